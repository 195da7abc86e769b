// Adjoint-sweep kernels (FP64): per-voxel transposed-Jacobian products of
// the local update by forward-mode dual numbers, and small reductions.
#include <cuda_runtime.h>

#include "adjoint_ops.h"
#include "common.cuh"

namespace rvk {

// ------------------------------------------------------------ dual numbers
// value and derivatives along N input directions
template <int N>
struct Dual {
  double v;
  double d[N];
};

template <int N>
__device__ __forceinline__ Dual<N> dc(double x) {
  Dual<N> r;
  r.v = x;
#pragma unroll
  for (int i = 0; i < N; i++) r.d[i] = 0.0;
  return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator+(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r;
  r.v = a.v + b.v;
#pragma unroll
  for (int i = 0; i < N; i++) r.d[i] = a.d[i] + b.d[i];
  return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator-(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r;
  r.v = a.v - b.v;
#pragma unroll
  for (int i = 0; i < N; i++) r.d[i] = a.d[i] - b.d[i];
  return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator*(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r;
  r.v = a.v * b.v;
#pragma unroll
  for (int i = 0; i < N; i++) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
  return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator*(double s, const Dual<N>& a) {
  Dual<N> r;
  r.v = s * a.v;
#pragma unroll
  for (int i = 0; i < N; i++) r.d[i] = s * a.d[i];
  return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator/(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r;
  r.v = a.v / b.v;
  const double ib = 1.0 / b.v;
#pragma unroll
  for (int i = 0; i < N; i++) r.d[i] = (a.d[i] - r.v * b.d[i]) * ib;
  return r;
}
template <int N>
__device__ __forceinline__ Dual<N> dsqrt(const Dual<N>& a) {
  Dual<N> r;
  r.v = sqrt(a.v);
  const double k = 0.5 / r.v;
#pragma unroll
  for (int i = 0; i < N; i++) r.d[i] = k * a.d[i];
  return r;
}

// --------------------------------------- positive part of a symmetric tensor
// Jacobi rotation zeroing (P, Q) that also accumulates the eigenvectors
// (columns of Vm); same rotation as in the forward return map.
template <int P, int Q>
__device__ __forceinline__ void jacobi_rot3v(double (&A)[3][3], double (&Vm)[3][3]) {
  const double apq = A[P][Q];
  if (apq == 0.0) return;
  constexpr int Rr = 3 - P - Q;
  const double th = (A[Q][Q] - A[P][P]) / (2.0 * apq);
  const double at = fabs(th);
  const double t = (at > 1e150 ? 0.5 / at : 1.0 / (at + sqrt(th * th + 1.0))) * (th >= 0.0 ? 1.0 : -1.0);
  const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
  A[P][P] -= t * apq;
  A[Q][Q] += t * apq;
  A[P][Q] = A[Q][P] = 0.0;
  const double arp = A[Rr][P], arq = A[Rr][Q];
  A[Rr][P] = A[P][Rr] = c * arp - s * arq;
  A[Rr][Q] = A[Q][Rr] = s * arp + c * arq;
#pragma unroll
  for (int r = 0; r < 3; r++) {
    const double vp = Vm[r][P], vq = Vm[r][Q];
    Vm[r][P] = c * vp - s * vq;
    Vm[r][Q] = s * vp + c * vq;
  }
}

// ||<e>_+|| and the Mandel components of <e>_+ (the positive spectral part)
__device__ __forceinline__ double positive_part(const double (&e)[6], double (&pp)[6]) {
  const double r2 = 0.70710678118654752440, s2 = 1.41421356237309504880;
  double A[3][3] = {{e[0], e[5] * r2, e[4] * r2}, {e[5] * r2, e[1], e[3] * r2}, {e[4] * r2, e[3] * r2, e[2]}};
  double Vm[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  const double n2 = e[0] * e[0] + e[1] * e[1] + e[2] * e[2] + e[3] * e[3] + e[4] * e[4] + e[5] * e[5];
  for (int sweep = 0; sweep < 12; sweep++) {
    const double off = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
    if (!(off > 1e-32 * n2)) break;
    jacobi_rot3v<0, 1>(A, Vm);
    jacobi_rot3v<0, 2>(A, Vm);
    jacobi_rot3v<1, 2>(A, Vm);
  }
  double k = 0.0, T[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  for (int i = 0; i < 3; i++) {
    const double l = A[i][i] > 0.0 ? A[i][i] : 0.0;
    k += l * l;
    for (int a = 0; a < 3; a++)
      for (int b = 0; b < 3; b++) T[a][b] += l * Vm[a][i] * Vm[b][i];
  }
  pp[0] = T[0][0];
  pp[1] = T[1][1];
  pp[2] = T[2][2];
  pp[3] = s2 * T[1][2];
  pp[4] = s2 * T[0][2];
  pp[5] = s2 * T[0][1];
  return sqrt(k);
}

// ------------------------------------------------------------ local VJP
constexpr int kDirs = 8;

__global__ void __launch_bounds__(kThreads)
k_local_vjp(Geo g, const PhaseTable* __restrict__ pt, int J, AdjState s, AdjCot w, AdjOut o, AdjDirs dirs) {
  using D8 = Dual<kDirs>;
  const long long V = g.V;
  const int nc = g.nc;
  const double s23 = 0.81649658092772603273;   // sqrt(2/3)
  for (long long v = blockIdx.x * (long long)kThreads + threadIdx.x; v < V; v += (long long)gridDim.x * kThreads) {
    const PhaseDev P = pt->p[s.phase[v]];
    // inputs as duals, seeded along this pass's directions
    D8 eps[6], pn[6];
    for (int c = 0; c < 6; c++) {
      eps[c] = dc<kDirs>(0.0);
      pn[c] = dc<kDirs>(s.epsp_prev[c * V + v]);
    }
    for (int c = 0; c < nc; c++) eps[g.cmap[c]].v = s.eps[c * V + v];
    D8 epn = dc<kDirs>(s.ep_prev[v]);
    D8 ab = dc<kDirs>(P.var >= 0 ? s.abar[P.var * V + v] : 0.0);
    D8 th[4] = {dc<kDirs>(P.sigma_y), dc<kDirs>(P.H), dc<kDirs>(P.eps_C), dc<kDirs>(P.eps_R)};
    D8 sc = dc<kDirs>(s.stiff ? s.stiff[v] : 1.0);
    for (int k = 0; k < dirs.n; k++) {
      const int i = dirs.idx[k];
      switch (dirs.kind[k]) {
        case AD_EPS: eps[g.cmap[i]].d[k] = 1.0; break;
        case AD_EPSP: pn[i].d[k] = 1.0; break;
        case AD_EP: epn.d[k] = 1.0; break;
        case AD_ABAR: if (i == P.var) ab.d[k] = 1.0; break;
        case AD_THETA: th[i].d[k] = 1.0; break;
        default: sc.d[k] = 1.0; break;
      }
    }
    // the local update (same equations as the forward return map)
    const D8 K = P.K * sc, mu = P.mu * sc;
    D8 e[6];
    for (int c = 0; c < 6; c++) e[c] = eps[c] - pn[c];
    const D8 tr = e[0] + e[1] + e[2];
    D8 dev[6];
    for (int c = 0; c < 6; c++) dev[c] = c < 3 ? e[c] - (1.0 / 3.0) * tr : e[c];
    D8 dl = dc<kDirs>(0.0), D = dc<kDirs>(0.0), epv = epn;
    D8 nh[6];
    for (int c = 0; c < 6; c++) nh[c] = dc<kDirs>(0.0);
    if (P.law == 1) {
      D8 q2 = dc<kDirs>(0.0);
      for (int c = 0; c < 6; c++) q2 = q2 + dev[c] * dev[c];
      if (q2.v > 0.0) {
        const D8 q = 2.0 * (mu * dsqrt(q2));
        const D8 f = q - s23 * (th[0] + th[1] * epn);
        if (f.v > 0.0) {
          dl = f / (2.0 * mu + (2.0 / 3.0) * th[1]);
          for (int c = 0; c < 6; c++) nh[c] = (2.0 * mu) * dev[c] / q;
        }
      }
      epv = epn + s23 * dl;
    } else if (P.law == 2) {
      double ev[6], pp[6];
      for (int c = 0; c < 6; c++) ev[c] = e[c].v;
      const double kn = positive_part(ev, pp);
      if (epn.v >= kn) {
        epv = epn;
      } else {
        epv = dc<kDirs>(kn);
        if (kn > 0.0)
          for (int c = 0; c < 6; c++)
            for (int k = 0; k < kDirs; k++) epv.d[k] += pp[c] / kn * e[c].d[k];
      }
    }
    if ((P.law == 1 || P.law == 2) && P.var >= 0) {
      const D8 Dr = (ab - th[2]) / (th[3] - th[2]);
      D = Dr.v < 0.0 ? dc<kDirs>(0.0) : (Dr.v > P.D_max ? dc<kDirs>(P.D_max) : Dr);
    }
    const D8 om = dc<kDirs>(1.0) - D;
    // contraction with the cotangent, output by output
    double acc[kDirs];
    for (int k = 0; k < kDirs; k++) acc[k] = 0.0;
    for (int c = 0; c < 6; c++) {
      double ws = c == 0 ? w.seed11 : 0.0;
      if (w.lam)
        for (int cc = 0; cc < nc; cc++)
          if (g.cmap[cc] == c) ws -= w.lam[cc * V + v];
      const D8 seff = (c < 3 ? K * tr : dc<kDirs>(0.0)) + 2.0 * (mu * dev[c]) - 2.0 * (mu * (dl * nh[c]));
      const D8 sg = om * seff;
      const double wp = w.w_epsp ? w.w_epsp[c * V + v] : 0.0;
      const D8 pnew = pn[c] + dl * nh[c];
      for (int k = 0; k < kDirs; k++) acc[k] += ws * sg.d[k] + wp * pnew.d[k];
    }
    if (w.w_ep)
      for (int k = 0; k < kDirs; k++) acc[k] += w.w_ep[v] * epv.d[k];
    if (w.w_alpha && P.var >= 0)
      for (int k = 0; k < kDirs; k++) acc[k] += w.w_alpha[P.var * V + v] * epv.d[k];
    for (int k = 0; k < dirs.n; k++) {
      const int i = dirs.idx[k];
      switch (dirs.kind[k]) {
        case AD_EPS: o.v_eps[i * V + v] = acc[k]; break;
        case AD_EPSP: o.v_epsp[i * V + v] = acc[k]; break;
        case AD_EP: o.v_ep[v] = acc[k]; break;
        case AD_ABAR: o.v_abar[i * V + v] = acc[k]; break;
        case AD_THETA: o.v_theta[i * V + v] = acc[k]; break;
        default: o.v_stiff[v] = acc[k]; break;
      }
    }
  }
}

void adj_local_vjp(const Geo& g, const PhaseTable* pt, int J, const AdjState& s, const AdjCot& w,
                   const AdjOut& o, const AdjDirs& dirs, int nblocks, cudaStream_t st) {
  k_local_vjp<<<nblocks, kThreads, 0, st>>>(g, pt, J, s, w, o, dirs);
}

// ------------------------------------------------------------ reductions
__global__ void __launch_bounds__(kThreads)
k_absmax2(long long n, const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ part,
          int pstride) {
  double m[2] = {0.0, 0.0};
  for (long long i = blockIdx.x * (long long)kThreads + threadIdx.x; i < n; i += (long long)gridDim.x * kThreads) {
    m[0] = fmax(m[0], fabs(a[i] - b[i]));
    m[1] = fmax(m[1], fabs(a[i]));
  }
  block_max_store<2>(m, part, pstride);
}

void adj_absmax2(long long n, const double* a, const double* b, double* part, int pstride, int nblocks,
                 cudaStream_t st) {
  k_absmax2<<<nblocks, kThreads, 0, st>>>(n, a, b, part, pstride);
}

__global__ void __launch_bounds__(kThreads)
k_weighted_dot(long long V, int d, const uint8_t* __restrict__ phase, PhaseWeights w,
               const double* __restrict__ ga, const double* __restrict__ gb, double* __restrict__ part,
               int pstride) {
  double acc[1] = {0.0};
  for (long long v = blockIdx.x * (long long)kThreads + threadIdx.x; v < V; v += (long long)gridDim.x * kThreads) {
    double s = 0.0;
    for (int k = 0; k < d; k++) s += ga[k * V + v] * gb[k * V + v];
    acc[0] += w.w[phase[v]] * s;
  }
  block_sum_store<1>(acc, part, pstride);
}

void adj_weighted_dot(long long V, int d, const uint8_t* phase, PhaseWeights w, const double* ga,
                      const double* gb, double* part, int pstride, int nblocks, cudaStream_t st) {
  k_weighted_dot<<<nblocks, kThreads, 0, st>>>(V, d, phase, w, ga, gb, part, pstride);
}

__global__ void __launch_bounds__(kThreads)
k_phase_sums(long long V, const uint8_t* __restrict__ phase, const double* __restrict__ vt,
             double* __restrict__ part, int pstride) {
  double acc[4 * kMaxPhases];
#pragma unroll
  for (int i = 0; i < 4 * kMaxPhases; i++) acc[i] = 0.0;
  for (long long v = blockIdx.x * (long long)kThreads + threadIdx.x; v < V; v += (long long)gridDim.x * kThreads) {
    const int q = phase[v];
#pragma unroll
    for (int p = 0; p < kMaxPhases; p++)
      if (p == q)
#pragma unroll
        for (int k = 0; k < 4; k++) acc[4 * p + k] += vt[k * V + v];
  }
  block_sum_store<4 * kMaxPhases>(acc, part, pstride);
}

void adj_phase_sums(long long V, const uint8_t* phase, const double* v_theta, double* part, int pstride,
                    int nblocks, cudaStream_t st) {
  k_phase_sums<<<nblocks, kThreads, 0, st>>>(V, phase, v_theta, part, pstride);
}

__global__ void k_axpy(long long n, double a, const double* __restrict__ x, double* __restrict__ y) {
  for (long long i = blockIdx.x * (long long)kThreads + threadIdx.x; i < n; i += (long long)gridDim.x * kThreads)
    y[i] += a * x[i];
}

void adj_axpy(long long n, double a, const double* x, double* y, int nblocks, cudaStream_t st) {
  k_axpy<<<nblocks, kThreads, 0, st>>>(n, a, x, y);
}

}  // namespace rvk
