// Precision-independent reductions: deterministic finalisation of per-CTA
// partial sums (FP64) into Krylov scalars, and the staggered-error sweeps
// of Algorithm 1 (iii).
#include <algorithm>

#include "ops.h"
#include "tma.cuh"

namespace rvk {

void tensor_map_evict(const void* base) { tensor_map_evict_impl(base); }

// Partial sums of the producing kernels (one per CTA and slot) are reduced
// in two levels, both in a fixed order so that results are reproducible:
// CTA c of the finalisation sums the contiguous block range c of every slot
// (its threads strided over the range, then a fixed tree) into fs->stage;
// the CTA that arrives last (atomic ticket) sums the stage entries of each
// slot in index order, applies the mode's Krylov update and re-arms the
// ticket.  At 256^3 the 64 K partials of the x1 passes take one load round
// per thread instead of eight sequential ones in a single CTA.
constexpr int kFinThreads = 256;

__global__ void __launch_bounds__(kFinThreads)
k_finalize_impl(const double* __restrict__ part, int nblocks, int stride, int nslots, int mode,
                KrylovCtl* ctl, double* out, double scale, int imax, int stall, FinScratch* __restrict__ fs) {
  __shared__ double red[kFinThreads / 32];
  __shared__ double vals[16];
  __shared__ int last;
  const bool is_max = mode == FIN_MAXS;
  const int chunk = (nblocks + gridDim.x - 1) / gridDim.x;
  const int b0 = blockIdx.x * chunk, b1 = min(nblocks, b0 + chunk);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int s = 0; s < nslots; s++) {
    const double* ps = part + (long long)s * stride;
    double a[4] = {0, 0, 0, 0};
    int b = b0 + threadIdx.x;
    for (; b + 3 * kFinThreads < b1; b += 4 * kFinThreads) {
      double x[4];
#pragma unroll
      for (int k = 0; k < 4; k++) x[k] = ps[b + k * kFinThreads];
#pragma unroll
      for (int k = 0; k < 4; k++) a[k] = is_max ? fmax(a[k], x[k]) : a[k] + x[k];
    }
    for (; b < b1; b += kFinThreads) a[0] = is_max ? fmax(a[0], ps[b]) : a[0] + ps[b];
    double acc = is_max ? fmax(fmax(a[0], a[1]), fmax(a[2], a[3])) : (a[0] + a[1]) + (a[2] + a[3]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double y = __shfl_down_sync(0xffffffffu, acc, o);
      acc = is_max ? fmax(acc, y) : acc + y;
    }
    if (lane == 0) red[wid] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = red[0];
      for (int w = 1; w < kFinThreads / 32; w++) t = is_max ? fmax(t, red[w]) : t + red[w];
      fs->stage[s * kFinMaxCtas + blockIdx.x] = t;
    }
    __syncthreads();
  }
  // the stage entries of this CTA are visible before its ticket is taken
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(&fs->ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (threadIdx.x < nslots) {
    const int s = threadIdx.x;
    double t = __ldcg(&fs->stage[s * kFinMaxCtas]);
    for (int c = 1; c < (int)gridDim.x; c++) {
      const double y = __ldcg(&fs->stage[s * kFinMaxCtas + c]);
      t = is_max ? fmax(t, y) : t + y;
    }
    vals[s] = t;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  fs->ticket = 0u;
  switch (mode) {
    case FIN_SUMS:
    case FIN_MAXS:
      for (int s = 0; s < nslots; s++) out[s] = vals[s] * scale;
      break;
    case FIN_CG_INIT:
      ctl->rtol2 = scale;
      ctl->maxit = imax;
      ctl->stall = stall;
      ctl->b2 = vals[0];
      ctl->tol2 = scale * vals[0];
      ctl->best = vals[0];
      ctl->best_it = 0;
      ctl->rr = vals[0];
      ctl->rnorm2 = vals[0];
      ctl->iter = 0;
      ctl->beta = 0.0;
      ctl->alpha = 0.0;
      ctl->status = 0;
      ctl->done = vals[0] == 0.0 ? 1 : 0;
      if (!(vals[0] == vals[0])) { ctl->done = 1; ctl->status = 3; }
      if (ctl->done && ctl->status == 0) ctl->status = 1;
      if (!ctl->done && imax <= 0) { ctl->done = 1; ctl->status = 2; }
      break;
    case FIN_PCG_INIT:
      ctl->rtol2 = scale;
      ctl->maxit = imax;
      ctl->stall = stall;
      ctl->tol2 = scale * vals[0];
      ctl->best = vals[0];
      ctl->best_it = 0;
      ctl->b2 = vals[0];
      ctl->rnorm2 = vals[0];
      ctl->rr = vals[1];
      ctl->iter = 0;
      ctl->beta = 0.0;
      ctl->alpha = 0.0;
      ctl->status = 0;
      ctl->done = vals[0] == 0.0 ? 1 : 0;
      if (!(vals[0] == vals[0])) { ctl->done = 1; ctl->status = 3; }
      if (ctl->done && ctl->status == 0) ctl->status = 1;
      if (!ctl->done && imax <= 0) { ctl->done = 1; ctl->status = 2; }
      break;
    case FIN_ALPHA:
      if (ctl->done) break;
      ctl->pAp = vals[0];
      // NaN: numeric failure; (p, Ap) <= 0: the SPD operator is at its
      // round-off floor, stop and keep the current iterate
      if (!(vals[0] == vals[0])) { ctl->done = 1; ctl->status = 3; break; }
      if (!(vals[0] > 0.0)) { ctl->done = 1; ctl->status = 4; break; }
      ctl->alpha = ctl->rr / vals[0];
      break;
    case FIN_CG_BETA:
    case FIN_PCG_BETA: {
      if (ctl->done) break;
      const double rn2 = vals[0];
      const double rrn = mode == FIN_CG_BETA ? vals[0] : vals[1];
      ctl->iter += 1;
      ctl->rnorm2 = rn2;
      if (!(rn2 == rn2)) { ctl->done = 1; ctl->status = 3; break; }
      if (rn2 <= ctl->tol2) { ctl->done = 1; ctl->status = 1; break; }
      if (ctl->iter >= ctl->maxit) { ctl->done = 1; ctl->status = 2; break; }
      if (rn2 < 0.25 * ctl->best) { ctl->best = rn2; ctl->best_it = ctl->iter; }
      else if (ctl->stall > 0 && (ctl->iter - ctl->best_it >= ctl->stall || rn2 > 1e2 * ctl->best)) {
        // FP32 solve at its attainable accuracy (stalled) or losing stability
        ctl->done = 1;
        ctl->status = 4;
        break;
      }
      ctl->beta = rrn / ctl->rr;
      ctl->rr = rrn;
      break;
    }
    default:
      break;
  }
}

void k_finalize(cudaStream_t st, FinScratch* fs, const double* part, int nblocks, int nblk_stride, int nslots,
                int mode, KrylovCtl* ctl, double* out, double scale, int imax, int stall) {
  // about 1024 partials per CTA of the first level
  const int ctas = std::max(1, std::min(kFinMaxCtas, (nblocks + 1023) / 1024));
  k_finalize_impl<<<ctas, kFinThreads, 0, st>>>(part, nblocks, nblk_stride, nslots, mode, ctl, out, scale, imax,
                                                stall, fs);
}

struct Add6 { double a[6]; };

__global__ void __launch_bounds__(kThreads)
k_copy_add_impl(long long V, int nc, const double* __restrict__ src, double* __restrict__ dst, Add6 add) {
  const long long n = (long long)nc * V;
  for (long long i = blockIdx.x * (long long)kThreads + threadIdx.x; i < n; i += (long long)gridDim.x * kThreads)
    dst[i] = src[i] + add.a[i / V];
}

// Corner derivatives of the rotated scheme (R5) in real space: out[j][n] is
// the mean of the forward differences along x_j on the 2^(d-1) cube edges
// parallel to x_j, at the voxel corner n + 1/2 (periodic).  With N3 = 1 the
// x3 neighbour is the voxel itself, which gives the 2D stencil.
__global__ void __launch_bounds__(kThreads)
k_corner_grad64_impl(Geo g, const double* __restrict__ a, double* __restrict__ out) {
  const long long V = g.V;
  const int n1 = g.n1, n2 = g.n2, n3 = g.n3;
  const double c0 = 1.0 / (4.0 * g.h[0]), c1 = 1.0 / (4.0 * g.h[1]), c2 = g.d == 3 ? 1.0 / (4.0 * g.h[2]) : 0.0;
  for (long long v = blockIdx.x * (long long)kThreads + threadIdx.x; v < V; v += (long long)gridDim.x * kThreads) {
    const int i = (int)(v % n1);
    const long long rest = v / n1;
    const int j = (int)(rest % n2), k = (int)(rest / n2);
    const int ip = i + 1 == n1 ? 0 : i + 1, jp = j + 1 == n2 ? 0 : j + 1, kp = k + 1 >= n3 ? 0 : k + 1;
    auto at = [&](int x, int y, int z) { return a[((long long)z * n2 + y) * n1 + x]; };
    const double q000 = at(i, j, k), q100 = at(ip, j, k), q010 = at(i, jp, k), q110 = at(ip, jp, k);
    const double q001 = at(i, j, kp), q101 = at(ip, j, kp), q011 = at(i, jp, kp), q111 = at(ip, jp, kp);
    out[v] = c0 * ((q100 - q000) + (q110 - q010) + (q101 - q001) + (q111 - q011));
    out[V + v] = c1 * ((q010 - q000) + (q110 - q100) + (q011 - q001) + (q111 - q101));
    if (g.d == 3) out[2 * V + v] = c2 * ((q001 - q000) + (q101 - q100) + (q011 - q010) + (q111 - q110));
  }
}

void k_corner_grad64(cudaStream_t st, const Geo& g, const double* a, double* out) {
  const long long nb = (g.V + kThreads - 1) / kThreads;
  k_corner_grad64_impl<<<(int)(nb < 8192 ? nb : 8192), kThreads, 0, st>>>(g, a, out);
}

__global__ void __launch_bounds__(kThreads)
k_fill_porosity_impl(long long V, const uint8_t* __restrict__ phase, const PhaseTable* __restrict__ pt,
                     double* __restrict__ f) {
  for (long long v = blockIdx.x * (long long)kThreads + threadIdx.x; v < V; v += (long long)gridDim.x * kThreads) {
    const PhaseDev& P = pt->p[phase[v]];
    f[v] = P.law == 3 ? P.f0 : 0.0;
  }
}

void k_fill_porosity(cudaStream_t st, long long V, const uint8_t* phase, const PhaseTable* pt, double* f) {
  const long long nb = (V + kThreads - 1) / kThreads;
  k_fill_porosity_impl<<<(int)(nb < 4096 ? nb : 4096), kThreads, 0, st>>>(V, phase, pt, f);
}

void k_copy_add(cudaStream_t st, long long V, int nc, const double* src, double* dst, const double* add_host6) {
  Add6 a;
  for (int c = 0; c < 6; c++) a.a[c] = add_host6[c];
  const long long n = (long long)nc * V;
  const long long nb = (n + kThreads - 1) / kThreads;
  k_copy_add_impl<<<(int)(nb < 4096 ? nb : 4096), kThreads, 0, st>>>(V, nc, src, dst, a);
}

__global__ void __launch_bounds__(kThreads)
k_err_eps_impl(Geo g, const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ part,
               int pstride) {
  double acc[6] = {0, 0, 0, 0, 0, 0};
  double mx[1] = {0.0};
  const long long V = g.V;
  for (long long v = blockIdx.x * (long long)kThreads + threadIdx.x; v < V; v += (long long)gridDim.x * kThreads) {
    for (int c = 0; c < g.nc; c++) {
      const double x = a[c * V + v];
      acc[c] += x;
      mx[0] = fmax(mx[0], fabs(x - b[c * V + v]));
    }
  }
  block_sum_store<6>(acc, part, pstride);
  __syncthreads();
  block_max_store<1>(mx, part + 6 * (long long)pstride, pstride);
}

__global__ void __launch_bounds__(kThreads)
k_err_abar_impl(long long n, const double* __restrict__ a, const double* __restrict__ b,
                double* __restrict__ part, int pstride) {
  double acc[2] = {0.0, 0.0};
  for (long long i = blockIdx.x * (long long)kThreads + threadIdx.x; i < n; i += (long long)gridDim.x * kThreads) {
    const double d = a[i] - b[i];
    acc[0] += d * d;
    acc[1] += a[i] * a[i];
  }
  block_sum_store<2>(acc, part, pstride);
}

void k_err_eps(const Geo& g, const LaunchCfg& lc, cudaStream_t st, const double* eps_new,
               const double* eps_old, double* part) {
  k_err_eps_impl<<<lc.n_ew_blocks, kThreads, 0, st>>>(g, eps_new, eps_old, part, lc.max_blocks);
}

void k_err_abar(const Geo& g, const LaunchCfg& lc, cudaStream_t st, const double* a_new, const double* a_old,
                double* part) {
  k_err_abar_impl<<<lc.n_ew_blocks, kThreads, 0, st>>>(g.V, a_new, a_old, part, lc.max_blocks);
}

}  // namespace rvk
