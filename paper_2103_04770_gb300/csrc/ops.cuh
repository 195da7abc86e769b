// Device operators of the non-local damage RVE library (templated on the
// precision R of the spectral and Krylov data).  See ops.h for the layout.
//
// Spectral sweeps (Section 3.2, Eq. eqdiscrete2 and Algorithm 2) are split
// into passes that each make one HBM round trip:
//   x1 pass   : R2C / C2R along the contiguous axis (half-length complex FFT
//               plus split), fused with the per-voxel prologue (tangent
//               C_T : p, residual source) or epilogue (store, dots, l^2)
//   y pass    : plain transform along x2 (3D only)
//   last pass : transform along the last axis fused with the pointwise
//               Fourier operator (modified projection G*, Helmholtz symbol
//               k, conj(k), preconditioner) and, for G*, the inverse.
#pragma once
#include <math.h>

#include <mutex>
#include <unordered_set>

#include "fft.cuh"
#include "fft256.cuh"
#include "fft_ct.cuh"
#include "ops.h"
#include "tma.cuh"

namespace rvk {

template <typename R> struct StridedE;
template <> struct StridedE<float> { static constexpr int E = 8; };
template <> struct StridedE<double> { static constexpr int E = 4; };

struct Mask6 { float m[6]; };

__device__ __forceinline__ long long lmin_(long long a, long long b) { return a < b ? a : b; }

template <typename K>
static void set_smem(K kernel, size_t bytes) {
  // The limit is a per-kernel attribute shared by every handle and thread.
  // It is raised once per kernel to the largest value the kernel accepts
  // (the device's opt-in maximum less the kernel's static shared memory) and
  // never lowered, so a concurrent caller with a smaller tile cannot shrink
  // it between another caller's check and launch.  Each launch still gets
  // only its own dynamic size.
  if (bytes <= 48 * 1024) return;
  static std::mutex mu;
  static std::unordered_set<const void*> done;
  const void* key = reinterpret_cast<const void*>(kernel);
  std::lock_guard<std::mutex> lock(mu);
  if (done.count(key)) return;
  int dev = 0, optin = 0;
  cudaFuncAttributes fa{};
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
      cudaFuncGetAttributes(&fa, kernel) != cudaSuccess) {
    cudaGetLastError();
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    return;
  }
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           optin - (int)fa.sharedSizeBytes) == cudaSuccess) {
    done.insert(key);
  } else {
    cudaGetLastError();
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  }
}

// ---------------------------------------------------------- Fourier symbols
// Rotated-scheme modified frequency (Willot): k_j = i e^{i phi} a_j with
// a_j = (2/h_j) sin(theta_j/2) prod_{m != j} cos(theta_m/2) and
// e^{i phi} = prod_m (cos(theta_m/2) + i sin(theta_m/2)).
template <typename R>
__device__ __forceinline__ void symbol(const Geo& g, const Tables<R>& t, int m0, int m1, int m2,
                                       R a[3], C2<R>& ph) {
  const R s0 = t.s[0][m0], c0 = t.c[0][m0];
  const R s1 = t.s[1][m1], c1 = t.c[1][m1];
  if (g.d == 3) {
    const R s2 = t.s[2][m2], c2 = t.c[2][m2];
    a[0] = t.two_over_h[0] * s0 * c1 * c2;
    a[1] = t.two_over_h[1] * s1 * c0 * c2;
    a[2] = t.two_over_h[2] * s2 * c0 * c1;
    ph = cmul(cmul(mk<R>(c0, s0), mk<R>(c1, s1)), mk<R>(c2, s2));
  } else {
    a[0] = t.two_over_h[0] * s0 * c1;
    a[1] = t.two_over_h[1] * s1 * c0;
    a[2] = R(0);
    ph = cmul(mk<R>(c0, s0), mk<R>(c1, s1));
  }
}

// Orthogonal projection onto compatible symmetric strains at one mode
// (Mandel components, real direction n):  G(T) = n(x)Tn + Tn(x)n - (nTn) n(x)n.
template <typename R>
__device__ __forceinline__ void gamma_mode(int d, const R n[3], C2<R>* t) {
  const R is2 = R(0.70710678118654752440);
  const R s2 = R(1.41421356237309504880);
  if (d == 3) {
    C2<R> v0 = cscale(t[0], n[0]) + cscale(cscale(t[5], n[1]) + cscale(t[4], n[2]), is2);
    C2<R> v1 = cscale(cscale(t[5], n[0]) + cscale(t[3], n[2]), is2) + cscale(t[1], n[1]);
    C2<R> v2 = cscale(cscale(t[4], n[0]) + cscale(t[3], n[1]), is2) + cscale(t[2], n[2]);
    C2<R> nt = cscale(v0, n[0]) + cscale(v1, n[1]) + cscale(v2, n[2]);
    t[0] = cscale(v0, R(2) * n[0]) - cscale(nt, n[0] * n[0]);
    t[1] = cscale(v1, R(2) * n[1]) - cscale(nt, n[1] * n[1]);
    t[2] = cscale(v2, R(2) * n[2]) - cscale(nt, n[2] * n[2]);
    t[3] = cscale(cscale(v2, n[1]) + cscale(v1, n[2]) - cscale(nt, n[1] * n[2]), s2);
    t[4] = cscale(cscale(v2, n[0]) + cscale(v0, n[2]) - cscale(nt, n[0] * n[2]), s2);
    t[5] = cscale(cscale(v1, n[0]) + cscale(v0, n[1]) - cscale(nt, n[0] * n[1]), s2);
  } else {
    C2<R> v0 = cscale(t[0], n[0]) + cscale(t[2], n[1] * is2);
    C2<R> v1 = cscale(t[2], n[0] * is2) + cscale(t[1], n[1]);
    C2<R> nt = cscale(v0, n[0]) + cscale(v1, n[1]);
    t[0] = cscale(v0, R(2) * n[0]) - cscale(nt, n[0] * n[0]);
    t[1] = cscale(v1, R(2) * n[1]) - cscale(nt, n[1] * n[1]);
    t[2] = cscale(cscale(v1, n[0]) + cscale(v0, n[1]) - cscale(nt, n[0] * n[1]), s2);
  }
}

// ------------------------------------------------ tile staging (cp.async)
// Tiles of the strided passes are rows of `cols` complex entries (row n of
// component c at src + c*cstride + n*astride) held in shared memory as
// buf[c][n][tx].  Loads go through cp.async in 16-byte chunks (8 bytes for
// an odd FP32 tail) so that each thread keeps many copies in flight; rows
// start on 16-byte boundaries (padded rows, even tile starts).
__device__ __forceinline__ void cp_async16(void* sm, const void* gm) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(sm);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gm) : "memory");
}
__device__ __forceinline__ void cp_async8(void* sm, const void* gm) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(sm);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gm) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// ================================================================ x1 passes
// Padding shift of the compile-time x1 kernels' shared buffers (one complex
// entry per 16 in FP32, per 8 in FP64; 0 for the runtime-sized kernels).
template <typename R, int MCT> struct XPad {
  static constexpr int v = MCT > 0 ? (sizeof(R) == 4 ? 4 : 3) : 0;
};
// complex entries reserved for rows * nc lines of M points, padding included
__host__ __device__ __forceinline__ size_t xbuf_c(int rows, int nc, int M) {
  const size_t n = (size_t)rows * nc * M;
  return n + (n >> 3) + 16;
}
// rows per CTA of the compile-time x1 kernels: the E = 4 row rule
// min(32, 4 kThreads / (NC M)) for M = MCT
template <int MCT, int NC> struct XRows {
  static constexpr int v = MCT > 0 ? x1_ct_rows(MCT, NC) : 0;
};

// real element ri of a padded complex buffer
template <typename R, int PADSH>
__device__ __forceinline__ R& rpad(R* rbuf, int ri) {
  return rbuf[2 * cpad<PADSH>(ri >> 1) + (ri & 1)];
}

// Kernels are specialised on the component count NC (so per-voxel vectors
// live in registers) and on E, the FFT elements staged per thread (4: one or
// a few rows per CTA and four CTAs per SM; 16: long rows).
template <typename R, int E> struct XMinBlocks {
  static constexpr int v = E <= 4 ? (sizeof(R) == 4 ? 3 : 2) : 1;
};

// MCT > 0: compile-time row of MCT = N1/2 complex points, one row per CTA.
template <typename R, int NC, int E, class PRO, int MCT = 0>
__global__ void __launch_bounds__(kThreads, XMinBlocks<R, E>::v)
k_xfwd(Geo g, FftPlan pl, const C2<R>* __restrict__ tw1, C2<R>* __restrict__ S, int nrows, PRO pro,
       const KrylovCtl* __restrict__ ctl) {
  if (ctl && ctl->done) return;
  constexpr int PS = XPad<R, MCT>::v;
  // row lengths: compile-time on the MCT path, so the index divisions fold
  const int n1 = MCT > 0 ? 2 * MCT : g.n1;
  const int M = MCT > 0 ? MCT : g.M;
  const int P1 = MCT > 0 ? MCT + 1 : g.P1;
  const int ps = MCT > 0 ? ((MCT + 1 + 15) / 16) * 16 : g.ps;
  extern __shared__ __align__(16) unsigned char smraw[];
  C2<R>* tws = reinterpret_cast<C2<R>*>(smraw);
  R* rbuf = reinterpret_cast<R*>(tws + g.n1);
  C2<R>* cbuf = reinterpret_cast<C2<R>*>(rbuf);
  const long long row0 = (long long)blockIdx.x * nrows;
  const int rows = (int)lmin_(nrows, g.nlines - row0);
  for (int i = threadIdx.x; i < g.n1; i += kThreads) tws[i] = tw1[i];
  pro.begin(ctl);
  R acc[1] = {R(0)};
  const int nvox = rows * n1;
  for (int e = threadIdx.x; e < nvox; e += kThreads) {
    const int r = e / n1, x = e - r * n1;
    const long long v = (row0 + r) * n1 + x;
    R val[NC];
    if constexpr (PRO::kDot) pro(v, val, acc[0]);
    else pro(v, val);
#pragma unroll
    for (int c = 0; c < NC; c++) rpad<R, PS>(rbuf, (r * NC + c) * n1 + x) = val[c];
  }
  if constexpr (PRO::kDot) {
    if (pro.part) block_sum_store<1>(acc, pro.part, pro.pstride);
  }
  __syncthreads();
  if constexpr (MCT > 0) fft_lines_ct<R, MCT, XRows<MCT, NC>::v * NC, 1, MCT, -1, true, 2, PS>(cbuf, tws);
  else fft_lines<R, E, -1>(cbuf, pl, rows * NC, 1, g.M, true, tws, 2);
  const int nout = rows * NC * P1;
  for (int e = threadIdx.x; e < nout; e += kThreads) {
    const int l = e / P1, k = e - l * P1;
    const int r = l / NC, c = l - r * NC;
    const C2<R> zk = cbuf[cpad<PS>(l * M + (k == M ? 0 : k))];
    const C2<R> zm = cbuf[cpad<PS>(l * M + (k == 0 ? 0 : M - k))];
    const C2<R> Ek = mk<R>(R(0.5) * (zk.x + zm.x), R(0.5) * (zk.y - zm.y));
    const C2<R> Ok = mk<R>(R(0.5) * (zk.y + zm.y), R(-0.5) * (zk.x - zm.x));
    S[c * g.sstride + (row0 + r) * ps + k] = Ek + cmul(tws[k], Ok);
  }
}

// Offset of the spectrum staging area behind the x1 pass buffers.
template <typename R>
__host__ __device__ __forceinline__ size_t xstage_off(int n1, int rows, int nc) {
  return (((size_t)n1 * sizeof(C2<R>) + xbuf_c(rows, nc, n1 / 2) * sizeof(C2<R>)) + 15) & ~(size_t)15;
}

// Stage the spectrum rows of the CTA with cp.async (xs[c][r][ps], r below
// XR rows per component slot), then split them into the half-length complex
// sequences (cbuf line r*NC + c).  MCT > 0: compile-time row length MCT and
// XR, so every index division folds into a multiply-shift.
template <typename R, int NC, int PS, int MCT = 0>
__device__ __forceinline__ void xinv_pre_staged(const Geo& g, const C2<R>* __restrict__ S, long long row0,
                                                int rows, int XRr, const C2<R>* tws, C2<R>* cbuf, C2<R>* xs) {
  const int M = MCT > 0 ? MCT : g.M;
  const int P1 = MCT > 0 ? MCT + 1 : g.P1;
  const int ps = MCT > 0 ? ((MCT + 1 + 15) / 16) * 16 : g.ps;
  const int XR = MCT > 0 ? XRows<MCT, NC>::v : XRr;
  {
    constexpr int PER = 16 / (int)sizeof(C2<R>);
    const int cpr = (P1 + PER - 1) / PER;
    const int total = NC * XR * cpr;
    for (int e = threadIdx.x; e < total; e += kThreads) {
      const int l = e / cpr, ch = e - l * cpr;
      const int c = l / XR, r = l - c * XR;
      if (r >= rows) continue;
      const int col = ch * PER;
      C2<R>* d = xs + (size_t)(c * XR + r) * ps + col;
      const C2<R>* sp = S + c * g.sstride + (row0 + r) * ps + col;
      if (PER == 2 && col + 1 >= P1) cp_async8(d, sp);
      else cp_async16(d, sp);
    }
    cp_async_wait_all();
  }
  __syncthreads();
  const int nin = rows * NC * M;
  for (int e = threadIdx.x; e < nin; e += kThreads) {
    const int l = e / M, k = e - l * M;
    const int r = l / NC, c = l - r * NC;
    const C2<R>* row = xs + (size_t)(c * XR + r) * ps;
    const C2<R> xk = row[k], xm = row[M - k];
    const C2<R> E = mk<R>(R(0.5) * (xk.x + xm.x), R(0.5) * (xk.y - xm.y));
    const C2<R> Dd = mk<R>(R(0.5) * (xk.x - xm.x), R(0.5) * (xk.y + xm.y));
    const C2<R> O = cmul(Dd, conj_(tws[k]));
    cbuf[cpad<PS>(l * M + k)] = mk<R>(E.x - O.y, E.y + O.x);
  }
}

// minimum resident CTAs of the x1 inverse kernels (the compile-time FP32
// variant fits 64 registers)
template <typename R, int E, int MCT> struct XInvMinBlocks {
  static constexpr int v = (MCT > 0 && sizeof(R) == 4) ? 4 : XMinBlocks<R, E>::v;
};

template <typename R, int NC, int E, class EPI, int NS, int MCT = 0>
__global__ void __launch_bounds__(kThreads, XInvMinBlocks<R, E, MCT>::v)
k_xinv(Geo g, FftPlan pl, const C2<R>* __restrict__ tw1, const C2<R>* __restrict__ S, int nrows, R scale,
       EPI epi, double* __restrict__ part, int pstride, const KrylovCtl* __restrict__ ctl) {
  if (ctl && ctl->done) return;
  constexpr int PS = XPad<R, MCT>::v;
  const int n1 = MCT > 0 ? 2 * MCT : g.n1;
  extern __shared__ __align__(16) unsigned char smraw[];
  C2<R>* tws = reinterpret_cast<C2<R>*>(smraw);
  R* rbuf = reinterpret_cast<R*>(tws + g.n1);
  C2<R>* cbuf = reinterpret_cast<C2<R>*>(rbuf);
  C2<R>* xs = reinterpret_cast<C2<R>*>(smraw + xstage_off<R>(g.n1, nrows, NC));
  const long long row0 = (long long)blockIdx.x * nrows;
  const int rows = (int)lmin_(nrows, g.nlines - row0);
  for (int i = threadIdx.x; i < g.n1; i += kThreads) tws[i] = tw1[i];
  // rows of the epilogue's input field, fetched together with the spectrum
  R* pre = reinterpret_cast<R*>(xs + (size_t)nrows * NC * g.ps);
  const int fs = nrows * NC * n1;   // stride between prefetched fields
  if constexpr (EPI::kPrefetch > 0) epi.prefetch(pre, row0, rows, n1, fs);
  xinv_pre_staged<R, NC, PS, MCT>(g, S, row0, rows, nrows, tws, cbuf, xs);
  __syncthreads();
  if constexpr (MCT > 0) fft_lines_ct<R, MCT, XRows<MCT, NC>::v * NC, 1, MCT, +1, true, 2, PS>(cbuf, tws);
  else fft_lines<R, E, +1>(cbuf, pl, rows * NC, 1, g.M, true, tws, 2);
  constexpr int NSA = NS > 0 ? NS : 1;
  R acc[NSA];
#pragma unroll
  for (int s = 0; s < NSA; s++) acc[s] = R(0);
  epi.begin(ctl);
  const int nvox = rows * n1;
  for (int e = threadIdx.x; e < nvox; e += kThreads) {
    const int r = e / n1, x = e - r * n1;
    const long long v = (row0 + r) * n1 + x;
    R val[NC];
#pragma unroll
    for (int c = 0; c < NC; c++) val[c] = rpad<R, PS>(rbuf, (r * NC + c) * n1 + x) * scale;
    if constexpr (EPI::kPrefetch > 0) epi(v, val, acc, pre + (r * NC) * n1 + x, n1, fs);
    else epi(v, val, acc);
  }
  if (NS > 0) block_sum_store<NSA>(acc, part, pstride);
}

// The Helmholtz operator of Algorithm 2 in real space (reading R15: the
// spectral GC(a) = a + sum_j conj(k_j) F(l^2 F^-1(k_j a)) with the rotated
// symbol k_j is, voxel by voxel, the stencil form q + sum_j D_j^T (l^2 D_j q)).
// This kernel computes the second part,
//     y = sum_j D_j^T (l^2 * D_j q),
// D_j the derivative along x_j at the voxel corner n + 1/2 (mean of the
// forward differences on the 2^(d-1) cube edges parallel to x_j, stored at
// index n) and l^2 taken at that index).
//
// Each warp owns a strip: 32 consecutive x1 columns (the first and last lane
// are halo: 30 outputs per warp), SYT rows along x2, and it marches along x3
// over zc planes.  Lane x holds q on its column for the strip's rows plus a
// one-row halo; q at x + 1 comes by shuffle, so a lane forms the fluxes of
// the corners at x + 1/2 alone.  Of the eight corners around a voxel, the
// four at x + 1/2 are the lane's own and the four at x - 1/2 belong to the
// lane on its left: each lane sums, per output row, the signed fluxes it owes
// itself (B) and its right neighbour (A), and one shuffle per output moves
// A.  The partial sums of corner plane k - 1/2 carry over to the next plane
// in registers, so every corner is formed once.  No shared memory, no block
// barrier; the next plane's loads are issued before the current plane's
// arithmetic.  With N3 = 1 the x3 neighbours are the plane itself, the x3
// flux vanishes and the kernel is the 2D stencil.
constexpr int kStencilWarps = 4;                   // warps per CTA (consecutive x2 strips)
constexpr int kStencilOut = 30;                    // outputs per warp along x1
template <typename R>
struct StencilRows {
  static constexpr int SYT = 4;
};

template <typename R>
__global__ void __launch_bounds__(32 * kStencilWarps)
k_helm_stencil(Geo g, const R* __restrict__ q, R* __restrict__ y, const uint8_t* __restrict__ phase,
               const R* __restrict__ ell2_tab, R c0, R c1, R c2, int zc, const KrylovCtl* __restrict__ ctl) {
  if (ctl && ctl->done) return;
  constexpr int SYT = StencilRows<R>::SYT;
  constexpr unsigned kAll = 0xffffffffu;
  __shared__ R l2[kMaxPhases];
  if (threadIdx.x < kMaxPhases) l2[threadIdx.x] = ell2_tab[threadIdx.x];
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int n1 = g.n1, n2 = g.n2, n3 = g.n3;
  const int y0 = (blockIdx.y * kStencilWarps + wid) * SYT;
  if (y0 >= n2) return;                            // whole warp (y0 is warp-uniform)
  const int x = blockIdx.x * kStencilOut - 1 + lane;
  const int xw = ((x % n1) + n1) % n1;
  const bool outx = lane >= 1 && lane <= kStencilOut && x < n1;
  const long long plane = (long long)n1 * n2;
  const int z0 = blockIdx.z * zc, z1 = min(z0 + zc, n3);
  int ro[SYT + 2];                                 // rows y0 - 1 .. y0 + SYT, periodic
#pragma unroll
  for (int r = 0; r < SYT + 2; r++) ro[r] = (((y0 - 1 + r) % n2 + n2) % n2) * n1 + xw;
  // planes k in [z0 - 1, z1] wrap at most once
  auto pbase = [&](int k) -> long long { return (long long)(k < 0 ? k + n3 : (k >= n3 ? k - n3 : k)) * plane; };
  R nq[SYT + 2];
  uint8_t nph[SYT + 1];
  auto fetch = [&](int k) {
    const long long b = pbase(k);
#pragma unroll
    for (int r = 0; r < SYT + 2; r++) nq[r] = q[b + ro[r]];
#pragma unroll
    for (int r = 0; r < SYT + 1; r++) nph[r] = phase[b + ro[r]];
  };
  // plane a (the lower plane of the current corner plane): q, q at x + 1,
  // l^2 at the corner index, and two terms of its corner derivatives kept
  // from the step where it was the upper plane: dx = q(x+1) - q(x) per row
  // and dy = the two x2 edge differences per corner row
  R qa[SYT + 2], qra[SYT + 2], wa[SYT + 1], dxa[SYT + 2], dya[SYT + 1];
  R Ap[SYT], Bp[SYT];                              // sums owed by corner plane k - 1/2
  auto take = [&](R* qv, R* qr, R* w, R* dx, R* dy) {
#pragma unroll
    for (int r = 0; r < SYT + 2; r++) {
      qv[r] = nq[r];
      qr[r] = __shfl_down_sync(kAll, nq[r], 1);
      dx[r] = qr[r] - qv[r];
    }
#pragma unroll
    for (int c = 0; c < SYT + 1; c++) dy[c] = (qv[c + 1] - qv[c]) + (qr[c + 1] - qr[c]);
#pragma unroll
    for (int r = 0; r < SYT + 1; r++) w[r] = l2[nph[r]];
  };
  // corner plane between planes a (low) and b (high): the sums it owes the
  // output plane above it (as its lower corner plane) and below it
  auto corner_plane = [&](const R* qb, const R* qrb, const R* dxb, const R* dyb, R* Alo, R* Blo, R* Ahi,
                          R* Bhi) {
    R zr[SYT + 2], fx[SYT + 1], fy[SYT + 1], fz[SYT + 1];
#pragma unroll
    for (int r = 0; r < SYT + 2; r++) zr[r] = (qb[r] - qa[r]) + (qrb[r] - qra[r]);
#pragma unroll
    for (int c = 0; c < SYT + 1; c++) {
      const R w = wa[c];
      fx[c] = (w * c0) * ((dxa[c] + dxa[c + 1]) + (dxb[c] + dxb[c + 1]));
      fy[c] = (w * c1) * (dya[c] + dyb[c]);
      fz[c] = (w * c2) * (zr[c] + zr[c + 1]);
    }
    // D_j^T: a corner on the low side of the voxel along x_j adds its flux
    // F_j, one on the high side subtracts it.  Row r's corners: c = r (at
    // y - 1/2) and c = r + 1 (at y + 1/2); the x3 flux enters with + for the
    // output plane above this corner plane and with - for the one below.
#pragma unroll
    for (int r = 0; r < SYT; r++) {
      const R P = (fx[r] + fy[r]) + (fx[r + 1] - fy[r + 1]);      // owed to the lane on the right
      const R Q = -((fx[r] - fy[r]) + (fx[r + 1] + fy[r + 1]));   // owed to this lane
      const R Z = fz[r] + fz[r + 1];
      Ahi[r] = P + Z;
      Bhi[r] = Q + Z;
      Alo[r] = P - Z;
      Blo[r] = Q - Z;
    }
  };
  fetch(z0 - 1);
  take(qa, qra, wa, dxa, dya);
  fetch(z0);
  {
    R qb[SYT + 2], qrb[SYT + 2], wb[SYT + 1], dxb[SYT + 2], dyb[SYT + 1], Ad[SYT], Bd[SYT];
    take(qb, qrb, wb, dxb, dyb);
    if (z0 + 1 <= z1) fetch(z0 + 1);
    corner_plane(qb, qrb, dxb, dyb, Ad, Bd, Ap, Bp);
#pragma unroll
    for (int r = 0; r < SYT + 2; r++) {
      qa[r] = qb[r];
      qra[r] = qrb[r];
      dxa[r] = dxb[r];
    }
#pragma unroll
    for (int r = 0; r < SYT + 1; r++) {
      wa[r] = wb[r];
      dya[r] = dyb[r];
    }
  }
  for (int k = z0; k < z1; k++) {
    R qb[SYT + 2], qrb[SYT + 2], wb[SYT + 1], dxb[SYT + 2], dyb[SYT + 1], Al[SYT], Bl[SYT], Ah[SYT], Bh[SYT];
    take(qb, qrb, wb, dxb, dyb);                   // plane k + 1
    if (k + 2 <= z1) fetch(k + 2);                 // in flight during this plane's arithmetic
    corner_plane(qb, qrb, dxb, dyb, Al, Bl, Ah, Bh);
    const long long ob = (long long)k * plane;
#pragma unroll
    for (int r = 0; r < SYT; r++) {
      const R v = __shfl_up_sync(kAll, Ap[r] + Al[r], 1) + (Bp[r] + Bl[r]);
      // the identity part of L is added to the spectrum, exactly, by the caller
      if (outx && y0 + r < n2) y[ob + ro[r + 1]] = v;
      Ap[r] = Ah[r];
      Bp[r] = Bh[r];
    }
#pragma unroll
    for (int r = 0; r < SYT + 2; r++) {
      qa[r] = qb[r];
      qra[r] = qrb[r];
      dxa[r] = dxb[r];
    }
#pragma unroll
    for (int r = 0; r < SYT + 1; r++) {
      wa[r] = wb[r];
      dya[r] = dyb[r];
    }
  }
}

// ------------------------------------------------------ x1 prologues / epilogues
// tau = C_T : p with the compact tangent descriptor
//   desc = [c1, c2, m_0 .. m_{NC-1}],  tau = c1 tr(p) 1 + c2 dev(p) - m (m . p)
// (c1 = (1-D) K, c2 = (1-D) 2 mu theta, m = sqrt((1-D) 2 mu thetabar) nhat).
// Inside CG the direction is refreshed first: p <- r (iter 0) or r + beta p.
template <typename R, int NC, bool EXT = false>
struct ProTangent {
  // (p, C_T : p) per CTA into part (when part is set): for p in the range of
  // the projection this equals (p, G*(C_T : p)), the CG curvature.
  // EXT: the descriptor holds A, B, C, D, nh (the GTN handles' tangent
  // A I(x)I + B P_dev + C nh(x)nh + D (I(x)nh + nh(x)I)); otherwise c1, c2, m
  // (c1 I(x)I + c2 P_dev - m(x)m).
  static constexpr bool kDot = true;
  R* p;
  const R* r;
  const R* desc;
  long long V;
  int update;
  R beta;
  bool first;
  double* part;
  int pstride;
  __device__ void begin(const KrylovCtl* ctl) {
    if (ctl) { first = ctl->iter == 0; beta = (R)ctl->beta; }
  }
  __device__ __forceinline__ void operator()(long long v, R (&out)[NC], R& acc) const {
    constexpr int NN = NC == 6 ? 3 : 2;
    // every load first (r, p, descriptor), then the store of the new p:
    // the store could alias the loads, so it would otherwise serialise them
    constexpr int M0 = EXT ? 4 : 2;
    R pv[NC], m[NC];
    const R c1 = desc[v], c2 = desc[V + v];
    R cc = R(0), dd = R(0);
    if constexpr (EXT) {
      cc = desc[2 * V + v];
      dd = desc[3 * V + v];
    }
#pragma unroll
    for (int c = 0; c < NC; c++) m[c] = desc[(M0 + c) * V + v];
    if (update) {
      R rv[NC], po[NC];
#pragma unroll
      for (int c = 0; c < NC; c++) {
        rv[c] = r[c * V + v];
        po[c] = first ? R(0) : p[c * V + v];
      }
#pragma unroll
      for (int c = 0; c < NC; c++) {
        pv[c] = first ? rv[c] : rv[c] + beta * po[c];
        p[c * V + v] = pv[c];
      }
    } else {
#pragma unroll
      for (int c = 0; c < NC; c++) pv[c] = p[c * V + v];
    }
    R tr = R(0), mp = R(0);
#pragma unroll
    for (int c = 0; c < NN; c++) tr += pv[c];
#pragma unroll
    for (int c = 0; c < NC; c++) mp += m[c] * pv[c];
    const R third = tr * R(1.0 / 3.0);
    // summed in the working precision per thread and warp, in FP64 above
    if constexpr (EXT) {
      const R w = cc * mp + dd * tr;
#pragma unroll
      for (int c = 0; c < NC; c++) {
        R o = c2 * pv[c] + w * m[c];
        if (c < NN) o += c1 * tr - c2 * third + dd * mp;
        out[c] = o;
        acc += pv[c] * o;
      }
    } else {
#pragma unroll
      for (int c = 0; c < NC; c++) {
        R o = c2 * pv[c] - m[c] * mp;
        if (c < NN) o += c1 * tr - c2 * third;
        out[c] = o;
        acc += pv[c] * o;
      }
    }
  }
};

// tau_c = f[map[c]][v] - mean[map[c]]  (FP64 source fields)
template <typename R, int NC>
struct ProField64 {
  static constexpr bool kDot = false;
  const double* f;
  const double* mean;   // device, may be null
  const double* f2;     // subtracted field (same layout as f), may be null
  const double* mean2;  // its mean, may be null
  long long V;
  int map[NC];
  double dm[NC];   // mean2 - mean per component
  __device__ void begin(const KrylovCtl*) {
#pragma unroll
    for (int c = 0; c < NC; c++) dm[c] = (mean2 ? mean2[map[c]] : 0.0) - (mean ? mean[map[c]] : 0.0);
  }
  __device__ __forceinline__ void operator()(long long v, R (&out)[NC]) const {
#pragma unroll
    for (int c = 0; c < NC; c++) {
      double x = f[map[c] * V + v];
      if (f2) x -= f2[map[c] * V + v];
      out[c] = (R)(x + dm[c]);
    }
  }
};

// cp.async of the CTA's rows of a [NC][V] field: pre[(r * NC + c) * n1 + x]
template <typename R, int NC>
__device__ __forceinline__ void prefetch_rows(R* pre, const R* f, long long V, long long row0, int rows,
                                              int n1) {
  constexpr int PER = 16 / (int)sizeof(R);
  const int cpr = n1 / PER;
  const int total = rows * NC * cpr;
  if (n1 % PER == 0) {
    for (int e = threadIdx.x; e < total; e += kThreads) {
      const int l = e / cpr, ch = e - l * cpr;
      const int r = l / NC, c = l - r * NC;
      cp_async16(pre + (size_t)l * n1 + ch * PER, f + c * V + (row0 + r) * n1 + ch * PER);
    }
  } else {
    for (int e = threadIdx.x; e < rows * NC * n1; e += kThreads) {
      const int l = e / n1, x = e - l * n1;
      const int r = l / NC, c = l - r * NC;
      pre[e] = f[c * V + (row0 + r) * n1 + x];
    }
  }
}

template <typename R, int NC>
struct EpiMatvec {       // Ap = val; acc0 += p . Ap   (p rows prefetched)
  static constexpr int kPrefetch = 1;
  R* Ap;
  const R* p;
  long long V;
  __device__ void begin(const KrylovCtl*) {}
  __device__ __forceinline__ void prefetch(R* pre, long long row0, int rows, int n1, int) const {
    prefetch_rows<R, NC>(pre, p, V, row0, rows, n1);
  }
  __device__ __forceinline__ void operator()(long long v, const R (&val)[NC], R* acc, const R* pv,
                                             int n1, int) const {
    // summed in the working precision per thread and warp, in FP64 above
#pragma unroll
    for (int c = 0; c < NC; c++) {
      Ap[c * V + v] = val[c];
      acc[0] += pv[c * n1] * val[c];
    }
  }
};

// CG step fused into the inverse x1 pass: with val = G*(C_T : p) at the
// voxel (never stored), x += alpha p, r -= alpha val, acc0 += r . r.  The
// rows of p, x and r are prefetched with the spectrum.
template <typename R, int NC>
struct EpiCG {
  static constexpr int kPrefetch = 3;
  R* x;
  R* r;
  const R* p;
  long long V;
  R alpha;
  __device__ void begin(const KrylovCtl* ctl) { alpha = (R)ctl->alpha; }
  __device__ __forceinline__ void prefetch(R* pre, long long row0, int rows, int n1, int fs) const {
    prefetch_rows<R, NC>(pre, p, V, row0, rows, n1);
    prefetch_rows<R, NC>(pre + fs, x, V, row0, rows, n1);
    prefetch_rows<R, NC>(pre + 2 * fs, r, V, row0, rows, n1);
  }
  __device__ __forceinline__ void operator()(long long v, const R (&val)[NC], R* acc, const R* pv,
                                             int n1, int fs) const {
#pragma unroll
    for (int c = 0; c < NC; c++) {
      const R pc = pv[c * n1], xc = pv[fs + c * n1], rc = pv[2 * fs + c * n1];
      x[c * V + v] = xc + alpha * pc;
      const R rn = rc - alpha * val[c];
      r[c * V + v] = rn;
      acc[0] += rn * rn;
    }
  }
};

template <typename R, typename RO, int NC>
// b = bref - (val + mask (mean_sigma - mean_ref - sbar)); acc0 += b . b
// (bref, mean_ref null for a plain residual)
struct EpiResidual {
  static constexpr int kPrefetch = 0;
  RO* b;
  const double* mean_sig;   // full Mandel (6)
  const double* mean_ref;   // full Mandel (6), may be null
  const RO* bref;           // [NC][V], may be null
  double mask[NC];
  double sbar[NC];
  int map[NC];
  long long V;
  double dc[NC];
  __device__ void begin(const KrylovCtl*) {
#pragma unroll
    for (int c = 0; c < NC; c++)
      dc[c] = mask[c] * (mean_sig[map[c]] - (mean_ref ? mean_ref[map[c]] : 0.0) - sbar[c]);
  }
  __device__ __forceinline__ void operator()(long long v, const R (&val)[NC], R* acc) const {
    RO part = RO(0);
#pragma unroll
    for (int c = 0; c < NC; c++) {
      RO br;
      if constexpr (sizeof(R) == 4) {
        // FP32 sweep: operands already FP32, the result stored in FP32
        br = (bref ? (R)bref[c * V + v] : R(0)) - (val[c] + (R)dc[c]);
      } else {
        const double bv = (bref ? (double)bref[c * V + v] : 0.0) - ((double)val[c] + dc[c]);
        br = (RO)bv;
      }
      b[c * V + v] = br;
      part += br * br;
    }
    acc[0] += (R)part;
  }
};

// out[v] = val (one component, working precision)
template <typename R>
struct EpiStoreR {
  static constexpr int kPrefetch = 0;
  R* out;
  __device__ void begin(const KrylovCtl*) {}
  __device__ __forceinline__ void operator()(long long v, const R (&val)[1], R*) const { out[v] = val[0]; }
};

// tau = f[v] (one component, working precision)
template <typename R>
struct ProFieldR {
  static constexpr bool kDot = false;
  const R* f;
  __device__ void begin(const KrylovCtl*) {}
  __device__ __forceinline__ void operator()(long long v, R (&out)[1]) const { out[0] = f[v]; }
};

template <typename R, int NC>
struct EpiStore64 {
  static constexpr int kPrefetch = 0;
  double* out;
  long long V;
  __device__ void begin(const KrylovCtl*) {}
  __device__ __forceinline__ void operator()(long long v, const R (&val)[NC], R*) const {
#pragma unroll
    for (int c = 0; c < NC; c++) out[c * V + v] = (double)val[c];
  }
};

// twiddle table bytes at the head of a strided kernel's shared memory,
// rounded up so that the tile behind it starts on a 16-byte boundary
template <typename R>
__host__ __device__ __forceinline__ size_t tw_bytes(int N) {
  return ((size_t)N * sizeof(C2<R>) + 15) & ~(size_t)15;
}

// Tile of ncomp components x N points x tx columns in shared memory:
// element (c, n, col) at (c N + n) tx + col, or with IL (components
// interleaved) at n rs + c tx + col (rs >= ncomp tx: the stride of one
// point's group of lines), where one batched transform of ncomp tx lines
// covers every component.  With SW (256-point axes) global row n maps to
// tile row reg_pos(n), the order of the register-pass spectrum.  Interleaved
// tiles are walked component-fastest so that a warp's shared-memory rows are
// adjacent.
template <bool IL, bool SW, int NAX = 256>
__device__ __forceinline__ int tile_off(int row, int ncomp, int N, int tx, int rs, long long cstride,
                                        long long astride, long long& goff) {
  int c, n;
  if (IL) { n = row / ncomp; c = row - n * ncomp; }
  else { c = row / N; n = row - c * N; }
  goff = c * cstride + n * astride;
  const int m = SW ? reg_pos<NAX>(n) : n;
  return IL ? m * rs + c * tx : (c * N + m) * tx;
}

template <typename R, bool IL = false, bool SW = false, int NAX = 256>
__device__ __forceinline__ void tile_load_async(C2<R>* buf, const C2<R>* src, int ncomp, long long cstride,
                                                int N, long long astride, int tx, int cols, int rs = 0) {
  constexpr int PER = 16 / (int)sizeof(C2<R>);
  const int cpr = (cols + PER - 1) / PER;
  const int total = ncomp * N * cpr;
  for (int e = threadIdx.x; e < total; e += kThreads) {
    const int row = e / cpr, ch = e - row * cpr;
    const int col = ch * PER;
    long long goff;
    C2<R>* d = buf + tile_off<IL, SW, NAX>(row, ncomp, N, tx, rs, cstride, astride, goff) + col;
    const C2<R>* sp = src + goff + col;
    if (PER == 2 && col + 1 >= cols) cp_async8(d, sp);
    else cp_async16(d, sp);
  }
  cp_async_wait_all();
}

template <typename R, bool IL = false, bool SW = false, int NAX = 256>
__device__ __forceinline__ void tile_store(const C2<R>* buf, C2<R>* dst, int ncomp, long long cstride, int N,
                                           long long astride, int tx, int cols, int rs = 0) {
  constexpr int PER = 16 / (int)sizeof(C2<R>);
  const int cpr = (cols + PER - 1) / PER;
  const int total = ncomp * N * cpr;
  for (int e = threadIdx.x; e < total; e += kThreads) {
    const int row = e / cpr, ch = e - row * cpr;
    const int col = ch * PER;
    long long goff;
    const C2<R>* sp = buf + tile_off<IL, SW, NAX>(row, ncomp, N, tx, rs, cstride, astride, goff) + col;
    C2<R>* d = dst + goff + col;
    if (PER == 2 && col + 1 >= cols) {
      d[0] = sp[0];
    } else if (PER == 2) {
      *reinterpret_cast<float4*>(d) = *reinterpret_cast<const float4*>(sp);
    } else {
      *reinterpret_cast<double2*>(d) = *reinterpret_cast<const double2*>(sp);
    }
  }
}

// ============================================================ strided passes
template <typename R>
struct StrideInfo { long long astride, ostride; int N; };

template <typename R>
static StrideInfo<R> stride_of(const Geo& g, int axis) {
  StrideInfo<R> s;
  if (axis == 1) { s.astride = g.ps; s.ostride = (long long)g.ps * g.n2; s.N = g.n2; }
  else { s.astride = (long long)g.ps * g.n2; s.ostride = g.ps; s.N = g.n3; }
  return s;
}

// Tile widths of the 256-point register-pass kernels (columns per CTA) for
// NCOMP components per tile: NCOMP * TX * 16 tasks per pass, about three per
// thread or fewer, and at most ~100 KB of shared memory.
template <typename R, int NCOMP> struct RegTx {
  static constexpr int v = sizeof(R) == 4 ? (NCOMP >= 3 ? 8 : 16) : (NCOMP >= 6 ? 4 : NCOMP >= 2 ? 8 : 16);
};
// Point stride of the interleaved tile: six-component tiles (four rows of a
// 32-lane warp per projection step) get 32 bytes of padding per point so
// that those rows fall on different banks.
template <typename R, int NCOMP> struct RegRs {
  static constexpr int v = NCOMP * RegTx<R, NCOMP>::v + (NCOMP >= 6 ? 32 / (int)sizeof(C2<R>) : 0);
};

// TXR > 0: NAX-point axis (64, 128 or 256) through the register passes, TXR
// columns per CTA.

template <typename R, int SIGN, int TXR = 0, int NAX = 256>
__global__ void __launch_bounds__(kThreads, (TXR > 0 && sizeof(R) == 4) ? 4 : 2)
k_strided_plain(Geo g, FftPlan pl, const C2<R>* __restrict__ tw, C2<R>* __restrict__ S, int tx,
                long long astride, long long ostride, const KrylovCtl* __restrict__ ctl) {
  if (ctl && ctl->done) return;
  constexpr int E = StridedE<R>::E;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int N = TXR ? NAX : pl.N;
  if (TXR) tx = TXR;
  C2<R>* tws = reinterpret_cast<C2<R>*>(smraw);
  C2<R>* buf = reinterpret_cast<C2<R>*>(smraw + tw_bytes<R>(N));
  const int q0 = blockIdx.x * tx;
  const int cols = min(tx, g.P1 - q0);
  C2<R>* base = S + blockIdx.z * g.sstride + blockIdx.y * ostride + q0;
  for (int i = threadIdx.x; i < N; i += kThreads) tws[i] = tw[i];
  if constexpr (TXR > 0) {
    // forward: natural rows in, spectrum stored from the reg_pos order;
    // inverse: spectrum loaded into the reg_pos order, natural rows out
    // full-width tiles (rows are padded to a multiple of 16 entries, so the
    // columns past P1 stay inside the row; their values are never used)
    tile_load_async<R, false, (SIGN > 0), NAX>(buf, base, 1, 0, NAX, astride, TXR, TXR);
    __syncthreads();
    if constexpr (SIGN < 0) fftreg_forward<R, NAX, TXR>(buf, tws);
    else fftreg_inverse<R, NAX, TXR>(buf, tws);
    tile_store<R, false, (SIGN < 0), NAX>(buf, base, 1, 0, NAX, astride, TXR, TXR);
  } else {
    tile_load_async(buf, base, 1, 0, N, astride, tx, cols);
    __syncthreads();
    fft_lines<R, E, SIGN>(buf, pl, cols, tx, 1, false, tws, 1);
    tile_store(buf, base, 1, 0, N, astride, tx, cols);
  }
}

// mode indices of element (n, col) of a last-axis tile
__device__ __forceinline__ void last_modes(const Geo& g, int q0, int col, int n, int& m0, int& m1,
                                           int& m2) {
  m0 = q0 + col;
  if (g.d == 3) { m1 = blockIdx.y; m2 = n; }
  else { m1 = n; m2 = 0; }
}

// Symbol factors of the last-axis kernels with the register passes: a
// thread keeps one column (axis-0 mode m0) and, in 3D, the CTA's y-plane
// (axis-1 mode m1) for all its points, so only the last-axis factors are
// looked up per point.  Same products, in the same order, as symbol().
template <typename R>
struct LastSym {
  R s0, c0, s1, c1;
  int m0, m1;
  __device__ __forceinline__ void init(const Geo& g, const Tables<R>& t, int m0_) {
    m0 = m0_;
    s0 = t.s[0][m0];
    c0 = t.c[0][m0];
    m1 = g.d == 3 ? (int)blockIdx.y : 0;
    s1 = t.s[1][m1];
    c1 = t.c[1][m1];
  }
  // 3D, last-axis factors s2 = sin, c2 = cos of mode f given (staged by the
  // caller): the same products as at()
  __device__ __forceinline__ void at3(const Tables<R>& t, int f, R s2, R c2, R a[3], bool& dc) const {
    a[0] = t.two_over_h[0] * s0 * c1 * c2;
    a[1] = t.two_over_h[1] * s1 * c0 * c2;
    a[2] = t.two_over_h[2] * s2 * c0 * c1;
    dc = m0 == 0 && m1 == 0 && f == 0;
  }
  // |k|^2 of mode (m0, m1, f) in 3D, (m0, f) in 2D (the preconditioner's
  // symbol; no phase factor)
  __device__ __forceinline__ R k2(const Geo& g, const Tables<R>& t, int f) const {
    if (g.d == 3) {
      const R s2 = t.s[2][f], c2 = t.c[2][f];
      const R a0 = t.two_over_h[0] * s0 * c1 * c2, a1 = t.two_over_h[1] * s1 * c0 * c2,
              a2 = t.two_over_h[2] * s2 * c0 * c1;
      return a0 * a0 + a1 * a1 + a2 * a2;
    }
    const R sf = t.s[1][f], cf = t.c[1][f];
    const R a0 = t.two_over_h[0] * s0 * cf, a1 = t.two_over_h[1] * sf * c0;
    return a0 * a0 + a1 * a1;
  }
  // modes (m0, m1, f) in 3D, (m0, f) in 2D
  __device__ __forceinline__ void at(const Geo& g, const Tables<R>& t, int f, R a[3], C2<R>& ph,
                                     bool& dc) const {
    if (g.d == 3) {
      const R s2 = t.s[2][f], c2 = t.c[2][f];
      a[0] = t.two_over_h[0] * s0 * c1 * c2;
      a[1] = t.two_over_h[1] * s1 * c0 * c2;
      a[2] = t.two_over_h[2] * s2 * c0 * c1;
      ph = cmul(cmul(mk<R>(c0, s0), mk<R>(c1, s1)), mk<R>(c2, s2));
      dc = m0 == 0 && m1 == 0 && f == 0;
    } else {
      const R sf = t.s[1][f], cf = t.c[1][f];
      a[0] = t.two_over_h[0] * s0 * cf;
      a[1] = t.two_over_h[1] * sf * c0;
      a[2] = R(0);
      ph = cmul(mk<R>(c0, s0), mk<R>(cf, sf));
      dc = m0 == 0 && f == 0;
    }
  }
};

template <typename R> __device__ __forceinline__ R inv_sqrt(R x);
template <> __device__ __forceinline__ float inv_sqrt<float>(float x) { return rsqrtf(x); }
template <> __device__ __forceinline__ double inv_sqrt<double>(double x) { return rsqrt(x); }

// Gamma* at one mode of symbol a: the projection for k != 0, the
// stress-control mask at the zero frequency (dc_mode 0), zero at the hidden
// zeros of the symbol
template <typename R, int NC>
__device__ __forceinline__ void gamma_apply(const R a[3], bool dc, const Mask6& mask, int dc_mode,
                                            C2<R> (&tv)[NC]) {
  const R a2 = a[0] * a[0] + a[1] * a[1] + a[2] * a[2];
  if (a2 > R(0)) {
    const R inv = inv_sqrt<R>(a2);
    R nv[3] = {a[0] * inv, a[1] * inv, a[2] * inv};
    gamma_mode<R>(NC == 6 ? 3 : 2, nv, tv);
  } else {
#pragma unroll
    for (int c = 0; c < NC; c++) tv[c] = (dc && !dc_mode) ? cscale(tv[c], (R)mask.m[c]) : mk<R>(0, 0);
  }
}

// TXR > 0: NAX-point last axis (64, 128, 256) through the register passes,
// TXR columns per CTA, the NC components interleaved in the tile and
// transformed as one
// batch of NC TXR lines; the projection runs on the reg_pos spectrum order.
template <typename R, int NC, int TXR = 0, int NAX = 256>
__global__ void __launch_bounds__(kThreads, 2)
k_gamma(Geo g, Tables<R> t, FftPlan pl, const C2<R>* __restrict__ tw, C2<R>* __restrict__ S, int tx,
        long long astride, long long ostride, Mask6 mask, int dc_mode,
        const KrylovCtl* __restrict__ ctl) {
  if (ctl && ctl->done) return;
  constexpr int E = StridedE<R>::E;
  constexpr int nc = NC;
  constexpr bool IL = TXR > 0;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int N = TXR ? NAX : pl.N;
  if (TXR) tx = TXR;
  C2<R>* tws = reinterpret_cast<C2<R>*>(smraw);
  C2<R>* buf = reinterpret_cast<C2<R>*>(smraw + tw_bytes<R>(N));
  const int q0 = blockIdx.x * tx;
  const int cols = min(tx, g.P1 - q0);
  C2<R>* base = S + blockIdx.y * ostride + q0;
  const int tile = N * tx;
  constexpr int RS = IL ? RegRs<R, NC>::v : 0;
  for (int i = threadIdx.x; i < N; i += kThreads) tws[i] = tw[i];
  tile_load_async<R, IL>(buf, base, nc, g.sstride, N, astride, tx, IL ? TXR : cols, RS);
  __syncthreads();
  if constexpr (IL) {
    fftreg_forward<R, NAX, NC * TXR, RS>(buf, tws);
  } else {
    for (int c = 0; c < nc; c++) fft_lines<R, E, -1>(buf + c * tile, pl, cols, tx, 1, false, tws, 1);
  }
  if constexpr (IL) {
    // the register passes leave frequency reg_freq(n) at tile row n
    constexpr int RPT = kThreads / TXR;
    const int col = threadIdx.x % TXR;
    if (col < cols) {
      LastSym<R> sy;
      sy.init(g, t, q0 + col);
#pragma unroll 2
      for (int n = threadIdx.x / TXR; n < NAX; n += RPT) {
        R a[3];
        C2<R> ph;
        bool dc;
        sy.at(g, t, reg_freq<NAX>(n), a, ph, dc);
        C2<R> tv[NC];
#pragma unroll
        for (int c = 0; c < nc; c++) tv[c] = buf[n * RS + c * TXR + col];
        gamma_apply<R, NC>(a, dc, mask, dc_mode, tv);
#pragma unroll
        for (int c = 0; c < nc; c++) buf[n * RS + c * TXR + col] = tv[c];
      }
    }
  } else {
    for (int e = threadIdx.x; e < tile; e += kThreads) {
      const int n = e / tx, col = e - n * tx;
      if (col >= cols) continue;
      int m0, m1, m2;
      last_modes(g, q0, col, n, m0, m1, m2);
      R a[3];
      C2<R> ph;
      symbol(g, t, m0, m1, m2, a, ph);
      C2<R> tv[NC];
#pragma unroll
      for (int c = 0; c < nc; c++) tv[c] = buf[e + c * tile];
      gamma_apply<R, NC>(a, m0 == 0 && m1 == 0 && m2 == 0, mask, dc_mode, tv);
#pragma unroll
      for (int c = 0; c < nc; c++) buf[e + c * tile] = tv[c];
    }
  }
  __syncthreads();
  if constexpr (IL) {
    fftreg_inverse<R, NAX, NC * TXR, RS>(buf, tws);
  } else {
    for (int c = 0; c < nc; c++) fft_lines<R, E, +1>(buf + c * tile, pl, cols, tx, 1, false, tws, 1);
  }
  tile_store<R, IL>(buf, base, nc, g.sstride, N, astride, tx, IL ? TXR : cols, RS);
}

// bytes ahead of the tile in the TMA last-axis pass: twiddles, the sin and
// cos tables of the last axis, rounded up to 128 bytes
template <typename R>
__host__ __device__ __forceinline__ size_t gamma_tma_head(int N) {
  return (tw_bytes<R>(N) + 2 * (size_t)N * sizeof(R) + 127) & ~(size_t)127;
}

// The same last-axis pass in 3D with the tile moved by the tensor memory
// accelerator: one box {TXR columns, NC components, one y plane, NAX z
// points} lands as [z][c][col] (point stride NC TXR, no padding), and goes
// back the same way.  A CTA that waits longer than wait_ns for its tile
// records it in *wait_err and skips the tile.  extra_tx > 0 (tests of that
// path only) adds bytes that no copy delivers to the expected count, so the
// wait runs out although the copy lands; the CTA then counts those bytes
// itself, so the phase completes and no copy is in flight when it returns.
//
// NTH threads per CTA: 256 with the default tile (two CTAs per SM), 128 with
// a tile half as wide (four CTAs per SM, so that more tiles are in flight
// per SM); the per-column arithmetic is the same, so are the results.
template <typename R, int NC, int TXR, int NAX, int NTH = kThreads>
__global__ void __launch_bounds__(NTH, NTH == kThreads ? 2 : 4)
k_gamma_tma(Geo g, Tables<R> t, const __grid_constant__ CUtensorMap tmap, const C2<R>* __restrict__ tw,
            Mask6 mask, int dc_mode, const KrylovCtl* __restrict__ ctl, int* __restrict__ wait_err,
            unsigned long long wait_ns, unsigned extra_tx) {
  if (ctl && ctl->done) return;
  constexpr int RS = NC * TXR;
  constexpr int U8 = (int)sizeof(C2<R>) / 8;    // 8-byte elements per complex entry
  constexpr uint32_t kBytes = (uint32_t)(NAX * RS * sizeof(C2<R>));
  extern __shared__ __align__(128) unsigned char smtma[];
  __shared__ __align__(8) uint64_t bar;
  C2<R>* tws = reinterpret_cast<C2<R>*>(smtma);
  R* zs = reinterpret_cast<R*>(smtma + tw_bytes<R>(NAX));   // sin, cos of the last-axis modes
  R* zc = zs + NAX;
  C2<R>* buf = reinterpret_cast<C2<R>*>(smtma + gamma_tma_head<R>(NAX));
  const int q0 = blockIdx.x * TXR;
  const int cols = min(TXR, g.P1 - q0);
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_expect_tx(&bar, kBytes + extra_tx);
    tma_load_4d(buf, &tmap, q0 * U8, 0, blockIdx.y, 0, &bar);
  }
  for (int i = threadIdx.x; i < NAX; i += NTH) {
    tws[i] = tw[i];
    zs[i] = t.s[2][i];
    zc[i] = t.c[2][i];
  }
  __syncthreads();
  if (!mbar_wait(&bar, 0, wait_ns)) {
    if (threadIdx.x == 0) {
      if (wait_err) atomicExch(wait_err, 1);
      if (extra_tx) mbar_complete_tx(&bar, extra_tx);
    }
    mbar_wait(&bar, 0, wait_ns);   // the copy in flight, once more bounded
    return;
  }
  fftreg_forward<R, NAX, NC * TXR, RS, NTH>(buf, tws);
  {
    // the register passes leave frequency reg_freq(n) at tile row n
    constexpr int RPT = NTH / TXR;
    const int col = threadIdx.x % TXR;
    if (col < cols) {
      LastSym<R> sy;
      sy.init(g, t, q0 + col);
#pragma unroll 2
      for (int n = threadIdx.x / TXR; n < NAX; n += RPT) {
        R a[3];
        bool dc;
        const int f = reg_freq<NAX>(n);
        sy.at3(t, f, zs[f], zc[f], a, dc);
        C2<R> tv[NC];
#pragma unroll
        for (int c = 0; c < NC; c++) tv[c] = buf[n * RS + c * TXR + col];
        gamma_apply<R, NC>(a, dc, mask, dc_mode, tv);
#pragma unroll
        for (int c = 0; c < NC; c++) buf[n * RS + c * TXR + col] = tv[c];
      }
    }
  }
  __syncthreads();
  fftreg_inverse<R, NAX, NC * TXR, RS, NTH>(buf, tws);
  tma_fence_smem();
  __syncthreads();
  if (threadIdx.x == 0) tma_store_4d_and_wait(&tmap, buf, q0 * U8, 0, blockIdx.y, 0);
}

template <typename R>
__device__ __forceinline__ R q1_weight(const Geo& g, int q1) {
  return (q1 == 0 || 2 * q1 == g.n1) ? R(1) : R(2);
}

// Helmholtz: p <- M r + beta p (M = 1/(1 + <l^2>|k|^2)); W = p (one
// component, D = 0: the operator is applied in real space) or W_j = k_j p
// (D > 0); inverse transform along the last axis.
template <typename R, int D, int TXR = 0, int NAX = 256>
__global__ void __launch_bounds__(kThreads, D == 0 && TXR > 0 && sizeof(R) == 4 ? 4 : 2)
k_expand(Geo g, Tables<R> t, FftPlan pl, const C2<R>* __restrict__ tw, C2<R>* __restrict__ W,
         C2<R>* __restrict__ p, const C2<R>* __restrict__ r, int tx, long long astride,
         long long ostride, R ell2m, const KrylovCtl* __restrict__ ctl, int raw) {
  if (ctl && ctl->done) return;
  constexpr int E = StridedE<R>::E;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int N = TXR ? NAX : pl.N;
  if (TXR) tx = TXR;
  constexpr int d = D > 0 ? D : 1;   // transformed components
  constexpr bool IL = TXR > 0;
  C2<R>* tws = reinterpret_cast<C2<R>*>(smraw);
  C2<R>* buf = reinterpret_cast<C2<R>*>(smraw + tw_bytes<R>(N));
  const int q0 = blockIdx.x * tx;
  const int cols = min(tx, g.P1 - q0);
  const long long off = blockIdx.y * ostride + q0;
  const int tile = N * tx;
  const bool first = ctl ? ctl->iter == 0 : true;
  const R beta = ctl ? (R)ctl->beta : R(0);
  for (int i = threadIdx.x; i < N; i += kThreads) tws[i] = tw[i];
  if constexpr (IL && D == 0) {
    // one column per thread; every load of the thread's entries first, then
    // p <- M r + beta p (only |k|^2 needed) into tile row reg_pos(n)
    constexpr int RPT = kThreads / TXR;
    constexpr int PER = NAX / RPT;
    const int col = threadIdx.x % TXR, r0 = threadIdx.x / TXR;
    if (col < cols) {
      // two halves of the thread's entries, each with all its loads issued
      // before it is used (registers for four CTAs per SM)
      constexpr int HALF = PER / 2;
      const bool upd = !raw && !first;
      LastSym<R> sy;
      sy.init(g, t, q0 + col);
#pragma unroll 1
      for (int h = 0; h < 2; h++) {
        C2<R> rv[HALF], pv[HALF];
#pragma unroll
        for (int k = 0; k < HALF; k++) {
          const long long idx = off + (long long)(r0 + (h * HALF + k) * RPT) * astride + col;
          rv[k] = r[idx];
          pv[k] = upd ? p[idx] : mk<R>(0, 0);
        }
#pragma unroll
        for (int k = 0; k < HALF; k++) {
          const int n = r0 + (h * HALF + k) * RPT;
          C2<R> pn = rv[k];
          if (!raw) {
            const R Mk = R(1) / (R(1) + ell2m * sy.k2(g, t, n));
            pn = cscale(rv[k], Mk);
            if (upd) pn = pn + cscale(pv[k], beta);
            p[off + (long long)n * astride + col] = pn;
          }
          buf[reg_pos<NAX>(n) * TXR + col] = pn;
        }
      }
    }
  } else if constexpr (IL) {
    // one column per thread; frequency n goes to tile row reg_pos(n)
    constexpr int RPT = kThreads / TXR;
    const int col = threadIdx.x % TXR;
    if (col < cols) {
      LastSym<R> sy;
      sy.init(g, t, q0 + col);
#pragma unroll 4
      for (int n = threadIdx.x / TXR; n < NAX; n += RPT) {
        R a[3];
        C2<R> ph;
        bool dc;
        sy.at(g, t, n, a, ph, dc);
        const R Mk = R(1) / (R(1) + ell2m * (a[0] * a[0] + a[1] * a[1] + a[2] * a[2]));
        const long long idx = off + n * astride + col;
        C2<R> pn;
        if (raw) {
          pn = r[idx];
        } else {
          pn = cscale(r[idx], Mk);
          if (!first) pn = pn + cscale(p[idx], beta);
          p[idx] = pn;
        }
        const int e0 = reg_pos<NAX>(n) * (d * TXR) + col;
        if constexpr (D == 0) {
          buf[e0] = pn;
        } else {
          const C2<R> ipp = mul_si<R, 1>(cmul(ph, pn));      // i e^{i phi} p
#pragma unroll
          for (int j = 0; j < d; j++) buf[e0 + j * TXR] = cscale(ipp, a[j]);
        }
      }
    }
  } else {
    for (int e = threadIdx.x; e < tile; e += kThreads) {
      const int n = e / tx, col = e - n * tx;
      if (col >= cols) continue;
      int m0, m1, m2;
      last_modes(g, q0, col, n, m0, m1, m2);
      R a[3];
      C2<R> ph;
      symbol(g, t, m0, m1, m2, a, ph);
      const R Mk = R(1) / (R(1) + ell2m * (a[0] * a[0] + a[1] * a[1] + a[2] * a[2]));
      const long long idx = off + n * astride + col;
      C2<R> pn;
      if (raw) {
        pn = r[idx];
      } else {
        pn = cscale(r[idx], Mk);
        if (!first) pn = pn + cscale(p[idx], beta);
        p[idx] = pn;
      }
      if constexpr (D == 0) {
        buf[e] = pn;
      } else {
        const C2<R> ipp = mul_si<R, 1>(cmul(ph, pn));      // i e^{i phi} p
        for (int j = 0; j < d; j++) buf[e + j * tile] = cscale(ipp, a[j]);
      }
    }
  }
  __syncthreads();
  if constexpr (IL) {
    fftreg_inverse<R, NAX, d * TXR>(buf, tws);
  } else {
    for (int j = 0; j < d; j++) fft_lines<R, E, +1>(buf + j * tile, pl, cols, tx, 1, false, tws, 1);
  }
  tile_store<R, IL>(buf, W + off, d, g.sstride, N, astride, tx, IL ? TXR : cols, d * tx);
}

// Helmholtz: forward transform along the last axis, y = p + W (D = 0: W is
// the transform of the real-space flux term, the identity added here exactly)
// or y = p + sum conj(k_j) W_j (D > 0); partial Hermitian-weighted (p, y).
template <typename R, int D, int TXR = 0, int NAX = 256>
__global__ void __launch_bounds__(kThreads, 3)
k_contract(Geo g, Tables<R> t, FftPlan pl, const C2<R>* __restrict__ tw, const C2<R>* __restrict__ W,
           const C2<R>* __restrict__ p, C2<R>* __restrict__ y, int tx, long long astride,
           long long ostride, double* __restrict__ part, int pstride,
           const KrylovCtl* __restrict__ ctl) {
  if (ctl && ctl->done) return;
  constexpr int E = StridedE<R>::E;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int N = TXR ? NAX : pl.N;
  if (TXR) tx = TXR;
  constexpr int d = D > 0 ? D : 1;   // transformed components
  constexpr bool IL = TXR > 0;
  C2<R>* tws = reinterpret_cast<C2<R>*>(smraw);
  C2<R>* buf = reinterpret_cast<C2<R>*>(smraw + tw_bytes<R>(N));
  const int q0 = blockIdx.x * tx;
  const int cols = min(tx, g.P1 - q0);
  const long long off = blockIdx.y * ostride + q0;
  const int tile = N * tx;
  for (int i = threadIdx.x; i < N; i += kThreads) tws[i] = tw[i];
  // register path: this thread's entries of p, fetched while the tile is
  // transformed
  constexpr int RPT = TXR ? kThreads / TXR : 1;
  constexpr int PER = TXR ? NAX / RPT : 1;
  C2<R> pv[PER];
  if constexpr (IL) {
    const int col = threadIdx.x % TXR;
    if (col < cols) {
#pragma unroll
      for (int k = 0; k < PER; k++) pv[k] = p[off + (threadIdx.x / TXR + k * RPT) * astride + col];
    }
  }
  tile_load_async<R, IL>(buf, W + off, d, g.sstride, N, astride, tx, IL ? TXR : cols, d * tx);
  __syncthreads();
  if constexpr (IL) {
    fftreg_forward<R, NAX, d * TXR>(buf, tws);
  } else {
    for (int j = 0; j < d; j++) fft_lines<R, E, -1>(buf + j * tile, pl, cols, tx, 1, false, tws, 1);
  }
  R acc[1] = {R(0)};
  if constexpr (IL) {
    const int col = threadIdx.x % TXR;
    if (col < cols) {
      LastSym<R> sy;
      sy.init(g, t, q0 + col);
      const R w1 = q1_weight<R>(g, q0 + col);
#pragma unroll
      for (int k = 0; k < PER; k++) {
        const int n = threadIdx.x / TXR + k * RPT;
        const int e0 = reg_pos<NAX>(n) * (d * TXR) + col;
        C2<R> yv;
        if constexpr (D == 0) {
          yv = pv[k] + buf[e0];
        } else {
          R a[3];
          C2<R> ph;
          bool dc;
          sy.at(g, t, n, a, ph, dc);
          C2<R> s = mk<R>(0, 0);
#pragma unroll
          for (int j = 0; j < d; j++) s = s + cscale(buf[e0 + j * TXR], a[j]);
          // conj(k_j) = -i e^{-i phi} a_j
          const C2<R> ks = mul_si<R, -1>(cmul(conj_(ph), s));
          yv = pv[k] + ks;
        }
        y[off + n * astride + col] = yv;
        acc[0] += w1 * (pv[k].x * yv.x + pv[k].y * yv.y);
      }
    }
  } else {
    for (int e = threadIdx.x; e < tile; e += kThreads) {
      const int n = e / tx, col = e - n * tx;
      if (col >= cols) continue;
      int m0, m1, m2;
      last_modes(g, q0, col, n, m0, m1, m2);
      const long long idx = off + n * astride + col;
      const C2<R> pn = p[idx];
      C2<R> yv;
      if constexpr (D == 0) {
        yv = pn + buf[e];
      } else {
        R a[3];
        C2<R> ph;
        symbol(g, t, m0, m1, m2, a, ph);
        C2<R> s = mk<R>(0, 0);
        for (int j = 0; j < d; j++) s = s + cscale(buf[e + j * tile], a[j]);
        // conj(k_j) = -i e^{-i phi} a_j
        const C2<R> ks = mul_si<R, -1>(cmul(conj_(ph), s));
        yv = pn + ks;
      }
      y[idx] = yv;
      acc[0] += q1_weight<R>(g, m0) * (pn.x * yv.x + pn.y * yv.y);
    }
  }
  block_sum_store<1>(acc, part, pstride);
}

// ============================================================ Krylov vectors
template <typename R>
__global__ void __launch_bounds__(kThreads)
k_cg_init(long long n, R* __restrict__ x, const R* __restrict__ r, double* __restrict__ part, int pstride) {
  double acc[1] = {0.0};
  for (long long i = blockIdx.x * (long long)kThreads + threadIdx.x; i < n; i += (long long)gridDim.x * kThreads) {
    x[i] = R(0);
    const double rv = r[i];
    acc[0] += rv * rv;
  }
  block_sum_store<1>(acc, part, pstride);
}

// 16-byte vector of the working precision
template <typename R> struct Vec16;
template <> struct Vec16<float> { using T = float4; static constexpr int n = 4; };
template <> struct Vec16<double> { using T = double2; static constexpr int n = 2; };

template <typename R>
__device__ __forceinline__ R vdot_self(const typename Vec16<R>::T& a);
template <> __device__ __forceinline__ float vdot_self<float>(const float4& a) {
  return a.x * a.x + a.y * a.y + a.z * a.z + a.w * a.w;
}
template <> __device__ __forceinline__ double vdot_self<double>(const double2& a) {
  return a.x * a.x + a.y * a.y;
}
template <typename R>
__device__ __forceinline__ void vaxpy(typename Vec16<R>::T& y, R a, const typename Vec16<R>::T& x);
template <> __device__ __forceinline__ void vaxpy<float>(float4& y, float a, const float4& x) {
  y.x += a * x.x; y.y += a * x.y; y.z += a * x.z; y.w += a * x.w;
}
template <> __device__ __forceinline__ void vaxpy<double>(double2& y, double a, const double2& x) {
  y.x += a * x.x; y.y += a * x.y;
}

// x += alpha p, r -= alpha Ap, partial (r, r): 16-byte vectors; the terms
// summed in the working precision per thread and warp, in FP64 above
template <typename R>
__global__ void __launch_bounds__(kThreads)
k_cg_update(long long n, R* __restrict__ x, R* __restrict__ r, const R* __restrict__ p,
            const R* __restrict__ Ap, double* __restrict__ part, int pstride,
            const KrylovCtl* __restrict__ ctl) {
  if (ctl->done) return;
  using VT = typename Vec16<R>::T;
  constexpr int VN = Vec16<R>::n;
  const R alpha = (R)ctl->alpha;
  R acc[1] = {R(0)};
  const long long nv = n / VN;
  VT* xv = reinterpret_cast<VT*>(x);
  VT* rv = reinterpret_cast<VT*>(r);
  const VT* pv = reinterpret_cast<const VT*>(p);
  const VT* av = reinterpret_cast<const VT*>(Ap);
  for (long long i = blockIdx.x * (long long)kThreads + threadIdx.x; i < nv; i += (long long)gridDim.x * kThreads) {
    VT xi = xv[i], ri = rv[i];
    const VT pi = pv[i], ai = av[i];
    vaxpy<R>(xi, alpha, pi);
    vaxpy<R>(ri, -alpha, ai);
    xv[i] = xi;
    rv[i] = ri;
    acc[0] += vdot_self<R>(ri);
  }
  for (long long i = nv * VN + blockIdx.x * (long long)kThreads + threadIdx.x; i < n;
       i += (long long)gridDim.x * kThreads) {
    x[i] += alpha * p[i];
    const R rn = r[i] - alpha * Ap[i];
    r[i] = rn;
    acc[0] += rn * rn;
  }
  block_sum_store<1>(acc, part, pstride);
}

template <typename R>
__device__ __forceinline__ R precond_at(const Geo& g, const Tables<R>& t, long long e, R ell2m,
                                        int& q1) {
  const long long line = e / g.P1;
  q1 = (int)(e - line * g.P1);
  const int m1 = (int)(line % g.n2), m2 = (int)(line / g.n2);
  R a[3];
  C2<R> ph;
  symbol(g, t, q1, m1, m2, a, ph);
  return R(1) / (R(1) + ell2m * (a[0] * a[0] + a[1] * a[1] + a[2] * a[2]));
}

template <typename R>
__global__ void __launch_bounds__(kThreads)
k_pcg_init(Geo g, Tables<R> t, C2<R>* __restrict__ x, const C2<R>* __restrict__ r, R ell2m,
           double* __restrict__ part, int pstride) {
  double acc[2] = {0.0, 0.0};
  const long long n = (long long)g.P1 * g.nlines;
  for (long long e = blockIdx.x * (long long)kThreads + threadIdx.x; e < n; e += (long long)gridDim.x * kThreads) {
    int q1;
    const R Mk = precond_at(g, t, e, ell2m, q1);
    const long long idx = (e / g.P1) * g.ps + q1;
    x[idx] = mk<R>(0, 0);
    const C2<R> rv = r[idx];
    const double w = q1_weight<R>(g, q1);
    const double rr = (double)rv.x * rv.x + (double)rv.y * rv.y;
    acc[0] += w * rr;
    acc[1] += w * (double)Mk * rr;
  }
  block_sum_store<2>(acc, part, pstride);
}

// Element e of the flat half spectrum (line e / P1, column e % P1), split
// without a 64-bit division: a float estimate of the quotient (off by at
// most one below about 5 M lines, by a few beyond) is corrected exactly.
__device__ __forceinline__ void split_flat(long long e, int P1, float invP1, long long& line, int& q1) {
  long long l = (long long)((float)e * invP1);
  long long r = e - l * P1;
  while (r < 0) { l -= 1; r += P1; }
  while (r >= P1) { l += 1; r -= P1; }
  line = l;
  q1 = (int)r;
}

// M = 1 / (1 + <l^2> |k|^2) at column q1 of the line with modes (m1, m2)
template <typename R>
__device__ __forceinline__ R precond_mode(const Geo& g, const Tables<R>& t, int q1, int m1, int m2, R ell2m) {
  R a[3];
  C2<R> ph;
  symbol(g, t, q1, m1, m2, a, ph);
  return R(1) / (R(1) + ell2m * (a[0] * a[0] + a[1] * a[1] + a[2] * a[2]));
}

// x += alpha p, r -= alpha y over the half spectrum; partial (r, r) and
// (r, M r) with the Hermitian weights.  One 16-byte vector of complex
// entries per thread and step over the padded rows (entries past P1 are
// updated too, their values are never used); the terms are summed in the
// working precision per thread and warp, in FP64 above.
template <typename R>
__global__ void __launch_bounds__(kThreads)
k_pcg_update(Geo g, Tables<R> t, C2<R>* __restrict__ x, C2<R>* __restrict__ r,
             const C2<R>* __restrict__ p, const C2<R>* __restrict__ y, R ell2m,
             double* __restrict__ part, int pstride, const KrylovCtl* __restrict__ ctl) {
  if (ctl->done) return;
  using VT = typename Vec16<R>::T;
  constexpr int U = 16 / (int)sizeof(C2<R>);   // complex entries per vector
  const R alpha = (R)ctl->alpha;
  R acc[2] = {R(0), R(0)};
  const int upl = g.ps / U;                    // vectors per padded row
  const long long nu = (long long)upl * g.nlines;
  const float inv_upl = 1.0f / (float)upl;
  for (long long u = blockIdx.x * (long long)kThreads + threadIdx.x; u < nu;
       u += (long long)gridDim.x * kThreads) {
    long long line;
    int jv;
    split_flat(u, upl, inv_upl, line, jv);
    // line = m1 + n2 m2 (32-bit: fewer than 2^31 lines)
    const int m2 = (int)((unsigned)line / (unsigned)g.n2), m1 = (int)line - m2 * g.n2;
    const long long base = line * g.ps + (long long)jv * U;
    alignas(16) C2<R> xe[U], re[U], pe[U], ye[U];
    *reinterpret_cast<VT*>(xe) = *reinterpret_cast<const VT*>(x + base);
    *reinterpret_cast<VT*>(re) = *reinterpret_cast<const VT*>(r + base);
    *reinterpret_cast<VT*>(pe) = *reinterpret_cast<const VT*>(p + base);
    *reinterpret_cast<VT*>(ye) = *reinterpret_cast<const VT*>(y + base);
#pragma unroll
    for (int i = 0; i < U; i++) {
      const int q1 = jv * U + i;
      xe[i] = xe[i] + cscale(pe[i], alpha);
      re[i] = re[i] - cscale(ye[i], alpha);
      if (q1 < g.P1) {
        const R Mk = precond_mode(g, t, q1, m1, m2, ell2m);
        const R wrr = q1_weight<R>(g, q1) * (re[i].x * re[i].x + re[i].y * re[i].y);
        acc[0] += wrr;
        acc[1] += Mk * wrr;
      }
    }
    *reinterpret_cast<VT*>(x + base) = *reinterpret_cast<const VT*>(xe);
    *reinterpret_cast<VT*>(r + base) = *reinterpret_cast<const VT*>(re);
  }
  block_sum_store<2>(acc, part, pstride);
}

// ============================================================ return map
// Backward-Euler Lemaitre update (Appendix A.2; readings R8-R11) at every
// voxel: radial return on the effective stress, D from the frozen non-local
// variable, sigma = (1 - D) sigma_eff, consistent tangent descriptor.
// One Jacobi rotation of a symmetric 3x3 matrix zeroing entry (P, Q)
// (Golub & Van Loan, Sec. 8.5: t = tan of the rotation angle, the smaller
// root of t^2 + 2 theta t - 1 = 0 with theta = (a_QQ - a_PP) / (2 a_PQ)).
template <int P, int Q>
__device__ __forceinline__ void jacobi_rot3(double (&A)[3][3]) {
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
}

// ||<eps>_+||: Euclidean norm of the positive eigenvalues of the symmetric
// strain tensor given in Mandel components (cyclic Jacobi sweeps until the
// off-diagonal part is below 1e-32 of the squared norm, at most 12 sweeps).
__device__ __forceinline__ double positive_principal_norm(const double (&e)[6]) {
  const double r2 = 0.70710678118654752440;
  double A[3][3] = {{e[0], e[5] * r2, e[4] * r2}, {e[5] * r2, e[1], e[3] * r2}, {e[4] * r2, e[3] * r2, e[2]}};
  const double n2 = e[0] * e[0] + e[1] * e[1] + e[2] * e[2] + e[3] * e[3] + e[4] * e[4] + e[5] * e[5];
  for (int sweep = 0; sweep < 12; sweep++) {
    const double off = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
    if (!(off > 1e-32 * n2)) break;
    jacobi_rot3<0, 1>(A);
    jacobi_rot3<0, 2>(A);
    jacobi_rot3<1, 2>(A);
  }
  double k = 0.0;
  for (int i = 0; i < 3; i++) {
    const double l = A[i][i] > 0.0 ? A[i][i] : 0.0;
    k += l * l;
  }
  return sqrt(k);
}

// Flow stress sigma_0(e) and slope d sigma_0 / d e of a phase.  Linear:
// sigma_y + H e.  Aravas power law (Section 4.1, Eq. aravas):
// y = sigma_0 / sigma_y solves g(y) = y - (y + c)^N = 0 with c = 3 mu e /
// sigma_y; g is increasing and convex on y >= 1 with g(1) <= 0, so Newton
// from y = 1 lands right of the root after one step and then decreases
// monotonically onto it.  Slope: 3 mu w / (1 - w), w = N (y + c)^(N - 1).
__device__ __forceinline__ void flow_stress(const PhaseDev& P, double e, double& s0, double& Hp) {
  if (P.hard == 0) {
    s0 = P.sigma_y + P.H * e;
    Hp = P.H;
    return;
  }
  const double c = P.c_hard * e;
  double y = 1.0;
  for (int it = 0; it < 60; it++) {
    const double z = pow(y + c, P.N);
    const double w = P.N * z / (y + c);
    const double dy = (y - z) / (1.0 - w);
    y -= dy;
    if (fabs(dy) <= 1e-16 * y) break;
  }
  const double w = P.N * pow(y + c, P.N - 1.0);
  s0 = P.sigma_y * y;
  Hp = P.sigma_y * P.c_hard * w / (1.0 - w);
}

// ------------------------------------------------ Gurson-Tvergaard-Needleman
// Backward-Euler update of one voxel of the non-local GTN model (Section
// 2.1.1, Section 2.2.2, Appendix A.1) with the porosity f (hence f*) fixed by
// the frozen non-local variables.  Unknowns x = (d_v, d_q, e0): the plastic
// strain increment d_v I/3 + d_q n along the trial direction n =
// (3/2) s_dev / s (normality of the cosh surface), the matrix equivalent
// plastic strain e0; pressure p = p_tr + K d_v, Mises stress s = s_tr -
// 3 mu d_q.  Residuals:
//   R1 = (s/s0)^2 + 2 f* q1 cosh(3 q2 p / (2 s0)) - 1 - q3 f*^2     (yield)
//   R2 = 2 s d_v / s0 + 3 q1 q2 f* sinh(3 q2 p / (2 s0)) d_q      (normality)
//   R3 = (1 - f)(e0 - e0_n) + (p d_v - s d_q) / s0                (work balance)
// solved by Newton with backtracking; the consistent tangent (f fixed) is
// A I(x)I + B P_dev + C nh(x)nh + D (I(x)nh + nh(x)I), nh = n / |n|, from the
// derivatives of x with respect to the trial invariants (s_tr, p_tr).
struct GtnPoint {
  double sig[6], dep[6];
  double e0, f, fs;
  double A, B, C, D, nh[6];
  int ok;
};

__device__ __forceinline__ void gtn_eval(const PhaseDev& P, double K, double mu, double f, double fs, double s_tr,
                                         double p_tr, double e0n, double dv, double dq, double e0, double (&Rv)[3],
                                         double (&Jm)[3][3], double (&Rs)[3], double (&Rp)[3]) {
  const double s = s_tr - 3.0 * mu * dq;
  const double p = p_tr + K * dv;
  double s0, H;
  flow_stress(P, e0, s0, H);
  const double is0 = 1.0 / s0;
  const double a = 1.5 * P.q2 * p * is0;
  const double ch = cosh(a), sh = sinh(a);
  const double so = s * is0;
  const double k3 = 3.0 * P.q1 * P.q2 * fs;
  Rv[0] = so * so + 2.0 * fs * P.q1 * ch - 1.0 - P.q3 * fs * fs;
  Rv[1] = 2.0 * so * dv + k3 * sh * dq;
  Rv[2] = (1.0 - f) * (e0 - e0n) + (p * dv - s * dq) * is0;
  Jm[0][0] = k3 * K * sh * is0;
  Jm[0][1] = -6.0 * mu * so * is0;
  Jm[0][2] = -H * is0 * (2.0 * so * so + 2.0 * fs * P.q1 * a * sh);
  Jm[1][0] = 2.0 * so + k3 * dq * ch * 1.5 * P.q2 * K * is0;
  Jm[1][1] = -6.0 * mu * dv * is0 + k3 * sh;
  Jm[1][2] = -2.0 * so * dv * H * is0 - k3 * dq * ch * a * H * is0;
  Jm[2][0] = (K * dv + p) * is0;
  Jm[2][1] = (3.0 * mu * dq - s) * is0;
  Jm[2][2] = (1.0 - f) - (p * dv - s * dq) * H * is0 * is0;
  Rs[0] = 2.0 * so * is0;
  Rs[1] = 2.0 * dv * is0;
  Rs[2] = -dq * is0;
  Rp[0] = k3 * sh * is0;
  Rp[1] = k3 * dq * ch * 1.5 * P.q2 * is0;
  Rp[2] = dv * is0;
}

// x = J^-1 b for a 3x3 system (Cramer's rule); false if singular
__device__ __forceinline__ bool solve3(const double (&Jm)[3][3], const double (&b)[3], double (&x)[3]) {
  const double c00 = Jm[1][1] * Jm[2][2] - Jm[1][2] * Jm[2][1];
  const double c01 = Jm[1][2] * Jm[2][0] - Jm[1][0] * Jm[2][2];
  const double c02 = Jm[1][0] * Jm[2][1] - Jm[1][1] * Jm[2][0];
  const double det = Jm[0][0] * c00 + Jm[0][1] * c01 + Jm[0][2] * c02;
  if (!(fabs(det) > 0.0)) return false;
  const double id = 1.0 / det;
  const double c10 = Jm[0][2] * Jm[2][1] - Jm[0][1] * Jm[2][2];
  const double c11 = Jm[0][0] * Jm[2][2] - Jm[0][2] * Jm[2][0];
  const double c12 = Jm[0][1] * Jm[2][0] - Jm[0][0] * Jm[2][1];
  const double c20 = Jm[0][1] * Jm[1][2] - Jm[0][2] * Jm[1][1];
  const double c21 = Jm[0][2] * Jm[1][0] - Jm[0][0] * Jm[1][2];
  const double c22 = Jm[0][0] * Jm[1][1] - Jm[0][1] * Jm[1][0];
  x[0] = (c00 * b[0] + c10 * b[1] + c20 * b[2]) * id;
  x[1] = (c01 * b[0] + c11 * b[1] + c21 * b[2]) * id;
  x[2] = (c02 * b[0] + c12 * b[1] + c22 * b[2]) * id;
  return true;
}

static __device__ __noinline__ void gtn_point(const PhaseDev& P, double K, double mu, const double (&ee)[6], double e0n,
                                       double fn, double a0, double a0n, double at, double atn, GtnPoint& o) {
  // porosity from the frozen non-local eps_0^p (a0) and tr eps^p (at)
  const double dat = at - atn;
  const double z = (a0 - P.eps_N) / P.s_N;
  const double AN = P.f_N / (P.s_N * 2.50662827463100050242) * exp(-0.5 * z * z);
  const double f = (fn + AN * (a0 - a0n) + dat) / (1.0 + dat);
  double fs = f < P.f_C ? f : (f < P.f_F ? P.f_C + (P.fV - P.f_C) / (P.f_F - P.f_C) * (f - P.f_C) : P.fV);
  fs = fmin(fmax(fs, 0.0), P.fstar_max);
  o.f = f;
  o.fs = fs;
  o.ok = 1;
  const double tr = ee[0] + ee[1] + ee[2];
  double dev[6], dd = 0.0;
  for (int c = 0; c < 6; c++) {
    dev[c] = ee[c] - (c < 3 ? tr * (1.0 / 3.0) : 0.0);
    dd += dev[c] * dev[c];
  }
  const double p_tr = -K * tr;
  const double s_tr = 2.0 * mu * sqrt(1.5 * dd);
  const double in = s_tr > 0.0 ? 3.0 * mu / s_tr : 0.0;   // n = 1.5 (2 mu dev) / s_tr
  double n[6];
  for (int c = 0; c < 6; c++) n[c] = in * dev[c];
  double s0n, hn;
  flow_stress(P, e0n, s0n, hn);
  const double atr = 1.5 * P.q2 * p_tr / s0n;
  const double phi_tr = (s_tr / s0n) * (s_tr / s0n) + 2.0 * fs * P.q1 * cosh(atr) - 1.0 - P.q3 * fs * fs;
  if (!(phi_tr > 0.0)) {
    for (int c = 0; c < 6; c++) {
      o.sig[c] = (c < 3 ? K * tr : 0.0) + 2.0 * mu * dev[c];
      o.dep[c] = 0.0;
      o.nh[c] = 0.0;
    }
    o.e0 = e0n;
    o.A = K;
    o.B = 2.0 * mu;
    o.C = 0.0;
    o.D = 0.0;
    return;
  }
  double x[3] = {0.0, 0.0, e0n}, Rv[3], Jm[3][3], Rs[3], Rp[3];
  gtn_eval(P, K, mu, f, fs, s_tr, p_tr, e0n, x[0], x[1], x[2], Rv, Jm, Rs, Rp);
  double r0 = sqrt(Rv[0] * Rv[0] + Rv[1] * Rv[1] + Rv[2] * Rv[2]);
  bool conv = false;
  for (int it = 0; it < 60 && !conv; it++) {
    double st[3];
    if (!solve3(Jm, Rv, st)) break;
    double lam = 1.0, xn[3], rn = 0.0;
    for (int bt = 0; bt < 40; bt++) {
      for (int k = 0; k < 3; k++) xn[k] = x[k] - lam * st[k];
      gtn_eval(P, K, mu, f, fs, s_tr, p_tr, e0n, xn[0], xn[1], xn[2], Rv, Jm, Rs, Rp);
      rn = sqrt(Rv[0] * Rv[0] + Rv[1] * Rv[1] + Rv[2] * Rv[2]);
      if (rn <= r0 * (1.0 - 1e-4 * lam) || !(r0 > 1e-15)) break;
      lam *= 0.5;
    }
    conv = true;
    for (int k = 0; k < 3; k++) {
      conv = conv && fabs(lam * st[k]) <= 1e-12 * fmax(fabs(xn[k]), 1e-4);
      x[k] = xn[k];
    }
    r0 = rn;
  }
  // x and the Jacobian at x (the last evaluation) give the update and tangent
  o.ok = conv && fabs(Rv[0]) <= 1e-10 && fabs(Rv[1]) <= 1e-10 && fabs(Rv[2]) <= 1e-10;
  const double dv = x[0], dq = x[1];
  const double s = s_tr - 3.0 * mu * dq, p = p_tr + K * dv;
  for (int c = 0; c < 6; c++) {
    o.sig[c] = (c < 3 ? -p : 0.0) + (2.0 / 3.0) * s * n[c];
    o.dep[c] = (c < 3 ? dv * (1.0 / 3.0) : 0.0) + dq * n[c];
  }
  o.e0 = x[2];
  double dxs[3], dxp[3];
  const double ms[3] = {-Rs[0], -Rs[1], -Rs[2]}, mp[3] = {-Rp[0], -Rp[1], -Rp[2]};
  if (!solve3(Jm, ms, dxs) || !solve3(Jm, mp, dxp)) o.ok = 0;
  const double sr = s_tr > 0.0 ? s / s_tr : 1.0;
  const double r23 = 0.81649658092772603273;   // sqrt(2/3): nh = sqrt(2/3) n
  o.A = K * (1.0 + K * dxp[0]);
  o.B = 2.0 * mu * sr;
  o.C = 2.0 * mu * (1.0 - 3.0 * mu * dxs[1]) - 2.0 * mu * sr;
  o.D = 1.22474487139158904909 * mu * K * (dxp[1] - dxs[0]);   // sqrt(3/2) mu K (b_p - a_s)
  for (int c = 0; c < 6; c++) o.nh[c] = r23 * n[c];
}

template <typename R, bool GTN>
__global__ void __launch_bounds__(kThreads)
k_return_map(Geo g, const PhaseTable* __restrict__ pt, int J, const uint8_t* __restrict__ phase,
             const double* __restrict__ eps, const double* __restrict__ epsp_n,
             const double* __restrict__ ep_n, const double* __restrict__ abar,
             double* __restrict__ sigma, double* __restrict__ epsp, double* __restrict__ ep,
             double* __restrict__ Dout, double* __restrict__ alpha, R* __restrict__ desc,
             double* __restrict__ part, int pstride, const double* __restrict__ stiff,
             const double* __restrict__ abar_n, const double* __restrict__ f_n, double* __restrict__ f_out) {
  const long long V = g.V;
  const int nc = g.nc;
  double acc[7] = {0, 0, 0, 0, 0, 0, 0};
  double dmx[1] = {0.0};
  const double s23 = 0.81649658092772603273;   // sqrt(2/3)
  for (long long v = blockIdx.x * (long long)kThreads + threadIdx.x; v < V; v += (long long)gridDim.x * kThreads) {
    const PhaseDev P = pt->p[phase[v]];
    double e[6] = {0, 0, 0, 0, 0, 0};
    for (int c = 0; c < nc; c++) e[g.cmap[c]] = eps[c * V + v];
    double pn[6];
    for (int c = 0; c < 6; c++) { pn[c] = epsp_n[c * V + v]; e[c] -= pn[c]; }
    const double tr = e[0] + e[1] + e[2];
    const double tr3 = tr * (1.0 / 3.0);
    double dev[6];
    for (int c = 0; c < 6; c++) dev[c] = e[c] - (c < 3 ? tr3 : 0.0);
    // per-voxel modulus factor (1 without a stiffness field)
    const double sc = stiff ? stiff[v] : 1.0;
    const double K = P.K * sc, mu = P.mu * sc;
    const double epn = ep_n[v];
    if constexpr (GTN) {
      if (P.law == 3) {
        GtnPoint o;
        const int j0 = P.var, j1 = P.var + 1;
        gtn_point(P, K, mu, e, epn, f_n[v], abar[j0 * V + v], abar_n[j0 * V + v], abar[j1 * V + v],
                  abar_n[j1 * V + v], o);
        // a local update that did not converge poisons the stress, so the
        // Newton residual turns non-finite and the increment is rejected
        const double bad = o.ok ? 0.0 : __longlong_as_double(0x7ff8000000000000LL);
        for (int c = 0; c < 6; c++) {
          const double sgc = o.sig[c] + bad;
          sigma[c * V + v] = sgc;
          epsp[c * V + v] = pn[c] + o.dep[c];
          acc[c] += sgc;
        }
        ep[v] = o.e0;
        Dout[v] = o.fs;
        f_out[v] = o.f;
        // the regularised variables: eps_0^p and the trace of the total
        // plastic strain (Eq. helmholta_gurson)
        const double trp = (pn[0] + o.dep[0]) + (pn[1] + o.dep[1]) + (pn[2] + o.dep[2]);
        for (int j = 0; j < J; j++) alpha[j * V + v] = j == j0 ? o.e0 : (j == j1 ? trp : 0.0);
        acc[6] += o.fs;
        dmx[0] = fmax(dmx[0], o.fs);
        desc[v] = (R)o.A;
        desc[V + v] = (R)o.B;
        desc[2 * V + v] = (R)o.C;
        desc[3 * V + v] = (R)o.D;
        for (int c = 0; c < nc; c++) desc[(4 + c) * V + v] = (R)o.nh[g.cmap[c]];
        continue;
      }
      f_out[v] = f_n[v];
    }
    double q = 0.0;
    for (int c = 0; c < 6; c++) q += dev[c] * dev[c];
    q = 2.0 * mu * sqrt(q);
    double dl = 0.0, theta = 1.0, thetab = 0.0, D = 0.0;
    double nh[6] = {0, 0, 0, 0, 0, 0};
    if (P.law == 1) {
      double s0n, hn;
      flow_stress(P, epn, s0n, hn);
      const double f = q - s23 * s0n;
      if (f > 0.0) {
        double ih;
        if (P.hard == 0) {
          // two FP64 divisions per plastic voxel (division is slow on the
          // FP64 pipe): 2 mu + 2H/3 = (2/3)(3 mu + H), so 1/(3 mu + H) serves
          // the multiplier and thetabar, 1/q the flow direction and theta
          ih = 1.0 / (3.0 * mu + P.H);
          dl = 1.5 * f * ih;
        } else {
          // q - 2 mu dl - sqrt(2/3) sigma_0(ep_n + sqrt(2/3) dl) = 0 is convex
          // and decreasing in dl and positive at 0: Newton from 0 rises
          // monotonically onto the root
          double x = 0.0, s0 = s0n, hp = hn;
          for (int it = 0; it < 60; it++) {
            const double r = q - 2.0 * mu * x - s23 * s0;
            const double dx = 1.5 * r / (3.0 * mu + hp);
            x += dx;
            flow_stress(P, epn + s23 * x, s0, hp);
            if (!(dx > 1e-16 * x)) break;
          }
          dl = x;
          ih = 1.0 / (3.0 * mu + hp);   // thetabar with the slope at the end point
        }
        const double iq = 1.0 / q;
        for (int c = 0; c < 6; c++) nh[c] = 2.0 * mu * dev[c] * iq;
        theta = 1.0 - 2.0 * mu * dl * iq;
        thetab = 3.0 * mu * ih - (1.0 - theta);
      }
      if (P.var >= 0) {
        const double ab = abar[P.var * V + v];
        D = (ab - P.eps_C) * P.inv_dCR;
        D = D < 0.0 ? 0.0 : (D > P.D_max ? P.D_max : D);
      }
    }
    // particle cracking: history kappa = max(kappa_n, ||<eps>_+||) in the ep
    // slot, damage from the non-local kappa on an elastic stress
    double kap = 0.0;
    if (P.law == 2) {
      kap = fmax(epn, positive_principal_norm(e));
      if (P.var >= 0) {
        const double ab = abar[P.var * V + v];
        D = (ab - P.eps_C) * P.inv_dCR;
        D = D < 0.0 ? 0.0 : (D > P.D_max ? P.D_max : D);
      }
    }
    const double om = 1.0 - D;
    double sg[6];
    for (int c = 0; c < 6; c++) {
      const double seff = (c < 3 ? K * tr : 0.0) + 2.0 * mu * dev[c] - 2.0 * mu * dl * nh[c];
      sg[c] = om * seff;
      sigma[c * V + v] = sg[c];
      epsp[c * V + v] = pn[c] + dl * nh[c];
      acc[c] += sg[c];
    }
    const double epv = P.law == 2 ? kap : epn + s23 * dl;
    ep[v] = epv;
    Dout[v] = D;
    for (int j = 0; j < J; j++) alpha[j * V + v] = (P.var == j) ? epv : 0.0;
    acc[6] += D;
    dmx[0] = fmax(dmx[0], D);
    desc[v] = (R)(om * K);
    desc[V + v] = (R)(om * 2.0 * mu * theta);
    if constexpr (GTN) {
      // extended layout A, B, C, D, nh (the GTN handles' tangent form)
      desc[2 * V + v] = (R)(-om * 2.0 * mu * thetab);
      desc[3 * V + v] = R(0);
      for (int c = 0; c < nc; c++) desc[(4 + c) * V + v] = (R)nh[g.cmap[c]];
    } else {
      // the descriptor is stored in the working precision: its square root
      // in that precision too
      const R ms = sqrt((R)(om * 2.0 * mu * thetab));
      for (int c = 0; c < nc; c++) desc[(2 + c) * V + v] = ms * (R)nh[g.cmap[c]];
    }
  }
  block_sum_store<7>(acc, part, pstride);
  __syncthreads();
  block_max_store<1>(dmx, part + 7 * (long long)pstride, pstride);
}

template <typename R>
__global__ void __launch_bounds__(kThreads)
k_tangent64(Geo g, const R* __restrict__ desc, const double* __restrict__ p, double* __restrict__ tau, int ext) {
  const long long V = g.V;
  const int nc = g.nc, nn = g.d == 3 ? 3 : 2;
  for (long long v = blockIdx.x * (long long)kThreads + threadIdx.x; v < V; v += (long long)gridDim.x * kThreads) {
    double pv[6], tr = 0.0, mp = 0.0;
    for (int c = 0; c < nc; c++) pv[c] = p[c * V + v];
    for (int c = 0; c < nn; c++) tr += pv[c];
    const int m0 = ext ? 4 : 2;
    for (int c = 0; c < nc; c++) mp += (double)desc[(m0 + c) * V + v] * pv[c];
    const double c1 = desc[v], c2 = desc[V + v];
    if (ext) {
      // A tr(p) I + B dev(p) + C (nh.p) nh + D ((nh.p) I + tr(p) nh)
      const double cc = desc[2 * V + v], dd = desc[3 * V + v];
      for (int c = 0; c < nc; c++) {
        const double n = desc[(4 + c) * V + v];
        double o = c2 * pv[c] + (cc * mp + dd * tr) * n;
        if (c < nn) o += (c1 - c2 / 3.0) * tr + dd * mp;
        tau[c * V + v] = o;
      }
      continue;
    }
    for (int c = 0; c < nc; c++) {
      double o = c2 * pv[c] - (double)desc[(2 + c) * V + v] * mp;
      if (c < nn) o += c1 * tr - c2 * tr / 3.0;
      tau[c * V + v] = o;
    }
  }
}

template <typename R>
__global__ void __launch_bounds__(kThreads)
k_eps_update(Geo g, double* __restrict__ eps, const R* __restrict__ x, double* __restrict__ part,
             int pstride) {
  const long long V = g.V;
  const int nc = g.nc;
  double acc[6] = {0, 0, 0, 0, 0, 0};
  R mxr = R(0);   // max |x| in the correction's own precision
  for (long long v = blockIdx.x * (long long)kThreads + threadIdx.x; v < V; v += (long long)gridDim.x * kThreads) {
    for (int c = 0; c < nc; c++) {
      const R xr = x[c * V + v];
      const double en = eps[c * V + v] + (double)xr;
      eps[c * V + v] = en;
      acc[c] += en;
      mxr = fmax(mxr, fabs(xr));
    }
  }
  double mx[1] = {(double)mxr};
  block_sum_store<6>(acc, part, pstride);
  __syncthreads();
  block_max_store<1>(mx, part + 6 * (long long)pstride, pstride);
}

template <typename R>
__global__ void k_to_r(long long n, const double* __restrict__ a, R* __restrict__ b) {
  for (long long i = blockIdx.x * (long long)kThreads + threadIdx.x; i < n; i += (long long)gridDim.x * kThreads) b[i] = (R)a[i];
}
template <typename R>
__global__ void k_from_r(long long n, const R* __restrict__ a, double* __restrict__ b) {
  for (long long i = blockIdx.x * (long long)kThreads + threadIdx.x; i < n; i += (long long)gridDim.x * kThreads) b[i] = (double)a[i];
}

// ============================================================ launchers
template <typename R>
static size_t xsmem(const Geo& g, int nrows, int nc) {
  return (size_t)g.n1 * sizeof(C2<R>) + xbuf_c(nrows, nc, g.M) * sizeof(C2<R>);
}
static inline int xgrid(const Geo& g, int nrows) { return (int)((g.nlines + nrows - 1) / nrows); }

// shared memory of an x1 kernel: STAGE 0 plain, 1 staged spectrum rows,
// 1 + k staged rows plus k prefetched real fields
template <typename R>
static size_t xinv_stage_smem(const Geo& g, int nr, int nc, int stage) {
  if (!stage) return xsmem<R>(g, nr, nc);
  return xstage_off<R>(g.n1, nr, nc) + (size_t)nr * nc * g.ps * sizeof(C2<R>) +
         (size_t)(stage - 1) * nr * nc * g.n1 * sizeof(R);
}

// launch an x1 kernel K<E> with E = 4 or 16 as chosen in the launch config
// x1 launch: compile-time variant KCT for rows of 128 complex points (N1 =
// 256) at one row per CTA, else KT4 / KT16 by the staged-element count
#define XLAUNCH(KCT, KT4, KT16, NCC, STAGE, ...)                                                        \
  do {                                                                                                  \
    const int nr = lc.nrows_c[NCC];                                                                     \
    const size_t sm = xinv_stage_smem<R>(g, nr, NCC, STAGE);                                           \
    if (lc.xe_c[NCC] == 4 && g.M == 128 && nr == XRows<128, NCC>::v) {                                  \
      auto k = KCT(128);                                                                                \
      set_smem(k, sm);                                                                                  \
      k<<<xgrid(g, nr), kThreads, sm, st>>>(__VA_ARGS__);                                               \
    } else if (lc.xe_c[NCC] == 4 && g.M == 64 && nr == XRows<64, NCC>::v) {                             \
      auto k = KCT(64);                                                                                 \
      set_smem(k, sm);                                                                                  \
      k<<<xgrid(g, nr), kThreads, sm, st>>>(__VA_ARGS__);                                               \
    } else if (lc.xe_c[NCC] == 4 && g.M == 48 && nr == XRows<48, NCC>::v) {                             \
      auto k = KCT(48);                                                                                 \
      set_smem(k, sm);                                                                                  \
      k<<<xgrid(g, nr), kThreads, sm, st>>>(__VA_ARGS__);                                               \
    } else if (lc.xe_c[NCC] == 4 && g.M == 32 && nr == XRows<32, NCC>::v) {                             \
      auto k = KCT(32);                                                                                 \
      set_smem(k, sm);                                                                                  \
      k<<<xgrid(g, nr), kThreads, sm, st>>>(__VA_ARGS__);                                               \
    } else if (lc.xe_c[NCC] == 4) {                                                                     \
      auto k = KT4;                                                                                     \
      set_smem(k, sm);                                                                                  \
      k<<<xgrid(g, nr), kThreads, sm, st>>>(__VA_ARGS__);                                               \
    } else {                                                                                            \
      auto k = KT16;                                                                                    \
      set_smem(k, sm);                                                                                  \
      k<<<xgrid(g, nr), kThreads, sm, st>>>(__VA_ARGS__);                                               \
    }                                                                                                   \
  } while (0)

// tile width of the strided / last-axis kernels with ncomp components per
// tile: the register-pass width on a 64/128/256-point axis, else the runtime
// width
template <typename R>
static int axis_tx(const LaunchCfg& lc, int N, int ncomp) {
  if (!reg_axis(N)) return lc.tx;
  switch (ncomp) {
    case 1: return RegTx<R, 1>::v;
    case 2: return RegTx<R, 2>::v;
    case 3: return RegTx<R, 3>::v;
    default: return RegTx<R, 6>::v;
  }
}

template <typename R, int NC, bool EXT>
static void xfwd_tangent_nc(const Geo& g, const Tables<R>& t, const LaunchCfg& lc, cudaStream_t st, R* p,
                            const R* r, const R* desc, C2<R>* S, const KrylovCtl* ctl, double* part) {
  ProTangent<R, NC, EXT> pro;
  pro.p = p; pro.r = r; pro.desc = desc; pro.V = g.V;
  pro.update = ctl != nullptr; pro.beta = R(0); pro.first = true;
  pro.part = part; pro.pstride = lc.max_blocks;
#define KCT_(M) (k_xfwd<R, NC, 4, ProTangent<R, NC, EXT>, M>)
  XLAUNCH(KCT_, (k_xfwd<R, NC, 4, ProTangent<R, NC, EXT>>),
          (k_xfwd<R, NC, 16, ProTangent<R, NC, EXT>>), NC, false,
          g, t.plan_x, t.tw[0], S, nr, pro, ctl);
#undef KCT_
}

template <typename R>
void Ops<R>::xfwd_tangent(const Geo& g, const Tables<R>& t, const LaunchCfg& lc, cudaStream_t st, R* p,
                          const R* r, const R* desc, C2<R>* S, const KrylovCtl* ctl, double* part, int ext) {
  if (ext) {
    if (g.nc == 6) xfwd_tangent_nc<R, 6, true>(g, t, lc, st, p, r, desc, S, ctl, part);
    else xfwd_tangent_nc<R, 3, true>(g, t, lc, st, p, r, desc, S, ctl, part);
  } else {
    if (g.nc == 6) xfwd_tangent_nc<R, 6, false>(g, t, lc, st, p, r, desc, S, ctl, part);
    else xfwd_tangent_nc<R, 3, false>(g, t, lc, st, p, r, desc, S, ctl, part);
  }
}

template <typename R, int NC>
static void xfwd_field64_nc(const Geo& g, const Tables<R>& t, const LaunchCfg& lc, cudaStream_t st,
                            const double* f, const int* fmap, const double* mean_dev, C2<R>* S,
                            const double* f2, const double* mean2) {
  ProField64<R, NC> pro;
  pro.f = f; pro.mean = mean_dev; pro.f2 = f2; pro.mean2 = mean2; pro.V = g.V;
  for (int c = 0; c < NC; c++) pro.map[c] = fmap[c];
#define KCT_(M) (k_xfwd<R, NC, 4, ProField64<R, NC>, M>)
  XLAUNCH(KCT_, (k_xfwd<R, NC, 4, ProField64<R, NC>>),
          (k_xfwd<R, NC, 16, ProField64<R, NC>>), NC, false,
          g, t.plan_x, t.tw[0], S, nr, pro, nullptr);
#undef KCT_
}

template <typename R>
void Ops<R>::xfwd_field64(const Geo& g, const Tables<R>& t, const LaunchCfg& lc, cudaStream_t st,
                          const double* f, int ncomp, const int* fmap, const double* mean_dev, C2<R>* S,
                          const double* f2, const double* mean2) {
  // component counts other than 6, 3 and 1 are transformed one by one
  if (ncomp == 6) xfwd_field64_nc<R, 6>(g, t, lc, st, f, fmap, mean_dev, S, f2, mean2);
  else if (ncomp == 3) xfwd_field64_nc<R, 3>(g, t, lc, st, f, fmap, mean_dev, S, f2, mean2);
  else
    for (int c = 0; c < ncomp; c++)
      xfwd_field64_nc<R, 1>(g, t, lc, st, f, fmap + c, mean_dev, S + (size_t)c * g.sstride, f2, mean2);
}

template <typename R, int NC>
static void xinv_matvec_nc(const Geo& g, const Tables<R>& t, const LaunchCfg& lc, cudaStream_t st,
                           const C2<R>* S, R* Ap, const R* p, double* part, const KrylovCtl* ctl) {
  EpiMatvec<R, NC> epi;
  epi.Ap = Ap; epi.p = p; epi.V = g.V;
#define KCT_(M) (k_xinv<R, NC, 4, EpiMatvec<R, NC>, 1, M>)
  XLAUNCH(KCT_, (k_xinv<R, NC, 4, EpiMatvec<R, NC>, 1>),
          (k_xinv<R, NC, 16, EpiMatvec<R, NC>, 1>), NC, 2,
          g, t.plan_x, t.tw[0], S, nr, R(2.0 / (double)g.V), epi, part, lc.max_blocks, ctl);
#undef KCT_
}

template <typename R>
void Ops<R>::xinv_matvec(const Geo& g, const Tables<R>& t, const LaunchCfg& lc, cudaStream_t st,
                         const C2<R>* S, R* Ap, const R* p, double* part, const KrylovCtl* ctl) {
  if (g.nc == 6) xinv_matvec_nc<R, 6>(g, t, lc, st, S, Ap, p, part, ctl);
  else xinv_matvec_nc<R, 3>(g, t, lc, st, S, Ap, p, part, ctl);
}

template <typename R, int NC>
static void xinv_cg_nc(const Geo& g, const Tables<R>& t, const LaunchCfg& lc, cudaStream_t st,
                       const C2<R>* S, R* x, R* r, const R* p, double* part, const KrylovCtl* ctl) {
  EpiCG<R, NC> epi;
  epi.x = x; epi.r = r; epi.p = p; epi.V = g.V; epi.alpha = R(0);
#define KCT_(M) (k_xinv<R, NC, 4, EpiCG<R, NC>, 1, M>)
  XLAUNCH(KCT_, (k_xinv<R, NC, 4, EpiCG<R, NC>, 1>),
          (k_xinv<R, NC, 16, EpiCG<R, NC>, 1>), NC, 4,
          g, t.plan_x, t.tw[0], S, nr, R(2.0 / (double)g.V), epi, part, lc.max_blocks, ctl);
#undef KCT_
}

template <typename R>
void Ops<R>::xinv_cg(const Geo& g, const Tables<R>& t, const LaunchCfg& lc, cudaStream_t st,
                     const C2<R>* S, R* x, R* r, const R* p, double* part, const KrylovCtl* ctl) {
  if (g.nc == 6) xinv_cg_nc<R, 6>(g, t, lc, st, S, x, r, p, part, ctl);
  else xinv_cg_nc<R, 3>(g, t, lc, st, S, x, r, p, part, ctl);
}

template <typename R>
size_t Ops<R>::xinv_cg_smem(const Geo& g, const LaunchCfg& lc) {
  return xinv_stage_smem<R>(g, lc.nrows_c[g.nc], g.nc, 4);
}

template <typename R, typename RO, int NC>
static void xinv_residual_nc(const Geo& g, const Tables<R>& t, const LaunchCfg& lc, cudaStream_t st,
                             const C2<R>* S, RO* b, const double* mean_sig_dev, const double* mask,
                             const double* sbar, double* part, const RO* bref, const double* mean_ref) {
  EpiResidual<R, RO, NC> epi;
  epi.b = b; epi.mean_sig = mean_sig_dev; epi.mean_ref = mean_ref; epi.bref = bref; epi.V = g.V;
  for (int c = 0; c < NC; c++) {
    epi.mask[c] = mask[c];
    epi.sbar[c] = sbar[c];
    epi.map[c] = g.cmap[c];
    epi.dc[c] = 0.0;
  }
#define KCT_(M) (k_xinv<R, NC, 4, EpiResidual<R, RO, NC>, 1, M>)
  XLAUNCH(KCT_, (k_xinv<R, NC, 4, EpiResidual<R, RO, NC>, 1>),
          (k_xinv<R, NC, 16, EpiResidual<R, RO, NC>, 1>), NC, true, g, t.plan_x, t.tw[0], S, nr, R(2.0 / (double)g.V), epi, part, lc.max_blocks, nullptr);
#undef KCT_
}

template <typename R>
template <typename RO>
void Ops<R>::xinv_residual(const Geo& g, const Tables<R>& t, const LaunchCfg& lc, cudaStream_t st,
                           const C2<R>* S, RO* b, const double* mean_sig_dev, const double* mask,
                           const double* sbar, double* part, const RO* bref, const double* mean_ref) {
  if (g.nc == 6) xinv_residual_nc<R, RO, 6>(g, t, lc, st, S, b, mean_sig_dev, mask, sbar, part, bref, mean_ref);
  else xinv_residual_nc<R, RO, 3>(g, t, lc, st, S, b, mean_sig_dev, mask, sbar, part, bref, mean_ref);
}

template <typename R, int NC>
static void xinv_store64_nc(const Geo& g, const Tables<R>& t, const LaunchCfg& lc, cudaStream_t st,
                            const C2<R>* S, double* out) {
  EpiStore64<R, NC> epi;
  epi.out = out; epi.V = g.V;
#define KCT_(M) (k_xinv<R, NC, 4, EpiStore64<R, NC>, 0, M>)
  XLAUNCH(KCT_, (k_xinv<R, NC, 4, EpiStore64<R, NC>, 0>),
          (k_xinv<R, NC, 16, EpiStore64<R, NC>, 0>), NC, true,
          g, t.plan_x, t.tw[0], S, nr, R(2.0 / (double)g.V), epi, nullptr, 0, nullptr);
#undef KCT_
}

template <typename R>
void Ops<R>::xinv_store64(const Geo& g, const Tables<R>& t, const LaunchCfg& lc, cudaStream_t st,
                          const C2<R>* S, int ncomp, double* out) {
  // component counts other than 6, 3 and 1 are stored one by one
  if (ncomp == 6) xinv_store64_nc<R, 6>(g, t, lc, st, S, out);
  else if (ncomp == 3) xinv_store64_nc<R, 3>(g, t, lc, st, S, out);
  else
    for (int c = 0; c < ncomp; c++) xinv_store64_nc<R, 1>(g, t, lc, st, S + (size_t)c * g.sstride, out + (size_t)c * g.V);
}

template <typename R>
void Ops<R>::xinv_storeR(const Geo& g, const Tables<R>& t, const LaunchCfg& lc, cudaStream_t st, const C2<R>* S,
                         R* out, const KrylovCtl* ctl) {
  EpiStoreR<R> epi;
  epi.out = out;
#define KCT_(M) (k_xinv<R, 1, 4, EpiStoreR<R>, 0, M>)
  XLAUNCH(KCT_, (k_xinv<R, 1, 4, EpiStoreR<R>, 0>), (k_xinv<R, 1, 16, EpiStoreR<R>, 0>), 1, true,
          g, t.plan_x, t.tw[0], S, nr, R(2.0 / (double)g.V), epi, nullptr, 0, ctl);
#undef KCT_
}

template <typename R>
void Ops<R>::xfwd_fieldR(const Geo& g, const Tables<R>& t, const LaunchCfg& lc, cudaStream_t st, const R* f,
                         C2<R>* S, const KrylovCtl* ctl) {
  ProFieldR<R> pro;
  pro.f = f;
#define KCT_(M) (k_xfwd<R, 1, 4, ProFieldR<R>, M>)
  XLAUNCH(KCT_, (k_xfwd<R, 1, 4, ProFieldR<R>>), (k_xfwd<R, 1, 16, ProFieldR<R>>), 1, false,
          g, t.plan_x, t.tw[0], S, nr, pro, ctl);
#undef KCT_
}

template <typename R>
void Ops<R>::helm_stencil(const Geo& g, const LaunchCfg& lc, cudaStream_t st, const R* q, R* y,
                          const uint8_t* phase, const R* ell2_tab, const KrylovCtl* ctl) {
  // corner derivative: mean of 2^(d-1) forward differences over h_j; the
  // kernel sums four edge differences per corner (twice the same two in 2D,
  // where the x3 neighbour is the plane itself), so 1 / (4 h_j) per D_j and
  // the same for D_j^T
  const R c0 = (R)(1.0 / (16.0 * g.h[0] * g.h[0]));
  const R c1 = (R)(1.0 / (16.0 * g.h[1] * g.h[1]));
  const R c2 = g.d == 3 ? (R)(1.0 / (16.0 * g.h[2] * g.h[2])) : R(0);
  constexpr int rows = kStencilWarps * StencilRows<R>::SYT;
  const int bx = (g.n1 + kStencilOut - 1) / kStencilOut, by = (g.n2 + rows - 1) / rows;
  // planes per CTA: each CTA also reads the two halo planes, and the last
  // wave of CTAs may leave SMs idle, so zc minimises (waves) x (zc + 2)
  // over the resident CTAs of the whole GPU
  static int slots = 0;
  if (slots == 0) {
    int dev = 0, nsm = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_helm_stencil<R>, 32 * kStencilWarps, 0) !=
            cudaSuccess || per < 1) {
      cudaGetLastError();
      nsm = 1;
      per = 1;
    }
    slots = nsm * per;
  }
  int zc = g.n3 < 16 ? g.n3 : 16;
  if (g.n3 > 16) {
    long long best = -1;
    for (int z = 8; z <= 32 && z <= g.n3; z++) {
      const long long ctas = (long long)bx * by * ((g.n3 + z - 1) / z);
      const long long cost = ((ctas + slots - 1) / slots) * (z + 2);
      if (best < 0 || cost < best) {
        best = cost;
        zc = z;
      }
    }
  }
  dim3 grid(bx, by, (g.n3 + zc - 1) / zc);
  k_helm_stencil<R><<<grid, 32 * kStencilWarps, 0, st>>>(g, q, y, phase, ell2_tab, c0, c1, c2, zc, ctl);
}

template <typename R>
void Ops<R>::strided_plain(const Geo& g, const Tables<R>& t, const LaunchCfg& lc, cudaStream_t st,
                           C2<R>* S, int ncomp, int axis, int sign, const KrylovCtl* ctl) {
  const StrideInfo<R> si = stride_of<R>(g, axis);
  const FftPlan& pl = axis == 1 ? t.plan_y : t.plan_z;
  const int tx = axis_tx<R>(lc, si.N, 1);
  const size_t sm = tw_bytes<R>(si.N) + (size_t)si.N * sizeof(C2<R>) * tx;
  dim3 grid((g.P1 + tx - 1) / tx, axis == 1 ? g.n3 : g.n2, ncomp);
  constexpr int TXR = RegTx<R, 1>::v;
  auto pick = [&](auto k256, auto k128, auto k64, auto kgen) {
    return si.N == 256 ? k256 : si.N == 128 ? k128 : si.N == 64 ? k64 : kgen;
  };
  if (sign < 0) {
    auto k = pick(k_strided_plain<R, -1, TXR, 256>, k_strided_plain<R, -1, TXR, 128>,
                  k_strided_plain<R, -1, TXR, 64>, k_strided_plain<R, -1>);
    set_smem(k, sm);
    k<<<grid, kThreads, sm, st>>>(g, pl, t.tw[axis], S, tx, si.astride, si.ostride, ctl);
  } else {
    auto k = pick(k_strided_plain<R, 1, TXR, 256>, k_strided_plain<R, 1, TXR, 128>,
                  k_strided_plain<R, 1, TXR, 64>, k_strided_plain<R, 1>);
    set_smem(k, sm);
    k<<<grid, kThreads, sm, st>>>(g, pl, t.tw[axis], S, tx, si.astride, si.ostride, ctl);
  }
}

template <typename R>
void Ops<R>::gamma(const Geo& g, const Tables<R>& t, const LaunchCfg& lc, cudaStream_t st, C2<R>* S,
                   const float* stress_mask, int dc_mode, const KrylovCtl* ctl, int* wait_err, double wait_s,
                   int extra_tx) {
  const unsigned long long wait_ns = (unsigned long long)(wait_s * 1e9);
  const int axis = g.d - 1;
  const StrideInfo<R> si = stride_of<R>(g, axis);
  const FftPlan& pl = axis == 1 ? t.plan_y : t.plan_z;
  const int tx = axis_tx<R>(lc, si.N, g.nc);
  const bool reg = reg_axis(si.N);
  const int rs = !reg ? g.nc * tx : g.nc == 6 ? RegRs<R, 6>::v : RegRs<R, 3>::v;
  const size_t sm = tw_bytes<R>(si.N) + (size_t)si.N * sizeof(C2<R>) * rs;
  dim3 grid((g.P1 + tx - 1) / tx, axis == 1 ? 1 : g.n2, 1);
  Mask6 m;
  for (int c = 0; c < 6; c++) m.m[c] = c < g.nc ? stress_mask[c] : 0.f;
  if (g.d == 3 && g.nc == 6 && reg) {
    // TMA path: the box {TX6 columns, 6 components, 1, N} of the half
    // spectrum seen as 8-byte elements [z][y][c][x]
    constexpr int TX6 = RegTx<R, 6>::v;
    constexpr int TXN = TX6 / 2;                  // the narrow tile (128 threads)
    const bool narrow = lc.gamma_narrow != 0;
    const int txc = narrow ? TXN : TX6;
    constexpr int U8 = (int)sizeof(C2<R>) / 8;
    const unsigned long long cb = sizeof(C2<R>);
    const unsigned long long dims[4] = {(unsigned long long)g.ps * U8, 6ULL, (unsigned long long)g.n2,
                                        (unsigned long long)g.n3};
    const unsigned long long strides[3] = {(unsigned long long)g.sstride * cb, (unsigned long long)g.ps * cb,
                                           (unsigned long long)g.ps * g.n2 * cb};
    const unsigned box[4] = {(unsigned)(txc * U8), 6u, 1u, (unsigned)si.N};
    const CUtensorMap* map = tensor_map_8b(S, 4, dims, strides, box);
    if (map) {
      // column tiles up to P1 (inside the padded row: ps is a multiple of 16)
      const size_t smt = gamma_tma_head<R>(si.N) + (size_t)si.N * 6 * txc * sizeof(C2<R>);
      dim3 gt((g.P1 + txc - 1) / txc, g.n2, 1);
      auto launch = [&](auto k, int nth) {
        set_smem(k, smt);
        k<<<gt, nth, smt, st>>>(g, t, *map, t.tw[axis], m, dc_mode, ctl, wait_err, wait_ns, (unsigned)extra_tx);
      };
      if (!narrow) {
        if (si.N == 256) launch(k_gamma_tma<R, 6, TX6, 256>, kThreads);
        else if (si.N == 128) launch(k_gamma_tma<R, 6, TX6, 128>, kThreads);
        else launch(k_gamma_tma<R, 6, TX6, 64>, kThreads);
      } else {
        constexpr int NT = kThreads / 2;
        if (si.N == 256) launch(k_gamma_tma<R, 6, TXN, 256, NT>, NT);
        else if (si.N == 128) launch(k_gamma_tma<R, 6, TXN, 128, NT>, NT);
        else launch(k_gamma_tma<R, 6, TXN, 64, NT>, NT);
      }
      return;
    }
  }
  auto pick = [&](auto k256, auto k128, auto k64, auto kgen) {
    return si.N == 256 ? k256 : si.N == 128 ? k128 : si.N == 64 ? k64 : kgen;
  };
  if (g.nc == 6) {
    constexpr int TX6 = RegTx<R, 6>::v;
    auto k = pick(k_gamma<R, 6, TX6, 256>, k_gamma<R, 6, TX6, 128>, k_gamma<R, 6, TX6, 64>, k_gamma<R, 6>);
    set_smem(k, sm);
    k<<<grid, kThreads, sm, st>>>(g, t, pl, t.tw[axis], S, tx, si.astride, si.ostride, m, dc_mode, ctl);
  } else {
    constexpr int TX3 = RegTx<R, 3>::v;
    auto k = pick(k_gamma<R, 3, TX3, 256>, k_gamma<R, 3, TX3, 128>, k_gamma<R, 3, TX3, 64>, k_gamma<R, 3>);
    set_smem(k, sm);
    k<<<grid, kThreads, sm, st>>>(g, t, pl, t.tw[axis], S, tx, si.astride, si.ostride, m, dc_mode, ctl);
  }
}

template <typename R>
void Ops<R>::helm_expand(const Geo& g, const Tables<R>& t, const LaunchCfg& lc, cudaStream_t st, C2<R>* W,
                         C2<R>* p, const C2<R>* r, double ell2_mean, const KrylovCtl* ctl, int raw) {
  const int axis = g.d - 1;
  const StrideInfo<R> si = stride_of<R>(g, axis);
  const FftPlan& pl = axis == 1 ? t.plan_y : t.plan_z;
  const int tx = axis_tx<R>(lc, si.N, 1);
  const size_t sm = tw_bytes<R>(si.N) + (size_t)si.N * sizeof(C2<R>) * tx;
  dim3 grid((g.P1 + tx - 1) / tx, axis == 1 ? 1 : g.n2, 1);
  auto pick = [&](auto k256, auto k128, auto k64, auto kgen) {
    return si.N == 256 ? k256 : si.N == 128 ? k128 : si.N == 64 ? k64 : kgen;
  };
  constexpr int T = RegTx<R, 1>::v;
  auto k = pick(k_expand<R, 0, T, 256>, k_expand<R, 0, T, 128>, k_expand<R, 0, T, 64>, k_expand<R, 0>);
  set_smem(k, sm);
  k<<<grid, kThreads, sm, st>>>(g, t, pl, t.tw[axis], W, p, r, tx, si.astride, si.ostride, (R)ell2_mean, ctl, raw);
}

template <typename R>
int Ops<R>::contract_blocks(const Geo& g, const LaunchCfg& lc) {
  const int tx = axis_tx<R>(lc, g.d == 3 ? g.n3 : g.n2, 1);
  return ((g.P1 + tx - 1) / tx) * (g.d == 3 ? g.n2 : 1);
}

template <typename R>
void Ops<R>::helm_contract(const Geo& g, const Tables<R>& t, const LaunchCfg& lc, cudaStream_t st,
                           const C2<R>* W, const C2<R>* p, C2<R>* y, double* part, const KrylovCtl* ctl) {
  const int axis = g.d - 1;
  const StrideInfo<R> si = stride_of<R>(g, axis);
  const FftPlan& pl = axis == 1 ? t.plan_y : t.plan_z;
  const int tx = axis_tx<R>(lc, si.N, 1);
  const size_t sm = tw_bytes<R>(si.N) + (size_t)si.N * sizeof(C2<R>) * tx;
  dim3 grid((g.P1 + tx - 1) / tx, axis == 1 ? 1 : g.n2, 1);
  auto pick = [&](auto k256, auto k128, auto k64, auto kgen) {
    return si.N == 256 ? k256 : si.N == 128 ? k128 : si.N == 64 ? k64 : kgen;
  };
  constexpr int T = RegTx<R, 1>::v;
  auto k = pick(k_contract<R, 0, T, 256>, k_contract<R, 0, T, 128>, k_contract<R, 0, T, 64>, k_contract<R, 0>);
  set_smem(k, sm);
  k<<<grid, kThreads, sm, st>>>(g, t, pl, t.tw[axis], W, p, y, tx, si.astride, si.ostride, part, lc.max_blocks,
                                ctl);
}

template <typename R>
void Ops<R>::cg_init(const Geo& g, const LaunchCfg& lc, cudaStream_t st, R* x, const R* r, double* part) {
  k_cg_init<R><<<lc.n_ew_blocks, kThreads, 0, st>>>((long long)g.nc * g.V, x, r, part, lc.max_blocks);
}

template <typename R>
void Ops<R>::cg_update(const Geo& g, const LaunchCfg& lc, cudaStream_t st, R* x, R* r, const R* p,
                       const R* Ap, double* part, const KrylovCtl* ctl) {
  k_cg_update<R><<<lc.n_ew_blocks, kThreads, 0, st>>>((long long)g.nc * g.V, x, r, p, Ap, part,
                                                      lc.max_blocks, ctl);
}

template <typename R>
void Ops<R>::pcg_init(const Geo& g, const Tables<R>& t, const LaunchCfg& lc, cudaStream_t st, C2<R>* x,
                      const C2<R>* r, double ell2_mean, double* part) {
  k_pcg_init<R><<<lc.n_ew_blocks, kThreads, 0, st>>>(g, t, x, r, (R)ell2_mean, part, lc.max_blocks);
}

template <typename R>
void Ops<R>::pcg_update(const Geo& g, const Tables<R>& t, const LaunchCfg& lc, cudaStream_t st, C2<R>* x,
                        C2<R>* r, const C2<R>* p, const C2<R>* y, double ell2_mean, double* part,
                        const KrylovCtl* ctl) {
  k_pcg_update<R><<<lc.n_ew_blocks, kThreads, 0, st>>>(g, t, x, r, p, y, (R)ell2_mean, part,
                                                       lc.max_blocks, ctl);
}

template <typename R>
void Ops<R>::return_map(const Geo& g, const LaunchCfg& lc, cudaStream_t st, const PhaseTable* pt, int J,
                        const uint8_t* phase, const double* eps, const double* epsp_n, const double* ep_n,
                        const double* abar, double* sigma, double* epsp, double* ep, double* D,
                        double* alpha, R* desc, double* part, const double* stiff, const double* abar_n,
                        const double* f_n, double* f_out, int gtn) {
  if (gtn)
    k_return_map<R, true><<<lc.n_ew_blocks, kThreads, 0, st>>>(g, pt, J, phase, eps, epsp_n, ep_n, abar, sigma,
                                                               epsp, ep, D, alpha, desc, part, lc.max_blocks,
                                                               stiff, abar_n, f_n, f_out);
  else
    k_return_map<R, false><<<lc.n_ew_blocks, kThreads, 0, st>>>(g, pt, J, phase, eps, epsp_n, ep_n, abar, sigma,
                                                                epsp, ep, D, alpha, desc, part, lc.max_blocks,
                                                                stiff, abar_n, f_n, f_out);
}

template <typename R>
void Ops<R>::tangent_apply64(const Geo& g, const LaunchCfg& lc, cudaStream_t st, const R* desc,
                             const double* p, double* tau, int ext) {
  k_tangent64<R><<<lc.n_ew_blocks, kThreads, 0, st>>>(g, desc, p, tau, ext);
}

template <typename R>
void Ops<R>::eps_update(const Geo& g, const LaunchCfg& lc, cudaStream_t st, double* eps, const R* x,
                        double* part) {
  k_eps_update<R><<<lc.n_ew_blocks, kThreads, 0, st>>>(g, eps, x, part, lc.max_blocks);
}

template <typename R>
void Ops<R>::to_r(cudaStream_t st, long long n, const double* a, R* b) {
  k_to_r<R><<<(int)((n + kThreads - 1) / kThreads < 4096 ? (n + kThreads - 1) / kThreads : 4096), kThreads, 0, st>>>(n, a, b);
}
template <typename R>
void Ops<R>::from_r(cudaStream_t st, long long n, const R* a, double* b) {
  k_from_r<R><<<(int)((n + kThreads - 1) / kThreads < 4096 ? (n + kThreads - 1) / kThreads : 4096), kThreads, 0, st>>>(n, a, b);
}

}  // namespace rvk
