// Shared device/host definitions of the GB300 non-local damage RVE library.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace rvk {

constexpr int kThreads = 256;           // threads per CTA of every kernel here
constexpr int kMaxPhases = 8;
constexpr int kMaxVars = 4;             // non-local variables J
constexpr int kMaxRadixStages = 16;

template <typename R> struct C2 { R x, y; };

template <typename R> __host__ __device__ __forceinline__ C2<R> mk(R a, R b) { C2<R> c; c.x = a; c.y = b; return c; }
template <typename R> __device__ __forceinline__ C2<R> operator+(C2<R> a, C2<R> b) { return mk<R>(a.x + b.x, a.y + b.y); }
template <typename R> __device__ __forceinline__ C2<R> operator-(C2<R> a, C2<R> b) { return mk<R>(a.x - b.x, a.y - b.y); }
template <typename R> __device__ __forceinline__ C2<R> cmul(C2<R> a, C2<R> b) {
  return mk<R>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename R> __device__ __forceinline__ C2<R> cscale(C2<R> a, R s) { return mk<R>(a.x * s, a.y * s); }
template <typename R> __device__ __forceinline__ C2<R> conj_(C2<R> a) { return mk<R>(a.x, -a.y); }
// multiply by sign * i
template <typename R, int SIGN> __device__ __forceinline__ C2<R> mul_si(C2<R> a) {
  return SIGN > 0 ? mk<R>(-a.y, a.x) : mk<R>(a.y, -a.x);
}

// Radix plan of a 1D FFT of length N (product of radices 2, 3, 4, 5, 8).
struct FftPlan {
  int N;
  int nst;
  int radix[kMaxRadixStages];
};

// Per-phase constitutive constants (device copy of rve_phase_params).
// Rows per CTA of the x1 passes.  Rows of a compile-time length (half
// length M in {32, 48, 64, 128}) are grouped so that about kX1CtElems
// complex points are transformed per CTA; other lengths stage at most
// e = 4 (or 16 for long rows) points per thread.  Shared by the launch
// configuration and the compile-time kernels.
#ifndef RVK_X1_CT_ELEMS
#define RVK_X1_CT_ELEMS 2048
#endif
constexpr int kX1CtElems = RVK_X1_CT_ELEMS;
__host__ __device__ constexpr bool x1_ct_length(int M) { return M == 32 || M == 48 || M == 64 || M == 128; }
__host__ __device__ constexpr int x1_ct_rows(int M, int c) {
  return kX1CtElems / (M * c) < 1 ? 1 : (kX1CtElems / (M * c) > 32 ? 32 : kX1CtElems / (M * c));
}

// strided / last axes of these lengths run the compile-time register passes
__host__ __device__ constexpr bool reg_axis(int N) { return N == 64 || N == 128 || N == 256; }

struct PhaseDev {
  double K, mu, sigma_y, H;
  double eps_C, eps_R, D_max;
  double inv_dCR;   // 1 / (eps_R - eps_C)
  int law;    // 0 elastic, 1 J2 + Lemaitre damage, 2 cracking particle, 3 GTN
  int var;    // non-local variable fed / read (law 3: var and var + 1), -1 none
  int hard;   // flow stress: 0 linear, 1 Aravas power law
  int pad_;
  double N;        // Aravas exponent
  double c_hard;   // 3 mu / sigma_y of the unscaled phase (Aravas law)
  // Gurson-Tvergaard-Needleman (law 3)
  double q1, q2, q3;
  double f_C, f_F, fV;       // coalescence onset, fracture, f_V* (surface at the origin)
  double f_N, eps_N, s_N;    // Chu-Needleman nucleation
  double f0, fstar_max;      // initial porosity, cap on f*
};

struct PhaseTable {
  PhaseDev p[kMaxPhases];
  int n_phases;
  float ell2f[kMaxVars][kMaxPhases];
  double ell2[kMaxVars][kMaxPhases];
};

// Scalars of one Krylov solve, kept on the device between kernels.
struct KrylovCtl {
  double rr;       // (r, r) for CG / (r, M r) for PCG
  double rnorm2;   // (r, r)
  double b2;       // (b, b)
  double pAp;
  double alpha, beta;
  double rtol2;
  double tol2;     // stop when (r, r) <= tol2 = max(rtol^2 (b, b), floor^2)
  double best;     // smallest (r, r) seen (stall detection)
  int best_it;
  int stall;       // > 0: stop after this many iterations without (r, r)
                   // falling below best / 4 (FP32 Krylov solves)
  // status: 0 running, 1 converged, 2 budget, 3 non-finite, 4 stopped at
  // the round-off floor ((p, Ap) <= 0)
  int iter, maxit, done, status;
  // set by a kernel whose tile copy did not complete within its wait budget
  // (never reset: the device is then not trustworthy)
  int wait_err;
};

__host__ __device__ inline int grid_linear_block() {
#ifdef __CUDA_ARCH__
  return blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
#else
  return 0;
#endif
}

// Deterministic block sum of NS doubles (fixed tree, fixed thread order).
template <int NS>
__device__ __forceinline__ void block_sum_store(double (&v)[NS], double* part, int nblk_stride) {
  __shared__ double red[kThreads / 32][NS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int s = 0; s < NS; s++) {
    double x = v[s];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) red[warp][s] = x;
  }
  __syncthreads();
  if (threadIdx.x < NS) {
    double acc = 0.0;
#pragma unroll
    for (int w = 0; w < kThreads / 32; w++) acc += red[w][threadIdx.x];
    part[threadIdx.x * nblk_stride + grid_linear_block()] = acc;
  }
}

// Deterministic block sum of per-thread FP32 partials: the warp tree runs in
// FP32 (each thread's partial covers a few voxels, a warp 32 of those), the
// warps' sums are added in FP64 in a fixed order.  Keeps the FP64 pipe,
// which is narrow, out of the per-voxel work.
template <int NS>
__device__ __forceinline__ void block_sum_store(float (&v)[NS], double* part, int nblk_stride) {
  __shared__ double redf[kThreads / 32][NS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int s = 0; s < NS; s++) {
    float x = v[s];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) redf[warp][s] = (double)x;
  }
  __syncthreads();
  if (threadIdx.x < NS) {
    double acc = 0.0;
#pragma unroll
    for (int w = 0; w < kThreads / 32; w++) acc += redf[w][threadIdx.x];
    part[threadIdx.x * nblk_stride + grid_linear_block()] = acc;
  }
}

// Block max of NS non-negative doubles.
template <int NS>
__device__ __forceinline__ void block_max_store(double (&v)[NS], double* part, int nblk_stride) {
  __shared__ double red[kThreads / 32][NS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int s = 0; s < NS; s++) {
    double x = v[s];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_down_sync(0xffffffffu, x, o));
    if (lane == 0) red[warp][s] = x;
  }
  __syncthreads();
  if (threadIdx.x < NS) {
    double acc = 0.0;
#pragma unroll
    for (int w = 0; w < kThreads / 32; w++) acc = fmax(acc, red[w][threadIdx.x]);
    part[threadIdx.x * nblk_stride + grid_linear_block()] = acc;
  }
}

}  // namespace rvk
