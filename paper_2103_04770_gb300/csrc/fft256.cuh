// 256-point transforms of lines held in shared memory, as two radix-16
// passes with every butterfly in registers.
//
// Write a position p in 0..255 as p = a + 16 b (a, b in 0..15).  The forward
// transform (exp(-2 pi i n k / 256)) runs
//   pass A: for each a, the 16-point DFT over b of x[a + 16 b], each output
//           r multiplied by W^(a r) (W = exp(-2 pi i / 256)) and written back
//           to position a + 16 r;
//   pass B: for each b, the 16-point DFT over a of the entries a + 16 b,
//           output k written back to position k + 16 b,
// which leaves X[b + 16 a] at position a + 16 b: the spectrum with its two
// base-16 digits swapped (swap16).  The inverse runs the mirror image from
// that order (pass B with the conjugate twiddles applied after its DFT, then
// pass A without twiddles) and ends in natural order.  In each pass a thread
// reads and writes back only its own 16 entries, so a pass needs no barrier
// between its loads and its stores; one barrier separates the two passes.
// Transforms are unnormalised.
//
// Lines are interleaved: element n of line l sits at buf[n * ES + l] (ES >=
// NL, the number of lines), so the lanes of a warp (consecutive l) touch
// consecutive entries.
#pragma once
#include "fft.cuh"

namespace rvk {

// cos(2 pi m / 16), m = 0..15
constexpr double kCos16[16] = {1.0,
                               0.92387953251128675613,
                               0.70710678118654752440,
                               0.38268343236508977173,
                               0.0,
                               -0.38268343236508977173,
                               -0.70710678118654752440,
                               -0.92387953251128675613,
                               -1.0,
                               -0.92387953251128675613,
                               -0.70710678118654752440,
                               -0.38268343236508977173,
                               0.0,
                               0.38268343236508977173,
                               0.70710678118654752440,
                               0.92387953251128675613};

// v * exp(SIGN 2 pi i M / 16)
template <typename R, int SIGN, int M>
__device__ __forceinline__ C2<R> w16(C2<R> v) {
  constexpr int m = M & 15;
  if constexpr (m == 0) {
    return v;
  } else if constexpr (m == 4) {
    return mul_si<R, SIGN>(v);
  } else if constexpr (m == 8) {
    return mk<R>(-v.x, -v.y);
  } else if constexpr (m == 12) {
    return mul_si<R, -SIGN>(v);
  } else {
    constexpr double c = kCos16[m];
    constexpr double s = SIGN * kCos16[(m + 12) & 15];   // sin(2 pi m / 16)
    return cmul(v, mk<R>((R)c, (R)s));
  }
}

// 16-point DFT in registers, natural order in and out: n = 4 n1 + n2,
// 4-point DFTs over n1, twiddles exp(SIGN 2 pi i n2 k1 / 16), 4-point DFTs
// over n2; output k1 + 4 k2.
template <typename R, int SIGN>
__device__ __forceinline__ void dft16(C2<R> (&v)[16]) {
  C2<R> a0[4] = {v[0], v[4], v[8], v[12]};
  C2<R> a1[4] = {v[1], v[5], v[9], v[13]};
  C2<R> a2[4] = {v[2], v[6], v[10], v[14]};
  C2<R> a3[4] = {v[3], v[7], v[11], v[15]};
  Dft<R, 4, SIGN>::run(a0);
  Dft<R, 4, SIGN>::run(a1);
  Dft<R, 4, SIGN>::run(a2);
  Dft<R, 4, SIGN>::run(a3);
  a1[1] = w16<R, SIGN, 1>(a1[1]);
  a1[2] = w16<R, SIGN, 2>(a1[2]);
  a1[3] = w16<R, SIGN, 3>(a1[3]);
  a2[1] = w16<R, SIGN, 2>(a2[1]);
  a2[2] = w16<R, SIGN, 4>(a2[2]);
  a2[3] = w16<R, SIGN, 6>(a2[3]);
  a3[1] = w16<R, SIGN, 3>(a3[1]);
  a3[2] = w16<R, SIGN, 6>(a3[2]);
  a3[3] = w16<R, SIGN, 9>(a3[3]);
#pragma unroll
  for (int k1 = 0; k1 < 4; k1++) {
    C2<R> b[4] = {a0[k1], a1[k1], a2[k1], a3[k1]};
    Dft<R, 4, SIGN>::run(b);
#pragma unroll
    for (int k2 = 0; k2 < 4; k2++) v[k1 + 4 * k2] = b[k2];
  }
}

// position of the spectrum entry X[f] after the forward transform (and the
// frequency held at position p): the two base-16 digits swapped
__host__ __device__ __forceinline__ int swap16(int p) { return ((p & 15) << 4) | (p >> 4); }

// One pass over NL lines: task (l, q) for q in 0..15 takes the entries
// q + 16 i (STRIDED) or 16 q + i (contiguous), i = 0..15, applies the
// 16-point DFT and, with TWID, the twiddles tw[q i] (conjugated for
// SIGN > 0), and writes them back in place.  tw[m] = exp(-2 pi i m / 256).
template <typename R, int NL, int ES, int SIGN, bool STRIDED, bool TWID>
__device__ __forceinline__ void fft256_pass(C2<R>* buf, const C2<R>* tw) {
  constexpr int NT = NL * 16;
#pragma unroll 1
  for (int t = threadIdx.x; t < NT; t += kThreads) {
    const int l = t % NL, q = t / NL;
    C2<R>* p = buf + l + (STRIDED ? q : 16 * q) * ES;
    constexpr int step = (STRIDED ? 16 : 1) * ES;
    C2<R> v[16];
#pragma unroll
    for (int i = 0; i < 16; i++) v[i] = p[i * step];
    dft16<R, SIGN>(v);
    if constexpr (TWID) {
#pragma unroll
      for (int i = 1; i < 16; i++) {
        C2<R> w = tw[q * i];
        if (SIGN > 0) w.y = -w.y;
        v[i] = cmul(v[i], w);
      }
    }
#pragma unroll
    for (int i = 0; i < 16; i++) p[i * step] = v[i];
  }
}

// Forward transform of NL lines, natural order in, swap16 order out.  The
// caller synchronises before the call (loads visible); the call ends with a
// barrier.
template <typename R, int NL, int ES = NL>
__device__ __forceinline__ void fft256_forward(C2<R>* buf, const C2<R>* tw) {
  fft256_pass<R, NL, ES, -1, true, true>(buf, tw);
  __syncthreads();
  fft256_pass<R, NL, ES, -1, false, false>(buf, tw);
  __syncthreads();
}

// Inverse transform of NL lines, swap16 order in, natural order out.
template <typename R, int NL, int ES = NL>
__device__ __forceinline__ void fft256_inverse(C2<R>* buf, const C2<R>* tw) {
  fft256_pass<R, NL, ES, 1, false, true>(buf, tw);
  __syncthreads();
  fft256_pass<R, NL, ES, 1, true, false>(buf, tw);
  __syncthreads();
}


// ------------------------------------------------ other lengths N = R1 R2
// The same two-pass scheme for N = R1 R2 (position p = a + R1 b):
//   forward  pass A: for each a < R1, the R2-point DFT over b of x[a + R1 b],
//                    output r times W_N^(a r) written to a + R1 r;
//            pass B: for each r < R2, the R1-point DFT over a of the entries
//                    a + R1 r, output k written to k + R1 r,
// leaving X[r + R2 k] at position k + R1 r; the inverse runs pass B (twiddles
// W_N^(-r a) after its DFT) then pass A and ends in natural order.  R1 = R2 =
// 16 is the 256-point scheme above.
template <int N> struct RegSplit;
template <> struct RegSplit<256> { static constexpr int r1 = 16, r2 = 16; };
template <> struct RegSplit<128> { static constexpr int r1 = 8, r2 = 16; };
template <> struct RegSplit<64> { static constexpr int r1 = 8, r2 = 8; };

// position of spectrum entry f after the forward transform
template <int N>
__host__ __device__ __forceinline__ int reg_pos(int f) {
  return f / RegSplit<N>::r2 + RegSplit<N>::r1 * (f % RegSplit<N>::r2);
}
// frequency held at position p after the forward transform
template <int N>
__host__ __device__ __forceinline__ int reg_freq(int p) {
  return p / RegSplit<N>::r1 + RegSplit<N>::r2 * (p % RegSplit<N>::r1);
}

template <typename R, int RAD, int SIGN>
__device__ __forceinline__ void dft_reg(C2<R> (&v)[RAD]) {
  if constexpr (RAD == 16) dft16<R, SIGN>(v);
  else Dft<R, RAD, SIGN>::run(v);
}

// One pass over NL lines of N = R1 R2 points (element n of line l at
// buf[n ES + l]), spread over the CTA's NTH threads: STRIDED takes, for task (l, a), a < R1, the R2 entries
// a + R1 i; otherwise, for task (l, r), r < R2, the R1 entries i + R1 r.
// TWID multiplies output i by tw[q i] (conjugated for SIGN > 0), q the
// task's a or r; tw[m] = exp(-2 pi i m / N).
template <typename R, int N, int NL, int ES, int SIGN, bool STRIDED, bool TWID, int NTH = kThreads>
__device__ __forceinline__ void fftreg_pass(C2<R>* buf, const C2<R>* tw) {
  constexpr int R1 = RegSplit<N>::r1, R2 = RegSplit<N>::r2;
  constexpr int L = STRIDED ? R2 : R1;          // DFT length
  constexpr int Q = STRIDED ? R1 : R2;          // tasks per line
  constexpr int NT = NL * Q;
#pragma unroll 1
  for (int t = threadIdx.x; t < NT; t += NTH) {
    const int l = t % NL, q = t / NL;
    C2<R>* p = buf + l + (STRIDED ? q : R1 * q) * ES;
    constexpr int step = (STRIDED ? R1 : 1) * ES;
    C2<R> v[L];
#pragma unroll
    for (int i = 0; i < L; i++) v[i] = p[i * step];
    dft_reg<R, L, SIGN>(v);
    if constexpr (TWID) {
#pragma unroll
      for (int i = 1; i < L; i++) {
        C2<R> w = tw[q * i];
        if (SIGN > 0) w.y = -w.y;
        v[i] = cmul(v[i], w);
      }
    }
#pragma unroll
    for (int i = 0; i < L; i++) p[i * step] = v[i];
  }
}

// Forward transform of NL lines, natural order in, reg_pos order out.  The
// caller synchronises before the call; the call ends with a barrier.
template <typename R, int N, int NL, int ES = NL, int NTH = kThreads>
__device__ __forceinline__ void fftreg_forward(C2<R>* buf, const C2<R>* tw) {
  fftreg_pass<R, N, NL, ES, -1, true, true, NTH>(buf, tw);
  __syncthreads();
  fftreg_pass<R, N, NL, ES, -1, false, false, NTH>(buf, tw);
  __syncthreads();
}

// Inverse transform of NL lines, reg_pos order in, natural order out.
template <typename R, int N, int NL, int ES = NL, int NTH = kThreads>
__device__ __forceinline__ void fftreg_inverse(C2<R>* buf, const C2<R>* tw) {
  fftreg_pass<R, N, NL, ES, 1, false, true, NTH>(buf, tw);
  __syncthreads();
  fftreg_pass<R, N, NL, ES, 1, true, false, NTH>(buf, tw);
  __syncthreads();
}

}  // namespace rvk
