// Mixed-radix (2, 3, 4, 5, 8) Stockham FFT on lines held in shared memory.
//
// A batch of `nl` lines of length N lives in shared memory; element n of
// line l sits at buf[l * ls + n * es].  Each stage of radix RAD combines RAD
// sub-transforms of length Ns into transforms of length Ns * RAD: butterfly
// j (0 <= j < N/RAD) reads the elements j + r N/RAD, applies the twiddles
// W^(k r N/(Ns RAD)) with k = j mod Ns, takes a RAD-point DFT and writes the
// results to (j / Ns) Ns RAD + k + r Ns.  Stages run in place: every thread
// first stages its inputs in registers (at most E elements per thread), the
// CTA synchronises, then the outputs are written.  Transforms are
// unnormalised; SIGN = -1 is the forward transform exp(-2 pi i n k / N).
//
// Twiddles come from a table tw[m * twmul] = exp(-2 pi i m / N), computed on
// the host in double precision.
#pragma once
#include "common.cuh"

namespace rvk {

template <typename R> struct RConst;
template <> struct RConst<float> {
  static __device__ __forceinline__ float s3() { return 0.866025403784438646763723f; }
  static __device__ __forceinline__ float h2() { return 0.707106781186547524400844f; }
  static __device__ __forceinline__ float c51() { return 0.309016994374947424102293f; }
  static __device__ __forceinline__ float c52() { return -0.809016994374947424102293f; }
  static __device__ __forceinline__ float s51() { return 0.951056516295153572116439f; }
  static __device__ __forceinline__ float s52() { return 0.587785252292473129168706f; }
};
template <> struct RConst<double> {
  static __device__ __forceinline__ double s3() { return 0.866025403784438646763723; }
  static __device__ __forceinline__ double h2() { return 0.707106781186547524400844; }
  static __device__ __forceinline__ double c51() { return 0.309016994374947424102293; }
  static __device__ __forceinline__ double c52() { return -0.809016994374947424102293; }
  static __device__ __forceinline__ double s51() { return 0.951056516295153572116439; }
  static __device__ __forceinline__ double s52() { return 0.587785252292473129168706; }
};

// ------------------------------------------------------------ small DFTs
template <typename R, int RAD, int SIGN> struct Dft;

template <typename R, int SIGN> struct Dft<R, 2, SIGN> {
  static __device__ __forceinline__ void run(C2<R>* v) {
    C2<R> a = v[0], b = v[1];
    v[0] = a + b;
    v[1] = a - b;
  }
};

template <typename R, int SIGN> struct Dft<R, 3, SIGN> {
  static __device__ __forceinline__ void run(C2<R>* v) {
    C2<R> t = v[1] + v[2];
    C2<R> u = v[1] - v[2];
    C2<R> a = v[0];
    v[0] = a + t;
    C2<R> m = a - cscale(t, R(0.5));
    C2<R> n = cscale(mul_si<R, SIGN>(u), RConst<R>::s3());
    v[1] = m + n;
    v[2] = m - n;
  }
};

template <typename R, int SIGN> struct Dft<R, 4, SIGN> {
  static __device__ __forceinline__ void run(C2<R>* v) {
    C2<R> t0 = v[0] + v[2], t1 = v[0] - v[2];
    C2<R> t2 = v[1] + v[3], t3 = mul_si<R, SIGN>(v[1] - v[3]);
    v[0] = t0 + t2;
    v[2] = t0 - t2;
    v[1] = t1 + t3;
    v[3] = t1 - t3;
  }
};

template <typename R, int SIGN> struct Dft<R, 5, SIGN> {
  static __device__ __forceinline__ void run(C2<R>* v) {
    C2<R> t1 = v[1] + v[4], t2 = v[2] + v[3];
    C2<R> t3 = v[1] - v[4], t4 = v[2] - v[3];
    C2<R> a = v[0];
    v[0] = a + t1 + t2;
    C2<R> m1 = a + cscale(t1, RConst<R>::c51()) + cscale(t2, RConst<R>::c52());
    C2<R> m2 = a + cscale(t1, RConst<R>::c52()) + cscale(t2, RConst<R>::c51());
    C2<R> n1 = mul_si<R, SIGN>(cscale(t3, RConst<R>::s51()) + cscale(t4, RConst<R>::s52()));
    C2<R> n2 = mul_si<R, SIGN>(cscale(t3, RConst<R>::s52()) - cscale(t4, RConst<R>::s51()));
    v[1] = m1 + n1;
    v[4] = m1 - n1;
    v[2] = m2 + n2;
    v[3] = m2 - n2;
  }
};

template <typename R, int SIGN> struct Dft<R, 8, SIGN> {
  static __device__ __forceinline__ void run(C2<R>* v) {
    C2<R> e[4] = {v[0], v[2], v[4], v[6]};
    C2<R> o[4] = {v[1], v[3], v[5], v[7]};
    Dft<R, 4, SIGN>::run(e);
    Dft<R, 4, SIGN>::run(o);
    const R h = RConst<R>::h2();
    // o[m] *= exp(SIGN 2 pi i m / 8)
    o[1] = cscale(o[1] + mul_si<R, SIGN>(o[1]), h);
    o[2] = mul_si<R, SIGN>(o[2]);
    o[3] = cscale(mul_si<R, SIGN>(o[3]) - o[3], h);
#pragma unroll
    for (int m = 0; m < 4; m++) {
      v[m] = e[m] + o[m];
      v[m + 4] = e[m] - o[m];
    }
  }
};

// ------------------------------------------------------------ one stage
template <typename R, int E, int RAD, int SIGN>
__device__ __forceinline__ void fft_stage(C2<R>* buf, int N, int Ns, int nl, int es, int ls,
                                          bool jfast, const C2<R>* tw, int twmul) {
  constexpr int NB = (E + RAD - 1) / RAD;
  const int NR = N / RAD;
  const int nbf = nl * NR;
  C2<R> v[NB][RAD];
#pragma unroll
  for (int i = 0; i < NB; i++) {
    const int b = threadIdx.x + i * kThreads;
    if (b < nbf) {
      int line, j;
      if (jfast) { line = b / NR; j = b - line * NR; }
      else { j = b / nl; line = b - j * nl; }
      const C2<R>* base = buf + line * ls;
#pragma unroll
      for (int r = 0; r < RAD; r++) v[i][r] = base[(j + r * NR) * es];
    }
  }
  __syncthreads();
  const int tstep = N / (Ns * RAD);
#pragma unroll
  for (int i = 0; i < NB; i++) {
    const int b = threadIdx.x + i * kThreads;
    if (b < nbf) {
      int line, j;
      if (jfast) { line = b / NR; j = b - line * NR; }
      else { j = b / nl; line = b - j * nl; }
      const int k = j % Ns;
      if (k) {
        const int st = k * tstep;
#pragma unroll
        for (int r = 1; r < RAD; r++) {
          int idx = (st * r) % N;
          C2<R> w = tw[idx * twmul];
          if (SIGN > 0) w.y = -w.y;
          v[i][r] = cmul(v[i][r], w);
        }
      }
      Dft<R, RAD, SIGN>::run(v[i]);
      C2<R>* base = buf + line * ls;
      const int o0 = (j / Ns) * Ns * RAD + k;
#pragma unroll
      for (int r = 0; r < RAD; r++) base[(o0 + r * Ns) * es] = v[i][r];
    }
  }
  __syncthreads();
}

// Full transform of nl lines; requires nl * N <= E * kThreads.
template <typename R, int E, int SIGN>
__device__ void fft_lines(C2<R>* buf, const FftPlan& pl, int nl, int es, int ls, bool jfast,
                          const C2<R>* tw, int twmul) {
  int Ns = 1;
  for (int s = 0; s < pl.nst; s++) {
    const int rad = pl.radix[s];
    switch (rad) {
      case 2: fft_stage<R, E, 2, SIGN>(buf, pl.N, Ns, nl, es, ls, jfast, tw, twmul); break;
      case 3: fft_stage<R, E, 3, SIGN>(buf, pl.N, Ns, nl, es, ls, jfast, tw, twmul); break;
      case 4: fft_stage<R, E, 4, SIGN>(buf, pl.N, Ns, nl, es, ls, jfast, tw, twmul); break;
      case 5: fft_stage<R, E, 5, SIGN>(buf, pl.N, Ns, nl, es, ls, jfast, tw, twmul); break;
      default: fft_stage<R, E, 8, SIGN>(buf, pl.N, Ns, nl, es, ls, jfast, tw, twmul); break;
    }
    Ns *= rad;
  }
}

}  // namespace rvk
