// Mixed-radix Stockham FFT with every size known at compile time.
//
// Same stage formulation as fft.cuh (butterfly j reads j + r N/RAD, applies
// W^(k r N/(Ns RAD)) with k = j mod Ns, writes (j/Ns) Ns RAD + k + r Ns), but
// the transform length N, the number of lines NL, the element and line
// strides ES / LS, the twiddle-table stride and the radix of every stage are
// template parameters, so all index arithmetic folds into constants and
// shifts and every register array is sized exactly.
#pragma once
#include "fft.cuh"

namespace rvk {

// radix of the next stage for the REM points still to combine
template <int REM> struct PickRadix {
  static constexpr int v = (REM % 8 == 0) ? 8 : (REM % 4 == 0) ? 4 : (REM % 2 == 0) ? 2 : (REM % 5 == 0) ? 5 : 3;
};

// shared-memory index with one padding entry every 2^PADSH entries (PADSH =
// 0: none); breaks the power-of-two strides of the Stockham writes
template <int PADSH>
__device__ __forceinline__ int cpad(int i) {
  return PADSH ? i + (i >> PADSH) : i;
}

template <typename R, int N, int NL, int ES, int LS, int SIGN, bool JFAST, int TWMUL, int Ns, int RAD,
          int PADSH = 0>
__device__ __forceinline__ void ct_stage(C2<R>* buf, const C2<R>* tw) {
  constexpr int NR = N / RAD;
  constexpr int NBF = NL * NR;
  constexpr int NB = (NBF + kThreads - 1) / kThreads;
  constexpr int TSTEP = N / (Ns * RAD);
  C2<R> v[NB][RAD];
#pragma unroll
  for (int i = 0; i < NB; i++) {
    const int b = threadIdx.x + i * kThreads;
    if (NBF % kThreads == 0 || b < NBF) {
      int line, j;
      if (JFAST) { line = b / NR; j = b - line * NR; }
      else { j = b / NL; line = b - j * NL; }
#pragma unroll
      for (int r = 0; r < RAD; r++) v[i][r] = buf[cpad<PADSH>(line * LS + (j + r * NR) * ES)];
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NB; i++) {
    const int b = threadIdx.x + i * kThreads;
    if (NBF % kThreads == 0 || b < NBF) {
      int line, j;
      if (JFAST) { line = b / NR; j = b - line * NR; }
      else { j = b / NL; line = b - j * NL; }
      const int k = j % Ns;
      if (Ns > 1) {
#pragma unroll
        for (int r = 1; r < RAD; r++) {
          C2<R> w = tw[(k * TSTEP * r) * TWMUL];
          if (SIGN > 0) w.y = -w.y;
          v[i][r] = cmul(v[i][r], w);
        }
      }
      Dft<R, RAD, SIGN>::run(v[i]);
      const int o0 = (j / Ns) * Ns * RAD + k;
#pragma unroll
      for (int r = 0; r < RAD; r++) buf[cpad<PADSH>(line * LS + (o0 + r * Ns) * ES)] = v[i][r];
    }
  }
  __syncthreads();
}

template <typename R, int N, int NL, int ES, int LS, int SIGN, bool JFAST, int TWMUL, int Ns, int PADSH>
struct CtStages {
  static __device__ __forceinline__ void run(C2<R>* buf, const C2<R>* tw) {
    if constexpr (Ns < N) {
      constexpr int RAD = PickRadix<N / Ns>::v;
      ct_stage<R, N, NL, ES, LS, SIGN, JFAST, TWMUL, Ns, RAD, PADSH>(buf, tw);
      CtStages<R, N, NL, ES, LS, SIGN, JFAST, TWMUL, Ns * RAD, PADSH>::run(buf, tw);
    }
  }
};

// NL lines of length N: element n of line l at buf[cpad(l * LS + n * ES)].
template <typename R, int N, int NL, int ES, int LS, int SIGN, bool JFAST, int TWMUL, int PADSH = 0>
__device__ __forceinline__ void fft_lines_ct(C2<R>* buf, const C2<R>* tw) {
  CtStages<R, N, NL, ES, LS, SIGN, JFAST, TWMUL, 1, PADSH>::run(buf, tw);
}

}  // namespace rvk
