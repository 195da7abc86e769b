// Allocation-free variant of the Galerkin projection G*(tau) for callers that
// cannot allocate device memory (see rve_op_apply_gamma_noalloc in rve.h).
//
// The half spectrum and the twiddle / half-angle tables of the call live in
// file-scope static device arrays; every GPU that loads the library holds
// them until the process exits.  In host code an array's name is only a
// host-side stand-in, so the device address of each array is looked up once
// per device with cudaGetSymbolAddress and passed to the kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "ops.h"
#include "rve.h"

using namespace rvk;

namespace {

constexpr size_t kScratchBytes = 32u << 20;   // 32 MiB of FP64 half spectrum
constexpr int kMaxAxis = 1024;                 // longest axis
constexpr int kMaxDevices = 64;
constexpr double kPiNA = 3.14159265358979323846;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];
static __device__ __align__(256) C2<double> g_tw[3][kMaxAxis];
static __device__ __align__(256) double g_s[3][kMaxAxis];
static __device__ __align__(256) double g_c[3][kMaxAxis];
// set by a CTA of the 3D projection pass whose tile copy did not arrive
// within its wait budget
static __device__ __align__(256) int g_wait_flag;

struct DevSymbols {
  bool ready = false;
  void* scratch = nullptr;
  C2<double>* tw = nullptr;
  double* s = nullptr;
  double* c = nullptr;
  int* wait_flag = nullptr;
};

std::mutex g_mutex;
DevSymbols g_dev[kMaxDevices];

// Device addresses of the static arrays on the current device (looked up
// on the first call made with that device current).
int symbols_for_current_device(DevSymbols** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return RVE_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return RVE_ERR_ARG;
  std::lock_guard<std::mutex> lock(g_mutex);
  DevSymbols& d = g_dev[dev];
  if (!d.ready) {
    if (cudaGetSymbolAddress(&d.scratch, g_scratch) != cudaSuccess ||
        cudaGetSymbolAddress((void**)&d.tw, g_tw) != cudaSuccess ||
        cudaGetSymbolAddress((void**)&d.s, g_s) != cudaSuccess ||
        cudaGetSymbolAddress((void**)&d.c, g_c) != cudaSuccess ||
        cudaGetSymbolAddress((void**)&d.wait_flag, g_wait_flag) != cudaSuccess) {
      cudaGetLastError();
      return RVE_ERR_CUDA;
    }
    d.ready = true;
  }
  *out = &d;
  return RVE_OK;
}

bool plan_of(int N, FftPlan& pl) {
  pl.N = N;
  pl.nst = 0;
  int m = N;
  const int rad[5] = {8, 4, 2, 5, 3};
  while (m > 1) {
    bool found = false;
    for (int r : rad) {
      if (m % r == 0) {
        if (pl.nst >= kMaxRadixStages) return false;
        pl.radix[pl.nst++] = r;
        m /= r;
        found = true;
        break;
      }
    }
    if (!found) return false;
  }
  return true;
}

}  // namespace

extern "C" int rve_op_apply_gamma_noalloc(int dim, const int n[3], const double L[3],
                                          const uint8_t strain_ctrl[6], const double* tau, double* out,
                                          void* cuda_stream) {
  if (!n || !L || !strain_ctrl || !tau || !out) return RVE_ERR_ARG;
  if (dim != 2 && dim != 3) return RVE_ERR_ARG;
  const int nn[3] = {n[0], n[1], dim == 3 ? n[2] : 1};
  const double LL[3] = {L[0], L[1], dim == 3 ? L[2] : 1.0};
  for (int j = 0; j < dim; j++)
    if (nn[j] < 1 || !(LL[j] > 0.0) || nn[j] > kMaxAxis) return RVE_ERR_ARG;
  if (nn[0] < 2 || nn[0] % 2) return RVE_ERR_ARG;
  for (int c = 0; c < 6; c++)
    if (strain_ctrl[c] > 1) return RVE_ERR_ARG;
  const int nc = dim == 3 ? 6 : 3;
  if ((nn[0] / 2) * nc > 16 * kThreads) return RVE_ERR_ARG;
  const int nmax = std::max(nn[1], nn[2]);
  if (nmax > 4 * kThreads) return RVE_ERR_ARG;
  FftPlan pl[3];
  if (!plan_of(nn[0] / 2, pl[0]) || !plan_of(nn[1], pl[1]) || !plan_of(nn[2], pl[2])) return RVE_ERR_ARG;

  Geo g{};
  g.d = dim;
  g.n1 = nn[0];
  g.n2 = nn[1];
  g.n3 = nn[2];
  g.M = nn[0] / 2;
  g.P1 = g.M + 1;
  g.ps = ((g.P1 + 15) / 16) * 16;
  g.nc = nc;
  const int cm3[6] = {0, 1, 2, 3, 4, 5}, cm2[6] = {0, 1, 5, 0, 0, 0};
  for (int c = 0; c < 6; c++) g.cmap[c] = dim == 3 ? cm3[c] : cm2[c];
  g.V = (long long)nn[0] * nn[1] * nn[2];
  g.nlines = (long long)nn[1] * nn[2];
  g.sstride = (long long)g.ps * nn[1] * nn[2];
  for (int j = 0; j < 3; j++) g.h[j] = LL[j] / nn[j];
  // sizes beyond the static scratch are rejected
  if ((size_t)nc * (size_t)g.sstride * sizeof(C2<double>) > kScratchBytes) return RVE_ERR_ARG;

  LaunchCfg lc{};
  for (int c = 1; c <= 6; c++) {
    const int e = (c * g.M <= 4 * kThreads) ? 4 : 16;
    lc.xe_c[c] = e;
    lc.nrows_c[c] = (e == 4 && x1_ct_length(g.M)) ? x1_ct_rows(g.M, c)
                                                  : std::max(1, std::min(32, (e * kThreads) / (c * g.M)));
  }
  lc.nrows_c[0] = 1;
  lc.xe_c[0] = 16;
  int tx = 1;
  while (tx * 2 * nmax <= 4 * kThreads && tx * 2 <= 32) tx *= 2;
  lc.tx = tx;
  lc.n_ew_blocks = 1;
  lc.max_blocks = 1;

  DevSymbols* sym = nullptr;
  int s = symbols_for_current_device(&sym);
  if (s != RVE_OK) return s;
  cudaStream_t st = (cudaStream_t)cuda_stream;

  // tables of this grid (host stack), copied into the static arrays
  C2<double> tw[kMaxAxis];
  double sv[kMaxAxis], cv[kMaxAxis];
  Tables<double> t;
  for (int j = 0; j < 3; j++) {
    const int N = nn[j];
    for (int m = 0; m < N; m++) {
      const double ang = -2.0 * kPiNA * (double)m / (double)N;
      tw[m].x = std::cos(ang);
      tw[m].y = std::sin(ang);
      const int q = m < (N + 1) / 2 ? m : m - N;
      const double half = kPiNA * (double)q / (double)N;
      sv[m] = std::sin(half);
      cv[m] = (2 * std::abs(q) == N) ? 0.0 : std::cos(half);
    }
    C2<double>* dtw = sym->tw + (size_t)j * kMaxAxis;
    double* ds = sym->s + (size_t)j * kMaxAxis;
    double* dc = sym->c + (size_t)j * kMaxAxis;
    if (cudaMemcpyAsync(dtw, tw, N * sizeof(C2<double>), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(ds, sv, N * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(dc, cv, N * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess) {
      cudaGetLastError();
      return RVE_ERR_CUDA;
    }
    t.tw[j] = dtw;
    t.s[j] = ds;
    t.c[j] = dc;
    t.two_over_h[j] = 2.0 / g.h[j];
  }
  t.plan_x = pl[0];
  t.plan_y = pl[1];
  t.plan_z = pl[2];

  float mask[6];
  for (int c = 0; c < 6; c++) mask[c] = c < nc ? (strain_ctrl[g.cmap[c]] ? 0.f : 1.f) : 0.f;
  int map[6] = {0, 1, 2, 3, 4, 5};
  C2<double>* S = (C2<double>*)sym->scratch;
  // the flag keeps the last call's value: clear it before this call's sweep
  if (cudaMemsetAsync(sym->wait_flag, 0, sizeof(int), st) != cudaSuccess) {
    cudaGetLastError();
    return RVE_ERR_CUDA;
  }
  Ops<double>::xfwd_field64(g, t, lc, st, tau, nc, map, nullptr, S);
  if (dim == 3) Ops<double>::strided_plain(g, t, lc, st, S, nc, 1, -1, nullptr);
  Ops<double>::gamma(g, t, lc, st, S, mask, 0, nullptr, sym->wait_flag);
  if (dim == 3) Ops<double>::strided_plain(g, t, lc, st, S, nc, 1, +1, nullptr);
  Ops<double>::xinv_store64(g, t, lc, st, S, nc, out);
  int waited_out = 0;
  if (cudaGetLastError() != cudaSuccess) return RVE_ERR_CUDA;
  if (cudaMemcpyAsync(&waited_out, sym->wait_flag, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) {
    cudaGetLastError();
    return RVE_ERR_CUDA;
  }
  if (cudaStreamSynchronize(st) != cudaSuccess) return RVE_ERR_CUDA;
  return waited_out ? RVE_ERR_TIMEOUT : RVE_OK;
}
