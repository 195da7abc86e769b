// C ABI and host drivers of the GB300 non-local damage RVE library.
//
// Host side of Algorithm 1 (iterated staggered scheme), the Newton /
// conjugate-gradient FFT-Galerkin mechanics of Section 3.2.2 and the
// preconditioned CG Helmholtz solve of Algorithm 2.  Every arithmetic step
// runs in the device operators of ops.cuh; the host only sequences launches,
// reads back a few scalars per Newton iteration and per chunk of Krylov
// iterations, and decides convergence.
#include <cuda_runtime.h>

#include <thread>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <new>
#include <vector>

#include "adjoint_ops.h"
#include "ops.h"
#include "rve.h"

using namespace rvk;

namespace {

constexpr int kSlots = 8;
constexpr double kPi = 3.14159265358979323846;
constexpr int kScal = 64;
enum {
  OFF_SIGMEAN = 0,    // 6 (+ D mean at 6)
  OFF_DMEAN = 6,
  OFF_DMAX = 7,
  OFF_EPSMEAN = 8,    // 6
  OFF_MAXDX = 14,
  OFF_ERRMEAN = 16,   // 6
  OFF_ERRMAX = 22,
  OFF_ABAR = 24,      // 2 per variable
  OFF_SIGREF = 40,    // 6: mean stress of the residual reference (mixed form)
};

// kernel classes of the launch accounting
enum {
  KC_RETURN_MAP = 0,
  KC_X_FWD_TANGENT,
  KC_X_FWD_FIELD,
  KC_Y_PASS,
  KC_GAMMA,
  KC_X_INV_MATVEC,
  KC_X_INV_RESIDUAL,
  KC_X_INV_STORE,
  KC_HELM_EXPAND,
  KC_HELM_X1,
  KC_HELM_CONTRACT,
  KC_CG_UPDATE,
  KC_PCG_UPDATE,
  KC_FINALIZE,
  KC_MISC,
  KC_RES_Y_PASS,
  KC_RES_GAMMA,
  KC_HELM_STENCIL,
  KC_COUNT
};
const char* const kClassNames[KC_COUNT] = {
    "return_map", "x1_fwd_tangent", "x1_fwd_field", "y_pass", "gamma_last_axis", "x1_inv_matvec",
    "x1_inv_residual", "x1_inv_store", "helmholtz_expand", "helmholtz_x1", "helmholtz_contract",
    "cg_update", "pcg_update", "finalize", "misc", "residual_y_pass", "residual_gamma", "helmholtz_stencil"};

struct PendingEv {
  int cls;
  cudaEvent_t a, b;
};

}  // namespace

struct AdjointStore;

struct rve {
  int dim = 0, prec = 0, J = 0;
  int n[3] = {1, 1, 1};
  double L[3] = {1, 1, 1};
  cudaStream_t st = nullptr;
  Geo g{};
  LaunchCfg lc{};
  rve_solver_options opt{};
  // phases
  int n_phases = 0;
  bool phases_set = false;
  PhaseTable pt_host{};
  PhaseTable* pt_dev = nullptr;
  double ell2_mean[kMaxVars] = {0, 0, 0, 0};
  void* ell2R = nullptr;         // [kMaxVars][kMaxPhases] in working precision
  // load path
  int n_incr = 0, n_done = 0;
  bool path_set = false;
  uint8_t ctrl[6] = {1, 1, 1, 1, 1, 1};
  std::vector<double> target;    // tensor shears
  double E_prev[6] = {0, 0, 0, 0, 0, 0};
  // stress targets of the stress-controlled components at the last
  // converged (sub-)step (interpolation origin of cut-back sub-steps)
  double S_prev[6] = {0, 0, 0, 0, 0, 0};
  double smask_d[6] = {0, 0, 0, 0, 0, 0};
  float smask_f[6] = {0, 0, 0, 0, 0, 0};
  // FP64 state
  uint8_t* phase = nullptr;
  double *eps = nullptr, *eps_conv = nullptr, *eps_prev = nullptr;
  double *epsp_n = nullptr, *epsp = nullptr, *ep_n = nullptr, *ep = nullptr;
  double *sigma = nullptr, *D = nullptr, *alpha = nullptr;
  double *abar_n = nullptr, *abar_k = nullptr, *abar_new = nullptr;
  // working precision
  void *x = nullptr, *r = nullptr, *p = nullptr, *Ap = nullptr, *desc = nullptr;
  void* S = nullptr;
  void *hx = nullptr, *hr = nullptr, *hp = nullptr, *hy = nullptr;
  void* tw[3] = {nullptr, nullptr, nullptr};
  void* ts[3] = {nullptr, nullptr, nullptr};
  void* tc[3] = {nullptr, nullptr, nullptr};
  // FP64 tables, spectrum and launch shape of the Newton residual sweep
  // (aliases of the above in the FP64 form)
  void* tw64[3] = {nullptr, nullptr, nullptr};
  void* ts64[3] = {nullptr, nullptr, nullptr};
  void* tc64[3] = {nullptr, nullptr, nullptr};
  void* S64 = nullptr;
  LaunchCfg lc64{};
  FftPlan plan[3]{};
  // reductions and control
  double* part = nullptr;
  KrylovCtl* ctl = nullptr;
  FinScratch* fin = nullptr;     // two-level reduction scratch of k_finalize
  double* dscal = nullptr;
  KrylovCtl* hctl = nullptr;     // pinned
  double* hscal = nullptr;       // pinned
  // results of the last converged increment
  double sig_mean[6] = {0, 0, 0, 0, 0, 0};
  double eps_mean[6] = {0, 0, 0, 0, 0, 0};
  double D_mean = 0, D_max = 0;
  std::vector<void*> allocs;
  // launch accounting / profiling
  bool prof = false;
  long long launches[KC_COUNT] = {};
  double prof_ms[KC_COUNT] = {};
  double prof_bytes[KC_COUNT] = {};
  std::vector<cudaEvent_t> ev_free;
  std::vector<PendingEv> ev_pending;
  cudaEvent_t ev_cur_a = nullptr;
  int fail_stage = 0;
  int verbose = 0;      // RVE_VERBOSE=1: trace solver progress on stderr
  // CUDA graphs of the Krylov chunks (captured at first use, replayed after)
  bool graphs = false;
  cudaGraphExec_t g_cg = nullptr;
  cudaGraphExec_t g_pcg[kMaxVars] = {};
  long long g_cg_n[KC_COUNT] = {};
  double g_cg_b[KC_COUNT] = {};
  long long g_pcg_n[kMaxVars][KC_COUNT] = {};
  double g_pcg_b[kMaxVars][KC_COUNT] = {};
  bool stepped = false;  // an increment has been attempted (autotuning closed)
  double* stiff = nullptr;  // per-voxel modulus factor (nullptr: 1 everywhere)
  // GTN (law 3): porosity of the last converged increment and of the
  // current return map; the tangent descriptor takes the extended layout
  bool gtn = false;
  double *f_n = nullptr, *f = nullptr;
  // wait budget of the 3D projection pass's tile copies, and bytes added to
  // their expected count (tests of the timeout path only)
  double tile_wait_s = 2.0;
  int tile_extra_tx = 0;
  // mixed form: stress and FP64-swept residual of the last FP64 sweep of the
  // current increment (reference of the FP32 difference sweeps)
  double* sig_ref = nullptr;
  void* r_ref = nullptr;
  bool ref_ok = false;
  AdjointStore* adj = nullptr;
  // CG step fused into the inverse x1 pass (its prefetch of p, x and r fits
  // the shared memory of one CTA)
  bool cg_fused = false;
};

namespace {

#define CK(call)                                \
  do {                                          \
    cudaError_t e_ = (call);                    \
    if (e_ != cudaSuccess) return RVE_ERR_CUDA; \
  } while (0)

bool factor_plan(int N, FftPlan& pl) {
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

int dalloc(rve* h, void** p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  const cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? RVE_ERR_OOM : RVE_ERR_CUDA;
  }
  h->allocs.push_back(*p);
  return RVE_OK;
}

template <typename T>
int dalloc_t(rve* h, T** p, size_t count) {
  void* v = nullptr;
  int s = dalloc(h, &v, count * sizeof(T));
  *p = (T*)v;
  return s;
}

size_t rsize(const rve* h) { return h->prec == RVE_MIXED ? sizeof(float) : sizeof(double); }

template <typename R>
Tables<R> tables(const rve* h) {
  Tables<R> t;
  for (int j = 0; j < 3; j++) {
    t.tw[j] = (C2<R>*)h->tw[j];
    t.s[j] = (R*)h->ts[j];
    t.c[j] = (R*)h->tc[j];
    t.two_over_h[j] = (R)(2.0 / h->g.h[j]);
  }
  t.plan_x = h->plan[0];
  t.plan_y = h->plan[1];
  t.plan_z = h->plan[2];
  return t;
}

// resolve recorded event pairs (the stream must be synchronised)
void prof_resolve(rve* h) {
  for (const PendingEv& e : h->ev_pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, e.a, e.b) == cudaSuccess) h->prof_ms[e.cls] += ms;
    h->ev_free.push_back(e.a);
    h->ev_free.push_back(e.b);
  }
  h->ev_pending.clear();
  cudaGetLastError();
}

cudaEvent_t prof_event(rve* h) {
  if (h->ev_free.empty()) {
    if (h->ev_pending.size() >= 2048) {
      cudaStreamSynchronize(h->st);
      prof_resolve(h);
    }
    if (h->ev_free.empty()) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
      return e;
    }
  }
  cudaEvent_t e = h->ev_free.back();
  h->ev_free.pop_back();
  return e;
}

inline void prof_begin(rve* h, int cls, double bytes) {
  h->launches[cls]++;
  h->prof_bytes[cls] += bytes;
  if (!h->prof) return;
  h->ev_cur_a = prof_event(h);
  if (h->ev_cur_a) cudaEventRecord(h->ev_cur_a, h->st);
}

inline void prof_end(rve* h, int cls) {
  if (!h->prof || !h->ev_cur_a) return;
  cudaEvent_t b = prof_event(h);
  if (!b) return;
  cudaEventRecord(b, h->st);
  h->ev_pending.push_back(PendingEv{cls, h->ev_cur_a, b});
  h->ev_cur_a = nullptr;
}

// RVE_VERBOSE=2: synchronise after every launch and name the first one
// that fails (debugging aid; graphs are not captured in this mode)
inline void launch_check(rve* h, int cls) {
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
  if (e != cudaSuccess) {
    std::fprintf(stderr, "[rve] launch of class %s failed: %s\n", kClassNames[cls], cudaGetErrorString(e));
    h->verbose = 1;
  }
}

// every launch is counted with its algorithmic bytes (each operand read
// once, each result written once) and, when profiling, timed by events
#define LAUNCHB(h, cls, bytes, call)     \
  do {                                   \
    prof_begin((h), (cls), (bytes));     \
    call;                                \
    prof_end((h), (cls));                \
    if ((h)->verbose >= 2) launch_check((h), (cls)); \
  } while (0)

Tables<double> tables64(const rve* h) {
  Tables<double> t;
  for (int j = 0; j < 3; j++) {
    t.tw[j] = (C2<double>*)h->tw64[j];
    t.s[j] = (double*)h->ts64[j];
    t.c[j] = (double*)h->tc64[j];
    t.two_over_h[j] = 2.0 / h->g.h[j];
  }
  t.plan_x = h->plan[0];
  t.plan_y = h->plan[1];
  t.plan_z = h->plan[2];
  return t;
}

int sync_read(rve* h) {
  CK(cudaMemcpyAsync(h->hscal, h->dscal, kScal * sizeof(double), cudaMemcpyDeviceToHost, h->st));
  CK(cudaMemcpyAsync(h->hctl, h->ctl, sizeof(KrylovCtl), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  CK(cudaGetLastError());
  if (h->prof) prof_resolve(h);
  if (h->hctl->wait_err) return RVE_ERR_TIMEOUT;
  return RVE_OK;
}

// drop the captured Krylov chunks (their launches bake in the load path's
// stress mask, the characteristic lengths, the chunk length and the launch
// shapes)
void graphs_reset(rve* h) {
  if (h->g_cg) cudaGraphExecDestroy(h->g_cg);
  h->g_cg = nullptr;
  for (int j = 0; j < kMaxVars; j++) {
    if (h->g_pcg[j]) cudaGraphExecDestroy(h->g_pcg[j]);
    h->g_pcg[j] = nullptr;
  }
}

// Launch one Krylov chunk: directly, or (graphs on, profiling off) from a
// graph captured the first time.  The launch tallies of the capture are
// replayed with the graph.  A capture the runtime refuses falls back to
// direct launches for the rest of the handle's life.
template <class F>
int run_chunk(rve* h, cudaGraphExec_t* ex, long long* tn, double* tb, F&& chunk) {
  if (!h->graphs || h->prof || h->verbose >= 2) {
    chunk();
    return RVE_OK;
  }
  if (!*ex) {
    long long n0[KC_COUNT];
    double b0[KC_COUNT];
    std::memcpy(n0, h->launches, sizeof(n0));
    std::memcpy(b0, h->prof_bytes, sizeof(b0));
    if (cudaStreamBeginCapture(h->st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      h->graphs = false;
      chunk();
      return RVE_OK;
    }
    chunk();
    cudaGraph_t gr = nullptr;
    cudaError_t e = cudaStreamEndCapture(h->st, &gr);
    for (int k = 0; k < KC_COUNT; k++) {
      tn[k] = h->launches[k] - n0[k];
      tb[k] = h->prof_bytes[k] - b0[k];
      h->launches[k] = n0[k];
      h->prof_bytes[k] = b0[k];
    }
    if (e == cudaSuccess && gr) e = cudaGraphInstantiate(ex, gr, 0);
    if (gr) cudaGraphDestroy(gr);
    if (e != cudaSuccess) {
      cudaGetLastError();
      *ex = nullptr;
      h->graphs = false;
      chunk();
      return RVE_OK;
    }
  }
  CK(cudaGraphLaunch(*ex, h->st));
  for (int k = 0; k < KC_COUNT; k++) {
    h->launches[k] += tn[k];
    h->prof_bytes[k] += tb[k];
  }
  return RVE_OK;
}

int xblocks(const rve* h, int nc) {
  return (int)((h->g.nlines + h->lc.nrows_c[nc] - 1) / h->lc.nrows_c[nc]);
}

template <typename R>
struct Alg {
  using Op = Ops<R>;
  static constexpr double RS = sizeof(R);
  static constexpr double CS = 2.0 * sizeof(R);
  static double VS(const rve* h) { return (double)h->g.P1 * (double)h->g.nlines; }
  static double VV(const rve* h) { return (double)h->g.V; }

  // G* on the x1-transformed spectrum S: y forward, last-axis G*, y inverse.
  static void gamma_sweep(rve* h, const Tables<R>& t, int dc_mode, const KrylovCtl* ctl) {
    C2<R>* S = (C2<R>*)h->S;
    if (h->g.d == 3) LAUNCHB(h, KC_Y_PASS, 2.0 * (double)h->g.nc * VS(h) * CS, Op::strided_plain(h->g, t, h->lc, h->st, S, h->g.nc, 1, -1, ctl));
    LAUNCHB(h, KC_GAMMA, 2.0 * (double)h->g.nc * VS(h) * CS,
            Op::gamma(h->g, t, h->lc, h->st, S, h->smask_f, dc_mode, ctl, &h->ctl->wait_err, h->tile_wait_s,
                      h->tile_extra_tx));
    if (h->g.d == 3) LAUNCHB(h, KC_Y_PASS, 2.0 * (double)h->g.nc * VS(h) * CS, Op::strided_plain(h->g, t, h->lc, h->st, S, h->g.nc, 1, +1, ctl));
  }

  static void return_map(rve* h, const double* abar_use) {
    const double gb = h->gtn ? VV(h) * (16.0 * h->J + 16.0 + 2.0 * RS) : 0.0;
    LAUNCHB(h, KC_RETURN_MAP, VV(h) * (8.0 * h->g.nc + 169.0 + 16.0 * h->J + (2.0 + h->g.nc) * RS) + gb,
            Op::return_map(h->g, h->lc, h->st, h->pt_dev, h->J, h->phase, h->eps, h->epsp_n, h->ep_n, abar_use,
                           h->sigma, h->epsp, h->ep, h->D, h->alpha, (R*)h->desc, h->part, h->stiff, h->abar_n,
                           h->f_n, h->f, h->gtn));
    LAUNCHB(h, KC_FINALIZE, 0.0, k_finalize(h->st, h->fin, h->part, h->lc.n_ew_blocks, h->lc.max_blocks, 7, FIN_SUMS, nullptr,
               h->dscal + OFF_SIGMEAN, 1.0 / (double)h->g.V));
    LAUNCHB(h, KC_FINALIZE, 0.0, k_finalize(h->st, h->fin, h->part + 7 * (size_t)h->lc.max_blocks, h->lc.n_ew_blocks, h->lc.max_blocks, 1,
               FIN_MAXS, nullptr, h->dscal + OFF_DMAX, 1.0));
  }

  // b = -G*(sigma - Sigma_bar), swept in FP64 in both forms and stored in
  // the working precision into r; ctl initialised for CG.
  static void residual(rve* h, const double* sbar_c, double rtol, int maxit) {
    const Tables<double> t64 = tables64(h);
    C2<double>* S64 = (C2<double>*)h->S64;
    const Geo& g = h->g;
    const double cs64 = 16.0, nc = g.nc;
    LAUNCHB(h, KC_X_FWD_FIELD, nc * (8.0 * VV(h) + VS(h) * cs64),
            Ops<double>::xfwd_field64(g, t64, h->lc64, h->st, h->sigma, g.nc, g.cmap, h->dscal + OFF_SIGMEAN,
                                      S64));
    if (g.d == 3)
      LAUNCHB(h, KC_RES_Y_PASS, 2.0 * nc * VS(h) * cs64,
              Ops<double>::strided_plain(g, t64, h->lc64, h->st, S64, g.nc, 1, -1, nullptr));
    LAUNCHB(h, KC_RES_GAMMA, 2.0 * nc * VS(h) * cs64,
            Ops<double>::gamma(g, t64, h->lc64, h->st, S64, h->smask_f, 1, nullptr, &h->ctl->wait_err,
                               h->tile_wait_s, h->tile_extra_tx));
    if (g.d == 3)
      LAUNCHB(h, KC_RES_Y_PASS, 2.0 * nc * VS(h) * cs64,
              Ops<double>::strided_plain(g, t64, h->lc64, h->st, S64, g.nc, 1, +1, nullptr));
    LAUNCHB(h, KC_X_INV_RESIDUAL, nc * (VS(h) * cs64 + VV(h) * RS),
            Ops<double>::template xinv_residual<R>(g, t64, h->lc64, h->st, S64, (R*)h->r,
                                                   h->dscal + OFF_SIGMEAN, h->smask_d, sbar_c, h->part));
    LAUNCHB(h, KC_FINALIZE, 0.0, k_finalize(h->st, h->fin, h->part, xblocks(h, g.nc), h->lc.max_blocks, 1, FIN_CG_INIT,
                                            h->ctl, nullptr, rtol * rtol, maxit, stall_window()));
  }

  // b = -G*(sigma - Sigma_bar) swept in the working precision (mixed form,
  // far from Newton convergence: FP32 rounding of the transform, about 1e-7
  // of |sigma|, is then at most 1 % of the residual itself).
  static void residual_lo(rve* h, const Tables<R>& t, const double* sbar_c, double rtol, int maxit) {
    const Geo& g = h->g;
    const double nc = g.nc;
    C2<R>* S = (C2<R>*)h->S;
    LAUNCHB(h, KC_X_FWD_FIELD, nc * (8.0 * VV(h) + VS(h) * CS),
            Op::xfwd_field64(g, t, h->lc, h->st, h->sigma, g.nc, g.cmap, h->dscal + OFF_SIGMEAN, S));
    gamma_sweep(h, t, 1, nullptr);
    LAUNCHB(h, KC_X_INV_RESIDUAL, nc * (VS(h) * CS + VV(h) * RS),
            Op::template xinv_residual<R>(g, t, h->lc, h->st, S, (R*)h->r, h->dscal + OFF_SIGMEAN, h->smask_d,
                                          sbar_c, h->part));
    LAUNCHB(h, KC_FINALIZE, 0.0, k_finalize(h->st, h->fin, h->part, xblocks(h, g.nc), h->lc.max_blocks, 1, FIN_CG_INIT,
                                            h->ctl, nullptr, rtol * rtol, maxit, stall_window()));
  }

  // Keep the stress and the residual of the FP64 sweep just made as the
  // reference of later difference sweeps in this increment.
  static int save_ref(rve* h) {
    const Geo& g = h->g;
    CK(cudaMemcpyAsync(h->sig_ref, h->sigma, 6 * (size_t)g.V * 8, cudaMemcpyDeviceToDevice, h->st));
    CK(cudaMemcpyAsync(h->r_ref, h->r, (size_t)g.nc * g.V * sizeof(R), cudaMemcpyDeviceToDevice, h->st));
    CK(cudaMemcpyAsync(h->dscal + OFF_SIGREF, h->dscal + OFF_SIGMEAN, 6 * sizeof(double),
                       cudaMemcpyDeviceToDevice, h->st));
    h->ref_ok = true;
    return RVE_OK;
  }

  // Near Newton convergence (mixed form): G* is linear, so the residual at
  // sigma is the FP64-swept reference residual minus the FP32 sweep of the
  // small difference sigma - sigma_ref (Sigma_bar cancels); FP32 rounding is
  // then about 1e-7 of |sigma - sigma_ref|, not of |sigma|.
  static void residual_delta(rve* h, const Tables<R>& t, double rtol, int maxit) {
    const Geo& g = h->g;
    const double nc = g.nc;
    const double zero[6] = {0, 0, 0, 0, 0, 0};
    C2<R>* S = (C2<R>*)h->S;
    LAUNCHB(h, KC_X_FWD_FIELD, nc * (16.0 * VV(h) + VS(h) * CS),
            Op::xfwd_field64(g, t, h->lc, h->st, h->sigma, g.nc, g.cmap, h->dscal + OFF_SIGMEAN, S, h->sig_ref,
                             h->dscal + OFF_SIGREF));
    gamma_sweep(h, t, 1, nullptr);
    LAUNCHB(h, KC_X_INV_RESIDUAL, nc * (VS(h) * CS + 2.0 * VV(h) * RS),
            Op::template xinv_residual<R>(g, t, h->lc, h->st, S, (R*)h->r, h->dscal + OFF_SIGMEAN, h->smask_d,
                                          zero, h->part, (const R*)h->r_ref, h->dscal + OFF_SIGREF));
    LAUNCHB(h, KC_FINALIZE, 0.0, k_finalize(h->st, h->fin, h->part, xblocks(h, g.nc), h->lc.max_blocks, 1, FIN_CG_INIT,
                                            h->ctl, nullptr, rtol * rtol, maxit, stall_window()));
  }

  // FP32 Krylov solves stop when (r, r) has not fallen below a quarter of its
  // best value for this many iterations (attainable accuracy reached).
  static int stall_window() { return sizeof(R) == sizeof(float) ? 150 : 0; }

  // CG on G*(C_T : x) = b (r holds b in the range of G*, ctl initialised, x
  // zeroed by caller).  Fused form: G* is an orthogonal projection and the
  // directions p stay in its range, so the curvature (p, G*(C_T : p)) equals
  // (p, C_T : p), summed in the forward x1 pass; alpha is then known before
  // the inverse pass, which applies x += alpha p, r -= alpha A p at once and
  // never stores A p.
  static int cg_loop(rve* h, const Tables<R>& t, int* iters) {
    const Geo& g = h->g;
    const int chunk = std::max(1, h->opt.check_every);
    const int nbx = xblocks(h, g.nc);
    for (;;) {
      int s = run_chunk(h, &h->g_cg, h->g_cg_n, h->g_cg_b, [&]() {
        for (int i = 0; i < chunk && h->cg_fused; i++) {
          LAUNCHB(h, KC_X_FWD_TANGENT, VV(h) * RS * (4.0 * h->g.nc + 2.0) + h->g.nc * VS(h) * CS,
                  Op::xfwd_tangent(g, t, h->lc, h->st, (R*)h->p, (const R*)h->r, (const R*)h->desc,
                                   (C2<R>*)h->S, h->ctl, h->part, h->gtn));
          LAUNCHB(h, KC_FINALIZE, 0.0, k_finalize(h->st, h->fin, h->part, nbx, h->lc.max_blocks, 1, FIN_ALPHA, h->ctl, nullptr, 1.0));
          gamma_sweep(h, t, 0, h->ctl);
          LAUNCHB(h, KC_X_INV_MATVEC, (double)h->g.nc * (VS(h) * CS + 5.0 * VV(h) * RS),
                  Op::xinv_cg(g, t, h->lc, h->st, (const C2<R>*)h->S, (R*)h->x, (R*)h->r, (const R*)h->p,
                              h->part, h->ctl));
          LAUNCHB(h, KC_FINALIZE, 0.0, k_finalize(h->st, h->fin, h->part, nbx, h->lc.max_blocks, 1, FIN_CG_BETA, h->ctl, nullptr, 1.0));
        }
        for (int i = 0; i < chunk && !h->cg_fused; i++) {
          LAUNCHB(h, KC_X_FWD_TANGENT, VV(h) * RS * (4.0 * h->g.nc + 2.0) + h->g.nc * VS(h) * CS, Op::xfwd_tangent(g, t, h->lc, h->st, (R*)h->p, (const R*)h->r, (const R*)h->desc, (C2<R>*)h->S,
                           h->ctl, nullptr, h->gtn));
          gamma_sweep(h, t, 0, h->ctl);
          LAUNCHB(h, KC_X_INV_MATVEC, (double)h->g.nc * (VS(h) * CS + 2.0 * VV(h) * RS), Op::xinv_matvec(g, t, h->lc, h->st, (const C2<R>*)h->S, (R*)h->Ap, (const R*)h->p, h->part, h->ctl));
          LAUNCHB(h, KC_FINALIZE, 0.0, k_finalize(h->st, h->fin, h->part, nbx, h->lc.max_blocks, 1, FIN_ALPHA, h->ctl, nullptr, 1.0));
          LAUNCHB(h, KC_CG_UPDATE, 6.0 * g.nc * VV(h) * RS, Op::cg_update(g, h->lc, h->st, (R*)h->x, (R*)h->r, (const R*)h->p, (const R*)h->Ap, h->part, h->ctl));
          LAUNCHB(h, KC_FINALIZE, 0.0, k_finalize(h->st, h->fin, h->part, h->lc.n_ew_blocks, h->lc.max_blocks, 1, FIN_CG_BETA, h->ctl, nullptr, 1.0));
        }
      });
      if (s) return s;
      s = sync_read(h);
      if (s) return s;
      if (h->hctl->done) break;
    }
    *iters = h->hctl->iter;
    if (h->hctl->status == 3) { h->fail_stage = 5; return RVE_ERR_NUMERIC; }
    if (h->hctl->status == 2) { h->fail_stage = 2; return RVE_ERR_NOT_CONVERGED; }
    return RVE_OK;
  }

  // Newton-Raphson on the Galerkin residual at fixed abar (Algorithm 1 (i)).
  static int mech_solve(rve* h, const Tables<R>& t, const double* abar_use, const double* sbar_c,
                        int* newton_out, long long* cg_out) {
    const Geo& g = h->g;
    double de_rel = -1.0, last_res = -1.0;
    int newton = 0;
    // mixed form: the residual is swept in FP32 while it exceeds res_lo
    // (relative), in FP64 below it and for every convergence decision
    const double res_lo = std::max(100.0 * h->opt.tol_newton, 1e-4);
    for (;;) {
      return_map(h, abar_use);
      const bool mixed = sizeof(R) == sizeof(float);
      bool lo = mixed && (last_res < 0.0 || last_res > res_lo);
      int s = RVE_OK;
      // near convergence: a difference sweep against this increment's FP64
      // reference, else a full FP64 sweep that becomes the reference
      auto near = [&]() -> int {
        if (mixed && h->ref_ok) {
          residual_delta(h, t, h->opt.cg_rtol, h->opt.max_cg);
          return RVE_OK;
        }
        residual(h, sbar_c, h->opt.cg_rtol, h->opt.max_cg);
        return mixed ? save_ref(h) : RVE_OK;
      };
      if (lo) residual_lo(h, t, sbar_c, h->opt.cg_rtol, h->opt.max_cg);
      else if ((s = near())) return s;
      s = sync_read(h);
      if (s) return s;
      double sm = 0.0;
      for (int c = 0; c < g.nc; c++) sm += h->hscal[OFF_SIGMEAN + g.cmap[c]] * h->hscal[OFF_SIGMEAN + g.cmap[c]];
      sm = std::sqrt(sm);
      double b2 = h->hctl->b2;
      if (!(b2 == b2)) { h->fail_stage = 5; return RVE_ERR_NUMERIC; }
      double res_rel = std::sqrt(b2) / (std::sqrt((double)g.V) * std::max(sm, 1e-300));
      if (lo && res_rel <= res_lo) {
        if ((s = near())) return s;
        if ((s = sync_read(h))) return s;
        b2 = h->hctl->b2;
        if (!(b2 == b2)) { h->fail_stage = 5; return RVE_ERR_NUMERIC; }
        res_rel = std::sqrt(b2) / (std::sqrt((double)g.V) * std::max(sm, 1e-300));
      }
      last_res = res_rel;
      if (h->verbose)
        std::fprintf(stderr, "[rve] newton %d res_rel %.3e de_rel %.3e |<sigma>| %.6e\n", newton, res_rel,
                     de_rel, sm);
      if (res_rel < h->opt.tol_newton && (de_rel < 0.0 || de_rel < h->opt.tol_newton)) break;
      if (newton >= h->opt.max_newton) { h->fail_stage = 1; *newton_out += newton; return RVE_ERR_NOT_CONVERGED; }
      CK(cudaMemsetAsync(h->x, 0, (size_t)g.nc * g.V * rsize(h), h->st));
      // absolute floor of the linear solve: 0.01 TOL_N sqrt(V) |<sigma>|
      const double floor_ = 0.01 * h->opt.tol_newton * std::sqrt((double)g.V) * sm;
      int it = 0;
      if (b2 <= floor_ * floor_) {
        h->hctl->done = 1;
        h->hctl->status = 1;
        h->hctl->iter = 0;
      } else {
        h->hctl->tol2 = std::max(h->hctl->tol2, floor_ * floor_);
        CK(cudaMemcpyAsync(h->ctl, h->hctl, sizeof(KrylovCtl), cudaMemcpyHostToDevice, h->st));
        s = cg_loop(h, t, &it);
      }
      *cg_out += it;
      if (h->verbose)
        std::fprintf(stderr, "[rve]   cg iters %d status %d pAp %.3e rnorm2 %.3e b2 %.3e -> %d\n", it,
                     h->hctl->status, h->hctl->pAp, h->hctl->rnorm2, h->hctl->b2, s);
      if (s) return s;
      LAUNCHB(h, KC_MISC, g.nc * VV(h) * (16.0 + RS), Op::eps_update(g, h->lc, h->st, h->eps, (const R*)h->x, h->part));
      LAUNCHB(h, KC_FINALIZE, 0.0, k_finalize(h->st, h->fin, h->part, h->lc.n_ew_blocks, h->lc.max_blocks, 6, FIN_SUMS, nullptr,
                 h->dscal + OFF_EPSMEAN, 1.0 / (double)g.V));
      LAUNCHB(h, KC_FINALIZE, 0.0, k_finalize(h->st, h->fin, h->part + 6 * (size_t)h->lc.max_blocks, h->lc.n_ew_blocks, h->lc.max_blocks, 1,
                 FIN_MAXS, nullptr, h->dscal + OFF_MAXDX, 1.0));
      s = sync_read(h);
      if (s) return s;
      newton++;
      double em = 0.0;
      for (int c = 0; c < g.nc; c++) em += h->hscal[OFF_EPSMEAN + c] * h->hscal[OFF_EPSMEAN + c];
      de_rel = h->hscal[OFF_MAXDX] / std::max(std::sqrt(em), 1e-300);
    }
    *newton_out += newton;
    return RVE_OK;
  }

  // Forward transform of one real FP64 field into the 1-component spectrum out.
  static void forward1(rve* h, const Tables<R>& t, const double* f, C2<R>* out) {
    const int map0[6] = {0, 0, 0, 0, 0, 0};
    LAUNCHB(h, KC_X_FWD_FIELD, 1.0 * (8.0 * VV(h) + VS(h) * CS), Op::xfwd_field64(h->g, t, h->lc, h->st, f, 1, map0, nullptr, out));
    LAUNCHB(h, KC_Y_PASS, 2.0 * 1.0 * VS(h) * CS, Op::strided_plain(h->g, t, h->lc, h->st, out, 1, 1, -1, nullptr));
    if (h->g.d == 3) LAUNCHB(h, KC_Y_PASS, 2.0 * 1.0 * VS(h) * CS, Op::strided_plain(h->g, t, h->lc, h->st, out, 1, 2, -1, nullptr));
  }

  static void inverse1(rve* h, const Tables<R>& t, C2<R>* in, double* f) {
    if (h->g.d == 3) LAUNCHB(h, KC_Y_PASS, 2.0 * 1.0 * VS(h) * CS, Op::strided_plain(h->g, t, h->lc, h->st, in, 1, 2, +1, nullptr));
    LAUNCHB(h, KC_Y_PASS, 2.0 * 1.0 * VS(h) * CS, Op::strided_plain(h->g, t, h->lc, h->st, in, 1, 1, +1, nullptr));
    LAUNCHB(h, KC_X_INV_STORE, 1.0 * (VS(h) * CS + 8.0 * VV(h)), Op::xinv_store64(h->g, t, h->lc, h->st, in, 1, f));
  }

  // Helmholtz operator application on the spectrum (GC of Algorithm 2):
  // y = p + F(sum_j D_j^T (l^2 D_j F^-1 p)), the flux term applied in real
  // space, equal to p + conj(k).F(l^2 F^-1(k p)) (reading R15); the identity
  // stays exact in the spectrum.  The real fields q and the flux term sit in
  // the mechanical Ap buffer, idle during the solve.
  static void helm_matvec(rve* h, const Tables<R>& t, int j, C2<R>* pvec, const C2<R>* rsrc, C2<R>* y,
                          const KrylovCtl* ctl, int raw) {
    const Geo& g = h->g;
    C2<R>* W = (C2<R>*)h->S;
    R* q = (R*)h->Ap;
    R* Lq = q + g.V;
    LAUNCHB(h, KC_HELM_EXPAND, (raw ? 2.0 : 4.0) * VS(h) * CS, Op::helm_expand(g, t, h->lc, h->st, W, pvec, rsrc, h->ell2_mean[j], ctl, raw));
    if (g.d == 3) LAUNCHB(h, KC_Y_PASS, 2.0 * VS(h) * CS, Op::strided_plain(g, t, h->lc, h->st, W, 1, 1, +1, ctl));
    LAUNCHB(h, KC_HELM_X1, VS(h) * CS + VV(h) * RS, Op::xinv_storeR(g, t, h->lc, h->st, W, q, ctl));
    LAUNCHB(h, KC_HELM_STENCIL, VV(h) * (2.0 * RS + 1.0),
            Op::helm_stencil(g, h->lc, h->st, q, Lq, h->phase, (const R*)h->ell2R + j * kMaxPhases, ctl));
    LAUNCHB(h, KC_HELM_X1, VS(h) * CS + VV(h) * RS, Op::xfwd_fieldR(g, t, h->lc, h->st, Lq, W, ctl));
    if (g.d == 3) LAUNCHB(h, KC_Y_PASS, 2.0 * VS(h) * CS, Op::strided_plain(g, t, h->lc, h->st, W, 1, 1, -1, ctl));
    LAUNCHB(h, KC_HELM_CONTRACT, 3.0 * VS(h) * CS, Op::helm_contract(g, t, h->lc, h->st, W, raw ? rsrc : pvec, y, h->part, ctl));
  }

  // Algorithm 2 for variable j: abar = F^-1 PCG(GC, M, F(alpha)).
  static int helm_solve(rve* h, const Tables<R>& t, int j, const double* alpha_j, double* abar_out,
                        double rtol, int maxit, int* iters) {
    const Geo& g = h->g;
    C2<R>* hx = (C2<R>*)h->hx;
    C2<R>* hr = (C2<R>*)h->hr;
    C2<R>* hp = (C2<R>*)h->hp;
    C2<R>* hy = (C2<R>*)h->hy;
    forward1(h, t, alpha_j, hr);
    LAUNCHB(h, KC_PCG_UPDATE, 2.0 * VS(h) * CS, Op::pcg_init(g, t, h->lc, h->st, hx, hr, h->ell2_mean[j], h->part));
    LAUNCHB(h, KC_FINALIZE, 0.0, k_finalize(h->st, h->fin, h->part, h->lc.n_ew_blocks, h->lc.max_blocks, 2, FIN_PCG_INIT, h->ctl, nullptr,
               rtol * rtol, maxit, stall_window()));
    const int chunk = std::max(1, h->opt.check_every);
    const int nbl = Op::contract_blocks(g, h->lc);
    for (;;) {
      int s = run_chunk(h, &h->g_pcg[j], h->g_pcg_n[j], h->g_pcg_b[j], [&]() {
        for (int i = 0; i < chunk; i++) {
          helm_matvec(h, t, j, hp, hr, hy, h->ctl, 0);
          LAUNCHB(h, KC_FINALIZE, 0.0, k_finalize(h->st, h->fin, h->part, nbl, h->lc.max_blocks, 1, FIN_ALPHA, h->ctl, nullptr, 1.0));
          LAUNCHB(h, KC_PCG_UPDATE, 6.0 * VS(h) * CS, Op::pcg_update(g, t, h->lc, h->st, hx, hr, hp, hy, h->ell2_mean[j], h->part, h->ctl));
          LAUNCHB(h, KC_FINALIZE, 0.0, k_finalize(h->st, h->fin, h->part, h->lc.n_ew_blocks, h->lc.max_blocks, 2, FIN_PCG_BETA, h->ctl, nullptr, 1.0));
        }
      });
      if (s) return s;
      s = sync_read(h);
      if (s) return s;
      if (h->hctl->done) break;
    }
    *iters = h->hctl->iter;
    inverse1(h, t, hx, abar_out);
    if (h->hctl->status == 3) { h->fail_stage = 5; return RVE_ERR_NUMERIC; }
    if (h->hctl->status == 2) { h->fail_stage = 3; return RVE_ERR_NOT_CONVERGED; }
    return RVE_OK;
  }

  // One load increment (Algorithm 1) to target tg (null: the next target of
  // the load path); advance: count it as the load path's next increment.
  static int step(rve* h, rve_step_info* info, const double* tg_in = nullptr, bool advance = true) {
    const Geo& g = h->g;
    const Tables<R> t = tables<R>(h);
    const double sq2 = std::sqrt(2.0);
    const double W6[6] = {1, 1, 1, sq2, sq2, sq2};
    const double* tg = tg_in ? tg_in : &h->target[(size_t)h->n_done * 6];
    double dE[6] = {0, 0, 0, 0, 0, 0}, sbar[6] = {0, 0, 0, 0, 0, 0};
    for (int c = 0; c < g.nc; c++) {
      const int m = g.cmap[c];
      const double tm = tg[m] * W6[m], tp = h->E_prev[m] * W6[m];
      dE[c] = h->ctrl[m] ? tm - tp : 0.0;
      sbar[c] = h->ctrl[m] ? 0.0 : tm;
    }
    // initial guess (eps_n + dE on strain-controlled components; abar_n)
    h->ref_ok = false;
    LAUNCHB(h, KC_MISC, 16.0 * g.nc * VV(h), k_copy_add(h->st, g.V, g.nc, h->eps_conv, h->eps, dE));
    CK(cudaMemcpyAsync(h->abar_k, h->abar_n, sizeof(double) * h->J * g.V, cudaMemcpyDeviceToDevice, h->st));
    int stag = 0, newton = 0;
    long long cg = 0, pcg = 0;
    double err = 0.0;
    int status = RVE_OK;
    h->fail_stage = 0;
    for (;;) {
      CK(cudaMemcpyAsync(h->eps_prev, h->eps, sizeof(double) * g.nc * g.V, cudaMemcpyDeviceToDevice, h->st));
      status = mech_solve(h, t, h->abar_k, sbar, &newton, &cg);
      if (status) break;
      for (int j = 0; j < h->J; j++) {
        int it = 0;
        status = helm_solve(h, t, j, h->alpha + (size_t)j * g.V, h->abar_new + (size_t)j * g.V,
                            h->opt.pcg_rtol, h->opt.max_pcg, &it);
        pcg += it;
        if (h->verbose)
          std::fprintf(stderr, "[rve]   pcg j=%d iters %d status %d b2 %.3e -> %d\n", j, it, h->hctl->status,
                       h->hctl->b2, status);
        if (status) break;
      }
      if (status) break;
      LAUNCHB(h, KC_MISC, 16.0 * g.nc * VV(h), k_err_eps(g, h->lc, h->st, h->eps, h->eps_prev, h->part));
      LAUNCHB(h, KC_FINALIZE, 0.0, k_finalize(h->st, h->fin, h->part, h->lc.n_ew_blocks, h->lc.max_blocks, 6, FIN_SUMS, nullptr,
                 h->dscal + OFF_ERRMEAN, 1.0 / (double)g.V));
      LAUNCHB(h, KC_FINALIZE, 0.0, k_finalize(h->st, h->fin, h->part + 6 * (size_t)h->lc.max_blocks, h->lc.n_ew_blocks, h->lc.max_blocks, 1,
                 FIN_MAXS, nullptr, h->dscal + OFF_ERRMAX, 1.0));
      for (int j = 0; j < h->J; j++) {
        LAUNCHB(h, KC_MISC, 16.0 * VV(h), k_err_abar(g, h->lc, h->st, h->abar_new + (size_t)j * g.V, h->abar_k + (size_t)j * g.V, h->part));
        LAUNCHB(h, KC_FINALIZE, 0.0, k_finalize(h->st, h->fin, h->part, h->lc.n_ew_blocks, h->lc.max_blocks, 2, FIN_SUMS, nullptr,
                   h->dscal + OFF_ABAR + 2 * j, 1.0));
      }
      status = sync_read(h);
      if (status) break;
      double em = 0.0;
      for (int c = 0; c < g.nc; c++) em += h->hscal[OFF_ERRMEAN + c] * h->hscal[OFF_ERRMEAN + c];
      err = h->hscal[OFF_ERRMAX] / std::max(std::sqrt(em), 1e-300);
      for (int j = 0; j < h->J; j++) {
        const double an = std::sqrt(h->hscal[OFF_ABAR + 2 * j + 1]);
        if (an >= 1e-30) err = std::max(err, std::sqrt(h->hscal[OFF_ABAR + 2 * j]) / an);
      }
      if (h->verbose) std::fprintf(stderr, "[rve] staggered %d err %.3e\n", stag, err);
      if (!(err == err)) { h->fail_stage = 5; status = RVE_ERR_NUMERIC; break; }
      std::swap(h->abar_k, h->abar_new);
      stag++;
      if (stag >= h->opt.min_stag && err <= h->opt.tol_stag) break;
      if (stag >= h->opt.max_stag) { h->fail_stage = 4; status = RVE_ERR_NOT_CONVERGED; break; }
    }
    if (status) {
      // roll back to the last converged increment
      cudaMemcpyAsync(h->eps, h->eps_conv, sizeof(double) * g.nc * g.V, cudaMemcpyDeviceToDevice, h->st);
      cudaStreamSynchronize(h->st);
      if (info) {
        info->status = status;
        info->increment = h->n_done + 1;
        info->staggered_iters = stag;
        info->newton_iters = newton;
        info->cg_iters = cg;
        info->pcg_iters = pcg;
        info->err = err;
        info->fail_stage = h->fail_stage;
      }
      return status;
    }
    // commit
    CK(cudaMemcpyAsync(h->eps_conv, h->eps, sizeof(double) * g.nc * g.V, cudaMemcpyDeviceToDevice, h->st));
    std::swap(h->epsp_n, h->epsp);
    std::swap(h->ep_n, h->ep);
    std::swap(h->abar_n, h->abar_k);
    if (h->gtn) std::swap(h->f_n, h->f);
    CK(cudaStreamSynchronize(h->st));
    for (int c = 0; c < 6; c++) h->sig_mean[c] = h->hscal[OFF_SIGMEAN + c] / W6[c];
    for (int c = 0; c < 6; c++) h->eps_mean[c] = 0.0;
    for (int c = 0; c < g.nc; c++) h->eps_mean[g.cmap[c]] = h->hscal[OFF_ERRMEAN + c] / W6[g.cmap[c]];
    for (int c = 0; c < 6; c++) {
      if (h->ctrl[c]) h->E_prev[c] = tg[c];
      else h->S_prev[c] = tg[c];
    }
    h->D_mean = h->hscal[OFF_DMEAN];
    h->D_max = h->hscal[OFF_DMAX];
    if (advance) h->n_done++;
    if (info) {
      info->status = RVE_OK;
      info->increment = h->n_done;
      info->staggered_iters = stag;
      info->newton_iters = newton;
      info->cg_iters = cg;
      info->pcg_iters = pcg;
      info->err = err;
      info->voxel_iterations = (double)g.V * (double)(cg + pcg);
      for (int c = 0; c < 6; c++) {
        info->sigma[c] = h->sig_mean[c];
        info->eps[c] = h->eps_mean[c];
      }
      info->D_mean = h->D_mean;
      info->D_max = h->D_max;
    }
    return RVE_OK;
  }

  // -------------------------------------------------------- operator level
  static int op_apply_gamma(rve* h, const double* tau, double* out) {
    const Tables<R> t = tables<R>(h);
    int map[6] = {0, 1, 2, 3, 4, 5};
    LAUNCHB(h, KC_X_FWD_FIELD, (double)h->g.nc * (8.0 * VV(h) + VS(h) * CS), Op::xfwd_field64(h->g, t, h->lc, h->st, tau, h->g.nc, map, nullptr, (C2<R>*)h->S));
    gamma_sweep(h, t, 0, nullptr);
    LAUNCHB(h, KC_X_INV_STORE, (double)h->g.nc * (VS(h) * CS + 8.0 * VV(h)), Op::xinv_store64(h->g, t, h->lc, h->st, (const C2<R>*)h->S, h->g.nc, out));
    // reads the control block: a tile wait that ran out is RVE_ERR_TIMEOUT
    return sync_read(h);
  }

  static int op_matvec(rve* h, const double* p, double* Ap) {
    const Tables<R> t = tables<R>(h);
    const long long n = (long long)h->g.nc * h->g.V;
    LAUNCHB(h, KC_MISC, (double)n * (8.0 + RS), Op::to_r(h->st, n, p, (R*)h->p));
    LAUNCHB(h, KC_X_FWD_TANGENT, VV(h) * RS * (2.0 * h->g.nc + 2.0) + h->g.nc * VS(h) * CS, Op::xfwd_tangent(h->g, t, h->lc, h->st, (R*)h->p, nullptr, (const R*)h->desc, (C2<R>*)h->S, nullptr, nullptr, h->gtn));
    gamma_sweep(h, t, 0, nullptr);
    LAUNCHB(h, KC_X_INV_MATVEC, (double)h->g.nc * (VS(h) * CS + 2.0 * VV(h) * RS), Op::xinv_matvec(h->g, t, h->lc, h->st, (const C2<R>*)h->S, (R*)h->Ap, (const R*)h->p, h->part, nullptr));
    LAUNCHB(h, KC_MISC, (double)n * (8.0 + RS), Op::from_r(h->st, n, (const R*)h->Ap, Ap));
    CK(cudaStreamSynchronize(h->st));
    CK(cudaGetLastError());
    return RVE_OK;
  }

  static int op_cg(rve* h, const double* b, double* x, double rtol, int maxit, int* iters) {
    const Tables<R> t = tables<R>(h);
    const long long n = (long long)h->g.nc * h->g.V;
    LAUNCHB(h, KC_MISC, (double)n * (8.0 + RS), Op::to_r(h->st, n, b, (R*)h->r));
    LAUNCHB(h, KC_CG_UPDATE, 2.0 * h->g.nc * VV(h) * RS, Op::cg_init(h->g, h->lc, h->st, (R*)h->x, (const R*)h->r, h->part));
    LAUNCHB(h, KC_FINALIZE, 0.0, k_finalize(h->st, h->fin, h->part, h->lc.n_ew_blocks, h->lc.max_blocks, 1, FIN_CG_INIT, h->ctl, nullptr,
               rtol * rtol, maxit));
    int it = 0;
    int s = cg_loop(h, t, &it);
    if (iters) *iters = it;
    LAUNCHB(h, KC_MISC, (double)n * (8.0 + RS), Op::from_r(h->st, n, (const R*)h->x, x));
    CK(cudaStreamSynchronize(h->st));
    CK(cudaGetLastError());
    return s;
  }

  static int op_helm_apply(rve* h, int j, const double* a, double* out) {
    const Tables<R> t = tables<R>(h);
    forward1(h, t, a, (C2<R>*)h->hr);
    helm_matvec(h, t, j, (C2<R>*)h->hp, (const C2<R>*)h->hr, (C2<R>*)h->hy, nullptr, 1);
    inverse1(h, t, (C2<R>*)h->hy, out);
    CK(cudaStreamSynchronize(h->st));
    CK(cudaGetLastError());
    return RVE_OK;
  }

  static int op_helm_solve(rve* h, int j, const double* alpha, double* abar, double rtol, int maxit,
                           int* iters) {
    const Tables<R> t = tables<R>(h);
    int it = 0;
    int s = helm_solve(h, t, j, alpha, abar, rtol, maxit, &it);
    if (iters) *iters = it;
    CK(cudaStreamSynchronize(h->st));
    CK(cudaGetLastError());
    return s;
  }
};

// Twiddles exp(-2 pi i m / N) and half-angle tables sin/cos(pi q / N) (cos
// exactly 0 at the Nyquist index) of the three axes, from double precision.
template <typename R>
int build_tables(rve* h, void* tw[3], void* ts[3], void* tc[3]) {
  const int Ns[3] = {h->g.n1, h->g.n2, h->g.n3};
  for (int j = 0; j < 3; j++) {
    const int N = Ns[j];
    std::vector<C2<R>> twv(N);
    std::vector<R> sv(N), cv(N);
    for (int m = 0; m < N; m++) {
      const double ang = -2.0 * kPi * (double)m / (double)N;
      twv[m] = mk<R>((R)std::cos(ang), (R)std::sin(ang));
      const int q = m < (N + 1) / 2 ? m : m - N;
      const double half = kPi * (double)q / (double)N;
      sv[m] = (R)std::sin(half);
      cv[m] = (2 * std::abs(q) == N) ? R(0) : (R)std::cos(half);
    }
    int st;
    if ((st = dalloc(h, &tw[j], N * sizeof(C2<R>)))) return st;
    if ((st = dalloc(h, &ts[j], N * sizeof(R)))) return st;
    if ((st = dalloc(h, &tc[j], N * sizeof(R)))) return st;
    CK(cudaMemcpy(tw[j], twv.data(), N * sizeof(C2<R>), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ts[j], sv.data(), N * sizeof(R), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(tc[j], cv.data(), N * sizeof(R), cudaMemcpyHostToDevice));
  }
  return RVE_OK;
}

int upload_ell2(rve* h) {
  if (h->prec == RVE_MIXED) {
    std::vector<float> v(kMaxVars * kMaxPhases, 0.f);
    for (int j = 0; j < kMaxVars; j++)
      for (int q = 0; q < kMaxPhases; q++) v[j * kMaxPhases + q] = (float)h->pt_host.ell2[j][q];
    CK(cudaMemcpy(h->ell2R, v.data(), v.size() * sizeof(float), cudaMemcpyHostToDevice));
  } else {
    std::vector<double> v(kMaxVars * kMaxPhases, 0.0);
    for (int j = 0; j < kMaxVars; j++)
      for (int q = 0; q < kMaxPhases; q++) v[j * kMaxPhases + q] = h->pt_host.ell2[j][q];
    CK(cudaMemcpy(h->ell2R, v.data(), v.size() * sizeof(double), cudaMemcpyHostToDevice));
  }
  return RVE_OK;
}

int reset_state(rve* h) {
  const size_t V = (size_t)h->g.V, nc = h->g.nc;
  CK(cudaMemsetAsync(h->eps, 0, nc * V * 8, h->st));
  CK(cudaMemsetAsync(h->eps_conv, 0, nc * V * 8, h->st));
  CK(cudaMemsetAsync(h->eps_prev, 0, nc * V * 8, h->st));
  CK(cudaMemsetAsync(h->epsp_n, 0, 6 * V * 8, h->st));
  CK(cudaMemsetAsync(h->epsp, 0, 6 * V * 8, h->st));
  CK(cudaMemsetAsync(h->ep_n, 0, V * 8, h->st));
  CK(cudaMemsetAsync(h->ep, 0, V * 8, h->st));
  CK(cudaMemsetAsync(h->sigma, 0, 6 * V * 8, h->st));
  CK(cudaMemsetAsync(h->D, 0, V * 8, h->st));
  const size_t JV = (size_t)std::max(h->J, 1) * V * 8;
  CK(cudaMemsetAsync(h->alpha, 0, JV, h->st));
  CK(cudaMemsetAsync(h->abar_n, 0, JV, h->st));
  CK(cudaMemsetAsync(h->abar_k, 0, JV, h->st));
  CK(cudaMemsetAsync(h->abar_new, 0, JV, h->st));
  CK(cudaMemsetAsync(h->f, 0, V * 8, h->st));
  if (h->phases_set || h->gtn) k_fill_porosity(h->st, (long long)V, h->phase, h->pt_dev, h->f_n);
  else CK(cudaMemsetAsync(h->f_n, 0, V * 8, h->st));
  CK(cudaStreamSynchronize(h->st));
  CK(cudaGetLastError());
  h->n_done = 0;
  for (int c = 0; c < 6; c++) { h->E_prev[c] = 0; h->S_prev[c] = 0; h->sig_mean[c] = 0; h->eps_mean[c] = 0; }
  h->D_mean = h->D_max = 0;
  return RVE_OK;
}

void free_all(rve* h) {
  // tensor maps are cached by buffer address (the spectra of the projection pass)
  for (void* p : h->allocs) tensor_map_evict(p);
  for (void* p : h->allocs) cudaFree(p);
  h->allocs.clear();
  if (h->hctl) cudaFreeHost(h->hctl);
  if (h->hscal) cudaFreeHost(h->hscal);
  h->hctl = nullptr;
  h->hscal = nullptr;
}

int create_impl(rve** out, int dim, const int n[3], const double L[3], int precision, int J, void* stream) {
  if (!out || !n || !L) return RVE_ERR_ARG;
  *out = nullptr;
  if (dim != 2 && dim != 3) return RVE_ERR_ARG;
  if (precision != RVE_FP64 && precision != RVE_MIXED) return RVE_ERR_ARG;
  if (J < 0 || J > kMaxVars) return RVE_ERR_ARG;
  int nn[3] = {n[0], n[1], dim == 3 ? n[2] : 1};
  double LL[3] = {L[0], L[1], dim == 3 ? L[2] : 1.0};
  for (int j = 0; j < dim; j++)
    if (nn[j] < 1 || !(LL[j] > 0.0)) return RVE_ERR_ARG;
  if (nn[0] < 2 || nn[0] % 2) return RVE_ERR_ARG;
  const int ET = (precision == RVE_MIXED ? 8 : 4) * kThreads;
  // the FP64 Newton residual sweep runs in both forms
  if (std::max(nn[1], nn[2]) > 4 * kThreads) return RVE_ERR_ARG;
  const int nc = dim == 3 ? 6 : 3;
  if ((nn[0] / 2) * nc > 16 * kThreads) return RVE_ERR_ARG;
  FftPlan pl[3];
  if (!factor_plan(nn[0] / 2, pl[0]) || !factor_plan(nn[1], pl[1]) || !factor_plan(nn[2], pl[2]))
    return RVE_ERR_ARG;

  rve* h = new (std::nothrow) rve();
  if (!h) return RVE_ERR_OOM;
  h->dim = dim;
  h->prec = precision;
  h->J = J;
  for (int j = 0; j < 3; j++) { h->n[j] = nn[j]; h->L[j] = LL[j]; h->plan[j] = pl[j]; }
  h->st = (cudaStream_t)stream;
  rve_default_options(precision, &h->opt);
  {
    const char* v = std::getenv("RVE_VERBOSE");
    h->verbose = (v && v[0] >= '1' && v[0] <= '9') ? v[0] - '0' : 0;
  }

  Geo& g = h->g;
  g.d = dim;
  g.n1 = nn[0]; g.n2 = nn[1]; g.n3 = nn[2];
  g.M = nn[0] / 2;
  g.P1 = g.M + 1;
  // rows padded to 16 complex entries in both precisions (128 B / 256 B)
  g.ps = ((g.P1 + 15) / 16) * 16;
  g.nc = nc;
  const int cm3[6] = {0, 1, 2, 3, 4, 5}, cm2[6] = {0, 1, 5, 0, 0, 0};
  for (int c = 0; c < 6; c++) g.cmap[c] = dim == 3 ? cm3[c] : cm2[c];
  g.V = (long long)nn[0] * nn[1] * nn[2];
  g.nlines = (long long)nn[1] * nn[2];
  g.sstride = (long long)g.ps * nn[1] * nn[2];
  for (int j = 0; j < 3; j++) g.h[j] = LL[j] / nn[j];

  LaunchCfg& lc = h->lc;
  // x1 passes: 4 staged FFT elements per thread when a row of c components
  // fits (several CTAs per SM), 16 otherwise
  for (int c = 1; c <= 6; c++) {
    const int e = (c * g.M <= 4 * kThreads) ? 4 : 16;
    lc.xe_c[c] = e;
    lc.nrows_c[c] = (e == 4 && x1_ct_length(g.M)) ? x1_ct_rows(g.M, c)
                                                  : std::max(1, std::min(32, (e * kThreads) / (c * g.M)));
  }
  lc.nrows_c[0] = 1;
  lc.xe_c[0] = 16;
  const int nmax = std::max(nn[1], nn[2]);
  auto tx_for = [&](int et) {
    int tx = 1;
    while (tx * 2 * nmax <= et && tx * 2 <= 32) tx *= 2;
    return tx;
  };
  const int ET64 = 4 * kThreads;
  lc.tx = tx_for(ET);
  long long ew = (g.V + kThreads - 1) / kThreads;
  lc.n_ew_blocks = (int)std::min<long long>(ew, 152LL * 16);
  long long mb = lc.n_ew_blocks;
  for (int c = 1; c <= 6; c++) mb = std::max<long long>(mb, (g.nlines + lc.nrows_c[c] - 1) / lc.nrows_c[c]);
  const int tx64 = tx_for(ET64);
  mb = std::max<long long>(mb, (long long)((g.P1 + tx64 - 1) / tx64) * std::max(nn[1], 1));
  lc.max_blocks = (int)mb;
  lc.gamma_narrow = 0;
  h->lc64 = lc;
  h->lc64.tx = tx64;
  {
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
      cudaGetLastError();
      optin = 0;
    }
    const size_t need = precision == RVE_MIXED ? Ops<float>::xinv_cg_smem(g, lc) : Ops<double>::xinv_cg_smem(g, lc);
    h->cg_fused = need + 1024 <= (size_t)optin;
  }

  int s = RVE_OK;
  const size_t V = (size_t)g.V;
  const size_t JV = (size_t)std::max(J, 1) * V;
  const size_t rs = rsize(h);
  const size_t cs = 2 * rs;
#define AL(expr)                 \
  if ((s = (expr)) != RVE_OK) {  \
    free_all(h);                 \
    delete h;                    \
    return s;                    \
  }
  AL(dalloc_t(h, &h->phase, V));
  AL(dalloc_t(h, &h->eps, nc * V));
  AL(dalloc_t(h, &h->eps_conv, nc * V));
  AL(dalloc_t(h, &h->eps_prev, nc * V));
  AL(dalloc_t(h, &h->epsp_n, 6 * V));
  AL(dalloc_t(h, &h->epsp, 6 * V));
  AL(dalloc_t(h, &h->ep_n, V));
  AL(dalloc_t(h, &h->ep, V));
  AL(dalloc_t(h, &h->sigma, 6 * V));
  AL(dalloc_t(h, &h->D, V));
  AL(dalloc_t(h, &h->alpha, JV));
  AL(dalloc_t(h, &h->abar_n, JV));
  AL(dalloc_t(h, &h->abar_k, JV));
  AL(dalloc_t(h, &h->abar_new, JV));
  AL(dalloc(h, &h->x, nc * V * rs));
  AL(dalloc(h, &h->r, nc * V * rs));
  AL(dalloc(h, &h->p, nc * V * rs));
  AL(dalloc(h, &h->Ap, nc * V * rs));
  // tangent descriptor: c1, c2, m (2 + nc rows) or A, B, C, D, nh (4 + nc)
  AL(dalloc(h, &h->desc, (4 + nc) * V * rs));
  AL(dalloc_t(h, &h->f_n, V));
  AL(dalloc_t(h, &h->f, V));
  AL(dalloc(h, &h->S, (size_t)nc * g.sstride * cs));
  AL(dalloc(h, &h->hx, (size_t)g.sstride * cs));
  AL(dalloc(h, &h->hr, (size_t)g.sstride * cs));
  AL(dalloc(h, &h->hp, (size_t)g.sstride * cs));
  AL(dalloc(h, &h->hy, (size_t)g.sstride * cs));
  AL(dalloc(h, &h->ell2R, kMaxVars * kMaxPhases * rs));
  AL(dalloc_t(h, &h->pt_dev, 1));
  AL(dalloc_t(h, &h->part, (size_t)kSlots * lc.max_blocks));
  AL(dalloc_t(h, &h->ctl, 1));
  AL(dalloc_t(h, &h->fin, 1));
  if (cudaMemset(h->ctl, 0, sizeof(KrylovCtl)) != cudaSuccess ||
      cudaMemset(h->fin, 0, sizeof(FinScratch)) != cudaSuccess) {
    cudaGetLastError();
    free_all(h);
    delete h;
    return RVE_ERR_CUDA;
  }
  AL(dalloc_t(h, &h->dscal, kScal));
  AL(build_tables<double>(h, h->tw64, h->ts64, h->tc64));
  if (precision == RVE_MIXED) {
    AL(build_tables<float>(h, h->tw, h->ts, h->tc));
    AL(dalloc(h, &h->S64, (size_t)nc * g.sstride * 16));
    AL(dalloc_t(h, &h->sig_ref, 6 * V));
    AL(dalloc(h, &h->r_ref, (size_t)nc * V * sizeof(float)));
  } else {
    for (int j = 0; j < 3; j++) { h->tw[j] = h->tw64[j]; h->ts[j] = h->ts64[j]; h->tc[j] = h->tc64[j]; }
    h->S64 = h->S;
  }
#undef AL
  if (cudaMallocHost((void**)&h->hctl, sizeof(KrylovCtl)) != cudaSuccess ||
      cudaMallocHost((void**)&h->hscal, kScal * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    free_all(h);
    delete h;
    return RVE_ERR_OOM;
  }
  // a (spectral) buffer that is never written in the padding stays defined
  cudaMemset(h->S, 0, (size_t)nc * g.sstride * cs);
  if (h->S64 != h->S) cudaMemset(h->S64, 0, (size_t)nc * g.sstride * 16);
  cudaMemset(h->hx, 0, (size_t)g.sstride * cs);
  cudaMemset(h->hr, 0, (size_t)g.sstride * cs);
  cudaMemset(h->hp, 0, (size_t)g.sstride * cs);
  cudaMemset(h->hy, 0, (size_t)g.sstride * cs);
  cudaMemset(h->dscal, 0, kScal * sizeof(double));
  cudaMemset(h->ctl, 0, sizeof(KrylovCtl));
  if (cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    free_all(h);
    delete h;
    return RVE_ERR_CUDA;
  }
  // default load path: pure strain control (operator-level calls)
  for (int c = 0; c < 6; c++) { h->smask_d[c] = 0.0; h->smask_f[c] = 0.f; }
  if ((s = reset_state(h)) != RVE_OK) {
    free_all(h);
    delete h;
    return s;
  }
  *out = h;
  return RVE_OK;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

// ====================================================================== C ABI
extern "C" {

int rve_profile(rve_t* h, int enable) {
  if (!h) return RVE_ERR_ARG;
  if (h->prof && !enable) {
    cudaStreamSynchronize(h->st);
    prof_resolve(h);
  }
  h->prof = enable != 0;
  return RVE_OK;
}

int rve_profile_read(rve_t* h, int n, double* ms, long long* launches, double* bytes) {
  if (!h || n < 0) return RVE_ERR_ARG;
  CK(cudaStreamSynchronize(h->st));
  prof_resolve(h);
  const int m = std::min(n, (int)KC_COUNT);
  for (int k = 0; k < m; k++) {
    if (ms) ms[k] = h->prof_ms[k];
    if (launches) launches[k] = h->launches[k];
    if (bytes) bytes[k] = h->prof_bytes[k];
  }
  return KC_COUNT;
}

int rve_profile_reset(rve_t* h) {
  if (!h) return RVE_ERR_ARG;
  cudaStreamSynchronize(h->st);
  prof_resolve(h);
  for (int k = 0; k < KC_COUNT; k++) { h->prof_ms[k] = 0.0; h->launches[k] = 0; h->prof_bytes[k] = 0.0; }
  return RVE_OK;
}

const char* rve_profile_class_name(int k) { return (k >= 0 && k < KC_COUNT) ? kClassNames[k] : nullptr; }

const char* rve_status_string(int s) {
  switch (s) {
    case RVE_OK: return "ok";
    case RVE_ERR_ARG: return "invalid argument";
    case RVE_ERR_STATE: return "call out of order";
    case RVE_ERR_CUDA: return "CUDA runtime error";
    case RVE_ERR_OOM: return "out of device memory";
    case RVE_ERR_NOT_CONVERGED: return "iteration budget exhausted";
    case RVE_ERR_NUMERIC: return "non-finite value or Krylov breakdown";
    case RVE_ERR_LOAD_PATH_END: return "load path finished";
    case RVE_ERR_TIMEOUT: return "device wait for a tile copy timed out";
    default: return "unknown status";
  }
}

int rve_default_options(int precision, rve_solver_options* o) {
  if (!o) return RVE_ERR_ARG;
  o->tol_stag = 1e-6;
  o->tol_newton = 1e-6;
  // the mixed form solves each Newton correction inexactly in FP32 and lets
  // the FP64 residual drive the outer convergence (iterative refinement)
  o->cg_rtol = precision == RVE_MIXED ? 1e-3 : 1e-8;
  // the FP32 PCG's recursive residual keeps falling below what FP32 vectors
  // can represent (unit round-off 6e-8); iterations past 1e-7 would not make
  // the non-local field more accurate
  o->pcg_rtol = precision == RVE_MIXED ? 1e-7 : 1e-8;
  o->max_stag = 50;
  o->max_newton = 30;
  o->max_cg = 2000;
  o->max_pcg = 2000;
  o->min_stag = 2;
  o->check_every = 8;
  return RVE_OK;
}

int rve_create(rve_t** out, int dim, const int n[3], const double L[3], int precision, int n_nonlocal,
               void* cuda_stream) {
  try {
    return create_impl(out, dim, n, L, precision, n_nonlocal, cuda_stream);
  } catch (...) {
    return RVE_ERR_OOM;
  }
}

void adjoint_free(rve* h);

void rve_free(rve_t* h) {
  if (!h) return;
  cudaStreamSynchronize(h->st);
  graphs_reset(h);
  adjoint_free(h);
  if (h->stiff) cudaFree(h->stiff);
  h->stiff = nullptr;
  prof_resolve(h);
  for (cudaEvent_t e : h->ev_free) cudaEventDestroy(e);
  h->ev_free.clear();
  free_all(h);
  delete h;
}

int rve_set_options(rve_t* h, const rve_solver_options* o) {
  if (!h || !o) return RVE_ERR_ARG;
  if (!(o->tol_stag > 0) || !(o->tol_newton > 0) || !(o->cg_rtol > 0) || !(o->pcg_rtol > 0)) return RVE_ERR_ARG;
  if (o->max_stag < 1 || o->max_newton < 0 || o->max_cg < 1 || o->max_pcg < 1 || o->min_stag < 1 ||
      o->check_every < 1)
    return RVE_ERR_ARG;
  h->opt = *o;
  graphs_reset(h);
  return RVE_OK;
}

int rve_set_phases(rve_t* h, const uint8_t* phase, int n_phases, const rve_phase_params* params,
                   const double* ell) {
  if (!h || !phase || !params) return RVE_ERR_ARG;
  if (n_phases < 1 || n_phases > kMaxPhases) return RVE_ERR_ARG;
  if (h->J > 0 && !ell) return RVE_ERR_ARG;
  const size_t V = (size_t)h->g.V;
  std::vector<uint8_t> hp;
  try {
    hp.resize(V);
  } catch (...) {
    return RVE_ERR_OOM;
  }
  if (is_device_ptr(phase)) {
    CK(cudaMemcpy(hp.data(), phase, V, cudaMemcpyDeviceToHost));
  } else {
    std::memcpy(hp.data(), phase, V);
  }
  std::vector<long long> count(n_phases, 0);
  for (size_t v = 0; v < V; v++) {
    if (hp[v] >= n_phases) return RVE_ERR_ARG;
    count[hp[v]]++;
  }
  PhaseTable pt{};
  pt.n_phases = n_phases;
  bool gtn = false;
  for (int q = 0; q < n_phases; q++) {
    const rve_phase_params& P = params[q];
    if (!(P.E > 0.0) || !(P.nu > -1.0 && P.nu < 0.5)) return RVE_ERR_ARG;
    if (P.damage_law < 0 || P.damage_law > 3) return RVE_ERR_ARG;
    if (P.nonlocal_var < -1 || P.nonlocal_var >= h->J) return RVE_ERR_ARG;
    const bool plastic = P.damage_law == 1 || P.damage_law == 3;
    if (plastic && (!(P.sigma_y > 0.0) || !(P.H >= 0.0))) return RVE_ERR_ARG;
    if (P.hardening < 0 || P.hardening > 1 || P.reserved != 0) return RVE_ERR_ARG;
    if (plastic && P.hardening == 1 && !(P.N > 0.0 && P.N < 1.0)) return RVE_ERR_ARG;
    if ((P.damage_law == 1 || P.damage_law == 2) && P.nonlocal_var >= 0 &&
        (!(P.eps_R > P.eps_C) || !(P.D_max >= 0.0 && P.D_max < 1.0)))
      return RVE_ERR_ARG;
    if (P.damage_law == 3) {
      // two non-local variables (eps_0^p, tr eps^p) at nonlocal_var, +1
      if (P.nonlocal_var < 0 || P.nonlocal_var + 1 >= h->J) return RVE_ERR_ARG;
      if (!(P.q1 > 0.0) || !(P.q2 > 0.0) || !(P.q3 > 0.0) || !(P.q1 * P.q1 >= P.q3)) return RVE_ERR_ARG;
      const double fV = (P.q1 + std::sqrt(P.q1 * P.q1 - P.q3)) / P.q3;
      if (!(P.f_C >= 0.0) || !(P.f_F > P.f_C) || !(P.f_F < 1.0)) return RVE_ERR_ARG;
      if (!(P.f_N >= 0.0) || !(P.s_N > 0.0) || !(P.f_0 >= 0.0 && P.f_0 < 1.0)) return RVE_ERR_ARG;
      if (!(P.fstar_max > 0.0 && P.fstar_max < fV)) return RVE_ERR_ARG;
    }
    PhaseDev& d = pt.p[q];
    d.K = P.E / (3.0 * (1.0 - 2.0 * P.nu));
    d.mu = P.E / (2.0 * (1.0 + P.nu));
    d.sigma_y = P.sigma_y;
    d.H = P.H;
    d.eps_C = P.eps_C;
    d.eps_R = P.eps_R;
    d.D_max = P.D_max;
    d.inv_dCR = P.eps_R > P.eps_C ? 1.0 / (P.eps_R - P.eps_C) : 0.0;
    d.law = P.damage_law;
    d.var = P.damage_law != 0 ? P.nonlocal_var : -1;
    d.hard = (P.damage_law == 1 || P.damage_law == 3) ? P.hardening : 0;
    d.pad_ = 0;
    d.N = P.N;
    d.c_hard = P.sigma_y > 0.0 ? 3.0 * d.mu / P.sigma_y : 0.0;
    d.q1 = P.q1; d.q2 = P.q2; d.q3 = P.q3;
    d.f_C = P.f_C; d.f_F = P.f_F;
    d.fV = P.q3 > 0.0 && P.q1 * P.q1 >= P.q3 ? (P.q1 + std::sqrt(P.q1 * P.q1 - P.q3)) / P.q3 : 0.0;
    d.f_N = P.f_N; d.eps_N = P.eps_N; d.s_N = P.s_N;
    d.f0 = P.f_0; d.fstar_max = P.fstar_max;
    if (P.damage_law == 3) gtn = true;
  }
  for (int j = 0; j < h->J; j++) {
    double m = 0.0;
    for (int q = 0; q < n_phases; q++) {
      const double l = ell[j * n_phases + q];
      if (!(l >= 0.0)) return RVE_ERR_ARG;
      pt.ell2[j][q] = l * l;
      pt.ell2f[j][q] = (float)(l * l);
      m += (double)count[q] * l * l;
    }
    h->ell2_mean[j] = m / (double)V;
  }
  h->pt_host = pt;
  h->n_phases = n_phases;
  h->gtn = gtn;
  CK(cudaMemcpy(h->phase, hp.data(), V, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(h->pt_dev, &pt, sizeof(PhaseTable), cudaMemcpyHostToDevice));
  int s = upload_ell2(h);
  if (s) return s;
  s = reset_state(h);
  if (s) return s;
  h->phases_set = true;
  h->stepped = false;
  graphs_reset(h);
  return RVE_OK;
}

int rve_set_load_path(rve_t* h, int n_incr, const uint8_t strain_ctrl[6], const double* target) {
  if (!h || !strain_ctrl || !target || n_incr < 1) return RVE_ERR_ARG;
  for (int c = 0; c < 6; c++)
    if (strain_ctrl[c] > 1) return RVE_ERR_ARG;
  if (h->dim == 2) {
    for (int c = 2; c <= 4; c++) {
      if (!strain_ctrl[c]) return RVE_ERR_ARG;
      for (int i = 0; i < n_incr; i++)
        if (target[i * 6 + c] != 0.0) return RVE_ERR_ARG;
    }
  }
  for (int i = 0; i < 6 * n_incr; i++)
    if (!std::isfinite(target[i])) return RVE_ERR_ARG;
  h->target.assign(target, target + 6 * (size_t)n_incr);
  h->n_incr = n_incr;
  h->n_done = 0;
  for (int c = 0; c < 6; c++) h->ctrl[c] = strain_ctrl[c];
  for (int c = 0; c < 6; c++) {
    const double m = (c < h->g.nc) ? (strain_ctrl[h->g.cmap[c]] ? 0.0 : 1.0) : 0.0;
    h->smask_d[c] = m;
    h->smask_f[c] = (float)m;
  }
  h->path_set = true;
  graphs_reset(h);
  return RVE_OK;
}

int rve_step_increment(rve_t* h, rve_step_info* info) {
  if (!h) return RVE_ERR_ARG;
  if (info) std::memset(info, 0, sizeof(*info));
  if (!h->phases_set || !h->path_set) return RVE_ERR_STATE;
  if (h->n_done >= h->n_incr) return RVE_ERR_LOAD_PATH_END;
  h->stepped = true;
  try {
    return h->prec == RVE_MIXED ? Alg<float>::step(h, info) : Alg<double>::step(h, info);
  } catch (...) {
    return RVE_ERR_OOM;
  }
}

int rve_step_increment_adaptive(rve_t* h, int max_cuts, rve_step_info* info) {
  if (!h || max_cuts < 0 || max_cuts > 60) return RVE_ERR_ARG;
  if (info) std::memset(info, 0, sizeof(*info));
  if (!h->phases_set || !h->path_set) return RVE_ERR_STATE;
  if (h->n_done >= h->n_incr) return RVE_ERR_LOAD_PATH_END;
  h->stepped = true;
  // the remaining path of this increment: from the last converged
  // (sub-)step's targets T0 to the increment's target T1
  const double* T1 = &h->target[(size_t)h->n_done * 6];
  double T0[6];
  for (int c = 0; c < 6; c++) T0[c] = h->ctrl[c] ? h->E_prev[c] : h->S_prev[c];
  const double min_step = std::ldexp(1.0, -max_cuts);
  double f = 0.0, step = 1.0;
  int subs = 0;
  rve_step_info acc{}, sub{};
  int s = RVE_OK;
  try {
    while (f < 1.0) {
      const double fn = std::min(1.0, f + step);
      double T[6];
      for (int c = 0; c < 6; c++) T[c] = fn >= 1.0 ? T1[c] : T0[c] + fn * (T1[c] - T0[c]);
      s = h->prec == RVE_MIXED ? Alg<float>::step(h, &sub, T, fn >= 1.0) : Alg<double>::step(h, &sub, T, fn >= 1.0);
      acc.staggered_iters += sub.staggered_iters;
      acc.newton_iters += sub.newton_iters;
      acc.cg_iters += sub.cg_iters;
      acc.pcg_iters += sub.pcg_iters;
      acc.voxel_iterations += (double)h->g.V * (double)(sub.cg_iters + sub.pcg_iters);
      if (s == RVE_OK) {
        f = fn;
        subs++;
        step *= 2.0;   // grow back after a success (the next try is capped at the rest)
      } else if (s == RVE_ERR_NOT_CONVERGED && step * 0.5 >= min_step) {
        step *= 0.5;   // the state is at the last converged sub-step
      } else {
        break;
      }
    }
  } catch (...) {
    s = RVE_ERR_OOM;
  }
  if (info) {
    *info = sub;   // the last sub-step (on failure: the attempt that failed)
    if (s != RVE_OK) {
      for (int c = 0; c < 6; c++) {
        info->sigma[c] = h->sig_mean[c];
        info->eps[c] = h->eps_mean[c];
      }
      info->D_mean = h->D_mean;
      info->D_max = h->D_max;
    }
    info->status = s;
    info->increment = s == RVE_OK ? h->n_done : h->n_done + 1;
    info->staggered_iters = acc.staggered_iters;
    info->newton_iters = acc.newton_iters;
    info->cg_iters = acc.cg_iters;
    info->pcg_iters = acc.pcg_iters;
    info->voxel_iterations = acc.voxel_iterations;
    info->reserved = subs;
  }
  return s;
}

int rve_homogenized_stress(const rve_t* h, double sigma[6]) {
  if (!h || !sigma) return RVE_ERR_ARG;
  for (int c = 0; c < 6; c++) sigma[c] = h->sig_mean[c];
  return RVE_OK;
}

int rve_homogenized_strain(const rve_t* h, double eps[6]) {
  if (!h || !eps) return RVE_ERR_ARG;
  for (int c = 0; c < 6; c++) eps[c] = h->eps_mean[c];
  return RVE_OK;
}

int rve_get_sizes(const rve_t* h, long long* nv, int* nc, int* J) {
  if (!h) return RVE_ERR_ARG;
  if (nv) *nv = h->g.V;
  if (nc) *nc = h->g.nc;
  if (J) *J = h->J;
  return RVE_OK;
}

int rve_get_field(const rve_t* h, int which, double* dst, size_t n) {
  if (!h || !dst) return RVE_ERR_ARG;
  const size_t V = (size_t)h->g.V;
  const double* src = nullptr;
  size_t cnt = 0;
  switch (which) {
    case 0: src = h->eps_conv; cnt = h->g.nc * V; break;
    case 1: src = h->sigma; cnt = 6 * V; break;
    case 2: src = h->D; cnt = V; break;
    case 3: src = h->abar_n; cnt = (size_t)h->J * V; break;
    case 4: src = h->ep_n; cnt = V; break;
    case 5: src = h->epsp_n; cnt = 6 * V; break;
    case 6: src = h->f_n; cnt = V; break;
    default: return RVE_ERR_ARG;
  }
  if (n < cnt) return RVE_ERR_ARG;
  if (cnt == 0) return RVE_OK;
  // dst may be device or host memory (the copy kind follows the address)
  CK(cudaMemcpyAsync(dst, src, cnt * sizeof(double), cudaMemcpyDefault, h->st));
  CK(cudaStreamSynchronize(h->st));
  return RVE_OK;
}

int rve_op_return_map(rve_t* h, const double* eps, const double* epsp_n, const double* ep_n,
                      const double* abar, double* sigma, double* epsp, double* ep, double* D,
                      double* alpha) {
  if (!h || !eps || !epsp_n || !ep_n || !sigma || !epsp || !ep || !D) return RVE_ERR_ARG;
  if (h->J > 0 && (!abar || !alpha)) return RVE_ERR_ARG;
  if (!h->phases_set) return RVE_ERR_STATE;
  return rve_op_return_map_ex(h, eps, epsp_n, ep_n, abar, nullptr, nullptr, sigma, epsp, ep, D, alpha, nullptr);
}

int rve_op_return_map_ex(rve_t* h, const double* eps, const double* epsp_n, const double* ep_n,
                         const double* abar, const double* abar_n, const double* f_n, double* sigma,
                         double* epsp, double* ep, double* D, double* alpha, double* f) {
  if (!h || !eps || !epsp_n || !ep_n || !sigma || !epsp || !ep || !D) return RVE_ERR_ARG;
  if (h->J > 0 && (!abar || !alpha)) return RVE_ERR_ARG;
  if (!h->phases_set) return RVE_ERR_STATE;
  double* alpha_use = alpha ? alpha : h->alpha;
  const double* abar_use = abar ? abar : h->abar_n;
  const double* abar_n_use = abar_n ? abar_n : h->abar_n;
  const double* f_n_use = f_n ? f_n : h->f_n;
  double* f_use = f ? f : h->f;
  if (h->prec == RVE_MIXED)
    Ops<float>::return_map(h->g, h->lc, h->st, h->pt_dev, h->J, h->phase, eps, epsp_n, ep_n, abar_use, sigma,
                           epsp, ep, D, alpha_use, (float*)h->desc, h->part, h->stiff, abar_n_use, f_n_use,
                           f_use, h->gtn);
  else
    Ops<double>::return_map(h->g, h->lc, h->st, h->pt_dev, h->J, h->phase, eps, epsp_n, ep_n, abar_use,
                            sigma, epsp, ep, D, alpha_use, (double*)h->desc, h->part, h->stiff, abar_n_use,
                            f_n_use, f_use, h->gtn);
  CK(cudaStreamSynchronize(h->st));
  CK(cudaGetLastError());
  return RVE_OK;
}

int rve_op_tangent_apply(rve_t* h, const double* p, double* tau) {
  if (!h || !p || !tau) return RVE_ERR_ARG;
  if (h->prec == RVE_MIXED)
    Ops<float>::tangent_apply64(h->g, h->lc, h->st, (const float*)h->desc, p, tau, h->gtn);
  else
    Ops<double>::tangent_apply64(h->g, h->lc, h->st, (const double*)h->desc, p, tau, h->gtn);
  CK(cudaStreamSynchronize(h->st));
  CK(cudaGetLastError());
  return RVE_OK;
}

int rve_op_apply_gamma(rve_t* h, const double* tau, double* out) {
  if (!h || !tau || !out) return RVE_ERR_ARG;
  return h->prec == RVE_MIXED ? Alg<float>::op_apply_gamma(h, tau, out) : Alg<double>::op_apply_gamma(h, tau, out);
}

int rve_test_tile_wait(rve_t* h, double wait_s, int extra_tx_bytes) {
  if (!h || !(wait_s > 0.0 && wait_s <= 60.0) || extra_tx_bytes < 0 || extra_tx_bytes > 4096) return RVE_ERR_ARG;
  h->tile_wait_s = wait_s;
  h->tile_extra_tx = extra_tx_bytes;
  graphs_reset(h);
  return RVE_OK;
}

int rve_op_matvec(rve_t* h, const double* p, double* Ap) {
  if (!h || !p || !Ap) return RVE_ERR_ARG;
  return h->prec == RVE_MIXED ? Alg<float>::op_matvec(h, p, Ap) : Alg<double>::op_matvec(h, p, Ap);
}

int rve_op_cg(rve_t* h, const double* b, double* x, double rtol, int maxit, int* iters) {
  if (!h || !b || !x || !(rtol > 0) || maxit < 1) return RVE_ERR_ARG;
  return h->prec == RVE_MIXED ? Alg<float>::op_cg(h, b, x, rtol, maxit, iters)
                              : Alg<double>::op_cg(h, b, x, rtol, maxit, iters);
}

int rve_op_helmholtz_apply(rve_t* h, int j, const double* a, double* out) {
  if (!h || !a || !out || j < 0 || j >= h->J) return RVE_ERR_ARG;
  if (!h->phases_set) return RVE_ERR_STATE;
  return h->prec == RVE_MIXED ? Alg<float>::op_helm_apply(h, j, a, out) : Alg<double>::op_helm_apply(h, j, a, out);
}

int rve_op_helmholtz_solve(rve_t* h, int j, const double* alpha, double* abar, double rtol, int maxit,
                           int* iters) {
  if (!h || !alpha || !abar || j < 0 || j >= h->J || !(rtol > 0) || maxit < 1) return RVE_ERR_ARG;
  if (!h->phases_set) return RVE_ERR_STATE;
  return h->prec == RVE_MIXED ? Alg<float>::op_helm_solve(h, j, alpha, abar, rtol, maxit, iters)
                              : Alg<double>::op_helm_solve(h, j, alpha, abar, rtol, maxit, iters);
}

}  // extern "C"

// ============================================================ graphs, autotuning, batches
int rve_set_gamma_tile(rve_t* h, int narrow) {
  if (!h || narrow < 0 || narrow > 1) return RVE_ERR_ARG;
  if (cudaStreamSynchronize(h->st) != cudaSuccess) return RVE_ERR_CUDA;
  graphs_reset(h);
  h->lc.gamma_narrow = narrow;
  return RVE_OK;
}

int rve_get_gamma_tile(const rve_t* h, int* narrow) {
  if (!h || !narrow) return RVE_ERR_ARG;
  *narrow = h->lc.gamma_narrow;
  return RVE_OK;
}

int rve_set_graphs(rve_t* h, int enable) {
  if (!h) return RVE_ERR_ARG;
  if (cudaStreamSynchronize(h->st) != cudaSuccess) return RVE_ERR_CUDA;
  graphs_reset(h);
  h->graphs = enable != 0;
  return RVE_OK;
}

namespace {

// ordered factorisations of N into the radices of the runtime FFT with the
// fewest stages (at most 12)
void radix_orders(int N, std::vector<FftPlan>& out) {
  const int rad[5] = {8, 5, 4, 3, 2};
  std::vector<std::vector<int>> found;
  std::vector<int> cur;
  size_t best = 100;
  std::function<void(int)> rec = [&](int m) {
    if (cur.size() > best || found.size() >= 64) return;
    if (m == 1) {
      if (cur.size() < best) { best = cur.size(); found.clear(); }
      found.push_back(cur);
      return;
    }
    if ((int)cur.size() >= kMaxRadixStages) return;
    for (int r : rad)
      if (m % r == 0) {
        cur.push_back(r);
        rec(m / r);
        cur.pop_back();
      }
  };
  rec(N);
  for (const auto& f : found) {
    if (f.size() != best) continue;
    FftPlan pl{};
    pl.N = N;
    pl.nst = (int)f.size();
    for (size_t i = 0; i < f.size(); i++) pl.radix[i] = f[i];
    out.push_back(pl);
    if (out.size() >= 12) break;
  }
}

// mean time of `reps` mechanical matvecs G*(C_T : p) with the handle's
// current launch shape and plans (Krylov scratch only; state untouched)
template <typename R>
double time_matvec(rve* h, int reps) {
  const Geo& g = h->g;
  const Tables<R> t = tables<R>(h);
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess) return 1e30;
  if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy(a); return 1e30; }
  auto once = [&]() {
    Ops<R>::xfwd_tangent(g, t, h->lc, h->st, (R*)h->p, (const R*)h->r, (const R*)h->desc, (C2<R>*)h->S, nullptr,
                         nullptr, h->gtn);
    Alg<R>::gamma_sweep(h, t, 0, nullptr);
    Ops<R>::xinv_matvec(g, t, h->lc, h->st, (const C2<R>*)h->S, (R*)h->Ap, (const R*)h->p, h->part, nullptr);
  };
  once();
  cudaEventRecord(a, h->st);
  for (int i = 0; i < reps; i++) once();
  cudaEventRecord(b, h->st);
  float ms = 1e30f;
  if (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&ms, a, b) != cudaSuccess) ms = 1e30f;
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaGetLastError();
  return ms / reps;
}

template <typename R>
int autotune_impl(rve* h, int reps, double* best_ms) {
  const Geo& g = h->g;
  const bool prof = h->prof;
  h->prof = false;
  long long n0[KC_COUNT];
  double b0[KC_COUNT];
  std::memcpy(n0, h->launches, sizeof(n0));
  std::memcpy(b0, h->prof_bytes, sizeof(b0));
  // the timed matvecs read r and the tangent descriptor as they are and
  // overwrite only the Krylov scratch (p, spectrum, Ap, partial sums)
  int s = RVE_OK;
  double best = time_matvec<R>(h, reps);
  // plan of each axis whose transforms run on the runtime mixed-radix path
  for (int ax = 0; ax < g.d && !s; ax++) {
    const int N = h->plan[ax].N;
    if (N <= 1 || (ax == 0 && x1_ct_length(N)) || (ax > 0 && reg_axis(N))) continue;
    std::vector<FftPlan> cands;
    radix_orders(N, cands);
    FftPlan keep = h->plan[ax];
    for (const FftPlan& pl : cands) {
      h->plan[ax] = pl;
      const double ms = time_matvec<R>(h, reps);
      if (ms < best * 0.98) { best = ms; keep = pl; }
    }
    h->plan[ax] = keep;
  }
  // tile width of the runtime strided passes (its partial-sum rows must fit)
  if (!s) {
    const int nmax = std::max(g.n2, g.n3);
    const int ET = (int)(sizeof(R) == 4 ? 8 : 4) * kThreads;
    const int keep0 = h->lc.tx;
    int keep = keep0;
    for (int tx = 1; tx <= 32; tx *= 2) {
      if (tx == keep0 || tx * nmax > ET) continue;
      const size_t smem = (size_t)nmax * sizeof(C2<R>) * (g.nc * tx + 1) + 16;
      if (smem > 200 * 1024) continue;
      const long long rows = (long long)((g.P1 + tx - 1) / tx) * (g.d == 3 ? g.n2 : 1);
      if (rows > h->lc.max_blocks) continue;
      h->lc.tx = tx;
      const double ms = time_matvec<R>(h, reps);
      if (ms < best * 0.98) { best = ms; keep = tx; }
    }
    h->lc.tx = keep;
  }
  // width of the 3D six-component last-axis TMA tile
  if (!s && g.d == 3 && g.nc == 6 && reg_axis(g.n3)) {
    const int keep0 = h->lc.gamma_narrow;
    h->lc.gamma_narrow = 1 - keep0;
    const double ms = time_matvec<R>(h, reps);
    if (ms < best * 0.98) best = ms;
    else h->lc.gamma_narrow = keep0;
  }
  std::memcpy(h->launches, n0, sizeof(n0));
  std::memcpy(h->prof_bytes, b0, sizeof(b0));
  h->prof = prof;
  graphs_reset(h);
  if (best_ms) *best_ms = best;
  if (cudaStreamSynchronize(h->st) != cudaSuccess) return RVE_ERR_CUDA;
  return s;
}

}  // namespace

int rve_autotune(rve_t* h, int reps, double* best_ms, int* tx, int radix[3][8]) {
  if (!h || reps < 1) return RVE_ERR_ARG;
  if (!h->phases_set || h->stepped) return RVE_ERR_STATE;
  int s;
  try {
    s = h->prec == RVE_MIXED ? autotune_impl<float>(h, reps, best_ms) : autotune_impl<double>(h, reps, best_ms);
  } catch (...) {
    return RVE_ERR_OOM;
  }
  if (s) return s;
  if (tx) *tx = h->lc.tx;
  if (radix)
    for (int j = 0; j < 3; j++)
      for (int i = 0; i < 8; i++) radix[j][i] = i < h->plan[j].nst ? h->plan[j].radix[i] : 0;
  return RVE_OK;
}

struct rve_batch {
  std::vector<rve*> m;
  std::vector<cudaStream_t> own, old;
};

int rve_batch_create(rve_batch_t** out, int count, rve_t* const* members, int autotune_reps) {
  if (!out || count < 1 || !members || autotune_reps < 0) return RVE_ERR_ARG;
  *out = nullptr;
  for (int i = 0; i < count; i++) {
    if (!members[i]) return RVE_ERR_ARG;
    if (!members[i]->phases_set || !members[i]->path_set) return RVE_ERR_STATE;
    for (int k = 0; k < i; k++)
      if (members[k] == members[i]) return RVE_ERR_ARG;
  }
  rve_batch* b = new (std::nothrow) rve_batch();
  if (!b) return RVE_ERR_OOM;
  b->m.assign(members, members + count);
  for (int i = 0; i < count; i++) {
    rve* h = b->m[i];
    cudaStream_t st = nullptr;
    if (cudaStreamSynchronize(h->st) != cudaSuccess ||
        cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      rve_batch_free(b);
      return RVE_ERR_CUDA;
    }
    b->own.push_back(st);
    b->old.push_back(h->st);
    h->st = st;
    graphs_reset(h);
    h->graphs = true;
  }
  if (autotune_reps > 0) {
    for (rve* h : b->m) {
      if (h->stepped) continue;
      const int s = rve_autotune(h, autotune_reps, nullptr, nullptr, nullptr);
      if (s) {
        rve_batch_free(b);
        return s;
      }
    }
  }
  *out = b;
  return RVE_OK;
}

int rve_batch_step(rve_batch_t* b, rve_step_info* infos) {
  if (!b || !infos) return RVE_ERR_ARG;
  const size_t n = b->m.size();
  std::vector<int> st(n, RVE_OK);
  std::vector<std::thread> th;
  th.reserve(n);
  for (size_t i = 0; i < n; i++) {
    rve* h = b->m[i];
    rve_step_info* inf = infos + i;
    int* out = &st[i];
    th.emplace_back([h, inf, out]() {
      if (h->n_done >= h->n_incr) {
        std::memset(inf, 0, sizeof(*inf));
        inf->status = RVE_ERR_LOAD_PATH_END;
        inf->increment = h->n_done;
        *out = RVE_OK;
        return;
      }
      *out = rve_step_increment(h, inf);
    });
  }
  for (auto& t : th) t.join();
  for (size_t i = 0; i < n; i++)
    if (st[i] != RVE_OK) return st[i];
  return RVE_OK;
}

int rve_batch_size(const rve_batch_t* b) { return b ? (int)b->m.size() : 0; }

void rve_batch_free(rve_batch_t* b) {
  if (!b) return;
  for (size_t i = 0; i < b->own.size(); i++) {
    rve* h = b->m[i];
    cudaStreamSynchronize(b->own[i]);
    graphs_reset(h);
    h->graphs = false;
    h->st = b->old[i];
    cudaStreamDestroy(b->own[i]);
  }
  delete b;
}

// ============================================================ adjoint sweep
// Saved converged state after n_done increments (restart point).
struct AdjCkpt {
  int n_done = 0;
  double E_prev[6], S_prev[6], sig_mean[6], eps_mean[6], D_mean = 0, D_max = 0;
  double *eps_conv = nullptr, *epsp_n = nullptr, *ep_n = nullptr, *abar_n = nullptr;
};

struct AdjointStore {
  int every = 0, n_total = 0;
  double J = 0;
  std::vector<AdjCkpt> ckpt;   // after 0, every, 2 every, ... increments
  AdjCkpt last;                // after the last increment
  // per increment of one segment: eps_n, abar_n and the history before it
  std::vector<double*> seg_eps, seg_abar, seg_epsp, seg_ep;
  double *eta_p = nullptr, *eta_e = nullptr, *eta_p2 = nullptr, *eta_e2 = nullptr;
  double *lam = nullptr, *lam2 = nullptr, *mu = nullptr, *mu2 = nullptr;
  double *v_eps = nullptr, *v_abar = nullptr, *v_theta = nullptr, *v_stiff = nullptr, *g_stiff = nullptr;
  double *b = nullptr, *G1 = nullptr, *G2 = nullptr, *red = nullptr;
  double* part = nullptr;      // [4 kMaxPhases][max_blocks] block partial sums
  std::vector<void*> allocs;
  bool forward_done = false;
};

void adjoint_free(rve* h) {
  if (!h->adj) return;
  for (void* p : h->adj->allocs) cudaFree(p);
  delete h->adj;
  h->adj = nullptr;
}

namespace {

int adj_alloc(AdjointStore* a, double** p, size_t n) {
  void* v = nullptr;
  const cudaError_t e = cudaMalloc(&v, std::max<size_t>(n, 2) * sizeof(double));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? RVE_ERR_OOM : RVE_ERR_CUDA;
  }
  a->allocs.push_back(v);
  *p = (double*)v;
  return RVE_OK;
}

int ckpt_alloc(rve* h, AdjointStore* a, AdjCkpt& c) {
  const size_t V = (size_t)h->g.V, J = (size_t)std::max(h->J, 1);
  int s;
  if ((s = adj_alloc(a, &c.eps_conv, h->g.nc * V)) || (s = adj_alloc(a, &c.epsp_n, 6 * V)) ||
      (s = adj_alloc(a, &c.ep_n, V)) || (s = adj_alloc(a, &c.abar_n, J * V)))
    return s;
  return RVE_OK;
}

int ckpt_save(rve* h, AdjCkpt& c) {
  const size_t V = (size_t)h->g.V, J = (size_t)std::max(h->J, 1);
  CK(cudaMemcpyAsync(c.eps_conv, h->eps_conv, h->g.nc * V * 8, cudaMemcpyDeviceToDevice, h->st));
  CK(cudaMemcpyAsync(c.epsp_n, h->epsp_n, 6 * V * 8, cudaMemcpyDeviceToDevice, h->st));
  CK(cudaMemcpyAsync(c.ep_n, h->ep_n, V * 8, cudaMemcpyDeviceToDevice, h->st));
  CK(cudaMemcpyAsync(c.abar_n, h->abar_n, J * V * 8, cudaMemcpyDeviceToDevice, h->st));
  c.n_done = h->n_done;
  for (int k = 0; k < 6; k++) {
    c.E_prev[k] = h->E_prev[k];
    c.S_prev[k] = h->S_prev[k];
    c.sig_mean[k] = h->sig_mean[k];
    c.eps_mean[k] = h->eps_mean[k];
  }
  c.D_mean = h->D_mean;
  c.D_max = h->D_max;
  return RVE_OK;
}

int ckpt_load(rve* h, const AdjCkpt& c) {
  const size_t V = (size_t)h->g.V, J = (size_t)std::max(h->J, 1);
  CK(cudaMemcpyAsync(h->eps_conv, c.eps_conv, h->g.nc * V * 8, cudaMemcpyDeviceToDevice, h->st));
  CK(cudaMemcpyAsync(h->eps, c.eps_conv, h->g.nc * V * 8, cudaMemcpyDeviceToDevice, h->st));
  CK(cudaMemcpyAsync(h->epsp_n, c.epsp_n, 6 * V * 8, cudaMemcpyDeviceToDevice, h->st));
  CK(cudaMemcpyAsync(h->ep_n, c.ep_n, V * 8, cudaMemcpyDeviceToDevice, h->st));
  CK(cudaMemcpyAsync(h->abar_n, c.abar_n, J * V * 8, cudaMemcpyDeviceToDevice, h->st));
  CK(cudaStreamSynchronize(h->st));
  h->n_done = c.n_done;
  for (int k = 0; k < 6; k++) {
    h->E_prev[k] = c.E_prev[k];
    h->S_prev[k] = c.S_prev[k];
    h->sig_mean[k] = c.sig_mean[k];
    h->eps_mean[k] = c.eps_mean[k];
  }
  h->D_mean = c.D_mean;
  h->D_max = c.D_max;
  return RVE_OK;
}

int adj_setup(rve* h, int every) {
  adjoint_free(h);
  AdjointStore* a = new (std::nothrow) AdjointStore();
  if (!a) return RVE_ERR_OOM;
  h->adj = a;
  a->every = every;
  a->n_total = h->n_incr;
  const size_t V = (size_t)h->g.V, nc = h->g.nc, J = (size_t)std::max(h->J, 1);
  const int nck = (h->n_incr + every - 1) / every;
  a->ckpt.resize(nck);
  int s;
  for (auto& c : a->ckpt)
    if ((s = ckpt_alloc(h, a, c))) return s;
  if ((s = ckpt_alloc(h, a, a->last))) return s;
  a->seg_eps.resize(every);
  a->seg_abar.resize(every);
  a->seg_epsp.resize(every);
  a->seg_ep.resize(every);
  for (int k = 0; k < every; k++)
    if ((s = adj_alloc(a, &a->seg_eps[k], nc * V)) || (s = adj_alloc(a, &a->seg_abar[k], J * V)) ||
        (s = adj_alloc(a, &a->seg_epsp[k], 6 * V)) || (s = adj_alloc(a, &a->seg_ep[k], V)))
      return s;
  if ((s = adj_alloc(a, &a->eta_p, 6 * V)) || (s = adj_alloc(a, &a->eta_e, V)) ||
      (s = adj_alloc(a, &a->eta_p2, 6 * V)) || (s = adj_alloc(a, &a->eta_e2, V)) ||
      (s = adj_alloc(a, &a->lam, nc * V)) || (s = adj_alloc(a, &a->lam2, nc * V)) ||
      (s = adj_alloc(a, &a->mu, J * V)) || (s = adj_alloc(a, &a->mu2, J * V)) ||
      (s = adj_alloc(a, &a->v_eps, nc * V)) || (s = adj_alloc(a, &a->v_abar, J * V)) ||
      (s = adj_alloc(a, &a->v_theta, 4 * V)) || (s = adj_alloc(a, &a->v_stiff, V)) ||
      (s = adj_alloc(a, &a->g_stiff, V)) || (s = adj_alloc(a, &a->b, nc * V)) ||
      (s = adj_alloc(a, &a->G1, 3 * V)) || (s = adj_alloc(a, &a->G2, 3 * V)) ||
      (s = adj_alloc(a, &a->red, 64)) || (s = adj_alloc(a, &a->part, (size_t)4 * kMaxPhases * h->lc.max_blocks)))
    return s;
  return RVE_OK;
}

struct AdjSums {
  double theta[kMaxPhases][4];
  double ell[kMaxVars];
  long long cg, pcg;
  int outer, outer_max;
};

// real-space gradient fields G_d a = F^-1(k_d F a), d = 0..dim-1, into out [d][V]
void grad_field(rve* h, const Tables<double>&, const double* a, double* out) {
  LAUNCHB(h, KC_MISC, 0.0, k_corner_grad64(h->st, h->g, a, out));
}

// read `n` finalised scalars from the adjoint reduction area
int red_read(rve* h, double* out, int n) {
  CK(cudaMemcpyAsync(h->hscal, h->adj->red, n * sizeof(double), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  CK(cudaGetLastError());
  for (int i = 0; i < n; i++) out[i] = h->hscal[i];
  return RVE_OK;
}

// One increment of the reverse sweep at segment slot k (state of increment
// n: eps_n, abar_n, history h_{n-1}); seed = dJ/V on sigma_11 at the last
// increment, 0 before.
int adj_increment(rve* h, int k, double seed, AdjSums& acc) {
  AdjointStore* a = h->adj;
  const Geo& g = h->g;
  const long long V = g.V;
  const int nc = g.nc, J = h->J;
  const Tables<double> t = tables<double>(h);
  const int nb = h->lc.n_ew_blocks, ps = h->lc.max_blocks;
  double* part = a->part;
  AdjState st{h->phase, a->seg_eps[k], a->seg_epsp[k], a->seg_ep[k], a->seg_abar[k], h->stiff};
  // consistent tangent at the converged state (descriptor used by CG)
  LAUNCHB(h, KC_RETURN_MAP, 0.0, Ops<double>::return_map(g, h->lc, h->st, h->pt_dev, J, h->phase, st.eps, st.epsp_prev,
                                                          st.ep_prev, st.abar, h->sigma, h->epsp, h->ep, h->D,
                                                          h->alpha, (double*)h->desc, h->part, h->stiff));
  CK(cudaMemsetAsync(a->lam, 0, nc * V * 8, h->st));
  CK(cudaMemsetAsync(a->mu, 0, std::max(J, 1) * V * 8, h->st));
  AdjDirs d_eps{nc, {}, {}}, d_abar{J, {}, {}}, d_hist{8, {}, {}}, d_theta{4, {}, {}};
  for (int c = 0; c < nc; c++) { d_eps.kind[c] = AD_EPS; d_eps.idx[c] = c; }
  for (int j = 0; j < J; j++) { d_abar.kind[j] = AD_ABAR; d_abar.idx[j] = j; }
  for (int c = 0; c < 6; c++) { d_hist.kind[c] = AD_EPSP; d_hist.idx[c] = c; }
  d_hist.kind[6] = AD_EP; d_hist.idx[6] = 0;
  d_hist.kind[7] = AD_STIFF; d_hist.idx[7] = 0;
  for (int i = 0; i < 4; i++) { d_theta.kind[i] = AD_THETA; d_theta.idx[i] = i; }
  AdjOut out{a->v_eps, a->eta_p2, a->eta_e2, a->v_abar, a->v_theta, a->v_stiff};
  const int maxo = std::max(1, h->opt.max_stag);
  int it = 0;
  for (;;) {
    // mechanical adjoint: P C_T lam = P [d(sigma, alpha, h)/d eps]^T (seed, mu, eta)
    LAUNCHB(h, KC_MISC, 0.0, adj_local_vjp(g, h->pt_dev, J, st, AdjCot{seed, nullptr, a->mu, a->eta_p, a->eta_e}, out, d_eps, nb, h->st));
    int s = Alg<double>::op_apply_gamma(h, a->v_eps, a->b);
    if (s) return s;
    int iters = 0;
    s = Alg<double>::op_cg(h, a->b, a->lam2, h->opt.cg_rtol, h->opt.max_cg, &iters);
    acc.cg += iters;
    if (s) return s;
    // Helmholtz adjoints: L_j mu_j = [d sigma / d abar_j]^T (seed e_11 - lam)
    if (J > 0) {
      LAUNCHB(h, KC_MISC, 0.0, adj_local_vjp(g, h->pt_dev, J, st, AdjCot{seed, a->lam2, nullptr, nullptr, nullptr}, out, d_abar, nb, h->st));
      for (int j = 0; j < J; j++) {
        s = Alg<double>::op_helm_solve(h, j, a->v_abar + (size_t)j * V, a->mu2 + (size_t)j * V, h->opt.pcg_rtol,
                                            h->opt.max_pcg, &iters);
        acc.pcg += iters;
        if (s) return s;
      }
    }
    // change of both adjoints since the last sweep
    double r[4] = {0, 0, 0, 0};
    LAUNCHB(h, KC_MISC, 0.0, adj_absmax2((long long)nc * V, a->lam2, a->lam, part, ps, nb, h->st));
    LAUNCHB(h, KC_FINALIZE, 0.0, k_finalize(h->st, h->fin, part, nb, ps, 2, FIN_MAXS, nullptr, a->red, 1.0));
    if (J > 0) {
      LAUNCHB(h, KC_MISC, 0.0, adj_absmax2((long long)J * V, a->mu2, a->mu, part, ps, nb, h->st));
      LAUNCHB(h, KC_FINALIZE, 0.0, k_finalize(h->st, h->fin, part, nb, ps, 2, FIN_MAXS, nullptr, a->red + 2, 1.0));
    }
    if ((s = red_read(h, r, 4))) return s;
    std::swap(a->lam, a->lam2);
    std::swap(a->mu, a->mu2);
    it++;
    const double dl = r[0] / std::max(r[1], 1e-300), dm = J > 0 ? r[2] / std::max(r[3], 1e-300) : 0.0;
    if (h->verbose)
      std::fprintf(stderr, "[rve] adjoint sweep %d d_lambda %.3e d_mu %.3e\n", it, dl, dm);
    if (!(dl == dl) || !(dm == dm)) return RVE_ERR_NUMERIC;
    if ((dl <= h->opt.tol_stag || r[1] == 0.0) && (dm <= h->opt.tol_stag || J == 0 || r[3] == 0.0)) break;
    if (it >= maxo) return RVE_ERR_NOT_CONVERGED;
  }
  acc.outer += it;
  acc.outer_max = std::max(acc.outer_max, it);
  // history adjoint, modulus-field and parameter products with the full cotangent
  const AdjCot full{seed, a->lam, a->mu, a->eta_p, a->eta_e};
  LAUNCHB(h, KC_MISC, 0.0, adj_local_vjp(g, h->pt_dev, J, st, full, out, d_hist, nb, h->st));
  LAUNCHB(h, KC_MISC, 0.0, adj_local_vjp(g, h->pt_dev, J, st, full, out, d_theta, nb, h->st));
  LAUNCHB(h, KC_MISC, 0.0, adj_axpy(V, 1.0, a->v_stiff, a->g_stiff, nb, h->st));
  LAUNCHB(h, KC_MISC, 0.0, adj_phase_sums(V, h->phase, a->v_theta, part, ps, nb, h->st));
  // the finaliser reduces at most 16 slots per call
  for (int half = 0; half < 4 * kMaxPhases; half += 16)
    LAUNCHB(h, KC_FINALIZE, 0.0, k_finalize(h->st, h->fin, part + (size_t)half * ps, nb, ps, 16, FIN_SUMS, nullptr, a->red + half, 1.0));
  double th[4 * kMaxPhases];
  int s = red_read(h, th, 4 * kMaxPhases);
  if (s) return s;
  for (int q = 0; q < kMaxPhases; q++)
    for (int i = 0; i < 4; i++) acc.theta[q][i] += th[4 * q + i];
  // characteristic lengths: - <mu_j, (dL_j/dl_j) abar_j>
  for (int j = 0; j < J; j++) {
    double own2 = 0.0;
    for (int q = 0; q < h->n_phases; q++) own2 = std::max(own2, h->pt_host.ell2[j][q]);
    if (!(own2 > 0.0)) continue;
    PhaseWeights w{};
    for (int q = 0; q < kMaxPhases; q++) w.w[q] = q < h->n_phases ? 2.0 * h->pt_host.ell2[j][q] / std::sqrt(own2) : 0.0;
    grad_field(h, t, a->mu + (size_t)j * V, a->G1);
    grad_field(h, t, a->seg_abar[k] + (size_t)j * V, a->G2);
    LAUNCHB(h, KC_MISC, 0.0, adj_weighted_dot(V, g.d, h->phase, w, a->G1, a->G2, part, ps, nb, h->st));
    LAUNCHB(h, KC_FINALIZE, 0.0, k_finalize(h->st, h->fin, part, nb, ps, 1, FIN_SUMS, nullptr, a->red, 1.0));
    double dv = 0.0;
    if ((s = red_read(h, &dv, 1))) return s;
    acc.ell[j] -= dv;
  }
  std::swap(a->eta_p, a->eta_p2);
  std::swap(a->eta_e, a->eta_e2);
  return RVE_OK;
}

}  // namespace

int rve_set_stiffness_field(rve_t* h, const double* s) {
  if (!h) return RVE_ERR_ARG;
  if (!s) {
    if (h->stiff) cudaFree(h->stiff);
    h->stiff = nullptr;
    return RVE_OK;
  }
  const size_t V = (size_t)h->g.V;
  for (size_t v = 0; v < V; v++)
    if (!(s[v] > 0.0) || !std::isfinite(s[v])) return RVE_ERR_ARG;
  if (!h->stiff) {
    void* p = nullptr;
    if (cudaMalloc(&p, V * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      return RVE_ERR_OOM;
    }
    h->stiff = (double*)p;
  }
  CK(cudaMemcpy(h->stiff, s, V * sizeof(double), cudaMemcpyHostToDevice));
  return RVE_OK;
}

int rve_adjoint_forward(rve_t* h, int checkpoint_every, double* J) {
  if (!h || checkpoint_every < 1) return RVE_ERR_ARG;
  if (h->prec != RVE_FP64) return RVE_ERR_ARG;
  if (!h->phases_set || !h->path_set) return RVE_ERR_STATE;
  // the local derivative products are written for linear hardening and
  // laws 0-2
  for (int q = 0; q < h->n_phases; q++)
    if (h->pt_host.p[q].hard != 0 || h->pt_host.p[q].law > 2) return RVE_ERR_ARG;
  try {
    int s = adj_setup(h, checkpoint_every);
    if (s) { adjoint_free(h); return s; }
    AdjointStore* a = h->adj;
    if ((s = reset_state(h))) return s;
    h->stepped = true;
    for (int n = 0; n < h->n_incr; n++) {
      if (n % checkpoint_every == 0 && (s = ckpt_save(h, a->ckpt[n / checkpoint_every]))) return s;
      if ((s = Alg<double>::step(h, nullptr))) return s;
    }
    if ((s = ckpt_save(h, a->last))) return s;
    CK(cudaStreamSynchronize(h->st));
    a->J = h->sig_mean[0];
    a->forward_done = true;
    if (J) *J = a->J;
    return RVE_OK;
  } catch (...) {
    return RVE_ERR_OOM;
  }
}

int rve_adjoint_backward(rve_t* h, double dJ, double* grad_params, double* grad_ell, double* grad_stiff,
                         rve_adjoint_info* info) {
  if (!h) return RVE_ERR_ARG;
  if (info) std::memset(info, 0, sizeof(*info));
  if (!h->adj || !h->adj->forward_done) return RVE_ERR_STATE;
  AdjointStore* a = h->adj;
  const long long V = h->g.V;
  AdjSums acc{};
  int recomputed = 0;
  try {
    CK(cudaMemsetAsync(a->eta_p, 0, 6 * V * 8, h->st));
    CK(cudaMemsetAsync(a->eta_e, 0, V * 8, h->st));
    CK(cudaMemsetAsync(a->g_stiff, 0, V * 8, h->st));
    const int N = a->n_total, every = a->every;
    int s = RVE_OK;
    for (int seg = (N - 1) / every; seg >= 0 && !s; seg--) {
      const int c0 = seg * every, c1 = std::min(N, c0 + every);
      if ((s = ckpt_load(h, a->ckpt[seg]))) break;
      // recompute the segment, keeping each increment's state
      for (int n = c0; n < c1 && !s; n++) {
        const int k = n - c0;
        CK(cudaMemcpyAsync(a->seg_epsp[k], h->epsp_n, 6 * V * 8, cudaMemcpyDeviceToDevice, h->st));
        CK(cudaMemcpyAsync(a->seg_ep[k], h->ep_n, V * 8, cudaMemcpyDeviceToDevice, h->st));
        if ((s = Alg<double>::step(h, nullptr))) break;
        recomputed++;
        CK(cudaMemcpyAsync(a->seg_eps[k], h->eps_conv, h->g.nc * V * 8, cudaMemcpyDeviceToDevice, h->st));
        CK(cudaMemcpyAsync(a->seg_abar[k], h->abar_n, std::max(h->J, 1) * V * 8, cudaMemcpyDeviceToDevice, h->st));
      }
      for (int n = c1 - 1; n >= c0 && !s; n--)
        s = adj_increment(h, n - c0, n == N - 1 ? dJ / (double)V : 0.0, acc);
    }
    int s2 = ckpt_load(h, a->last);
    if (info) {
      info->status = s;
      info->increments = N;
      info->recomputed = recomputed;
      info->checkpoints = (int)a->ckpt.size();
      info->transposed_staggered_iters = acc.outer;
      info->max_transposed_staggered_iters = acc.outer_max;
      info->cg_iters = acc.cg;
      info->pcg_iters = acc.pcg;
    }
    if (s) return s;
    if (s2) return s2;
    if (grad_params)
      for (int q = 0; q < h->n_phases; q++)
        for (int i = 0; i < 4; i++) grad_params[4 * q + i] = acc.theta[q][i];
    if (grad_ell)
      for (int j = 0; j < h->J; j++) grad_ell[j] = acc.ell[j];
    if (grad_stiff) CK(cudaMemcpy(grad_stiff, a->g_stiff, V * 8, cudaMemcpyDeviceToHost));
    return RVE_OK;
  } catch (...) {
    return RVE_ERR_OOM;
  }
}

// ============================================================ checkpoint / resume
namespace {
struct StateHeader {
  char magic[8];
  int version, dim, prec, J;
  int n[3], nc;
  long long V;
  int n_done, pad;
  double E_prev[6], S_prev[6], sig_mean[6], eps_mean[6], D_mean, D_max;
};
const char kStateMagic[8] = {'R', 'V', 'E', 'S', 'T', 'A', 'T', '1'};
constexpr int kStateVersion = 3;
}  // namespace

long long rve_state_bytes(const rve_t* h) {
  if (!h) return 0;
  const long long V = h->g.V;
  return (long long)sizeof(StateHeader) + (long long)(h->g.nc + 8 + h->J) * V * 8;
}

int rve_save_state(const rve_t* h, void* buf, long long bytes) {
  if (!h || !buf || bytes < rve_state_bytes(h)) return RVE_ERR_ARG;
  if (!h->phases_set) return RVE_ERR_STATE;
  StateHeader hd{};
  std::memcpy(hd.magic, kStateMagic, 8);
  hd.version = kStateVersion;
  hd.dim = h->dim;
  hd.prec = h->prec;
  hd.J = h->J;
  for (int j = 0; j < 3; j++) hd.n[j] = h->n[j];
  hd.nc = h->g.nc;
  hd.V = h->g.V;
  hd.n_done = h->n_done;
  for (int c = 0; c < 6; c++) {
    hd.E_prev[c] = h->E_prev[c];
    hd.S_prev[c] = h->S_prev[c];
    hd.sig_mean[c] = h->sig_mean[c];
    hd.eps_mean[c] = h->eps_mean[c];
  }
  hd.D_mean = h->D_mean;
  hd.D_max = h->D_max;
  unsigned char* p = (unsigned char*)buf;
  std::memcpy(p, &hd, sizeof(hd));
  p += sizeof(hd);
  const size_t V = (size_t)h->g.V;
  CK(cudaStreamSynchronize(h->st));
  CK(cudaMemcpy(p, h->eps_conv, h->g.nc * V * 8, cudaMemcpyDeviceToHost));
  p += h->g.nc * V * 8;
  CK(cudaMemcpy(p, h->epsp_n, 6 * V * 8, cudaMemcpyDeviceToHost));
  p += 6 * V * 8;
  CK(cudaMemcpy(p, h->ep_n, V * 8, cudaMemcpyDeviceToHost));
  p += V * 8;
  if (h->J > 0) CK(cudaMemcpy(p, h->abar_n, (size_t)h->J * V * 8, cudaMemcpyDeviceToHost));
  p += (size_t)h->J * V * 8;
  CK(cudaMemcpy(p, h->f_n, V * 8, cudaMemcpyDeviceToHost));
  return RVE_OK;
}

int rve_load_state(rve_t* h, const void* buf, long long bytes) {
  if (!h || !buf || bytes < (long long)sizeof(StateHeader)) return RVE_ERR_ARG;
  if (!h->phases_set) return RVE_ERR_STATE;
  StateHeader hd;
  std::memcpy(&hd, buf, sizeof(hd));
  if (std::memcmp(hd.magic, kStateMagic, 8) != 0 || hd.version != kStateVersion || hd.dim != h->dim ||
      hd.J != h->J || hd.nc != h->g.nc || hd.V != h->g.V || hd.n[0] != h->n[0] || hd.n[1] != h->n[1] ||
      hd.n[2] != h->n[2] || bytes < rve_state_bytes(h) || hd.n_done < 0)
    return RVE_ERR_ARG;
  const unsigned char* p = (const unsigned char*)buf + sizeof(hd);
  const size_t V = (size_t)h->g.V;
  CK(cudaStreamSynchronize(h->st));
  CK(cudaMemcpy(h->eps_conv, p, h->g.nc * V * 8, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(h->eps, p, h->g.nc * V * 8, cudaMemcpyHostToDevice));
  p += h->g.nc * V * 8;
  CK(cudaMemcpy(h->epsp_n, p, 6 * V * 8, cudaMemcpyHostToDevice));
  p += 6 * V * 8;
  CK(cudaMemcpy(h->ep_n, p, V * 8, cudaMemcpyHostToDevice));
  p += V * 8;
  if (h->J > 0) CK(cudaMemcpy(h->abar_n, p, (size_t)h->J * V * 8, cudaMemcpyHostToDevice));
  p += (size_t)h->J * V * 8;
  CK(cudaMemcpy(h->f_n, p, V * 8, cudaMemcpyHostToDevice));
  h->n_done = hd.n_done;
  for (int c = 0; c < 6; c++) {
    h->E_prev[c] = hd.E_prev[c];
    h->S_prev[c] = hd.S_prev[c];
    h->sig_mean[c] = hd.sig_mean[c];
    h->eps_mean[c] = hd.eps_mean[c];
  }
  h->D_mean = hd.D_mean;
  h->D_max = hd.D_max;
  return RVE_OK;
}
