// Host-side interface of the device operators (kernel launchers) of the
// non-local damage RVE library.  Implemented in ops.cuh and instantiated for
// R = float (mixed precision) and R = double (FP64) in ops_f32.cu / ops_f64.cu.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace rvk {

// Grid geometry and the spectral layout.  Real fields are component-major
// [c][N3][N2][N1] (x1 fastest).  The half spectrum of a real field is
// [c][N3][N2][ps] complex with q1 = 0..N1/2 valid in each row of ps entries.
struct Geo {
  int d;                 // 2 or 3
  int n1, n2, n3;        // n3 = 1 in 2D
  int M;                 // n1 / 2
  int P1;                // n1 / 2 + 1
  int ps;                // padded spectral row (complex entries)
  int nc;                // carried Mandel components (3 in 2D, 6 in 3D)
  int cmap[6];           // carried -> full Mandel index
  long long V;           // voxels
  long long nlines;      // n2 * n3
  long long sstride;     // spectral component stride = ps * n2 * n3
  double h[3];           // voxel sizes
};

template <typename R>
struct Tables {
  C2<R>* tw[3];          // exp(-2 pi i m / N_j), m < N_j
  R* s[3];               // sin(pi q / N_j) in mode storage order
  R* c[3];               // cos(pi q / N_j), exactly 0 at the Nyquist index
  FftPlan plan_x;        // length n1 / 2
  FftPlan plan_y;        // n2
  FftPlan plan_z;        // n3
  R two_over_h[3];
};

// Launch configuration chosen once per grid.
struct LaunchCfg {
  int nrows_c[7];        // rows per CTA of the x1 pass for 1..6 components
  int xe_c[7];           // FFT elements staged per thread in that x1 pass (4 or 16)
  int tx;                // q1 columns per CTA of the strided passes
  int n_ew_blocks;       // CTAs of element-wise kernels
  int max_blocks;        // upper bound of CTAs of any reducing kernel
  int gamma_narrow;      // 3D six-component last-axis pass: half-width TMA tile, 128 threads
};

template <typename R>
struct Ops {
  // ---------------------------------------------------------------- x1 passes
  // forward: tau = C_T : p  (with p <- r + beta p when ctl != null and iter > 0);
  // partial (p, tau) into part when part != null
  // ext: descriptor in the extended layout A, B, C, D, nh (handles with a
  // GTN phase), else c1, c2, m
  static void xfwd_tangent(const Geo& g, const Tables<R>& t, const LaunchCfg& lc, cudaStream_t st,
                           R* p, const R* r, const R* desc, C2<R>* S, const KrylovCtl* ctl,
                           double* part = nullptr, int ext = 0);
  // forward: tau_c = f[map c][v] - mean[c] (ncomp components, comp stride V),
  // minus f2[map c][v] - mean2[c] when f2 / mean2 are given
  static void xfwd_field64(const Geo& g, const Tables<R>& t, const LaunchCfg& lc, cudaStream_t st,
                           const double* f, int ncomp, const int* fmap, const double* mean_dev,
                           C2<R>* S, const double* f2 = nullptr, const double* mean2 = nullptr);
  // inverse: Ap = scale * C2R(S); partial (p, Ap)
  static void xinv_matvec(const Geo& g, const Tables<R>& t, const LaunchCfg& lc, cudaStream_t st,
                          const C2<R>* S, R* Ap, const R* p, double* part, const KrylovCtl* ctl);
  // inverse with the CG step fused: Ap = scale * C2R(S) (not stored),
  // x += alpha p, r -= alpha Ap (alpha from ctl); partial (r, r)
  static void xinv_cg(const Geo& g, const Tables<R>& t, const LaunchCfg& lc, cudaStream_t st,
                      const C2<R>* S, R* x, R* r, const R* p, double* part, const KrylovCtl* ctl);
  // shared memory that xinv_cg asks for (it must fit the device's opt-in limit)
  static size_t xinv_cg_smem(const Geo& g, const LaunchCfg& lc);
  // inverse: b = bref - (C2R + mask (mean_sigma - mean_ref - sbar)) stored in
  // precision RO (bref, mean_ref may be null); partial (b, b) of the stored values
  template <typename RO>
  static void xinv_residual(const Geo& g, const Tables<R>& t, const LaunchCfg& lc, cudaStream_t st,
                            const C2<R>* S, RO* b, const double* mean_sig_dev, const double* dcterm_mask,
                            const double* sbar, double* part, const RO* bref = nullptr,
                            const double* mean_ref = nullptr);
  // inverse: out64[c][v] = scale * C2R(S)
  static void xinv_store64(const Geo& g, const Tables<R>& t, const LaunchCfg& lc, cudaStream_t st,
                           const C2<R>* S, int ncomp, double* out);
  // inverse along x1 of one spectral component into a real field in the
  // working precision: out[v] = C2R(S)[v] / V
  static void xinv_storeR(const Geo& g, const Tables<R>& t, const LaunchCfg& lc, cudaStream_t st,
                          const C2<R>* S, R* out, const KrylovCtl* ctl);
  // forward along x1 of one real field in the working precision
  static void xfwd_fieldR(const Geo& g, const Tables<R>& t, const LaunchCfg& lc, cudaStream_t st,
                          const R* f, C2<R>* S, const KrylovCtl* ctl);
  // y = sum_j D_j^T (l^2(phase) D_j q) in real space (the flux term of the
  // Helmholtz operator of Algorithm 2 with the rotated-scheme corner
  // derivative; the identity part is added to the spectrum by helm_contract)
  static void helm_stencil(const Geo& g, const LaunchCfg& lc, cudaStream_t st, const R* q, R* y,
                           const uint8_t* phase, const R* ell2_tab, const KrylovCtl* ctl);

  // ---------------------------------------------------------- strided passes
  // plain transform along axis (1 = y, 2 = z) of ncomp components
  static void strided_plain(const Geo& g, const Tables<R>& t, const LaunchCfg& lc, cudaStream_t st,
                            C2<R>* S, int ncomp, int axis, int sign, const KrylovCtl* ctl);
  // last axis: forward, modified projection (dc_mode 0: stress-mask at xi=0,
  // 1: zero at xi=0), inverse.  In 3D the tiles move by TMA; a CTA whose
  // tile did not arrive within wait_s seconds sets *wait_err (if given).
  // extra_tx > 0 only in tests of that path (bytes no copy delivers).
  static void gamma(const Geo& g, const Tables<R>& t, const LaunchCfg& lc, cudaStream_t st,
                    C2<R>* S, const float* stress_mask, int dc_mode, const KrylovCtl* ctl,
                    int* wait_err = nullptr, double wait_s = 2.0, int extra_tx = 0);
  // last axis inverse of one component with p <- M r + beta p, W = p
  // raw = 1: W = r without touching p (operator application only)
  static void helm_expand(const Geo& g, const Tables<R>& t, const LaunchCfg& lc, cudaStream_t st,
                          C2<R>* W, C2<R>* p, const C2<R>* r, double ell2_mean, const KrylovCtl* ctl,
                          int raw = 0);
  // last axis forward of one component; y = p + W; partial (p, y)
  // CTAs of helm_contract (rows of partial sums it writes)
  static int contract_blocks(const Geo& g, const LaunchCfg& lc);
  static void helm_contract(const Geo& g, const Tables<R>& t, const LaunchCfg& lc, cudaStream_t st,
                            const C2<R>* W, const C2<R>* p, C2<R>* y, double* part,
                            const KrylovCtl* ctl);

  // ------------------------------------------------------------- Krylov
  static void cg_init(const Geo& g, const LaunchCfg& lc, cudaStream_t st, R* x, const R* r,
                      double* part);
  static void cg_update(const Geo& g, const LaunchCfg& lc, cudaStream_t st, R* x, R* r, const R* p,
                        const R* Ap, double* part, const KrylovCtl* ctl);
  static void pcg_init(const Geo& g, const Tables<R>& t, const LaunchCfg& lc, cudaStream_t st,
                       C2<R>* x, const C2<R>* r, double ell2_mean, double* part);
  static void pcg_update(const Geo& g, const Tables<R>& t, const LaunchCfg& lc, cudaStream_t st,
                         C2<R>* x, C2<R>* r, const C2<R>* p, const C2<R>* y, double ell2_mean,
                         double* part, const KrylovCtl* ctl);

  // ------------------------------------------------------------- local
  // gtn != 0: a phase follows the GTN law (law 3); it reads the converged
  // non-local variables abar_n and porosity f_n, writes the new porosity to
  // f_out (f_n copied elsewhere) and the descriptor in the extended layout
  static void return_map(const Geo& g, const LaunchCfg& lc, cudaStream_t st, const PhaseTable* pt,
                         int J, const uint8_t* phase, const double* eps, const double* epsp_n,
                         const double* ep_n, const double* abar, double* sigma, double* epsp,
                         double* ep, double* D, double* alpha, R* desc, double* part,
                         const double* stiff = nullptr, const double* abar_n = nullptr,
                         const double* f_n = nullptr, double* f_out = nullptr, int gtn = 0);
  static void tangent_apply64(const Geo& g, const LaunchCfg& lc, cudaStream_t st, const R* desc,
                              const double* p, double* tau, int ext = 0);
  // eps += x; partials: max |x| per comp, sum eps per comp
  static void eps_update(const Geo& g, const LaunchCfg& lc, cudaStream_t st, double* eps,
                         const R* x, double* part);
  static void to_r(cudaStream_t st, long long n, const double* a, R* b);
  static void from_r(cudaStream_t st, long long n, const R* a, double* b);
};

// Precision-independent element-wise kernels (ops_common.cu).
// slot 0..nc-1: sum of eps_new per component; slot 6: max |eps_new - eps_old|
void k_err_eps(const Geo& g, const LaunchCfg& lc, cudaStream_t st, const double* eps_new,
               const double* eps_old, double* part);
void k_err_abar(const Geo& g, const LaunchCfg& lc, cudaStream_t st, const double* a_new,
                const double* a_old, double* part);
// finalize: reduce nslots (<= 16) slots of per-CTA partials; INIT modes
// also store rtol2 = scale and maxit = imax into ctl.  fs: the handle's
// scratch of the two-level reduction (ticket zero between launches; the
// launches of one handle are serialised on its stream).
constexpr int kFinMaxCtas = 64;
struct FinScratch {
  double stage[16 * kFinMaxCtas];
  unsigned ticket;
};
void k_finalize(cudaStream_t st, FinScratch* fs, const double* part, int nblocks, int nblk_stride, int nslots,
                int mode, KrylovCtl* ctl, double* out, double scale, int imax = 0, int stall = 0);
// out[j][v] = rotated-scheme derivative along x_j of the FP64 field a at the
// voxel corner v + 1/2 (j < d)
void k_corner_grad64(cudaStream_t st, const Geo& g, const double* a, double* out);
// forget the cached TMA tensor maps over a device buffer before it is freed
void tensor_map_evict(const void* base);
// f[v] = initial porosity f0 of the voxel's phase (GTN, law 3), else 0
void k_fill_porosity(cudaStream_t st, long long V, const uint8_t* phase, const PhaseTable* pt, double* f);
// dst[c][v] = src[c][v] + add[c]  (c < nc, FP64)
void k_copy_add(cudaStream_t st, long long V, int nc, const double* src, double* dst, const double* add_host6);

// finalize modes
enum {
  FIN_SUMS = 0,       // out[s] = scale * sum of slot s
  FIN_MAXS = 1,       // out[s] = max of slot s
  FIN_CG_INIT = 2,    // slot0 = (b,b) -> ctl init (CG)
  FIN_PCG_INIT = 3,   // slot0 = (r,r), slot1 = (r,Mr) -> ctl init (PCG)
  FIN_ALPHA = 4,      // slot0 = (p,Ap) -> alpha
  FIN_CG_BETA = 5,    // slot0 = (r,r)
  FIN_PCG_BETA = 6,   // slot0 = (r,r), slot1 = (r,Mr)
};

}  // namespace rvk
