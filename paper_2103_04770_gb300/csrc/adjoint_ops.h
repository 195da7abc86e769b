// Kernels of the adjoint (reverse) sweep over converged increments, FP64.
//
// The paper has no adjoint.  The reverse sweep of the discrete problem
// needs, per voxel, products of the transposed Jacobian of the local update
// (the return map of Section 2.1.2 / Appendix A.2 and the particle-cracking
// variable) with a cotangent of its outputs, and a few reductions.  The
// linear solves of the sweep reuse the forward kernels (G*, CG, Helmholtz
// PCG).
#pragma once
#include "ops.h"

namespace rvk {

// Input directions of one forward-mode pass of the local Jacobian (at most
// eight per pass).
enum AdjDirKind { AD_EPS = 0, AD_EPSP = 1, AD_EP = 2, AD_ABAR = 3, AD_THETA = 4, AD_STIFF = 5 };
struct AdjDirs {
  int n;
  int kind[8];
  int idx[8];   // carried component (AD_EPS), Mandel component (AD_EPSP),
                // variable (AD_ABAR), parameter sigma_y/H/eps_C/eps_R (AD_THETA)
};

// State at which the local update is differentiated: the converged strain
// eps_n [nc][V], the history it started from (eps^p [6][V], e [V]), the
// converged non-local variables [J][V] and the modulus factor (or null).
struct AdjState {
  const uint8_t* phase;
  const double* eps;
  const double* epsp_prev;
  const double* ep_prev;
  const double* abar;
  const double* stiff;
};

// Cotangent of the outputs (sigma [6], alpha [J], eps^p [6], e) per voxel:
// w_sigma = seed11 e_11 - embed(lam); any pointer may be null (zero).
struct AdjCot {
  double seed11;
  const double* lam;       // [nc][V]
  const double* w_alpha;   // [J][V]
  const double* w_epsp;    // [6][V]
  const double* w_ep;      // [V]
};

// Products written for the directions of the pass (other arrays untouched).
struct AdjOut {
  double* v_eps;    // [nc][V]
  double* v_epsp;   // [6][V]
  double* v_ep;     // [V]
  double* v_abar;   // [J][V]
  double* v_theta;  // [4][V]: own phase's sigma_y, H, eps_C, eps_R
  double* v_stiff;  // [V]
};

struct PhaseWeights {
  double w[kMaxPhases];
};

void adj_local_vjp(const Geo& g, const PhaseTable* pt, int J, const AdjState& s, const AdjCot& w,
                   const AdjOut& o, const AdjDirs& dirs, int nblocks, cudaStream_t st);

// part slot 0: max |a - b|, slot 1: max |a| over n entries
void adj_absmax2(long long n, const double* a, const double* b, double* part, int pstride, int nblocks,
                 cudaStream_t st);

// part slot 0: sum_x w[phase(x)] sum_k ga[k][x] gb[k][x]
void adj_weighted_dot(long long V, int d, const uint8_t* phase, PhaseWeights w, const double* ga,
                      const double* gb, double* part, int pstride, int nblocks, cudaStream_t st);

// part slot 4 q + k: sum over the voxels of phase q of v_theta[k]
void adj_phase_sums(long long V, const uint8_t* phase, const double* v_theta, double* part, int pstride,
                    int nblocks, cudaStream_t st);

// y += a x
void adj_axpy(long long n, double a, const double* x, double* y, int nblocks, cudaStream_t st);

}  // namespace rvk
