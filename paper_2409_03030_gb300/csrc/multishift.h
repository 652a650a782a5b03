// Multi-shift CG on Mhat^dag Mhat (multishift.cu).
#pragma once
#include <cuda_runtime.h>

#include <string>

#include "jqcd.h"

namespace jqcd {

constexpr int kMsMaxShifts = 32;

// Device-resident scalars of one multi-shift solve.
struct MsScalars {
  double rr, alpha, alpha_prev, beta, stop_rr, rhs2;
  double sigma[kMsMaxShifts], zeta_prev[kMsMaxShifts], zeta[kMsMaxShifts], zeta_next[kMsMaxShifts];
  double alpha_s[kMsMaxShifts], beta_s[kMsMaxShifts], true_rr[kMsMaxShifts];
  int active[kMsMaxShifts], conv_iter[kMsMaxShifts];
  int xact[kMsMaxShifts];  // shifts whose x_i takes this iteration's update (active before beta)
  float2 alpha_dw;         // alpha as a (hi, lo) pair for the fused r update
  int nshift, iters, max_iters;
  int done;  // 1 every shift converged, 2 breakdown, 3 maxiter
  int halt;
  int final_x;  // beta halted the solve: the x_i update of that iteration is still due
};

// Per-shift solution and search direction (even parity, double-word).
struct MsVectors {
  float4 *x[kMsMaxShifts];
  float4 *p[kMsMaxShifts];
};

struct GaugeEntry;

cudaError_t launch_ms_start(const double *partials, int n, MsScalars *S, double tol2, int max_iters,
                            cudaStream_t s);
// alpha from the per-hop-block partials of ||Mhat p||^2.
cudaError_t launch_ms_alpha(const double *partials, int nhop, MsScalars *S, cudaStream_t s);
// beta from the per-hop-block partials of ||r||^2, then x_i += alpha_i p_i,
// p = r + beta p and p_i = zeta_i r + beta_i p_i in one pass over the shifts.
cudaError_t launch_ms_beta_xp(const double *partials, int nhop, int nblas, MsScalars *S, const MsVectors &V,
                              const float4 *r, float4 *pb, int64_t n, cudaStream_t s);
cudaError_t launch_ms_resid(const float4 *rhs, const float4 *Ax, const float4 *x, double sigma, int64_t n,
                            double *partials, int nblocks, cudaStream_t s);

// Solve (Mhat^dag Mhat + shifts[i]) x_i = rhs for the double-word even-parity
// rhs in G.vrhs (even half); x_even[i]: caller's even-parity buffers.
jqcd_status solve_multishift(GaugeEntry &G, const jqcd_solve_params &P, int nshift, const double *shifts,
                             float4 *const *x_even, cudaStream_t s, jqcd_solve_info *infos,
                             std::string *msg);

}  // namespace jqcd
