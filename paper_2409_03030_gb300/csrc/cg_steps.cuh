// Scalar steps of the conjugate gradient of the paper's solver (section
// "Definition of Dirac operators", solve_DinvX! with eps_CG): alpha =
// ||r||^2 / <p, A p>, beta = ||r_new||^2 / ||r||^2, the stopping test; run
// by thread 0 of the block that holds the fixed-order sum of a hop's
// per-block partials.  The single-block kernels of blas.cu and blas_mixed.cu
// call them; on small grids the last block of the hop that writes the
// partials calls them itself (hop_finish_scalars), which saves the launch of
// the single-block kernel.
#pragma once
#include <cuda_runtime.h>

#include "kernels.h"
#include "reduce.cuh"

namespace jqcd {

__device__ __forceinline__ float2 split_double(double v) {
  const float h = __double2float_rn(v);
  return make_float2(h, __double2float_rn(v - (double)h));
}

// alpha = rr / pAp; a non-positive or non-finite pAp ends the solve (breakdown)
__device__ __forceinline__ void cg_alpha_step(double pAp, SolverScalars *S) {
  S->pAp = pAp;
  if (!(pAp > 0.0) || !isfinite(pAp)) {
    S->done = 2;
    S->halt = 1;
    return;
  }
  const double a = S->rr / pAp;
  S->alpha = a;
  S->alpha_dw = split_double(a);
  S->malpha_dw = split_double(-a);
  S->alpha_f = (float)a;
  S->malpha_f = (float)-a;
}

// beta = rr_new / rr, the stopping test on rr_new and the iteration cap
__device__ __forceinline__ void cg_beta_step(double rr_new, SolverScalars *S) {
  S->rr_new = rr_new;
  S->iters += 1;
  if (!isfinite(rr_new)) {
    S->done = 2;
    S->halt = 1;
    return;
  }
  if (rr_new <= S->stop_rr) {
    S->rr = rr_new;
    S->done = 1;
    S->halt = 1;
    return;
  }
  if (S->iters >= S->max_iters) {
    S->done = 3;
    S->halt = 1;
  }
  const double b = rr_new / S->rr;
  S->beta = b;
  S->beta_dw = split_double(b);
  S->beta_f = (float)b;
  S->rr = rr_new;
}

// The inner solver of the mixed-precision CG: the same beta, and a reliable
// update requested (need_update, halt) when rr_new reaches the tolerance,
// drops below delta^2 max ||r||^2 since the last update, or at the cap.
__device__ __forceinline__ void mixed_beta_step(double rr_new, SolverScalars *S) {
  S->rr_new = rr_new;
  S->iters += 1;
  if (!isfinite(rr_new)) {
    S->done = 2;
    S->halt = 1;
    return;
  }
  if (rr_new <= S->stop_rr || rr_new < S->delta2 * S->rr_max || S->iters >= S->max_iters) {
    S->need_update = 1;  // the host runs the double-word update next
    S->halt = 1;
    return;
  }
  const double b = rr_new / S->rr;
  S->beta = b;
  S->beta_f = (float)b;
  S->rr = rr_new;
  if (rr_new > S->rr_max) S->rr_max = rr_new;
}

// block_sum_partials with its loads from L2 (ld.global.cg): the partials
// were written by other blocks of the same launch.
__device__ __forceinline__ double block_sum_partials_l2(const double *partials, int n) {
  double v = 0.0;
  constexpr int kU = 16;
  for (int base = threadIdx.x; base < n; base += kU * blockDim.x) {
    double t[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int i = base + u * (int)blockDim.x;
      t[u] = i < n ? __ldcg(partials + i) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) v += t[u];
  }
  return block_sum_d(v);
}

// Called by every thread of every block of a hop launch after thread 0 has
// written the block's partial (P.partials[blockIdx.x]) when P.fin is set: the
// block that finishes last (a counter in P.fin_S, no waiting) sums all the
// partials in the fixed order of the single-block kernels and takes the
// scalar step P.fin.  The fences order each block's partial before its
// count, and the counts before the last block's reads.
__device__ __forceinline__ void hop_finish_scalars(const HopParams &P) {
  __shared__ int is_last;
  if (threadIdx.x == 0) {
    __threadfence();
    const int done_blocks = atomicAdd(&P.fin_S->fin_count, 1);
    is_last = done_blocks == (int)gridDim.x - 1;
  }
  __syncthreads();
  if (!is_last) return;  // uniform over the block
  __threadfence();
  const double v = block_sum_partials_l2(P.partials, (int)gridDim.x);
  if (threadIdx.x == 0) {
    SolverScalars *S = P.fin_S;
    S->fin_count = 0;
    if (P.fin == FIN_ALPHA) cg_alpha_step(v, S);
    else if (P.fin == FIN_BETA) cg_beta_step(v, S);
    else mixed_beta_step(v, S);
  }
}

}  // namespace jqcd
