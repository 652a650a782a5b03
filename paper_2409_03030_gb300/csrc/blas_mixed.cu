// Vector and scalar kernels of mixed-precision CG with reliable updates.
//
// The inner CG runs on the even-parity Schur system in low precision: the
// operator and the search direction p (and A p) in FP32 or FP16 with a
// per-site norm, the iterate x_s and residual r_s in FP32.  Whenever the
// inner residual has dropped by a factor delta since the last update (or the
// inner loop thinks it has converged), the host folds x_s into the
// double-word solution x, recomputes r = rhs - A x in double-word arithmetic,
// and restarts the inner residual from it while keeping the search direction
// (reliable updates; Sleijpen and van der Vorst 1996).  Every decision is
// taken on the device in single-block kernels; the host only polls.
#include <cuda_runtime.h>

#include "fields.cuh"
#include "kernels.h"
#include "pdl.cuh"
#include "cg_steps.cuh"
#include "reduce.cuh"

namespace jqcd {

// FP32 spinor chunks of one site <-> registers
__device__ __forceinline__ void load_f32(const float4 *base, int64_t vh, int64_t i, cf (&s)[4][3]) {
  PT<PREC_F32>::load_spinor(base, vh, i, s);
}
__device__ __forceinline__ void store_f32(float4 *base, int64_t vh, int64_t i, const cf (&s)[4][3]) {
  PT<PREC_F32>::store_spinor(base, vh, i, s);
}

template <int PREC>
__global__ void mixed_xpay_kernel(void *__restrict__ p, const float4 *__restrict__ rs, int64_t vh,
                                  const SolverScalars *S) {
  pdl_enter();
  if (S->halt) return;
  const float b = S->beta_f;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= vh) return;
  cf pv[4][3], rv[4][3];
  PT<PREC>::load_spinor(p, vh, i, pv);
  load_f32(rs, vh, i, rv);
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    cf &q = pv[k / 3][k % 3];
    const cf r = rv[k / 3][k % 3];
    q.re = fmaf(b, q.re, r.re);
    q.im = fmaf(b, q.im, r.im);
  }
  PT<PREC>::store_spinor(p, vh, i, pv);
}

template <int PREC>
__global__ void mixed_copy_kernel(void *__restrict__ p, const float4 *__restrict__ rs, int64_t vh) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= vh) return;
  cf rv[4][3];
  load_f32(rs, vh, i, rv);
  PT<PREC>::store_spinor(p, vh, i, rv);
}

// FP32 chunk j of a site holds complex components 2j and 2j+1; double-word
// chunk k holds component k.  One thread per (site, FP32 chunk).
__global__ void dw_to_f32_kernel(float4 *__restrict__ rs, const float4 *__restrict__ r, int64_t vh) {
  const int64_t n = 6 * vh;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = q / vh, i = q % vh;
    const float4 a = r[(2 * j) * vh + i], b = r[(2 * j + 1) * vh + i];
    rs[q] = make_float4(a.x, a.y, b.x, b.y);  // normalised pairs: hi = nearest float
  }
}

__global__ void dw_add_f32_kernel(float4 *__restrict__ x, float4 *__restrict__ xs, int64_t vh) {
  const int64_t n = 6 * vh;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = q / vh, i = q % vh;
    const float4 s = xs[q];
    float4 *xa = x + (2 * j) * vh + i, *xb = x + (2 * j + 1) * vh + i;
    dw ar, ai, br, bi;
    dwc_unpack(*xa, ar, ai);
    dwc_unpack(*xb, br, bi);
    *xa = dwc_pack(dw_add(ar, dw_make(s.x, 0.f)), dw_add(ai, dw_make(s.y, 0.f)));
    *xb = dwc_pack(dw_add(br, dw_make(s.z, 0.f)), dw_add(bi, dw_make(s.w, 0.f)));
    xs[q] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

__global__ void mixed_beta_kernel(const double *partials, int n, SolverScalars *S) {
  pdl_enter();
  if (S->halt) return;
  const double rr_new = block_sum_partials(partials, n);
  if (threadIdx.x == 0) mixed_beta_step(rr_new, S);
}

__global__ void mixed_after_update_kernel(const double *partials, int n, SolverScalars *S) {
  const double rr_true = block_sum_partials(partials, n);
  if (threadIdx.x == 0) {
    S->reliable_updates += 1;
    S->need_update = 0;
    S->true_rr = rr_true;
    if (!isfinite(rr_true)) { S->done = 2; S->halt = 1; return; }
    if (rr_true <= S->stop_rr) { S->rr = rr_true; S->done = 1; S->halt = 1; return; }
    if (S->iters >= S->max_iters) { S->rr = rr_true; S->done = 3; S->halt = 1; return; }
    const double b = rr_true / S->rr;
    S->beta = b;
    S->beta_f = (float)b;
    S->rr = rr_true;
    S->rr_max = rr_true;
    S->halt = 0;
  }
}

static unsigned site_blocks(int64_t vh) { return (unsigned)((vh + kBlasThreads - 1) / kBlasThreads); }

cudaError_t launch_mixed_xpay(int hop_prec, void *p, const float4 *rs, int64_t vh,
                              const SolverScalars *S, cudaStream_t s) {
  note_launch();
  if (hop_prec == PREC_F16N)
    return launch_pdl(mixed_xpay_kernel<PREC_F16N>, site_blocks(vh), kBlasThreads, 0, s, p, rs, vh, S);
  else
    return launch_pdl(mixed_xpay_kernel<PREC_F32>, site_blocks(vh), kBlasThreads, 0, s, p, rs, vh, S);
}

cudaError_t launch_mixed_copy(int hop_prec, void *p, const float4 *rs, int64_t vh, cudaStream_t s) {
  note_launch();
  if (hop_prec == PREC_F16N)
    mixed_copy_kernel<PREC_F16N><<<site_blocks(vh), kBlasThreads, 0, s>>>(p, rs, vh);
  else
    mixed_copy_kernel<PREC_F32><<<site_blocks(vh), kBlasThreads, 0, s>>>(p, rs, vh);
  return cudaGetLastError();
}

cudaError_t launch_dw_to_f32(float4 *rs, const float4 *r, int64_t vh, cudaStream_t s) {
  note_launch();
  dw_to_f32_kernel<<<blas_blocks(6 * vh), kBlasThreads, 0, s>>>(rs, r, vh);
  return cudaGetLastError();
}

cudaError_t launch_dw_add_f32(float4 *x, float4 *xs, int64_t vh, cudaStream_t s) {
  note_launch();
  dw_add_f32_kernel<<<blas_blocks(6 * vh), kBlasThreads, 0, s>>>(x, xs, vh);
  return cudaGetLastError();
}

cudaError_t launch_mixed_beta(const double *partials, int n, SolverScalars *S, cudaStream_t s) {
  note_launch();
  return launch_pdl(mixed_beta_kernel, 1, kReduceThreads, 0, s, partials, n, S);
}

cudaError_t launch_mixed_after_update(const double *partials, int n, SolverScalars *S,
                                      cudaStream_t s) {
  note_launch();
  mixed_after_update_kernel<<<1, kReduceThreads, 0, s>>>(partials, n, S);
  return cudaGetLastError();
}

}  // namespace jqcd
