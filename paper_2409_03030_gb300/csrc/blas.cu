// Vector kernels and the scalar steps of conjugate gradient.
//
// Double-word vectors are handled as flat arrays of float4 = one complex
// double-word number (re.h, im.h, re.l, im.l).  Vector kernels use a fixed
// grid with grid-stride loops, so the number of partial sums (and with it the
// rounding of every reduction) depends only on the vector length.
#include <cuda_runtime.h>

#include "dw.cuh"
#include "kernels.h"
#include "pdl.cuh"
#include "cg_steps.cuh"
#include "reduce.cuh"

namespace jqcd {

unsigned blas_blocks(int64_t n) {
  const int64_t per = (int64_t)kBlasThreads * 4;
  int64_t b = (n + per - 1) / per;
  if (b > 152 * 8) b = 152 * 8;
  if (b < 1) b = 1;
  return (unsigned)b;
}

__device__ __forceinline__ dw lo_dw(float h, float l) { return dw_make(h, l); }

__device__ __forceinline__ void accum_sq4(dwacc &A, float4 v) {
  dw re, im;
  dwc_unpack(v, re, im);
  acc_sq(A, re);
  acc_sq(A, im);
}

__global__ void dw_copy_kernel(float4 *__restrict__ d, const float4 *__restrict__ s, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    d[i] = s[i];
}

__global__ void dw_zero_kernel(float4 *__restrict__ d, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    d[i] = make_float4(0.f, 0.f, 0.f, 0.f);
}

__global__ void dw_norm2_kernel(const float4 *__restrict__ a, int64_t n, double *partials) {
  dwacc A{0.f, 0.f};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    accum_sq4(A, a[i]);
  const double s = block_sum_dw(A);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__global__ void dw_xmy_norm_kernel(float4 *__restrict__ r, const float4 *__restrict__ b,
                                   const float4 *__restrict__ y, int64_t n, double *partials) {
  dwacc A{0.f, 0.f};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    dw br, bi, yr, yi;
    dwc_unpack(b[i], br, bi);
    dwc_unpack(y[i], yr, yi);
    const dw re = dw_add(br, dw_neg(yr));
    const dw im = dw_add(bi, dw_neg(yi));
    r[i] = dwc_pack(re, im);
    acc_sq(A, re);
    acc_sq(A, im);
  }
  const double s = block_sum_dw(A);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__global__ void dw_cg_update_kernel(float4 *__restrict__ x, float4 *__restrict__ r,
                                    const float4 *__restrict__ p, const float4 *__restrict__ Ap,
                                    int64_t n, const SolverScalars *S, double *partials) {
  if (S->halt) return;
  const dw al = dw_make(S->alpha_dw.x, S->alpha_dw.y);
  const dw mal = dw_neg(al);
  dwacc A{0.f, 0.f};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    dw x_r, x_i, p_r, p_i, r_r, r_i, a_r, a_i;
    dwc_unpack(x[i], x_r, x_i);
    dwc_unpack(p[i], p_r, p_i);
    dwc_unpack(r[i], r_r, r_i);
    dwc_unpack(Ap[i], a_r, a_i);
    const dw xr = dw_add(x_r, dw_mul(al, p_r));
    const dw xi = dw_add(x_i, dw_mul(al, p_i));
    const dw rr = dw_add(r_r, dw_mul(mal, a_r));
    const dw ri = dw_add(r_i, dw_mul(mal, a_i));
    x[i] = dwc_pack(xr, xi);
    r[i] = dwc_pack(rr, ri);
    acc_sq(A, rr);
    acc_sq(A, ri);
  }
  const double s = block_sum_dw(A);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__global__ void dw_xpay_kernel(float4 *__restrict__ p, const float4 *__restrict__ r, int64_t n,
                               const SolverScalars *S) {
  pdl_enter();
  if (S->halt) return;
  const dw be = dw_make(S->beta_dw.x, S->beta_dw.y);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    dw p_r, p_i, r_r, r_i;
    dwc_unpack(p[i], p_r, p_i);
    dwc_unpack(r[i], r_r, r_i);
    p[i] = dwc_pack(dw_add(r_r, dw_mul(be, p_r)), dw_add(r_i, dw_mul(be, p_i)));
  }
}

// ---- single-block scalar steps -------------------------------------------------

__global__ void finalize_sum_kernel(const double *partials, int n, double *out) {
  const double s = block_sum_partials(partials, n);
  if (threadIdx.x == 0) *out = s;
}

__global__ void cg_alpha_kernel(const double *partials, int n, SolverScalars *S) {
  pdl_enter();
  if (S->halt) return;
  const double pAp = block_sum_partials(partials, n);
  if (threadIdx.x == 0) cg_alpha_step(pAp, S);
}

__global__ void cg_beta_kernel(const double *partials, int n, SolverScalars *S) {
  pdl_enter();
  if (S->halt) return;
  const double rr_new = block_sum_partials(partials, n);
  if (threadIdx.x == 0) cg_beta_step(rr_new, S);
}

__global__ void cg_start_kernel(const double *partials, int n, SolverScalars *S, double tol2,
                                int max_iters, double delta2) {
  const double rr = block_sum_partials(partials, n);
  if (threadIdx.x == 0) {
    S->rr = rr;
    S->true_rr = rr;  // the start residual is computed from x, not recursively
    S->stop_rr = tol2 * S->rhs2;
    S->max_iters = max_iters;
    S->delta2 = delta2;
    S->done = rr <= S->stop_rr ? 1 : (S->iters >= max_iters ? 3 : 0);
    S->halt = S->done != 0;
    S->need_update = 0;
    S->rr_max = rr;
    S->fin_count = 0;
  }
}

cudaError_t launch_finalize_sum(const double *partials, int n, double *out, cudaStream_t s) {
  note_launch();
  finalize_sum_kernel<<<1, kReduceThreads, 0, s>>>(partials, n, out);
  return cudaGetLastError();
}
cudaError_t launch_dw_copy(float4 *dst, const float4 *src, int64_t n, cudaStream_t s) {
  note_launch();
  dw_copy_kernel<<<blas_blocks(n), kBlasThreads, 0, s>>>(dst, src, n);
  return cudaGetLastError();
}
cudaError_t launch_dw_zero(float4 *dst, int64_t n, cudaStream_t s) {
  note_launch();
  dw_zero_kernel<<<blas_blocks(n), kBlasThreads, 0, s>>>(dst, n);
  return cudaGetLastError();
}
cudaError_t launch_dw_norm2(const float4 *a, int64_t n, double *partials, cudaStream_t s) {
  note_launch();
  dw_norm2_kernel<<<blas_blocks(n), kBlasThreads, 0, s>>>(a, n, partials);
  return cudaGetLastError();
}
cudaError_t launch_dw_xmy_norm(float4 *r, const float4 *b, const float4 *y, int64_t n,
                               double *partials, cudaStream_t s) {
  note_launch();
  dw_xmy_norm_kernel<<<blas_blocks(n), kBlasThreads, 0, s>>>(r, b, y, n, partials);
  return cudaGetLastError();
}
cudaError_t launch_dw_cg_update(float4 *x, float4 *r, const float4 *p, const float4 *Ap, int64_t n,
                                const SolverScalars *S, double *partials, cudaStream_t s) {
  note_launch();
  dw_cg_update_kernel<<<blas_blocks(n), kBlasThreads, 0, s>>>(x, r, p, Ap, n, S, partials);
  return cudaGetLastError();
}
cudaError_t launch_dw_xpay(float4 *p, const float4 *r, int64_t n, const SolverScalars *S,
                           cudaStream_t s) {
  note_launch();
  return launch_pdl(dw_xpay_kernel, blas_blocks(n), kBlasThreads, 0, s, p, r, n, S);
}
cudaError_t launch_cg_alpha(const double *partials, int n, SolverScalars *S, cudaStream_t s) {
  note_launch();
  return launch_pdl(cg_alpha_kernel, 1, kReduceThreads, 0, s, partials, n, S);
}
cudaError_t launch_cg_beta(const double *partials, int n, SolverScalars *S, cudaStream_t s) {
  note_launch();
  return launch_pdl(cg_beta_kernel, 1, kReduceThreads, 0, s, partials, n, S);
}
cudaError_t launch_cg_start(const double *partials, int n, SolverScalars *S, double tol2,
                            int max_iters, double delta2, cudaStream_t s) {
  note_launch();
  cg_start_kernel<<<1, kReduceThreads, 0, s>>>(partials, n, S, tol2, max_iters, delta2);
  return cudaGetLastError();
}

}  // namespace jqcd
