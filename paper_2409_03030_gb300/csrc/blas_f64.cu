// Vector kernels of the native FP64 conjugate gradient (JQCD_CG_F64).
//
// FP64 vectors are flat arrays of double2 = one complex number (re, im), in
// the per-parity chunk order of the JQCD_PREC_F64 spinor layout, so a whole
// lattice is 24 * vh complex numbers (even half first).  Every product and
// sum is IEEE FP64 (DFMA / DADD); reductions accumulate in FP64 per thread,
// per warp in a fixed shuffle tree and per block in warp order, and the
// block partials are summed by the single-block scalar kernels of blas.cu,
// so each reduction rounds the same way for a given vector length.
//
// The conversions between the double-word layout (float4 = re.h, im.h,
// re.l, im.l) and FP64 let the FP64 solver take and return double-word
// vectors: widening is exact (h + l has at most 49 significant bits),
// narrowing rounds each real to the nearest double-word pair.
#include <cuda_runtime.h>

#include "kernels.h"
#include "pdl.cuh"
#include "reduce.cuh"

namespace jqcd {

namespace {

#define GRID_STRIDE(i, n) \
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

__global__ void f64_copy_kernel(double2 *__restrict__ d, const double2 *__restrict__ s, int64_t n) {
  GRID_STRIDE(i, n) d[i] = s[i];
}

__global__ void f64_zero_kernel(double2 *__restrict__ d, int64_t n) {
  GRID_STRIDE(i, n) d[i] = make_double2(0.0, 0.0);
}

__global__ void f64_norm2_kernel(const double2 *__restrict__ a, int64_t n, double *partials) {
  double A = 0.0;
  GRID_STRIDE(i, n) {
    const double2 v = a[i];
    A = fma(v.x, v.x, A);
    A = fma(v.y, v.y, A);
  }
  const double s = block_sum_d(A);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// r = b - y, partials of ||r||^2
__global__ void f64_xmy_norm_kernel(double2 *__restrict__ r, const double2 *__restrict__ b,
                                    const double2 *__restrict__ y, int64_t n, double *partials) {
  double A = 0.0;
  GRID_STRIDE(i, n) {
    const double2 bv = b[i], yv = y[i];
    const double2 v = make_double2(bv.x - yv.x, bv.y - yv.y);
    r[i] = v;
    A = fma(v.x, v.x, A);
    A = fma(v.y, v.y, A);
  }
  const double s = block_sum_d(A);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// x += alpha p, r -= alpha Ap, partials of ||r||^2 (alpha = S->alpha)
__global__ void f64_cg_update_kernel(double2 *__restrict__ x, double2 *__restrict__ r,
                                     const double2 *__restrict__ p, const double2 *__restrict__ Ap,
                                     int64_t n, const SolverScalars *S, double *partials) {
  pdl_enter();
  if (S->halt) return;  // uniform across the grid
  const double al = S->alpha;
  double A = 0.0;
  GRID_STRIDE(i, n) {
    const double2 xv = x[i], pv = p[i], rv = r[i], av = Ap[i];
    x[i] = make_double2(fma(al, pv.x, xv.x), fma(al, pv.y, xv.y));
    const double2 rn = make_double2(fma(-al, av.x, rv.x), fma(-al, av.y, rv.y));
    r[i] = rn;
    A = fma(rn.x, rn.x, A);
    A = fma(rn.y, rn.y, A);
  }
  const double s = block_sum_d(A);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// p = r + beta p (beta = S->beta)
__global__ void f64_xpay_kernel(double2 *__restrict__ p, const double2 *__restrict__ r, int64_t n,
                                const SolverScalars *S) {
  pdl_enter();
  if (S->halt) return;
  const double be = S->beta;
  GRID_STRIDE(i, n) {
    const double2 pv = p[i], rv = r[i];
    p[i] = make_double2(fma(be, pv.x, rv.x), fma(be, pv.y, rv.y));
  }
}

__global__ void dw_to_f64_kernel(double2 *__restrict__ d, const float4 *__restrict__ s, int64_t n) {
  GRID_STRIDE(i, n) {
    const float4 v = s[i];
    d[i] = make_double2((double)v.x + (double)v.z, (double)v.y + (double)v.w);
  }
}

__device__ __forceinline__ float2 split_rn(double v) {
  const float h = __double2float_rn(v);
  return make_float2(h, __double2float_rn(v - (double)h));
}

__global__ void f64_to_dw_kernel(float4 *__restrict__ d, const double2 *__restrict__ s, int64_t n) {
  GRID_STRIDE(i, n) {
    const double2 v = s[i];
    const float2 re = split_rn(v.x), im = split_rn(v.y);
    d[i] = make_float4(re.x, im.x, re.y, im.y);
  }
}

#undef GRID_STRIDE

}  // namespace

cudaError_t launch_f64_copy(double2 *dst, const double2 *src, int64_t n, cudaStream_t s) {
  note_launch();
  f64_copy_kernel<<<blas_blocks(n), kBlasThreads, 0, s>>>(dst, src, n);
  return cudaGetLastError();
}
cudaError_t launch_f64_zero(double2 *dst, int64_t n, cudaStream_t s) {
  note_launch();
  f64_zero_kernel<<<blas_blocks(n), kBlasThreads, 0, s>>>(dst, n);
  return cudaGetLastError();
}
cudaError_t launch_f64_norm2(const double2 *a, int64_t n, double *partials, cudaStream_t s) {
  note_launch();
  f64_norm2_kernel<<<blas_blocks(n), kBlasThreads, 0, s>>>(a, n, partials);
  return cudaGetLastError();
}
cudaError_t launch_f64_xmy_norm(double2 *r, const double2 *b, const double2 *y, int64_t n,
                                double *partials, cudaStream_t s) {
  note_launch();
  f64_xmy_norm_kernel<<<blas_blocks(n), kBlasThreads, 0, s>>>(r, b, y, n, partials);
  return cudaGetLastError();
}
cudaError_t launch_f64_cg_update(double2 *x, double2 *r, const double2 *p, const double2 *Ap,
                                 int64_t n, const SolverScalars *S, double *partials,
                                 cudaStream_t s) {
  note_launch();
  return launch_pdl(f64_cg_update_kernel, blas_blocks(n), kBlasThreads, 0, s, x, r, p, Ap, n, S,
                    partials);
}
cudaError_t launch_f64_xpay(double2 *p, const double2 *r, int64_t n, const SolverScalars *S,
                            cudaStream_t s) {
  note_launch();
  return launch_pdl(f64_xpay_kernel, blas_blocks(n), kBlasThreads, 0, s, p, r, n, S);
}
cudaError_t launch_dw_to_f64(double2 *dst, const float4 *src, int64_t n, cudaStream_t s) {
  note_launch();
  dw_to_f64_kernel<<<blas_blocks(n), kBlasThreads, 0, s>>>(dst, src, n);
  return cudaGetLastError();
}
cudaError_t launch_f64_to_dw(float4 *dst, const double2 *src, int64_t n, cudaStream_t s) {
  note_launch();
  f64_to_dw_kernel<<<blas_blocks(n), kBlasThreads, 0, s>>>(dst, src, n);
  return cudaGetLastError();
}

}  // namespace jqcd
