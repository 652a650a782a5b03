// Last hop of the double-word even-odd normal operator fused with the CG
// update (conjugate gradient on Mhat^dag Mhat, the paper's solve_DinvX! in
// section "Definition of Dirac operators"), for the double-word solver and
// for the FP32 / FP16-with-norm inner solver of the mixed-precision CG.
//
// In one CG iteration alpha = ||r||^2 / <p, Mhat^dag Mhat p> and
// <p, Mhat^dag Mhat p> = ||Mhat p||^2 are known once the second hop has
// formed w = Mhat p.  The fourth hop, Ap = w - k^2 H^dag_eo t, therefore
// applies x += alpha p and r -= alpha Ap at its own site and forms the
// block partial of ||r||^2: Ap never reaches memory and the separate update
// kernel (which read x, r, p, Ap and wrote x, r) is gone.
#include <cuda_runtime.h>

#include "fields.cuh"
#include "hop_dwp.cuh"
#include "hop_lp.cuh"
#include "kernels.h"
#include "pdl.cuh"
#include "cg_steps.cuh"
#include "reduce.cuh"
#include "solver.h"

namespace jqcd {

namespace {

// q = a*w + b*v is (Ap)(idx) for the NC components k0 .. k0 + NC - 1 of the
// site; x += alpha p (XUPD) and r -= alpha q in place; returns their
// contribution to ||r||^2.  Every operand is a 16-byte double-word chunk.
template <bool XUPD, int NC>
__device__ __forceinline__ dwacc dwp_store_cg(const p2 (&v)[NC], int k0, const float4 *__restrict__ w_base,
                                              const float4 *__restrict__ p_base,
                                              float4 *__restrict__ x_base, float4 *__restrict__ r_base,
                                              int64_t vh, int64_t idx, float2 a_split, float2 b_split,
                                              float2 alpha) {
  idx += (int64_t)k0 * vh;
  const mul2 Bm{f2_make(b_split.x, b_split.x), f2_make(b_split.y, b_split.y)};
  const mul2 Am{f2_make(a_split.x, a_split.x), f2_make(a_split.y, a_split.y)};
  const mul2 Al{f2_make(alpha.x, alpha.x), f2_make(alpha.y, alpha.y)};
  const mul2 Ml{f2_neg(Al.h), f2_neg(Al.l)};
  const ulonglong2 *__restrict__ wp = reinterpret_cast<const ulonglong2 *>(w_base) + idx;
  const ulonglong2 *__restrict__ pp = reinterpret_cast<const ulonglong2 *>(p_base) + idx;
  ulonglong2 *__restrict__ xp = reinterpret_cast<ulonglong2 *>(x_base) + idx;
  ulonglong2 *__restrict__ rp = reinterpret_cast<ulonglong2 *>(r_base) + idx;
  acc2 nq{0ull, 0ull};
#pragma unroll
  for (int k = 0; k < NC; ++k) {
    const ulonglong2 wv = __ldg(wp + k * vh), rv = rp[k * vh];
    acc2 R = acc2_first(Bm, p2_norm(v[k]));
    acc2_mad(R, Am, p2{wv.x, wv.y});
    const p2 q = p2_norm(acc2_get(R));
    if (XUPD) {
      const ulonglong2 pv = __ldg(pp + k * vh), xv = xp[k * vh];
      const p2 xn = p2_norm(p2_add(p2{xv.x, xv.y}, acc2_get(acc2_first(Al, p2{pv.x, pv.y}))));
      xp[k * vh] = make_ulonglong2(xn.h, xn.l);
    }
    const p2 rn = p2_norm(p2_add(p2{rv.x, rv.y}, acc2_get(acc2_first(Ml, q))));
    rp[k * vh] = make_ulonglong2(rn.h, rn.l);
    const mul2 Q{rn.h, rn.l};
    if (k == 0) nq = acc2_first(Q, rn);
    else acc2_mad(nq, Q, rn);
  }
  float s0, s1, c0, c1;
  f2_split(nq.s, s0, s1);
  f2_split(nq.c, c0, c1);
  float s, e;
  two_sum(s0, s1, s, e);
  return dwacc{s, __fadd_rn(__fadd_rn(c0, c1), e)};
}

template <bool XUPD, int MINB>
__global__ void __launch_bounds__(kDwp1Threads, MINB)
    hop_dwp_cg_kernel(const HopParams P, const float4 *__restrict__ p, float4 *__restrict__ xs,
                      float4 *__restrict__ r, const float2 *__restrict__ alpha) {
  extern __shared__ float4 dsm[];
  pdl_enter();
  if (P.guard && *P.guard) return;  // uniform across the grid
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  dwacc nrm{0.f, 0.f};
  if (idx < P.g.vh) {
    p2 acc[4][3];
    dwp_hop_site<true, kDwp1Threads>(dsm, reinterpret_cast<const float4 *>(P.in),
                                     reinterpret_cast<const float4 *>(P.gauge), P.g, P.out_parity, idx, acc);
    p2 v[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) v[k] = acc[k / 3][k % 3];
    nrm = dwp_store_cg<XUPD, 12>(v, 0, reinterpret_cast<const float4 *>(P.x), p, xs, r, P.g.vh, idx,
                                 P.a_split, P.b_split, *alpha);
  }
  const double s = block_sum_dw(nrm);
  if (threadIdx.x == 0) P.partials[blockIdx.x] = s;
}

// The same with two threads per output site (small lattices, see
// dwp_pair_combine): thread q updates components 6q .. 6q + 5.
template <bool XUPD>
__global__ void __launch_bounds__(kDwp2Threads, JQCD_DWP2_MIN_BLOCKS)
    hop_dwp2_cg_kernel(const HopParams P, const float4 *__restrict__ p, float4 *__restrict__ xs,
                       float4 *__restrict__ r, const float2 *__restrict__ alpha) {
  extern __shared__ float4 dsm[];
  pdl_enter();
  if (P.guard && *P.guard) return;  // uniform across the grid
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t idx = gid >> 1;
  const int q = (int)(gid & 1);
  const bool active = idx < P.g.vh;
  p2 acc[4][3];
  if (active) {
    dwp_hop_dirs<true, kDwp2Threads>(dsm, reinterpret_cast<const float4 *>(P.in),
                                      reinterpret_cast<const float4 *>(P.gauge), P.g, P.out_parity, idx, q, 2,
                                      4, acc);
  } else {
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c = 0; c < 3; ++c) acc[a][c] = p2{0ull, 0ull};
  }
  p2 o[6];
  dwp_pair_combine(acc, q, o);
  dwacc nrm{0.f, 0.f};
  if (active)
    nrm = dwp_store_cg<XUPD, 6>(o, 6 * q, reinterpret_cast<const float4 *>(P.x), p, xs, r, P.g.vh, idx,
                                P.a_split, P.b_split, *alpha);
  const double s = block_sum_dw(nrm);
  if (threadIdx.x == 0) P.partials[blockIdx.x] = s;
}

// Low-precision form for the inner CG: Ap = a w + b H^dag t in FP32 registers
// (never rounded to the storage precision), then the FP32 update of the
// inner solution xs and residual rs with alpha_f, as the unfused update
// kernel does, and ||rs||^2 per hop block.
template <int PREC>
__global__ void __launch_bounds__(kHopThreads)
    hop_lp_cg_kernel(const HopParams P, const void *__restrict__ p, float4 *__restrict__ xs,
                     float4 *__restrict__ rs, const SolverScalars *__restrict__ S) {
  typedef PT<PREC> T;
  extern __shared__ float4 lsm[];
  pdl_enter();
  if (P.guard && *P.guard) return;  // uniform across the grid
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  float n2 = 0.f;
  if (idx < P.g.vh) {
    cf acc[4][3];
    lp_hop_site<PREC, true, false>(lsm, P.in, reinterpret_cast<const float4 *>(P.gauge), P.g,
                                   P.out_parity, idx, acc);
    const float a = (float)P.a, b = (float)P.b, al = S->alpha_f;
    cf w[4][3], pv[4][3], xv[4][3], rv[4][3];
    T::load_spinor(P.x, P.g.vh, idx, w);
    T::load_spinor(p, P.g.vh, idx, pv);
    PT<PREC_F32>::load_spinor(xs, P.g.vh, idx, xv);
    PT<PREC_F32>::load_spinor(rs, P.g.vh, idx, rv);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      const cf q = T::axpby(a, w[k / 3][k % 3], b, acc[k / 3][k % 3]);
      cf &x = xv[k / 3][k % 3], &r = rv[k / 3][k % 3];
      const cf pp = pv[k / 3][k % 3];
      x.re = fmaf(al, pp.re, x.re);
      x.im = fmaf(al, pp.im, x.im);
      r.re = fmaf(-al, q.re, r.re);
      r.im = fmaf(-al, q.im, r.im);
      n2 = fmaf(r.re, r.re, fmaf(r.im, r.im, n2));
    }
    PT<PREC_F32>::store_spinor(xs, P.g.vh, idx, xv);
    PT<PREC_F32>::store_spinor(rs, P.g.vh, idx, rv);
  }
  const double s = block_sum_f(n2);
  if (threadIdx.x == 0) P.partials[blockIdx.x] = s;
  if (P.fin) hop_finish_scalars(P);  // uniform over the grid
}

template <int PREC>
cudaError_t launch_lp_cg_t(const HopParams &P, const void *p, float4 *xs, float4 *rs,
                           const SolverScalars *S, cudaStream_t s) {
  return launch_pdl(hop_lp_cg_kernel<PREC>, hop_blocks(P.g.vh), kHopThreads, lp_stage_smem<PREC>(), s, P, p,
                    xs, rs, S);
}

}  // namespace

cudaError_t launch_hop_lp_cg(int prec, const HopParams &P, const void *p, float4 *xs, float4 *rs,
                             const SolverScalars *S, cudaStream_t s) {
  note_launch();
  if (P.fin && (!P.fin_S || hop_blocks(P.g.vh) > (unsigned)JQCD_FIN_MAX_BLOCKS)) return cudaErrorInvalidValue;
  switch (prec) {
    case PREC_F32: return launch_lp_cg_t<PREC_F32>(P, p, xs, rs, S, s);
    case PREC_F16N: return launch_lp_cg_t<PREC_F16N>(P, p, xs, rs, S, s);
    default: return cudaErrorInvalidValue;
  }
}

template <bool XUPD>
static cudaError_t launch_dw_cg_t(const HopParams &P, const float4 *p, float4 *x, float4 *r, const float2 *alpha,
                                  cudaStream_t s) {
  note_launch();
  static bool configured = false;  // one attribute call per instantiation
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(hop_dwp_cg_kernel<XUPD, JQCD_DWP_MIN_BLOCKS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDwp1Smem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(hop_dwp_cg_kernel<XUPD, JQCD_DWP_SMALL_MIN_BLOCKS>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDwp1Smem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(hop_dwp2_cg_kernel<XUPD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)kDwp2Smem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  if (dw_hop_split(P.g.vh))
    return launch_pdl(hop_dwp2_cg_kernel<XUPD>, dw_hop_blocks(P.g.vh), kDwp2Threads, kDwp2Smem, s, P, p, x,
                      r, alpha);
  if (dw_hop_small(P.g.vh))
    return launch_pdl(hop_dwp_cg_kernel<XUPD, JQCD_DWP_SMALL_MIN_BLOCKS>, dw_hop_blocks(P.g.vh), kDwp1Threads,
                      kDwp1Smem, s, P, p, x, r, alpha);
  return launch_pdl(hop_dwp_cg_kernel<XUPD, JQCD_DWP_MIN_BLOCKS>, dw_hop_blocks(P.g.vh), kDwp1Threads, kDwp1Smem,
                    s, P, p, x, r, alpha);
}

cudaError_t launch_hop_dw_cg(const HopParams &P, const float4 *p, float4 *x, float4 *r,
                             const SolverScalars *S, cudaStream_t s) {
  return launch_dw_cg_t<true>(P, p, x, r, &S->alpha_dw, s);
}

cudaError_t launch_hop_dw_r(const HopParams &P, float4 *r, const float2 *alpha_dw, cudaStream_t s) {
  return launch_dw_cg_t<false>(P, nullptr, nullptr, r, alpha_dw, s);
}

}  // namespace jqcd
