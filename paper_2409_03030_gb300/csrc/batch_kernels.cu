// Kernels of the batched mixed-precision CG (see batch.h).
//
// Tile kernels are persistent: block b handles tiles b, b + gridDim.x, ...
// of the device tile list; a tile is tile_sites consecutive sites (one per
// thread) of one group of right-hand sides sharing a gauge field.  Per-slot
// kernels run one block per slot.  Every skip condition below depends only on
// values all threads of a block read alike, so block reductions stay
// convergent.
#include <cuda_runtime.h>

#include "batch.h"
#include "hop_dw.cuh"
#include "hop_dwp.cuh"
#include "hop_lp.cuh"
#include "hop_lp2.cuh"
#include "reduce.cuh"

namespace jqcd {

__device__ __forceinline__ bool slot_running(const BatchArgs &A, int si) {
  return A.slots[si].active && !A.S[si].halt;
}

// Low-precision hop stages of the batched operator.  Work items are
// (slot, block of 128 sites); consecutive items are the right-hand sides of
// one group on the same sites, so their link loads meet in L2.  The site
// loop (hop_lp.cuh) prefetches the next hop's neighbour and link into shared
// memory while the current hop computes.
// STAGE 0: t = H_oe p;  1: w = p - kappa^2 H_eo t, ||w||^2;  2: t = H^dag_oe w;
// STAGE 3: Ap = w - kappa^2 H^dag_eo t, then (UPDATE) x_s += alpha p,
//          r_s -= alpha Ap, ||r_s||^2 without storing Ap.
// The per-site epilogue of a low-precision stage for one slot: acc is
// (H in)(idx); AXPY stages add the slot's own operand, stage 3 with UPDATE
// applies x_s += alpha p, r_s -= alpha Ap; returns this site's part of the
// stage's norm (NORM stages).
template <int PREC, int STAGE, bool UPDATE>
__device__ __forceinline__ float lp_stage_epilogue(const cf (&acc)[4][3], const SlotDev &Sl,
                                                   const SolverScalars &Ss, int64_t vh, int64_t idx) {
  constexpr bool AXPY = STAGE == 1 || STAGE == 3;
  constexpr bool NORM = STAGE == 1 || (STAGE == 3 && UPDATE);
  float n2 = 0.f;
  const void *xv = STAGE == 1 ? Sl.p : Sl.w;
  void *out = STAGE == 0 || STAGE == 2 ? Sl.t : (STAGE == 1 ? Sl.w : Sl.Ap);
      cf o[4][3];
      if (AXPY) {
        cf xs[4][3];
        PT<PREC>::load_spinor(xv, vh, idx, xs);
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int c = 0; c < 3; ++c) o[a][c] = PT<PREC>::axpby(1.f, xs[a][c], Sl.k2, acc[a][c]);
      } else {
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int c = 0; c < 3; ++c) o[a][c] = acc[a][c];
      }
      if (STAGE == 3 && UPDATE) {
        const float al = Ss.alpha_f;
        cf pv[4][3], xv4[4][3], rv[4][3];
        PT<PREC>::load_spinor(Sl.p, vh, idx, pv);
        PT<PREC_F32>::load_spinor(Sl.xs, vh, idx, xv4);
        PT<PREC_F32>::load_spinor(Sl.rs, vh, idx, rv);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
          cf &xq = xv4[k / 3][k % 3], &rq = rv[k / 3][k % 3];
          const cf pp = pv[k / 3][k % 3], aa = o[k / 3][k % 3];
          xq.re = fmaf(al, pp.re, xq.re);
          xq.im = fmaf(al, pp.im, xq.im);
          rq.re = fmaf(-al, aa.re, rq.re);
          rq.im = fmaf(-al, aa.im, rq.im);
          n2 = fmaf(rq.re, rq.re, fmaf(rq.im, rq.im, n2));
        }
        PT<PREC_F32>::store_spinor(Sl.xs, vh, idx, xv4);
        PT<PREC_F32>::store_spinor(Sl.rs, vh, idx, rv);
      } else {
        PT<PREC>::store_spinor(out, vh, idx, o);
        if (NORM) {
#pragma unroll
          for (int k = 0; k < 12; ++k)
            n2 = fmaf(o[k / 3][k % 3].re, o[k / 3][k % 3].re, fmaf(o[k / 3][k % 3].im, o[k / 3][k % 3].im, n2));
        }
      }
  return n2;
}

// SINGLES: walk the single-slot items beside the packed kernel (lp1_tiles),
// else every slot's items (lp_tiles).
template <int PREC, int STAGE, bool UPDATE, bool SINGLES>
__global__ void __launch_bounds__(kLpThreads) batch_lp_hop_kernel(const BatchArgs A) {
  extern __shared__ float4 lsm[];
  constexpr bool DAG = STAGE >= 2;
  constexpr int OUTP = (STAGE == 0 || STAGE == 2) ? 1 : 0;
  constexpr bool NORM = STAGE == 1 || (STAGE == 3 && UPDATE);
  const int n = SINGLES ? *A.n_lp1_tiles : *A.n_lp_tiles;
  const int2 *items = SINGLES ? A.lp1_tiles : A.lp_tiles;
  // the next item is loaded while this one computes (a block's items are
  // gridDim.x apart, each one a fresh L2 access at the head of a chain of
  // dependent descriptor loads)
  int2 Wnext = blockIdx.x < n ? items[blockIdx.x] : make_int2(0, 0);
  for (int it = blockIdx.x; it < n; it += gridDim.x) {
    const int2 W = Wnext;
    if (it + (int)gridDim.x < n) Wnext = items[it + gridDim.x];
    // single items carry the slot itself; the others (group, slot in group)
    const int si = SINGLES ? W.x : A.groups[W.x >> 4].slot[W.x & 15];
    if (!slot_running(A, si)) continue;  // uniform over the block
    const SlotDev &Sl = A.slots[si];
    const Geom g = Sl.g;
    const int64_t idx = (int64_t)W.y * kLpThreads + threadIdx.x;
    float n2 = 0.f;
    if (idx < g.vh) {
      const void *in = STAGE == 0 ? Sl.p : (STAGE == 2 ? Sl.w : Sl.t);
      cf acc[4][3];
      // a single solve's links are read once per site: streamed past L1
      lp_hop_site<PREC, DAG, !SINGLES>(lsm, in, Sl.gauge_f32, g, OUTP, idx, acc);
      n2 = lp_stage_epilogue<PREC, STAGE, UPDATE>(acc, Sl, A.S[si], g.vh, idx);
    }
    if (NORM) {
      const double sum = block_sum_f(n2);
      if (threadIdx.x == 0) Sl.part[W.y] = sum;
    }
  }
}

// The same stages for two right-hand sides of a group per work item, in
// packed two-lane arithmetic (hop_lp2.cuh): items are (group, first slot of
// a pair, block of kLpThreads sites) from the pair list lp2_tiles.  An item
// with a single running slot (an odd group, or a pair one of whose solves
// has stopped) takes the one-lane site loop of hop_lp.cuh.
// Resident blocks per SM the packed kernels' register budget is cut for.
// Measured (ncu launch lists of the 24-solve batch, serialised): FP16 inner
// operator 236 ms with one right-hand side per thread (5 blocks/SM), 267 ms
// packed at 3 blocks/SM (155-168 registers), 222 ms packed at 4 blocks/SM
// (128 registers, 8-160 B spilled); FP32 297, 300 and 277 ms.
#ifndef JQCD_BATCH_LP2_MIN_BLOCKS
#define JQCD_BATCH_LP2_MIN_BLOCKS 4
#endif
template <int PREC, int STAGE, bool UPDATE>
__global__ void __launch_bounds__(kLpThreads, JQCD_BATCH_LP2_MIN_BLOCKS) batch_lp2_hop_kernel(const BatchArgs A) {
  extern __shared__ float4 lsm[];
  constexpr bool DAG = STAGE >= 2;
  constexpr int OUTP = (STAGE == 0 || STAGE == 2) ? 1 : 0;
  constexpr bool NORM = STAGE == 1 || (STAGE == 3 && UPDATE);
  const int n = *A.n_lp2_tiles;
  int2 Wnext = blockIdx.x < n ? A.lp2_tiles[blockIdx.x] : make_int2(0, 0);  // loaded one item ahead
  for (int it = blockIdx.x; it < n; it += gridDim.x) {
    const int2 W = Wnext;
    if (it + (int)gridDim.x < n) Wnext = A.lp2_tiles[it + gridDim.x];
    const GroupDev *G = A.groups + (W.x >> 4);
    const int r0 = W.x & 15;
    const int s0 = G->slot[r0];
    const int s1 = r0 + 1 < G->nslots ? G->slot[r0 + 1] : -1;
    const bool run0 = slot_running(A, s0), run1 = s1 >= 0 && slot_running(A, s1);
    if (!run0 && !run1) continue;  // uniform over the block
    const int sa = run0 ? s0 : s1;
    const int sb = run0 && run1 ? s1 : sa;
    const bool two = run0 && run1;
    const SlotDev &S0 = A.slots[sa], &S1 = A.slots[sb];
    const Geom g = G->g;
    const int64_t idx = (int64_t)W.y * kLpThreads + threadIdx.x;
    float n2a = 0.f, n2b = 0.f;
    if (idx < g.vh) {
      const void *in0 = STAGE == 0 ? S0.p : (STAGE == 2 ? S0.w : S0.t);
      cf acc[4][3];
      if (two) {
        const void *in1 = STAGE == 0 ? S1.p : (STAGE == 2 ? S1.w : S1.t);
        cp2 acc2[4][3];
        lp2_hop_site<PREC, DAG>(lsm, in0, in1, G->gauge_f32, g, OUTP, idx, acc2);
        lp2_lane(acc2, 0, acc);
        n2a = lp_stage_epilogue<PREC, STAGE, UPDATE>(acc, S0, A.S[sa], g.vh, idx);
        lp2_lane(acc2, 1, acc);
        n2b = lp_stage_epilogue<PREC, STAGE, UPDATE>(acc, S1, A.S[sb], g.vh, idx);
      } else {  // a single running slot: the one-lane site loop
        lp_hop_site<PREC, DAG, true, Lp2Stage<PREC>::kChunks, 2 * Lp2Stage<PREC>::kSpin>(lsm, in0, G->gauge_f32,
                                                                                     g, OUTP, idx, acc);
        n2a = lp_stage_epilogue<PREC, STAGE, UPDATE>(acc, S0, A.S[sa], g.vh, idx);
      }
    }
    if (NORM) {
      const double sum0 = block_sum_f(n2a);
      if (threadIdx.x == 0) S0.part[W.y] = sum0;
      if (two) {
        const double sum1 = block_sum_f(n2b);
        if (threadIdx.x == 0) S1.part[W.y] = sum1;
      }
    }
  }
}

// p = r_s + beta p for running slots (CONVERT = false) or, after a reliable
// update, r_s = FP32(r) and then p = r_s + beta p (CONVERT = true).
template <int PREC, bool CONVERT>
__global__ void __launch_bounds__(256) batch_xpay_kernel(const BatchArgs A) {
  if (CONVERT && *A.any_update == 0) return;
  const int tid = threadIdx.x, bd = blockDim.x;
  const int nt = *A.ntiles;
  for (int ti = blockIdx.x; ti < nt; ti += gridDim.x) {
    const int2 T = A.tiles[ti];
    const GroupDev *G = A.groups + T.x;
    const int64_t vh = G->g.vh;
    const int64_t i = (int64_t)T.y * bd + tid;
    if (i >= vh) continue;
    for (int s = 0; s < G->nslots; ++s) {
      const int si = G->slot[s];
      const SlotDev &Sl = A.slots[si];
      if (CONVERT) {
        if (!Sl.active || A.S[si].need_update != 2) continue;
      } else if (!slot_running(A, si)) {
        continue;
      }
      const float b = A.S[si].beta_f;
      cf rv[4][3], pv[4][3];
      if (CONVERT) {
        const float4 *r = Sl.r + i;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
          const float4 v = r[k * vh];
          rv[k / 3][k % 3] = cf{v.x, v.y};  // normalised pairs: hi = nearest float
        }
        PT<PREC_F32>::store_spinor(Sl.rs, vh, i, rv);
      } else {
        PT<PREC_F32>::load_spinor(Sl.rs, vh, i, rv);
      }
      PT<PREC>::load_spinor(Sl.p, vh, i, pv);
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        cf &q = pv[k / 3][k % 3];
        q.re = fmaf(b, q.re, rv[k / 3][k % 3].re);
        q.im = fmaf(b, q.im, rv[k / 3][k % 3].im);
      }
      PT<PREC>::store_spinor(Sl.p, vh, i, pv);
    }
  }
}

// ---- reliable updates (slots with need_update == 1) ---------------------------

// x_e += x_s; x_s = 0
__global__ void __launch_bounds__(256) batch_dw_add_kernel(const BatchArgs A) {
  if (*A.any_update == 0) return;
  const int tid = threadIdx.x, bd = blockDim.x;
  const int nt = *A.ntiles;
  for (int ti = blockIdx.x; ti < nt; ti += gridDim.x) {
    const int2 T = A.tiles[ti];
    const GroupDev *G = A.groups + T.x;
    const int64_t vh = G->g.vh;
    const int64_t i = (int64_t)T.y * bd + tid;
    if (i >= vh) continue;
    for (int s = 0; s < G->nslots; ++s) {
      const int si = G->slot[s];
      const SlotDev &Sl = A.slots[si];
      if (!Sl.active || A.S[si].need_update != 1) continue;
      cf xv[4][3];
      PT<PREC_F32>::load_spinor(Sl.xs, vh, i, xv);
      float4 *x = Sl.x + i;
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        dw re, im;
        dwc_unpack(x[k * vh], re, im);
        re = dw_add(re, dw_make(xv[k / 3][k % 3].re, 0.f));
        im = dw_add(im, dw_make(xv[k / 3][k % 3].im, 0.f));
        x[k * vh] = dwc_pack(re, im);
      }
      float4 *xs = Sl.xs + i;
#pragma unroll
      for (int j = 0; j < 6; ++j) xs[j * vh] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
}

// Double-word Mhat^dag Mhat x in four stages (as the low-precision stages, on
// x, tdw, wdw, Adw) for the slots that asked for a reliable update.  Work
// items are those of the low-precision stages (slot, kLpThreads sites); the
// site loop is the packed double-word hop of the single-field kernel.
static_assert(kLpThreads == kHopThreads, "batched double-word stages reuse the hop staging");

template <int STAGE>
__global__ void __launch_bounds__(kLpThreads, 3) batch_dw_hop_kernel(const BatchArgs A) {
  extern __shared__ float4 dsm[];
  if (*A.any_update == 0) return;
  constexpr bool DAG = STAGE >= 2;
  constexpr int OUTP = (STAGE == 0 || STAGE == 2) ? 1 : 0;
  constexpr bool AXPY = STAGE == 1 || STAGE == 3;
  const int n = *A.n_lp_tiles;
  for (int it = blockIdx.x; it < n; it += gridDim.x) {
    const int2 W = A.lp_tiles[it];
    const GroupDev *G = A.groups + (W.x >> 4);
    const int si = G->slot[W.x & 15];
    const SlotDev &Sl = A.slots[si];
    if (!Sl.active || A.S[si].need_update != 1) continue;  // uniform over the block
    const int64_t idx = (int64_t)W.y * kLpThreads + threadIdx.x;
    if (idx >= G->g.vh) continue;  // no block-wide step follows
    const float4 *in = STAGE == 0 ? Sl.x : (STAGE == 2 ? Sl.wdw : Sl.tdw);
    const float4 *xv = STAGE == 1 ? Sl.x : Sl.wdw;
    float4 *out = STAGE == 0 || STAGE == 2 ? Sl.tdw : (STAGE == 1 ? Sl.wdw : Sl.Adw);
    p2 acc[4][3];
    dwp_hop_site<DAG>(dsm, in, G->gauge_dw, G->g, OUTP, idx, acc);
    dwp_store<AXPY, false>(acc, out, xv, G->g.vh, idx, make_float2(1.f, 0.f),
                           AXPY ? Sl.k2_dw : make_float2(1.f, 0.f));  // t = H v;  w = v - kappa^2 H t
  }
}

// r = rhs - Adw, partial ||r||^2
__global__ void __launch_bounds__(256) batch_dw_resid_kernel(const BatchArgs A) {
  if (*A.any_update == 0) return;
  const int tid = threadIdx.x, bd = blockDim.x;
  const int nt = *A.ntiles;
  for (int ti = blockIdx.x; ti < nt; ti += gridDim.x) {
    const int2 T = A.tiles[ti];
    const GroupDev *G = A.groups + T.x;
    const int64_t vh = G->g.vh;
    const int64_t i = (int64_t)T.y * bd + tid;
    for (int s = 0; s < G->nslots; ++s) {
      const int si = G->slot[s];
      const SlotDev &Sl = A.slots[si];
      if (!Sl.active || A.S[si].need_update != 1) continue;
      dwacc n2{0.f, 0.f};
      if (i < vh) {
#pragma unroll
        for (int k = 0; k < 12; ++k) {
          dw br, bi, yr, yi;
          dwc_unpack(Sl.rhs[k * vh + i], br, bi);
          dwc_unpack(Sl.Adw[k * vh + i], yr, yi);
          const dw re = dw_add(br, dw_neg(yr));
          const dw im = dw_add(bi, dw_neg(yi));
          Sl.r[k * vh + i] = dwc_pack(re, im);
          acc_sq(n2, re);
          acc_sq(n2, im);
        }
      }
      const double sum = block_sum_dw(n2);
      if (tid == 0) Sl.part[T.y] = sum;
    }
  }
}

// ---- per-slot scalar steps (one block per slot) --------------------------------
__device__ __forceinline__ double slot_sum(const SlotDev &Sl, int n) {
  double v = 0.0;
  // all of a thread's loads are in flight before its first add; the adds keep
  // the fixed order i = tid, tid + blockDim.x, ... (out-of-range slots add 0)
  constexpr int kU = 16;
  for (int base = threadIdx.x; base < n; base += kU * blockDim.x) {
    double t[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int i = base + u * (int)blockDim.x;
      t[u] = i < n ? Sl.part[i] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) v += t[u];
  }
  return block_sum_d(v);
}

__global__ void batch_alpha_kernel(const BatchArgs A) {
  const int si = blockIdx.x;
  if (si >= A.nslots || !slot_running(A, si)) return;
  const double pAp = slot_sum(A.slots[si], A.slots[si].nblk_lp);
  if (threadIdx.x == 0) {
    SolverScalars *S = A.S + si;
    S->pAp = pAp;
    if (!(pAp > 0.0) || !isfinite(pAp)) { S->done = 2; S->halt = 1; return; }
    const double a = S->rr / pAp;
    S->alpha = a;
    S->alpha_f = (float)a;
  }
}

__global__ void batch_beta_kernel(const BatchArgs A) {
  const int si = blockIdx.x;
  if (si >= A.nslots || !slot_running(A, si)) return;
  const double rr_new = slot_sum(A.slots[si], A.slots[si].nblk_lp);
  if (threadIdx.x == 0) {
    SolverScalars *S = A.S + si;
    S->rr_new = rr_new;
    S->iters += 1;
    if (!isfinite(rr_new)) { S->done = 2; S->halt = 1; return; }
    if (rr_new <= S->stop_rr || rr_new < S->delta2 * S->rr_max || S->iters >= S->max_iters) {
      S->need_update = 1;
      S->halt = 1;
      *A.any_update = 1;
      return;
    }
    const double b = rr_new / S->rr;
    S->beta = b;
    S->beta_f = (float)b;
    S->rr = rr_new;
    if (rr_new > S->rr_max) S->rr_max = rr_new;
  }
}

__global__ void batch_after_update_kernel(const BatchArgs A) {
  if (*A.any_update == 0) return;
  const int si = blockIdx.x;
  if (si >= A.nslots || !A.slots[si].active || A.S[si].need_update != 1) return;
  const double rr_true = slot_sum(A.slots[si], A.slots[si].nblocks);
  if (threadIdx.x == 0) {
    SolverScalars *S = A.S + si;
    S->reliable_updates += 1;
    S->true_rr = rr_true;
    S->need_update = 0;
    if (!isfinite(rr_true)) { S->done = 2; return; }
    if (rr_true <= S->stop_rr) { S->rr = rr_true; S->done = 1; return; }
    if (S->iters >= S->max_iters) { S->rr = rr_true; S->done = 3; return; }
    const double b = rr_true / S->rr;
    S->beta = b;
    S->beta_f = (float)b;
    S->rr = rr_true;
    S->rr_max = rr_true;
    S->need_update = 2;  // convert the residual, then resume
  }
}

__global__ void batch_resume_kernel(const BatchArgs A) {
  const int si = blockIdx.x;
  if (si < A.nslots && threadIdx.x == 0 && A.slots[si].active && A.S[si].need_update == 2) {
    A.S[si].need_update = 0;
    A.S[si].halt = 0;
  }
  if (si == 0 && threadIdx.x == 0) *A.any_update = 0;
}

// ---- launchers -------------------------------------------------------------------
template <int PREC>
static cudaError_t configure_lp2() {
  const void *k[5] = {(const void *)batch_lp2_hop_kernel<PREC, 0, false>,
                      (const void *)batch_lp2_hop_kernel<PREC, 1, false>,
                      (const void *)batch_lp2_hop_kernel<PREC, 2, false>,
                      (const void *)batch_lp2_hop_kernel<PREC, 3, false>,
                      (const void *)batch_lp2_hop_kernel<PREC, 3, true>};
  for (const void *f : k) {
    const cudaError_t e =
        cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lp2_stage_smem<PREC>());
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t batch_configure() {
  const void *k[4] = {(const void *)batch_dw_hop_kernel<0>, (const void *)batch_dw_hop_kernel<1>,
                      (const void *)batch_dw_hop_kernel<2>, (const void *)batch_dw_hop_kernel<3>};
  for (const void *f : k) {
    const cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDwpSmem);
    if (e != cudaSuccess) return e;
  }
  cudaError_t e = configure_lp2<PREC_F32>();
  if (e == cudaSuccess) e = configure_lp2<PREC_F16N>();
  return e;
}

int batch_lp_blocks_per_sm(int hp) {
  int n = 0;
  const cudaError_t e =
      hp == PREC_F16N
          ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_lp2_hop_kernel<PREC_F16N, 0, false>,
                                                          kLpThreads, lp2_stage_smem<PREC_F16N>())
          : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_lp2_hop_kernel<PREC_F32, 0, false>,
                                                          kLpThreads, lp2_stage_smem<PREC_F32>());
  return (e == cudaSuccess && n > 0) ? n : 2;
}

// One low-precision stage: with pairing, the packed kernel over the pair
// items and the one-lane kernel over the single items (a group's odd last
// slot: in serving, most groups hold one solve); else the one-lane kernel
// over every slot's items.
template <int PREC, int STAGE, bool UPDATE>
static void lp_stage(const BatchArgs &A, const LpGrids &lp, cudaStream_t s) {
  if (kBatchLpPairs) {
    note_launch(2);
    batch_lp2_hop_kernel<PREC, STAGE, UPDATE><<<lp.pairs, kLpThreads, lp2_stage_smem<PREC>(), s>>>(A);
    batch_lp_hop_kernel<PREC, STAGE, UPDATE, true><<<lp.singles, kLpThreads, lp_stage_smem<PREC>(), s>>>(A);
  } else {
    note_launch();
    batch_lp_hop_kernel<PREC, STAGE, UPDATE, false><<<lp.all, kLpThreads, lp_stage_smem<PREC>(), s>>>(A);
  }
}

template <int PREC>
static cudaError_t iteration(const BatchArgs &A, int ts, int grid, const LpGrids &lp, cudaStream_t s) {
  const int lp_grid = lp.all;
  lp_stage<PREC, 0, false>(A, lp, s);
  lp_stage<PREC, 1, false>(A, lp, s);
  note_launch();
  batch_alpha_kernel<<<A.nslots, kReduceThreads, 0, s>>>(A);
  lp_stage<PREC, 2, false>(A, lp, s);
  lp_stage<PREC, 3, true>(A, lp, s);  // Ap and the x_s, r_s update
  note_launch();
  batch_beta_kernel<<<A.nslots, kReduceThreads, 0, s>>>(A);
  note_launch();
  batch_xpay_kernel<PREC, false><<<grid, ts, 0, s>>>(A);
  // reliable updates of the slots that asked for one (no-ops otherwise)
  note_launch();
  batch_dw_add_kernel<<<grid, ts, 0, s>>>(A);
  note_launch();
  batch_dw_hop_kernel<0><<<lp_grid, kLpThreads, kDwpSmem, s>>>(A);
  note_launch();
  batch_dw_hop_kernel<1><<<lp_grid, kLpThreads, kDwpSmem, s>>>(A);
  note_launch();
  batch_dw_hop_kernel<2><<<lp_grid, kLpThreads, kDwpSmem, s>>>(A);
  note_launch();
  batch_dw_hop_kernel<3><<<lp_grid, kLpThreads, kDwpSmem, s>>>(A);
  note_launch();
  batch_dw_resid_kernel<<<grid, ts, 0, s>>>(A);
  note_launch();
  batch_after_update_kernel<<<A.nslots, kReduceThreads, 0, s>>>(A);
  note_launch();
  batch_xpay_kernel<PREC, true><<<grid, ts, 0, s>>>(A);
  note_launch();
  batch_resume_kernel<<<A.nslots, 32, 0, s>>>(A);
  return cudaGetLastError();
}

static bool valid(const LpGrids &lp) { return lp.all >= 1 && lp.pairs >= 1 && lp.singles >= 1; }

cudaError_t launch_batch_iteration(const BatchArgs &A, int hp, int tile_sites, int grid,
                                   const LpGrids &lp, cudaStream_t s) {
  if (tile_sites < 32 || tile_sites > 256 || (tile_sites & 31) || grid < 1 || !valid(lp))
    return cudaErrorInvalidValue;
  return hp == PREC_F16N ? iteration<PREC_F16N>(A, tile_sites, grid, lp, s)
                         : iteration<PREC_F32>(A, tile_sites, grid, lp, s);
}

cudaError_t launch_batch_lp_apply(const BatchArgs &A, int hp, const LpGrids &lp, cudaStream_t s) {
  if (!valid(lp)) return cudaErrorInvalidValue;
  if (hp == PREC_F16N) {
    lp_stage<PREC_F16N, 0, false>(A, lp, s);
    lp_stage<PREC_F16N, 1, false>(A, lp, s);
    lp_stage<PREC_F16N, 2, false>(A, lp, s);
    lp_stage<PREC_F16N, 3, false>(A, lp, s);
  } else {
    lp_stage<PREC_F32, 0, false>(A, lp, s);
    lp_stage<PREC_F32, 1, false>(A, lp, s);
    lp_stage<PREC_F32, 2, false>(A, lp, s);
    lp_stage<PREC_F32, 3, false>(A, lp, s);
  }
  return cudaGetLastError();
}

}  // namespace jqcd
