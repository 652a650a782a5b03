// Low-precision hop (FP32 or FP16 with per-site norm; 12-real FP32 links)
// for two right-hand sides on the same gauge field at once, in packed
// two-lane FP32 arithmetic: lane 0 holds the first right-hand side, lane 1
// the second, and every add, multiply and fma of the hop is one
// add/mul/fma.rn.f32x2 for both.  The link is loaded, its third row rebuilt
// and its components broadcast to both lanes once for the pair.  This
// halves the arithmetic instructions per site and right-hand side of the
// batched operator, which is bound by instruction issue once its links are
// shared by a group of right-hand sides.
//
// Staging follows hop_lp.cuh: the next hop's two neighbour spinors and its
// link are copied into shared memory with cp.async while the current hop
// computes (two stages, chunk-major [chunk][thread], each thread touching
// only its own column).
#pragma once
#include "dw2.cuh"
#include "hop_lp.cuh"

namespace jqcd {

// A complex number of each of two right-hand sides: re = (re_0, re_1),
// im = (im_0, im_1).
struct cp2 {
  f2 re, im;
};

template <int PREC> struct Lp2Stage {
  static constexpr int kSpin = LpStage<PREC>::kSpin;   // chunks of one spinor (+ norm slot)
  static constexpr int kChunks = 2 * kSpin + 3;        // two spinors and one link
};
template <int PREC> constexpr size_t lp2_stage_smem() {
  return 2ull * Lp2Stage<PREC>::kChunks * kHopThreads * 16;
}
// The packed kernels fall back to the one-lane site loop in the same buffer,
// laid out as the packed stages (lp_hop_site with C = kChunks, LK = 2 kSpin).

// a + PH * b for a phase code PH (0: +1, 1: +i, 2: -1, 3: -i), lane-wise.
template <int PH> __device__ __forceinline__ cp2 add_phase(cp2 a, cp2 b) {
  if (PH == 0) return cp2{f2_add(a.re, b.re), f2_add(a.im, b.im)};
  if (PH == 1) return cp2{f2_sub(a.re, b.im), f2_add(a.im, b.re)};
  if (PH == 2) return cp2{f2_sub(a.re, b.re), f2_sub(a.im, b.im)};
  return cp2{f2_add(a.re, b.im), f2_sub(a.im, b.re)};
}

// Copies of one spinor of hop d's neighbour site nb into a stage slot.
template <int PREC>
__device__ __forceinline__ void lp2_issue_spinor(float4 *st, const void *in, int64_t vh, int64_t nb) {
  const int tid = threadIdx.x;
  if (PREC == PREC_F32) {
    const float4 *src = reinterpret_cast<const float4 *>(in) + nb;
#pragma unroll
    for (int k = 0; k < 6; ++k) cp_async16(st + k * kHopThreads + tid, src + k * vh, true);
  } else {
    const uint4 *src = reinterpret_cast<const uint4 *>(in);
#pragma unroll
    for (int k = 0; k < 3; ++k) cp_async16(st + k * kHopThreads + tid, src + k * vh + nb, true);
    cp_async4(lp_norm_slot(st + 3 * kHopThreads, tid), reinterpret_cast<const float *>(src + 3 * vh) + nb);
  }
}

template <int PREC>
__device__ __forceinline__ void lp2_issue(float4 *st, const void *in0, const void *in1,
                                          const float4 *gauge, int64_t vh, int p, int64_t idx, int d,
                                          int64_t nb) {
  typedef Lp2Stage<PREC> S;
  lp2_issue_spinor<PREC>(st, in0, vh, nb);
  lp2_issue_spinor<PREC>(st + S::kSpin * kHopThreads, in1, vh, nb);
  const int tid = threadIdx.x;
  const int mu = d >> 1;
  const bool bwd = (d & 1) != 0;
  const float4 *L = gauge + (size_t)(((bwd ? 1 - p : p) * 4 + mu) * 3) * vh + (bwd ? nb : idx);
#pragma unroll
  for (int k = 0; k < 3; ++k) cp_async16(st + (2 * S::kSpin + k) * kHopThreads + tid, L + k * vh, true);
}

// The two spinors of a stage slot (st offset by the thread) as packed
// complex numbers; for FP16 the values come back unscaled and nrm holds the
// two site norms (the caller scales the projected half-spinor).
template <int PREC>
__device__ __forceinline__ void lp2_read_spinors(const float4 *st, cp2 (&psi)[4][3], f2 &nrm) {
  typedef Lp2Stage<PREC> S;
  if (PREC == PREC_F32) {
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      const float4 a = st[j * kHopThreads], b = st[(S::kSpin + j) * kHopThreads];
      psi[(2 * j) / 3][(2 * j) % 3] = cp2{f2_make(a.x, b.x), f2_make(a.y, b.y)};
      psi[(2 * j + 1) / 3][(2 * j + 1) % 3] = cp2{f2_make(a.z, b.z), f2_make(a.w, b.w)};
    }
    nrm = f2_make(1.f, 1.f);
  } else {
    nrm = f2_make(lp_norm_read(st + 3 * kHopThreads, threadIdx.x),
                  lp_norm_read(st + (S::kSpin + 3) * kHopThreads, threadIdx.x));
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const uint4 va = reinterpret_cast<const uint4 *>(st)[j * kHopThreads];
      const uint4 vb = reinterpret_cast<const uint4 *>(st)[(S::kSpin + j) * kHopThreads];
      const unsigned wa[4] = {va.x, va.y, va.z, va.w}, wb[4] = {vb.x, vb.y, vb.z, vb.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float2 fa = __half22float2(*reinterpret_cast<const __half2 *>(&wa[q]));
        const float2 fb = __half22float2(*reinterpret_cast<const __half2 *>(&wb[q]));
        const int k = 4 * j + q;
        psi[k / 3][k % 3] = cp2{f2_make(fa.x, fb.x), f2_make(fa.y, fb.y)};
      }
    }
  }
}

// r[s][a] = sum_b W_ab h[s][b] for both spins, W = u (forward) or u^dag
// (backward), the link's components broadcast to both lanes once per (a, b).
template <bool ADJ>
__device__ __forceinline__ void lp2_matvec(const cf (&u)[3][3], const cp2 (&h)[2][3], cp2 (&r)[2][3]) {
  // the one operand each product needs negated: -h.im (W = u), -h.re (W = u^dag)
  f2 nh[2][3];
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int b = 0; b < 3; ++b) nh[s][b] = f2_neg(ADJ ? h[s][b].re : h[s][b].im);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const cf w = ADJ ? u[b][a] : u[a][b];  // ADJ: conj(u_ba), sign carried by nh
      const f2 wr = f2_make(w.re, w.re), wi = f2_make(w.im, w.im);
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        // W = u:     re += w.re h.re - w.im h.im,  im += w.re h.im + w.im h.re
        // W = u^dag: re += w.re h.re + w.im h.im,  im += w.re h.im - w.im h.re
        if (b == 0) {
          r[s][a].re = f2_mul(wr, h[s][b].re);
          r[s][a].im = f2_mul(wr, h[s][b].im);
        } else {
          r[s][a].re = f2_fma(wr, h[s][b].re, r[s][a].re);
          r[s][a].im = f2_fma(wr, h[s][b].im, r[s][a].im);
        }
        r[s][a].re = f2_fma(wi, ADJ ? h[s][b].im : nh[s][b], r[s][a].re);
        r[s][a].im = f2_fma(wi, ADJ ? nh[s][b] : h[s][b].re, r[s][a].im);
      }
    }
  }
}

// One hop for both right-hand sides: project, scale (FP16 norms, boundary
// sign), link multiply, reconstruct into acc (phases as in hop.cuh).
template <int PREC, int MU, bool BWD, bool DAG>
__device__ __forceinline__ void lp2_apply(const cp2 (&psi)[4][3], const cf (&u)[3][3], f2 nrm, bool neg,
                                          cp2 (&acc)[4][3]) {
  typedef SpinTab<MU> T;
  constexpr int S = (BWD != DAG) ? 1 : -1;
  constexpr int P0 = (T::p0 + (S < 0 ? 2 : 0)) & 3, P1 = (T::p1 + (S < 0 ? 2 : 0)) & 3;
  constexpr int Q2 = (T::q2 + (S < 0 ? 2 : 0)) & 3, Q3 = (T::q3 + (S < 0 ? 2 : 0)) & 3;
  cp2 h[2][3], r[2][3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    h[0][c] = add_phase<P0>(psi[0][c], psi[T::j0][c]);
    h[1][c] = add_phase<P1>(psi[1][c], psi[T::j1][c]);
  }
  if (PREC == PREC_F16N || MU == 3) {
    const f2 f = (MU == 3 && neg) ? f2_neg(nrm) : nrm;
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int c = 0; c < 3; ++c) h[a][c] = cp2{f2_mul(h[a][c].re, f), f2_mul(h[a][c].im, f)};
  }
  lp2_matvec<BWD>(u, h, r);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    acc[0][c] = add_phase<0>(acc[0][c], r[0][c]);
    acc[1][c] = add_phase<0>(acc[1][c], r[1][c]);
    acc[2][c] = add_phase<Q2>(acc[2][c], r[T::k2][c]);
    acc[3][c] = add_phase<Q3>(acc[3][c], r[T::k3][c]);
  }
}

// acc = (H_{p,1-p} in0)(idx) in lane 0 and (H_{p,1-p} in1)(idx) in lane 1
// (DAG: the adjoint hop); smem: this block's lp2_stage_smem<PREC>() bytes;
// blockDim.x must be kHopThreads.
template <int PREC, bool DAG>
__device__ __forceinline__ void lp2_hop_site(float4 *smem, const void *in0, const void *in1,
                                             const float4 *gauge, const Geom &g, int p, int64_t idx,
                                             cp2 (&acc)[4][3]) {
  constexpr int C = Lp2Stage<PREC>::kChunks;
  constexpr int K = Lp2Stage<PREC>::kSpin;
  const int64_t vh = g.vh;
  int x, y, z, t;
  cb_coords(g, idx, p, x, y, z, t);
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c) acc[a][c] = cp2{0ull, 0ull};
  const int tid = threadIdx.x;
  bool neg_next;
  int64_t nb = hop_neighbour(g, x, y, z, t, 0, neg_next);
  lp2_issue<PREC>(smem, in0, in1, gauge, vh, p, idx, 0, nb);
  cp_async_commit();
#pragma unroll
  for (int d = 0; d < 8; ++d) {
    const bool neg = neg_next;
    if (d < 7) {
      nb = hop_neighbour(g, x, y, z, t, d + 1, neg_next);
      lp2_issue<PREC>(smem + ((d + 1) & 1) * C * kHopThreads, in0, in1, gauge, vh, p, idx, d + 1, nb);
    }
    cp_async_commit();
    cp_async_wait1();  // this thread's copies of hop d have landed
    const float4 *st = smem + (d & 1) * C * kHopThreads + tid;
    cp2 psi[4][3];
    f2 nrm;
    lp2_read_spinors<PREC>(st, psi, nrm);
    cf u[3][3];
    PT_F32Links::link_from_chunks(st[(2 * K) * kHopThreads], st[(2 * K + 1) * kHopThreads],
                                  st[(2 * K + 2) * kHopThreads], u);
    switch (d) {  // d is a constant after unrolling
      case 0: lp2_apply<PREC, 0, false, DAG>(psi, u, nrm, neg, acc); break;
      case 1: lp2_apply<PREC, 0, true, DAG>(psi, u, nrm, neg, acc); break;
      case 2: lp2_apply<PREC, 1, false, DAG>(psi, u, nrm, neg, acc); break;
      case 3: lp2_apply<PREC, 1, true, DAG>(psi, u, nrm, neg, acc); break;
      case 4: lp2_apply<PREC, 2, false, DAG>(psi, u, nrm, neg, acc); break;
      case 5: lp2_apply<PREC, 2, true, DAG>(psi, u, nrm, neg, acc); break;
      case 6: lp2_apply<PREC, 3, false, DAG>(psi, u, nrm, neg, acc); break;
      default: lp2_apply<PREC, 3, true, DAG>(psi, u, nrm, neg, acc);
    }
  }
}

// Lane `lane` of a packed spinor as plain complex numbers.
__device__ __forceinline__ void lp2_lane(const cp2 (&v)[4][3], int lane, cf (&o)[4][3]) {
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float r0, r1, i0, i1;
      f2_split(v[a][c].re, r0, r1);
      f2_split(v[a][c].im, i0, i1);
      o[a][c] = lane ? cf{r1, i1} : cf{r0, i0};
    }
}

}  // namespace jqcd
