// Low-precision (FP32 or FP16 with per-site norm; 12-real FP32 links) hop
// for one output site, shared by the single-field kernel (dslash.cu) and the
// batched operator (batch_kernels.cu).
//
// The plain form of this hop waits on every neighbour load in turn (memory
// latency bound: long-scoreboard stalls dominate).  Here the neighbour
// spinor and the link of hop d+1 are copied into shared memory with cp.async
// while hop d computes: two stages of chunk-major [chunk][thread] slots, each
// thread touching only its own column, so no block-wide barrier is needed.
// The eight hops are unrolled, so spin projection, reconstruction and the
// adjoint are resolved at compile time.
#pragma once
#include "fields.cuh"
#include "hop.cuh"
#include "hop_dw.cuh"

namespace jqcd {

template <int PREC> struct LpStage;
template <> struct LpStage<PREC_F32> {
  static constexpr int kSpin = 6;    // six 16-byte spinor chunks
  static constexpr int kChunks = 9;  // + three link chunks
};
template <> struct LpStage<PREC_F16N> {
  static constexpr int kSpin = 4;    // three half chunks + one slot for the site norm
  static constexpr int kChunks = 7;
};
// Dynamic shared memory of a kHopThreads block.
template <int PREC> constexpr size_t lp_stage_smem() {
  return 2ull * LpStage<PREC>::kChunks * kHopThreads * 16;
}

// The FP16 site norm of a stage slot sits in the fourth chunk plane at a
// 4-byte stride (thread t at float t of the plane): one 128-byte wavefront
// per warp to write and to read, where a 16-byte stride took four.  A thread's
// norm is then not in its own column of the plane, so a kernel that mixes
// stage layouts in one buffer must keep every word's owner (lp_hop_site).
__device__ __forceinline__ float *lp_norm_slot(float4 *plane, int tid) {
  return reinterpret_cast<float *>(plane) + tid;
}
// The same from a thread-offset stage pointer (st = stage + tid).
__device__ __forceinline__ float lp_norm_read(const float4 *st_plane_tid, int tid) {
  return reinterpret_cast<const float *>(st_plane_tid - tid)[tid];
}

__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}

// Copies of hop d's neighbour spinor (site nb of the input parity) and link
// (forward: U_mu(idx) of parity p; backward: U_mu(nb) of parity 1-p); the
// link goes to chunk planes LK .. LK + 2 of the stage.
template <int PREC, bool LINK_L1, int LK = LpStage<PREC>::kSpin>
__device__ __forceinline__ void lp_stage_issue(float4 *st, const void *in, const float4 *gauge,
                                               int64_t vh, int p, int64_t idx, int d, int64_t nb) {
  typedef LpStage<PREC> S;
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
  const int mu = d >> 1;
  const bool bwd = (d & 1) != 0;
  const float4 *L = gauge + (size_t)(((bwd ? 1 - p : p) * 4 + mu) * 3) * vh + (bwd ? nb : idx);
#pragma unroll
  for (int k = 0; k < 3; ++k) cp_async16(st + (LK + k) * kHopThreads + tid, L + k * vh, LINK_L1);
}

// Spinor and link of one stage slot (st already offset by the thread).  For
// FP16 the spinor comes back unscaled and *norm holds the site norm (the
// caller scales the projected half-spinor: 12 multiplies instead of 24);
// for FP32 *norm = 1.
template <int PREC, int LK = LpStage<PREC>::kSpin>
__device__ __forceinline__ void lp_stage_read(const float4 *st, cf (&psi)[4][3], cf (&u)[3][3], float *norm) {
  if (PREC == PREC_F32) {
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      const float4 v = st[j * kHopThreads];
      psi[(2 * j) / 3][(2 * j) % 3] = cf{v.x, v.y};
      psi[(2 * j + 1) / 3][(2 * j + 1) % 3] = cf{v.z, v.w};
    }
    *norm = 1.f;
  } else {
    *norm = lp_norm_read(st + 3 * kHopThreads, threadIdx.x);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const uint4 v = reinterpret_cast<const uint4 *>(st)[j * kHopThreads];
      const unsigned w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float2 f = __half22float2(*reinterpret_cast<const __half2 *>(&w[q]));
        const int k = 4 * j + q;
        psi[k / 3][k % 3] = cf{f.x, f.y};
      }
    }
  }
  PT_F32Links::link_from_chunks(st[LK * kHopThreads], st[(LK + 1) * kHopThreads], st[(LK + 2) * kHopThreads],
                                u);
}

// One hop: project, site norm (FP16) and boundary sign, link multiply,
// reconstruct into acc.
template <int PREC, int MU, bool BWD, bool DAG>
__device__ __forceinline__ void lp_apply(const cf (&psi)[4][3], const cf (&u)[3][3], float norm, bool neg,
                                         cf (&acc)[4][3]) {
  constexpr int S = (BWD != DAG) ? 1 : -1;
  cf h[2][3], r[2][3];
  project<MU, S>(psi, h);
  if (PREC == PREC_F16N) {
    const float f = (MU == 3 && neg) ? -norm : norm;
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int c = 0; c < 3; ++c) h[a][c] = cf{h[a][c].re * f, h[a][c].im * f};
  } else if (MU == 3) {
    PT_F32Links::negate_if(h, neg);  // only time hops cross the boundary
  }
  matvec2<BWD>(u, h, r);
  reconstruct<MU, S>(r, acc);
}

// acc = (H_{p,1-p} in)(idx) (DAG: the adjoint hop); smem: this block's
// lp_stage_smem<PREC>() bytes; blockDim.x must be kHopThreads.  C and LK: the
// chunk planes of a stage and the first link plane; a kernel that also runs
// the two-lane hop of hop_lp2.cuh in the same buffer passes that layout's,
// so that every shared-memory word keeps one owner thread in both (the site
// norms are not in their thread's own column).
template <int PREC, bool DAG, bool LINK_L1, int C = LpStage<PREC>::kChunks, int LK = LpStage<PREC>::kSpin>
__device__ __forceinline__ void lp_hop_site(float4 *smem, const void *in, const float4 *gauge,
                                            const Geom &g, int p, int64_t idx, cf (&acc)[4][3]) {
  const int64_t vh = g.vh;
  int x, y, z, t;
  cb_coords(g, idx, p, x, y, z, t);
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c) acc[a][c] = cf{0.f, 0.f};
  const int tid = threadIdx.x;
  bool neg_next;
  int64_t nb = hop_neighbour(g, x, y, z, t, 0, neg_next);
  lp_stage_issue<PREC, LINK_L1, LK>(smem, in, gauge, vh, p, idx, 0, nb);
  cp_async_commit();
#pragma unroll
  for (int d = 0; d < 8; ++d) {
    const bool neg = neg_next;
    if (d < 7) {
      nb = hop_neighbour(g, x, y, z, t, d + 1, neg_next);
      lp_stage_issue<PREC, LINK_L1, LK>(smem + ((d + 1) & 1) * C * kHopThreads, in, gauge, vh, p, idx, d + 1,
                                        nb);
    }
    cp_async_commit();
    cp_async_wait1();  // this thread's copies of hop d have landed
    cf psi[4][3], u[3][3];
    float nrm;
    lp_stage_read<PREC, LK>(smem + (d & 1) * C * kHopThreads + tid, psi, u, &nrm);
    switch (d) {  // d is a constant after unrolling
      case 0: lp_apply<PREC, 0, false, DAG>(psi, u, nrm, neg, acc); break;
      case 1: lp_apply<PREC, 0, true, DAG>(psi, u, nrm, neg, acc); break;
      case 2: lp_apply<PREC, 1, false, DAG>(psi, u, nrm, neg, acc); break;
      case 3: lp_apply<PREC, 1, true, DAG>(psi, u, nrm, neg, acc); break;
      case 4: lp_apply<PREC, 2, false, DAG>(psi, u, nrm, neg, acc); break;
      case 5: lp_apply<PREC, 2, true, DAG>(psi, u, nrm, neg, acc); break;
      case 6: lp_apply<PREC, 3, false, DAG>(psi, u, nrm, neg, acc); break;
      default: lp_apply<PREC, 3, true, DAG>(psi, u, nrm, neg, acc);
    }
  }
}

}  // namespace jqcd
