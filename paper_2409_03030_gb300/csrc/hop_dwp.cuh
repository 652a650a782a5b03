// Double-word hop in packed two-lane arithmetic, shared by the single-field
// kernel (dslash.cu) and the batched reliable-update stages (batch_kernels.cu).
//
// Every complex double-word operation runs its real and imaginary lanes in
// one fma/add/mul.rn.f32x2: projection and reconstruction by sign-carrying
// TwoSums, the SU(3) product W h = h.re W + i (h.im W) as sums of exact
// products on a fixed offset grid with broadcast half-spinor multipliers.  (Folding the link's signs into the
// multipliers instead saves FP32 multiplies but costs registers: the kernel
// then spills and runs slower on sm_103.)
//
// Neighbour spinors and links of the next hop are prefetched into shared
// memory with cp.async (chunk-major [k][thread], each thread touching only
// its own column).
#pragma once
#include "dw2.cuh"
#include "hop_dw.cuh"

namespace jqcd {

constexpr int kDwpStageChunks = 12;  // one double-word spinor per thread
constexpr int kDwpLinkChunks = 9;    // one double-word link per thread and stage
// one neighbour-spinor stage and two link stages, chunk-major [k][thread],
// for blocks of nt threads
constexpr size_t dwp_smem(int nt = kHopThreads) {
  return (size_t)(kDwpStageChunks + 2 * kDwpLinkChunks) * nt * 16;
}
constexpr size_t kDwpSmem = dwp_smem();

// Launch shapes of the single-field kernels: threads per block and the
// resident blocks per SM their register budget is cut for, one thread per
// output site (DWP) and two (DWP2, small lattices).  One-warp blocks spread
// a small lattice's split grid over more SMs (measured on GB300: 8^4 hop
// 7.35 -> 5.87 us, 12^4 10.9 -> 8.85 us against 128-thread blocks).  The
// one-thread kernel keeps 128: with one-warp blocks its plain hop ran 1%
// faster at 24^3x48 but the solve 1.2% slower (four times the norm partials).
#ifndef JQCD_DWP_THREADS
#define JQCD_DWP_THREADS 128
#endif
#ifndef JQCD_DWP_MIN_BLOCKS
#define JQCD_DWP_MIN_BLOCKS 3
#endif
// Lattices whose one-thread grid fits in SMs x JQCD_DWP_SMALL_MIN_BLOCKS
// blocks (16^4) run the same kernel compiled for that many blocks per SM:
// the register budget, not the occupancy, limits them there.
#ifndef JQCD_DWP_SMALL_MIN_BLOCKS
#define JQCD_DWP_SMALL_MIN_BLOCKS 2
#endif
#ifndef JQCD_DWP2_THREADS
#define JQCD_DWP2_THREADS 32
#endif
#ifndef JQCD_DWP2_MIN_BLOCKS
#define JQCD_DWP2_MIN_BLOCKS 12
#endif
constexpr int kDwp1Threads = JQCD_DWP_THREADS;
constexpr size_t kDwp1Smem = dwp_smem(kDwp1Threads);
constexpr int kDwp2Threads = JQCD_DWP2_THREADS;
constexpr size_t kDwp2Smem = dwp_smem(kDwp2Threads);

// Issue the copies of the neighbour spinor of one hop into its stage (NT:
// threads per block, the stride of the chunk-major stage).
template <int NT = kHopThreads>
__device__ __forceinline__ void stage_hop_p(float4 *st, const float4 *in, int64_t vh, int64_t nb) {
  const int tid = threadIdx.x;
#pragma unroll
  for (int k = 0; k < 12; ++k) cp_async16(st + k * NT + tid, in + k * vh + nb, true);
}

// Issue the copies of the link of hop d (mu = d/2, backward when d is odd)
// into a link stage, element (a, b) at chunk 3a + b: U_mu(x) for a forward
// hop, the transpose of U_mu(x - mu) (conjugated at use) for a backward one.
template <int NT = kHopThreads>
__device__ __forceinline__ void stage_link_p(float4 *st, const float4 *gauge, int64_t vh, int p, int d,
                                             int64_t idx, int64_t nb) {
  const int tid = threadIdx.x;
  const int mu = d >> 1;
  const bool bwd = (d & 1) != 0;
  const float4 *L = gauge + (size_t)(((bwd ? 1 - p : p) * 4 + mu) * 9) * vh + (bwd ? nb : idx);
  const int sa = bwd ? 1 : 3, sb = bwd ? 3 : 1;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b)
      cp_async16(st + (a * 3 + b) * NT + tid, L + (int64_t)(a * sa + b * sb) * vh, false);
}

__device__ __forceinline__ p2 ld_p2(const float4 *p) {
  const ulonglong2 v = *reinterpret_cast<const ulonglong2 *>(p);
  return p2{v.x, v.y};
}

// (1 + S gamma_mu) psi, rows 0 and 1, DeGrand-Rossi basis.  With phi = i the
// swapped operand (im, re) carries the lane signs (-S, S).
template <int MU>
__device__ __forceinline__ void project_p(const p2 (&psi)[4][3], p2 (&h)[2][3], float S) {
  const f2 sS = f2_make(S, S), nS = f2_make(-S, -S), sI = f2_make(-S, S), sIm = f2_make(S, -S);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if (MU == 0) { h[0][c] = p2_add_sgn(psi[0][c], p2_swap(psi[3][c]), sI); h[1][c] = p2_add_sgn(psi[1][c], p2_swap(psi[2][c]), sI); }
    if (MU == 1) { h[0][c] = p2_add_sgn(psi[0][c], psi[3][c], nS);          h[1][c] = p2_add_sgn(psi[1][c], psi[2][c], sS); }
    if (MU == 2) { h[0][c] = p2_add_sgn(psi[0][c], p2_swap(psi[2][c]), sI); h[1][c] = p2_add_sgn(psi[1][c], p2_swap(psi[3][c]), sIm); }
    if (MU == 3) { h[0][c] = p2_add_sgn(psi[0][c], psi[2][c], sS);          h[1][c] = p2_add_sgn(psi[1][c], psi[3][c], sS); }
  }
}

// r[a] = sum_b W_ab h[b] with TwoSum-compensated sums of exact products
// (twelve packed operations per product, error about 2^-48 |W||h|): the
// accumulation of the staggered hop, which is bound by HBM bandwidth.
__device__ __forceinline__ void matvec_half_ts(const p2 (&W)[3][3], const p2 (&h)[3], p2 (&r)[3]) {
  mul2 mr[3], mi[3];
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    mr[b] = mul2{f2_lo(h[b].h), f2_lo(h[b].l)};
    mi[b] = mul2{f2_hi(h[b].h), f2_hi(h[b].l)};
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    acc2 A = acc2_first(mr[0], W[a][0]);
    acc2 B = acc2_first(mi[0], W[a][0]);
#pragma unroll
    for (int b = 1; b < 3; ++b) {
      acc2_mad(A, mr[b], W[a][b]);
      acc2_mad(B, mi[b], W[a][b]);
    }
    // i B = (-B.im, B.re): swap the lanes, flip the sign of lane 0
    constexpr f2 kLane0 = 0x0000000080000000ull;
    r[a] = p2_add(acc2_get(A), p2{f2_swap(B.s) ^ kLane0, f2_swap(B.c) ^ kLane0});
  }
}

// Largest |component| of the link's high words, the bound its products need.
__device__ __forceinline__ float link_max_hi(const p2 (&W)[3][3]) {
  float m = 0.f;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    float u, v;
    f2_split(W[k / 3][k % 3].h, u, v);
    m = fmaxf(m, fmaxf(fabsf(u), fabsf(v)));
  }
  return m;
}

// One exact-product step of an offset-grid sum: T = T0 + (partial sum) stays
// in the binade [sigma, 2 sigma), so the fma rounds the exact high product
// onto that binade's fixed grid, T - T_new is exact (Sterbenz lemma) and one
// more fma returns the part of the product below the grid to the low-order
// sum c, together with the two cross products of the low words.
__device__ __forceinline__ void grid_mad(f2 &T, f2 &c, const mul2 &A, p2 B, bool first) {
  const f2 Tn = f2_fma(A.h, B.h, T);
  const f2 d = f2_fma(A.h, B.h, f2_sub(T, Tn));  // product - (Tn - T), rounded
  f2 t = first ? d : f2_add(c, d);
  t = f2_fma(A.h, B.l, t);
  c = f2_fma(A.l, B.h, t);
  T = Tn;
}

// r[a] = sum_b W_ab h[b] = A + i B with A = sum_b h.re W_ab and
// B = sum_b h.im W_ab for one spin of the half-spinor (half-spinor
// components broadcast to both lanes against the same link lanes).  Both
// sums run on one fixed grid: sigma is a power of two with every partial sum
// below sigma/2 in magnitude (bound wmax * max(sum_b |h_b.re|, sum_b |h_b.im|),
// raised by 2^-19 to cover its own rounding and that of the grid steps); A
// starts at (T0, T0) and B at (-T0, T0), T0 = 1.5 sigma, so every
// accumulator lane stays in a binade of magnitude [sigma, 2 sigma).  The
// high words of A + i B = (A.re - B.im, A.im + B.re) are then differences of
// two such lanes with the offsets cancelling: exact, multiples of the grid
// step below sigma in magnitude.  The low words carry everything below the
// grid.  Six packed
// operations per product instead of the twelve of a TwoSum accumulation; the
// low words are coarser (about 2^-48 sigma per operation), giving a
// relative error of a few 1e-14 per product W h.
__device__ __forceinline__ void matvec_half_p(const p2 (&W)[3][3], float wmax, const p2 (&h)[3],
                                              p2 (&r)[3]) {
  mul2 mr[3], mi[3];
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    mr[b] = mul2{f2_lo(h[b].h), f2_lo(h[b].l)};
    mi[b] = mul2{f2_hi(h[b].h), f2_hi(h[b].l)};
  }
  f2 TA0, TB0;
  {
    float r0, i0, r1, i1, r2, i2;
    f2_split(h[0].h, r0, i0);
    f2_split(h[1].h, r1, i1);
    f2_split(h[2].h, r2, i2);
    const float sr = fabsf(r0) + fabsf(r1) + fabsf(r2);
    const float si = fabsf(i0) + fabsf(i1) + fabsf(i2);
    const float m = fmaxf(sr, si) * wmax;
    // sigma = 2^(e + 2) for m in [2^e, 2^(e+1)); T0 = 1.5 sigma
    const unsigned tb = (__float_as_uint(m) & 0x7f800000u) + (2u << 23) + (1u << 22);
    const float t0 = __uint_as_float(tb);
    TA0 = f2_make(t0, t0);
    TB0 = f2_make(-t0, t0);
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    f2 TA = TA0, TB = TB0, cA = 0ull, cB = 0ull;
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      grid_mad(TA, cA, mr[b], W[a][b], b == 0);
      grid_mad(TB, cB, mi[b], W[a][b], b == 0);
    }
    // i B = (-B.im, B.re): swap the lanes, flip the sign of lane 0; the high
    // lanes are (T0 + A.re) - (T0 + B.im) and (T0 + A.im) + (-T0 + B.re)
    constexpr f2 kLane0 = 0x0000000080000000ull;
    r[a] = p2{f2_add(TA, f2_swap(TB) ^ kLane0), f2_add(cA, f2_swap(cB) ^ kLane0)};
  }
}

// Reconstruction of one spin s of the two-spin result: out_s += r and the
// lower spin that (1 + S gamma_mu) ties to s gets the phase times r.
template <int MU, int SP>
__device__ __forceinline__ void reconstruct_half_p(const p2 (&r)[3], p2 (&acc)[4][3], float S) {
  const f2 sS = f2_make(S, S), nS = f2_make(-S, -S), sI = f2_make(-S, S), sIm = f2_make(S, -S);
  constexpr int L = (MU <= 1) ? 3 - SP : 2 + SP;  // lower spin fed by spin SP
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    acc[SP][c] = p2_add(acc[SP][c], r[c]);
    if (MU == 0) acc[L][c] = p2_add_sgn(acc[L][c], p2_swap(r[c]), sIm);
    if (MU == 1) acc[L][c] = p2_add_sgn(acc[L][c], r[c], SP == 0 ? nS : sS);
    if (MU == 2) acc[L][c] = p2_add_sgn(acc[L][c], p2_swap(r[c]), SP == 0 ? sIm : sI);
    if (MU == 3) acc[L][c] = p2_add_sgn(acc[L][c], r[c], sS);
  }
}

template <int SP>
__device__ __forceinline__ void reconstruct_half_mu(int mu, const p2 (&r)[3], p2 (&acc)[4][3], float S) {
  switch (mu) {
    case 0: reconstruct_half_p<0, SP>(r, acc, S); break;
    case 1: reconstruct_half_p<1, SP>(r, acc, S); break;
    case 2: reconstruct_half_p<2, SP>(r, acc, S); break;
    default: reconstruct_half_p<3, SP>(r, acc, S);
  }
}

// acc = the sum over the hops d = d0, d0 + dstep, ... (nd of them; hop d
// has mu = d/2 and is backward when d is odd) of H_{p,1-p} in at output site
// idx of parity p (DAG: the adjoint hop), unnormalised double-word
// accumulators.  All eight hops (d0 = 0, dstep = 1, nd = 8) give
// (H_{p,1-p} in)(idx).  dsm: this block's kDwpSmem bytes of shared memory;
// blockDim.x must be NT.
//
// Copies run one hop ahead: the links of the next hop are issued when hop d
// starts (two link stages), the neighbour spinor of the next hop as soon as
// hop d's has been read into registers and projected (one stage).  Every
// thread reads and overwrites only its own column, so no block barrier is
// needed; the completed-group wait of each hop covers both of its copies.
template <bool DAG, int NT = kHopThreads>
__device__ __forceinline__ void dwp_hop_dirs(float4 *dsm, const float4 *in, const float4 *gauge,
                                             const Geom &g, int p, int64_t idx, int d0, int dstep,
                                             int nd, p2 (&acc)[4][3]) {
  const int64_t vh = g.vh;
  int x, y, z, t;
  cb_coords(g, idx, p, x, y, z, t);
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c) acc[a][c] = p2{0ull, 0ull};
  const int tid = threadIdx.x;
  float4 *const lnk = dsm + kDwpStageChunks * NT;  // two link stages
  bool neg_next;
  int64_t nb = hop_neighbour(g, x, y, z, t, d0, neg_next);
  stage_hop_p<NT>(dsm, in, vh, nb);
  stage_link_p<NT>(lnk, gauge, vh, p, d0, idx, nb);
  cp_async_commit();
#pragma unroll 1
  for (int j = 0; j < nd; ++j) {
    const int d = d0 + j * dstep;
    const bool neg = neg_next;
    const int mu = d >> 1;
    const bool bwd = (d & 1) != 0;
    const bool more = j + 1 < nd;
    if (more) {  // the other link stage was read during the previous hop
      nb = hop_neighbour(g, x, y, z, t, d + dstep, neg_next);
      stage_link_p<NT>(lnk + ((j + 1) & 1) * kDwpLinkChunks * NT, gauge, vh, p, d + dstep, idx, nb);
    }
    cp_async_commit();
    cp_async_wait1();  // this thread's spinor and link copies of hop d have landed
    p2 psi[4][3];
#pragma unroll
    for (int k = 0; k < 12; ++k) psi[k / 3][k % 3] = ld_p2(dsm + k * NT + tid);
    p2 W[3][3];
    {
      const float4 *ls = lnk + (j & 1) * kDwpLinkChunks * NT + tid;
#pragma unroll
      for (int k = 0; k < 9; ++k) W[k / 3][k % 3] = ld_p2(ls + k * NT);
    }
    const float S = (bwd != DAG) ? 1.f : -1.f;
    p2 h[2][3];
    switch (mu) {
      case 0: project_p<0>(psi, h, S); break;
      case 1: project_p<1>(psi, h, S); break;
      case 2: project_p<2>(psi, h, S); break;
      default: project_p<3>(psi, h, S);
    }
    if (more) stage_hop_p<NT>(dsm, in, vh, nb);  // the spinor stage has been read
    cp_async_commit();
    if (neg) {
      const f2 mm = f2_make(-1.f, -1.f);
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) h[a][c] = p2_scale_sgn(h[a][c], mm);
    }
    if (bwd) {
      // conjugation of the adjoint link on backward hops only, by sign bits
      // (off the FMA pipe: 1.4% faster than multiplying every link by (1, +-1))
#pragma unroll
      for (int k = 0; k < 9; ++k) W[k / 3][k % 3] = p2_conj(W[k / 3][k % 3]);
    }
    // bound of the link's high words, raised by 2^-19 (see matvec_half_p)
    const float wmax = link_max_hi(W) * 1.0000019f;
    {  // spin 0 of the half-spinor, then spin 1: one three-colour result live
      p2 r[3];
      matvec_half_p(W, wmax, h[0], r);
      reconstruct_half_mu<0>(mu, r, acc, S);
      matvec_half_p(W, wmax, h[1], r);
      reconstruct_half_mu<1>(mu, r, acc, S);
    }
  }
}

// (H_{p,1-p} in)(idx): all eight hops in one thread.
template <bool DAG, int NT = kHopThreads>
__device__ __forceinline__ void dwp_hop_site(float4 *dsm, const float4 *in, const float4 *gauge,
                                             const Geom &g, int p, int64_t idx, p2 (&acc)[4][3]) {
  dwp_hop_dirs<DAG, NT>(dsm, in, gauge, g, p, idx, 0, 1, 8, acc);
}

// Two threads per output site (lanes 2i and 2i + 1 of a warp, q = lane & 1):
// thread q runs the forward (q = 0) or backward (q = 1) hops of the four
// directions, then the pair exchanges partial sums so that thread q holds
// the whole result of spins 2q and 2q + 1, components 6q .. 6q + 5 in the
// order of the spinor layout.  Every lane of the warp must call this.
__device__ __forceinline__ void dwp_pair_combine(const p2 (&acc)[4][3], int q, p2 (&o)[6]) {
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const p2 up = acc[k / 3][k % 3], dn = acc[2 + k / 3][k % 3];
    const p2 keep = q ? dn : up, send = q ? up : dn;
    p2 recv;
    recv.h = __shfl_xor_sync(0xffffffffu, send.h, 1);
    recv.l = __shfl_xor_sync(0xffffffffu, send.l, 1);
    o[k] = p2_add(keep, recv);
  }
}

// out = a x + b v (AXPY) or b v for NC consecutive components k0 .. k0 + NC - 1
// of the site's spinor, each scalar a double-word (hi, lo) float pair;
// returns their contribution to ||out||^2 when NORM.
template <bool AXPY, bool NORM, int NC>
__device__ __forceinline__ dwacc dwp_store_chunks(const p2 (&v)[NC], int k0, float4 *out_base,
                                                  const float4 *x_base, int64_t vh, int64_t idx,
                                                  float2 a_split, float2 b_split) {
  const f2 bh = f2_make(b_split.x, b_split.x);
  const mul2 Bm{bh, f2_make(b_split.y, b_split.y)};
  const f2 ah = f2_make(a_split.x, a_split.x);
  const mul2 Am{ah, f2_make(a_split.y, a_split.y)};
  acc2 nq{0ull, 0ull};
  ulonglong2 *__restrict__ o = reinterpret_cast<ulonglong2 *>(out_base) + idx + (int64_t)k0 * vh;
  p2 xs[NC];
  if (AXPY) {  // all loads before the first store
    const ulonglong2 *__restrict__ xp =
        reinterpret_cast<const ulonglong2 *>(x_base) + idx + (int64_t)k0 * vh;
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      const ulonglong2 u = __ldg(xp + k * vh);
      xs[k] = p2{u.x, u.y};
    }
  }
#pragma unroll
  for (int k = 0; k < NC; ++k) {
    acc2 R = acc2_first(Bm, p2_norm(v[k]));
    if (AXPY) acc2_mad(R, Am, xs[k]);
    const p2 q = p2_norm(acc2_get(R));
    o[k * vh] = make_ulonglong2(q.h, q.l);
    if (NORM) {
      const mul2 Q{q.h, q.l};
      if (k == 0) nq = acc2_first(Q, q);
      else acc2_mad(nq, Q, q);
    }
  }
  dwacc nrm{0.f, 0.f};
  if (NORM) {
    float s0, s1, c0, c1;
    f2_split(nq.s, s0, s1);
    f2_split(nq.c, c0, c1);
    float s, e;
    two_sum(s0, s1, s, e);
    nrm = dwacc{s, __fadd_rn(__fadd_rn(c0, c1), e)};
  }
  return nrm;
}

// out = a x + b acc (AXPY) or b acc for the whole site; returns ||out||^2
// when NORM.
template <bool AXPY, bool NORM>
__device__ __forceinline__ dwacc dwp_store(const p2 (&acc)[4][3], float4 *out_base,
                                           const float4 *x_base, int64_t vh, int64_t idx,
                                           float2 a_split, float2 b_split) {
  p2 v[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) v[k] = acc[k / 3][k % 3];
  return dwp_store_chunks<AXPY, NORM, 12>(v, 0, out_base, x_base, vh, idx, a_split, b_split);
}

}  // namespace jqcd
