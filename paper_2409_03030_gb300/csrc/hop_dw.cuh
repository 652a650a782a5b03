// Double-word hop building blocks shared by the single-field and batched
// kernels: projection and reconstruction with runtime signs, neighbour
// lookup, cp.async helpers, per-site norms, and a direct-load hop body.
#pragma once
#include "fields.cuh"
#include "hop.cuh"
#include "kernels.h"

namespace jqcd {

template <int PREC> __device__ __forceinline__ dwacc site_norm2(const typename PT<PREC>::C (&o)[4][3]);
template <> __device__ __forceinline__ dwacc site_norm2<PREC_DW>(const cw (&o)[4][3]) {
  dwacc A = acc_first(o[0][0].re, o[0][0].re);
  acc_sq(A, o[0][0].im);
#pragma unroll
  for (int k = 1; k < 12; ++k) {
    acc_sq(A, o[k / 3][k % 3].re);
    acc_sq(A, o[k / 3][k % 3].im);
  }
  return A;
}
template <> __device__ __forceinline__ dwacc site_norm2<PREC_F64>(const cd (&o)[4][3]) {
  double s = 0.;
#pragma unroll
  for (int k = 0; k < 12; ++k) s += o[k / 3][k % 3].re * o[k / 3][k % 3].re + o[k / 3][k % 3].im * o[k / 3][k % 3].im;
  float h = (float)s;
  return dwacc{h, (float)(s - (double)h)};
}
template <int PREC> __device__ __forceinline__ dwacc site_norm2_f(const cf (&o)[4][3]) {
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < 12; ++k) s = fmaf(o[k / 3][k % 3].re, o[k / 3][k % 3].re, fmaf(o[k / 3][k % 3].im, o[k / 3][k % 3].im, s));
  return dwacc{s, 0.f};
}
template <> __device__ __forceinline__ dwacc site_norm2<PREC_F32>(const cf (&o)[4][3]) { return site_norm2_f<PREC_F32>(o); }
template <> __device__ __forceinline__ dwacc site_norm2<PREC_F16N>(const cf (&o)[4][3]) { return site_norm2_f<PREC_F16N>(o); }

// ---------------------------------------------------------------------------
// Double-word hop: one runtime loop over the eight hops.  The body
// (projection, compensated mat-vec, reconstruction) exists once in the
// instruction stream; the direction only selects a small
// projection/reconstruction case and the neighbour.  A fully unrolled
// double-word body is ~10k instructions per site and does not fit the
// instruction caches.  Forward/backward and dagger signs ride on the FMAs of
// the error-free additions (dw_add_sgn), so they cost nothing.

// h = a + sg * phi * b with phi = 1 (I = false) or i (I = true).
template <bool I> __device__ __forceinline__ cw cadd_ph(const cw &a, const cw &b, float sg) {
  if (I) return cw{dw_add_sgn(a.re, b.im, -sg), dw_add_sgn(a.im, b.re, sg)};
  return cw{dw_add_sgn(a.re, b.re, sg), dw_add_sgn(a.im, b.im, sg)};
}
// acc += sg * phi * r
template <bool I> __device__ __forceinline__ void cacc_ph(cw &acc, const cw &r, float sg) {
  if (I) { acc.re = dw_add_sgn(acc.re, r.im, -sg); acc.im = dw_add_sgn(acc.im, r.re, sg); }
  else { acc.re = dw_add_sgn(acc.re, r.re, sg); acc.im = dw_add_sgn(acc.im, r.im, sg); }
}

// (1 + S gamma_mu) psi, rows 0 and 1, DeGrand-Rossi basis (see hop.cuh).
template <int MU> __device__ __forceinline__ void project_dw(const cw (&psi)[4][3], cw (&h)[2][3], float S) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if (MU == 0) { h[0][c] = cadd_ph<true>(psi[0][c], psi[3][c], S);   h[1][c] = cadd_ph<true>(psi[1][c], psi[2][c], S); }
    if (MU == 1) { h[0][c] = cadd_ph<false>(psi[0][c], psi[3][c], -S); h[1][c] = cadd_ph<false>(psi[1][c], psi[2][c], S); }
    if (MU == 2) { h[0][c] = cadd_ph<true>(psi[0][c], psi[2][c], S);   h[1][c] = cadd_ph<true>(psi[1][c], psi[3][c], -S); }
    if (MU == 3) { h[0][c] = cadd_ph<false>(psi[0][c], psi[2][c], S);  h[1][c] = cadd_ph<false>(psi[1][c], psi[3][c], S); }
  }
}

template <int MU> __device__ __forceinline__ void reconstruct_dw(const cw (&r)[2][3], cw (&acc)[4][3], float S) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    cacc(acc[0][c], r[0][c]);
    cacc(acc[1][c], r[1][c]);
    if (MU == 0) { cacc_ph<true>(acc[2][c], r[1][c], -S);  cacc_ph<true>(acc[3][c], r[0][c], -S); }
    if (MU == 1) { cacc_ph<false>(acc[2][c], r[1][c], S);  cacc_ph<false>(acc[3][c], r[0][c], -S); }
    if (MU == 2) { cacc_ph<true>(acc[2][c], r[0][c], -S);  cacc_ph<true>(acc[3][c], r[1][c], S); }
    if (MU == 3) { cacc_ph<false>(acc[2][c], r[0][c], S);  cacc_ph<false>(acc[3][c], r[1][c], S); }
  }
}

// ---------------------------------------------------------------------------
// Double-word hop with the operands of the next hop prefetched into shared
// memory (cp.async, two stages), so each warp's memory latency overlaps its
// own arithmetic instead of depending on other resident warps.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, bool keep_l1) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  if (keep_l1)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
  else
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// Neighbour of hop d (mu = d/2, backward when d is odd) and its boundary sign.
__device__ __forceinline__ int64_t hop_neighbour(const Geom &g, int x, int y, int z, int t, int d,
                                                 bool &neg) {
  const int mu = d >> 1;
  const bool bwd = (d & 1) != 0;
  neg = false;
  if (!bwd) {
    switch (mu) {
      case 0: x = (x + 1 == g.nx) ? 0 : x + 1; break;
      case 1: y = (y + 1 == g.ny) ? 0 : y + 1; break;
      case 2: z = (z + 1 == g.nz) ? 0 : z + 1; break;
      default: if (t + 1 == g.nt) { t = 0; neg = g.tanti != 0; } else t = t + 1;
    }
  } else {
    switch (mu) {
      case 0: x = (x == 0) ? g.nx - 1 : x - 1; break;
      case 1: y = (y == 0) ? g.ny - 1 : y - 1; break;
      case 2: z = (z == 0) ? g.nz - 1 : z - 1; break;
      default: if (t == 0) { t = g.nt - 1; neg = g.tanti != 0; } else t = t - 1;
    }
  }
  return cb_index(g, x, y, z, t);
}


// (H in)(x) for one output site in double-word arithmetic, one runtime loop
// over the eight hops, operands loaded directly (read-only path for the
// spinor, streaming for the links).  DAG selects the adjoint hop.
template <bool DAG>
__device__ __forceinline__ void dw_hop_site(const float4 *in, const float4 *gauge, const Geom &g,
                                            int p, int64_t idx, cw (&acc)[4][3]) {
  typedef PT<PREC_DW> T;
  int x, y, z, t;
  cb_coords(g, idx, p, x, y, z, t);
  const int64_t vh = g.vh;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c) acc[a][c] = T::zero();
#pragma unroll 1
  for (int d = 0; d < 8; ++d) {
    const int mu = d >> 1;
    const bool bwd = (d & 1) != 0;
    bool neg;
    const int64_t nb = hop_neighbour(g, x, y, z, t, d, neg);
    cw psi[4][3];
    T::load_spinor(in, vh, nb, psi);
    const float S = (bwd != DAG) ? 1.f : -1.f;
    cw h[2][3];
    switch (mu) {
      case 0: project_dw<0>(psi, h, S); break;
      case 1: project_dw<1>(psi, h, S); break;
      case 2: project_dw<2>(psi, h, S); break;
      default: project_dw<3>(psi, h, S);
    }
    if (neg) T::negate_if(h, true);
    const float4 *L = gauge + (size_t)(((bwd ? 1 - p : p) * 4 + mu) * 9) * vh + (bwd ? nb : idx);
    const int sa = bwd ? 1 : 3, sb = bwd ? 3 : 1;
    const float cs = bwd ? -1.f : 1.f;
    cw u[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        dw ur, ui;
        dwc_unpack(__ldcs(L + (int64_t)(a * sa + b * sb) * vh), ur, ui);
        u[a][b] = cw{ur, dw_make(cs * ui.h, cs * ui.l)};
      }
    cw r[2][3];
    matvec2<false>(u, h, r);
    switch (mu) {
      case 0: reconstruct_dw<0>(r, acc, S); break;
      case 1: reconstruct_dw<1>(r, acc, S); break;
      case 2: reconstruct_dw<2>(r, acc, S); break;
      default: reconstruct_dw<3>(r, acc, S);
    }
  }
}

}  // namespace jqcd
