// Even-odd Wilson hop H_{p,1-p} for one output site, generic over precision.
//
// (H psi)(x) = sum_mu [ (1 - gamma_mu) U_mu(x) psi(x+mu)
//                     + (1 + gamma_mu) U_mu(x-mu)^dag psi(x-mu) ]
// (the hopping term of the Wilson-Dirac operator D = 1 - kappa H; paper,
// "Definition of Dirac operators").  The adjoint hop swaps (1 -/+ gamma_mu).
//
// In the DeGrand-Rossi basis every (1 + s gamma_mu), s = +-1, has rank 2: its
// rows 2 and 3 are phases times rows 1 and 0.  So each neighbour is first
// projected to a two-spin half-spinor h (two complex adds per colour), the
// link multiplies only h, and the result r is spread back to four spins:
//   mu=x: h0 = psi0 + s*i*psi3, h1 = psi1 + s*i*psi2, out2 += -s*i*r1, out3 += -s*i*r0
//   mu=y: h0 = psi0 -   s*psi3, h1 = psi1 +   s*psi2, out2 +=    s*r1, out3 +=   -s*r0
//   mu=z: h0 = psi0 + s*i*psi2, h1 = psi1 - s*i*psi3, out2 += -s*i*r0, out3 +=  s*i*r1
//   mu=t: h0 = psi0 +   s*psi2, h1 = psi1 +   s*psi3, out2 +=    s*r0, out3 +=    s*r1
// (out0 += r0, out1 += r1 always).  Forward hops use s = -1, backward s = +1;
// the adjoint flips both.
#pragma once
#include "dw.cuh"
#include "lattice.cuh"

namespace jqcd {

// ---- complex register types ----------------------------------------------
struct cf { float re, im; };
struct cd { double re, im; };
struct cw { dw re, im; };

// Phase codes: 0 -> +1, 1 -> +i, 2 -> -1, 3 -> -i.
template <int PH> __device__ __forceinline__ cf phase(cf a) {
  if (PH == 0) return a;
  if (PH == 1) return cf{-a.im, a.re};
  if (PH == 2) return cf{-a.re, -a.im};
  return cf{a.im, -a.re};
}
template <int PH> __device__ __forceinline__ cd phase(cd a) {
  if (PH == 0) return a;
  if (PH == 1) return cd{-a.im, a.re};
  if (PH == 2) return cd{-a.re, -a.im};
  return cd{a.im, -a.re};
}
template <int PH> __device__ __forceinline__ cw phase(cw a) {
  if (PH == 0) return a;
  if (PH == 1) return cw{dw_neg(a.im), a.re};
  if (PH == 2) return cw{dw_neg(a.re), dw_neg(a.im)};
  return cw{a.im, dw_neg(a.re)};
}

__device__ __forceinline__ cf cadd(cf a, cf b) { return cf{a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ cd cadd(cd a, cd b) { return cd{a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ cw cadd(cw a, cw b) { return cw{dw_add_u(a.re, b.re), dw_add_u(a.im, b.im)}; }

// accumulate: a += b
__device__ __forceinline__ void cacc(cf &a, cf b) { a.re += b.re; a.im += b.im; }
__device__ __forceinline__ void cacc(cd &a, cd b) { a.re += b.re; a.im += b.im; }
__device__ __forceinline__ void cacc(cw &a, cw b) { dw_accum(a.re, b.re); dw_accum(a.im, b.im); }

__device__ __forceinline__ cf cscale(cf a, float s) { return cf{a.re * s, a.im * s}; }
__device__ __forceinline__ cd cscale(cd a, double s) { return cd{a.re * s, a.im * s}; }
__device__ __forceinline__ cw cscale(cw a, float s) {  // s = +-1 only
  return s < 0 ? cw{dw_neg(a.re), dw_neg(a.im)} : a;
}

// ---- colour mat-vec: r[s] = W h[s], W = U or U^dag -------------------------
template <bool ADJ>
__device__ __forceinline__ void matvec2(const cf (&u)[3][3], const cf (&h)[2][3], cf (&r)[2][3]) {
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      float re = 0.f, im = 0.f;
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        cf w = ADJ ? cf{u[b][a].re, -u[b][a].im} : u[a][b];
        re = fmaf(w.re, h[s][b].re, re);
        re = fmaf(-w.im, h[s][b].im, re);
        im = fmaf(w.re, h[s][b].im, im);
        im = fmaf(w.im, h[s][b].re, im);
      }
      r[s][a] = cf{re, im};
    }
}

template <bool ADJ>
__device__ __forceinline__ void matvec2(const cd (&u)[3][3], const cd (&h)[2][3], cd (&r)[2][3]) {
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      double re = 0., im = 0.;
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        cd w = ADJ ? cd{u[b][a].re, -u[b][a].im} : u[a][b];
        re = fma(w.re, h[s][b].re, re);
        re = fma(-w.im, h[s][b].im, re);
        im = fma(w.re, h[s][b].im, im);
        im = fma(w.im, h[s][b].re, im);
      }
      r[s][a] = cd{re, im};
    }
}

// Double-word: every output real is a 6-term compensated dot product.
template <bool ADJ>
__device__ __forceinline__ void matvec2(const cw (&u)[3][3], const cw (&h)[2][3], cw (&r)[2][3]) {
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      cw w0 = ADJ ? cw{u[0][a].re, dw_neg(u[0][a].im)} : u[a][0];
      dwacc re = acc_first(w0.re, h[s][0].re);
      dwacc im = acc_first(w0.re, h[s][0].im);
      acc_mad(re, dw_neg(w0.im), h[s][0].im);
      acc_mad(im, w0.im, h[s][0].re);
#pragma unroll
      for (int b = 1; b < 3; ++b) {
        cw w = ADJ ? cw{u[b][a].re, dw_neg(u[b][a].im)} : u[a][b];
        acc_mad(re, w.re, h[s][b].re);
        acc_mad(re, dw_neg(w.im), h[s][b].im);
        acc_mad(im, w.re, h[s][b].im);
        acc_mad(im, w.im, h[s][b].re);
      }
      r[s][a] = cw{acc_get(re), acc_get(im)};
    }
}

// ---- projection / reconstruction --------------------------------------------
// Phase codes for (1 + s gamma_mu) with s = +1; s = -1 adds 2 (negation).
// Columns: spin index read into h0 and h1, phases p0, p1 (h_k = psi_k + p*psi_j),
// and the reconstruction sources and phases of out2, out3.
template <int MU> struct SpinTab;
template <> struct SpinTab<0> { enum { j0 = 3, p0 = 1, j1 = 2, p1 = 1, k2 = 1, q2 = 3, k3 = 0, q3 = 3 }; };
template <> struct SpinTab<1> { enum { j0 = 3, p0 = 2, j1 = 2, p1 = 0, k2 = 1, q2 = 0, k3 = 0, q3 = 2 }; };
template <> struct SpinTab<2> { enum { j0 = 2, p0 = 1, j1 = 3, p1 = 3, k2 = 0, q2 = 3, k3 = 1, q3 = 1 }; };
template <> struct SpinTab<3> { enum { j0 = 2, p0 = 0, j1 = 3, p1 = 0, k2 = 0, q2 = 0, k3 = 1, q3 = 0 }; };

// h = (1 + S gamma_mu) psi, rows 0 and 1 (S = +1 or -1); bc = +-1 boundary factor
// is folded into h.
template <int MU, int S, typename C>
__device__ __forceinline__ void project(const C (&psi)[4][3], C (&h)[2][3]) {
  typedef SpinTab<MU> T;
  constexpr int P0 = (T::p0 + (S < 0 ? 2 : 0)) & 3;
  constexpr int P1 = (T::p1 + (S < 0 ? 2 : 0)) & 3;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    h[0][c] = cadd(psi[0][c], phase<P0>(psi[T::j0][c]));
    h[1][c] = cadd(psi[1][c], phase<P1>(psi[T::j1][c]));
  }
}

template <int MU, int S, typename C>
__device__ __forceinline__ void reconstruct(const C (&r)[2][3], C (&acc)[4][3]) {
  typedef SpinTab<MU> T;
  constexpr int Q2 = (T::q2 + (S < 0 ? 2 : 0)) & 3;
  constexpr int Q3 = (T::q3 + (S < 0 ? 2 : 0)) & 3;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    cacc(acc[0][c], r[0][c]);
    cacc(acc[1][c], r[1][c]);
    cacc(acc[2][c], phase<Q2>(r[T::k2][c]));
    cacc(acc[3][c], phase<Q3>(r[T::k3][c]));
  }
}

}  // namespace jqcd
