// Double-word ("double-float") arithmetic on the FP32 pipes.
//
// A value is the unevaluated sum h + l of two floats with |l| <= ulp(h)
// (after normalisation); the pair carries about 48 significant bits, so the
// relative representation error of an FP64 input is below 2^-48.  GB300's
// native FP64 rate is about 1/58 of its FP32 rate, so FP64-accurate stencil
// and vector arithmetic runs here on error-free transformations of FP32
// operations instead of on DFMA:
//   TwoSum (Knuth 1969, 6 flops), Fast2Sum (Dekker 1971, 3 flops) and
//   TwoProd with FMA (2 flops), combined as in the double-word algorithms of
//   Joldes, Muller and Popescu (ACM TOMS 2017) and the compensated dot
//   product of Ogita, Rump and Oishi (SIAM J. Sci. Comput. 2005).
// Every primitive uses the __f*_rn intrinsics, which the compiler never
// contracts into FMAs: contraction would destroy the exactness of TwoSum.
#pragma once
#include <cuda_runtime.h>

namespace jqcd {

struct dw {
  float h, l;
};

__device__ __forceinline__ dw dw_make(float h, float l) { dw r; r.h = h; r.l = l; return r; }
__device__ __forceinline__ dw dw_neg(dw a) { return dw_make(-a.h, -a.l); }

// s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// s + e == a + b exactly, requires |a| >= |b| (or a == 0).
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ dw dw_norm(float h, float l) {
  float s, e;
  fast_two_sum(h, l, s, e);
  return dw_make(s, e);
}

// a + b, result left unnormalised (|l| may reach a few ulp(h)); error is a
// few units of 2^-48 relative to |a| + |b|.
__device__ __forceinline__ dw dw_add_u(dw a, dw b) {
  float s, e;
  two_sum(a.h, b.h, s, e);
  return dw_make(s, __fadd_rn(__fadd_rn(a.l, b.l), e));
}
__device__ __forceinline__ dw dw_sub_u(dw a, dw b) { return dw_add_u(a, dw_neg(b)); }
__device__ __forceinline__ dw dw_add(dw a, dw b) {
  dw r = dw_add_u(a, b);
  return dw_norm(r.h, r.l);
}

// a * b (normalised).
__device__ __forceinline__ dw dw_mul(dw a, dw b) {
  float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  return dw_norm(p, e);
}

// Compensated accumulator for sums of products: the exact products of the
// high parts are summed with TwoSum into s; every rounding error, the
// products' low halves and the cross terms go to c.  Result s + c.
struct dwacc {
  float s, c;
};

__device__ __forceinline__ dwacc acc_first(dw a, dw b) {
  dwacc A;
  A.s = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -A.s);
  e = __fmaf_rn(a.h, b.l, e);
  A.c = __fmaf_rn(a.l, b.h, e);
  return A;
}

__device__ __forceinline__ void acc_mad(dwacc &A, dw a, dw b) {
  float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  float c = __fmaf_rn(a.h, b.l, A.c);
  c = __fmaf_rn(a.l, b.h, c);
  float s, t;
  two_sum(A.s, p, s, t);
  A.s = s;
  A.c = __fadd_rn(__fadd_rn(c, e), t);
}

__device__ __forceinline__ dw acc_get(dwacc A) { return dw_make(A.s, A.c); }  // unnormalised

// x += v for an unnormalised running sum.
__device__ __forceinline__ void dw_accum(dw &x, dw v) {
  float s, e;
  two_sum(x.h, v.h, s, e);
  x.h = s;
  x.l = __fadd_rn(__fadd_rn(x.l, v.l), e);
}

// a + s*b for s = +1 or -1, unnormalised.  The sign rides on FMAs, which are
// exact here (s*b is exact), so TwoSum keeps its error-free property.
__device__ __forceinline__ dw dw_add_sgn(dw a, dw b, float s) {
  const float sum = __fmaf_rn(s, b.h, a.h);
  const float bb = __fsub_rn(sum, a.h);
  const float e = __fadd_rn(__fsub_rn(a.h, __fsub_rn(sum, bb)), __fmaf_rn(s, b.h, -bb));
  return dw_make(sum, __fadd_rn(__fmaf_rn(s, b.l, a.l), e));
}

// x += s*v for s = +1 or -1 (running sum, unnormalised).
__device__ __forceinline__ void dw_accum_sgn(dw &x, dw v, float s) { x = dw_add_sgn(x, v, s); }

// Square-accumulate a*a into (s, c) (for norms).
__device__ __forceinline__ void acc_sq(dwacc &A, dw a) { acc_mad(A, a, a); }

// A complex double-word number in one 16-byte chunk, laid out
// (re.h, im.h, re.l, im.l) so that the high and the low halves each form an
// aligned pair of floats (packed two-lane FP32 arithmetic reads them as is).
__device__ __forceinline__ void dwc_unpack(float4 v, dw &re, dw &im) {
  re = dw_make(v.x, v.z);
  im = dw_make(v.y, v.w);
}
__device__ __forceinline__ float4 dwc_pack(dw re, dw im) { return make_float4(re.h, im.h, re.l, im.l); }

__host__ __device__ __forceinline__ float2 dw_split_host(double v) {
  float h = (float)v;
  float l = (float)(v - (double)h);
  return make_float2(h, l);
}

}  // namespace jqcd
