// Packed double-word arithmetic: two FP32 lanes per 64-bit register pair,
// using the packed fma/add/mul.rn.f32x2 instructions of sm_100-family GPUs
// (one instruction per two lanes, same FP32 datapath rate).  A complex
// double-word number is held as p2{h = (re.h, im.h), l = (re.l, im.l)}, which
// is exactly how a 16-byte double-word chunk is laid out in memory.
// The error-free transformations are those of dw.cuh applied lane-wise.
#pragma once
#include <cuda_runtime.h>

#include "dw.cuh"

namespace jqcd {

typedef unsigned long long f2;  // lane 0 = low 32 bits, lane 1 = high 32 bits

__device__ __forceinline__ f2 f2_make(float a, float b) {
  f2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void f2_split(f2 v, float &a, float &b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ f2 f2_add(f2 a, f2 b) {
  f2 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2 f2_sub(f2 a, f2 b) {
  f2 d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2 f2_mul(f2 a, f2 b) {
  f2 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2 f2_fma(f2 a, f2 b, f2 c) {
  f2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ f2 f2_swap(f2 v) {
  float a, b;
  f2_split(v, a, b);
  return f2_make(b, a);
}
__device__ __forceinline__ f2 f2_lo(f2 v) {  // (lane0, lane0)
  float a, b;
  f2_split(v, a, b);
  return f2_make(a, a);
}
__device__ __forceinline__ f2 f2_hi(f2 v) {  // (lane1, lane1)
  float a, b;
  f2_split(v, a, b);
  return f2_make(b, b);
}
__device__ __forceinline__ f2 f2_neg(f2 v) { return v ^ 0x8000000080000000ull; }

struct p2 {
  f2 h, l;
};

// Lane-wise TwoSum: s + e == a + b exactly in each lane.
__device__ __forceinline__ void two_sum2(f2 a, f2 b, f2 &s, f2 &e) {
  s = f2_add(a, b);
  const f2 bb = f2_sub(s, a);
  e = f2_add(f2_sub(a, f2_sub(s, bb)), f2_sub(b, bb));
}

// a + sg*b lane-wise, sg = +-1 per lane (exact product), unnormalised.
__device__ __forceinline__ p2 p2_add_sgn(p2 a, p2 b, f2 sg) {
  const f2 sb = f2_mul(sg, b.h);
  f2 s, e;
  two_sum2(a.h, sb, s, e);
  return p2{s, f2_add(f2_fma(sg, b.l, a.l), e)};
}
__device__ __forceinline__ p2 p2_add(p2 a, p2 b) {
  f2 s, e;
  two_sum2(a.h, b.h, s, e);
  return p2{s, f2_add(f2_add(a.l, b.l), e)};
}
__device__ __forceinline__ p2 p2_norm(p2 a) {  // Fast2Sum per lane
  const f2 s = f2_add(a.h, a.l);
  return p2{s, f2_sub(a.l, f2_sub(s, a.h))};
}
__device__ __forceinline__ p2 p2_swap(p2 a) { return p2{f2_swap(a.h), f2_swap(a.l)}; }
__device__ __forceinline__ p2 p2_scale_sgn(p2 a, f2 sg) { return p2{f2_mul(sg, a.h), f2_mul(sg, a.l)}; }
// complex conjugate of a double-word complex number: the sign bits of both
// words' imaginary lanes flipped (integer ALU, no floating-point operation)
__device__ __forceinline__ p2 p2_conj(p2 a) {
  constexpr f2 kLane1Sign = 0x8000000000000000ull;
  return p2{a.h ^ kLane1Sign, a.l ^ kLane1Sign};
}

// Compensated accumulator pair: sum of exact high products in s (TwoSum),
// every error and low-order term in c.
struct acc2 {
  f2 s, c;
};
// A = multiplier (h, l), B = multiplicand.  The error of the high product
// is e = fma(A.h, B.h, -p), exact; the negation is a sign flip of p.
struct mul2 {
  f2 h, l;
};
__device__ __forceinline__ acc2 acc2_first(const mul2 &A, p2 B) {
  acc2 R;
  R.s = f2_mul(A.h, B.h);
  const f2 e = f2_fma(A.h, B.h, f2_neg(R.s));  // A.h*B.h - s, exact
  const f2 c = f2_fma(A.h, B.l, e);
  R.c = f2_fma(A.l, B.h, c);
  return R;
}
__device__ __forceinline__ void acc2_mad(acc2 &R, const mul2 &A, p2 B) {
  const f2 p = f2_mul(A.h, B.h);
  const f2 e = f2_fma(A.h, B.h, f2_neg(p));
  f2 c = f2_fma(A.h, B.l, R.c);
  c = f2_fma(A.l, B.h, c);
  f2 s, t;
  two_sum2(R.s, p, s, t);
  R.s = s;
  R.c = f2_add(f2_add(c, e), t);
}
__device__ __forceinline__ p2 acc2_get(const acc2 &R) { return p2{R.s, R.c}; }

}  // namespace jqcd
