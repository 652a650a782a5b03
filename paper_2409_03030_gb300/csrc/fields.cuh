// Register-level loads and stores of spinors and links in each device layout
// (layouts are described in lattice.cuh).
#pragma once
#include <cuda_fp16.h>

#include "hop.cuh"
#include "lattice.cuh"

namespace jqcd {

template <int PREC> struct PT;

// ---------------------------------------------------------------- double-word
template <> struct PT<PREC_DW> {
  typedef cw C;
  typedef dw Scalar;
  static constexpr int kLinkChunks = kLinkChunksDW;

  __device__ static __forceinline__ void load_spinor(const void *base, int64_t vh, int64_t i,
                                                     C (&s)[4][3]) {
    const float4 *p = reinterpret_cast<const float4 *>(base) + i;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      dwc_unpack(__ldg(p + k * vh), s[k / 3][k % 3].re, s[k / 3][k % 3].im);
    }
  }
  __device__ static __forceinline__ void store_spinor(void *base, int64_t vh, int64_t i,
                                                      const C (&s)[4][3]) {
    float4 *p = reinterpret_cast<float4 *>(base) + i;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      const dw re = dw_norm(s[k / 3][k % 3].re.h, s[k / 3][k % 3].re.l);
      const dw im = dw_norm(s[k / 3][k % 3].im.h, s[k / 3][k % 3].im.l);
      p[k * vh] = dwc_pack(re, im);
    }
  }
  // link chunks start at `base` (already offset to parity and direction)
  __device__ static __forceinline__ void load_link(const void *base, int64_t vh, int64_t i,
                                                   C (&u)[3][3]) {
    const float4 *p = reinterpret_cast<const float4 *>(base) + i;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      dwc_unpack(__ldcs(p + k * vh), u[k / 3][k % 3].re, u[k / 3][k % 3].im);
    }
  }
  __device__ static __forceinline__ void negate_if(C (&h)[2][3], bool neg) {
    const float s = neg ? -1.f : 1.f;
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        h[a][c].re.h *= s; h[a][c].re.l *= s;
        h[a][c].im.h *= s; h[a][c].im.l *= s;
      }
  }
  // out = alpha * x + beta * acc
  __device__ static __forceinline__ C axpby(Scalar alpha, C x, Scalar beta, C acc) {
    C r;
    r.re = dw_add(dw_mul(alpha, x.re), dw_mul(beta, dw_norm(acc.re.h, acc.re.l)));
    r.im = dw_add(dw_mul(alpha, x.im), dw_mul(beta, dw_norm(acc.im.h, acc.im.l)));
    return r;
  }
  __device__ static __forceinline__ C scale(Scalar beta, C acc) {
    C r;
    r.re = dw_mul(beta, dw_norm(acc.re.h, acc.re.l));
    r.im = dw_mul(beta, dw_norm(acc.im.h, acc.im.l));
    return r;
  }
  __device__ static __forceinline__ C zero() { return cw{dw_make(0.f, 0.f), dw_make(0.f, 0.f)}; }
  __device__ static __forceinline__ Scalar scalar(double v, float2 split) {
    return dw_make(split.x, split.y);
  }
};

// ---------------------------------------------------------------- native FP64
template <> struct PT<PREC_F64> {
  typedef cd C;
  typedef double Scalar;
  static constexpr int kLinkChunks = kLinkChunksF64;

  __device__ static __forceinline__ void load_spinor(const void *base, int64_t vh, int64_t i,
                                                     C (&s)[4][3]) {
    const double2 *p = reinterpret_cast<const double2 *>(base) + i;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      double2 v = __ldg(p + k * vh);
      s[k / 3][k % 3] = cd{v.x, v.y};
    }
  }
  __device__ static __forceinline__ void store_spinor(void *base, int64_t vh, int64_t i,
                                                      const C (&s)[4][3]) {
    double2 *p = reinterpret_cast<double2 *>(base) + i;
#pragma unroll
    for (int k = 0; k < 12; ++k) p[k * vh] = make_double2(s[k / 3][k % 3].re, s[k / 3][k % 3].im);
  }
  __device__ static __forceinline__ void load_link(const void *base, int64_t vh, int64_t i,
                                                   C (&u)[3][3]) {
    const double2 *p = reinterpret_cast<const double2 *>(base) + i;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      double2 v = __ldcs(p + k * vh);
      u[k / 3][k % 3] = cd{v.x, v.y};
    }
  }
  __device__ static __forceinline__ void negate_if(C (&h)[2][3], bool neg) {
    if (!neg) return;
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int c = 0; c < 3; ++c) h[a][c] = cd{-h[a][c].re, -h[a][c].im};
  }
  __device__ static __forceinline__ C axpby(Scalar alpha, C x, Scalar beta, C acc) {
    return cd{fma(alpha, x.re, beta * acc.re), fma(alpha, x.im, beta * acc.im)};
  }
  __device__ static __forceinline__ C scale(Scalar beta, C acc) {
    return cd{beta * acc.re, beta * acc.im};
  }
  __device__ static __forceinline__ C zero() { return cd{0., 0.}; }
  __device__ static __forceinline__ Scalar scalar(double v, float2) { return v; }
};

// ---------------------------------------------------------------- FP32 (12-real links)
struct PT_F32Links {
  __device__ static __forceinline__ void load_link(const void *base, int64_t vh, int64_t i,
                                                   cf (&u)[3][3]) {
    const float4 *p = reinterpret_cast<const float4 *>(base) + i;
    float4 c0 = __ldcs(p), c1 = __ldcs(p + vh), c2 = __ldcs(p + 2 * vh);
    u[0][0] = cf{c0.x, c0.y}; u[0][1] = cf{c0.z, c0.w};
    u[0][2] = cf{c1.x, c1.y}; u[1][0] = cf{c1.z, c1.w};
    u[1][1] = cf{c2.x, c2.y}; u[1][2] = cf{c2.z, c2.w};
    reconstruct_row2(u);
  }
  // rows 0 and 1 from three 16-byte chunks (U00,U01) (U02,U10) (U11,U12)
  __device__ static __forceinline__ void link_from_chunks(float4 c0, float4 c1, float4 c2,
                                                          cf (&u)[3][3]) {
    u[0][0] = cf{c0.x, c0.y}; u[0][1] = cf{c0.z, c0.w};
    u[0][2] = cf{c1.x, c1.y}; u[1][0] = cf{c1.z, c1.w};
    u[1][1] = cf{c2.x, c2.y}; u[1][2] = cf{c2.z, c2.w};
    reconstruct_row2(u);
  }
  // row 2 = conj(row0 x row1), exact for SU(3)
  __device__ static __forceinline__ void reconstruct_row2(cf (&u)[3][3]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const int c1i = (c + 1) % 3, c2i = (c + 2) % 3;
      cf a = u[0][c1i], b = u[1][c2i], d = u[0][c2i], e = u[1][c1i];
      float re = a.re * b.re - a.im * b.im - (d.re * e.re - d.im * e.im);
      float im = a.re * b.im + a.im * b.re - (d.re * e.im + d.im * e.re);
      u[2][c] = cf{re, -im};
    }
  }
  __device__ static __forceinline__ void negate_if(cf (&h)[2][3], bool neg) {
    const float s = neg ? -1.f : 1.f;
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int c = 0; c < 3; ++c) h[a][c] = cf{h[a][c].re * s, h[a][c].im * s};
  }
  __device__ static __forceinline__ cf axpby(float alpha, cf x, float beta, cf acc) {
    return cf{fmaf(alpha, x.re, beta * acc.re), fmaf(alpha, x.im, beta * acc.im)};
  }
  __device__ static __forceinline__ cf scale(float beta, cf acc) {
    return cf{beta * acc.re, beta * acc.im};
  }
  __device__ static __forceinline__ cf zero() { return cf{0.f, 0.f}; }
  __device__ static __forceinline__ float scalar(double v, float2) { return (float)v; }
};

template <> struct PT<PREC_F32> : PT_F32Links {
  typedef cf C;
  typedef float Scalar;
  static constexpr int kLinkChunks = kLinkChunksF32;
  __device__ static __forceinline__ void load_spinor(const void *base, int64_t vh, int64_t i,
                                                     C (&s)[4][3]) {
    const float4 *p = reinterpret_cast<const float4 *>(base) + i;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      float4 v = __ldg(p + j * vh);
      s[(2 * j) / 3][(2 * j) % 3] = cf{v.x, v.y};
      s[(2 * j + 1) / 3][(2 * j + 1) % 3] = cf{v.z, v.w};
    }
  }
  __device__ static __forceinline__ void store_spinor(void *base, int64_t vh, int64_t i,
                                                      const C (&s)[4][3]) {
    float4 *p = reinterpret_cast<float4 *>(base) + i;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      cf a = s[(2 * j) / 3][(2 * j) % 3], b = s[(2 * j + 1) / 3][(2 * j + 1) % 3];
      p[j * vh] = make_float4(a.re, a.im, b.re, b.im);
    }
  }
};

// ---------------------------------------------------------------- FP16 + per-site norm
template <> struct PT<PREC_F16N> : PT_F32Links {
  typedef cf C;
  typedef float Scalar;
  static constexpr int kLinkChunks = kLinkChunksF32;
  __device__ static __forceinline__ void load_spinor(const void *base, int64_t vh, int64_t i,
                                                     C (&s)[4][3]) {
    const uint4 *p = reinterpret_cast<const uint4 *>(base) + i;
    const float n = __ldg(reinterpret_cast<const float *>(reinterpret_cast<const uint4 *>(base) +
                                                          3 * vh) + i);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      uint4 v = __ldg(p + j * vh);
      const unsigned w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        __half2 h2 = *reinterpret_cast<const __half2 *>(&w[q]);
        float2 f = __half22float2(h2);
        const int k = 4 * j + q;
        s[k / 3][k % 3] = cf{f.x * n, f.y * n};
      }
    }
  }
  __device__ static __forceinline__ void store_spinor(void *base, int64_t vh, int64_t i,
                                                      const C (&s)[4][3]) {
    float m = 0.f;
#pragma unroll
    for (int k = 0; k < 12; ++k) m = fmaxf(m, fmaxf(fabsf(s[k / 3][k % 3].re), fabsf(s[k / 3][k % 3].im)));
    // A site whose largest component is below 1e-30 is stored as exact zeros:
    // 1/m would overflow for denormal m (point sources reach such values at
    // the edge of their support).  NaN is kept so breakdowns stay visible.
    if (m < 1e-30f) m = 0.f;
    const float inv = m > 0.f ? 1.f / m : (m == 0.f ? 0.f : m);
    uint4 *p = reinterpret_cast<uint4 *>(base) + i;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      unsigned w[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int k = 4 * j + q;
        __half2 h2 = __floats2half2_rn(s[k / 3][k % 3].re * inv, s[k / 3][k % 3].im * inv);
        w[q] = *reinterpret_cast<unsigned *>(&h2);
      }
      p[j * vh] = make_uint4(w[0], w[1], w[2], w[3]);
    }
    reinterpret_cast<float *>(reinterpret_cast<uint4 *>(base) + 3 * vh)[i] = m;
  }
};

}  // namespace jqcd
