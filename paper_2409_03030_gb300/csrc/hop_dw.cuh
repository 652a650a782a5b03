// Building blocks shared by the hop kernels of every precision: per-site
// norms of a hop's output, the cp.async helpers of the staged hops, and the
// neighbour lookup with its boundary sign.
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
// FP64 sum of squares of an FP64 site (the native FP64 hop's norm).
__device__ __forceinline__ double site_norm2_d(const cd (&o)[4][3]) {
  double s = 0.;
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    s = fma(o[k / 3][k % 3].re, o[k / 3][k % 3].re, s);
    s = fma(o[k / 3][k % 3].im, o[k / 3][k % 3].im, s);
  }
  return s;
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
// Staged hops copy the operands of the next hop into shared memory (cp.async,
// two stages), so each warp's memory latency overlaps its own arithmetic
// instead of depending on other resident warps.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, bool keep_l1) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  if (keep_l1)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
  else
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

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


}  // namespace jqcd
