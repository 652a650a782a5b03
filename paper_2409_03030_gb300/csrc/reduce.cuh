// Deterministic block reductions: a fixed warp-shuffle tree, then warps summed
// in order by thread 0.  Per-block results go to a partials array that a
// single-block kernel later sums in a fixed order, so a reduction over a
// given launch shape always rounds the same way.
#pragma once
#include "dw.cuh"

namespace jqcd {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ dwacc warp_sum_dw(dwacc v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    float s2 = __shfl_down_sync(kFull, v.s, o);
    float c2 = __shfl_down_sync(kFull, v.c, o);
    float s, e;
    two_sum(v.s, s2, s, e);
    v.s = s;
    v.c = __fadd_rn(__fadd_rn(v.c, c2), e);
  }
  return v;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
  return v;
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
  return v;
}

// Block sum of one double per warp (given by lane 0); result in thread 0.
// blockDim.x must be a multiple of 32 and <= 1024.
__device__ __forceinline__ double block_sum_warp_values(double warp_value) {
  __shared__ double sh[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) sh[warp] = warp_value;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0) {
    const int nw = blockDim.x >> 5;
    for (int w = 0; w < nw; ++w) r += sh[w];
  }
  __syncthreads();
  return r;
}

__device__ __forceinline__ double block_sum_dw(dwacc v) {
  v = warp_sum_dw(v);
  return block_sum_warp_values((double)v.s + (double)v.c);
}

__device__ __forceinline__ double block_sum_f(float v) {
  v = warp_sum_f(v);
  return block_sum_warp_values((double)v);
}

__device__ __forceinline__ double block_sum_d(double v) {
  v = warp_sum_d(v);
  return block_sum_warp_values(v);
}

// sum of partials[0..n) by the whole block in a fixed order (valid in
// thread 0): all of a thread's loads are in flight before its first add;
// the adds keep the order i = tid, tid + blockDim.x, ... (out-of-range
// slots add 0), then the block tree.
__device__ __forceinline__ double block_sum_partials(const double *partials, int n) {
  double v = 0.0;
  constexpr int kU = 16;
  for (int base = threadIdx.x; base < n; base += kU * blockDim.x) {
    double t[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int i = base + u * (int)blockDim.x;
      t[u] = i < n ? partials[i] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) v += t[u];
  }
  return block_sum_d(v);
}

}  // namespace jqcd
