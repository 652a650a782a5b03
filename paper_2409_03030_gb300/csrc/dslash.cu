// Even-odd Wilson hop kernels: out_p = a * x_p + b * H_{p,1-p} in_{1-p}
// with an optional fused per-block partial of ||out_p||^2.
//
// One thread per output site.  Each of the 8 neighbours is loaded as a full
// spinor (16-byte chunks, read-only path), spin-projected to a half-spinor,
// multiplied by its link (streamed, each link is used once per hop) and
// spread back onto four spins in registers.  Neighbour reuse across threads
// is served by L1/L2: in the checkerboard order the x, y, z neighbours of a
// warp's sites are within a few kB and the t neighbours within one time slice.
#include <cuda_runtime.h>

#include "fields.cuh"
#include "hop.cuh"
#include "kernels.h"
#include "pdl.cuh"
#include "hop_dw.cuh"
#include "hop_dwp.cuh"
#include "hop_lp.cuh"
#include "cg_steps.cuh"
#include "reduce.cuh"

namespace jqcd {

template <int MU, int PREC, bool DAG>
__device__ __forceinline__ void hop_dir(const HopParams &P, int x, int y, int z, int t,
                                        int64_t idx, typename PT<PREC>::C (&acc)[4][3]) {
  typedef PT<PREC> T;
  typedef typename T::C C;
  const Geom &g = P.g;
  const int p = P.out_parity;
  const char *gbase = reinterpret_cast<const char *>(P.gauge);
  const size_t link_bytes = (size_t)T::kLinkChunks * 16 * g.vh;  // one (parity, mu) block
  // forward neighbour x + mu: (1 - gamma_mu) U_mu(x) psi(x+mu)
  {
    int xf = x, yf = y, zf = z, tf = t;
    bool neg = false;
    if (MU == 0) xf = (x + 1 == g.nx) ? 0 : x + 1;
    if (MU == 1) yf = (y + 1 == g.ny) ? 0 : y + 1;
    if (MU == 2) zf = (z + 1 == g.nz) ? 0 : z + 1;
    if (MU == 3) {
      if (t + 1 == g.nt) { tf = 0; neg = g.tanti != 0; } else tf = t + 1;
    }
    const int64_t nf = cb_index(g, xf, yf, zf, tf);
    C psi[4][3], h[2][3], r[2][3], u[3][3];
    T::load_spinor(P.in, g.vh, nf, psi);
    project<MU, DAG ? 1 : -1>(psi, h);
    T::negate_if(h, neg);
    T::load_link(gbase + link_bytes * (size_t)(p * 4 + MU), g.vh, idx, u);
    matvec2<false>(u, h, r);
    reconstruct<MU, DAG ? 1 : -1>(r, acc);
  }
  // backward neighbour x - mu: (1 + gamma_mu) U_mu(x-mu)^dag psi(x-mu)
  {
    int xb = x, yb = y, zb = z, tb = t;
    bool neg = false;
    if (MU == 0) xb = (x == 0) ? g.nx - 1 : x - 1;
    if (MU == 1) yb = (y == 0) ? g.ny - 1 : y - 1;
    if (MU == 2) zb = (z == 0) ? g.nz - 1 : z - 1;
    if (MU == 3) {
      if (t == 0) { tb = g.nt - 1; neg = g.tanti != 0; } else tb = t - 1;
    }
    const int64_t nb = cb_index(g, xb, yb, zb, tb);
    C psi[4][3], h[2][3], r[2][3], u[3][3];
    T::load_spinor(P.in, g.vh, nb, psi);
    project<MU, DAG ? -1 : 1>(psi, h);
    T::negate_if(h, neg);
    T::load_link(gbase + link_bytes * (size_t)((1 - p) * 4 + MU), g.vh, nb, u);
    matvec2<true>(u, h, r);
    reconstruct<MU, DAG ? -1 : 1>(r, acc);
  }
}

template <int PREC, bool DAG, bool AXPY, bool NORM>
__global__ void __launch_bounds__(kHopThreads) hop_kernel(const HopParams P) {
  typedef PT<PREC> T;
  typedef typename T::C C;
  pdl_enter();
  if (P.guard && *P.guard) return;  // uniform across the grid
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = idx < P.g.vh;
  dwacc nrm{0.f, 0.f};
  double nrm64 = 0.0;  // FP64 hops accumulate their norm in FP64
  if (active) {
    int x, y, z, t;
    cb_coords(P.g, idx, P.out_parity, x, y, z, t);
    C acc[4][3];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c = 0; c < 3; ++c) acc[a][c] = T::zero();
    hop_dir<0, PREC, DAG>(P, x, y, z, t, idx, acc);
    hop_dir<1, PREC, DAG>(P, x, y, z, t, idx, acc);
    hop_dir<2, PREC, DAG>(P, x, y, z, t, idx, acc);
    hop_dir<3, PREC, DAG>(P, x, y, z, t, idx, acc);
    const typename T::Scalar b = T::scalar(P.b, P.b_split);
    C o[4][3];
    if (AXPY) {
      const typename T::Scalar a = T::scalar(P.a, P.a_split);
      C xs[4][3];
      T::load_spinor(P.x, P.g.vh, idx, xs);
#pragma unroll
      for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) o[s][c] = T::axpby(a, xs[s][c], b, acc[s][c]);
    } else {
#pragma unroll
      for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) o[s][c] = T::scale(b, acc[s][c]);
    }
    T::store_spinor(P.out, P.g.vh, idx, o);
    if (NORM) {
      if constexpr (PREC == PREC_F64) nrm64 = site_norm2_d(o);
      else nrm = site_norm2<PREC>(o);
    }
  }
  if (NORM) {
    const double s = PREC == PREC_F64 ? block_sum_d(nrm64) : block_sum_dw(nrm);
    if (threadIdx.x == 0) P.partials[blockIdx.x] = s;
    if (P.fin) hop_finish_scalars(P);  // uniform over the grid
  }
}

// Low-precision hop with the next hop's neighbour and link prefetched into
// shared memory (hop_lp.cuh); same epilogue as hop_kernel.
template <int PREC, bool DAG, bool AXPY, bool NORM>
__global__ void __launch_bounds__(kHopThreads) hop_lp_kernel(const HopParams P) {
  typedef PT<PREC> T;
  extern __shared__ float4 lsm[];
  pdl_enter();
  if (P.guard && *P.guard) return;  // uniform across the grid
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  dwacc nrm{0.f, 0.f};
  if (idx < P.g.vh) {
    cf acc[4][3];
    lp_hop_site<PREC, DAG, false>(lsm, P.in, reinterpret_cast<const float4 *>(P.gauge), P.g,
                                  P.out_parity, idx, acc);
    const float b = (float)P.b;
    cf o[4][3];
    if (AXPY) {
      const float a = (float)P.a;
      cf xs[4][3];
      T::load_spinor(P.x, P.g.vh, idx, xs);
#pragma unroll
      for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) o[s][c] = T::axpby(a, xs[s][c], b, acc[s][c]);
    } else {
#pragma unroll
      for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) o[s][c] = T::scale(b, acc[s][c]);
    }
    T::store_spinor(P.out, P.g.vh, idx, o);
    if (NORM) nrm = site_norm2<PREC>(o);
  }
  if (NORM) {
    const double s = block_sum_dw(nrm);
    if (threadIdx.x == 0) P.partials[blockIdx.x] = s;
    if (P.fin) hop_finish_scalars(P);  // uniform over the grid
  }
}

template <int PREC, bool DAG, bool AXPY, bool NORM>
static cudaError_t launch_hop_t(const HopParams &P, cudaStream_t s) {
  const unsigned blocks = hop_blocks(P.g.vh);
  note_launch();
  // FP16: staged (measured faster); FP32: plain loads (its six-chunk stages
  // cost more occupancy than the prefetch gains); FP64: plain.
  if (PREC == PREC_F16N)
    return launch_pdl(hop_lp_kernel<PREC_F16N, DAG, AXPY, NORM>, blocks, kHopThreads,
                      lp_stage_smem<PREC_F16N>(), s, P);
  else
    return launch_pdl(hop_kernel<PREC, DAG, AXPY, NORM>, blocks, kHopThreads, 0, s, P);
}

template <int PREC>
static cudaError_t launch_hop_p(const HopParams &P, bool dag, bool axpy, bool norm, cudaStream_t s) {
  const int key = (dag ? 4 : 0) | (axpy ? 2 : 0) | (norm ? 1 : 0);
  switch (key) {
    case 0: return launch_hop_t<PREC, false, false, false>(P, s);
    case 1: return launch_hop_t<PREC, false, false, true>(P, s);
    case 2: return launch_hop_t<PREC, false, true, false>(P, s);
    case 3: return launch_hop_t<PREC, false, true, true>(P, s);
    case 4: return launch_hop_t<PREC, true, false, false>(P, s);
    case 5: return launch_hop_t<PREC, true, false, true>(P, s);
    case 6: return launch_hop_t<PREC, true, true, false>(P, s);
    default: return launch_hop_t<PREC, true, true, true>(P, s);
  }
}

// ---------------------------------------------------------------------------
// Double-word hop in packed two-lane arithmetic (hop_dwp.cuh): one fma/add/
// mul.rn.f32x2 per complex operation halves the instruction issue of a
// scalar double-word hop, which was bound by issue rather than by the FP32
// datapath.
template <bool DAG, bool AXPY, bool NORM, int MINB>
__global__ void __launch_bounds__(kDwp1Threads, MINB) hop_dwp_kernel(const HopParams P) {
  extern __shared__ float4 dsm[];
  pdl_enter();
  if (P.guard && *P.guard) return;  // uniform across the grid
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  dwacc nrm{0.f, 0.f};
  if (idx < P.g.vh) {
    p2 acc[4][3];
    dwp_hop_site<DAG, kDwp1Threads>(dsm, reinterpret_cast<const float4 *>(P.in),
                                    reinterpret_cast<const float4 *>(P.gauge), P.g, P.out_parity, idx, acc);
    nrm = dwp_store<AXPY, NORM>(acc, reinterpret_cast<float4 *>(P.out),
                                reinterpret_cast<const float4 *>(P.x), P.g.vh, idx, P.a_split, P.b_split);
  }
  if (NORM) {
    const double s = block_sum_dw(nrm);
    if (threadIdx.x == 0) P.partials[blockIdx.x] = s;
  }
}

// Small lattices: two threads per output site (dwp_pair_combine), so the
// grid holds twice as many warps when one thread per site cannot fill the
// GPU.  Blocks of kDwp2Threads threads cover kDwp2Threads / 2 sites.
template <bool DAG, bool AXPY, bool NORM>
__global__ void __launch_bounds__(kDwp2Threads, JQCD_DWP2_MIN_BLOCKS) hop_dwp2_kernel(const HopParams P) {
  extern __shared__ float4 dsm[];
  pdl_enter();
  if (P.guard && *P.guard) return;  // uniform across the grid
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t idx = gid >> 1;
  const int q = (int)(gid & 1);
  const bool active = idx < P.g.vh;  // the same for both threads of a site
  p2 acc[4][3];
  if (active) {
    dwp_hop_dirs<DAG, kDwp2Threads>(dsm, reinterpret_cast<const float4 *>(P.in),
                                     reinterpret_cast<const float4 *>(P.gauge), P.g, P.out_parity, idx, q,
                                     2, 4, acc);
  } else {
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c = 0; c < 3; ++c) acc[a][c] = p2{0ull, 0ull};
  }
  p2 o[6];
  dwp_pair_combine(acc, q, o);  // every lane of the warp takes part
  dwacc nrm{0.f, 0.f};
  if (active)
    nrm = dwp_store_chunks<AXPY, NORM, 6>(o, 6 * q, reinterpret_cast<float4 *>(P.out),
                                          reinterpret_cast<const float4 *>(P.x), P.g.vh, idx,
                                          P.a_split, P.b_split);
  if (NORM) {
    const double s = block_sum_dw(nrm);
    if (threadIdx.x == 0) P.partials[blockIdx.x] = s;
  }
}

// Two threads per site pay off only while their grid fits in one wave of
// resident warps (measured on GB300: 8^4 hop 9.6 -> 5.9 us; at 16^4, where
// the split grid needs 1.12 waves, 19.1 -> 18.6 us and the solve slower;
// 16^3x32 at 2.25 waves 24.8 -> 30.4 us).  Twelve warps per SM is the most
// the split kernel's 164-168 registers allow: a thirteenth puts a fourth
// warp on one SM sub-partition, whose register file then caps every thread
// at 128 registers (the kernel spilled 402 bytes and ran 25-40% slower).
bool dw_hop_split(int64_t vh) {
  static const int64_t max_vh = [] {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
      return (int64_t)0;
    return (int64_t)sms * JQCD_DWP2_MIN_BLOCKS * kDwp2Threads / 2;
  }();
  return vh <= max_vh && vh <= JQCD_DWP_SPLIT_MAX_VH;
}

// A one-thread grid of at most SMs x JQCD_DWP_SMALL_MIN_BLOCKS blocks takes
// the form compiled for that occupancy: 184 instead of 166 registers, so
// fewer dependent chains are serialised to save registers (measured on
// GB300: 16^4 hop 18.75 -> 13.94 us, its double-word solve 5.34 -> 4.60 ms;
// at 24^3x48 the same form, at 2 blocks/SM, ran 110.5 against 97.9 us).
bool dw_hop_small(int64_t vh) {
  static const int64_t max_vh = [] {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
      return (int64_t)0;
    return (int64_t)sms * JQCD_DWP_SMALL_MIN_BLOCKS * kDwp1Threads;
  }();
  return !dw_hop_split(vh) && vh <= max_vh && vh <= JQCD_DWP_SMALL_MAX_VH;
}

unsigned dw_hop_blocks(int64_t vh) {
  return dw_hop_split(vh) ? (unsigned)((2 * vh + kDwp2Threads - 1) / kDwp2Threads)
                          : (unsigned)((vh + kDwp1Threads - 1) / kDwp1Threads);
}

unsigned hop_norm_partials(int prec, int64_t vh) {
  return prec == PREC_DW ? dw_hop_blocks(vh) : hop_blocks(vh);
}

template <bool DAG, bool AXPY, bool NORM>
static cudaError_t launch_hop_dw_t(const HopParams &P, cudaStream_t s) {
  note_launch();
  static bool configured = false;  // one attribute call per instantiation
  auto kern = hop_dwp_kernel<DAG, AXPY, NORM, JQCD_DWP_MIN_BLOCKS>;
  auto kern_s = hop_dwp_kernel<DAG, AXPY, NORM, JQCD_DWP_SMALL_MIN_BLOCKS>;
  auto kern2 = hop_dwp2_kernel<DAG, AXPY, NORM>;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDwp1Smem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(kern_s, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDwp1Smem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(kern2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDwp2Smem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  if (dw_hop_split(P.g.vh)) return launch_pdl(kern2, dw_hop_blocks(P.g.vh), kDwp2Threads, kDwp2Smem, s, P);
  if (dw_hop_small(P.g.vh)) return launch_pdl(kern_s, dw_hop_blocks(P.g.vh), kDwp1Threads, kDwp1Smem, s, P);
  return launch_pdl(kern, dw_hop_blocks(P.g.vh), kDwp1Threads, kDwp1Smem, s, P);
}

static cudaError_t launch_hop_dw(const HopParams &P, bool dag, bool axpy, bool norm, cudaStream_t s) {
  const int key = (dag ? 4 : 0) | (axpy ? 2 : 0) | (norm ? 1 : 0);
  switch (key) {
    case 0: return launch_hop_dw_t<false, false, false>(P, s);
    case 1: return launch_hop_dw_t<false, false, true>(P, s);
    case 2: return launch_hop_dw_t<false, true, false>(P, s);
    case 3: return launch_hop_dw_t<false, true, true>(P, s);
    case 4: return launch_hop_dw_t<true, false, false>(P, s);
    case 5: return launch_hop_dw_t<true, false, true>(P, s);
    case 6: return launch_hop_dw_t<true, true, false>(P, s);
    default: return launch_hop_dw_t<true, true, true>(P, s);
  }
}

cudaError_t launch_hop(int prec, const HopParams &P, bool dag, bool axpy, bool norm,
                       cudaStream_t s) {
  // the last-block scalar step (FP64, FP32 and FP16 hops) needs the partials
  // and at most JQCD_FIN_MAX_BLOCKS of them
  if (P.fin && (prec == PREC_DW || !norm || !P.fin_S ||
                hop_norm_partials(prec, P.g.vh) > (unsigned)JQCD_FIN_MAX_BLOCKS))
    return cudaErrorInvalidValue;
  switch (prec) {
    case PREC_DW: return launch_hop_dw(P, dag, axpy, norm, s);
    case PREC_F64: return launch_hop_p<PREC_F64>(P, dag, axpy, norm, s);
    case PREC_F32: return launch_hop_p<PREC_F32>(P, dag, axpy, norm, s);
    case PREC_F16N: return launch_hop_p<PREC_F16N>(P, dag, axpy, norm, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace jqcd
