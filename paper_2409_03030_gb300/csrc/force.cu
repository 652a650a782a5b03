// Two-flavour Wilson fermion action S = eta^dag (D^dag D)^{-1} eta and its
// link derivative U dS/dU (paper: evaluate_FermiAction and calc_UdSfdU,
// section "Definition of fermion actions"), in double-word arithmetic.
//
// With X = (D^dag D)^{-1} eta and Y = D X, a variation dU of the links gives
// dS = 2 kappa Re(Y^dag dH X); U_mu(x) enters H at site x through
// (1 - gamma_mu) U_mu(x) psi(x+mu) and at site x+mu through
// (1 + gamma_mu) U_mu(x)^dag psi(x), both times the boundary sign s.  With the
// convention dS = Re Tr[(dS/dU) dU]:
//   U dS/dU = 2 kappa s U (A + B^dag),
//   A_ba = sum_alpha [(1 - gamma_mu) X(x+mu)]_alpha,b conj(Y_alpha,a(x)),
//   B_ba = sum_alpha [(1 + gamma_mu) X(x)]_alpha,b    conj(Y_alpha,a(x+mu)).
// (1 +- gamma_mu) has rank two: rows 2 and 3 are phases times rows k2, k3 (the
// reconstruction table of the hop), so each spin sum is two colour outer
// products, h_s conj(w_s)^T, with h the projected half-spinor of X and
// w_s = Y_s + conj-phase * Y_alpha for the lower spins alpha that map to s.
// Arithmetic: the packed two-lane double-word operations of the hop
// (sums of exact products on a fixed offset grid, hop_dwp.cuh).
#include <cuda_runtime.h>

#include "fields.cuh"
#include "hop.cuh"
#include "hop_dw.cuh"
#include "hop_dwp.cuh"
#include "kernels.h"
#include "reduce.cuh"

namespace jqcd {

namespace {

constexpr int kForceThreads = 128;
constexpr int kForceOwnChunks = 24;  // X and Y of the thread's own site
constexpr int kForceNbChunks = 12;   // the neighbour spinor of the next part
constexpr size_t kForceSmem = (size_t)(kForceOwnChunks + kForceNbChunks) * kForceThreads * 16;  // 72 KB

// Issue the copies of one double-word spinor of site i into a stage column.
__device__ __forceinline__ void stage_spinor_force(float4 *st, const float4 *f, int64_t vh, int64_t i) {
#pragma unroll
  for (int k = 0; k < 12; ++k) cp_async16(st + k * kForceThreads, f + k * vh + i, false);
}

// a + phase<PH> b for complex double-word pairs (PH: 0 -> 1, 1 -> i, 2 -> -1,
// 3 -> -i); i b = (-b.im, b.re).
template <int PH>
__device__ __forceinline__ p2 p2_add_phase(p2 a, p2 b) {
  if (PH == 0) return p2_add(a, b);
  if (PH == 2) return p2_add_sgn(a, b, f2_make(-1.f, -1.f));
  if (PH == 1) return p2_add_sgn(a, p2_swap(b), f2_make(-1.f, 1.f));
  return p2_add_sgn(a, p2_swap(b), f2_make(1.f, -1.f));
}

// w_s = Y_s + sum over the lower spins alpha with k_alpha = s of
// conj(phase_alpha) Y_alpha, for the projector (1 + S gamma_mu): then
// sum_alpha [(1 + S gamma_mu) Z]_alpha conj(Y_alpha) = sum_s h_s conj(w_s).
template <int MU, int S>
__device__ __forceinline__ void adjoint_half_p(const p2 (&y)[4][3], p2 (&w)[2][3]) {
  typedef SpinTab<MU> T;
  constexpr int Q2 = (T::q2 + (S < 0 ? 2 : 0)) & 3;
  constexpr int Q3 = (T::q3 + (S < 0 ? 2 : 0)) & 3;
  constexpr int C2 = (4 - Q2) & 3, C3 = (4 - Q3) & 3;  // conjugate phases
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    w[0][c] = y[0][c];
    w[1][c] = y[1][c];
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    w[T::k2][c] = p2_add_phase<C2>(w[T::k2][c], y[2][c]);
    w[T::k3][c] = p2_add_phase<C3>(w[T::k3][c], y[3][c]);
  }
}

// Broadcast multiplier of the real part of conj(z) (both lanes z.re) and of
// its imaginary part (both lanes -z.im).
__device__ __forceinline__ mul2 conj_re(p2 z) { return mul2{f2_lo(z.h), f2_lo(z.l)}; }
__device__ __forceinline__ mul2 conj_im(p2 z) { return mul2{f2_neg(f2_hi(z.h)), f2_neg(f2_hi(z.l))}; }

// Projected half-spinor (rows 0, 1 of (1 + S gamma_mu) psi) with a runtime
// direction: only this small step exists once per direction in the code.
__device__ __forceinline__ void project_rt(int mu, const p2 (&s4)[4][3], p2 (&h)[2][3], float S) {
  switch (mu) {
    case 0: project_p<0>(s4, h, S); break;
    case 1: project_p<1>(s4, h, S); break;
    case 2: project_p<2>(s4, h, S); break;
    default: project_p<3>(s4, h, S);
  }
}
__device__ __forceinline__ void adjoint_rt(int mu, int S, const p2 (&s4)[4][3], p2 (&w)[2][3]) {
  switch (mu + (S > 0 ? 4 : 0)) {
    case 0: adjoint_half_p<0, -1>(s4, w); break;
    case 1: adjoint_half_p<1, -1>(s4, w); break;
    case 2: adjoint_half_p<2, -1>(s4, w); break;
    case 3: adjoint_half_p<3, -1>(s4, w); break;
    case 4: adjoint_half_p<0, 1>(s4, w); break;
    case 5: adjoint_half_p<1, 1>(s4, w); break;
    case 6: adjoint_half_p<2, 1>(s4, w); break;
    default: adjoint_half_p<3, 1>(s4, w);
  }
}

// X and Y of both parities as double-word spinor fields.
struct FieldPair {
  const float4 *xe, *xo, *ye, *yo;
};

// U dS/dU of direction mu for the link at site (p, cb), packed double-word
// arithmetic.  M_ba = A_ba + conj(B_ab) is built in two parts, each
// P_ba = sum_s v_sb conj(c_sa) (complex scalars conj(c) times the vector
// components v, split into the scalars' real and imaginary parts):
//   part 0 (A):      v = projected (1 - gamma_mu) X(x+mu), c = adjoint half of Y(x);
//   part 1 (B^dag):  v = adjoint half of Y(x+mu), c = projected (1 + gamma_mu) X(x).
// Then G = 2 kappa s U M column by column through the hop's mat-vec.  The
// direction and the part are runtime values, so the heavy arithmetic exists
// once in the instruction stream (the per-direction copies overflowed the
// instruction cache).
// own: this thread's column of the block's shared memory, X(x) in chunks
// 0..11 and Y(x) in chunks 12..23 (stride kForceThreads).  nst: the column of
// the neighbour stage, holding X(x + mu) (copies issued by the caller or the
// previous direction) when the call starts; Y(x + mu) is copied in during
// part 0 and X(x + mu + 1) during part 1, each as soon as the stage has been
// read.
__device__ __forceinline__ void force_link(const Geom &g, int p, int64_t cb, int x, int y, int z, int t, int mu,
                                           const FieldPair &F, const float4 *own, float4 *nst,
                                           const float4 *gauge, float2 two_kappa, float4 *out) {
  const int64_t vh = g.vh;
  bool neg;
  const int64_t nb = hop_neighbour(g, x, y, z, t, 2 * mu, neg);  // x + mu, parity 1-p
  const float4 *Xn = p ? F.xe : F.xo, *Yn = p ? F.ye : F.yo;
  constexpr f2 kLane0 = 0x0000000080000000ull;
  p2 M[3][3];
#pragma unroll 1
  for (int part = 0; part < 2; ++part) {
    p2 v[2][3], c[2][3];
    {
      p2 s4[4][3];
      asm volatile("cp.async.wait_group 0;\n" ::: "memory");  // only this thread's column is read
#pragma unroll
      for (int k = 0; k < 12; ++k) s4[k / 3][k % 3] = ld_p2(nst + k * kForceThreads);
      if (part == 0) {
        stage_spinor_force(nst, Yn, vh, nb);
      } else if (mu < 3) {
        bool neg1;
        stage_spinor_force(nst, Xn, vh, hop_neighbour(g, x, y, z, t, 2 * mu + 2, neg1));
      }
      cp_async_commit();
      if (part) adjoint_rt(mu, 1, s4, v);
      else project_rt(mu, s4, v, -1.f);
      {
        const float4 *o = own + (part ? 0 : 12) * kForceThreads;
#pragma unroll
        for (int k = 0; k < 12; ++k) s4[k / 3][k % 3] = ld_p2(o + k * kForceThreads);
      }
      if (part) project_rt(mu, s4, c, 1.f);
      else adjoint_rt(mu, -1, s4, c);
    }
    // One offset grid for the part's nine entries (as in matvec_half_p): every
    // partial sum is below max|v.hi| * max_a max(|c_0a.re| + |c_1a.re|,
    // |c_0a.im| + |c_1a.im|), raised by 2^-19, and sigma is the power of two
    // above twice that; A starts at (1.5 sigma, 1.5 sigma), B at
    // (-1.5 sigma, 1.5 sigma).
    f2 TA0, TB0;
    {
      float vm = 0.f, cm = 0.f;
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        float u, w;
        f2_split(v[k / 3][k % 3].h, u, w);
        vm = fmaxf(vm, fmaxf(fabsf(u), fabsf(w)));
      }
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        float r0, i0, r1, i1;
        f2_split(c[0][a].h, r0, i0);
        f2_split(c[1][a].h, r1, i1);
        cm = fmaxf(cm, fmaxf(fabsf(r0) + fabsf(r1), fabsf(i0) + fabsf(i1)));
      }
      const float m = vm * cm * 1.0000019f;
      const float t0 = __uint_as_float((__float_as_uint(m) & 0x7f800000u) + (2u << 23) + (1u << 22));
      TA0 = f2_make(t0, t0);
      TB0 = f2_make(-t0, t0);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const mul2 r0 = conj_re(c[0][a]), r1 = conj_re(c[1][a]);
      const mul2 i0 = conj_im(c[0][a]), i1 = conj_im(c[1][a]);
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        f2 TA = TA0, TB = TB0, cA = 0ull, cB = 0ull;
        grid_mad(TA, cA, r0, v[0][b], true);
        grid_mad(TA, cA, r1, v[1][b], false);
        grid_mad(TB, cB, i0, v[0][b], true);
        grid_mad(TB, cB, i1, v[1][b], false);
        // A + i B; the offsets cancel exactly in the high words
        const p2 P{f2_add(TA, f2_swap(TB) ^ kLane0), f2_add(cA, f2_swap(cB) ^ kLane0)};
        M[b][a] = part ? p2_norm(p2_add(M[b][a], P)) : P;
      }
    }
  }
  p2 U[3][3];
  {
    const ulonglong2 *L = reinterpret_cast<const ulonglong2 *>(gauge) + (size_t)((p * 4 + mu) * 9) * vh + cb;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const ulonglong2 v = __ldcs(L + k * vh);
      U[k / 3][k % 3] = p2{v.x, v.y};
    }
  }
  const float umax = link_max_hi(U) * 1.0000019f;  // bound of the grid mat-vec
  const float fs = neg ? -1.f : 1.f;  // boundary sign, exact
  const f2 fh = f2_make(fs * two_kappa.x, fs * two_kappa.x);
  const mul2 Fm{fh, f2_make(fs * two_kappa.y, fs * two_kappa.y)};
  ulonglong2 *o = reinterpret_cast<ulonglong2 *>(out) + (size_t)((p * 4 + mu) * 9) * vh + cb;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const p2 col[3] = {M[0][a], M[1][a], M[2][a]};
    p2 Gc[3];
    matvec_half_p(U, umax, col, Gc);  // G_ia = sum_b U_ib M_ba
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const p2 q = p2_norm(acc2_get(acc2_first(Fm, p2_norm(Gc[i]))));
      __stcs(o + (3 * i + a) * vh, make_ulonglong2(q.h, q.l));
    }
  }
}

// The site's own X and Y are read by all four directions: they are copied
// once into this thread's column of shared memory (an L1-cached reload would
// not survive the ~350 KB per SM that the neighbours and links of one
// direction stream through).
__global__ void __launch_bounds__(kForceThreads, 3) force_kernel(Geom g, FieldPair F,
                                                                 const float4 *__restrict__ gauge,
                                                                 float2 two_kappa, float4 *__restrict__ out) {
  extern __shared__ float4 fsm[];  // kForceOwnChunks x kForceThreads
  // Blocks 2k and 2k + 1 take the same checkerboard sites of parity 0 and 1:
  // the spinors one parity reads as its neighbours are the other's own, loaded
  // at the same time, so each is read from DRAM about once (all of parity 0
  // before parity 1 read 1.22x the algorithmic bytes).
  const int p = (int)(blockIdx.x & 1);
  const int64_t cb = (int64_t)(blockIdx.x >> 1) * blockDim.x + threadIdx.x;
  if (cb >= g.vh) return;
  const float4 *Xh = p ? F.xo : F.xe, *Yh = p ? F.yo : F.ye;
  float4 *own = fsm + threadIdx.x;
  float4 *nst = fsm + kForceOwnChunks * kForceThreads + threadIdx.x;
  int x, y, z, t;
  cb_coords(g, cb, p, x, y, z, t);
  stage_spinor_force(own, Xh, g.vh, cb);
  stage_spinor_force(own + 12 * kForceThreads, Yh, g.vh, cb);
  {
    bool neg0;
    stage_spinor_force(nst, p ? F.xe : F.xo, g.vh, hop_neighbour(g, x, y, z, t, 0, neg0));  // X(x + 0)
  }
  cp_async_commit();
#pragma unroll 1
  for (int mu = 0; mu < 4; ++mu) force_link(g, p, cb, x, y, z, t, mu, F, own, nst, gauge, two_kappa, out);
}

// out = gamma5 in on a whole-lattice double-word spinor (chunks k = 3*spin + c;
// spins 2 and 3 change sign).  In place allowed.
__global__ void gamma5_dw_kernel(float4 *out, const float4 *in, int64_t vh) {
  const int64_t n = 24 * vh;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)((q / vh) % 12);
    const float4 v = in[q];
    out[q] = k >= 6 ? make_float4(-v.x, -v.y, -v.z, -v.w) : v;
  }
}

// Per-block partial of Re <a, b> over n double-word complex numbers.
__global__ void dw_dot_re_kernel(const float4 *__restrict__ a, const float4 *__restrict__ b, int64_t n,
                                 double *partials, const int *guard) {
  if (guard && *guard) return;  // uniform across the grid
  dwacc A{0.f, 0.f};
  bool first = true;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
    dw ar, ai, br, bi;
    dwc_unpack(a[q], ar, ai);
    dwc_unpack(b[q], br, bi);
    if (first) {
      A = acc_first(ar, br);
      first = false;
    } else {
      acc_mad(A, ar, br);
    }
    acc_mad(A, ai, bi);
  }
  const double s = block_sum_dw(A);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// Double-word link field [2][4][9][vh] -> canonical links a + 3(b + 3(site + V mu)).
__global__ void linkfield_unpack_kernel(Geom g, const float4 *__restrict__ dwf, double *__restrict__ canon) {
  const int64_t V = 2 * g.vh;
  const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= 4 * V) return;
  const int mu = (int)(l / V);
  const int64_t s = l % V;
  const int x = (int)(s % g.nx);
  int64_t r = s / g.nx;
  const int y = (int)(r % g.ny);
  r /= g.ny;
  const int z = (int)(r % g.nz);
  const int t = (int)(r / g.nz);
  const int p = (x + y + z + t) & 1;
  const int64_t cb = s >> 1;
  double2 *dst = reinterpret_cast<double2 *>(canon) + 9 * (s + V * mu);
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      const float4 v = dwf[((int64_t)(p * 4 + mu) * 9 + 3 * a + b) * g.vh + cb];
      dst[a + 3 * b] = make_double2((double)v.x + (double)v.z, (double)v.y + (double)v.w);
    }
}

}  // namespace

cudaError_t launch_fermi_force(const Geom &g, const float4 *xe, const float4 *xo, const float4 *ye,
                               const float4 *yo, const float4 *gauge_dw, double kappa, float4 *out,
                               cudaStream_t s) {
  static bool configured = false;  // 72 KB of dynamic shared memory needs the opt-in
  if (!configured) {
    const cudaError_t e = cudaFuncSetAttribute(force_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)kForceSmem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  note_launch();
  const float2 tk = dw_split_host(2.0 * kappa);
  const unsigned blocks = 2 * (unsigned)((g.vh + kForceThreads - 1) / kForceThreads);
  force_kernel<<<blocks, kForceThreads, kForceSmem, s>>>(g, FieldPair{xe, xo, ye, yo}, gauge_dw, tk, out);
  return cudaGetLastError();
}

cudaError_t launch_gamma5_dw(float4 *out, const float4 *in, int64_t vh, cudaStream_t s) {
  note_launch();
  gamma5_dw_kernel<<<blas_blocks(24 * vh), kBlasThreads, 0, s>>>(out, in, vh);
  return cudaGetLastError();
}

cudaError_t launch_dw_dot_re(const float4 *a, const float4 *b, int64_t n, double *partials, int nblocks,
                             cudaStream_t s, const int *guard) {
  note_launch();
  dw_dot_re_kernel<<<nblocks, kBlasThreads, 0, s>>>(a, b, n, partials, guard);
  return cudaGetLastError();
}

cudaError_t launch_linkfield_unpack(const Geom &g, const float4 *dwf, double *canon, cudaStream_t s) {
  note_launch();
  const int64_t n = 8 * g.vh;
  linkfield_unpack_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(g, dwf, canon);
  return cudaGetLastError();
}

}  // namespace jqcd
