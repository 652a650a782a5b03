// Staggered (Kogut-Susskind) fermions (paper: Dirac_operator "staggered"
// with a "mass"), double-word arithmetic:
//   (D psi)(x) = m psi(x) + D_hop psi,
//   (D_hop psi)(x) = 1/2 sum_mu eta_mu(x) [U_mu(x) psi(x+mu) - U_mu(x-mu)^dag psi(x-mu)],
//   eta_mu(x) = (-1)^(x_0 + ... + x_{mu-1}), antiperiodic time boundary.
// D_hop is anti-Hermitian and couples opposite parities, so the even-odd
// system M_ee = m^2 - D_eo D_oe = m^2 + D_oe^dag D_oe is Hermitian positive
// definite: solve M_ee x_e = m b_e - D_eo b_o by CG, then
// x_o = (b_o - D_oe x_e) / m.
//
// Layout: one colour vector per site; per parity three 16-byte double-word
// chunks (re.h, im.h, re.l, im.l), chunk c of site cb at c*vh + cb.  Links:
// the double-word gauge field of the Wilson path.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>

#include "hop_dwp.cuh"
#include "kernels.h"
#include "pdl.cuh"
#include "reduce.cuh"
#include "solver.h"
#include "staggered.h"

namespace jqcd {

namespace {

constexpr int kStagThreads = 128;

// eta_mu(x) for checkerboard coordinates
__device__ __forceinline__ float stag_eta(int mu, int x, int y, int z) {
  const int s = mu == 0 ? 0 : (mu == 1 ? x : (mu == 2 ? x + y : x + y + z));
  return (s & 1) ? -1.f : 1.f;
}

// acc = sum over the 8 hops of eta_mu(x) * (+U_mu(x) in(x+mu) or -U_mu(x-mu)^dag in(x-mu)),
// with the boundary sign (DAG: negated), at output site cb of parity p.
template <bool DAG>
__device__ __forceinline__ void stag_hop_sum(const Geom &g, int p, int64_t cb, const float4 *__restrict__ in,
                                             const float4 *__restrict__ gauge, p2 (&acc)[3]) {
  const int64_t vh = g.vh;
  int x, y, z, t;
  cb_coords(g, cb, p, x, y, z, t);
  acc[0] = acc[1] = acc[2] = p2{0ull, 0ull};
#pragma unroll 1
  for (int d = 0; d < 8; ++d) {
    const int mu = d >> 1;
    const bool bwd = (d & 1) != 0;
    bool neg;
    const int64_t nb = hop_neighbour(g, x, y, z, t, d, neg);
    // link: forward U_mu(x); backward U_mu(x-mu)^dag (transposed here, conjugated below)
    const ulonglong2 *L = reinterpret_cast<const ulonglong2 *>(gauge) +
                          (size_t)(((bwd ? 1 - p : p) * 4 + mu) * 9) * vh + (bwd ? nb : cb);
    const int sa = bwd ? 1 : 3, sb = bwd ? 3 : 1;
    p2 W[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const ulonglong2 v = __ldcs(L + (int64_t)(a * sa + b * sb) * vh);
        W[a][b] = p2{v.x, v.y};
      }
    p2 h[3];
    const ulonglong2 *P = reinterpret_cast<const ulonglong2 *>(in) + nb;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const ulonglong2 v = __ldg(P + c * vh);
      h[c] = p2{v.x, v.y};
    }
    if (bwd) {
      // conjugation by multiplies: sign-bit flips here (p2_conj) ran the
      // staggered hop 26% slower on GB300 (80.4 against 63.7 us at 24^3x48)
      const f2 cc = f2_make(1.f, -1.f);
#pragma unroll
      for (int k = 0; k < 9; ++k) W[k / 3][k % 3] = p2_scale_sgn(W[k / 3][k % 3], cc);
    }
    p2 r[3];
    matvec_half_ts(W, h, r);
    // sign: eta, boundary, +forward / -backward, and -1 for the adjoint
    float sg = stag_eta(mu, x, y, z) * (neg ? -1.f : 1.f) * (bwd ? -1.f : 1.f);
    if (DAG) sg = -sg;
    const f2 sv = f2_make(sg, sg);
#pragma unroll
    for (int c = 0; c < 3; ++c) acc[c] = p2_add_sgn(acc[c], r[c], sv);
  }
}

// out_p = a x_p + b D_hop(p <- 1-p) in   (DAG: D_hop^dag = -D_hop)
template <bool DAG, bool AXPY, bool NORM>
__global__ void __launch_bounds__(kStagThreads) stag_hop_kernel(Geom g, int p, const float4 *__restrict__ in,
                                                                const float4 *__restrict__ xv,
                                                                float4 *__restrict__ out,
                                                                const float4 *__restrict__ gauge, float2 a_split,
                                                                float2 b_split, double *partials,
                                                                const int *guard) {
  pdl_enter();
  if (guard && *guard) return;  // uniform across the grid
  const int64_t cb = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t vh = g.vh;
  dwacc nrm{0.f, 0.f};
  if (cb < vh) {
    p2 acc[3];
    stag_hop_sum<DAG>(g, p, cb, in, gauge, acc);
    // out = a x + (b / 2) acc  (the 1/2 is exact)
    const f2 bh = f2_make(0.5f * b_split.x, 0.5f * b_split.x);
    const mul2 Bm{bh, f2_make(0.5f * b_split.y, 0.5f * b_split.y)};
    const mul2 Am{f2_make(a_split.x, a_split.x), f2_make(a_split.y, a_split.y)};
    ulonglong2 *o = reinterpret_cast<ulonglong2 *>(out) + cb;
    p2 xs[3];
    if (AXPY) {
      const ulonglong2 *X = reinterpret_cast<const ulonglong2 *>(xv) + cb;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const ulonglong2 v = __ldg(X + c * vh);
        xs[c] = p2{v.x, v.y};
      }
    }
    acc2 nq{0ull, 0ull};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      acc2 R = acc2_first(Bm, p2_norm(acc[c]));
      if (AXPY) acc2_mad(R, Am, xs[c]);
      const p2 q = p2_norm(acc2_get(R));
      o[c * vh] = make_ulonglong2(q.h, q.l);
      if (NORM) {
        const mul2 Q{q.h, q.l};
        if (c == 0) nq = acc2_first(Q, q);
        else acc2_mad(nq, Q, q);
      }
    }
    if (NORM) {
      float s0, s1, c0, c1;
      f2_split(nq.s, s0, s1);
      f2_split(nq.c, c0, c1);
      float s, e;
      two_sum(s0, s1, s, e);
      nrm = dwacc{s, __fadd_rn(__fadd_rn(c0, c1), e)};
    }
  }
  if (NORM) {
    const double s = block_sum_dw(nrm);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
  }
}

__device__ __forceinline__ float2 split_dev2(double v) {
  const float h = __double2float_rn(v);
  return make_float2(h, __double2float_rn(v - (double)h));
}

// canonical (colour + 3*site, complex double) <-> double-word parity fields
__global__ void stag_pack_kernel(Geom g, const double *__restrict__ canon, float4 *even, float4 *odd) {
  const int64_t V = 2 * g.vh;
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  const int x = (int)(s % g.nx);
  int64_t r = s / g.nx;
  const int y = (int)(r % g.ny);
  r /= g.ny;
  const int z = (int)(r % g.nz);
  const int t = (int)(r / g.nz);
  float4 *base = ((x + y + z + t) & 1) ? odd : even;
  const int64_t cb = s >> 1;
  const double2 *src = reinterpret_cast<const double2 *>(canon) + 3 * s;
  for (int c = 0; c < 3; ++c) {
    const double2 v = src[c];
    const float2 re = split_dev2(v.x), im = split_dev2(v.y);
    base[c * g.vh + cb] = make_float4(re.x, im.x, re.y, im.y);
  }
}

__global__ void stag_unpack_kernel(Geom g, const float4 *even, const float4 *odd, double *__restrict__ canon) {
  const int64_t V = 2 * g.vh;
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  const int x = (int)(s % g.nx);
  int64_t r = s / g.nx;
  const int y = (int)(r % g.ny);
  r /= g.ny;
  const int z = (int)(r % g.nz);
  const int t = (int)(r / g.nz);
  const float4 *base = ((x + y + z + t) & 1) ? odd : even;
  const int64_t cb = s >> 1;
  double2 *dst = reinterpret_cast<double2 *>(canon) + 3 * s;
  for (int c = 0; c < 3; ++c) {
    const float4 v = base[c * g.vh + cb];
    dst[c] = make_double2((double)v.x + (double)v.z, (double)v.y + (double)v.w);
  }
}

// Second hop of the even-odd CG on m^2 - D_eo D_oe fused with the update:
// Ap = a p + (b/2) H t at the site in registers (a = m^2, b = -1), then
// x += alpha p, r -= alpha Ap and the block partial of ||r||^2; Ap is never
// stored.
__global__ void __launch_bounds__(kStagThreads)
    stag_hop_cg_kernel(Geom g, const float4 *__restrict__ t, const float4 *__restrict__ pv,
                       float4 *__restrict__ xs, float4 *__restrict__ r, const float4 *__restrict__ gauge,
                       float2 a_split, float2 b_split, const SolverScalars *__restrict__ S, double *partials) {
  pdl_enter();
  if (S->halt) return;  // uniform across the grid
  const int64_t cb = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t vh = g.vh;
  dwacc nrm{0.f, 0.f};
  if (cb < vh) {
    p2 acc[3];
    stag_hop_sum<false>(g, 0, cb, t, gauge, acc);
    const mul2 Bm{f2_make(0.5f * b_split.x, 0.5f * b_split.x), f2_make(0.5f * b_split.y, 0.5f * b_split.y)};
    const mul2 Am{f2_make(a_split.x, a_split.x), f2_make(a_split.y, a_split.y)};
    const float2 al = S->alpha_dw;
    const mul2 Al{f2_make(al.x, al.x), f2_make(al.y, al.y)};
    const mul2 Ml{f2_neg(Al.h), f2_neg(Al.l)};
    const ulonglong2 *P = reinterpret_cast<const ulonglong2 *>(pv) + cb;
    ulonglong2 *X = reinterpret_cast<ulonglong2 *>(xs) + cb;
    ulonglong2 *R = reinterpret_cast<ulonglong2 *>(r) + cb;
    acc2 nq{0ull, 0ull};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const ulonglong2 pw = __ldg(P + c * vh), xw = X[c * vh], rw = R[c * vh];
      const p2 pc{pw.x, pw.y};
      acc2 Q = acc2_first(Bm, p2_norm(acc[c]));
      acc2_mad(Q, Am, pc);
      const p2 q = p2_norm(acc2_get(Q));
      const p2 xn = p2_norm(p2_add(p2{xw.x, xw.y}, acc2_get(acc2_first(Al, pc))));
      const p2 rn = p2_norm(p2_add(p2{rw.x, rw.y}, acc2_get(acc2_first(Ml, q))));
      X[c * vh] = make_ulonglong2(xn.h, xn.l);
      R[c * vh] = make_ulonglong2(rn.h, rn.l);
      const mul2 Rm{rn.h, rn.l};
      if (c == 0) nq = acc2_first(Rm, rn);
      else acc2_mad(nq, Rm, rn);
    }
    float s0, s1, c0, c1;
    f2_split(nq.s, s0, s1);
    f2_split(nq.c, c0, c1);
    float sum, e;
    two_sum(s0, s1, sum, e);
    nrm = dwacc{sum, __fadd_rn(__fadd_rn(c0, c1), e)};
  }
  const double bs = block_sum_dw(nrm);
  if (threadIdx.x == 0) partials[blockIdx.x] = bs;
}

// p = r + beta p (beta = S->beta_dw) with the block partial of ||p||^2.
__global__ void stag_xpay_norm_kernel(float4 *__restrict__ p, const float4 *__restrict__ r, int64_t n,
                                      const SolverScalars *S, double *partials) {
  pdl_enter();
  if (S->halt) return;  // uniform across the grid
  const dw be = dw_make(S->beta_dw.x, S->beta_dw.y);
  dwacc A{0.f, 0.f};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    dw p_r, p_i, r_r, r_i;
    dwc_unpack(p[i], p_r, p_i);
    dwc_unpack(r[i], r_r, r_i);
    const dw nr = dw_add(r_r, dw_mul(be, p_r)), ni = dw_add(r_i, dw_mul(be, p_i));
    p[i] = dwc_pack(nr, ni);
    acc_sq(A, nr);
    acc_sq(A, ni);
  }
  const double bs = block_sum_dw(A);
  if (threadIdx.x == 0) partials[blockIdx.x] = bs;
}

// alpha = ||r||^2 / <p, (m^2 - D_eo D_oe) p> with <p, A p> = m^2 ||p||^2 + ||D_oe p||^2
// (D_eo^dag = -D_oe): the two norms come as per-block partials of the first
// hop (pt) and of the p update (pp); breakdown when the sum is not positive.
// This thread's share of sum(a[0..n)) in the fixed order i = tid, tid +
// blockDim.x, ...; all of its loads are in flight before its first add
// (out-of-range slots add 0).
__device__ __forceinline__ double thread_sum(const double *a, int n) {
  constexpr int kU = 16;
  double v = 0.0;
  for (int base = threadIdx.x; base < n; base += kU * blockDim.x) {
    double t[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int i = base + u * (int)blockDim.x;
      t[u] = i < n ? a[i] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) v += t[u];
  }
  return v;
}

__global__ void stag_alpha_kernel(const double *pt, int nt, const double *pp, int np, double m2,
                                  SolverScalars *S) {
  pdl_enter();
  if (S->halt) return;
  double vt = thread_sum(pt, nt), vp = thread_sum(pp, np);
  vt = block_sum_d(vt);
  vp = block_sum_d(vp);
  if (threadIdx.x == 0) {
    const double pAp = m2 * vp + vt;
    S->pAp = pAp;
    if (!(pAp > 0.0) || !isfinite(pAp)) {
      S->done = 2;
      S->halt = 1;
      return;
    }
    const double a = S->rr / pAp;
    S->alpha = a;
    S->alpha_dw = split_dev2(a);
    S->malpha_dw = split_dev2(-a);
    S->alpha_f = (float)a;
    S->malpha_f = (float)-a;
  }
}

}  // namespace

unsigned stag_blocks(int64_t vh) { return (unsigned)((vh + kStagThreads - 1) / kStagThreads); }

cudaError_t launch_stag_hop(const Geom &g, int out_parity, bool dagger, const float4 *in, const float4 *x,
                            float4 *out, const float4 *gauge_dw, double a, double b, double *partials,
                            cudaStream_t s, const int *guard) {
  note_launch();
  const float2 as = dw_split_host(a), bs = dw_split_host(b);
  const unsigned nb = stag_blocks(g.vh);
  const int key = (dagger ? 4 : 0) | (x ? 2 : 0) | (partials ? 1 : 0);
#define STAG_LAUNCH(D, A, N) \
  return launch_pdl(stag_hop_kernel<D, A, N>, nb, kStagThreads, 0, s, g, out_parity, in, x, out, gauge_dw, as, bs, \
                    partials, guard)
  switch (key) {
    case 0: STAG_LAUNCH(false, false, false);
    case 1: STAG_LAUNCH(false, false, true);
    case 2: STAG_LAUNCH(false, true, false);
    case 3: STAG_LAUNCH(false, true, true);
    case 4: STAG_LAUNCH(true, false, false);
    case 5: STAG_LAUNCH(true, false, true);
    case 6: STAG_LAUNCH(true, true, false);
    default: STAG_LAUNCH(true, true, true);
  }
#undef STAG_LAUNCH
}

cudaError_t launch_stag_pack(const Geom &g, const double *canon, float4 *even, float4 *odd, cudaStream_t s) {
  note_launch();
  stag_pack_kernel<<<(unsigned)((2 * g.vh + 255) / 256), 256, 0, s>>>(g, canon, even, odd);
  return cudaGetLastError();
}

cudaError_t launch_stag_unpack(const Geom &g, const float4 *even, const float4 *odd, double *canon,
                               cudaStream_t s) {
  note_launch();
  stag_unpack_kernel<<<(unsigned)((2 * g.vh + 255) / 256), 256, 0, s>>>(g, even, odd, canon);
  return cudaGetLastError();
}

cudaError_t GaugeEntry::ensure_staggered() {
  cudaError_t e = ensure_canon();
  if (e == cudaSuccess) e = ensure_reduce();
  const size_t full = 2 * stag_parity_bytes(g.vh);
  float4 **vs[] = {&sb, &sx, &sr, &sp, &sAp, &st, &srhs};
  for (float4 **v : vs)
    if (e == cudaSuccess && !*v) e = alloc_t(v, full);
  return e;
}

// Solve the staggered D x = b for the double-word b in G.sb (whole lattice,
// even half first); x into G.sx.
jqcd_status solve_staggered(GaugeEntry &G, double mass, const jqcd_solve_params &P, cudaStream_t s,
                            jqcd_solve_info *info, std::string *msg) {
#define CKT(call)                                                            \
  do {                                                                       \
    cudaError_t e_ = (call);                                                 \
    if (e_ != cudaSuccess) {                                                 \
      *msg = cudaGetErrorString(e_);                                         \
      return e_ == cudaErrorMemoryAllocation ? JQCD_ENOMEM : JQCD_ECUDA;     \
    }                                                                        \
  } while (0)
  if (!(mass > 0.0) || !std::isfinite(mass) || !(P.tol > 0.0) || P.maxiter < 1) {
    *msg = "staggered solve: mass > 0, tol > 0, maxiter >= 1";
    return JQCD_EINVAL;
  }
  CKT(G.ensure_staggered());
  const int64_t vh = G.g.vh;
  const int64_t n = 3 * vh;  // complex double-word numbers of one parity
  const int nblas = (int)blas_blocks(n);
  const float4 *U = (const float4 *)G.gauge_dw;
  float4 *be = G.sb, *bo = G.sb + n, *xe = G.sx, *xo = G.sx + n;
  float4 *r = G.sr, *p = G.sp, *Ap = G.sAp, *t = G.st, *rhs = G.srhs;
  SolverScalars *S = G.S;
  const double m2 = mass * mass;
  const double tol2 = P.tol * P.tol;
  CKT(cudaEventRecord(G.ev0, s));
  CKT(cudaMemsetAsync(S, 0, sizeof(SolverScalars), s));
  CKT(launch_dw_norm2(G.sb, 2 * n, G.partials, s));
  CKT(launch_finalize_sum(G.partials, (int)blas_blocks(2 * n), &S->b2, s));
  // rhs_e = m b_e - D_eo b_o
  CKT(launch_stag_hop(G.g, 0, false, bo, be, rhs, U, mass, -1.0, nullptr, s));
  CKT(launch_dw_norm2(rhs, n, G.partials, s));
  CKT(launch_finalize_sum(G.partials, nblas, &S->rhs2, s));
  CKT(launch_dw_zero(xe, n, s));
  CKT(launch_dw_copy(r, rhs, n, s));
  CKT(launch_dw_norm2(r, n, G.partials, s));
  CKT(launch_cg_start(G.partials, nblas, S, tol2, P.maxiter, 0.0, s));
  CKT(launch_dw_copy(p, r, n, s));
  // partials: ||t||^2 and ||r||^2 per hop block from the start, ||p||^2 per
  // vector block after them
  const int nstag = (int)stag_blocks(vh);
  double *part_t = G.partials, *part_p = G.partials + nstag;
  CKT(launch_dw_norm2(p, n, part_p, s));
  long long hops = 1;
  int restarts = 0;
  jqcd_status st = JQCD_OK;
  auto apply = [&](const float4 *in, float4 *out, const int *guard) -> cudaError_t {
    // t_o = D_oe in; out = m^2 in - D_eo t_o
    cudaError_t e = launch_stag_hop(G.g, 1, false, in, nullptr, t, U, 0.0, 1.0, nullptr, s, guard);
    if (!e) e = launch_stag_hop(G.g, 0, false, t, in, out, U, m2, -1.0, nullptr, s, guard);
    return e;
  };
  for (;;) {
    for (;;) {
      for (int k = 0; k < 8; ++k) {
        // t = D_oe p with ||t||^2; alpha from m^2 ||p||^2 + ||t||^2; the second
        // hop applies the update and forms ||r||^2; beta; p = r + beta p, ||p||^2
        CKT(launch_stag_hop(G.g, 1, false, p, nullptr, t, U, 0.0, 1.0, part_t, s, &S->halt));
        note_launch();
        CKT(launch_pdl(stag_alpha_kernel, 1, kReduceThreads, 0, s, part_t, nstag, part_p, nblas, m2, S));
        note_launch();
        CKT(launch_pdl(stag_hop_cg_kernel, nstag, kStagThreads, 0, s, G.g, t, p, xe, r, U, dw_split_host(m2),
                       dw_split_host(-1.0), S, part_t));
        CKT(launch_cg_beta(part_t, nstag, S, s));
        note_launch();
        CKT(launch_pdl(stag_xpay_norm_kernel, nblas, kBlasThreads, 0, s, p, r, n, S, part_p));
      }
      CKT(cudaMemcpyAsync(G.S_host, S, sizeof(SolverScalars), cudaMemcpyDeviceToHost, s));
      CKT(cudaStreamSynchronize(s));
      if (G.S_host->done || G.S_host->iters >= P.maxiter) break;
    }
    if (G.S_host->done == 2) {
      *msg = "staggered CG breakdown (<p,Ap> <= 0 or not finite)";
      st = JQCD_EBREAKDOWN;
      break;
    }
    // true residual
    CKT(apply(xe, Ap, nullptr));
    hops += 2;
    CKT(launch_dw_xmy_norm(r, rhs, Ap, n, G.partials, s));
    CKT(launch_finalize_sum(G.partials, nblas, &S->true_rr, s));
    CKT(cudaMemcpyAsync(G.S_host, S, sizeof(SolverScalars), cudaMemcpyDeviceToHost, s));
    CKT(cudaStreamSynchronize(s));
    if (G.S_host->true_rr <= tol2 * G.S_host->rhs2) break;
    if (G.S_host->iters >= P.maxiter || restarts >= 8) {
      st = JQCD_ENOCONV;
      *msg = "maximum iterations reached";
      break;
    }
    ++restarts;
    CKT(launch_cg_start(G.partials, nblas, S, tol2, P.maxiter, 0.0, s));
    CKT(launch_dw_copy(p, r, n, s));
    CKT(launch_dw_norm2(p, n, part_p, s));
  }
  // x_o = (b_o - D_oe x_e) / m
  CKT(launch_stag_hop(G.g, 1, false, xe, bo, xo, U, 1.0 / mass, -1.0 / mass, nullptr, s));
  hops += 1;
  CKT(cudaEventRecord(G.ev1, s));
  // ||b - D x|| (whole lattice): t = D x into Ap (even) and t (odd)
  CKT(launch_stag_hop(G.g, 0, false, xo, xe, Ap, U, mass, 1.0, nullptr, s));
  CKT(launch_stag_hop(G.g, 1, false, xe, xo, t, U, mass, 1.0, nullptr, s));
  CKT(launch_dw_xmy_norm(r, be, Ap, n, G.partials, s));
  CKT(launch_finalize_sum(G.partials, nblas, &S->full_rr, s));
  CKT(launch_dw_xmy_norm(rhs, bo, t, n, G.partials, s));  // rhs reused as scratch
  CKT(launch_finalize_sum(G.partials, nblas, &S->rr_new, s));
  CKT(cudaMemcpyAsync(G.S_host, S, sizeof(SolverScalars), cudaMemcpyDeviceToHost, s));
  CKT(cudaStreamSynchronize(s));
  float ms = 0.f;
  CKT(cudaEventElapsedTime(&ms, G.ev0, G.ev1));
  const SolverScalars &H = *G.S_host;
  memset(info, 0, sizeof *info);
  info->iters = H.iters;
  info->restarts = restarts;
  info->true_rel_resid = H.rhs2 > 0 ? std::sqrt(H.true_rr / H.rhs2) : 0.0;
  info->full_rel_resid = H.b2 > 0 ? std::sqrt((H.full_rr + H.rr_new) / H.b2) : 0.0;
  info->gpu_seconds = ms * 1e-3;
  hops += 2LL * H.iters;
  info->hop_count = (double)hops;
  info->hop_bytes = (double)hops * (double)vh * kStagHopBytes;
  info->status = st;
  return st;
#undef CKT
}

}  // namespace jqcd
