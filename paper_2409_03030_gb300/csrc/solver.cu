// Solver drivers: conjugate gradient on the normal equations, even-odd
// source preparation and reconstruction (paper: solve_DinvX! with eps_CG).
//
// Conjugate gradient (Hestenes-Stiefel) on A x = rhs, A Hermitian positive
// definite (A = Mhat^dag Mhat on the even sites, or D^dag D):
//   r = rhs - A x, p = r, rr = <r,r>
//   loop: alpha = rr / <p,Ap>;  x += alpha p;  r -= alpha Ap;
//         rr' = <r,r>;  stop if rr' <= tol^2 <rhs,rhs>;  p = r + (rr'/rr) p
// All scalars live on the device: <p,Ap> = ||Mhat p||^2 comes fused out of
// the second hop, <r,r> out of the vector update, and single-block kernels
// turn the partial sums into alpha and beta.  The host only polls the
// scalars every kCheckEvery iterations; kernels of finished solves return
// at once.  After the loop the residual is recomputed from x; if it misses
// the tolerance CG restarts from x.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>

#include "kernels.h"
#include "solver.h"

namespace jqcd {

namespace {
constexpr int kCheckEvery = 8;
constexpr int kMaxRestarts = 8;
}  // namespace

GaugeEntry::~GaugeEntry() {
  for (void *p : device_allocs) cudaFree(p);
  if (S_host) cudaFreeHost(S_host);
  if (ms_S_host) cudaFreeHost(ms_S_host);
  if (ev0) cudaEventDestroy(ev0);
  if (ev1) cudaEventDestroy(ev1);
  if (ev_fork) cudaEventDestroy(ev_fork);
  if (ev_join) cudaEventDestroy(ev_join);
  if (side) cudaStreamDestroy(side);
}

cudaError_t GaugeEntry::alloc(void **p, size_t bytes) {
  *p = nullptr;
  cudaError_t e = cudaMalloc(p, bytes < 256 ? 256 : bytes);
  if (e == cudaSuccess) device_allocs.push_back(*p);
  return e;
}

cudaError_t GaugeEntry::ensure_canon() {
  if (canon) return cudaSuccess;
  return alloc_t(&canon, canon_bytes());
}

int GaugeEntry::n_partials() const {
  return 2 * (int)dw_hop_blocks(g.vh) + (int)blas_blocks(24 * g.vh) + 64;
}

cudaError_t GaugeEntry::ensure_reduce() {
  cudaError_t e = cudaSuccess;
  if (!side) e = cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking);
  if (e == cudaSuccess && !ev_fork) e = cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming);
  if (e == cudaSuccess && !ev_join) e = cudaEventCreateWithFlags(&ev_join, cudaEventDisableTiming);
  if (!partials) e = alloc_t(&partials, sizeof(double) * n_partials());
  if (e == cudaSuccess && !S) e = alloc_t(&S, sizeof(SolverScalars));
  if (e == cudaSuccess && !S_host) e = cudaMallocHost(&S_host, sizeof(SolverScalars));
  if (e == cudaSuccess && !ev0) e = cudaEventCreate(&ev0);
  if (e == cudaSuccess && !ev1) e = cudaEventCreate(&ev1);
  return e;
}

cudaError_t GaugeEntry::ensure_tmp(int prec) {
  cudaError_t e = cudaSuccess;
  const size_t b = spinor_parity_bytes(prec, g.vh);
  if (!tmp[prec]) e = alloc(&tmp[prec], b);
  if (e == cudaSuccess && !tmp2[prec]) e = alloc(&tmp2[prec], b);
  return e;
}

cudaError_t GaugeEntry::ensure_solver() {
  cudaError_t e = ensure_canon();
  if (e == cudaSuccess) e = ensure_reduce();
  const size_t full = 2 * spinor_parity_bytes(PREC_DW, g.vh);
  float4 **vs[] = {&vb, &vsol, &vr, &vp, &vAp, &vw, &vt, &vrhs};
  for (float4 **v : vs)
    if (e == cudaSuccess && !*v) e = alloc_t(v, full);
  return e;
}

cudaError_t GaugeEntry::ensure_force() {
  cudaError_t e = ensure_solver();
  const size_t full = 2 * spinor_parity_bytes(PREC_DW, g.vh);
  float4 **vs[] = {&feta, &fX, &fY};
  for (float4 **v : vs)
    if (e == cudaSuccess && !*v) e = alloc_t(v, full);
  if (e == cudaSuccess && !fout) e = alloc_t(&fout, linkfield_bytes());
  if (e == cudaSuccess && !lcanon) e = alloc_t(&lcanon, link_canon_bytes());
  return e;
}

cudaError_t GaugeEntry::ensure_mixed(int hop_prec) {
  const int k = hop_prec == PREC_F16N ? 1 : 0;
  const size_t f32 = spinor_parity_bytes(PREC_F32, g.vh);
  const size_t hb = spinor_parity_bytes(hop_prec, g.vh);
  cudaError_t e = cudaSuccess;
  if (!mx) e = alloc(&mx, f32);
  if (e == cudaSuccess && !mr) e = alloc(&mr, f32);
  void **vs[] = {&mp[k], &mw[k], &mt[k]};
  for (void **v : vs)
    if (e == cudaSuccess && !*v) e = alloc(v, hb);
  return e;
}

cudaError_t GaugeEntry::ensure_f64() {
  cudaError_t e = ensure_canon();
  if (e == cudaSuccess) e = ensure_reduce();
  const size_t full = 2 * spinor_parity_bytes(PREC_F64, g.vh);
  double2 **vs[] = {&fb, &fsol, &fr, &fp, &fAp, &fw, &ft, &frhs};
  for (double2 **v : vs)
    if (e == cudaSuccess && !*v) e = alloc_t(v, full);
  return e;
}

const void *GaugeEntry::gauge_for(int prec) const {
  switch (prec) {
    case PREC_DW: return gauge_dw;
    case PREC_F64: return gauge_f64;
    default: return gauge_f32;
  }
}

HopParams GaugeEntry::hop_params(int prec, int out_parity, const void *in, const void *x, void *out,
                                 double a, double b, double *parts) const {
  HopParams P;
  memset(&P, 0, sizeof P);
  P.out = out;
  P.in = in;
  P.x = x;
  P.gauge = gauge_for(prec);
  P.g = g;
  P.out_parity = out_parity;
  P.a = a;
  P.b = b;
  const float ah = (float)a, bh = (float)b;
  P.a_split = make_float2(ah, (float)(a - (double)ah));
  P.b_split = make_float2(bh, (float)(b - (double)bh));
  P.partials = parts;
  P.guard = nullptr;
  return P;
}

cudaError_t apply_mdagm(const GaugeEntry &G, int prec, double kappa, const void *in, void *out,
                        void *t_odd, void *w_even, double *partials, const int *guard,
                        cudaStream_t s) {
  const double k2 = -kappa * kappa;
  HopParams P = G.hop_params(prec, 1, in, nullptr, t_odd, 0.0, 1.0, nullptr);
  P.guard = guard;
  cudaError_t e = launch_hop(prec, P, false, false, false, s);           // t = H_oe in
  if (e) return e;
  P = G.hop_params(prec, 0, t_odd, in, w_even, 1.0, k2, partials);
  P.guard = guard;
  e = launch_hop(prec, P, false, true, partials != nullptr, s);          // w = in - k^2 H_eo t
  if (e) return e;
  P = G.hop_params(prec, 1, w_even, nullptr, t_odd, 0.0, 1.0, nullptr);
  P.guard = guard;
  e = launch_hop(prec, P, true, false, false, s);                        // t = H^dag_oe w
  if (e) return e;
  P = G.hop_params(prec, 0, t_odd, w_even, out, 1.0, k2, nullptr);
  P.guard = guard;
  return launch_hop(prec, P, true, true, false, s);                      // out = w - k^2 H^dag_eo t
}

namespace {

// Whole-lattice D (or D^dag) on double-word vectors: out = in - kappa H in,
// optional per-block partials of ||out||^2 (2 * dw_hop_blocks entries).
cudaError_t apply_dirac_dw(const GaugeEntry &G, double kappa, bool dag, float4 *in, float4 *out,
                           double *partials, const int *guard, cudaStream_t s) {
  const int nb = (int)dw_hop_blocks(G.g.vh);
  HopParams Pe = G.hop_params(PREC_DW, 0, G.vec_odd(in), G.vec_even(in), G.vec_even(out), 1.0,
                              -kappa, partials);
  Pe.guard = guard;
  cudaError_t e = launch_hop(PREC_DW, Pe, dag, true, partials != nullptr, s);
  if (e) return e;
  HopParams Po = G.hop_params(PREC_DW, 1, G.vec_even(in), G.vec_odd(in), G.vec_odd(out), 1.0,
                              -kappa, partials ? partials + nb : nullptr);
  Po.guard = guard;
  return launch_hop(PREC_DW, Po, dag, true, partials != nullptr, s);
}

struct DwSystem {
  GaugeEntry &G;
  double kappa;
  bool eo;
  cudaStream_t s;
  int64_t n;      // complex elements of the system's vectors
  int n_hop_partials;
  long long hops = 0;
  double hop_bytes = 0;

  void count(int plain, int axpy) {
    hops += plain + axpy;
    hop_bytes += (double)G.g.vh * (1536.0 * (plain + axpy) + 192.0 * axpy);
  }

  // out = A in, partials <- ||M in||^2 (M = Mhat or D).  Guarded applies
  // inside the CG loop are counted from the iteration count instead.
  cudaError_t apply(float4 *in, float4 *out, double *partials, const int *guard) {
    if (!guard) count(eo ? 2 : 0, eo ? 2 : 4);
    if (eo) {
      return apply_mdagm(G, PREC_DW, kappa, in, out, G.vec_odd(G.vt), G.vec_even(G.vw), partials,
                         guard, s);
    }
    cudaError_t e = apply_dirac_dw(G, kappa, false, in, G.vw, partials, guard, s);
    if (e) return e;
    return apply_dirac_dw(G, kappa, true, G.vw, out, nullptr, guard, s);
  }
};

// One double-word CG iteration on the even-odd system, p -> (x, r, p):
// w = Mhat p with ||w||^2 = <p, Mhat^dag Mhat p> fused into the second hop,
// alpha, then the last hop of Mhat^dag w applies x += alpha p, r -= alpha Ap
// and forms ||r||^2 itself (Ap is never stored), beta, p = r + beta p.
// The inner solver of the mixed CG on small grids (at most
// JQCD_FIN_MAX_BLOCKS hop blocks) takes alpha and beta in the last block of
// the hop that writes their partials (cg_steps.cuh) instead of a
// single-block launch after it (measured on GB300: mixed FP16 solve at 16^4
// 3.08 -> 2.83 ms).  The double-word iteration keeps the separate launches:
// there the last-block form gained nothing at 16^4 and lost 2% at 8^4.
static bool fuse_scalar_steps(int nb) { return nb <= JQCD_FIN_MAX_BLOCKS; }

// alpha = rr / <p, A p> from the partials of the hop just queued on s, on
// the side stream: the next hop (t = H^dag_oe w) does not read alpha, so the
// single-block step runs beside it; s waits for it before the last hop
// (measured on GB300: double-word solve 33.62 -> 33.53 ms at 24^3x48, 4.48 ->
// 4.39 ms at 16^4; mixed FP16 13.90 -> 13.81 ms).
static cudaError_t alpha_fork(GaugeEntry &G, int nb, SolverScalars *S, cudaStream_t s) {
  if (!G.side) return launch_cg_alpha(G.partials, nb, S, s);
  cudaError_t e = cudaEventRecord(G.ev_fork, s);
  if (!e) e = cudaStreamWaitEvent(G.side, G.ev_fork, 0);
  if (!e) e = launch_cg_alpha(G.partials, nb, S, G.side);
  if (!e) e = cudaEventRecord(G.ev_join, G.side);
  return e;
}
static cudaError_t alpha_join(GaugeEntry &G, cudaStream_t s) {
  if (!G.side) return cudaSuccess;
  return cudaStreamWaitEvent(s, G.ev_join, 0);
}

cudaError_t dw_eo_cg_iteration(GaugeEntry &G, double kappa, SolverScalars *S, cudaStream_t s) {
  const double k2 = -kappa * kappa;
  const int nb = (int)dw_hop_blocks(G.g.vh);
  const int *guard = &S->halt;
  float4 *t = G.vec_odd(G.vt), *w = G.vec_even(G.vw);
  HopParams P = G.hop_params(PREC_DW, 1, G.vp, nullptr, t, 0.0, 1.0, nullptr);
  P.guard = guard;
  cudaError_t e = launch_hop(PREC_DW, P, false, false, false, s);  // t = H_oe p
  if (e) return e;
  P = G.hop_params(PREC_DW, 0, t, G.vp, w, 1.0, k2, G.partials);
  P.guard = guard;
  e = launch_hop(PREC_DW, P, false, true, true, s);  // w = p - k^2 H_eo t, ||w||^2
  if (e) return e;
  e = alpha_fork(G, nb, S, s);
  if (e) return e;
  P = G.hop_params(PREC_DW, 1, w, nullptr, t, 0.0, 1.0, nullptr);
  P.guard = guard;
  e = launch_hop(PREC_DW, P, true, false, false, s);  // t = H^dag_oe w
  if (e) return e;
  e = alpha_join(G, s);
  if (e) return e;
  P = G.hop_params(PREC_DW, 0, t, w, nullptr, 1.0, k2, G.partials);
  P.guard = guard;
  e = launch_hop_dw_cg(P, G.vp, G.vsol, G.vr, S, s);  // Ap = w - k^2 H^dag_eo t; x, r, ||r||^2
  if (e) return e;
  e = launch_cg_beta(G.partials, nb, S, s);
  if (e) return e;
  return launch_dw_xpay(G.vp, G.vr, 12 * G.g.vh, S, s);
}

// One iteration of the inner CG of the mixed solver in hop precision hp on
// the vectors p, t, w of that precision (FP32 xs and rs): the same order as
// the double-word iteration, the update fused into the last hop.
cudaError_t lp_eo_cg_iteration(GaugeEntry &G, int hp, int mk, double kappa, SolverScalars *S,
                               cudaStream_t s) {
  const double k2 = -kappa * kappa;
  const int nb = (int)hop_blocks(G.g.vh);
  const bool fuse = fuse_scalar_steps(nb);
  const int *guard = &S->halt;
  void *p = G.mp[mk], *t = G.mt[mk], *w = G.mw[mk];
  HopParams P = G.hop_params(hp, 1, p, nullptr, t, 0.0, 1.0, nullptr);
  P.guard = guard;
  cudaError_t e = launch_hop(hp, P, false, false, false, s);  // t = H_oe p
  if (e) return e;
  P = G.hop_params(hp, 0, t, p, w, 1.0, k2, G.partials);
  P.guard = guard;
  if (fuse) {
    P.fin = FIN_ALPHA;
    P.fin_S = S;
  }
  e = launch_hop(hp, P, false, true, true, s);  // w = p - k^2 H_eo t, ||w||^2
  if (e) return e;
  if (!fuse && (e = alpha_fork(G, nb, S, s))) return e;
  P = G.hop_params(hp, 1, w, nullptr, t, 0.0, 1.0, nullptr);
  P.guard = guard;
  e = launch_hop(hp, P, true, false, false, s);  // t = H^dag_oe w
  if (e) return e;
  if (!fuse && (e = alpha_join(G, s))) return e;
  P = G.hop_params(hp, 0, t, w, nullptr, 1.0, k2, G.partials);
  P.guard = guard;
  if (fuse) {
    P.fin = FIN_MIXED_BETA;
    P.fin_S = S;
  }
  e = launch_hop_lp_cg(hp, P, p, (float4 *)G.mx, (float4 *)G.mr, S, s);
  if (e) return e;
  if (!fuse && (e = launch_mixed_beta(G.partials, nb, S, s))) return e;
  return launch_mixed_xpay(hp, p, (const float4 *)G.mr, G.g.vh, S, s);
}

// ---- native FP64 system (JQCD_CG_F64) -------------------------------------
double2 *f64_even(double2 *v) { return v; }
double2 *f64_odd(const GaugeEntry &G, double2 *v) { return v + 12 * G.g.vh; }

// Whole-lattice D (or D^dag) on FP64 vectors: out = in - kappa H in, optional
// per-block partials of ||out||^2 (2 * hop_blocks entries).
cudaError_t apply_dirac_f64(const GaugeEntry &G, double kappa, bool dag, double2 *in, double2 *out,
                            double *partials, const int *guard, cudaStream_t s) {
  const int nb = (int)hop_blocks(G.g.vh);
  HopParams Pe = G.hop_params(PREC_F64, 0, f64_odd(G, in), f64_even(in), f64_even(out), 1.0,
                              -kappa, partials);
  Pe.guard = guard;
  cudaError_t e = launch_hop(PREC_F64, Pe, dag, true, partials != nullptr, s);
  if (e) return e;
  HopParams Po = G.hop_params(PREC_F64, 1, f64_even(in), f64_odd(G, in), f64_odd(G, out), 1.0,
                              -kappa, partials ? partials + nb : nullptr);
  Po.guard = guard;
  return launch_hop(PREC_F64, Po, dag, true, partials != nullptr, s);
}

// out = A in for the FP64 CG system (A = Mhat^dag Mhat on the even sites, or
// D^dag D on the whole lattice); partials <- ||M in||^2 per hop block.
cudaError_t apply_a_f64(GaugeEntry &G, double kappa, bool eo, double2 *in, double2 *out,
                        double *partials, const int *guard, cudaStream_t s) {
  if (eo)
    return apply_mdagm(G, PREC_F64, kappa, in, out, f64_odd(G, G.ft), f64_even(G.fw), partials,
                       guard, s);
  cudaError_t e = apply_dirac_f64(G, kappa, false, in, G.fw, partials, guard, s);
  if (e) return e;
  return apply_dirac_f64(G, kappa, true, G.fw, out, nullptr, guard, s);
}

}  // namespace

// Bytes per output site of one hop in precision `prec` (+ the axpy operand).
static double hop_site_bytes(int prec, bool axpy) {
  switch (prec) {
    case PREC_F32: return 576.0 + (axpy ? 96.0 : 0.0);
    case PREC_F16N: return 488.0 + (axpy ? 52.0 : 0.0);
    default: return 1536.0 + (axpy ? 192.0 : 0.0);
  }
}

// Conjugate gradient on the normal equations.  mode JQCD_CG_DW: every vector
// and operator in double-word precision.  Mixed modes: inner CG in FP32 or
// FP16+norm on the even-odd system, reliable updates in double-word.
static jqcd_status solve_cg(GaugeEntry &G, const jqcd_solve_params &P, cudaStream_t s,
                            jqcd_solve_info *info, std::string *msg) {
  const bool eo = P.eo != 0;
  const bool mixed = P.mode == JQCD_CG_MIXED_F32 || P.mode == JQCD_CG_MIXED_F16;
  const int hp = P.mode == JQCD_CG_MIXED_F16 ? PREC_F16N : PREC_F32;
  const int mk = hp == PREC_F16N ? 1 : 0;  // index of the hop-precision vectors
  DwSystem A{G, P.kappa, eo, s, (eo ? 12 : 24) * G.g.vh, (eo ? 1 : 2) * (int)dw_hop_blocks(G.g.vh)};
  const int nblas = (int)blas_blocks(A.n);
  const double tol2 = P.tol * P.tol;
  const double delta = P.delta > 0.0 ? P.delta : 0.01;
  const int64_t vh = G.g.vh;
  SolverScalars *S = G.S;
  double low_bytes = 0.0;
  long long low_hops = 0;
#define CKS(call)                                              \
  do {                                                         \
    cudaError_t e_ = (call);                                   \
    if (e_ != cudaSuccess) {                                   \
      *msg = cudaGetErrorString(e_);                           \
      return e_ == cudaErrorMemoryAllocation ? JQCD_ENOMEM : JQCD_ECUDA; \
    }                                                          \
  } while (0)
  if (mixed) CKS(G.ensure_mixed(hp));

  CKS(cudaEventRecord(G.ev0, s));
  CKS(cudaMemsetAsync(S, 0, sizeof(SolverScalars), s));
  // ||b||^2 of D x = b
  CKS(launch_dw_norm2(G.vb, 24 * vh, G.partials, s));
  CKS(launch_finalize_sum(G.partials, (int)blas_blocks(24 * vh), &S->b2, s));
  // right-hand side of the CG system
  if (eo) {
    // bhat_e = b_e + kappa H_eo b_o  (into vw even)
    HopParams Pb = G.hop_params(PREC_DW, 0, G.vec_odd(G.vb), G.vec_even(G.vb), G.vec_even(G.vw),
                                1.0, P.kappa, nullptr);
    CKS(launch_hop(PREC_DW, Pb, false, true, false, s));
    // rhs = Mhat^dag bhat: t = H^dag_oe bhat; rhs = bhat - kappa^2 H^dag_eo t
    HopParams P1 = G.hop_params(PREC_DW, 1, G.vec_even(G.vw), nullptr, G.vec_odd(G.vt), 0.0, 1.0,
                                nullptr);
    CKS(launch_hop(PREC_DW, P1, true, false, false, s));
    HopParams P2 = G.hop_params(PREC_DW, 0, G.vec_odd(G.vt), G.vec_even(G.vw), G.vec_even(G.vrhs),
                                1.0, -P.kappa * P.kappa, nullptr);
    CKS(launch_hop(PREC_DW, P2, true, true, false, s));
    A.count(2, 1);
  } else {
    CKS(apply_dirac_dw(G, P.kappa, true, G.vb, G.vrhs, nullptr, nullptr, s));  // rhs = D^dag b
    A.count(0, 2);
  }
  CKS(launch_dw_norm2(G.vrhs, A.n, G.partials, s));
  CKS(launch_finalize_sum(G.partials, nblas, &S->rhs2, s));
  // start vector and residual
  if (P.use_x0) {
    CKS(A.apply(G.vsol, G.vAp, nullptr, nullptr));
    CKS(launch_dw_xmy_norm(G.vr, G.vrhs, G.vAp, A.n, G.partials, s));
  } else {
    CKS(launch_dw_zero(G.vsol, 24 * vh, s));
    CKS(launch_dw_copy(G.vr, G.vrhs, A.n, s));
    CKS(launch_dw_norm2(G.vr, A.n, G.partials, s));
  }
  CKS(launch_cg_start(G.partials, nblas, S, tol2, P.maxiter, delta * delta, s));
  auto start_direction = [&]() -> cudaError_t {
    if (!mixed) return launch_dw_copy(G.vp, G.vr, A.n, s);
    cudaError_t e = launch_dw_to_f32((float4 *)G.mr, G.vr, vh, s);
    if (!e) e = cudaMemsetAsync(G.mx, 0, spinor_parity_bytes(PREC_F32, vh), s);
    if (!e) e = launch_mixed_copy(hp, G.mp[mk], (const float4 *)G.mr, vh, s);
    return e;
  };
  CKS(start_direction());

  int restarts = 0;
  jqcd_status st = JQCD_OK;
  for (;;) {
    // main loop: poll the device scalars every kCheckEvery iterations
    for (;;) {
      for (int k = 0; k < kCheckEvery; ++k) {
        if (!mixed && eo) {
          CKS(dw_eo_cg_iteration(G, P.kappa, S, s));
        } else if (!mixed) {
          CKS(A.apply(G.vp, G.vAp, G.partials, &S->halt));
          CKS(launch_cg_alpha(G.partials, A.n_hop_partials, S, s));
          CKS(launch_dw_cg_update(G.vsol, G.vr, G.vp, G.vAp, A.n, S, G.partials, s));
          CKS(launch_cg_beta(G.partials, nblas, S, s));
          CKS(launch_dw_xpay(G.vp, G.vr, A.n, S, s));
        } else {
          CKS(lp_eo_cg_iteration(G, hp, mk, P.kappa, S, s));
        }
      }
      CKS(cudaMemcpyAsync(G.S_host, S, sizeof(SolverScalars), cudaMemcpyDeviceToHost, s));
      CKS(cudaStreamSynchronize(s));
      if (mixed && G.S_host->need_update && !G.S_host->done) {
        // reliable update: x += x_s; r = rhs - A x in double-word; resume
        CKS(launch_dw_add_f32(G.vsol, (float4 *)G.mx, vh, s));
        CKS(A.apply(G.vsol, G.vAp, nullptr, nullptr));
        CKS(launch_dw_xmy_norm(G.vr, G.vrhs, G.vAp, A.n, G.partials, s));
        CKS(launch_mixed_after_update(G.partials, nblas, S, s));
        CKS(launch_dw_to_f32((float4 *)G.mr, G.vr, vh, s));
        CKS(launch_mixed_xpay(hp, G.mp[mk], (const float4 *)G.mr, vh, S, s));
        CKS(cudaMemcpyAsync(G.S_host, S, sizeof(SolverScalars), cudaMemcpyDeviceToHost, s));
        CKS(cudaStreamSynchronize(s));
      }
      if (P.verbose >= 3)
        fprintf(stderr, "jqcd cg: iter %d  |r|/|rhs| = %.3e  reliable updates %d\n",
                G.S_host->iters,
                G.S_host->rhs2 > 0 ? std::sqrt(G.S_host->rr / G.S_host->rhs2) : 0.0,
                G.S_host->reliable_updates);
      if (G.S_host->done) break;
      if (!mixed && G.S_host->iters >= P.maxiter) break;
    }
    if (G.S_host->done == 2) {
      *msg = "CG breakdown (<p,Ap> <= 0 or not finite)";
      st = JQCD_EBREAKDOWN;
      break;
    }
    if (!mixed) {
      // true residual of the CG system (the mixed loop ends on one)
      CKS(A.apply(G.vsol, G.vAp, nullptr, nullptr));
      CKS(launch_dw_xmy_norm(G.vr, G.vrhs, G.vAp, A.n, G.partials, s));
      CKS(launch_finalize_sum(G.partials, nblas, &S->true_rr, s));
      CKS(cudaMemcpyAsync(G.S_host, S, sizeof(SolverScalars), cudaMemcpyDeviceToHost, s));
      CKS(cudaStreamSynchronize(s));
    }
    const double rhs2 = G.S_host->rhs2;
    const bool ok = G.S_host->true_rr <= tol2 * rhs2;
    if (ok) break;
    if (G.S_host->iters >= P.maxiter || restarts >= kMaxRestarts) {
      st = JQCD_ENOCONV;
      *msg = "maximum iterations reached";
      break;
    }
    ++restarts;  // restart from x with the recomputed residual
    CKS(launch_cg_start(G.partials, nblas, S, tol2, P.maxiter, delta * delta, s));
    CKS(start_direction());
  }
  // even-odd reconstruction x_o = b_o + kappa H_oe x_e
  if (eo) {
    HopParams Pr = G.hop_params(PREC_DW, 1, G.vec_even(G.vsol), G.vec_odd(G.vb), G.vec_odd(G.vsol),
                                1.0, P.kappa, nullptr);
    CKS(launch_hop(PREC_DW, Pr, false, true, false, s));
    A.count(0, 1);
  }
  CKS(cudaEventRecord(G.ev1, s));
  G.x_host_queued = false;
  if (G.x_host_out && G.side && (st == JQCD_OK || st == JQCD_ENOCONV)) {
    // x is final: its unpack and copy to the host overlap the residual below
    CKS(cudaStreamWaitEvent(G.side, G.ev1, 0));
    CKS(launch_spinor_unpack(G.g, PREC_DW, G.vec_even(G.vsol), G.vec_odd(G.vsol), G.canon, G.side));
    CKS(cudaMemcpyAsync(G.x_host_out, G.canon, G.canon_bytes(), cudaMemcpyDeviceToHost, G.side));
    CKS(cudaEventRecord(G.ev_join, G.side));
    G.x_host_queued = true;
  }
  // ||b - D x||^2 (not part of the timed solve)
  CKS(apply_dirac_dw(G, P.kappa, false, G.vsol, G.vw, nullptr, nullptr, s));
  CKS(launch_dw_xmy_norm(G.vAp, G.vb, G.vw, 24 * vh, G.partials, s));
  CKS(launch_finalize_sum(G.partials, (int)blas_blocks(24 * vh), &S->full_rr, s));
  CKS(cudaMemcpyAsync(G.S_host, S, sizeof(SolverScalars), cudaMemcpyDeviceToHost, s));
  CKS(cudaStreamSynchronize(s));
  float ms = 0.f;
  CKS(cudaEventElapsedTime(&ms, G.ev0, G.ev1));
  const SolverScalars &H = *G.S_host;
  info->iters = H.iters;
  info->restarts = restarts;
  info->reliable_updates = H.reliable_updates;
  info->true_rel_resid = H.rhs2 > 0 ? std::sqrt(H.true_rr / H.rhs2) : 0.0;
  info->full_rel_resid = H.b2 > 0 ? std::sqrt(H.full_rr / H.b2) : 0.0;
  info->gpu_seconds = ms * 1e-3;
  if (!mixed) {
    // loop hops: four per completed iteration
    for (int i = 0; i < H.iters; ++i) A.count(eo ? 2 : 0, eo ? 2 : 4);
  } else {
    low_hops = 4LL * H.iters;
    low_bytes = (double)vh * H.iters * 2.0 * (hop_site_bytes(hp, false) + hop_site_bytes(hp, true));
    // double-word applications of A in the reliable updates (counted by apply)
  }
  info->hop_count = (double)(A.hops + low_hops);
  info->hop_bytes = A.hop_bytes + low_bytes;
  return st;
#undef CKS
}

// Plain conjugate gradient in native FP64: every vector, operator and
// reduction in IEEE double (the hop is hop_kernel<PREC_F64>, the vector
// kernels blas_f64.cu).  Same iteration, stopping rule, true-residual check
// and restarts as the double-word solver; b in G.fb, x (start vector when
// use_x0) and the solution in G.fsol, whole lattice in the JQCD_PREC_F64
// layout.  One iteration is eight launches: t = H_oe p; w = p - k^2 H_eo t
// with ||w||^2; alpha; t = H^dag_oe w; Ap = w - k^2 H^dag_eo t; x, r, ||r||^2;
// beta; p = r + beta p.
static jqcd_status solve_cg_f64(GaugeEntry &G, const jqcd_solve_params &P, cudaStream_t s,
                                jqcd_solve_info *info, std::string *msg) {
  const bool eo = P.eo != 0;
  const int64_t vh = G.g.vh;
  const int64_t n = (eo ? 12 : 24) * vh;  // complex elements of the system's vectors
  const int nblas = (int)blas_blocks(n);
  const int nhop = (eo ? 1 : 2) * (int)hop_blocks(vh);
  const double tol2 = P.tol * P.tol;
  const double k2 = -P.kappa * P.kappa;
  SolverScalars *S = G.S;
  long long hops = 0;
  double hop_bytes = 0.0;
  auto count = [&](int plain, int axpy) {
    hops += plain + axpy;
    hop_bytes += (double)vh * (1536.0 * (plain + axpy) + 192.0 * axpy);
  };
  auto count_a = [&]() { count(eo ? 2 : 0, eo ? 2 : 4); };
#define CKS(call)                                              \
  do {                                                         \
    cudaError_t e_ = (call);                                   \
    if (e_ != cudaSuccess) {                                   \
      *msg = cudaGetErrorString(e_);                           \
      return e_ == cudaErrorMemoryAllocation ? JQCD_ENOMEM : JQCD_ECUDA; \
    }                                                          \
  } while (0)
  CKS(G.ensure_f64());
  CKS(cudaEventRecord(G.ev0, s));
  CKS(cudaMemsetAsync(S, 0, sizeof(SolverScalars), s));
  CKS(launch_f64_norm2(G.fb, 24 * vh, G.partials, s));  // ||b||^2 of D x = b
  CKS(launch_finalize_sum(G.partials, (int)blas_blocks(24 * vh), &S->b2, s));
  if (eo) {
    // bhat_e = b_e + kappa H_eo b_o (into fw even); rhs = Mhat^dag bhat
    HopParams Pb = G.hop_params(PREC_F64, 0, f64_odd(G, G.fb), f64_even(G.fb), f64_even(G.fw), 1.0,
                                P.kappa, nullptr);
    CKS(launch_hop(PREC_F64, Pb, false, true, false, s));
    HopParams P1 = G.hop_params(PREC_F64, 1, f64_even(G.fw), nullptr, f64_odd(G, G.ft), 0.0, 1.0,
                                nullptr);
    CKS(launch_hop(PREC_F64, P1, true, false, false, s));
    HopParams P2 = G.hop_params(PREC_F64, 0, f64_odd(G, G.ft), f64_even(G.fw), f64_even(G.frhs),
                                1.0, k2, nullptr);
    CKS(launch_hop(PREC_F64, P2, true, true, false, s));
    count(2, 1);
  } else {
    CKS(apply_dirac_f64(G, P.kappa, true, G.fb, G.frhs, nullptr, nullptr, s));  // rhs = D^dag b
    count(0, 2);
  }
  CKS(launch_f64_norm2(G.frhs, n, G.partials, s));
  CKS(launch_finalize_sum(G.partials, nblas, &S->rhs2, s));
  if (P.use_x0) {
    CKS(apply_a_f64(G, P.kappa, eo, G.fsol, G.fAp, nullptr, nullptr, s));
    count_a();
    CKS(launch_f64_xmy_norm(G.fr, G.frhs, G.fAp, n, G.partials, s));
  } else {
    CKS(launch_f64_zero(G.fsol, 24 * vh, s));
    CKS(launch_f64_copy(G.fr, G.frhs, n, s));
    CKS(launch_f64_norm2(G.fr, n, G.partials, s));
  }
  CKS(launch_cg_start(G.partials, nblas, S, tol2, P.maxiter, 0.0, s));
  CKS(launch_f64_copy(G.fp, G.fr, n, s));

  int restarts = 0;
  jqcd_status st = JQCD_OK;
  const int *guard = &S->halt;
  for (;;) {
    for (;;) {
      for (int k = 0; k < kCheckEvery; ++k) {
        CKS(apply_a_f64(G, P.kappa, eo, G.fp, G.fAp, G.partials, guard, s));
        CKS(launch_cg_alpha(G.partials, nhop, S, s));
        CKS(launch_f64_cg_update(G.fsol, G.fr, G.fp, G.fAp, n, S, G.partials, s));
        CKS(launch_cg_beta(G.partials, nblas, S, s));
        CKS(launch_f64_xpay(G.fp, G.fr, n, S, s));
      }
      CKS(cudaMemcpyAsync(G.S_host, S, sizeof(SolverScalars), cudaMemcpyDeviceToHost, s));
      CKS(cudaStreamSynchronize(s));
      if (P.verbose >= 3)
        fprintf(stderr, "jqcd cg (fp64): iter %d  |r|/|rhs| = %.3e\n", G.S_host->iters,
                G.S_host->rhs2 > 0 ? std::sqrt(G.S_host->rr / G.S_host->rhs2) : 0.0);
      if (G.S_host->done || G.S_host->iters >= P.maxiter) break;
    }
    if (G.S_host->done == 2) {
      *msg = "CG breakdown (<p,Ap> <= 0 or not finite)";
      st = JQCD_EBREAKDOWN;
      break;
    }
    // true residual of the CG system
    CKS(apply_a_f64(G, P.kappa, eo, G.fsol, G.fAp, nullptr, nullptr, s));
    count_a();
    CKS(launch_f64_xmy_norm(G.fr, G.frhs, G.fAp, n, G.partials, s));
    CKS(launch_finalize_sum(G.partials, nblas, &S->true_rr, s));
    CKS(cudaMemcpyAsync(G.S_host, S, sizeof(SolverScalars), cudaMemcpyDeviceToHost, s));
    CKS(cudaStreamSynchronize(s));
    if (G.S_host->true_rr <= tol2 * G.S_host->rhs2) break;
    if (G.S_host->iters >= P.maxiter || restarts >= kMaxRestarts) {
      st = JQCD_ENOCONV;
      *msg = "maximum iterations reached";
      break;
    }
    ++restarts;  // restart from x with the recomputed residual
    CKS(launch_cg_start(G.partials, nblas, S, tol2, P.maxiter, 0.0, s));
    CKS(launch_f64_copy(G.fp, G.fr, n, s));
  }
  if (eo) {  // x_o = b_o + kappa H_oe x_e
    HopParams Pr = G.hop_params(PREC_F64, 1, f64_even(G.fsol), f64_odd(G, G.fb),
                                f64_odd(G, G.fsol), 1.0, P.kappa, nullptr);
    CKS(launch_hop(PREC_F64, Pr, false, true, false, s));
    count(0, 1);
  }
  CKS(cudaEventRecord(G.ev1, s));
  // ||b - D x||^2 (not part of the timed solve)
  CKS(apply_dirac_f64(G, P.kappa, false, G.fsol, G.fw, nullptr, nullptr, s));
  CKS(launch_f64_xmy_norm(G.fAp, G.fb, G.fw, 24 * vh, G.partials, s));
  CKS(launch_finalize_sum(G.partials, (int)blas_blocks(24 * vh), &S->full_rr, s));
  CKS(cudaMemcpyAsync(G.S_host, S, sizeof(SolverScalars), cudaMemcpyDeviceToHost, s));
  CKS(cudaStreamSynchronize(s));
  float ms = 0.f;
  CKS(cudaEventElapsedTime(&ms, G.ev0, G.ev1));
  const SolverScalars &H = *G.S_host;
  for (int i = 0; i < H.iters; ++i) count_a();  // loop hops: four per completed iteration
  info->iters = H.iters;
  info->restarts = restarts;
  info->reliable_updates = 0;
  info->true_rel_resid = H.rhs2 > 0 ? std::sqrt(H.true_rr / H.rhs2) : 0.0;
  info->full_rel_resid = H.b2 > 0 ? std::sqrt(H.full_rr / H.b2) : 0.0;
  info->gpu_seconds = ms * 1e-3;
  info->hop_count = (double)hops;
  info->hop_bytes = hop_bytes;
  return st;
#undef CKS
}

static jqcd_status check_params(const jqcd_solve_params &P, std::string *msg) {
  if (!(P.tol > 0.0) || P.maxiter < 1 || !(P.kappa >= 0.0)) {
    *msg = "bad solve parameters (tol > 0, maxiter >= 1, kappa >= 0)";
    return JQCD_EINVAL;
  }
  return JQCD_OK;
}

jqcd_status solve_resident_f64(GaugeEntry &G, const jqcd_solve_params &P, cudaStream_t s,
                               jqcd_solve_info *info, std::string *msg) {
  jqcd_status st = check_params(P, msg);
  if (st) return st;
  return solve_cg_f64(G, P, s, info, msg);
}

jqcd_status solve_resident(GaugeEntry &G, const jqcd_solve_params &P, cudaStream_t s,
                           jqcd_solve_info *info, std::string *msg) {
  jqcd_status st = check_params(P, msg);
  if (st) return st;
  switch (P.mode) {
    case JQCD_CG_DW: return solve_cg(G, P, s, info, msg);
    case JQCD_CG_F64: {
      // double-word b (and start vector) widened exactly to FP64, the FP64
      // solution rounded back to double-word
      cudaError_t e = G.ensure_f64();
      if (e == cudaSuccess) e = launch_dw_to_f64(G.fb, G.vb, 24 * G.g.vh, s);
      if (e == cudaSuccess && P.use_x0) e = launch_dw_to_f64(G.fsol, G.vsol, 24 * G.g.vh, s);
      if (e != cudaSuccess) {
        *msg = cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? JQCD_ENOMEM : JQCD_ECUDA;
      }
      st = solve_cg_f64(G, P, s, info, msg);
      if (st == JQCD_OK || st == JQCD_ENOCONV) {
        e = launch_f64_to_dw(G.vsol, G.fsol, 24 * G.g.vh, s);
        if (e != cudaSuccess) {
          *msg = cudaGetErrorString(e);
          return JQCD_ECUDA;
        }
      }
      return st;
    }
    case JQCD_CG_MIXED_F32:
    case JQCD_CG_MIXED_F16:
      if (!P.eo) {
        *msg = "mixed-precision modes solve the even-odd system only (eo = 1)";
        return JQCD_EINVAL;
      }
      if (!(P.delta >= 0.0 && P.delta < 1.0)) {
        *msg = "delta must lie in [0, 1)";
        return JQCD_EINVAL;
      }
      return solve_cg(G, P, s, info, msg);
    default:
      *msg = "solver mode not available";
      return JQCD_EINVAL;
  }
}

}  // namespace jqcd
