// Multi-shift conjugate gradient: (A + sigma_i) x_i = rhs for all shifts at
// once, A = Mhat^dag Mhat on the even sites, in double-word arithmetic (the
// rational approximations of RHMC; the paper lists RHMC among its
// algorithms, section on the package's features).
//
// All shifted systems share the Krylov space of the unshifted CG: the shifted
// residuals are collinear, r_i = zeta_i r, so one operator application per
// iteration serves every shift.  With alpha, beta of the unshifted CG and
// zeta_i^{-1} = zeta_i^0 = 1, alpha^{-1} = 1, beta^{-1} = 0 (Jegerlehner's
// recurrences, written for A + sigma):
//   zeta_i^{k+1} = zeta_i^k zeta_i^{k-1} alpha^{k-1} /
//                  [alpha^k beta^{k-1} (zeta_i^{k-1} - zeta_i^k) + zeta_i^{k-1} alpha^{k-1} (1 + sigma_i alpha^k)]
//   alpha_i^k = alpha^k zeta_i^{k+1} / zeta_i^k,   x_i += alpha_i^k p_i
//   beta_i^k  = beta^k (zeta_i^{k+1} / zeta_i^k)^2, p_i = zeta_i^{k+1} r + beta_i^k p_i
// Shift i stops (x_i frozen) once |zeta_i| |r| <= tol |rhs|; the loop ends
// when every shift has.  Scalars live on the device; the host polls.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "dw.cuh"
#include "kernels.h"
#include "multishift.h"
#include "pdl.cuh"
#include "reduce.cuh"
#include "solver.h"

namespace jqcd {

namespace {

constexpr int kMsCheckEvery = 8;

__device__ __forceinline__ dw dw_from_double(double v) {
  const float h = __double2float_rn(v);
  return dw_make(h, __double2float_rn(v - (double)h));
}

__device__ __forceinline__ double sum_partials(const double *partials, int n) {
  double v = 0.0;
  // all of a thread's loads are in flight before its first add; the adds keep
  // the fixed order i = tid, tid + blockDim.x, ... (out-of-range slots add 0)
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

__global__ void ms_start_kernel(const double *partials, int n, MsScalars *S, double tol2, int max_iters) {
  const double rhs2 = sum_partials(partials, n);
  if (threadIdx.x == 0) {
    S->rhs2 = rhs2;
    S->rr = rhs2;
    S->stop_rr = tol2 * rhs2;
    S->alpha = 0.0;
    S->alpha_prev = 1.0;
    S->beta = 0.0;
    S->iters = 0;
    S->max_iters = max_iters;
    S->done = 0;
    S->halt = 0;
    S->final_x = 0;
    for (int i = 0; i < S->nshift; ++i) {
      S->zeta_prev[i] = S->zeta[i] = S->zeta_next[i] = 1.0;
      S->alpha_s[i] = S->beta_s[i] = 0.0;
      S->active[i] = rhs2 > 0.0;
      S->conv_iter[i] = 0;
    }
    if (!(rhs2 > 0.0)) {
      S->done = 1;
      S->halt = 1;
    }
  }
}

__global__ void ms_alpha_kernel(const double *partials, int n, MsScalars *S) {
  pdl_enter();
  if (S->halt) {  // a queued iteration after the halt: the last x_i update is done
    if (threadIdx.x == 0) S->final_x = 0;
    return;
  }
  const double pAp = sum_partials(partials, n);
  if (threadIdx.x == 0) {
    if (!(pAp > 0.0) || !isfinite(pAp)) { S->done = 2; S->halt = 1; return; }
    const double a = S->rr / pAp, ap = S->alpha_prev, b = S->beta;
    S->alpha = a;
    const float ah = __double2float_rn(a);
    S->alpha_dw = make_float2(ah, __double2float_rn(a - (double)ah));
    for (int i = 0; i < S->nshift; ++i) {
      if (!S->active[i]) continue;
      const double z = S->zeta[i], zp = S->zeta_prev[i];
      const double zn = z * zp * ap / (a * b * (zp - z) + zp * ap * (1.0 + S->sigma[i] * a));
      S->zeta_next[i] = zn;
      S->alpha_s[i] = a * zn / z;
    }
  }
}

__global__ void ms_beta_kernel(const double *partials, int n, MsScalars *S) {
  pdl_enter();
  if (S->halt) return;
  const double rr_new = sum_partials(partials, n);
  if (threadIdx.x == 0) {
    S->iters += 1;
    if (!isfinite(rr_new)) { S->done = 2; S->halt = 1; return; }
    const double b = rr_new / S->rr;
    int any = 0;
    for (int i = 0; i < S->nshift; ++i) {
      S->xact[i] = S->active[i];
      if (!S->active[i]) continue;
      const double z = S->zeta[i], zn = S->zeta_next[i];
      S->beta_s[i] = b * (zn / z) * (zn / z);
      S->zeta_prev[i] = z;
      S->zeta[i] = zn;
      if (zn * zn * rr_new <= S->stop_rr) {
        S->active[i] = 0;
        S->conv_iter[i] = S->iters;
      } else {
        any = 1;
      }
    }
    S->beta = b;
    S->alpha_prev = S->alpha;
    S->rr = rr_new;
    if (!any) { S->done = 1; S->halt = 1; S->final_x = 1; }
    else if (S->iters >= S->max_iters) { S->done = 3; S->halt = 1; S->final_x = 1; }
  }
}

// After beta: x_i += alpha_i p_i for the shifts active in this iteration
// (xact; alpha_i from this iteration's alpha step) and p_i = zeta_i r +
// beta_i p_i for those still active, p = r + beta p: each p_i is read once.
// Runs while the solve iterates, and once more after the beta step that
// halted it (final_x).
__global__ void ms_xp_kernel(float4 *__restrict__ pb, const float4 *__restrict__ r, MsVectors V, int64_t n,
                             const MsScalars *S) {
  __shared__ float4 cp[kMsMaxShifts];  // (zeta.h, zeta.l, beta.h, beta.l)
  __shared__ float2 cx[kMsMaxShifts];  // alpha_i (h, l)
  __shared__ int ax[kMsMaxShifts], ap[kMsMaxShifts];
  pdl_enter();
  if (S->halt && !S->final_x) return;  // uniform across the grid
  const int ns = S->nshift;
  for (int i = threadIdx.x; i < ns; i += blockDim.x) {
    const double z = S->zeta[i], b = S->beta_s[i], a = S->alpha_s[i];
    const float zh = __double2float_rn(z), bh = __double2float_rn(b), ah = __double2float_rn(a);
    cp[i] = make_float4(zh, __double2float_rn(z - (double)zh), bh, __double2float_rn(b - (double)bh));
    cx[i] = make_float2(ah, __double2float_rn(a - (double)ah));
    ax[i] = S->xact[i];
    ap[i] = S->active[i] && !S->halt;
  }
  __syncthreads();
  const dw beta = dw_from_double(S->beta);
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
    dw rr, ri, pr, pi;
    dwc_unpack(r[q], rr, ri);
    dwc_unpack(pb[q], pr, pi);
    pb[q] = dwc_pack(dw_add(rr, dw_mul(beta, pr)), dw_add(ri, dw_mul(beta, pi)));
    for (int i = 0; i < ns; ++i) {
      if (!ax[i]) continue;
      dwc_unpack(V.p[i][q], pr, pi);
      const dw a = dw_make(cx[i].x, cx[i].y);
      dw xr, xi;
      dwc_unpack(V.x[i][q], xr, xi);
      V.x[i][q] = dwc_pack(dw_add(xr, dw_mul(a, pr)), dw_add(xi, dw_mul(a, pi)));
      if (!ap[i]) continue;
      const dw z = dw_make(cp[i].x, cp[i].y), b = dw_make(cp[i].z, cp[i].w);
      V.p[i][q] = dwc_pack(dw_add(dw_mul(z, rr), dw_mul(b, pr)), dw_add(dw_mul(z, ri), dw_mul(b, pi)));
    }
  }
}

// r = rhs - Ax - sigma x, per-block partials of ||r||^2 (true residual).
__global__ void ms_resid_kernel(const float4 *__restrict__ rhs, const float4 *__restrict__ Ax,
                                const float4 *__restrict__ x, double sigma, int64_t n, double *partials) {
  const dw ms = dw_from_double(-sigma);
  dwacc A{0.f, 0.f};
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
    dw br, bi, yr, yi, xr, xi;
    dwc_unpack(rhs[q], br, bi);
    dwc_unpack(Ax[q], yr, yi);
    dwc_unpack(x[q], xr, xi);
    const dw re = dw_add(dw_add(br, dw_neg(yr)), dw_mul(ms, xr));
    const dw im = dw_add(dw_add(bi, dw_neg(yi)), dw_mul(ms, xi));
    acc_sq(A, re);
    acc_sq(A, im);
  }
  const double s = block_sum_dw(A);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

}  // namespace

cudaError_t GaugeEntry::ensure_multishift(int nshift) {
  cudaError_t e = ensure_solver();
  const size_t half = spinor_parity_bytes(PREC_DW, g.vh);
  while (e == cudaSuccess && (int)ms_p.size() < nshift) {
    float4 *p = nullptr;
    e = alloc_t(&p, half);
    if (e == cudaSuccess) ms_p.push_back(p);
  }
  if (e == cudaSuccess && !ms_S) e = alloc_t(&ms_S, sizeof(MsScalars));
  if (e == cudaSuccess && !ms_S_host) e = cudaMallocHost(&ms_S_host, sizeof(MsScalars));
  return e;
}

jqcd_status solve_multishift(GaugeEntry &G, const jqcd_solve_params &P, int nshift, const double *shifts,
                             float4 *const *x_even, cudaStream_t s, jqcd_solve_info *infos,
                             std::string *msg) {
#define CKM(call)                                                            \
  do {                                                                       \
    cudaError_t e_ = (call);                                                 \
    if (e_ != cudaSuccess) {                                                 \
      *msg = cudaGetErrorString(e_);                                         \
      return e_ == cudaErrorMemoryAllocation ? JQCD_ENOMEM : JQCD_ECUDA;     \
    }                                                                        \
  } while (0)
  if (nshift < 1 || nshift > kMsMaxShifts) {
    *msg = "nshift must lie in [1, 32]";
    return JQCD_EINVAL;
  }
  for (int i = 0; i < nshift; ++i)
    if (!(shifts[i] >= 0.0) || !std::isfinite(shifts[i])) {
      *msg = "shifts must be finite and >= 0 (A + sigma must stay positive definite)";
      return JQCD_EINVAL;
    }
  if (!(P.tol > 0.0) || P.maxiter < 1 || !(P.kappa >= 0.0) || !P.eo || P.mode != JQCD_CG_DW) {
    *msg = "multi-shift CG: eo = 1, mode JQCD_CG_DW, tol > 0, maxiter >= 1, kappa >= 0";
    return JQCD_EINVAL;
  }
  CKM(G.ensure_multishift(nshift));
  const int64_t vh = G.g.vh;
  const int64_t n = 12 * vh;  // complex double-word numbers of one parity
  const int nblas = (int)blas_blocks(n);
  const int nhop = (int)dw_hop_blocks(vh);  // partials of the double-word hops
  float4 *rhs = G.vec_even(G.vrhs), *r = G.vec_even(G.vr), *pb = G.vec_even(G.vp), *Ap = G.vec_even(G.vAp);
  MsVectors V;
  memset(&V, 0, sizeof V);
  for (int i = 0; i < nshift; ++i) {
    V.x[i] = x_even[i];
    V.p[i] = G.ms_p[i];
  }
  MsScalars *S = G.ms_S;
  MsScalars *H = G.ms_S_host;
  memset(H, 0, sizeof(MsScalars));
  H->nshift = nshift;
  for (int i = 0; i < nshift; ++i) H->sigma[i] = shifts[i];
  CKM(cudaEventRecord(G.ev0, s));
  CKM(cudaMemcpyAsync(S, H, sizeof(MsScalars), cudaMemcpyHostToDevice, s));
  CKM(launch_dw_norm2(rhs, n, G.partials, s));
  CKM(launch_ms_start(G.partials, nblas, S, P.tol * P.tol, P.maxiter, s));
  CKM(launch_dw_copy(r, rhs, n, s));
  CKM(launch_dw_copy(pb, rhs, n, s));
  for (int i = 0; i < nshift; ++i) {
    CKM(launch_dw_copy(V.p[i], rhs, n, s));
    CKM(launch_dw_zero(V.x[i], n, s));
  }
  // One iteration: t = H_oe p; w = p - k^2 H_eo t with ||w||^2 = <p, Mhat^dag Mhat p>;
  // alpha; t = H^dag_oe w; the last hop forms Ap at its site and applies
  // r -= alpha Ap with ||r||^2 (Ap is not stored); beta; then the x_i and p_i
  // of every shift in one pass.
  const double k2 = -P.kappa * P.kappa;
  float4 *t = G.vec_odd(G.vt), *w = G.vec_even(G.vw);
  auto iteration = [&]() -> cudaError_t {
    HopParams H = G.hop_params(PREC_DW, 1, pb, nullptr, t, 0.0, 1.0, nullptr);
    H.guard = &S->halt;
    cudaError_t e = launch_hop(PREC_DW, H, false, false, false, s);
    if (e) return e;
    H = G.hop_params(PREC_DW, 0, t, pb, w, 1.0, k2, G.partials);
    H.guard = &S->halt;
    if ((e = launch_hop(PREC_DW, H, false, true, true, s))) return e;
    // the alpha step runs on the side stream beside t = H^dag_oe w, which
    // does not read it; the last hop waits for it
    if (G.side) {
      if ((e = cudaEventRecord(G.ev_fork, s))) return e;
      if ((e = cudaStreamWaitEvent(G.side, G.ev_fork, 0))) return e;
      if ((e = launch_ms_alpha(G.partials, nhop, S, G.side))) return e;
      if ((e = cudaEventRecord(G.ev_join, G.side))) return e;
    } else if ((e = launch_ms_alpha(G.partials, nhop, S, s))) {
      return e;
    }
    H = G.hop_params(PREC_DW, 1, w, nullptr, t, 0.0, 1.0, nullptr);
    H.guard = &S->halt;
    if ((e = launch_hop(PREC_DW, H, true, false, false, s))) return e;
    if (G.side && (e = cudaStreamWaitEvent(s, G.ev_join, 0))) return e;
    H = G.hop_params(PREC_DW, 0, t, w, nullptr, 1.0, k2, G.partials);
    H.guard = &S->halt;
    if ((e = launch_hop_dw_r(H, r, &S->alpha_dw, s))) return e;
    return launch_ms_beta_xp(G.partials, nhop, nblas, S, V, r, pb, n, s);
  };
  for (;;) {
    for (int k = 0; k < kMsCheckEvery; ++k) CKM(iteration());
    CKM(cudaMemcpyAsync(H, S, sizeof(MsScalars), cudaMemcpyDeviceToHost, s));
    CKM(cudaStreamSynchronize(s));
    if (P.verbose >= 3)
      fprintf(stderr, "jqcd multishift: iter %d  |r|/|rhs| = %.3e\n", H->iters,
              H->rhs2 > 0 ? std::sqrt(H->rr / H->rhs2) : 0.0);
    if (H->done) break;
  }
  CKM(cudaEventRecord(G.ev1, s));
  jqcd_status st = JQCD_OK;
  if (H->done == 2) {
    *msg = "multi-shift CG breakdown (<p,Ap> <= 0 or not finite)";
    st = JQCD_EBREAKDOWN;
  }
  // true residual of every shifted system
  std::vector<double> tr(nshift, 0.0);
  for (int i = 0; i < nshift && st == JQCD_OK; ++i) {
    CKM(apply_mdagm(G, PREC_DW, P.kappa, V.x[i], Ap, G.vec_odd(G.vt), G.vec_even(G.vw), nullptr, nullptr, s));
    CKM(launch_ms_resid(rhs, Ap, V.x[i], shifts[i], n, G.partials, nblas, s));
    CKM(launch_finalize_sum(G.partials, nblas, &S->true_rr[i], s));
  }
  CKM(cudaMemcpyAsync(H, S, sizeof(MsScalars), cudaMemcpyDeviceToHost, s));
  CKM(cudaStreamSynchronize(s));
  float ms = 0.f;
  CKM(cudaEventElapsedTime(&ms, G.ev0, G.ev1));
  const double hop_iter = (double)vh * (1536.0 * 4 + 192.0 * 2);  // 4 hops, 2 with axpy
  for (int i = 0; i < nshift; ++i) {
    jqcd_solve_info &f = infos[i];
    memset(&f, 0, sizeof f);
    f.iters = H->conv_iter[i] ? H->conv_iter[i] : H->iters;
    f.true_rel_resid = H->rhs2 > 0 ? std::sqrt(H->true_rr[i] / H->rhs2) : 0.0;
    f.gpu_seconds = ms * 1e-3;
    f.hop_count = 4.0 * H->iters;
    f.hop_bytes = hop_iter * H->iters;
    f.status = st;
    if (st == JQCD_OK && (H->conv_iter[i] == 0 && H->rhs2 > 0)) f.status = JQCD_ENOCONV;
    else if (st == JQCD_OK && f.true_rel_resid > P.tol * (1.0 + 1e-6)) f.status = JQCD_ENOCONV;
  }
  if (st == JQCD_OK)
    for (int i = 0; i < nshift; ++i)
      if (infos[i].status != JQCD_OK) {
        st = JQCD_ENOCONV;
        *msg = H->done == 3 ? "maximum iterations reached" : "a shifted system misses its tolerance";
      }
  return st;
#undef CKM
}

cudaError_t launch_ms_start(const double *partials, int n, MsScalars *S, double tol2, int max_iters,
                            cudaStream_t s) {
  note_launch();
  ms_start_kernel<<<1, kReduceThreads, 0, s>>>(partials, n, S, tol2, max_iters);
  return cudaGetLastError();
}

cudaError_t launch_ms_alpha(const double *partials, int nhop, MsScalars *S, cudaStream_t s) {
  note_launch();
  return launch_pdl(ms_alpha_kernel, 1, kReduceThreads, 0, s, partials, nhop, S);
}

cudaError_t launch_ms_beta_xp(const double *partials, int nhop, int nblas, MsScalars *S, const MsVectors &V,
                              const float4 *r, float4 *pb, int64_t n, cudaStream_t s) {
  note_launch(2);
  const cudaError_t e = launch_pdl(ms_beta_kernel, 1, kReduceThreads, 0, s, partials, nhop, S);
  if (e != cudaSuccess) return e;
  return launch_pdl(ms_xp_kernel, nblas, kBlasThreads, 0, s, pb, r, V, n, S);
}

cudaError_t launch_ms_resid(const float4 *rhs, const float4 *Ax, const float4 *x, double sigma, int64_t n,
                            double *partials, int nblocks, cudaStream_t s) {
  note_launch();
  ms_resid_kernel<<<nblocks, kBlasThreads, 0, s>>>(rhs, Ax, x, sigma, n, partials);
  return cudaGetLastError();
}

}  // namespace jqcd
