// Hybrid Monte Carlo on the resident gauge field (paper: section "Hybrid
// Monte Carlo", MDstep!): Wilson plaquette gauge action with beta, su(3)
// momenta, leapfrog steps U(dt/2) P(dt) U(dt/2), two-flavour Wilson fermions
// through the action/force of force.cu, Metropolis on H = K + S_g + S_f.
//
// Conventions (U dS/dU as in force.cu: dS = Re Tr[(dS/dU) dU]):
//   S_g = -(beta/3) sum_x sum_{mu<nu} Re Tr P_munu(x),
//   U dS_g/dU_mu(x) = -(beta/3) U_mu(x) V_mu(x) (V: the six staples),
//   P = i sum_a p^a T^a, T^a = lambda^a / 2, K = -sum Tr P^2 = sum (p^a)^2 / 2,
//   dP/dt = TA(U dS/dU) / 2, dU/dt = P U, TA(G) = (G - G^dag)/2 - Tr(G - G^dag)/6.
// The FP64 links are the master copy (link update, plaquette and momenta in
// native FP64); the double-word and 12-real FP32 copies are refreshed from
// them after every update, and the staple force runs on the double-word copy.  Layouts: FP64 link-type fields double2[2][4][9][vh] (parity, mu,
// element 3a+b, checkerboard site), like the uploaded FP64 gauge field.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>

#include "dw.cuh"
#include "hmc.h"
#include "hop_dwp.cuh"
#include "kernels.h"
#include "reduce.cuh"
#include "solver.h"

namespace jqcd {

namespace {

constexpr int kHmcThreads = 128;

struct m3 {
  double2 e[3][3];
};

__device__ __forceinline__ double2 cmul_d(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cadd_d(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }

// 3x3 complex product accumulated in FMAs: 2 multiplies and 10 FMAs per
// element (the FP64 pipe bounds the FP64 gauge kernels).
__device__ __forceinline__ m3 m3_mul(const m3 &A, const m3 &B) {
  m3 r;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      double re = A.e[a][0].x * B.e[0][b].x, im = A.e[a][0].x * B.e[0][b].y;
      re = fma(-A.e[a][0].y, B.e[0][b].y, re);
      im = fma(A.e[a][0].y, B.e[0][b].x, im);
#pragma unroll
      for (int k = 1; k < 3; ++k) {
        re = fma(A.e[a][k].x, B.e[k][b].x, re);
        re = fma(-A.e[a][k].y, B.e[k][b].y, re);
        im = fma(A.e[a][k].x, B.e[k][b].y, im);
        im = fma(A.e[a][k].y, B.e[k][b].x, im);
      }
      r.e[a][b] = make_double2(re, im);
    }
  return r;
}
__device__ __forceinline__ m3 m3_dag(const m3 &A) {
  m3 r;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) r.e[a][b] = make_double2(A.e[b][a].x, -A.e[b][a].y);
  return r;
}
__device__ __forceinline__ m3 m3_load(const double2 *F, int64_t vh, int p, int mu, int64_t cb) {
  m3 r;
  const double2 *q = F + (size_t)((p * 4 + mu) * 9) * vh + cb;
#pragma unroll
  for (int k = 0; k < 9; ++k) r.e[k / 3][k % 3] = q[k * vh];
  return r;
}
__device__ __forceinline__ void m3_store(double2 *F, int64_t vh, int p, int mu, int64_t cb, const m3 &A) {
  double2 *q = F + (size_t)((p * 4 + mu) * 9) * vh + cb;
#pragma unroll
  for (int k = 0; k < 9; ++k) q[k * vh] = A.e[k / 3][k % 3];
}

// link U_nu at the site c shifted by (s1 in mu1) and (s2 in mu2)
__device__ __forceinline__ m3 link_at(const double2 *U, const Geom &g, const int c[4], int nu, int mu1, int s1,
                                      int mu2, int s2) {
  int d[4] = {c[0], c[1], c[2], c[3]};
  const int n1 = mu1 == 0 ? g.nx : (mu1 == 1 ? g.ny : (mu1 == 2 ? g.nz : g.nt));
  const int n2 = mu2 == 0 ? g.nx : (mu2 == 1 ? g.ny : (mu2 == 2 ? g.nz : g.nt));
  if (s1) d[mu1] = (d[mu1] + s1 + n1) % n1;
  if (s2) d[mu2] = (d[mu2] + s2 + n2) % n2;
  return m3_load(U, g.vh, (d[0] + d[1] + d[2] + d[3]) & 1, nu, cb_index(g, d[0], d[1], d[2], d[3]));
}

__device__ __forceinline__ void site_of_thread(const Geom &g, int64_t q, int *p, int64_t *cb, int c[4]) {
  *p = (int)(q / g.vh);
  *cb = q - (int64_t)*p * g.vh;
  cb_coords(g, *cb, *p, c[0], c[1], c[2], c[3]);
}

// ---- U dS_g/dU for every link, in double-word arithmetic -------------------
// One thread per (site, mu) sums the six staples of its link on the
// double-word copy of the links (refreshed from the FP64 masters after every
// link update) and multiplies by U_mu(x).  Each 3x3 product is three
// offset-grid mat-vecs (matvec_half_p: exact products on a fixed grid, a few
// 1e-14 relative per product) on the FP32 pipes; in native FP64 the same
// sums were bound by the FP64 pipe (707.6 against 143 us at 16^4 on GB300).
struct m3p {
  p2 e[3][3];
};

__device__ __forceinline__ m3p m3p_load(const float4 *U, int64_t vh, int p, int mu, int64_t cb) {
  m3p r;
  const ulonglong2 *q = reinterpret_cast<const ulonglong2 *>(U) + (size_t)((p * 4 + mu) * 9) * vh + cb;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const ulonglong2 v = __ldg(q + k * vh);
    r.e[k / 3][k % 3] = p2{v.x, v.y};
  }
  return r;
}
__device__ __forceinline__ m3p m3p_dag(const m3p &A) {
  m3p r;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) r.e[a][b] = p2_conj(A.e[b][a]);
  return r;
}
// C = A B, column by column; the results normalised (Fast2Sum per lane)
__device__ __forceinline__ m3p m3p_mul(const m3p &A, const m3p &B) {
  const float amax = link_max_hi(A.e) * 1.0000019f;  // raised as in the hop (matvec_half_p)
  m3p C;
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    const p2 col[3] = {B.e[0][b], B.e[1][b], B.e[2][b]};
    p2 r[3];
    matvec_half_p(A.e, amax, col, r);
#pragma unroll
    for (int a = 0; a < 3; ++a) C.e[a][b] = p2_norm(r[a]);
  }
  return C;
}
__device__ __forceinline__ m3p link_at_dw(const float4 *U, const Geom &g, const int c[4], int nu, int mu1, int s1,
                                          int mu2, int s2) {
  int d[4] = {c[0], c[1], c[2], c[3]};
  const int n1 = mu1 == 0 ? g.nx : (mu1 == 1 ? g.ny : (mu1 == 2 ? g.nz : g.nt));
  const int n2 = mu2 == 0 ? g.nx : (mu2 == 1 ? g.ny : (mu2 == 2 ? g.nz : g.nt));
  if (s1) d[mu1] = (d[mu1] + s1 + n1) % n1;
  if (s2) d[mu2] = (d[mu2] + s2 + n2) % n2;
  return m3p_load(U, g.vh, (d[0] + d[1] + d[2] + d[3]) & 1, nu, cb_index(g, d[0], d[1], d[2], d[3]));
}

__global__ void __launch_bounds__(kHmcThreads) gauge_force_dw_kernel(Geom g, const float4 *__restrict__ U,
                                                                     double beta, double2 *__restrict__ out) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= 8 * g.vh) return;
  const int mu = (int)(q / (2 * g.vh));
  int p, c[4];
  int64_t cb;
  site_of_thread(g, q % (2 * g.vh), &p, &cb, c);
  m3p V;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) V.e[a][b] = p2{0ull, 0ull};
#pragma unroll 1
  for (int nu = 0; nu < 4; ++nu) {
    if (nu == mu) continue;
    // upper staple U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag
    m3p T = m3p_mul(link_at_dw(U, g, c, nu, mu, 1, nu, 0), m3p_dag(link_at_dw(U, g, c, mu, nu, 1, mu, 0)));
    m3p S = m3p_mul(T, m3p_dag(link_at_dw(U, g, c, nu, mu, 0, nu, 0)));
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) V.e[a][b] = p2_add(V.e[a][b], S.e[a][b]);
    // lower staple U_nu(x+mu-nu)^dag U_mu(x-nu)^dag U_nu(x-nu)
    T = m3p_mul(m3p_dag(link_at_dw(U, g, c, nu, mu, 1, nu, -1)), m3p_dag(link_at_dw(U, g, c, mu, nu, -1, mu, 0)));
    S = m3p_mul(T, link_at_dw(U, g, c, nu, nu, -1, mu, 0));
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) V.e[a][b] = p2_norm(p2_add(V.e[a][b], S.e[a][b]));
  }
  const m3p G = m3p_mul(m3p_load(U, g.vh, p, mu, cb), V);
  const double f = -beta / 3.0;
  double2 *o = out + (size_t)((p * 4 + mu) * 9) * g.vh + cb;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    float hr, hi, lr, li;
    f2_split(G.e[k / 3][k % 3].h, hr, hi);
    f2_split(G.e[k / 3][k % 3].l, lr, li);
    o[k * g.vh] = make_double2(f * ((double)hr + (double)lr), f * ((double)hi + (double)li));
  }
}

// per-block partials of sum_{mu<nu} Re Tr P_munu(x): one thread per site
__global__ void __launch_bounds__(kHmcThreads) plaquette_kernel(Geom g, const double2 *__restrict__ U,
                                                                double *partials) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double s = 0.0;
  if (q < 2 * g.vh) {
    int p, c[4];
    int64_t cb;
    site_of_thread(g, q, &p, &cb, c);
    for (int mu = 0; mu < 4; ++mu)
      for (int nu = mu + 1; nu < 4; ++nu) {
        const m3 A = m3_mul(m3_load(U, g.vh, p, mu, cb), link_at(U, g, c, nu, mu, 1, nu, 0));
        const m3 B = m3_mul(m3_dag(link_at(U, g, c, mu, nu, 1, mu, 0)), m3_dag(m3_load(U, g.vh, p, nu, cb)));
        // Re Tr (A B)
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
          for (int k = 0; k < 3; ++k) s += A.e[a][k].x * B.e[k][a].x - A.e[a][k].y * B.e[k][a].y;
      }
  }
  const double t = block_sum_d(s);
  if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

// P = i sum_a p^a T^a from normals [link l = site + V*mu][8] (canonical order)
__global__ void mom_set_kernel(Geom g, const double *__restrict__ normals, double2 *__restrict__ P) {
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
  const double *a = normals + 8 * l;
  const double r3 = 0.5773502691896258;  // 1/sqrt(3)
  // i * (1/2) * sum_a p^a lambda^a  (Gell-Mann matrices)
  m3 M;
  M.e[0][0] = make_double2(0.0, 0.5 * (a[2] + r3 * a[7]));
  M.e[1][1] = make_double2(0.0, 0.5 * (-a[2] + r3 * a[7]));
  M.e[2][2] = make_double2(0.0, 0.5 * (-2.0 * r3 * a[7]));
  M.e[0][1] = make_double2(0.5 * a[1], 0.5 * a[0]);
  M.e[1][0] = make_double2(-0.5 * a[1], 0.5 * a[0]);
  M.e[0][2] = make_double2(0.5 * a[4], 0.5 * a[3]);
  M.e[2][0] = make_double2(-0.5 * a[4], 0.5 * a[3]);
  M.e[1][2] = make_double2(0.5 * a[6], 0.5 * a[5]);
  M.e[2][1] = make_double2(-0.5 * a[6], 0.5 * a[5]);
  m3_store(P, g.vh, p, mu, cb, M);
}

// per-block partials of sum over links of -Tr P^2
__global__ void kinetic_kernel(Geom g, const double2 *__restrict__ P, double *partials) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double s = 0.0;
  if (q < 8 * g.vh) {
    const int mu = (int)(q / (2 * g.vh));
    const int64_t r = q % (2 * g.vh);
    const int p = (int)(r / g.vh);
    const m3 A = m3_load(P, g.vh, p, mu, r - (int64_t)p * g.vh);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int k = 0; k < 3; ++k) s -= A.e[a][k].x * A.e[k][a].x - A.e[a][k].y * A.e[k][a].y;
  }
  const double t = block_sum_d(s);
  if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

// P += coef * TA(Gg + Gf); Gf: double-word link field or null
__global__ void mom_update_kernel(Geom g, double2 *__restrict__ P, const double2 *__restrict__ Gg,
                                  const float4 *__restrict__ Gf, double coef) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= 8 * g.vh) return;
  const int mu = (int)(q / (2 * g.vh));
  const int64_t r = q % (2 * g.vh);
  const int p = (int)(r / g.vh);
  const int64_t cb = r - (int64_t)p * g.vh;
  m3 G = m3_load(Gg, g.vh, p, mu, cb);
  if (Gf) {
    const float4 *F = Gf + (size_t)((p * 4 + mu) * 9) * g.vh + cb;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const float4 v = F[k * g.vh];
      G.e[k / 3][k % 3].x += (double)v.x + (double)v.z;
      G.e[k / 3][k % 3].y += (double)v.y + (double)v.w;
    }
  }
  // TA(G) = (G - G^dag)/2 - i Im Tr(G)/3 on the diagonal
  const double tr = (G.e[0][0].y + G.e[1][1].y + G.e[2][2].y) / 3.0;
  m3 A = m3_load(P, g.vh, p, mu, cb);
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      double re = 0.5 * (G.e[a][b].x - G.e[b][a].x);
      double im = 0.5 * (G.e[a][b].y + G.e[b][a].y);
      if (a == b) im -= tr;
      A.e[a][b] = make_double2(A.e[a][b].x + coef * re, A.e[a][b].y + coef * im);
    }
  m3_store(P, g.vh, p, mu, cb, A);
}

// exp(X) for a 3x3 complex X with |X|_F <= 1, by the Cayley-Hamilton identity
// X^3 = t X^2 - s X + d (t = tr X, s = ((tr X)^2 - tr X^2)/2, d = det X):
// X^n = a_n + b_n X + c_n X^2 with a_{n+1} = d c_n, b_{n+1} = a_n - s c_n,
// c_{n+1} = b_n + t c_n, so exp X = F0 + F1 X + F2 X^2 with
// F = sum_n (a_n, b_n, c_n) / n!.  One matrix product (X^2) replaces the
// products of a matrix Taylor series; the F are divided differences of exp
// on the spectrum, smooth also for degenerate eigenvalues, and 18 terms
// reach double precision for |X|_F <= 1 (checked against a dense matrix
// exponential, degenerate spectra and a small trace included).  The count
// of terms is fixed by nu >= |X|_F: the series' remainder after N terms is at
// most nu^(N+1) / (N+1)! / (1 - nu / (N+2)), below 1e-17 for N = 10, 12, 15,
// 18 at nu <= 1/8, 1/4, 1/2, 1 (a leapfrog step's eps P has |eps P|_F of
// about 0.1; the 16^4 trajectory went 0.0649 -> 0.0634 s against 18 terms
// always).  A count fixed per call measured faster than stopping at the
// first negligible term.
__device__ __forceinline__ m3 m3_exp(const m3 &X, double nu) {
  const int nterms = nu <= 0.125 ? 10 : (nu <= 0.25 ? 12 : (nu <= 0.5 ? 15 : 18));
  const m3 X2 = m3_mul(X, X);
  const double2 t = cadd_d(cadd_d(X.e[0][0], X.e[1][1]), X.e[2][2]);
  const double2 tr2 = cadd_d(cadd_d(X2.e[0][0], X2.e[1][1]), X2.e[2][2]);
  const double2 tt = cmul_d(t, t);
  const double2 sI = make_double2(0.5 * (tt.x - tr2.x), 0.5 * (tt.y - tr2.y));
  const double2 m0 = cadd_d(cmul_d(X.e[1][1], X.e[2][2]), cmul_d(make_double2(-X.e[1][2].x, -X.e[1][2].y), X.e[2][1]));
  const double2 m1 = cadd_d(cmul_d(X.e[1][0], X.e[2][2]), cmul_d(make_double2(-X.e[1][2].x, -X.e[1][2].y), X.e[2][0]));
  const double2 m2 = cadd_d(cmul_d(X.e[1][0], X.e[2][1]), cmul_d(make_double2(-X.e[1][1].x, -X.e[1][1].y), X.e[2][0]));
  const double2 d0 = cmul_d(X.e[0][0], m0), d1 = cmul_d(X.e[0][1], m1), d2 = cmul_d(X.e[0][2], m2);
  const double2 d = make_double2(d0.x - d1.x + d2.x, d0.y - d1.y + d2.y);
  double2 a = make_double2(1.0, 0.0), b = make_double2(0.0, 0.0), c = b;
  double2 F0 = a, F1 = b, F2 = b;
#pragma unroll
  for (int n = 1; n <= 18; ++n) {
    if (n > nterms) break;
    const double inv = 1.0 / n;
    const double2 dc = cmul_d(d, c), sc = cmul_d(sI, c), tc = cmul_d(t, c);
    const double2 na = make_double2(dc.x * inv, dc.y * inv);
    const double2 nb = make_double2((a.x - sc.x) * inv, (a.y - sc.y) * inv);
    const double2 nc = make_double2((b.x + tc.x) * inv, (b.y + tc.y) * inv);
    a = na;
    b = nb;
    c = nc;
    F0 = cadd_d(F0, a);
    F1 = cadd_d(F1, b);
    F2 = cadd_d(F2, c);
  }
  m3 E;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      double2 v = cadd_d(cmul_d(F1, X.e[i][j]), cmul_d(F2, X2.e[i][j]));
      if (i == j) v = cadd_d(v, F0);
      E.e[i][j] = v;
    }
  return E;
}

// U <- exp(eps P) U: exp(eps P / 2^k) with |eps P / 2^k|_F <= 1 by m3_exp,
// squared k times (k = 0 for the step sizes of a trajectory)
__global__ void exp_update_kernel(Geom g, double2 *__restrict__ U, const double2 *__restrict__ P, double eps) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= 8 * g.vh) return;
  const int mu = (int)(q / (2 * g.vh));
  const int64_t r = q % (2 * g.vh);
  const int p = (int)(r / g.vh);
  const int64_t cb = r - (int64_t)p * g.vh;
  m3 A = m3_load(P, g.vh, p, mu, cb);
  double nrm = 0.0;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) nrm += A.e[a][b].x * A.e[a][b].x + A.e[a][b].y * A.e[a][b].y;
  nrm = fabs(eps) * sqrt(nrm);  // Frobenius norm of eps P
  int k = 0;
  double sc = eps;
  while (nrm > 1.0 && k < 40) {
    nrm *= 0.5;
    sc *= 0.5;
    ++k;
  }
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) A.e[a][b] = make_double2(sc * A.e[a][b].x, sc * A.e[a][b].y);
  m3 E = m3_exp(A, nrm);
  for (int i = 0; i < k; ++i) E = m3_mul(E, E);
  m3_store(U, g.vh, p, mu, cb, m3_mul(E, m3_load(U, g.vh, p, mu, cb)));
}

// FP64 links -> double-word and 12-real FP32 copies (same per-link layout as gauge_pack)
__global__ void links_refresh_kernel(Geom g, const double2 *__restrict__ U, float4 *__restrict__ dwo,
                                     float4 *__restrict__ f32o) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= 8 * g.vh) return;
  const int mu = (int)(q / (2 * g.vh));
  const int64_t r = q % (2 * g.vh);
  const int p = (int)(r / g.vh);
  const int64_t cb = r - (int64_t)p * g.vh;
  const m3 A = m3_load(U, g.vh, p, mu, cb);
  const int64_t blk = (int64_t)(p * 4 + mu);
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const double2 v = A.e[k / 3][k % 3];
    const float rh = __double2float_rn(v.x), ih = __double2float_rn(v.y);
    dwo[(blk * 9 + k) * g.vh + cb] =
        make_float4(rh, ih, __double2float_rn(v.x - (double)rh), __double2float_rn(v.y - (double)ih));
  }
  const double2 e[6] = {A.e[0][0], A.e[0][1], A.e[0][2], A.e[1][0], A.e[1][1], A.e[1][2]};
#pragma unroll
  for (int j = 0; j < 3; ++j)
    f32o[(blk * 3 + j) * g.vh + cb] = make_float4((float)e[2 * j].x, (float)e[2 * j].y, (float)e[2 * j + 1].x,
                                                  (float)e[2 * j + 1].y);
}

// FP64 link field -> canonical host layout a + 3(b + 3(site + V mu))
__global__ void links_unpack_kernel(Geom g, const double2 *__restrict__ U, double2 *__restrict__ canon) {
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
  const m3 A = m3_load(U, g.vh, (x + y + z + t) & 1, mu, s >> 1);
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) canon[9 * l + a + 3 * b] = A.e[a][b];
}

unsigned link_blocks(int64_t vh) { return (unsigned)((8 * vh + kHmcThreads - 1) / kHmcThreads); }
unsigned site_blocks2(int64_t vh) { return (unsigned)((2 * vh + kHmcThreads - 1) / kHmcThreads); }

}  // namespace

// out = a x + b y over n double-word complex numbers (a, b real, given as
// (hi, lo) float pairs); out may alias x or y.
__global__ void dw_lincomb_kernel(float4 *out, const float4 *x, const float4 *y, float2 a, float2 b, int64_t n) {
  const dw A = dw_make(a.x, a.y), B = dw_make(b.x, b.y);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    dw xr, xi, yr, yi;
    dwc_unpack(x[i], xr, xi);
    dwc_unpack(y[i], yr, yi);
    out[i] = dwc_pack(dw_add(dw_mul(A, xr), dw_mul(B, yr)), dw_add(dw_mul(A, xi), dw_mul(B, yi)));
  }
}

cudaError_t launch_dw_lincomb(float4 *out, const float4 *x, const float4 *y, double a, double b, int64_t n,
                              cudaStream_t s) {
  const float ah = (float)a, bh = (float)b;
  note_launch();
  dw_lincomb_kernel<<<blas_blocks(n), kBlasThreads, 0, s>>>(
      out, x, y, make_float2(ah, (float)(a - (double)ah)), make_float2(bh, (float)(b - (double)bh)), n);
  return cudaGetLastError();
}

cudaError_t GaugeEntry::ensure_hmc() {
  cudaError_t e = ensure_reduce();
  const size_t lf = (size_t)72 * 16 * g.vh;  // FP64 link field, double2[2][4][9][vh]
  double2 **vs[] = {&hP, &hG, &hUbak};
  for (double2 **v : vs)
    if (e == cudaSuccess && !*v) e = alloc_t(v, lf);
  if (e == cudaSuccess && !hNormals) e = alloc_t(&hNormals, sizeof(double) * 8 * 4 * (size_t)(2 * g.vh));
  if (e == cudaSuccess && !hPart) e = alloc_t(&hPart, sizeof(double) * (link_blocks(g.vh) + 2));
  return e;
}

cudaError_t GaugeEntry::ensure_hmc_history() {
  cudaError_t e = cudaSuccess;
  const size_t full = 2 * spinor_parity_bytes(PREC_DW, g.vh);
  float4 **vs[] = {&hXp, &hYp, &hS1, &hS2};
  for (float4 **v : vs)
    if (e == cudaSuccess && !*v) e = alloc_t(v, full);
  return e;
}

cudaError_t launch_hmc_links_refresh(GaugeEntry &G, cudaStream_t s) {
  note_launch();
  links_refresh_kernel<<<link_blocks(G.g.vh), kHmcThreads, 0, s>>>(G.g, (const double2 *)G.gauge_f64,
                                                                      (float4 *)G.gauge_dw, (float4 *)G.gauge_f32);
  return cudaGetLastError();
}

cudaError_t launch_links_unpack(const GaugeEntry &G, double *canon, cudaStream_t s) {
  note_launch();
  links_unpack_kernel<<<(unsigned)((8 * G.g.vh + 255) / 256), 256, 0, s>>>(G.g, (const double2 *)G.gauge_f64,
                                                                             (double2 *)canon);
  return cudaGetLastError();
}

namespace {

// sum of the per-block partials in G.hPart into its last slot, then to the host
cudaError_t reduce_to_host(GaugeEntry &G, int nblocks, double *host, cudaStream_t s) {
  double *dev = G.hPart + link_blocks(G.g.vh) + 1;
  cudaError_t e = launch_finalize_sum(G.hPart, nblocks, dev, s);
  if (!e) e = cudaMemcpyAsync(host, dev, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (!e) e = cudaStreamSynchronize(s);
  return e;
}

}  // namespace

cudaError_t hmc_plaquette_sum(GaugeEntry &G, double *out, cudaStream_t s) {
  const unsigned nb = site_blocks2(G.g.vh);
  note_launch();
  plaquette_kernel<<<nb, kHmcThreads, 0, s>>>(G.g, (const double2 *)G.gauge_f64, G.hPart);
  cudaError_t e = cudaGetLastError();
  if (!e) e = reduce_to_host(G, (int)nb, out, s);
  return e;
}

cudaError_t hmc_kinetic(GaugeEntry &G, double *out, cudaStream_t s) {
  const unsigned nb = link_blocks(G.g.vh);
  note_launch();
  kinetic_kernel<<<nb, kHmcThreads, 0, s>>>(G.g, G.hP, G.hPart);
  cudaError_t e = cudaGetLastError();
  if (!e) e = reduce_to_host(G, (int)nb, out, s);
  return e;
}

cudaError_t hmc_momenta_set(GaugeEntry &G, const double *normals_dev, cudaStream_t s) {
  note_launch();
  mom_set_kernel<<<(unsigned)((8 * G.g.vh + 255) / 256), 256, 0, s>>>(G.g, normals_dev, G.hP);
  return cudaGetLastError();
}

cudaError_t hmc_gauge_force(GaugeEntry &G, double beta, cudaStream_t s) {
  note_launch();
  gauge_force_dw_kernel<<<link_blocks(G.g.vh), kHmcThreads, 0, s>>>(G.g, (const float4 *)G.gauge_dw, beta, G.hG);
  return cudaGetLastError();
}

cudaError_t hmc_momenta_update(GaugeEntry &G, const float4 *Gf, double coef, cudaStream_t s) {
  note_launch();
  mom_update_kernel<<<link_blocks(G.g.vh), kHmcThreads, 0, s>>>(G.g, G.hP, G.hG, Gf, coef);
  return cudaGetLastError();
}

cudaError_t hmc_links_update(GaugeEntry &G, double eps, cudaStream_t s) {
  note_launch();
  exp_update_kernel<<<link_blocks(G.g.vh), kHmcThreads, 0, s>>>(G.g, (double2 *)G.gauge_f64, G.hP, eps);
  cudaError_t e = cudaGetLastError();
  if (!e) e = launch_hmc_links_refresh(G, s);
  return e;
}

}  // namespace jqcd
