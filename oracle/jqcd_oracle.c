/*
 * jqcd oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, FP64 CPU implementation of the Wilson-Dirac operator, its
 * even-odd Schur complement and the conjugate-gradient solves built on them.
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * may load this library; the product path never calls it and shares no code
 * with it.
 *
 * Operator (paper: Wilson fermions with hopping parameter kappa, section
 * "Definition of Dirac operators", `mul!(y,D,x)`):
 *   (D psi)(x) = psi(x) - kappa * (H psi)(x)
 *   (H psi)(x) = sum_mu [ (1 - gamma_mu) U_mu(x) psi(x+mu)
 *                       + (1 + gamma_mu) U_mu(x-mu)^dagger psi(x-mu) ]
 * with periodic boundaries in x, y, z and, when t_antiperiodic != 0, a factor
 * -1 on every hop that crosses the time boundary (t = NT-1 <-> 0).
 * The adjoint `D'` is the same sum with gamma_mu -> -gamma_mu (written out from
 * the definition of the adjoint, not through gamma5).
 *
 * Everything is written from the definitions: explicit 4x4 gamma matrices
 * (DeGrand-Rossi chiral basis), a colour mat-vec per neighbour followed by the
 * full 4x4 spin matrix (1 -/+ gamma_mu) -- no spin projection.
 *
 * Layouts are the canonical host layouts (complex128, interleaved re/im):
 *   site   = ix + NX*(iy + NY*(iz + NZ*it))
 *   spinor (ic, site, alpha)  -> ic + 3*(site + V*alpha)
 *   link   (a, b) of U_mu(x)  -> a + 3*(b + 3*(site + V*mu))
 * Even-odd: parity(x) = (ix+iy+iz+it) mod 2, even = 0.  Even-odd routines take
 * full-lattice arrays; only the sites of the stated parity are meaningful and
 * the other parity of every output is written as zero.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct { double re, im; } cplx;

static inline cplx cm(double r, double i) { cplx z = {r, i}; return z; }
static inline cplx cadd(cplx a, cplx b) { return cm(a.re + b.re, a.im + b.im); }
static inline cplx csub(cplx a, cplx b) { return cm(a.re - b.re, a.im - b.im); }
static inline cplx cmul(cplx a, cplx b) {
  return cm(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
static inline cplx cconj(cplx a) { return cm(a.re, -a.im); }
static inline cplx cscale(cplx a, double s) { return cm(a.re * s, a.im * s); }

/* gamma_mu[alpha][beta], mu = 0..3 <-> x, y, z, t (DeGrand-Rossi basis). */
static const double GRE[4][4][4] = {
    {{0, 0, 0, 0}, {0, 0, 0, 0}, {0, 0, 0, 0}, {0, 0, 0, 0}},
    {{0, 0, 0, -1}, {0, 0, 1, 0}, {0, 1, 0, 0}, {-1, 0, 0, 0}},
    {{0, 0, 0, 0}, {0, 0, 0, 0}, {0, 0, 0, 0}, {0, 0, 0, 0}},
    {{0, 0, 1, 0}, {0, 0, 0, 1}, {1, 0, 0, 0}, {0, 1, 0, 0}}};
static const double GIM[4][4][4] = {
    {{0, 0, 0, 1}, {0, 0, 1, 0}, {0, -1, 0, 0}, {-1, 0, 0, 0}},
    {{0, 0, 0, 0}, {0, 0, 0, 0}, {0, 0, 0, 0}, {0, 0, 0, 0}},
    {{0, 0, 1, 0}, {0, 0, 0, -1}, {-1, 0, 0, 0}, {0, 1, 0, 0}},
    {{0, 0, 0, 0}, {0, 0, 0, 0}, {0, 0, 0, 0}, {0, 0, 0, 0}}};

/* Copy of the gamma matrices for the tests (re, im interleaved, [mu][a][b]). */
void jo_gamma(double *out) {
  for (int mu = 0; mu < 4; ++mu)
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) {
        out[2 * (16 * mu + 4 * a + b)] = GRE[mu][a][b];
        out[2 * (16 * mu + 4 * a + b) + 1] = GIM[mu][a][b];
      }
}

typedef struct {
  int64_t n[4];
  int64_t V;
  int tanti;
} lat_t;

static int lat_init(lat_t *L, const int dims[4], int tanti) {
  if (!dims) return -1;
  L->V = 1;
  for (int d = 0; d < 4; ++d) {
    if (dims[d] < 1) return -1;
    L->n[d] = dims[d];
    L->V *= dims[d];
  }
  L->tanti = tanti;
  return 0;
}

static inline void site_coords(const lat_t *L, int64_t s, int64_t c[4]) {
  c[0] = s % L->n[0]; s /= L->n[0];
  c[1] = s % L->n[1]; s /= L->n[1];
  c[2] = s % L->n[2]; s /= L->n[2];
  c[3] = s;
}

static inline int64_t site_index(const lat_t *L, const int64_t c[4]) {
  return c[0] + L->n[0] * (c[1] + L->n[1] * (c[2] + L->n[2] * c[3]));
}

static inline int site_parity(const int64_t c[4]) {
  return (int)((c[0] + c[1] + c[2] + c[3]) & 1);
}

static inline cplx ld(const double *p, int64_t k) { return cm(p[2 * k], p[2 * k + 1]); }
static inline void st(double *p, int64_t k, cplx z) { p[2 * k] = z.re; p[2 * k + 1] = z.im; }

/* U_mu(site)[a][b] */
static inline cplx link(const lat_t *L, const double *U, int mu, int64_t site, int a, int b) {
  return ld(U, a + 3 * (b + 3 * (site + L->V * mu)));
}
/* psi(site)[colour c][spin alpha] */
static inline cplx spin_ld(const lat_t *L, const double *p, int64_t site, int c, int alpha) {
  return ld(p, c + 3 * (site + L->V * alpha));
}

/* (H psi)(x) at one site x, both hop directions, all mu.  sgn = +1 for H,
 * -1 for the adjoint hop (gamma_mu -> -gamma_mu).  res[alpha][c]. */
static void hop_site(const lat_t *L, const double *U, const double *in, int64_t x, int sgn,
                     cplx res[4][3]) {
  int64_t c[4];
  site_coords(L, x, c);
  for (int a = 0; a < 4; ++a)
    for (int k = 0; k < 3; ++k) res[a][k] = cm(0, 0);
  for (int mu = 0; mu < 4; ++mu) {
    for (int dir = 0; dir < 2; ++dir) { /* dir 0: forward x+mu, dir 1: backward x-mu */
      int64_t nc[4] = {c[0], c[1], c[2], c[3]};
      double bc = 1.0;
      if (dir == 0) {
        nc[mu] = c[mu] + 1;
        if (nc[mu] == L->n[mu]) {
          nc[mu] = 0;
          if (mu == 3 && L->tanti) bc = -1.0;
        }
      } else {
        nc[mu] = c[mu] - 1;
        if (nc[mu] < 0) {
          nc[mu] = L->n[mu] - 1;
          if (mu == 3 && L->tanti) bc = -1.0;
        }
      }
      int64_t y = site_index(L, nc);
      /* chi[beta][a] = W psi(y)[.][beta] with W = U_mu(x) (forward) or
       * U_mu(x-mu)^dagger (backward, x-mu = y). */
      cplx chi[4][3];
      for (int beta = 0; beta < 4; ++beta)
        for (int a = 0; a < 3; ++a) {
          cplx acc = cm(0, 0);
          for (int b = 0; b < 3; ++b) {
            cplx w = (dir == 0) ? link(L, U, mu, x, a, b) : cconj(link(L, U, mu, y, b, a));
            acc = cadd(acc, cmul(w, spin_ld(L, in, y, b, beta)));
          }
          chi[beta][a] = cscale(acc, bc);
        }
      /* spin matrix: forward (1 - s gamma_mu), backward (1 + s gamma_mu) */
      double s = (dir == 0) ? -(double)sgn : (double)sgn;
      for (int alpha = 0; alpha < 4; ++alpha)
        for (int beta = 0; beta < 4; ++beta) {
          cplx g = cm((alpha == beta ? 1.0 : 0.0) + s * GRE[mu][alpha][beta], s * GIM[mu][alpha][beta]);
          if (g.re == 0.0 && g.im == 0.0) continue;
          for (int a = 0; a < 3; ++a) res[alpha][a] = cadd(res[alpha][a], cmul(g, chi[beta][a]));
        }
    }
  }
}

static void zero_parity(const lat_t *L, double *out, int parity) {
  for (int64_t x = 0; x < L->V; ++x) {
    int64_t c[4];
    site_coords(L, x, c);
    if (site_parity(c) != parity) continue;
    for (int alpha = 0; alpha < 4; ++alpha)
      for (int a = 0; a < 3; ++a) st(out, a + 3 * (x + L->V * alpha), cm(0, 0));
  }
}

/* out = a_in * in + b_hop * H in, at sites of parity `out_parity` (all sites if
 * out_parity < 0); the other parity of `out` is set to zero.  `in` and `out`
 * must not alias. */
static void hop_axpy(const lat_t *L, const double *U, const double *in, double *out, int sgn,
                     int out_parity, double a_in, double b_hop) {
#pragma omp parallel for schedule(static)
  for (int64_t x = 0; x < L->V; ++x) {
    int64_t c[4];
    site_coords(L, x, c);
    if (out_parity >= 0 && site_parity(c) != out_parity) {
      for (int alpha = 0; alpha < 4; ++alpha)
        for (int a = 0; a < 3; ++a) st(out, a + 3 * (x + L->V * alpha), cm(0, 0));
      continue;
    }
    cplx h[4][3];
    hop_site(L, U, in, x, sgn, h);
    for (int alpha = 0; alpha < 4; ++alpha)
      for (int a = 0; a < 3; ++a) {
        int64_t k = a + 3 * (x + L->V * alpha);
        cplx v = cscale(h[alpha][a], b_hop);
        if (a_in != 0.0) v = cadd(v, cscale(ld(in, k), a_in));
        st(out, k, v);
      }
  }
}

/* ---- public: operator applications ------------------------------------- */

/* out = H in (dagger: adjoint hop), restricted to output parity `out_parity`
 * (-1: whole lattice).  H_{p,1-p} of the even-odd decomposition is
 * out_parity = p: the neighbours of a site of parity p all have parity 1-p. */
int jo_hop(const int dims[4], int tanti, const double *U, const double *in, double *out,
           int dagger, int out_parity) {
  lat_t L;
  if (lat_init(&L, dims, tanti) || !U || !in || !out || in == out) return -1;
  hop_axpy(&L, U, in, out, dagger ? -1 : 1, out_parity, 0.0, 1.0);
  return 0;
}

/* out = D in = in - kappa H in (paper: mul!(y, D, x)); dagger: D' . */
int jo_dirac(const int dims[4], int tanti, double kappa, const double *U, const double *in,
             double *out, int dagger) {
  lat_t L;
  if (lat_init(&L, dims, tanti) || !U || !in || !out || in == out) return -1;
  hop_axpy(&L, U, in, out, dagger ? -1 : 1, -1, 1.0, -kappa);
  return 0;
}

/* H at a list of sites only (for sampled checks at large volumes).
 * out_sites[i*24 + 2*(a + 3*alpha) + {0,1}] = (H in)(sites[i])[alpha][a]. */
int jo_hop_sites(const int dims[4], int tanti, const double *U, const double *in, int dagger,
                 const int64_t *sites, int64_t nsites, double *out_sites) {
  lat_t L;
  if (lat_init(&L, dims, tanti) || !U || !in || !sites || !out_sites) return -1;
  for (int64_t i = 0; i < nsites; ++i) {
    if (sites[i] < 0 || sites[i] >= L.V) return -1;
    cplx h[4][3];
    hop_site(&L, U, in, sites[i], dagger ? -1 : 1, h);
    for (int alpha = 0; alpha < 4; ++alpha)
      for (int a = 0; a < 3; ++a) st(out_sites + 24 * i, a + 3 * alpha, h[alpha][a]);
  }
  return 0;
}

/* Schur complement on the even sites: out_e = in_e - kappa^2 H_eo H_oe in_e.
 * With D = [[1, -kappa H_eo], [-kappa H_oe, 1]] in (even, odd) blocks this is
 * D_ee - D_eo D_oo^{-1} D_oe.  dagger: its adjoint, which is the same product
 * of adjoint hops.  `tmp` is a full-lattice scratch array. */
static void schur(const lat_t *L, double kappa, const double *U, const double *in, double *out,
                  int sgn, double *tmp) {
  hop_axpy(L, U, in, tmp, sgn, 1, 0.0, 1.0);            /* tmp_o = H_oe in_e */
  hop_axpy(L, U, tmp, out, sgn, 0, 0.0, -kappa * kappa); /* out_e = -k^2 H_eo tmp_o */
  for (int64_t x = 0; x < L->V; ++x) {
    int64_t c[4];
    site_coords(L, x, c);
    if (site_parity(c) != 0) continue;
    for (int alpha = 0; alpha < 4; ++alpha)
      for (int a = 0; a < 3; ++a) {
        int64_t k = a + 3 * (x + L->V * alpha);
        st(out, k, cadd(ld(in, k), ld(out, k)));
      }
  }
}

int jo_schur(const int dims[4], int tanti, double kappa, const double *U, const double *in,
             double *out, int dagger) {
  lat_t L;
  if (lat_init(&L, dims, tanti) || !U || !in || !out || in == out) return -1;
  double *tmp = (double *)malloc(sizeof(double) * 24 * (size_t)L.V);
  if (!tmp) return -2;
  schur(&L, kappa, U, in, out, dagger ? -1 : 1, tmp);
  free(tmp);
  return 0;
}

/* ---- BLAS-1 on full-lattice arrays (sequential, fixed order) ------------- */
static double norm2(const double *a, int64_t nreal) {
  double s = 0;
  for (int64_t i = 0; i < nreal; ++i) s += a[i] * a[i];
  return s;
}
static double redot(const double *a, const double *b, int64_t nreal) { /* Re <a, b> */
  double s = 0;
  for (int64_t i = 0; i < nreal; ++i) s += a[i] * b[i];
  return s;
}

/* Normal-equation operators.  op 0: A = D^dagger D (whole lattice).
 * op 1: A = Mhat^dagger Mhat (even sites).  Applied as A + shift (shift = 0
 * except for the shifted systems of multi-shift solves). */
typedef struct {
  lat_t L;
  int op;
  double kappa;
  double shift;
  const double *U;
  double *t1, *t2;
} normal_op;

static void apply_A(normal_op *A, const double *in, double *out) {
  if (A->op == 0) {
    hop_axpy(&A->L, A->U, in, A->t1, 1, -1, 1.0, -A->kappa);  /* D in */
    hop_axpy(&A->L, A->U, A->t1, out, -1, -1, 1.0, -A->kappa); /* D^dag (D in) */
  } else {
    schur(&A->L, A->kappa, A->U, in, A->t1, 1, A->t2);
    schur(&A->L, A->kappa, A->U, A->t1, out, -1, A->t2);
  }
  if (A->shift != 0.0)
    for (int64_t i = 0; i < 24 * A->L.V; ++i) out[i] += A->shift * in[i];
}

/* out = A in for op 0 (D^dag D) or op 1 (Mhat^dag Mhat); paper: DdagD_operator. */
int jo_normal_apply(const int dims[4], int tanti, double kappa, const double *U, int op,
                    const double *in, double *out) {
  normal_op A;
  if (lat_init(&A.L, dims, tanti) || !U || !in || !out || in == out || op < 0 || op > 1) return -1;
  A.op = op; A.kappa = kappa; A.U = U;
  size_t n = 24 * (size_t)A.L.V;
  A.t1 = (double *)malloc(sizeof(double) * n);
  A.t2 = (double *)malloc(sizeof(double) * n);
  if (!A.t1 || !A.t2) { free(A.t1); free(A.t2); return -2; }
  apply_A(&A, in, out);
  free(A.t1); free(A.t2);
  return 0;
}

/* Conjugate gradient (Hestenes-Stiefel) on the Hermitian positive-definite
 * system (A + shift) x = rhs, A = D^dag D (op 0) or Mhat^dag Mhat (op 1), in FP64
 * (A stands for A + shift below):
 *   r = rhs - A x, p = r;
 *   repeat: alpha = <r,r>/<p,Ap>; x += alpha p; r -= alpha Ap;
 *           beta = <r',r'>/<r,r>; p = r' + beta p
 *   until ||r||/||rhs|| <= tol (recursive residual) or maxiter.
 * x holds the start vector on entry (x0 = 0 unless the caller sets it).
 * On return *true_rel = ||rhs - A x|| / ||rhs|| recomputed from x.
 * Paper: solve_DinvX! with the stopping tolerance eps_CG.
 * Returns 0 on convergence, 1 if maxiter was reached, <0 on error. */
static int cg_impl(const int dims[4], int tanti, double kappa, const double *U, int op, double shift,
                   const double *rhs, double *x, double tol, int maxiter, int *iters, double *true_rel) {
  normal_op A;
  if (lat_init(&A.L, dims, tanti) || !U || !rhs || !x || op < 0 || op > 1) return -1;
  A.op = op; A.kappa = kappa; A.U = U; A.shift = shift;
  int64_t n = 24 * A.L.V;
  double *r = (double *)malloc(sizeof(double) * n);
  double *p = (double *)malloc(sizeof(double) * n);
  double *Ap = (double *)malloc(sizeof(double) * n);
  A.t1 = (double *)malloc(sizeof(double) * n);
  A.t2 = (double *)malloc(sizeof(double) * n);
  if (!r || !p || !Ap || !A.t1 || !A.t2) {
    free(r); free(p); free(Ap); free(A.t1); free(A.t2);
    return -2;
  }
  double bnorm = sqrt(norm2(rhs, n));
  int k = 0, rc = 1;
  if (bnorm == 0.0) {
    memset(x, 0, sizeof(double) * n);
    rc = 0;
  } else {
    apply_A(&A, x, Ap);
    for (int64_t i = 0; i < n; ++i) r[i] = rhs[i] - Ap[i];
    memcpy(p, r, sizeof(double) * n);
    double rr = norm2(r, n);
    if (sqrt(rr) <= tol * bnorm) rc = 0;
    while (rc != 0 && k < maxiter) {
      apply_A(&A, p, Ap);
      double pAp = redot(p, Ap, n);
      double alpha = rr / pAp;
      for (int64_t i = 0; i < n; ++i) x[i] += alpha * p[i];
      for (int64_t i = 0; i < n; ++i) r[i] -= alpha * Ap[i];
      double rr_new = norm2(r, n);
      ++k;
      if (sqrt(rr_new) <= tol * bnorm) { rc = 0; rr = rr_new; break; }
      double beta = rr_new / rr;
      for (int64_t i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
      rr = rr_new;
    }
  }
  if (iters) *iters = k;
  if (true_rel) {
    if (bnorm == 0.0) *true_rel = 0.0;
    else {
      apply_A(&A, x, Ap);
      for (int64_t i = 0; i < n; ++i) r[i] = rhs[i] - Ap[i];
      *true_rel = sqrt(norm2(r, n)) / bnorm;
    }
  }
  free(r); free(p); free(Ap); free(A.t1); free(A.t2);
  return rc;
}

/* cg_impl without a shift: the CG of solve_DinvX!. */
int jo_cg(const int dims[4], int tanti, double kappa, const double *U, int op, const double *rhs,
          double *x, double tol, int maxiter, int *iters, double *true_rel) {
  return cg_impl(dims, tanti, kappa, U, op, 0.0, rhs, x, tol, maxiter, iters, true_rel);
}

/* The same CG on the shifted system (A + shift) x = rhs (shift >= 0): the
 * definition of what a multi-shift solve returns for each of its shifts. */
int jo_cg_shift(const int dims[4], int tanti, double kappa, const double *U, int op, double shift,
                const double *rhs, double *x, double tol, int maxiter, int *iters, double *true_rel) {
  return cg_impl(dims, tanti, kappa, U, op, shift, rhs, x, tol, maxiter, iters, true_rel);
}

/* Solve D x = b (paper: solve_DinvX!(x, D, b)).
 * eo == 0: CG on D^dag D x = D^dag b over the whole lattice.
 * eo == 1: even-odd.  From the block form of D,
 *   bhat_e = b_e + kappa H_eo b_o,
 *   Mhat^dag Mhat x_e = Mhat^dag bhat_e   (CG, op 1),
 *   x_o = b_o + kappa H_oe x_e.
 * `tol` applies to the CG system (relative 2-norm of its residual);
 * *sys_rel is that system's true relative residual, *full_rel is
 * ||b - D x|| / ||b||.  Returns as jo_cg. */
int jo_solve(const int dims[4], int tanti, double kappa, const double *U, int eo, const double *b,
             double *x, double tol, int maxiter, int *iters, double *sys_rel, double *full_rel) {
  lat_t L;
  if (lat_init(&L, dims, tanti) || !U || !b || !x || b == x) return -1;
  int64_t n = 24 * L.V;
  double *rhs = (double *)malloc(sizeof(double) * n);
  double *t = (double *)malloc(sizeof(double) * n);
  double *t2 = (double *)malloc(sizeof(double) * n);
  if (!rhs || !t || !t2) { free(rhs); free(t); free(t2); return -2; }
  int rc;
  memset(x, 0, sizeof(double) * n);
  if (!eo) {
    hop_axpy(&L, U, b, rhs, -1, -1, 1.0, -kappa); /* D^dag b */
    rc = jo_cg(dims, tanti, kappa, U, 0, rhs, x, tol, maxiter, iters, sys_rel);
  } else {
    /* bhat_e = b_e + kappa H_eo b_o  (H_eo reads only odd sites of b) */
    hop_axpy(&L, U, b, t, 1, 0, 0.0, kappa);
    for (int64_t xs = 0; xs < L.V; ++xs) {
      int64_t c[4];
      site_coords(&L, xs, c);
      if (site_parity(c) != 0) continue;
      for (int k = 0; k < 12; ++k) {
        int64_t i = (k % 3) + 3 * (xs + L.V * (k / 3));
        st(t, i, cadd(ld(t, i), ld(b, i)));
      }
    }
    schur(&L, kappa, U, t, rhs, -1, t2); /* Mhat^dag bhat_e */
    rc = jo_cg(dims, tanti, kappa, U, 1, rhs, x, tol, maxiter, iters, sys_rel);
    /* x_o = b_o + kappa H_oe x_e */
    hop_axpy(&L, U, x, t, 1, 1, 0.0, kappa);
    for (int64_t xs = 0; xs < L.V; ++xs) {
      int64_t c[4];
      site_coords(&L, xs, c);
      if (site_parity(c) != 1) continue;
      for (int k = 0; k < 12; ++k) {
        int64_t i = (k % 3) + 3 * (xs + L.V * (k / 3));
        st(x, i, cadd(ld(t, i), ld(b, i)));
      }
    }
  }
  if (full_rel && rc >= 0) {
    hop_axpy(&L, U, x, t, 1, -1, 1.0, -kappa);
    double num = 0, den = norm2(b, n);
    for (int64_t i = 0; i < n; ++i) num += (b[i] - t[i]) * (b[i] - t[i]);
    *full_rel = den > 0 ? sqrt(num / den) : 0.0;
  }
  free(rhs); free(t); free(t2);
  return rc;
}

/* Zero the sites of one parity of a full-lattice spinor (test helper). */
int jo_zero_parity(const int dims[4], double *psi, int parity) {
  lat_t L;
  if (lat_init(&L, dims, 0) || !psi) return -1;
  zero_parity(&L, psi, parity);
  return 0;
}

/* Threads of the site loop (OpenMP builds; returns the count now in force,
 * 1 without OpenMP).  n <= 0 leaves the setting unchanged.  Used to time the
 * oracle single-threaded next to the all-core run; no arithmetic changes. */
#ifdef _OPENMP
#include <omp.h>
#endif
int jo_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

/* Derivative of the two-flavour Wilson fermion action
 *   S = eta^dag (D^dag D)^{-1} eta          (paper: evaluate_FermiAction)
 * with respect to every link (paper: calc_UdSfdU, "U dSf/dU").
 *
 * Given X = (D^dag D)^{-1} eta and Y = D X, a change dU of the links gives
 *   dS = -X^dag d(D^dag D) X = -2 Re(Y^dag dD X) = 2 kappa Re(Y^dag dH X),
 * and U_mu(x) enters H twice: (1 - gamma_mu) U_mu(x) psi(x+mu) at site x and
 * (1 + gamma_mu) U_mu(x)^dag psi(x) at site x+mu, both times the boundary sign
 * s (-1 for a link crossing the antiperiodic time boundary).  Hence, with the
 * convention dS = Re Tr[(dS/dU) dU] for every complex 3x3 variation dU,
 *   dS/dU_mu(x) = 2 kappa s (A + B^dag),
 *   A_{ba} = sum_{alpha,beta} (1 - gamma_mu)_{alpha beta} X_{beta b}(x+mu) conj(Y_{alpha a}(x)),
 *   B_{ba} = sum_{alpha,beta} (1 + gamma_mu)_{alpha beta} X_{beta b}(x)    conj(Y_{alpha a}(x+mu)),
 * and out = U_mu(x) dS/dU_mu(x) in the canonical link layout.  For the
 * variation U -> exp(eps w) U (w in su(3)) this gives dS/deps = Re Tr[out w].
 * Written from the definition: explicit 4x4 gamma matrices, no spin projection.
 */
/* U_mu(x) dS/dU_mu(x) of one link into res[i][a] (element (i, a)). */
static void force_link(const lat_t *L, double kappa, const double *U, const double *X, const double *Y,
                       int64_t x, int mu, cplx res[3][3]) {
  int64_t c[4];
  site_coords(L, x, c);
  int64_t nc[4] = {c[0], c[1], c[2], c[3]};
  double s = 1.0;
  nc[mu] = c[mu] + 1;
  if (nc[mu] == L->n[mu]) {
    nc[mu] = 0;
    if (mu == 3 && L->tanti) s = -1.0;
  }
  const int64_t xp = site_index(L, nc);
  cplx M[3][3];  /* M[b][a] = A_{ba} + conj(B_{ab}) */
  for (int b = 0; b < 3; ++b)
    for (int a = 0; a < 3; ++a) {
      cplx acc = cm(0, 0);
      for (int alpha = 0; alpha < 4; ++alpha)
        for (int beta = 0; beta < 4; ++beta) {
          const double d = (alpha == beta) ? 1.0 : 0.0;
          const cplx gm = cm(d - GRE[mu][alpha][beta], -GIM[mu][alpha][beta]);  /* 1 - gamma */
          const cplx gp = cm(d + GRE[mu][alpha][beta], GIM[mu][alpha][beta]);   /* 1 + gamma */
          /* A_{ba} term */
          acc = cadd(acc, cmul(gm, cmul(spin_ld(L, X, xp, b, beta), cconj(spin_ld(L, Y, x, a, alpha)))));
          /* conj(B_{ab}) term: B_{ab} = (1+gamma)_{alpha beta} X_{beta a}(x) conj(Y_{alpha b}(x+mu)) */
          acc = cadd(acc, cconj(cmul(gp, cmul(spin_ld(L, X, x, a, beta), cconj(spin_ld(L, Y, xp, b, alpha))))));
        }
      M[b][a] = acc;
    }
  for (int i = 0; i < 3; ++i)
    for (int a = 0; a < 3; ++a) {
      cplx acc = cm(0, 0);
      for (int b = 0; b < 3; ++b) acc = cadd(acc, cmul(link(L, U, mu, x, i, b), M[b][a]));
      res[i][a] = cscale(acc, 2.0 * kappa * s);
    }
}

int jo_fermi_force(const int dims[4], int tanti, double kappa, const double *U, const double *X,
                   const double *Y, double *out) {
  lat_t L;
  if (lat_init(&L, dims, tanti) || !U || !X || !Y || !out) return -1;
#pragma omp parallel for schedule(static)
  for (int64_t x = 0; x < L.V; ++x)
    for (int mu = 0; mu < 4; ++mu) {
      cplx r[3][3];
      force_link(&L, kappa, U, X, Y, x, mu, r);
      for (int i = 0; i < 3; ++i)
        for (int a = 0; a < 3; ++a) st(out, i + 3 * (a + 3 * (x + L.V * mu)), r[i][a]);
    }
  return 0;
}

/* The same for n links only: links[k] = site + V*mu (lexicographic site);
 * out[k] holds the 3x3 matrix, element (i, a) at i + 3*a (complex). */
int jo_fermi_force_links(const int dims[4], int tanti, double kappa, const double *U, const double *X,
                         const double *Y, const int64_t *links, int64_t n, double *out) {
  lat_t L;
  if (lat_init(&L, dims, tanti) || !U || !X || !Y || !links || !out || n < 0) return -1;
  for (int64_t k = 0; k < n; ++k) {
    if (links[k] < 0 || links[k] >= 4 * L.V) return -1;
    cplx r[3][3];
    force_link(&L, kappa, U, X, Y, links[k] % L.V, (int)(links[k] / L.V), r);
    for (int i = 0; i < 3; ++i)
      for (int a = 0; a < 3; ++a) st(out, 9 * k + i + 3 * a, r[i][a]);
  }
  return 0;
}

/* ---- staggered fermions (paper: Dirac_operator "staggered" with "mass") ----
 * Kogut-Susskind operator on one colour vector per site:
 *   (D psi)(x) = m psi(x) + (1/2) sum_mu eta_mu(x) [ U_mu(x) psi(x+mu)
 *                                                  - U_mu(x-mu)^dagger psi(x-mu) ]
 * eta_mu(x) = (-1)^(x_0 + ... + x_{mu-1}) (mu = x, y, z, t), and the same
 * antiperiodic time boundary sign as the Wilson operator.  The hopping part is
 * anti-Hermitian, so D^dagger = m - D_hop.  Layout: colour c of site s at
 * c + 3*s (complex). */
static inline int stag_eta(const int64_t c[4], int mu) {
  int64_t s = 0;
  for (int nu = 0; nu < mu; ++nu) s += c[nu];
  return (s & 1) ? -1 : 1;
}

/* out = a_in * in + b_hop * D_hop in at sites of parity out_parity (all if < 0);
 * sgn = +1 for D_hop, -1 for D_hop^dagger = -D_hop. */
static void stag_hop_axpy(const lat_t *L, const double *U, const double *in, double *out, int sgn,
                          int out_parity, double a_in, double b_hop) {
#pragma omp parallel for schedule(static)
  for (int64_t x = 0; x < L->V; ++x) {
    int64_t c[4];
    site_coords(L, x, c);
    if (out_parity >= 0 && site_parity(c) != out_parity) {
      for (int a = 0; a < 3; ++a) st(out, a + 3 * x, cm(0, 0));
      continue;
    }
    cplx h[3] = {cm(0, 0), cm(0, 0), cm(0, 0)};
    for (int mu = 0; mu < 4; ++mu) {
      const double eta = stag_eta(c, mu);
      for (int dir = 0; dir < 2; ++dir) {
        int64_t nc[4] = {c[0], c[1], c[2], c[3]};
        double bc = 1.0;
        if (dir == 0) {
          nc[mu] = c[mu] + 1;
          if (nc[mu] == L->n[mu]) { nc[mu] = 0; if (mu == 3 && L->tanti) bc = -1.0; }
        } else {
          nc[mu] = c[mu] - 1;
          if (nc[mu] < 0) { nc[mu] = L->n[mu] - 1; if (mu == 3 && L->tanti) bc = -1.0; }
        }
        const int64_t y = site_index(L, nc);
        const double f = 0.5 * eta * bc * (dir == 0 ? 1.0 : -1.0) * sgn;
        for (int a = 0; a < 3; ++a) {
          cplx acc = cm(0, 0);
          for (int b = 0; b < 3; ++b) {
            const cplx w = (dir == 0) ? link(L, U, mu, x, a, b) : cconj(link(L, U, mu, y, b, a));
            acc = cadd(acc, cmul(w, ld(in, b + 3 * y)));
          }
          h[a] = cadd(h[a], cscale(acc, f));
        }
      }
    }
    for (int a = 0; a < 3; ++a) {
      cplx v = cscale(h[a], b_hop);
      if (a_in != 0.0) v = cadd(v, cscale(ld(in, a + 3 * x), a_in));
      st(out, a + 3 * x, v);
    }
  }
}

/* out = D_hop in (dagger: D_hop^dagger) at sites of parity out_parity (all if < 0). */
int jo_stag_hop(const int dims[4], int tanti, const double *U, const double *in, double *out, int dagger,
                int out_parity) {
  lat_t L;
  if (lat_init(&L, dims, tanti) || !U || !in || !out || in == out) return -1;
  stag_hop_axpy(&L, U, in, out, dagger ? -1 : 1, out_parity, 0.0, 1.0);
  return 0;
}

/* out = D in = m in + D_hop in (dagger: m in - D_hop in), whole lattice. */
int jo_stag_dirac(const int dims[4], int tanti, double mass, const double *U, const double *in, double *out,
                  int dagger) {
  lat_t L;
  if (lat_init(&L, dims, tanti) || !U || !in || !out || in == out) return -1;
  stag_hop_axpy(&L, U, in, out, dagger ? -1 : 1, -1, mass, 1.0);
  return 0;
}

/* Solve D x = b by textbook CG on D^dag D x = D^dag b (whole lattice, FP64),
 * the plain definition of a staggered solve (paper: solve_DinvX! with the
 * staggered operator).  x0 = 0.  *true_rel = ||D^dag b - D^dag D x|| / ||D^dag b||,
 * *full_rel = ||b - D x|| / ||b||.  Returns 0 on convergence, 1 at maxiter. */
int jo_stag_solve(const int dims[4], int tanti, double mass, const double *U, const double *b, double *x,
                  double tol, int maxiter, int *iters, double *true_rel, double *full_rel) {
  lat_t L;
  if (lat_init(&L, dims, tanti) || !U || !b || !x) return -1;
  const int64_t n = 6 * L.V;
  double *rhs = (double *)malloc(sizeof(double) * n), *r = (double *)malloc(sizeof(double) * n);
  double *p = (double *)malloc(sizeof(double) * n), *Ap = (double *)malloc(sizeof(double) * n);
  double *t = (double *)malloc(sizeof(double) * n);
  if (!rhs || !r || !p || !Ap || !t) { free(rhs); free(r); free(p); free(Ap); free(t); return -2; }
#define STAG_A(in_, out_) do { stag_hop_axpy(&L, U, in_, t, 1, -1, mass, 1.0); \
                               stag_hop_axpy(&L, U, t, out_, -1, -1, mass, 1.0); } while (0)
  stag_hop_axpy(&L, U, b, rhs, -1, -1, mass, 1.0);  /* D^dag b */
  memset(x, 0, sizeof(double) * n);
  memcpy(r, rhs, sizeof(double) * n);
  memcpy(p, r, sizeof(double) * n);
  const double bnorm = sqrt(norm2(rhs, n));
  double rr = norm2(r, n);
  int k = 0, rc = 1;
  if (bnorm == 0.0 || sqrt(rr) <= tol * bnorm) rc = 0;
  while (rc != 0 && k < maxiter) {
    STAG_A(p, Ap);
    const double alpha = rr / redot(p, Ap, n);
    for (int64_t i = 0; i < n; ++i) x[i] += alpha * p[i];
    for (int64_t i = 0; i < n; ++i) r[i] -= alpha * Ap[i];
    const double rr_new = norm2(r, n);
    ++k;
    if (sqrt(rr_new) <= tol * bnorm) { rc = 0; break; }
    const double beta = rr_new / rr;
    for (int64_t i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
    rr = rr_new;
  }
  if (iters) *iters = k;
  if (true_rel) {
    STAG_A(x, Ap);
    for (int64_t i = 0; i < n; ++i) r[i] = rhs[i] - Ap[i];
    *true_rel = bnorm > 0 ? sqrt(norm2(r, n)) / bnorm : 0.0;
  }
  if (full_rel) {
    stag_hop_axpy(&L, U, x, t, 1, -1, mass, 1.0);
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] - t[i];
    const double bn = sqrt(norm2(b, n));
    *full_rel = bn > 0 ? sqrt(norm2(r, n)) / bn : 0.0;
  }
#undef STAG_A
  free(rhs); free(r); free(p); free(Ap); free(t);
  return rc;
}

/* ---- pure-gauge part of the HMC (paper: section "Hybrid Monte Carlo") -----
 * Wilson plaquette action, as the paper's example builds it (plaquette loops
 * and their adjoints, Sg = -evaluate_GaugeAction / NC):
 *   S_g = -(beta / 3) sum_x sum_{mu<nu} Re Tr P_munu(x),
 *   P_munu(x) = U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag.
 * Its link derivative in the convention of jo_fermi_force (dS = Re Tr[(dS/dU) dU]):
 *   U dS_g/dU_mu(x) = -(beta / 3) U_mu(x) V_mu(x),  V = sum over the six staples
 *   V_mu(x) = sum_{nu != mu} [ U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag
 *                            + U_nu(x+mu-nu)^dag U_mu(x-nu)^dag U_nu(x-nu) ]. */
typedef struct { cplx m[3][3]; } mat3;

static mat3 mat_link(const lat_t *L, const double *U, int mu, int64_t s) {
  mat3 r;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) r.m[a][b] = link(L, U, mu, s, a, b);
  return r;
}
static mat3 mat_mul(mat3 A, mat3 B) {
  mat3 r;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      cplx acc = cm(0, 0);
      for (int k = 0; k < 3; ++k) acc = cadd(acc, cmul(A.m[a][k], B.m[k][b]));
      r.m[a][b] = acc;
    }
  return r;
}
static mat3 mat_dag(mat3 A) {
  mat3 r;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) r.m[a][b] = cconj(A.m[b][a]);
  return r;
}
static int64_t shift_site(const lat_t *L, int64_t s, int mu, int step) {
  int64_t c[4];
  site_coords(L, s, c);
  c[mu] = (c[mu] + step + L->n[mu]) % L->n[mu];
  return site_index(L, c);
}

/* Sum over x and mu < nu of Re Tr P_munu(x). */
double jo_plaquette_sum(const int dims[4], const double *U) {
  lat_t L;
  if (lat_init(&L, dims, 0) || !U) return NAN;
  double sum = 0.0;
  for (int64_t x = 0; x < L.V; ++x)
    for (int mu = 0; mu < 4; ++mu)
      for (int nu = mu + 1; nu < 4; ++nu) {
        const mat3 P = mat_mul(mat_mul(mat_link(&L, U, mu, x), mat_link(&L, U, nu, shift_site(&L, x, mu, 1))),
                               mat_mul(mat_dag(mat_link(&L, U, mu, shift_site(&L, x, nu, 1))),
                                       mat_dag(mat_link(&L, U, nu, x))));
        sum += P.m[0][0].re + P.m[1][1].re + P.m[2][2].re;
      }
  return sum;
}

/* out = U dS_g/dU for every link (canonical link layout). */
int jo_gauge_force(const int dims[4], double beta, const double *U, double *out) {
  lat_t L;
  if (lat_init(&L, dims, 0) || !U || !out) return -1;
  for (int64_t x = 0; x < L.V; ++x)
    for (int mu = 0; mu < 4; ++mu) {
      mat3 V;
      memset(&V, 0, sizeof V);
      const int64_t xpm = shift_site(&L, x, mu, 1);
      for (int nu = 0; nu < 4; ++nu) {
        if (nu == mu) continue;
        const int64_t xpn = shift_site(&L, x, nu, 1), xmn = shift_site(&L, x, nu, -1);
        const int64_t xpmmn = shift_site(&L, xpm, nu, -1);
        const mat3 up = mat_mul(mat_mul(mat_link(&L, U, nu, xpm), mat_dag(mat_link(&L, U, mu, xpn))),
                                mat_dag(mat_link(&L, U, nu, x)));
        const mat3 dn = mat_mul(mat_mul(mat_dag(mat_link(&L, U, nu, xpmmn)), mat_dag(mat_link(&L, U, mu, xmn))),
                                mat_link(&L, U, nu, xmn));
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) V.m[a][b] = cadd(V.m[a][b], cadd(up.m[a][b], dn.m[a][b]));
      }
      const mat3 G = mat_mul(mat_link(&L, U, mu, x), V);
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) st(out, a + 3 * (b + 3 * (x + L.V * mu)), cscale(G.m[a][b], -beta / 3.0));
    }
  return 0;
}
