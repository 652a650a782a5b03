/*
 * Seeded synthetic inputs for the Wilson-Dirac operator and its solvers.
 *
 * This module only DRAWS inputs: random SU(3) gauge links, Gaussian and point
 * sources.  It holds none of the operator's or the solver's arithmetic, and it
 * is the one piece of code that both the CUDA library's tests/benchmarks and
 * the CPU oracle consume.
 *
 * Canonical host layouts (JuliaQCD's column-major index order, paper section
 * "Definition of pseudo-fermion fields": x[ic,ix,iy,iz,it,ialpha], and the
 * gauge field shape (NC,NC,NX,NY,NZ,NT) per direction):
 *   site  = ix + NX*(iy + NY*(iz + NZ*it))
 *   spinor element (ic, site, alpha) -> complex index ic + 3*(site + V*alpha)
 *   link   element (a, b) of U_mu(site) -> complex index
 *                                       a + 3*(b + 3*(site + V*mu))
 * Complex numbers are interleaved (re, im) doubles.  mu = 0..3 is x,y,z,t.
 *
 * Random numbers: a counter-based generator.  Element i of a draw seeded with
 * `seed` starts its own SplitMix64 stream (Steele, Lea, Flood 2014) at state
 * mix(seed, i), so results do not depend on thread count or call order.
 * Uniforms take the top 53 bits and lie in (0, 1]; normals come from the
 * Box-Muller transform.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

typedef struct { double re, im; } cplx;

static inline cplx c_make(double r, double i) { cplx z = {r, i}; return z; }
static inline cplx c_add(cplx a, cplx b) { return c_make(a.re + b.re, a.im + b.im); }
static inline cplx c_sub(cplx a, cplx b) { return c_make(a.re - b.re, a.im - b.im); }
static inline cplx c_mul(cplx a, cplx b) {
  return c_make(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
static inline cplx c_conj(cplx a) { return c_make(a.re, -a.im); }
static inline cplx c_scale(cplx a, double s) { return c_make(a.re * s, a.im * s); }

/* ---- SplitMix64, counter-seeded ---------------------------------------- */
static inline uint64_t sm64_next(uint64_t *s) {
  uint64_t z = (*s += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* Start of the stream of element `i` of a draw seeded with `seed`. */
static inline uint64_t stream_start(uint64_t seed, uint64_t i) {
  uint64_t s = seed * 0xD1B54A32D192ED03ULL + 0x8CB92BA72F3D8DD7ULL;
  uint64_t h = sm64_next(&s);
  s = h ^ (i * 0x9E3779B97F4A7C15ULL + 0x632BE59BD9B4E019ULL);
  (void)sm64_next(&s); /* decorrelate neighbouring counters */
  return s;
}

static inline double uniform01(uint64_t *s) { /* (0, 1] */
  return (double)((sm64_next(s) >> 11) + 1) * (1.0 / 9007199254740992.0);
}

/* One complex normal with independent re, im ~ N(0, 1/2), so E|z|^2 = 1. */
static inline cplx cnormal(uint64_t *s) {
  double u1 = uniform01(s), u2 = uniform01(s);
  double r = sqrt(-log(u1)); /* sqrt(-2 ln u1) * sqrt(1/2) */
  double th = 6.283185307179586476925286766559 * u2;
  return c_make(r * cos(th), r * sin(th));
}

/* ---- 3x3 complex helpers (row-major m[a][b] in registers) --------------- */
typedef struct { cplx m[3][3]; } mat3;

static mat3 m3_mul(const mat3 *x, const mat3 *y) {
  mat3 r;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      cplx acc = c_make(0, 0);
      for (int k = 0; k < 3; ++k) acc = c_add(acc, c_mul(x->m[a][k], y->m[k][b]));
      r.m[a][b] = acc;
    }
  return r;
}

static cplx m3_det(const mat3 *q) {
  const cplx(*m)[3] = q->m;
  cplx t0 = c_sub(c_mul(m[1][1], m[2][2]), c_mul(m[1][2], m[2][1]));
  cplx t1 = c_sub(c_mul(m[1][0], m[2][2]), c_mul(m[1][2], m[2][0]));
  cplx t2 = c_sub(c_mul(m[1][0], m[2][1]), c_mul(m[1][1], m[2][0]));
  return c_add(c_sub(c_mul(m[0][0], t0), c_mul(m[0][1], t1)), c_mul(m[0][2], t2));
}

static void store_link(double *links, uint64_t V, int mu, uint64_t site, const mat3 *u) {
  double *base = links + 2 * (9 * (site + V * (uint64_t)mu));
  for (int b = 0; b < 3; ++b)
    for (int a = 0; a < 3; ++a) {
      base[2 * (a + 3 * b) + 0] = u->m[a][b].re;
      base[2 * (a + 3 * b) + 1] = u->m[a][b].im;
    }
}

/* Haar-random SU(3): QR of a complex Gaussian matrix by modified Gram-Schmidt
 * on its columns (R has a positive real diagonal, so Q is Haar on U(3),
 * Mezzadri 2007), then Q <- Q * det(Q)^(-1/3) with the principal cube root. */
static mat3 draw_haar(uint64_t *s) {
  mat3 z;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) z.m[a][b] = cnormal(s);
  for (int j = 0; j < 3; ++j) {
    for (int k = 0; k < j; ++k) {
      cplx proj = c_make(0, 0); /* <q_k, z_j> */
      for (int a = 0; a < 3; ++a) proj = c_add(proj, c_mul(c_conj(z.m[a][k]), z.m[a][j]));
      for (int a = 0; a < 3; ++a) z.m[a][j] = c_sub(z.m[a][j], c_mul(proj, z.m[a][k]));
    }
    double nrm = 0;
    for (int a = 0; a < 3; ++a) nrm += z.m[a][j].re * z.m[a][j].re + z.m[a][j].im * z.m[a][j].im;
    nrm = 1.0 / sqrt(nrm);
    for (int a = 0; a < 3; ++a) z.m[a][j] = c_scale(z.m[a][j], nrm);
  }
  cplx d = m3_det(&z);
  double phi = atan2(d.im, d.re) / 3.0;
  cplx f = c_make(cos(phi), -sin(phi));
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) z.m[a][b] = c_mul(z.m[a][b], f);
  return z;
}

/* U = exp(i eps H) with H = (A + A^dag)/2 - tr(...)/3 traceless Hermitian from a
 * complex Gaussian A.  Computed by scaling and squaring with a Taylor series
 * that runs to machine precision. */
static mat3 draw_expi(uint64_t *s, double eps) {
  mat3 A, X;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) A.m[a][b] = cnormal(s);
  double tr = 0;
  for (int a = 0; a < 3; ++a) tr += A.m[a][a].re; /* tr(A + A^dag)/2 is real */
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      cplx h = c_scale(c_add(A.m[a][b], c_conj(A.m[b][a])), 0.5);
      if (a == b) h.re -= tr / 3.0;
      X.m[a][b] = c_make(-eps * h.im, eps * h.re); /* i * eps * h */
    }
  double nrm = 0; /* max row sum norm */
  for (int a = 0; a < 3; ++a) {
    double r = 0;
    for (int b = 0; b < 3; ++b) r += hypot(X.m[a][b].re, X.m[a][b].im);
    if (r > nrm) nrm = r;
  }
  int sq = 0;
  while (nrm > 0.25) { nrm *= 0.5; ++sq; }
  double sc = ldexp(1.0, -sq);
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) X.m[a][b] = c_scale(X.m[a][b], sc);
  mat3 E, T; /* E = sum_k X^k / k!, T = current term */
  memset(&E, 0, sizeof E);
  memset(&T, 0, sizeof T);
  for (int a = 0; a < 3; ++a) { E.m[a][a] = c_make(1, 0); T.m[a][a] = c_make(1, 0); }
  for (int k = 1; k <= 24; ++k) {
    mat3 n = m3_mul(&T, &X);
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) T.m[a][b] = c_scale(n.m[a][b], 1.0 / k);
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) E.m[a][b] = c_add(E.m[a][b], T.m[a][b]);
  }
  for (int i = 0; i < sq; ++i) E = m3_mul(&E, &E);
  return E;
}

static uint64_t volume(const int dims[4]) {
  return (uint64_t)dims[0] * dims[1] * dims[2] * dims[3];
}

/* kind: 0 = unit links (cold start), 1 = Haar SU(3), 2 = exp(i eps H). */
int synth_gauge(double *links, const int dims[4], int kind, double eps, uint64_t seed) {
  if (!links || !dims) return -1;
  for (int d = 0; d < 4; ++d)
    if (dims[d] < 1) return -1;
  if (kind < 0 || kind > 2) return -1;
  uint64_t V = volume(dims);
  int64_t n = (int64_t)(4 * V);
#pragma omp parallel for schedule(static)
  for (int64_t l = 0; l < n; ++l) {
    int mu = (int)(l / (int64_t)V);
    uint64_t site = (uint64_t)l % V;
    uint64_t s = stream_start(seed, (uint64_t)l);
    mat3 u;
    if (kind == 0) {
      memset(&u, 0, sizeof u);
      for (int a = 0; a < 3; ++a) u.m[a][a] = c_make(1, 0);
    } else if (kind == 1) {
      u = draw_haar(&s);
    } else {
      u = draw_expi(&s, eps);
    }
    store_link(links, V, mu, site, &u);
  }
  return 0;
}

/* Gaussian spinor: every complex component independently re, im ~ N(0, 1/2). */
int synth_gaussian_spinor(double *psi, const int dims[4], uint64_t seed) {
  if (!psi || !dims) return -1;
  uint64_t n = 12 * volume(dims);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < (int64_t)n; ++i) {
    uint64_t s = stream_start(seed, (uint64_t)i);
    cplx z = cnormal(&s);
    psi[2 * i] = z.re;
    psi[2 * i + 1] = z.im;
  }
  return 0;
}

/* Point source delta_{x,0} delta_{alpha,spin} delta_{ic,colour} at the origin. */
int synth_point_source(double *psi, const int dims[4], int spin, int colour) {
  if (!psi || !dims || spin < 0 || spin > 3 || colour < 0 || colour > 2) return -1;
  uint64_t V = volume(dims);
  memset(psi, 0, sizeof(double) * 2 * 12 * V);
  psi[2 * (colour + 3 * (0 + V * (uint64_t)spin))] = 1.0;
  return 0;
}

/* Random SU(3) gauge transformation Omega(x), Haar, one 3x3 per site stored
 * like one direction of the links: a + 3*(b + 3*site). */
int synth_gauge_transform(double *omega, const int dims[4], uint64_t seed) {
  if (!omega || !dims) return -1;
  uint64_t V = volume(dims);
#pragma omp parallel for schedule(static)
  for (int64_t site = 0; site < (int64_t)V; ++site) {
    uint64_t s = stream_start(seed, (uint64_t)site);
    mat3 u = draw_haar(&s);
    store_link(omega, V, 0, (uint64_t)site, &u);
  }
  return 0;
}

/* Raw uniforms of the counter-based generator, for distribution tests. */
int synth_uniforms(double *out, uint64_t n, uint64_t seed) {
  if (!out) return -1;
  for (uint64_t i = 0; i < n; ++i) {
    uint64_t s = stream_start(seed, i);
    out[i] = uniform01(&s);
  }
  return 0;
}
