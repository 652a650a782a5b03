/*
 * jqcd -- even-odd preconditioned Wilson-Dirac operator and conjugate-gradient
 * solvers for one NVIDIA GB300 GPU (sm_103a).  C ABI.
 *
 * The method is the fermion part of JuliaQCD's two-flavour Wilson HMC
 * (Nagai & Tomiya, arXiv:2409.03030): applying the Wilson-Dirac operator with
 * hopping parameter kappa,
 *     D = 1 - kappa H,
 *     (H psi)(x) = sum_mu [ (1 - gamma_mu) U_mu(x) psi(x+mu)
 *                         + (1 + gamma_mu) U_mu(x-mu)^dag psi(x-mu) ],
 * its adjoint D' and the normal operator D'D (paper, section "Definition of
 * Dirac operators": Dirac_operator(U,x,params) with params "kappa",
 * "eps_CG", "verbose_level"; mul!(y,D,x); solve_DinvX!(y,D,x); D';
 * DdagD_operator), and the CG solve that dominates the fermion action and
 * force (paper, "Definition of fermion actions" and "Hybrid Monte Carlo").
 *
 * Conventions fixed by this library where the paper is silent:
 *  - gamma matrices: DeGrand-Rossi chiral basis, mu = 0..3 <-> x, y, z, t;
 *  - boundaries periodic in x, y, z; if t_antiperiodic, every hop crossing
 *    the time boundary carries a factor -1;
 *  - even-odd: parity (x+y+z+t) mod 2, all extents even; the preconditioned
 *    operator is the Schur complement on the even sites
 *        Mhat = 1 - kappa^2 H_eo H_oe,
 *    where H_eo maps odd sites to even sites;
 *  - CG tolerance: relative 2-norm of the residual of the CG system,
 *    ||rhs - A x|| / ||rhs|| <= tol, A = Mhat'Mhat (even-odd) or D'D.
 *
 * Host layouts (canonical; the column-major index order of JuliaQCD's
 * x[ic,ix,iy,iz,it,ialpha] and U[a,b,ix,iy,iz,it], paper "Definition of
 * pseudo-fermion fields"), complex numbers as interleaved (re, im) doubles:
 *     site = ix + NX*(iy + NY*(iz + NZ*it))
 *     spinor element (ic, site, alpha)  at complex index ic + 3*(site + V*alpha)
 *     link element (a, b) of U_mu(site) at complex index a + 3*(b + 3*(site + V*mu))
 *
 * Device layouts are per parity (V/2 sites) and per precision; their sizes
 * come from jqcd_spinor_bytes.  JQCD_PREC_DW ("double-word") stores every
 * real as a pair of floats (hi, lo) -- 8 bytes per real like FP64, about 48
 * significant bits -- and computes with error-free FP32 transformations; it
 * is the library's FP64-class precision.  The Wilson hop forms its SU(3)
 * products as sums of exact products on a fixed offset grid, which agrees
 * with FP64 to about 1e-13 relative per apply (a few 1e-14 typical).
 * Double-word values have FP32's exponent range: the hop and the fermion
 * force are accurate as stated while every |link| x |spinor| product sum
 * of a site stays between about 2^-100 and 2^125 in magnitude (inputs scaled
 * by 2^+-60 are tested).  From about 2^125 up the grid offset leaves the
 * FP32 range: those outputs are Inf, NaN or inaccurate, so scale such
 * inputs first.
 * JQCD_PREC_F64 is IEEE double with native FP64 arithmetic.
 *
 * Errors: every call returns a jqcd_status and never aborts.  A message for
 * the last failure is available from jqcd_last_error.  After a CUDA error
 * raised by a kernel the context is poisoned: later calls return JQCD_ECUDA.
 * Ownership: the library never frees caller memory.  Host inputs are copied
 * during the call; device buffers passed to kernel-level calls stay owned by
 * the caller and must stay valid until the work on `stream` has completed.
 * Threading: one caller thread per context, except jqcd_serve_submit and
 * jqcd_serve_poll, which may be called from any thread while a server runs.
 */
#ifndef JQCD_H
#define JQCD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define JQCD_ABI_VERSION 1

#if defined(__GNUC__)
#define JQCD_API __attribute__((visibility("default")))
#else
#define JQCD_API
#endif

typedef struct jqcd_ctx jqcd_ctx;
typedef int32_t jqcd_status;

enum {
  JQCD_OK = 0,
  JQCD_EINVAL = -1,     /* bad argument (null pointer, odd extent, unknown id ...) */
  JQCD_ENOMEM = -2,     /* device or host allocation failed */
  JQCD_ECUDA = -3,      /* CUDA error; the context is poisoned */
  JQCD_ENOCONV = -4,    /* solver reached maxiter; info is filled in */
  JQCD_EBUSY = -5,      /* queue full (serving) */
  JQCD_ETIMEOUT = -6,   /* a bounded device wait gave up */
  JQCD_ENOTFOUND = -7,  /* unknown gauge id or ticket */
  JQCD_EBREAKDOWN = -8, /* CG breakdown: <p, A p> <= 0 or not finite */
  JQCD_PENDING = 1      /* serving: request not finished yet */
};

/* Device storage/arithmetic precisions. */
enum {
  JQCD_PREC_DW = 0,   /* FP64-class: float pairs, 8 B per real */
  JQCD_PREC_F32 = 1,  /* FP32 spinors; FP32 links with 12 stored reals */
  JQCD_PREC_F16N = 2, /* FP16 spinors scaled by a per-site FP32 norm; FP32 links */
  JQCD_PREC_F64 = 3   /* IEEE FP64 spinors and links, native FP64 arithmetic */
};

typedef struct {
  int32_t dims[4];        /* NX, NY, NZ, NT: each even and >= 2 */
  int32_t t_antiperiodic; /* 1: antiperiodic in time, 0: periodic */
} jqcd_lattice;

JQCD_API int32_t jqcd_abi_version(void);

/* Number of CUDA kernel launches the library has issued in this process
 * (all contexts).  Used to count the kernels inside a timed region. */
JQCD_API uint64_t jqcd_kernel_launches(void);

/* Create a context on CUDA device `device` (makes it current for the calling
 * thread).  *out receives the context; release it with jqcd_finalize. */
JQCD_API jqcd_status jqcd_init(int device, jqcd_ctx **out);
/* Free every gauge field and workspace of the context, then the context. */
JQCD_API jqcd_status jqcd_finalize(jqcd_ctx *ctx);
/* Message of the last failed call on ctx (never NULL; "" if none). */
JQCD_API const char *jqcd_last_error(const jqcd_ctx *ctx);

/* Upload a gauge field U_mu(x) (paper: Initialize_Gaugefields / the U passed
 * to Dirac_operator).  `links`: host, 4*V SU(3) matrices in the canonical
 * link layout, copied during the call.  The device copy is stored in every
 * layout the precisions need (double-word 18 reals, FP64 18 reals, FP32 12
 * reals with the third row recomputed as conj(row0 x row1), which assumes
 * det U = 1).  flags: reserved, pass 0.  *gauge_id names the field in later
 * calls. */
JQCD_API jqcd_status jqcd_gauge_upload(jqcd_ctx *ctx, const jqcd_lattice *lat, const double *links,
                              uint32_t flags, uint64_t *gauge_id);
JQCD_API jqcd_status jqcd_gauge_free(jqcd_ctx *ctx, uint64_t gauge_id);

/* Bytes of one parity of a spinor field of lattice `lat` in precision `prec`. */
JQCD_API jqcd_status jqcd_spinor_bytes(const jqcd_lattice *lat, int32_t prec, size_t *bytes_per_parity);

/* Convert a whole-lattice spinor between the canonical host layout (`host`,
 * 12*V complex doubles) and the device layout of `prec` (two caller-owned
 * device buffers of jqcd_spinor_bytes each), on `stream` (a cudaStream_t;
 * NULL = legacy default stream).  pack returns once `host` has been read;
 * unpack synchronises `stream` and returns with `host` written. */
JQCD_API jqcd_status jqcd_spinor_pack(jqcd_ctx *ctx, uint64_t gauge_id, const double *host, int32_t prec,
                             void *dev_even, void *dev_odd, void *stream);
JQCD_API jqcd_status jqcd_spinor_unpack(jqcd_ctx *ctx, uint64_t gauge_id, int32_t prec,
                               const void *dev_even, const void *dev_odd, double *host,
                               void *stream);

/* Even-odd hop (the hopping term of mul!(y,D,x), paper "Definition of Dirac
 * operators"):
 *     out_p = a * x_p + b * H_{p,1-p} in_{1-p}
 * with p = out_parity (0 even, 1 odd); dagger != 0 uses the adjoint hop
 * (gamma_mu -> -gamma_mu).  in, x, out: caller-owned device buffers in the
 * layout of `prec`; x may be NULL (then a is ignored); out must not alias in.
 * norm2_dev: NULL or a device double that receives ||out_p||^2.
 * Asynchronous on `stream`. */
JQCD_API jqcd_status jqcd_dslash_eo(jqcd_ctx *ctx, uint64_t gauge_id, int32_t prec, int32_t out_parity,
                           int32_t dagger, const void *in, const void *x, void *out, double a,
                           double b, double *norm2_dev, void *stream);

/* Same operation as jqcd_dslash_eo, for callers that must not have the
 * library allocate device memory during the call.  This entry point has no
 * counterpart in the paper; it exists for users such as a solve server that
 * budgets every byte of HBM up front, or code that overlaps work on several
 * streams and cannot afford the device-wide synchronisation that cudaMalloc
 * and cudaFree may cause.  jqcd_dslash_eo allocates its norm scratch on first
 * use; this variant instead uses one fixed array of
 * JQCD_NOALLOC_MAX_SITES_PER_PARITY / 128 doubles (128 KiB) compiled into the
 * library, present on every device that loads the library until the process
 * exits.  Lattices with more than JQCD_NOALLOC_MAX_SITES_PER_PARITY sites per
 * parity are rejected with JQCD_EINVAL.
 * The first call on a device that asks for a norm looks up the array's
 * device address (cudaGetSymbolAddress) with that device current; make that
 * first call before any stream capture.  The address is kept for the life of
 * the process: resetting the device (cudaDeviceReset) or otherwise
 * re-creating its primary context while the library is loaded is not
 * supported by this entry point.
 * All calls share the one array and each call overwrites what it reads, so
 * nothing needs clearing, but calls whose work overlaps on the GPU (other
 * streams, other host threads) race on it: serialise them.
 * Arguments, layouts and results are those of jqcd_dslash_eo. */
#define JQCD_NOALLOC_MAX_SITES_PER_PARITY (16384 * 128)
JQCD_API jqcd_status jqcd_dslash_eo_noalloc(jqcd_ctx *ctx, uint64_t gauge_id, int32_t prec,
                                            int32_t out_parity, int32_t dagger, const void *in,
                                            const void *x, void *out, double a, double b,
                                            double *norm2_dev, void *stream);

/* out = Mhat' Mhat in on the even sites, Mhat = 1 - kappa^2 H_eo H_oe (the
 * even-odd form of DdagD_operator, paper "Definition of Dirac operators").
 * in, out: even-parity device buffers of `prec`, out must not alias in.
 * norm2_dev: NULL or a device double receiving ||Mhat in||^2 = <in, out>.
 * Uses a context-owned odd-parity temporary; asynchronous on `stream`. */
JQCD_API jqcd_status jqcd_mdagm(jqcd_ctx *ctx, uint64_t gauge_id, int32_t prec, double kappa, const void *in,
                       void *out, double *norm2_dev, void *stream);

/* Whole-lattice out = D in (dagger: D' in), paper mul!(y,D,x) and D'.
 * Four caller-owned device buffers of `prec` (in and out must not alias). */
JQCD_API jqcd_status jqcd_dirac_apply(jqcd_ctx *ctx, uint64_t gauge_id, int32_t prec, double kappa,
                             int32_t dagger, const void *in_even, const void *in_odd,
                             void *out_even, void *out_odd, void *stream);

/* Solver modes. */
enum {
  JQCD_CG_DW = 0,        /* every vector and operator in double-word precision */
  JQCD_CG_F64 = 1,       /* plain FP64 CG: every vector, hop (native DFMA, the
                            JQCD_PREC_F64 layout) and reduction in IEEE double;
                            eo = 0 or 1; no reliable updates */
  JQCD_CG_MIXED_F32 = 2, /* FP32 inner CG, double-word reliable updates */
  JQCD_CG_MIXED_F16 = 3  /* FP16+norm inner operator, FP32 inner vectors,
                            double-word reliable updates */
};

typedef struct {
  double kappa;      /* hopping parameter (paper params["kappa"]) */
  double tol;        /* relative residual of the CG system (paper params["eps_CG"]) */
  int32_t maxiter;   /* iteration cap, counted in operator applications of A */
  int32_t eo;        /* 1: even-odd preconditioned, 0: CG on D'D, whole lattice */
  int32_t mode;      /* JQCD_CG_* */
  int32_t verbose;   /* 0 quiet; >= 3 prints residuals to stderr (paper verbose_level) */
  double delta;      /* mixed modes: reliable-update threshold, 0 -> 0.01 */
  int32_t use_x0;    /* 1: x holds the start vector on entry; 0: start from 0 */
  int32_t reserved;
} jqcd_solve_params;

typedef struct {
  int32_t iters;            /* CG iterations (applications of A) */
  int32_t reliable_updates; /* mixed modes */
  int32_t restarts;         /* restarts after a true-residual check failed */
  int32_t status;           /* same as the return value */
  double true_rel_resid;    /* ||rhs - A x|| / ||rhs|| of the CG system, recomputed
                               in double-word after exit */
  double full_rel_resid;    /* ||b - D x|| / ||b|| */
  double seconds;           /* host wall time of the call */
  double gpu_seconds;       /* device time of the solve proper (CUDA events) */
  double hop_bytes;         /* algorithmic bytes moved by hop kernels */
  double hop_count;         /* number of hop launches */
} jqcd_solve_info;

/* Solve D x = b (paper: solve_DinvX!(x, D, b) -- note this call orders its
 * arguments input first, output second).  b, x: host, 12*V complex doubles
 * in the canonical spinor layout; b is copied, x is written before return.
 * Even-odd: bhat_e = b_e + kappa H_eo b_o, CG on Mhat'Mhat x_e = Mhat' bhat_e,
 * x_o = b_o + kappa H_oe x_e.  Returns JQCD_OK on convergence of the CG
 * system to `tol` (checked on the recomputed residual), JQCD_ENOCONV if
 * maxiter was hit (x holds the last iterate).  info may be NULL. */
JQCD_API jqcd_status jqcd_cg_solve(jqcd_ctx *ctx, uint64_t gauge_id, const jqcd_solve_params *params,
                          const double *b, double *x, jqcd_solve_info *info);

/* The same solve on device-resident fields: b_even, b_odd, x_even, x_odd are
 * caller-owned device buffers in the JQCD_PREC_DW layout (x is used as the
 * start vector when params->use_x0).  Synchronises `stream` before return.
 * In mode JQCD_CG_F64, b is widened exactly to FP64, the solve runs in FP64
 * and x is rounded back to double-word (jqcd_cg_solve instead packs the host
 * FP64 b straight into the FP64 layout, so it rounds nowhere). */
JQCD_API jqcd_status jqcd_cg_solve_dev(jqcd_ctx *ctx, uint64_t gauge_id, const jqcd_solve_params *params,
                              const void *b_even, const void *b_odd, void *x_even, void *x_odd,
                              jqcd_solve_info *info, void *stream);

/* Solve n systems D_i x_i = b_i together (batched mixed-precision CG):
 * every solve advances one iteration per pass of persistent kernels that
 * walk all active solves at once; solves on the same gauge field share each
 * link load (multi right-hand-side hops); one iteration is captured in a
 * CUDA graph and replayed; sites per tile and grid size are autotuned per
 * batch shape.  Each solve has its own kappa, tol and maxiter (params[i]);
 * all must use the same mixed mode (JQCD_CG_MIXED_F32 or _F16) and eo = 1.
 * b[i], x[i]: host canonical spinors of solve i's lattice (b copied, x
 * written before return).  Page-locked (pinned) b and x are copied on a
 * second stream: a solution goes to the host while the other solves iterate;
 * pageable ones are copied in order on the compute stream.  infos:
 * NULL or n entries.  Returns JQCD_OK when every solve converged, else the
 * first failing status (all infos filled). */
JQCD_API jqcd_status jqcd_cg_solve_batch(jqcd_ctx *ctx, int32_t n, const uint64_t *gauge_ids,
                                         const jqcd_solve_params *params, const double *const *b,
                                         double *const *x, jqcd_solve_info *infos);

/* ---- serving: continuous batching of solves -------------------------------
 * Requests go to one of three lanes by lattice size: at most 65,536 sites
 * per parity (16^3x32 and smaller), at most 524,288 (up to 32^3x32, e.g.
 * 24^3x48), and larger.  Each lane has a scheduler thread owned by the
 * context that admits its queued requests as engine slots and device memory
 * free up, advances every admitted solve of the lane together (the batched
 * engine of jqcd_cg_solve_batch), and completes each request as soon as it
 * converges.  The smaller a lane's lattices, the higher its stream priority,
 * so its solves iterate at their own pace instead of in lockstep with larger
 * ones; the lanes' work overlaps on the GPU.  Requests that arrive while
 * others run join their lane at the next iteration boundary.  Admission is
 * first come, first served within a lane, by HBM footprint: a request is
 * admitted when a slot of its lane is free and the device memory held by the
 * slot buffers of all lanes, plus what this request adds, stays within
 * hbm_budget_bytes (resident gauge fields are not counted).
 * Sources and solutions move on a copy stream of their own, so with pinned
 * (page-locked) host buffers they overlap the iterations of other requests;
 * pageable buffers work too, copied in order on the compute stream.
 * This mode of operation has no counterpart in the paper; it serves the
 * paper's solves (solve_DinvX! with per-request kappa and eps_CG). */
typedef struct {
  uint64_t gauge_id;         /* resident gauge field (jqcd_gauge_upload) */
  jqcd_solve_params params;  /* kappa, tol, maxiter; mode must match the server's; eo = 1 */
  const double *b;           /* host canonical source, read during admission */
  double *x;                 /* host canonical solution, written before completion */
} jqcd_request;              /* b and x must stay valid until the request has completed */

typedef struct {
  int64_t completed;      /* requests finished */
  int64_t rejected;       /* requests whose footprint exceeds the budget */
  double p50_s, p99_s;    /* latency percentiles, submit -> completion */
  double mean_s;
  double solves_per_s;    /* completed / (last completion - first submit) */
  double wall_s;
  double peak_hbm_bytes;  /* peak device bytes held by solve slots */
  int32_t peak_active;    /* largest number of solves iterating together (all lanes) */
  int32_t peak_queue;     /* largest number of requests waiting for admission */
} jqcd_serve_stats;

/* Start the scheduler threads.  max_slots: solves iterating together in each
 * lane (>= 1); max_queue: waiting requests of all lanes before submit
 * returns JQCD_EBUSY (0 = unbounded);
 * mode: JQCD_CG_MIXED_F16 or JQCD_CG_MIXED_F32.  One server per context. */
JQCD_API jqcd_status jqcd_serve_start(jqcd_ctx *ctx, size_t hbm_budget_bytes, int32_t max_slots,
                                      int32_t max_queue, int32_t mode);
/* Queue a request; *ticket identifies it.  Thread-safe.  JQCD_EBUSY when the
 * queue is full, JQCD_ENOTFOUND for an unknown gauge id. */
JQCD_API jqcd_status jqcd_serve_submit(jqcd_ctx *ctx, const jqcd_request *req, uint64_t *ticket);
/* JQCD_PENDING while queued or running; otherwise the request's final status
 * (info filled, x written) and the ticket is released.  Thread-safe. */
JQCD_API jqcd_status jqcd_serve_poll(jqcd_ctx *ctx, uint64_t ticket, jqcd_solve_info *info);
/* Wait for every submitted request to finish, stop the thread, report stats. */
JQCD_API jqcd_status jqcd_serve_stop(jqcd_ctx *ctx, jqcd_serve_stats *stats);

/* ---- fermion action and force (paper, section "Definition of fermion
 * actions": FermiAction, evaluate_FermiAction, calc_UdSfdU) ----------------
 * Two-flavour Wilson action of a pseudofermion eta,
 *   S = eta^dag (D^dag D)^{-1} eta = |(D^dag)^{-1} eta|^2,
 * computed from two solves of D z = c (each even-odd preconditioned, as
 * jqcd_cg_solve, in params->mode): Y = gamma5 D^{-1} gamma5 eta = (D^dag)^{-1}
 * eta and X = D^{-1} Y = (D^dag D)^{-1} eta; S = Re <eta, X>.
 * The pseudofermion heatbath eta = D^dag xi (paper: sample_pseudofermions!)
 * is jqcd_dirac_apply with dagger = 1; then S = |xi|^2.
 *
 * U dS/dU (one 3x3 complex matrix per link): with dS = Re Tr[(dS/dU) dU] for
 * every complex variation dU of a link, the library returns
 *   G_mu(x) = U_mu(x) dS/dU_mu(x) = 2 kappa s U_mu(x) (A + B^dag),
 *   A_ba = sum_alpha [(1 - gamma_mu) X(x+mu)]_alpha,b conj(Y_alpha,a(x)),
 *   B_ba = sum_alpha [(1 + gamma_mu) X(x)]_alpha,b    conj(Y_alpha,a(x+mu)),
 * s = -1 for links that cross the antiperiodic time boundary, else 1.  For
 * U -> exp(eps w) U with w in su(3): dS/deps = Re Tr[G w].  The HMC momentum
 * update takes the traceless anti-Hermitian part of G.  Layout: the canonical
 * link layout of jqcd_gauge_upload (4*V matrices, element (a, b) of link
 * (site, mu) at a + 3*(b + 3*(site + V*mu))), complex doubles.  Arithmetic is
 * double-word (FP64-class); X and Y are accurate to the solves' tol. */

/* S only.  eta: host canonical spinor (copied).  info (may be NULL) sums the
 * two solves' iterations, hop bytes and times; its residuals are the larger
 * of the two. */
JQCD_API jqcd_status jqcd_fermi_action(jqcd_ctx *ctx, uint64_t gauge_id, const jqcd_solve_params *params,
                                       const double *eta, double *action, jqcd_solve_info *info);
/* S and G.  udsdu: host, 4*V*9 complex doubles (written); action may be NULL. */
JQCD_API jqcd_status jqcd_fermi_force(jqcd_ctx *ctx, uint64_t gauge_id, const jqcd_solve_params *params,
                                      const double *eta, double *udsdu, double *action,
                                      jqcd_solve_info *info);
/* G from given X and Y (host canonical spinors): the per-link kernel alone. */
JQCD_API jqcd_status jqcd_fermi_force_xy(jqcd_ctx *ctx, uint64_t gauge_id, double kappa, const double *X,
                                         const double *Y, double *udsdu);
/* Device form: X_*, Y_* caller-owned JQCD_PREC_DW spinors per parity; out:
 * caller-owned device buffer of jqcd_linkfield_bytes() holding G as a
 * double-word link field ([parity][mu][3*a+b][site] chunks of
 * (re.h, im.h, re.l, im.l), the layout of the uploaded double-word gauge
 * field).  Asynchronous on `stream`. */
JQCD_API jqcd_status jqcd_fermi_force_dev(jqcd_ctx *ctx, uint64_t gauge_id, double kappa, const void *X_even,
                                          const void *X_odd, const void *Y_even, const void *Y_odd, void *out,
                                          void *stream);
JQCD_API jqcd_status jqcd_linkfield_bytes(const jqcd_lattice *lat, size_t *bytes);

/* ---- multi-shift CG (rational HMC; the paper lists RHMC among its
 * algorithms) -------------------------------------------------------------
 * Solves (Mhat^dag Mhat + shifts[i]) x_i = rhs, i < nshift (1..32), on the
 * even sites in one Krylov space: one operator application per iteration for
 * all shifts (double-word arithmetic; params: eo = 1, mode JQCD_CG_DW, kappa,
 * tol, maxiter).  Shifts must be finite and >= 0.  Shift i stops once its
 * recursive residual |zeta_i r| <= tol |rhs|; every x_i's true residual
 * ||rhs - (A + sigma_i) x_i|| / ||rhs|| is recomputed and reported in
 * infos[i] (iters = the iteration at which shift i stopped).  Returns
 * JQCD_OK when every shift meets tol, JQCD_ENOCONV otherwise (x_i hold the
 * last iterates), JQCD_EBREAKDOWN on a non-positive <p, Ap>. */
/* rhs: host canonical spinor (odd sites ignored); x[i]: host canonical
 * spinors written with zeros on the odd sites; infos: NULL or nshift entries. */
JQCD_API jqcd_status jqcd_cg_multishift(jqcd_ctx *ctx, uint64_t gauge_id, const jqcd_solve_params *params,
                                        int32_t nshift, const double *shifts, const double *rhs,
                                        double *const *x, jqcd_solve_info *infos);
/* Device form: rhs_even one JQCD_PREC_DW parity; x_even[i] caller-owned
 * JQCD_PREC_DW parity buffers (a host array of nshift device pointers).
 * Synchronises `stream` before return. */
JQCD_API jqcd_status jqcd_cg_multishift_dev(jqcd_ctx *ctx, uint64_t gauge_id, const jqcd_solve_params *params,
                                            int32_t nshift, const double *shifts, const void *rhs_even,
                                            void *const *x_even, jqcd_solve_info *infos, void *stream);

/* ---- staggered fermions (paper: Dirac_operator "staggered" with "mass") ----
 * Kogut-Susskind operator on one colour vector per site:
 *   (D psi)(x) = m psi(x) + D_hop psi,
 *   (D_hop psi)(x) = 1/2 sum_mu eta_mu(x) [U_mu(x) psi(x+mu) - U_mu(x-mu)^dag psi(x-mu)],
 *   eta_mu(x) = (-1)^(x_0 + ... + x_{mu-1}) (mu = x, y, z, t),
 * with the lattice's time boundary sign on hops across t = NT-1 <-> 0.  D_hop
 * is anti-Hermitian: D^dag = m - D_hop.  Host layout: colour c of site s
 * (s = ix + NX*(iy + NY*(iz + NZ*it))) at c + 3*s, complex doubles (3*V).
 * Device layout: per parity three double-word chunks per site
 * (jqcd_staggered_bytes), the links of the uploaded gauge field.  Arithmetic
 * is double-word (FP64-class). */
JQCD_API jqcd_status jqcd_staggered_bytes(const jqcd_lattice *lat, size_t *bytes_per_parity);
JQCD_API jqcd_status jqcd_staggered_pack(jqcd_ctx *ctx, uint64_t gauge_id, const double *host, void *dev_even,
                                         void *dev_odd, void *stream);
/* Synchronises `stream` before return. */
JQCD_API jqcd_status jqcd_staggered_unpack(jqcd_ctx *ctx, uint64_t gauge_id, const void *dev_even,
                                           const void *dev_odd, double *host, void *stream);
/* out_p = a * x_p + b * D_hop(p <- 1-p) in  (dagger: -D_hop); x may be NULL;
 * norm2_dev (device double, may be NULL) receives ||out_p||^2.  in and out
 * must not alias.  Asynchronous on `stream`. */
JQCD_API jqcd_status jqcd_staggered_dslash_eo(jqcd_ctx *ctx, uint64_t gauge_id, int32_t out_parity,
                                              int32_t dagger, const void *in, const void *x, void *out, double a,
                                              double b, double *norm2_dev, void *stream);
/* Whole lattice: out = D in (dagger: D^dag in) = m in +- D_hop in. */
JQCD_API jqcd_status jqcd_staggered_apply(jqcd_ctx *ctx, uint64_t gauge_id, double mass, int32_t dagger,
                                          const void *in_even, const void *in_odd, void *out_even, void *out_odd,
                                          void *stream);
/* Solve D x = b (paper: solve_DinvX! with the staggered operator): CG on the
 * even-odd system (m^2 - D_eo D_oe) x_e = m b_e - D_eo b_o (Hermitian
 * positive definite), x_o = (b_o - D_oe x_e) / m.  params: tol (checked on the
 * recomputed residual of that system), maxiter, verbose; kappa, eo, mode are
 * ignored (always even-odd, double-word).  mass > 0.  b, x: host (3*V
 * complex doubles; b copied, x written).  info->full_rel_resid = ||b - Dx||/||b||. */
JQCD_API jqcd_status jqcd_staggered_solve(jqcd_ctx *ctx, uint64_t gauge_id, const jqcd_solve_params *params,
                                          double mass, const double *b, double *x, jqcd_solve_info *info);
/* The same on device fields (JQCD staggered double-word parities). */
JQCD_API jqcd_status jqcd_staggered_solve_dev(jqcd_ctx *ctx, uint64_t gauge_id, const jqcd_solve_params *params,
                                              double mass, const void *b_even, const void *b_odd, void *x_even,
                                              void *x_odd, jqcd_solve_info *info, void *stream);

/* ---- hybrid Monte Carlo (paper: section "Hybrid Monte Carlo", MDstep!) ----
 * One trajectory on the resident gauge field: momenta refresh from the given
 * normals, pseudofermion eta = D^dag xi, n_md leapfrog steps
 * U(dt/2) P(dt) U(dt/2) with dt = tau / n_md, and the Metropolis test with the
 * given uniform u: accepted iff u <= exp(-dH).  A rejected trajectory leaves
 * the gauge field as it was.
 *   H = K + S_g + S_f,  K = -sum_links Tr P^2 = sum (p^a)^2 / 2, P = i sum_a p^a T^a
 *   (T^a = Gell-Mann / 2), S_g = -(beta/3) sum_{x, mu<nu} Re Tr P_munu(x)
 *   (the paper's plaquette action, Sg = -evaluate_GaugeAction / NC),
 *   S_f = eta^dag (D^dag D)^{-1} eta (jqcd_fermi_action; S_f before = |xi|^2),
 *   dU/dt = P U, dP/dt = TA(U dS/dU) / 2 (U dS/dU: gauge part plus jqcd_fermi_force).
 * Gauge-field kernels run in FP64; the FP64 links are the master copy and the
 * double-word and FP32 copies are refreshed after every update.  Random
 * numbers are inputs: normals[8*l + a] (l = site + V*mu, a < 8) are the
 * momentum coefficients p^a, xi (host canonical spinor, ignored without
 * fermions) the Gaussian pseudofermion source. */
typedef struct {
  double beta;       /* plaquette coupling (paper's example: 5.5) */
  double kappa;      /* Wilson hopping parameter */
  double tau;        /* trajectory length (paper: 1) */
  double tol;        /* CG tolerance of the fermion solves */
  int32_t n_md;      /* leapfrog steps (paper: MDsteps = 10) */
  int32_t fermions;  /* 1: two-flavour Wilson fermions; 0: pure gauge */
  int32_t mode;      /* CG mode of the fermion solves (JQCD_CG_DW, _MIXED_F32, _MIXED_F16) */
  int32_t maxiter;   /* per fermion solve; the solves start from the linear extrapolation
                        of the previous two solutions on the same pseudofermion (the first
                        from gamma5 xi), since the links move by O(tau / n_md) in between,
                        and stop at tol like a cold start */
} jqcd_hmc_params;
typedef struct {
  double H_old, H_new, dH;
  double plaquette;  /* sum Re Tr P / (18 V) of the field after the trajectory */
  double seconds;
  int32_t accepted;
  int32_t cg_iters;  /* iterations of every fermion solve */
} jqcd_hmc_info;
JQCD_API jqcd_status jqcd_hmc_trajectory(jqcd_ctx *ctx, uint64_t gauge_id, const jqcd_hmc_params *params,
                                         const double *normals, const double *xi, double u, jqcd_hmc_info *info);
/* Average plaquette sum Re Tr P / (18 V) of the resident field (paper's
 * calculate_Plaquette normalisation: 1 for the cold start). */
JQCD_API jqcd_status jqcd_gauge_plaquette(jqcd_ctx *ctx, uint64_t gauge_id, double *plaquette);
/* Copy the resident FP64 links to the host (canonical link layout, 36*V complex doubles). */
JQCD_API jqcd_status jqcd_gauge_download(jqcd_ctx *ctx, uint64_t gauge_id, double *links);

#ifdef __cplusplus
}
#endif
#endif /* JQCD_H */
