// Internal launch interface of the jqcd kernels (host side of the library).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "lattice.cuh"

namespace jqcd {

// Process-wide count of kernel launches issued by the library (n may be
// negative to take back launches recorded into a graph that is replayed).
void note_launch(int64_t n = 1);

constexpr int kHopThreads = 128;
inline unsigned hop_blocks(int64_t vh) { return (unsigned)((vh + kHopThreads - 1) / kHopThreads); }

struct SolverScalars;
// Scalar step the last block of a hop launch with norm takes (cg_steps.cuh)
enum { FIN_NONE = 0, FIN_ALPHA = 1, FIN_BETA = 2, FIN_MIXED_BETA = 3 };
// Grids of at most this many blocks take the scalar steps in their last block
// instead of a separate single-block launch.
#ifndef JQCD_FIN_MAX_BLOCKS
#define JQCD_FIN_MAX_BLOCKS 1024
#endif

struct HopParams {
  void *out;
  const void *in;
  const void *x;      // same parity as out, used when axpy
  const void *gauge;  // gauge field in the layout of the precision
  Geom g;
  int out_parity;
  double a, b;        // out = a*x + b*H in
  float2 a_split, b_split;
  double *partials;   // one per hop block when norm
  const int *guard;   // when non-null and *guard != 0 the launch does nothing
  SolverScalars *fin_S;  // with fin != FIN_NONE (and norm): the scalars the last block updates
  int fin;
};

// out_p = a x_p + b H_{p,1-p} in (dag: adjoint hop); partials get per-block
// ||out||^2 when norm: hop_norm_partials(prec, vh) of them.
cudaError_t launch_hop(int prec, const HopParams &P, bool dag, bool axpy, bool norm,
                       cudaStream_t s);

// The double-word hops run two threads per output site on lattices small
// enough that the two-thread grid fits in one wave of resident blocks (and
// of at most JQCD_DWP_SPLIT_MAX_VH sites per parity), where one thread per
// site leaves the GPU short of warps; their grids (and per-block partial
// sums) are then twice as many blocks.
#ifndef JQCD_DWP_SPLIT_MAX_VH
#define JQCD_DWP_SPLIT_MAX_VH 65536
#endif
bool dw_hop_split(int64_t vh);
// Lattices one size up (at most JQCD_DWP_SMALL_MAX_VH sites per parity and a
// one-thread grid that fits in one wave at a lower occupancy) run one thread
// per site compiled with a larger register budget.
#ifndef JQCD_DWP_SMALL_MAX_VH
#define JQCD_DWP_SMALL_MAX_VH 65536
#endif
bool dw_hop_small(int64_t vh);
unsigned dw_hop_blocks(int64_t vh);                 // blocks of a double-word hop launch
unsigned hop_norm_partials(int prec, int64_t vh);   // partials of a hop launch with norm

// ---- layouts ----------------------------------------------------------------
// Canonical FP64 links on the device -> every device layout requested
// (null destination pointers are skipped).
cudaError_t launch_gauge_pack(const Geom &g, const double *canon, void *dw, void *f64, void *f32,
                              cudaStream_t s);
// Canonical FP64 spinor (device) <-> per-parity device layout.
cudaError_t launch_spinor_pack(const Geom &g, int prec, const double *canon, void *even, void *odd,
                               cudaStream_t s);
cudaError_t launch_spinor_unpack(const Geom &g, int prec, const void *even, const void *odd,
                                 double *canon, cudaStream_t s);

// ---- BLAS-1 and reductions ---------------------------------------------------
constexpr int kBlasThreads = 256;
constexpr int kReduceThreads = 256;
unsigned blas_blocks(int64_t n);   // grid of the grid-stride vector kernels

// Device-resident solver scalars.
struct SolverScalars {
  double rr;        // current ||r||^2
  double rr_new;
  double pAp;
  double alpha, beta;
  double stop_rr;   // stop when rr <= stop_rr
  double rhs2;      // ||rhs||^2
  double rr_max;    // mixed precision: max ||r_inner||^2 since last reliable update
  double delta2;    // reliable update threshold (squared)
  double true_rr;   // ||rhs - A x||^2 recomputed after the loop
  double b2;        // ||b||^2 of the original system D x = b
  double full_rr;   // ||b - D x||^2
  double tmp0, tmp1;
  float2 alpha_dw, beta_dw, malpha_dw;
  float alpha_f, beta_f, malpha_f;
  int done;         // 0 running, 1 converged, 2 breakdown, 3 iteration cap reached
  int iters;
  int need_update;  // mixed: reliable update requested
  int max_iters;
  int halt;         // loop kernels return at once while nonzero (done or need_update)
  int reliable_updates;
  int fin_count;    // blocks of the current hop launch that have written their partial
  int pad1;
};

// sum of partials[0..n) in a fixed order -> *out
cudaError_t launch_finalize_sum(const double *partials, int n, double *out, cudaStream_t s);

// Flat double-word complex vectors (float4 = one complex DW), n elements.
cudaError_t launch_dw_copy(float4 *dst, const float4 *src, int64_t n, cudaStream_t s);
cudaError_t launch_dw_zero(float4 *dst, int64_t n, cudaStream_t s);
cudaError_t launch_dw_norm2(const float4 *a, int64_t n, double *partials, cudaStream_t s);
// r = b - y, partials of ||r||^2
cudaError_t launch_dw_xmy_norm(float4 *r, const float4 *b, const float4 *y, int64_t n,
                               double *partials, cudaStream_t s);
// x += alpha p; r -= alpha Ap; partials ||r||^2 (alpha from S; skipped when S->done)
cudaError_t launch_dw_cg_update(float4 *x, float4 *r, const float4 *p, const float4 *Ap, int64_t n,
                                const SolverScalars *S, double *partials, cudaStream_t s);
// p = r + beta p (skipped when S->done)
cudaError_t launch_dw_xpay(float4 *p, const float4 *r, int64_t n, const SolverScalars *S,
                           cudaStream_t s);

// ---- native FP64 vectors (blas_f64.cu): flat double2 = one complex FP64 ----
cudaError_t launch_f64_copy(double2 *dst, const double2 *src, int64_t n, cudaStream_t s);
cudaError_t launch_f64_zero(double2 *dst, int64_t n, cudaStream_t s);
cudaError_t launch_f64_norm2(const double2 *a, int64_t n, double *partials, cudaStream_t s);
// r = b - y, partials of ||r||^2
cudaError_t launch_f64_xmy_norm(double2 *r, const double2 *b, const double2 *y, int64_t n,
                                double *partials, cudaStream_t s);
// x += alpha p; r -= alpha Ap; partials ||r||^2 (alpha = S->alpha; skipped when S->halt)
cudaError_t launch_f64_cg_update(double2 *x, double2 *r, const double2 *p, const double2 *Ap,
                                 int64_t n, const SolverScalars *S, double *partials,
                                 cudaStream_t s);
// p = r + beta p (beta = S->beta; skipped when S->halt)
cudaError_t launch_f64_xpay(double2 *p, const double2 *r, int64_t n, const SolverScalars *S,
                            cudaStream_t s);
// double-word <-> FP64 complex vectors of n elements (widening is exact)
cudaError_t launch_dw_to_f64(double2 *dst, const float4 *src, int64_t n, cudaStream_t s);
cudaError_t launch_f64_to_dw(float4 *dst, const double2 *src, int64_t n, cudaStream_t s);

// ---- mixed precision (inner CG in FP32 or FP16+norm, even parity) ----------
// p = r_s + beta p in the hop precision (guarded)
cudaError_t launch_mixed_xpay(int hop_prec, void *p, const float4 *rs, int64_t vh,
                              const SolverScalars *S, cudaStream_t s);
// p = r_s converted to the hop precision
cudaError_t launch_mixed_copy(int hop_prec, void *p, const float4 *rs, int64_t vh, cudaStream_t s);
// r_s = FP32(r) for a double-word r of vh sites
cudaError_t launch_dw_to_f32(float4 *rs, const float4 *r, int64_t vh, cudaStream_t s);
// x += x_s (double-word += FP32), then x_s = 0
cudaError_t launch_dw_add_f32(float4 *x, float4 *xs, int64_t vh, cudaStream_t s);
// inner step: rr_new = sum; iters++; request a reliable update when
// rr_new <= stop, rr_new < delta^2 rr_max or the iteration cap is reached;
// otherwise beta = rr_new / rr
cudaError_t launch_mixed_beta(const double *partials, int n, SolverScalars *S, cudaStream_t s);
// after x += x_s and r = rhs - A x: rr_true = sum; done when rr_true <= stop
// (or cap reached); otherwise beta = rr_true / rr and the inner loop resumes
cudaError_t launch_mixed_after_update(const double *partials, int n, SolverScalars *S,
                                      cudaStream_t s);

// CG scalar steps (single block): alpha = rr / sum(partials)
cudaError_t launch_cg_alpha(const double *partials, int n, SolverScalars *S, cudaStream_t s);
// rr_new = sum(partials); iters++; done when rr_new <= stop_rr; beta = rr_new/rr
cudaError_t launch_cg_beta(const double *partials, int n, SolverScalars *S, cudaStream_t s);
// S->rr = sum(partials) and reset the loop state (start or restart of CG)
cudaError_t launch_cg_start(const double *partials, int n, SolverScalars *S, double tol2,
                            int max_iters, double delta2, cudaStream_t s);

// ---- fermion action and force (force.cu) ------------------------------------
// out [2][4][9][vh] double-word link field = U dS/dU from X = (D^dag D)^-1 eta
// and Y = D X (double-word spinors per parity).
cudaError_t launch_fermi_force(const Geom &g, const float4 *xe, const float4 *xo, const float4 *ye,
                               const float4 *yo, const float4 *gauge_dw, double kappa, float4 *out,
                               cudaStream_t s);
// out = gamma5 in, whole-lattice double-word spinor (24 vh chunks); in place allowed.
cudaError_t launch_gamma5_dw(float4 *out, const float4 *in, int64_t vh, cudaStream_t s);
// Per-block partials of Re <a, b> over n double-word complex numbers (skipped
// when guard is set and *guard != 0).
cudaError_t launch_dw_dot_re(const float4 *a, const float4 *b, int64_t n, double *partials, int nblocks,
                             cudaStream_t s, const int *guard = nullptr);
// Double-word link field -> canonical host-layout links (complex double).
cudaError_t launch_linkfield_unpack(const Geom &g, const float4 *dwf, double *canon, cudaStream_t s);

}  // namespace jqcd
