// Host-side state of one resident gauge field and the solver drivers.
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "jqcd.h"
#include "kernels.h"
#include "multishift.h"

namespace jqcd {

struct GaugeEntry {
  Geom g{};
  void *gauge_dw = nullptr, *gauge_f64 = nullptr, *gauge_f32 = nullptr;

  // workspace, allocated on first use
  double *canon = nullptr;        // 12*V complex doubles: host <-> device staging
  double *partials = nullptr;     // reduction partial sums
  SolverScalars *S = nullptr;     // device scalars of the running solve
  SolverScalars *S_host = nullptr;  // pinned mirror
  void *tmp[4] = {nullptr, nullptr, nullptr, nullptr};   // odd-parity temporaries per precision
  void *tmp2[4] = {nullptr, nullptr, nullptr, nullptr};  // even-parity temporaries per precision
  // whole-lattice double-word solver vectors (even half first, then odd)
  float4 *vb = nullptr, *vsol = nullptr, *vr = nullptr, *vp = nullptr, *vAp = nullptr,
         *vw = nullptr, *vt = nullptr, *vrhs = nullptr;
  // mixed-precision inner vectors (even parity): x, r in FP32; p, w in the
  // hop precision; t odd in the hop precision
  void *mx = nullptr, *mr = nullptr, *mp[2] = {nullptr, nullptr}, *mw[2] = {nullptr, nullptr},
       *mt[2] = {nullptr, nullptr};
  // native FP64 solver vectors (whole lattice)
  double2 *fb = nullptr, *fsol = nullptr, *fr = nullptr, *fp = nullptr, *fAp = nullptr,
          *fw = nullptr, *ft = nullptr, *frhs = nullptr;
  // fermion action / force workspace: eta, X, Y (whole-lattice double-word),
  // the double-word link-field result and its canonical host-layout staging
  float4 *feta = nullptr, *fX = nullptr, *fY = nullptr, *fout = nullptr;
  double *lcanon = nullptr;
  // multi-shift CG workspace: per-shift search directions and scalars
  std::vector<float4 *> ms_p, ms_x;  // ms_x: solutions of the host-buffer entry
  MsScalars *ms_S = nullptr;
  MsScalars *ms_S_host = nullptr;  // pinned mirror
  // staggered workspace (double-word, whole lattice: even half then odd half)
  float4 *sb = nullptr, *sx = nullptr, *sr = nullptr, *sp = nullptr, *sAp = nullptr, *st = nullptr,
         *srhs = nullptr;
  // HMC workspace: momenta, gauge force, backup of the FP64 links (FP64 link
  // fields) and the momentum normals of one refresh
  double2 *hP = nullptr, *hG = nullptr, *hUbak = nullptr;
  double *hNormals = nullptr;
  double *hPart = nullptr;  // per-block partials of the HMC reductions
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // a second stream for the CG's alpha step, which runs beside the hop that
  // follows it (fork and join events)
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // host destination of the canonical solution: when set, the solve queues
  // its unpack and copy on the side stream as soon as x is final (while the
  // full-system residual is computed) and sets x_host_queued; the caller
  // then waits for ev_join instead of copying x itself
  double *x_host_out = nullptr;
  bool x_host_queued = false;
  std::vector<void *> device_allocs;

  ~GaugeEntry();
  cudaError_t alloc(void **p, size_t bytes);
  template <typename T> cudaError_t alloc_t(T **p, size_t bytes) {
    void *v = nullptr;
    cudaError_t e = alloc(&v, bytes);
    *p = reinterpret_cast<T *>(v);
    return e;
  }
  size_t canon_bytes() const { return sizeof(double) * 2 * 12 * (size_t)(2 * g.vh); }
  cudaError_t ensure_canon();
  cudaError_t ensure_reduce();
  cudaError_t ensure_tmp(int prec);
  cudaError_t ensure_solver();
  cudaError_t ensure_mixed(int hop_prec);
  cudaError_t ensure_f64();
  cudaError_t ensure_force();
  cudaError_t ensure_multishift(int nshift);
  cudaError_t ensure_staggered();
  cudaError_t ensure_hmc();
  // fermion-solve history of a trajectory: previous X, Y and two start vectors
  float4 *hXp = nullptr, *hYp = nullptr, *hS1 = nullptr, *hS2 = nullptr;
  cudaError_t ensure_hmc_history();
  size_t linkfield_bytes() const { return (size_t)72 * 16 * g.vh; }  // [2][4][9][vh] float4
  size_t link_canon_bytes() const { return sizeof(double) * 2 * 9 * 4 * (size_t)(2 * g.vh); }
  int n_partials() const;
  float4 *vec_even(float4 *v) const { return v; }
  float4 *vec_odd(float4 *v) const { return v + 12 * g.vh; }
  const void *gauge_for(int prec) const;
  HopParams hop_params(int prec, int out_parity, const void *in, const void *x, void *out, double a,
                       double b, double *partials) const;
};

// out = Mhat^dag Mhat in (even sites) in precision `prec`; t_odd and w_even are
// temporaries; partials (if not null) receive ||Mhat in||^2 per hop block.
cudaError_t apply_mdagm(const GaugeEntry &G, int prec, double kappa, const void *in, void *out,
                        void *t_odd, void *w_even, double *partials, const int *guard,
                        cudaStream_t s);

// Last hop of the double-word even-odd normal operator fused with the CG
// update: P as for out = w - k^2 H^dag_eo t (P.x = w, P.in = t, P.out unused);
// x += alpha p and r -= alpha Ap in place (alpha = S->alpha_dw), P.partials
// gets one ||r||^2 per hop block.  Returns at once while *P.guard != 0.
cudaError_t launch_hop_dw_cg(const HopParams &P, const float4 *p, float4 *x, float4 *r,
                             const SolverScalars *S, cudaStream_t s);

// The same without x: Ap stays in registers, r -= alpha Ap with alpha =
// *alpha_dw (device, hi/lo pair), P.partials gets ||r||^2 per hop block
// (multi-shift CG, whose x_i are updated per shift elsewhere).
cudaError_t launch_hop_dw_r(const HopParams &P, float4 *r, const float2 *alpha_dw, cudaStream_t s);

// The same for the inner CG of the mixed solver in hop precision prec (FP32 or
// FP16 with norm): p, t and w in that precision, xs and rs FP32, alpha =
// S->alpha_f.
cudaError_t launch_hop_lp_cg(int prec, const HopParams &P, const void *p, float4 *xs, float4 *rs,
                             const SolverScalars *S, cudaStream_t s);

// Run the solve of D x = b for the double-word b in G.vb; the solution is
// left in G.vsol (whole lattice, double-word).  Mode JQCD_CG_F64 widens b to
// FP64, solves in FP64 and rounds the solution back to double-word.
jqcd_status solve_resident(GaugeEntry &G, const jqcd_solve_params &P, cudaStream_t s,
                           jqcd_solve_info *info, std::string *msg);

// The native FP64 solve (mode JQCD_CG_F64, any eo) of D x = b for the FP64 b
// in G.fb (whole lattice, JQCD_PREC_F64 layout); start vector (use_x0) and
// solution in G.fsol.  The caller has run G.ensure_f64().
jqcd_status solve_resident_f64(GaugeEntry &G, const jqcd_solve_params &P, cudaStream_t s,
                               jqcd_solve_info *info, std::string *msg);

}  // namespace jqcd
