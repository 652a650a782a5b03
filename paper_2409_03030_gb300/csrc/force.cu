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
#include <cuda_runtime.h>

#include "fields.cuh"
#include "hop.cuh"
#include "hop_dw.cuh"
#include "kernels.h"
#include "reduce.cuh"

namespace jqcd {

namespace {

constexpr int kForceThreads = 128;

// w_s = Y_s + sum over the lower spins alpha with k_alpha = s of
// conj(phase_alpha) Y_alpha, for the projector (1 + S gamma_mu).
template <int MU, int S>
__device__ __forceinline__ void adjoint_half(const cw (&y)[4][3], cw (&w)[2][3]) {
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
    w[T::k2][c] = cadd(w[T::k2][c], phase<C2>(y[2][c]));
    w[T::k3][c] = cadd(w[T::k3][c], phase<C3>(y[3][c]));
  }
}

__device__ __forceinline__ void load_dw_spinor(const float4 *base, int64_t vh, int64_t i, cw (&s)[4][3]) {
#pragma unroll
  for (int k = 0; k < 12; ++k) dwc_unpack(__ldg(base + k * vh + i), s[k / 3][k % 3].re, s[k / 3][k % 3].im);
}

// X and Y of both parities as double-word spinor fields.
struct FieldPair {
  const float4 *xe, *xo, *ye, *yo;
};

// U dS/dU of direction MU for the link at site (p, cb).
template <int MU>
__device__ __forceinline__ void force_link(const Geom &g, int p, int64_t cb, int x, int y, int z, int t,
                                           const FieldPair &F, const float4 *gauge, dw two_kappa,
                                           float4 *out) {
  const int64_t vh = g.vh;
  bool neg;
  const int64_t nb = hop_neighbour(g, x, y, z, t, 2 * MU, neg);  // x + mu, parity 1-p
  const float4 *Xh = p ? F.xo : F.xe, *Yh = p ? F.yo : F.ye;
  const float4 *Xn = p ? F.xe : F.xo, *Yn = p ? F.ye : F.yo;
  cw h[2][3], w[2][3], hp[2][3], wp[2][3];
  {
    cw s4[4][3];
    load_dw_spinor(Xn, vh, nb, s4);
    project<MU, -1>(s4, h);     // rows 0, 1 of (1 - gamma_mu) X(x+mu)
    load_dw_spinor(Yh, vh, cb, s4);
    adjoint_half<MU, -1>(s4, w);  // partner of Y(x)
    load_dw_spinor(Xh, vh, cb, s4);
    project<MU, 1>(s4, hp);     // rows 0, 1 of (1 + gamma_mu) X(x)
    load_dw_spinor(Yn, vh, nb, s4);
    adjoint_half<MU, 1>(s4, wp);  // partner of Y(x+mu)
  }
  // M_ba = A_ba + conj(B_ab) = sum_s h_sb conj(w_sa) + conj(hp_sa) wp_sb
  cw M[3][3];
#pragma unroll
  for (int b = 0; b < 3; ++b)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      dwacc re = acc_first(h[0][b].re, w[0][a].re), im = acc_first(h[0][b].im, w[0][a].re);
      acc_mad(re, h[0][b].im, w[0][a].im);
      acc_mad(im, dw_neg(h[0][b].re), w[0][a].im);
      acc_mad(re, h[1][b].re, w[1][a].re);
      acc_mad(re, h[1][b].im, w[1][a].im);
      acc_mad(im, h[1][b].im, w[1][a].re);
      acc_mad(im, dw_neg(h[1][b].re), w[1][a].im);
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        acc_mad(re, hp[s][a].re, wp[s][b].re);
        acc_mad(re, hp[s][a].im, wp[s][b].im);
        acc_mad(im, hp[s][a].re, wp[s][b].im);
        acc_mad(im, dw_neg(hp[s][a].im), wp[s][b].re);
      }
      const dw r = acc_get(re), i = acc_get(im);
      M[b][a] = cw{dw_norm(r.h, r.l), dw_norm(i.h, i.l)};
    }
  // G = 2 kappa s U M
  const dw f = neg ? dw_neg(two_kappa) : two_kappa;
  const float4 *L = gauge + (size_t)((p * 4 + MU) * 9) * vh + cb;
  cw u[3][3];
#pragma unroll
  for (int k = 0; k < 9; ++k) dwc_unpack(__ldcs(L + k * vh), u[k / 3][k % 3].re, u[k / 3][k % 3].im);
  float4 *o = out + (size_t)((p * 4 + MU) * 9) * vh + cb;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      dwacc re = acc_first(u[i][0].re, M[0][a].re), im = acc_first(u[i][0].re, M[0][a].im);
      acc_mad(re, dw_neg(u[i][0].im), M[0][a].im);
      acc_mad(im, u[i][0].im, M[0][a].re);
#pragma unroll
      for (int b = 1; b < 3; ++b) {
        acc_mad(re, u[i][b].re, M[b][a].re);
        acc_mad(re, dw_neg(u[i][b].im), M[b][a].im);
        acc_mad(im, u[i][b].re, M[b][a].im);
        acc_mad(im, u[i][b].im, M[b][a].re);
      }
      const dw r = acc_get(re), m = acc_get(im);
      __stcs(o + (3 * i + a) * vh, dwc_pack(dw_mul(f, dw_norm(r.h, r.l)), dw_mul(f, dw_norm(m.h, m.l))));
    }
}

__global__ void __launch_bounds__(kForceThreads) force_kernel(Geom g, FieldPair F,
                                                              const float4 *__restrict__ gauge,
                                                              float2 two_kappa, float4 *__restrict__ out) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= 2 * g.vh) return;
  const int p = (int)(q / g.vh);
  const int64_t cb = q - (int64_t)p * g.vh;
  int x, y, z, t;
  cb_coords(g, cb, p, x, y, z, t);
  const dw tk = dw_make(two_kappa.x, two_kappa.y);
  force_link<0>(g, p, cb, x, y, z, t, F, gauge, tk, out);
  force_link<1>(g, p, cb, x, y, z, t, F, gauge, tk, out);
  force_link<2>(g, p, cb, x, y, z, t, F, gauge, tk, out);
  force_link<3>(g, p, cb, x, y, z, t, F, gauge, tk, out);
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
                                 double *partials) {
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
  note_launch();
  const float2 tk = dw_split_host(2.0 * kappa);
  force_kernel<<<(unsigned)((2 * g.vh + kForceThreads - 1) / kForceThreads), kForceThreads, 0, s>>>(
      g, FieldPair{xe, xo, ye, yo}, gauge_dw, tk, out);
  return cudaGetLastError();
}

cudaError_t launch_gamma5_dw(float4 *out, const float4 *in, int64_t vh, cudaStream_t s) {
  note_launch();
  gamma5_dw_kernel<<<blas_blocks(24 * vh), kBlasThreads, 0, s>>>(out, in, vh);
  return cudaGetLastError();
}

cudaError_t launch_dw_dot_re(const float4 *a, const float4 *b, int64_t n, double *partials, int nblocks,
                             cudaStream_t s) {
  note_launch();
  dw_dot_re_kernel<<<nblocks, kBlasThreads, 0, s>>>(a, b, n, partials);
  return cudaGetLastError();
}

cudaError_t launch_linkfield_unpack(const Geom &g, const float4 *dwf, double *canon, cudaStream_t s) {
  note_launch();
  const int64_t n = 8 * g.vh;
  linkfield_unpack_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(g, dwf, canon);
  return cudaGetLastError();
}

}  // namespace jqcd
