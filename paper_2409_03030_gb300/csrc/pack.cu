// Conversions between the canonical FP64 host layouts and the device layouts.
//
// Canonical layouts (JuliaQCD's column-major index order x[ic,ix,iy,iz,it,ialpha]
// and U[a,b,ix,iy,iz,it] per direction), complex interleaved:
//   site = ix + NX*(iy + NY*(iz + NZ*it))
//   spinor (ic, site, alpha) -> ic + 3*(site + V*alpha)
//   link (a, b, site, mu)    -> a + 3*(b + 3*(site + V*mu))
// One thread per lattice site.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "dw.cuh"
#include "kernels.h"

namespace jqcd {

__device__ __forceinline__ void site_of(const Geom &g, int64_t s, int &x, int &y, int &z, int &t) {
  x = (int)(s % g.nx);
  int64_t r = s / g.nx;
  y = (int)(r % g.ny);
  r /= g.ny;
  z = (int)(r % g.nz);
  t = (int)(r / g.nz);
}

__device__ __forceinline__ float2 split_dev(double v) {
  const float h = __double2float_rn(v);
  return make_float2(h, __double2float_rn(v - (double)h));
}

__global__ void gauge_pack_kernel(Geom g, const double *__restrict__ canon, float4 *dwo,
                                  double2 *f64o, float4 *f32o) {
  const int64_t V = 2 * g.vh;
  const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= 4 * V) return;
  const int mu = (int)(l / V);
  const int64_t s = l % V;
  int x, y, z, t;
  site_of(g, s, x, y, z, t);
  const int p = (x + y + z + t) & 1;
  const int64_t cb = s >> 1;
  double2 u[3][3];
  const double2 *src = reinterpret_cast<const double2 *>(canon) + 9 * (s + V * mu);
  for (int b = 0; b < 3; ++b)
    for (int a = 0; a < 3; ++a) u[a][b] = src[a + 3 * b];
  const int64_t blk = (int64_t)(p * 4 + mu);
  if (dwo) {
    for (int k = 0; k < 9; ++k) {
      float2 re = split_dev(u[k / 3][k % 3].x), im = split_dev(u[k / 3][k % 3].y);
      dwo[(blk * 9 + k) * g.vh + cb] = make_float4(re.x, im.x, re.y, im.y);  // (re.h, im.h, re.l, im.l)
    }
  }
  if (f64o) {
    for (int k = 0; k < 9; ++k) f64o[(blk * 9 + k) * g.vh + cb] = u[k / 3][k % 3];
  }
  if (f32o) {
    // rows 0 and 1: (U00,U01) (U02,U10) (U11,U12)
    const double2 e[6] = {u[0][0], u[0][1], u[0][2], u[1][0], u[1][1], u[1][2]};
    for (int j = 0; j < 3; ++j)
      f32o[(blk * 3 + j) * g.vh + cb] =
          make_float4((float)e[2 * j].x, (float)e[2 * j].y, (float)e[2 * j + 1].x, (float)e[2 * j + 1].y);
  }
}

__global__ void spinor_pack_kernel(Geom g, int prec, const double *__restrict__ canon, void *even,
                                   void *odd) {
  const int64_t V = 2 * g.vh;
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  int x, y, z, t;
  site_of(g, s, x, y, z, t);
  void *base = ((x + y + z + t) & 1) ? odd : even;
  const int64_t cb = s >> 1;
  const int64_t vh = g.vh;
  const double2 *src = reinterpret_cast<const double2 *>(canon);
  double2 v[12];
  for (int k = 0; k < 12; ++k) v[k] = src[(k % 3) + 3 * (s + V * (k / 3))];  // k = 3*alpha + ic
  if (prec == PREC_DW) {
    float4 *o = reinterpret_cast<float4 *>(base);
    for (int k = 0; k < 12; ++k) {
      float2 re = split_dev(v[k].x), im = split_dev(v[k].y);
      o[k * vh + cb] = make_float4(re.x, im.x, re.y, im.y);  // (re.h, im.h, re.l, im.l)
    }
  } else if (prec == PREC_F64) {
    double2 *o = reinterpret_cast<double2 *>(base);
    for (int k = 0; k < 12; ++k) o[k * vh + cb] = v[k];
  } else if (prec == PREC_F32) {
    float4 *o = reinterpret_cast<float4 *>(base);
    for (int j = 0; j < 6; ++j)
      o[j * vh + cb] = make_float4((float)v[2 * j].x, (float)v[2 * j].y, (float)v[2 * j + 1].x,
                                   (float)v[2 * j + 1].y);
  } else {  // PREC_F16N
    double m = 0.0;
    for (int k = 0; k < 12; ++k) m = fmax(m, fmax(fabs(v[k].x), fabs(v[k].y)));
    const float n = (float)m;
    const double inv = n > 0.f ? 1.0 / (double)n : 0.0;
    uint4 *o = reinterpret_cast<uint4 *>(base);
    for (int j = 0; j < 3; ++j) {
      unsigned w[4];
      for (int q = 0; q < 4; ++q) {
        __half2 h2 = __floats2half2_rn((float)(v[4 * j + q].x * inv), (float)(v[4 * j + q].y * inv));
        w[q] = *reinterpret_cast<unsigned *>(&h2);
      }
      o[j * vh + cb] = make_uint4(w[0], w[1], w[2], w[3]);
    }
    reinterpret_cast<float *>(o + 3 * vh)[cb] = n;
  }
}

__global__ void spinor_unpack_kernel(Geom g, int prec, const void *even, const void *odd,
                                     double *canon) {
  const int64_t V = 2 * g.vh;
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  int x, y, z, t;
  site_of(g, s, x, y, z, t);
  const void *base = ((x + y + z + t) & 1) ? odd : even;
  const int64_t cb = s >> 1;
  const int64_t vh = g.vh;
  double2 v[12];
  if (prec == PREC_DW) {
    const float4 *o = reinterpret_cast<const float4 *>(base);
    for (int k = 0; k < 12; ++k) {
      float4 q = o[k * vh + cb];
      v[k] = make_double2((double)q.x + (double)q.z, (double)q.y + (double)q.w);
    }
  } else if (prec == PREC_F64) {
    const double2 *o = reinterpret_cast<const double2 *>(base);
    for (int k = 0; k < 12; ++k) v[k] = o[k * vh + cb];
  } else if (prec == PREC_F32) {
    const float4 *o = reinterpret_cast<const float4 *>(base);
    for (int j = 0; j < 6; ++j) {
      float4 q = o[j * vh + cb];
      v[2 * j] = make_double2(q.x, q.y);
      v[2 * j + 1] = make_double2(q.z, q.w);
    }
  } else {
    const uint4 *o = reinterpret_cast<const uint4 *>(base);
    const float n = reinterpret_cast<const float *>(o + 3 * vh)[cb];
    for (int j = 0; j < 3; ++j) {
      uint4 q = o[j * vh + cb];
      const unsigned w[4] = {q.x, q.y, q.z, q.w};
      for (int k = 0; k < 4; ++k) {
        float2 f = __half22float2(*reinterpret_cast<const __half2 *>(&w[k]));
        v[4 * j + k] = make_double2((double)f.x * n, (double)f.y * n);
      }
    }
  }
  double2 *dst = reinterpret_cast<double2 *>(canon);
  for (int k = 0; k < 12; ++k) dst[(k % 3) + 3 * (s + V * (k / 3))] = v[k];
}

cudaError_t launch_gauge_pack(const Geom &g, const double *canon, void *dw, void *f64, void *f32,
                              cudaStream_t s) {
  const int64_t n = 8 * g.vh;
  note_launch();
  gauge_pack_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(
      g, canon, reinterpret_cast<float4 *>(dw), reinterpret_cast<double2 *>(f64),
      reinterpret_cast<float4 *>(f32));
  return cudaGetLastError();
}

cudaError_t launch_spinor_pack(const Geom &g, int prec, const double *canon, void *even, void *odd,
                               cudaStream_t s) {
  const int64_t n = 2 * g.vh;
  note_launch();
  spinor_pack_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(g, prec, canon, even, odd);
  return cudaGetLastError();
}

cudaError_t launch_spinor_unpack(const Geom &g, int prec, const void *even, const void *odd,
                                 double *canon, cudaStream_t s) {
  const int64_t n = 2 * g.vh;
  note_launch();
  spinor_unpack_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(g, prec, even, odd, canon);
  return cudaGetLastError();
}

}  // namespace jqcd
