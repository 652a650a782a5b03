// Lattice geometry and device data layouts shared by the jqcd kernels.
//
// Even-odd (checkerboard) site order: a site (x,y,z,t) has parity
// (x+y+z+t) mod 2 and, within its parity, the index
//   cb = (x + NX*(y + NY*(z + NZ*t))) / 2          (NX even)
// so x/2 runs fastest.  Every field is stored per parity as a structure of
// arrays of 16-byte chunks: chunk k of site cb lives at  base[k*vh + cb],
// which makes each chunk load of a warp one fully coalesced 512-byte access.
//
// Spinor layouts (per parity, vh = V/2 sites; component k = 3*spin + colour):
//   DW   float4[12][vh]  (re.h, im.h, re.l, im.l) of component k
//   F64  double2[12][vh] (re, im) of component k
//   F32  float4[6][vh]   components 2j, 2j+1 as (re, im, re, im)
//   F16N uint4[3][vh]    components 4j..4j+3 as half2 (re, im), scaled by
//        1/n(site), followed by float n[vh], n = max |real| over the site
// Gauge layouts (parity p, direction mu, forward link U_mu(x) of the sites x
// of parity p; element (a,b) is chunk 3a+b; double-word chunks are
// (re.h, im.h, re.l, im.l) as for spinors):
//   DW   float4[2][4][9][vh]   F64  double2[2][4][9][vh]
//   F32  float4[2][4][3][vh]   rows 0 and 1 only (12 reals); row 2 is
//        recomputed as conj(row0 x row1), exact for SU(3).
// The antiperiodic time boundary is never folded into the links; hops that
// cross t = NT-1 <-> 0 multiply by -1 in the kernel.
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace jqcd {

struct Geom {
  int nx, ny, nz, nt;
  int nxh;       // nx / 2
  int64_t vh;    // sites per parity
  int tanti;     // 1: antiperiodic in time
};

// Coordinates of checkerboard site cb of parity p.
__device__ __forceinline__ void cb_coords(const Geom &g, int64_t cb, int p, int &x, int &y, int &z,
                                          int &t) {
  int xh = (int)(cb % g.nxh);
  int64_t r = cb / g.nxh;
  y = (int)(r % g.ny);
  r /= g.ny;
  z = (int)(r % g.nz);
  t = (int)(r / g.nz);
  x = 2 * xh + ((y + z + t + p) & 1);
}

__device__ __forceinline__ int64_t cb_index(const Geom &g, int x, int y, int z, int t) {
  return ((int64_t)x + (int64_t)g.nx * (y + (int64_t)g.ny * (z + (int64_t)g.nz * t))) >> 1;
}

// ---- chunk counts (16-byte units per site) -------------------------------
constexpr int kSpinorChunksDW = 12;
constexpr int kSpinorChunksF64 = 12;
constexpr int kSpinorChunksF32 = 6;
constexpr int kSpinorChunksF16 = 3;
constexpr int kLinkChunksDW = 9;
constexpr int kLinkChunksF64 = 9;
constexpr int kLinkChunksF32 = 3;

enum Prec { PREC_DW = 0, PREC_F32 = 1, PREC_F16N = 2, PREC_F64 = 3 };

// Bytes of one parity of a spinor field in precision `prec`.
__host__ __device__ inline size_t spinor_parity_bytes(int prec, int64_t vh) {
  switch (prec) {
    case PREC_DW: return (size_t)vh * 16 * kSpinorChunksDW;
    case PREC_F64: return (size_t)vh * 16 * kSpinorChunksF64;
    case PREC_F32: return (size_t)vh * 16 * kSpinorChunksF32;
    case PREC_F16N: return (size_t)vh * (16 * kSpinorChunksF16 + 4);
    default: return 0;
  }
}

}  // namespace jqcd
