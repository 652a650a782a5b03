// Staggered (Kogut-Susskind) operator and solver (staggered.cu).
#pragma once
#include <cuda_runtime.h>

#include <string>

#include "jqcd.h"
#include "kernels.h"

namespace jqcd {

// Bytes of one parity of a double-word staggered field (three chunks per site).
inline size_t stag_parity_bytes(int64_t vh) { return (size_t)vh * 16 * 3; }
// Algorithmic bytes per output site of one staggered hop: the input colour
// vector once, 8 double-word links, the output.
constexpr double kStagHopBytes = 48.0 + 8 * 144.0 + 48.0;

unsigned stag_blocks(int64_t vh);
// out_p = a x_p + b D_hop(p <- 1-p) in (dagger: -D_hop); x may be null (no
// axpy); partials (one per block) of ||out||^2 when not null; the kernel
// returns at once when guard is set and *guard != 0.
cudaError_t launch_stag_hop(const Geom &g, int out_parity, bool dagger, const float4 *in, const float4 *x,
                            float4 *out, const float4 *gauge_dw, double a, double b, double *partials,
                            cudaStream_t s, const int *guard = nullptr);
cudaError_t launch_stag_pack(const Geom &g, const double *canon, float4 *even, float4 *odd, cudaStream_t s);
cudaError_t launch_stag_unpack(const Geom &g, const float4 *even, const float4 *odd, double *canon,
                               cudaStream_t s);

struct GaugeEntry;
// Solve D x = b, b in G.sb (double-word, whole lattice, even half first), x
// into G.sx; even-odd CG on m^2 - D_eo D_oe in double-word arithmetic.
jqcd_status solve_staggered(GaugeEntry &G, double mass, const jqcd_solve_params &P, cudaStream_t s,
                            jqcd_solve_info *info, std::string *msg);

}  // namespace jqcd
