// Device pieces of the HMC trajectory (hmc.cu).
#pragma once
#include <cuda_runtime.h>

namespace jqcd {

struct GaugeEntry;

// FP64 master links -> double-word and 12-real FP32 copies
cudaError_t launch_hmc_links_refresh(GaugeEntry &G, cudaStream_t s);
// FP64 master links -> canonical host-layout links (device buffer)
cudaError_t launch_links_unpack(const GaugeEntry &G, double *canon, cudaStream_t s);
// sum over x, mu < nu of Re Tr P_munu(x), to the host (synchronises)
cudaError_t hmc_plaquette_sum(GaugeEntry &G, double *out, cudaStream_t s);
// K = -sum Tr P^2 of the momenta G.hP, to the host (synchronises)
cudaError_t hmc_kinetic(GaugeEntry &G, double *out, cudaStream_t s);
// G.hP = i sum_a p^a T^a from device normals [link][8]
cudaError_t hmc_momenta_set(GaugeEntry &G, const double *normals_dev, cudaStream_t s);
// G.hG = U dS_g/dU of the plaquette action
cudaError_t hmc_gauge_force(GaugeEntry &G, double beta, cudaStream_t s);
// G.hP += coef * TA(G.hG + Gf)   (Gf: double-word link field or null)
cudaError_t hmc_momenta_update(GaugeEntry &G, const float4 *Gf, double coef, cudaStream_t s);
// U <- exp(eps P) U and refresh of the link copies
cudaError_t hmc_links_update(GaugeEntry &G, double eps, cudaStream_t s);
// out = a x + b y over n double-word complex numbers (out may alias x or y)
cudaError_t launch_dw_lincomb(float4 *out, const float4 *x, const float4 *y, double a, double b, int64_t n,
                              cudaStream_t s);

}  // namespace jqcd
