// C-ABI entry points: context, gauge fields, spinor conversion, operator
// applications and the conjugate-gradient drivers.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <vector>
#include <vector>

#include <mutex>

#include "batch_engine.h"
#include "jqcd.h"
#include "kernels.h"
#include "serve.h"
#include "solver.h"
#include "staggered.h"
#include "hmc.h"
#include <nvtx3/nvToolsExt.h>

using namespace jqcd;

namespace {
std::atomic<uint64_t> g_launches{0};
}
void jqcd::note_launch(int64_t n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }

struct jqcd_ctx {
  int device = 0;
  int sm_count = 0;
  cudaStream_t stream = nullptr;
  bool poisoned = false;
  std::string err;
  uint64_t next_id = 1;
  std::map<uint64_t, std::unique_ptr<GaugeEntry>> gauges;
  std::unique_ptr<BatchEngine> engine[2];  // batched solves: FP32 and FP16 inner precision
  Server *server = nullptr;                // continuous-batching solve server
  int server_mode = 0;
  std::mutex gauges_mu;                    // gauge map vs. serve_submit from other threads
};

namespace {

jqcd_status fail(jqcd_ctx *ctx, jqcd_status st, const char *fmt, ...) {
  if (ctx) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    ctx->err = buf;
  }
  return st;
}

jqcd_status cuda_fail(jqcd_ctx *ctx, cudaError_t e, const char *where) {
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return fail(ctx, JQCD_ENOMEM, "%s: out of device memory", where);
  }
  ctx->poisoned = true;
  return fail(ctx, JQCD_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define CK(call, where)                                   \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, where); \
  } while (0)

jqcd_status check_ctx(jqcd_ctx *ctx) {
  if (!ctx) return JQCD_EINVAL;
  if (ctx->poisoned) return fail(ctx, JQCD_ECUDA, "context poisoned by an earlier CUDA error");
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
  return JQCD_OK;
}

jqcd_status lattice_geom(jqcd_ctx *ctx, const jqcd_lattice *lat, Geom *g) {
  if (!lat) return fail(ctx, JQCD_EINVAL, "lattice is NULL");
  for (int d = 0; d < 4; ++d)
    if (lat->dims[d] < 2 || (lat->dims[d] & 1))
      return fail(ctx, JQCD_EINVAL, "extent %d of direction %d must be even and >= 2",
                  lat->dims[d], d);
  g->nx = lat->dims[0];
  g->ny = lat->dims[1];
  g->nz = lat->dims[2];
  g->nt = lat->dims[3];
  g->nxh = g->nx / 2;
  const int64_t V = (int64_t)g->nx * g->ny * g->nz * g->nt;
  if (V > ((int64_t)1 << 34)) return fail(ctx, JQCD_EINVAL, "lattice too large");
  g->vh = V / 2;
  g->tanti = lat->t_antiperiodic ? 1 : 0;
  return JQCD_OK;
}

GaugeEntry *find_gauge(jqcd_ctx *ctx, uint64_t id) {
  auto it = ctx->gauges.find(id);
  return it == ctx->gauges.end() ? nullptr : it->second.get();
}

bool valid_prec(int32_t p) { return p >= 0 && p <= 3; }

}  // namespace

// NVTX range over one C ABI call, named after the call: visible to
// profilers, a no-op when none is attached.
struct AbiRange {
  explicit AbiRange(const char *name) { nvtxRangePushA(name); }
  ~AbiRange() { nvtxRangePop(); }
  AbiRange(const AbiRange &) = delete;
  AbiRange &operator=(const AbiRange &) = delete;
};
#define JQCD_RANGE() AbiRange jqcd_range_(__func__)

extern "C" {

int32_t jqcd_abi_version(void) { return JQCD_ABI_VERSION; }

uint64_t jqcd_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

jqcd_status jqcd_init(int device, jqcd_ctx **out) {
  JQCD_RANGE();
  if (!out) return JQCD_EINVAL;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || n <= 0) {
    cudaGetLastError();
    return JQCD_ECUDA;
  }
  if (device < 0 || device >= n) return JQCD_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) return JQCD_ECUDA;
  std::unique_ptr<jqcd_ctx> ctx(new (std::nothrow) jqcd_ctx());
  if (!ctx) return JQCD_ENOMEM;
  ctx->device = device;
  cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device);
  if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) return JQCD_ECUDA;
  *out = ctx.release();
  return JQCD_OK;
}

jqcd_status jqcd_finalize(jqcd_ctx *ctx) {
  JQCD_RANGE();
  if (!ctx) return JQCD_EINVAL;
  cudaSetDevice(ctx->device);
  if (ctx->server) {
    std::string err;
    serve_destroy(ctx->server, nullptr, &err);
    ctx->server = nullptr;
  }
  if (!ctx->poisoned) cudaStreamSynchronize(ctx->stream);
  ctx->engine[0].reset();
  ctx->engine[1].reset();
  ctx->gauges.clear();
  if (ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
  return JQCD_OK;
}

const char *jqcd_last_error(const jqcd_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

jqcd_status jqcd_gauge_upload(jqcd_ctx *ctx, const jqcd_lattice *lat, const double *links,
                              uint32_t flags, uint64_t *gauge_id) {
  JQCD_RANGE();
  jqcd_status st = check_ctx(ctx);
  if (st) return st;
  if (!links || !gauge_id) return fail(ctx, JQCD_EINVAL, "links or gauge_id is NULL");
  if (flags != 0) return fail(ctx, JQCD_EINVAL, "flags must be 0");
  Geom g;
  if ((st = lattice_geom(ctx, lat, &g))) return st;
  std::unique_ptr<GaugeEntry> G(new GaugeEntry());
  G->g = g;
  const size_t canon_bytes = sizeof(double) * 2 * 9 * 4 * (size_t)(2 * g.vh);
  const size_t dw_bytes = (size_t)16 * kLinkChunksDW * 8 * g.vh;
  const size_t f64_bytes = (size_t)16 * kLinkChunksF64 * 8 * g.vh;
  const size_t f32_bytes = (size_t)16 * kLinkChunksF32 * 8 * g.vh;
  double *canon = nullptr;
  CK(G->alloc(&G->gauge_dw, dw_bytes), "gauge alloc");
  CK(G->alloc(&G->gauge_f64, f64_bytes), "gauge alloc");
  CK(G->alloc(&G->gauge_f32, f32_bytes), "gauge alloc");
  CK(cudaMalloc(&canon, canon_bytes), "gauge staging alloc");
  cudaError_t e = cudaMemcpyAsync(canon, links, canon_bytes, cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess)
    e = launch_gauge_pack(g, canon, G->gauge_dw, G->gauge_f64, G->gauge_f32, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  cudaFree(canon);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "gauge upload");
  std::lock_guard<std::mutex> lk(ctx->gauges_mu);
  const uint64_t id = ctx->next_id++;
  ctx->gauges[id] = std::move(G);
  *gauge_id = id;
  return JQCD_OK;
}

jqcd_status jqcd_gauge_free(jqcd_ctx *ctx, uint64_t gauge_id) {
  JQCD_RANGE();
  if (!ctx) return JQCD_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->gauges_mu);
  auto it = ctx->gauges.find(gauge_id);
  if (it != ctx->gauges.end() && ctx->server && serve_uses_gauge(ctx->server, it->second.get()))
    return fail(ctx, JQCD_EBUSY, "gauge %llu has requests in flight", (unsigned long long)gauge_id);
  if (it == ctx->gauges.end()) return fail(ctx, JQCD_ENOTFOUND, "unknown gauge id %llu",
                                           (unsigned long long)gauge_id);
  cudaSetDevice(ctx->device);
  if (!ctx->poisoned) cudaDeviceSynchronize();
  ctx->gauges.erase(it);
  return JQCD_OK;
}

jqcd_status jqcd_spinor_bytes(const jqcd_lattice *lat, int32_t prec, size_t *bytes) {
  JQCD_RANGE();
  if (!bytes || !valid_prec(prec)) return JQCD_EINVAL;
  Geom g;
  if (lattice_geom(nullptr, lat, &g)) return JQCD_EINVAL;
  *bytes = spinor_parity_bytes(prec, g.vh);
  return JQCD_OK;
}

jqcd_status jqcd_spinor_pack(jqcd_ctx *ctx, uint64_t gauge_id, const double *host, int32_t prec,
                             void *dev_even, void *dev_odd, void *stream) {
  JQCD_RANGE();
  jqcd_status st = check_ctx(ctx);
  if (st) return st;
  GaugeEntry *G = find_gauge(ctx, gauge_id);
  if (!G) return fail(ctx, JQCD_ENOTFOUND, "unknown gauge id");
  if (!host || !dev_even || !dev_odd || !valid_prec(prec))
    return fail(ctx, JQCD_EINVAL, "spinor_pack: bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  CK(G->ensure_canon(), "staging alloc");
  CK(cudaMemcpyAsync(G->canon, host, G->canon_bytes(), cudaMemcpyHostToDevice, s), "spinor H2D");
  CK(launch_spinor_pack(G->g, prec, G->canon, dev_even, dev_odd, s), "spinor pack");
  return JQCD_OK;
}

jqcd_status jqcd_spinor_unpack(jqcd_ctx *ctx, uint64_t gauge_id, int32_t prec,
                               const void *dev_even, const void *dev_odd, double *host,
                               void *stream) {
  JQCD_RANGE();
  jqcd_status st = check_ctx(ctx);
  if (st) return st;
  GaugeEntry *G = find_gauge(ctx, gauge_id);
  if (!G) return fail(ctx, JQCD_ENOTFOUND, "unknown gauge id");
  if (!host || !dev_even || !dev_odd || !valid_prec(prec))
    return fail(ctx, JQCD_EINVAL, "spinor_unpack: bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  CK(G->ensure_canon(), "staging alloc");
  CK(launch_spinor_unpack(G->g, prec, dev_even, dev_odd, G->canon, s), "spinor unpack");
  CK(cudaMemcpyAsync(host, G->canon, G->canon_bytes(), cudaMemcpyDeviceToHost, s), "spinor D2H");
  CK(cudaStreamSynchronize(s), "spinor unpack sync");
  return JQCD_OK;
}

jqcd_status jqcd_dslash_eo(jqcd_ctx *ctx, uint64_t gauge_id, int32_t prec, int32_t out_parity,
                           int32_t dagger, const void *in, const void *x, void *out, double a,
                           double b, double *norm2_dev, void *stream) {
  JQCD_RANGE();
  jqcd_status st = check_ctx(ctx);
  if (st) return st;
  GaugeEntry *G = find_gauge(ctx, gauge_id);
  if (!G) return fail(ctx, JQCD_ENOTFOUND, "unknown gauge id");
  if (!in || !out || in == out || (out_parity != 0 && out_parity != 1) || !valid_prec(prec))
    return fail(ctx, JQCD_EINVAL, "dslash_eo: bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  if (norm2_dev) CK(G->ensure_reduce(), "workspace alloc");
  HopParams P = G->hop_params(prec, out_parity, in, x, out, a, b, norm2_dev ? G->partials : nullptr);
  CK(launch_hop(prec, P, dagger != 0, x != nullptr, norm2_dev != nullptr, s), "hop launch");
  if (norm2_dev)
    CK(launch_finalize_sum(G->partials, (int)hop_norm_partials(prec, G->g.vh), norm2_dev, s), "norm");
  return JQCD_OK;
}

jqcd_status jqcd_mdagm(jqcd_ctx *ctx, uint64_t gauge_id, int32_t prec, double kappa, const void *in,
                       void *out, double *norm2_dev, void *stream) {
  JQCD_RANGE();
  jqcd_status st = check_ctx(ctx);
  if (st) return st;
  GaugeEntry *G = find_gauge(ctx, gauge_id);
  if (!G) return fail(ctx, JQCD_ENOTFOUND, "unknown gauge id");
  if (!in || !out || in == out || !valid_prec(prec)) return fail(ctx, JQCD_EINVAL, "mdagm: bad argument");
  CK(G->ensure_tmp(prec), "workspace alloc");
  CK(G->ensure_reduce(), "workspace alloc");
  CK(apply_mdagm(*G, prec, kappa, in, out, G->tmp[prec], G->tmp2[prec],
                 norm2_dev ? G->partials : nullptr, nullptr, (cudaStream_t)stream),
     "mdagm");
  if (norm2_dev)
    CK(launch_finalize_sum(G->partials, (int)hop_norm_partials(prec, G->g.vh), norm2_dev,
                           (cudaStream_t)stream), "norm");
  return JQCD_OK;
}

jqcd_status jqcd_dirac_apply(jqcd_ctx *ctx, uint64_t gauge_id, int32_t prec, double kappa,
                             int32_t dagger, const void *in_even, const void *in_odd,
                             void *out_even, void *out_odd, void *stream) {
  JQCD_RANGE();
  jqcd_status st = check_ctx(ctx);
  if (st) return st;
  GaugeEntry *G = find_gauge(ctx, gauge_id);
  if (!G) return fail(ctx, JQCD_ENOTFOUND, "unknown gauge id");
  if (!in_even || !in_odd || !out_even || !out_odd || !valid_prec(prec) || in_even == out_even ||
      in_odd == out_odd || in_even == out_odd || in_odd == out_even)
    return fail(ctx, JQCD_EINVAL, "dirac_apply: bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  HopParams Pe = G->hop_params(prec, 0, in_odd, in_even, out_even, 1.0, -kappa, nullptr);
  HopParams Po = G->hop_params(prec, 1, in_even, in_odd, out_odd, 1.0, -kappa, nullptr);
  CK(launch_hop(prec, Pe, dagger != 0, true, false, s), "hop launch");
  CK(launch_hop(prec, Po, dagger != 0, true, false, s), "hop launch");
  return JQCD_OK;
}

// jqcd_cg_solve in mode JQCD_CG_F64: the canonical FP64 b (and start vector)
// is packed straight into the FP64 layout and the FP64 solution unpacked from
// it, so no step of the solve rounds below IEEE double.
static jqcd_status cg_solve_f64(jqcd_ctx *ctx, GaugeEntry *G, const jqcd_solve_params *params,
                                const double *b, double *x, jqcd_solve_info *info,
                                std::chrono::steady_clock::time_point t0) {
  cudaStream_t s = ctx->stream;
  const int64_t nh = 12 * G->g.vh;  // complex numbers per parity
  CK(G->ensure_f64(), "solver workspace alloc");
  CK(cudaMemcpyAsync(G->canon, b, G->canon_bytes(), cudaMemcpyHostToDevice, s), "b H2D");
  CK(launch_spinor_pack(G->g, PREC_F64, G->canon, G->fb, G->fb + nh, s), "b pack");
  if (params->use_x0) {
    CK(cudaMemcpyAsync(G->canon, x, G->canon_bytes(), cudaMemcpyHostToDevice, s), "x0 H2D");
    CK(launch_spinor_pack(G->g, PREC_F64, G->canon, G->fsol, G->fsol + nh, s), "x0 pack");
  }
  jqcd_solve_info inf;
  memset(&inf, 0, sizeof inf);
  std::string msg;
  jqcd_status st = solve_resident_f64(*G, *params, s, &inf, &msg);
  if (st == JQCD_ECUDA) ctx->poisoned = true;
  if (st == JQCD_OK || st == JQCD_ENOCONV) {
    CK(launch_spinor_unpack(G->g, PREC_F64, G->fsol, G->fsol + nh, G->canon, s), "x unpack");
    CK(cudaMemcpyAsync(x, G->canon, G->canon_bytes(), cudaMemcpyDeviceToHost, s), "x D2H");
    CK(cudaStreamSynchronize(s), "solve sync");
  }
  inf.status = st;
  inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (info) *info = inf;
  if (st != JQCD_OK) return fail(ctx, st, "cg_solve: %s", msg.c_str());
  return JQCD_OK;
}

jqcd_status jqcd_cg_solve(jqcd_ctx *ctx, uint64_t gauge_id, const jqcd_solve_params *params,
                          const double *b, double *x, jqcd_solve_info *info) {
  JQCD_RANGE();
  const auto t0 = std::chrono::steady_clock::now();
  jqcd_status st = check_ctx(ctx);
  if (st) return st;
  GaugeEntry *G = find_gauge(ctx, gauge_id);
  if (!G) return fail(ctx, JQCD_ENOTFOUND, "unknown gauge id");
  if (!params || !b || !x) return fail(ctx, JQCD_EINVAL, "cg_solve: bad argument");
  cudaStream_t s = ctx->stream;
  if (params->mode == JQCD_CG_F64) return cg_solve_f64(ctx, G, params, b, x, info, t0);
  CK(G->ensure_solver(), "solver workspace alloc");
  // host -> device: canonical b (and x0) into the solver's double-word vectors
  CK(cudaMemcpyAsync(G->canon, b, G->canon_bytes(), cudaMemcpyHostToDevice, s), "b H2D");
  CK(launch_spinor_pack(G->g, PREC_DW, G->canon, G->vec_even(G->vb), G->vec_odd(G->vb), s), "b pack");
  if (params->use_x0) {
    CK(cudaMemcpyAsync(G->canon, x, G->canon_bytes(), cudaMemcpyHostToDevice, s), "x0 H2D");
    CK(launch_spinor_pack(G->g, PREC_DW, G->canon, G->vec_even(G->vsol), G->vec_odd(G->vsol), s),
       "x0 pack");
  }
  jqcd_solve_info inf;
  memset(&inf, 0, sizeof inf);
  std::string msg;
  G->x_host_out = x;  // the solve copies x out while it computes the full residual
  st = solve_resident(*G, *params, s, &inf, &msg);
  G->x_host_out = nullptr;
  const bool queued = G->x_host_queued;
  G->x_host_queued = false;
  if (st == JQCD_ECUDA) ctx->poisoned = true;
  if (queued) {
    CK(cudaEventSynchronize(G->ev_join), "x copy");
  } else if (st == JQCD_OK || st == JQCD_ENOCONV) {
    CK(launch_spinor_unpack(G->g, PREC_DW, G->vec_even(G->vsol), G->vec_odd(G->vsol), G->canon, s),
       "x unpack");
    CK(cudaMemcpyAsync(x, G->canon, G->canon_bytes(), cudaMemcpyDeviceToHost, s), "x D2H");
    CK(cudaStreamSynchronize(s), "solve sync");
  }
  inf.status = st;
  inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (info) *info = inf;
  if (st != JQCD_OK) return fail(ctx, st, "cg_solve: %s", msg.c_str());
  return JQCD_OK;
}

jqcd_status jqcd_cg_solve_dev(jqcd_ctx *ctx, uint64_t gauge_id, const jqcd_solve_params *params,
                              const void *b_even, const void *b_odd, void *x_even, void *x_odd,
                              jqcd_solve_info *info, void *stream) {
  JQCD_RANGE();
  const auto t0 = std::chrono::steady_clock::now();
  jqcd_status st = check_ctx(ctx);
  if (st) return st;
  GaugeEntry *G = find_gauge(ctx, gauge_id);
  if (!G) return fail(ctx, JQCD_ENOTFOUND, "unknown gauge id");
  if (!params || !b_even || !b_odd || !x_even || !x_odd)
    return fail(ctx, JQCD_EINVAL, "cg_solve_dev: bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  CK(G->ensure_solver(), "solver workspace alloc");
  const int64_t nh = 12 * G->g.vh;  // complex DW numbers per parity
  CK(launch_dw_copy(G->vec_even(G->vb), (const float4 *)b_even, nh, s), "copy b");
  CK(launch_dw_copy(G->vec_odd(G->vb), (const float4 *)b_odd, nh, s), "copy b");
  if (params->use_x0) {
    CK(launch_dw_copy(G->vec_even(G->vsol), (const float4 *)x_even, nh, s), "copy x0");
    CK(launch_dw_copy(G->vec_odd(G->vsol), (const float4 *)x_odd, nh, s), "copy x0");
  }
  jqcd_solve_info inf;
  memset(&inf, 0, sizeof inf);
  std::string msg;
  st = solve_resident(*G, *params, s, &inf, &msg);
  if (st == JQCD_ECUDA) ctx->poisoned = true;
  if (st == JQCD_OK || st == JQCD_ENOCONV) {
    CK(launch_dw_copy((float4 *)x_even, G->vec_even(G->vsol), nh, s), "copy x");
    CK(launch_dw_copy((float4 *)x_odd, G->vec_odd(G->vsol), nh, s), "copy x");
    CK(cudaStreamSynchronize(s), "solve sync");
  }
  inf.status = st;
  inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (info) *info = inf;
  if (st != JQCD_OK) return fail(ctx, st, "cg_solve_dev: %s", msg.c_str());
  return JQCD_OK;
}


jqcd_status jqcd_cg_solve_batch(jqcd_ctx *ctx, int32_t n, const uint64_t *gauge_ids,
                                const jqcd_solve_params *params, const double *const *b,
                                double *const *x, jqcd_solve_info *infos) {
  JQCD_RANGE();
  jqcd_status st = check_ctx(ctx);
  if (st) return st;
  if (n < 1 || !gauge_ids || !params || !b || !x) return fail(ctx, JQCD_EINVAL, "cg_solve_batch: bad argument");
  const int32_t mode = params[0].mode;
  if (mode != JQCD_CG_MIXED_F32 && mode != JQCD_CG_MIXED_F16)
    return fail(ctx, JQCD_EINVAL, "cg_solve_batch: mode must be JQCD_CG_MIXED_F32 or JQCD_CG_MIXED_F16");
  std::vector<GaugeEntry *> G(n);
  for (int i = 0; i < n; ++i) {
    const jqcd_solve_params &P = params[i];
    if (P.mode != mode || !P.eo || !(P.tol > 0.0) || P.maxiter < 1 || !(P.kappa >= 0.0) ||
        !(P.delta >= 0.0 && P.delta < 1.0) || !b[i] || !x[i])
      return fail(ctx, JQCD_EINVAL, "cg_solve_batch: solve %d: bad parameters (one mixed mode for "
                  "all, eo = 1, tol > 0, maxiter >= 1)", i);
    G[i] = find_gauge(ctx, gauge_ids[i]);
    if (!G[i]) return fail(ctx, JQCD_ENOTFOUND, "cg_solve_batch: solve %d: unknown gauge id", i);
    if (G[i]->g.vh >= ((int64_t)1 << 31)) return fail(ctx, JQCD_EINVAL, "lattice too large for batching");
  }
  const int hp = mode == JQCD_CG_MIXED_F16 ? PREC_F16N : PREC_F32;
  std::unique_ptr<BatchEngine> &E = ctx->engine[hp == PREC_F16N ? 1 : 0];
  if (!E || E->max_slots() < n) {
    E.reset(new BatchEngine(hp, n, ctx->stream, ctx->sm_count));
    CK(E->init(), "batch engine init");
  }
  const bool timing = params[0].verbose >= 2;  // phase times on stderr
  auto tnow = [&]() {
    if (timing) cudaStreamSynchronize(ctx->stream);
    return std::chrono::steady_clock::now();
  };
  const auto t0 = tnow();
  for (int i = 0; i < n; ++i) CK(E->admit(i, G[i], params[i], b[i]), "batch admit");
  const auto t1 = tnow();
  CK(E->autotune(), "batch autotune");
  const auto t2 = tnow();
  int left = n;
  std::vector<int> done;
  jqcd_status worst = JQCD_OK;
  double t_collect = 0.0;
  // verbose >= 2: device time of the iteration graphs beside the wall time
  struct EventPair {
    cudaEvent_t a = nullptr, b = nullptr;
    ~EventPair() {
      if (a) cudaEventDestroy(a);
      if (b) cudaEventDestroy(b);
    }
  } ev;
  const bool graph_time = timing && cudaEventCreate(&ev.a) == cudaSuccess && cudaEventCreate(&ev.b) == cudaSuccess;
  double t_graphs = 0.0;
  int n_polls = 0;
  auto finish_one = [&](int i) {
    jqcd_solve_info inf;
    E->finish(i, &inf);
    if (infos) infos[i] = inf;
    if (inf.status != JQCD_OK && worst == JQCD_OK) worst = inf.status;
    --left;
  };
  // The device waits on the host between polls; keeping the next graph
  // queued during a poll was measured slower (0.159 against 0.155 s of
  // iterations for the 24-solve batch on GB300), so the loop stays simple.
  while (E->running() > 0) {
    if (graph_time) cudaEventRecord(ev.a, ctx->stream);
    CK(E->run(8), "batch iterations");
    if (graph_time) cudaEventRecord(ev.b, ctx->stream);
    done.clear();
    CK(E->poll(&done), "batch poll");
    ++n_polls;
    float ms = 0.f;
    if (graph_time && cudaEventElapsedTime(&ms, ev.a, ev.b) == cudaSuccess) t_graphs += 1e-3 * ms;
    // solutions of finished solves go to the host while the others iterate
    const auto c0 = std::chrono::steady_clock::now();
    for (int i : done) CK(E->collect_async(i, x[i]), "batch collect");
    for (int i = 0; i < n; ++i)
      if (E->drained(i)) finish_one(i);
    t_collect += std::chrono::duration<double>(std::chrono::steady_clock::now() - c0).count();
  }
  const auto c0 = std::chrono::steady_clock::now();
  for (int i = 0; i < n; ++i)
    if (E->collecting(i)) {
      CK(E->wait_collect(i), "batch collect");
      finish_one(i);
    }
  t_collect += std::chrono::duration<double>(std::chrono::steady_clock::now() - c0).count();
  if (left != 0) return fail(ctx, JQCD_ECUDA, "cg_solve_batch: %d solves not collected", left);
  if (timing) {
    const auto t3 = tnow();
    auto sec = [](std::chrono::steady_clock::time_point a, std::chrono::steady_clock::time_point b) {
      return std::chrono::duration<double>(b - a).count();
    };
    fprintf(stderr,
            "jqcd batch: admit %.4f s, autotune %.4f s, iterate+collect %.4f s (collect %.4f s; "
            "iteration graphs %.4f s of device time over %d polls)\n",
            sec(t0, t1), sec(t1, t2), sec(t2, t3), t_collect, t_graphs, n_polls);
  }
  if (worst != JQCD_OK) return fail(ctx, worst, "cg_solve_batch: a solve did not converge");
  return JQCD_OK;
}


jqcd_status jqcd_serve_start(jqcd_ctx *ctx, size_t hbm_budget_bytes, int32_t max_slots,
                             int32_t max_queue, int32_t mode) {
  JQCD_RANGE();
  jqcd_status st = check_ctx(ctx);
  if (st) return st;
  if (ctx->server) return fail(ctx, JQCD_EBUSY, "a server is already running on this context");
  if (max_slots < 1 || max_queue < 0 || (mode != JQCD_CG_MIXED_F16 && mode != JQCD_CG_MIXED_F32))
    return fail(ctx, JQCD_EINVAL, "serve_start: max_slots >= 1, max_queue >= 0, mixed mode");
  std::string err;
  Server *S = serve_create(ctx->device, ctx->sm_count, mode == JQCD_CG_MIXED_F16 ? PREC_F16N : PREC_F32,
                           hbm_budget_bytes, max_slots, max_queue, &err);
  if (!S) return fail(ctx, JQCD_ECUDA, "serve_start: %s", err.c_str());
  ctx->server = S;
  ctx->server_mode = mode;
  return JQCD_OK;
}

jqcd_status jqcd_serve_submit(jqcd_ctx *ctx, const jqcd_request *req, uint64_t *ticket) {
  JQCD_RANGE();
  if (!ctx || !req || !ticket || !req->b || !req->x) return JQCD_EINVAL;
  if (!ctx->server) return JQCD_EINVAL;
  const jqcd_solve_params &P = req->params;
  if (P.mode != ctx->server_mode || !P.eo || !(P.tol > 0.0) || P.maxiter < 1 ||
      !(P.kappa >= 0.0) || !(P.delta >= 0.0 && P.delta < 1.0))
    return JQCD_EINVAL;
  GaugeEntry *G;
  {
    std::lock_guard<std::mutex> lk(ctx->gauges_mu);
    G = find_gauge(ctx, req->gauge_id);
  }
  if (!G) return JQCD_ENOTFOUND;
  if (G->g.vh >= ((int64_t)1 << 31)) return JQCD_EINVAL;
  return serve_submit(ctx->server, G, *req, ticket);
}

jqcd_status jqcd_serve_poll(jqcd_ctx *ctx, uint64_t ticket, jqcd_solve_info *info) {
  JQCD_RANGE();
  if (!ctx || !ctx->server) return JQCD_EINVAL;
  return serve_poll(ctx->server, ticket, info, true);
}

jqcd_status jqcd_serve_stop(jqcd_ctx *ctx, jqcd_serve_stats *stats) {
  JQCD_RANGE();
  if (!ctx) return JQCD_EINVAL;
  if (!ctx->server) return fail(ctx, JQCD_EINVAL, "no server running");
  std::string err;
  jqcd_status st = serve_destroy(ctx->server, stats, &err);
  ctx->server = nullptr;
  if (st != JQCD_OK) {
    ctx->poisoned = true;
    return fail(ctx, st, "serve: %s", err.c_str());
  }
  return JQCD_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free variant of jqcd_dslash_eo (declared in jqcd.h).
//
// jqcd_dslash_eo allocates its reduction scratch from the device heap the
// first time a norm is requested.  This variant keeps that scratch -- one
// double per 128-site block of the hop -- in a fixed array compiled into the
// library instead, so the call itself never allocates.  The array lives in
// every device that loads the library until the process exits.
#include <mutex>

namespace {
constexpr int kNoAllocMaxBlocks = JQCD_NOALLOC_MAX_SITES_PER_PARITY / kHopThreads;
static_assert(JQCD_NOALLOC_MAX_SITES_PER_PARITY % kHopThreads == 0, "limit must be whole blocks");
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_partials[kNoAllocMaxBlocks];

std::mutex g_noalloc_mu;
double *g_noalloc_addr[kNoAllocMaxDevices] = {};

// Device address of g_noalloc_partials on the current device `dev`, looked up
// once per device (the host-side name of the array is not a device address).
cudaError_t noalloc_scratch(int dev, double **out) {
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess) return e;
    g_noalloc_addr[dev] = static_cast<double *>(p);
  }
  *out = g_noalloc_addr[dev];
  return cudaSuccess;
}
}  // namespace

extern "C" jqcd_status jqcd_dslash_eo_noalloc(jqcd_ctx *ctx, uint64_t gauge_id, int32_t prec,
                                              int32_t out_parity, int32_t dagger, const void *in,
                                              const void *x, void *out, double a, double b,
                                              double *norm2_dev, void *stream) {
  JQCD_RANGE();
  jqcd_status st = check_ctx(ctx);
  if (st) return st;
  GaugeEntry *G = find_gauge(ctx, gauge_id);
  if (!G) return fail(ctx, JQCD_ENOTFOUND, "unknown gauge id");
  if (!in || !out || in == out || (out_parity != 0 && out_parity != 1) || !valid_prec(prec))
    return fail(ctx, JQCD_EINVAL, "dslash_eo_noalloc: bad argument");
  if (G->g.vh > (int64_t)JQCD_NOALLOC_MAX_SITES_PER_PARITY ||
      hop_norm_partials(prec, G->g.vh) > (unsigned)kNoAllocMaxBlocks)
    return fail(ctx, JQCD_EINVAL,
                "dslash_eo_noalloc: %lld sites per parity exceed the fixed scratch limit of %d",
                (long long)G->g.vh, JQCD_NOALLOC_MAX_SITES_PER_PARITY);
  if (ctx->device < 0 || ctx->device >= kNoAllocMaxDevices)
    return fail(ctx, JQCD_EINVAL, "dslash_eo_noalloc: device index %d not supported", ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  double *scratch = nullptr;
  if (norm2_dev) CK(noalloc_scratch(ctx->device, &scratch), "cudaGetSymbolAddress(noalloc scratch)");
  // Every partial the finalize step reads is written by the hop launch of this
  // same call, so nothing in the scratch has to be cleared first.
  HopParams P = G->hop_params(prec, out_parity, in, x, out, a, b, scratch);
  CK(launch_hop(prec, P, dagger != 0, x != nullptr, norm2_dev != nullptr, s), "hop launch");
  if (norm2_dev)
    CK(launch_finalize_sum(scratch, (int)hop_norm_partials(prec, G->g.vh), norm2_dev, s), "norm");
  return JQCD_OK;
}

// ---- fermion action and force ------------------------------------------------
namespace {

void add_info(jqcd_solve_info *acc, const jqcd_solve_info &s) {
  acc->iters += s.iters;
  acc->reliable_updates += s.reliable_updates;
  acc->restarts += s.restarts;
  acc->true_rel_resid = std::max(acc->true_rel_resid, s.true_rel_resid);
  acc->full_rel_resid = std::max(acc->full_rel_resid, s.full_rel_resid);
  acc->gpu_seconds += s.gpu_seconds;
  acc->hop_bytes += s.hop_bytes;
  acc->hop_count += s.hop_count;
}

// X = (D^dag D)^{-1} eta into G->fX and Y = (D^dag)^{-1} eta into G->fY for the
// double-word eta in G->feta, by two solves of D z = c:
// Y = gamma5 D^{-1} gamma5 eta, X = D^{-1} Y.  Then S = Re <eta, X>.
// start1, start2: null (start from 0) or whole-lattice double-word start
// vectors of D x = gamma5 eta and of D x = Y (read before either is
// overwritten; they may be fX or fY).
jqcd_status fermi_solves(jqcd_ctx *ctx, GaugeEntry *G, const jqcd_solve_params &params,
                         jqcd_solve_info *inf, double *action, const float4 *start1 = nullptr,
                         const float4 *start2 = nullptr) {
  cudaStream_t s = ctx->stream;
  const int64_t vh = G->g.vh;
  jqcd_solve_params P = params;
  P.use_x0 = start1 ? 1 : 0;
  std::string msg;
  jqcd_solve_info one;
  CK(launch_gamma5_dw(G->vb, G->feta, vh, s), "gamma5");
  if (start1) CK(launch_dw_copy(G->vsol, start1, 24 * vh, s), "start vector");
  memset(&one, 0, sizeof one);
  jqcd_status st = solve_resident(*G, P, s, &one, &msg);
  add_info(inf, one);
  if (st != JQCD_OK) {
    if (st == JQCD_ECUDA) ctx->poisoned = true;
    return fail(ctx, st, "fermion action, first solve: %s", msg.c_str());
  }
  CK(launch_gamma5_dw(G->fY, G->vsol, vh, s), "gamma5");
  CK(launch_dw_copy(G->vb, G->fY, 24 * vh, s), "copy");
  P.use_x0 = start2 ? 1 : 0;
  if (start2) CK(launch_dw_copy(G->vsol, start2, 24 * vh, s), "start vector");
  memset(&one, 0, sizeof one);
  st = solve_resident(*G, P, s, &one, &msg);
  add_info(inf, one);
  if (st != JQCD_OK) {
    if (st == JQCD_ECUDA) ctx->poisoned = true;
    return fail(ctx, st, "fermion action, second solve: %s", msg.c_str());
  }
  CK(launch_dw_copy(G->fX, G->vsol, 24 * vh, s), "copy");
  const int nb = (int)blas_blocks(24 * vh);
  double *S_dev = G->partials + (G->n_partials() - 1);
  CK(launch_dw_dot_re(G->feta, G->fX, 24 * vh, G->partials, nb, s), "dot");
  CK(launch_finalize_sum(G->partials, nb, S_dev, s), "dot finalize");
  double S = 0.0;
  CK(cudaMemcpyAsync(&S, S_dev, sizeof S, cudaMemcpyDeviceToHost, s), "action D2H");
  CK(cudaStreamSynchronize(s), "action sync");
  if (action) *action = S;
  return JQCD_OK;
}

jqcd_status fermi_common(jqcd_ctx *ctx, uint64_t gauge_id, const jqcd_solve_params *params,
                         const double *eta, double *udsdu, double *action, jqcd_solve_info *info,
                         const char *what) {
  const auto t0 = std::chrono::steady_clock::now();
  jqcd_status st = check_ctx(ctx);
  if (st) return st;
  GaugeEntry *G = find_gauge(ctx, gauge_id);
  if (!G) return fail(ctx, JQCD_ENOTFOUND, "unknown gauge id");
  if (!params || !eta) return fail(ctx, JQCD_EINVAL, "%s: bad argument", what);
  cudaStream_t s = ctx->stream;
  CK(G->ensure_force(), "force workspace alloc");
  CK(cudaMemcpyAsync(G->canon, eta, G->canon_bytes(), cudaMemcpyHostToDevice, s), "eta H2D");
  CK(launch_spinor_pack(G->g, PREC_DW, G->canon, G->vec_even(G->feta), G->vec_odd(G->feta), s), "eta pack");
  jqcd_solve_info inf;
  memset(&inf, 0, sizeof inf);
  st = fermi_solves(ctx, G, *params, &inf, action);
  if (st == JQCD_OK && udsdu) {
    const int64_t nh = 12 * G->g.vh;
    CK(launch_fermi_force(G->g, G->fX, G->fX + nh, G->fY, G->fY + nh, (const float4 *)G->gauge_dw,
                          params->kappa, G->fout, s), "force");
    CK(launch_linkfield_unpack(G->g, G->fout, G->lcanon, s), "force unpack");
    CK(cudaMemcpyAsync(udsdu, G->lcanon, G->link_canon_bytes(), cudaMemcpyDeviceToHost, s), "force D2H");
    CK(cudaStreamSynchronize(s), "force sync");
  }
  inf.status = st;
  inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (info) *info = inf;
  return st;
}

}  // namespace

extern "C" {

jqcd_status jqcd_fermi_action(jqcd_ctx *ctx, uint64_t gauge_id, const jqcd_solve_params *params,
                              const double *eta, double *action, jqcd_solve_info *info) {
  JQCD_RANGE();
  if (!action) return fail(ctx, JQCD_EINVAL, "fermi_action: action is NULL");
  return fermi_common(ctx, gauge_id, params, eta, nullptr, action, info, "fermi_action");
}

jqcd_status jqcd_fermi_force(jqcd_ctx *ctx, uint64_t gauge_id, const jqcd_solve_params *params,
                             const double *eta, double *udsdu, double *action, jqcd_solve_info *info) {
  JQCD_RANGE();
  if (!udsdu) return fail(ctx, JQCD_EINVAL, "fermi_force: udsdu is NULL");
  return fermi_common(ctx, gauge_id, params, eta, udsdu, action, info, "fermi_force");
}

jqcd_status jqcd_fermi_force_xy(jqcd_ctx *ctx, uint64_t gauge_id, double kappa, const double *X,
                                const double *Y, double *udsdu) {
  JQCD_RANGE();
  jqcd_status st = check_ctx(ctx);
  if (st) return st;
  GaugeEntry *G = find_gauge(ctx, gauge_id);
  if (!G) return fail(ctx, JQCD_ENOTFOUND, "unknown gauge id");
  if (!X || !Y || !udsdu) return fail(ctx, JQCD_EINVAL, "fermi_force_xy: bad argument");
  cudaStream_t s = ctx->stream;
  CK(G->ensure_force(), "force workspace alloc");
  const int64_t nh = 12 * G->g.vh;
  CK(cudaMemcpyAsync(G->canon, X, G->canon_bytes(), cudaMemcpyHostToDevice, s), "X H2D");
  CK(launch_spinor_pack(G->g, PREC_DW, G->canon, G->fX, G->fX + nh, s), "X pack");
  CK(cudaMemcpyAsync(G->canon, Y, G->canon_bytes(), cudaMemcpyHostToDevice, s), "Y H2D");
  CK(launch_spinor_pack(G->g, PREC_DW, G->canon, G->fY, G->fY + nh, s), "Y pack");
  CK(launch_fermi_force(G->g, G->fX, G->fX + nh, G->fY, G->fY + nh, (const float4 *)G->gauge_dw, kappa,
                        G->fout, s), "force");
  CK(launch_linkfield_unpack(G->g, G->fout, G->lcanon, s), "force unpack");
  CK(cudaMemcpyAsync(udsdu, G->lcanon, G->link_canon_bytes(), cudaMemcpyDeviceToHost, s), "force D2H");
  CK(cudaStreamSynchronize(s), "force sync");
  return JQCD_OK;
}

jqcd_status jqcd_fermi_force_dev(jqcd_ctx *ctx, uint64_t gauge_id, double kappa, const void *X_even,
                                 const void *X_odd, const void *Y_even, const void *Y_odd, void *out,
                                 void *stream) {
  JQCD_RANGE();
  jqcd_status st = check_ctx(ctx);
  if (st) return st;
  GaugeEntry *G = find_gauge(ctx, gauge_id);
  if (!G) return fail(ctx, JQCD_ENOTFOUND, "unknown gauge id");
  if (!X_even || !X_odd || !Y_even || !Y_odd || !out)
    return fail(ctx, JQCD_EINVAL, "fermi_force_dev: bad argument");
  CK(launch_fermi_force(G->g, (const float4 *)X_even, (const float4 *)X_odd, (const float4 *)Y_even,
                        (const float4 *)Y_odd, (const float4 *)G->gauge_dw, kappa, (float4 *)out,
                        (cudaStream_t)stream), "force");
  return JQCD_OK;
}

jqcd_status jqcd_linkfield_bytes(const jqcd_lattice *lat, size_t *bytes) {
  JQCD_RANGE();
  if (!bytes) return JQCD_EINVAL;
  Geom g;
  if (lattice_geom(nullptr, lat, &g)) return JQCD_EINVAL;
  *bytes = (size_t)72 * 16 * g.vh;
  return JQCD_OK;
}

}  // extern "C"

// ---- multi-shift CG ------------------------------------------------------------
extern "C" {

jqcd_status jqcd_cg_multishift(jqcd_ctx *ctx, uint64_t gauge_id, const jqcd_solve_params *params,
                               int32_t nshift, const double *shifts, const double *rhs, double *const *x,
                               jqcd_solve_info *infos) {
  JQCD_RANGE();
  const auto t0 = std::chrono::steady_clock::now();
  jqcd_status st = check_ctx(ctx);
  if (st) return st;
  GaugeEntry *G = find_gauge(ctx, gauge_id);
  if (!G) return fail(ctx, JQCD_ENOTFOUND, "unknown gauge id");
  if (!params || !shifts || !rhs || !x || nshift < 1 || nshift > kMsMaxShifts)
    return fail(ctx, JQCD_EINVAL, "cg_multishift: bad argument");
  for (int i = 0; i < nshift; ++i)
    if (!x[i]) return fail(ctx, JQCD_EINVAL, "cg_multishift: x[%d] is NULL", i);
  cudaStream_t s = ctx->stream;
  CK(G->ensure_multishift(nshift), "multishift workspace alloc");
  // per-shift solution buffers (one double-word parity each), kept for reuse
  std::vector<float4 *> xs(nshift);
  for (int i = 0; i < nshift; ++i) {
    while ((int)G->ms_x.size() <= i) {
      float4 *p = nullptr;
      CK(G->alloc_t(&p, spinor_parity_bytes(PREC_DW, G->g.vh)), "multishift x alloc");
      G->ms_x.push_back(p);
    }
    xs[i] = G->ms_x[i];
  }
  CK(cudaMemcpyAsync(G->canon, rhs, G->canon_bytes(), cudaMemcpyHostToDevice, s), "rhs H2D");
  CK(launch_spinor_pack(G->g, PREC_DW, G->canon, G->vec_even(G->vrhs), G->vec_odd(G->vrhs), s), "rhs pack");
  std::vector<jqcd_solve_info> inf(nshift);
  std::string msg;
  st = solve_multishift(*G, *params, nshift, shifts, xs.data(), s, inf.data(), &msg);
  if (st == JQCD_ECUDA) ctx->poisoned = true;
  if (st == JQCD_OK || st == JQCD_ENOCONV) {
    float4 *zero_odd = G->vec_odd(G->vt);
    CK(launch_dw_zero(zero_odd, 12 * G->g.vh, s), "zero");
    for (int i = 0; i < nshift; ++i) {
      CK(launch_spinor_unpack(G->g, PREC_DW, xs[i], zero_odd, G->canon, s), "x unpack");
      CK(cudaMemcpyAsync(x[i], G->canon, G->canon_bytes(), cudaMemcpyDeviceToHost, s), "x D2H");
    }
    CK(cudaStreamSynchronize(s), "multishift sync");
  }
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (infos)
    for (int i = 0; i < nshift; ++i) {
      infos[i] = inf[i];
      infos[i].seconds = secs;
    }
  if (st != JQCD_OK) return fail(ctx, st, "cg_multishift: %s", msg.c_str());
  return JQCD_OK;
}

jqcd_status jqcd_cg_multishift_dev(jqcd_ctx *ctx, uint64_t gauge_id, const jqcd_solve_params *params,
                                   int32_t nshift, const double *shifts, const void *rhs_even,
                                   void *const *x_even, jqcd_solve_info *infos, void *stream) {
  JQCD_RANGE();
  const auto t0 = std::chrono::steady_clock::now();
  jqcd_status st = check_ctx(ctx);
  if (st) return st;
  GaugeEntry *G = find_gauge(ctx, gauge_id);
  if (!G) return fail(ctx, JQCD_ENOTFOUND, "unknown gauge id");
  if (!params || !shifts || !rhs_even || !x_even || nshift < 1 || nshift > kMsMaxShifts)
    return fail(ctx, JQCD_EINVAL, "cg_multishift_dev: bad argument");
  std::vector<float4 *> xs(nshift);
  for (int i = 0; i < nshift; ++i) {
    if (!x_even[i]) return fail(ctx, JQCD_EINVAL, "cg_multishift_dev: x_even[%d] is NULL", i);
    xs[i] = (float4 *)x_even[i];
  }
  cudaStream_t s = (cudaStream_t)stream;
  CK(G->ensure_multishift(nshift), "multishift workspace alloc");
  CK(launch_dw_copy(G->vec_even(G->vrhs), (const float4 *)rhs_even, 12 * G->g.vh, s), "copy rhs");
  std::vector<jqcd_solve_info> inf(nshift);
  std::string msg;
  st = solve_multishift(*G, *params, nshift, shifts, xs.data(), s, inf.data(), &msg);
  if (st == JQCD_ECUDA) ctx->poisoned = true;
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (infos)
    for (int i = 0; i < nshift; ++i) {
      infos[i] = inf[i];
      infos[i].seconds = secs;
    }
  if (st != JQCD_OK) return fail(ctx, st, "cg_multishift_dev: %s", msg.c_str());
  return JQCD_OK;
}

}  // extern "C"

// ---- staggered fermions ------------------------------------------------------------
extern "C" {

jqcd_status jqcd_staggered_bytes(const jqcd_lattice *lat, size_t *bytes) {
  JQCD_RANGE();
  if (!bytes) return JQCD_EINVAL;
  Geom g;
  if (lattice_geom(nullptr, lat, &g)) return JQCD_EINVAL;
  *bytes = stag_parity_bytes(g.vh);
  return JQCD_OK;
}

jqcd_status jqcd_staggered_pack(jqcd_ctx *ctx, uint64_t gauge_id, const double *host, void *dev_even,
                                void *dev_odd, void *stream) {
  JQCD_RANGE();
  jqcd_status st = check_ctx(ctx);
  if (st) return st;
  GaugeEntry *G = find_gauge(ctx, gauge_id);
  if (!G) return fail(ctx, JQCD_ENOTFOUND, "unknown gauge id");
  if (!host || !dev_even || !dev_odd) return fail(ctx, JQCD_EINVAL, "staggered_pack: bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  CK(G->ensure_canon(), "staging alloc");
  const size_t bytes = sizeof(double) * 2 * 3 * (size_t)(2 * G->g.vh);
  CK(cudaMemcpyAsync(G->canon, host, bytes, cudaMemcpyHostToDevice, s), "H2D");
  CK(launch_stag_pack(G->g, G->canon, (float4 *)dev_even, (float4 *)dev_odd, s), "pack");
  return JQCD_OK;
}

jqcd_status jqcd_staggered_unpack(jqcd_ctx *ctx, uint64_t gauge_id, const void *dev_even, const void *dev_odd,
                                  double *host, void *stream) {
  JQCD_RANGE();
  jqcd_status st = check_ctx(ctx);
  if (st) return st;
  GaugeEntry *G = find_gauge(ctx, gauge_id);
  if (!G) return fail(ctx, JQCD_ENOTFOUND, "unknown gauge id");
  if (!host || !dev_even || !dev_odd) return fail(ctx, JQCD_EINVAL, "staggered_unpack: bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  CK(G->ensure_canon(), "staging alloc");
  const size_t bytes = sizeof(double) * 2 * 3 * (size_t)(2 * G->g.vh);
  CK(launch_stag_unpack(G->g, (const float4 *)dev_even, (const float4 *)dev_odd, G->canon, s), "unpack");
  CK(cudaMemcpyAsync(host, G->canon, bytes, cudaMemcpyDeviceToHost, s), "D2H");
  CK(cudaStreamSynchronize(s), "unpack sync");
  return JQCD_OK;
}

jqcd_status jqcd_staggered_dslash_eo(jqcd_ctx *ctx, uint64_t gauge_id, int32_t out_parity, int32_t dagger,
                                     const void *in, const void *x, void *out, double a, double b,
                                     double *norm2_dev, void *stream) {
  JQCD_RANGE();
  jqcd_status st = check_ctx(ctx);
  if (st) return st;
  GaugeEntry *G = find_gauge(ctx, gauge_id);
  if (!G) return fail(ctx, JQCD_ENOTFOUND, "unknown gauge id");
  if (!in || !out || in == out || (out_parity != 0 && out_parity != 1))
    return fail(ctx, JQCD_EINVAL, "staggered_dslash_eo: bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  double *parts = nullptr;
  if (norm2_dev) {
    CK(G->ensure_reduce(), "reduce alloc");
    parts = G->partials;
  }
  CK(launch_stag_hop(G->g, out_parity, dagger != 0, (const float4 *)in, (const float4 *)x, (float4 *)out,
                     (const float4 *)G->gauge_dw, a, b, parts, s), "staggered hop");
  if (norm2_dev) CK(launch_finalize_sum(parts, (int)stag_blocks(G->g.vh), norm2_dev, s), "norm");
  return JQCD_OK;
}

jqcd_status jqcd_staggered_apply(jqcd_ctx *ctx, uint64_t gauge_id, double mass, int32_t dagger,
                                 const void *in_even, const void *in_odd, void *out_even, void *out_odd,
                                 void *stream) {
  JQCD_RANGE();
  jqcd_status st = check_ctx(ctx);
  if (st) return st;
  GaugeEntry *G = find_gauge(ctx, gauge_id);
  if (!G) return fail(ctx, JQCD_ENOTFOUND, "unknown gauge id");
  if (!in_even || !in_odd || !out_even || !out_odd || in_even == out_even || in_odd == out_odd)
    return fail(ctx, JQCD_EINVAL, "staggered_apply: bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  const float4 *U = (const float4 *)G->gauge_dw;
  CK(launch_stag_hop(G->g, 0, dagger != 0, (const float4 *)in_odd, (const float4 *)in_even, (float4 *)out_even,
                     U, mass, 1.0, nullptr, s), "staggered hop");
  CK(launch_stag_hop(G->g, 1, dagger != 0, (const float4 *)in_even, (const float4 *)in_odd, (float4 *)out_odd,
                     U, mass, 1.0, nullptr, s), "staggered hop");
  return JQCD_OK;
}

jqcd_status jqcd_staggered_solve(jqcd_ctx *ctx, uint64_t gauge_id, const jqcd_solve_params *params, double mass,
                                 const double *b, double *x, jqcd_solve_info *info) {
  JQCD_RANGE();
  const auto t0 = std::chrono::steady_clock::now();
  jqcd_status st = check_ctx(ctx);
  if (st) return st;
  GaugeEntry *G = find_gauge(ctx, gauge_id);
  if (!G) return fail(ctx, JQCD_ENOTFOUND, "unknown gauge id");
  if (!params || !b || !x) return fail(ctx, JQCD_EINVAL, "staggered_solve: bad argument");
  cudaStream_t s = ctx->stream;
  CK(G->ensure_staggered(), "staggered workspace alloc");
  const int64_t n = 3 * G->g.vh;
  const size_t bytes = sizeof(double) * 2 * 3 * (size_t)(2 * G->g.vh);
  CK(cudaMemcpyAsync(G->canon, b, bytes, cudaMemcpyHostToDevice, s), "b H2D");
  CK(launch_stag_pack(G->g, G->canon, G->sb, G->sb + n, s), "b pack");
  jqcd_solve_info inf;
  memset(&inf, 0, sizeof inf);
  std::string msg;
  st = solve_staggered(*G, mass, *params, s, &inf, &msg);
  if (st == JQCD_ECUDA) ctx->poisoned = true;
  if (st == JQCD_OK || st == JQCD_ENOCONV) {
    CK(launch_stag_unpack(G->g, G->sx, G->sx + n, G->canon, s), "x unpack");
    CK(cudaMemcpyAsync(x, G->canon, bytes, cudaMemcpyDeviceToHost, s), "x D2H");
    CK(cudaStreamSynchronize(s), "solve sync");
  }
  inf.status = st;
  inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (info) *info = inf;
  if (st != JQCD_OK) return fail(ctx, st, "staggered_solve: %s", msg.c_str());
  return JQCD_OK;
}

jqcd_status jqcd_staggered_solve_dev(jqcd_ctx *ctx, uint64_t gauge_id, const jqcd_solve_params *params,
                                     double mass, const void *b_even, const void *b_odd, void *x_even, void *x_odd,
                                     jqcd_solve_info *info, void *stream) {
  JQCD_RANGE();
  const auto t0 = std::chrono::steady_clock::now();
  jqcd_status st = check_ctx(ctx);
  if (st) return st;
  GaugeEntry *G = find_gauge(ctx, gauge_id);
  if (!G) return fail(ctx, JQCD_ENOTFOUND, "unknown gauge id");
  if (!params || !b_even || !b_odd || !x_even || !x_odd)
    return fail(ctx, JQCD_EINVAL, "staggered_solve_dev: bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  CK(G->ensure_staggered(), "staggered workspace alloc");
  const int64_t n = 3 * G->g.vh;
  CK(launch_dw_copy(G->sb, (const float4 *)b_even, n, s), "copy b");
  CK(launch_dw_copy(G->sb + n, (const float4 *)b_odd, n, s), "copy b");
  jqcd_solve_info inf;
  memset(&inf, 0, sizeof inf);
  std::string msg;
  st = solve_staggered(*G, mass, *params, s, &inf, &msg);
  if (st == JQCD_ECUDA) ctx->poisoned = true;
  if (st == JQCD_OK || st == JQCD_ENOCONV) {
    CK(launch_dw_copy((float4 *)x_even, G->sx, n, s), "copy x");
    CK(launch_dw_copy((float4 *)x_odd, G->sx + n, n, s), "copy x");
    CK(cudaStreamSynchronize(s), "solve sync");
  }
  inf.status = st;
  inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (info) *info = inf;
  if (st != JQCD_OK) return fail(ctx, st, "staggered_solve_dev: %s", msg.c_str());
  return JQCD_OK;
}

}  // extern "C"

// ---- hybrid Monte Carlo ------------------------------------------------------------
extern "C" {

jqcd_status jqcd_gauge_plaquette(jqcd_ctx *ctx, uint64_t gauge_id, double *plaquette) {
  JQCD_RANGE();
  jqcd_status st = check_ctx(ctx);
  if (st) return st;
  GaugeEntry *G = find_gauge(ctx, gauge_id);
  if (!G) return fail(ctx, JQCD_ENOTFOUND, "unknown gauge id");
  if (!plaquette) return fail(ctx, JQCD_EINVAL, "gauge_plaquette: plaquette is NULL");
  CK(G->ensure_hmc(), "hmc workspace alloc");
  double sum = 0.0;
  CK(hmc_plaquette_sum(*G, &sum, ctx->stream), "plaquette");
  *plaquette = sum / (18.0 * (double)(2 * G->g.vh));
  return JQCD_OK;
}

jqcd_status jqcd_gauge_download(jqcd_ctx *ctx, uint64_t gauge_id, double *links) {
  JQCD_RANGE();
  jqcd_status st = check_ctx(ctx);
  if (st) return st;
  GaugeEntry *G = find_gauge(ctx, gauge_id);
  if (!G) return fail(ctx, JQCD_ENOTFOUND, "unknown gauge id");
  if (!links) return fail(ctx, JQCD_EINVAL, "gauge_download: links is NULL");
  cudaStream_t s = ctx->stream;
  CK(G->ensure_force(), "staging alloc");  // lcanon: 36 V complex doubles
  CK(launch_links_unpack(*G, G->lcanon, s), "links unpack");
  CK(cudaMemcpyAsync(links, G->lcanon, G->link_canon_bytes(), cudaMemcpyDeviceToHost, s), "links D2H");
  CK(cudaStreamSynchronize(s), "download sync");
  return JQCD_OK;
}

jqcd_status jqcd_hmc_trajectory(jqcd_ctx *ctx, uint64_t gauge_id, const jqcd_hmc_params *hp, const double *normals,
                                const double *xi, double u, jqcd_hmc_info *info) {
  JQCD_RANGE();
  const auto t0 = std::chrono::steady_clock::now();
  jqcd_status st = check_ctx(ctx);
  if (st) return st;
  GaugeEntry *G = find_gauge(ctx, gauge_id);
  if (!G) return fail(ctx, JQCD_ENOTFOUND, "unknown gauge id");
  if (!hp || !normals || (hp->fermions && !xi)) return fail(ctx, JQCD_EINVAL, "hmc_trajectory: bad argument");
  if (hp->n_md < 1 || !(hp->tau > 0.0) || !std::isfinite(hp->beta) || !(hp->beta >= 0.0))
    return fail(ctx, JQCD_EINVAL, "hmc_trajectory: n_md >= 1, tau > 0, beta >= 0");
  cudaStream_t s = ctx->stream;
  const int64_t V = 2 * G->g.vh, nh = 12 * G->g.vh;
  CK(G->ensure_hmc(), "hmc workspace alloc");
  if (hp->fermions) CK(G->ensure_force(), "force workspace alloc");
  if (hp->fermions) CK(G->ensure_hmc_history(), "solve history alloc");
  const size_t lf = (size_t)72 * 16 * G->g.vh;
  jqcd_solve_params sp;
  memset(&sp, 0, sizeof sp);
  sp.kappa = hp->kappa;
  sp.tol = hp->tol;
  sp.maxiter = hp->maxiter > 0 ? hp->maxiter : 20000;
  sp.eo = 1;
  sp.mode = hp->mode;
  jqcd_hmc_info out;
  memset(&out, 0, sizeof out);
  jqcd_solve_info inf;
  memset(&inf, 0, sizeof inf);
  // save the links, refresh the momenta
  CK(cudaMemcpyAsync(G->hUbak, G->gauge_f64, lf, cudaMemcpyDeviceToDevice, s), "links backup");
  CK(cudaMemcpyAsync(G->hNormals, normals, sizeof(double) * 32 * (size_t)V, cudaMemcpyHostToDevice, s),
     "normals H2D");
  CK(hmc_momenta_set(*G, G->hNormals, s), "momenta");
  double S_f = 0.0;
  if (hp->fermions) {
    // eta = D^dag xi into feta (xi staged in fY); S_f,old = |xi|^2
    CK(cudaMemcpyAsync(G->canon, xi, G->canon_bytes(), cudaMemcpyHostToDevice, s), "xi H2D");
    CK(launch_spinor_pack(G->g, PREC_DW, G->canon, G->fY, G->fY + nh, s), "xi pack");
    HopParams Pe = G->hop_params(PREC_DW, 0, G->fY + nh, G->fY, G->feta, 1.0, -hp->kappa, nullptr);
    HopParams Po = G->hop_params(PREC_DW, 1, G->fY, G->fY + nh, G->feta + nh, 1.0, -hp->kappa, nullptr);
    CK(launch_hop(PREC_DW, Pe, true, true, false, s), "heatbath hop");
    CK(launch_hop(PREC_DW, Po, true, true, false, s), "heatbath hop");
    const int nb = (int)blas_blocks(2 * nh);
    double *dev = G->partials + (G->n_partials() - 1);
    CK(launch_dw_norm2(G->fY, 2 * nh, G->partials, s), "norm");
    CK(launch_finalize_sum(G->partials, nb, dev, s), "norm");
    CK(cudaMemcpyAsync(&S_f, dev, sizeof(double), cudaMemcpyDeviceToHost, s), "norm D2H");
    CK(cudaStreamSynchronize(s), "sync");
  }
  double K = 0.0, plaq = 0.0;
  CK(hmc_kinetic(*G, &K, s), "kinetic");
  CK(hmc_plaquette_sum(*G, &plaq, s), "plaquette");
  out.H_old = K - hp->beta / 3.0 * plaq + S_f;
  // Start vectors of the fermion solves (chronological): the solutions X(t),
  // Y(t) at the force times t_k = (k + 1/2) dt are smooth in t, so step k
  // starts from the linear extrapolation 2 x_{k-1} - x_{k-2} (error O(dt^2)),
  // step 1 from x_0, step 0's first solve from gamma5 xi (exact at t = 0:
  // eta = D^dag xi) and its second from 0.  hS1 holds gamma5 of Y's start.
  const int64_t nfull = 24 * G->g.vh;
  int nhist = 0;  // force-time solutions available (fX, fY newest; hXp, hYp before)
  auto starts = [&](double ahead, const float4 **s1, const float4 **s2) -> cudaError_t {
    // ahead: distance to the next solve time in units of dt
    cudaError_t e = cudaSuccess;
    if (nhist >= 2) {
      e = launch_dw_lincomb(G->hS1, G->fY, G->hYp, 1.0 + ahead, -ahead, nfull, s);
      if (!e) e = launch_dw_lincomb(G->hS2, G->fX, G->hXp, 1.0 + ahead, -ahead, nfull, s);
      *s2 = G->hS2;
    } else {
      e = launch_dw_copy(G->hS1, G->fY, nfull, s);  // Y_0, or xi before the first solves
      *s2 = nhist == 1 ? G->hS2 : nullptr;
      if (!e && nhist == 1) e = launch_dw_copy(G->hS2, G->fX, nfull, s);
    }
    if (!e) e = launch_gamma5_dw(G->hS1, G->hS1, G->g.vh, s);
    *s1 = G->hS1;
    // the newest solutions become the history before the solves replace them
    if (!e && nhist >= 1) e = launch_dw_copy(G->hYp, G->fY, nfull, s);
    if (!e && nhist >= 1) e = launch_dw_copy(G->hXp, G->fX, nfull, s);
    return e;
  };
  // leapfrog
  const double dt = hp->tau / hp->n_md;
  for (int step = 0; step < hp->n_md; ++step) {
    CK(hmc_links_update(*G, 0.5 * dt, s), "link update");
    CK(hmc_gauge_force(*G, hp->beta, s), "gauge force");
    if (hp->fermions) {
      jqcd_solve_info fi;
      memset(&fi, 0, sizeof fi);
      const float4 *s1 = nullptr, *s2 = nullptr;
      CK(starts(1.0, &s1, &s2), "start vectors");
      st = fermi_solves(ctx, G, sp, &fi, nullptr, s1, s2);
      ++nhist;
      add_info(&inf, fi);
      if (st != JQCD_OK) break;
      CK(launch_fermi_force(G->g, G->fX, G->fX + nh, G->fY, G->fY + nh, (const float4 *)G->gauge_dw, hp->kappa,
                            G->fout, s), "fermion force");
    }
    CK(hmc_momenta_update(*G, hp->fermions ? G->fout : nullptr, 0.5 * dt, s), "momenta update");
    CK(hmc_links_update(*G, 0.5 * dt, s), "link update");
  }
  if (st == JQCD_OK) {
    S_f = 0.0;
    if (hp->fermions) {
      jqcd_solve_info fi;
      memset(&fi, 0, sizeof fi);
      const float4 *s1 = nullptr, *s2 = nullptr;
      CK(starts(0.5, &s1, &s2), "start vectors");  // t = tau, half a step after the last force
      st = fermi_solves(ctx, G, sp, &fi, &S_f, s1, s2);
      add_info(&inf, fi);
    }
  }
  if (st == JQCD_OK) {
    CK(hmc_kinetic(*G, &K, s), "kinetic");
    CK(hmc_plaquette_sum(*G, &plaq, s), "plaquette");
    out.H_new = K - hp->beta / 3.0 * plaq + S_f;
    out.dH = out.H_new - out.H_old;
    out.accepted = std::isfinite(out.dH) && u <= std::exp(-out.dH);
  }
  if (!out.accepted) {  // restore the links (also after a failed solve)
    CK(cudaMemcpyAsync(G->gauge_f64, G->hUbak, lf, cudaMemcpyDeviceToDevice, s), "links restore");
    CK(launch_hmc_links_refresh(*G, s), "links refresh");
  }
  CK(hmc_plaquette_sum(*G, &plaq, s), "plaquette");
  out.plaquette = plaq / (18.0 * (double)V);
  out.cg_iters = inf.iters;
  out.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (info) *info = out;
  return st;  // fermi_solves has set the error text on failure
}

}  // extern "C"
