// Host side of the batched mixed-precision CG engine.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>

#include "batch_engine.h"
#include "jqcd.h"

namespace jqcd {

namespace {
constexpr int kGraphIters = 4;  // CG iterations per captured graph

float2 split(double v) {
  const float h = (float)v;
  return make_float2(h, (float)(v - (double)h));
}
}  // namespace

// ---- slot buffers -------------------------------------------------------------
SlotBuffers::~SlotBuffers() { release(); }

void SlotBuffers::release() {
  for (void *p : allocs) cudaFree(p);
  allocs.clear();
  vh_cap = 0;
  hp = -1;
  bytes = 0;
}

int64_t SlotBuffers::n_part(int64_t vh) { return vh / 32 + 4096; }

size_t SlotBuffers::footprint(int64_t vh, int hp) {
  const size_t lp = spinor_parity_bytes(hp, vh), f32 = spinor_parity_bytes(PREC_F32, vh),
               dw = spinor_parity_bytes(PREC_DW, vh);
  return 4 * lp + 2 * f32 + 9 * dw + sizeof(double) * (size_t)n_part(vh);
}

cudaError_t SlotBuffers::ensure(int64_t vh, int hp_) {
  if (vh <= vh_cap && hp_ == hp) return cudaSuccess;
  release();
  const size_t lp = spinor_parity_bytes(hp_, vh), f32 = spinor_parity_bytes(PREC_F32, vh),
               dw = spinor_parity_bytes(PREC_DW, vh);
  struct Want { void **dst; size_t n; };
  Want wants[] = {{&p, lp}, {&Ap, lp}, {&w, lp}, {&t, lp},
                  {(void **)&xs, f32}, {(void **)&rs, f32},
                  {(void **)&b, 2 * dw}, {(void **)&x, 2 * dw}, {(void **)&r, dw},
                  {(void **)&rhs, dw}, {(void **)&wdw, dw}, {(void **)&Adw, dw},
                  {(void **)&tdw, dw}, {(void **)&part, sizeof(double) * (size_t)n_part(vh)}};
  for (const Want &wt : wants) {
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, wt.n);
    if (e != cudaSuccess) {
      release();
      return e;
    }
    allocs.push_back(q);
    *wt.dst = q;
  }
  vh_cap = vh;
  hp = hp_;
  bytes = footprint(vh, hp_);
  return cudaSuccess;
}

// ---- engine -----------------------------------------------------------------------
// True for page-locked (pinned or registered) host memory.  Only such buffers
// take the copy stream: a pageable buffer is staged by the driver, which
// blocks the calling thread and synchronises with the copy stream's queue
// (measured: serving latencies grew 20x), so it keeps the compute stream.
static bool page_locked(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeHost;
}

BatchEngine::BatchEngine(int hp, int max_slots, cudaStream_t s, int sm_count)
    : hp_(hp), sm_count_(sm_count > 0 ? sm_count : 152), s_(s), slots_(max_slots),
      h_slots_(max_slots) {
  memset(h_slots_.data(), 0, sizeof(SlotDev) * h_slots_.size());
  grid_ = sm_count_ * 4;
  lp_grid_ = sm_count_ * 2;
  t0_ = now();
}

BatchArgs BatchEngine::args() const {
  BatchArgs A;
  A.slots = d_slots_;
  A.S = d_S_;
  A.groups = d_groups_;
  A.tiles = d_tiles_;
  A.ntiles = d_ntiles_;
  A.lp_tiles = d_lp_tiles_;
  A.n_lp_tiles = d_n_lp_tiles_;
  A.lp2_tiles = d_lp_tiles_ ? d_lp_tiles_ + max_lp_tiles_ : nullptr;      // second third of the buffer
  A.n_lp2_tiles = d_n_lp2_tiles_;
  A.lp1_tiles = d_lp_tiles_ ? d_lp_tiles_ + 2 * max_lp_tiles_ : nullptr;  // last third
  A.n_lp1_tiles = d_n_lp1_tiles_;
  A.any_update = d_any_update_;
  A.nslots = (int)slots_.size();
  return A;
}

BatchEngine::~BatchEngine() {
  cudaStreamSynchronize(s_);
  if (cs_) cudaStreamSynchronize(cs_);
  drop_graphs();
  for (void *p : {(void *)d_slots_, (void *)d_S_, (void *)d_groups_, (void *)d_tiles_,
                  (void *)d_ntiles_, (void *)d_lp_tiles_, (void *)d_n_lp_tiles_,
                  (void *)d_n_lp2_tiles_, (void *)d_n_lp1_tiles_, (void *)d_any_update_})
    if (p) cudaFree(p);
  for (auto *v : {&ev_in_, &ev_out_, &ev_done_})
    for (cudaEvent_t ev : *v) cudaEventDestroy(ev);
  if (cs_) cudaStreamDestroy(cs_);
  if (h_S_) cudaFreeHost(h_S_);
}

double BatchEngine::now() const {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count() - t0_;
}

cudaError_t BatchEngine::init() {
  const int n = (int)slots_.size();
  cudaError_t e = batch_configure();
  // persistent low-precision grid: one full wave of resident blocks (the
  // autotuner of jqcd_cg_solve_batch may choose another; the server keeps it)
  if (!e) lp_grid_ = sm_count_ * batch_lp_blocks_per_sm(hp_);
  if (!e) e = cudaMalloc(&d_slots_, sizeof(SlotDev) * n);
  if (!e) e = cudaMalloc(&d_S_, sizeof(SolverScalars) * n);
  if (!e) e = cudaMallocHost(&h_S_, sizeof(SolverScalars) * n);
  if (!e) e = cudaMalloc(&d_groups_, sizeof(GroupDev) * n);
  if (!e) e = cudaMalloc(&d_ntiles_, sizeof(int));
  if (!e) e = cudaMalloc(&d_n_lp_tiles_, sizeof(int));
  if (!e) e = cudaMemsetAsync(d_n_lp_tiles_, 0, sizeof(int), s_);
  if (!e) e = cudaMalloc(&d_n_lp2_tiles_, sizeof(int));
  if (!e) e = cudaMemsetAsync(d_n_lp2_tiles_, 0, sizeof(int), s_);
  if (!e) e = cudaMalloc(&d_n_lp1_tiles_, sizeof(int));
  if (!e) e = cudaMemsetAsync(d_n_lp1_tiles_, 0, sizeof(int), s_);
  if (!e) e = cudaMalloc(&d_any_update_, sizeof(int));
  if (!e) e = cudaMemsetAsync(d_S_, 0, sizeof(SolverScalars) * n, s_);
  if (!e) e = cudaMemsetAsync(d_ntiles_, 0, sizeof(int), s_);
  if (!e) e = cudaMemsetAsync(d_any_update_, 0, sizeof(int), s_);
  if (!e) memset(h_S_, 0, sizeof(SolverScalars) * n);
  if (!e) e = cudaStreamCreateWithFlags(&cs_, cudaStreamNonBlocking);
  for (auto *v : {&ev_in_, &ev_out_, &ev_done_}) {
    v->assign(n, nullptr);
    for (int i = 0; i < n && !e; ++i) e = cudaEventCreateWithFlags(&(*v)[i], cudaEventDisableTiming);
  }
  max_groups_ = n;
  return e;
}

int BatchEngine::free_slot() const {
  for (size_t i = 0; i < slots_.size(); ++i)
    if (slots_[i].state == 0) return (int)i;
  return -1;
}

int BatchEngine::pick_slot(int64_t vh, int64_t *extra) const {
  const size_t need = SlotBuffers::footprint(vh, hp_);
  int best = -1, empty = -1, largest = -1;
  for (size_t i = 0; i < slots_.size(); ++i) {
    const SlotHost &S = slots_[i];
    if (S.state != 0) continue;
    if (S.buf.vh_cap >= vh && S.buf.hp == hp_) {
      if (best < 0 || S.buf.bytes < slots_[best].buf.bytes) best = (int)i;
    } else if (S.buf.vh_cap == 0) {
      if (empty < 0) empty = (int)i;
    } else if (largest < 0 || S.buf.bytes > slots_[largest].buf.bytes) {
      largest = (int)i;
    }
  }
  if (best >= 0) { *extra = 0; return best; }
  if (empty >= 0) { *extra = (int64_t)need; return empty; }
  if (largest >= 0) { *extra = (int64_t)need - (int64_t)slots_[largest].buf.bytes; return largest; }
  *extra = 0;
  return -1;
}

void BatchEngine::release_idle(int keep) {
  for (size_t i = 0; i < slots_.size(); ++i)
    if ((int)i != keep && slots_[i].state == 0 && slots_[i].buf.vh_cap > 0) slots_[i].buf.release();
}

size_t BatchEngine::allocated_bytes() const {
  size_t b = 0;
  for (const SlotHost &S : slots_) b += S.buf.bytes;
  return b;
}

int BatchEngine::running() const {
  int r = 0;
  for (const SlotHost &s : slots_) r += s.state == 1;
  return r;
}

cudaError_t BatchEngine::admit(int slot, GaugeEntry *G, const jqcd_solve_params &P,
                               const double *b_host) {
  if (slot < 0 || slot >= (int)slots_.size() || slots_[slot].state != 0) return cudaErrorInvalidValue;
  SlotHost &H = slots_[slot];
  const Geom &g = G->g;
  const int64_t vh = g.vh;
  cudaError_t e = H.buf.ensure(vh, hp_);
  if (e) return e;
  SlotBuffers &B = H.buf;
  SolverScalars *S = d_S_ + slot;
  const double k = P.kappa;
  const double tol2 = P.tol * P.tol;
  const double delta = P.delta > 0.0 ? P.delta : 0.01;
  float4 *b_e = B.b, *b_o = B.b + 12 * vh;
  const int nb24 = (int)blas_blocks(24 * vh), nb12 = (int)blas_blocks(12 * vh);
#define CKE(call) do { e = (call); if (e) return e; } while (0)
  CKE(cudaMemsetAsync(S, 0, sizeof(SolverScalars), s_));
  // canonical source staged in the slot's x buffer (same 384 B per site; x is
  // zeroed below), copied on the copy stream: after any earlier copy of this
  // slot there, and before the pack on the compute stream
  double *stage = reinterpret_cast<double *>(B.x);
  const size_t bytes = sizeof(double) * 24 * (size_t)(2 * vh);
  if (page_locked(b_host)) {
    CKE(cudaMemcpyAsync(stage, b_host, bytes, cudaMemcpyHostToDevice, cs_));
    CKE(cudaEventRecord(ev_in_[slot], cs_));
    CKE(cudaStreamWaitEvent(s_, ev_in_[slot], 0));
  } else {
    CKE(cudaMemcpyAsync(stage, b_host, bytes, cudaMemcpyHostToDevice, s_));
  }
  CKE(launch_spinor_pack(g, PREC_DW, stage, b_e, b_o, s_));
  CKE(launch_dw_norm2(B.b, 24 * vh, B.part, s_));
  CKE(launch_finalize_sum(B.part, nb24, &S->b2, s_));
  // bhat_e = b_e + kappa H_eo b_o; rhs = Mhat^dag bhat_e
  CKE(launch_hop(PREC_DW, G->hop_params(PREC_DW, 0, b_o, b_e, B.wdw, 1.0, k, nullptr), false, true, false, s_));
  CKE(launch_hop(PREC_DW, G->hop_params(PREC_DW, 1, B.wdw, nullptr, B.tdw, 0.0, 1.0, nullptr), true, false, false, s_));
  CKE(launch_hop(PREC_DW, G->hop_params(PREC_DW, 0, B.tdw, B.wdw, B.rhs, 1.0, -k * k, nullptr), true, true, false, s_));
  CKE(launch_dw_norm2(B.rhs, 12 * vh, B.part, s_));
  CKE(launch_finalize_sum(B.part, nb12, &S->rhs2, s_));
  // x = 0, r = rhs, inner vectors
  CKE(launch_dw_zero(B.x, 24 * vh, s_));
  CKE(launch_dw_copy(B.r, B.rhs, 12 * vh, s_));
  CKE(launch_dw_norm2(B.r, 12 * vh, B.part, s_));
  CKE(launch_cg_start(B.part, nb12, S, tol2, P.maxiter, delta * delta, s_));
  CKE(cudaMemsetAsync(B.xs, 0, spinor_parity_bytes(PREC_F32, vh), s_));
  CKE(launch_dw_to_f32(B.rs, B.r, vh, s_));
  CKE(launch_mixed_copy(hp_, B.p, B.rs, vh, s_));
#undef CKE
  SlotDev &D = h_slots_[slot];
  memset(&D, 0, sizeof D);
  D.g = g;
  D.gauge_f32 = (const float4 *)G->gauge_f32;
  D.gauge_dw = (const float4 *)G->gauge_dw;
  D.kappa = k;
  D.k2 = (float)(-k * k);
  D.k2_dw = split(-k * k);
  D.kap_dw = split(k);
  D.p = B.p; D.Ap = B.Ap; D.w = B.w; D.t = B.t;
  D.xs = B.xs; D.rs = B.rs;
  D.b = B.b; D.x = B.x; D.r = B.r; D.rhs = B.rhs; D.wdw = B.wdw; D.Adw = B.Adw; D.tdw = B.tdw;
  D.part = B.part;
  D.active = 1;
  H.state = 1;
  H.G = G;
  H.P = P;
  H.t_admit = now();
  dirty_ = true;
  return cudaSuccess;
}

cudaError_t BatchEngine::rebuild() {
  // groups: running slots on the same gauge field, at most kBatchMaxRhs each
  std::vector<GroupDev> groups;
  std::map<const void *, int> open;  // gauge -> index of its group being filled
  for (size_t i = 0; i < slots_.size(); ++i) {
    SlotDev &D = h_slots_[i];
    if (slots_[i].state != 1) {
      D.active = 0;
      continue;
    }
    D.nblocks = (int)((D.g.vh + tile_sites_ - 1) / tile_sites_);
    D.nblk_lp = (int)((D.g.vh + kLpThreads - 1) / kLpThreads);
    auto it = open.find(D.gauge_f32);
    if (it == open.end() || groups[it->second].nslots == kBatchMaxRhs) {
      GroupDev Gd;
      memset(&Gd, 0, sizeof Gd);
      Gd.g = D.g;
      Gd.gauge_f32 = D.gauge_f32;
      Gd.gauge_dw = D.gauge_dw;
      groups.push_back(Gd);
      open[D.gauge_f32] = (int)groups.size() - 1;
      it = open.find(D.gauge_f32);
    }
    GroupDev &Gd = groups[it->second];
    Gd.slot[Gd.nslots++] = (int)i;
  }
  std::vector<int2> tiles, lp_tiles, lp2_tiles, lp1_tiles;
  for (size_t gi = 0; gi < groups.size(); ++gi) {
    const int nbk = (int)((groups[gi].g.vh + tile_sites_ - 1) / tile_sites_);
    for (int j = 0; j < nbk; ++j) tiles.push_back(make_int2((int)gi, j));
    groups[gi].tpb = 1;
    const int nlp = (int)((groups[gi].g.vh + kLpThreads - 1) / kLpThreads);
    const int ns = groups[gi].nslots;
    for (int j = 0; j < nlp; ++j)
      for (int r = 0; r < ns; ++r) {
        lp_tiles.push_back(make_int2((int)gi * 16 + r, j));
        if (r % 2 == 0 && r + 1 < ns) lp2_tiles.push_back(make_int2((int)gi * 16 + r, j));
        if (r % 2 == 0 && r + 1 == ns) lp1_tiles.push_back(make_int2(groups[gi].slot[r], j));
      }
  }
  if ((int64_t)lp_tiles.size() > max_lp_tiles_) {
    if (d_lp_tiles_) cudaFree(d_lp_tiles_);
    d_lp_tiles_ = nullptr;
    const int64_t cap = std::max<int64_t>((int64_t)lp_tiles.size() * 2, 1024);
    // per-slot items in the first third, pair items in the second, single items in the last
    cudaError_t e0 = cudaMalloc(&d_lp_tiles_, 3 * sizeof(int2) * cap);
    if (e0) { max_lp_tiles_ = 0; return e0; }
    max_lp_tiles_ = cap;
    drop_graphs();  // pointer changed
  }
  cudaError_t e = cudaSuccess;
  if ((int64_t)tiles.size() > max_tiles_) {
    if (d_tiles_) cudaFree(d_tiles_);
    d_tiles_ = nullptr;
    const int64_t cap = std::max<int64_t>((int64_t)tiles.size() * 2, 1024);
    e = cudaMalloc(&d_tiles_, sizeof(int2) * cap);
    if (e) { max_tiles_ = 0; return e; }
    max_tiles_ = cap;
    drop_graphs();  // pointer changed
  }
  const int ntiles = (int)tiles.size();
  n_tiles_ = ntiles;
  n_lp_items_ = (int64_t)lp_tiles.size();
  e = cudaMemcpyAsync(d_slots_, h_slots_.data(), sizeof(SlotDev) * h_slots_.size(),
                      cudaMemcpyHostToDevice, s_);
  if (!e && !groups.empty())
    e = cudaMemcpyAsync(d_groups_, groups.data(), sizeof(GroupDev) * groups.size(),
                        cudaMemcpyHostToDevice, s_);
  if (!e && ntiles)
    e = cudaMemcpyAsync(d_tiles_, tiles.data(), sizeof(int2) * tiles.size(), cudaMemcpyHostToDevice, s_);
  if (!e) e = cudaMemcpyAsync(d_ntiles_, &ntiles, sizeof(int), cudaMemcpyHostToDevice, s_);
  const int n_lp = (int)lp_tiles.size();
  if (!e && n_lp)
    e = cudaMemcpyAsync(d_lp_tiles_, lp_tiles.data(), sizeof(int2) * lp_tiles.size(),
                        cudaMemcpyHostToDevice, s_);
  if (!e) e = cudaMemcpyAsync(d_n_lp_tiles_, &n_lp, sizeof(int), cudaMemcpyHostToDevice, s_);
  const int n_lp2 = (int)lp2_tiles.size();
  if (!e && n_lp2)
    e = cudaMemcpyAsync(d_lp_tiles_ + max_lp_tiles_, lp2_tiles.data(), sizeof(int2) * lp2_tiles.size(),
                        cudaMemcpyHostToDevice, s_);
  if (!e) e = cudaMemcpyAsync(d_n_lp2_tiles_, &n_lp2, sizeof(int), cudaMemcpyHostToDevice, s_);
  const int n_lp1 = (int)lp1_tiles.size();
  if (!e && n_lp1)
    e = cudaMemcpyAsync(d_lp_tiles_ + 2 * max_lp_tiles_, lp1_tiles.data(), sizeof(int2) * lp1_tiles.size(),
                        cudaMemcpyHostToDevice, s_);
  if (!e) e = cudaMemcpyAsync(d_n_lp1_tiles_, &n_lp1, sizeof(int), cudaMemcpyHostToDevice, s_);
  n_lp2_items_ = n_lp2;
  n_lp1_items_ = n_lp1;
  // pageable sources: make the copies complete before the vectors go away
  if (!e) e = cudaStreamSynchronize(s_);
  if (!e) dirty_ = false;
  return e;
}

// Persistent grids no larger than the work: the tile and low-precision
// grids are capped at the next power of two of their item counts (a few
// solves on an 8^4 lattice have tens of items, not 2-4 x SMs), so each launch
// asks the block scheduler for no more blocks than it can use.  One captured
// graph is kept per (tile size, grid, low-precision grid).
static int pow2_at_least(int64_t n) {
  int p = 1;
  while (p < n && p < (1 << 30)) p <<= 1;
  return p;
}

void BatchEngine::drop_graphs() {
  for (auto &kv : graphs_) cudaGraphExecDestroy(kv.second.first);
  graphs_.clear();
  graph_ = nullptr;
}

LpGrids BatchEngine::lp_grids(int lp_grid) const {
  auto cap = [lp_grid](int64_t n) { return std::min<int>(lp_grid, pow2_at_least(std::max<int64_t>(n, 1))); };
  return LpGrids{cap(n_lp_items_), cap(n_lp2_items_), cap(n_lp1_items_)};
}

cudaError_t BatchEngine::ensure_graph() {
  const int grid = std::min<int>(grid_, pow2_at_least(std::max<int64_t>(n_tiles_, 1)));
  const LpGrids lp = lp_grids(lp_grid_);
  const std::tuple<int, int, int, int, int> key{tile_sites_, grid, lp.all, lp.pairs, lp.singles};
  auto it = graphs_.find(key);
  if (it != graphs_.end()) {
    graph_ = it->second.first;
    graph_kernels_ = it->second.second;
    return cudaSuccess;
  }
  const BatchArgs A = args();
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(s_, cudaStreamCaptureModeThreadLocal);
  if (e) return e;
  const uint64_t before = jqcd_kernel_launches();
  for (int k = 0; k < kGraphIters && !e; ++k)
    e = launch_batch_iteration(A, hp_, tile_sites_, grid, lp, s_);
  const int64_t kernels = (int64_t)(jqcd_kernel_launches() - before);
  note_launch(-kernels);  // recorded, not run: counted at each replay instead
  cudaError_t e2 = cudaStreamEndCapture(s_, &g);
  if (e) { if (g) cudaGraphDestroy(g); return e; }
  if (e2) return e2;
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, g, 0);
  cudaGraphDestroy(g);
  if (e) return e;
  graphs_[key] = {exec, kernels};
  graph_ = exec;
  graph_kernels_ = kernels;
  return cudaSuccess;
}

cudaError_t BatchEngine::run(int iters) {
  cudaError_t e = cudaSuccess;
  if (dirty_ && (e = rebuild())) return e;
  if ((e = ensure_graph())) return e;
  const int n = (iters + kGraphIters - 1) / kGraphIters;
  for (int i = 0; i < n && !e; ++i) {
    e = cudaGraphLaunch(graph_, s_);
    note_launch(graph_kernels_);  // kernels inside the graph
  }
  return e;
}

cudaError_t BatchEngine::poll(std::vector<int> *finished) {
  const int n = (int)slots_.size();
  cudaError_t e = cudaMemcpyAsync(h_S_, d_S_, sizeof(SolverScalars) * n, cudaMemcpyDeviceToHost, s_);
  if (!e) e = cudaStreamSynchronize(s_);
  if (e) return e;
  const double t = now();
  for (int i = 0; i < n; ++i) {
    if (slots_[i].state == 1 && h_S_[i].done != 0) {
      slots_[i].state = 2;
      slots_[i].t_done = t;
      h_slots_[i].active = 0;
      dirty_ = true;
      if (finished) finished->push_back(i);
    }
  }
  return cudaSuccess;
}

cudaError_t BatchEngine::collect(int slot, double *x_host, jqcd_solve_info *info) {
  cudaError_t e = collect_async(slot, x_host);
  if (!e) e = cudaEventSynchronize(ev_done_[slot]);
  if (e) return e;
  finish(slot, info);
  return cudaSuccess;
}

cudaError_t BatchEngine::collect_async(int slot, double *x_host) {
  if (slot < 0 || slot >= (int)slots_.size() || slots_[slot].state != 2) return cudaErrorInvalidValue;
  SlotHost &H = slots_[slot];
  GaugeEntry *G = H.G;
  SlotBuffers &B = H.buf;
  const Geom &g = G->g;
  const int64_t vh = g.vh;
  const double k = H.P.kappa;
  SolverScalars *S = d_S_ + slot;
  float4 *x_e = B.x, *x_o = B.x + 12 * vh, *b_e = B.b, *b_o = B.b + 12 * vh;
  const int nb12 = (int)blas_blocks(12 * vh);
  cudaError_t e;
#define CKE(call) do { e = (call); if (e) return e; } while (0)
  // x_o = b_o + kappa H_oe x_e
  CKE(launch_hop(PREC_DW, G->hop_params(PREC_DW, 1, x_e, b_o, x_o, 1.0, k, nullptr), false, true, false, s_));
  // ||b - D x||^2 over both parities
  CKE(launch_hop(PREC_DW, G->hop_params(PREC_DW, 0, x_o, x_e, B.wdw, 1.0, -k, nullptr), false, true, false, s_));
  CKE(launch_hop(PREC_DW, G->hop_params(PREC_DW, 1, x_e, x_o, B.tdw, 1.0, -k, nullptr), false, true, false, s_));
  CKE(launch_dw_xmy_norm(B.Adw, b_e, B.wdw, 12 * vh, B.part, s_));
  CKE(launch_dw_xmy_norm(B.r, b_o, B.tdw, 12 * vh, B.part + nb12, s_));
  CKE(launch_finalize_sum(B.part, 2 * nb12, &S->full_rr, s_));
  // canonical x unpacked into the slot's b buffer (b is not read after the
  // residual above), then both copies on the copy stream
  double *stage = reinterpret_cast<double *>(B.b);
  if (x_host) CKE(launch_spinor_unpack(g, PREC_DW, x_e, x_o, stage, s_));
  // pageable x: copied on the compute stream (the copy returns when done)
  cudaStream_t cs = (!x_host || page_locked(x_host)) ? cs_ : s_;
  if (cs == cs_) {
    CKE(cudaEventRecord(ev_out_[slot], s_));
    CKE(cudaStreamWaitEvent(cs_, ev_out_[slot], 0));
  }
  if (x_host)
    CKE(cudaMemcpyAsync(x_host, stage, sizeof(double) * 24 * (size_t)(2 * vh), cudaMemcpyDeviceToHost, cs));
  CKE(cudaMemcpyAsync(h_S_ + slot, S, sizeof(SolverScalars), cudaMemcpyDeviceToHost, cs));
  CKE(cudaEventRecord(ev_done_[slot], cs));
#undef CKE
  H.state = 3;
  return cudaSuccess;
}

bool BatchEngine::drained(int slot) const {
  return slots_[slot].state == 3 && cudaEventQuery(ev_done_[slot]) == cudaSuccess;
}

cudaError_t BatchEngine::wait_collect(int slot) const { return cudaEventSynchronize(ev_done_[slot]); }

int BatchEngine::draining() const {
  int r = 0;
  for (const SlotHost &s : slots_) r += s.state == 3;
  return r;
}

void BatchEngine::finish(int slot, jqcd_solve_info *info) {
  SlotHost &H = slots_[slot];
  const int64_t vh = H.G->g.vh;
  const SolverScalars &Sh = h_S_[slot];
  if (info) {
    memset(info, 0, sizeof *info);
    info->iters = Sh.iters;
    info->reliable_updates = Sh.reliable_updates;
    info->status = Sh.done == 1 ? JQCD_OK : (Sh.done == 3 ? JQCD_ENOCONV : JQCD_EBREAKDOWN);
    info->true_rel_resid = Sh.rhs2 > 0 ? std::sqrt(Sh.true_rr / Sh.rhs2) : 0.0;
    info->full_rel_resid = Sh.b2 > 0 ? std::sqrt(Sh.full_rr / Sh.b2) : 0.0;
    info->gpu_seconds = H.t_done - H.t_admit;
    info->seconds = now() - H.t_admit;
    // algorithmic bytes as if every hop ran alone (the batch shares link loads)
    const double lpb = hp_ == PREC_F16N ? (2 * 488.0 + 2 * (488.0 + 52.0)) : (2 * 576.0 + 2 * (576.0 + 96.0));
    const double dwb = 2 * 1536.0 + 2 * (1536.0 + 192.0);
    info->hop_count = 4.0 * Sh.iters + 4.0 * Sh.reliable_updates + 6.0;
    info->hop_bytes = (double)vh * (lpb * Sh.iters + dwb * Sh.reliable_updates + 6 * (1536.0 + 192.0));
  }
  H.state = 0;
  H.G = nullptr;
  h_slots_[slot].active = 0;
  dirty_ = true;
}

std::string BatchEngine::tune_key() const {
  std::vector<std::pair<int64_t, int>> shape;
  std::map<const void *, std::pair<int64_t, int>> by;
  for (size_t i = 0; i < slots_.size(); ++i)
    if (slots_[i].state == 1) {
      auto &v = by[h_slots_[i].gauge_f32];
      v.first = h_slots_[i].g.vh;
      v.second += 1;
    }
  for (auto &kv : by) shape.push_back(kv.second);
  std::sort(shape.begin(), shape.end());
  std::string key = std::to_string(hp_) + ":";
  for (auto &s : shape) key += std::to_string(s.first) + "x" + std::to_string(s.second) + ",";
  return key;
}

cudaError_t BatchEngine::autotune() {
  const std::string key = tune_key();
  auto it = tuned_.find(key);
  if (it != tuned_.end()) {
    lp_grid_ = it->second.first;
    return cudaSuccess;
  }
  cudaError_t e = cudaSuccess;
  if (dirty_ && (e = rebuild())) return e;
  const int m_cand[] = {2, 4, 6, 8, 12};
  float best = 1e30f;
  int best_grid = lp_grid_;
  cudaEvent_t a, b;
  if ((e = cudaEventCreate(&a))) return e;
  if ((e = cudaEventCreate(&b))) { cudaEventDestroy(a); return e; }
  const BatchArgs A = args();
  for (int m : m_cand) {
    const int grid = sm_count_ * m;
    const LpGrids lp = lp_grids(grid);
    if ((e = launch_batch_lp_apply(A, hp_, lp, s_))) break;  // warm-up
    if ((e = cudaEventRecord(a, s_))) break;
    for (int r = 0; r < 3 && !e; ++r) e = launch_batch_lp_apply(A, hp_, lp, s_);
    if (!e) e = cudaEventRecord(b, s_);
    if (!e) e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (!e) e = cudaEventElapsedTime(&ms, a, b);
    if (e) break;
    if (ms < best) { best = ms; best_grid = grid; }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (e) return e;
  lp_grid_ = best_grid;
  tuned_[key] = {best_grid, 0};
  return cudaSuccess;
}

}  // namespace jqcd
