// Host side of the batched mixed-precision CG engine (kernels in batch.h).
#pragma once
#include <cuda_runtime.h>

#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "batch.h"
#include "jqcd.h"
#include "solver.h"

namespace jqcd {

// Device buffers of one slot, sized for `vh_cap` sites per parity.
struct SlotBuffers {
  int64_t vh_cap = 0;
  int hp = -1;
  void *p = nullptr, *Ap = nullptr, *w = nullptr, *t = nullptr;
  float4 *xs = nullptr, *rs = nullptr;
  float4 *b = nullptr, *x = nullptr, *r = nullptr, *rhs = nullptr, *wdw = nullptr, *Adw = nullptr,
         *tdw = nullptr;
  double *part = nullptr;
  size_t bytes = 0;
  std::vector<void *> allocs;
  ~SlotBuffers();
  void release();
  cudaError_t ensure(int64_t vh, int hp);
  static size_t footprint(int64_t vh, int hp);
  static int64_t n_part(int64_t vh);
};

struct SlotHost {
  int state = 0;  // 0 free, 1 iterating, 2 converged or stopped, waiting for collect,
                  // 3 result copy to the host in flight (collect_async), waiting for finish
  GaugeEntry *G = nullptr;
  jqcd_solve_params P{};
  SlotBuffers buf;
  double t_admit = 0.0, t_done = 0.0;  // seconds on the engine's host clock
};

class BatchEngine {
 public:
  BatchEngine(int hp, int max_slots, cudaStream_t s, int sm_count);
  ~BatchEngine();
  cudaError_t init();
  int hop_prec() const { return hp_; }
  int max_slots() const { return (int)slots_.size(); }
  int free_slot() const;
  int running() const;
  // Prepare slot `slot` for D x = b (b: host canonical spinor).  Even-odd
  // source, normal-equation right-hand side, start residual; the slot joins
  // the next iteration.  b is copied on the engine's copy stream into the
  // slot's own buffers, so the copy overlaps the iterations of other slots,
  // when b is page-locked; a pageable b is copied on the compute stream.
  cudaError_t admit(int slot, GaugeEntry *G, const jqcd_solve_params &P, const double *b_host);
  // Run `iters` iterations of every running slot (graph replays).
  cudaError_t run(int iters);
  // Copy the device scalars; slots that finished move to state 2.
  cudaError_t poll(std::vector<int> *finished);
  // Reconstruct x_o, compute ||b - D x||, copy x to the host, fill info and
  // free the slot (collect_async, then a wait for the copy, then finish).
  cudaError_t collect(int slot, double *x_host, jqcd_solve_info *info);
  // The same without waiting: the reconstruction and residual are queued on
  // the compute stream, the copies of x and of the slot's scalars on the copy
  // stream (compute stream for a pageable x_host); the slot stays in state 3
  // until finish().  x_host must stay valid and untouched until drained(slot).
  cudaError_t collect_async(int slot, double *x_host);
  // True once the copies queued by collect_async(slot) have completed.
  bool drained(int slot) const;
  // True while slot is in state 3; wait_collect blocks until it is drained.
  bool collecting(int slot) const { return slots_[slot].state == 3; }
  cudaError_t wait_collect(int slot) const;
  // Fill info from the copied scalars and free the slot; slot must be drained.
  void finish(int slot, jqcd_solve_info *info);
  // Slots in state 3.
  int draining() const;
  // Choose sites per tile and grid size for the current active set.
  cudaError_t autotune();
  const SolverScalars &scalars(int slot) const { return h_S_[slot]; }
  // Free slot for a lattice of vh sites: best fit among free slots whose
  // buffers already suffice (extra = 0), else an unused slot or the largest
  // free one (extra = bytes the admission will add).  -1 if none is free.
  int pick_slot(int64_t vh, int64_t *extra_bytes) const;
  // Device bytes held by all slot buffers.
  size_t allocated_bytes() const;
  // Free the buffers of every idle slot except `keep`.
  void release_idle(int keep);
  double now() const;
  int tile_sites() const { return tile_sites_; }
  int grid() const { return grid_; }
  int lp_grid() const { return lp_grid_; }
  cudaStream_t stream() const { return s_; }

 private:
  cudaError_t rebuild();
  BatchArgs args() const;
  cudaError_t ensure_graph();
  std::string tune_key() const;

  int hp_;
  int sm_count_;
  cudaStream_t s_;
  std::vector<SlotHost> slots_;
  std::vector<SlotDev> h_slots_;
  SlotDev *d_slots_ = nullptr;
  SolverScalars *d_S_ = nullptr;
  SolverScalars *h_S_ = nullptr;  // pinned
  GroupDev *d_groups_ = nullptr;
  int2 *d_tiles_ = nullptr;
  int *d_ntiles_ = nullptr;
  int2 *d_lp_tiles_ = nullptr;
  int *d_n_lp_tiles_ = nullptr;
  int *d_n_lp2_tiles_ = nullptr;  // pair items live in d_lp_tiles_ + max_lp_tiles_
  int *d_n_lp1_tiles_ = nullptr;  // single items in d_lp_tiles_ + 2 * max_lp_tiles_
  int64_t max_lp_tiles_ = 0;
  int lp_grid_ = 0;
  int *d_any_update_ = nullptr;
  int max_groups_ = 0;
  int64_t max_tiles_ = 0;
  cudaStream_t cs_ = nullptr;        // host <-> device copies of sources and solutions
  std::vector<cudaEvent_t> ev_in_;   // per slot: source copy landed (copy stream)
  std::vector<cudaEvent_t> ev_out_;  // per slot: solution unpacked (compute stream)
  std::vector<cudaEvent_t> ev_done_; // per slot: solution and scalars on the host
  int tile_sites_ = 128;
  int grid_ = 0;
  bool dirty_ = true;
  cudaGraphExec_t graph_ = nullptr;  // the graph of the current grids (owned by graphs_)
  int64_t graph_kernels_ = 0;
  std::map<std::tuple<int, int, int, int, int>, std::pair<cudaGraphExec_t, int64_t>> graphs_;
  int64_t n_tiles_ = 0, n_lp_items_ = 0, n_lp2_items_ = 0, n_lp1_items_ = 0;  // current work items
  void drop_graphs();
  // grids of the low-precision kernels for a persistent grid of lp_grid
  // blocks, each capped at the next power of two of its item count
  LpGrids lp_grids(int lp_grid) const;
  std::map<std::string, std::pair<int, int>> tuned_;
  double t0_ = 0.0;
};

}  // namespace jqcd
