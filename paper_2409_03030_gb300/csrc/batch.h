// Batched mixed-precision CG: many concurrent solves (any lattice, kappa and
// tolerance) advanced together, one iteration of every active solve per
// pass, by persistent kernels that walk a device-resident tile list.
//
// Solves on the same gauge field form a group; a tile is one block of
// consecutive sites of one group, and the low-precision hop kernels stage
// the tile's links in shared memory once and apply them to every right-hand
// side of the group (link bytes amortised over the group).  Each slot keeps
// its own device-resident CG scalars (SolverScalars), its own reliable-update
// flag and its own partial sums, so slots join, converge and leave
// independently.  Kernel arguments point at the descriptor arrays, which lets
// one captured CUDA graph of an iteration serve every change of the active
// set.
#pragma once
#include <cuda_runtime.h>

#include "kernels.h"

namespace jqcd {

constexpr int kBatchMaxRhs = 16;  // right-hand sides per group (one tile pass)

struct SlotDev {
  Geom g;
  const float4 *gauge_f32;  // [2][4][3][vh]  12-real FP32 links
  const float4 *gauge_dw;   // [2][4][9][vh]  double-word links
  double kappa;
  float k2;                 // -kappa^2
  float2 k2_dw;             // -kappa^2 as a double-word number
  float2 kap_dw;            // kappa as a double-word number
  void *p, *Ap, *w, *t;     // hop precision (t odd parity, others even)
  float4 *xs, *rs;          // FP32 inner iterate and residual (even)
  float4 *b, *x;            // double-word, whole lattice (even then odd half)
  float4 *r, *rhs, *wdw, *Adw, *tdw;  // double-word (tdw odd, others even)
  double *part;             // partial sums, one per site block
  int active;               // 1 while the solve iterates
  int nblocks;              // site blocks of this lattice for the current tile size
  int nblk_lp;              // kLpThreads-site blocks of this lattice (hop partials)
  int pad;
};

struct GroupDev {
  Geom g;
  const float4 *gauge_f32;
  const float4 *gauge_dw;
  int nslots;
  int slot[kBatchMaxRhs];
  int tpb;                  // reserved
};

struct BatchArgs {
  SlotDev *slots;
  SolverScalars *S;      // one per slot
  GroupDev *groups;
  int2 *tiles;           // (group, site block of tile_sites)
  const int *ntiles;
  int2 *lp_tiles;        // (16 * group + slot in group, block of kLpThreads sites)
  const int *n_lp_tiles;
  int2 *lp2_tiles;       // the same with the first slot of each pair of a group (slots
  const int *n_lp2_tiles;  // 0, 2, 4, ...): items of the packed low-precision stages
  int2 *lp1_tiles;       // (slot, block of kLpThreads sites) for the last slot of each group
  const int *n_lp1_tiles;  // with an odd count: items of the one-lane stages beside the packed ones
  int *any_update;       // nonzero when some slot requested a reliable update
  int nslots;            // descriptors allocated (grid of per-slot kernels)
};

// Shared-memory limits of the batch kernels; call once before launching.
cudaError_t batch_configure();

// Blocks of the low-precision operator kernel in hop precision hp that one SM
// holds at once (after batch_configure): a persistent grid of this many per
// SM fills the GPU in one wave.
int batch_lp_blocks_per_sm(int hp);

// Low-precision hop blocks: one thread per site, kLpThreads sites per item.
constexpr int kLpThreads = 128;

// Low-precision hop items carry two right-hand sides of a group (packed
// two-lane arithmetic, hop_lp2.cuh) when set, one otherwise.
#ifndef JQCD_BATCH_LP_PAIRS
#define JQCD_BATCH_LP_PAIRS 1
#endif
constexpr bool kBatchLpPairs = JQCD_BATCH_LP_PAIRS != 0;

// Persistent grids (blocks of kLpThreads threads) of the kernels that walk
// the per-slot items (all: the double-word reliable-update stages, and the
// low-precision stages without pairing), the pair items and the single items.
struct LpGrids {
  int all, pairs, singles;
};

// One CG iteration of every active slot (inner hop precision hp): the
// low-precision hops on the persistent grids lp, the other tile kernels on
// `grid` blocks of `tile_sites` threads.
cudaError_t launch_batch_iteration(const BatchArgs &A, int hp, int tile_sites, int grid,
                                   const LpGrids &lp, cudaStream_t s);
// Only the four low-precision hops of one iteration (for the autotuner; the
// last stage also updates x_s and r_s, so run it on a copy of the state).
cudaError_t launch_batch_lp_apply(const BatchArgs &A, int hp, const LpGrids &lp, cudaStream_t s);

}  // namespace jqcd
