// Batched stepping of many independent 2D Euler problems (degrees 3 and 4) in
// one launch per phase, or in one persistent launch for all phases and steps.
// The kernels run the same per-block bodies as the single-problem kernels
// (local_body, face_body, update_body), so a batched step computes exactly
// what the single-problem step computes.  Interface between cr_batch.cu (the
// kernels) and cr_host.cu (the C ABI).
#pragma once
#include "cr_common.cuh"

namespace crk {

// One unit of work: block blk of problem prob (a tile).
struct BatchTile {
  int prob, blk;
};

template <typename real>
struct BatchArgs {
  Tab<real> tb[2];              // tables of degree 3 and 4 in the bulk type (kernel parameters,
  Tab<double> td[2];            // like the single-problem kernels'), and in FP64
  const KParams<real>* P;       // [nprob] parameters of every problem (device)
  const int* deg;               // [nprob] degree, 3 or 4
  const int* nblk_el;           // [nprob] element blocks of the problem (update phase count)
  const int* nblk_face;         // [nprob] face-node blocks of the problem
  const BatchTile* t_el;        // element tiles (local and update phases), all problems
  int n_el;
  const BatchTile* t_face;      // face-node tiles, all problems
  int n_face;
  const BatchTile* t_upd;       // element tiles of the update phase (blocks of upd_threads)
  int n_upd;
  const int* nblk_upd;          // [nprob] update blocks of the problem
  int upd_threads;              // threads per block of the update phase
  int el_first[2], el_count[2];   // element tiles of degree 3 and 4 (t_el holds them in that order)
  int upd_first[2], upd_count[2]; // likewise for t_upd
  int nprob;
  int tiles;                    // fused launch: tiles per claim = kFusedClaim * tiles
  unsigned* queue;              // fused launch: [0] next unclaimed work item, then the tiles
                                // finished per (phase, problem) [3][nprob]; zeroed before each launch
  int* err;                     // set when a wait of the fused launch gave up
  unsigned long long spin_limit;  // polls (>= 64 ns each) before a wait gives up
  int phantom;                  // extra completions every wait requires (0; > 0 only in tests
                                // of the timeout path: they never come)
  int nsteps;                   // steps per fused launch
};

// Threads per block the batched kernels are built for, and tiles per block.
constexpr int kBatchThreadChoices[2] = {128, 256};
constexpr int kBatchTileChoices[3] = {1, 2, 4};
// Tiles per claim of the fused kernel for each tile of cr_batch_config's
// tiles: few claims on the queue's one counter, and one dependency check and
// one publication per run of tiles of the same (phase, problem).
constexpr int kFusedClaim = 8;

// Shared memory (bytes) of the largest body for a block of `threads` threads.
size_t batch_smem(int threads, bool fp32);
// Set the kernels' shared-memory limits; returns the first error.
cudaError_t batch_configure(int threads, bool fp32);
// Blocks of the fused kernel that fit on the device at once (cooperative grid).
cudaError_t batch_fused_max_blocks(int threads, bool fp32, int* blocks);
// phase 0 local, 1 face, 2 update: one launch over all tiles of the phase.
cudaError_t batch_launch_phase(int threads, int phase, const void* args, bool fp32,
                               cudaStream_t s);
// Start a run on every problem (t_final, CFL time step; plans the first step).
cudaError_t batch_set_run(const void* P, int n, double t_final, bool fp32, cudaStream_t s);
// All phases of A.nsteps steps in one cooperative launch of `grid` blocks.
cudaError_t batch_launch_fused(int threads, int grid, const void* args, bool fp32, cudaStream_t s);

}  // namespace crk
