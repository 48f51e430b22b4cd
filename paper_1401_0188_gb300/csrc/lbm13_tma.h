// lbm13_tma.h -- tensor-map staging of the batched FP32 step (lbm13_batch.cu)
// and its host-side description (lbm13_api.cu).
#pragma once

#include <cuda.h>  // CUtensorMap (the type only: the encoder is fetched through the runtime)

#include "lbm13_internal.h"

namespace lbm13 {

// Tiles of the staged step: 32 columns x 8-row slabs, each slab loaded with
// its halo (2 columns and 2 rows each side; the box starts 4 columns left so
// that its first column is 16-byte aligned) for all 13 planes by one tensor
// copy: a box of 40 x 12 x 13 floats.  One slab per block in shared memory
// (25 KB): six blocks per SM keep 24 warps resident, which measured faster
// than two slabs in flight per block with fewer blocks.
constexpr int kTmaX = 40;
constexpr int kTmaRows = 8;
constexpr int kTmaY = kTmaRows + 4;
constexpr int kTmaStage = Q * kTmaY * kTmaX;              // floats per slab
constexpr unsigned kTmaBytes = unsigned(kTmaStage) * 4u;   // bytes per slab
constexpr int kTmaSmem = kTmaStage * 4;                    // one slab per block

// Ring-staged tiles (batch_ring_kernel): a block steps a strip of 64 columns
// over `groups` 4-row output groups.  One producer warp streams the strip's
// input rows in 4-row chunks -- a box of 72 x 4 x 13 floats, starting 4
// columns left of the strip so that its first column is 16-byte aligned --
// through a ring of kRingSlots shared-memory slots; output group g reads
// chunks g, g + 1 and g + 2 (rows -2 .. +5 around it), so every input row is
// loaded once per strip.  Eight consumer warps (two column halves x four rows)
// each step one row of 32 nodes per group.  Full and empty mbarriers per slot
// hand the chunks over; no block-wide barrier after the set-up.
constexpr int kRingW = 64;
constexpr int kRingX = kRingW + 8;
constexpr int kRingRows = 4;
constexpr int kRingSlots = 6;
constexpr int kRingChunk = Q * kRingRows * kRingX;        // floats per chunk
constexpr unsigned kRingBytes = unsigned(kRingChunk) * 4u;  // bytes per chunk (14,976)
constexpr int kRingConsumers = 8;
constexpr int kRingThreads = 32 * (kRingConsumers + 1);
// ring slots, then one 13-float row per consumer thread for the edge gathers
constexpr int kRingSmem = kRingSlots * int(kRingBytes) + 32 * kRingConsumers * Q * 4;

// One lattice's tensor maps: map[p] describes the buffer read when the step's
// parity is p, as a 3-D tensor (x: nx, y: ny, plane: 13) with row stride
// pitch and plane stride plane (in bytes), in boxes of the slab tile; ring[p]
// the same buffers in boxes of the ring tile.  use / ring_use = 0: the
// lattice is stepped through global loads (too small for the box, or the map
// could not be made).
struct LatticeMaps {
    CUtensorMap map[2];
    CUtensorMap ring[2];
    int use;
    int ring_use;
};

// Staged batched step: one block per tile of 32 columns x 16 groups rows (two
// slabs per row group of the R = 4, BY = 4 tile shape); the wait for each
// slab is bounded (wait_ns by the global timer, 1 s in a step), after which
// the block sets *err, waits (bounded) for its copy in flight and returns.
// issue = 0 withholds the copies, so that every wait runs out (the self-check
// of the bounded wait; nothing is written then).
cudaError_t launch_batch_tma(const BatchDesc<float, float> *descs, const LatticeMaps *maps, const int2 *work,
                             int ntiles, int parity, int groups, unsigned *err, cudaStream_t s, int issue = 1,
                             unsigned long long wait_ns = 1000000000ull);

// Ring-staged batched step (FP32): one block per work item (lattice, strip of
// 64 columns x groups 4-row groups), packed as (segment << 16) | strip.  Every
// mbarrier wait is bounded by wait_ns of the global timer; after a timeout the
// warp sets *err and leaves, and the producer waits (bounded) for the copies it
// issued before it leaves.  issue = 0 withholds the copies (self-check of the
// bounded waits; nothing is written then).
cudaError_t launch_batch_ring(const BatchDesc<float, float> *descs, const LatticeMaps *maps, const int2 *work,
                              int ntiles, int parity, int groups, unsigned *err, cudaStream_t s, int issue = 1,
                              unsigned long long wait_ns = 1000000000ull);

}  // namespace lbm13
