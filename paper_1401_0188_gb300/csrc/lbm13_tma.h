// lbm13_tma.h -- tensor-map staging of the batched FP32 step (lbm13_batch.cu)
// and its host-side description (lbm13_api.cu).  The paired steps' tile
// constants are in lbm13_pair.h.
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

// Ring-staged tiles (batch_ring_kernel): a block steps a strip of W columns
// (W = 64 with eight warps, or W = 32 with four) over `groups` 4-row output
// groups.  The strip's input rows stream in 4-row chunks through a ring of
// kRingRowsTotal rows of shared memory, laid out [ring row][plane][W + 8
// columns]: chunk k holds input rows yb - 2 + 4k .. yb + 1 + 4k (columns
// x0 - 4 .. x0 + W + 3, so that its first column is 16-byte aligned) in ring
// rows 4 (k mod kRingSlots) .. + 3, loaded by one tensor copy whose map orders
// the lattice as (x, plane, y).  Output group g (rows yb + 4g .. + 3) reads
// chunks g and g + 1 only, so with four slots two chunks are in flight while
// two are read.  Each warp (W / 32 column slices x four rows) steps one row
// of 32 nodes per group.  Full and empty mbarriers per slot hand the chunks
// over; no block-wide barrier after the set-up.  W = 64: two blocks per SM
// (16 warps), W = 32: five (20 warps, the register cap 96, which the strips
// meet without spilling; six blocks would cap it at 80 and spill).
constexpr int kRingRows = 4;
constexpr int kRingSlots = 4;
constexpr int kRingRowsTotal = kRingRows * kRingSlots;     // 16: ring row = relative row & 15
static_assert((kRingRowsTotal & (kRingRowsTotal - 1)) == 0, "ring rows must be a power of two");

template <int W>
struct Ring {
    static constexpr int X = W + 8;                        // box width
    static constexpr int Consumers = (W / 32) * kRingRows;  // warps
    static constexpr int Threads = 32 * Consumers;
    static constexpr int RowFloats = Q * X;                // one ring row, all planes
    static constexpr int Chunk = kRingRows * RowFloats;    // floats per chunk
    static constexpr unsigned Bytes = unsigned(Chunk) * 4u;
    // ring slots, then one 13-float row per thread for the edge gathers
    static constexpr int Smem = kRingSlots * int(Bytes) + Threads * Q * 4;
    static constexpr int BlocksPerSm = W == 64 ? 2 : 5;
    static_assert(Bytes % 128 == 0, "ring slots are tensor-copy destinations: 128-byte aligned");
    // nodes of one edge work item: one per thread of the block
    static constexpr int EdgeNodes = Threads;
};

// The nodes of a lattice within two links of an edge, in the order the edge
// work items of the ring-staged strips take them: rows 0, 1, ny - 2, ny - 1
// across the lattice, then columns 0, 1, nx - 2, nx - 1 of rows 2 .. ny - 3
// (four per row).  The strips step every other node from the staged rows.
__host__ __device__ inline long long ring_edge_count(int nx, int ny)
{
    return 4LL * nx + 4LL * (ny > 4 ? ny - 4 : 0);
}

// One lattice's tensor maps: map[p] describes the buffer read when the step's
// parity is p, as a 3-D tensor (x: nx, y: ny, plane: 13) with row stride
// pitch and plane stride plane (in bytes), in boxes of the slab tile; ring[p]
// the same buffers in boxes of the ring tile.  use / ring_use = 0: the
// lattice is stepped through global loads (too small for the box, or the map
// could not be made).
struct LatticeMaps {
    CUtensorMap map[2];
    CUtensorMap ring[2];    // boxes of the 64-column strips
    CUtensorMap ring32[2];  // boxes of the 32-column strips
    int use;
    int ring_use;
    int ring32_use;
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
// `width` = 64 or 32 columns x groups 4-row groups), packed as
// (segment << 16) | strip, or (lattice, edge item e) packed as -1 - e: its
// share of the lattice's edge nodes (Ring<W>::EdgeNodes per item, in
// ring_edge_count's order), stepped with global loads.  Every
// mbarrier wait is bounded by wait_ns of the global timer; after a timeout the
// warp sets *err and leaves, and the producer lane waits (bounded) for the
// copies it issued before it leaves.  issue = 0 withholds the copies (self-check of the
// bounded waits; nothing is written then).
cudaError_t launch_batch_ring(const BatchDesc<float, float> *descs, const LatticeMaps *maps, const int2 *work,
                              int ntiles, int parity, int groups, int width, unsigned *err, cudaStream_t s,
                              int issue = 1, unsigned long long wait_ns = 1000000000ull);

}  // namespace lbm13
