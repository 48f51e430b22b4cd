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

// One lattice's tensor maps: map[p] describes the buffer read when the step's
// parity is p, as a 3-D tensor (x: nx, y: ny, plane: 13) with row stride
// pitch and plane stride plane (in bytes).  use = 0: the lattice is stepped
// through global loads (too small for the box, or the map could not be made).
struct LatticeMaps {
    CUtensorMap map[2];
    int use;
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

}  // namespace lbm13
