// lbm13_pair.h -- paired time steps of one FP32 lattice periodic in x and y
// (pair_step_kernel, lbm13_step2.cu): tile constants and the launch.
#pragma once

#include <cuda.h>  // CUtensorMap (the type only: the encoder is fetched through the runtime)

#include "lbm13_internal.h"

namespace lbm13 {

// Two time steps per launch.  Persistent blocks, one per SM,
// take output tiles of kPairX x kPairY nodes in turn.  For each tile the rows
// and columns within four links of it (kPairInX x kPairInY nodes, all 13
// planes, [row][plane][column]) arrive in shared memory (a tensor copy issued
// while the previous tile is stepped: two input buffers), the kPairMidX x
// kPairMidY nodes within two links are stepped into a third tile, and the
// output tile is stepped from that and written to the other buffer: one read
// and one write of every population per two updates.  The intermediate tile
// is one warp wide (every warp steps whole rows of 32 nodes), the output
// tile 28 columns of it.
constexpr int kPairX = 28, kPairY = 28;
constexpr int kPairInX = kPairX + 8, kPairInY = kPairY + 8;
constexpr int kPairMidX = kPairX + 4, kPairMidY = kPairY + 4;
constexpr int kPairIn = kPairInY * Q * kPairInX;     // floats of one input box
constexpr int kPairInStride = (kPairIn + 31) / 32 * 32;  // input buffers 128 bytes apart
constexpr int kPairMid = kPairMidY * Q * kPairMidX;  // floats
constexpr int kPairThreads = 512;
constexpr int kPairBlocksPerSm = 1;
constexpr int kPairSmem = (2 * kPairInStride + kPairMid) * 4;  // 188,160 bytes: one block per SM
static_assert(kPairMidX == 32, "the intermediate tile is one warp wide");
// a tensor copy's shared-memory destination must be 128-byte aligned
static_assert(kPairInStride * 4 % 128 == 0, "paired-step input buffers 128-byte aligned");

// Paired steps of one FP32 lattice periodic in x and y: reads a.fin, writes
// the state two steps later to a.fout.  map describes a.fin as (x: nx, plane:
// 13, y: ny) in boxes of kPairInX x 13 x kPairInY; tiles clear of the periodic
// seam load through it, the others by wrapped global loads.  Every tensor
// copy's wait is bounded by wait_ns of the global timer; after a timeout the
// block sets *err, waits (bounded) for its copies in flight and leaves without
// writing the tile (issue = 0 withholds the copies: the self-check of that
// wait).
cudaError_t launch_pair_step(const StepArgs<float, float> &a, const CUtensorMap &map, bool force, unsigned *err,
                             cudaStream_t s, int issue = 1, unsigned long long wait_ns = 1000000000ull);

}  // namespace lbm13
