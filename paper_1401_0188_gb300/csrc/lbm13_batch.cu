// lbm13_batch.cu -- many lattices stepped by one launch: the fused
// pull-stream + wall + MRT-collision step of lbm13_step.cu over a work list of
// (lattice, tile) pairs, each lattice's arguments read from a descriptor array.
// The per-node device code is the one-lattice kernel's (lbm13_stepdev.cuh), so
// a lattice gives bit-identical results alone or in a plan.
#include <atomic>

#include "lbm13_internal.h"
#include "lbm13_tma.h"
#include "lbm13_mbar.cuh"

// Each launch reads only what earlier launches wrote: the read-only path.
#define LBM13_LDG(p) __ldg(p)
#include "lbm13_stepdev.cuh"

namespace lbm13 {

namespace {

// Many lattices in one launch.  The work list holds (lattice, tile) pairs; a
// tile is 32 columns x (groups BY R) rows of one lattice, packed as
// (tile row << 16) | tile column, and the block walks its `groups` row groups
// of BY R rows in turn.  Each block takes a contiguous run of the work list
// (one tile when the grid has a block per tile; a longer run in a persistent
// grid), so consecutive tiles of a block mostly belong to one lattice; the next
// work item is fetched while the current one runs.  The block copies a
// lattice's arguments for this step's buffer parity into shared memory with
// 16-byte loads spread over its threads, only when the lattice changes.
// One row per thread keeps to 64 registers (half the SM's warps resident),
// two rows to 80 (24 warps: as many loads in flight as the one-lattice
// kernel); more rows per thread take what they need.
template <typename T, typename C, int R, int BY>
__global__ void __launch_bounds__(32 * BY, sizeof(T) == 4 ? (R == 1 ? 32 / BY : R == 2 ? 24 / BY : 1) : 1) batch_step_kernel(const BatchDesc<T, C> *__restrict__ descs,
                                                            const int2 *__restrict__ work, int ntiles, int parity,
                                                            int groups)
{
    __shared__ StepArgs<T, C> sa;
    __shared__ int s_force;
    __shared__ C slots[32 * BY][Q];
    constexpr int kWords = int(sizeof(StepArgs<T, C>) / 16);
    static_assert(sizeof(StepArgs<T, C>) % 16 == 0, "StepArgs must be a whole number of 16-byte words");
    const int tid = threadIdx.y * 32 + threadIdx.x;
    const int per = (ntiles + gridDim.x - 1) / gridDim.x;
    const int t0 = blockIdx.x * per;
    const int t_end = min(ntiles, t0 + per);
    int lattice = -1;
    int2 w = t0 < t_end ? __ldg(work + t0) : make_int2(0, 0);
    for (int t = t0; t < t_end; ++t) {
        const int2 wn = t + 1 < t_end ? __ldg(work + t + 1) : w;
        if (w.x != lattice) {
            __syncthreads();
            const int4 *src = reinterpret_cast<const int4 *>(&descs[w.x].a[parity]);
            int4 *dst = reinterpret_cast<int4 *>(&sa);
            for (int i = tid; i < kWords; i += 32 * BY) dst[i] = __ldg(src + i);
            if (tid == 0) s_force = descs[w.x].force;
            __syncthreads();
            lattice = w.x;
        }
        const int x = (w.y & 0xffff) * 32 + threadIdx.x;
        const int yb = (w.y >> 16) * groups * (BY * R);
        for (int g = 0; g < groups; ++g) {
            const int y = yb + g * (BY * R);
            if (y >= sa.ny) break;
            if (s_force)
                process_column<T, C, true, R>(sa, x, y + threadIdx.y * R, slots[tid]);
            else
                process_column<T, C, false, R>(sa, x, y + threadIdx.y * R, slots[tid]);
        }
        w = wn;
    }
}

// One block per tile (the grid the autotuner picks on uneven lattices): the
// same per-node code without the run loop, the next-item prefetch and the
// lattice comparison, so fewer registers stay live across the row groups.
template <typename T, typename C, int R, int BY>
__global__ void __launch_bounds__(32 * BY, sizeof(T) == 4 ? (R == 1 ? 32 / BY : R == 2 ? 24 / BY : 1) : 1) batch_tile_kernel(const BatchDesc<T, C> *__restrict__ descs,
                                                            const int2 *__restrict__ work, int parity, int groups)
{
    __shared__ StepArgs<T, C> sa;
    __shared__ int s_force;
    __shared__ C slots[32 * BY][Q];
    constexpr int kWords = int(sizeof(StepArgs<T, C>) / 16);
    const int tid = threadIdx.y * 32 + threadIdx.x;
    const int2 w = __ldg(work + blockIdx.x);
    {
        const int4 *src = reinterpret_cast<const int4 *>(&descs[w.x].a[parity]);
        int4 *dst = reinterpret_cast<int4 *>(&sa);
        for (int i = tid; i < kWords; i += 32 * BY) dst[i] = __ldg(src + i);
        if (tid == 0) s_force = descs[w.x].force;
    }
    __syncthreads();
    const int x = (w.y & 0xffff) * 32 + threadIdx.x;
    const int yb = (w.y >> 16) * groups * (BY * R);
    for (int g = 0; g < groups; ++g) {
        const int y = yb + g * (BY * R);
        if (y >= sa.ny) break;
        if (s_force)
            process_column<T, C, true, R>(sa, x, y + threadIdx.y * R, slots[tid]);
        else
            process_column<T, C, false, R>(sa, x, y + threadIdx.y * R, slots[tid]);
    }
}

// ------------------------------------------------ tensor-map staged tiles
//
// FP32 only.  Each block takes one tile of 32 columns x 16 `groups` rows in
// slabs of 8; one elected thread loads each slab (with its halo, all 13
// planes) by one tensor copy into shared memory, completion signalled on an
// mbarrier, the next slab issued once every warp is done with the current
// one.  A warp takes rows w and w + 4 of the slab and pulls its 13
// populations from shared memory; the lanes at an x edge replace
// the links that cross it with process_column's rules (global loads), and the
// rows within two of a y edge go through process_column itself, so the results
// are bit-identical to the other kernels.

__device__ __forceinline__ void mbar_init(unsigned bar) { mbar_init_count(bar, 1u); }

__device__ __forceinline__ void tma_slab(unsigned dst, const CUtensorMap *map, int x, int y, unsigned bar)
{
    tma_box_3d(dst, map, x, y, 0, bar, kTmaBytes);
}

// Row r of the slab in `tile` (its row 0 is the slab's first row minus 2,
// its column 0 is x0 - 4): node (x, y) of a row at least two from the bottom
// and top edges.
template <bool Force>
__device__ __forceinline__ void tma_row(const StepArgs<float, float> &a, const float *tile, int r, int x, int y)
{
    const int nx = a.nx;
    const bool xedge = x < nx && (x < 2 || x >= nx - 2) && !a.per_x;
    const int side = x < 2 ? WEST : EAST;
    WallState<float> st = {0.0f, 0.0f};
    if (xedge && a.wall[side].needs_data) {
        const WallArgs<float> &w = a.wall[side];
        if (w.kind == WALL_MIXED && w.mass_flux) {
            int x0, y0w, x1, y1w;
            wall_nodes(a, side, y, x0, y0w, x1, y1w);
            st = zero_flux_state(w, ld(a, out_unit(side), x0, y0w) + ld(a, out_two(side), x0, y0w) +
                                        ld(a, out_two(side), x1, y1w));
        } else {
            st = wall_state(a, side, y);
        }
    }
    float f[Q];
    const int lane = threadIdx.x;
#pragma unroll
    for (int j = 0; j < Q; ++j) f[j] = tile[(j * kTmaY + r + 2 - cvy(j)) * kTmaX + lane + 4 - cvx(j)];
    if (x >= nx) return;
    if (x < 2 || x >= nx - 2) {
#pragma unroll
        for (int j = 0; j < Q; ++j) {
            if (cvx(j) == 0) continue;
            const int sx = x - cvx(j);
            if (sx >= 0 && sx < nx) continue;
            if (a.per_x)
                f[j] = ld(a, j, sx < 0 ? sx + nx : sx - nx, y - cvy(j));
            else
                f[j] = cross_wall(a, side, j, x, y, st);
        }
    }
    collide<Force>(f, a.k);
    store(a, x, y, f);
}

template <bool Force>
__device__ __forceinline__ void tma_slabs(const StepArgs<float, float> &a, const CUtensorMap *map, float *stage,
                                          unsigned bar0, int x0, int yb, int nslab, int tid, float *slot,
                                          unsigned *err, int issue, unsigned long long wait_ns)
{
    const int x = x0 + threadIdx.x, ny = a.ny;
    const unsigned st0 = static_cast<unsigned>(__cvta_generic_to_shared(stage));
    if (tid == 0 && issue) tma_slab(st0, map, x0 - 4, yb - 2, bar0);
    for (int g = 0; g < nslab; ++g) {
        const bool ok = mbar_wait(bar0, g & 1, wait_ns);
        if (__syncthreads_or(!ok)) {
            // the copy did not complete in time: report, wait (bounded) once
            // more so that it does not land after the block, leave
            if (tid == 0) atomicOr(err, 1u);
            if (issue) mbar_wait(bar0, g & 1, wait_ns);
            return;
        }
        const float *tile = stage;
#pragma unroll 1
        for (int i = 0; i < kTmaRows / 4; ++i) {
            const int r = threadIdx.y + 4 * i;
            const int y = yb + g * kTmaRows + r;
            if (y >= ny) break;
            if (__all_sync(0xffffffffu, y >= 2 && y + 1 <= ny - 2))
                tma_row<Force>(a, tile, r, x, y);
            else
                process_column<float, float, Force, 1>(a, x, y, slot);
        }
        __syncthreads();
        if (tid == 0 && issue && g + 1 < nslab) tma_slab(st0, map, x0 - 4, yb + (g + 1) * kTmaRows - 2, bar0);
    }
}

__global__ void __launch_bounds__(128, 6) batch_tma_kernel(const BatchDesc<float, float> *__restrict__ descs,
                                                           const LatticeMaps *__restrict__ maps,
                                                           const int2 *__restrict__ work, int parity, int groups,
                                                           unsigned *err, int issue, unsigned long long wait_ns)
{
    extern __shared__ __align__(128) unsigned char tma_smem[];
    __shared__ StepArgs<float, float> sa;
    __shared__ float slots[128][Q];
    __shared__ __align__(8) unsigned long long bars[1];
    __shared__ int s_force, s_use;
    constexpr int kWords = int(sizeof(StepArgs<float, float>) / 16);
    const int tid = threadIdx.y * 32 + threadIdx.x;
    const int2 w = __ldg(work + blockIdx.x);
    {
        const int4 *src = reinterpret_cast<const int4 *>(&descs[w.x].a[parity]);
        int4 *dst = reinterpret_cast<int4 *>(&sa);
        for (int i = tid; i < kWords; i += 128) dst[i] = __ldg(src + i);
    }
    const unsigned bar0 = static_cast<unsigned>(__cvta_generic_to_shared(&bars[0]));
    if (tid == 0) {
        s_force = descs[w.x].force;
        s_use = maps[w.x].use;
        mbar_init(bar0);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    const int x0 = (w.y & 0xffff) * 32;
    const int yb = (w.y >> 16) * groups * 16;
    const int ny = sa.ny;
    const int nslab = min(groups * (16 / kTmaRows), (ny - yb + kTmaRows - 1) / kTmaRows);
    float *stage = reinterpret_cast<float *>(tma_smem);
    if (s_use) {
        const CUtensorMap *map = &maps[w.x].map[parity];
        if (s_force)
            tma_slabs<true>(sa, map, stage, bar0, x0, yb, nslab, tid, slots[tid], err, issue, wait_ns);
        else
            tma_slabs<false>(sa, map, stage, bar0, x0, yb, nslab, tid, slots[tid], err, issue, wait_ns);
        return;
    }
    // a lattice without tensor maps: one row per thread through global loads
    const int x = x0 + threadIdx.x;
    for (int g = 0; g < nslab; ++g) {
        for (int i = 0; i < kTmaRows / 4; ++i) {
            const int y = yb + g * kTmaRows + threadIdx.y + 4 * i;
            if (y >= ny) break;
            if (s_force)
                process_column<float, float, true, 1>(sa, x, y, slots[tid]);
            else
                process_column<float, float, false, 1>(sa, x, y, slots[tid]);
        }
    }
}

// ------------------------------------------------- ring-staged strips
//
// FP32 only.  A block of eight warps steps a strip of 64 columns of one
// lattice over `groups` 4-row output groups (rows yb .. yb + 4 groups - 1).
// Input chunk k (rows yb - 2 + 4k .. yb + 1 + 4k, columns x0 - 4 .. x0 + 67,
// all 13 planes) arrives by one tensor copy in ring slot k % kRingSlots, laid
// out [row][plane][column], so input row r (relative to yb - 2) sits in ring
// row r & 15.  The first lane of warp 0 is also the producer: it issues the
// first kRingSlots chunks at once, then, at the top of each group g >= 1,
// chunk g + 3 into the slot of chunk g - 1 once every warp has released that
// chunk.  Warp w steps row yb + 4g + (w & 3) of output group g in the column
// half w >> 2, pulling its 13 populations from chunks g and g + 1, and
// releases chunk g when the group is done (group g + 1 reads chunks g + 1 and
// g + 2).  The lattice's collision coefficients live in registers for the
// whole strip; every warp runs the same code (the row within the group only
// moves five ring-row addresses), and the loop makes no out-of-line call: the
// strips step only the nodes at least two links from every edge.  The edge
// nodes are work items of their own in the same launch (ring_edge_item):
// blocks that step them through process_column (periodic wraps and wall
// rules) with global loads, latency-bound, beside strips that keep
// streaming; the results are bit-identical to the other kernels.  (Edge work
// inside the strips' loop, even from the staged rows, slowed every strip: it
// costs the loop registers and instruction-cache room; a separate edge kernel
// ran latency-bound on its own instead of beside the streams.)

// One chunk: the box at (column x, plane 0, row y) of a map ordered (x, plane, y).
__device__ __forceinline__ void ring_chunk(unsigned dst, const CUtensorMap *map, int x, int y, unsigned bar,
                                           unsigned bytes)
{
    tma_box_3d(dst, map, x, 0, y, bar, bytes);
}

// Chunk k of the strip into its slot (the producer lane).
template <int W>
__device__ __forceinline__ void ring_issue(const CUtensorMap *map, unsigned st0, unsigned full0, int x0, int yb, int k)
{
    const int slot = k % kRingSlots;
    ring_chunk(st0 + unsigned(slot) * Ring<W>::Bytes, map, x0 - 4, yb - 2 + kRingRows * k, full0 + 8u * slot,
               Ring<W>::Bytes);
}

// Before the producer's warp leaves (normally or after a wait ran out), the
// copies issued into slots that no later copy re-armed must have landed, so
// that none lands in the block's shared memory after the block has left.
__device__ __forceinline__ void ring_drain(unsigned full0, int issued, unsigned long long wait_ns)
{
    for (int j = issued > kRingSlots ? issued - kRingSlots : 0; j < issued; ++j)
        mbar_wait(full0 + 8u * (j % kRingSlots), unsigned((j / kRingSlots) & 1), wait_ns);
}

// The 13 populations of a node from the staged rows: rb[d] is the address of
// ring row (input row of the node minus d) at the node's column (d = v_y in
// -2 .. 2, index d + 2); link j reads plane j of ring row rb[v_y] at column
// offset -v_x.
template <int W>
__device__ __forceinline__ void ring_pull(const float *const rb[5], float f[Q])
{
#pragma unroll
    for (int j = 0; j < Q; ++j) f[j] = rb[cvy(j) + 2][j * Ring<W>::X - cvx(j)];
}

// Staged phase of a consumer warp: the nodes of its row that lie at least two
// links from every edge, from the staged rows, with the coefficients in
// registers and no out-of-line call.  Returns false after a wait ran out.
template <bool Force, int W>
__device__ bool ring_consume(const StepArgs<float, float> &a, const float *stage, unsigned full0, unsigned empty0,
                             int x0, int yb, int ngroups, int wr, int half, const CUtensorMap *map, int producer,
                             unsigned *err, unsigned long long wait_ns)
{
    const Coef<float> k = a.k;  // in registers for the whole strip
    const int lane = threadIdx.x & 31;
    const int nchunks = ngroups + 1;
    const unsigned st0 = static_cast<unsigned>(__cvta_generic_to_shared(stage));
    int issued = producer ? min(nchunks, kRingSlots) : 0;  // the first ones went out with the set-up
    const int nx = a.nx, ny = a.ny;
    const int x = x0 + 32 * half + lane;
    const float *const colp = stage + 32 * half + lane + 4;  // the node's column in ring row 0
    const bool xin = x >= 2 && x < nx - 2;
    float *const fout = a.fout;
    const long long pitch = a.pitch, plane = a.plane;
    for (int g = 0; g < ngroups; ++g) {
        bool ok = true;
        if (producer && lane == 0 && g >= 1 && issued < nchunks) {
            // chunk g + 3 takes the slot of chunk g - 1: wait until every warp
            // has released that chunk
            const int c = g - 1;
            ok = mbar_wait(empty0 + 8u * (c % kRingSlots), unsigned((c / kRingSlots) & 1), wait_ns);
            if (ok) ring_issue<W>(map, st0, full0, x0, yb, issued++);
        }
        if (g == 0) ok = ok && mbar_wait(full0, 0u, wait_ns);
        {
            const int c = g + 1;
            ok = ok && mbar_wait(full0 + 8u * (c % kRingSlots), unsigned((c / kRingSlots) & 1), wait_ns);
        }
        if (!__all_sync(0xffffffffu, ok)) {
            if (lane == 0) {
                atomicOr(err, 1u);
                if (producer) ring_drain(full0, issued, wait_ns);
            }
            return false;
        }
        const int y = yb + kRingRows * g + wr;
        if (xin && y >= 2 && y <= ny - 3) {
            // input row of the node relative to yb - 2
            const int r = kRingRows * g + wr + 2;
            const float *rb[5];
#pragma unroll
            for (int d = -2; d <= 2; ++d) rb[d + 2] = colp + ((r - d) & (kRingRowsTotal - 1)) * Ring<W>::RowFloats;
            float f[Q];
            ring_pull<W>(rb, f);
            collide<Force>(f, k);
#ifdef LBM13_DEBUG
            store(a, x, y, f);
#else
            float *p = fout + (long long)y * pitch + x;
#pragma unroll
            for (int j = 0; j < Q; ++j) p[(long long)j * plane] = f[j];
#endif
        }
        // chunk g is needed by no later group: release its slot
        __syncwarp();
        if (lane == 0) mbar_arrive(empty0 + 8u * (g % kRingSlots));
    }
    if (producer && lane == 0) ring_drain(full0, issued, wait_ns);
    return true;
}

// An edge work item: nodes item * EdgeNodes .. (item + 1) * EdgeNodes - 1 of
// the lattice's edge nodes (in ring_edge_count's order), one per thread, each
// link resolved on its own (gather_body compiled in, global loads: every load
// of the node, its wall states' included, in one round trip), then collided
// and stored.  Lanes past the last node have nothing to do; the halo rows of
// a y-slab are written by the exchange, never stepped.
template <bool Force>
__device__ __forceinline__ void edge_node(const StepArgs<float, float> &a, int x, int y)
{
    float f[Q];
    gather_body(a, x, y, f, GlobalInlineSrc<float, float>());
    collide<Force>(f, a.k);
    store(a, x, y, f);
}

template <int W>
__device__ void ring_edge_item(const StepArgs<float, float> &a, int force, int item)
{
    const int nx = a.nx, ny = a.ny;
    const long long rows_part = 4LL * nx, total = ring_edge_count(nx, ny);
    const long long i = (long long)item * Ring<W>::EdgeNodes + threadIdx.x;
    int x = nx, y = min(2, ny - 1);
    if (i < rows_part) {
        // rows 0, 1, ny - 2, ny - 1
        const int r = int(i / nx);
        x = int(i - (long long)r * nx);
        y = r < 2 ? r : ny - 4 + r;
    } else if (i < total) {
        // columns 0, 1, nx - 2, nx - 1 of rows 2 .. ny - 3
        const long long k = i - rows_part;
        const int c = int(k & 3);
        y = 2 + int(k >> 2);
        x = c < 2 ? c : nx - 4 + c;
    }
    if (x >= nx) return;
    if ((y < 2 && a.wall[SOUTH].kind == HALO) || (y >= ny - 2 && a.wall[NORTH].kind == HALO)) return;
    if (force)
        edge_node<true>(a, x, y);
    else
        edge_node<false>(a, x, y);
}

template <int W>
__global__ void __launch_bounds__(Ring<W>::Threads, Ring<W>::BlocksPerSm) batch_ring_kernel(const BatchDesc<float, float> *__restrict__ descs,
                                                                     const LatticeMaps *__restrict__ maps,
                                                                     const int2 *__restrict__ work, int parity,
                                                                     int groups, unsigned *err, int issue,
                                                                     unsigned long long wait_ns)
{
    extern __shared__ __align__(128) unsigned char ring_smem[];
    __shared__ StepArgs<float, float> sa;
    __shared__ __align__(8) unsigned long long bars[2 * kRingSlots];  // full[slots], empty[slots]
    __shared__ int s_force, s_use;
    constexpr int kWords = int(sizeof(StepArgs<float, float>) / 16);
    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int2 w = __ldg(work + blockIdx.x);
    {
        const int4 *src = reinterpret_cast<const int4 *>(&descs[w.x].a[parity]);
        int4 *dst = reinterpret_cast<int4 *>(&sa);
        for (int i = tid; i < kWords; i += Ring<W>::Threads) dst[i] = __ldg(src + i);
    }
    const unsigned full0 = static_cast<unsigned>(__cvta_generic_to_shared(&bars[0]));
    const unsigned empty0 = full0 + 8u * kRingSlots;
    if (tid == 0) {
        s_force = descs[w.x].force;
        s_use = W == 64 ? maps[w.x].ring_use : maps[w.x].ring32_use;
        for (int i = 0; i < kRingSlots; ++i) {
            mbar_init_count(full0 + 8u * i, 1u);
            mbar_init_count(empty0 + 8u * i, unsigned(Ring<W>::Consumers));
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    float *stage = reinterpret_cast<float *>(ring_smem);
    float *slots = stage + kRingSlots * Ring<W>::Chunk;
    if (w.y < 0) {
        // an edge item (none in a check launch, whose copies are withheld)
        if (issue) ring_edge_item<W>(sa, s_force, -1 - w.y);
        return;
    }
    const int x0 = (w.y & 0xffff) * W;
    const int yb = (w.y >> 16) * groups * kRingRows;
    const int ny = sa.ny;
    const int ngroups = min(groups, (ny - yb + kRingRows - 1) / kRingRows);
    if (!s_use) {
        // a lattice without a ring tensor map: the warps step it through
        // global loads, one row per warp and group
        const int x = x0 + 32 * (warp >> 2) + (tid & 31);  // W / 32 slices x 4 rows
        for (int g = 0; g < ngroups; ++g) {
            const int y = yb + kRingRows * g + (warp & 3);
            if (y >= ny) break;
            if (s_force)
                process_column<float, float, true, 1>(sa, x, y, slots + tid * Q);
            else
                process_column<float, float, false, 1>(sa, x, y, slots + tid * Q);
        }
        return;
    }
    const CUtensorMap *map = W == 64 ? &maps[w.x].ring[parity] : &maps[w.x].ring32[parity];
    const int producer = warp == 0 && issue;
    if (producer && (tid & 31) == 0) {
        const unsigned st0 = static_cast<unsigned>(__cvta_generic_to_shared(stage));
        for (int k = 0; k < ngroups + 1 && k < kRingSlots; ++k) ring_issue<W>(map, st0, full0, x0, yb, k);
    }
    if (s_force)
        ring_consume<true, W>(sa, stage, full0, empty0, x0, yb, ngroups, warp & 3, warp >> 2, map, producer, err,
                              wait_ns);
    else
        ring_consume<false, W>(sa, stage, full0, empty0, x0, yb, ngroups, warp & 3, warp >> 2, map, producer, err,
                               wait_ns);
}

template <typename T, typename C, int R, int BY>
cudaError_t launch_batch_rb(const BatchDesc<T, C> *descs, const int2 *work, int ntiles, int parity, int groups,
                            int grid, cudaStream_t s)
{
    if (grid >= ntiles)
        batch_tile_kernel<T, C, R, BY><<<ntiles, dim3(32, BY), 0, s>>>(descs, work, parity, groups);
    else
        batch_step_kernel<T, C, R, BY><<<grid, dim3(32, BY), 0, s>>>(descs, work, ntiles, parity, groups);
    return cudaGetLastError();
}

} // namespace

bool batch_shape_supported(int R, int BY)
{
    return (R == 1 && BY == 4) || (R == 2 && BY == 4) || (R == 4 && BY == 4) || (R == 2 && BY == 2) ||
           (R == 1 && BY == 8) || (R == 0 && (BY == 8 || BY == 4));
}

template <typename T, typename C>
cudaError_t launch_batch(const BatchDesc<T, C> *descs, const int2 *work, int ntiles, int parity, int R, int BY,
                         int groups, int grid, cudaStream_t s)
{
    if (ntiles <= 0) return cudaSuccess;
    if (groups < 1) return cudaErrorInvalidValue;
    if (R == 1 && BY == 4) return launch_batch_rb<T, C, 1, 4>(descs, work, ntiles, parity, groups, grid, s);
    if (R == 2 && BY == 4) return launch_batch_rb<T, C, 2, 4>(descs, work, ntiles, parity, groups, grid, s);
    if (R == 4 && BY == 4) return launch_batch_rb<T, C, 4, 4>(descs, work, ntiles, parity, groups, grid, s);
    if (R == 2 && BY == 2) return launch_batch_rb<T, C, 2, 2>(descs, work, ntiles, parity, groups, grid, s);
    if (R == 1 && BY == 8) return launch_batch_rb<T, C, 1, 8>(descs, work, ntiles, parity, groups, grid, s);
    return cudaErrorInvalidValue;
}

cudaError_t launch_batch_tma(const BatchDesc<float, float> *descs, const LatticeMaps *maps, const int2 *work,
                             int ntiles, int parity, int groups, unsigned *err, cudaStream_t s, int issue,
                             unsigned long long wait_ns)
{
    if (ntiles <= 0) return cudaSuccess;
    if (groups < 1) return cudaErrorInvalidValue;
    // the kernel's shared-memory allowance is a per-device attribute: raise
    // it once on each device that launches it
    static std::atomic<unsigned long long> raised{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = dev < 64 ? 1ull << dev : 0ull;
    if (!bit || !(raised.load() & bit)) {
        e = cudaFuncSetAttribute(batch_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kTmaSmem);
        if (e != cudaSuccess) return e;
        raised.fetch_or(bit);
    }
    batch_tma_kernel<<<ntiles, dim3(32, 4), kTmaSmem, s>>>(descs, maps, work, parity, groups, err, issue, wait_ns);
    return cudaGetLastError();
}

template <int W>
cudaError_t launch_ring_w(const BatchDesc<float, float> *descs, const LatticeMaps *maps, const int2 *work, int ntiles,
                          int parity, int groups, unsigned *err, cudaStream_t s, int issue, unsigned long long wait_ns)
{
    // the kernel's shared-memory allowance and carveout are per-device
    // attributes: set them once on each device that launches it
    static std::atomic<unsigned long long> raised{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = dev < 64 ? 1ull << dev : 0ull;
    if (!bit || !(raised.load() & bit)) {
        e = cudaFuncSetAttribute(batch_ring_kernel<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, Ring<W>::Smem);
        // several blocks per SM need the largest shared-memory carveout
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(batch_ring_kernel<W>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     int(cudaSharedmemCarveoutMaxShared));
        if (e != cudaSuccess) return e;
        raised.fetch_or(bit);
    }
    batch_ring_kernel<W><<<ntiles, Ring<W>::Threads, Ring<W>::Smem, s>>>(descs, maps, work, parity, groups, err, issue,
                                                                         wait_ns);
    return cudaGetLastError();
}

cudaError_t launch_batch_ring(const BatchDesc<float, float> *descs, const LatticeMaps *maps, const int2 *work,
                              int ntiles, int parity, int groups, int width, unsigned *err, cudaStream_t s, int issue,
                              unsigned long long wait_ns)
{
    if (ntiles <= 0) return cudaSuccess;
    if (groups < 1) return cudaErrorInvalidValue;
    if (width == 64) return launch_ring_w<64>(descs, maps, work, ntiles, parity, groups, err, s, issue, wait_ns);
    if (width == 32) return launch_ring_w<32>(descs, maps, work, ntiles, parity, groups, err, s, issue, wait_ns);
    return cudaErrorInvalidValue;
}

template cudaError_t launch_batch<double, double>(const BatchDesc<double, double> *, const int2 *, int, int, int, int,
                                                  int, int, cudaStream_t);
template cudaError_t launch_batch<float, float>(const BatchDesc<float, float> *, const int2 *, int, int, int, int, int,
                                                int, cudaStream_t);

} // namespace lbm13
