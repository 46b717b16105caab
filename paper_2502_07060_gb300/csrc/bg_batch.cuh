// bg_batch.cuh -- persistent kernel for a batch of uneven groups: points of
// different n, d, D_s and metric (one number type per kernel) in one launch.
//
// The batch is cut into tiles of consecutive work items of one group.  A
// group runs one work item per thread, or -- when the configuration asks for
// it and the group is small -- one per group of 4 or 8 lanes (the lane-group
// body of bg_lanes.cuh, on the same table region).  Tiles
// are ordered by decreasing cost per point (longest-processing-time first, so
// the cheap tiles fill the tail) and handed out by one atomic counter: each
// resident block takes the next tile, runs the recursion of bg_compact.cuh on
// its items (the (D, D_s, metric) body the group needs), and repeats until the
// queue is empty.  The tables of a block live in a global scratch region sized
// for the largest group of the batch; a one-item-per-thread item drops its
// table lines from L2 when it is done.  Blocks never wait for one another.
#pragma once
#include <cstdint>

#include "bg_compact.cuh"
#include "bg_lanes.cuh"

namespace bgk {

// (D, D_s) pairs compiled for the batch kernel, and the variant index
// variant = 2 * pair + metric, plus kBatchVariants for complex groups with
// real momenta (run by the complex kernel).
constexpr int kBatchPairs = 6;
constexpr int kBatchVariants = 2 * kBatchPairs;
__host__ __device__ constexpr int batch_pair_index(int D, int DS) {
    return D == 4 ? (DS == 4 ? 0 : DS == 6 ? 1 : 2) : D == 6 ? (DS == 6 ? 3 : 4) : 5;
}

struct BatchGroup {
    CompactArgs args;       // n, E, H, S, dims, device buffers (ws unused)
    int variant;            // 2 * batch_pair_index(D, D_s) + metric (+ kBatchVariants)
    int lanes;              // 0: one work item per thread; 4 or 8: per group of lanes
    FpOps fp;               // Montgomery constants (F_p groups)
};

struct BatchTile {
    int group;
    int count;              // work items in the tile
    int64_t first;          // first work item (point * H + assignment)
};

struct BatchArgs {
    const BatchGroup* groups;
    const BatchTile* tiles;
    int n_tiles;
    int* counter;           // next tile; zero before the launch
    void* tables;           // per-block table regions
    int words;              // table elements per thread (largest group)
};

template <class F>
__device__ __forceinline__ F batch_field(const BatchGroup& g);
template <>
__device__ __forceinline__ FpOps batch_field<FpOps>(const BatchGroup& g) { return g.fp; }
template <>
__device__ __forceinline__ C64Ops batch_field<C64Ops>(const BatchGroup&) { return C64Ops{}; }

// One (D, D_s, metric) body as a function of its own (not inlined): each body
// gets its own register allocation instead of the union of all of them
template <class F, int D, int DS, int M, int BLOCK>
__device__ __noinline__ void batch_point(const F f, const CompactArgs* a, typename F::T* tab, int64_t u) {
    bg_point<F, D, DS, M, BLOCK>(f, *a, tab, u);
    // the item's table is dead: drop its lines from L2 (bg_compact.cuh)
    const Geometry g{a->n - 1};
    discard_point_table<F, D, DS, BLOCK, true>(g, tab, tab + g.off_k(DS) * BLOCK);
}

template <class F, int BLOCK>
__device__ __forceinline__ void batch_dims(const F& f, const CompactArgs& a, int variant,
                                           typename F::T* tab, int64_t u) {
    switch (variant) {
        case 0: batch_point<F, 4, 4, 0, BLOCK>(f, &a, tab, u); break;
        case 1: batch_point<F, 4, 4, 1, BLOCK>(f, &a, tab, u); break;
        case 2: batch_point<F, 4, 6, 0, BLOCK>(f, &a, tab, u); break;
        case 3: batch_point<F, 4, 6, 1, BLOCK>(f, &a, tab, u); break;
        case 4: batch_point<F, 4, 8, 0, BLOCK>(f, &a, tab, u); break;
        case 5: batch_point<F, 4, 8, 1, BLOCK>(f, &a, tab, u); break;
        case 6: batch_point<F, 6, 6, 0, BLOCK>(f, &a, tab, u); break;
        case 7: batch_point<F, 6, 6, 1, BLOCK>(f, &a, tab, u); break;
        case 8: batch_point<F, 6, 8, 0, BLOCK>(f, &a, tab, u); break;
        case 9: batch_point<F, 6, 8, 1, BLOCK>(f, &a, tab, u); break;
        case 10: batch_point<F, 8, 8, 0, BLOCK>(f, &a, tab, u); break;
        default: batch_point<F, 8, 8, 1, BLOCK>(f, &a, tab, u); break;
    }
}

template <class F, int BLOCK>
__device__ __forceinline__ void batch_item(const F& f, const CompactArgs& a, int variant,
                                           typename F::T* tab, int64_t u) {
    if constexpr (!F::kIsFp) {
        if (variant >= kBatchVariants) {         // same table element type (double2)
            batch_dims<C64ROps, BLOCK>(C64ROps{}, a, variant - kBatchVariants, tab, u);
            return;
        }
    }
    batch_dims<F, BLOCK>(f, a, variant, tab, u);
}

// The lane-group body (bg_lanes.cuh) for a group of small size: one work
// item per group of L lanes, the lane table in the block's global region.
template <class F, int L, int M, int BLOCK>
__device__ __noinline__ void batch_lanes_point(const F f, const CompactArgs* a, unsigned char* tab, int64_t u) {
    lanes_point<F, L, M, BLOCK>(f, *a, tab, u);
}

template <class F, int BLOCK>
__device__ __forceinline__ void batch_lanes_dims(const F& f, const CompactArgs& a, int L, int metric,
                                                 unsigned char* tab, int64_t u) {
    if (L == 4) {
        if (metric) batch_lanes_point<F, 4, 1, BLOCK>(f, &a, tab, u);
        else batch_lanes_point<F, 4, 0, BLOCK>(f, &a, tab, u);
    } else {
        if (metric) batch_lanes_point<F, 8, 1, BLOCK>(f, &a, tab, u);
        else batch_lanes_point<F, 8, 0, BLOCK>(f, &a, tab, u);
    }
}

template <class F, int BLOCK>
__device__ __forceinline__ void batch_lanes_item(const F& f, const CompactArgs& a, int variant, int L,
                                                 unsigned char* tab, int64_t u) {
    if constexpr (!F::kIsFp) {
        if (variant >= kBatchVariants) {
            batch_lanes_dims<C64ROps, BLOCK>(C64ROps{}, a, L, (variant - kBatchVariants) & 1, tab, u);
            return;
        }
    }
    batch_lanes_dims<F, BLOCK>(f, a, L, variant & 1, tab, u);
}

// MINB: resident blocks per SM the kernel is built for.  The bodies are
// functions of their own, so the kernel's register count covers the largest
// of them: built for one block (up to 255 registers) no body spills much;
// built for four F_p blocks (at most 128 registers) some bodies spill but
// twice as many warps hide the table loads' latency.
template <class F, int BLOCK, int MINB>
__global__ void __launch_bounds__(BLOCK, MINB) bg_batch_kernel(const BatchArgs a) {
    using T = typename F::T;
    __shared__ int s_tile;
    T* tab = reinterpret_cast<T*>(a.tables) + static_cast<size_t>(blockIdx.x) * a.words * BLOCK;
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(a.counter, 1);
        __syncthreads();
        const int ti = s_tile;
        __syncthreads();                       // every thread has read s_tile
        if (ti >= a.n_tiles) break;
        const BatchTile td = a.tiles[ti];
        const BatchGroup& gd = a.groups[td.group];
        const F f = batch_field<F>(gd);
        const int variant = gd.variant;
        if (gd.lanes) {                        // groups of L lanes share one work item
            const int L = gd.lanes;
            for (int k = threadIdx.x / L; k < td.count; k += BLOCK / L)
                batch_lanes_item<F, BLOCK>(f, gd.args, variant, L, reinterpret_cast<unsigned char*>(tab),
                                           td.first + k);
        } else {
            for (int k = threadIdx.x; k < td.count; k += BLOCK)
                batch_item<F, BLOCK>(f, gd.args, variant, tab, td.first + k);
        }
    }
}

// The batch kernels are instantiated in translation units of their own
// (bg_batch_fp.cu, bg_batch_c64.cu): each holds the recursion body of every
// (D, D_s, metric), and compiled apart they build in parallel.  F_p has two
// builds: `wide` for one resident block per SM and up (two fit), the other
// for four (kFpNarrowBlocks); complex has one (four 64-thread blocks fit).
constexpr int kBlockFpBatch = 128;
constexpr int kBlockC64Batch = 64;
constexpr int kFpNarrowBlocks = 4;
const void* batch_kernel_fp(bool wide);   // the __global__ functions (occupancy queries)
const void* batch_kernel_c64();
void launch_batch_fp(const BatchArgs& a, int blocks, bool wide, cudaStream_t s);
void launch_batch_c64(const BatchArgs& a, int blocks, cudaStream_t s);

}  // namespace bgk
