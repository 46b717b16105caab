// bg_instances.cuh -- compile-time kernel variants and their registry rows.
//
// One row per (field, D, D_s, metric, table placement, mixed); n is a
// run-time parameter of every kernel.  Momentum and
// polarisation dimensions are compiled for D, D_s in {4, 6, 8}; a request
// with odd d or D_s runs on the next even instance with zero padding, which
// leaves the amplitude unchanged (Sec. 2.3: lower-dimensional vectors are
// embedded by appending zeros).
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "bg_compact.cuh"

namespace bgk {

struct KernelEntry {
    int field;          // bg_field: 0 = C64, 1 = F_p, 2 = C64 with real momenta
    int D, DS, metric;
    bool global_table;  // (part of the) table in global scratch: the workspace is needed
    bool split;         // currents in global scratch, the rest in shared memory
    bool mixed;         // evaluates ranges of four-dimensional legs with four components
    int block;          // threads per block
    int elem_bytes;     // sizeof(T)
    const void* func;   // the __global__ function
    // launch(field params, CompactArgs, grid, smem, stream)
    void (*launch)(const void* field_params, const void* args, dim3 grid, size_t smem,
                   cudaStream_t stream);
};

template <class F, int D, int DS, int M, int B, int G, bool X>
void launch_compact(const void* fp, const void* args, dim3 grid, size_t smem, cudaStream_t s) {
    const F& f = *static_cast<const F*>(fp);
    bg_compact_kernel<F, D, DS, M, B, G, X><<<grid, B, smem, s>>>(f, *static_cast<const CompactArgs*>(args));
}

template <class F, int D, int DS, int M, int B, int G, bool X = false>
KernelEntry make_compact() {
    KernelEntry e;
    e.field = F::kField;
    e.D = D;
    e.DS = DS;
    e.metric = M;
    e.global_table = G != kPlaceShared;
    e.split = G == kPlaceSplit;
    e.mixed = X;
    e.block = B;
    e.elem_bytes = sizeof(typename F::T);
    e.func = reinterpret_cast<const void*>(&bg_compact_kernel<F, D, DS, M, B, G, X>);
    e.launch = &launch_compact<F, D, DS, M, B, G, X>;
    return e;
}

// Compact kernels: every (D, D_s) pair with D <= D_s in {4, 6, 8}, both
// metrics; F_p with shared or global table, the complex fields (complex or
// real momenta) with global table.
constexpr int kBlockFpCompactSmem = 64;
constexpr int kBlockFpCompactGlobal = 128;
constexpr int kBlockC64Compact = 64;

// Mixed-dimension variants (plans with four-dimensional legs) exist where a
// current has more than four components: F_p with shared or global table,
// the complex fields with global table.
template <class F, int D, int DS, int M>
void add_compact_dims(std::vector<KernelEntry>& v) {
    if constexpr (F::kIsFp) {
        v.push_back(make_compact<F, D, DS, M, kBlockFpCompactSmem, kPlaceShared>());
        v.push_back(make_compact<F, D, DS, M, kBlockFpCompactGlobal, kPlaceGlobal>());
        v.push_back(make_compact<F, D, DS, M, kBlockFpCompactGlobal, kPlaceSplit>());
        if constexpr (DS > 4) {
            v.push_back(make_compact<F, D, DS, M, kBlockFpCompactSmem, kPlaceShared, true>());
            v.push_back(make_compact<F, D, DS, M, kBlockFpCompactGlobal, kPlaceGlobal, true>());
        }
    } else {
        v.push_back(make_compact<F, D, DS, M, kBlockC64Compact, kPlaceGlobal>());
        if constexpr (DS > 4) v.push_back(make_compact<F, D, DS, M, kBlockC64Compact, kPlaceGlobal, true>());
    }
}

template <class F, int D, int DS>
void register_compact(std::vector<KernelEntry>& v) {
    add_compact_dims<F, D, DS, 0>(v);
    add_compact_dims<F, D, DS, 1>(v);
}

}  // namespace bgk

#define BG_DEFINE_COMPACT(D, DS, OPS, TAG)                                    \
    void bg_register_compact_##TAG##_##D##_##DS(std::vector<bgk::KernelEntry>& v) { \
        bgk::register_compact<bgk::OPS, D, DS>(v);                            \
    }
