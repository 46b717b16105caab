// bg_instances.cuh -- compile-time kernel variants and their registry rows.
//
// One row per (field, n, D, D_s, metric, table placement).  Momentum and
// polarisation dimensions are compiled for D, D_s in {4, 6, 8}; a request
// with odd d or D_s runs on the next even instance with zero padding, which
// leaves the amplitude unchanged (Sec. 2.3: lower-dimensional vectors are
// embedded by appending zeros).
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "bg_kernel.cuh"

namespace bgk {

struct KernelEntry {
    int field;          // 0 = C64, 1 = F_p (bg_field)
    int n, D, DS, metric;
    bool global_table;  // table in global scratch (true) or shared memory
    int block;          // threads per block
    int words;          // table elements per thread
    int elem_bytes;     // sizeof(T)
    const void* func;   // the __global__ function
    void (*launch)(const void* field_params, const LaunchArgs& a, dim3 grid, size_t smem,
                   cudaStream_t stream);
};

template <class F, int NLEG, int D, int DS, int M, int B, bool G>
void launch_impl(const void* fp, const LaunchArgs& a, dim3 grid, size_t smem, cudaStream_t s) {
    const F& f = *static_cast<const F*>(fp);
    bg_recursion_kernel<F, NLEG, D, DS, M, B, G><<<grid, B, smem, s>>>(f, a);
}

template <class F, int NLEG, int D, int DS, int M, int B, bool G>
KernelEntry make_entry() {
    KernelEntry e;
    e.field = F::kIsFp ? 1 : 0;
    e.n = NLEG;
    e.D = D;
    e.DS = DS;
    e.metric = M;
    e.global_table = G;
    e.block = B;
    e.words = Frame<NLEG - 1, D, DS>::WORDS;
    e.elem_bytes = sizeof(typename F::T);
    e.func = reinterpret_cast<const void*>(&bg_recursion_kernel<F, NLEG, D, DS, M, B, G>);
    e.launch = &launch_impl<F, NLEG, D, DS, M, B, G>;
    return e;
}

// Thread-block sizes: F_p with the table in shared memory uses 64 threads
// (n = 8, D_s = 6: 1000 B per thread, three blocks per SM); global-table
// variants use 128 (F_p) and 64 (C64) threads.
constexpr int kBlockFpSmem = 64;
constexpr int kBlockFpGlobal = 128;
constexpr int kBlockC64 = 64;

// Table placement per n: F_p keeps the table in shared memory up to n = 9
// and in global scratch from n = 8 (both are built for n = 8, 9 so they can
// be compared); C64 always uses global scratch (16-byte elements).
template <int NLEG, int D, int M, bool FP>
void add_dims(std::vector<KernelEntry>& v) {
    if constexpr (FP) {
        if constexpr (NLEG <= 9) v.push_back(make_entry<FieldFp, NLEG, D, D, M, kBlockFpSmem, false>());
        if constexpr (NLEG >= 8) v.push_back(make_entry<FieldFp, NLEG, D, D, M, kBlockFpGlobal, true>());
    } else {
        v.push_back(make_entry<FieldC64, NLEG, D, D, M, kBlockC64, true>());
    }
}

// (D, D_s) are compiled square, D = D_s in {4, 6, 8}; a request (d, D_s)
// runs on the smallest instance with D >= max(d, D_s), zero padded.
template <int NLEG, bool FP>
void register_n(std::vector<KernelEntry>& v) {
    add_dims<NLEG, 4, 0, FP>(v);
    add_dims<NLEG, 6, 0, FP>(v);
    add_dims<NLEG, 8, 0, FP>(v);
    add_dims<NLEG, 4, 1, FP>(v);
    add_dims<NLEG, 6, 1, FP>(v);
    add_dims<NLEG, 8, 1, FP>(v);
}

}  // namespace bgk

#define BG_DEFINE_REGISTRY(NLEG, FP, TAG)                                     \
    void bg_register_##TAG##_n##NLEG(std::vector<bgk::KernelEntry>& v) {      \
        bgk::register_n<NLEG, FP>(v);                                         \
    }
