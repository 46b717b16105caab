// bg_internal.h -- definitions shared by the translation units of libbg.so
// (not part of the public C-ABI).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "../../include/bg.h"
#include "bg_instances.cuh"

struct bg_plan {
    int n, d, Ds;
    bg_field field;
    uint32_t p;
    bg_metric metric;
    int S, H;
    std::vector<uint8_t> assign;      // host copy [H][n]
    uint8_t* d_assign = nullptr;      // device copy when H > 1
    int device = -1;                  // device of d_assign / attribute setup
    const bgk::KernelEntry* entry = nullptr;
    int words = 0;                    // table elements per thread
    bgk::FieldFp fp{};                // unrolled kernels
    bgk::FieldC64 c64{};
    bgk::FpOps fpo{};                 // compact kernels
    bgk::C64Ops c64o{};
    int sm_count = 0;
    int blocks_per_sm = 0;
    size_t smem_bytes = 0;            // dynamic shared memory per block
};

namespace bgi {
const std::vector<bgk::KernelEntry>& registry();
bg_status fail(bg_status s, const char* fmt, ...);
bg_status check_device_ptr(const void* ptr, const char* what, int device);
int round_dim(int x);
bg_status ensure_smem_limit(const void* func, int device, size_t bytes);
}  // namespace bgi
