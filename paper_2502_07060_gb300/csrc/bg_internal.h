// bg_internal.h -- definitions shared by the translation units of libbg.so
// (not part of the public C-ABI).
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstdint>
#include <vector>

#include "../../include/bg.h"
#include "bg_instances.cuh"
#include "bg_lanes.cuh"
#include "bg_states.cuh"

struct bg_plan {
    int n, d, Ds;
    bg_field field;
    uint32_t p;
    bg_metric metric;
    int S, H;
    std::vector<uint8_t> assign;      // host copy [H][n]
    uint32_t four_d_legs = 0;         // bit l: leg l four-dimensional (mixed plans)
    uint8_t* d_assign = nullptr;      // device copy when H > 1
    int device = -1;                  // device of d_assign / attribute setup
    const bgk::KernelEntry* entry = nullptr;
    int words = 0;                    // table elements per thread (or per thread in global
                                      // scratch for the split placement)
    bgk::FpOps fpo{};                 // field constants of the kernels
    bgk::C64Ops c64o{};
    bgk::C64ROps c64ro{};
    int sm_count = 0;
    int blocks_per_sm = 0;
    size_t smem_bytes = 0;            // dynamic shared memory per block
    // small batches: one point per group of L lanes (bg_lanes.cuh), used by
    // bg_eval for at most lanes_max_items work items
    const bgk::LanesEntry* lentry = nullptr;
    size_t lanes_smem = 0;
    int lanes_blocks_per_sm = 0;
    int64_t lanes_max_items = 0;
    // the same kernel with one point per team (a warp of groups), for at most
    // team_max_items work items (checked before lanes_max_items)
    const bgk::LanesEntry* tentry = nullptr;
    size_t team_smem = 0;
    int team_blocks_per_sm = 0;
    int64_t team_max_items = 0;
    // all S^n assignments with sub-current reuse (assign == NULL, H == S^n > 1)
    bool all_states = false;
    const bgk::StatesEntry* sentry = nullptr;
    bgk::StatesGeometry sgeo{};
    bool states_global = false;       // states table in global scratch
};

namespace bgi {
// True when the current operation at `site` (a bg_fault_site) is one that
// bg_debug_inject_fault asked to fail; counts the operation either way.
bool fault(int site);

// Device word receiving the first out-of-range table index of a launch in
// builds compiled with BG_CHECKED (null otherwise): a static __device__
// variable whose address is looked up once per device -- nothing allocated.
unsigned long long* violation_word(int device);

// NVTX range around an entry point (visible in Nsight; no cost without a tool)
struct Range {
    explicit Range(const char* name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range&) = delete;
    Range& operator=(const Range&) = delete;
};

const std::vector<bgk::KernelEntry>& registry();
const std::vector<bgk::StatesEntry>& states_registry();
const std::vector<bgk::LanesEntry>& lanes_registry();
bg_status fail(bg_status s, const char* fmt, ...);
// One line on stderr, prefixed "bg: ", when the environment variable BG_LOG
// is set to anything but "" or "0" (read once); otherwise nothing.
void log(const char* fmt, ...);
bg_status check_device_ptr(const void* ptr, const char* what, int device);
bg_status check_kernel_ptr(const void* ptr, const char* what, int device, bool mapped_host_ok);
// bg_eval that also takes page-locked host buffers mapped at the same address
// (momenta, eps, out, status; the workspace stays device memory): the kernel
// reads and writes them over the host link.
bg_status eval_mapped(const bg_plan* plan, int64_t E, const void* momenta, const void* eps, void* out,
                      uint8_t* status, void* workspace, size_t workspace_bytes, cudaStream_t stream);
// bg_eval on part of a larger batch of batch_items work items (a chunk of
// bg_eval_host): the kernel is the one bg_eval takes for the whole batch, so
// every chunk gives the whole batch's values.
bg_status eval_part(const bg_plan* plan, int64_t E, const void* momenta, const void* eps, void* out,
                    uint8_t* status, void* workspace, size_t workspace_bytes, cudaStream_t stream,
                    int64_t batch_items);
// Whether a batch of select_items work items runs on the plan's lane-group
// kernel (one point per group or per team), and the device workspace for E
// points when the kernel is chosen by select_items (bg_workspace_size:
// select_items = E * H).
bool uses_lanes(const bg_plan* plan, int64_t select_items);
// One launch of the plan's lane-group kernel on E points (checked
// arguments), one point per team when select_items allows it.
bg_status launch_lanes(const bg_plan* plan, int64_t E, const void* momenta, const void* eps, void* out,
                       uint8_t* status, int dev, cudaStream_t stream, int64_t select_items);
size_t workspace_bytes(const bg_plan* plan, int64_t E, int64_t select_items);
// True when `p` is page-locked host memory mapped into the device's address
// space at the same address (the kernels can read and write it directly).
bool mapped_host(const void* p);
// Whether kernels should read a batch of E points from mapped host memory in
// place rather than have it copied in first: always for batches of at most
// kInPlaceBytes of host data (latency dominates), and otherwise when the
// recursion's arithmetic per point hides the traffic over the host link.
constexpr size_t kInPlaceBytes = size_t(64) << 20;
bool in_place_pays(const bg_plan* plan, int64_t E, size_t host_bytes);
bool in_place_pays_for(int field, int n, int d, int Ds, int H, int64_t E, size_t host_bytes, double sm_scale,
                       double link_bytes_per_s);
// Bytes per second of the host-link probe, reading page-locked host memory in
// place on the current device (measured once, bg_host.cu); the default is the
// figure measured on a GB300 host.
constexpr double kMappedReadRateDefault = 1.35e11;
double mapped_read_rate();
double ops_per_amplitude(int n, int d, int D);
int round_dim(int x);
bg_status ensure_smem_limit(const void* func, int device, size_t bytes);

// bytes of one polarisation / amplitude element (uint32 residue or double2)
inline size_t value_bytes(bg_field f) { return f == BG_FIELD_FP ? 4 : 16; }
// bytes of one momentum component (uint32, double2, or double for real momenta)
inline size_t momentum_bytes(bg_field f) {
    return f == BG_FIELD_FP ? 4 : f == BG_FIELD_C64_REAL ? 8 : 16;
}
// field constants passed to the compact kernel of the plan's field
inline const void* compact_params(const bg_plan* pl) {
    return pl->field == BG_FIELD_FP ? (const void*)&pl->fpo
         : pl->field == BG_FIELD_C64_REAL ? (const void*)&pl->c64ro : (const void*)&pl->c64o;
}
inline const char* field_name(bg_field f) {
    return f == BG_FIELD_FP ? "fp" : f == BG_FIELD_C64_REAL ? "c64_real" : "c64";
}
}  // namespace bgi
