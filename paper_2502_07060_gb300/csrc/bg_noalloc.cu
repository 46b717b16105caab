// bg_noalloc.cu -- bg_eval_noalloc: evaluation that allocates no memory.
//
// Some callers cannot call cudaMalloc: a host framework that owns the whole
// device-memory budget through its own allocator and forbids allocations by
// libraries, a latency-critical loop where cudaMalloc's implicit device-wide
// synchronisation is not acceptable, or code that runs where CUDA allocation
// calls are not permitted at all (for example a host function enqueued on a
// stream).  bg_eval needs such callers to provide a device workspace; this
// entry point instead runs the global-table kernel on a scratch table that
// lives in this file as a statically sized __device__ array, so the call
// itself allocates nothing.
//
// The array is kNoAllocScratchBytes (64 MiB) per device.  Every GPU on which
// the library's module is loaded holds it until the process exits.  Host code
// must not pass the array's name to a kernel (on the host it names a stand-in
// object, not device memory): its device address is obtained once per device
// with cudaGetSymbolAddress, with that device current, during the first call
// on that device.  That first call should therefore come before any stream
// capture begins.  The cached address belongs to the device's primary
// context: after cudaDeviceReset it is stale, and the library must not be
// used again in that process.  All calls share the array and it keeps the previous call's
// contents; the kernel writes every table entry before reading it, so nothing
// needs clearing, but calls whose kernels overlap on the GPU (different
// streams, or without ordering between them) race on the array.
#include <cuda_runtime.h>

#include <mutex>

#include "bg_internal.h"

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(64) << 20;
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char bg_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_setup_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on device `dev` (the current device).
bg_status scratch_address(int dev, void** out) {
    if (dev < 0 || dev >= kMaxDevices) return bgi::fail(BG_ERR_CUDA, "device index %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        cudaError_t err = cudaGetSymbolAddress(&p, bg_noalloc_scratch);
        if (err != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return bgi::fail(BG_ERR_CUDA, "cudaGetSymbolAddress of the scratch array failed: %s",
                             cudaGetErrorString(err));
        }
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return BG_OK;
}

}  // namespace

extern "C" bg_status bg_eval_noalloc(const bg_plan* plan, int64_t E, const void* momenta,
                                     const void* eps, void* out, uint8_t* status,
                                     cudaStream_t stream) {
    bgi::Range nvtx("bg_eval_noalloc");
    if (!plan) return bgi::fail(BG_ERR_INVALID_ARG, "plan is NULL");
    if (E < 0) return bgi::fail(BG_ERR_INVALID_ARG, "E = %lld < 0", (long long)E);
    if (E == 0) return BG_OK;
    if (!momenta || !eps || !out)
        return bgi::fail(BG_ERR_INVALID_ARG, "momenta, eps and out must be non-NULL");
    if (plan->all_states)
        return bgi::fail(BG_ERR_UNSUPPORTED, "all-assignment plans (assign == NULL, H = S^n) are not supported here");
    if (E > (int64_t(1) << 40) / plan->H)
        return bgi::fail(BG_ERR_INVALID_ARG, "E * n_assign exceeds the maximum of 2^40 work items");
    const size_t elem = bgi::value_bytes(plan->field), kelem = bgi::momentum_bytes(plan->field);
    if (((uintptr_t)eps | (uintptr_t)out) % elem || (uintptr_t)momenta % kelem)
        return bgi::fail(BG_ERR_INVALID_ARG, "momenta, eps and out must be aligned to their element sizes "
                         "(%zu, %zu, %zu bytes)", kelem, elem, elem);
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return bgi::fail(BG_ERR_CUDA, "no current CUDA device");
    }
    if (plan->d_assign && dev != plan->device)
        return bgi::fail(BG_ERR_CUDA, "plan was created on device %d, current device is %d", plan->device, dev);
    bg_status st;
    if ((st = bgi::check_device_ptr(momenta, "momenta", dev)) != BG_OK) return st;
    if ((st = bgi::check_device_ptr(eps, "eps", dev)) != BG_OK) return st;
    if ((st = bgi::check_device_ptr(out, "out", dev)) != BG_OK) return st;
    if (status && (st = bgi::check_device_ptr(status, "status", dev)) != BG_OK) return st;

    // Small batches take the lane-group kernel as bg_eval does; its table is
    // in shared memory, so it needs no scratch at all.
    if (bgi::uses_lanes(plan, E * plan->H)) {
        if (bgi::fault(BG_FAULT_LAUNCH)) return bgi::fail(BG_ERR_CUDA, "launch failed: injected fault");
        return bgi::launch_lanes(plan, E, momenta, eps, out, status, dev, stream, E * plan->H);
    }
    // The compact kernel with its table in global memory, same dimensions and
    // metric as the plan's own kernel.
    const int D = bgi::round_dim(plan->d), DS = bgi::round_dim(plan->Ds);
    const bgk::KernelEntry* e = nullptr;
    for (const auto& k : bgi::registry())
        if (k.global_table && !k.split && k.field == (int)plan->field && k.D == D &&
            k.DS == DS && k.metric == (int)plan->metric && k.mixed == plan->entry->mixed)
            e = &k;
    if (!e) return bgi::fail(BG_ERR_UNSUPPORTED, "no global-table kernel for this plan");
    const bgk::Geometry geo{plan->n - 1};
    const size_t per_block = (size_t)geo.words(D, DS) * e->block * e->elem_bytes;
    if (per_block > kNoAllocScratchBytes)
        return bgi::fail(BG_ERR_UNSUPPORTED, "one block needs %zu B of scratch, above the maximum of %zu B",
                         per_block, kNoAllocScratchBytes);

    void* scratch = nullptr;
    if ((st = scratch_address(dev, &scratch)) != BG_OK) return st;

    int occ = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, e->func, e->block, 0) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return bgi::fail(BG_ERR_CUDA, "occupancy query failed");
    }
    const int64_t items = E * plan->H;
    int64_t blocks = (items + e->block - 1) / e->block;
    const int64_t resident = (int64_t)(occ > 0 ? occ : 1) * sms;
    const int64_t fit = (int64_t)(kNoAllocScratchBytes / per_block);
    if (blocks > resident) blocks = resident;
    if (blocks > fit) blocks = fit;

    if (bgi::fault(BG_FAULT_LAUNCH)) return bgi::fail(BG_ERR_CUDA, "launch failed: injected fault");
    bgk::CompactArgs a;
    a.E = E; a.H = plan->H; a.S = plan->S; a.n = plan->n;
    a.d_in = plan->d; a.ds_in = plan->Ds;
    a.k = momenta; a.eps = eps; a.out = out; a.status = status;
    a.assign = plan->d_assign; a.ws = scratch;
    a.four_d_legs = plan->four_d_legs;
    a.violation = bgi::violation_word(dev);
    e->launch(bgi::compact_params(plan), &a, dim3((unsigned)blocks), 0, stream);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return bgi::fail(BG_ERR_CUDA, "launch failed: %s", cudaGetErrorString(err));
    return BG_OK;
}
