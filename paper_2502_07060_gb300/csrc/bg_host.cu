// bg_host.cu -- bg_eval_host: evaluation with inputs and outputs in host
// memory, pipelined so that host-to-device copies, the kernel and the
// device-to-host copies of consecutive chunks overlap.
//
// The batch is cut into chunks of `chunk` points and two staging slots in
// caller-provided device memory are used alternately.  Chunk c (slot c % 2):
//   copy-in stream : wait until the kernel that last read the slot is done,
//                    copy momenta and polarisations in, record "in ready";
//   caller's stream: wait for "in ready" and for the slot's previous outputs
//                    to have left, run the kernel (bg_eval), record "done";
//   copy-out stream: wait for "done", copy amplitudes and status out,
//                    record "out done".
// Finally the caller's stream waits for both slots' "out done", so the host
// results are valid once the caller's stream reaches the call (the usual
// stream-ordered semantics).  On a failure part-way, the call returns after
// the copies it had enqueued have finished.  Host memory should be page-locked for the copies
// to overlap; pageable memory works but serialises.
//
// When all four buffers are page-locked host memory mapped into the device's
// address space and the batch's arithmetic hides the host-link traffic
// (bgi::in_place_pays: small batches, or large ones heavy enough per point,
// such as complex FP64 at n = 8), one kernel reads the inputs and writes the
// results in place instead: no copies, no chunk boundaries.
#include <cuda_runtime.h>

#include <cstdint>

#include <mutex>

#include "bg_internal.h"

namespace {

constexpr int kMaxDevices = 64;

struct HostPipe {
    bool ready = false;
    cudaStream_t s_in = nullptr, s_out = nullptr;
    cudaEvent_t in_ready[2] = {}, k_done[2] = {}, out_done[2] = {};
};

std::mutex g_pipe_mutex;              // also serialises enqueueing of calls
HostPipe g_pipe[kMaxDevices];

bg_status pipe_for(int dev, HostPipe** out) {
    HostPipe& hp = g_pipe[dev];
    if (!hp.ready) {
        bool ok = cudaStreamCreateWithFlags(&hp.s_in, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaStreamCreateWithFlags(&hp.s_out, cudaStreamNonBlocking) == cudaSuccess;
        for (int s = 0; s < 2 && ok; ++s)
            ok = cudaEventCreateWithFlags(&hp.in_ready[s], cudaEventDisableTiming) == cudaSuccess &&
                 cudaEventCreateWithFlags(&hp.k_done[s], cudaEventDisableTiming) == cudaSuccess &&
                 cudaEventCreateWithFlags(&hp.out_done[s], cudaEventDisableTiming) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            return bgi::fail(BG_ERR_CUDA, "could not create the copy streams");
        }
        hp.ready = true;
    }
    *out = &hp;
    return BG_OK;
}

size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

struct Slot {
    size_t k, eps, out, status;   // bytes per chunk of each buffer (256-rounded)
    size_t total() const { return k + eps + out + status; }
};

Slot slot_sizes(const bg_plan* pl, int64_t chunk) {
    const size_t elem = bgi::value_bytes(pl->field);
    Slot s;
    s.k = up256((size_t)chunk * pl->n * pl->d * bgi::momentum_bytes(pl->field));
    s.eps = up256((size_t)chunk * pl->n * pl->S * pl->Ds * elem);
    s.out = up256((size_t)chunk * pl->H * elem);
    s.status = up256((size_t)chunk);
    return s;
}

}  // namespace

extern "C" bg_status bg_host_staging_size(const bg_plan* plan, int64_t chunk, size_t* bytes) {
    if (!plan || !bytes || chunk < 1) return bgi::fail(BG_ERR_INVALID_ARG, "bad argument to bg_host_staging_size");
    // a chunk of a large batch runs the kernel of the whole batch, which may
    // need a workspace even where a batch of `chunk` points alone would not
    const size_t ws = bgi::workspace_bytes(plan, chunk, INT64_MAX);
    *bytes = 2 * slot_sizes(plan, chunk).total() + up256(ws);
    return BG_OK;
}

extern "C" bg_status bg_eval_host(const bg_plan* plan, int64_t E, const void* momenta, const void* eps,
                                  void* out, uint8_t* status, int64_t chunk, void* staging,
                                  size_t staging_bytes, cudaStream_t stream) {
    bgi::Range nvtx("bg_eval_host");
    if (!plan) return bgi::fail(BG_ERR_INVALID_ARG, "plan is NULL");
    if (E < 0 || chunk < 1) return bgi::fail(BG_ERR_INVALID_ARG, "E must be >= 0 and chunk >= 1");
    if (E == 0) return BG_OK;
    if (!momenta || !eps || !out || !status || !staging)
        return bgi::fail(BG_ERR_INVALID_ARG, "momenta, eps, out, status and staging must be non-NULL");
    if ((uintptr_t)staging % 256) return bgi::fail(BG_ERR_INVALID_ARG, "staging must be 256-byte aligned");
    size_t need = 0;
    bg_status st = bg_host_staging_size(plan, chunk, &need);
    if (st != BG_OK) return st;
    if (staging_bytes < need)
        return bgi::fail(BG_ERR_INVALID_ARG, "staging of %zu B needed, %zu B given", need, staging_bytes);
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return bgi::fail(BG_ERR_CUDA, "no usable current CUDA device");
    }
    if ((st = bgi::check_device_ptr(staging, "staging", dev)) != BG_OK) return st;
    for (const void* hp : {momenta, eps, (const void*)out, (const void*)status}) {
        cudaPointerAttributes attr;
        if (cudaPointerGetAttributes(&attr, hp) == cudaSuccess && attr.type == cudaMemoryTypeDevice)
            return bgi::fail(BG_ERR_INVALID_ARG, "bg_eval_host takes host buffers (got device memory)");
        cudaGetLastError();
    }

    const Slot sz = slot_sizes(plan, chunk);
    unsigned char* base = static_cast<unsigned char*>(staging);
    unsigned char* slot_base[2] = {base, base + sz.total()};
    void* ws = base + 2 * sz.total();
    size_t ws_bytes = staging_bytes - 2 * sz.total();
    const size_t elem = bgi::value_bytes(plan->field);
    const size_t k_pt = (size_t)plan->n * plan->d * bgi::momentum_bytes(plan->field);
    const size_t e_pt = (size_t)plan->n * plan->S * plan->Ds * elem;
    const size_t o_pt = (size_t)plan->H * elem;

    // Page-locked host buffers mapped into the device's address space are
    // read and written in place by one launch when the recursion's arithmetic
    // hides the host-link traffic (the workspace then sits at the start of
    // the staging buffer); otherwise the chunked copy pipeline below runs.
    if (bgi::mapped_host(momenta) && bgi::mapped_host(eps) && bgi::mapped_host(out) && bgi::mapped_host(status) &&
        bgi::in_place_pays(plan, E, (size_t)E * (k_pt + e_pt + o_pt + 1))) {
        size_t ws_need = 0;
        if ((st = bg_workspace_size(plan, E, &ws_need)) != BG_OK) return st;
        if (ws_need <= staging_bytes)
            return bgi::eval_mapped(plan, E, momenta, eps, out, status, ws_need ? staging : nullptr, ws_need,
                                    stream);
    }

    std::lock_guard<std::mutex> lock(g_pipe_mutex);
    HostPipe* hp = nullptr;
    if ((st = pipe_for(dev, &hp)) != BG_OK) return st;
    const unsigned char* kin = static_cast<const unsigned char*>(momenta);
    const unsigned char* ein = static_cast<const unsigned char*>(eps);
    unsigned char* oh = static_cast<unsigned char*>(out);
    // A failure after earlier chunks were enqueued returns only once the
    // copies already enqueued have finished (they read and write the
    // caller's buffers); kernels enqueued on `stream` stay ordered there.
    auto drained = [&](bg_status st) {
        cudaStreamSynchronize(hp->s_in);
        cudaStreamSynchronize(hp->s_out);
        cudaGetLastError();
        return st;
    };
    int64_t c = 0;
    for (int64_t start = 0; start < E; start += chunk, ++c) {
        const int s = (int)(c & 1);
        const int64_t m = (E - start < chunk) ? E - start : chunk;
        unsigned char* dk = slot_base[s];
        unsigned char* de = dk + sz.k;
        unsigned char* dout = de + sz.eps;
        uint8_t* dst = reinterpret_cast<uint8_t*>(dout + sz.out);
        if (bgi::fault(BG_FAULT_COPY))
            return drained(bgi::fail(BG_ERR_CUDA, "enqueueing chunk %lld: injected copy fault", (long long)c));
        cudaError_t err = cudaStreamWaitEvent(hp->s_in, hp->k_done[s], 0);
        if (!err) err = cudaMemcpyAsync(dk, kin + start * k_pt, m * k_pt, cudaMemcpyHostToDevice, hp->s_in);
        if (!err) err = cudaMemcpyAsync(de, ein + start * e_pt, m * e_pt, cudaMemcpyHostToDevice, hp->s_in);
        if (!err) err = cudaEventRecord(hp->in_ready[s], hp->s_in);
        if (!err) err = cudaStreamWaitEvent(stream, hp->in_ready[s], 0);
        if (!err) err = cudaStreamWaitEvent(stream, hp->out_done[s], 0);
        if (err) {
            cudaGetLastError();
            return drained(bgi::fail(BG_ERR_CUDA, "enqueueing chunk %lld: %s", (long long)c, cudaGetErrorString(err)));
        }
        if ((st = bgi::eval_part(plan, m, dk, de, dout, dst, ws, ws_bytes, stream, E * plan->H)) != BG_OK)
            return drained(st);
        err = cudaEventRecord(hp->k_done[s], stream);
        if (!err) err = cudaStreamWaitEvent(hp->s_out, hp->k_done[s], 0);
        if (!err) err = cudaMemcpyAsync(oh + start * o_pt, dout, m * o_pt, cudaMemcpyDeviceToHost, hp->s_out);
        if (!err) err = cudaMemcpyAsync(status + start, dst, m, cudaMemcpyDeviceToHost, hp->s_out);
        if (!err) err = cudaEventRecord(hp->out_done[s], hp->s_out);
        if (err) {
            cudaGetLastError();
            return drained(bgi::fail(BG_ERR_CUDA, "enqueueing chunk %lld: %s", (long long)c, cudaGetErrorString(err)));
        }
    }
    cudaError_t err = cudaStreamWaitEvent(stream, hp->out_done[0], 0);
    if (!err) err = cudaStreamWaitEvent(stream, hp->out_done[1], 0);
    if (err) {
        cudaGetLastError();
        return bgi::fail(BG_ERR_CUDA, "final wait: %s", cudaGetErrorString(err));
    }
    return BG_OK;
}
