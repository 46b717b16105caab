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
#include <cstring>

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

// Probe of the host link as the kernels use it when they read page-locked
// host memory in place: each thread reads whole rows of 384 bytes (one point's
// F_p inputs at n = 8, d = 6) with streaming 16-byte loads, consecutive
// threads consecutive rows.  `sink` keeps the loads from being removed.
constexpr int kProbeRowVec = 24;            // 16-byte vectors per row
__global__ void host_link_probe(const uint4* __restrict__ rows, int64_t n_rows, unsigned* sink) {
    unsigned acc = 0;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n_rows; r += (int64_t)gridDim.x * blockDim.x) {
        const uint4* q = rows + r * kProbeRowVec;
#pragma unroll 4
        for (int v = 0; v < kProbeRowVec; ++v) {
            const uint4 x = __ldcs(q + v);
            acc ^= x.x + x.y + x.z + x.w;
        }
    }
    if (acc == 0x9e3779b9u) sink[0] = acc;  // practically never taken
}

// Bytes per second of in-place reads over the host link, measured on the
// current device: 32 MiB of page-locked memory read twice by four resident
// blocks of 128 threads per SM (the compute kernels' residency), timed with
// events after one warm-up pass.  0 when the probe cannot run.
double probe_mapped_read_rate(int dev) {
    constexpr size_t kBytes = size_t(32) << 20;
    const int64_t n_rows = (int64_t)(kBytes / (kProbeRowVec * sizeof(uint4)));
    void* host = nullptr;
    unsigned* sink = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    double rate = 0;
    int sms = 0;
    void* dptr = nullptr;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
        cudaHostAlloc(&host, kBytes, cudaHostAllocMapped) == cudaSuccess &&
        cudaHostGetDevicePointer(&dptr, host, 0) == cudaSuccess && cudaMalloc(&sink, sizeof(unsigned)) == cudaSuccess &&
        cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess &&
        cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
        memset(host, 1, kBytes);
        const int blocks = 4 * sms;
        host_link_probe<<<blocks, 128, 0, st>>>(static_cast<const uint4*>(dptr), n_rows, sink);
        cudaEventRecord(e0, st);
        for (int rep = 0; rep < 2; ++rep)
            host_link_probe<<<blocks, 128, 0, st>>>(static_cast<const uint4*>(dptr), n_rows, sink);
        cudaEventRecord(e1, st);
        float ms = 0;
        if (cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms > 0)
            rate = 2.0 * (double)kBytes / (ms * 1e-3);
    }
    cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (sink) cudaFree(sink);
    if (host) cudaFreeHost(host);
    cudaGetLastError();
    return rate;
}

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

namespace bgi {

// Measured once per device (the first large in-place decision, or a server's
// creation), then cached.  The probe's cudaFreeHost waits for the device, so
// the first call may wait for work already queued.
double mapped_read_rate() {
    static std::mutex mu;
    static bool done[kMaxDevices] = {};
    static double rate[kMaxDevices] = {};
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return kMappedReadRateDefault;
    }
    std::lock_guard<std::mutex> lk(mu);
    if (!done[dev]) {
        done[dev] = true;
        const double r = probe_mapped_read_rate(dev);
        rate[dev] = r > 0 ? r : kMappedReadRateDefault;
        log("device %d: in-place reads over the host link %.1f GB/s (%s)", dev, rate[dev] / 1e9,
            r > 0 ? "measured" : "probe failed, default");
    }
    return rate[dev];
}

}  // namespace bgi

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
