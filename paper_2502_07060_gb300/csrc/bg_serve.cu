// bg_serve.cu -- a request server for evaluation requests of mixed size and
// configuration (the request stream of a reconstruction or Monte Carlo
// consumer of these amplitudes).
//
// Design:
//   * one device arena of `budget` bytes, allocated at bg_serve_create and
//     sub-allocated first-fit (256-byte granules) for each admitted request:
//     its inputs, outputs and kernel workspace;
//   * a dispatcher thread admits pending requests while memory and a stream
//     slot are free -- continuously, not in rounds: a request that arrives
//     while others run is admitted as soon as a slot and memory free up, and
//     its copies and kernel overlap with the work already on the device;
//   * admission is first-come-first-served, except that a request that does
//     not fit may be overtaken by later ones until it has waited kStarveMs,
//     after which nothing overtakes it;
//   * each admitted request runs on its own stream slot: host->device copies,
//     one bg_eval launch, device->host copies, then a host function (run by
//     the CUDA driver, no CUDA calls in it) that marks the slot finished;
//     buffers already in device memory (a resident pool of momenta and
//     states, outputs kept on the device) are used in place, with no copy and
//     no arena bytes, and so are page-locked host buffers mapped into the
//     device's address space: the kernel reads its inputs and writes its
//     results over the host link.  A copy-engine transfer costs tens of
//     microseconds before its first byte moves, small copies queue behind
//     large ones and a staged request holds its slot through its copy, while
//     the kernels read each input once.  Pageable host buffers, and mapped
//     ones of large requests whose kernels the link would bound
//     (bgi::in_place_pays), are staged through the arena by copies;
//   * the dispatcher enqueues copies and kernels with the server mutex
//     released, so the completion host functions never wait on it;
//   * each slot records an event after its request's work; when the host
//     function reports the slot finished, the dispatcher queries that event,
//     so an asynchronous error of the request's copies or kernel marks the
//     request failed (BG_ERR_CUDA from its wait) instead of done;
//   * bg_serve_wait blocks on a condition variable with a deadline and
//     returns BG_ERR_TIMEOUT when the request is not done by then.  Several
//     threads may wait on one ticket: each gets the request's result, and the
//     request is freed when the last of them returns.
#include <cuda_runtime.h>

#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "bg_internal.h"

namespace {

constexpr size_t kGranule = 256;
constexpr double kStarveMs = 50.0;

using Clock = std::chrono::steady_clock;

size_t up_granule(size_t x) { return (x + kGranule - 1) & ~(kGranule - 1); }

// First-fit allocator over [0, size) with coalescing (host bookkeeping only).
class Arena {
public:
    explicit Arena(size_t size) { free_[0] = size; }
    bool alloc(size_t bytes, size_t* off) {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes, start = it->first + bytes;
                free_.erase(it);
                if (rest) free_[start] = rest;
                used_ += bytes;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t used() const { return used_; }

private:
    std::map<size_t, size_t> free_;
    size_t used_ = 0;
};

enum class State { Pending, Running, Done, Failed };

struct Request {
    uint64_t id;
    const bg_plan* plan;
    int64_t E;
    const void* k;
    const void* eps;
    void* out;
    uint8_t* status;
    // buffers used in place (device memory, or mapped page-locked host
    // memory) rather than staged through the arena
    bool k_dev = false, e_dev = false, out_dev = false, st_dev = false;
    bool mapped = false;                     // some buffer in place is mapped host memory
    size_t bytes_k, bytes_e, bytes_o, bytes_s, bytes_ws, total;
    Clock::time_point submitted;
    State state = State::Pending;
    bg_status result = BG_OK;
    size_t off = 0;
    int slot = -1;
    int waiters = 0;                         // threads inside bg_serve_wait on this ticket
    bool retired = false;                    // finished and removed from the ticket map
};

}  // namespace

struct bg_server {
    int device = -1;
    size_t budget = 0;
    unsigned char* arena_mem = nullptr;
    Arena* arena = nullptr;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> slot_event;     // recorded after each request's work
    std::vector<Request*> slot_req;          // request running on each slot (or null)
    std::vector<int> slot_done;              // set by the host function
    std::mutex mu;
    std::condition_variable cv_work;         // dispatcher: new request or slot finished
    std::condition_variable cv_done;         // waiters
    std::deque<Request*> pending;
    std::map<uint64_t, Request*> requests;   // all not yet collected
    uint64_t next_id = 1;
    bool stop = false;
    std::thread thread;
    // statistics
    uint64_t n_submitted = 0, n_completed = 0;
    size_t peak_used = 0;
};

namespace {

struct SlotDone {
    bg_server* srv;
    int slot;
};

void CUDART_CB slot_finished(void* arg) {
    SlotDone* sd = static_cast<SlotDone*>(arg);
    {
        std::lock_guard<std::mutex> lk(sd->srv->mu);
        sd->srv->slot_done[sd->slot] = 1;
    }
    sd->srv->cv_work.notify_one();
    delete sd;
}

// Enqueue the copies, the kernel and the completion callback of r on its slot.
bg_status launch_request(bg_server* s, Request* r) {
    cudaStream_t st = s->streams[r->slot];
    unsigned char* base = s->arena_mem + r->off;
    // arena layout: staged momenta, eps, outputs, status, then the workspace;
    // device-resident buffers take no arena bytes and are used in place
    unsigned char* ak = base;
    unsigned char* ae = ak + r->bytes_k;
    unsigned char* aout = ae + r->bytes_e;
    unsigned char* ast = aout + r->bytes_o;
    unsigned char* ws = ast + r->bytes_s;
    const void* dk = r->k_dev ? r->k : ak;
    const void* de = r->e_dev ? r->eps : ae;
    void* dout = r->out_dev ? r->out : aout;
    uint8_t* dst = r->st_dev ? r->status : reinterpret_cast<uint8_t*>(ast);
    const size_t elem = bgi::value_bytes(r->plan->field);
    const size_t nk = (size_t)r->E * r->plan->n * r->plan->d * bgi::momentum_bytes(r->plan->field);
    const size_t ne = (size_t)r->E * r->plan->n * r->plan->S * r->plan->Ds * elem;
    const size_t no = (size_t)r->E * r->plan->H * elem;
    bgi::Range nvtx("bg_serve_request");
    if (bgi::fault(BG_FAULT_COPY)) return BG_ERR_CUDA;
    cudaError_t err = cudaSuccess;
    if (!r->k_dev) err = cudaMemcpyAsync(ak, r->k, nk, cudaMemcpyHostToDevice, st);
    if (!err && !r->e_dev) err = cudaMemcpyAsync(ae, r->eps, ne, cudaMemcpyHostToDevice, st);
    if (err) { cudaGetLastError(); return BG_ERR_CUDA; }
    bg_status bs = r->mapped
        ? bgi::eval_mapped(r->plan, r->E, dk, de, dout, dst, r->bytes_ws ? ws : nullptr, r->bytes_ws, st)
        : bg_eval(r->plan, r->E, dk, de, dout, dst, r->bytes_ws ? ws : nullptr, r->bytes_ws, st);
    if (bs != BG_OK) return bs;
    if (!r->out_dev) err = cudaMemcpyAsync(r->out, dout, no, cudaMemcpyDeviceToHost, st);
    if (!err && r->status && !r->st_dev)
        err = cudaMemcpyAsync(r->status, dst, (size_t)r->E, cudaMemcpyDeviceToHost, st);
    SlotDone* sd = new (std::nothrow) SlotDone{s, r->slot};
    if (!sd) return BG_ERR_NOMEM;
    if (!err) err = cudaEventRecord(s->slot_event[r->slot], st);
    if (!err) err = cudaLaunchHostFunc(st, slot_finished, sd);
    if (err) { delete sd; cudaGetLastError(); return BG_ERR_CUDA; }
    return BG_OK;
}

// The dispatcher decides admissions under the server mutex but enqueues the
// copies, kernels and host functions with the mutex released: the host
// function of a finishing request takes the mutex on the driver's callback
// thread, and a dispatcher holding it across CUDA calls would hold up every
// stream's completion behind those calls.
void dispatcher(bg_server* s) {
    cudaSetDevice(s->device);
    std::vector<Request*> admitted;
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        // collect finished slots
        bool progressed = false;
        for (size_t i = 0; i < s->streams.size(); ++i) {
            if (s->slot_req[i] && s->slot_done[i]) {
                Request* r = s->slot_req[i];
                s->arena->release(r->off, r->total);
                // the host function ran after the work, so the event has
                // completed -- unless that work raised an asynchronous error
                const cudaError_t ev = cudaEventQuery(s->slot_event[i]);
                if (ev == cudaSuccess) {
                    r->state = State::Done;
                } else {
                    cudaGetLastError();
                    r->result = BG_ERR_CUDA;
                    r->state = State::Failed;
                }
                s->slot_req[i] = nullptr;
                s->slot_done[i] = 0;
                ++s->n_completed;
                progressed = true;
            }
        }
        if (progressed) s->cv_done.notify_all();
        // admit: reserve a slot and arena bytes for each request that fits
        const auto now = Clock::now();
        bool blocked_head = false;
        admitted.clear();
        for (auto it = s->pending.begin(); it != s->pending.end();) {
            int slot = -1;
            for (size_t i = 0; i < s->slot_req.size(); ++i)
                if (!s->slot_req[i]) { slot = (int)i; break; }
            if (slot < 0) break;
            Request* r = *it;
            size_t off = 0;
            if (!blocked_head && s->arena->alloc(r->total, &off)) {
                r->off = off;
                r->slot = slot;
                r->state = State::Running;
                s->slot_req[slot] = r;
                s->slot_done[slot] = 0;
                if (s->arena->used() > s->peak_used) s->peak_used = s->arena->used();
                it = s->pending.erase(it);
                admitted.push_back(r);
                continue;
            }
            // does not fit: later requests may overtake unless this one starves
            const double waited = std::chrono::duration<double, std::milli>(now - r->submitted).count();
            if (waited > kStarveMs) blocked_head = true;
            ++it;
        }
        if (!admitted.empty()) {
            // enqueue outside the mutex; a running request is neither freed
            // by bg_serve_wait nor touched by submit, and its slot stays
            // reserved until the dispatcher itself releases it
            lk.unlock();
            for (Request* r : admitted) {
                r->result = launch_request(s, r);
                if (r->result != BG_OK)         // nothing of r was enqueued after the failure point
                    cudaStreamSynchronize(s->streams[r->slot]);
            }
            lk.lock();
            bool failed = false;
            for (Request* r : admitted) {
                if (r->result == BG_OK) continue;
                s->arena->release(r->off, r->total);
                s->slot_req[r->slot] = nullptr;
                s->slot_done[r->slot] = 0;
                r->state = State::Failed;
                failed = true;
            }
            if (failed) s->cv_done.notify_all();
            continue;                           // completions may have arrived meanwhile
        }
        if (s->stop && s->pending.empty()) {
            bool busy = false;
            for (auto* r : s->slot_req) busy |= (r != nullptr);
            if (!busy) break;
        }
        s->cv_work.wait_for(lk, std::chrono::milliseconds(2));
    }
}

}  // namespace

extern "C" {

bg_status bg_serve_create(size_t budget_bytes, int max_inflight, bg_server** out) {
    if (!out) return bgi::fail(BG_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (budget_bytes < kGranule || max_inflight < 1 || max_inflight > 64)
        return bgi::fail(BG_ERR_INVALID_ARG, "budget >= 256 B and 1 <= max_inflight <= 64 required");
    bg_server* s = new (std::nothrow) bg_server();
    if (!s) return bgi::fail(BG_ERR_NOMEM, "host allocation failed");
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return bgi::fail(BG_ERR_CUDA, "no current CUDA device");
    }
    s->budget = budget_bytes & ~(kGranule - 1);
    bgi::mapped_read_rate();          // measured now, not in a submit while requests run
    if (bgi::fault(BG_FAULT_DEVICE_ALLOC) || cudaMalloc(&s->arena_mem, s->budget) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return bgi::fail(BG_ERR_NOMEM, "device arena of %zu B could not be allocated", budget_bytes);
    }
    s->arena = new Arena(s->budget);
    s->streams.resize(max_inflight);
    s->slot_event.resize(max_inflight);
    s->slot_req.assign(max_inflight, nullptr);
    s->slot_done.assign(max_inflight, 0);
    for (int i = 0; i < max_inflight; ++i) {
        if (cudaStreamCreateWithFlags(&s->streams[i], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&s->slot_event[i], cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            for (int j = 0; j < i; ++j) {
                cudaStreamDestroy(s->streams[j]);
                cudaEventDestroy(s->slot_event[j]);
            }
            cudaFree(s->arena_mem);
            delete s->arena;
            delete s;
            return bgi::fail(BG_ERR_CUDA, "stream or event creation failed");
        }
    }
    s->thread = std::thread(dispatcher, s);
    *out = s;
    return BG_OK;
}

bg_status bg_serve_submit(bg_server* srv, const bg_plan* plan, int64_t E, const void* momenta,
                          const void* eps, void* out, uint8_t* status, uint64_t* ticket) {
    if (!srv || !plan || !ticket) return bgi::fail(BG_ERR_INVALID_ARG, "server, plan and ticket are required");
    if (E < 1 || !momenta || !eps || !out) return bgi::fail(BG_ERR_INVALID_ARG, "E >= 1 and buffers required");
    if (plan->d_assign && plan->device != srv->device)
        return bgi::fail(BG_ERR_INVALID_ARG, "plan and server are on different devices");
    // each buffer is host memory (staged through the arena) or device memory
    // of the server's device (used in place: resident inputs, outputs left on
    // the device)
    int where[4] = {0, 0, 0, 0};      // 0 host, 1 this device, 2 mapped page-locked host memory
    const void* bufs[4] = {momenta, eps, out, status};
    for (int b = 0; b < 4; ++b) {
        if (!bufs[b]) continue;
        cudaPointerAttributes attr;
        if (cudaPointerGetAttributes(&attr, bufs[b]) != cudaSuccess) {
            cudaGetLastError();
            continue;                 // unregistered host memory
        }
        if (attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged) {
            if (attr.type == cudaMemoryTypeDevice && attr.device != srv->device)
                return bgi::fail(BG_ERR_INVALID_ARG, "buffer %d is on device %d, the server's is %d", b,
                                 attr.device, srv->device);
            where[b] = 1;
        } else if (attr.type == cudaMemoryTypeHost && attr.devicePointer == bufs[b]) {
            where[b] = 2;
        }
    }
    Request* r = new (std::nothrow) Request();
    if (!r) return bgi::fail(BG_ERR_NOMEM, "host allocation failed");
    const size_t elem = bgi::value_bytes(plan->field);
    r->plan = plan;
    r->E = E;
    r->k = momenta;
    r->eps = eps;
    r->out = out;
    r->status = status;
    // device memory is used in place, and so is mapped page-locked host
    // memory unless the request is large and light enough per point for the
    // host link to bound its kernel (then copies, overlapping other requests'
    // kernels, serve it better)
    const size_t sizes[4] = {(size_t)E * plan->n * plan->d * bgi::momentum_bytes(plan->field),
                             (size_t)E * plan->n * plan->S * plan->Ds * elem, (size_t)E * plan->H * elem,
                             (size_t)E};
    size_t mapped_bytes = 0;
    for (int b = 0; b < 4; ++b)
        if (where[b] == 2) mapped_bytes += sizes[b];
    const bool use_mapped = mapped_bytes > 0 && bgi::in_place_pays(plan, E, mapped_bytes);
    bool in_place[4];
    for (int b = 0; b < 4; ++b) {
        in_place[b] = where[b] == 1 || (where[b] == 2 && use_mapped);
        r->mapped |= where[b] == 2 && use_mapped;
    }
    r->k_dev = in_place[0];
    r->e_dev = in_place[1];
    r->out_dev = in_place[2];
    r->st_dev = in_place[3];
    r->bytes_k = r->k_dev ? 0 : up_granule((size_t)E * plan->n * plan->d * bgi::momentum_bytes(plan->field));
    r->bytes_e = r->e_dev ? 0 : up_granule((size_t)E * plan->n * plan->S * plan->Ds * elem);
    r->bytes_o = r->out_dev ? 0 : up_granule((size_t)E * plan->H * elem);
    r->bytes_s = r->st_dev ? 0 : up_granule((size_t)E);
    size_t ws = 0;
    bg_workspace_size(plan, E, &ws);
    r->bytes_ws = up_granule(ws);
    r->total = r->bytes_k + r->bytes_e + r->bytes_o + r->bytes_s + r->bytes_ws;
    if (r->total > srv->budget) {
        const size_t need = r->total;
        delete r;
        return bgi::fail(BG_ERR_INVALID_ARG, "request needs %zu B, above the server budget of %zu B", need,
                         srv->budget);
    }
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        if (srv->stop) {
            delete r;
            return bgi::fail(BG_ERR_BUSY, "server is shutting down");
        }
        r->id = srv->next_id++;
        r->submitted = Clock::now();
        srv->pending.push_back(r);
        srv->requests[r->id] = r;
        ++srv->n_submitted;
        *ticket = r->id;
    }
    srv->cv_work.notify_one();
    return BG_OK;
}

bg_status bg_serve_wait(bg_server* srv, uint64_t ticket, int64_t timeout_ms) {
    if (!srv) return bgi::fail(BG_ERR_INVALID_ARG, "server is NULL");
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->requests.find(ticket);
    if (it == srv->requests.end()) return bgi::fail(BG_ERR_INVALID_ARG, "unknown ticket %llu", (unsigned long long)ticket);
    Request* r = it->second;
    auto finished = [r] { return r->state == State::Done || r->state == State::Failed; };
    ++r->waiters;
    bool done = true;
    if (timeout_ms < 0) srv->cv_done.wait(lk, finished);
    else done = srv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), finished);
    --r->waiters;
    if (!done)
        return bgi::fail(BG_ERR_TIMEOUT, "request %llu not finished after %lld ms", (unsigned long long)ticket,
                         (long long)timeout_ms);
    const bg_status result = r->state == State::Done ? BG_OK : r->result;
    if (!r->retired) {                          // the first waiter to return retires the ticket
        r->retired = true;
        srv->requests.erase(r->id);
    }
    if (r->waiters == 0) delete r;              // the last one frees the request
    if (result != BG_OK) return bgi::fail(result, "request failed");
    return BG_OK;
}

bg_status bg_serve_stats(bg_server* srv, uint64_t* submitted, uint64_t* completed, uint64_t* pending,
                         size_t* bytes_in_use, size_t* peak_bytes) {
    if (!srv) return bgi::fail(BG_ERR_INVALID_ARG, "server is NULL");
    std::lock_guard<std::mutex> lk(srv->mu);
    if (submitted) *submitted = srv->n_submitted;
    if (completed) *completed = srv->n_completed;
    if (pending) *pending = srv->pending.size();
    if (bytes_in_use) *bytes_in_use = srv->arena->used();
    if (peak_bytes) *peak_bytes = srv->peak_used;
    return BG_OK;
}

bg_status bg_serve_destroy(bg_server* srv) {
    if (!srv) return BG_OK;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
    }
    srv->cv_work.notify_all();
    if (srv->thread.joinable()) srv->thread.join();
    for (cudaStream_t st : srv->streams) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    for (cudaEvent_t ev : srv->slot_event) cudaEventDestroy(ev);
    cudaFree(srv->arena_mem);
    for (auto& kv : srv->requests) delete kv.second;
    delete srv->arena;
    delete srv;
    return BG_OK;
}

}  // extern "C"
