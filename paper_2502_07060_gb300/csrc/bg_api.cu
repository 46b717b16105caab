// bg_api.cu -- the C-ABI of libbg.so (declared in include/bg.h): plan
// validation, kernel selection and the single launch of bg_eval.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <utility>
#include <string>
#include <vector>

#include "bg_internal.h"

#define BG_REGC(TAG, D, DS) void bg_register_compact_##TAG##_##D##_##DS(std::vector<bgk::KernelEntry>&);
BG_REGC(fp, 4, 4) BG_REGC(fp, 4, 6) BG_REGC(fp, 4, 8) BG_REGC(fp, 6, 6) BG_REGC(fp, 6, 8) BG_REGC(fp, 8, 8)
BG_REGC(c64, 4, 4) BG_REGC(c64, 4, 6) BG_REGC(c64, 4, 8) BG_REGC(c64, 6, 6) BG_REGC(c64, 6, 8)
BG_REGC(c64, 8, 8)
BG_REGC(c64r, 4, 4) BG_REGC(c64r, 4, 6) BG_REGC(c64r, 4, 8) BG_REGC(c64r, 6, 6) BG_REGC(c64r, 6, 8)
BG_REGC(c64r, 8, 8)
#undef BG_REGC
void bg_register_lanes_fp(std::vector<bgk::LanesEntry>&);
void bg_register_lanes_c64(std::vector<bgk::LanesEntry>&);
void bg_register_lanes_c64r(std::vector<bgk::LanesEntry>&);
#define BG_REGS(TAG, D) void bg_register_states_##TAG##_##D(std::vector<bgk::StatesEntry>&);
BG_REGS(fp, 4) BG_REGS(fp, 6) BG_REGS(fp, 8) BG_REGS(c64, 4) BG_REGS(c64, 6) BG_REGS(c64, 8)
BG_REGS(c64r, 4) BG_REGS(c64r, 6) BG_REGS(c64r, 8)
#undef BG_REGS

namespace {
thread_local std::string g_last_error;
#ifdef BG_CHECKED
__device__ unsigned long long g_bounds_violation;   // first out-of-range table index (checked builds)
#endif
}  // namespace

namespace bgi {

namespace {
struct FaultPlan {
    std::atomic<int64_t> seen{0};     // operations at the site since the last arming
    std::atomic<int64_t> first{0};    // first failing operation
    std::atomic<int64_t> end{0};      // one past the last failing operation
};
FaultPlan g_fault[4];
}  // namespace

unsigned long long* violation_word(int device) {
#ifdef BG_CHECKED
    static std::mutex mu;
    static void* addr[64] = {};
    if (device < 0 || device >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(mu);
    if (!addr[device] && cudaGetSymbolAddress(&addr[device], g_bounds_violation) != cudaSuccess) {
        cudaGetLastError();
        addr[device] = nullptr;
    }
    return static_cast<unsigned long long*>(addr[device]);
#else
    (void)device;
    return nullptr;
#endif
}

bool fault(int site) {
    if (site < 1 || site > 3) return false;
    FaultPlan& f = g_fault[site];
    if (f.end.load(std::memory_order_relaxed) == 0) return false;
    const int64_t k = f.seen.fetch_add(1);
    return k >= f.first.load() && k < f.end.load();
}

bg_status fail(bg_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return s;
}

void log(const char* fmt, ...) {
    static const bool on = [] {
        const char* v = getenv("BG_LOG");
        return v && *v && strcmp(v, "0") != 0;
    }();
    if (!on) return;
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    fprintf(stderr, "bg: %s\n", buf);
}

const std::vector<bgk::KernelEntry>& registry() {
    static std::vector<bgk::KernelEntry> v;
    static std::once_flag once;
    std::call_once(once, [] {
#define BG_ADDC(TAG, D, DS) bg_register_compact_##TAG##_##D##_##DS(v);
        BG_ADDC(fp, 4, 4) BG_ADDC(fp, 4, 6) BG_ADDC(fp, 4, 8) BG_ADDC(fp, 6, 6) BG_ADDC(fp, 6, 8)
        BG_ADDC(fp, 8, 8) BG_ADDC(c64, 4, 4) BG_ADDC(c64, 4, 6) BG_ADDC(c64, 4, 8) BG_ADDC(c64, 6, 6)
        BG_ADDC(c64, 6, 8) BG_ADDC(c64, 8, 8)
        BG_ADDC(c64r, 4, 4) BG_ADDC(c64r, 4, 6) BG_ADDC(c64r, 4, 8) BG_ADDC(c64r, 6, 6)
        BG_ADDC(c64r, 6, 8) BG_ADDC(c64r, 8, 8)
#undef BG_ADDC
    });
    return v;
}

const std::vector<bgk::StatesEntry>& states_registry() {
    static std::vector<bgk::StatesEntry> v;
    static std::once_flag once;
    std::call_once(once, [] {
        bg_register_states_fp_4(v); bg_register_states_fp_6(v); bg_register_states_fp_8(v);
        bg_register_states_c64_4(v); bg_register_states_c64_6(v); bg_register_states_c64_8(v);
        bg_register_states_c64r_4(v); bg_register_states_c64r_6(v); bg_register_states_c64r_8(v);
    });
    return v;
}

const std::vector<bgk::LanesEntry>& lanes_registry() {
    static std::vector<bgk::LanesEntry> v;
    static std::once_flag once;
    std::call_once(once, [] {
        bg_register_lanes_fp(v);
        bg_register_lanes_c64(v);
        bg_register_lanes_c64r(v);
    });
    return v;
}

static uint64_t mulmod64(uint64_t a, uint64_t b, uint64_t m) { return (a * b) % m; }   // a, b < 2^31

static uint64_t powmod64(uint64_t a, uint64_t e, uint64_t m) {
    uint64_t r = 1 % m;
    a %= m;
    while (e) {
        if (e & 1) r = mulmod64(r, a, m);
        a = mulmod64(a, a, m);
        e >>= 1;
    }
    return r;
}

// Deterministic Miller-Rabin for n < 2^32 (bases 2, 3, 5, 7 suffice below 3.2e9).
static bool is_prime_u32(uint32_t n) {
    if (n < 2) return false;
    for (uint32_t q : {2u, 3u, 5u, 7u}) {
        if (n == q) return true;
        if (n % q == 0) return false;
    }
    uint64_t d = n - 1;
    int r = 0;
    while ((d & 1) == 0) { d >>= 1; ++r; }
    for (uint64_t a : {2ull, 3ull, 5ull, 7ull}) {
        uint64_t x = powmod64(a, d, n);
        if (x == 1 || x == n - 1) continue;
        bool comp = true;
        for (int i = 1; i < r; ++i) {
            x = mulmod64(x, x, n);
            if (x == n - 1) { comp = false; break; }
        }
        if (comp) return false;
    }
    return true;
}

bg_status check_device_ptr(const void* ptr, const char* what, int device) {
    cudaPointerAttributes attr;
    cudaError_t err = cudaPointerGetAttributes(&attr, ptr);
    if (err != cudaSuccess) {
        cudaGetLastError();
        return fail(BG_ERR_INVALID_ARG, "%s: not a CUDA pointer (%s)", what, cudaGetErrorString(err));
    }
    if (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged)
        return fail(BG_ERR_INVALID_ARG, "%s: must be device memory", what);
    if (attr.type == cudaMemoryTypeDevice && attr.device != device)
        return fail(BG_ERR_INVALID_ARG, "%s: lives on device %d, current device is %d", what,
                    attr.device, device);
    return BG_OK;
}

// Memory a kernel on `device` may read and write: device memory of that
// device, or -- where the caller allows it -- page-locked host memory mapped
// into the device's address space at the same address (unified addressing),
// which kernels access over the host link without a copy.
bg_status check_kernel_ptr(const void* ptr, const char* what, int device, bool mapped_host_ok) {
    if (mapped_host_ok) {
        cudaPointerAttributes attr;
        if (cudaPointerGetAttributes(&attr, ptr) == cudaSuccess && attr.type == cudaMemoryTypeHost &&
            attr.devicePointer == ptr)
            return BG_OK;
        cudaGetLastError();
    }
    return check_device_ptr(ptr, what, device);
}

bool mapped_host(const void* p) {
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return attr.type == cudaMemoryTypeHost && attr.devicePointer == p;
}

// Field multiplications per amplitude of the literal recursion (three- and
// four-gluon splits of every range, propagators, final contraction; momenta
// d-, currents D-dimensional): C(n,3)(3D+3d) + C(n,4) 6D + (C(n,2)-n)(d+D) + D.
double ops_per_amplitude(int n, int d, int D) {
    const double c2 = n * (n - 1.0) / 2, c3 = c2 * (n - 2) / 3, c4 = c3 * (n - 3) / 4;
    return c3 * (3.0 * D + 3.0 * d) + c4 * 6.0 * D + (c2 - n) * (d + D) + D;
}

// The kernels sustain about 4.3e12 (F_p), 2.5e11 (complex, real momenta) and
// 1.9e11 (complex momenta) of these multiplications per second (n = 8, d = 6
// on a GB300).  link_bytes_per_s is the rate of the host-link probe
// (mapped_read_rate); the kernels' own loads of mapped host memory, mixed
// with their arithmetic, reach about three quarters of it (103 against 135
// GB/s on a GB300 host), and in place pays while the batch needs at most 80 %
// of that.  At n = 8, d = 6 that keeps F_p batches (about 350 GB/s) on copies
// and takes complex ones (about 60 GB/s) in place.
bool in_place_pays_for(int field, int n, int d, int Ds, int H, int64_t E, size_t host_bytes, double sm_scale,
                       double link_bytes_per_s) {
    if (host_bytes <= kInPlaceBytes) return true;
    const double rate = sm_scale * (field == BG_FIELD_FP ? 4.3e12 : field == BG_FIELD_C64_REAL ? 2.5e11 : 1.9e11);
    const double seconds = (double)E * H * ops_per_amplitude(n, d, Ds) / rate;
    return (double)host_bytes <= 0.8 * 0.76 * link_bytes_per_s * seconds;
}

// The compute rates above were measured on a 152-SM GB300; a device with
// another SM count scales them (the kernels are bound by per-SM pipes).  The
// host-link rate is measured on the device itself (mapped_read_rate), since
// it differed from host to host.
bool in_place_pays(const bg_plan* plan, int64_t E, size_t host_bytes) {
    if (host_bytes <= kInPlaceBytes) return true;
    const double sm_scale = plan->sm_count > 0 ? plan->sm_count / 152.0 : 1.0;
    return in_place_pays_for(plan->field, plan->n, plan->d, plan->Ds, plan->H, E, host_bytes, sm_scale,
                             mapped_read_rate());
}

int round_dim(int x) { return x <= 4 ? 4 : (x <= 6 ? 6 : 8); }

// The dynamic shared-memory limit is an attribute of the kernel function, not
// of a plan: raise it to `bytes` on `device` if it is lower, never lower it
// (plans sharing a kernel may need different sizes).
bg_status ensure_smem_limit(const void* func, int device, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<const void*, int>, size_t> limit;
    std::lock_guard<std::mutex> lk(mu);
    size_t& cur = limit[{func, device}];
    if (cur >= bytes) return BG_OK;
    cudaError_t err = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (err != cudaSuccess) {
        cudaGetLastError();
        return fail(BG_ERR_UNSUPPORTED, "shared memory %zu B: %s", bytes, cudaGetErrorString(err));
    }
    cur = bytes;
    return BG_OK;
}

}  // namespace bgi

using bgi::check_device_ptr;
using bgi::fail;
using bgi::registry;
using bgi::round_dim;
using bgi::is_prime_u32;
using bgi::mulmod64;
using bgi::value_bytes;
using bgi::momentum_bytes;
using bgi::compact_params;
using bgi::field_name;

namespace {

// Table bytes of one block of the states kernel above which the table moves
// to global scratch: at most this much shared memory keeps four or more
// blocks (16 warps) resident per SM.
constexpr size_t kStatesSmemMax = 56 * 1024;

// States-kernel choice, table placement and occupancy of a plan over the
// product of per-leg state sets (radix[l] states on leg l).
bg_status setup_states(bg_plan* pl, const int* radix, const char* tenv) {
    const int D = round_dim(pl->d), DS = round_dim(pl->Ds);
    bool uniform = true;
    for (int l = 1; l < pl->n; ++l) uniform &= radix[l] == radix[0];
    for (const auto& e : bgi::states_registry())
        if (e.field == (int)pl->field && e.D == D && e.DS == DS && e.metric == (int)pl->metric &&
            e.uniform == uniform)
            pl->sentry = &e;
    if (!pl->sentry) return fail(BG_ERR_UNSUPPORTED, "no all-assignment kernel for this plan");
    pl->sgeo = bgk::make_states_geometry(pl->n, pl->S, radix, D, DS, pl->sentry->elem_bytes,
                                         pl->sentry->elem_k_bytes);
    pl->all_states = true;
    const size_t smem = (size_t)bgk::kStatesWarps * pl->sgeo.P * pl->sgeo.words * pl->sentry->elem_bytes;
    bool global = smem > kStatesSmemMax;
    if (tenv) global = strcmp(tenv, "global") == 0 || smem > 227 * 1024;
    pl->states_global = global;
    pl->smem_bytes = global ? 0 : smem;
    if (pl->smem_bytes > 0) {
        bg_status st = bgi::ensure_smem_limit(pl->sentry->func, pl->device, pl->smem_bytes);
        if (st != BG_OK) return st;
    }
    int occ = 0;
    cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, pl->sentry->func,
                                                                    32 * bgk::kStatesWarps, pl->smem_bytes);
    if (err != cudaSuccess || occ < 1) {
        cudaGetLastError();
        return fail(BG_ERR_UNSUPPORTED, "all-assignment kernel cannot be resident (%s)", cudaGetErrorString(err));
    }
    pl->blocks_per_sm = occ;
    return BG_OK;
}

// The lane-group kernel of a plan with one recursion per work item, and the
// batch sizes it takes.  A batch of E H work items on the compact kernel
// runs one item per thread: while E H is far below the kernel's resident
// threads most of the GPU idles and the call lasts as long as one thread's
// whole recursion.  The lanes kernel spreads each item over L lanes, which
// shortens that recursion for the complex fields (FP64 vector updates split
// over the lanes: 2.1x at n = 8, 2.8x at n = 12, d = 8, up to 2048 points)
// and less over F_p, where the shuffled contractions lengthen its dependency
// chains (1.24x at n = 8, 1.5x at n = 12; none at n <= 5).  Measured on
// GB300, the lanes kernel stops paying between 16 and 32 items per SM for
// the complex fields at n = 8..12 and between 24 and 48 for F_p, and at about
// half of one resident wave of lane groups when the groups are small (L = 4,
// short tables): BG_LANES unset takes it up to max(16 (complex) or 24 (F_p,
// n >= 7) items per SM, half a resident wave of the lanes kernel);
// BG_LANES=0 never, BG_LANES=1 always (when the plan has one).
// The entry of the lanes kernel with L lanes per group and G groups per
// point, its shared memory and resident blocks per SM; false (entry cleared)
// when the plan's tables do not fit.
bool lanes_variant(bg_plan* pl, int L, int G, const bgk::LanesEntry** entry, size_t* smem_out, int* occ_out) {
    *entry = nullptr;
    for (const auto& e : bgi::lanes_registry())
        if (e.field == (int)pl->field && e.L == L && e.G == G && e.metric == (int)pl->metric) *entry = &e;
    if (!*entry) return false;
    const size_t smem = (size_t)bgk::LaneGeometry{pl->n - 1}.words() * ((*entry)->block / G) * (*entry)->elem_bytes;
    int occ = 0;
    if (smem > 227 * 1024 || bgi::ensure_smem_limit((*entry)->func, pl->device, smem) != BG_OK ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, (*entry)->func, (*entry)->block, smem) != cudaSuccess ||
        occ < 1) {
        cudaGetLastError();
        g_last_error.clear();
        *entry = nullptr;                // the compact kernel serves every size
        return false;
    }
    *smem_out = smem;
    *occ_out = occ;
    return true;
}

// One point per team (a warp of G = 32 / L groups evaluating the ranges of
// each length in parallel) shortens a point's recursion further (measured on
// GB300 up to 512 points: complex n = 8, d = 6 0.10 against 0.18 ms, n = 12,
// d = 8 0.35 against 0.82 ms; F_p n = 12, d = 8 0.066 against 0.128 ms) but
// takes G times the lanes per point, so it stops paying once the warps fill
// the schedulers: at about 5 points per scheduler for F_p and n - 5 for the
// complex fields (more ranges per length at larger n keep more of a team's
// groups busy).  BG_LANES=2 takes the team form always.
bg_status setup_lanes(bg_plan* pl) {
    const int L = round_dim(pl->Ds) <= 4 ? 4 : 8;
    if (!lanes_variant(pl, L, 1, &pl->lentry, &pl->lanes_smem, &pl->lanes_blocks_per_sm)) return BG_OK;
    lanes_variant(pl, L, 32 / L, &pl->tentry, &pl->team_smem, &pl->team_blocks_per_sm);
    const char* env = getenv("BG_LANES");
    if (env && strcmp(env, "0") == 0) {
        pl->lanes_max_items = 0;
    } else if (env && strcmp(env, "1") == 0) {
        pl->lanes_max_items = INT64_MAX;
    } else if (env && strcmp(env, "2") == 0) {
        pl->lanes_max_items = INT64_MAX;
        pl->team_max_items = pl->tentry ? INT64_MAX : 0;
    } else {
        const int64_t wave = (int64_t)pl->lanes_blocks_per_sm * pl->sm_count * (pl->lentry->block / L);
        const int64_t per_sm = pl->field == BG_FIELD_FP ? 24 : 16;
        pl->lanes_max_items = (pl->field == BG_FIELD_FP && pl->n < 7) ? 0
                            : std::max(per_sm * pl->sm_count, wave / 2);
        if (pl->tentry && pl->lanes_max_items > 0) {
            const int64_t per_scheduler = pl->field == BG_FIELD_FP ? 5 : std::max(1, pl->n - 5);
            pl->team_max_items = std::min(pl->lanes_max_items, per_scheduler * 4 * pl->sm_count);
        }
    }
    return BG_OK;
}

}  // namespace

extern "C" {

const char* bg_strerror(bg_status s) {
    switch (s) {
        case BG_OK: return "success";
        case BG_ERR_INVALID_ARG: return "invalid argument";
        case BG_ERR_UNSUPPORTED: return "unsupported configuration";
        case BG_ERR_NOMEM: return "out of memory";
        case BG_ERR_CUDA: return "CUDA error";
        case BG_ERR_TIMEOUT: return "timed out";
        case BG_ERR_BUSY: return "busy";
    }
    return "unknown status";
}

const char* bg_last_error(void) { return g_last_error.c_str(); }

int bg_version(void) { return BG_VERSION; }

bg_status bg_debug_bounds_report(int* checked, uint64_t* first_violation) {
    if (!checked || !first_violation) return fail(BG_ERR_INVALID_ARG, "checked and first_violation must be non-NULL");
    *checked = 0;
    *first_violation = 0;
#ifdef BG_CHECKED
    unsigned long long v = 0, zero = 0;
    if (cudaMemcpyFromSymbol(&v, g_bounds_violation, sizeof v) != cudaSuccess ||
        cudaMemcpyToSymbol(g_bounds_violation, &zero, sizeof zero) != cudaSuccess) {
        cudaGetLastError();
        return fail(BG_ERR_CUDA, "could not read the bounds-violation word");
    }
    *checked = 1;
    *first_violation = v;
#endif
    return BG_OK;
}

bg_status bg_debug_in_place_pays(bg_field field, int n, int d, int D_s, int H, int64_t E, size_t host_bytes,
                                 int* in_place, double* ops) {
    if (!in_place || !ops || n < 4 || n > 12 || d < 4 || D_s < d || D_s > 8 || H < 1 || E < 0 ||
        (field != BG_FIELD_C64 && field != BG_FIELD_FP && field != BG_FIELD_C64_REAL))
        return fail(BG_ERR_INVALID_ARG, "bad argument to bg_debug_in_place_pays");
    *ops = bgi::ops_per_amplitude(n, d, D_s);
    *in_place = bgi::in_place_pays_for((int)field, n, d, D_s, H, E, host_bytes, 1.0, bgi::kMappedReadRateDefault) ? 1 : 0;
    return BG_OK;
}

bg_status bg_debug_inject_fault(bg_fault_site site, int skip, int count) {
    if ((int)site < 1 || (int)site > 3 || skip < 0 || count < 0)
        return fail(BG_ERR_INVALID_ARG, "bad fault site %d, skip %d or count %d", (int)site, skip, count);
    bgi::FaultPlan& f = bgi::g_fault[(int)site];
    f.end.store(0);
    f.seen.store(0);
    f.first.store(skip);
    f.end.store(count > 0 ? (int64_t)skip + count : 0);
    return BG_OK;
}

}  // extern "C"

// Plan creation; product_radix (or NULL) gives the states per leg of a
// product plan (all assignments of the product of per-leg state sets).
static bg_status create_plan(int n, int d, int D_s, bg_field field, uint32_t p, bg_metric metric,
                             int n_states, int n_assign, const uint8_t* assign, const uint8_t* product_radix,
                             uint32_t four_d_legs, bg_plan** out) {
    g_last_error.clear();
    if (!out) return fail(BG_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n < 4 || n > 12) return fail(BG_ERR_INVALID_ARG, "n = %d outside [4, 12]", n);
    if (d < 4 || d > 8) return fail(BG_ERR_INVALID_ARG, "d = %d outside [4, 8]", d);
    if (D_s < d || D_s > 8) return fail(BG_ERR_INVALID_ARG, "D_s = %d outside [d, 8]", D_s);
    if (field != BG_FIELD_FP && field != BG_FIELD_C64 && field != BG_FIELD_C64_REAL)
        return fail(BG_ERR_INVALID_ARG, "unknown field %d", (int)field);
    if (metric != BG_METRIC_MOSTLY_MINUS && metric != BG_METRIC_ALTERNATING)
        return fail(BG_ERR_INVALID_ARG, "unknown metric %d", (int)metric);
    if (field == BG_FIELD_FP) {
        if (p < 3 || p >= (1u << 31) || !is_prime_u32(p))
            return fail(BG_ERR_INVALID_ARG, "p = %u is not an odd prime below 2^31", p);
    } else if (p != 0) {
        return fail(BG_ERR_INVALID_ARG, "p must be 0 for the complex field");
    }
    if (n_states < 1 || n_states > 255) return fail(BG_ERR_INVALID_ARG, "n_states = %d", n_states);
    if (n_assign < 1 || (int64_t)n_assign * n > (1 << 20))
        return fail(BG_ERR_INVALID_ARG, "n_assign = %d", n_assign);
    // assign == NULL with H > 1: all S^n assignments (H must equal S^n),
    // evaluated with sub-currents shared between assignments
    bool all_states = product_radix != nullptr;
    if (n_assign > 1 && !assign && !product_radix) {
        int64_t h = 1;
        for (int l = 0; l < n && h <= n_assign; ++l) h *= n_states;
        if (n_states < 2 || h != n_assign)
            return fail(BG_ERR_INVALID_ARG, "assign is NULL with n_assign = %d != n_states^n", n_assign);
        all_states = true;
    }
    if (four_d_legs >> n) return fail(BG_ERR_INVALID_ARG, "four_dim_legs has bits above leg n-1");
    if (four_d_legs && all_states)
        return fail(BG_ERR_UNSUPPORTED, "four-dimensional legs with all-assignment plans");
    if (assign) {
        for (int64_t i = 0; i < (int64_t)n_assign * n; ++i)
            if (assign[i] >= n_states)
                return fail(BG_ERR_INVALID_ARG, "assign[%lld] = %d >= n_states", (long long)i, assign[i]);
    }

    // Kernel choice: the compact kernel (run-time n) for the plan's (D, D_s,
    // metric).  Table placement: shared memory for small tables, else global
    // scratch, or split (currents global, the rest on chip)
    // (BG_TABLE=shared|global|split overrides).
    const char* tenv = getenv("BG_TABLE");
    const int Dk = round_dim(d), DSk = round_dim(D_s);
    // mixed kernels only pay where a current has more than four components
    const bool want_mixed = four_d_legs != 0 && DSk > 4;
    const bgk::KernelEntry* best = nullptr;
    const bgk::Geometry geo{n - 1};
    int words = geo.words(Dk, DSk);
    {
        const size_t elem = value_bytes(field);
        int want = bgk::kPlaceGlobal;
        if (tenv) {
            want = strcmp(tenv, "shared") == 0 ? bgk::kPlaceShared
                 : strcmp(tenv, "split") == 0 ? bgk::kPlaceSplit : bgk::kPlaceGlobal;
        } else if (field == BG_FIELD_FP) {
            // measured on GB300 (n = 5..12): shared wins while a block's table
            // is at most ~40 KB (five or more blocks per SM), global beyond
            const size_t smem = (size_t)words * bgk::kBlockFpCompactSmem * elem;
            want = smem > 40 * 1024 ? bgk::kPlaceGlobal : bgk::kPlaceShared;
        }
        for (const auto& e : registry()) {
            const int place = e.split ? bgk::kPlaceSplit : e.global_table ? bgk::kPlaceGlobal : bgk::kPlaceShared;
            if (e.field == (int)field && e.D == Dk && e.DS == DSk && e.metric == (int)metric && place == want &&
                e.mixed == want_mixed)
                best = &e;
        }
        // F_p with D_s = 8 and the table in global scratch: the prefix sums, SA
        // and 1/P^2 in shared memory (split) measured 3.7-7 % faster on GB300
        // at n = 6..8 while it keeps the resident blocks per SM; from n = 9 it
        // loses blocks and time, and at D_s = 6 it did not pay at n = 8.
        if (!tenv && best && field == BG_FIELD_FP && DSk == 8 && !want_mixed && best->global_table && !best->split) {
            const bgk::KernelEntry* sp = nullptr;
            for (const auto& e : registry())
                if (e.field == (int)field && e.D == Dk && e.DS == DSk && e.metric == (int)metric && e.split &&
                    !e.mixed)
                    sp = &e;
            int dev = -1, occ_g = 0, occ_s = 0;
            const size_t ssm = sp ? (size_t)geo.aux_words(Dk, DSk) * sp->block * sp->elem_bytes : 0;
            const std::string kept = g_last_error;           // a refused smem limit is not this call's error
            if (sp && cudaGetDevice(&dev) == cudaSuccess &&
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_g, best->func, best->block, 0) == cudaSuccess &&
                ssm <= 227 * 1024 && bgi::ensure_smem_limit(sp->func, dev, ssm) == BG_OK &&
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_s, sp->func, sp->block, ssm) == cudaSuccess &&
                occ_s >= occ_g && occ_s > 0)
                best = sp;
            cudaGetLastError();
            g_last_error = kept;
        }
        if (best && best->split) words = geo.cur_words(DSk);
        if (!best)      // the complex fields have only the global placement, mixed F_p no split
            for (const auto& e : registry())
                if (e.field == (int)field && e.D == Dk && e.DS == DSk && e.metric == (int)metric &&
                    e.mixed == want_mixed && !e.split)
                    best = &e;
    }
    if (!best) return fail(BG_ERR_UNSUPPORTED, "no kernel for n=%d d=%d D_s=%d field=%d metric=%d", n, d,
                           D_s, (int)field, (int)metric);

    bg_plan* pl = new (std::nothrow) bg_plan();
    if (!pl) return fail(BG_ERR_NOMEM, "host allocation failed");
    pl->n = n; pl->d = d; pl->Ds = D_s; pl->field = field; pl->p = p; pl->metric = metric;
    pl->S = n_states; pl->H = n_assign; pl->entry = best; pl->words = words;
    pl->four_d_legs = best->mixed ? four_d_legs : 0u;
    if (assign) pl->assign.assign(assign, assign + (size_t)n_assign * n);
    if (field == BG_FIELD_FP) {
        uint32_t inv = p;                         // p^-1 mod 2^32 by Newton iteration
        for (int i = 0; i < 5; ++i) inv *= 2u - p * inv;
        const uint64_t r1 = (uint64_t(1) << 32) % p;
        const uint64_t r2 = mulmod64(r1, r1, p);
        const uint64_t r3 = mulmod64(r2, r1, p);
        pl->fpo.p = p;
        pl->fpo.pinv = 0u - inv;
        pl->fpo.one = (uint32_t)r1;
        pl->fpo.r2 = (uint32_t)r2;
        pl->fpo.r3 = (uint32_t)r3;
        pl->fpo.pm2 = p - 2;
        uint64_t rn3 = r3;                        // R^(n+3): states enter unconverted
        for (int i = 0; i < n; ++i) rn3 = mulmod64(rn3, r1, p);
        pl->fpo.rn3 = (uint32_t)rn3;
    }

    if (cudaGetDevice(&pl->device) != cudaSuccess) {
        cudaGetLastError();
        delete pl;
        return fail(BG_ERR_CUDA, "no CUDA device");
    }
    cudaDeviceGetAttribute(&pl->sm_count, cudaDevAttrMultiProcessorCount, pl->device);
    pl->smem_bytes = best->split ? (size_t)bgk::Geometry{n - 1}.aux_words(round_dim(d), round_dim(D_s)) *
                                       best->block * best->elem_bytes
                   : best->global_table ? 0 : (size_t)words * best->block * best->elem_bytes;
    if (pl->smem_bytes > 0) {
        bg_status st = bgi::ensure_smem_limit(best->func, pl->device, pl->smem_bytes);
        if (st != BG_OK) {
            delete pl;
            return st;
        }
    }
    int occ = 0;
    cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, best->func, best->block,
                                                                    pl->smem_bytes);
    if (err != cudaSuccess || occ < 1) {
        cudaGetLastError();
        delete pl;
        return fail(BG_ERR_UNSUPPORTED, "kernel cannot be resident (%s)", cudaGetErrorString(err));
    }
    pl->blocks_per_sm = occ;
    if (all_states) {
        int radix[bgk::kStatesMaxLegs];
        for (int l = 0; l < n; ++l) radix[l] = product_radix ? product_radix[l] : n_states;
        bg_status st = setup_states(pl, radix, tenv);
        if (st != BG_OK) {
            delete pl;
            return st;
        }
    }
    if (!all_states) setup_lanes(pl);
    if (n_assign > 1 && !all_states) {
        size_t bytes = pl->assign.size();
        if (bgi::fault(BG_FAULT_DEVICE_ALLOC) || cudaMalloc(&pl->d_assign, bytes) != cudaSuccess) {
            cudaGetLastError();
            delete pl;
            return fail(BG_ERR_NOMEM, "device allocation of %zu B failed", bytes);
        }
        if (cudaMemcpy(pl->d_assign, pl->assign.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(pl->d_assign);
            delete pl;
            return fail(BG_ERR_CUDA, "copy of the assignment table failed");
        }
    }
    *out = pl;
    if (pl->all_states)
        bgi::log("plan n=%d d=%d D_s=%d field=%d: all-assignment kernel, %s table, %d blocks/SM", n, d, D_s,
                 (int)field, pl->states_global ? "global" : "shared", pl->blocks_per_sm);
    else
        bgi::log("plan n=%d d=%d D_s=%d field=%d: compact kernel D=%d D_s=%d, %s table, block %d, %d blocks/SM",
                 n, d, D_s, (int)field, best->D, best->DS,
                 best->split ? "split" : best->global_table ? "global" : "shared", best->block, pl->blocks_per_sm);
    return BG_OK;
}

extern "C" {

bg_status bg_plan_create(int n, int d, int D_s, bg_field field, uint32_t p, bg_metric metric,
                         int n_states, int n_assign, const uint8_t* assign, bg_plan** out) {
    return create_plan(n, d, D_s, field, p, metric, n_states, n_assign, assign, nullptr, 0u, out);
}

bg_status bg_plan_create_mixed(int n, int d, int D_s, bg_field field, uint32_t p, bg_metric metric,
                               int n_states, int n_assign, const uint8_t* assign, uint32_t four_dim_legs,
                               bg_plan** out) {
    if (n_assign > 1 && !assign) {
        g_last_error.clear();
        if (out) *out = nullptr;
        return fail(BG_ERR_UNSUPPORTED, "mixed plans take an explicit assignment table");
    }
    return create_plan(n, d, D_s, field, p, metric, n_states, n_assign, assign, nullptr, four_dim_legs, out);
}

bg_status bg_plan_create_product(int n, int d, int D_s, bg_field field, uint32_t p, bg_metric metric,
                                 int n_states, const uint8_t* states_per_leg, bg_plan** out) {
    g_last_error.clear();
    if (!out) return fail(BG_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!states_per_leg) return fail(BG_ERR_INVALID_ARG, "states_per_leg is NULL");
    if (n < 4 || n > 12) return fail(BG_ERR_INVALID_ARG, "n = %d outside [4, 12]", n);
    if (n_states < 1 || n_states > 255) return fail(BG_ERR_INVALID_ARG, "n_states = %d", n_states);
    int64_t h = 1;
    for (int l = 0; l < n; ++l) {
        if (states_per_leg[l] < 1 || states_per_leg[l] > n_states)
            return fail(BG_ERR_INVALID_ARG, "states_per_leg[%d] = %d outside [1, n_states]", l, states_per_leg[l]);
        h *= states_per_leg[l];
        if (h * n > (1 << 20)) return fail(BG_ERR_INVALID_ARG, "product of states_per_leg too large");
    }
    return create_plan(n, d, D_s, field, p, metric, n_states, (int)h, nullptr, states_per_leg, 0u, out);
}

bg_status bg_plan_destroy(bg_plan* plan) {
    if (!plan) return BG_OK;
    if (plan->d_assign) cudaFree(plan->d_assign);
    delete plan;
    return BG_OK;
}

static int64_t resident_blocks(const bg_plan* pl) { return (int64_t)pl->blocks_per_sm * pl->sm_count; }

bg_status bg_workspace_size(const bg_plan* plan, int64_t E, size_t* bytes) {
    if (!plan || !bytes || E < 0) return fail(BG_ERR_INVALID_ARG, "bad argument to bg_workspace_size");
    *bytes = bgi::workspace_bytes(plan, E, E * plan->H);
    return BG_OK;
}

}  // extern "C"

namespace bgi {

bool uses_lanes(const bg_plan* plan, int64_t select_items) {
    return !plan->all_states && plan->lentry && select_items <= plan->lanes_max_items;
}

bg_status launch_lanes(const bg_plan* plan, int64_t E, const void* momenta, const void* eps, void* out,
                       uint8_t* status, int dev, cudaStream_t stream, int64_t select_items) {
    const bool team = plan->tentry && select_items <= plan->team_max_items;
    const bgk::LanesEntry* le = team ? plan->tentry : plan->lentry;
    const size_t smem = team ? plan->team_smem : plan->lanes_smem;
    bg_status st;
    if (dev != plan->device && (st = ensure_smem_limit(le->func, dev, smem)) != BG_OK) return st;
    const int64_t items = E * plan->H;
    const int64_t ppb = le->block / (le->L * le->G);
    int64_t blocks = (items + ppb - 1) / ppb;
    const int64_t cap = (int64_t)(team ? plan->team_blocks_per_sm : plan->lanes_blocks_per_sm) * plan->sm_count;
    if (blocks > cap) blocks = cap;
    bgk::CompactArgs a;
    a.E = E; a.H = plan->H; a.S = plan->S; a.n = plan->n;
    a.d_in = plan->d; a.ds_in = plan->Ds;
    a.k = momenta; a.eps = eps; a.out = out; a.status = status;
    a.assign = plan->d_assign; a.ws = nullptr;
    a.four_d_legs = 0;
    a.violation = violation_word(dev);
    le->launch(compact_params(plan), &a, dim3((unsigned)blocks), smem, stream);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return fail(BG_ERR_CUDA, "launch failed: %s", cudaGetErrorString(err));
    return BG_OK;
}

size_t workspace_bytes(const bg_plan* plan, int64_t E, int64_t select_items) {
    if (E <= 0) return 0;
    if (plan->all_states) {
        if (!plan->states_global) return 0;
        const int64_t per_block = (int64_t)bgk::kStatesWarps * plan->sgeo.P;
        int64_t blocks = (E + per_block - 1) / per_block;
        if (blocks > resident_blocks(plan)) blocks = resident_blocks(plan);
        return (size_t)blocks * per_block * plan->sgeo.words * plan->sentry->elem_bytes;
    }
    if (!plan->entry->global_table) return 0;
    if (uses_lanes(plan, select_items)) return 0;      // lanes kernel: shared memory only
    const int64_t items = E * plan->H;
    const int B = plan->entry->block;
    int64_t blocks = (items + B - 1) / B;
    if (blocks > resident_blocks(plan)) blocks = resident_blocks(plan);
    return (size_t)blocks * B * plan->words * plan->entry->elem_bytes;
}

}  // namespace bgi

extern "C" {

bg_status bg_plan_describe(const bg_plan* plan, char* buf, size_t len) {
    if (!plan || !buf) return fail(BG_ERR_INVALID_ARG, "bad argument to bg_plan_describe");
    const auto* e = plan->entry;
    if (plan->all_states) {
        int w = snprintf(buf, len,
                         "field=%s n=%d d=%d D_s=%d kernel=states kernel_D=%d kernel_D_s=%d metric=%s "
                         "table=%s states=%d assignments=%d warps_per_block=%d points_per_warp=%d "
                         "blocks_per_sm=%d smem=%zu words_per_point=%d elem_bytes=%d",
                         field_name(plan->field), plan->n, plan->d, plan->Ds, plan->sentry->D,
                         plan->sentry->DS, plan->metric == BG_METRIC_MOSTLY_MINUS ? "mostly_minus" : "alternating",
                         plan->states_global ? "global" : "shared", plan->S, plan->H, bgk::kStatesWarps,
                         plan->sgeo.P, plan->blocks_per_sm, plan->smem_bytes, plan->sgeo.words, plan->sentry->elem_bytes);
        if (w < 0 || (size_t)w >= len) return fail(BG_ERR_INVALID_ARG, "buffer too small");
        return BG_OK;
    }
    int w = snprintf(buf, len,
                     "field=%s n=%d d=%d D_s=%d kernel=compact kernel_D=%d kernel_D_s=%d metric=%s "
                     "table=%s block=%d blocks_per_sm=%d smem=%zu words_per_thread=%d elem_bytes=%d "
                     "four_dim_legs=0x%x lanes=%d lanes_max_items=%lld team_max_items=%lld",
                     field_name(plan->field), plan->n, plan->d, plan->Ds, e->D, e->DS,
                     plan->metric == BG_METRIC_MOSTLY_MINUS ? "mostly_minus" : "alternating",
                     e->split ? "split" : e->global_table ? "global" : "shared", e->block, plan->blocks_per_sm,
                     plan->smem_bytes, plan->words, e->elem_bytes, plan->four_d_legs,
                     plan->lentry ? plan->lentry->L : 0, (long long)plan->lanes_max_items,
                     (long long)plan->team_max_items);
    if (w < 0 || (size_t)w >= len) return fail(BG_ERR_INVALID_ARG, "buffer too small");
    return BG_OK;
}

namespace {

bg_status eval_impl(const bg_plan* plan, int64_t E, const void* momenta, const void* eps, void* out,
                    uint8_t* status, void* workspace, size_t workspace_bytes, cudaStream_t stream,
                    bool mapped_host_ok, int64_t select_items) {
    g_last_error.clear();
    if (!plan) return fail(BG_ERR_INVALID_ARG, "plan is NULL");
    if (E < 0) return fail(BG_ERR_INVALID_ARG, "E = %lld < 0", (long long)E);
    if (E == 0) return BG_OK;
    if (!momenta || !eps || !out) return fail(BG_ERR_INVALID_ARG, "momenta, eps and out must be non-NULL");
    if (E > (int64_t(1) << 40) / plan->H) return fail(BG_ERR_INVALID_ARG, "E too large");
    const size_t elem = value_bytes(plan->field), kelem = momentum_bytes(plan->field);
    if (((uintptr_t)eps | (uintptr_t)out) % elem || (uintptr_t)momenta % kelem)
        return fail(BG_ERR_INVALID_ARG, "momenta, eps and out must be aligned to their element sizes "
                    "(%zu, %zu, %zu bytes)", kelem, elem, elem);
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return fail(BG_ERR_CUDA, "no current CUDA device");
    }
    if (plan->d_assign && dev != plan->device)
        return fail(BG_ERR_CUDA, "plan was created on device %d, current device is %d", plan->device, dev);
    bg_status st;
    if ((st = bgi::check_kernel_ptr(momenta, "momenta", dev, mapped_host_ok)) != BG_OK) return st;
    if ((st = bgi::check_kernel_ptr(eps, "eps", dev, mapped_host_ok)) != BG_OK) return st;
    if ((st = bgi::check_kernel_ptr(out, "out", dev, mapped_host_ok)) != BG_OK) return st;
    if (status && (st = bgi::check_kernel_ptr(status, "status", dev, mapped_host_ok)) != BG_OK) return st;

    const bgk::KernelEntry* e = plan->entry;
    const size_t need = bgi::workspace_bytes(plan, E, select_items);
    if (need > 0) {
        if (!workspace || workspace_bytes < need)
            return fail(BG_ERR_INVALID_ARG, "workspace of %zu B needed, %zu B given", need, workspace_bytes);
        if ((uintptr_t)workspace % 256) return fail(BG_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
        if ((st = check_device_ptr(workspace, "workspace", dev)) != BG_OK) return st;
    }
    if (!plan->all_states && dev != plan->device && plan->smem_bytes > 0) {
        if ((st = bgi::ensure_smem_limit(e->func, dev, plan->smem_bytes)) != BG_OK) return st;
    }

    if (plan->all_states) {
        if (dev != plan->device && plan->smem_bytes > 0) {
            if ((st = bgi::ensure_smem_limit(plan->sentry->func, dev, plan->smem_bytes)) != BG_OK) return st;
        }
        const int64_t per_block = (int64_t)bgk::kStatesWarps * plan->sgeo.P;
        int64_t blocks = (E + per_block - 1) / per_block;
        if (blocks > resident_blocks(plan)) blocks = resident_blocks(plan);
        bgk::StatesArgs a;
        a.E = E; a.n = plan->n; a.d_in = plan->d; a.ds_in = plan->Ds;
        a.k = momenta; a.eps = eps; a.out = out; a.status = status;
        a.ws = plan->states_global ? workspace : nullptr;
        a.violation = bgi::violation_word(dev);
        if (bgi::fault(BG_FAULT_LAUNCH)) return fail(BG_ERR_CUDA, "launch failed: injected fault");
        plan->sentry->launch(compact_params(plan), a, plan->sgeo, dim3((unsigned)blocks), plan->smem_bytes,
                             stream);
        cudaError_t err = cudaGetLastError();
        if (err != cudaSuccess) return fail(BG_ERR_CUDA, "launch failed: %s", cudaGetErrorString(err));
        return BG_OK;
    }
    if (bgi::fault(BG_FAULT_LAUNCH)) return fail(BG_ERR_CUDA, "launch failed: injected fault");
    const int64_t items = E * plan->H;
    if (bgi::uses_lanes(plan, select_items))
        return bgi::launch_lanes(plan, E, momenta, eps, out, status, dev, stream, select_items);
    int64_t blocks = (items + e->block - 1) / e->block;
    const int64_t cap = e->global_table ? resident_blocks(plan) : resident_blocks(plan) * 256;
    if (blocks > cap) blocks = cap;
    bgk::CompactArgs a;
    a.E = E; a.H = plan->H; a.S = plan->S; a.n = plan->n;
    a.d_in = plan->d; a.ds_in = plan->Ds;
    a.k = momenta; a.eps = eps; a.out = out; a.status = status;
    a.assign = plan->d_assign; a.ws = workspace;
    a.four_d_legs = plan->four_d_legs;
    a.violation = bgi::violation_word(dev);
    e->launch(compact_params(plan), &a, dim3((unsigned)blocks), plan->smem_bytes, stream);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return fail(BG_ERR_CUDA, "launch failed: %s", cudaGetErrorString(err));
    return BG_OK;
}

}  // namespace

bg_status bg_eval(const bg_plan* plan, int64_t E, const void* momenta, const void* eps, void* out,
                  uint8_t* status, void* workspace, size_t workspace_bytes, cudaStream_t stream) {
    bgi::Range nvtx("bg_eval");
    return eval_impl(plan, E, momenta, eps, out, status, workspace, workspace_bytes, stream, false,
                     plan ? E * plan->H : 0);
}

}  // extern "C"

namespace bgi {

bg_status eval_mapped(const bg_plan* plan, int64_t E, const void* momenta, const void* eps, void* out,
                      uint8_t* status, void* workspace, size_t workspace_bytes, cudaStream_t stream) {
    Range nvtx("bg_eval_mapped");
    return eval_impl(plan, E, momenta, eps, out, status, workspace, workspace_bytes, stream, true,
                     plan ? E * plan->H : 0);
}

bg_status eval_part(const bg_plan* plan, int64_t E, const void* momenta, const void* eps, void* out,
                    uint8_t* status, void* workspace, size_t workspace_bytes, cudaStream_t stream,
                    int64_t batch_items) {
    return eval_impl(plan, E, momenta, eps, out, status, workspace, workspace_bytes, stream, false, batch_items);
}

}  // namespace bgi
