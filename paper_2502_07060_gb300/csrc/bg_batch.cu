// bg_batch.cu -- uneven batches: many groups of points with different n, d,
// D_s, metric and number type evaluated by one CUDA-graph launch.
//
// A batch is built once from its groups (each group: a plan and its device
// buffers).  The host orders the groups by decreasing cost per point, cuts
// them into tiles, stores the group and tile tables in the caller's workspace
// and captures a graph: reset the tile counters, then the F_p and the complex
// persistent kernels as two parallel branches (they use different pipes: the
// integer multiply pipe and the FP64 pipe, so they can share SMs).  Each
// branch's grid is one resident wave, optionally capped per SM; the caps and
// the tile size are the knobs that bg_batch_autotune searches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "bg_batch.cuh"
#include "bg_internal.h"

namespace {

using bgk::kBlockC64Batch;
using bgk::kBlockFpBatch;
constexpr int kTuneTiles[] = {64, 256, 1024, 4096}; // autotune candidates (points per tile)
constexpr int kTuneFpCaps[] = {0, 3, 2};            // F_p blocks per SM (0 = all that fit; see fp_wide)
constexpr int kTuneC64Caps[] = {0, 3, 2, 1};        // C64 blocks per SM
constexpr int kTuneLanes[] = {0, 2048};             // lane groups for groups of at most this many items

size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

// relative cost of one point (field multiplications of the regrouped form;
// complex points weighted by their FP64 FMAs, the FP64 pipe being far slower
// per operation than the integer multiply pipe)
double point_cost(int n, int D, int DS, bg_field field) {
    const int N = n - 1;
    double tot = 0;
    const double kw = field == BG_FIELD_C64_REAL ? 0.5 : 1.0;    // momentum terms
    for (int m = 2; m <= N; ++m) {
        const double per = (m - 1) * (3.0 * DS + 3.0 * kw * D) + (m - 1) * (m - 2) * DS;
        tot += (N - m + 1) * per;
    }
    return field == BG_FIELD_FP ? tot : 8.0 * tot;
}

struct FieldPart {
    std::vector<bgk::BatchGroup> groups;
    std::vector<bgk::BatchTile> tiles;
    int words = 0;                      // largest table, elements per thread
    int blocks = 0;                     // grid
    bool wide = true;                   // F_p: the kernel built for 1-2 blocks per SM
    size_t off_groups = 0, off_tiles = 0, off_tables = 0;
};

struct Layout {
    FieldPart part[2];                  // [0] = complex (C64, C64_REAL), [1] = F_p
    size_t bytes = 0;
};

// The F_p kernel build a residency cap selects: caps of one or two blocks per
// SM take the build for few blocks (no body spills much); no cap or three to
// four blocks take the build for four (bg_batch.cuh).
bool fp_wide(int cap) { return cap == 1 || cap == 2; }

bg_status build_layout(const bg_group* groups, int n_groups, const bg_batch_config* cfg, int dev,
                       Layout* L) {
    if (!groups || n_groups < 1) return bgi::fail(BG_ERR_INVALID_ARG, "no groups");
    const int tile = cfg && cfg->tile_points > 0 ? cfg->tile_points : 1024;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    struct Item { int idx; double cost; };
    std::vector<Item> order;
    for (int gi = 0; gi < n_groups; ++gi) {
        const bg_group& g = groups[gi];
        if (!g.plan) return bgi::fail(BG_ERR_INVALID_ARG, "group %d has no plan", gi);
        if (g.E < 0) return bgi::fail(BG_ERR_INVALID_ARG, "group %d has E < 0", gi);
        if (g.E == 0) continue;
        if (!g.momenta || !g.eps || !g.out) return bgi::fail(BG_ERR_INVALID_ARG, "group %d: NULL buffer", gi);
        const bg_plan* pl = g.plan;
        if (pl->all_states)
            return bgi::fail(BG_ERR_UNSUPPORTED, "group %d: all-assignment plans are evaluated by bg_eval", gi);
        if (g.E > (int64_t(1) << 40) / pl->H) return bgi::fail(BG_ERR_INVALID_ARG, "group %d too large", gi);
        const int D = bgi::round_dim(pl->d), DS = bgi::round_dim(pl->Ds);
        order.push_back({gi, point_cost(pl->n, D, DS, pl->field) * pl->H});
    }
    std::stable_sort(order.begin(), order.end(), [](const Item& a, const Item& b) { return a.cost > b.cost; });
    for (const Item& it : order) {
        const bg_group& g = groups[it.idx];
        const bg_plan* pl = g.plan;
        FieldPart& fpart = L->part[pl->field == BG_FIELD_FP ? 1 : 0];
        const int D = bgi::round_dim(pl->d), DS = bgi::round_dim(pl->Ds);
        bgk::BatchGroup bgd{};
        bgd.args.E = g.E;
        bgd.args.H = pl->H;
        bgd.args.S = pl->S;
        bgd.args.n = pl->n;
        bgd.args.d_in = pl->d;
        bgd.args.ds_in = pl->Ds;
        bgd.args.k = g.momenta;
        bgd.args.eps = g.eps;
        bgd.args.out = g.out;
        bgd.args.status = g.status;
        bgd.args.assign = pl->d_assign;
        bgd.args.ws = nullptr;
        bgd.args.four_d_legs = 0;   // full width: exact for mixed plans as well
        bgd.args.violation = bgi::violation_word(pl->device);
        bgd.variant = 2 * bgk::batch_pair_index(D, DS) + (int)pl->metric +
                      (pl->field == BG_FIELD_C64_REAL ? bgk::kBatchVariants : 0);
        bgd.fp = pl->fpo;
        const int64_t items_g = g.E * pl->H;
        bgd.lanes = (cfg && cfg->lanes_max_items > 0 && items_g <= cfg->lanes_max_items) ? (DS <= 4 ? 4 : 8) : 0;
        const int gidx = (int)fpart.groups.size();
        fpart.groups.push_back(bgd);
        fpart.words = std::max(fpart.words, bgk::Geometry{pl->n - 1}.words(D, DS));
        fpart.words = std::max(fpart.words, bgk::LaneGeometry{pl->n - 1}.words());
        const int64_t items = g.E * pl->H;
        // a group on lane groups takes tiles of one pass of a block (block / L
        // items): its items have the longest latency per block, so they spread
        // over as many blocks as possible
        const int gtile = bgd.lanes ? (pl->field == BG_FIELD_FP ? kBlockFpBatch : kBlockC64Batch) / bgd.lanes : tile;
        for (int64_t first = 0; first < items; first += gtile) {
            bgk::BatchTile t;
            t.group = gidx;
            t.first = first;
            t.count = (int)std::min<int64_t>(gtile, items - first);
            fpart.tiles.push_back(t);
        }
    }
    // grids: one resident wave, capped per SM by the configuration
    size_t off = 256;                    // [0, 256): the two tile counters
    for (int f = 0; f < 2; ++f) {
        FieldPart& P = L->part[f];
        if (P.tiles.empty()) continue;
        const int cap = cfg ? (f ? cfg->fp_blocks_per_sm : cfg->c64_blocks_per_sm) : 0;
        if (f) P.wide = fp_wide(cap);
        const void* func = f ? bgk::batch_kernel_fp(P.wide) : bgk::batch_kernel_c64();
        const int block = f ? kBlockFpBatch : kBlockC64Batch;
        int occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, func, block, 0) != cudaSuccess || occ < 1) {
            cudaGetLastError();
            return bgi::fail(BG_ERR_UNSUPPORTED, "batch kernel cannot be resident");
        }
        if (cap > 0 && cap < occ) occ = cap;
        P.blocks = std::min<int64_t>((int64_t)occ * sms, (int64_t)P.tiles.size());
        const size_t elem = f ? 4 : 16;
        P.off_groups = off;
        off += up256(P.groups.size() * sizeof(bgk::BatchGroup));
        P.off_tiles = off;
        off += up256(P.tiles.size() * sizeof(bgk::BatchTile));
        P.off_tables = off;
        off += up256((size_t)P.blocks * block * P.words * elem);
    }
    L->bytes = off;
    return BG_OK;
}

}  // namespace

struct bg_batch {
    int device = -1;
    Layout L;
    unsigned char* ws = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

extern "C" {

bg_status bg_batch_workspace_size(const bg_group* groups, int n_groups, const bg_batch_config* cfg,
                                  size_t* bytes) {
    if (!bytes) return bgi::fail(BG_ERR_INVALID_ARG, "bytes is NULL");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return bgi::fail(BG_ERR_CUDA, "no current CUDA device");
    }
    if (cfg) {
        Layout L;
        bg_status st = build_layout(groups, n_groups, cfg, dev, &L);
        if (st != BG_OK) return st;
        *bytes = L.bytes;
        return BG_OK;
    }
    // no configuration: the largest workspace any autotune candidate (or the
    // default configuration of bg_batch_create) needs; uncapped residency is
    // the largest grid
    size_t mx = 0;
    for (int t : kTuneTiles)
        for (int ln : kTuneLanes) {
            bg_batch_config c{t, 0, 0, ln};
            Layout L;
            bg_status st = build_layout(groups, n_groups, &c, dev, &L);
            if (st != BG_OK) return st;
            mx = std::max(mx, L.bytes);
        }
    *bytes = mx;
    return BG_OK;
}

bg_status bg_batch_create(const bg_group* groups, int n_groups, const bg_batch_config* cfg,
                          void* workspace, size_t workspace_bytes, bg_batch** out) {
    if (!out) return bgi::fail(BG_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return bgi::fail(BG_ERR_CUDA, "no current CUDA device");
    }
    bg_batch* b = new (std::nothrow) bg_batch();
    if (!b) return bgi::fail(BG_ERR_NOMEM, "host allocation failed");
    b->device = dev;
    // cfg NULL: the configuration the autotuner picked most often on GB300 --
    // small tiles, lane groups for small groups, and the F_p kernel build
    // below (the 54-group uneven batch measured 92.5 ms with 1024-point tiles,
    // no lane groups and a single F_p build)
    bg_batch_config dflt{256, 0, 0, 2048};
    if (!cfg && groups) {
        bool fp = false;
        for (int gi = 0; gi < n_groups; ++gi)
            if (groups[gi].plan && groups[gi].E > 0 && groups[gi].plan->field == BG_FIELD_FP) fp = true;
        // the F_p kernel built for four blocks per SM when most F_p work items
        // run one per thread (large groups), the one for two when most run on
        // lane groups (small groups): the autotuner's picks on GB300 (54-group
        // batch of 77672 points per group: 82.6 ms against 83.2 ms with the
        // two-block build; 27 F_p groups of 155344 points: 7.85 against
        // 9.15 ms; of 512 points: 0.155 ms against 0.26 ms the other way)
        int64_t thread_items = 0, lane_items = 0;
        for (int gi = 0; gi < n_groups; ++gi)
            if (groups[gi].plan && groups[gi].E > 0 && groups[gi].plan->field == BG_FIELD_FP) {
                const int64_t items = groups[gi].E * groups[gi].plan->H;
                (items <= dflt.lanes_max_items ? lane_items : thread_items) += items;
            }
        if (fp) dflt.fp_blocks_per_sm = thread_items >= lane_items ? 0 : 2;
        cfg = &dflt;
    }
    bg_status st = build_layout(groups, n_groups, cfg, dev, &b->L);
    if (st != BG_OK) { delete b; return st; }
    if (!workspace || workspace_bytes < b->L.bytes || (uintptr_t)workspace % 256) {
        const size_t need = b->L.bytes;
        delete b;
        return bgi::fail(BG_ERR_INVALID_ARG, "workspace of %zu B (256-byte aligned) needed", need);
    }
    if ((st = bgi::check_device_ptr(workspace, "workspace", dev)) != BG_OK) { delete b; return st; }
    for (int gi = 0; gi < n_groups; ++gi) {
        if (groups[gi].E == 0) continue;
        const bg_plan* pl = groups[gi].plan;
        if (pl->d_assign && pl->device != dev) { delete b; return bgi::fail(BG_ERR_CUDA, "group %d: plan on another device", gi); }
        if ((st = bgi::check_device_ptr(groups[gi].momenta, "momenta", dev)) != BG_OK ||
            (st = bgi::check_device_ptr(groups[gi].eps, "eps", dev)) != BG_OK ||
            (st = bgi::check_device_ptr(groups[gi].out, "out", dev)) != BG_OK ||
            (groups[gi].status && (st = bgi::check_device_ptr(groups[gi].status, "status", dev)) != BG_OK)) {
            delete b;
            return st;
        }
    }
    b->ws = static_cast<unsigned char*>(workspace);
    // group and tile tables -> workspace
    for (int f = 0; f < 2; ++f) {
        FieldPart& P = b->L.part[f];
        if (P.tiles.empty()) continue;
        if (cudaMemcpy(b->ws + P.off_groups, P.groups.data(), P.groups.size() * sizeof(bgk::BatchGroup),
                       cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(b->ws + P.off_tiles, P.tiles.data(), P.tiles.size() * sizeof(bgk::BatchTile),
                       cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaGetLastError();
            delete b;
            return bgi::fail(BG_ERR_CUDA, "upload of the batch tables failed");
        }
    }
    // capture: reset counters; F_p and C64 kernels on two parallel branches
    cudaStream_t s0 = nullptr, s1 = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    cudaError_t err = cudaStreamCreateWithFlags(&s0, cudaStreamNonBlocking);
    if (!err) err = cudaStreamCreateWithFlags(&s1, cudaStreamNonBlocking);
    if (!err) err = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
    if (!err) err = cudaEventCreateWithFlags(&join, cudaEventDisableTiming);
    if (!err) err = cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal);
    if (!err) err = cudaMemsetAsync(b->ws, 0, 256, s0);
    if (!err) err = cudaEventRecord(fork, s0);
    if (!err) err = cudaStreamWaitEvent(s1, fork, 0);
    for (int f = 0; f < 2 && !err; ++f) {
        FieldPart& P = b->L.part[f];
        if (P.tiles.empty()) continue;
        bgk::BatchArgs a;
        a.groups = reinterpret_cast<const bgk::BatchGroup*>(b->ws + P.off_groups);
        a.tiles = reinterpret_cast<const bgk::BatchTile*>(b->ws + P.off_tiles);
        a.n_tiles = (int)P.tiles.size();
        a.counter = reinterpret_cast<int*>(b->ws) + f;
        a.tables = b->ws + P.off_tables;
        a.words = P.words;
        if (f) bgk::launch_batch_fp(a, P.blocks, P.wide, s0);
        else bgk::launch_batch_c64(a, P.blocks, s1);
        err = cudaGetLastError();
    }
    if (!err) err = cudaEventRecord(join, s1);
    if (!err) err = cudaStreamWaitEvent(s0, join, 0);
    cudaGraph_t graph = nullptr;
    cudaError_t end = cudaStreamEndCapture(s0, &graph);
    if (!err) err = end;
    if (!err) err = cudaGraphInstantiate(&b->exec, graph, 0);
    b->graph = graph;
    if (fork) cudaEventDestroy(fork);
    if (join) cudaEventDestroy(join);
    if (s0) cudaStreamDestroy(s0);
    if (s1) cudaStreamDestroy(s1);
    if (err) {
        cudaGetLastError();
        bg_batch_destroy(b);
        return bgi::fail(BG_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(err));
    }
    *out = b;
    return BG_OK;
}

bg_status bg_batch_launch(const bg_batch* batch, cudaStream_t stream) {
    bgi::Range nvtx("bg_batch_launch");
    if (!batch || !batch->exec) return bgi::fail(BG_ERR_INVALID_ARG, "batch is NULL");
    if (bgi::fault(BG_FAULT_LAUNCH)) return bgi::fail(BG_ERR_CUDA, "graph launch failed: injected fault");
    cudaError_t err = cudaGraphLaunch(batch->exec, stream);
    if (err != cudaSuccess) {
        cudaGetLastError();
        return bgi::fail(BG_ERR_CUDA, "graph launch failed: %s", cudaGetErrorString(err));
    }
    return BG_OK;
}

bg_status bg_batch_describe(const bg_batch* batch, char* buf, size_t len) {
    if (!batch || !buf) return bgi::fail(BG_ERR_INVALID_ARG, "bad argument to bg_batch_describe");
    const FieldPart& F = batch->L.part[1];
    const FieldPart& C = batch->L.part[0];
    int w = snprintf(buf, len,
                     "fp: groups=%zu tiles=%zu blocks=%d words=%d kernel=%s; c64: groups=%zu tiles=%zu "
                     "blocks=%d words=%d; workspace=%zu",
                     F.groups.size(), F.tiles.size(), F.blocks, F.words, F.wide ? "wide" : "narrow",
                     C.groups.size(), C.tiles.size(),
                     C.blocks, C.words, batch->L.bytes);
    if (w < 0 || (size_t)w >= len) return bgi::fail(BG_ERR_INVALID_ARG, "buffer too small");
    return BG_OK;
}

bg_status bg_batch_destroy(bg_batch* batch) {
    if (!batch) return BG_OK;
    if (batch->exec) cudaGraphExecDestroy(batch->exec);
    if (batch->graph) cudaGraphDestroy(batch->graph);
    delete batch;
    return BG_OK;
}

}  // extern "C"

namespace {

// Key of a batch's group mix for the autotune cache: the device, the library
// version and, for every non-empty group in a canonical order, its
// configuration and its size rounded up to a power of two (FNV-1a, 64 bit).
std::string tune_key(const bg_group* groups, int n_groups, int dev) {
    std::vector<std::string> parts;
    for (int g = 0; g < n_groups; ++g) {
        const bg_plan* pl = groups[g].plan;
        if (!pl || groups[g].E <= 0) continue;
        int lg = 0;
        while ((int64_t(1) << lg) < groups[g].E) ++lg;
        char buf[128];
        snprintf(buf, sizeof buf, "%d:%d:%d:%d:%d:%u:%d:%d:%x:%d", (int)pl->field, pl->n, pl->d, pl->Ds,
                 (int)pl->metric, pl->p, pl->S, pl->H, pl->four_d_legs, lg);
        parts.push_back(buf);
    }
    std::sort(parts.begin(), parts.end());
    cudaDeviceProp prop{};
    cudaGetDeviceProperties(&prop, dev);
    std::string all = std::string(prop.name) + "/" + std::to_string(prop.multiProcessorCount) + "/v" +
                      std::to_string(BG_VERSION);
    for (const auto& x : parts) all += "|" + x;
    uint64_t h = 1469598103934665603ull;
    for (unsigned char c : all) {
        h ^= c;
        h *= 1099511628211ull;
    }
    char hex[17];
    snprintf(hex, sizeof hex, "%016llx", (unsigned long long)h);
    return hex;
}

// A cached result for `key` in the file `path` (lines "key tile fp_cap
// c64_cap lanes_max_items ms"; the last matching line wins).
bool tune_lookup(const char* path, const std::string& key, bg_batch_config* cfg, double* ms) {
    FILE* f = fopen(path, "r");
    if (!f) return false;
    char k[64];
    int t, fc, cc, ln;
    double m;
    bool found = false;
    while (fscanf(f, "%63s %d %d %d %d %lf", k, &t, &fc, &cc, &ln, &m) == 6) {
        if (key == k && t > 0 && fc >= 0 && cc >= 0 && ln >= 0) {
            *cfg = bg_batch_config{t, fc, cc, ln};
            *ms = m;
            found = true;
        }
    }
    fclose(f);
    return found;
}

void tune_store(const char* path, const std::string& key, const bg_batch_config& cfg, double ms) {
    FILE* f = fopen(path, "a");
    if (!f) {
        bgi::log("autotune cache %s not writable", path);
        return;
    }
    fprintf(f, "%s %d %d %d %d %.6f\n", key.c_str(), cfg.tile_points, cfg.fp_blocks_per_sm, cfg.c64_blocks_per_sm,
            cfg.lanes_max_items, ms);
    fclose(f);
}

}  // namespace

extern "C" {

// Time every candidate configuration (tile size x residency caps) on the
// caller's batch and return the fastest.  Each candidate: one warm-up launch
// and `reps` timed launches of its graph on `stream`.  With BG_AUTOTUNE_CACHE
// naming a file, a result stored there for the same device and group mix is
// returned without timing, and a new result is appended.
bg_status bg_batch_autotune(const bg_group* groups, int n_groups, void* workspace, size_t workspace_bytes,
                            int reps, cudaStream_t stream, bg_batch_config* best, double* best_ms) {
    if (!best) return bgi::fail(BG_ERR_INVALID_ARG, "best is NULL");
    if (!groups || n_groups < 1) return bgi::fail(BG_ERR_INVALID_ARG, "groups required");
    if (reps < 1) reps = 1;
    const char* cache = getenv("BG_AUTOTUNE_CACHE");
    std::string key;
    if (cache && *cache) {
        int dev = 0;
        cudaGetDevice(&dev);
        key = tune_key(groups, n_groups, dev);
        double ms = 0;
        if (tune_lookup(cache, key, best, &ms)) {
            if (best_ms) *best_ms = ms;
            bgi::log("autotune cache hit %s: tile %d, caps %d/%d, lanes %d, %.3f ms", key.c_str(), best->tile_points,
                     best->fp_blocks_per_sm, best->c64_blocks_per_sm, best->lanes_max_items, ms);
            return BG_OK;
        }
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        return bgi::fail(BG_ERR_CUDA, "event creation failed");
    }
    double best_t = -1.0;
    bg_status result = BG_OK;
    for (int t : kTuneTiles)
        for (int fc : kTuneFpCaps)
            for (int cc : kTuneC64Caps)
              for (int ln : kTuneLanes) {
                bg_batch_config cfg{t, fc, cc, ln};
                bg_batch* b = nullptr;
                bg_status st = bg_batch_create(groups, n_groups, &cfg, workspace, workspace_bytes, &b);
                if (st != BG_OK) { result = st; continue; }
                float ms = 0.f;
                bool ok = bg_batch_launch(b, stream) == BG_OK && cudaEventRecord(e0, stream) == cudaSuccess;
                for (int r = 0; r < reps && ok; ++r) ok = bg_batch_launch(b, stream) == BG_OK;
                ok = ok && cudaEventRecord(e1, stream) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
                     cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
                bg_batch_destroy(b);
                if (!ok) {
                    cudaGetLastError();
                    result = bgi::fail(BG_ERR_CUDA, "timing a candidate failed");
                    continue;
                }
                const double per = ms / reps;
                if (best_t < 0 || per < best_t) {
                    best_t = per;
                    *best = cfg;
                }
              }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (best_t < 0) return result != BG_OK ? result : bgi::fail(BG_ERR_CUDA, "no candidate ran");
    if (best_ms) *best_ms = best_t;
    bgi::log("autotune: tile %d, caps %d/%d, lanes %d, %.3f ms", best->tile_points, best->fp_blocks_per_sm,
             best->c64_blocks_per_sm, best->lanes_max_items, best_t);
    if (!key.empty()) tune_store(cache, key, *best, best_t);
    return BG_OK;
}

}  // extern "C"
