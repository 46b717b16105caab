// bg_lanes.cuh -- the recursion for SMALL batches: one point per group of L
// lanes (L = 4 when D_s <= 4, else 8), lane mu owning component mu of every
// vector of its point.
//
// With one point per thread (bg_compact.cuh) a batch of a few thousand
// points occupies a few thousand threads, and each thread runs the whole
// recursion serially: the latency of one point bounds the call (the flat
// part of the time-against-points curve of Sec. 3.2).  Here the component
// loops of that recursion run across the lanes of a group: a vector update
// (scalar times current, J = R / P^2) is one component per lane with no
// communication, and a Minkowski contraction is one product per lane summed
// over the group with xor shuffles.  The loops over lengths, ranges, splits
// and gaps are the compact kernel's (same regrouped sum, same Sec. 2.2
// recursion), run in lock step by the L lanes of a point.
//
// Each lane keeps its own words in shared memory (bg_lanes_kernel) or in its
// block's global table region (the uneven-batch kernel) -- its component of
// every current and prefix sum, and its copy of every per-range scalar (SA,
// 1/P^2, which all lanes of a point compute identically) -- at
// [word][thread], so no lane ever reads another lane's words and only the
// shuffles exchange data.  Per lane: NJ + (N+1) + 2 NS words (75 at n = 8).
//
// Teams (G = 32 / L groups, one warp, per point) serve the smallest batches:
// the groups evaluate the ranges of each length in parallel and share one
// table per team, lane mu of every group reading and writing the words of
// component mu ([word][team][mu]); group 0 stages the inputs, prefix sums and
// inverses, and a warp barrier separates the lengths.  Every range runs the
// same operations as in a group of its own, so the values are identical.
//
// F_p: the same Montgomery levels as FpOps; a contraction sums the lanes'
// products (L = 4: four products below 2^64; L = 8: each product first taken
// to 33 bits by redc_full) and reduces twice, so every coefficient equals
// the compact kernel's up to its representative and the stored currents and
// the amplitude are the same canonical residues.  Complex FP64: the lanes'
// partial products are summed by the shuffle tree, a different order from
// the compact kernel's sequential FMAs (rounding differences only).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>
#include <vector>

#include "bg_compact.cuh"

namespace bgk {

// Lane-group arithmetic: each lane holds one component (index mu) of its
// point's vectors.  Shuffles stay inside the group (xor offsets < L) and use
// the group's own mask, so groups of a warp may leave a grid-stride loop at
// different iterations.
template <class F, int L>
struct LaneOps;

template <int L>
struct LaneOps<FpOps, L> {
    using T = uint32_t;
    const FpOps& f;
    unsigned mask;
    __device__ __forceinline__ uint64_t sum64(uint64_t x) const {
#pragma unroll
        for (int o = L / 2; o > 0; o >>= 1) x += __shfl_xor_sync(mask, x, o, L);
        return x;
    }
    // sum over the group of eta_mu a b (a, b < p, or a = p - x for eta = -1
    // is formed here): level 2 products -> level 0 coefficient in [0, p)
    template <int METRIC>
    __device__ __forceinline__ uint32_t dot(uint32_t a, uint32_t b, int mu) const {
        const uint32_t x = msign<METRIC>(mu) > 0 ? a : f.p - a;
        const uint64_t t = static_cast<uint64_t>(x) * b;          // < p^2 < 2^62
        uint64_t S;
        if constexpr (L <= 4) {
            S = f.redc_full(sum64(t));                             // four products < 2^64
        } else {
            S = sum64(f.redc_full(t));                              // eight values < 2^33
        }
        return f.fold(f.redc(S));
    }
};

template <int L>
struct LaneOpsC {
    __device__ __forceinline__ static double2 sum(double2 v, unsigned mask) {
#pragma unroll
        for (int o = L / 2; o > 0; o >>= 1) {
            v.x += __shfl_xor_sync(mask, v.x, o, L);
            v.y += __shfl_xor_sync(mask, v.y, o, L);
        }
        return v;
    }
};

template <int L>
struct LaneOps<C64Ops, L> {
    using T = double2;
    const C64Ops& f;
    unsigned mask;
    template <int METRIC>
    __device__ __forceinline__ double2 dot(double2 a, double2 b, int mu) const {
        const double s = msign<METRIC>(mu);
        double2 t = make_double2(s * fma(a.x, b.x, -a.y * b.y), s * fma(a.x, b.y, a.y * b.x));
        return LaneOpsC<L>::sum(t, mask);
    }
};

template <int L>
struct LaneOps<C64ROps, L> {
    using T = double2;
    const C64ROps& f;
    unsigned mask;
    template <int METRIC>
    __device__ __forceinline__ double2 dot(double2 a, double2 b, int mu) const {
        const double s = msign<METRIC>(mu);
        double2 t = make_double2(s * fma(a.x, b.x, -a.y * b.y), s * fma(a.x, b.y, a.y * b.x));
        return LaneOpsC<L>::sum(t, mask);
    }
    // real momentum component times complex current component
    template <int METRIC>
    __device__ __forceinline__ double2 kdot(double a, double2 b, int mu) const {
        const double s = msign<METRIC>(mu) * a;
        return LaneOpsC<L>::sum(make_double2(s * b.x, s * b.y), mask);
    }
    template <int METRIC>
    __device__ __forceinline__ double2 kkdot(double a, double b, int mu) const {
        double2 t = make_double2(msign<METRIC>(mu) * a * b, 0.0);
        return LaneOpsC<L>::sum(t, mask);
    }
};

// Words per lane of the lane table for N = n - 1 legs.
struct LaneGeometry {
    int N;
    __host__ __device__ int nj() const { return Geometry{N}.nj(); }
    __host__ __device__ int ns() const { return Geometry{N}.ns(); }
    __host__ __device__ int off_k() const { return nj(); }
    __host__ __device__ int off_sa() const { return off_k() + N + 1; }
    __host__ __device__ int off_inv() const { return off_sa() + ns(); }
    __host__ __device__ int words() const { return off_inv() + ns(); }
};

// G = 1: one point per group of L lanes, each lane's words its own.  G > 1
// (L * G = 32): one point per warp ("team"): the G groups of the warp evaluate
// the ranges of each length in parallel (group gi takes the ranges starting
// at i = gi, gi + G, ...), with one table per team shared by its groups --
// component mu of every vector at the word of lane mu of the team -- and a
// warp barrier between lengths; group 0 loads the inputs and forms the prefix
// sums and the inverses alone (a serial chain either way).
template <class F, int L, int METRIC, int BLOCK, int G = 1>
__device__ __forceinline__ void lanes_point(const F& f, const CompactArgs& a, unsigned char* smem, int64_t u) {
    static_assert(G == 1 || L * G == 32, "a team is one warp");
    using T = typename F::T;
    using C = typename F::C;
    using Acc = typename F::A;
    using io_t = typename F::io_t;
    using TK = typename F::TK;
    using kio_t = typename F::kio_t;
    const int t = threadIdx.x;
    const int mu = t & (L - 1);
    const unsigned mask = ((1u << L) - 1u) << ((t & 31) & ~(L - 1));
    const LaneOps<F, L> lo{f, mask};
    const int NLEG = a.n;
    const LaneGeometry lg{NLEG - 1};
    const Geometry g{NLEG - 1};
    const int N = lg.N;
    // word w of this lane's table at [w][column]: the column is the thread
    // (G = 1) or lane mu of the team (G > 1), BLOCK / G columns per word
    constexpr int STRIDE = BLOCK / G;
    const int gi = G > 1 ? (t / L) % G : 0;
    const int col = G > 1 ? (t / 32) * L + mu : t;
    T* W = reinterpret_cast<T*>(smem) + col;
    TK* KW = reinterpret_cast<TK*>(reinterpret_cast<T*>(smem) + lg.off_k() * STRIDE) + col;
    const int NJ = lg.nj(), NSW = lg.ns();
    // word addressing of the four regions (checked in BG_CHECKED builds)
    auto J = [&](int slot) -> T& { return W[checked_slot(a.violation, slot, NJ, 21) * STRIDE]; };
    auto Kv = [&](int i) -> TK& { return KW[checked_slot(a.violation, i, N + 1, 22) * STRIDE]; };
    auto SA = [&](int s) -> T& { return W[(lg.off_sa() + checked_slot(a.violation, s, NSW, 23)) * STRIDE]; };
    auto IV = [&](int s) -> T& { return W[(lg.off_inv() + checked_slot(a.violation, s, NSW, 23)) * STRIDE]; };

    int64_t e = u;
    int h = 0;
    if (a.H > 1) {
        e = u / a.H;
        h = static_cast<int>(u - e * a.H);
    }
#ifdef BG_CHECKED
    const bool violated = !inputs_meet_preconditions<F, METRIC>(f, a.k, a.eps, e, NLEG, a.d_in, a.ds_in, a.S);
#else
    constexpr bool violated = false;
#endif
    // a1: this lane's components of the prefix sums and of the states (in a
    // team, group 0 alone: the other groups read them after the barrier)
    const bool stage = G == 1 || gi == 0;
    if (stage) {
        const kio_t* kp = static_cast<const kio_t*>(a.k) + e * NLEG * a.d_in;
        TK K = f.kzero();
        Kv(0) = K;
#pragma unroll 1
        for (int l = 0; l < N; ++l) {
            if (mu < a.d_in) K = f.kadd(K, f.kfrom_io(ld_once(kp + l * a.d_in + mu)));
            Kv(l + 1) = K;
        }
    }
    T eL = f.zero();
#pragma unroll 1
    for (int l = 0; l < (stage ? NLEG : 0); ++l) {
        const int s = (a.assign != nullptr) ? a.assign[h * NLEG + l] : 0;
        const io_t* ep = static_cast<const io_t*>(a.eps) + ((e * NLEG + l) * a.S + s) * a.ds_in;
        T v = f.zero();
        if constexpr (F::kIsFp) {
            if (mu < a.ds_in) v = ld_once(ep + mu);        // canonical residues, level 0 (as bg_compact)
        } else {
            if (mu < a.ds_in) v = f.from_io(ld_once(ep + mu));
        }
        if (l < N) J(l) = v;
        else eL = v;
    }
    // a2: P^2 of every internal range; a3: inverses (every lane the same scalars)
    auto kdot = [&](TK k, T v) -> C {
        if constexpr (F::kField == 2) return lo.template kdot<METRIC>(k, v, mu);
        else return lo.template dot<METRIC>(k, v, mu);
    };
    auto kkdot = [&](TK x, TK y) -> C {
        if constexpr (F::kField == 2) return lo.template kkdot<METRIC>(x, y, mu);
        else return lo.template dot<METRIC>(x, y, mu);
    };
#pragma unroll 1
    for (int m = 2; m < (stage ? N : 0); ++m) {
#pragma unroll 1
        for (int i = 0; i + m - 1 < N; ++i) {
            const TK P = f.ksub(Kv(i + m), Kv(i));
            SA(g.sbase(m) + i) = f.inv_input(kkdot(P, P));
        }
    }
    bool singular = false;
    const int NS = g.ns();
    if (!stage) {
    } else if constexpr (F::kIsFp) {
        T c = SA(0);
        IV(0) = c;
#pragma unroll 1
        for (int s = 1; s < NS; ++s) {
            c = f.inv_mul(c, SA(s));
            IV(s) = c;
        }
        singular = f.is_zero(c);
        T r = f.inv_scalar(c);
#pragma unroll 1
        for (int s = NS - 1; s > 0; --s) {
            const T x = SA(s);
            IV(s) = f.inv_store(f.inv_mul(IV(s - 1), r));
            r = f.inv_mul(r, x);
        }
        IV(0) = f.inv_store(r);
    } else {
#pragma unroll 1
        for (int s = 0; s < NS; ++s) {
            const T x = SA(s);
            singular |= f.is_zero(x);
            IV(s) = f.inv_scalar(x);
        }
    }
    if constexpr (G > 1) __syncwarp();      // the team's staged words are visible

    // a4: every range [i, i+m-1]; one point per group: by right end, as in
    // bg_compact.cuh; a team: by length, the ranges of one length spread over
    // the groups and a barrier before the next length reads them
    io_t result = f.zero_io();
    auto range = [&](const int m, const int i) {
        const TK Ki = Kv(i), Kj = Kv(i + m);
        const TK KiKj = f.kadd(Ki, Kj), P = f.ksub(Kj, Ki);
        Acc acc[1];
        f.template acc_zero<1>(acc);
        C sa = f.czero();
        int ps = i, ss = g.jbase(m - 1) + i + 1, es = i - N;
#pragma unroll 1
        for (int b = 0; b < m - 1; ++b) {
            const int lenA = b + 1, lenB = m - 1 - b;
            const T pb = J(ps), sf = J(ss);
            const TK Kt = Kv(i + b + 1);
            const C adj = lo.template dot<METRIC>(pb, sf, mu);
            const C pa_jb = kdot(P, sf);
            const C pb_ja = kdot(P, pb);
            sa = f.cadd(sa, adj);
            C csuf = f.cdbl(pb_ja);
            if (lenA >= 2) csuf = f.csub(csuf, f.t_to_c(SA(ps - N)));
            C cpre = f.cneg(f.cdbl(pa_jb));
            if (lenB >= 2) cpre = f.csub(cpre, f.t_to_c(SA(ss - N)));
            f.template acc2<1>(acc, csuf, &sf, cpre, &pb);
            f.template kacc1<1>(acc, f.cdbl(adj), &Kt);
            // gaps in pairs: two independent shuffle contractions in flight
            int pq = i, dp = N, iq = es, di = N - b + 1;
            int q = 0;
#pragma unroll 1
            for (; q + 1 < b; q += 2) {
                const T pa0 = J(pq), in0 = J(iq);
                pq += dp; iq -= di;
                const T pa1 = J(pq), in1 = J(iq);
                pq += dp - 1; iq -= di + 1;
                dp -= 2; di += 2;
                const C g0 = f.cdbl(lo.template dot<METRIC>(pa0, sf, mu));
                const C g1 = f.cdbl(lo.template dot<METRIC>(pa1, sf, mu));
                f.template acc2<1>(acc, g0, &in0, g1, &in1);
            }
            if (q < b) {
                const T pa0 = J(pq), in0 = J(iq);
                const C g0 = f.cdbl(lo.template dot<METRIC>(pa0, sf, mu));
                f.template acc1<1>(acc, g0, &in0);
            }
            ps += N - b;
            ss -= N - lenB + 1;
            es += N - b + 1;
        }
        f.template kacc1<1>(acc, f.cneg(sa), &KiKj);
        if (m < N) {
            const int sidx = g.sbase(m) + i;
            T Jn;
            f.template finish<1>(acc, IV(sidx), &Jn);
            J(g.jbase(m) + i) = Jn;
            SA(sidx) = f.c_to_t(sa);
        } else {
            if constexpr (F::kIsFp) {
                const T r = f.mmul(f.reduce96(acc[0]), f.rn3);
                const C amp = lo.template dot<METRIC>(eL, r, mu);
                result = amp == f.p ? 0u : amp;
            } else {
                result = lo.template dot<METRIC>(eL, acc[0], mu);
            }
        }
    };
    if constexpr (G == 1) {
#pragma unroll 1
        for (int jj = 1; jj < N; ++jj) {
#pragma unroll 1
            for (int i = jj - 1; i >= 0; --i) range(jj - i + 1, i);
        }
    } else {
#pragma unroll 1
        for (int m = 2; m <= N; ++m) {
#pragma unroll 1
            for (int i = gi; i + m - 1 < N; i += G) range(m, i);
            __syncwarp();
        }
    }
    if (mu == 0 && gi == 0) {
        st_once(static_cast<io_t*>(a.out) + u, (singular || violated) ? f.zero_io() : result);
        if (a.status != nullptr && h == 0) a.status[e] = violated ? 2 : singular ? 1 : 0;
    }
}

// One point per group of L lanes (L >= D_s: lanes beyond D_s hold zeros), or
// per team of G such groups (one warp), BLOCK / (L G) points per block,
// grid-stride over the work items; the tables of the block in dynamic shared
// memory (LaneGeometry::words() x BLOCK / G elements).  A team's lanes run
// the point loop together, so its barriers see the whole warp.
template <class F, int L, int METRIC, int BLOCK, int G>
__global__ void __launch_bounds__(BLOCK) bg_lanes_kernel(const F f, const CompactArgs a) {
    constexpr int PPB = BLOCK / (L * G);
    extern __shared__ __align__(16) unsigned char bg_lane_smem[];
    const int64_t total = a.E * a.H;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * PPB;
    for (int64_t u = static_cast<int64_t>(blockIdx.x) * PPB + threadIdx.x / (L * G); u < total; u += stride)
        lanes_point<F, L, METRIC, BLOCK, G>(f, a, bg_lane_smem, u);
}

// Registry row of a lanes kernel.
struct LanesEntry {
    int field;          // bg_field
    int L;              // lanes per group (>= D_s)
    int G;              // groups per point: 1, or 32 / L (a team of one warp)
    int metric;
    int block;          // threads per block
    int elem_bytes;     // sizeof(T)
    const void* func;
    void (*launch)(const void* field_params, const void* args, dim3 grid, size_t smem, cudaStream_t stream);
};

template <class F, int L, int M, int B, int G>
void launch_lanes(const void* fp, const void* args, dim3 grid, size_t smem, cudaStream_t s) {
    bg_lanes_kernel<F, L, M, B, G><<<grid, B, smem, s>>>(*static_cast<const F*>(fp),
                                                         *static_cast<const CompactArgs*>(args));
}

// F_p: 128 threads (16 points) per block; complex: 64 threads (8 points),
// their lane tables being four times larger.
constexpr int kBlockLanesFp = 128;
constexpr int kBlockLanesC64 = 64;

template <class F>
void register_lanes(std::vector<LanesEntry>& v) {
    constexpr int B = F::kIsFp ? kBlockLanesFp : kBlockLanesC64;
    auto add = [&](auto l, auto m, auto g) {
        constexpr int L = decltype(l)::value, M = decltype(m)::value, G = decltype(g)::value;
        v.push_back(LanesEntry{F::kField, L, G, M, B, static_cast<int>(sizeof(typename F::T)),
                               reinterpret_cast<const void*>(&bg_lanes_kernel<F, L, M, B, G>),
                               &launch_lanes<F, L, M, B, G>});
    };
    using one = std::integral_constant<int, 1>;
    add(std::integral_constant<int, 4>{}, std::integral_constant<int, 0>{}, one{});
    add(std::integral_constant<int, 4>{}, std::integral_constant<int, 1>{}, one{});
    add(std::integral_constant<int, 8>{}, std::integral_constant<int, 0>{}, one{});
    add(std::integral_constant<int, 8>{}, std::integral_constant<int, 1>{}, one{});
    add(std::integral_constant<int, 4>{}, std::integral_constant<int, 0>{}, std::integral_constant<int, 8>{});
    add(std::integral_constant<int, 4>{}, std::integral_constant<int, 1>{}, std::integral_constant<int, 8>{});
    add(std::integral_constant<int, 8>{}, std::integral_constant<int, 0>{}, std::integral_constant<int, 4>{});
    add(std::integral_constant<int, 8>{}, std::integral_constant<int, 1>{}, std::integral_constant<int, 4>{});
}

}  // namespace bgk

#define BG_DEFINE_LANES(OPS, TAG)                                             \
    void bg_register_lanes_##TAG(std::vector<bgk::LanesEntry>& v) { bgk::register_lanes<bgk::OPS>(v); }
