// bg_states.cuh -- every state assignment of a point in one recursion, with
// sub-currents shared between the assignments that agree on their legs.
//
// With S states per leg and all H = S^n assignments requested (the helicity
// sums of Sec. 2.3 and the state sums over cut trees of Sec. 2.1), the current
// of a range [i, j] depends only on the states of legs i..j: it has S^m
// versions for length m = j - i + 1, however many assignments share it.  The
// recursion of Sec. 2.2 is run once per (range, version) instead of once per
// (assignment, range): at n = 8, S = 2 that is 8.2k instead of 47k range
// evaluations per point, and the propagators 1/P^2, which depend on no state,
// are inverted once per point.
//
// Work decomposition: one warp per point.  For each length m the warp's lanes
// share the (range, version) items of that length; __syncwarp separates the
// lengths.  The warp's table (all versions of the currents of lengths
// 1..N-1, SA per version, prefix sums K, 1/P^2 per internal range, the last
// leg's states) lives in shared memory, or in a global scratch region when
// it does not fit.  Each version's vector is contiguous, so lanes reading
// consecutive versions of a sub-current read consecutive vectors.
//
// Version numbering: version sigma of a range of length m starting at leg i is
// sum_l s_{i+l} S^l (little endian in the legs); the output index of an
// assignment is h = sum_l s_l S^l over all n legs.  A split of [i, j] into
// A = [i, i+b] and B = [i+b+1, j] takes version sigma mod S^(b+1) of A and
// sigma / S^(b+1) of B.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "bg_compact.cuh"

namespace bgk {

constexpr int kStatesMaxLen = 12;           // pw[], cur[] ... indexed by length 0..11
constexpr int kStatesWarps = 4;             // warps (points in flight) per block

// x / d for x < 2^24 by a multiply and a shift (division by an invariant
// integer, Granlund and Montgomery 1994): magic = ceil(2^k / d) with
// k = 24 + ceil(log2 d), so that the error term stays below 1/d.
struct DivU {
    uint32_t magic;
    int shift;
    __host__ __device__ uint32_t div(uint32_t x) const {
        return static_cast<uint32_t>((static_cast<uint64_t>(x) * magic) >> shift);
    }
};

inline DivU make_divu(uint32_t d) {
    int lg = 0;
    while ((1ull << lg) < d) ++lg;
    const int k = 24 + lg;
    const uint64_t m = ((1ull << k) + d - 1) / d;
    return DivU{static_cast<uint32_t>(m), k};
}

// Table geometry of one point, in table elements (T); host-computed.
struct StatesGeometry {
    int N, S;                        // recursion legs (n - 1), states per leg
    int pw[kStatesMaxLen];           // S^L, L = 0..N
    int cur[kStatesMaxLen];          // first element of the currents of length L (L = 1..N-1)
    int sa[kStatesMaxLen];           // first SA entry of length L (L = 2..N-1)
    int inv[kStatesMaxLen];          // first 1/P^2 entry of length L (L = 2..N-1), from off_inv
    int ns;                          // internal ranges
    int off_inv, off_el, off_k;      // 1/P^2, last leg's states [S][D_s], prefix sums [N+1][D]
    int words;                       // elements per point
    DivU div_s;                      // x / S
    DivU div_pw[kStatesMaxLen];      // x / S^L
};

inline int states_up4(int x) { return (x + 3) & ~3; }

// elem_t = sizeof(T), elem_k = sizeof(momentum element)
inline StatesGeometry make_states_geometry(int n, int S, int D, int DS, int elem_t, int elem_k) {
    StatesGeometry g{};
    g.N = n - 1;
    g.S = S;
    const int N = g.N;
    g.pw[0] = 1;
    for (int L = 1; L <= N; ++L) g.pw[L] = g.pw[L - 1] * S;
    int off = 0;
    for (int L = 1; L < N; ++L) {
        g.cur[L] = off;
        off += (N - L + 1) * g.pw[L] * DS;
    }
    off = states_up4(off);
    for (int L = 2; L < N; ++L) {
        g.sa[L] = off;
        off += (N - L + 1) * g.pw[L];
    }
    g.off_inv = states_up4(off);
    int idx = 0;
    for (int L = 2; L < N; ++L) {
        g.inv[L] = idx;
        idx += N - L + 1;
    }
    g.ns = idx;
    g.off_el = states_up4(g.off_inv + idx);
    g.off_k = states_up4(g.off_el + S * DS);
    const int k_elems = ((N + 1) * D * elem_k + elem_t - 1) / elem_t;
    g.words = states_up4(g.off_k + k_elems);
    g.div_s = make_divu(S);
    for (int L = 0; L <= N; ++L) g.div_pw[L] = make_divu(g.pw[L]);
    return g;
}

struct StatesArgs {
    int64_t E;                  // points
    int n, d_in, ds_in;
    const void* k;              // [E][n][d_in]
    const void* eps;            // [E][n][S][ds_in]
    void* out;                  // [E][S^n]
    uint8_t* status;            // [E] or null
    void* ws;                   // global tables (global placement) or null
};

// All S^n assignments of point e by the warp whose table is `tab`.
template <class F, int D, int DS, int METRIC>
__device__ __forceinline__ void states_point(const F& f, const StatesArgs& a, const StatesGeometry& g,
                                             typename F::T* tab, int64_t e, int lane) {
    using T = typename F::T;
    using C = typename F::C;
    using Acc = typename F::A;
    using io_t = typename F::io_t;
    using TK = typename F::TK;
    using kio_t = typename F::kio_t;
    using IO = TableIO<T, F::kIsFp, 1>;         // contiguous vectors
    using KIO = TableIO<TK, F::kIsFp, 1>;
    const int N = g.N, S = g.S, n = N + 1;
    TK* Kr = reinterpret_cast<TK*>(tab + g.off_k);
    const T* Y = tab + g.off_inv;
    const T* EL = tab + g.off_el;
    auto cur = [&](int len, int start, uint32_t ver) {
        return tab + g.cur[len] + (start * g.pw[len] + static_cast<int>(ver)) * DS;
    };
    auto sav = [&](int len, int start, uint32_t ver) {
        return tab[g.sa[len] + start * g.pw[len] + static_cast<int>(ver)];
    };

    // s1: prefix sums K_0 = 0, K_{l+1} = K_l + k_l, one lane per component
    if (lane < D) {
        const kio_t* kp = static_cast<const kio_t*>(a.k) + e * n * a.d_in;
        TK acc = f.kzero();
        Kr[lane] = acc;
        for (int l = 0; l < N; ++l) {
            if (lane < a.d_in) acc = f.kadd(acc, f.kfrom_io(kp[l * a.d_in + lane]));
            Kr[(l + 1) * D + lane] = acc;
        }
    }
    // s2: polarisations -> currents of length 1 (version = state) and the
    // last leg's states
    {
        const io_t* ep = static_cast<const io_t*>(a.eps) + e * n * S * a.ds_in;
        const int total = n * S * DS;
        for (int x = lane; x < total; x += 32) {
            const int mu = x % DS;
            const int ls = x / DS;                 // l * S + t
            const T v = mu < a.ds_in ? f.from_io(ep[ls * a.ds_in + mu]) : f.zero();
            if (ls < N * S) tab[g.cur[1] + x] = v;
            else tab[g.off_el + (x - N * S * DS)] = v;
        }
    }
    __threadfence_block();
    __syncwarp();
    // s3: 1/P^2 of every internal range, one lane per range
    bool sing = false;
    for (int r = lane; r < g.ns; r += 32) {
        int L = 2, i = r;
        while (i >= N - L + 1) {
            i -= N - L + 1;
            ++L;
        }
        TK Ka[D], Kb[D], P[D];
        KIO::template load<D>(Kr + i * D, Ka);
        KIO::template load<D>(Kr + (i + L) * D, Kb);
#pragma unroll
        for (int mu = 0; mu < D; ++mu) P[mu] = f.ksub(Kb[mu], Ka[mu]);
        const T x = f.inv_input(f.template kkdot<D, METRIC>(P, P));
        sing |= f.is_zero(x);
        tab[g.off_inv + r] = f.inv_store(f.inv_scalar(x));
    }
    const bool singular = __any_sync(0xffffffffu, sing);
    __threadfence_block();
    __syncwarp();

    // s4: the recursion by length; items (range start i, version sigma)
    io_t* out = static_cast<io_t*>(a.out);
    const int64_t H = static_cast<int64_t>(g.pw[N]) * S;
    for (int m = 2; m <= N; ++m) {
        const int nver = g.pw[m];
        const int count = (N - m + 1) * nver;
        for (int it = lane; it < count; it += 32) {
            const int i = static_cast<int>(g.div_pw[m].div(static_cast<uint32_t>(it)));
            const uint32_t sig = static_cast<uint32_t>(it - i * nver);
            TK Ki[D], Kj[D];
            KIO::template load<D>(Kr + i * D, Ki);
            KIO::template load<D>(Kr + (i + m) * D, Kj);
            Acc acc[DS];
            f.template acc_zero<DS>(acc);
            C sa = f.czero();
            C mom_c = f.czero();
            TK mom_v[D];
            bool mom_pending = false;
            uint32_t qB = sig;                  // sigma / S^(b+1): version of the suffix
            for (int b = 0; b < m - 1; ++b) {
                const int lenA = b + 1, lenB = m - 1 - b;
                qB = g.div_s.div(qB);
                const uint32_t sA = sig - qB * static_cast<uint32_t>(g.pw[lenA]);
                T pb[DS], sf[DS];
                TK Kt[D], PA[D], PB[D];
                IO::template load<DS>(cur(lenA, i, sA), pb);
                IO::template load<DS>(cur(lenB, i + b + 1, qB), sf);
                KIO::template load<D>(Kr + (i + b + 1) * D, Kt);
#pragma unroll
                for (int mu = 0; mu < D; ++mu) {
                    PA[mu] = f.ksub(Kt[mu], Ki[mu]);
                    PB[mu] = f.ksub(Kj[mu], Kt[mu]);
                }
                const C adj = f.template dot<DS, METRIC>(pb, sf);
                const C pa_jb = f.template kdot<D, METRIC>(PA, sf);
                const C pb_ja = f.template kdot<D, METRIC>(PB, pb);
                sa = f.cadd(sa, adj);
                C csuf = f.cdbl(pb_ja);
                if (lenA >= 2) csuf = f.csub(csuf, f.t_to_c(sav(lenA, i, sA)));
                C cpre = f.cneg(f.cdbl(pa_jb));
                if (lenB >= 2) cpre = f.csub(cpre, f.t_to_c(sav(lenB, i + b + 1, qB)));
                f.template acc2<DS>(acc, csuf, sf, cpre, pb);
                if (mom_pending) {
                    f.template kacc2<D>(acc, mom_c, mom_v, f.cdbl(adj), Kt);
                    mom_pending = false;
                } else {
                    mom_c = f.cdbl(adj);
#pragma unroll
                    for (int mu = 0; mu < D; ++mu) mom_v[mu] = Kt[mu];
                    mom_pending = true;
                }
                // four-gluon vertex: prefix [i, i+q], inner [i+q+1, i+b], suffix sf;
                // Q = sigma / S^(q+1), prefix version sigma - Q S^(q+1), inner
                // version Q - qB S^(b-q)
                uint32_t Q = sig;
                int q = 0;
                for (; q + 1 < b; q += 2) {
                    const uint32_t Q0 = g.div_s.div(Q);
                    const uint32_t Q1 = g.div_s.div(Q0);
                    Q = Q1;
                    T pa0[DS], pa1[DS], in0[DS], in1[DS];
                    IO::template load<DS>(cur(q + 1, i, sig - Q0 * static_cast<uint32_t>(g.pw[q + 1])), pa0);
                    IO::template load<DS>(cur(b - q, i + q + 1, Q0 - qB * static_cast<uint32_t>(g.pw[b - q])), in0);
                    IO::template load<DS>(cur(q + 2, i, sig - Q1 * static_cast<uint32_t>(g.pw[q + 2])), pa1);
                    IO::template load<DS>(cur(b - q - 1, i + q + 2, Q1 - qB * static_cast<uint32_t>(g.pw[b - q - 1])), in1);
                    const C g0 = f.cdbl(f.template dot<DS, METRIC>(pa0, sf));
                    const C g1 = f.cdbl(f.template dot<DS, METRIC>(pa1, sf));
                    f.template acc2<DS>(acc, g0, in0, g1, in1);
                }
                if (q < b) {
                    const uint32_t Q0 = g.div_s.div(Q);
                    T pa0[DS], in0[DS];
                    IO::template load<DS>(cur(q + 1, i, sig - Q0 * static_cast<uint32_t>(g.pw[q + 1])), pa0);
                    IO::template load<DS>(cur(b - q, i + q + 1, Q0 - qB * static_cast<uint32_t>(g.pw[b - q])), in0);
                    const C g0 = f.cdbl(f.template dot<DS, METRIC>(pa0, sf));
                    f.template acc1<DS>(acc, g0, in0);
                }
            }
            {
                TK KiKj[D];
#pragma unroll
                for (int mu = 0; mu < D; ++mu) KiKj[mu] = f.kadd(Ki[mu], Kj[mu]);
                if (mom_pending) f.template kacc2<D>(acc, mom_c, mom_v, f.cneg(sa), KiKj);
                else f.template kacc1<D>(acc, f.cneg(sa), KiKj);
            }
            if (m < N) {
                T J[DS];
                f.template finish<DS>(acc, Y[g.inv[m] + i], J);
                IO::template store<DS>(tab + g.cur[m] + it * DS, J);
                tab[g.sa[m] + it] = f.c_to_t(sa);
            } else {
                // the top range: contract with each state of the last leg
                io_t* o = out + e * H + sig;
                for (int t = 0; t < S; ++t) {
                    T eL[DS];
                    IO::template load<DS>(EL + t * DS, eL);
                    o[static_cast<int64_t>(t) * nver] = singular ? f.zero_io()
                                                                 : f.template amplitude<DS, METRIC>(acc, eL);
                }
            }
        }
        __threadfence_block();
        __syncwarp();
    }
    if (lane == 0 && a.status != nullptr) a.status[e] = singular ? 1 : 0;
}

template <class F, int D, int DS, int METRIC>
__global__ void __launch_bounds__(32 * kStatesWarps)
bg_states_kernel(const F f, const StatesArgs a, const StatesGeometry g) {
    using T = typename F::T;
    extern __shared__ __align__(16) unsigned char bg_states_smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t slot = static_cast<int64_t>(blockIdx.x) * kStatesWarps + warp;
    T* tab = a.ws != nullptr ? reinterpret_cast<T*>(a.ws) + slot * g.words
                             : reinterpret_cast<T*>(bg_states_smem) + warp * g.words;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * kStatesWarps;
    for (int64_t e = slot; e < a.E; e += stride) states_point<F, D, DS, METRIC>(f, a, g, tab, e, lane);
}

}  // namespace bgk

namespace bgk {

// Registry row of a states kernel (one per field, D, D_s, metric).
struct StatesEntry {
    int field, D, DS, metric;
    int elem_bytes, elem_k_bytes;     // sizeof(T), sizeof(momentum element)
    const void* func;
    void (*launch)(const void* field_params, const StatesArgs& a, const StatesGeometry& g, dim3 grid,
                   size_t smem, cudaStream_t stream);
};

template <class F, int D, int DS, int M>
void launch_states(const void* fp, const StatesArgs& a, const StatesGeometry& g, dim3 grid, size_t smem,
                   cudaStream_t s) {
    bg_states_kernel<F, D, DS, M><<<grid, 32 * kStatesWarps, smem, s>>>(*static_cast<const F*>(fp), a, g);
}

template <class F, int D, int DS, int M>
StatesEntry make_states() {
    StatesEntry e;
    e.field = F::kField;
    e.D = D;
    e.DS = DS;
    e.metric = M;
    e.elem_bytes = sizeof(typename F::T);
    e.elem_k_bytes = sizeof(typename F::TK);
    e.func = reinterpret_cast<const void*>(&bg_states_kernel<F, D, DS, M>);
    e.launch = &launch_states<F, D, DS, M>;
    return e;
}

template <class F, int D, int DS>
void register_states(std::vector<StatesEntry>& v) {
    v.push_back(make_states<F, D, DS, 0>());
    v.push_back(make_states<F, D, DS, 1>());
}

}  // namespace bgk

// Instances for one field and momentum dimension D: every D_s >= D.
#define BG_DEFINE_STATES(D, OPS, TAG)                                            \
    void bg_register_states_##TAG##_##D(std::vector<bgk::StatesEntry>& v) {      \
        if constexpr (D == 4) {                                                  \
            bgk::register_states<bgk::OPS, 4, 4>(v);                             \
            bgk::register_states<bgk::OPS, 4, 6>(v);                             \
            bgk::register_states<bgk::OPS, 4, 8>(v);                             \
        } else if constexpr (D == 6) {                                           \
            bgk::register_states<bgk::OPS, 6, 6>(v);                             \
            bgk::register_states<bgk::OPS, 6, 8>(v);                             \
        } else {                                                                 \
            bgk::register_states<bgk::OPS, 8, 8>(v);                             \
        }                                                                        \
    }
