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

constexpr int kStatesMaxLegs = 12;          // legs (n <= 12)
constexpr int kStatesWarps = 4;             // warps per block

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

// Table geometry of one point, in table elements (T); host-computed.  Leg l
// has radix[l] states; range (i, L) = legs i..i+L-1 has W[i][L] versions.
struct StatesGeometry {
    int N, S;                                    // recursion legs (n - 1); eps slots per leg
    int P;                                       // points per warp
    int H;                                       // outputs per point = W[0][N] * radix[N]
    int radix[kStatesMaxLegs];
    DivU div_leg[kStatesMaxLegs];                // x / radix[l]
    int W[kStatesMaxLegs][kStatesMaxLegs + 1];   // W[i][L] = radix[i] ... radix[i+L-1]
    int cur[kStatesMaxLegs][kStatesMaxLegs];     // [L][i] first element of the currents of (i, L)
    int sa[kStatesMaxLegs][kStatesMaxLegs];      // [L][i] first SA entry of (i, L), L >= 2
    int inv[kStatesMaxLegs];                     // [L] first 1/P^2 entry of length L (from off_inv)
    int count[kStatesMaxLegs + 1];               // [m] (range, version) items of length m
    int first[kStatesMaxLegs + 1][kStatesMaxLegs + 1];   // [m][i] first item of range i; [m][N-m+1] = count
    DivU div_count[kStatesMaxLegs + 1];          // x / count[m]
    int ns;                                      // internal ranges
    int off_inv, off_el, off_k, off_flag;        // 1/P^2, last leg's states, prefix sums, singular flag
    int words;                                   // elements per point
};

inline int states_up4(int x) { return (x + 3) & ~3; }

// radix[0..n): states per leg (1 <= radix[l] <= S); elem_t = sizeof(T),
// elem_k = sizeof(momentum element)
inline StatesGeometry make_states_geometry(int n, int S, const int* radix, int D, int DS, int elem_t,
                                           int elem_k) {
    StatesGeometry g{};
    g.N = n - 1;
    g.S = S;
    const int N = g.N;
    for (int l = 0; l < n; ++l) {
        g.radix[l] = radix[l];
        g.div_leg[l] = make_divu(radix[l]);
    }
    for (int i = 0; i < n; ++i) {
        g.W[i][0] = 1;
        for (int L = 1; i + L <= n; ++L) g.W[i][L] = g.W[i][L - 1] * radix[i + L - 1];
    }
    g.H = g.W[0][N] * radix[N];
    int off = 0;
    for (int L = 1; L < N; ++L)
        for (int i = 0; i + L <= N; ++i) {
            g.cur[L][i] = off;
            off += g.W[i][L] * DS;
        }
    off = states_up4(off);
    for (int L = 2; L < N; ++L)
        for (int i = 0; i + L <= N; ++i) {
            g.sa[L][i] = off;
            off += g.W[i][L];
        }
    g.off_inv = states_up4(off);
    int idx = 0;
    for (int L = 2; L < N; ++L) {
        g.inv[L] = idx;
        idx += N - L + 1;
    }
    g.ns = idx;
    g.off_el = states_up4(g.off_inv + idx);
    g.off_k = states_up4(g.off_el + radix[N] * DS);
    const int k_elems = ((N + 1) * D * elem_k + elem_t - 1) / elem_t;
    g.off_flag = states_up4(g.off_k + k_elems);
    g.words = g.off_flag + 4;
    int maxc = 1;
    for (int m = 2; m <= N; ++m) {
        int c = 0;
        for (int i = 0; i + m <= N; ++i) {
            g.first[m][i] = c;
            c += g.W[i][m];
        }
        g.first[m][N - m + 1] = c;
        g.count[m] = c;
        g.div_count[m] = make_divu(c);
        if (c > maxc) maxc = c;
    }
    // points per warp: enough (point, item) pairs of the top length to fill the lanes
    g.P = 32 / g.count[N];
    if (g.P < 1) g.P = 1;
    (void)maxc;
    return g;
}

struct StatesArgs {
    int64_t E;                  // points
    int n, d_in, ds_in;
    const void* k;              // [E][n][d_in]
    const void* eps;            // [E][n][S][ds_in]
    void* out;                  // [E][H]
    uint8_t* status;            // [E] or null
    void* ws;                   // global tables (global placement) or null
    unsigned long long* violation;   // checked builds: first out-of-range table index
};

// The assignments of the points e0 .. e0+np-1 (np <= P) by one warp; point p's
// table is tab + p * words.
template <class F, int D, int DS, int METRIC, bool UNIFORM>
__device__ __forceinline__ void states_group(const F& f, const StatesArgs& a, const StatesGeometry& g,
                                             typename F::T* tab, int64_t e0, int np, int lane) {
    using T = typename F::T;
    using C = typename F::C;
    using Acc = typename F::A;
    using io_t = typename F::io_t;
    using TK = typename F::TK;
    using kio_t = typename F::kio_t;
    using IO = TableIO<T, F::kIsFp, 1>;         // contiguous vectors
    using KIO = TableIO<TK, F::kIsFp, 1>;
    const int N = g.N, S = g.S, n = N + 1, W = g.words;
    // every leg with the same number of states: one divisor and W[i][L] = S^L
    // for every i (loop-invariant constants)
    auto divl = [&](int leg) -> const DivU& {
        if constexpr (UNIFORM) return g.div_leg[0];
        else return g.div_leg[leg];
    };
    auto wv = [&](int i, int L) -> uint32_t {
        if constexpr (UNIFORM) return static_cast<uint32_t>(g.W[0][L]);
        else return static_cast<uint32_t>(g.W[i][L]);
    };
    auto kr = [&](int p) { return reinterpret_cast<TK*>(tab + p * W + g.off_k); };
    auto flag = [&](int p) { return reinterpret_cast<int*>(tab + p * W + g.off_flag); };
    // offset of a `width`-element access in a point's table (checked in
    // BG_CHECKED builds), and of a prefix-sum component in the K region
    auto at = [&](int off, int width, int site) { return checked_slot(a.violation, off, W - width + 1, site); };
    auto kat = [&](int idx) { return checked_slot(a.violation, idx, (N + 1) * D, 14); };

    // s1: prefix sums K_0 = 0, K_{l+1} = K_l + k_l, one lane per (point, component)
    for (int x = lane; x < np * D; x += 32) {
        const int p = x / D, mu = x - p * D;
        const kio_t* kp = static_cast<const kio_t*>(a.k) + (e0 + p) * n * a.d_in;
        TK* Kr = kr(p);
        TK acc = f.kzero();
        Kr[kat(mu)] = acc;
        for (int l = 0; l < N; ++l) {
            if (mu < a.d_in) acc = f.kadd(acc, f.kfrom_io(kp[l * a.d_in + mu]));
            Kr[kat((l + 1) * D + mu)] = acc;
        }
    }
    // s2: polarisations -> currents of length 1 (version = state) and the last
    // leg's states; singular flags cleared
    {
        const int per = n * S * DS;
        for (int x = lane; x < np * per; x += 32) {
            const int p = x / per, y = x - p * per;
            const int mu = y % DS;
            const int ls = y / DS;                 // l * S + t
            const int l = ls / S, t = ls - l * S;
            if (t >= g.radix[l]) continue;
            const io_t* ep = static_cast<const io_t*>(a.eps) + (e0 + p) * n * S * a.ds_in;
            const T v = mu < a.ds_in ? f.from_io(ep[ls * a.ds_in + mu]) : f.zero();
            T* tp = tab + p * W;
            if (l < N) tp[at(g.cur[1][l] + t * DS + mu, 1, 11)] = v;
            else tp[at(g.off_el + t * DS + mu, 1, 12)] = v;
        }
        for (int p = lane; p < np; p += 32) {
            int fl = 0;
#ifdef BG_CHECKED
            // bit 1: the point's inputs break a precondition of the boundary
            if (!inputs_meet_preconditions<F, METRIC>(f, a.k, a.eps, e0 + p, n, a.d_in, a.ds_in, S, g.radix))
                fl = 2;
#endif
            *flag(p) = fl;
        }
    }
    __threadfence_block();
    __syncwarp();
    // s3: 1/P^2 of every internal range, one lane per (point, range)
    for (int x = lane; x < np * g.ns; x += 32) {
        const int p = x / g.ns, r = x - p * g.ns;
        int L = 2, i = r;
        while (i >= N - L + 1) {
            i -= N - L + 1;
            ++L;
        }
        const TK* Kr = kr(p);
        TK Ka[D], Kb[D], Pv[D];
        KIO::template load<D>(Kr + kat(i * D), Ka);
        KIO::template load<D>(Kr + kat((i + L) * D), Kb);
#pragma unroll
        for (int mu = 0; mu < D; ++mu) Pv[mu] = f.ksub(Kb[mu], Ka[mu]);
        const T xv = f.inv_input(f.template kkdot<D, METRIC>(Pv, Pv));
        if (f.is_zero(xv)) *flag(p) |= 1;    // bit 0: singular propagator
        tab[p * W + at(g.off_inv + r, 1, 13)] = f.inv_store(f.inv_scalar(xv));
    }
    __threadfence_block();
    __syncwarp();

    // s4: the recursion by length; items (point, range start i, version sigma)
    io_t* out = static_cast<io_t*>(a.out);
    for (int m = 2; m <= N; ++m) {
        const int count = g.count[m];
        for (int x = lane; x < np * count; x += 32) {
            const int p = static_cast<int>(g.div_count[m].div(static_cast<uint32_t>(x)));
            const int it = x - p * count;
            int i = 0;
            while (it >= g.first[m][i + 1]) ++i;
            const uint32_t sig = static_cast<uint32_t>(it - g.first[m][i]);
            T* tp = tab + p * W;
            const TK* Kr = kr(p);
            auto cur = [&](int len, int start, uint32_t ver) {
                return tp + at(g.cur[len][start] + static_cast<int>(ver) * DS, DS, 15);
            };
            auto sav = [&](int len, int start, uint32_t ver) {
                return tp[at(g.sa[len][start] + static_cast<int>(ver), 1, 16)];
            };
            // K_i + K_{j+1} and the range momentum P (current conservation:
            // P_B . J_A = P . J_A and P_A . J_B = P . J_B, as in bg_compact.cuh)
            TK KiKj[D], P[D];
            {
                TK Ki[D], Kj[D];
                KIO::template load<D>(Kr + kat(i * D), Ki);
                KIO::template load<D>(Kr + kat((i + m) * D), Kj);
#pragma unroll
                for (int mu = 0; mu < D; ++mu) {
                    KiKj[mu] = f.kadd(Ki[mu], Kj[mu]);
                    P[mu] = f.ksub(Kj[mu], Ki[mu]);
                }
            }
            Acc acc[DS];
            f.template acc_zero<DS>(acc);
            C sa = f.czero();
            C mom_c = f.czero();
            TK mom_v[D];
            bool mom_pending = false;
            uint32_t qB = sig;                  // sigma / W[i][b+1]: version of the suffix
            for (int b = 0; b < m - 1; ++b) {
                const int lenA = b + 1, lenB = m - 1 - b;
                qB = divl(i + b).div(qB);
                const uint32_t sA = sig - qB * wv(i, lenA);
                T pb[DS], sf[DS];
                TK Kt[D];
                IO::template load<DS>(cur(lenA, i, sA), pb);
                IO::template load<DS>(cur(lenB, i + b + 1, qB), sf);
                KIO::template load<D>(Kr + kat((i + b + 1) * D), Kt);
                const C adj = f.template dot<DS, METRIC>(pb, sf);
                const C pa_jb = f.template kdot<D, METRIC>(P, sf);
                const C pb_ja = f.template kdot<D, METRIC>(P, pb);
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
                // Q = sigma / W[i][q+1], prefix version sigma - Q W[i][q+1],
                // inner version Q - qB W[i+q+1][b-q]
                uint32_t Q = sig;
                int q = 0;
                for (; q + 1 < b; q += 2) {
                    const uint32_t Q0 = divl(i + q).div(Q);
                    const uint32_t Q1 = divl(i + q + 1).div(Q0);
                    Q = Q1;
                    T pa0[DS], pa1[DS], in0[DS], in1[DS];
                    IO::template load<DS>(cur(q + 1, i, sig - Q0 * wv(i, q + 1)), pa0);
                    IO::template load<DS>(cur(b - q, i + q + 1, Q0 - qB * wv(i + q + 1, b - q)), in0);
                    IO::template load<DS>(cur(q + 2, i, sig - Q1 * wv(i, q + 2)), pa1);
                    IO::template load<DS>(cur(b - q - 1, i + q + 2, Q1 - qB * wv(i + q + 2, b - q - 1)), in1);
                    const C g0 = f.cdbl(f.template dot<DS, METRIC>(pa0, sf));
                    const C g1 = f.cdbl(f.template dot<DS, METRIC>(pa1, sf));
                    f.template acc2<DS>(acc, g0, in0, g1, in1);
                }
                if (q < b) {
                    const uint32_t Q0 = divl(i + q).div(Q);
                    T pa0[DS], in0[DS];
                    IO::template load<DS>(cur(q + 1, i, sig - Q0 * wv(i, q + 1)), pa0);
                    IO::template load<DS>(cur(b - q, i + q + 1, Q0 - qB * wv(i + q + 1, b - q)), in0);
                    const C g0 = f.cdbl(f.template dot<DS, METRIC>(pa0, sf));
                    f.template acc1<DS>(acc, g0, in0);
                }
            }
            if (mom_pending) f.template kacc2<D>(acc, mom_c, mom_v, f.cneg(sa), KiKj);
            else f.template kacc1<D>(acc, f.cneg(sa), KiKj);
            if (m < N) {
                T J[DS];
                f.template finish<DS>(acc, tp[at(g.off_inv + g.inv[m] + i, 1, 17)], J);
                IO::template store<DS>(cur(m, i, sig), J);
                tp[at(g.sa[m][i] + static_cast<int>(sig), 1, 18)] = f.c_to_t(sa);
            } else {
                // the top range: contract with each state of the last leg
                const bool singular = *flag(p) != 0;
                io_t* o = out + (e0 + p) * g.H + sig;
                for (int t = 0; t < g.radix[N]; ++t) {
                    T eL[DS];
                    IO::template load<DS>(tp + at(g.off_el + t * DS, DS, 19), eL);
                    o[static_cast<int64_t>(t) * count] = singular ? f.zero_io()
                                                                  : f.template amplitude<DS, METRIC>(acc, eL);
                }
            }
        }
        __threadfence_block();
        __syncwarp();
    }
    if (a.status != nullptr)
        for (int p = lane; p < np; p += 32) a.status[e0 + p] = (*flag(p) & 2) ? 2 : (*flag(p) ? 1 : 0);
    __syncwarp();
}

template <class F, int D, int DS, int METRIC, bool UNIFORM>
__global__ void __launch_bounds__(32 * kStatesWarps)
bg_states_kernel(const F f, const StatesArgs a, const StatesGeometry g) {
    using T = typename F::T;
    extern __shared__ __align__(16) unsigned char bg_states_smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t slot = static_cast<int64_t>(blockIdx.x) * kStatesWarps + warp;
    T* tab = a.ws != nullptr ? reinterpret_cast<T*>(a.ws) + slot * g.P * g.words
                             : reinterpret_cast<T*>(bg_states_smem) + warp * g.P * g.words;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * kStatesWarps * g.P;
    for (int64_t e0 = slot * g.P; e0 < a.E; e0 += stride) {
        const int np = a.E - e0 < g.P ? static_cast<int>(a.E - e0) : g.P;
        states_group<F, D, DS, METRIC, UNIFORM>(f, a, g, tab, e0, np, lane);
    }
}

}  // namespace bgk

namespace bgk {

// Registry row of a states kernel (one per field, D, D_s, metric).
struct StatesEntry {
    int field, D, DS, metric;
    bool uniform;                     // every leg with the same number of states
    int elem_bytes, elem_k_bytes;     // sizeof(T), sizeof(momentum element)
    const void* func;
    void (*launch)(const void* field_params, const StatesArgs& a, const StatesGeometry& g, dim3 grid,
                   size_t smem, cudaStream_t stream);
};

template <class F, int D, int DS, int M, bool U>
void launch_states(const void* fp, const StatesArgs& a, const StatesGeometry& g, dim3 grid, size_t smem,
                   cudaStream_t s) {
    bg_states_kernel<F, D, DS, M, U><<<grid, 32 * kStatesWarps, smem, s>>>(*static_cast<const F*>(fp), a, g);
}

template <class F, int D, int DS, int M, bool U>
StatesEntry make_states() {
    StatesEntry e;
    e.field = F::kField;
    e.D = D;
    e.DS = DS;
    e.metric = M;
    e.uniform = U;
    e.elem_bytes = sizeof(typename F::T);
    e.elem_k_bytes = sizeof(typename F::TK);
    e.func = reinterpret_cast<const void*>(&bg_states_kernel<F, D, DS, M, U>);
    e.launch = &launch_states<F, D, DS, M, U>;
    return e;
}

template <class F, int D, int DS>
void register_states(std::vector<StatesEntry>& v) {
    v.push_back(make_states<F, D, DS, 0, true>());
    v.push_back(make_states<F, D, DS, 1, true>());
    v.push_back(make_states<F, D, DS, 0, false>());
    v.push_back(make_states<F, D, DS, 1, false>());
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
