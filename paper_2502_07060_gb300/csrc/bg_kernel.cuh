// bg_kernel.cuh -- fused Berends-Giele recursion, one phase-space point (and
// state assignment) per thread.
//
// Method (arXiv:2502.07060, Sec. 2.2): currents over consecutive leg ranges,
//   J(i,j) = (-i/P_ij^2) [ sum_s V3(P_A,P_B) J_A J_B + sum_{s<t} V4 J_A J_B J_C ],
// with the vertices of Sec. 2.2.  Contracted with the currents, and with the
// i of each vertex cancelled against the -i of the propagator,
//   R(i,j) = sum_s   (J_A.J_B)(P_A - P_B) + 2(P_B.J_A) J_B - 2(P_A.J_B) J_A
//          + sum_s<t 2(J_A.J_C) J_B - (J_B.J_C) J_A - (J_A.J_B) J_C,
//   J(i,j) = R(i,j) / P_ij^2 (internal ranges),   A = eps_n . R(1, n-1).
//
// GB300 design (not the paper's TensorFlow op-per-launch design, Sec. 3):
// * the whole recursion for a point runs in ONE thread, fully specialised at
//   compile time on (n, D, D_s, metric); the loop over ranges of equal length
//   runs at run time so the code size grows with n^3, not n^4;
// * the sum above is regrouped by the current it multiplies, which removes
//   repeated dot products without changing the value (exact over F_p):
//     - prefix  A=[i,s]:   coefficient -2 P_A.J_[s+1,j] - SA([s+1,j])
//     - suffix  C=[t+1,j]: coefficient +2 P_C.J_[i,t]   - SA([i,t])
//     - inner   B=[s+1,t]: coefficient  2 J_[i,s].J_[t+1,j]
//     - momentum part sum_s (J_A.J_B)(P_A - P_B)
//   where SA(X) = sum over the splits X = Y|Z of J_Y.J_Z is a by-product of
//   the range X itself and is stored with its current;
// * the per-point table (currents, prefix sums K_t of the momenta,
//   P_ij = K_{j+1} - K_i, SA and 1/P^2) lives in shared memory (thread-
//   interleaved: element w of thread t at [w * BLOCK + t], conflict free) or,
//   for large tables, in a global scratch buffer with the same layout that
//   stays resident in the 126 MB L2;
// * 1/P^2 for all internal ranges: Montgomery simultaneous inversion with a
//   single Fermat inverse per point (F_p), or per-range reciprocal (C64).
#pragma once
#include <cstdint>
#include <utility>

#include "bg_c64.cuh"
#include "bg_fp.cuh"

namespace bgk {

// Slot bookkeeping for a recursion over N = n - 1 legs.
template <int N>
struct Slots {
    __host__ __device__ static constexpr int count(int len) { return N - len + 1; }
    __host__ __device__ static constexpr int jbase(int len) {   // first current of length `len`
        int b = 0;
        for (int l = 1; l < len; ++l) b += count(l);
        return b;
    }
    __host__ __device__ static constexpr int sbase(int len) {   // first scalar slot of length `len` >= 2
        int b = 0;
        for (int l = 2; l < len; ++l) b += count(l);
        return b;
    }
    static constexpr int NJ = jbase(N);     // currents of length 1..N-1
    static constexpr int NS = sbase(N);     // internal ranges, length 2..N-1
};

template <int N, int D, int DS>
struct Frame {
    using S = Slots<N>;
    static constexpr int OFF_J = 0;
    static constexpr int OFF_K = S::NJ * DS;
    static constexpr int OFF_SA = OFF_K + (N + 1) * D;
    static constexpr int OFF_INV = OFF_SA + S::NS;
    static constexpr int WORDS = OFF_INV + S::NS;   // elements of T per point
};

struct LaunchArgs {
    int64_t E;                  // points
    int H;                      // state assignments per point
    int S;                      // states per leg
    int d_in, ds_in;            // dimensions of the inputs (<= D, D_s)
    const void* k;              // [E][n][d_in]
    const void* eps;            // [E][n][S][ds_in]
    void* out;                  // [E][H]
    uint8_t* status;            // [E] or null
    const uint8_t* assign;      // device [H][n] or null (H == 1)
    void* ws;                   // global table (GLOBAL_TABLE variants)
};

template <class F, int N, int D, int DS, int METRIC, int BLOCK>
struct Rec {
    using T = typename F::T;
    using Sl = Slots<N>;
    using Fr = Frame<N, D, DS>;

    // Cache the prefixes of a range in registers while they fit in a budget.
    template <int LEN>
    __host__ __device__ static constexpr bool cache_prefixes() {
        return (LEN - 1) * DS * int(sizeof(T) / 4) <= 96;
    }

    __device__ static __forceinline__ void load_vec(const T* p, T* v, int n) {
#pragma unroll
        for (int mu = 0; mu < DS; ++mu)
            if (mu < n) v[mu] = p[mu * BLOCK];
    }

    // One length LEN of the recursion: every range [i, i+LEN-1].
    template <int LEN>
    __device__ static __forceinline__ void range_len(const F& f, T* base, T* top) {
        constexpr bool CACHE = cache_prefixes<LEN>();
        constexpr int NPF = CACHE ? LEN - 1 : 1;
#pragma unroll 1
        for (int i = 0; i + LEN - 1 < N; ++i) {
            T* Jb = base + (Fr::OFF_J + i * DS) * BLOCK;   // current (len, i + c)
            T* Kb = base + (Fr::OFF_K + i * D) * BLOCK;    // K_{i + c}
            T* Sb = base + (Fr::OFF_SA + i) * BLOCK;       // SA (len, i + c)
            T* Ib = base + (Fr::OFF_INV + i) * BLOCK;      // 1/P^2 (len, i + c)
            auto jslot = [&](int len, int c) { return Jb + ((Sl::jbase(len) + c) * DS) * BLOCK; };

            T pfc[NPF][DS];
            if constexpr (CACHE) {
#pragma unroll
                for (int b = 0; b < LEN - 1; ++b) load_vec(jslot(b + 1, 0), pfc[b], DS);
            }
            T Ki[D], Kj1[D];
            load_vec(Kb, Ki, D);
            load_vec(Kb + (LEN * D) * BLOCK, Kj1, D);

            T acc[DS];
#pragma unroll
            for (int mu = 0; mu < DS; ++mu) acc[mu] = f.zero();
            T sa = f.zero();

#pragma unroll
            for (int b = 0; b < LEN - 1; ++b) {
                const int lenB = LEN - 1 - b;                    // suffix [i+b+1, j]
                T pb[DS];                                         // prefix [i, i+b]
                if constexpr (CACHE) {
#pragma unroll
                    for (int mu = 0; mu < DS; ++mu) pb[mu] = pfc[b][mu];
                } else {
                    load_vec(jslot(b + 1, 0), pb, DS);
                }
                T sf[DS];
                load_vec(jslot(lenB, b + 1), sf, DS);
                T Kt[D], PA[D], PB[D], dP[D];
                load_vec(Kb + ((b + 1) * D) * BLOCK, Kt, D);
#pragma unroll
                for (int mu = 0; mu < D; ++mu) {
                    PA[mu] = f.sub(Kt[mu], Ki[mu]);
                    PB[mu] = f.sub(Kj1[mu], Kt[mu]);
                    dP[mu] = f.sub(PA[mu], PB[mu]);
                }
                // three-gluon vertex of the split at s = i + b
                const T adj = f.template dot<DS, METRIC>(pb, sf);
                sa = (b == 0) ? adj : f.add(sa, adj);
                const T pa_jb = f.template dot<D, METRIC>(PA, sf);
                const T pb_ja = f.template dot<D, METRIC>(PB, pb);
                f.template axpy<D>(acc, adj, dP);        // momentum part of V3
                T csuf = f.dbl(pb_ja);
                if (b + 1 >= 2) csuf = f.sub(csuf, Sb[Sl::sbase(b + 1) * BLOCK]);
                f.template axpy<DS>(acc, csuf, sf);
                T cpre = f.neg(f.dbl(pa_jb));
                if (lenB >= 2) cpre = f.sub(cpre, Sb[(Sl::sbase(lenB) + b + 1) * BLOCK]);
                f.template axpy<DS>(acc, cpre, pb);
                // four-gluon vertex: prefix [i, i+a], inner [i+a+1, i+b], suffix
#pragma unroll
                for (int a = 0; a < b; ++a) {
                    T pa[DS];
                    if constexpr (CACHE) {
#pragma unroll
                        for (int mu = 0; mu < DS; ++mu) pa[mu] = pfc[a][mu];
                    } else {
                        load_vec(jslot(a + 1, 0), pa, DS);
                    }
                    const T g = f.template dot<DS, METRIC>(pa, sf);
                    T inner[DS];
                    load_vec(jslot(b - a, a + 1), inner, DS);
                    f.template axpy<DS>(acc, f.dbl(g), inner);
                }
            }

            if constexpr (LEN < N) {
                const T inv = Ib[Sl::sbase(LEN) * BLOCK];
                T* dst = jslot(LEN, 0);
#pragma unroll
                for (int mu = 0; mu < DS; ++mu) dst[mu * BLOCK] = f.mul(acc[mu], inv);
                Sb[Sl::sbase(LEN) * BLOCK] = sa;
            } else {
#pragma unroll
                for (int mu = 0; mu < DS; ++mu) top[mu] = acc[mu];
            }
        }
    }

    template <int LEN>
    __device__ static __forceinline__ void p2_len(const F& f, T* base) {
#pragma unroll 1
        for (int i = 0; i + LEN - 1 < N; ++i) {
            const T* Kb = base + (Fr::OFF_K + i * D) * BLOCK;
            T P[D];
#pragma unroll
            for (int mu = 0; mu < D; ++mu) P[mu] = f.sub(Kb[(LEN * D + mu) * BLOCK], Kb[mu * BLOCK]);
            base[(Fr::OFF_SA + Sl::sbase(LEN) + i) * BLOCK] = f.template dot<D, METRIC>(P, P);
        }
    }

    template <int... Ls>
    __device__ static __forceinline__ void all_p2(const F& f, T* base, std::integer_sequence<int, Ls...>) {
        (p2_len<Ls + 2>(f, base), ...);
    }
    template <int... Ls>
    __device__ static __forceinline__ void all_ranges(const F& f, T* base, T* top,
                                                      std::integer_sequence<int, Ls...>) {
        (range_len<Ls + 2>(f, base, top), ...);
    }

    // 1/P^2 for every internal range into the INV slots; returns "singular".
    __device__ static __forceinline__ bool inverses(const F& f, T* base) {
        T* X = base + Fr::OFF_SA * BLOCK;
        T* Y = base + Fr::OFF_INV * BLOCK;
        if constexpr (F::kIsFp) {
            // Montgomery simultaneous inversion: prefix products, one inverse,
            // then the backward sweep.
            T c = X[0];
            Y[0] = c;
#pragma unroll 1
            for (int s = 1; s < Sl::NS; ++s) {
                c = f.mul(c, X[s * BLOCK]);
                Y[s * BLOCK] = c;
            }
            const bool singular = f.is_zero(c);
            T r = f.inv(c);
#pragma unroll 1
            for (int s = Sl::NS - 1; s > 0; --s) {
                const T x = X[s * BLOCK];
                Y[s * BLOCK] = f.mul(Y[(s - 1) * BLOCK], r);
                r = f.mul(r, x);
            }
            Y[0] = r;
            return singular;
        } else {
            bool singular = false;
#pragma unroll 1
            for (int s = 0; s < Sl::NS; ++s) {
                const T x = X[s * BLOCK];
                singular |= f.is_zero(x);
                Y[s * BLOCK] = f.inv(x);
            }
            return singular;
        }
    }
};

template <class F, int NLEG, int D, int DS, int METRIC, int BLOCK, bool GLOBAL_TABLE>
__global__ void __launch_bounds__(BLOCK)
bg_recursion_kernel(const F f, const LaunchArgs a) {
    constexpr int N = NLEG - 1;
    using T = typename F::T;
    using io_t = typename F::io_t;
    using R = Rec<F, N, D, DS, METRIC, BLOCK>;
    using Fr = Frame<N, D, DS>;

    extern __shared__ __align__(16) unsigned char bg_smem[];
    T* base;
    if constexpr (GLOBAL_TABLE) {
        base = reinterpret_cast<T*>(a.ws) + static_cast<size_t>(blockIdx.x) * Fr::WORDS * BLOCK + threadIdx.x;
    } else {
        base = reinterpret_cast<T*>(bg_smem) + threadIdx.x;
    }
    const io_t* kin = static_cast<const io_t*>(a.k);
    const io_t* ein = static_cast<const io_t*>(a.eps);
    io_t* out = static_cast<io_t*>(a.out);
    const int64_t total = a.E * a.H;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * BLOCK;

    for (int64_t u = static_cast<int64_t>(blockIdx.x) * BLOCK + threadIdx.x; u < total; u += stride) {
        int64_t e = u;
        int h = 0;
        if (a.H > 1) {
            e = u / a.H;
            h = static_cast<int>(u - e * a.H);
        }
        // a1: load momenta into the prefix-sum table K_0..K_N (K_0 = 0); leg n
        // is not needed (P_{1,n-1} = -k_n is never used).  Zero padding to D.
        {
            const io_t* kp = kin + e * NLEG * a.d_in;
            T Kacc[D];
#pragma unroll
            for (int mu = 0; mu < D; ++mu) {
                Kacc[mu] = f.zero();
                base[(Fr::OFF_K + mu) * BLOCK] = Kacc[mu];
            }
#pragma unroll
            for (int l = 0; l < N; ++l) {
#pragma unroll
                for (int mu = 0; mu < D; ++mu) {
                    if (mu < a.d_in) Kacc[mu] = f.add(Kacc[mu], f.from_io(kp[l * a.d_in + mu]));
                    base[(Fr::OFF_K + (l + 1) * D + mu) * BLOCK] = Kacc[mu];
                }
            }
        }
        // currents of length 1 are the polarisations (Sec. 2.2)
        T eL[DS];
#pragma unroll
        for (int l = 0; l < NLEG; ++l) {
            const int s = (a.assign != nullptr) ? a.assign[h * NLEG + l] : 0;
            const io_t* ep = ein + ((e * NLEG + l) * a.S + s) * a.ds_in;
#pragma unroll
            for (int mu = 0; mu < DS; ++mu) {
                const T v = (mu < a.ds_in) ? f.from_io(ep[mu]) : f.zero();
                if (l < N) base[(Fr::OFF_J + (Slots<N>::jbase(1) + l) * DS + mu) * BLOCK] = v;
                else eL[mu] = v;
            }
        }
        // a2, a3: P^2 of every internal range, then all inverses
        R::all_p2(f, base, std::make_integer_sequence<int, N - 2>{});
        const bool singular = R::inverses(f, base);
        // a4: the recursion, length by length
        T top[DS];
        R::all_ranges(f, base, top, std::make_integer_sequence<int, N - 1>{});
        // a5: contract with the last polarisation
        const T A = f.template dot<DS, METRIC>(eL, top);
        out[u] = singular ? f.to_io(f.zero()) : f.to_io(A);
        if (a.status != nullptr && h == 0) a.status[e] = singular ? 1 : 0;
    }
}

}  // namespace bgk
