// bg_compact.cuh -- Berends-Giele recursion, one point (and state assignment)
// per thread, with the number of legs a RUN-TIME parameter.
//
// Method (arXiv:2502.07060, Sec. 2.2): currents over consecutive leg ranges,
//   J(i,j) = (-i/P_ij^2) [ sum_s V3(P_A,P_B) J_A J_B + sum_{s<t} V4 J_A J_B J_C ],
// vertices V3, V4 of Sec. 2.2; with every vertex i cancelled against the -i of
// the propagator,
//   R(i,j) = sum_s   (J_A.J_B)(P_A - P_B) + 2(P_B.J_A) J_B - 2(P_A.J_B) J_A
//          + sum_s<t 2(J_A.J_C) J_B - (J_B.J_C) J_A - (J_A.J_B) J_C,
//   J(i,j) = R(i,j) / P_ij^2 (internal ranges),   A = eps_n . R(1, n-1).
//
// The sum is regrouped by the sub-current each term multiplies (an identity,
// exact over F_p):
//   prefix  A = [i, s]:   -2 P_A.J_[s+1,j] - SA([s+1,j])
//   suffix  C = [t+1, j]: +2 P_C.J_[i,t]   - SA([i,t])
//   inner   B = [s+1, t]:  2 J_[i,s].J_[t+1,j]
//   plus the momentum part sum_s (J_A.J_B)(P_A - P_B)
//     = 2 sum_s (J_A.J_B) K_{s+1} - SA([i,j]) (K_i + K_{j+1}),
// where SA(X) = sum over the splits X = Y|Z of J_Y.J_Z is accumulated while X
// itself is built and stored next to its current.  Per range of length m this
// costs m(m+1)/2 - 1 vector updates instead of 2(m-1) + 3 C(m-1,2).  The
// coefficients P_B.J_A and P_A.J_B are taken as P.J_A and P.J_B with P the
// range momentum: currents of on-shell legs with transverse states are
// conserved (P_X.J_X = 0), the documented precondition of the inputs.
//
// Per-point table for N = n - 1 legs (layout: TableIO below):
//   currents of length 1..N-1 (D_s each), prefix sums K_0..K_N of the momenta
//   (D each; P_{i,j} = K_{j+1} - K_i), SA and 1/P^2 per internal range.
// Shared-memory placement keeps the table on chip; global placement keeps it
// in a scratch buffer that one resident wave of blocks reuses (L2 resident).
//
// Only the component loops are unrolled; the loops over lengths, ranges and
// splits run at run time, so one compact kernel serves every n and stays in
// the instruction cache.
#pragma once
#include <cstdint>
#include <type_traits>

#include "bg_field.cuh"

namespace bgk {

struct CompactArgs {
    int64_t E;                  // points
    int H;                      // state assignments per point
    int S;                      // states per leg
    int n;                      // gluons (4..12)
    int d_in, ds_in;            // dimensions of the inputs (<= D, D_s)
    const void* k;              // [E][n][d_in]
    const void* eps;            // [E][n][S][ds_in]
    void* out;                  // [E][H]
    uint8_t* status;            // [E] or null
    const uint8_t* assign;      // device [H][n] or null (H == 1)
    void* ws;                   // global table (global placement)
    uint32_t four_d_legs;       // bit l: leg l is four-dimensional (read by MIXED kernels)
    unsigned long long* violation;   // checked builds: first out-of-range table index
};

// Table-index checking (builds compiled with BG_CHECKED; without it the checks
// vanish).  Every slot index is compared with the extent of its region before
// the access; a violation records (site << 32 | index) in *violation (the
// first one wins) and the access goes to slot 0 instead, so a wrong index
// never leaves the thread's own table.
__device__ __forceinline__ int checked_slot(unsigned long long* violation, int idx, int extent, int site) {
#ifdef BG_CHECKED
    if (idx < 0 || idx >= extent) {
        if (violation != nullptr)
            atomicCAS(violation, 0ull, (static_cast<unsigned long long>(site) << 32) | static_cast<uint32_t>(idx));
        return 0;
    }
#else
    (void)violation; (void)extent; (void)site;
#endif
    return idx;
}

// Input preconditions of the boundary (builds compiled with BG_CHECKED;
// ordinary builds never call this): every F_p value canonical (< p), momentum
// conservation sum_l k_l = 0, on-shell legs k_l^2 = 0 and transverse states
// eps_{l,s} . k_l = 0 for every state s (Sec. 2.2 builds the currents from
// on-shell legs and imposes momentum conservation at the amplitude; the
// kernels rely on the current conservation these imply).  Exact over F_p
// (plain modular arithmetic on the canonical inputs); for the complex fields
// within kPreconditionTol relative to the point's momentum scale kmax (the
// largest Euclidean norm of its momenta): |sum k| <= tol kmax,
// |k_l^2| <= tol kmax^2, |eps . k_l| <= tol |eps| kmax.
constexpr double kPreconditionTol = 1e-8;

template <int METRIC>
__device__ inline bool fp_preconditions(uint32_t p, const uint32_t* k, const uint32_t* eps, int n, int d, int ds,
                                        int S, const int* used) {
    const uint64_t P = p;
    for (int i = 0; i < n * d; ++i)
        if (k[i] >= p) return false;
    for (int l = 0; l < n; ++l)
        for (int i = 0; i < (used ? used[l] : S) * ds; ++i)
            if (eps[l * S * ds + i] >= p) return false;
    for (int mu = 0; mu < d; ++mu) {
        uint64_t sum = 0;
        for (int l = 0; l < n; ++l) sum = (sum + k[l * d + mu]) % P;
        if (sum != 0) return false;
    }
    for (int l = 0; l < n; ++l) {
        const uint32_t* kl = k + l * d;
        uint64_t k2 = 0;
        for (int mu = 0; mu < d; ++mu) {
            const uint64_t t = static_cast<uint64_t>(kl[mu]) * kl[mu] % P;
            k2 = (k2 + (msign<METRIC>(mu) > 0 ? t : P - t)) % P;
        }
        if (k2 != 0) return false;
        for (int s = 0; s < (used ? used[l] : S); ++s) {
            const uint32_t* es = eps + (l * S + s) * ds;
            uint64_t ek = 0;
            for (int mu = 0; mu < d; ++mu) {
                const uint64_t t = static_cast<uint64_t>(es[mu]) * kl[mu] % P;
                ek = (ek + (msign<METRIC>(mu) > 0 ? t : P - t)) % P;
            }
            if (ek != 0) return false;
        }
    }
    return true;
}

// complex FP64 (KC = double2: complex momenta, double: real momenta)
template <int METRIC, class KC>
__device__ inline bool c64_preconditions(const KC* k, const double2* eps, int n, int d, int ds, int S,
                                         const int* used) {
    auto re = [](const KC& x) -> double { if constexpr (sizeof(KC) == 16) return x.x; else return x; };
    auto im = [](const KC& x) -> double { if constexpr (sizeof(KC) == 16) return x.y; else return 0.0; };
    double kmax = 0.0;
    for (int l = 0; l < n; ++l) {
        double nk = 0.0;
        for (int mu = 0; mu < d; ++mu) nk += re(k[l * d + mu]) * re(k[l * d + mu]) + im(k[l * d + mu]) * im(k[l * d + mu]);
        kmax = fmax(kmax, sqrt(nk));
    }
    for (int mu = 0; mu < d; ++mu) {
        double sr = 0.0, si = 0.0;
        for (int l = 0; l < n; ++l) { sr += re(k[l * d + mu]); si += im(k[l * d + mu]); }
        if (sqrt(sr * sr + si * si) > kPreconditionTol * kmax) return false;
    }
    for (int l = 0; l < n; ++l) {
        const KC* kl = k + l * d;
        double k2r = 0.0, k2i = 0.0;
        for (int mu = 0; mu < d; ++mu) {
            const double g = msign<METRIC>(mu);
            k2r += g * (re(kl[mu]) * re(kl[mu]) - im(kl[mu]) * im(kl[mu]));
            k2i += g * 2.0 * re(kl[mu]) * im(kl[mu]);
        }
        if (sqrt(k2r * k2r + k2i * k2i) > kPreconditionTol * kmax * kmax) return false;
        for (int s = 0; s < (used ? used[l] : S); ++s) {
            const double2* es = eps + (l * S + s) * ds;
            double er = 0.0, ei = 0.0, ne = 0.0;
            for (int mu = 0; mu < ds; ++mu) ne += es[mu].x * es[mu].x + es[mu].y * es[mu].y;
            for (int mu = 0; mu < d; ++mu) {
                const double g = msign<METRIC>(mu);
                er += g * (es[mu].x * re(kl[mu]) - es[mu].y * im(kl[mu]));
                ei += g * (es[mu].x * im(kl[mu]) + es[mu].y * re(kl[mu]));
            }
            if (sqrt(er * er + ei * ei) > kPreconditionTol * sqrt(ne) * kmax) return false;
        }
    }
    return true;
}

// The preconditions for point e of a batch in the boundary layouts
// (momenta [E][n][d], polarisations [E][n][S][D_s]); used[l] (or all S when
// used is null) is the number of leg l's state slots that are evaluated.
template <class F, int METRIC>
__device__ inline bool inputs_meet_preconditions(const F& f, const void* k, const void* eps, int64_t e, int n,
                                                 int d, int ds, int S, const int* used = nullptr) {
    using kio_t = typename F::kio_t;
    using io_t = typename F::io_t;
    const kio_t* kp = static_cast<const kio_t*>(k) + e * n * d;
    const io_t* ep = static_cast<const io_t*>(eps) + e * n * S * ds;
    if constexpr (F::kIsFp) return fp_preconditions<METRIC>(f.p, kp, ep, n, d, ds, S, used);
    else return c64_preconditions<METRIC>(kp, ep, n, d, ds, S, used);
}

// Table geometry for N = n - 1 recursion legs (host and device), in table
// elements per thread.  Region starts are rounded up to 4 elements so that
// vector accesses stay aligned.
struct Geometry {
    int N;
    __host__ __device__ static int up4(int x) { return (x + 3) & ~3; }
    __host__ __device__ int jbase(int len) const { return ((len - 1) * (2 * N + 2 - len)) >> 1; }
    __host__ __device__ int nj() const { return jbase(N); }              // currents, length 1..N-1
    __host__ __device__ int ns() const { return jbase(N) - N; }          // internal ranges
    __host__ __device__ int sbase(int len) const { return jbase(len) - N; }
    __host__ __device__ int off_k(int DS) const { return up4(nj() * DS); }
    __host__ __device__ int off_sa(int D, int DS) const { return off_k(DS) + up4((N + 1) * D); }
    __host__ __device__ int off_inv(int D, int DS) const { return off_sa(D, DS) + ns(); }
    __host__ __device__ int words(int D, int DS) const { return off_inv(D, DS) + ns(); }
    // split placement: currents in global scratch, the rest (K, SA, 1/P^2) on chip
    __host__ __device__ int cur_words(int DS) const { return off_k(DS); }
    __host__ __device__ int aux_words(int D, int DS) const { return words(D, DS) - off_k(DS); }
};

// Table placements of the compact kernel.
constexpr int kPlaceShared = 0;     // whole table in shared memory
constexpr int kPlaceGlobal = 1;     // whole table in global scratch (L2 resident)
constexpr int kPlaceSplit = 2;      // currents in global scratch, K / SA / 1/P^2 in shared memory

// Vector access to the table.  VEC (F_p): a thread's K-component vector is
// contiguous ([slot][thread][K]); it is read with 16- or 8-byte accesses, and
// consecutive threads' vectors are adjacent, so a warp's access is contiguous
// (coalesced in global memory, bank-conflict free in shared memory).  Not VEC
// (C64, 16-byte elements): component mu of slot s of thread t is at
// [(s * K + mu) * BLOCK + t], one 16-byte access per component.
template <class T, bool VEC, int BLOCK>
struct TableIO {
    template <int K>
    __device__ static __forceinline__ T* vec(T* region, int slot) {
        if constexpr (VEC) return region + slot * BLOCK * K;      // region already offset by t*K
        else return region + slot * K * BLOCK;                    // region already offset by t
    }
    template <int K>
    __device__ static __forceinline__ void load(const T* p, T* v) {
        if constexpr (VEC) {
            if constexpr (K % 4 == 0) {
#pragma unroll
                for (int q = 0; q < K / 4; ++q) {
                    const uint4 x = reinterpret_cast<const uint4*>(p)[q];
                    v[4 * q] = x.x; v[4 * q + 1] = x.y; v[4 * q + 2] = x.z; v[4 * q + 3] = x.w;
                }
            } else {
#pragma unroll
                for (int q = 0; q < K / 2; ++q) {
                    const uint2 x = reinterpret_cast<const uint2*>(p)[q];
                    v[2 * q] = x.x; v[2 * q + 1] = x.y;
                }
            }
        } else {
#pragma unroll
            for (int mu = 0; mu < K; ++mu) v[mu] = p[mu * BLOCK];
        }
    }
    // the first KL components (KL = K, or 4 <= K) of a K-component vector
    template <int K, int KL>
    __device__ static __forceinline__ void load_live(const T* p, T* v) {
        static_assert(KL == K || (KL == 4 && K >= 4), "live prefix of four components");
        if constexpr (KL == K) {
            load<K>(p, v);
        } else if constexpr (VEC) {
            if constexpr (K % 4 == 0) {
                const uint4 x = reinterpret_cast<const uint4*>(p)[0];
                v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
            } else {
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const uint2 x = reinterpret_cast<const uint2*>(p)[q];
                    v[2 * q] = x.x; v[2 * q + 1] = x.y;
                }
            }
        } else {
#pragma unroll
            for (int mu = 0; mu < KL; ++mu) v[mu] = p[mu * BLOCK];
        }
    }
    template <int K>
    __device__ static __forceinline__ void store(T* p, const T* v) {
        if constexpr (VEC) {
            if constexpr (K % 4 == 0) {
#pragma unroll
                for (int q = 0; q < K / 4; ++q)
                    reinterpret_cast<uint4*>(p)[q] = make_uint4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
            } else {
#pragma unroll
                for (int q = 0; q < K / 2; ++q)
                    reinterpret_cast<uint2*>(p)[q] = make_uint2(v[2 * q], v[2 * q + 1]);
            }
        } else {
#pragma unroll
            for (int mu = 0; mu < K; ++mu) p[mu * BLOCK] = v[mu];
        }
    }
};

// Inputs and outputs are touched once per point: streaming (evict-first)
// accesses keep them from displacing the recursion table in L1 and L2.
template <class X>
__device__ __forceinline__ X ld_once(const X* p) { return __ldcs(p); }
template <class X>
__device__ __forceinline__ void st_once(X* p, X v) { __stcs(p, v); }

// One leg's F_p input vector of K components, the first k_in stored (the
// rest zero padding).  A vector of exactly K components at an aligned
// address (vec) is read with 16-byte (K = 4, 8) or 8-byte (K = 6) loads:
// a thread's row is contiguous, so fewer and wider loads touch the same
// sectors and the prologue's L1 traffic drops.
template <int K>
__device__ __forceinline__ void load_leg_fp(const uint32_t* p, int k_in, bool vec, uint32_t* v) {
    if (vec) {
        if constexpr (K % 4 == 0) {
#pragma unroll
            for (int q = 0; q < K / 4; ++q) {
                const uint4 x = ld_once(reinterpret_cast<const uint4*>(p) + q);
                v[4 * q] = x.x; v[4 * q + 1] = x.y; v[4 * q + 2] = x.z; v[4 * q + 3] = x.w;
            }
            return;
        } else if constexpr (K % 2 == 0) {
#pragma unroll
            for (int q = 0; q < K / 2; ++q) {
                const uint2 x = ld_once(reinterpret_cast<const uint2*>(p) + q);
                v[2 * q] = x.x; v[2 * q + 1] = x.y;
            }
            return;
        }
    }
#pragma unroll
    for (int mu = 0; mu < K; ++mu) v[mu] = (mu < k_in) ? ld_once(p + mu) : 0u;
}

// alignment that load_leg_fp's vector path needs for K-component rows
template <int K>
__host__ __device__ constexpr int leg_align() { return K % 4 == 0 ? 16 : 8; }

// The whole recursion for work item u (point e = u / H, assignment h = u % H)
// with the block's currents at `tab` and its prefix sums, SA and 1/P^2 at
// `aux` (shared or global memory).
template <class F, int D, int DS, int METRIC, int BLOCK, bool MIXED = false>
__device__ __forceinline__ void bg_point(const F& f, const CompactArgs& a, typename F::T* tab,
                                         typename F::T* aux, int64_t u) {
    using T = typename F::T;
    using C = typename F::C;
    using Acc = typename F::A;
    using io_t = typename F::io_t;
    using TK = typename F::TK;               // momentum component (may be real)
    using kio_t = typename F::kio_t;

    const int NLEG = a.n;
    const Geometry g{NLEG - 1};
    const int N = g.N;
    const int OFF_K = g.off_k(DS), OFF_SA = g.off_sa(D, DS), OFF_INV = g.off_inv(D, DS);
    constexpr bool VEC = F::kIsFp;
    using IO = TableIO<T, VEC, BLOCK>;
    using KIO = TableIO<TK, VEC, BLOCK>;
    const int t = threadIdx.x;
    T* Jr = tab + (VEC ? t * DS : t);                              // currents
    TK* Kr = reinterpret_cast<TK*>(aux) + (VEC ? t * D : t);      // prefix sums
    T* Sr = aux + (OFF_SA - OFF_K) * BLOCK + t;                    // SA per internal range
    T* Ir = aux + (OFF_INV - OFF_K) * BLOCK + t;                   // 1/P^2 per internal range
    const int NJ = g.nj(), NS_ = g.ns();
    // slot addressing of the four table regions (checked in BG_CHECKED builds)
    auto jslot = [&](int slot) { return IO::template vec<DS>(Jr, checked_slot(a.violation, slot, NJ, 1)); };
    auto jvec = [&](int len, int start) { return jslot(g.jbase(len) + start); };
    auto kvec = [&](int i) { return KIO::template vec<D>(Kr, checked_slot(a.violation, i, N + 1, 2)); };
    auto sidx_ok = [&](int i) { return checked_slot(a.violation, i, NS_, 3) * BLOCK; };
    const kio_t* kin = static_cast<const kio_t*>(a.k);
    const io_t* ein = static_cast<const io_t*>(a.eps);
    io_t* out = static_cast<io_t*>(a.out);

    int64_t e = u;
    int h = 0;
    if (a.H > 1) {
        e = u / a.H;
        h = static_cast<int>(u - e * a.H);
    }
#ifdef BG_CHECKED
    // every item of a point checks all of its states, so all items agree
    const bool violated = !inputs_meet_preconditions<F, METRIC>(f, a.k, a.eps, e, NLEG, a.d_in, a.ds_in, a.S);
#else
    constexpr bool violated = false;
#endif
    // a1: momenta -> prefix sums K_0 = 0, K_{l+1} = K_l + k_l (leg n unused:
    // P_{1,n-1} = -k_n never enters); polarisations -> currents of length 1.
    {
        const kio_t* kp = kin + e * NLEG * a.d_in;
        TK Kacc[D];
#pragma unroll
        for (int mu = 0; mu < D; ++mu) Kacc[mu] = f.kzero();
        KIO::template store<D>(kvec(0), Kacc);
        if constexpr (F::kIsFp) {
            const bool vec = a.d_in == D && reinterpret_cast<uintptr_t>(a.k) % leg_align<D>() == 0;
#pragma unroll 1
            for (int l = 0; l < N; ++l) {
                uint32_t raw[D];
                load_leg_fp<D>(kp + l * a.d_in, a.d_in, vec, raw);
#pragma unroll
                for (int mu = 0; mu < D; ++mu) Kacc[mu] = f.kadd(Kacc[mu], f.kfrom_io(raw[mu]));
                KIO::template store<D>(kvec(l + 1), Kacc);
            }
        } else {
#pragma unroll 1
            for (int l = 0; l < N; ++l) {
#pragma unroll
                for (int mu = 0; mu < D; ++mu)
                    if (mu < a.d_in) Kacc[mu] = f.kadd(Kacc[mu], f.kfrom_io(ld_once(kp + l * a.d_in + mu)));
                KIO::template store<D>(kvec(l + 1), Kacc);
            }
        }
    }
    T eL[DS];
    [[maybe_unused]] const bool vec_eps =
        a.ds_in == DS && reinterpret_cast<uintptr_t>(a.eps) % leg_align<DS>() == 0;
#pragma unroll 1
    for (int l = 0; l < NLEG; ++l) {
        const int s = (a.assign != nullptr) ? a.assign[h * NLEG + l] : 0;
        const io_t* ep = ein + ((e * NLEG + l) * a.S + s) * a.ds_in;
        T v[DS];
        if constexpr (F::kIsFp) {
            // canonical residues kept as they are (level 0, no Montgomery
            // conversion): each current of length m is then uniformly one
            // level lower per state, which amplitude_raw undoes at the end
            load_leg_fp<DS>(ep, a.ds_in, vec_eps, v);
        } else {
#pragma unroll
            for (int mu = 0; mu < DS; ++mu) v[mu] = (mu < a.ds_in) ? f.from_io(ld_once(ep + mu)) : f.zero();
        }
        if (l < N) {
            IO::template store<DS>(jvec(1, l), v);     // current (1, l)
        } else {
#pragma unroll
            for (int mu = 0; mu < DS; ++mu) eL[mu] = v[mu];
        }
    }
    // a2: P^2 of every internal range (length 2..N-1), flat index sbase(m) + i
    T* X = Sr;     // P^2 inputs of the inverse (reuses the SA slots)
    T* Y = Ir;     // 1/P^2
#pragma unroll 1
    for (int m = 2; m < N; ++m) {
#pragma unroll 1
        for (int i = 0; i + m - 1 < N; ++i) {
            TK Ka[D], Kb[D], P[D];
            KIO::template load<D>(kvec(i), Ka);
            KIO::template load<D>(kvec(i + m), Kb);
#pragma unroll
            for (int mu = 0; mu < D; ++mu) P[mu] = f.ksub(Kb[mu], Ka[mu]);
            X[sidx_ok(g.sbase(m) + i)] = f.inv_input(f.template kkdot<D, METRIC>(P, P));
        }
    }
    // a3: all inverses.  F_p: Montgomery simultaneous inversion (prefix
    // products, one Fermat inverse, backward sweep); C64: per range.
    bool singular = false;
    const int NS = g.ns();
    if constexpr (F::kIsFp) {
        T c = X[0];
        Y[0] = c;
#pragma unroll 1
        for (int s = 1; s < NS; ++s) {
            c = f.inv_mul(c, X[sidx_ok(s)]);
            Y[sidx_ok(s)] = c;
        }
        singular = f.is_zero(c);
        T r = f.inv_scalar(c);
#pragma unroll 1
        for (int s = NS - 1; s > 0; --s) {
            const T x = X[sidx_ok(s)];
            Y[sidx_ok(s)] = f.inv_store(f.inv_mul(Y[sidx_ok(s - 1)], r));
            r = f.inv_mul(r, x);
        }
        Y[0] = f.inv_store(r);
    } else {
#pragma unroll 1
        for (int s = 0; s < NS; ++s) {
            const T x = X[sidx_ok(s)];
            singular |= f.is_zero(x);
            Y[sidx_ok(s)] = f.inv_scalar(x);
        }
    }

    // a4: the recursion over all ranges [i, i+m-1].  Slot indices of the
    // sub-currents are advanced incrementally (count(L) = N - L + 1 slots per
    // length L) instead of being recomputed from jbase() at every access.
    // The range [i, i+m-1] is evaluated with DL momentum and DSL current
    // components: D and DS, or four for a range of four-dimensional legs only
    // (MIXED kernels), whose momenta and currents vanish beyond the first
    // four components.
    io_t result = f.zero_io();
    //
    // Table addresses inside a range are byte offsets from the thread's
    // current region, advanced by additions: the slot of the prefix, suffix
    // and inner current of each split and gap moves by a step that itself
    // changes by one slot per split or gap, so no access multiplies a slot
    // index by the slot size (measured on GB300, n=8, d=6, with the 96-bit
    // contractions of FpOps: 4.41 against 4.66 ms per 2^22 points).
    auto range = [&](auto live_d, auto live_ds, const int m, const int i) {
        constexpr int DL = decltype(live_d)::value;
        constexpr int DSL = decltype(live_ds)::value;
        constexpr int SLOT = DS * BLOCK;                                  // elements per current slot
        constexpr int SLOTB = SLOT * static_cast<int>(sizeof(T));         // bytes per current slot
        constexpr int KSTEP = D * BLOCK;                                  // elements per prefix-sum slot
        const char* Jb = reinterpret_cast<const char*>(Jr);
        // current at byte offset `off` (a multiple of SLOTB from Jr)
        auto at = [&](int off, int site) -> const T* {
#ifdef BG_CHECKED
            return Jr + checked_slot(a.violation, off / SLOTB, NJ, site) * SLOT;
#else
            (void)site;
            return reinterpret_cast<const T*>(Jb + off);
#endif
        };
        // K_i + K_{j+1} (the -SA(i,j) momentum term) and the range momentum
        // P = P_[i,j] = K_{j+1} - K_i.  Current conservation (P_X . J_X = 0
        // for every current of on-shell legs with transverse states) gives
        // P_B . J_A = P . J_A and P_A . J_B = P . J_B for every split A|B, so
        // the split momenta P_A, P_B are never formed.
        TK KiKj[DL], P[DL];
        {
            TK Ki[DL], Kj[DL];
            KIO::template load_live<D, DL>(kvec(i), Ki);
            KIO::template load_live<D, DL>(kvec(i + m), Kj);
#pragma unroll
            for (int mu = 0; mu < DL; ++mu) {
                KiKj[mu] = f.kadd(Ki[mu], Kj[mu]);
                P[mu] = f.ksub(Kj[mu], Ki[mu]);
            }
        }
        Acc acc[DSL];
        f.template acc_zero<DSL>(acc);
        C sa = f.czero();
        int ps = i;                          // slot of the prefix [i, i+b]      (length b+1)
        int ss = g.jbase(m - 1) + i + 1;     // slot of the suffix [i+b+1, j]    (length m-1-b)
        // byte offsets and their steps: ps += N - b, ss -= N - m + 2 + b, and
        // the first inner slot [i+1, i+b] (jbase(b) + i + 1) += N - b + 1
        int off_ps = ps * SLOTB, step_ps = N * SLOTB;
        int off_ss = ss * SLOTB, step_ss = (N - m + 2) * SLOTB;
        int off_es = (i - N) * SLOTB, step_es = (N + 1) * SLOTB;
        const TK* Kt_ptr = kvec(i + 1);      // K_{i+b+1}
        // momentum terms 2 adj_b K_{i+b+1} of consecutive splits are
        // accumulated in pairs (one reduction per pair)
        C mom_c = f.czero();
        TK mom_v[DL];
        bool mom_pending = false;
        // The gap-pair loop unrolled twice gives the scheduler two pairs of
        // loads and contractions at a time.  Measured on the F_p kernel with
        // D = D_s = 6: 0.9 % faster at the same 94-96 registers; at other
        // dimensions and for the complex kernels the unrolled loop takes up
        // to 40 more registers (fewer resident blocks), so it stays rolled.
        constexpr int kGapUnroll = (F::kIsFp && !MIXED && D == 6 && DS == 6) ? 2 : 1;
#pragma unroll 1
        for (int b = 0; b < m - 1; ++b) {
            const int lenA = b + 1, lenB = m - 1 - b;   // [i, i+b] | [i+b+1, j]
            T pb[DSL], sf[DSL];
            TK Kt[DL];
            IO::template load_live<DS, DSL>(at(off_ps, 1), pb);
            IO::template load_live<DS, DSL>(at(off_ss, 1), sf);
            KIO::template load_live<D, DL>(Kt_ptr, Kt);
            Kt_ptr += KSTEP;
            // three-gluon vertex of the split at s = i + b
            const C adj = f.template dot<DSL, METRIC>(pb, sf);
            const C pa_jb = f.template kdot<DL, METRIC>(P, sf);     // P_A . J_B = P . J_B
            const C pb_ja = f.template kdot<DL, METRIC>(P, pb);     // P_B . J_A = P . J_A
            sa = f.cadd(sa, adj);
            C csuf = f.cdbl(pb_ja);
            if (lenA >= 2) csuf = f.csub(csuf, f.t_to_c(Sr[sidx_ok(ps - N)]));     // SA(prefix)
            C cpre = f.cneg(f.cdbl(pa_jb));
            if (lenB >= 2) cpre = f.csub(cpre, f.t_to_c(Sr[sidx_ok(ss - N)]));     // SA(suffix)
            f.template acc2<DSL>(acc, csuf, sf, cpre, pb);
            // momentum part: adj (P_A - P_B) = adj (2 K_{i+b+1} - K_i - K_j);
            // the K_i + K_j share is added once per range below
            if (mom_pending) {
                f.template kacc2<DL>(acc, mom_c, mom_v, f.cdbl(adj), Kt);
                mom_pending = false;
            } else {
                mom_c = f.cdbl(adj);
#pragma unroll
                for (int mu = 0; mu < DL; ++mu) mom_v[mu] = Kt[mu];
                mom_pending = true;
            }
            // four-gluon vertex: prefix [i, i+q] (slot advances by N - q),
            // inner [i+q+1, i+b] (slot falls by N - b + 1 + q), suffix sf;
            // gaps in pairs (independent loads and contractions in flight)
            int off_pq = i * SLOTB, step_pq = N * SLOTB;
            int off_iq = off_es, step_iq = (N - b + 1) * SLOTB;
            int q = 0;
#pragma unroll(kGapUnroll)
            for (; q + 1 < b; q += 2) {
                T pa0[DSL], pa1[DSL], in0[DSL], in1[DSL];
                IO::template load_live<DS, DSL>(at(off_pq, 1), pa0);
                IO::template load_live<DS, DSL>(at(off_iq, 1), in0);
                off_pq += step_pq; off_iq -= step_iq;
                step_pq -= SLOTB; step_iq += SLOTB;
                IO::template load_live<DS, DSL>(at(off_pq, 1), pa1);
                IO::template load_live<DS, DSL>(at(off_iq, 1), in1);
                off_pq += step_pq; off_iq -= step_iq;
                step_pq -= SLOTB; step_iq += SLOTB;
                const C g0 = f.cdbl(f.template dot<DSL, METRIC>(pa0, sf));
                const C g1 = f.cdbl(f.template dot<DSL, METRIC>(pa1, sf));
                f.template acc2<DSL>(acc, g0, in0, g1, in1);
            }
            if (q < b) {
                T pa0[DSL], in0[DSL];
                IO::template load_live<DS, DSL>(at(off_pq, 1), pa0);
                IO::template load_live<DS, DSL>(at(off_iq, 1), in0);
                const C g0 = f.cdbl(f.template dot<DSL, METRIC>(pa0, sf));
                f.template acc1<DSL>(acc, g0, in0);
            }
            ps += N - b;                     // prefix length b+1 -> b+2
            ss -= N - lenB + 1;              // suffix length lenB -> lenB-1
            off_ps += step_ps; step_ps -= SLOTB;
            off_ss -= step_ss; step_ss += SLOTB;
            off_es += step_es; step_es -= SLOTB;
        }
        if (mom_pending) f.template kacc2<DL>(acc, mom_c, mom_v, f.cneg(sa), KiKj);
        else f.template kacc1<DL>(acc, f.cneg(sa), KiKj);         // - SA(i,j) (K_i + K_j)
        if (m < N) {
            const int sidx = g.sbase(m) + i;
            T J[DS];
            f.template finish<DSL>(acc, Y[sidx_ok(sidx)], J);
#pragma unroll
            for (int mu = DSL; mu < DS; ++mu) J[mu] = f.zero();     // components beyond a 4d range
            IO::template store<DS>(jvec(m, i), J);
            Sr[sidx_ok(sidx)] = f.c_to_t(sa);
        } else {
            // a5: contract the top bracket with the last polarisation
            if constexpr (F::kIsFp) result = f.template amplitude_raw<DSL, METRIC>(acc, eL);
            else result = f.template amplitude<DSL, METRIC>(acc, eL);
        }
    };
#pragma unroll 1
    // Ranges by right end j, and for each j from the shortest [j-1, j] to the
    // longest [0, j]: every sub-range is finished before it is read, and
    // consecutive ranges share their suffix currents [s+1, j] (better L1 reuse
    // than ordering by length; measured 1-3 % at n = 8).
    for (int jj = 1; jj < N; ++jj) {
#pragma unroll 1
        for (int i = jj - 1; i >= 0; --i) {
            const int m = jj - i + 1;
            if constexpr (MIXED && DS > 4) {
                const uint32_t legs = ((1u << m) - 1u) << i;
                if ((a.four_d_legs & legs) == legs) {
                    range(std::integral_constant<int, 4>{}, std::integral_constant<int, 4>{}, m, i);
                    continue;
                }
            }
            range(std::integral_constant<int, D>{}, std::integral_constant<int, DS>{}, m, i);
        }
    }
    st_once(out + u, (singular || violated) ? f.zero_io() : result);
    if (a.status != nullptr && h == 0) a.status[e] = violated ? 2 : singular ? 1 : 0;
}

// bg_point with the whole table at `tab` (one region, as in the batch kernel).
template <class F, int D, int DS, int METRIC, int BLOCK>
__device__ __forceinline__ void bg_point(const F& f, const CompactArgs& a, typename F::T* tab, int64_t u) {
    bg_point<F, D, DS, METRIC, BLOCK>(f, a, tab, tab + Geometry{a.n - 1}.off_k(DS) * BLOCK, u);
}

// Dead table lines out of L2.  A point's table in global scratch is dead once
// the point is done: the next point of the same thread writes every slot
// before it reads it.  Without help L2 writes those dirty lines back to DRAM
// when it evicts them (at n = 8, d = 6 about three times the algorithmic
// bytes of a launch); discard.global.L2 drops them instead.  The warp's part
// of every table row is whole 128-byte lines that no other warp touches (rows
// of 32 x K x 4 bytes in the F_p layout, of 32 x element bytes in the complex
// one; every region starts on a multiple of 128 bytes), so once all 32 lanes
// are past the point each lane drops a share of the lines.  A partial warp (the
// last points of the grid) keeps its lines: dropping them is only a saving.
// Measured on GB300, n = 8, d = 6, 2^19 points: DRAM bytes 696 -> 413 MB per
// launch (algorithmic 204 MB), time within 1 %.

// Drops `rows` rows of PER_ROW lines each (row r at base + r * row_stride):
// line l = lane + 32 k of the warp's share goes to this lane, its address
// advanced by additions only.
template <int PER_ROW>
__device__ __forceinline__ void discard_rows(const void* base, int rows, int row_stride, int lane) {
    static_assert(PER_ROW >= 1 && PER_ROW <= 32, "lines per row");
    constexpr int DR = 32 / PER_ROW, DC = 32 % PER_ROW;
    const int lines = rows * PER_ROW;
    int c = lane % PER_ROW;
    const char* q = static_cast<const char*>(base) + static_cast<size_t>(lane / PER_ROW) * row_stride + (c << 7);
    const int step = DR * row_stride + (DC << 7), wrap = row_stride - (PER_ROW << 7);
    for (int l = lane; l < lines; l += 32) {
        asm volatile("discard.global.L2 [%0], 128;" ::"l"(q) : "memory");
        q += step;
        c += DC;
        if (c >= PER_ROW) {
            c -= PER_ROW;
            q += wrap;
        }
    }
}

template <class F, int D, int DS, int BLOCK, bool AUX>
__device__ __forceinline__ void discard_point_table_body(const Geometry& g, const typename F::T* tab,
                                                         const typename F::T* aux) {
    using T = typename F::T;
    using TK = typename F::TK;
    // every entry point hands the kernels 256-byte aligned scratch; a table
    // that is not 128-byte aligned is never discarded (the lines would not
    // be the warp's own)
    if (__activemask() != 0xffffffffu || (reinterpret_cast<uintptr_t>(tab) & 127u) != 0) return;
    __syncwarp();                                   // every lane is done with the point
    // opaque to the compiler, so that the line addresses are formed here and
    // not hoisted out of the point loop into registers held across the points
    asm volatile("" : "+l"(tab), "+l"(aux));
    const int lane = threadIdx.x & 31, w0 = threadIdx.x & ~31;
    constexpr int ES = sizeof(T), KS = sizeof(TK);
    const T* sa = aux + (g.off_sa(D, DS) - g.off_k(DS)) * BLOCK + w0;     // SA and 1/P^2, 2 ns rows
    if constexpr (F::kIsFp) {                       // [slot][thread][K]: a row is the warp's whole slot
        discard_rows<DS * ES / 4>(tab + w0 * DS, g.nj(), BLOCK * DS * ES, lane);
        if constexpr (AUX) {
            discard_rows<D * KS / 4>(reinterpret_cast<const TK*>(aux) + w0 * D, g.N + 1, BLOCK * D * KS, lane);
            discard_rows<ES / 4>(sa, 2 * g.ns(), BLOCK * ES, lane);
        }
    } else {                                        // [slot][K][thread]: a row is one component
        discard_rows<ES / 4>(tab + w0, g.nj() * DS, BLOCK * ES, lane);
        if constexpr (AUX) {
            discard_rows<KS / 4>(reinterpret_cast<const TK*>(aux) + w0, (g.N + 1) * D, BLOCK * KS, lane);
            discard_rows<ES / 4>(sa, 2 * g.ns(), BLOCK * ES, lane);
        }
    }
    __syncwarp();                                   // before any lane writes the next point's table
}

// The same as a function of its own (not inlined).  Which of the two keeps
// the point loop faster depends on the kernel's register pressure (measured on
// GB300, F_p): inlined, the D = D_s = 6 kernel ran 3-5 % slower at n = 8..12;
// called, the D_s = 8 kernel ran 2-8 % slower (n = 6..12), and inlined it ran
// as fast as without any discard.  The complex kernels measured the same
// either way and call it.
template <class F, int D, int DS, int BLOCK, bool AUX>
__device__ __noinline__ void discard_point_table_call(const Geometry g, const typename F::T* tab,
                                                      const typename F::T* aux) {
    discard_point_table_body<F, D, DS, BLOCK, AUX>(g, tab, aux);
}

template <class F, int D, int DS, int BLOCK, bool AUX>
__device__ __forceinline__ void discard_point_table(const Geometry& g, const typename F::T* tab,
                                                    const typename F::T* aux) {
    if constexpr (F::kIsFp && DS == 8) discard_point_table_body<F, D, DS, BLOCK, AUX>(g, tab, aux);
    else discard_point_table_call<F, D, DS, BLOCK, AUX>(g, tab, aux);
}

template <class F, int D, int DS, int METRIC, int BLOCK, int PLACE, bool MIXED>
__device__ __forceinline__ void compact_body(const F& f, const CompactArgs& a) {
    using T = typename F::T;
    extern __shared__ __align__(16) unsigned char bg_smem[];
    const Geometry g{a.n - 1};
    T* tab;                                   // this block's currents
    T* aux;                                   // its prefix sums, SA, 1/P^2
    if constexpr (PLACE == kPlaceGlobal) {
        tab = reinterpret_cast<T*>(a.ws) + static_cast<size_t>(blockIdx.x) * g.words(D, DS) * BLOCK;
        aux = tab + g.off_k(DS) * BLOCK;
    } else if constexpr (PLACE == kPlaceSplit) {
        tab = reinterpret_cast<T*>(a.ws) + static_cast<size_t>(blockIdx.x) * g.cur_words(DS) * BLOCK;
        aux = reinterpret_cast<T*>(bg_smem);
    } else {
        tab = reinterpret_cast<T*>(bg_smem);
        aux = tab + g.off_k(DS) * BLOCK;
    }
    const int64_t total = a.E * a.H;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * BLOCK;
    for (int64_t u = static_cast<int64_t>(blockIdx.x) * BLOCK + threadIdx.x; u < total; u += stride) {
        bg_point<F, D, DS, METRIC, BLOCK, MIXED>(f, a, tab, aux, u);
        if constexpr (PLACE != kPlaceShared) discard_point_table<F, D, DS, BLOCK, PLACE == kPlaceGlobal>(g, tab, aux);
    }
}

template <class F, int D, int DS, int METRIC, int BLOCK, int PLACE, bool MIXED = false>
__global__ void __launch_bounds__(BLOCK)
bg_compact_kernel(const F f, const CompactArgs a) {
    compact_body<F, D, DS, METRIC, BLOCK, PLACE, MIXED>(f, a);
}

}  // namespace bgk
