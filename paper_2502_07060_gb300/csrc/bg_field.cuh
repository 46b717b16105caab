// bg_field.cuh -- arithmetic policies of the compact recursion kernel.
//
// Both policies expose the same operations so that bg_compact.cuh is written
// once:
//   T   stored element (table entries: currents, momenta, SA, 1/P^2)
//   C   coefficient (result of a dot product, scalar arithmetic)
//   A   accumulator element of R(i,j)
//   dot<D, METRIC>(a, b)          metric dot over D components -> C
//   cadd / csub / cdbl / cneg     coefficient arithmetic
//   acc1<K>(acc, c, v)            acc[0..K) += c v
//   acc2<K>(acc, c1, v1, c2, v2)  acc[0..K) += c1 v1 + c2 v2
//   finish(acc, inv) -> T[]       J = R / P^2 from the accumulator
//   amplitude(acc, eps_last)      A = eps_n . R_top
//   TK, kdot / kkdot / kacc1 / kacc2: the same for momentum components
//                                 (field elements, complex, or real doubles
//                                 for physical points in C64ROps)
//
// F_p (Sec. 3: p < 2^31, every intermediate reduced mod p).  Montgomery
// representation with R = 2^32; a value "at level L" is x R^L mod p.
//   * stored table entries are at level 1 and fully reduced (< p);
//   * redc(t) = t R^-1 mod p in [0, 2p) for t < p 2^32: one 32-bit multiply
//     (m = lo(t) (-p^-1)) and one 32x32+64 multiply-add whose high word is
//     the result; redc_full(t) = t R^-1 mod p for any t < 2^64, as the 33-bit
//     sum hi(t) + hi(m p + lo(t));
//   * a product of two reduced values is < p^2 < 2^62, so FOUR products fit
//     in 64 bits without reduction;
//   * a dot product of up to four products (< 2^64) applies redc_full and
//     redc; of five to eight, adds two 64-bit sums of four into a 96-bit
//     value and applies reduce96 (the same two Montgomery steps): the
//     coefficient is at level 0, in [0, p];
//   * R(i,j) accumulates the unreduced products (level 0 coefficient) x
//     (level 1 entry) -- level-1 integers below 2^62 -- in a 96-bit
//     accumulator (64-bit sums of up to four products are added with one
//     carry chain); finish() reduces the 96-bit sum twice (level -1) and
//     multiplies by 1/P^2 stored at level 3, giving level 1.  Measured on
//     GB300: the 64-bit multiply-add runs at half the rate of the 32-bit one,
//     and this accumulation sustains 27 field multiplications per SM per
//     clock against 15.6 when every pair of products is reduced;
//   * metric signs: terms with eta = -1 are summed as products with the
//     negated operand (p - a), so every sum is a plain sum.
// C64 (Sec. 3, complex double): FMA-based complex arithmetic; dot products and
// accumulations are 4 FP64 FMAs per complex term; the metric sign becomes the
// sign of an FMA operand.  C64ROps: real momenta, 2 FMAs per momentum term.
#pragma once
#include <cstdint>

namespace bgk {

template <int METRIC>
__host__ __device__ constexpr int msign(int mu) {
    return METRIC == 0 ? (mu == 0 ? 1 : -1) : ((mu & 1) ? -1 : 1);
}

// 96-bit accumulator of the F_p recursion: lo + 2^64 hi
struct Acc96 {
    uint64_t lo;
    uint32_t hi;
};

__device__ __forceinline__ void add96(Acc96& a, uint64_t t) {
    asm("{\n\t.reg .u32 a0, a1, t0, t1;\n\t"
        "mov.b64 {a0, a1}, %0;\n\tmov.b64 {t0, t1}, %2;\n\t"
        "add.cc.u32 a0, a0, t0;\n\taddc.cc.u32 a1, a1, t1;\n\taddc.u32 %1, %1, 0;\n\t"
        "mov.b64 %0, {a0, a1};\n\t}"
        : "+l"(a.lo), "+r"(a.hi)
        : "l"(t));
}

struct FpOps {
    using T = uint32_t;
    using C = uint32_t;
    using A = Acc96;
    using io_t = uint32_t;
    using TK = uint32_t;            // momentum component
    using kio_t = uint32_t;         // momentum input element
    static constexpr bool kIsFp = true;
    static constexpr int kField = 1;

    uint32_t p, pinv, r2, r3, one, pm2;   // r2 = R^2, r3 = R^3, one = R (mod p)
    uint32_t rn3;                          // R^(n+3) mod p for the plan's n (amplitude_raw)

    __device__ __forceinline__ uint32_t redc(uint64_t t) const {
        const uint32_t m = static_cast<uint32_t>(t) * pinv;
        return static_cast<uint32_t>((static_cast<uint64_t>(m) * p + t) >> 32);
    }
    // t R^-1 mod p for any t < 2^64, in [0, 2^32 + p): t + m p = 0 mod 2^32,
    // so (t + m p) / 2^32 = hi(t) + hi(m p + lo(t)) exactly
    __device__ __forceinline__ uint64_t redc_full(uint64_t t) const {
        const uint32_t lo = static_cast<uint32_t>(t);
        const uint32_t m = lo * pinv;
        return (t >> 32) + ((static_cast<uint64_t>(m) * p + lo) >> 32);
    }
    __device__ __forceinline__ uint32_t fold(uint32_t x) const { return min(x, x - p); }
    // full Montgomery product of reduced operands, level la + lb - 1, in [0, p)
    __device__ __forceinline__ uint32_t mmul(uint32_t a, uint32_t b) const {
        return fold(redc(static_cast<uint64_t>(a) * b));
    }
    __device__ __forceinline__ uint32_t madd(uint32_t a, uint32_t b) const { return fold(a + b); }
    __device__ __forceinline__ uint32_t msub(uint32_t a, uint32_t b) const {
        const uint32_t d = a - b;
        return min(d, d + p);
    }

    __device__ __forceinline__ T zero() const { return 0u; }
    __device__ __forceinline__ T from_io(io_t x) const { return mmul(x, r2); }      // level 1
    __device__ __forceinline__ T tadd(T a, T b) const { return madd(a, b); }
    __device__ __forceinline__ T tsub(T a, T b) const { return msub(a, b); }

    // sum_mu eta_mu a_mu b_mu -> level 0, in [0, p].  All terms of the sign
    // that occurs most often are summed directly; the others use p - a.
    // Up to four products (< 4 p^2 < 2^64): one 64-bit sum, redc_full and
    // redc.  Five to eight: two 64-bit sums of four added into a 96-bit value
    // (hi <= 1) and reduced twice by reduce96 -- one reduction fewer than
    // reducing each group (measured 3 % on the n=8, d=6 kernel).
    template <int D, int METRIC>
    __device__ __forceinline__ C dot(const T* a, const T* b) const {
        constexpr int nneg = []() { int c = 0; for (int mu = 0; mu < D; ++mu) c += msign<METRIC>(mu) < 0; return c; }();
        constexpr int flip = (nneg * 2 > D) ? -1 : 1;   // sign that is NOT negated
        static_assert(D <= 8, "two groups of four products at most");
        // products summed as a tree (pairs, then pairs of pairs): the sums are
        // exact, and the dependency chain is two additions deep instead of
        // four multiply-adds (measured 0.5 % on the n=8, d=6 kernel, the same
        // time as two chains of four at d=8)
        uint64_t pr[8];
#pragma unroll
        for (int mu = 0; mu < D; ++mu) {
            const uint32_t x = (msign<METRIC>(mu) == flip) ? a[mu] : (p - a[mu]);
            pr[mu] = static_cast<uint64_t>(x) * b[mu];
        }
#pragma unroll
        for (int mu = D; mu < 8; ++mu) pr[mu] = 0;
        const uint64_t s0 = (pr[0] + pr[1]) + (pr[2] + pr[3]);
        const uint64_t s1 = (pr[4] + pr[5]) + (pr[6] + pr[7]);
        uint32_t r;
        if constexpr (D <= 4) {
            r = fold(redc(redc_full(s0)));             // flip * dot, level 0, [0, p)
        } else {
            A acc{s0, 0u};
            add96(acc, s1);
            r = fold(reduce96(acc));
        }
        return flip > 0 ? r : p - r;               // [0, p]
    }
    __device__ __forceinline__ C cadd(C a, C b) const { return madd(a, b); }        // [0, p)
    __device__ __forceinline__ C csub(C a, C b) const { return msub(a, b); }        // [0, p]
    __device__ __forceinline__ C cdbl(C a) const { return fold(a + a); }            // a <= p -> [0, p]
    __device__ __forceinline__ C cneg(C a) const { return p - a; }                  // [0, p]
    __device__ __forceinline__ C czero() const { return 0u; }
    __device__ __forceinline__ T c_to_t(C a) const { return fold(a); }              // stored SA
    __device__ __forceinline__ C t_to_c(T a) const { return a; }

    template <int K>
    __device__ __forceinline__ void acc_zero(A* acc) const {
#pragma unroll
        for (int mu = 0; mu < K; ++mu) {
            acc[mu].lo = 0;
            acc[mu].hi = 0;
        }
    }
    // c <= p and v < p: every product is below 2^62
    template <int K>
    __device__ __forceinline__ void acc1(A* acc, C c, const T* v) const {
#pragma unroll
        for (int mu = 0; mu < K; ++mu) add96(acc[mu], static_cast<uint64_t>(c) * v[mu]);
    }
    template <int K>
    __device__ __forceinline__ void acc2(A* acc, C c1, const T* v1, C c2, const T* v2) const {
#pragma unroll
        for (int mu = 0; mu < K; ++mu)
            add96(acc[mu], static_cast<uint64_t>(c1) * v1[mu] + static_cast<uint64_t>(c2) * v2[mu]);
    }
    // 96-bit sum -> divided by R^2 (two Montgomery steps), in [0, 2p): redc_full of
    // the low word shifts the sum down by 2^32 (it stays far below p 2^32:
    // a range sums fewer than 2^8 products, a contraction eight), then one redc
    __device__ __forceinline__ uint32_t reduce96(const A& a) const {
        const uint32_t lo = static_cast<uint32_t>(a.lo);
        const uint32_t m = lo * pinv;
        const uint64_t shifted = ((static_cast<uint64_t>(a.hi) << 32) | (a.lo >> 32)) +
                                 ((static_cast<uint64_t>(m) * p + lo) >> 32);
        return redc(shifted);
    }
    // J = R / P^2: reduce96(acc) is level -1; times 1/P^2 at level 3 -> level 1.
    template <int K>
    __device__ __forceinline__ void finish(const A* acc, T inv3, T* out) const {
#pragma unroll
        for (int mu = 0; mu < K; ++mu) out[mu] = mmul(reduce96(acc[mu]), inv3);
    }
    template <int K, int METRIC>
    __device__ __forceinline__ io_t amplitude(const A* acc, const T* eps_last) const {
        T r[K];
#pragma unroll
        for (int mu = 0; mu < K; ++mu) r[mu] = mmul(reduce96(acc[mu]), r3);   // level 1
        const C a = dot<K, METRIC>(eps_last, r);                               // level 0 = canonical
        return a == p ? 0u : a;
    }
    // The same contraction when the states were taken as canonical residues
    // (level 0) instead of level 1: every current is multilinear in the
    // states of its legs, so a current of length m then sits at level 1 - m
    // (one level lower per state, uniformly in all its terms), R_top at
    // level 2 - n.  reduce96 gives level -n, times R^(n+3) level 2, and the
    // contraction with the level-0 last state level 0 = canonical.
    template <int K, int METRIC>
    __device__ __forceinline__ io_t amplitude_raw(const A* acc, const T* eps_last) const {
        T r[K];
#pragma unroll
        for (int mu = 0; mu < K; ++mu) r[mu] = mmul(reduce96(acc[mu]), rn3);
        const C a = dot<K, METRIC>(eps_last, r);
        return a == p ? 0u : a;
    }
    // P^2 (level 0 coefficient) -> level 1 input of the batched inverse
    __device__ __forceinline__ T inv_input(C p2) const { return mmul(fold(p2), r2); }
    __device__ __forceinline__ T inv_mul(T a, T b) const { return mmul(a, b); }
    __device__ __forceinline__ T inv_scalar(T x) const {     // x^(p-2), level 1 in and out
        T r = one;
#pragma unroll 1
        for (int bit = 30; bit >= 0; --bit) {
            r = mmul(r, r);
            if ((pm2 >> bit) & 1u) r = mmul(r, x);
        }
        return r;
    }
    __device__ __forceinline__ T inv_store(T inv1) const { return mmul(inv1, r3); }   // level 3

    // momentum operations: momenta are field elements like the currents
    __device__ __forceinline__ TK kzero() const { return 0u; }
    __device__ __forceinline__ TK kfrom_io(kio_t x) const { return from_io(x); }
    __device__ __forceinline__ TK kadd(TK a, TK b) const { return tadd(a, b); }
    __device__ __forceinline__ TK ksub(TK a, TK b) const { return tsub(a, b); }
    template <int D, int METRIC>
    __device__ __forceinline__ C kdot(const TK* a, const T* b) const { return dot<D, METRIC>(a, b); }
    template <int D, int METRIC>
    __device__ __forceinline__ C kkdot(const TK* a, const TK* b) const { return dot<D, METRIC>(a, b); }
    template <int K>
    __device__ __forceinline__ void kacc1(A* acc, C c, const TK* v) const { acc1<K>(acc, c, v); }
    template <int K>
    __device__ __forceinline__ void kacc2(A* acc, C c1, const TK* v1, C c2, const TK* v2) const {
        acc2<K>(acc, c1, v1, c2, v2);
    }
    __device__ __forceinline__ bool is_zero(T x) const { return x == 0u; }
    __device__ __forceinline__ io_t zero_io() const { return 0u; }
};

struct C64Ops {
    using T = double2;
    using C = double2;
    using A = double2;
    using io_t = double2;
    using TK = double2;
    using kio_t = double2;
    static constexpr bool kIsFp = false;
    static constexpr int kField = 0;

    __device__ __forceinline__ T zero() const { return make_double2(0.0, 0.0); }
    __device__ __forceinline__ T from_io(io_t x) const { return x; }
    __device__ __forceinline__ T tadd(T a, T b) const { return make_double2(a.x + b.x, a.y + b.y); }
    __device__ __forceinline__ T tsub(T a, T b) const { return make_double2(a.x - b.x, a.y - b.y); }

    template <int D, int METRIC>
    __device__ __forceinline__ C dot(const T* a, const T* b) const {
        double re = 0.0, im = 0.0;
#pragma unroll
        for (int mu = 0; mu < D; ++mu) {
            if (msign<METRIC>(mu) > 0) {
                re = fma(a[mu].x, b[mu].x, re);
                re = fma(-a[mu].y, b[mu].y, re);
                im = fma(a[mu].x, b[mu].y, im);
                im = fma(a[mu].y, b[mu].x, im);
            } else {
                re = fma(-a[mu].x, b[mu].x, re);
                re = fma(a[mu].y, b[mu].y, re);
                im = fma(-a[mu].x, b[mu].y, im);
                im = fma(-a[mu].y, b[mu].x, im);
            }
        }
        return make_double2(re, im);
    }
    __device__ __forceinline__ C cadd(C a, C b) const { return make_double2(a.x + b.x, a.y + b.y); }
    __device__ __forceinline__ C csub(C a, C b) const { return make_double2(a.x - b.x, a.y - b.y); }
    __device__ __forceinline__ C cdbl(C a) const { return make_double2(a.x + a.x, a.y + a.y); }
    __device__ __forceinline__ C cneg(C a) const { return make_double2(-a.x, -a.y); }
    __device__ __forceinline__ C czero() const { return make_double2(0.0, 0.0); }
    __device__ __forceinline__ T c_to_t(C a) const { return a; }
    __device__ __forceinline__ C t_to_c(T a) const { return a; }

    template <int K>
    __device__ __forceinline__ void acc_zero(A* acc) const {
#pragma unroll
        for (int mu = 0; mu < K; ++mu) acc[mu] = make_double2(0.0, 0.0);
    }
    template <int K>
    __device__ __forceinline__ void acc1(A* acc, C c, const T* v) const {
#pragma unroll
        for (int mu = 0; mu < K; ++mu) {
            acc[mu].x = fma(c.x, v[mu].x, acc[mu].x);
            acc[mu].x = fma(-c.y, v[mu].y, acc[mu].x);
            acc[mu].y = fma(c.x, v[mu].y, acc[mu].y);
            acc[mu].y = fma(c.y, v[mu].x, acc[mu].y);
        }
    }
    template <int K>
    __device__ __forceinline__ void acc2(A* acc, C c1, const T* v1, C c2, const T* v2) const {
        acc1<K>(acc, c1, v1);
        acc1<K>(acc, c2, v2);
    }
    template <int K>
    __device__ __forceinline__ void finish(const A* acc, T inv, T* out) const {
#pragma unroll
        for (int mu = 0; mu < K; ++mu)
            out[mu] = make_double2(fma(acc[mu].x, inv.x, -acc[mu].y * inv.y),
                                   fma(acc[mu].x, inv.y, acc[mu].y * inv.x));
    }
    template <int K, int METRIC>
    __device__ __forceinline__ io_t amplitude(const A* acc, const T* eps_last) const {
        return dot<K, METRIC>(eps_last, acc);
    }
    __device__ __forceinline__ T inv_input(C p2) const { return p2; }
    __device__ __forceinline__ T inv_mul(T a, T b) const { return a; }   // unused
    __device__ __forceinline__ T inv_scalar(T z) const {                  // 1/z = conj(z)/|z|^2
        const double w = fma(z.x, z.x, z.y * z.y);
        const double r = __drcp_rn(w);
        return make_double2(z.x * r, -z.y * r);
    }
    __device__ __forceinline__ T inv_store(T v) const { return v; }
    __device__ __forceinline__ bool is_zero(T z) const { return z.x == 0.0 && z.y == 0.0; }
    __device__ __forceinline__ io_t zero_io() const { return make_double2(0.0, 0.0); }

    // complex momenta
    __device__ __forceinline__ TK kzero() const { return zero(); }
    __device__ __forceinline__ TK kfrom_io(kio_t x) const { return x; }
    __device__ __forceinline__ TK kadd(TK a, TK b) const { return tadd(a, b); }
    __device__ __forceinline__ TK ksub(TK a, TK b) const { return tsub(a, b); }
    template <int D, int METRIC>
    __device__ __forceinline__ C kdot(const TK* a, const T* b) const { return dot<D, METRIC>(a, b); }
    template <int D, int METRIC>
    __device__ __forceinline__ C kkdot(const TK* a, const TK* b) const { return dot<D, METRIC>(a, b); }
    template <int K>
    __device__ __forceinline__ void kacc1(A* acc, C c, const TK* v) const { acc1<K>(acc, c, v); }
    template <int K>
    __device__ __forceinline__ void kacc2(A* acc, C c1, const TK* v1, C c2, const TK* v2) const {
        acc2<K>(acc, c1, v1, c2, v2);
    }
};

// Complex FP64 with real momenta (physical phase-space points, Sec. 3): the
// currents and polarisations stay complex, momenta are real doubles.  A
// momentum-current contraction is then two FMAs per component (real times
// complex) instead of four, P^2 is real and so is its inverse, and the
// momentum term of the three-gluon vertex accumulates with two FMAs per
// component.
struct C64ROps : C64Ops {
    using TK = double;
    using kio_t = double;
    static constexpr int kField = 2;

    __device__ __forceinline__ TK kzero() const { return 0.0; }
    __device__ __forceinline__ TK kfrom_io(kio_t x) const { return x; }
    __device__ __forceinline__ TK kadd(TK a, TK b) const { return a + b; }
    __device__ __forceinline__ TK ksub(TK a, TK b) const { return a - b; }
    template <int D, int METRIC>
    __device__ __forceinline__ C kdot(const TK* a, const T* b) const {
        double re = 0.0, im = 0.0;
#pragma unroll
        for (int mu = 0; mu < D; ++mu) {
            const double s = msign<METRIC>(mu) > 0 ? a[mu] : -a[mu];
            re = fma(s, b[mu].x, re);
            im = fma(s, b[mu].y, im);
        }
        return make_double2(re, im);
    }
    template <int D, int METRIC>
    __device__ __forceinline__ C kkdot(const TK* a, const TK* b) const {
        double re = 0.0;
#pragma unroll
        for (int mu = 0; mu < D; ++mu) re = fma(msign<METRIC>(mu) > 0 ? a[mu] : -a[mu], b[mu], re);
        return make_double2(re, 0.0);
    }
    template <int K>
    __device__ __forceinline__ void kacc1(A* acc, C c, const TK* v) const {
#pragma unroll
        for (int mu = 0; mu < K; ++mu) {
            acc[mu].x = fma(c.x, v[mu], acc[mu].x);
            acc[mu].y = fma(c.y, v[mu], acc[mu].y);
        }
    }
    template <int K>
    __device__ __forceinline__ void kacc2(A* acc, C c1, const TK* v1, C c2, const TK* v2) const {
        kacc1<K>(acc, c1, v1);
        kacc1<K>(acc, c2, v2);
    }
    // P^2 is real: its inverse is the correctly rounded reciprocal, and the
    // current is R scaled by it
    __device__ __forceinline__ T inv_scalar(T z) const { return make_double2(__drcp_rn(z.x), 0.0); }
    template <int K>
    __device__ __forceinline__ void finish(const A* acc, T inv, T* out) const {
#pragma unroll
        for (int mu = 0; mu < K; ++mu) out[mu] = make_double2(acc[mu].x * inv.x, acc[mu].y * inv.x);
    }
};

}  // namespace bgk
