// bg_fp.cuh -- F_p arithmetic for the recursion kernel (device side).
//
// The paper works over F_p with p < 2^31, reducing every intermediate modulo
// p and dividing through an inverse (Sec. 3).  Here residues live in
// Montgomery form x*R mod p with R = 2^32, fully reduced to [0, p).
//
//   redc(t)   = t * R^-1 mod p, in [0, 2p), for t < p * 2^32.  Two integer-
//               multiply instructions: m = lo(t) * (-p^-1) and the 32x32+64
//               multiply-add m*p + t, whose high word is the result (no
//               carry can be lost: t + m*p < 2 p 2^32 < 2^64 for p < 2^31).
//   mul(a, b) = redc(a*b) folded to [0, p).
//
// Products of two reduced residues are < p^2, and the sum of two such
// products is < 2 p^2 < p * 2^32 (as 2p < 2^32), so dot products reduce once
// per PAIR of products.  Signs of the metric are handled by grouping terms of
// equal sign.  Constants are computed on the host (bg_api.cu) per plan.
#pragma once
#include <cstdint>

namespace bgk {

template <int METRIC>
__host__ __device__ constexpr int metric_sign(int mu) {
    // 0: mostly minus (Sec. 2.3); 1: alternating diag(+,-,+,-,...) (Sec. 3.1)
    return METRIC == 0 ? (mu == 0 ? 1 : -1) : ((mu & 1) ? -1 : 1);
}

struct FieldFp {
    using T = uint32_t;       // Montgomery residue in [0, p)
    using io_t = uint32_t;    // canonical residue at the boundary
    static constexpr bool kIsFp = true;

    uint32_t p;       // the prime, odd, < 2^31
    uint32_t pinv;    // -p^-1 mod 2^32
    uint32_t r2;      // R^2 mod p      (canonical -> Montgomery)
    uint32_t one;     // R mod p        (Montgomery form of 1)
    uint32_t pm2;     // p - 2          (Fermat exponent)

    __device__ __forceinline__ uint32_t redc(uint64_t t) const {
        const uint32_t m = static_cast<uint32_t>(t) * pinv;
        return static_cast<uint32_t>((static_cast<uint64_t>(m) * p + t) >> 32);
    }
    __device__ __forceinline__ uint32_t fold(uint32_t x) const {   // [0,2p) -> [0,p)
        return min(x, x - p);
    }
    __device__ __forceinline__ T zero() const { return 0u; }
    __device__ __forceinline__ T mul(T a, T b) const {
        return fold(redc(static_cast<uint64_t>(a) * b));
    }
    __device__ __forceinline__ T add(T a, T b) const { return fold(a + b); }
    __device__ __forceinline__ T sub(T a, T b) const {
        const uint32_t d = a - b;
        return min(d, d + p);
    }
    __device__ __forceinline__ T neg(T a) const { return fold(p - a); }
    __device__ __forceinline__ T dbl(T a) const { return add(a, a); }

    __device__ __forceinline__ T from_io(io_t x) const { return mul(x, r2); }
    __device__ __forceinline__ io_t to_io(T x) const { return fold(redc(x)); }

    // sum_{mu < D} eta_mu a_mu b_mu; pairs of equal-sign products share one redc.
    template <int D, int METRIC>
    __device__ __forceinline__ T dot(const T* a, const T* b) const {
        uint64_t tp = 0, tn = 0;
        int cp = 0, cn = 0;
        T pos = 0, neg_ = 0;
        bool hp = false, hn = false;
#pragma unroll
        for (int mu = 0; mu < D; ++mu) {
            const uint64_t prod = static_cast<uint64_t>(a[mu]) * b[mu];
            if (metric_sign<METRIC>(mu) > 0) {
                tp += prod;
                if (++cp == 2) {
                    const T r = fold(redc(tp));
                    pos = hp ? add(pos, r) : r;
                    hp = true; tp = 0; cp = 0;
                }
            } else {
                tn += prod;
                if (++cn == 2) {
                    const T r = fold(redc(tn));
                    neg_ = hn ? add(neg_, r) : r;
                    hn = true; tn = 0; cn = 0;
                }
            }
        }
        if (cp) { const T r = fold(redc(tp)); pos = hp ? add(pos, r) : r; hp = true; }
        if (cn) { const T r = fold(redc(tn)); neg_ = hn ? add(neg_, r) : r; hn = true; }
        if (!hn) return pos;
        if (!hp) return neg(neg_);
        return sub(pos, neg_);
    }

    // acc[mu] += c * v[mu] for mu < D
    template <int D>
    __device__ __forceinline__ void axpy(T* acc, T c, const T* v) const {
#pragma unroll
        for (int mu = 0; mu < D; ++mu) acc[mu] = add(acc[mu], mul(c, v[mu]));
    }

    // x^(p-2) = x^-1 (x != 0), 0 -> 0; square-and-multiply on the bits of p-2
    // (uniform across the warp: every thread has the same exponent).
    __device__ __forceinline__ T inv(T x) const {
        T r = one;
#pragma unroll 1
        for (int bit = 30; bit >= 0; --bit) {
            r = mul(r, r);
            if ((pm2 >> bit) & 1u) r = mul(r, x);
        }
        return r;
    }
    __device__ __forceinline__ bool is_zero(T x) const { return x == 0u; }
};

}  // namespace bgk
