// bg_c64.cuh -- complex FP64 arithmetic for the recursion kernel.
//
// The paper evaluates the recursion over complex double as well as F_p
// (Sec. 3).  Every complex multiply-accumulate is four fused multiply-adds on
// the FP64 pipe; metric signs fold into the sign of an FMA operand, so dots
// cost exactly 4 FMAs per component.  The propagator inverse is
// conj(z) / |z|^2 with a correctly rounded FP64 reciprocal.
#pragma once
#include <cstdint>
#include "bg_fp.cuh"   // metric_sign

namespace bgk {

struct FieldC64 {
    using T = double2;
    using io_t = double2;
    static constexpr bool kIsFp = false;

    __device__ __forceinline__ T zero() const { return make_double2(0.0, 0.0); }
    __device__ __forceinline__ T mul(T a, T b) const {
        return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
    }
    __device__ __forceinline__ T add(T a, T b) const { return make_double2(a.x + b.x, a.y + b.y); }
    __device__ __forceinline__ T sub(T a, T b) const { return make_double2(a.x - b.x, a.y - b.y); }
    __device__ __forceinline__ T neg(T a) const { return make_double2(-a.x, -a.y); }
    __device__ __forceinline__ T dbl(T a) const { return make_double2(a.x + a.x, a.y + a.y); }
    __device__ __forceinline__ T from_io(io_t x) const { return x; }
    __device__ __forceinline__ io_t to_io(T x) const { return x; }

    template <int D, int METRIC>
    __device__ __forceinline__ T dot(const T* a, const T* b) const {
        double re = 0.0, im = 0.0;
#pragma unroll
        for (int mu = 0; mu < D; ++mu) {
            const double s = static_cast<double>(metric_sign<METRIC>(mu));
            const double ax = s * a[mu].x, ay = s * a[mu].y;   // exact sign flip
            re = fma(ax, b[mu].x, re);
            re = fma(-ay, b[mu].y, re);
            im = fma(ax, b[mu].y, im);
            im = fma(ay, b[mu].x, im);
        }
        return make_double2(re, im);
    }

    template <int D>
    __device__ __forceinline__ void axpy(T* acc, T c, const T* v) const {
#pragma unroll
        for (int mu = 0; mu < D; ++mu) {
            acc[mu].x = fma(c.x, v[mu].x, acc[mu].x);
            acc[mu].x = fma(-c.y, v[mu].y, acc[mu].x);
            acc[mu].y = fma(c.x, v[mu].y, acc[mu].y);
            acc[mu].y = fma(c.y, v[mu].x, acc[mu].y);
        }
    }

    __device__ __forceinline__ T inv(T z) const {
        const double w = fma(z.x, z.x, z.y * z.y);
        const double r = __drcp_rn(w);
        return make_double2(z.x * r, -z.y * r);
    }
    __device__ __forceinline__ bool is_zero(T z) const { return z.x == 0.0 && z.y == 0.0; }
};

}  // namespace bgk
