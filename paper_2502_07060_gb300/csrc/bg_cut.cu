// bg_cut.cu -- bg_cut_trace: the state sum over a ring of tree amplitudes.
//
// A one-loop cut joins k tree amplitudes in a ring by k internal legs; its
// leading pole is the sum over the internal states of the product of the
// trees (Sec. 2.1), with the states of Sec. 2.3 on one side of each internal
// leg and their duals (the tilde states) on the other.  When tree i is
// evaluated by a product plan whose only legs with several states are its
// incoming internal leg (leg 0) and its outgoing one (leg n-1), its output
// row [E][S * S] is the matrix M_i[e][s_out][s_in], and the state sum is
//     sum_{s_1..s_k} prod_i M_i[e][s_{i+1}][s_i]  (s_{k+1} = s_1)
//     = trace(M_k ... M_2 M_1).
// One thread per point: the running product stays in registers, and each
// block stages its points' matrices in shared memory with coalesced loads.
#include <cuda_runtime.h>

#include "bg_internal.h"

namespace {

constexpr int kCutStageBytes = 32768;      // shared staging per block
constexpr int kCutMaxS = 8;
constexpr int kCutMaxK = 16;

struct CutArgs {
    int64_t E;
    int k;
    const void* M[kCutMaxK];
    void* out;
};

struct ModP {
    using T = uint32_t;
    uint32_t p;
    __device__ T zero() const { return 0u; }
    __device__ T mul_add(T acc, T a, T b) const {
        return static_cast<T>((static_cast<uint64_t>(a) * b + acc) % p);
    }
    __device__ T add(T a, T b) const {
        const uint32_t s = a + b;
        return s >= p ? s - p : s;
    }
};

struct CplxD {
    using T = double2;
    __device__ T zero() const { return make_double2(0.0, 0.0); }
    __device__ T mul_add(T acc, T a, T b) const {
        return make_double2(fma(a.x, b.x, fma(-a.y, b.y, acc.x)), fma(a.x, b.y, fma(a.y, b.x, acc.y)));
    }
    __device__ T add(T a, T b) const { return make_double2(a.x + b.x, a.y + b.y); }
};

// points per block: as many as the staging buffer holds, 32 to 128
template <class T, int S>
__host__ __device__ constexpr int cut_block() {
    return kCutStageBytes / (S * S * (int)sizeof(T)) >= 128 ? 128
         : (kCutStageBytes / (S * S * (int)sizeof(T))) / 32 * 32;
}

template <class F, int S>
__global__ void __launch_bounds__(cut_block<typename F::T, S>()) bg_cut_kernel(const F f, const CutArgs a) {
    using T = typename F::T;
    constexpr int kCutBlock = cut_block<T, S>();
    static_assert(kCutBlock >= 32, "staging buffer too small");
    __shared__ T stage[kCutBlock * S * S];
    const int64_t base = static_cast<int64_t>(blockIdx.x) * kCutBlock;
    const int t = threadIdx.x;
    const int nloc = a.E - base < kCutBlock ? static_cast<int>(a.E - base) : kCutBlock;
    T R[S][S];
    for (int i = 0; i < a.k; ++i) {
        // coalesced copy of this block's matrices M_i[base .. base+nloc)
        const T* src = static_cast<const T*>(a.M[i]) + base * S * S;
        for (int x = t; x < nloc * S * S; x += kCutBlock) stage[x] = src[x];
        __syncthreads();
        if (t < nloc) {
            const T* m = stage + t * S * S;
            if (i == 0) {
#pragma unroll
                for (int r = 0; r < S; ++r)
#pragma unroll
                    for (int c = 0; c < S; ++c) R[r][c] = m[r * S + c];
            } else {
                T N[S][S];
#pragma unroll
                for (int r = 0; r < S; ++r)
#pragma unroll
                    for (int c = 0; c < S; ++c) {
                        T acc = f.zero();
#pragma unroll
                        for (int q = 0; q < S; ++q) acc = f.mul_add(acc, m[r * S + q], R[q][c]);
                        N[r][c] = acc;
                    }
#pragma unroll
                for (int r = 0; r < S; ++r)
#pragma unroll
                    for (int c = 0; c < S; ++c) R[r][c] = N[r][c];
            }
        }
        __syncthreads();
    }
    if (t < nloc) {
        T tr = f.zero();
#pragma unroll
        for (int r = 0; r < S; ++r) tr = f.add(tr, R[r][r]);
        static_cast<T*>(a.out)[base + t] = tr;
    }
}

template <class F, int S>
void launch_cut_s(const F& f, const CutArgs& a, cudaStream_t s) {
    constexpr int B = cut_block<typename F::T, S>();
    const unsigned grid = (unsigned)((a.E + B - 1) / B);
    bg_cut_kernel<F, S><<<grid, B, 0, s>>>(f, a);
}

template <class F>
void launch_cut(const F& f, int S, const CutArgs& a, cudaStream_t s) {
    switch (S) {
        case 1: launch_cut_s<F, 1>(f, a, s); break;
        case 2: launch_cut_s<F, 2>(f, a, s); break;
        case 3: launch_cut_s<F, 3>(f, a, s); break;
        case 4: launch_cut_s<F, 4>(f, a, s); break;
        case 5: launch_cut_s<F, 5>(f, a, s); break;
        case 6: launch_cut_s<F, 6>(f, a, s); break;
        case 7: launch_cut_s<F, 7>(f, a, s); break;
        default: launch_cut_s<F, 8>(f, a, s); break;
    }
}

}  // namespace

extern "C" bg_status bg_cut_trace(bg_field field, uint32_t p, int64_t E, int k, int S,
                                  const void* const* M, void* out, cudaStream_t stream) {
    if (field != BG_FIELD_FP && field != BG_FIELD_C64 && field != BG_FIELD_C64_REAL)
        return bgi::fail(BG_ERR_INVALID_ARG, "unknown field %d", (int)field);
    if (field == BG_FIELD_FP && (p < 3 || p >= (1u << 31)))
        return bgi::fail(BG_ERR_INVALID_ARG, "p = %u outside [3, 2^31)", p);
    if (E < 0 || k < 1 || k > kCutMaxK || S < 1 || S > kCutMaxS)
        return bgi::fail(BG_ERR_INVALID_ARG, "need E >= 0, 1 <= k <= %d, 1 <= S <= %d", kCutMaxK, kCutMaxS);
    if (E == 0) return BG_OK;
    if (E > (int64_t(1) << 40)) return bgi::fail(BG_ERR_INVALID_ARG, "E too large");
    if (!M || !out) return bgi::fail(BG_ERR_INVALID_ARG, "M and out must be non-NULL");
    const size_t elem = bgi::value_bytes(field);
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return bgi::fail(BG_ERR_CUDA, "no current CUDA device");
    }
    CutArgs a;
    a.E = E;
    a.k = k;
    a.out = out;
    bg_status st;
    for (int i = 0; i < k; ++i) {
        if (!M[i]) return bgi::fail(BG_ERR_INVALID_ARG, "M[%d] is NULL", i);
        if ((uintptr_t)M[i] % elem) return bgi::fail(BG_ERR_INVALID_ARG, "M[%d] misaligned", i);
        if ((st = bgi::check_device_ptr(M[i], "M[i]", dev)) != BG_OK) return st;
        a.M[i] = M[i];
    }
    if ((uintptr_t)out % elem) return bgi::fail(BG_ERR_INVALID_ARG, "out misaligned");
    if ((st = bgi::check_device_ptr(out, "out", dev)) != BG_OK) return st;
    if (bgi::fault(BG_FAULT_LAUNCH)) return bgi::fail(BG_ERR_CUDA, "launch failed: injected fault");
    bgi::Range nvtx("bg_cut_trace");
    if (field == BG_FIELD_FP) launch_cut(ModP{p}, S, a, stream);
    else launch_cut(CplxD{}, S, a, stream);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return bgi::fail(BG_ERR_CUDA, "launch failed: %s", cudaGetErrorString(err));
    return BG_OK;
}
