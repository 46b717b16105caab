// pipe_throughput.cu -- stand-alone measurement of the integer-multiply and
// FP64 pipes (the denominators of the ALU rooflines reported by bench.py).
//
// Each thread runs 8 independent dependency chains of one operation; every
// bit of every result stays live (the chains feed both 32-bit halves of a
// 64-bit result back into the next operand and the kernel stores all of it),
// so the compiler cannot narrow a 64-bit operation to a 32-bit one.  The
// rate is printed in operations per SM per clock at the maximum SM clock.
//
// Besides single instructions it times the two field-multiplication kernels
// of the F_p recursion in isolation:
//   mont2:  t = a b + c d (two 32x32+64 products), Montgomery reduction
//           m = lo(t) (-p^-1), r = hi(m p + t), 64-bit accumulation of r --
//           two field multiplications;
//   lazy4:  four 32x32+64 products summed unreduced into a 96-bit
//           accumulator (one carry chain) -- four field multiplications.
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o pipe_throughput pipe_throughput.cu
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>
#define CK(x) do{cudaError_t e=(x); if(e){printf("err %s line %d\n", cudaGetErrorString(e), __LINE__); return 1;}}while(0)
constexpr int ITERS = 2048;

__device__ __forceinline__ uint32_t mix(uint64_t x) { return (uint32_t)x ^ (uint32_t)(x >> 32); }

__global__ void k_madlo(uint64_t* out, uint32_t s) {
  uint32_t a[8];
  for (int k = 0; k < 8; ++k) a[k] = threadIdx.x * 8 + k + s;
  for (int i = 0; i < ITERS; i++) {
#pragma unroll
    for (int k = 0; k < 8; ++k) asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(a[k]) : "r"(s), "r"(a[(k + 1) & 7]));
  }
  uint64_t r = 0;
  for (int k = 0; k < 8; ++k) r += a[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = r;
}
__global__ void k_mulhi(uint64_t* out, uint32_t s) {
  uint32_t a[8];
  for (int k = 0; k < 8; ++k) a[k] = threadIdx.x * 8 + k + s;
  for (int i = 0; i < ITERS; i++) {
#pragma unroll
    for (int k = 0; k < 8; ++k) asm volatile("mad.hi.u32 %0, %0, %1, %2;" : "+r"(a[k]) : "r"(s), "r"(a[(k + 1) & 7]));
  }
  uint64_t r = 0;
  for (int k = 0; k < 8; ++k) r += a[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = r;
}
// 64-bit result of a 32x32+64 multiply-add; the next multiplicand is the xor
// of both halves of the previous result, so both halves are live.
__global__ void k_madwide(uint64_t* out, uint32_t s) {
  uint64_t a[8];
  for (int k = 0; k < 8; ++k) a[k] = (uint64_t)(threadIdx.x * 8 + k + s) << 17;
  for (int i = 0; i < ITERS; i++) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      uint32_t x = mix(a[(k + 1) & 7]);
      asm volatile("mad.wide.u32 %0, %1, %2, %0;" : "+l"(a[k]) : "r"(x), "r"(s));
    }
  }
  uint64_t r = 0;
  for (int k = 0; k < 8; ++k) r ^= a[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = r;
}
// the same xor feedback with a 32-bit multiply-add, to separate the cost of
// the xor from the multiply
__global__ void k_madlo_xor(uint64_t* out, uint32_t s) {
  uint64_t a[8];
  for (int k = 0; k < 8; ++k) a[k] = (uint64_t)(threadIdx.x * 8 + k + s) << 17;
  for (int i = 0; i < ITERS; i++) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      uint32_t x = mix(a[(k + 1) & 7]);
      uint32_t lo = (uint32_t)a[k], hi = (uint32_t)(a[k] >> 32);
      asm volatile("mad.lo.u32 %0, %1, %2, %0;" : "+r"(lo) : "r"(x), "r"(s));
      a[k] = ((uint64_t)hi << 32) | lo;
    }
  }
  uint64_t r = 0;
  for (int k = 0; k < 8; ++k) r ^= a[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = r;
}
__global__ void k_iadd(uint64_t* out, uint32_t s) {
  uint32_t a[8];
  for (int k = 0; k < 8; ++k) a[k] = threadIdx.x * 8 + k + s;
  for (int i = 0; i < ITERS; i++) {
#pragma unroll
    for (int k = 0; k < 8; ++k) asm volatile("add.u32 %0, %0, %1;" : "+r"(a[k]) : "r"(a[(k + 1) & 7]));
  }
  uint64_t r = 0;
  for (int k = 0; k < 8; ++k) r += a[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = r;
}
// two field multiplications per step: Montgomery reduction of a pair
__global__ void k_mont2(uint64_t* out, uint32_t p, uint32_t pinv) {
  uint32_t v[8];
  uint64_t acc[8];
  for (int k = 0; k < 8; ++k) { v[k] = (threadIdx.x * 8 + k) % p; acc[k] = 0; }
  for (int i = 0; i < ITERS; i++) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const uint32_t c = v[(k + 1) & 7], d = v[(k + 3) & 7];
      const uint64_t t = (uint64_t)c * v[k] + (uint64_t)d * v[(k + 5) & 7];
      const uint32_t m = (uint32_t)t * pinv;
      const uint32_t r = (uint32_t)(((uint64_t)m * p + t) >> 32);
      acc[k] += r;
      v[k] = min(r, r - p);
    }
  }
  uint64_t r = 0;
  for (int k = 0; k < 8; ++k) r ^= acc[k] + v[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = r;
}
__device__ __forceinline__ void add96(uint64_t& lo, uint32_t& hi, uint64_t t) {
  asm("{\n\t.reg .u32 a0, a1, t0, t1;\n\tmov.b64 {a0, a1}, %0;\n\tmov.b64 {t0, t1}, %2;\n\t"
      "add.cc.u32 a0, a0, t0;\n\taddc.cc.u32 a1, a1, t1;\n\taddc.u32 %1, %1, 0;\n\tmov.b64 %0, {a0, a1};\n\t}"
      : "+l"(lo), "+r"(hi) : "l"(t));
}
// four field multiplications per step: unreduced products into a 96-bit sum
__global__ void k_lazy4(uint64_t* out, uint32_t p) {
  uint32_t v[8];
  uint64_t lo[8];
  uint32_t hi[8];
  for (int k = 0; k < 8; ++k) { v[k] = (threadIdx.x * 8 + k) % p; lo[k] = 0; hi[k] = 0; }
  for (int i = 0; i < ITERS; i++) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const uint64_t t = (uint64_t)v[(k + 1) & 7] * v[k] + (uint64_t)v[(k + 2) & 7] * v[(k + 3) & 7] +
                         (uint64_t)v[(k + 4) & 7] * v[(k + 5) & 7] + (uint64_t)v[(k + 6) & 7] * v[(k + 7) & 7];
      add96(lo[k], hi[k], t);
      v[k] ^= (uint32_t)lo[k] & 0x3fffffffu;
    }
  }
  uint64_t r = 0;
  for (int k = 0; k < 8; ++k) r ^= lo[k] + hi[k] + v[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = r;
}
__global__ void k_dfma(double* out, double s) {
  double a0=threadIdx.x*1e-3, a1=a0+1, a2=a0+2, a3=a0+3, a4=a0+4, a5=a0+5, a6=a0+6, a7=a0+7;
  for (int i=0;i<ITERS/8;i++){
    asm volatile("fma.rn.f64 %0, %0, %1, %2;" : "+d"(a0) : "d"(s), "d"(a1));
    asm volatile("fma.rn.f64 %0, %0, %1, %2;" : "+d"(a1) : "d"(s), "d"(a2));
    asm volatile("fma.rn.f64 %0, %0, %1, %2;" : "+d"(a2) : "d"(s), "d"(a3));
    asm volatile("fma.rn.f64 %0, %0, %1, %2;" : "+d"(a3) : "d"(s), "d"(a4));
    asm volatile("fma.rn.f64 %0, %0, %1, %2;" : "+d"(a4) : "d"(s), "d"(a5));
    asm volatile("fma.rn.f64 %0, %0, %1, %2;" : "+d"(a5) : "d"(s), "d"(a6));
    asm volatile("fma.rn.f64 %0, %0, %1, %2;" : "+d"(a6) : "d"(s), "d"(a7));
    asm volatile("fma.rn.f64 %0, %0, %1, %2;" : "+d"(a7) : "d"(s), "d"(a0));
  }
  out[blockIdx.x*blockDim.x+threadIdx.x] = a0+a1+a2+a3+a4+a5+a6+a7;
}
__global__ void k_ffma(float* out, float s) {
  float a0=threadIdx.x*1e-3f, a1=a0+1, a2=a0+2, a3=a0+3, a4=a0+4, a5=a0+5, a6=a0+6, a7=a0+7;
  for (int i=0;i<ITERS;i++){
    asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(a0) : "f"(s), "f"(a1));
    asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(a1) : "f"(s), "f"(a2));
    asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(a2) : "f"(s), "f"(a3));
    asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(a3) : "f"(s), "f"(a4));
    asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(a4) : "f"(s), "f"(a5));
    asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(a5) : "f"(s), "f"(a6));
    asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(a6) : "f"(s), "f"(a7));
    asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(a7) : "f"(s), "f"(a0));
  }
  out[blockIdx.x*blockDim.x+threadIdx.x] = a0+a1+a2+a3+a4+a5+a6+a7;
}
template<typename K, typename... A> int run(const char* name, K kern, int blocks, int threads, double ops_per_thread, A... args) {
  kern<<<blocks, threads>>>(args...); CK(cudaDeviceSynchronize());
  cudaEvent_t a,b; cudaEventCreate(&a); cudaEventCreate(&b);
  cudaEventRecord(a); for(int r=0;r<5;r++) kern<<<blocks, threads>>>(args...); cudaEventRecord(b); CK(cudaEventSynchronize(b));
  float ms; cudaEventElapsedTime(&ms,a,b); ms/=5;
  double ops = ops_per_thread*blocks*threads;
  int sm=0, clk=0; cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, 0); cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, 0);
  printf("%-12s blocks=%d thr=%d  %.3f ms  %.3f Tops/s  %.2f ops/clk/SM (at %d MHz max)\n", name, blocks, threads, ms, ops/ms*1e-9, ops/(ms*1e-3)/sm/(clk*1e3), clk/1000);
  return 0;
}
int main(){
  int sm; cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, 0);
  uint64_t* u; double* dd; float* ff;
  const uint32_t p = 2147483629u;
  uint32_t inv = p;
  for (int i = 0; i < 5; ++i) inv *= 2u - p * inv;
  const uint32_t pinv = 0u - inv;
  CK(cudaMalloc(&u, 1<<27)); CK(cudaMalloc(&dd, 1<<27)); CK(cudaMalloc(&ff, 1<<26));
  for (int tpb : {256, 512}) {
    int blocks = sm*4*256/tpb*2;
    run("madlo", k_madlo, blocks, tpb, 8.0*ITERS, u, 12345u);
    run("madlo_xor", k_madlo_xor, blocks, tpb, 8.0*ITERS, u, 12345u);
    run("madhi", k_mulhi, blocks, tpb, 8.0*ITERS, u, 12345u);
    run("madwide", k_madwide, blocks, tpb, 8.0*ITERS, u, 12345u);
    run("iadd", k_iadd, blocks, tpb, 8.0*ITERS, u, 12345u);
    run("mont2_fmul", k_mont2, blocks, tpb, 2*8.0*ITERS, u, p, pinv);
    run("lazy4_fmul", k_lazy4, blocks, tpb, 4*8.0*ITERS, u, p);
    run("ffma", k_ffma, blocks, tpb, 8.0*ITERS, ff, 0.999f);
    run("dfma", k_dfma, blocks, tpb, 8.0*ITERS/8, dd, 0.999);
  }
  return 0;
}
