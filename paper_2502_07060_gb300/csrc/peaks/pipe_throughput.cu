// pipe_throughput.cu -- stand-alone measurement of the integer-multiply and
// FP64 pipes (the denominators of the ALU rooflines reported by bench.py).
// Each thread runs 8 independent dependency chains of one instruction; the
// rate is printed in operations per SM per clock at the maximum SM clock.
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o pipe_throughput pipe_throughput.cu
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>
#define CK(x) do{cudaError_t e=(x); if(e){printf("err %s line %d\n", cudaGetErrorString(e), __LINE__); return 1;}}while(0)
constexpr int ITERS = 4096;
__global__ void k_madlo(uint32_t* out, uint32_t s) {
  uint32_t a0=threadIdx.x+s, a1=a0^1, a2=a0^2, a3=a0^3, a4=a0^4, a5=a0^5, a6=a0^6, a7=a0^7;
  for (int i=0;i<ITERS;i++){
    asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(a0) : "r"(s), "r"(a1));
    asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(a1) : "r"(s), "r"(a2));
    asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(a2) : "r"(s), "r"(a3));
    asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(a3) : "r"(s), "r"(a4));
    asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(a4) : "r"(s), "r"(a5));
    asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(a5) : "r"(s), "r"(a6));
    asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(a6) : "r"(s), "r"(a7));
    asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(a7) : "r"(s), "r"(a0));
  }
  out[blockIdx.x*blockDim.x+threadIdx.x] = a0+a1+a2+a3+a4+a5+a6+a7;
}
__global__ void k_mulhi(uint32_t* out, uint32_t s) {
  uint32_t a0=threadIdx.x+s, a1=a0^1, a2=a0^2, a3=a0^3, a4=a0^4, a5=a0^5, a6=a0^6, a7=a0^7;
  for (int i=0;i<ITERS;i++){
    asm volatile("mul.hi.u32 %0, %0, %1;" : "+r"(a0) : "r"(s));
    asm volatile("mul.hi.u32 %0, %0, %1;" : "+r"(a1) : "r"(s));
    asm volatile("mul.hi.u32 %0, %0, %1;" : "+r"(a2) : "r"(s));
    asm volatile("mul.hi.u32 %0, %0, %1;" : "+r"(a3) : "r"(s));
    asm volatile("mul.hi.u32 %0, %0, %1;" : "+r"(a4) : "r"(s));
    asm volatile("mul.hi.u32 %0, %0, %1;" : "+r"(a5) : "r"(s));
    asm volatile("mul.hi.u32 %0, %0, %1;" : "+r"(a6) : "r"(s));
    asm volatile("mul.hi.u32 %0, %0, %1;" : "+r"(a7) : "r"(s));
  }
  out[blockIdx.x*blockDim.x+threadIdx.x] = a0+a1+a2+a3+a4+a5+a6+a7;
}
__global__ void k_mulwide(uint32_t* out, uint32_t s) {
  uint64_t a0=threadIdx.x+s, a1=a0^1, a2=a0^2, a3=a0^3, a4=a0^4, a5=a0^5, a6=a0^6, a7=a0^7;
  for (int i=0;i<ITERS;i++){
    asm volatile("mad.wide.u32 %0, %1, %2, %0;" : "+l"(a0) : "r"((uint32_t)a1), "r"(s));
    asm volatile("mad.wide.u32 %0, %1, %2, %0;" : "+l"(a1) : "r"((uint32_t)a2), "r"(s));
    asm volatile("mad.wide.u32 %0, %1, %2, %0;" : "+l"(a2) : "r"((uint32_t)a3), "r"(s));
    asm volatile("mad.wide.u32 %0, %1, %2, %0;" : "+l"(a3) : "r"((uint32_t)a4), "r"(s));
    asm volatile("mad.wide.u32 %0, %1, %2, %0;" : "+l"(a4) : "r"((uint32_t)a5), "r"(s));
    asm volatile("mad.wide.u32 %0, %1, %2, %0;" : "+l"(a5) : "r"((uint32_t)a6), "r"(s));
    asm volatile("mad.wide.u32 %0, %1, %2, %0;" : "+l"(a6) : "r"((uint32_t)a7), "r"(s));
    asm volatile("mad.wide.u32 %0, %1, %2, %0;" : "+l"(a7) : "r"((uint32_t)a0), "r"(s));
  }
  out[blockIdx.x*blockDim.x+threadIdx.x] = (uint32_t)(a0+a1+a2+a3+a4+a5+a6+a7);
}
__global__ void k_iadd(uint32_t* out, uint32_t s) {
  uint32_t a0=threadIdx.x+s, a1=a0^1, a2=a0^2, a3=a0^3, a4=a0^4, a5=a0^5, a6=a0^6, a7=a0^7;
  for (int i=0;i<ITERS;i++){
    asm volatile("add.u32 %0, %0, %1;" : "+r"(a0) : "r"(a1));
    asm volatile("add.u32 %0, %0, %1;" : "+r"(a1) : "r"(a2));
    asm volatile("add.u32 %0, %0, %1;" : "+r"(a2) : "r"(a3));
    asm volatile("add.u32 %0, %0, %1;" : "+r"(a3) : "r"(a4));
    asm volatile("add.u32 %0, %0, %1;" : "+r"(a4) : "r"(a5));
    asm volatile("add.u32 %0, %0, %1;" : "+r"(a5) : "r"(a6));
    asm volatile("add.u32 %0, %0, %1;" : "+r"(a6) : "r"(a7));
    asm volatile("add.u32 %0, %0, %1;" : "+r"(a7) : "r"(a0));
  }
  out[blockIdx.x*blockDim.x+threadIdx.x] = a0+a1+a2+a3+a4+a5+a6+a7;
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
template<typename K, typename T> int run(const char* name, K kern, T* buf, T s, int blocks, int threads, double ops_per_thread) {
  kern<<<blocks, threads>>>(buf, s); CK(cudaDeviceSynchronize());
  cudaEvent_t a,b; cudaEventCreate(&a); cudaEventCreate(&b);
  cudaEventRecord(a); for(int r=0;r<5;r++) kern<<<blocks, threads>>>(buf, s); cudaEventRecord(b); CK(cudaEventSynchronize(b));
  float ms; cudaEventElapsedTime(&ms,a,b); ms/=5;
  double ops = ops_per_thread*blocks*threads;
  int sm=0, clk=0; cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, 0); cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, 0);
  printf("%-10s blocks=%d thr=%d  %.3f ms  %.3f Tops/s  %.2f ops/clk/SM (at %d MHz max)\n", name, blocks, threads, ms, ops/ms*1e-9, ops/(ms*1e-3)/sm/(clk*1e3), clk/1000);
  return 0;
}
int main(){
  int sm; cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, 0);
  uint32_t* u; double* dd; float* ff;
  CK(cudaMalloc(&u, 1<<26)); CK(cudaMalloc(&dd, 1<<27)); CK(cudaMalloc(&ff, 1<<26));
  for (int tpb : {256, 512, 1024}) {
    int blocks = sm*4*256/tpb*2;
    run("madlo", k_madlo, u, 12345u, blocks, tpb, 8.0*ITERS);
    run("mulhi", k_mulhi, u, 12345u, blocks, tpb, 8.0*ITERS);
    run("madwide", k_mulwide, u, 12345u, blocks, tpb, 8.0*ITERS);
    run("iadd", k_iadd, u, 12345u, blocks, tpb, 8.0*ITERS);
    run("ffma", k_ffma, ff, 0.999f, blocks, tpb, 8.0*ITERS);
    run("dfma", k_dfma, dd, 0.999, blocks, tpb, 8.0*ITERS/8);
  }
  return 0;
}
