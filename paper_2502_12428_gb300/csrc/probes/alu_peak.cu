// Throughput probe for the roofline denominators: IMAD, IDP4A and mma.sync s8 (and f16, for context) on one GPU.
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>
#define CK(x) do{cudaError_t e=(x); if(e!=cudaSuccess){printf("err %s line %d\n",cudaGetErrorString(e),__LINE__); return 1;}}while(0)

__global__ void k_imad(int* out, int a, int b, int iters) {
  int x0=threadIdx.x, x1=x0+1, x2=x0+2, x3=x0+3, x4=x0+4, x5=x0+5, x6=x0+6, x7=x0+7;
  for (int i=0;i<iters;i++){
#pragma unroll
    for(int j=0;j<16;j++){
      x0 = x0*a + b; x1 = x1*a + b; x2 = x2*a + b; x3 = x3*a + b;
      x4 = x4*a + b; x5 = x5*a + b; x6 = x6*a + b; x7 = x7*a + b;
    }
  }
  out[blockIdx.x*blockDim.x+threadIdx.x] = x0^x1^x2^x3^x4^x5^x6^x7;
}
__global__ void k_dp4a(int* out, int a, int b, int iters) {
  int x0=threadIdx.x, x1=x0+1, x2=x0+2, x3=x0+3, x4=x0+4, x5=x0+5, x6=x0+6, x7=x0+7;
  for (int i=0;i<iters;i++){
#pragma unroll
    for(int j=0;j<16;j++){
      x0 = __dp4a(a, b, x0); x1 = __dp4a(a, b, x1); x2 = __dp4a(a, b, x2); x3 = __dp4a(a, b, x3);
      x4 = __dp4a(a, b, x4); x5 = __dp4a(a, b, x5); x6 = __dp4a(a, b, x6); x7 = __dp4a(a, b, x7);
    }
    a ^= x0;
  }
  out[blockIdx.x*blockDim.x+threadIdx.x] = x0^x1^x2^x3^x4^x5^x6^x7;
}
__global__ void k_iadd(int* out, int a, int b, int iters) {
  int x0=threadIdx.x, x1=x0+1, x2=x0+2, x3=x0+3, x4=x0+4, x5=x0+5, x6=x0+6, x7=x0+7;
  for (int i=0;i<iters;i++){
#pragma unroll
    for(int j=0;j<16;j++){
      x0 = x0 + a; x1 = x1 ^ a; x2 = x2 + b; x3 = x3 ^ b;
      x4 = x4 + x0; x5 = x5 ^ x1; x6 = x6 + x2; x7 = x7 ^ x3;
    }
  }
  out[blockIdx.x*blockDim.x+threadIdx.x] = x0^x1^x2^x3^x4^x5^x6^x7;
}
__global__ void k_mma(int* out, int a, int b, int iters) {
  int c[4][4] = {};
  int a0=a^threadIdx.x, a1=a+1, a2=a+2, a3=a+3, b0=b^threadIdx.x, b1=b+1;
  for (int i=0;i<iters;i++){
#pragma unroll
    for(int j=0;j<4;j++){
#pragma unroll
      for(int q=0;q<4;q++)
      asm volatile("mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
       : "+r"(c[q][0]),"+r"(c[q][1]),"+r"(c[q][2]),"+r"(c[q][3]) : "r"(a0),"r"(a1),"r"(a2),"r"(a3),"r"(b0),"r"(b1));
    }
  }
  int s=0;
  for(int q=0;q<4;q++) s ^= c[q][0]^c[q][1]^c[q][2]^c[q][3];
  out[blockIdx.x*blockDim.x+threadIdx.x] = s;
}
__global__ void k_mma_f16(int* out, int a, int b, int iters) {
  float c[4][4] = {};
  int a0=a^threadIdx.x, a1=a+1, a2=a+2, a3=a+3, b0=b^threadIdx.x, b1=b+1;
  for (int i=0;i<iters;i++){
#pragma unroll
    for(int j=0;j<4;j++){
#pragma unroll
      for(int q=0;q<4;q++)
      asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
       : "+f"(c[q][0]),"+f"(c[q][1]),"+f"(c[q][2]),"+f"(c[q][3]) : "r"(a0),"r"(a1),"r"(a2),"r"(a3),"r"(b0),"r"(b1));
    }
  }
  float s=0;
  for(int q=0;q<4;q++) s += c[q][0]+c[q][1]+c[q][2]+c[q][3];
  out[blockIdx.x*blockDim.x+threadIdx.x] = (int)s;
}

int main(){
  int dev; CK(cudaGetDevice(&dev)); cudaDeviceProp pr; CK(cudaGetDeviceProperties(&pr,dev));
  int sms = pr.multiProcessorCount;
  int clk=0; cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, dev);
  printf("gpu %s sms %d clock_khz %d smem/blk optin %zu l2 %d\n", pr.name, sms, clk, pr.sharedMemPerBlockOptin, pr.l2CacheSize);
  int blocks = sms*8, threads=256, iters=4096;
  int* out; CK(cudaMalloc(&out, sizeof(int)*blocks*threads));
  cudaEvent_t e0,e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  struct { const char* name; void(*fn)(int*,int,int,int); double ops_per_thread_iter; } ks[] = {
    {"imad (ops=MAC)", k_imad, 8*16}, {"dp4a (ops=4 MAC)", k_dp4a, 8*16*4}, {"iadd/xor", k_iadd, 8*16},
    {"mma s8 m16n8k32 (per thread share of MACs)", k_mma, 16.0*4096/32}, {"mma f16 m16n8k16 (MAC)", k_mma_f16, 16.0*2048/32}};
  for (auto& k : ks) {
    for (int rep=0; rep<3; rep++){
      k.fn<<<blocks,threads>>>(out, 3, 5, iters/16);
      CK(cudaGetLastError());
      CK(cudaEventRecord(e0));
      k.fn<<<blocks,threads>>>(out, 3, 5, iters);
      CK(cudaEventRecord(e1));
      CK(cudaEventSynchronize(e1));
      float ms; cudaEventElapsedTime(&ms,e0,e1);
      double ops = (double)blocks*threads*iters*k.ops_per_thread_iter;
      printf("%-45s  %.3f ms  %.2f T(ops)/s   per-SM-per-clk(at max clk %.0f MHz) %.1f\n", k.name, ms, ops/ms/1e9, clk/1e3, ops/(ms*1e-3)/sms/(clk*1e3));
    }
  }
  CK(cudaDeviceSynchronize());
  return 0;
}
