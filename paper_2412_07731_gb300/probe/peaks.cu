// Throughput probe for the roofline denominators: FP64 FMA, FP32 FMA, FP64
// mma.sync (DMMA) and TF32 mma.sync, register-only, timed with CUDA events.
#include <cstdio>
#include <cuda_runtime.h>
#define CK(x) do{cudaError_t e=(x); if(e!=cudaSuccess){printf("ERR %s line %d: %s\n",#x,__LINE__,cudaGetErrorString(e)); return 1;}}while(0)

template<int ITERS>
__global__ void fma64(double* out, double s) {
  double a0=threadIdx.x*1e-3, a1=a0+1, a2=a0+2, a3=a0+3, a4=a0+4, a5=a0+5, a6=a0+6, a7=a0+7;
  for (int i=0;i<ITERS;i++){
#pragma unroll
    for(int u=0;u<8;u++){
      a0=fma(a0,s,0.5); a1=fma(a1,s,0.5); a2=fma(a2,s,0.5); a3=fma(a3,s,0.5);
      a4=fma(a4,s,0.5); a5=fma(a5,s,0.5); a6=fma(a6,s,0.5); a7=fma(a7,s,0.5);
    }
  }
  out[blockIdx.x*blockDim.x+threadIdx.x]=a0+a1+a2+a3+a4+a5+a6+a7;
}
template<int ITERS>
__global__ void fma32(float* out, float s) {
  float a[16];
#pragma unroll
  for(int u=0;u<16;u++) a[u]=threadIdx.x*1e-3f+u;
  for (int i=0;i<ITERS;i++){
#pragma unroll
    for(int r=0;r<8;r++)
#pragma unroll
    for(int u=0;u<16;u++) a[u]=fmaf(a[u],s,0.5f);
  }
  float t=0; for(int u=0;u<16;u++) t+=a[u];
  out[blockIdx.x*blockDim.x+threadIdx.x]=t;
}
template<int ITERS>
__global__ void dmma(double* out) {
  double a = threadIdx.x*1e-3, b = 1.0 - threadIdx.x*1e-4;
  double c[4][2];
  for(int u=0;u<4;u++){c[u][0]=0;c[u][1]=0;}
  for (int i=0;i<ITERS;i++){
#pragma unroll
    for(int u=0;u<4;u++){
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
        : "+d"(c[u][0]), "+d"(c[u][1]) : "d"(a), "d"(b));
    }
  }
  double t=0; for(int u=0;u<4;u++) t+=c[u][0]+c[u][1];
  out[blockIdx.x*blockDim.x+threadIdx.x]=t;
}
template<int ITERS>
__global__ void tf32mma(float* out) {
  unsigned a0=__float_as_uint(1.0f+threadIdx.x*1e-3f), a1=a0, a2=a0, a3=a0, b0=__float_as_uint(0.5f), b1=b0;
  float c[4][4];
  for(int u=0;u<4;u++) for(int v=0;v<4;v++) c[u][v]=0;
  for (int i=0;i<ITERS;i++){
#pragma unroll
    for(int u=0;u<4;u++){
      asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(c[u][0]), "+f"(c[u][1]), "+f"(c[u][2]), "+f"(c[u][3]) : "r"(a0),"r"(a1),"r"(a2),"r"(a3),"r"(b0),"r"(b1));
    }
  }
  float t=0; for(int u=0;u<4;u++) for(int v=0;v<4;v++) t+=c[u][v];
  out[blockIdx.x*blockDim.x+threadIdx.x]=t;
}

int main(){
  int dev=0; cudaDeviceProp p; CK(cudaGetDeviceProperties(&p,dev));
  printf("device %s SMs %d cc %d.%d\n", p.name, p.multiProcessorCount, p.major, p.minor);
  int nsm=p.multiProcessorCount;
  const int threads=256; const int blocks=nsm*8;
  double* d64; float* d32;
  CK(cudaMalloc(&d64, sizeof(double)*threads*blocks));
  CK(cudaMalloc(&d32, sizeof(float)*threads*blocks));
  cudaEvent_t e0,e1; CK(cudaEventCreate(&e0)); CK(cudaEventCreate(&e1));
  float ms;
  const int IT=2000;
  for(int rep=0;rep<3;rep++){
    fma64<IT><<<blocks,threads>>>(d64, 0.999); CK(cudaGetLastError());
    CK(cudaEventRecord(e0)); fma64<IT><<<blocks,threads>>>(d64, 0.999); CK(cudaEventRecord(e1)); CK(cudaEventSynchronize(e1));
    CK(cudaEventElapsedTime(&ms,e0,e1));
    double fl = 2.0*IT*64.0*threads*blocks; printf("fp64_fma_tflops %.3f (%.3f ms)\n", fl/ms/1e9, ms);
    fma32<IT><<<blocks,threads>>>(d32, 0.999f); CK(cudaGetLastError());
    CK(cudaEventRecord(e0)); fma32<IT><<<blocks,threads>>>(d32, 0.999f); CK(cudaEventRecord(e1)); CK(cudaEventSynchronize(e1));
    CK(cudaEventElapsedTime(&ms,e0,e1));
    fl = 2.0*IT*128.0*threads*blocks; printf("fp32_fma_tflops %.3f (%.3f ms)\n", fl/ms/1e9, ms);
    dmma<IT><<<blocks,threads>>>(d64); CK(cudaGetLastError());
    CK(cudaEventRecord(e0)); dmma<IT><<<blocks,threads>>>(d64); CK(cudaEventRecord(e1)); CK(cudaEventSynchronize(e1));
    CK(cudaEventElapsedTime(&ms,e0,e1));
    fl = 2.0*8*8*4*4.0*IT*(threads/32)*blocks; printf("fp64_dmma_tflops %.3f (%.3f ms)\n", fl/ms/1e9, ms);
    tf32mma<IT><<<blocks,threads>>>(d32); CK(cudaGetLastError());
    CK(cudaEventRecord(e0)); tf32mma<IT><<<blocks,threads>>>(d32); CK(cudaEventRecord(e1)); CK(cudaEventSynchronize(e1));
    CK(cudaEventElapsedTime(&ms,e0,e1));
    fl = 2.0*16*8*8*4.0*IT*(threads/32)*blocks; printf("tf32_mmasync_tflops %.3f (%.3f ms)\n", fl/ms/1e9, ms);
  }
  CK(cudaDeviceSynchronize());
  printf("OK\n");
  return 0;
}
