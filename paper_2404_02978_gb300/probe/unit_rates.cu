// Unit-rate probe (sin.approx, cos.approx, ex2.approx, FFMA, DFMA, paired FFMA2, and the 32 x 32 -> 64-bit
// and 32-bit integer multiply-adds, per SM per clock): the denominators of the ALU rooflines.  Build and run on the GPU:
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o /tmp/unit_rates paper_2404_02978_gb300/probe/unit_rates.cu && /tmp/unit_rates
#include <cstdio>
#include <cuda_runtime.h>
#define CK(x) do{cudaError_t e=(x); if(e!=cudaSuccess){printf("CUDA %s @%d\n",cudaGetErrorString(e),__LINE__);return 1;}}while(0)
template<int OP>
__global__ void k(float* out, int iters, float a) {
  float x0=threadIdx.x*1e-3f, x1=x0+0.1f, x2=x0+0.2f, x3=x0+0.3f, x4=x0+0.4f, x5=x0+0.5f, x6=x0+0.6f, x7=x0+0.7f;
  for (int i=0;i<iters;i++){
#define S(x) if(OP==0){asm volatile("sin.approx.ftz.f32 %0,%0;":"+f"(x));} \
             else if(OP==1){asm volatile("cos.approx.ftz.f32 %0,%0;":"+f"(x));} \
             else if(OP==2){asm volatile("ex2.approx.ftz.f32 %0,%0;":"+f"(x));} \
             else {asm volatile("fma.rn.f32 %0,%0,%1,%1;":"+f"(x):"f"(a));}
    S(x0) S(x1) S(x2) S(x3) S(x4) S(x5) S(x6) S(x7)
  }
  out[blockIdx.x*blockDim.x+threadIdx.x]=x0+x1+x2+x3+x4+x5+x6+x7;
}
__global__ void kd(double* out, int iters, double a) {
  double x0=threadIdx.x*1e-3, x1=x0+0.1, x2=x0+0.2, x3=x0+0.3, x4=x0+0.4, x5=x0+0.5, x6=x0+0.6, x7=x0+0.7;
  for (int i=0;i<iters;i++){
#define D(x) asm volatile("fma.rn.f64 %0,%0,%1,%1;":"+d"(x):"d"(a));
    D(x0) D(x1) D(x2) D(x3) D(x4) D(x5) D(x6) D(x7)
  }
  out[blockIdx.x*blockDim.x+threadIdx.x]=x0+x1+x2+x3+x4+x5+x6+x7;
}
// Paired FP32 FMA (FFMA2: two lanes' FMAs in one instruction), 8 independent float2 chains.
__global__ void k2(float* out, int iters, float a) {
  const float2 av = make_float2(a, a);
  float2 x[8];
  for (int j = 0; j < 8; ++j) x[j] = make_float2(threadIdx.x * 1e-3f + 0.1f * j, threadIdx.x * 1e-3f - 0.1f * j);
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = __ffma2_rn(x[j], av, av);
  }
  float t = 0.0f;
  for (int j = 0; j < 8; ++j) t += x[j].x + x[j].y;
  out[blockIdx.x * blockDim.x + threadIdx.x] = t;
}
// Integer multiply-adds, 8 independent chains per thread, each step depending on the last through
// its multiplicand (nothing to hoist): OP 0 = mad.wide.s32 w = lo(w) a + w (64-bit addend and
// result), OP 1 = mad.lo.s32, OP 2 = mul.hi.s32 feeding an add.
template <int OP>
__global__ void ki(long long* out, int iters, int a) {
  long long w[8];
  int v[8];
  for (int j = 0; j < 8; ++j) { w[j] = threadIdx.x * 7 + j; v[j] = threadIdx.x * 13 + j; }
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if (OP == 0) asm volatile("{.reg .s32 l; cvt.u32.u64 l, %0; mad.wide.s32 %0, l, %1, %0;}" : "+l"(w[j]) : "r"(a));
      else if (OP == 1) asm volatile("mad.lo.s32 %0, %0, %1, %1;" : "+r"(v[j]) : "r"(a));
      else asm volatile("{.reg .s32 t; mul.hi.s32 t, %0, %1; add.s32 %0, %0, t;}" : "+r"(v[j]) : "r"(a));
    }
  }
  long long t = 0;
  for (int j = 0; j < 8; ++j) t += w[j] + v[j];
  out[blockIdx.x * blockDim.x + threadIdx.x] = t;
}
int main(){
  cudaDeviceProp p; CK(cudaGetDeviceProperties(&p,0));
  int clk=0; cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, 0);
  printf("name=%s SMs=%d cc=%d.%d clockRate_kHz=%d smem/block optin=%zu\n",p.name,p.multiProcessorCount,p.major,p.minor,clk,p.sharedMemPerBlockOptin);
  int nsm=p.multiProcessorCount, blocks=nsm*8, thr=256;
  float* o; CK(cudaMalloc(&o, blocks*thr*sizeof(double)));
  cudaEvent_t a,b; cudaEventCreate(&a); cudaEventCreate(&b);
  const char* names[4]={"sin.approx","cos.approx","ex2.approx","ffma"};
  for(int op=0;op<6;op++){
    int iters = op==4? 256 : 4096;
    for(int rep=0;rep<3;rep++){
      cudaEventRecord(a);
      if(op==0)k<0><<<blocks,thr>>>(o,iters,0.999f);
      if(op==1)k<1><<<blocks,thr>>>(o,iters,0.999f);
      if(op==2)k<2><<<blocks,thr>>>(o,iters,0.999f);
      if(op==3)k<3><<<blocks,thr>>>(o,iters,0.999f);
      if(op==4)kd<<<blocks,thr>>>((double*)o,iters,0.999);
      if(op==5)k2<<<blocks,thr>>>(o,iters,0.999f);
      cudaEventRecord(b); CK(cudaEventSynchronize(b));
      float ms; cudaEventElapsedTime(&ms,a,b);
      double ops=(double)blocks*thr*iters*8*(op==5?2:1);  // FFMA2: two FMAs per instruction
      if(rep==2) printf("%-11s %.3f ms  %.3e ops/s  per-SM-per-clk@2070MHz=%.2f  @1900=%.2f\n", op==4?"dfma":op==5?"ffma2 (FMAs)":names[op], ms, ops/(ms*1e-3), ops/(ms*1e-3)/nsm/2.07e9, ops/(ms*1e-3)/nsm/1.9e9);
    }
  }
  const char* inames[3] = {"mad.wide.s32", "mad.lo.s32", "mul.hi+add"};
  for (int op = 0; op < 3; op++) {
    for (int rep = 0; rep < 3; rep++) {
      cudaEventRecord(a);
      if (op == 0) ki<0><<<blocks, thr>>>((long long*)o, 4096, 0x12345);
      if (op == 1) ki<1><<<blocks, thr>>>((long long*)o, 4096, 0x12345);
      if (op == 2) ki<2><<<blocks, thr>>>((long long*)o, 4096, 0x12345);
      cudaEventRecord(b); CK(cudaEventSynchronize(b));
      float ms; cudaEventElapsedTime(&ms, a, b);
      double ops = (double)blocks * thr * 4096 * 8;
      if (rep == 2) printf("%-11s %.3f ms  %.3e ops/s  per-SM-per-clk@2070MHz=%.2f\n", inames[op], ms, ops / (ms * 1e-3),
                           ops / (ms * 1e-3) / nsm / 2.07e9);
    }
  }
  CK(cudaGetLastError());
  return 0;
}
