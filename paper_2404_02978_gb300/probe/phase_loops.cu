// Inner-loop probe: (point, term) throughput of the fused synthesis inner loop with the
// double-float phase, the 64-bit fixed-point phase, and no reduction (the MUFU bound).
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o /tmp/phase_loops paper_2404_02978_gb300/probe/phase_loops.cu && /tmp/phase_loops
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>
#define CK(x) do{cudaError_t e=(x); if(e!=cudaSuccess){printf("CUDA %s @%d\n",cudaGetErrorString(e),__LINE__);return 1;}}while(0)
constexpr int TPB=256, PPT=8, NT=4096;
__device__ __forceinline__ float sinr(float x){float y; asm("sin.approx.ftz.f32 %0,%1;":"=f"(y):"f"(x)); return y;}
__device__ __forceinline__ float cosr(float x){float y; asm("cos.approx.ftz.f32 %0,%1;":"=f"(y):"f"(x)); return y;}
template<int V>
__global__ void __launch_bounds__(TPB) k(const float4* terms, const float2* xy, float* out, int reps){
  __shared__ float4 st[1024];
  float x[PPT], y[PPT], acc[PPT]; int xi[PPT], yi[PPT];
  for(int j=0;j<PPT;j++){ float2 p=xy[(blockIdx.x*PPT+j)*TPB+threadIdx.x]; x[j]=p.x; y[j]=p.y; acc[j]=0.f;
    xi[j]=__float2int_rn(p.x*536870912.f); yi[j]=__float2int_rn(p.y*536870912.f);}
  for(int rep=0;rep<reps;rep++)
  for(int c=0;c<NT;c+=1024){
    __syncthreads();
    for(int i=threadIdx.x;i<1024;i+=TPB) st[i]=terms[c+i];
    __syncthreads();
    #pragma unroll 2
    for(int t=0;t<1024;t++){
      float4 T=st[t];
      if(V==0){
        #pragma unroll
        for(int j=0;j<PPT;j++){
          float p1=__fmul_rn(T.x,x[j]); float e1=__fmaf_rn(T.x,x[j],-p1);
          float p2=__fmul_rn(T.y,y[j]); float e2=__fmaf_rn(T.y,y[j],-p2);
          const float M=12582912.f;
          float n1=__fsub_rn(__fadd_rn(p1,M),M), n2=__fsub_rn(__fadd_rn(p2,M),M);
          float r=__fadd_rn(__fsub_rn(p1,n1),__fsub_rn(p2,n2));
          float ph=__fadd_rn(r,__fadd_rn(e1,e2));
          float a=ph*6.2831853f;
          float s=sinr(a), co=cosr(a);
          acc[j]=fmaf(T.z,co,acc[j]); acc[j]=fmaf(T.w,s,acc[j]);
        }
      } else if(V==1){
        int fx=__float_as_int(T.x), fy=__float_as_int(T.y); // pretend fixed-point ints
        #pragma unroll
        for(int j=0;j<PPT;j++){
          long long pr=(long long)fx*xi[j]; pr+=(long long)fy*yi[j];
          uint32_t lo=(uint32_t)pr, hi=(uint32_t)(pr>>32);
          uint32_t ph; asm("shf.l.wrap.b32 %0,%1,%2,8;":"=r"(ph):"r"(lo),"r"(hi));
          float f=__int_as_float((ph>>9)|0x3F800000u)-1.5f;
          float a=f*6.2831853f;
          float s=sinr(a), co=cosr(a);
          acc[j]=fmaf(T.z,co,acc[j]); acc[j]=fmaf(T.w,s,acc[j]);
        }
      } else {
        #pragma unroll
        for(int j=0;j<PPT;j++){
          float a=fmaf(T.x,x[j],T.y*y[j]);
          float s=sinr(a), co=cosr(a);
          acc[j]=fmaf(T.z,co,acc[j]); acc[j]=fmaf(T.w,s,acc[j]);
        }
      }
    }
  }
  for(int j=0;j<PPT;j++) out[(blockIdx.x*PPT+j)*TPB+threadIdx.x]=acc[j];
}
int main(){
  int nsm; cudaDeviceGetAttribute(&nsm,cudaDevAttrMultiProcessorCount,0);
  int blocks=nsm*4*8; size_t np=(size_t)blocks*TPB*PPT;
  float4* terms; float2* xy; float* out;
  CK(cudaMalloc(&terms,NT*sizeof(float4))); CK(cudaMalloc(&xy,np*sizeof(float2))); CK(cudaMalloc(&out,np*4));
  float4 h[NT]; for(int i=0;i<NT;i++) h[i]=make_float4(0.01f*(i%97)-0.4f,0.013f*(i%89)-0.5f,0.1f,-0.1f);
  CK(cudaMemcpy(terms,h,sizeof(h),cudaMemcpyHostToDevice)); CK(cudaMemset(xy,0,np*sizeof(float2)));
  cudaEvent_t a,b; cudaEventCreate(&a); cudaEventCreate(&b);
  const char* nm[3]={"doublefloat13","fixedpoint64","noreduce"};
  for(int v=0;v<3;v++){ for(int rep=0;rep<3;rep++){
    cudaEventRecord(a);
    if(v==0)k<0><<<blocks,TPB>>>(terms,xy,out,2); if(v==1)k<1><<<blocks,TPB>>>(terms,xy,out,2); if(v==2)k<2><<<blocks,TPB>>>(terms,xy,out,2);
    cudaEventRecord(b); CK(cudaEventSynchronize(b)); float ms; cudaEventElapsedTime(&ms,a,b);
    double tp=(double)np*NT*2;
    if(rep==2) printf("%-14s %.3f ms %.3e term-pts/s  per-SM-clk@1995=%.2f\n",nm[v],ms,tp/(ms*1e-3),tp/(ms*1e-3)/nsm/1.995e9);
  }}
  CK(cudaGetLastError()); return 0;
}
