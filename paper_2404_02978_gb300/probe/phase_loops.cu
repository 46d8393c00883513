// Inner-loop probe: (point, term) throughput of the fused synthesis inner loop with the
// double-float phase, the 64-bit fixed-point phase, and no reduction (the MUFU bound); then the
// same in amplitude-phase form (one cosine per (point, term)): no reduction, the fixed-point
// phase with the fraction in the high word (scalar and with paired FP32 instructions), a
// bare cosine per (point, term), and variants of the integer phase (alone; one 64-bit product;
// two independent products; 32-bit halves with an explicit carry; explicit mad.wide.s32; unsigned products).
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
      } else if(V==2){
        #pragma unroll
        for(int j=0;j<PPT;j++){
          float a=fmaf(T.x,x[j],T.y*y[j]);
          float s=sinr(a), co=cosr(a);
          acc[j]=fmaf(T.z,co,acc[j]); acc[j]=fmaf(T.w,s,acc[j]);
        }
      } else if(V==3){
        #pragma unroll
        for(int j=0;j<PPT;j++){
          float a=fmaf(T.x,x[j],T.y*y[j]);
          acc[j]=fmaf(T.z,cosr(a),acc[j]);
        }
      } else if(V==4 || V==5){
        int fx=__float_as_int(T.x), fy=__float_as_int(T.y);
        const uint64_t C=(uint64_t)__float_as_uint(T.w)*(1u<<30)+(1ull<<31);
        if(V==4){
          #pragma unroll
          for(int j=0;j<PPT;j++){
            uint64_t pr=C+(uint64_t)((long long)fy*yi[j]); pr+=(uint64_t)((long long)fx*xi[j]);
            uint32_t hi=(uint32_t)(pr>>32);
            float a=fmaf(__uint_as_float((hi&0x007FFFFFu)|0x3F800000u),6.2831853f,-6.2831853f);
            acc[j]=fmaf(T.z,cosr(a),acc[j]);
          }
        } else {
          const float2 A=make_float2(T.z,T.z), tp=make_float2(6.2831853f,6.2831853f), ntp=make_float2(-6.2831853f,-6.2831853f);
          #pragma unroll
          for(int q=0;q<PPT/2;q++){
            uint64_t p0=C+(uint64_t)((long long)fy*yi[2*q]); p0+=(uint64_t)((long long)fx*xi[2*q]);
            uint64_t p1=C+(uint64_t)((long long)fy*yi[2*q+1]); p1+=(uint64_t)((long long)fx*xi[2*q+1]);
            const float2 m=make_float2(__uint_as_float(((uint32_t)(p0>>32)&0x007FFFFFu)|0x3F800000u),
                                       __uint_as_float(((uint32_t)(p1>>32)&0x007FFFFFu)|0x3F800000u));
            const float2 a=__ffma2_rn(m,tp,ntp);
            float2 pa=make_float2(acc[2*q],acc[2*q+1]);
            pa=__ffma2_rn(A,make_float2(cosr(a.x),cosr(a.y)),pa);
            acc[2*q]=pa.x; acc[2*q+1]=pa.y;
          }
        }
      } else if(V==6){
        #pragma unroll
        for(int j=0;j<PPT;j++) acc[j]+=cosr(T.x*x[j]);
      } else {
        int fx=__float_as_int(T.x), fy=__float_as_int(T.y);
        const uint64_t C=(uint64_t)__float_as_uint(T.w)*(1u<<30)+(1ull<<31);
        #pragma unroll
        for(int j=0;j<PPT;j++){
          uint32_t hi;
          if(V==7){         // the integer phase alone, no cosine
            uint64_t pr=C+(uint64_t)((long long)fy*yi[j]); pr+=(uint64_t)((long long)fx*xi[j]); hi=(uint32_t)(pr>>32);
          } else if(V==8){  // one 64-bit product per (point, term)
            uint64_t pr=C+(uint64_t)((long long)fx*xi[j]); hi=(uint32_t)(pr>>32);
          } else if(V==9){  // two independent 64-bit products, then a 64-bit add
            uint64_t p1=C+(uint64_t)((long long)fy*yi[j]); uint64_t p2=(uint64_t)((long long)fx*xi[j]); hi=(uint32_t)((p1+p2)>>32);
          } else if(V==11 || V==12){  // the two products as explicit mad.wide.s32 (64-bit addend)
            uint64_t pr;
            asm("mad.wide.s32 %0, %1, %2, %3;" : "=l"(pr) : "r"(fy), "r"(yi[j]), "l"(C));
            asm("mad.wide.s32 %0, %1, %2, %0;" : "+l"(pr) : "r"(fx), "r"(xi[j]));
            hi=(uint32_t)(pr>>32);
          } else if(V==13 || V==14){  // unsigned 32 x 32 -> 64 products (C++), with and without the cosine
            uint64_t pr=C+(uint64_t)(uint32_t)fy*(uint32_t)yi[j]; pr+=(uint64_t)(uint32_t)fx*(uint32_t)xi[j];
            hi=(uint32_t)(pr>>32);
          } else {          // 32-bit halves: lo and hi products, carry by add.cc
            uint32_t l1=(uint32_t)fy*(uint32_t)yi[j], h1=__mulhi(fy,yi[j]);
            uint32_t l2=(uint32_t)fx*(uint32_t)xi[j], h2=__mulhi(fx,xi[j]);
            uint32_t lo, hh;
            asm("{.reg .u32 c1; add.cc.u32 c1, %2, %3; addc.u32 %1, %4, %5; add.cc.u32 %0, c1, %6; addc.u32 %1, %1, %7;}"
                : "=r"(lo), "=r"(hh) : "r"(l1), "r"(l2), "r"(h1), "r"(h2), "r"((uint32_t)C), "r"((uint32_t)(C>>32)));
            hi=hh; (void)lo;
          }
          float a=fmaf(__uint_as_float((hi&0x007FFFFFu)|0x3F800000u),6.2831853f,-6.2831853f);
          if(V==7 || V==12 || V==14) acc[j]=fmaf(T.z,a,acc[j]); else acc[j]=fmaf(T.z,cosr(a),acc[j]);
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
  const char* nm[15]={"doublefloat13","fixedpoint64","noreduce","noreduce-1cos","fixedhi-1cos","fixedhi-1cos-x2","cos-only",
                      "fixedhi-nocos","onewide-1cos","twoindep-1cos","halves-1cos","madwide-1cos","madwide-nocos","unsigned-1cos","unsigned-nocos"};
  for(int v=0;v<15;v++){ for(int rep=0;rep<3;rep++){
    cudaEventRecord(a);
    if(v==0)k<0><<<blocks,TPB>>>(terms,xy,out,2); if(v==1)k<1><<<blocks,TPB>>>(terms,xy,out,2); if(v==2)k<2><<<blocks,TPB>>>(terms,xy,out,2);
    if(v==3)k<3><<<blocks,TPB>>>(terms,xy,out,2); if(v==4)k<4><<<blocks,TPB>>>(terms,xy,out,2);
    if(v==5)k<5><<<blocks,TPB>>>(terms,xy,out,2); if(v==6)k<6><<<blocks,TPB>>>(terms,xy,out,2);
    if(v==7)k<7><<<blocks,TPB>>>(terms,xy,out,2); if(v==8)k<8><<<blocks,TPB>>>(terms,xy,out,2);
    if(v==9)k<9><<<blocks,TPB>>>(terms,xy,out,2); if(v==10)k<10><<<blocks,TPB>>>(terms,xy,out,2);
    if(v==11)k<11><<<blocks,TPB>>>(terms,xy,out,2); if(v==12)k<12><<<blocks,TPB>>>(terms,xy,out,2);
    if(v==13)k<13><<<blocks,TPB>>>(terms,xy,out,2); if(v==14)k<14><<<blocks,TPB>>>(terms,xy,out,2);
    cudaEventRecord(b); CK(cudaEventSynchronize(b)); float ms; cudaEventElapsedTime(&ms,a,b);
    double tp=(double)np*NT*2;
    if(rep==2) printf("%-14s %.3f ms %.3e term-pts/s  per-SM-clk@2070=%.2f\n",nm[v],ms,tp/(ms*1e-3),tp/(ms*1e-3)/nsm/2.07e9);
  }}
  CK(cudaGetLastError()); return 0;
}
