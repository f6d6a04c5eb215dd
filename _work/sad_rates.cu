// sad_rates.cu -- throughput of candidate packed-SAD formulations on the
// GPU it runs on: 16 independent accumulator chains per thread, 8 CTAs of
// 256 threads per SM, ITERS iterations; prints ops per SM per clock (at
// 2070 MHz).  Standalone program, not part of the library:
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o sad_rates sad_rates.cu && ./sad_rates
// Run under ncu with pipe counters to see how many instructions, on which
// pipe, each formulation costs.
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>

#define ITERS 4096

__device__ __forceinline__ uint32_t v4add(uint32_t a, uint32_t b, uint32_t c){uint32_t d;asm volatile("vabsdiff4.u32.u32.u32.add %0,%1,%2,%3;":"=r"(d):"r"(a),"r"(b),"r"(c));return d;}
__device__ __forceinline__ uint32_t v2add(uint32_t a, uint32_t b, uint32_t c){uint32_t d;asm volatile("vabsdiff2.u32.u32.u32.add %0,%1,%2,%3;":"=r"(d):"r"(a),"r"(b),"r"(c));return d;}
__device__ __forceinline__ uint32_t v4(uint32_t a, uint32_t b){return __vabsdiffu4(a,b);}
__device__ __forceinline__ uint32_t v2(uint32_t a, uint32_t b){return __vabsdiffu2(a,b);}
__device__ __forceinline__ uint32_t max2(uint32_t a, uint32_t b){uint32_t d;asm volatile("max.u16x2 %0,%1,%2;":"=r"(d):"r"(a),"r"(b));return d;}
__device__ __forceinline__ uint32_t min2(uint32_t a, uint32_t b){uint32_t d;asm volatile("min.u16x2 %0,%1,%2;":"=r"(d):"r"(a),"r"(b));return d;}

template<int K> __global__ void __launch_bounds__(256) probe(uint32_t* out, uint32_t a0, uint32_t b){
  uint32_t x[16], acc[16];
  for(int j=0;j<16;++j){x[j]=a0^(j*0x01030507u)^threadIdx.x; acc[j]=j;}
  for(int it=0;it<ITERS;++it){
#pragma unroll
    for(int j=0;j<16;++j){
      if(K==0) acc[j]=v4add(x[j],b,acc[j]);                 // vabsdiff4.add
      else if(K==1) acc[j]=v2add(x[j],b,acc[j]);            // vabsdiff2.add
      else if(K==2) acc[j]=__dp4a(v4(x[j],b),0x01010101u,acc[j]);  // absdiff bytes + dp4a
      else if(K==3) acc[j]=acc[j]+max2(x[j],b)-min2(x[j],b);  // packed 16-bit |a-b| accumulate
      else if(K==4) acc[j]=acc[j]+v2(x[j],b);                // vabsdiff2 (no add) + 32-bit add of packed halves
      else if(K==5) acc[j]=min(acc[j]^x[j], b+j);            // min.u32 + xor
      else if(K==6) acc[j]=__sad(x[j],b,acc[j]);             // scalar sad
      else if(K==7) { uint32_t d=v4(x[j],b); acc[j]=acc[j]+d; }   // vabsdiff4 (no add) + packed byte add (wraps)
    }
    b += 0x01010101u;
  }
  uint32_t s=0; for(int j=0;j<16;++j) s+=acc[j];
  if(s==0xdeadbeef) out[0]=s;
}

template<int K> float run(int blocks, uint32_t* out){
  cudaEvent_t a,b; cudaEventCreate(&a); cudaEventCreate(&b);
  probe<K><<<blocks,256>>>(out,1,0x12345678); cudaDeviceSynchronize();
  cudaEventRecord(a); probe<K><<<blocks,256>>>(out,1,0x12345678); cudaEventRecord(b); cudaEventSynchronize(b);
  float ms; cudaEventElapsedTime(&ms,a,b); return ms;
}

int main(){
  int dev=0; cudaDeviceProp p; cudaGetDeviceProperties(&p,dev);
  int sms=p.multiProcessorCount;
  uint32_t* out; cudaMalloc(&out,4);
  const char* names[8]={"vabsdiff4.add","vabsdiff2.add","vabsdiff4+dp4a","max/min.u16x2+add","vabsdiff2+add","min.u32+xor","sad","vabsdiff4+add"};
  int blocks=sms*8;
  float ms[8];
  ms[0]=run<0>(blocks,out); ms[1]=run<1>(blocks,out); ms[2]=run<2>(blocks,out); ms[3]=run<3>(blocks,out);
  ms[4]=run<4>(blocks,out); ms[5]=run<5>(blocks,out); ms[6]=run<6>(blocks,out); ms[7]=run<7>(blocks,out);
  for(int k=0;k<8;++k){
    double ops=(double)blocks*256*ITERS*16;
    printf("%-20s %.3f ms  %.1f ops/SM/clk(@2070MHz)\n",names[k],ms[k],ops/(ms[k]*1e-3)/sms/2.07e9);
  }
  printf("err=%s SMs=%d\n",cudaGetErrorString(cudaGetLastError()),sms);
  return 0;
}
