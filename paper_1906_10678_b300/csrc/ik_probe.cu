// Peak probes: the rates that bound the boolean set propagation, measured on
// the device itself.  No datasheet gives them: the propagation's inner step
// is shared-memory word loads, funnel shifts and 3-input logic ops (LOP3), so
// its rooflines are the SM's issue rate for those instructions and its
// shared-memory word-load rate, both multiplied by the SMs and the clock the
// probe sees.
//
// Each probe is a throughput loop: every thread runs several independent
// dependency chains of one instruction kind, enough warps per SM to hide its
// latency, and the result is folded into a value that is written only when
// it takes an impossible value (so nothing can be optimised away).  The
// instructions are inline PTX, so each counted op is one instruction.

#include <cuda_runtime.h>
#include <stdint.h>

#include "ik_internal.h"

namespace {

constexpr int kProbeThreads = 256;
constexpr int kUnroll = 16;

// Elapsed SM clocks and nanoseconds of the first block, for the effective clock.
__device__ __forceinline__ void stamp(long long* t, int slot) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    long long ns;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(ns));
    t[2 * slot] = clock64();
    t[2 * slot + 1] = ns;
  }
}

// 8 chains of a ^ (b & c) (LUT 0x78): 8 LOP3 per unrolled step and thread.
__global__ void __launch_bounds__(kProbeThreads) k_probe_lop3(int iters, uint32_t seed, uint32_t* sink,
                                                             long long* t) {
  stamp(t, 0);
  uint32_t a[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) a[i] = seed * (threadIdx.x + 1 + 97 * i) ^ (blockIdx.x << i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int i = 0; i < 8; ++i)
        asm volatile("lop3.b32 %0, %0, %1, %2, 0x78;" : "+r"(a[i]) : "r"(a[(i + 1) & 7]), "r"(a[(i + 3) & 7]));
    }
  }
  __syncthreads();
  stamp(t, 1);
  uint32_t x = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) x ^= a[i];
  if (x == 0x9e3779b9u && seed == 0u) sink[blockIdx.x] = x;
}

// 8 chains of funnel shifts (shf.r.wrap): 8 SHF per unrolled step and thread.
__global__ void __launch_bounds__(kProbeThreads) k_probe_shf(int iters, uint32_t seed, uint32_t* sink,
                                                            long long* t) {
  stamp(t, 0);
  uint32_t a[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) a[i] = seed * (threadIdx.x + 1 + 97 * i) ^ (blockIdx.x << i);
  const uint32_t sh = (seed >> 3) | 1u;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int i = 0; i < 8; ++i)
        asm volatile("shf.r.wrap.b32 %0, %0, %1, %2;" : "+r"(a[i]) : "r"(a[(i + 1) & 7]), "r"(sh + i));
    }
  }
  __syncthreads();
  stamp(t, 1);
  uint32_t x = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) x ^= a[i];
  if (x == 0x9e3779b9u && seed == 0u) sink[blockIdx.x] = x;
}

// Conflict-free 32-bit shared-memory loads: lane l of a warp reads words
// base + 64 u + l and base + 64 u + 32 + l (one word per bank), kUnroll x 2
// loads per step, folded two at a time by one LOP3.
constexpr int kSmemWords = 8192;  // 32 KiB per block

__global__ void __launch_bounds__(kProbeThreads) k_probe_lds(int iters, uint32_t seed, uint32_t* sink,
                                                            long long* t) {
  __shared__ uint32_t s[kSmemWords];
  for (int i = threadIdx.x; i < kSmemWords; i += blockDim.x) s[i] = seed * (i + 1);
  __syncthreads();
  stamp(t, 0);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t acc0 = 0, acc1 = 0;
  const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(s);
  for (int it = 0; it < iters; ++it) {
    // a multiple of 32 words, so the warp's 32 lanes hit 32 distinct banks;
    // the largest word read is 223 * 32 + 64 * 15 + 32 + 31 = 8159 < kSmemWords
    const uint32_t base = (uint32_t)((it * 7 + warp) % 224) * 32u + (uint32_t)lane;
    const uint32_t a = sbase + 4u * base;
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      uint32_t v0, v1;
      asm volatile("ld.volatile.shared.b32 %0, [%1];" : "=r"(v0) : "r"(a + 256u * u));
      asm volatile("ld.volatile.shared.b32 %0, [%1];" : "=r"(v1) : "r"(a + 256u * u + 128u));
      asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(acc0) : "r"(v0), "r"(v1));
    }
    acc1 += acc0;
  }
  __syncthreads();
  stamp(t, 1);
  if ((acc0 ^ acc1) == 0x9e3779b9u && seed == 0u) sink[blockIdx.x] = acc0;
}

}  // namespace

extern "C" {

int ik_probe_peak(int kind, int blocks_per_sm, int iters, void* cuda_stream, double* ops_per_s_out,
                  double* ms_out, double* sm_mhz_out) {
  if (kind < 0 || kind > 2 || blocks_per_sm < 1 || blocks_per_sm > 8 || iters < 1 || iters > (1 << 24))
    return IK_ERR_ARG;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return IK_ERR_CUDA;
  const int blocks = sms * blocks_per_sm;
  uint32_t* sink = nullptr;
  long long* t = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = IK_OK;
  if (cudaMalloc(&sink, (size_t)blocks * 4) != cudaSuccess || cudaMalloc(&t, 4 * sizeof(long long)) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    rc = IK_ERR_CUDA;
  } else {
    const uint32_t seed = 0x2545f491u;
    cudaEventRecord(e0, st);
    if (kind == 0) k_probe_lop3<<<blocks, kProbeThreads, 0, st>>>(iters, seed, sink, t);
    else if (kind == 1) k_probe_shf<<<blocks, kProbeThreads, 0, st>>>(iters, seed, sink, t);
    else k_probe_lds<<<blocks, kProbeThreads, 0, st>>>(iters, seed, sink, t);
    cudaEventRecord(e1, st);
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
      rc = IK_ERR_CUDA;
    } else {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      long long h[4] = {0, 0, 0, 0};
      cudaMemcpy(h, t, sizeof(h), cudaMemcpyDeviceToHost);
      // ops per thread and iteration: 8 chains x kUnroll for the ALU probes,
      // 2 x kUnroll word loads for the shared-memory probe
      const double per = (kind == 2 ? 2.0 : 8.0) * kUnroll;
      const double ops = (double)blocks * kProbeThreads * (double)iters * per;
      if (ops_per_s_out) *ops_per_s_out = ops / (ms * 1e-3);
      if (ms_out) *ms_out = ms;
      if (sm_mhz_out) *sm_mhz_out = (h[3] > h[1]) ? (double)(h[2] - h[0]) / (double)(h[3] - h[1]) * 1e3 : 0.0;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(sink);
  cudaFree(t);
  return rc;
}

}  // extern "C"
