// On-chip ceilings of the current device (libed_probes.so, include/ed_probes.h):
// the rates that bound the H v kernel when DRAM does not.  Each probe runs a
// plain kernel whose work is fixed and counted, after one warm-up launch,
// timed with CUDA events on one stream.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/ed_probes.h"

namespace {

constexpr int kThreads = 256;

// Every thread reads float4 words through L2 only (ld.global.cg), grid-stride
// over an n4-word buffer, `passes` times; the XOR of the words goes to out
// only if it equals a value the data never produces (keeps the loads alive).
__global__ void __launch_bounds__(kThreads) k_read_cg(const float4* buf, int64_t n4, int passes,
                                                      unsigned* out) {
  unsigned acc = 0u;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int p = 0; p < passes; ++p)
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4; i += 4 * stride) {
      float4 v[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int64_t k = i + q * stride;
        v[q] = k < n4 ? __ldcg(buf + k) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int q = 0; q < 4; ++q)
        acc ^= __float_as_uint(v[q].x) ^ __float_as_uint(v[q].y) ^ __float_as_uint(v[q].z) ^
               __float_as_uint(v[q].w);
    }
  if (acc == 0x7F7F7F7Fu) out[0] = acc;
}

// Streaming read (evict-first) of a buffer larger than L2: DRAM read rate.
__global__ void __launch_bounds__(kThreads) k_read_cs(const float4* buf, int64_t n4,
                                                      unsigned* out) {
  unsigned acc = 0u;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4; i += 4 * stride) {
    float4 v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t k = i + q * stride;
      v[q] = k < n4 ? __ldcs(buf + k) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
      acc ^= __float_as_uint(v[q].x) ^ __float_as_uint(v[q].w);
  }
  if (acc == 0x7F7F7F7Fu) out[0] = acc;
}

// Shared memory: each CTA fills 32 KB and reads it back `iters` times with
// conflict-free 16-byte loads (lane l of a warp reads word l of a 512-byte
// run), 4 loads in flight per thread.  The loads are volatile PTX loads
// (ld.volatile), so neither compiler stage can hoist or merge them.
constexpr int kSmemWords = 2048;   // float4 words = 32 KB
__device__ __forceinline__ float4 lds128(const float4* p) {
  float4 v;
  asm volatile("ld.volatile.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "r"((uint32_t)__cvta_generic_to_shared(p)));
  return v;
}
__global__ void __launch_bounds__(kThreads) k_smem_read(int iters, unsigned* out) {
  __shared__ float4 sm[kSmemWords];
  for (int i = threadIdx.x; i < kSmemWords; i += blockDim.x)
    sm[i] = make_float4((float)i, (float)(i + 1), (float)(i + 2), (float)(i + 3));
  __syncthreads();
  unsigned acc = 0u;
  int idx = threadIdx.x;
  for (int it = 0; it < iters; ++it) {
    float4 v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) v[q] = lds128(sm + ((idx + q * kThreads) & (kSmemWords - 1)));
#pragma unroll
    for (int q = 0; q < 4; ++q) acc += __float_as_uint(v[q].x) ^ __float_as_uint(v[q].w);
    idx = (idx + 4 * kThreads) & (kSmemWords - 1);
  }
  if (acc == 0x7F7F7F7Fu) out[0] = acc;
}

// FMA throughput: 8 independent chains per thread, `iters` rounds.
__global__ void __launch_bounds__(kThreads) k_ffma(int iters, float a, float b, float* out) {
  float x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = (float)(threadIdx.x + k);
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = fmaf(x[k], a, b);
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  if (s == 1234.5f) out[0] = s;
}

__device__ __forceinline__ unsigned long long ffma2(unsigned long long a, unsigned long long b,
                                                   unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__global__ void __launch_bounds__(kThreads) k_ffma2(int iters, float a, float b, float* out) {
  unsigned long long x[8], pa, pb;
  asm("mov.b64 %0, {%1, %2};" : "=l"(pa) : "f"(a), "f"(a));
  asm("mov.b64 %0, {%1, %2};" : "=l"(pb) : "f"(b), "f"(b));
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const float f = (float)(threadIdx.x + k);
    asm("mov.b64 %0, {%1, %2};" : "=l"(x[k]) : "f"(f), "f"(f));
  }
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = ffma2(x[k], pa, pb);
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    float lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(x[k]));
    s += lo + hi;
  }
  if (s == 1234.5f) out[0] = s;
}

__global__ void __launch_bounds__(kThreads) k_dfma(int iters, double a, double b, double* out) {
  double x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = (double)(threadIdx.x + k);
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  if (s == 1234.5) out[0] = s;
}

struct Timer {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t init() {
    cudaError_t e = cudaEventCreate(&e0);
    return e == cudaSuccess ? cudaEventCreate(&e1) : e;
  }
  ~Timer() {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  }
};

#define PCK(call)                                 \
  do {                                            \
    cudaError_t e_ = (call);                      \
    if (e_ != cudaSuccess) return (int)e_;        \
  } while (0)

// Times launch() (after one warm-up launch); returns milliseconds in *ms.
template <typename F>
int time_ms(Timer& t, F launch, float* ms) {
  launch();
  PCK(cudaGetLastError());
  PCK(cudaEventRecord(t.e0));
  launch();
  PCK(cudaGetLastError());
  PCK(cudaEventRecord(t.e1));
  PCK(cudaEventSynchronize(t.e1));
  return (int)cudaEventElapsedTime(ms, t.e0, t.e1);
}

}  // namespace

extern "C" int ed_probe_ceilings(ed_ceilings* out) {
  if (!out) return (int)cudaErrorInvalidValue;
  int dev = 0, sms = 0;
  PCK(cudaGetDevice(&dev));
  PCK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  Timer t;
  PCK(t.init());
  unsigned* sink = nullptr;
  PCK(cudaMalloc(&sink, 64));
  float* fsink = reinterpret_cast<float*>(sink);
  double* dsink = reinterpret_cast<double*>(sink);
  const int grid = sms * 8;   // 8 CTAs of 256 threads per SM
  float ms = 0.f;
  int rc = 0;
  // L2: a 32 MB buffer (a quarter of the L2), written once, read 100 times
  {
    const int64_t bytes = 32ll << 20, n4 = bytes / 16;
    const int passes = 100;
    float4* buf = nullptr;
    if ((rc = (int)cudaMalloc(&buf, bytes)) != 0) { cudaFree(sink); return rc; }
    cudaMemset(buf, 1, bytes);
    rc = time_ms(t, [&] { k_read_cg<<<grid, kThreads>>>(buf, n4, passes, sink); }, &ms);
    cudaFree(buf);
    if (rc) { cudaFree(sink); return rc; }
    out->l2_read_gbs = (double)bytes * passes / (ms * 1e-3) / 1e9;
  }
  // DRAM: one streaming read of 4 GB
  {
    const int64_t bytes = 4ll << 30, n4 = bytes / 16;
    float4* buf = nullptr;
    if ((rc = (int)cudaMalloc(&buf, bytes)) != 0) { cudaFree(sink); return rc; }
    cudaMemset(buf, 1, bytes);
    rc = time_ms(t, [&] { k_read_cs<<<grid, kThreads>>>(buf, n4, sink); }, &ms);
    cudaFree(buf);
    if (rc) { cudaFree(sink); return rc; }
    out->hbm_read_gbs = (double)bytes / (ms * 1e-3) / 1e9;
  }
  // shared memory
  {
    const int iters = 4096;
    rc = time_ms(t, [&] { k_smem_read<<<grid, kThreads>>>(iters, sink); }, &ms);
    if (rc) { cudaFree(sink); return rc; }
    out->smem_read_gbs = (double)grid * kThreads * iters * 4 * 16 / (ms * 1e-3) / 1e9;
  }
  // FMA rates (2 flops per FMA, 8 chains per thread)
  {
    const int iters = 2048;
    rc = time_ms(t, [&] { k_ffma<<<grid, kThreads>>>(iters, 0.999f, 0.001f, fsink); }, &ms);
    if (rc) { cudaFree(sink); return rc; }
    out->fp32_fma_tflops = 2.0 * 8 * iters * (double)grid * kThreads / (ms * 1e-3) / 1e12;
    rc = time_ms(t, [&] { k_ffma2<<<grid, kThreads>>>(iters, 0.999f, 0.001f, fsink); }, &ms);
    if (rc) { cudaFree(sink); return rc; }
    out->fp32x2_fma_tflops = 4.0 * 8 * iters * (double)grid * kThreads / (ms * 1e-3) / 1e12;
    const int diters = 1024;   // long enough that launch and tail do not count
    rc = time_ms(t, [&] { k_dfma<<<grid, kThreads>>>(diters, 0.999, 0.001, dsink); }, &ms);
    if (rc) { cudaFree(sink); return rc; }
    out->fp64_fma_tflops = 2.0 * 8 * diters * (double)grid * kThreads / (ms * 1e-3) / 1e12;
  }
  out->sms = sms;
  cudaFree(sink);
  return 0;
}

namespace {

// Access patterns of 16-byte shared-memory loads, one warp, for reading the
// wavefronts each pattern costs with a profiler
// (l1tex__data_pipe_lsu_wavefronts_mem_shared_op_ld.sum over
// smsp__inst_executed_op_shared_ld.sum).  Every index is masked to the
// 256 float4 words of the buffer.
//   MODE 0: one address for all lanes (a broadcast)
//   MODE 1: 32 consecutive words (conflict-free)
//   MODE 2: every quarter warp 2-way in four bank groups, the two quarters
//           of each half warp in disjoint bank groups (8 wavefronts if
//           conflicts are resolved per quarter warp, 4 if per half warp)
//   MODE 3: the eight lanes of every quarter warp in one bank group, the
//           four quarters at the same addresses (8-way)
template <int MODE>
__global__ void __launch_bounds__(32) k_probe_lds(float* out, int salt) {
  __shared__ float4 buf[256];
  const int l = threadIdx.x;
  for (int i = l; i < 256; i += 32) buf[i] = make_float4(i, i + 1, i + 2, i + 3);
  __syncthreads();
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int it = 0; it < 1024; ++it) {
    int idx;
    if (MODE == 0) idx = (it * 7 + salt) & 255;
    else if (MODE == 1) idx = (l + 32 * (it & 7)) & 255;
    else if (MODE == 2)
      idx = ((((l & 7) >> 1) + 4 * ((l >> 3) & 1)) + 8 * ((l & 1) + 2 * (l >> 4)) + 32 * (it & 3)) & 255;
    else idx = ((l & 7) * 8 + (it & 7)) & 255;
    const float4 v = buf[idx];
    acc.x += v.x; acc.y += v.y; acc.z += v.z; acc.w += v.w;
  }
  out[l] = acc.x + acc.y + acc.z + acc.w;
}

}  // namespace

extern "C" int ed_probe_shared_loads(void) {
  float* d = nullptr;
  cudaError_t e = cudaMalloc(&d, 32 * sizeof(float));
  if (e != cudaSuccess) return (int)e;
  k_probe_lds<0><<<1, 32>>>(d, 3);
  k_probe_lds<1><<<1, 32>>>(d, 3);
  k_probe_lds<2><<<1, 32>>>(d, 3);
  k_probe_lds<3><<<1, 32>>>(d, 3);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  cudaFree(d);
  return (int)e;
}
