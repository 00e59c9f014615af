// ed_double_occupation_static: the double-occupancy reduction of
// ed_double_occupation with its scratch memory in a fixed device array of
// this library instead of a per-call allocation.  It serves callers that
// must not allocate device memory while they run: code inside a region whose
// device memory is fixed up front (a latency-critical step loop, a memory
// budget enforced by the host application), or hosts that cannot call
// cudaMalloc at that point.
#include <cuda_runtime.h>

#include <mutex>

#include "ctx.h"

namespace ed {

namespace {

constexpr int kStaticSlots = kMaxSites + 1;          // total + one per site
constexpr int kStaticBlocks = 1024;                   // per-block partial rows
constexpr int64_t kStaticChunk = 65536;               // elements per block
constexpr int64_t kStaticMaxElems = kStaticChunk * kStaticBlocks;  // 67,108,864
constexpr int kStaticMaxDevices = 64;

// Partial sums of every block (kStaticBlocks rows) followed by the final
// sums (one row): (1024 + 1) * 17 doubles = 139,400 bytes per device.
__device__ __align__(256) double g_docc_scratch[(kStaticBlocks + 1) * kStaticSlots];

std::mutex g_scratch_mutex;
double* g_scratch_ptr[kStaticMaxDevices] = {nullptr};

// Device address of the scratch array on the current device, looked up once
// per device.  In host code the array's name is only a host-side stand-in, so
// the address must come from cudaGetSymbolAddress.
cudaError_t scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kStaticMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_docc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

template <typename C>
__global__ void __launch_bounds__(256)
k_docc_sites_static(const C* psi, SectorDev sd, double* scratch) {
  __shared__ double red[32][kStaticSlots];
  const int64_t D = (int64_t)sd.dim_up * sd.dim_dn;
  const int64_t i0 = blockIdx.x * kStaticChunk;
  const int64_t i1 = i0 + kStaticChunk < D ? i0 + kStaticChunk : D;
  double v[kStaticSlots];
#pragma unroll
  for (int i = 0; i < kStaticSlots; ++i) v[i] = 0.0;
  for (int64_t t = i0 + threadIdx.x; t < i1; t += blockDim.x) {
    const int u = (int)(t / sd.dim_dn);
    const int d = (int)(t - (int64_t)u * sd.dim_dn);
    const C p = psi[t];
    const double q = (double)p.x * p.x + (double)p.y * p.y;
    const uint32_t both = sd.up_word[u] & sd.dn_word[d];
    v[0] += __popc(both) * q;
#pragma unroll
    for (int i = 0; i < kMaxSites; ++i)
      if ((both >> i) & 1u) v[1 + i] += q;
  }
  // warp sums, then one warp sums the warps in a fixed order
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < kStaticSlots; ++i) {
    double s = v[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) red[wid][i] = s;
  }
  __syncthreads();
  if (threadIdx.x < kStaticSlots) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w][threadIdx.x];
    scratch[(size_t)blockIdx.x * kStaticSlots + threadIdx.x] = s;   // every slot rewritten
  }
}

__global__ void k_docc_sum_static(double* scratch, int nblk) {
  const int i = threadIdx.x;
  if (i >= kStaticSlots) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += scratch[(size_t)b * kStaticSlots + i];
  scratch[(size_t)kStaticBlocks * kStaticSlots + i] = s;
}

}  // namespace
}  // namespace ed

using namespace ed;

extern "C" ed_status ed_double_occupation_static(ed_ctx* ctx, const void* psi, ed_dtype dtype,
                                                 double* d_avg, double* d_site, void* stream) {
  if (!ctx || !psi || !d_avg) return fail(ctx, ED_ERR_ARG, "NULL argument");
  if (dtype != ED_C128 && dtype != ED_C64) return fail(ctx, ED_ERR_ARG, "bad dtype");
  const int64_t D = ctx->dim_up * ctx->dim_dn;
  if (D > kStaticMaxElems)
    return fail(ctx, ED_ERR_UNSUPPORTED,
                "ed_double_occupation_static: sector dimension " + std::to_string(D) +
                    " exceeds its fixed scratch (at most 67,108,864 elements); use "
                    "ed_double_occupation");
  if (!ctx->lattice_set || !ctx->sec.uploaded)
    return fail(ctx, ED_ERR_STATE,
                "ed_double_occupation_static needs the context's tables on the device "
                "already (call any GPU entry point on this context first)");
  if (!is_device_ptr(psi)) return fail(ctx, ED_ERR_ARG, "psi must be a device pointer");
  // the tables and psi must live on the current device, whose scratch array
  // the kernels below use
  if (ed_status e = check_device(ctx, {psi})) return e;
  double* scratch = nullptr;
  CK(ctx, scratch_address(&scratch));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int nblk = (int)((D + kStaticChunk - 1) / kStaticChunk);
  if (dtype == ED_C128)
    k_docc_sites_static<double2><<<nblk, 256, 0, s>>>(static_cast<const double2*>(psi),
                                                       ctx->sec.dev, scratch);
  else
    k_docc_sites_static<float2><<<nblk, 256, 0, s>>>(static_cast<const float2*>(psi),
                                                      ctx->sec.dev, scratch);
  CK(ctx, cudaGetLastError());
  k_docc_sum_static<<<1, 32, 0, s>>>(scratch, nblk);
  CK(ctx, cudaGetLastError());
  double h[kStaticSlots];
  CK(ctx, cudaMemcpyAsync(h, scratch + (size_t)kStaticBlocks * kStaticSlots, sizeof(h),
                          cudaMemcpyDeviceToHost, s));
  CK(ctx, cudaStreamSynchronize(s));
  *d_avg = h[0] / ctx->Ns;
  if (d_site)
    for (int i = 0; i < ctx->Ns; ++i) d_site[i] = h[1 + i];
  return ED_OK;
}
