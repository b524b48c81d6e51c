// wave_misfit_static: the FP64 misfit of `misfit`, for callers that cannot
// allocate device memory.
//
// Who needs it: code that runs where no allocation may happen -- a plugin
// inside a host framework that has already reserved all device memory for
// its own allocator, a latency-critical loop that must not take the
// allocator's locks or trigger a device synchronisation, or a caller that
// simply has no scratch buffer to hand.  `misfit` asks such callers for a
// scratch buffer of partial sums; this variant keeps those partial sums in a
// fixed array that lives in the library's own device memory instead.
//
// The array is a file-scope static __device__ array.  Every GPU that loads
// the library holds it until the process exits, and every call on that GPU
// shares it: two calls whose kernels overlap on the GPU (different streams,
// no ordering between them) race on it and give wrong sums.  The array keeps
// whatever the previous call left; nothing has to start at zero because the
// first kernel writes every partial sum that the second kernel reads.
//
// The first call on a device looks up the array's device address with
// cudaGetSymbolAddress (with that device current) and caches it together with
// the device's current context; a later call in another context (after a
// device reset) looks it up again.  Make the first call on a device before
// any stream capture begins.  The call itself never allocates: no
// cudaMalloc, cudaFree or allocating library routine.
#include <cuda.h>   // CUcontext (cuCtxGetCurrent is looked up at run time)

#include <mutex>

#include "wave_internal.cuh"

namespace {

// One partial sum per block of kChunk samples: the array bounds the input at
// kStaticParts * kChunk samples (33,554,432 FP32 samples, 32 KB of scratch).
constexpr int kStaticParts = 4096;
constexpr int64_t kChunk = 8192;
constexpr int kThreads = 256;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_misfit_partials[kStaticParts];

std::mutex g_addr_mutex;
double* g_addr[kMaxDevices] = {nullptr};
CUcontext g_ctx[kMaxDevices] = {nullptr};   // context the cached address belongs to

typedef CUresult (*CtxGetCurrent)(CUcontext*);

// The calling thread's current context (null if it cannot be read).
CUcontext current_context() {
  static CtxGetCurrent fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<CtxGetCurrent>(p);
  });
  CUcontext c = nullptr;
  if (fn) fn(&c);
  return c;
}

__device__ __forceinline__ double block_reduce(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (warp == 0) {
    s = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  }
  return s;
}

// Block b sums (syn - obs)^2 over samples [b*kChunk, min((b+1)*kChunk, n)).
__global__ void __launch_bounds__(kThreads)
chunk_partial_kernel(const float* __restrict__ syn, const float* __restrict__ obs, int64_t n,
                     double* __restrict__ partials) {
  __shared__ double red[kThreads / 32];
  const int64_t begin = (int64_t)blockIdx.x * kChunk;
  const int64_t end = begin + kChunk < n ? begin + kChunk : n;
  double acc = 0.0;
  for (int64_t i = begin + threadIdx.x; i < end; i += kThreads) {
    const double d = (double)syn[i] - (obs ? (double)obs[i] : 0.0);
    acc = fma(d, d, acc);
  }
  const double s = block_reduce(acc, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads)
chunk_final_kernel(const double* __restrict__ partials, int nparts, double scale, double* out) {
  __shared__ double red[kThreads / 32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < nparts; i += kThreads) acc += partials[i];
  const double s = block_reduce(acc, red);
  if (threadIdx.x == 0) out[0] = scale * s;
}

// Device address of the static array on the current device: looked up once
// per device and context.
cudaError_t scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_addr_mutex);
  const CUcontext ctx = current_context();
  if (g_addr[dev] == nullptr || ctx == nullptr || ctx != g_ctx[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_misfit_partials);
    if (e != cudaSuccess) return e;
    g_addr[dev] = static_cast<double*>(p);
    g_ctx[dev] = current_context();   // the lookup may have made the primary context current
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" wave_status wave_misfit_static(const float* syn_dev, const float* obs_dev, int64_t count, double dt,
                                          double weight, double* out_dev, void* stream) {
  if (!out_dev || count < 0 || !(dt > 0)) return WAVE_EINVAL;
  if (count > 0 && !syn_dev) return WAVE_EINVAL;
  if (count > (int64_t)kStaticParts * kChunk) return WAVE_EINVAL;  // beyond the static scratch
  double* partials = nullptr;
  cudaError_t e = scratch_address(&partials);
  if (e != cudaSuccess) {
    wave::set_last_error("cudaGetSymbolAddress (static misfit scratch)", e);
    return WAVE_ECUDA;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int nparts = (int)((count + kChunk - 1) / kChunk);
  if (nparts > 0) {
    chunk_partial_kernel<<<nparts, kThreads, 0, s>>>(syn_dev, obs_dev, count, partials);
    wave::count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) {
      wave::set_last_error("chunk_partial_kernel launch", e);
      return WAVE_ECUDA;
    }
  }
  chunk_final_kernel<<<1, kThreads, 0, s>>>(partials, nparts, 0.5 * weight * dt, out_dev);
  wave::count_launch();
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    wave::set_last_error("chunk_final_kernel launch", e);
    return WAVE_ECUDA;
  }
  return WAVE_OK;
}
