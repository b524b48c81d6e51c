// Auxiliary kernels of libwave: coefficient preparation (Eq. FDstencil1/2
// prefactors and the Sec. 2.3 material interpolation), the stability bound,
// layout conversions, the per-step source/receiver kernel (Algorithm 1's
// computeAdjointSource and the injection of f and k f_adj, Eq.
// superposedforce), the FP64 misfit / norm reductions (Eq. cost1), the
// choice of k, the final scaling K~ = acc / (2 k dt) (Eq. superposedkernel)
// and the source time functions (Eq. source2 and the Ricker wavelet).
#include <atomic>
#include <math.h>
#include <mutex>
#include <set>
#include <utility>

#include "wave_internal.cuh"

namespace wave {

static std::atomic<uint64_t> g_launches{0};

// Dynamic shared-memory limit of a kernel, set once per device (the attribute
// is per device; setting it again while the kernel runs is not allowed).
cudaError_t set_smem_limit_once(const void* func, int bytes) {
  static std::mutex mu;
  static std::set<std::pair<int, const void*>> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    note_error("cudaGetDevice", e);
    return e;
  }
  std::lock_guard<std::mutex> lock(mu);
  if (done.count({dev, func})) return cudaSuccess;
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) done.insert({dev, func});
  else note_error("cudaFuncSetAttribute(max dynamic shared memory)", e);
  return e;
}
void count_launch(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }
uint64_t launches() { return g_launches.load(std::memory_order_relaxed); }

static unsigned grid_for(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  if (b > (1LL << 20)) b = 1LL << 20;   // grid-stride loops cover the rest
  if (b < 1) b = 1;
  return (unsigned)b;
}

// ---- materials of the acoustic model (Sec. 2.3) ---------------------------
constexpr double kRhoAir = 1.204, kKappaAir = 1.419e5;
constexpr double kRhoSolid = 2643.0, kKappaSolid = 6.87e8;

__global__ void coef_velocity_kernel(Geom g, const float* __restrict__ v, float dt_over_h,
                                     float* __restrict__ coef) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.cells;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t x = i % g.px, row = i / g.px;
    float c = 0.f;
    if (x < g.nx) {
      const float s = v[row * g.nx + x] * dt_over_h;
      c = s * s;
    }
    coef[i] = c;
  }
}

__global__ void coef_density_kernel(Geom g, const float* __restrict__ gamma, double dt2_over_h2,
                                    float* __restrict__ ca, float* __restrict__ b) {
  const double a_air = 1.0 / kKappaAir, da = 1.0 / kKappaSolid - 1.0 / kKappaAir;
  const double b_air = 1.0 / kRhoAir, db = 1.0 / kRhoSolid - 1.0 / kRhoAir;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.cells;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t x = i % g.px, row = i / g.px;
    float cav = 0.f, bv = 1.f;  // padding: no mass term, unit (finite) material
    if (x < g.nx) {
      const double gm = gamma[row * g.nx + x];
      cav = (float)(dt2_over_h2 / (a_air + gm * da));
      bv = (float)(b_air + gm * db);
    }
    ca[i] = cav;
    b[i] = bv;
  }
}

cudaError_t launch_coef_velocity(const Geom& g, const float* v, float dt_over_h, float* coef, cudaStream_t s) {
  coef_velocity_kernel<<<grid_for(g.cells, 256), 256, 0, s>>>(g, v, dt_over_h, coef);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_coef_density(const Geom& g, const float* gamma, double dt2_over_h2, float* ca, float* b,
                                cudaStream_t s) {
  coef_density_kernel<<<grid_for(g.cells, 256), 256, 0, s>>>(g, gamma, dt2_over_h2, ca, b);
  count_launch();
  return cudaGetLastError();
}

// ---- stability bound ---------------------------------------------------------
// Gershgorin bound of dt^2 * rho(A^-1 L): velocity coef_i * ndim * S;
// density 2 ca_i sum_faces b_f (boundary faces: b_i under Dirichlet, 0 under
// Neumann).  Leapfrog is stable while it is <= 4.
__device__ __forceinline__ float hmean(float a, float b) { return 2.f * a * b / (a + b); }

// max that keeps a NaN (fmaxf drops it), so a NaN parameter reaches the check
__device__ __forceinline__ float max_keep_nan(float a, float b) {
  return (a != a || b != b) ? __int_as_float(0x7fffffff) : fmaxf(a, b);
}

__global__ void stability_kernel(Geom g, int physics, float sym, const float* __restrict__ coef,
                                 const float* __restrict__ b, float* __restrict__ partial) {
  __shared__ float red[256];
  float m = 0.f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.cells;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t x = i % g.px;
    if (x >= g.nx) continue;
    float val;
    if (physics == WAVE_VELOCITY) {
      val = coef[i] * sym;
    } else {
      const int64_t row = i / g.px, y = row % g.ny, z = row / g.ny;
      const float bi = b[i];
      float s = 0.f;
      const float edge = g.bc == WAVE_DIRICHLET ? bi : 0.f;
      s += x > 0 ? hmean(bi, b[i - 1]) : edge;
      s += x < g.nx - 1 ? hmean(bi, b[i + 1]) : edge;
      s += y > 0 ? hmean(bi, b[i - g.px]) : edge;
      s += y < g.ny - 1 ? hmean(bi, b[i + g.px]) : edge;
      if (g.ndim == 3) {
        s += z > 0 ? hmean(bi, b[i - g.plane]) : edge;
        s += z < g.nz - 1 ? hmean(bi, b[i + g.plane]) : edge;
      }
      val = 2.f * coef[i] * s;
    }
    m = max_keep_nan(m, val);
  }
  red[threadIdx.x] = m;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] = max_keep_nan(red[threadIdx.x], red[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void max_final_kernel(const float* __restrict__ partial, int n, float* out) {
  __shared__ float red[256];
  float m = 0.f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) m = max_keep_nan(m, partial[i]);
  red[threadIdx.x] = m;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] = max_keep_nan(red[threadIdx.x], red[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = red[0];
}

cudaError_t launch_stability(const Geom& g, int physics, double sym, const float* coef, const float* b,
                             float* partial, int nparts, cudaStream_t s) {
  stability_kernel<<<nparts, 256, 0, s>>>(g, physics, (float)sym, coef, b, partial);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_max_final(const float* partial, int nparts, float* out, cudaStream_t s) {
  max_final_kernel<<<1, 256, 0, s>>>(partial, nparts, out);
  count_launch();
  return cudaGetLastError();
}

// ---- layout conversions --------------------------------------------------------
__global__ void pitch_indices_kernel(Geom g, const int64_t* __restrict__ flat, int32_t n,
                                     int64_t* __restrict__ pitched) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int64_t i = flat[t];
  const int64_t total = g.nx * g.ny * g.nz;
  pitched[t] = (i < 0 || i >= total) ? -1 : (i / g.nx) * g.px + (i % g.nx);
}

cudaError_t launch_pitch_indices(const Geom& g, const int64_t* flat, int32_t n, int64_t* pitched, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  pitch_indices_kernel<<<grid_for(n, 256), 256, 0, s>>>(g, flat, n, pitched);
  count_launch();
  return cudaGetLastError();
}

template <typename T>
__global__ void dense_to_pitched_kernel(Geom g, const float* __restrict__ dense, T* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.cells;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t x = i % g.px, row = i / g.px;
    out[i] = T(x < g.nx ? dense[row * g.nx + x] : 0.f);
  }
}

template <typename T>
__global__ void pitched_to_dense_kernel(Geom g, const T* __restrict__ in, float* __restrict__ dense) {
  const int64_t total = g.nx * g.ny * g.nz;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    dense[i] = float(in[(i / g.nx) * g.px + (i % g.nx)]);
  }
}

cudaError_t launch_dense_to_pitched(const Geom& g, const float* dense, void* pitched, int storage, cudaStream_t s) {
  const unsigned grid = grid_for(g.cells, 256);
  if (storage == WAVE_F32) dense_to_pitched_kernel<float><<<grid, 256, 0, s>>>(g, dense, (float*)pitched);
  else if (storage == WAVE_BF16) dense_to_pitched_kernel<__nv_bfloat16><<<grid, 256, 0, s>>>(g, dense, (__nv_bfloat16*)pitched);
  else dense_to_pitched_kernel<__half><<<grid, 256, 0, s>>>(g, dense, (__half*)pitched);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_pitched_to_dense(const Geom& g, const void* pitched, float* dense, int storage, cudaStream_t s) {
  const unsigned grid = grid_for(g.nx * g.ny * g.nz, 256);
  if (storage == WAVE_F32) pitched_to_dense_kernel<float><<<grid, 256, 0, s>>>(g, (const float*)pitched, dense);
  else if (storage == WAVE_BF16) pitched_to_dense_kernel<__nv_bfloat16><<<grid, 256, 0, s>>>(g, (const __nv_bfloat16*)pitched, dense);
  else pitched_to_dense_kernel<__half><<<grid, 256, 0, s>>>(g, (const __half*)pitched, dense);
  count_launch();
  return cudaGetLastError();
}

// ---- per-step source / receiver kernel -----------------------------------
// Threads 0..nrec-1 handle receivers, thread nrec the source.
//  gather:  u_r = level `glevel` at the receiver; residual e = u_r - d_r
//           stored time-major (computeAdjointSource of Algorithm 1 keeps
//           f_adj = -w e implicitly) and/or the raw trace receiver-major.
//  inject:  pre-subtract the force of the coming step from the level about to
//           be overwritten: u^{n+1} = 2u^n - (u^{n-1} - dt^2/a f) + ..., i.e.
//           dst -= (dt^2/a) * f with f = psi (source) and k f_adj = -k w e
//           (receivers, Eq. superposedforce).  Atomic: cells may repeat.
template <typename T>
__global__ void sparse_kernel(SparseArgs a) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < a.nrec) {
    const int64_t p = a.rec_p[t];
    if (p < 0) {  // skipped receiver: zero trace, zero residual
      if (a.gsrc != nullptr && a.glevel >= 0) {
        if (a.traces) a.traces[t * a.tr_ld + a.glevel] = 0.f;
        if (a.resid) a.resid[(int64_t)a.glevel * a.nrec + t] = 0.f;
      }
      return;
    }
    if (a.gsrc != nullptr && a.glevel >= 0) {
      const float u = Stor<T>::get(reinterpret_cast<const T*>(a.gsrc) + p);
      if (a.traces) a.traces[t * a.tr_ld + a.glevel] = u;
      if (a.resid) {
        const float d = a.observed ? a.observed[t * a.obs_ld + a.glevel] : 0.f;
        a.resid[(int64_t)a.glevel * a.nrec + t] = u - d;
      }
    }
    if (a.dst != nullptr && a.resid_in != nullptr) {
      const float e = a.resid_in[(int64_t)a.ilevel * a.nrec + t];
      const float inj = a.coef[p] * a.h2;
      const float kw = (float)(*a.k_dev) * a.weight;
      Stor<T>::atomic_add(reinterpret_cast<T*>(a.dst) + p, -a.inj_sign * inj * (kw * e));
    }
  } else if (t == a.nrec) {
    if (a.dst != nullptr && a.src_p >= 0 && a.wavelet != nullptr) {
      const float inj = a.coef[a.src_p] * a.h2;
      Stor<T>::atomic_add(reinterpret_cast<T*>(a.dst) + a.src_p, a.inj_sign * inj * a.wavelet[a.ilevel]);
    }
  }
}

cudaError_t launch_sparse(const SparseArgs& a, int storage, cudaStream_t s) {
  const int64_t n = (int64_t)a.nrec + 1;
  const unsigned grid = (unsigned)((n + 255) / 256);
  if (storage == WAVE_F32) sparse_kernel<float><<<grid, 256, 0, s>>>(a);
  else if (storage == WAVE_BF16) sparse_kernel<__nv_bfloat16><<<grid, 256, 0, s>>>(a);
  else sparse_kernel<__half><<<grid, 256, 0, s>>>(a);
  count_launch();
  return cudaGetLastError();
}

// ---- FP64 reductions -----------------------------------------------------
// Deterministic two-pass: a fixed number of blocks each write one partial sum
// of (x - y)^2 (grid-stride order fixed by the launch shape), then one block
// adds the partials in a fixed tree order.
int reduce_parts(int64_t count) {
  int64_t p = (count + 8191) / 8192;
  if (p < 1) p = 1;
  if (p > 1024) p = 1024;
  return (int)p;
}

__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (warp == 0) {
    s = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  }
  return s;  // valid in thread 0
}

__global__ void sumsq_partial_kernel(const float* __restrict__ x, const float* __restrict__ y, int64_t n,
                                     double* __restrict__ partial) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double d = (double)x[i] - (y ? (double)y[i] : 0.0);
    acc = fma(d, d, acc);
  }
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void sum_final_kernel(const double* __restrict__ partial, int n, double scale, int accumulate,
                                 double* out, double* root) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += partial[i];
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) {
    const double v = accumulate ? out[0] + scale * s : scale * s;
    out[0] = v;
    if (root) root[0] = sqrt(v);
  }
}

cudaError_t launch_sumsq_partial(const float* x, const float* y, int64_t count, double* partial, int nparts,
                                 cudaStream_t s) {
  sumsq_partial_kernel<<<nparts, 256, 0, s>>>(x, y, count, partial);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_sum_final(const double* partial, int nparts, double scale, int accumulate, double* out,
                             cudaStream_t s, double* root) {
  sum_final_kernel<<<1, 256, 0, s>>>(partial, nparts, scale, accumulate, out, root);
  count_launch();
  return cudaGetLastError();
}

// ---- k -------------------------------------------------------------------
__global__ void set_k_kernel(double* k_dev, double k) { k_dev[0] = k; }

// k = ratio * ||psi|| / ||f_adj||, ||f_adj||^2 = w^2 sum e^2 (levels 1..N of
// the first shot).  A stand-in for the calibration of Sec. 4.1: it fixes the
// size of k u_adj relative to u, which sets both the neglected k^2 term and the
// FP32 cancellation in K(u^s,u^s) - K(u,u).
__global__ void auto_k_kernel(const double* psi2, const double* e2, double ratio, double w, double* k_dev) {
  const double g2 = w * w * e2[0];
  k_dev[0] = (g2 > 0.0 && psi2[0] > 0.0) ? ratio * sqrt(psi2[0] / g2) : 1.0;
}

cudaError_t launch_set_k(double* k_dev, double k, cudaStream_t s) {
  set_k_kernel<<<1, 1, 0, s>>>(k_dev, k);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_auto_k(const double* psi2, const double* e2, double ratio, double w, double* k_dev,
                          cudaStream_t s) {
  auto_k_kernel<<<1, 1, 0, s>>>(psi2, e2, ratio, w, k_dev);
  count_launch();
  return cudaGetLastError();
}

// ---- finish: K~ = acc / (2 k dt) (or acc / dt for the exact mode), with the
// per-block FP64 partial sums of K~^2 for the norm (fixed grid, fixed order) --
int finish_parts(int64_t cells) {
  int64_t b = (cells + 255) / 256;
  if (b > 1024) b = 1024;
  if (b < 1) b = 1;
  return (int)b;
}

__global__ void finish_kernel(Geom g, const float* __restrict__ acc, const double* k_dev, double inv_dt,
                              int superposition, int chain_v, const float* __restrict__ param,
                              float* __restrict__ grad, double* __restrict__ partial) {
  __shared__ double red[32];
  const double sc = superposition ? inv_dt / (2.0 * k_dev[0]) : inv_dt;
  const float s = (float)sc;
  const int64_t total = g.nx * g.ny * g.nz;
  double ss = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    float v = acc[(i / g.nx) * g.px + (i % g.nx)] * s;
    if (chain_v) {
      const float p = param[i];
      v *= -2.f / (p * p * p);   // dC/dv = dC/dm * dm/dv, m = 1/v^2
    }
    grad[i] = v;
    ss = fma((double)v, (double)v, ss);
  }
  const double bs = block_sum(ss, red);
  if (threadIdx.x == 0) partial[blockIdx.x] = bs;
}

cudaError_t launch_finish(const Geom& g, const float* acc, const double* k_dev, double inv_dt, int superposition,
                          int chain_v, const float* param, float* grad, double* partial, cudaStream_t s) {
  finish_kernel<<<finish_parts(g.nx * g.ny * g.nz), 256, 0, s>>>(g, acc, k_dev, inv_dt, superposition, chain_v,
                                                                  param, grad, partial);
  count_launch();
  return cudaGetLastError();
}

// ---- source time functions ----------------------------------------------
__global__ void wavelet_kernel(int kind, double f, int nc, double psi0, double dt, int nt, float* out) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n > nt) return;
  const double t = n * dt;
  const double pi = 3.14159265358979323846;
  double v;
  if (kind == 0) {
    const double tau = t - 1.0 / f;
    const double a = (pi * f * tau) * (pi * f * tau);
    v = psi0 * (1.0 - 2.0 * a) * exp(-a);
  } else {
    const double w = 2.0 * pi * f;
    const double s = sin(w * t / (2.0 * nc));
    v = (t >= 0.0 && t <= 2.0 * pi * nc / w) ? psi0 * sin(w * t) * s * s : 0.0;
  }
  out[n] = (float)v;
}

cudaError_t launch_wavelet(int kind, double f, int nc, double psi0, double dt, int nt, float* out, cudaStream_t s) {
  wavelet_kernel<<<(nt + 1 + 255) / 256, 256, 0, s>>>(kind, f, nc, psi0, dt, nt, out);
  count_launch();
  return cudaGetLastError();
}

}  // namespace wave
