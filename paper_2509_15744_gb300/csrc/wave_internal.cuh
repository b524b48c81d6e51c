// Internal declarations shared by the libwave translation units (not part of
// the C ABI).  Layout of every resident grid: pitched, C order, x fastest,
// row pitch px = nx rounded up to 128 cells, so each 32-lane warp owns one
// 128-cell strip of a row as one float4 (four cells) per lane.  Cells with
// x in [nx, px) are padding and stay exactly zero in every buffer.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "../../include/wave.h"

namespace wave {

constexpr int kStrip = 128;          // cells per warp strip (32 lanes x 4)
constexpr int kRowW = kStrip + 8;    // staged row: 4 halo cells each side

struct Geom {
  int ndim;
  int r;             // stencil radius = order / 2
  int bc;            // wave_bc
  int64_t nx, ny, nz;
  int64_t px;        // pitch (cells) of a row
  int64_t plane;     // px * ny
  int64_t cells;     // px * ny * nz (pitched grid size)
};

// Mirror an index of an axis of length n onto the domain (Sec. 3.1 ghost
// cells).  Neumann: even mirror about the half cell, u_{-1-j} = u_j.
// Dirichlet: odd mirror about the virtual nodes -1 and n, u_{-1} = 0,
// u_{-1-j} = -u_{j-1}.  Valid for overshoots up to n - 1; sign 0 marks a zero.
__host__ __device__ __forceinline__ int64_t mirror_index(int64_t i, int64_t n, int bc, float* sign) {
  if (i >= 0 && i < n) { *sign = 1.f; return i; }
  if (bc == WAVE_NEUMANN) { *sign = 1.f; return i < 0 ? -1 - i : 2 * n - 1 - i; }
  if (i == -1 || i == n) { *sign = 0.f; return 0; }
  *sign = -1.f;
  return i < 0 ? -2 - i : 2 * n - i;
}

// ---- storage types of the resident time levels ---------------------------
template <typename T> struct Stor;
template <> struct Stor<float> {
  static __device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
  static __device__ __forceinline__ float4 ld4_nc(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }
  static __device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
  static __device__ __forceinline__ float ld1(const float* p) { return __ldg(p); }
  static __device__ __forceinline__ void atomic_add(float* p, float v) { atomicAdd(p, v); }
  static __device__ __forceinline__ float get(const float* p) { return *p; }
};
template <> struct Stor<__nv_bfloat16> {
  typedef __nv_bfloat16 T;
  static __device__ __forceinline__ float4 ld4(const T* p) {
    uint2 raw = *reinterpret_cast<const uint2*>(p);
    __nv_bfloat162 a = *reinterpret_cast<__nv_bfloat162*>(&raw.x);
    __nv_bfloat162 b = *reinterpret_cast<__nv_bfloat162*>(&raw.y);
    float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
    return make_float4(fa.x, fa.y, fb.x, fb.y);
  }
  static __device__ __forceinline__ float4 ld4_nc(const T* p) {
    uint2 raw = __ldg(reinterpret_cast<const uint2*>(p));
    __nv_bfloat162 a = *reinterpret_cast<__nv_bfloat162*>(&raw.x);
    __nv_bfloat162 b = *reinterpret_cast<__nv_bfloat162*>(&raw.y);
    float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
    return make_float4(fa.x, fa.y, fb.x, fb.y);
  }
  static __device__ __forceinline__ void st4(T* p, float4 v) {
    __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y), b = __floats2bfloat162_rn(v.z, v.w);
    uint2 raw;
    raw.x = *reinterpret_cast<uint32_t*>(&a);
    raw.y = *reinterpret_cast<uint32_t*>(&b);
    *reinterpret_cast<uint2*>(p) = raw;
  }
  static __device__ __forceinline__ float ld1(const T* p) { return __bfloat162float(*p); }
  static __device__ __forceinline__ void atomic_add(T* p, float v) { atomicAdd(p, __float2bfloat16_rn(v)); }
  static __device__ __forceinline__ float get(const T* p) { return __bfloat162float(*p); }
};
template <> struct Stor<__half> {
  typedef __half T;
  static __device__ __forceinline__ float4 ld4(const T* p) {
    uint2 raw = *reinterpret_cast<const uint2*>(p);
    __half2 a = *reinterpret_cast<__half2*>(&raw.x);
    __half2 b = *reinterpret_cast<__half2*>(&raw.y);
    float2 fa = __half22float2(a), fb = __half22float2(b);
    return make_float4(fa.x, fa.y, fb.x, fb.y);
  }
  static __device__ __forceinline__ float4 ld4_nc(const T* p) {
    uint2 raw = __ldg(reinterpret_cast<const uint2*>(p));
    __half2 a = *reinterpret_cast<__half2*>(&raw.x);
    __half2 b = *reinterpret_cast<__half2*>(&raw.y);
    float2 fa = __half22float2(a), fb = __half22float2(b);
    return make_float4(fa.x, fa.y, fb.x, fb.y);
  }
  static __device__ __forceinline__ void st4(T* p, float4 v) {
    __half2 a = __floats2half2_rn(v.x, v.y), b = __floats2half2_rn(v.z, v.w);
    uint2 raw;
    raw.x = *reinterpret_cast<uint32_t*>(&a);
    raw.y = *reinterpret_cast<uint32_t*>(&b);
    *reinterpret_cast<uint2*>(p) = raw;
  }
  static __device__ __forceinline__ float ld1(const T* p) { return __half2float(*p); }
  static __device__ __forceinline__ void atomic_add(T* p, float v) { atomicAdd(p, __float2half_rn(v)); }
  static __device__ __forceinline__ float get(const T* p) { return __half2float(*p); }
};

__device__ __forceinline__ float4 f4_scale(float4 v, float s) {
  return make_float4(v.x * s, v.y * s, v.z * s, v.w * s);
}
__device__ __forceinline__ float f4_get(const float4& v, int i) {
  return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
}

// ---- step kernel arguments ----------------------------------------------
// One leapfrog step u_next = 2 u_cur - u_prev + coef * (h^2 L u_cur), written
// over u_prev, with the sensitivity increment acc += acc_scale * c where
//   velocity: c = (u_next - u_cur)^2
//   density:  c = da (u_next - u_cur)^2 - dbs * sum_faces dbf (D_f u_cur)^2
// (dt times the per-step discrete Frechet kernel of Eq. kernel1 / kernel2).
struct StepArgs {
  Geom g;
  const void* u_cur;     // level n (read)
  void* u_prev;          // level n-1 (read) -> level n+1 (written)
  const float* coef;     // velocity: v^2 dt^2 / h^2; density: dt^2 / (a h^2)
  const float* bmat;     // density: b = 1/rho per cell
  float* acc;            // sensitivity accumulator (nullable)
  float* comp;           // Kahan compensation (nullable)
  float acc_scale;       // +1 forward (subtracts K(u,u)), -1 superposed pass (adds K(u^s,u^s))
  int acc_mass;          // accumulate the half-level (mass) term
  int acc_stiff;         // accumulate the level (stiffness) term (density)
  float da;              // d a / d gamma (density); 1 for velocity
  float dbs;             // (dt^2/h^2) d b / d gamma (density)
  int64_t zblock;        // cells of the march axis per CTA (3D) / warp (2D)
  int tile_rows;         // 3D ring kernel: rows per CTA (8 or 16)
  int ring_depth;        // 3D ring kernel: planes copied ahead (2 or 3)
  int pipeline;          // 3D FP32: 0 cp.async ring, 3 register queue, 4 two fields per pass, 5 TMA tiles with the
                         // accumulator in registers
  int cta_order;         // 3D pipelines 3 and 4: 0 z-block fastest in launch order, 1 plane-major (x strip fastest,
                         // then y tile, then z-block)
  int* err;              // device error word (bounded waits)
  long long wait_limit_cycles;
  int debug_stall;
  // Exact (stored-history) mode, FP32 velocity only:
  const float* mix_a;    // stored u^j (nullable): accumulate the mixed term
  const float* mix_b;    // stored u^{j-1}: acc += acc_scale (u_cur - u_next)(mix_a - mix_b)
};

// Launchers (defined in step_*.cu).  Return cudaGetLastError() of the launch.
cudaError_t launch_step_velocity(const StepArgs& a, int order, int storage, cudaStream_t s);
cudaError_t launch_step_density(const StepArgs& a, int storage, cudaStream_t s);
cudaError_t launch_step3d_ring(const StepArgs& a, int order, cudaStream_t s);

// Batched 3D step: every listed shot advances one step; the shots' sensitivity
// increments are summed per cell before one accumulator update.
constexpr int kMaxBatch = 32;
struct BatchArgs {
  StepArgs base;                 // geometry, coef, acc, comp, acc_scale, zblock, ring_depth
  int nshots;
  const float* cur[kMaxBatch];   // level n of each shot
  float* prev[kMaxBatch];        // level n-1 -> n+1 of each shot
  float accf[kMaxBatch];         // per-shot factor on acc_scale this step (0: no increment)
  int pair_mix;                  // two fields (u, lambda) in the two-shots-per-pass kernel:
                                 // acc += acc_scale accf[1] (lambda - lambda_new)(u - u_new)
  // TMA-tiled pipeline only:
  int* err;                      // set to 1 when a bounded wait gives up
  long long wait_limit_cycles;   // bound of every wait (clock64 cycles)
  int debug_stall;               // test only: issue no copies, so the first wait runs out
};
cudaError_t launch_step3d_batched(const BatchArgs& b, int order, cudaStream_t s);
cudaError_t launch_step3d_queue(const BatchArgs& b, int order, cudaStream_t s);
cudaError_t launch_step3d_pair(const BatchArgs& b, int order, cudaStream_t s);
cudaError_t launch_step3d_stream(const BatchArgs& b, int order, cudaStream_t s);
bool stream_supported(const BatchArgs& b);


// ---- sparse (source / receiver) kernel -----------------------------------
struct SparseArgs {
  const void* gsrc;       // buffer holding level `glevel` (gather), or null
  int32_t glevel;
  const int64_t* rec_p;   // pitched receiver cells, -1 = skip
  int32_t nrec;
  const float* observed;  // [nrec][obs_ld], nullable
  int64_t obs_ld;
  float* resid;           // time-major [.][nrec]: resid[level * nrec + r] = u - d, nullable
  float* traces;          // receiver-major traces[r * tr_ld + level] = u, nullable
  int64_t tr_ld;
  void* dst;              // injection target (level about to be overwritten), or null
  const float* coef;      // injection scale is coef * h2 = dt^2 / a
  float h2;
  int64_t src_p;          // pitched source cell (-1: none)
  const float* wavelet;
  int32_t ilevel;         // wavelet sample injected
  const float* resid_in;  // time-major residuals of level ilevel (receivers), nullable
  const double* k_dev;    // superposition factor
  float weight;           // objective weight w (f_adj = -w e)
  float inj_sign;         // -1: pre-subtract the force of the coming step from
                          //     the level it overwrites; +1: add the force of
                          //     the step just taken to its output level
};
cudaError_t launch_sparse(const SparseArgs& a, int storage, cudaStream_t s);

// ---- auxiliary kernels (aux.cu) -----------------------------------------
cudaError_t launch_coef_velocity(const Geom& g, const float* v, float dt_over_h, float* coef, cudaStream_t s);
cudaError_t launch_coef_density(const Geom& g, const float* gamma, double dt2_over_h2, float* ca, float* b, cudaStream_t s);
cudaError_t launch_stability(const Geom& g, int physics, double sym, const float* coef, const float* b,
                             float* partial, int nparts, cudaStream_t s);
cudaError_t launch_max_final(const float* partial, int nparts, float* out, cudaStream_t s);
cudaError_t launch_pitch_indices(const Geom& g, const int64_t* flat, int32_t n, int64_t* pitched, cudaStream_t s);
cudaError_t launch_dense_to_pitched(const Geom& g, const float* dense, void* pitched, int storage, cudaStream_t s);
cudaError_t launch_pitched_to_dense(const Geom& g, const void* pitched, float* dense, int storage, cudaStream_t s);
cudaError_t launch_sumsq_partial(const float* x, const float* y, int64_t count, double* partial, int nparts, cudaStream_t s);
// out = scale * sum (+ out if accumulate); root, if not null, receives sqrt(out).
cudaError_t launch_sum_final(const double* partial, int nparts, double scale, int accumulate, double* out, cudaStream_t s,
                             double* root = nullptr);
cudaError_t launch_set_k(double* k_dev, double k, cudaStream_t s);
cudaError_t launch_auto_k(const double* psi2, const double* e2, double ratio, double w, double* k_dev, cudaStream_t s);
// Writes grad and finish_parts(cells) FP64 partial sums of grad^2 to partial.
cudaError_t launch_finish(const Geom& g, const float* acc, const double* k_dev, double inv_dt, int superposition,
                          int chain_v, const float* param, float* grad, double* partial, cudaStream_t s);
int finish_parts(int64_t cells);
cudaError_t launch_wavelet(int kind, double f, int nc, double psi0, double dt, int nt, float* out, cudaStream_t s);

int reduce_parts(int64_t count);   // number of partial sums used for `count` samples
// Raises a kernel's dynamic shared-memory limit once per device.
cudaError_t set_smem_limit_once(const void* func, int bytes);
// Records the text wave_last_error() returns for a failed CUDA call.
void set_last_error(const char* what, cudaError_t e);
// Names the call that failed inside a launcher; the entry point adds it to
// the text of wave_last_error().
void note_error(const char* what, cudaError_t e);
void count_launch(int n = 1);

}  // namespace wave
