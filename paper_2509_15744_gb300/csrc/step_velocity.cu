// Fused leapfrog step for the constant-density (velocity) wave equation,
// orders 2/4/6/8, 2D and 3D, with the sensitivity increment of the
// superposition method fused into the epilogue.
//
//   u^{n+1} = 2 u^n - u^{n-1} + (v dt/h)^2 * sum_axes sum_j c_j (u_{+j} + u_{-j})
//   acc    += acc_scale * (u^{n+1} - u^n)^2
//
// Sec. 3.1 (Eq. FDstencil1 with the mass written as m = 1/v^2) for the update;
// Sec. 4 / Algorithm 1 (incrementKernel, Eq. kernel1's -int u_t u_t dt term)
// for the accumulation.  Orders 4-8 use the textbook central weights.
//
// Mapping (GB300, HBM-bound): one warp owns a 128-cell x strip of one row,
// four cells per lane, so every global access is a coalesced 128-bit (FP32)
// or 64-bit (16-bit storage) load of a 512-byte warp row.  2D: each warp
// marches down y over a block of rows keeping the 2r+1 rows of u^n it needs
// in a register queue.  3D: a CTA of TY warps (TY rows) marches up z over a
// block of planes; z neighbours come from the per-lane register queue, y
// neighbours from a double-buffered shared-memory plane staged by the CTA
// (own rows from the queue, 2r halo rows loaded by the first 2r warps), x
// neighbours from the same staged rows (4-cell halos each side).
#include "stencil_common.cuh"

namespace wave {

// Common epilogue: update, store, sensitivity increment.
template <typename T>
__device__ __forceinline__ void update_store(const StepArgs& a, int64_t off, const float4& u,
                                             const float4& u_old, const float4& cf, const float lap[4]) {
  float4 un;
  un.x = fmaf(cf.x, lap[0], 2.f * u.x - u_old.x);
  un.y = fmaf(cf.y, lap[1], 2.f * u.y - u_old.y);
  un.z = fmaf(cf.z, lap[2], 2.f * u.z - u_old.z);
  un.w = fmaf(cf.w, lap[3], 2.f * u.w - u_old.w);
  Stor<T>::st4(reinterpret_cast<T*>(a.u_prev) + off, un);
  if (a.mix_a) {  // exact mode: acc += acc_scale (u_cur - u_next)(mix_a - mix_b)
    const float4 ma = *reinterpret_cast<const float4*>(a.mix_a + off);
    const float4 mb = *reinterpret_cast<const float4*>(a.mix_b + off);
    float4* accp = reinterpret_cast<float4*>(a.acc + off);
    float4 ac = *accp;
    ac.x = fmaf(a.acc_scale * (u.x - un.x), ma.x - mb.x, ac.x);
    ac.y = fmaf(a.acc_scale * (u.y - un.y), ma.y - mb.y, ac.y);
    ac.z = fmaf(a.acc_scale * (u.z - un.z), ma.z - mb.z, ac.z);
    ac.w = fmaf(a.acc_scale * (u.w - un.w), ma.w - mb.w, ac.w);
    *accp = ac;
  } else if (a.acc_mass) {
    const float4 ur = round_to_storage<T>(un);
    const float d0 = ur.x - u.x, d1 = ur.y - u.y, d2 = ur.z - u.z, d3 = ur.w - u.w;
    float4* accp = reinterpret_cast<float4*>(a.acc + off);
    float4 ac = *accp;
    if (a.comp) {
      float4* cpp = reinterpret_cast<float4*>(a.comp + off);
      float4 cp = *cpp;
      kahan_add(ac.x, cp.x, a.acc_scale * d0 * d0);
      kahan_add(ac.y, cp.y, a.acc_scale * d1 * d1);
      kahan_add(ac.z, cp.z, a.acc_scale * d2 * d2);
      kahan_add(ac.w, cp.w, a.acc_scale * d3 * d3);
      *cpp = cp;
    } else {
      ac.x = fmaf(a.acc_scale * d0, d0, ac.x);
      ac.y = fmaf(a.acc_scale * d1, d1, ac.y);
      ac.z = fmaf(a.acc_scale * d2, d2, ac.z);
      ac.w = fmaf(a.acc_scale * d3, d3, ac.w);
    }
    *accp = ac;
  }
}

// ---------------------------------------------------------------------------
// 2D: warp-per-strip, march in y
// ---------------------------------------------------------------------------
template <int R, typename T, int WPB>
__global__ void __launch_bounds__(WPB * 32)
step2d_velocity_kernel(StepArgs a) {
  __shared__ __align__(16) float sm[WPB][kRowW];
  const Geom& g = a.g;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int64_t nstrips = (g.nx + kStrip - 1) / kStrip;
  const int64_t gw = (int64_t)blockIdx.x * WPB + warp;
  const int64_t strip = gw % nstrips;
  const int64_t y0 = (gw / nstrips) * a.zblock;
  if (y0 >= g.ny) return;  // warp-uniform; this kernel synchronises only within warps
  const int64_t y1 = min(y0 + a.zblock, g.ny);
  const int64_t x0 = strip * kStrip;
  const int64_t xl = x0 + 4 * lane;
  const bool xin = (x0 >= 4) && (x0 + kStrip + 4 <= g.nx);
  const T* __restrict__ uc = reinterpret_cast<const T*>(a.u_cur);
  const T* __restrict__ up = reinterpret_cast<const T*>(a.u_prev);
  float* srow = sm[warp];
  // Staged rows start at zero so that never-written halo slots are finite.
  for (int i = lane; i < kRowW; i += 32) srow[i] = 0.f;

  auto qload = [&](int64_t yy) -> float4 {
    float s;
    const int64_t ys = mirror_index(yy, g.ny, g.bc, &s);
    if (s == 0.f) return make_float4(0.f, 0.f, 0.f, 0.f);
    return f4_scale(Stor<T>::ld4_nc(uc + ys * g.px + xl), s);
  };

  float4 q[2 * R + 1];
#pragma unroll
  for (int j = 1; j <= 2 * R; ++j) q[j] = qload(y0 - R + (j - 1));

  for (int64_t y = y0; y < y1; ++y) {
#pragma unroll
    for (int j = 0; j < 2 * R; ++j) q[j] = q[j + 1];
    q[2 * R] = qload(y + R);
    const int64_t off = y * g.px + xl;
    const float4 u_old = Stor<T>::ld4(up + off);
    const float4 cf = __ldg(reinterpret_cast<const float4*>(a.coef + off));
    __syncwarp();
    *reinterpret_cast<float4*>(srow + 4 + 4 * lane) = q[R];
    stage_x_halo<R, T>(srow, uc, y * g.px, x0, xin, lane, g);
    __syncwarp();
    float lap[4];
    x_terms<R>(srow, lane, lap, 2.f * cw<R>(0));
#pragma unroll
    for (int j = 1; j <= R; ++j) {
      lap[0] = fmaf(cw<R>(j), q[R - j].x + q[R + j].x, lap[0]);
      lap[1] = fmaf(cw<R>(j), q[R - j].y + q[R + j].y, lap[1]);
      lap[2] = fmaf(cw<R>(j), q[R - j].z + q[R + j].z, lap[2]);
      lap[3] = fmaf(cw<R>(j), q[R - j].w + q[R + j].w, lap[3]);
    }
    update_store<T>(a, off, q[R], u_old, cf, lap);
  }
}

// ---------------------------------------------------------------------------
// 3D: CTA of TY rows x 128 cells, march in z (2.5D)
// ---------------------------------------------------------------------------
template <int R, typename T, int TY>
__global__ void __launch_bounds__(TY * 32)
step3d_velocity_kernel(StepArgs a) {
  static_assert(TY >= 2 * R, "the first 2r warps stage the y halo rows");
  __shared__ __align__(16) float sm[2][TY + 2 * R][kRowW];
  const Geom& g = a.g;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int64_t x0 = (int64_t)blockIdx.x * kStrip;
  const int64_t ty0 = (int64_t)blockIdx.y * TY;
  const int64_t y = ty0 + warp;
  const int64_t z0 = (int64_t)blockIdx.z * a.zblock;
  const int64_t z1 = min(z0 + a.zblock, g.nz);
  const int64_t xl = x0 + 4 * lane;
  const bool xin = (x0 >= 4) && (x0 + kStrip + 4 <= g.nx);
  const T* __restrict__ uc = reinterpret_cast<const T*>(a.u_cur);
  const T* __restrict__ up = reinterpret_cast<const T*>(a.u_prev);

  // Own row (mirrored if it lies beyond ny, zero if not needed).
  const bool row_valid = y < g.ny;
  float ysg = 0.f;
  int64_t ysrc = 0;
  if (y < g.ny + R) ysrc = mirror_index(y, g.ny, g.bc, &ysg);
  const int64_t row_off = ysrc * g.px + xl;

  // Halo rows y0-R..y0-1 (slots 0..R-1) and y0+TY..y0+TY+R-1 (slots R+TY..).
  int halo_slot = -1;
  float hsg = 0.f;
  int64_t hrow_off = 0;
  if (warp < 2 * R) {
    const int64_t yh = warp < R ? ty0 - R + warp : ty0 + TY + (warp - R);
    halo_slot = warp < R ? warp : TY + warp;
    if (yh >= -R && yh < g.ny + R) {
      const int64_t ys = mirror_index(yh, g.ny, g.bc, &hsg);
      hrow_off = ys * g.px + xl;
    }
  }

  for (int i = threadIdx.x; i < 2 * (TY + 2 * R) * kRowW; i += TY * 32) (&sm[0][0][0])[i] = 0.f;
  __syncthreads();

  auto qload = [&](int64_t z) -> float4 {
    float zs;
    const int64_t zsrc = mirror_index(z, g.nz, g.bc, &zs);
    const float s = zs * ysg;
    if (s == 0.f) return make_float4(0.f, 0.f, 0.f, 0.f);
    return f4_scale(Stor<T>::ld4_nc(uc + zsrc * g.plane + row_off), s);
  };

  float4 q[2 * R + 1];
#pragma unroll
  for (int j = 1; j <= 2 * R; ++j) q[j] = qload(z0 - R + (j - 1));

  int buf = 0;
  for (int64_t z = z0; z < z1; ++z) {
#pragma unroll
    for (int j = 0; j < 2 * R; ++j) q[j] = q[j + 1];
    q[2 * R] = qload(z + R);
    const int64_t zoff = z * g.plane;
    float4 u_old = make_float4(0.f, 0.f, 0.f, 0.f), cf = u_old;
    if (row_valid) {
      u_old = Stor<T>::ld4(up + zoff + row_off);
      cf = __ldg(reinterpret_cast<const float4*>(a.coef + zoff + row_off));
    }
    float* srow = &sm[buf][R + warp][0];
    *reinterpret_cast<float4*>(srow + 4 + 4 * lane) = q[R];
    if (row_valid) stage_x_halo<R, T>(srow, uc, zoff + ysrc * g.px, x0, xin, lane, g);
    if (halo_slot >= 0) {
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (hsg != 0.f) v = f4_scale(Stor<T>::ld4_nc(uc + zoff + hrow_off), hsg);
      *reinterpret_cast<float4*>(&sm[buf][halo_slot][4 + 4 * lane]) = v;
    }
    __syncthreads();
    if (row_valid) {
      float lap[4];
      x_terms<R>(srow, lane, lap, 3.f * cw<R>(0));
#pragma unroll
      for (int j = 1; j <= R; ++j) {
        const float4 ym = *reinterpret_cast<const float4*>(&sm[buf][R + warp - j][4 + 4 * lane]);
        const float4 yp = *reinterpret_cast<const float4*>(&sm[buf][R + warp + j][4 + 4 * lane]);
        const float c = cw<R>(j);
        lap[0] = fmaf(c, ym.x + yp.x + q[R - j].x + q[R + j].x, lap[0]);
        lap[1] = fmaf(c, ym.y + yp.y + q[R - j].y + q[R + j].y, lap[1]);
        lap[2] = fmaf(c, ym.z + yp.z + q[R - j].z + q[R + j].z, lap[2]);
        lap[3] = fmaf(c, ym.w + yp.w + q[R - j].w + q[R + j].w, lap[3]);
      }
      update_store<T>(a, zoff + row_off, q[R], u_old, cf, lap);
    }
    buf ^= 1;
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
constexpr int kWarps2D = 4;
constexpr int kRows3D = 8;

template <int R, typename T>
static cudaError_t launch_vel(const StepArgs& a, cudaStream_t s) {
  const Geom& g = a.g;
  const int64_t nstrips = (g.nx + kStrip - 1) / kStrip;
  if (g.ndim == 2) {
    const int64_t nyb = (g.ny + a.zblock - 1) / a.zblock;
    const int64_t warps = nstrips * nyb;
    const int64_t blocks = (warps + kWarps2D - 1) / kWarps2D;
    step2d_velocity_kernel<R, T, kWarps2D><<<(unsigned)blocks, kWarps2D * 32, 0, s>>>(a);
  } else {
    dim3 grid((unsigned)nstrips, (unsigned)((g.ny + kRows3D - 1) / kRows3D),
              (unsigned)((g.nz + a.zblock - 1) / a.zblock));
    if constexpr (sizeof(T) == 4) {
      return launch_step3d_ring(a, 2 * R, s);
    } else {
      step3d_velocity_kernel<R, T, kRows3D><<<grid, kRows3D * 32, 0, s>>>(a);
    }
  }
  count_launch();
  return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_vel_t(const StepArgs& a, int order, cudaStream_t s) {
  switch (order) {
    case 2: return launch_vel<1, T>(a, s);
    case 4: return launch_vel<2, T>(a, s);
    case 6: return launch_vel<3, T>(a, s);
    case 8: return launch_vel<4, T>(a, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_step_velocity(const StepArgs& a, int order, int storage, cudaStream_t s) {
  switch (storage) {
    case WAVE_F32: return launch_vel_t<float>(a, order, s);
    case WAVE_BF16: return launch_vel_t<__nv_bfloat16>(a, order, s);
    case WAVE_F16: return launch_vel_t<__half>(a, order, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace wave
