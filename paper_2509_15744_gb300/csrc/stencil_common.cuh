// Device helpers shared by the velocity step kernels (2D, 3D register-queue
// and 3D shared-memory ring): stencil weights, x-halo staging with the ghost
// rule, x part of the stencil, Kahan update.
#pragma once

#include "wave_internal.cuh"

namespace wave {

// Central second-derivative weights c_0..c_r (before 1/h^2).
template <int R>
__device__ __forceinline__ float cw(int j) {
  if (R == 1) return j == 0 ? -2.f : 1.f;
  if (R == 2) return j == 0 ? -2.5f : (j == 1 ? 4.f / 3.f : -1.f / 12.f);
  if (R == 3) return j == 0 ? -49.f / 18.f : (j == 1 ? 1.5f : (j == 2 ? -0.15f : 1.f / 90.f));
  return j == 0 ? -205.f / 72.f
                : (j == 1 ? 1.6f : (j == 2 ? -0.2f : (j == 3 ? 8.f / 315.f : -1.f / 560.f)));
}

template <typename T>
__device__ __forceinline__ float4 round_to_storage(float4 v) {
  if constexpr (sizeof(T) == 4) {
    return v;
  } else {
    T buf[4];
    buf[0] = T(v.x); buf[1] = T(v.y); buf[2] = T(v.z); buf[3] = T(v.w);
    return make_float4(float(buf[0]), float(buf[1]), float(buf[2]), float(buf[3]));
  }
}

// Value of u at (row offset `rowbase`, column gx) with the x ghost rule.
template <typename T>
__device__ __forceinline__ float ghost_x(const T* __restrict__ u, int64_t rowbase, int64_t gx,
                                         const Geom& g) {
  float s;
  int64_t m = mirror_index(gx, g.nx, g.bc, &s);
  return s == 0.f ? 0.f : s * Stor<T>::ld1(u + rowbase + m);
}

// Stage the x halo of one 128-cell row in `srow` (positions 0..3 and
// 132..135 hold cells x0-4..x0-1 and x0+128..x0+131; positions of cells
// beyond nx receive their mirror values).  `rowbase` = offset of the row.
template <int R, typename T>
__device__ __forceinline__ void stage_x_halo(float* srow, const T* __restrict__ u, int64_t rowbase,
                                             int64_t x0, bool xin, int lane, const Geom& g) {
  if (xin) {
    if (lane == 0) *reinterpret_cast<float4*>(srow) = Stor<T>::ld4_nc(u + rowbase + x0 - 4);
    if (lane == 31) *reinterpret_cast<float4*>(srow + 4 + kStrip) = Stor<T>::ld4_nc(u + rowbase + x0 + kStrip);
  } else {
    __syncwarp();
    if (lane < R) {
      const int64_t gx = x0 - 1 - lane;
      srow[3 - lane] = ghost_x<T>(u, rowbase, gx, g);
    } else if (lane >= 8 && lane < 8 + R) {
      const int64_t base = g.nx < x0 + kStrip ? g.nx : x0 + kStrip;
      const int64_t gx = base + (lane - 8);
      srow[gx - x0 + 4] = ghost_x<T>(u, rowbase, gx, g);
    }
  }
}

// x part of the stencil for the 4 cells of a lane: positions 4+4l+i in srow.
// The lane's own float4 is read back from the staged row, not taken from the
// register queue: when the row ends inside it (nx not a multiple of 4), its
// cells beyond nx hold the mirrored ghost values written by stage_x_halo.
template <int R>
__device__ __forceinline__ void x_terms(const float* srow, int lane, float lap[4], float ndim_c0) {
  const float4 A = *reinterpret_cast<const float4*>(srow + 4 * lane);
  const float4 B = *reinterpret_cast<const float4*>(srow + 4 + 4 * lane);
  const float4 C = *reinterpret_cast<const float4*>(srow + 8 + 4 * lane);
  const float e[12] = {A.x, A.y, A.z, A.w, B.x, B.y, B.z, B.w, C.x, C.y, C.z, C.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    float s = ndim_c0 * e[4 + i];
#pragma unroll
    for (int j = 1; j <= R; ++j) s = fmaf(cw<R>(j), e[4 + i + j] + e[4 + i - j], s);
    lap[i] = s;
  }
}

// The same x part from the three float4 A (cells x-4..x-1), B (x..x+3) and
// C (x+4..x+7) already in registers, with the same operation order.
template <int R>
__device__ __forceinline__ void x_terms_abc(const float4& A, const float4& B, const float4& C, float lap[4],
                                            float ndim_c0) {
  const float e[12] = {A.x, A.y, A.z, A.w, B.x, B.y, B.z, B.w, C.x, C.y, C.z, C.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    float s = ndim_c0 * e[4 + i];
#pragma unroll
    for (int j = 1; j <= R; ++j) s = fmaf(cw<R>(j), e[4 + i + j] + e[4 + i - j], s);
    lap[i] = s;
  }
}

// x ghosts of a row whose ends fall on float4 boundaries (nx a multiple of
// 128): the four cells beyond the left end (A of lane 0) and beyond the right
// end (C of lane 31) from the lane's own cells B by the boundary rule.
// Dirichlet: u_{-1} = 0, u_{-1-j} = -u_{j-1}; Neumann: u_{-1-j} = u_j.
__device__ __forceinline__ float4 left_ghosts(const float4& B, int bc) {
  return bc == WAVE_NEUMANN ? make_float4(B.w, B.z, B.y, B.x) : make_float4(-B.z, -B.y, -B.x, 0.f);
}
__device__ __forceinline__ float4 right_ghosts(const float4& B, int bc) {
  return bc == WAVE_NEUMANN ? make_float4(B.w, B.z, B.y, B.x) : make_float4(0.f, -B.w, -B.z, -B.y);
}

// In the shared-memory ring kernels the lane's own float4 is read from the
// staged row, whose cells at x >= nx hold mirrored ghost values; zeroing them
// there (u = u_old = coef = 0 in the row padding) keeps the padding at zero
// and its sensitivity increment at zero.
__device__ __forceinline__ float4 mask_row_padding(float4 u, int64_t xl, int64_t nx) {
  if (xl + 4 > nx) {
    if (xl >= nx) u.x = 0.f;
    if (xl + 1 >= nx) u.y = 0.f;
    if (xl + 2 >= nx) u.z = 0.f;
    if (xl + 3 >= nx) u.w = 0.f;
  }
  return u;
}

// Compensated sum acc += v.  The explicitly rounded operations keep the
// compiler from fusing the caller's product into v - comp, so every kernel
// rounds the update the same way.
__device__ __forceinline__ void kahan_add(float& acc, float& comp, float v) {
  const float y = __fsub_rn(v, comp);
  const float t = __fadd_rn(acc, y);
  comp = __fsub_rn(__fsub_rn(t, acc), y);
  acc = t;
}

}  // namespace wave
