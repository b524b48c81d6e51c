// Fused leapfrog step for the variable-density acoustic equation (Eq.
// wavetopopt) with the second-order stencil of Eq. FDstencil2:
//
//   u^{n+1} = 2 u^n - u^{n-1} + dt^2/(a h^2) sum_faces b_f (u_j - u_i),
//   b_f = 2 b_i b_j / (b_i + b_j)   (harmonic mean of b = 1/rho, Sec. 3.1),
//
// ghost material = boundary material (even mirror of b), ghost u per the BC.
// Sensitivity increment (dt times the per-step discrete Eq. kernel2):
//
//   acc += acc_scale * [ da (u^{n+1} - u^n)^2 - dbs sum_faces dbf (u_j - u_i)^2 ]
//
// with dbs = (dt^2/h^2) db/dgamma and dbf = d b_f / d b_i = 2 b_j^2/(b_i+b_j)^2
// (1 for a Dirichlet ghost face, whose material follows cell i).  The mass
// term belongs to the half level n+1/2, the stiffness term to level n.
//
// Mapping (2D): as the 2D velocity kernel (warp per 128-cell strip, march in
// y), with a second staged field b; 3D below.
#include "wave_internal.cuh"

namespace wave {

template <typename T>
__device__ __forceinline__ float4 round_storage(float4 v) {
  if constexpr (sizeof(T) == 4) {
    return v;
  } else {
    T b0 = T(v.x), b1 = T(v.y), b2 = T(v.z), b3 = T(v.w);
    return make_float4(float(b0), float(b1), float(b2), float(b3));
  }
}

// Face contribution of one neighbour j of cell i.
struct Face {
  float flux;   // b_f (u_j - u_i)
  float grad;   // dbf (u_j - u_i)^2
};

__device__ __forceinline__ Face face(float ui, float uj, float bi, float bj, bool dirichlet_ghost) {
  const float du = uj - ui;
  const float sum = bi + bj;
  const float bf = 2.f * bi * bj / sum;
  const float dbf = dirichlet_ghost ? 1.f : 2.f * bj * bj / (sum * sum);
  Face f;
  f.flux = bf * du;
  f.grad = dbf * du * du;
  return f;
}

__device__ __forceinline__ void kahan_add_d(float& acc, float& comp, float v) {
  const float y = v - comp;
  const float t = acc + y;
  comp = (t - acc) - y;
  acc = t;
}

// Stage one row of a field with its 4-cell x halos (ghost rule per `bc`).
template <typename T>
__device__ __forceinline__ void stage_row(float* srow, const T* __restrict__ f, int64_t rowbase, float4 own,
                                          int64_t x0, bool xin, int lane, const Geom& g, int bc) {
  *reinterpret_cast<float4*>(srow + 4 + 4 * lane) = own;
  if (xin) {
    if (lane == 0) *reinterpret_cast<float4*>(srow) = Stor<T>::ld4_nc(f + rowbase + x0 - 4);
    if (lane == 31) *reinterpret_cast<float4*>(srow + 4 + kStrip) = Stor<T>::ld4_nc(f + rowbase + x0 + kStrip);
  } else {
    __syncwarp();
    int64_t gx = -1;
    int p = 0;
    if (lane == 0) { gx = x0 - 1; p = 3; }
    if (lane == 8) { gx = g.nx < x0 + kStrip ? g.nx : x0 + kStrip; p = (int)(gx - x0 + 4); }
    if (lane == 0 || lane == 8) {
      float s;
      const int64_t m = mirror_index(gx, g.nx, bc, &s);
      srow[p] = s == 0.f ? 0.f : s * Stor<T>::ld1(f + rowbase + m);
    }
  }
}

template <typename T, int WPB>
__global__ void __launch_bounds__(WPB * 32)
step2d_density_kernel(StepArgs a) {
  __shared__ __align__(16) float su[WPB][kRowW];
  __shared__ __align__(16) float sb[WPB][kRowW];
  const Geom& g = a.g;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int64_t nstrips = (g.nx + kStrip - 1) / kStrip;
  const int64_t gw = (int64_t)blockIdx.x * WPB + warp;
  const int64_t strip = gw % nstrips;
  const int64_t y0 = (gw / nstrips) * a.zblock;
  if (y0 >= g.ny) return;
  const int64_t y1 = min(y0 + a.zblock, g.ny);
  const int64_t x0 = strip * kStrip;
  const int64_t xl = x0 + 4 * lane;
  const bool xin = (x0 >= 4) && (x0 + kStrip + 4 <= g.nx);
  const T* __restrict__ uc = reinterpret_cast<const T*>(a.u_cur);
  const T* __restrict__ up = reinterpret_cast<const T*>(a.u_prev);
  const float* __restrict__ bm = a.bmat;
  const bool dir = g.bc == WAVE_DIRICHLET;
  for (int i = lane; i < kRowW; i += 32) { su[warp][i] = 0.f; sb[warp][i] = 1.f; }

  auto uload = [&](int64_t yy) -> float4 {
    float s;
    const int64_t ys = mirror_index(yy, g.ny, g.bc, &s);
    if (s == 0.f) return make_float4(0.f, 0.f, 0.f, 0.f);
    return f4_scale(Stor<T>::ld4_nc(uc + ys * g.px + xl), s);
  };
  auto bload = [&](int64_t yy) -> float4 {   // material ghost = boundary material
    float s;
    const int64_t ys = mirror_index(yy, g.ny, WAVE_NEUMANN, &s);
    return __ldg(reinterpret_cast<const float4*>(bm + ys * g.px + xl));
  };

  float4 qu0 = uload(y0 - 1), qu1 = uload(y0);
  float4 qb0 = bload(y0 - 1), qb1 = bload(y0);
  for (int64_t y = y0; y < y1; ++y) {
    const float4 qu2 = uload(y + 1);
    const float4 qb2 = bload(y + 1);
    const int64_t off = y * g.px + xl;
    const float4 u_old = Stor<T>::ld4(up + off);
    const float4 ca = __ldg(reinterpret_cast<const float4*>(a.coef + off));
    __syncwarp();
    stage_row<T>(su[warp], uc, y * g.px, qu1, x0, xin, lane, g, g.bc);
    stage_row<float>(sb[warp], bm, y * g.px, qb1, x0, xin, lane, g, WAVE_NEUMANN);
    __syncwarp();
    const float* ru = su[warp];
    const float* rb = sb[warp];
    float flux[4], grad[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int p = 4 + 4 * lane + i;
      const int64_t x = xl + i;
      const float ui = ru[p], bi = rb[p];
      const float uy_m = f4_get(qu0, i), uy_p = f4_get(qu2, i);
      const float by_m = f4_get(qb0, i), by_p = f4_get(qb2, i);
      Face fxm = face(ui, ru[p - 1], bi, rb[p - 1], dir && x == 0);
      Face fxp = face(ui, ru[p + 1], bi, rb[p + 1], dir && x == g.nx - 1);
      Face fym = face(ui, uy_m, bi, by_m, dir && y == 0);
      Face fyp = face(ui, uy_p, bi, by_p, dir && y == g.ny - 1);
      flux[i] = (fxm.flux + fxp.flux) + (fym.flux + fyp.flux);
      grad[i] = x < g.nx ? (fxm.grad + fxp.grad) + (fym.grad + fyp.grad) : 0.f;   // row padding stays zero
    }
    float4 un;
    un.x = fmaf(ca.x, flux[0], 2.f * qu1.x - u_old.x);
    un.y = fmaf(ca.y, flux[1], 2.f * qu1.y - u_old.y);
    un.z = fmaf(ca.z, flux[2], 2.f * qu1.z - u_old.z);
    un.w = fmaf(ca.w, flux[3], 2.f * qu1.w - u_old.w);
    Stor<T>::st4(reinterpret_cast<T*>(a.u_prev) + off, un);
    if (a.acc_mass || a.acc_stiff) {
      const float4 ur = round_storage<T>(un);
      const float d[4] = {ur.x - qu1.x, ur.y - qu1.y, ur.z - qu1.z, ur.w - qu1.w};
      float c[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        float v = 0.f;
        if (a.acc_mass) v = a.da * d[i] * d[i];
        if (a.acc_stiff) v = fmaf(-a.dbs, grad[i], v);
        c[i] = a.acc_scale * v;
      }
      float4* accp = reinterpret_cast<float4*>(a.acc + off);
      float4 ac = *accp;
      if (a.comp) {
        float4* cpp = reinterpret_cast<float4*>(a.comp + off);
        float4 cp = *cpp;
        kahan_add_d(ac.x, cp.x, c[0]);
        kahan_add_d(ac.y, cp.y, c[1]);
        kahan_add_d(ac.z, cp.z, c[2]);
        kahan_add_d(ac.w, cp.w, c[3]);
        *cpp = cp;
      } else {
        ac.x += c[0]; ac.y += c[1]; ac.z += c[2]; ac.w += c[3];
      }
      *accp = ac;
    }
    qu0 = qu1; qu1 = qu2;
    qb0 = qb1; qb1 = qb2;
  }
}

// 3D: a warp owns one 128-cell strip of a (y, z) row and marches up z over a
// block of planes.  z neighbours come from a three-plane register queue, y
// neighbours from direct loads of the rows y-1 and y+1 (L1/L2-resident: the
// warps of the neighbouring rows read them too), x neighbours from the
// staged own row.  Same face arithmetic and sensitivity increment as 2D.
template <typename T, int WPB>
__global__ void __launch_bounds__(WPB * 32)
step3d_density_kernel(StepArgs a) {
  __shared__ __align__(16) float su[WPB][kRowW];
  __shared__ __align__(16) float sb[WPB][kRowW];
  const Geom& g = a.g;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int64_t nstrips = (g.nx + kStrip - 1) / kStrip;
  const int64_t nzb = (g.nz + a.zblock - 1) / a.zblock;
  const int64_t gw = (int64_t)blockIdx.x * WPB + warp;
  const int64_t strip = gw % nstrips;
  const int64_t rest = gw / nstrips;
  const int64_t y = rest % g.ny;
  const int64_t zb = rest / g.ny;
  if (zb >= nzb) return;   // whole warps only; the kernel has no block-wide barrier
  const int64_t z0 = zb * a.zblock;
  const int64_t z1 = min(z0 + a.zblock, g.nz);
  const int64_t x0 = strip * kStrip;
  const int64_t xl = x0 + 4 * lane;
  const bool xin = (x0 >= 4) && (x0 + kStrip + 4 <= g.nx);
  const T* __restrict__ uc = reinterpret_cast<const T*>(a.u_cur);
  const T* __restrict__ up = reinterpret_cast<const T*>(a.u_prev);
  const float* __restrict__ bm = a.bmat;
  const bool dir = g.bc == WAVE_DIRICHLET;
  for (int i = lane; i < kRowW; i += 32) { su[warp][i] = 0.f; sb[warp][i] = 1.f; }

  auto uload = [&](int64_t yy, int64_t zz) -> float4 {   // u with the ghost rule in y and z
    float sy, sz;
    const int64_t ys = mirror_index(yy, g.ny, g.bc, &sy);
    const int64_t zs = mirror_index(zz, g.nz, g.bc, &sz);
    const float sg = sy * sz;
    if (sg == 0.f) return make_float4(0.f, 0.f, 0.f, 0.f);
    return f4_scale(Stor<T>::ld4_nc(uc + zs * g.plane + ys * g.px + xl), sg);
  };
  auto bload = [&](int64_t yy, int64_t zz) -> float4 {   // material ghost = boundary material
    float sy, sz;
    const int64_t ys = mirror_index(yy, g.ny, WAVE_NEUMANN, &sy);
    const int64_t zs = mirror_index(zz, g.nz, WAVE_NEUMANN, &sz);
    return __ldg(reinterpret_cast<const float4*>(bm + zs * g.plane + ys * g.px + xl));
  };

  float4 qu0 = uload(y, z0 - 1), qu1 = uload(y, z0);
  float4 qb0 = bload(y, z0 - 1), qb1 = bload(y, z0);
  for (int64_t z = z0; z < z1; ++z) {
    const float4 qu2 = uload(y, z + 1);
    const float4 qb2 = bload(y, z + 1);
    const float4 uym4 = uload(y - 1, z), uyp4 = uload(y + 1, z);
    const float4 bym4 = bload(y - 1, z), byp4 = bload(y + 1, z);
    const int64_t rowbase = z * g.plane + y * g.px;
    const int64_t off = rowbase + xl;
    const float4 u_old = Stor<T>::ld4(up + off);
    const float4 ca = __ldg(reinterpret_cast<const float4*>(a.coef + off));
    __syncwarp();
    stage_row<T>(su[warp], uc, rowbase, qu1, x0, xin, lane, g, g.bc);
    stage_row<float>(sb[warp], bm, rowbase, qb1, x0, xin, lane, g, WAVE_NEUMANN);
    __syncwarp();
    const float* ru = su[warp];
    const float* rb = sb[warp];
    float flux[4], grad[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int p = 4 + 4 * lane + i;
      const int64_t x = xl + i;
      const float ui = ru[p], bi = rb[p];
      Face fxm = face(ui, ru[p - 1], bi, rb[p - 1], dir && x == 0);
      Face fxp = face(ui, ru[p + 1], bi, rb[p + 1], dir && x == g.nx - 1);
      Face fym = face(ui, f4_get(uym4, i), bi, f4_get(bym4, i), dir && y == 0);
      Face fyp = face(ui, f4_get(uyp4, i), bi, f4_get(byp4, i), dir && y == g.ny - 1);
      Face fzm = face(ui, f4_get(qu0, i), bi, f4_get(qb0, i), dir && z == 0);
      Face fzp = face(ui, f4_get(qu2, i), bi, f4_get(qb2, i), dir && z == g.nz - 1);
      flux[i] = ((fxm.flux + fxp.flux) + (fym.flux + fyp.flux)) + (fzm.flux + fzp.flux);
      grad[i] = x < g.nx ? ((fxm.grad + fxp.grad) + (fym.grad + fyp.grad)) + (fzm.grad + fzp.grad)
                         : 0.f;   // row padding stays zero
    }
    float4 un;
    un.x = fmaf(ca.x, flux[0], 2.f * qu1.x - u_old.x);
    un.y = fmaf(ca.y, flux[1], 2.f * qu1.y - u_old.y);
    un.z = fmaf(ca.z, flux[2], 2.f * qu1.z - u_old.z);
    un.w = fmaf(ca.w, flux[3], 2.f * qu1.w - u_old.w);
    Stor<T>::st4(reinterpret_cast<T*>(a.u_prev) + off, un);
    if (a.acc_mass || a.acc_stiff) {
      const float4 ur = round_storage<T>(un);
      const float d[4] = {ur.x - qu1.x, ur.y - qu1.y, ur.z - qu1.z, ur.w - qu1.w};
      float c[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        float v = 0.f;
        if (a.acc_mass) v = a.da * d[i] * d[i];
        if (a.acc_stiff) v = fmaf(-a.dbs, grad[i], v);
        c[i] = a.acc_scale * v;
      }
      float4* accp = reinterpret_cast<float4*>(a.acc + off);
      float4 ac = *accp;
      if (a.comp) {
        float4* cpp = reinterpret_cast<float4*>(a.comp + off);
        float4 cp = *cpp;
        kahan_add_d(ac.x, cp.x, c[0]);
        kahan_add_d(ac.y, cp.y, c[1]);
        kahan_add_d(ac.z, cp.z, c[2]);
        kahan_add_d(ac.w, cp.w, c[3]);
        *cpp = cp;
      } else {
        ac.x += c[0]; ac.y += c[1]; ac.z += c[2]; ac.w += c[3];
      }
      *accp = ac;
    }
    qu0 = qu1; qu1 = qu2;
    qb0 = qb1; qb1 = qb2;
  }
}

constexpr int kWarpsDen = 4;

template <typename T>
static cudaError_t launch_den(const StepArgs& a, cudaStream_t s) {
  const Geom& g = a.g;
  const int64_t nstrips = (g.nx + kStrip - 1) / kStrip;
  if (g.ndim == 3) {
    const int64_t warps = nstrips * g.ny * ((g.nz + a.zblock - 1) / a.zblock);
    const int64_t blocks = (warps + kWarpsDen - 1) / kWarpsDen;
    step3d_density_kernel<T, kWarpsDen><<<(unsigned)blocks, kWarpsDen * 32, 0, s>>>(a);
    count_launch();
    return cudaGetLastError();
  }
  if (g.ndim != 2) return cudaErrorInvalidValue;
  const int64_t warps = nstrips * ((g.ny + a.zblock - 1) / a.zblock);
  const int64_t blocks = (warps + kWarpsDen - 1) / kWarpsDen;
  step2d_density_kernel<T, kWarpsDen><<<(unsigned)blocks, kWarpsDen * 32, 0, s>>>(a);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_step_density(const StepArgs& a, int storage, cudaStream_t s) {
  switch (storage) {
    case WAVE_F32: return launch_den<float>(a, s);
    case WAVE_BF16: return launch_den<__nv_bfloat16>(a, s);
    case WAVE_F16: return launch_den<__half>(a, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace wave
