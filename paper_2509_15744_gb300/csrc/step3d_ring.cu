// 3D fused leapfrog step, FP32 storage, orders 2-8, one or many shots per
// launch: shared-memory plane ring filled by cp.async.  Same arithmetic as
// the register-queue kernel (Eq. FDstencil1 in squared-slowness form,
// sensitivity increment of Algorithm 1 / Eq. kernel1) with a different
// mapping:
//
// * the grid runs z-blocks fastest, so vertically adjacent CTAs (which share
//   r halo planes) run side by side and the halo planes come from L2;
// * with several shots (batched mode), a CTA advances each listed shot in
//   turn over its tile; the shots' increments go into the one accumulator
//   K~ (summed over sources), whose tile stays in L2 between shots, so per
//   shot and cell HBM sees u^n, u^{n-1}, u^{n+1} (12 B) and coef / acc only
//   once per step for all shots;
//
// * a CTA of TY warps owns TY rows x 128 cells and marches up z over a block
//   of planes;
// * it keeps P = 2r+1+D planes of its tile (own rows + r halo rows above and
//   below, each row with 4 halo cells per side) in a shared-memory ring;
//   plane z+r+D is copied asynchronously (cp.async, 16-byte chunks, L2 ->
//   shared memory) while plane z is computed, so D planes of u^n are in
//   flight per CTA without occupying registers;
// * the streaming operands of plane z+1 (u^{n-1}, coef, acc[, comp]) are
//   loaded into registers while plane z is computed;
// * rows and planes outside the domain are staged from their mirror images
//   (negated for a Dirichlet mirror, zero on the wall node); the x ghosts of
//   the own rows are filled warp-locally right before use;
// * one __syncthreads per plane.
#include <string.h>

#include "stencil_common.cuh"

namespace wave {

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

template <int R, int TY, int D>
struct Ring {
  static constexpr int P = 2 * R + 1 + D;       // planes held
  static constexpr int ROWS = TY + 2 * R;       // staged rows per plane
  static constexpr int CH = kRowW / 4;          // 16-byte chunks per staged row
  static constexpr int NT = TY * 32;            // threads
  static constexpr int K = (ROWS * CH + NT - 1) / NT;  // chunks per thread per plane
  static constexpr int PLANE = ROWS * kRowW;    // floats per staged plane
  static constexpr size_t bytes() { return (size_t)P * PLANE * sizeof(float); }
};

template <int R, int TY, int D>
__global__ void __launch_bounds__(TY * 32, (TY == 8 ? 2 : 1))
step3d_velocity_ring_kernel(BatchArgs b) {
  using RG = Ring<R, TY, D>;
  extern __shared__ __align__(16) float ring[];
  const StepArgs& a = b.base;
  const Geom& g = a.g;
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const int z0 = (int)((int64_t)blockIdx.x * a.zblock);
  const int z1 = (int)min((int64_t)z0 + a.zblock, g.nz);
  const int64_t x0 = (int64_t)blockIdx.y * kStrip;
  const int64_t ty0 = (int64_t)blockIdx.z * TY;
  const int64_t y = ty0 + warp;
  const int64_t xl = x0 + 4 * lane;
  const bool row_valid = y < g.ny;
  const bool xfix = (x0 == 0) || (x0 + kStrip + R > g.nx);
  const int64_t row_off = y * g.px + xl;

  // Per-thread staging descriptors, fixed for the whole march: source row
  // offset in a plane, mirror sign of the row (0: zero chunk), offset in a
  // staged plane.
  int64_t c_off[RG::K];
  float c_sgn[RG::K];
  int c_dst[RG::K];
#pragma unroll
  for (int k = 0; k < RG::K; ++k) {
    const int c = tid + k * RG::NT;
    c_sgn[k] = 0.f;
    c_off[k] = 0;
    c_dst[k] = -1;
    if (c < RG::ROWS * RG::CH) {
      const int rr = c / RG::CH, ch = c - rr * RG::CH;
      const int64_t yy = ty0 - R + rr;
      const int64_t xx = x0 - 4 + 4 * ch;
      c_dst[k] = rr * kRowW + 4 * ch;
      if (yy >= -R && yy < g.ny + R && xx >= 0 && xx + 4 <= g.px) {
        float ys;
        const int64_t ysrc = mirror_index(yy, g.ny, g.bc, &ys);
        c_sgn[k] = ys;
        c_off[k] = ysrc * g.px + xx;
      }
    }
  }

  for (int shot = 0; shot < b.nshots; ++shot) {
    const float* __restrict__ uc = b.cur[shot];
    float* __restrict__ up = b.prev[shot];
    const bool acc_on = b.accf[shot] != 0;
    const float acc_sc = a.acc_scale * b.accf[shot];  // per-shot sign and on/off
    // Stage plane p into ring slot `slot`; always commits one group.
    auto issue = [&](int p, int slot) {
      if (p < z1 + R) {
        float zs;
        const int64_t zsrc = mirror_index(p, g.nz, g.bc, &zs);
        const float* src0 = uc + zsrc * g.plane;
        float* dst0 = ring + slot * RG::PLANE;
  #pragma unroll
        for (int k = 0; k < RG::K; ++k) {
          if (c_dst[k] < 0) continue;
          const float sgn = c_sgn[k] * zs;
          float* dst = dst0 + c_dst[k];
          if (sgn == 0.f) {
            *reinterpret_cast<float4*>(dst) = make_float4(0.f, 0.f, 0.f, 0.f);
          } else if (sgn > 0.f) {
            cp_async16(dst, src0 + c_off[k]);
          } else {
            *reinterpret_cast<float4*>(dst) = f4_scale(__ldg(reinterpret_cast<const float4*>(src0 + c_off[k])), sgn);
          }
        }
      }
      cp_async_commit();
    };

    // prologue: planes z0-R .. z0+R+D-1 into slots 0 .. 2R+D-1 (drained and
    // fenced by the __syncthreads at the end of the previous shot)
  #pragma unroll 1
    for (int i = 0; i < 2 * R + D; ++i) issue(z0 - R + i, i);
    int s0 = 0;  // slot of plane z - R

    float4 u_old = make_float4(0.f, 0.f, 0.f, 0.f), cf = u_old, ac = u_old, cp = u_old;
    auto load_streams = [&](int z, float4& uo, float4& c, float4& acv, float4& cpv) {
      const int64_t off = (int64_t)z * g.plane + row_off;
      uo = *reinterpret_cast<const float4*>(up + off);
      c = __ldg(reinterpret_cast<const float4*>(a.coef + off));
      if (acc_on) {
        acv = *reinterpret_cast<const float4*>(a.acc + off);
        if (a.comp) cpv = *reinterpret_cast<const float4*>(a.comp + off);
      }
    };
    if (row_valid && z0 < z1) load_streams(z0, u_old, cf, ac, cp);

    const int col = 4 + 4 * lane;
    for (int z = z0; z < z1; ++z) {
      cp_async_wait<D - 1>();
      __syncthreads();
      // plane z+R+D reuses the slot of plane z-R-1 (read last in iteration z-1)
      {
        int sn = s0 + 2 * R + D;
        sn -= sn >= RG::P ? RG::P : 0;
        issue(z + R + D, sn);
      }
      float4 n_old = u_old, n_cf = cf, n_ac = ac, n_cp = cp;
      if (row_valid && z + 1 < z1) load_streams(z + 1, n_old, n_cf, n_ac, n_cp);
      if (row_valid) {
        int sl[2 * R + 1];   // slots of planes z-R .. z+R
  #pragma unroll
        for (int j = 0; j <= 2 * R; ++j) {
          const int t = s0 + j;
          sl[j] = t >= RG::P ? t - RG::P : t;
        }
        const float* cplane = ring + sl[R] * RG::PLANE;
        float* srow = const_cast<float*>(cplane) + (R + warp) * kRowW;
        if (xfix) {
          float val = 0.f;
          int pos = -1;
          int64_t gx = 0;
          if (lane < R && x0 == 0) {
            gx = -1 - lane;
            pos = 3 - lane;
          } else if (lane >= 8 && lane < 8 + R) {
            gx = (g.nx < x0 + kStrip ? g.nx : x0 + kStrip) + (lane - 8);
            if (gx >= g.nx) pos = (int)(gx - x0 + 4);
          }
          __syncwarp();
          if (pos >= 0) {
            float sx;
            const int64_t m = mirror_index(gx, g.nx, g.bc, &sx);
            val = sx == 0.f ? 0.f : sx * srow[m - x0 + 4];
          }
          __syncwarp();
          if (pos >= 0) srow[pos] = val;
          __syncwarp();
        }
        float lap[4];
        x_terms<R>(srow, lane, lap, 3.f * cw<R>(0));
        const float4 u = mask_row_padding(*reinterpret_cast<const float4*>(srow + 4 + 4 * lane), xl, g.nx);
  #pragma unroll
        for (int j = 1; j <= R; ++j) {
          const float4 ym = *reinterpret_cast<const float4*>(cplane + (R + warp - j) * kRowW + col);
          const float4 yp = *reinterpret_cast<const float4*>(cplane + (R + warp + j) * kRowW + col);
          const float4 zm = *reinterpret_cast<const float4*>(ring + sl[R - j] * RG::PLANE + (R + warp) * kRowW + col);
          const float4 zp = *reinterpret_cast<const float4*>(ring + sl[R + j] * RG::PLANE + (R + warp) * kRowW + col);
          const float c = cw<R>(j);
          lap[0] = fmaf(c, (ym.x + yp.x) + (zm.x + zp.x), lap[0]);
          lap[1] = fmaf(c, (ym.y + yp.y) + (zm.y + zp.y), lap[1]);
          lap[2] = fmaf(c, (ym.z + yp.z) + (zm.z + zp.z), lap[2]);
          lap[3] = fmaf(c, (ym.w + yp.w) + (zm.w + zp.w), lap[3]);
        }
        float4 un;
        un.x = fmaf(cf.x, lap[0], 2.f * u.x - u_old.x);
        un.y = fmaf(cf.y, lap[1], 2.f * u.y - u_old.y);
        un.z = fmaf(cf.z, lap[2], 2.f * u.z - u_old.z);
        un.w = fmaf(cf.w, lap[3], 2.f * u.w - u_old.w);
        const int64_t off = (int64_t)z * g.plane + row_off;
        *reinterpret_cast<float4*>(up + off) = un;
        if (a.mix_a) {  // exact mode (one shot): acc += acc_scale (u_cur - u_next)(mix_a - mix_b)
          const float4 ma = *reinterpret_cast<const float4*>(a.mix_a + off);
          const float4 mb = *reinterpret_cast<const float4*>(a.mix_b + off);
          ac.x = fmaf(acc_sc * (u.x - un.x), ma.x - mb.x, ac.x);
          ac.y = fmaf(acc_sc * (u.y - un.y), ma.y - mb.y, ac.y);
          ac.z = fmaf(acc_sc * (u.z - un.z), ma.z - mb.z, ac.z);
          ac.w = fmaf(acc_sc * (u.w - un.w), ma.w - mb.w, ac.w);
          *reinterpret_cast<float4*>(a.acc + off) = ac;
        } else if (acc_on) {
          const float d0 = un.x - u.x, d1 = un.y - u.y, d2 = un.z - u.z, d3 = un.w - u.w;
          if (a.comp) {
            kahan_add(ac.x, cp.x, acc_sc * d0 * d0);
            kahan_add(ac.y, cp.y, acc_sc * d1 * d1);
            kahan_add(ac.z, cp.z, acc_sc * d2 * d2);
            kahan_add(ac.w, cp.w, acc_sc * d3 * d3);
            *reinterpret_cast<float4*>(a.comp + off) = cp;
          } else {
            ac.x = fmaf(acc_sc * d0, d0, ac.x);
            ac.y = fmaf(acc_sc * d1, d1, ac.y);
            ac.z = fmaf(acc_sc * d2, d2, ac.z);
            ac.w = fmaf(acc_sc * d3, d3, ac.w);
          }
          *reinterpret_cast<float4*>(a.acc + off) = ac;
        }
      }
      u_old = n_old;
      cf = n_cf;
      ac = n_ac;
      cp = n_cp;
      s0 = s0 + 1 == RG::P ? 0 : s0 + 1;
    }
    cp_async_wait<0>();
    __syncthreads();  // the ring is refilled for the next shot
  }
}

template <int R, int TY, int D>
static cudaError_t launch_ring(const BatchArgs& a, cudaStream_t s) {
  using RG = Ring<R, TY, D>;
  cudaError_t e = set_smem_limit_once(reinterpret_cast<const void*>(step3d_velocity_ring_kernel<R, TY, D>), (int)RG::bytes());
  if (e != cudaSuccess) return e;
  const Geom& g = a.base.g;
  dim3 grid((unsigned)((g.nz + a.base.zblock - 1) / a.base.zblock), (unsigned)((g.nx + kStrip - 1) / kStrip),
            (unsigned)((g.ny + TY - 1) / TY));
  step3d_velocity_ring_kernel<R, TY, D><<<grid, TY * 32, RG::bytes(), s>>>(a);
  count_launch();
  e = cudaGetLastError();
  if (e != cudaSuccess) note_error("step kernel launch", e);
  return e;
}

template <int R>
static cudaError_t launch_ring_r(const BatchArgs& a, cudaStream_t s) {
  if (a.base.tile_rows == 16)
    return a.base.ring_depth == 2 ? launch_ring<R, 16, 2>(a, s) : launch_ring<R, 16, 3>(a, s);
  return a.base.ring_depth == 2 ? launch_ring<R, 8, 2>(a, s) : launch_ring<R, 8, 3>(a, s);
}

cudaError_t launch_step3d_batched(const BatchArgs& b, int order, cudaStream_t s) {
  // The plane-major launch order of pipelines 3 and 4 puts the z-blocks in
  // gridDim.z (at most 65535); a grid with more z-blocks launches in the
  // z-block-fastest order (z-blocks in gridDim.x), which computes the same.
  if (b.base.cta_order && b.base.zblock > 0 && (b.base.g.nz + b.base.zblock - 1) / b.base.zblock > 65535) {
    BatchArgs c = b;
    c.base.cta_order = 0;
    return launch_step3d_batched(c, order, s);
  }
  // Pipelines: 0 this cp.async ring (64-bit offsets: any grid, the fallback);
  // 3 register queue in z; 4 two fields per pass; 5 two fields per pass with
  // TMA tensor tiles.  A launch of one field goes to the register queue from
  // pipelines 3-5.  Pipeline 5 takes every launch of two or more fields it
  // supports.
  if (b.base.pipeline == 5 && b.nshots >= 2 && stream_supported(b)) return launch_step3d_stream(b, order, s);
  // the fused (u, lambda) pair of the exact reverse-time mode runs only in the pair kernels
  if (b.pair_mix) return b.nshots == 2 && b.base.g.plane < (int64_t)1 << 31 ? launch_step3d_pair(b, order, s)
                                                                           : cudaErrorInvalidValue;
  // pipeline 4 pairs the fields of a launch; a launch of one field gains nothing from it
  if (b.base.pipeline >= 4 && b.nshots >= 2 && b.base.g.plane < (int64_t)1 << 31 && !b.base.mix_a)
    return launch_step3d_pair(b, order, s);
  if (b.base.pipeline >= 3 && b.base.g.plane < (int64_t)1 << 31) return launch_step3d_queue(b, order, s);
  switch (order) {
    case 2: return launch_ring_r<1>(b, s);
    case 4: return launch_ring_r<2>(b, s);
    case 6: return launch_ring_r<3>(b, s);
    case 8: return launch_ring_r<4>(b, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_step3d_ring(const StepArgs& a, int order, cudaStream_t s) {
  BatchArgs b;
  memset(&b, 0, sizeof(b));
  b.base = a;
  b.nshots = 1;
  b.cur[0] = reinterpret_cast<const float*>(a.u_cur);
  b.prev[0] = reinterpret_cast<float*>(a.u_prev);
  b.accf[0] = a.acc_mass;
  b.err = a.err;
  b.wait_limit_cycles = a.wait_limit_cycles;
  b.debug_stall = a.debug_stall;
  return launch_step3d_batched(b, order, s);
}

}  // namespace wave
