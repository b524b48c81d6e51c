// 3D fused leapfrog step, FP32 storage, one or many shots per launch:
// shared-memory plane ring fed by cp.async, two planes per CTA barrier.
//
// Same tile, ring and arithmetic as step3d_ring.cu (Eq. FDstencil1 in
// squared-slowness form; Algorithm 1's incrementKernel of Eq. kernel1); the
// march advances two planes per __syncthreads / cp.async wait, the
// streaming operands alternate between two register sets instead of being
// copied every plane, and the staging uses precomputed 32-bit in-plane
// offsets with a sign-free fast path for tiles and planes away from the
// domain boundary.  With P = 2r + D + 2 ring slots, the two planes issued in
// an iteration reuse the slots of the two planes the previous iteration
// released.
#include "stencil_common.cuh"

namespace wave {

namespace {

__device__ __forceinline__ void cp16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void wait_groups() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

template <int R, int TY, int D>
struct Ring2 {
  static constexpr int P = 2 * R + D + 2;        // planes held
  static constexpr int ROWS = TY + 2 * R;
  static constexpr int CH = kRowW / 4;
  static constexpr int NT = TY * 32;
  static constexpr int K = (ROWS * CH + NT - 1) / NT;
  static constexpr int PLANE = ROWS * kRowW;
  static constexpr size_t bytes() { return (size_t)P * PLANE * sizeof(float); }
};

template <int R, int TY, int D>
__global__ void __launch_bounds__(TY * 32, 2)
step3d_velocity_ring2_kernel(BatchArgs b) {
  using RG = Ring2<R, TY, D>;
  static_assert(D >= 2, "two planes are staged per iteration");
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
  const bool row_valid = y < g.ny;
  const bool xfix = (x0 == 0) || (x0 + kStrip + R > g.nx);
  const int64_t row_off = y * g.px + x0 + 4 * lane;
  const int col = 4 + 4 * lane;
  const int own = (R + warp) * kRowW + col;      // own cells in a staged plane
  // tiles whose staged rows and columns all lie inside the grid copy every
  // chunk with cp.async (no mirror signs)
  const bool tile_inside = (ty0 - R >= 0) && (ty0 + TY + R <= g.ny) && (x0 >= 4) && (x0 + kStrip + 4 <= g.px);

  // staging descriptors: 32-bit in-plane source offset, row mirror sign,
  // destination offset in a staged plane (-1: no chunk)
  int c_off[RG::K];
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
        c_off[k] = (int)(ysrc * g.px + xx);
      }
    }
  }

  for (int shot = 0; shot < b.nshots; ++shot) {
    const float* __restrict__ uc = b.cur[shot];
    float* __restrict__ up = b.prev[shot];
    const bool acc_on = b.accf[shot] != 0;
    const float acc_sc = a.acc_scale * b.accf[shot];  // per-shot sign and on/off

    auto issue = [&](int p, int slot) {
      if (p < z1 + R) {
        float* dst0 = ring + slot * RG::PLANE;
        if (tile_inside && p >= 0 && p < g.nz) {
          const float* src0 = uc + (int64_t)p * g.plane;
#pragma unroll
          for (int k = 0; k < RG::K; ++k)
            if (c_dst[k] >= 0) cp16(dst0 + c_dst[k], src0 + c_off[k]);
        } else {
          float zs;
          const int64_t zsrc = mirror_index(p, g.nz, g.bc, &zs);
          const float* src0 = uc + zsrc * g.plane;
#pragma unroll
          for (int k = 0; k < RG::K; ++k) {
            if (c_dst[k] < 0) continue;
            const float sgn = c_sgn[k] * zs;
            float* dst = dst0 + c_dst[k];
            if (sgn == 0.f) {
              *reinterpret_cast<float4*>(dst) = make_float4(0.f, 0.f, 0.f, 0.f);
            } else if (sgn > 0.f) {
              cp16(dst, src0 + c_off[k]);
            } else {
              *reinterpret_cast<float4*>(dst) = f4_scale(__ldg(reinterpret_cast<const float4*>(src0 + c_off[k])), sgn);
            }
          }
        }
      }
      commit();
    };

    // prologue: planes z0-R .. z0+R+D-1 into slots 0 .. 2R+D-1
#pragma unroll 1
    for (int i = 0; i < 2 * R + D; ++i) issue(z0 - R + i, i);
    int s0 = 0;  // slot of plane z - R

    auto load = [&](int z, float4& uo, float4& c, float4& acv, float4& cpv) {
      const int64_t off = (int64_t)z * g.plane + row_off;
      uo = *reinterpret_cast<const float4*>(up + off);
      c = __ldg(reinterpret_cast<const float4*>(a.coef + off));
      if (acc_on) {
        acv = *reinterpret_cast<const float4*>(a.acc + off);
        if (a.comp) cpv = *reinterpret_cast<const float4*>(a.comp + off);
      }
    };
    // One plane z of this warp's row; slot of plane z-R is `lo`.
    auto compute = [&](int z, int lo, const float4& u_old, const float4& cf, float4& ac, float4& cp) {
      int sl[2 * R + 1];
#pragma unroll
      for (int j = 0; j <= 2 * R; ++j) {
        const int t = lo + j;
        sl[j] = t >= RG::P ? t - RG::P : t;
      }
      float* cplane = ring + sl[R] * RG::PLANE;
      float* srow = cplane + (R + warp) * kRowW;
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
      const float4 u = mask_row_padding(*reinterpret_cast<const float4*>(cplane + own), x0 + 4 * lane, g.nx);
      // y / z terms and the update on pairs of cells (paired FP32 ops of
      // sm_100-class GPUs; each element rounds as the scalar code would)
      float2 l01 = make_float2(lap[0], lap[1]), l23 = make_float2(lap[2], lap[3]);
#pragma unroll
      for (int j = 1; j <= R; ++j) {
        const float4 ym = *reinterpret_cast<const float4*>(cplane + own - j * kRowW);
        const float4 yp = *reinterpret_cast<const float4*>(cplane + own + j * kRowW);
        const float4 zm = *reinterpret_cast<const float4*>(ring + sl[R - j] * RG::PLANE + own);
        const float4 zp = *reinterpret_cast<const float4*>(ring + sl[R + j] * RG::PLANE + own);
        const float2 c2 = make_float2(cw<R>(j), cw<R>(j));
        l01 = __ffma2_rn(c2, __fadd2_rn(__fadd2_rn(make_float2(ym.x, ym.y), make_float2(yp.x, yp.y)),
                                        __fadd2_rn(make_float2(zm.x, zm.y), make_float2(zp.x, zp.y))), l01);
        l23 = __ffma2_rn(c2, __fadd2_rn(__fadd2_rn(make_float2(ym.z, ym.w), make_float2(yp.z, yp.w)),
                                        __fadd2_rn(make_float2(zm.z, zm.w), make_float2(zp.z, zp.w))), l23);
      }
      const float2 two = make_float2(2.f, 2.f);
      const float2 n01 = __ffma2_rn(make_float2(cf.x, cf.y), l01,
                                    __ffma2_rn(two, make_float2(u.x, u.y), make_float2(-u_old.x, -u_old.y)));
      const float2 n23 = __ffma2_rn(make_float2(cf.z, cf.w), l23,
                                    __ffma2_rn(two, make_float2(u.z, u.w), make_float2(-u_old.z, -u_old.w)));
      float4 un = make_float4(n01.x, n01.y, n23.x, n23.y);
      const int64_t off = (int64_t)z * g.plane + row_off;
      *reinterpret_cast<float4*>((a.u_out ? reinterpret_cast<float*>(a.u_out) : up) + off) = un;
      if (a.mix_a) {
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
          const float2 sc = make_float2(acc_sc, acc_sc);
          const float2 e01 = make_float2(d0, d1), e23 = make_float2(d2, d3);
          const float2 r01 = __ffma2_rn(__fmul2_rn(sc, e01), e01, make_float2(ac.x, ac.y));
          const float2 r23 = __ffma2_rn(__fmul2_rn(sc, e23), e23, make_float2(ac.z, ac.w));
          ac = make_float4(r01.x, r01.y, r23.x, r23.y);
        }
        *reinterpret_cast<float4*>(a.acc + off) = ac;
      }
    };

    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 oa = zero4, ca = zero4, aa = zero4, pa = zero4;   // streams of plane z
    float4 ob = zero4, cb = zero4, ab = zero4, pb = zero4;   // streams of plane z+1
    if (row_valid) load(z0, oa, ca, aa, pa);
    for (int z = z0; z < z1; z += 2) {
      // planes up to z+1+R are complete once at most D-2 newer groups remain
      wait_groups<D - 2>();
      __syncthreads();
      {
        int sn = s0 + 2 * R + D;         // slot of plane z+R+D (was plane z-R-2)
        sn -= sn >= RG::P ? RG::P : 0;
        int sm = sn + 1;                 // slot of plane z+R+D+1 (was plane z-R-1)
        sm -= sm >= RG::P ? RG::P : 0;
        issue(z + R + D, sn);
        issue(z + R + D + 1, sm);
      }
      const bool two = z + 1 < z1;
      if (row_valid && two) load(z + 1, ob, cb, ab, pb);
      if (row_valid) compute(z, s0, oa, ca, aa, pa);
      int s1 = s0 + 1;
      s1 -= s1 >= RG::P ? RG::P : 0;
      if (row_valid && z + 2 < z1) load(z + 2, oa, ca, aa, pa);
      if (row_valid && two) compute(z + 1, s1, ob, cb, ab, pb);
      s0 = s1 + 1;
      s0 -= s0 >= RG::P ? RG::P : 0;
    }
    wait_groups<0>();
    __syncthreads();  // the ring is refilled for the next shot
  }
}

template <int R, int TY, int D>
cudaError_t launch_r2(const BatchArgs& b, cudaStream_t s) {
  using RG = Ring2<R, TY, D>;
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(step3d_velocity_ring2_kernel<R, TY, D>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)RG::bytes());
    if (e != cudaSuccess) return e;
    configured = true;
  }
  const Geom& g = b.base.g;
  dim3 grid((unsigned)((g.nz + b.base.zblock - 1) / b.base.zblock), (unsigned)((g.nx + kStrip - 1) / kStrip),
            (unsigned)((g.ny + TY - 1) / TY));
  step3d_velocity_ring2_kernel<R, TY, D><<<grid, TY * 32, RG::bytes(), s>>>(b);
  count_launch();
  return cudaGetLastError();
}

template <int R>
cudaError_t launch_r2_r(const BatchArgs& b, cudaStream_t s) {
  return b.base.ring_depth == 2 ? launch_r2<R, 8, 2>(b, s) : launch_r2<R, 8, 3>(b, s);
}

}  // namespace

cudaError_t launch_step3d_ring2(const BatchArgs& b, int order, cudaStream_t s) {
  switch (order) {
    case 2: return launch_r2_r<1>(b, s);
    case 4: return launch_r2_r<2>(b, s);
    case 6: return launch_r2_r<3>(b, s);
    case 8: return launch_r2_r<4>(b, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace wave
