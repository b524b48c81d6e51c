// 3D fused leapfrog step, FP32 storage, one or many shots per launch, with
// the u^n planes staged by TMA bulk copies (cp.async.bulk, one per row)
// into a shared-memory ring managed by mbarriers.  Same arithmetic as the
// other velocity step kernels (Eq. FDstencil1 in squared-slowness form;
// Algorithm 1's incrementKernel of Eq. kernel1).
//
// Pipeline (per CTA: TY consumer warps = TY rows x 128 cells, one z-block):
// * the sequence of plane loads of the CTA runs over all listed shots
//   (planes z0-r .. z1+r-1 of shot 0, then of shot 1, ...); load L goes to
//   ring slot L mod P (P = 2r+1+D);
// * the producer duty rotates over the warps (the warp whose turn it is in
//   consumer iteration i issues that iteration's loads), keeping the loads
//   D planes ahead of the newest plane a warp needs.  Lane i copies row i of
//   the staged tile (r halo rows, TY own rows, r halo rows; 4 halo cells per
//   side) with one bulk copy; lane 0 posts the expected bytes on the slot's
//   "full" mbarrier.
//   Rows and planes that are zero under the Dirichlet mirror are zero-filled
//   with ordinary stores instead; mirrored rows / planes are copied from
//   their mirror images and the consumers apply the mirror sign;
// * each consumer warp waits on the "full" barrier of every load it has
//   not waited on yet, computes its row of plane z, and releases the oldest
//   load of its window on the slot's "empty" barrier; the producer waits on
//   "empty" before it reuses a slot.  There is no CTA-wide barrier per
//   plane, and the next shot's first planes are prefetched while the current
//   shot finishes;
// * every wait is bounded (about one second of clock cycles): on time-out the
//   kernel records an error word and every warp leaves its loop.  Copies in
//   flight are waited for (bounded) before the CTA exits.
#include "stencil_common.cuh"

namespace wave {

namespace {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// Bounded wait on an mbarrier phase.  Returns false on time-out or when the
// CTA has already aborted.
__device__ __forceinline__ bool wait_phase(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                           long long limit) {
  const long long t0 = clock64();
  for (uint32_t it = 0;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 63) == 63) {
      if (*abort_flag) return false;
      if (clock64() - t0 > limit) {
        *abort_flag = 1;
        return false;
      }
    }
  }
}

template <int R, int TY, int D>
struct Tma {
  static constexpr int P = 2 * R + 1 + D;
  static constexpr int ROWS = TY + 2 * R;
  static constexpr int PLANE = ROWS * kRowW;
  static constexpr size_t bytes() { return (size_t)P * PLANE * sizeof(float) + 2 * P * sizeof(uint64_t) + 16; }
};

template <int R, int TY, int D>
__global__ void __launch_bounds__(TY * 32, (TY == 8 ? 2 : 1))
step3d_velocity_tma_kernel(BatchArgs b) {
  static_assert(TY + 2 * R <= 32, "one producer lane per staged row");
  using TM = Tma<R, TY, D>;
  extern __shared__ __align__(128) float ring[];
  uint64_t* full = reinterpret_cast<uint64_t*>(ring + TM::P * TM::PLANE);
  uint64_t* empty = full + TM::P;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(empty + TM::P);

  const StepArgs& a = b.base;
  const Geom& g = a.g;
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const int z0 = (int)((int64_t)blockIdx.x * a.zblock);
  const int z1 = (int)min((int64_t)z0 + a.zblock, g.nz);
  const int nzb = z1 - z0;
  const int per_shot = nzb + 2 * R;                 // loads per shot
  const int nloads = b.nshots * per_shot;
  const int64_t x0 = (int64_t)blockIdx.y * kStrip;
  const int64_t ty0 = (int64_t)blockIdx.z * TY;
  const int64_t y = ty0 + warp;
  const int64_t xl = x0 + 4 * lane;
  const bool row_valid = y < g.ny;
  const bool xfix = (x0 == 0) || (x0 + kStrip + R > g.nx);
  const int64_t row_off = y * g.px + xl;
  const int col = 4 + 4 * lane;
  const long long limit = b.wait_limit_cycles;

  if (tid == 0) {
    for (int s = 0; s < TM::P; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], TY);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();

  // ---- producer state (warp 0): the staged row `lane` of every plane -------
  const int rr = lane;
  const int64_t yy = ty0 - R + rr;
  float prow_sign = 0.f;
  int64_t prow_off = 0;
  if (rr < TM::ROWS && yy >= -R && yy < g.ny + R) prow_off = mirror_index(yy, g.ny, g.bc, &prow_sign) * g.px;
  const int64_t xs = x0 - 4 < 0 ? 0 : x0 - 4;
  const int64_t xe = x0 + kStrip + 4 > g.px ? g.px : x0 + kStrip + 4;
  const uint32_t row_bytes = (uint32_t)((xe - xs) * sizeof(float));
  const int row_dst = rr * kRowW + (int)(xs - (x0 - 4));
  int issued = 0;

  auto issue = [&](int L) -> bool {  // warp 0, all lanes
    const int slot = L % TM::P;
    const int use = L / TM::P;
    bool w = true;
    if (use >= 1) w = wait_phase(&empty[slot], (uint32_t)((use - 1) & 1), abort_flag, limit);
    if (!__all_sync(0xffffffffu, w)) return false;  // warp-uniform decision
    const int s = L / per_shot;
    const int p = z0 - R + (L - s * per_shot);
    float zs;
    const int64_t zsrc = mirror_index(p, g.nz, g.bc, &zs);
    float* dst0 = ring + slot * TM::PLANE;
    const bool copy = b.debug_stall == 0 && rr < TM::ROWS && zs != 0.f && prow_sign != 0.f;
    if (rr < TM::ROWS && !copy && b.debug_stall == 0) {  // zero row (Dirichlet wall or unused)
      float4* d = reinterpret_cast<float4*>(dst0 + rr * kRowW);
      for (int c = 0; c < kRowW / 4; ++c) d[c] = make_float4(0.f, 0.f, 0.f, 0.f);
      fence_proxy_async();  // ordered before later bulk copies into this slot
    }
    const unsigned m = __ballot_sync(0xffffffffu, copy);
    const uint32_t total = (uint32_t)__popc(m) * row_bytes;
    __syncwarp();
    if (lane == 0 && b.debug_stall == 0) mbar_arrive_expect_tx(&full[slot], total);
    __syncwarp();
    if (copy) {
      const float* src = b.cur[s] + zsrc * g.plane + prow_off + xs;
      bulk_g2s(dst0 + row_dst, src, row_bytes, &full[slot]);
    }
    return true;
  };

  bool ok = true;
  // prologue: the first P loads, spread over the warps
  const int first = min(nloads, TM::P);
  for (int L = warp; L < first; L += TY) issue(L);
  issued = first;   // loads issued by all warps so far (identical in every warp)
  int iter = 0;     // consumer iteration over all shots (identical in every warp)

  // ---- consumers --------------------------------------------------------
  // mirror signs of the y-neighbour rows of this warp's row (constant in z)
  float ysm[R + 1], ysp[R + 1];
  bool yone = true;
#pragma unroll
  for (int j = 1; j <= R; ++j) {
    float s1 = 0.f, s2 = 0.f;
    if (y - j >= -R) mirror_index(y - j, g.ny, g.bc, &s1);
    if (y + j < g.ny + R) mirror_index(y + j, g.ny, g.bc, &s2);
    ysm[j] = s1;
    ysp[j] = s2;
    yone = yone && s1 == 1.f && s2 == 1.f;
  }
  int waited = 0;  // loads this warp has waited on
  for (int s = 0; s < b.nshots && ok; ++s) {
    float* __restrict__ up = b.prev[s];
    const bool acc_on = b.accf[s] != 0;
    const float acc_sc = a.acc_scale * b.accf[s];  // per-shot sign and on/off
    const int base = s * per_shot;  // load index of plane z0-R of this shot
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
    if (row_valid && nzb > 0) load_streams(z0, u_old, cf, ac, cp);
    for (int z = z0; z < z1; ++z) {
      const int lnew = base + (z - z0) + 2 * R;  // load of plane z+R
      const int target = min(nloads, lnew + D + 1);
      if (warp == iter % TY) {
        for (int L = issued; L < target && ok; ++L) ok = issue(L);
      }
      issued = target > issued ? target : issued;
      ++iter;
      while (ok && waited <= lnew) {
        const bool w = wait_phase(&full[waited % TM::P], (uint32_t)((waited / TM::P) & 1), abort_flag, limit);
        ok = __all_sync(0xffffffffu, w);  // warp-uniform decision
        if (ok) ++waited;
      }
      if (!ok) break;
      float4 n_old = u_old, n_cf = cf, n_ac = ac, n_cp = cp;
      if (row_valid && z + 1 < z1) load_streams(z + 1, n_old, n_cf, n_ac, n_cp);
      if (row_valid) {
        const int lz = base + (z - z0) + R;  // load of plane z
        const float* cplane = ring + (lz % TM::P) * TM::PLANE;
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
        const float4 u = mask_row_padding(*reinterpret_cast<const float4*>(srow + col), xl, g.nx);
        const bool zone = (z - R >= 0) && (z + R < g.nz);
#pragma unroll
        for (int j = 1; j <= R; ++j) {
          float4 ym = *reinterpret_cast<const float4*>(cplane + (R + warp - j) * kRowW + col);
          float4 yp = *reinterpret_cast<const float4*>(cplane + (R + warp + j) * kRowW + col);
          float4 zm = *reinterpret_cast<const float4*>(ring + ((lz - j) % TM::P) * TM::PLANE + (R + warp) * kRowW + col);
          float4 zp = *reinterpret_cast<const float4*>(ring + ((lz + j) % TM::P) * TM::PLANE + (R + warp) * kRowW + col);
          if (!yone) {
            ym = f4_scale(ym, ysm[j]);
            yp = f4_scale(yp, ysp[j]);
          }
          if (!zone) {
            float sm = 1.f, sp = 1.f;
            mirror_index(z - j, g.nz, g.bc, &sm);
            mirror_index(z + j, g.nz, g.bc, &sp);
            zm = f4_scale(zm, sm);
            zp = f4_scale(zp, sp);
          }
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
            ac.x = fmaf(acc_sc * d0, d0, ac.x);
            ac.y = fmaf(acc_sc * d1, d1, ac.y);
            ac.z = fmaf(acc_sc * d2, d2, ac.z);
            ac.w = fmaf(acc_sc * d3, d3, ac.w);
          }
          *reinterpret_cast<float4*>(a.acc + off) = ac;
        }
        if (xfix) fence_proxy_async();  // generic writes above precede the slot's next bulk copy
      }
      u_old = n_old;
      cf = n_cf;
      ac = n_ac;
      cp = n_cp;
      // release the oldest load of the window; after the shot's last plane,
      // release its remaining 2r loads as well
      __syncwarp();
      if (lane == 0) {
        const int lo = base + (z - z0);
        const int hi = z + 1 == z1 ? base + per_shot - 1 : lo;
        for (int l = lo; l <= hi; ++l) mbar_arrive(&empty[l % TM::P]);
      }
    }
  }
  if (!ok && b.err) atomicOr(b.err, 1);
  // Copies this CTA issued must land before it exits.  On the normal path
  // every warp has waited on every load; after a time-out, wait (bounded,
  // briefly per load) for the loads this warp has not seen complete.
  if (!ok && b.debug_stall == 0) {
    for (int l = waited; l < issued; ++l) {
      const long long t0 = clock64();
      while (!mbar_try_wait(&full[l % TM::P], (uint32_t)((l / TM::P) & 1)) && clock64() - t0 < (limit >> 6)) {
      }
    }
  }
  __syncthreads();
}

template <int R, int TY, int D>
cudaError_t launch_tma(const BatchArgs& b, cudaStream_t s) {
  using TM = Tma<R, TY, D>;
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(step3d_velocity_tma_kernel<R, TY, D>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TM::bytes());
    if (e != cudaSuccess) return e;
    configured = true;
  }
  const Geom& g = b.base.g;
  dim3 grid((unsigned)((g.nz + b.base.zblock - 1) / b.base.zblock), (unsigned)((g.nx + kStrip - 1) / kStrip),
            (unsigned)((g.ny + TY - 1) / TY));
  step3d_velocity_tma_kernel<R, TY, D><<<grid, TY * 32, TM::bytes(), s>>>(b);
  count_launch();
  return cudaGetLastError();
}

template <int R>
cudaError_t launch_tma_r(const BatchArgs& b, cudaStream_t s) {
  if (b.base.tile_rows == 16) return b.base.ring_depth == 2 ? launch_tma<R, 16, 2>(b, s) : launch_tma<R, 16, 3>(b, s);
  return b.base.ring_depth == 2 ? launch_tma<R, 8, 2>(b, s) : launch_tma<R, 8, 3>(b, s);
}

}  // namespace

cudaError_t launch_step3d_tma(const BatchArgs& b, int order, cudaStream_t s) {
  switch (order) {
    case 2: return launch_tma_r<1>(b, s);
    case 4: return launch_tma_r<2>(b, s);
    case 6: return launch_tma_r<3>(b, s);
    case 8: return launch_tma_r<4>(b, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace wave
