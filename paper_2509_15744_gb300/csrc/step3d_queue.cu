// 3D fused leapfrog step, FP32 storage, orders 2-8, one or many shots per
// launch: z neighbours in a register queue fed from deep-staged plane tiles.
//
// Same arithmetic, element by element, as the plane-ring kernels (Eq.
// FDstencil1 in squared-slowness form; sensitivity increment of Algorithm 1),
// so every pipeline gives bit-identical results.  The mapping:
//
// * a CTA of TY warps owns TY rows x 128 cells and marches up z over a block
//   of planes; each lane keeps its 4 cells of planes z-r .. z+r in registers
//   (a queue of 2r+1 float4, rotated statically by unrolling the march by
//   2r+1 planes), so the z part of the stencil needs no shared-memory loads
//   and no slot arithmetic;
// * the tile of each plane (own rows + r halo rows, 4 halo cells per side)
//   is staged by cp.async D = r+1+depth planes ahead into D+1 buffers; the
//   tile of plane z gives the x and y neighbours, the own row of plane z+r+1
//   (already staged) gives the next queue entry, so u^n is read from HBM once;
// * staging is branch-free: per thread a fixed list of 16-byte chunks with
//   precomputed shared addresses and in-plane offsets, chunks outside the
//   grid zero-filled by the copy itself; only rows behind a Dirichlet
//   mirror (negated) are copied by hand;
// * planes above the domain are staged from their mirror images and enter
//   the queue with the mirror sign; rows outside it are staged from theirs;
//   the x ghosts of the own row are filled warp-locally from precomputed
//   mirror positions;
// * the streaming operands of plane z+1 (u^{n-1}, coef, acc[, comp]) are
//   loaded into registers while plane z is computed; one __syncthreads per
//   plane;
// * with several shots (batched mode) the CTA advances each shot in turn
//   over its tile; their increments go into the one accumulator, whose tile
//   stays in L2 between shots.
// In-plane offsets are 32-bit: the launcher requires px * ny < 2^31.
#include "stencil_common.cuh"

namespace wave {
namespace {

__device__ __forceinline__ void cpa16z(uint32_t sdst, const float* gsrc, uint32_t nbytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sdst), "l"(gsrc), "r"(nbytes) : "memory");
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cpa_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

template <int R, int TY, int DX>
struct QTile {
  static constexpr int Q = 2 * R + 1;            // queue length (planes z-r .. z+r)
  static constexpr int D = R + 1 + DX;           // planes staged ahead of the centre plane
  static constexpr int W = DX - 1;               // copy groups left in flight at each wait
  static constexpr int NB = D + 1;               // tile buffers
  static constexpr int ROWS = TY + 2 * R;        // staged rows per tile
  static constexpr int CH = kRowW / 4;           // 16-byte chunks per staged row
  static constexpr int NT = TY * 32;             // threads
  static constexpr int K = (ROWS * CH + NT - 1) / NT;  // chunks per thread per tile
  static constexpr int TILE = ROWS * kRowW;      // floats per tile
  static constexpr size_t bytes() { return (size_t)NB * TILE * sizeof(float); }
  static_assert(K <= 32, "chunk masks are 32-bit");
};

template <int R, int TY, int DX>
__global__ void __launch_bounds__(TY * 32, (TY == 8 ? 2 : 1))
step3d_velocity_queue_kernel(BatchArgs b) {
  using QT = QTile<R, TY, DX>;
  constexpr int Q = QT::Q;
  constexpr int D = QT::D;
  constexpr int NB = QT::NB;
  extern __shared__ __align__(16) float tiles[];
  const StepArgs& a = b.base;
  const Geom& g = a.g;
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  // launch order: z-block fastest, or plane-major (x strip, y tile, z-block)
  const unsigned bzb = a.cta_order ? blockIdx.z : blockIdx.x;
  const unsigned bxs = a.cta_order ? blockIdx.x : blockIdx.y;
  const unsigned byt = a.cta_order ? blockIdx.y : blockIdx.z;
  const int z0 = (int)((int64_t)bzb * a.zblock);
  const int z1 = (int)min((int64_t)z0 + a.zblock, g.nz);
  const int zs_end = z1 + R;                     // planes z0 .. zs_end-1 are staged
  const int64_t x0 = (int64_t)bxs * kStrip;
  const int64_t ty0 = (int64_t)byt * TY;
  const int64_t y = ty0 + warp;
  const int64_t xl = x0 + 4 * lane;
  const bool row_valid = y < g.ny;
  const bool xfix = (x0 == 0) || (x0 + kStrip + R > g.nx);
  const int row_off = (int)(y * g.px + xl);      // in-plane offset of the lane's cells
  const int own = (R + warp) * kRowW + 4 + 4 * lane;   // own cells in a tile
  const uint32_t smem0 = (uint32_t)__cvta_generic_to_shared(tiles);

  // staging descriptors: shared offset (floats), in-plane source offset,
  // bytes copied (16, or 0 to zero-fill); chunks copied by cp.async and
  // chunks copied negated by hand (rows behind a Dirichlet mirror)
  int s_dst[QT::K];
  int c_off[QT::K];
  uint32_t c_sz[QT::K];
  uint32_t cp_mask = 0, neg_mask = 0;
#pragma unroll
  for (int k = 0; k < QT::K; ++k) {
    const int c = tid + k * QT::NT;
    s_dst[k] = 0;
    c_off[k] = 0;
    c_sz[k] = 0;
    if (c < QT::ROWS * QT::CH) {
      const int rr = c / QT::CH, ch = c - rr * QT::CH;
      const int64_t yy = ty0 - R + rr;
      const int64_t xx = x0 - 4 + 4 * ch;
      s_dst[k] = rr * kRowW + 4 * ch;
      float ys = 0.f;
      if (yy >= -R && yy < g.ny + R && xx >= 0 && xx + 4 <= g.px) {
        const int64_t ysrc = mirror_index(yy, g.ny, g.bc, &ys);
        c_off[k] = (int)(ysrc * g.px + xx);
      }
      if (ys < 0.f) {
        neg_mask |= 1u << k;
      } else {
        cp_mask |= 1u << k;
        c_sz[k] = ys > 0.f ? 16u : 0u;
      }
    }
  }
  // x ghosts of the own row: position in the staged row, mirror source, sign
  int fx_pos = -1, fx_src = 0;
  float fx_sgn = 0.f;
  if (xfix) {
    int64_t gx = 0;
    if (lane < R && x0 == 0) {
      gx = -1 - lane;
      fx_pos = 3 - lane;
    } else if (lane >= 8 && lane < 8 + R) {
      gx = (g.nx < x0 + kStrip ? g.nx : x0 + kStrip) + (lane - 8);
      if (gx >= g.nx) fx_pos = (int)(gx - x0 + 4);
    }
    if (fx_pos >= 0) {
      const int64_t m = mirror_index(gx, g.nx, g.bc, &fx_sgn);
      fx_src = (int)(m - x0 + 4);
    }
  }
  const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);

  for (int shot = 0; shot < b.nshots; ++shot) {
    const float* __restrict__ uc = b.cur[shot];
    float* __restrict__ up = b.prev[shot];
    const bool acc_on = b.accf[shot] != 0;
    const float acc_sc = a.acc_scale * b.accf[shot];  // per-shot sign and on/off

    // Tile of plane p (z0 <= p < zs_end; above the domain: its mirror
    // source, positive) into buffer buf; always commits one group.
    auto stage = [&](int p, int buf) {
      if (p < zs_end) {
        float zsg = 1.f;
        const int64_t ps = p < g.nz ? p : mirror_index(p, g.nz, g.bc, &zsg);
        if (zsg != 0.f) {
          const float* src0 = uc + ps * g.plane;
          const uint32_t sb = smem0 + (uint32_t)(buf * QT::TILE) * 4u;
#pragma unroll
          for (int k = 0; k < QT::K; ++k)
            if (cp_mask & (1u << k)) cpa16z(sb + 4u * (uint32_t)s_dst[k], src0 + c_off[k], c_sz[k]);
          if (neg_mask) {
            float* tb = tiles + buf * QT::TILE;
#pragma unroll
            for (int k = 0; k < QT::K; ++k)
              if (neg_mask & (1u << k))
                *reinterpret_cast<float4*>(tb + s_dst[k]) =
                    f4_scale(__ldg(reinterpret_cast<const float4*>(src0 + c_off[k])), -1.f);
          }
        }
      }
      cpa_commit();
    };
    // sign with which plane p's staged own row enters the queue
    auto qsign = [&](int p) -> float {
      if (p < g.nz) return 1.f;
      float s;
      mirror_index(p, g.nz, g.bc, &s);
      return s;
    };
    auto qtile = [&](int p, int buf) -> float4 {   // plane p's own cells from its staged tile
      const float4 v = *reinterpret_cast<const float4*>(tiles + buf * QT::TILE + own);
      if (p < g.nz) return v;
      const float sg = qsign(p);
      return sg == 0.f ? zero4 : f4_scale(v, sg);   // a wall plane is never staged: do not read it
    };

    // prologue: tiles of planes z0 .. z0+D-1, queue of plane z0
#pragma unroll 1
    for (int i = 0; i < D; ++i) stage(z0 + i, i);
    float4 q[Q];
#pragma unroll
    for (int i = 0; i < R; ++i) {   // planes z0-r .. z0-1: below the block, from global memory
      const int p = z0 - R + i;
      float zsg;
      const int64_t ps = mirror_index(p, g.nz, g.bc, &zsg);
      q[i] = (row_valid && zsg != 0.f)
                 ? f4_scale(__ldg(reinterpret_cast<const float4*>(uc + ps * g.plane + row_off)), zsg)
                 : zero4;
    }
    int64_t off = (int64_t)z0 * g.plane + row_off;   // the lane's cells in plane z
    float4 u_old = zero4, cf = zero4, ac = zero4, cp = zero4;
    auto load = [&](int64_t o, float4& uo, float4& c, float4& acv, float4& cpv) {
      uo = *reinterpret_cast<const float4*>(up + o);
      c = __ldg(reinterpret_cast<const float4*>(a.coef + o));
      if (acc_on) {
        acv = *reinterpret_cast<const float4*>(a.acc + o);
        if (a.comp) cpv = *reinterpret_cast<const float4*>(a.comp + o);
      }
    };
    if (row_valid) load(off, u_old, cf, ac, cp);
    cpa_wait<QT::W>();   // tiles of planes z0 .. z0+r+1 have landed
    __syncthreads();
#pragma unroll
    for (int i = 0; i <= R; ++i) q[R + i] = row_valid ? qtile(z0 + i, i) : zero4;   // planes z0 .. z0+r
    int bz = 0;   // buffer of plane z

    for (int zb = z0; zb < z1; zb += Q) {
#pragma unroll
      for (int J = 0; J < Q; ++J) {
        const int z = zb + J;
        if (z < z1) {   // uniform over the CTA
          {
            int bn = bz + D;   // the buffer of plane z-1
            bn -= bn >= NB ? NB : 0;
            stage(z + D, bn);
          }
          float4 qn = zero4;   // plane z+r+1, staged at least one plane ago
          float4 n_old = u_old, n_cf = cf, n_ac = ac, n_cp = cp;
          if (row_valid && z + 1 < z1) {
            int bq = bz + R + 1;
            bq -= bq >= NB ? NB : 0;
            qn = qtile(z + R + 1, bq);
            load(off + g.plane, n_old, n_cf, n_ac, n_cp);
          }
          if (row_valid) {
            float* tile = tiles + bz * QT::TILE;
            float* srow = tile + (R + warp) * kRowW;
            if (xfix) {
              const float val = (fx_pos >= 0 && fx_sgn != 0.f) ? fx_sgn * srow[fx_src] : 0.f;
              __syncwarp();
              if (fx_pos >= 0) srow[fx_pos] = val;
              __syncwarp();
            }
            float lap[4];
            x_terms<R>(srow, lane, lap, 3.f * cw<R>(0));
            const float4 u = mask_row_padding(*reinterpret_cast<const float4*>(tile + own), xl, g.nx);
            // y terms from the tile, z terms from the queue, in pairs of cells
            // (paired FP32 ops; each element rounds as the scalar code would)
            float2 l01 = make_float2(lap[0], lap[1]), l23 = make_float2(lap[2], lap[3]);
#pragma unroll
            for (int j = 1; j <= R; ++j) {
              const float4 ym = *reinterpret_cast<const float4*>(tile + own - j * kRowW);
              const float4 yp = *reinterpret_cast<const float4*>(tile + own + j * kRowW);
              const float4 zm = q[(J + R - j) % Q];
              const float4 zp = q[(J + R + j) % Q];
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
            const float4 un = make_float4(n01.x, n01.y, n23.x, n23.y);
            *reinterpret_cast<float4*>(up + off) = un;
            if (a.mix_a) {   // exact modes (one shot): acc += acc_scale (u_cur - u_next)(mix_a - mix_b)
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
          }
          q[J] = qn;   // plane z+r+1 takes the slot of plane z-r
          u_old = n_old;
          cf = n_cf;
          ac = n_ac;
          cp = n_cp;
          off += g.plane;
          bz = bz + 1 == NB ? 0 : bz + 1;
          cpa_wait<QT::W>();   // tiles up to plane z+r+2 have landed
          __syncthreads();
        }
      }
    }
    cpa_wait<0>();
    __syncthreads();   // the buffers are refilled for the next shot
  }
}

template <int R, int TY, int DX>
cudaError_t launch_q(const BatchArgs& b, cudaStream_t s) {
  using QT = QTile<R, TY, DX>;
  cudaError_t e = set_smem_limit_once(reinterpret_cast<const void*>(step3d_velocity_queue_kernel<R, TY, DX>), (int)QT::bytes());
  if (e != cudaSuccess) return e;
  const Geom& g = b.base.g;
  const unsigned nzb = (unsigned)((g.nz + b.base.zblock - 1) / b.base.zblock);
  const unsigned nxs = (unsigned)((g.nx + kStrip - 1) / kStrip), nyt = (unsigned)((g.ny + TY - 1) / TY);
  const dim3 grid = b.base.cta_order ? dim3(nxs, nyt, nzb) : dim3(nzb, nxs, nyt);
  step3d_velocity_queue_kernel<R, TY, DX><<<grid, TY * 32, QT::bytes(), s>>>(b);
  count_launch();
  e = cudaGetLastError();
  if (e != cudaSuccess) note_error("step kernel launch", e);
  return e;
}

template <int R>
cudaError_t launch_q_r(const BatchArgs& b, cudaStream_t s) {
  if (b.base.tile_rows == 16)
    return b.base.ring_depth == 2 ? launch_q<R, 16, 1>(b, s) : launch_q<R, 16, 2>(b, s);
  return b.base.ring_depth == 2 ? launch_q<R, 8, 1>(b, s) : launch_q<R, 8, 2>(b, s);
}

}  // namespace

cudaError_t launch_step3d_queue(const BatchArgs& b, int order, cudaStream_t s) {
  switch (order) {
    case 2: return launch_q_r<1>(b, s);
    case 4: return launch_q_r<2>(b, s);
    case 6: return launch_q_r<3>(b, s);
    case 8: return launch_q_r<4>(b, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace wave
