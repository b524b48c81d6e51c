// 3D fused leapfrog step, FP32 storage, orders 2-8, batched mode: two shots
// advanced together in one pass of a CTA over its tile.
//
// Same arithmetic, element by element, as the other pipelines (Eq.
// FDstencil1 in squared-slowness form; sensitivity increment of Algorithm 1,
// shot A's increment added before shot B's), so results are bit-identical.
// The mapping:
//
// * a CTA of 16 warps owns 16 rows x 128 cells and marches up z over a block
//   of planes, advancing the shots of the launch two at a time; the two
//   fields share the march: one barrier and one set of index and loop
//   bookkeeping per plane, one load of coef and one update of the
//   accumulator (both increments) per cell and plane;
// * with more than two shots and a z-block of at most 32 planes (16 with
//   Kahan compensation) the accumulator tile stays in tensor memory between
//   the pairs: read from HBM by the first pair, written back by the last, so
//   it crosses HBM once per launch instead of once per pair;
// * per shot, the tile of each plane (own rows + r halo rows, 4 halo cells
//   per side) is staged by cp.async r+1+depth planes ahead (ring depth 2 or
//   3 of the tiling) into r+2+depth buffers: the
//   tile of plane z gives the x and y neighbours and the own rows of planes
//   z+1 .. z+r give the upper z neighbours; the lower ones (planes z-r ..
//   z-1) stay in a register queue of r float4 per shot, rotated statically;
// * staging is branch-free (precomputed chunk list, chunks outside the grid
//   zero-filled by the copy); rows behind a Dirichlet mirror are copied
//   negated by hand; planes above the domain are staged from their mirror
//   images (the wall plane as zeros) and read with the mirror sign;
// * the streaming operands of plane z+1 are loaded into registers while
//   plane z is computed;
// * the exact reverse-time mode runs u (field A) and lambda (field B) here
//   and accumulates their mixed term from registers (no re-read of u).
// In-plane offsets are 32-bit: the launcher requires px * ny < 2^31.
#include "stencil_common.cuh"

namespace wave {
namespace {

__device__ __forceinline__ void pcp16(uint32_t sdst, const float* gsrc, uint32_t nbytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sdst), "l"(gsrc), "r"(nbytes) : "memory");
}
__device__ __forceinline__ void pcp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void pcp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

enum { kPairNone = 0, kPairSq = 1, kPairKahan = 2, kPairMix = 3 };

// x part of the stencil for the lane's 4 cells from A (cells x-4..x-1), B
// (x..x+3) and C (x+4..x+7), as two cell pairs (0,1) and (2,3).  Per cell the
// operations and their order are those of x_terms_abc (c0' u, then
// fma(c_j, u[+j] + u[-j], s) for j = 1..r); the offsets j that keep both
// operands of a pair in one aligned register pair (even j) run as packed
// FP32x2 instructions, the odd ones per cell.
// Order 2 keeps the scalar helper: its one weight c_1 = 1 turns
// fma(c_1, s, .) into an add that the compiler may fuse with the product
// c0' u, and every kernel must round that the same way.
template <int R>
__device__ __forceinline__ void x_terms_pair(const float4& A, const float4& B, const float4& C, float ndim_c0,
                                             float2& l01, float2& l23) {
  if constexpr (R == 1) {
    float lap[4];
    x_terms_abc<R>(A, B, C, lap, ndim_c0);
    l01 = make_float2(lap[0], lap[1]);
    l23 = make_float2(lap[2], lap[3]);
    return;
  }
  const float e[12] = {A.x, A.y, A.z, A.w, B.x, B.y, B.z, B.w, C.x, C.y, C.z, C.w};
  const float2 c0 = make_float2(ndim_c0, ndim_c0);
  l01 = __fmul2_rn(c0, make_float2(B.x, B.y));
  l23 = __fmul2_rn(c0, make_float2(B.z, B.w));
#pragma unroll
  for (int j = 1; j <= R; ++j) {
    if (j % 2 == 0) {
      const float2 cj = make_float2(cw<R>(j), cw<R>(j));
      l01 = __ffma2_rn(cj, __fadd2_rn(make_float2(e[4 + j], e[5 + j]), make_float2(e[4 - j], e[5 - j])), l01);
      l23 = __ffma2_rn(cj, __fadd2_rn(make_float2(e[6 + j], e[7 + j]), make_float2(e[6 - j], e[7 - j])), l23);
    } else {
      l01.x = fmaf(cw<R>(j), e[4 + j] + e[4 - j], l01.x);
      l01.y = fmaf(cw<R>(j), e[5 + j] + e[5 - j], l01.y);
      l23.x = fmaf(cw<R>(j), e[6 + j] + e[6 - j], l23.x);
      l23.y = fmaf(cw<R>(j), e[7 + j] + e[7 - j], l23.y);
    }
  }
}

// Tensor memory (TMEM, 128 lanes x 512 columns of 32 bits per SM) holds the
// accumulator (and Kahan compensation) tile of the CTA's z-block between the
// shot pairs of a launch.  Warp w reaches lanes 32 (w mod 4) .. +31, one per
// thread; a thread's 4 cells of plane z - z0 take 4 columns, so the four warps
// sharing a lane quarter and a z-block of P planes fill 16 P columns:
// P <= 32 for the accumulator alone, P <= 16 with the compensation beside it
// (columns 256..511).
constexpr int kTmemPlanes = 32;
constexpr int kTmemPlanesKahan = 16;
__device__ __forceinline__ void tm_ld4(uint32_t ta, float4& v) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(ta) : "memory");
}
// wait for the loads; the registers pass through so that no use moves above it
__device__ __forceinline__ void tm_wait_ld(float4& v, float4& w) {
  asm volatile("tcgen05.wait::ld.sync.aligned;" : "+f"(v.x), "+f"(v.y), "+f"(v.z), "+f"(v.w),
               "+f"(w.x), "+f"(w.y), "+f"(w.z), "+f"(w.w) :: "memory");
}
__device__ __forceinline__ void tm_st4(uint32_t ta, const float4& v) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};"
               :: "r"(ta), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w) : "memory");
}
__device__ __forceinline__ void tm_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

template <int R, int TY, int DX>
struct PTile {
  static constexpr int D = R + 1 + DX;           // planes staged ahead of the centre plane
  static constexpr int W = D - R - 1;            // copy groups left in flight at each wait
  static constexpr int NB = D + 1;               // tile buffers per shot
  static constexpr int ROWS = TY + 2 * R;        // staged rows per tile
  static constexpr int CH = kRowW / 4;           // 16-byte chunks per staged row
  static constexpr int NT = TY * 32;             // threads
  static constexpr int K = (ROWS * CH + NT - 1) / NT;  // chunks per thread per tile
  static constexpr int TILE = ROWS * kRowW;      // floats per tile
  static constexpr size_t bytes() { return (size_t)2 * NB * TILE * sizeof(float); }
  static_assert(K <= 32, "chunk masks are 32-bit");
};

template <int R, int TY, int DX, int ACC, bool TM>
__global__ void __launch_bounds__(TY * 32, 1)
step3d_velocity_pair_kernel(BatchArgs b) {
  using PT = PTile<R, TY, DX>;
  constexpr int D = PT::D;
  constexpr int NB = PT::NB;
  extern __shared__ __align__(16) float tiles[];   // [2][NB][TILE]
  const StepArgs& a = b.base;
  const Geom& g = a.g;
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  // Launch order (grid built by the launcher to match): plane-major puts the
  // x strips and then the y tiles of one z-block next to each other, so the
  // CTAs whose halo rows overlap run at the same time and share them in L2.
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
  const bool xfast = (g.nx % kStrip) == 0;   // row ends on strip boundaries: x ghosts in registers
  const int row_off = (int)(y * g.px + xl);
  const int own = (R + warp) * kRowW + 4 + 4 * lane;   // own cells in a tile
  const uint32_t smem0 = (uint32_t)__cvta_generic_to_shared(tiles);

  // staging descriptors (as in the register-queue kernel)
  int s_dst[PT::K];
  int c_off[PT::K];
  uint32_t c_sz[PT::K];
  uint32_t cp_mask = 0, neg_mask = 0;
#pragma unroll
  for (int k = 0; k < PT::K; ++k) {
    const int c = tid + k * PT::NT;
    s_dst[k] = 0;
    c_off[k] = 0;
    c_sz[k] = 0;
    if (c < PT::ROWS * PT::CH) {
      const int rr = c / PT::CH, ch = c - rr * PT::CH;
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
  // x ghosts of a ragged own row (nx not a multiple of the strip): lanes
  // 0..r-1 (left end) and 8..8+r-1 (right end) write the mirror values into
  // the staged row; computed where used, so that grids whose rows end on strip
  // boundaries keep no registers for it
  auto ragged_x_ghosts = [&](float* srow) {
    int fx_pos = -1, fx_src = 0;
    float fx_sgn = 0.f;
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
    const float val = (fx_pos >= 0 && fx_sgn != 0.f) ? fx_sgn * srow[fx_src] : 0.f;
    __syncwarp();
    if (fx_pos >= 0) srow[fx_pos] = val;
    __syncwarp();
  };
  const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);

  __shared__ uint32_t tm_slot;
  uint32_t tm_base = 0;
  const uint32_t tm_ncols = ACC == kPairKahan ? 512u : (a.zblock * 16 <= 256 ? 256u : 512u);
  if constexpr (TM) {
    if (warp == 0) {
      const uint32_t sa = (uint32_t)__cvta_generic_to_shared(&tm_slot);
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sa), "r"(tm_ncols)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    tm_base = tm_slot;
  }
  // this warp's TMEM lanes (32 per warp of a group of four) and first column
  const uint32_t tm_row = tm_base + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)((warp >> 2) * a.zblock * 4);

  for (int s0 = 0; s0 < b.nshots; s0 += 2) {
    const bool first = s0 == 0, last = s0 + 2 >= b.nshots;
    const bool two = s0 + 1 < b.nshots;   // uniform: a second field in this pass
    const float* __restrict__ ucA = b.cur[s0];
    const float* __restrict__ ucB = two ? b.cur[s0 + 1] : b.cur[s0];
    float* __restrict__ upA = b.prev[s0];
    float* __restrict__ upB = two ? b.prev[s0 + 1] : b.prev[s0];
    const float fA = b.accf[s0], fB = two ? b.accf[s0 + 1] : 0.f;
    const bool onA = ACC != kPairNone && ACC != kPairMix && fA != 0.f;
    const bool onB = ACC != kPairNone && (ACC == kPairMix ? two : fB != 0.f);
    const bool acc_on = onA || onB;
    const float scA = a.acc_scale * fA, scB = a.acc_scale * fB;

    // Tiles of plane p for both fields into buffer buf; one commit group.
    // Above the domain: the mirror source plane with the mirror sign applied
    // (the wall plane of a Dirichlet box as zeros; the planes behind it
    // negated, copied by hand: the top r planes of the grid only), so the
    // stencil reads every staged plane as it is.
    auto stage = [&](int p, int buf) {
      if (p < zs_end) {
        float zsg = 1.f;
        const int64_t ps = p < g.nz ? p : mirror_index(p, g.nz, g.bc, &zsg);
        const uint32_t zmask = zsg != 0.f ? 0xffffffffu : 0u;   // 0: zero-fill every chunk
        const int64_t pofs = ps * g.plane;
#pragma unroll
        for (int f = 0; f < 2; ++f) {
          if (f == 1 && !two) break;
          const float* src0 = (f == 0 ? ucA : ucB) + pofs;
          float* tb = tiles + (f * NB + buf) * PT::TILE;
          if (zsg < 0.f) {
#pragma unroll
            for (int k = 0; k < PT::K; ++k) {
              const float4 v = __ldg(reinterpret_cast<const float4*>(src0 + c_off[k]));
              if (cp_mask & (1u << k))
                *reinterpret_cast<float4*>(tb + s_dst[k]) = c_sz[k] ? f4_scale(v, -1.f) : zero4;
              else if (neg_mask & (1u << k))
                *reinterpret_cast<float4*>(tb + s_dst[k]) = v;
            }
            continue;
          }
          const uint32_t sb = smem0 + (uint32_t)(((f * NB) + buf) * PT::TILE) * 4u;
#pragma unroll
          for (int k = 0; k < PT::K; ++k)
            if (cp_mask & (1u << k)) pcp16(sb + 4u * (uint32_t)s_dst[k], src0 + c_off[k], c_sz[k] & zmask);
          if (neg_mask) {
#pragma unroll
            for (int k = 0; k < PT::K; ++k)
              if (neg_mask & (1u << k))
                *reinterpret_cast<float4*>(tb + s_dst[k]) =
                    zsg != 0.f ? f4_scale(__ldg(reinterpret_cast<const float4*>(src0 + c_off[k])), -1.f) : zero4;
          }
        }
      }
      pcp_commit();
    };

    // prologue: tiles of planes z0 .. z0+D-1, lower queues of plane z0
#pragma unroll 1
    for (int i = 0; i < D; ++i) stage(z0 + i, i);
    float4 qa[R], qb[R];   // planes z-r .. z-1 of each field
#pragma unroll
    for (int i = 0; i < R; ++i) {
      const int p = z0 - R + i;
      float zsg;
      const int64_t ps = mirror_index(p, g.nz, g.bc, &zsg);
      const bool ld = row_valid && zsg != 0.f;
      qa[i] = ld ? f4_scale(__ldg(reinterpret_cast<const float4*>(ucA + ps * g.plane + row_off)), zsg) : zero4;
      qb[i] = (ld && two) ? f4_scale(__ldg(reinterpret_cast<const float4*>(ucB + ps * g.plane + row_off)), zsg)
                          : zero4;
    }
    int64_t off = (int64_t)z0 * g.plane + row_off;
    float4 oa = zero4, ob = zero4, cf = zero4, ac = zero4, cp = zero4;   // streams of plane z
    auto load = [&](int64_t o, float4& uoa, float4& uob, float4& c, float4& acv, float4& cpv) {
      uoa = *reinterpret_cast<const float4*>(upA + o);
      if (two) uob = *reinterpret_cast<const float4*>(upB + o);
      c = __ldg(reinterpret_cast<const float4*>(a.coef + o));
      if (TM ? first : acc_on) {
        acv = *reinterpret_cast<const float4*>(a.acc + o);
        if (ACC == kPairKahan) cpv = *reinterpret_cast<const float4*>(a.comp + o);
      }
    };
    if (row_valid) load(off, oa, ob, cf, ac, cp);
    int bz = 0;   // buffer of plane z
    pcp_wait<PT::W>();   // tiles of planes z0 .. z0+r have landed
    __syncthreads();

    // One field f at plane z (buffer bz; lower queue ql): new level un and
    // the centre value u the increment is taken against.
    auto field = [&](int f, int J, int bz_, const float4 (&ql)[R], const float4& u_old,
                     const int (&zoff)[R], float4& u, float4& un) {
      float* tile = tiles + (f * NB + bz_) * PT::TILE;
      float* srow = tile + (R + warp) * kRowW;
      u = *reinterpret_cast<const float4*>(tile + own);
      float2 l01, l23;
      if (xfix && !xfast) {   // ragged row end: ghosts written into the staged row
        ragged_x_ghosts(srow);
        u = mask_row_padding(u, xl, g.nx);
        float lap[4];
        x_terms<R>(srow, lane, lap, 3.f * cw<R>(0));
        l01 = make_float2(lap[0], lap[1]);
        l23 = make_float2(lap[2], lap[3]);
      } else {
        float4 xa = *reinterpret_cast<const float4*>(srow + 4 * lane);
        float4 xc = *reinterpret_cast<const float4*>(srow + 8 + 4 * lane);
        if (xfix) {   // row ends on a strip boundary: ghosts from the lane's own cells
          if (lane == 0 && x0 == 0) xa = left_ghosts(u, g.bc);
          if (lane == 31 && x0 + kStrip == g.nx) xc = right_ghosts(u, g.bc);
        }
        x_terms_pair<R>(xa, u, xc, 3.f * cw<R>(0), l01, l23);
      }
#pragma unroll
      for (int j = 1; j <= R; ++j) {
        const float4 ym = *reinterpret_cast<const float4*>(tile + own - j * kRowW);
        const float4 yp = *reinterpret_cast<const float4*>(tile + own + j * kRowW);
        const float4 zm = ql[(J - j + R) % R];
        const float4 zp = *reinterpret_cast<const float4*>(tiles + f * NB * PT::TILE + zoff[j - 1]);
        const float2 c2 = make_float2(cw<R>(j), cw<R>(j));
        l01 = __ffma2_rn(c2, __fadd2_rn(__fadd2_rn(make_float2(ym.x, ym.y), make_float2(yp.x, yp.y)),
                                        __fadd2_rn(make_float2(zm.x, zm.y), make_float2(zp.x, zp.y))), l01);
        l23 = __ffma2_rn(c2, __fadd2_rn(__fadd2_rn(make_float2(ym.z, ym.w), make_float2(yp.z, yp.w)),
                                        __fadd2_rn(make_float2(zm.z, zm.w), make_float2(zp.z, zp.w))), l23);
      }
      const float2 tw = make_float2(2.f, 2.f);
      const float2 n01 = __ffma2_rn(make_float2(cf.x, cf.y), l01,
                                    __ffma2_rn(tw, make_float2(u.x, u.y), make_float2(-u_old.x, -u_old.y)));
      const float2 n23 = __ffma2_rn(make_float2(cf.z, cf.w), l23,
                                    __ffma2_rn(tw, make_float2(u.z, u.w), make_float2(-u_old.z, -u_old.w)));
      un = make_float4(n01.x, n01.y, n23.x, n23.y);
    };
    // acc (+ comp) += sc (un - u)^2, element order as the single-field kernels
    auto accumulate = [&](float sc, const float4& u, const float4& un) {
      const float d0 = un.x - u.x, d1 = un.y - u.y, d2 = un.z - u.z, d3 = un.w - u.w;
      if (ACC == kPairKahan) {
        kahan_add(ac.x, cp.x, sc * d0 * d0);
        kahan_add(ac.y, cp.y, sc * d1 * d1);
        kahan_add(ac.z, cp.z, sc * d2 * d2);
        kahan_add(ac.w, cp.w, sc * d3 * d3);
      } else {
        const float2 s2 = make_float2(sc, sc);
        const float2 e01 = make_float2(d0, d1), e23 = make_float2(d2, d3);
        const float2 r01 = __ffma2_rn(__fmul2_rn(s2, e01), e01, make_float2(ac.x, ac.y));
        const float2 r23 = __ffma2_rn(__fmul2_rn(s2, e23), e23, make_float2(ac.z, ac.w));
        ac = make_float4(r01.x, r01.y, r23.x, r23.y);
      }
    };

    for (int zb = z0; zb < z1; zb += R) {
#pragma unroll
      for (int J = 0; J < R; ++J) {   // lower-queue slot of plane z-j is (J-j) mod r
        const int z = zb + J;
        if (z < z1) {   // uniform over the CTA
          {
            int bn = bz + D;   // the buffer of plane z-1
            bn -= bn >= NB ? NB : 0;
            stage(z + D, bn);
          }
          float4 n_oa = oa, n_ob = ob, n_cf = cf, n_ac = ac, n_cp = cp;
          if (row_valid && z + 1 < z1) load(off + g.plane, n_oa, n_ob, n_cf, n_ac, n_cp);
          if (row_valid) {
            const bool tm_in = TM && !first && (acc_on || last);
            const uint32_t tm_a = tm_row + (uint32_t)(4 * (z - z0));
            if (tm_in) {
              tm_ld4(tm_a, ac);
              if (ACC == kPairKahan) tm_ld4(tm_a + 256u, cp);
            }
            int zoff[R];   // own cells of planes z+1 .. z+r in the tile ring (both fields)
#pragma unroll
            for (int j = 1; j <= R; ++j) {
              int bj = bz + j;
              bj -= bj >= NB ? NB : 0;
              zoff[j - 1] = bj * PT::TILE + own;
            }
            float4 ua, una;
            field(0, J, bz, qa, oa, zoff, ua, una);
            *reinterpret_cast<float4*>(upA + off) = una;
            float4 ubv = zero4, unb = zero4;
            if (two) {
              field(1, J, bz, qb, ob, zoff, ubv, unb);
              *reinterpret_cast<float4*>(upB + off) = unb;
            }
            if (ACC == kPairMix && acc_on) {
              // exact reverse-time mode: field A is u, field B is lambda (Eq.
              // kernel1 mixed term, same operand order as the one-field kernels)
              ac.x = fmaf(scB * (ubv.x - unb.x), ua.x - una.x, ac.x);
              ac.y = fmaf(scB * (ubv.y - unb.y), ua.y - una.y, ac.y);
              ac.z = fmaf(scB * (ubv.z - unb.z), ua.z - una.z, ac.z);
              ac.w = fmaf(scB * (ubv.w - unb.w), ua.w - una.w, ac.w);
              *reinterpret_cast<float4*>(a.acc + off) = ac;
            } else if (TM) {
              if (tm_in) tm_wait_ld(ac, cp);
              if (onA) accumulate(scA, ua, una);
              if (onB) accumulate(scB, ubv, unb);
              if (last) {
                *reinterpret_cast<float4*>(a.acc + off) = ac;
                if (ACC == kPairKahan) *reinterpret_cast<float4*>(a.comp + off) = cp;
              } else if (acc_on || first) {
                tm_st4(tm_a, ac);
                if (ACC == kPairKahan) tm_st4(tm_a + 256u, cp);
                tm_wait_st();
              }
            } else if (acc_on) {
              if (onA) accumulate(scA, ua, una);
              if (onB) accumulate(scB, ubv, unb);
              *reinterpret_cast<float4*>(a.acc + off) = ac;
              if (ACC == kPairKahan) *reinterpret_cast<float4*>(a.comp + off) = cp;
            }
            qa[J] = ua;   // plane z enters the lower queues in place of plane z-r
            qb[J] = ubv;
          }
          oa = n_oa;
          ob = n_ob;
          cf = n_cf;
          ac = n_ac;
          cp = n_cp;
          off += g.plane;
          bz = bz + 1 == NB ? 0 : bz + 1;
          pcp_wait<PT::W>();   // tiles up to plane z+1+r have landed
          __syncthreads();
        }
      }
    }
    pcp_wait<0>();
    __syncthreads();   // the buffers are refilled for the next pair
  }
  if constexpr (TM) {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tm_base), "r"(tm_ncols) : "memory");
    }
  }
}

template <int R, int TY, int DX, int ACC, bool TM = false>
cudaError_t launch_p(const BatchArgs& b, cudaStream_t s) {
  using PT = PTile<R, TY, DX>;
  cudaError_t e = set_smem_limit_once(reinterpret_cast<const void*>(step3d_velocity_pair_kernel<R, TY, DX, ACC, TM>), (int)PT::bytes());
  if (e != cudaSuccess) return e;
  const Geom& g = b.base.g;
  const unsigned nzb = (unsigned)((g.nz + b.base.zblock - 1) / b.base.zblock);
  const unsigned nxs = (unsigned)((g.nx + kStrip - 1) / kStrip), nyt = (unsigned)((g.ny + TY - 1) / TY);
  const dim3 grid = b.base.cta_order ? dim3(nxs, nyt, nzb) : dim3(nzb, nxs, nyt);
  step3d_velocity_pair_kernel<R, TY, DX, ACC, TM><<<grid, TY * 32, PT::bytes(), s>>>(b);
  count_launch();
  e = cudaGetLastError();
  if (e != cudaSuccess) note_error("step kernel launch", e);
  return e;
}

template <int R, int DX>
cudaError_t launch_p_d(const BatchArgs& b, cudaStream_t s) {
  if (b.pair_mix) return launch_p<R, 16, DX, kPairMix>(b, s);
  bool any = false;
  for (int i = 0; i < b.nshots; ++i) any |= b.accf[i] != 0.f;
  if (!any) return launch_p<R, 16, DX, kPairNone>(b, s);
  if (b.nshots > 2 && b.base.zblock <= (b.base.comp ? kTmemPlanesKahan : kTmemPlanes)) {
    if (b.base.comp) return launch_p<R, 16, DX, kPairKahan, true>(b, s);
    return launch_p<R, 16, DX, kPairSq, true>(b, s);
  }
  if (b.base.comp) return launch_p<R, 16, DX, kPairKahan>(b, s);
  return launch_p<R, 16, DX, kPairSq>(b, s);
}

template <int R>
cudaError_t launch_p_r(const BatchArgs& b, cudaStream_t s) {
  return b.base.ring_depth == 2 ? launch_p_d<R, 1>(b, s) : launch_p_d<R, 2>(b, s);
}

}  // namespace

cudaError_t launch_step3d_pair(const BatchArgs& b, int order, cudaStream_t s) {
  switch (order) {
    case 2: return launch_p_r<1>(b, s);
    case 4: return launch_p_r<2>(b, s);
    case 6: return launch_p_r<3>(b, s);
    case 8: return launch_p_r<4>(b, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace wave
