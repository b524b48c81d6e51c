// 3D fused leapfrog step, FP32 storage, orders 2-8, batched launches: the
// shots of a launch advance two per pass of a CTA over its tile, the u^n
// tiles arriving by TMA tensor copies from a producer warp.
//
// Arithmetic, element by element, is that of the other velocity pipelines
// (Eq. FDstencil1 in squared-slowness form; Algorithm 1's sensitivity
// increment of Eq. kernel1, shot A's increment added before shot B's), so
// the results are bit-identical to theirs.  The mapping:
//
// * a CTA owns 16 rows x 128 cells (one consumer warp per row, four cells
//   per lane) and a z-block of 8 planes; grid x runs over z-blocks fastest,
//   so the CTAs of neighbouring z-blocks run side by side and the planes one
//   of them stages as halo the other reads as its own shortly before or after
//   (an L2 hit);
// * for each pass (fields A and B = the next two shots of the launch) the
//   CTA needs the tiles of planes z0-r .. z0+8+r-1 of both fields: 8 + 2r
//   tiles per field, each 16 + 2r rows x 136 cells (4 halo cells per side).
//   A 17th warp copies them with cp.async.bulk.tensor.3d into a ring of
//   (8 + 2r) / 2 slots, so every slot is used exactly twice per pass and the
//   slot and mbarrier parity of every tile are compile-time constants of the
//   unrolled pass.  The copies run on across passes: the next pass's first
//   tiles arrive while the current pass finishes;
// * a consumer warp keeps planes z-r .. z-1 of its row in a register queue
//   per field and reads the x and y neighbours from the tile of plane z and
//   the upper z neighbours from the tiles of planes z+1 .. z+r; it releases
//   a tile on its slot's "empty" mbarrier after its last use;
// * the streaming operands (u^{n-1} of both fields, coef, the accumulator
//   and its compensation) of the next plane -- across the pass boundary, of
//   the next pass's first plane -- are loaded into registers while the
//   current plane is computed; the accumulator of a cell is read and written
//   once per pass (both increments);
// * ghost values: out-of-range tile rows and planes arrive as zeros (the
//   copy's out-of-bounds fill).  Rows behind a y boundary are then filled from
//   their mirror rows by the producer warp before the consumers may read the
//   tile (a second "ready" mbarrier, only in CTAs at a y boundary); planes
//   behind a z boundary are copied from their mirror planes and read with the
//   mirror sign; the x ghosts of a warp's own row are written by that warp;
// * every wait is bounded (wait_limit_cycles): on time-out the kernel sets
//   the device error word, every warp leaves, and the producer waits
//   (bounded) for the copies it has in flight before the CTA exits.
#include <cuda.h>   // CUtensorMap and its encoder's types (the encoder is looked up at run time)

#include <mutex>
#include <unordered_map>

#include "stencil_common.cuh"

namespace wave {
namespace {

constexpr int kZB = 8;                    // planes per z-block (compile-time: the pass is unrolled)
constexpr int kTY = 16;                   // rows per CTA = consumer warps
constexpr int kThreads = kTY * 32;

template <int R>
struct SCfg {
  static constexpr int ROWS = kTY + 2 * R;       // staged rows per tile
  static constexpr int TILE = ROWS * kRowW;      // floats per tile
  static constexpr int TILE_BYTES = TILE * 4;
  static constexpr int STRIDE = (TILE + 31) / 32 * 32;   // floats between tiles: 128-byte aligned copies
  static constexpr int PER_PASS = kZB + 2 * R;   // tiles per field and pass
  static constexpr int NB = PER_PASS / 2;        // ring slots (two fields each)
  static constexpr size_t BAR_OFF = (size_t)2 * NB * STRIDE * 4;
  static constexpr size_t bytes() { return BAR_OFF + NB * sizeof(uint64_t) + 2 * NB * sizeof(int) + 16; }
  static_assert(PER_PASS % 2 == 0, "each slot is used twice per pass");
};

struct StreamArgs {
  BatchArgs b;
  CUtensorMap map[kMaxBatch];   // u^n of each listed field: (px, ny, nz) FP32, box (136, 16 + 2r, 1)
};

__device__ __forceinline__ uint32_t sa(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(sa(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void bar_expect(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(sa(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool bar_test(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(sa(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase of the given parity; false on time-out or when
// another warp has already given up.
__device__ __forceinline__ bool bar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                         long long limit) {
  if (bar_test(bar, parity)) return true;
  const long long t0 = clock64();
  for (uint32_t it = 0;; ++it) {
    if (bar_test(bar, parity)) return true;
    if ((it & 31) == 31) {
      if (*abort_flag) return false;
      if (clock64() - t0 > limit) {
        *abort_flag = 1;
        return false;
      }
    }
  }
}
__device__ __forceinline__ void tma_load_3d(float* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];\n" ::"r"(sa(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(sa(bar))
      : "memory");
}
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

enum { kAccNone = 0, kAccSq = 1, kAccKahan = 2, kAccMix = 3 };

// Plane that tile q of a pass holds (z0 - r + q), where its data come from,
// and the sign it is read with.  Outside [-r, nz + r) (tiles of a partial
// z-block nobody reads) and on a Dirichlet wall plane the source coordinate
// is out of range, so the copy fills zeros.
__device__ __forceinline__ int tile_source(int p, const Geom& g, int R, float* sign) {
  if (p < -R || p >= g.nz + R) {
    *sign = 0.f;
    return p < 0 ? -1 : (int)g.nz;
  }
  float s;
  const int64_t m = mirror_index(p, g.nz, g.bc, &s);
  *sign = s;
  if (s == 0.f) return p;   // Dirichlet wall: -1 or nz, out of range
  return (int)m;
}

template <int R, int ACC>
__global__ void __launch_bounds__(kThreads, 1) step3d_velocity_stream_kernel(const __grid_constant__ StreamArgs P) {
  using C = SCfg<R>;
  constexpr int NB = C::NB;
  constexpr int PP = C::PER_PASS;
  extern __shared__ __align__(128) float tiles[];   // [NB][2][STRIDE]
  uint64_t* full = reinterpret_cast<uint64_t*>(reinterpret_cast<char*>(tiles) + C::BAR_OFF);
  int* released = reinterpret_cast<int*>(full + NB);   // warps done with the slot's tile
  int* nissued = released + NB;                        // copies issued into the slot
  volatile int* abort_flag = nissued + NB;

  const BatchArgs& b = P.b;
  const StepArgs& a = b.base;
  const Geom& g = a.g;
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const int z0 = blockIdx.x * kZB;
  const int nzb = (int)min((int64_t)kZB, g.nz - z0);
  const int x0 = blockIdx.y * kStrip;
  const int ty0 = blockIdx.z * kTY;
  const long long limit = b.wait_limit_cycles;
  const int npass = (b.nshots + 1) / 2;

  // Copy tile q of pass p (both fields of the pass) into slot q mod NB.
  auto issue = [&](int p, int q) {
    const int s = q % NB;
    const bool two = 2 * p + 1 < b.nshots;
    float sg;
    const int zsrc = tile_source(z0 - R + q, g, R, &sg);
    bar_expect(&full[s], (uint32_t)C::TILE_BYTES * (two ? 2u : 1u));
    tma_load_3d(tiles + (2 * s) * C::STRIDE, &P.map[2 * p], x0 - 4, ty0 - R, zsrc, &full[s]);
    if (two) tma_load_3d(tiles + (2 * s + 1) * C::STRIDE, &P.map[2 * p + 1], x0 - 4, ty0 - R, zsrc, &full[s]);
    nissued[s] += 1;
  };

  if (tid == 0) {
    for (int s = 0; s < NB; ++s) {
      bar_init(&full[s], 1);
      released[s] = 0;
      nissued[s] = 0;
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  if (tid == 0 && !b.debug_stall)
    for (int q = 0; q < NB; ++q) issue(0, q);

  // A warp is done with tile q of pass p: the last of the 16 warps to say so
  // refills the slot with the tile that uses it next (q + NB of this pass, or
  // of the next pass).  The fence orders the warps' reads (and ghost writes)
  // of the slot before the copy that overwrites it.
  auto release = [&](int p, int q) {
    __syncwarp();
    if (lane == 0) {
      const int s = q % NB;
      __threadfence_block();
      if (atomicAdd(&released[s], 1) == kTY - 1) {
        released[s] = 0;
        __threadfence_block();
        fence_async_smem();
        int np = p, nq = q + NB;
        if (nq >= PP) {
          nq -= PP;
          ++np;
        }
        if (np < npass && !b.debug_stall && !*abort_flag) issue(np, nq);
      }
    }
  };

  const int y = ty0 + warp;
  const bool row_valid = y < g.ny;
  const int xl = x0 + 4 * lane;
  const bool xfix = (x0 == 0) || (x0 + kStrip + R > g.nx);
  // rows behind a y boundary are filled from their mirror rows by the warps
  // once a centre tile has landed (then a CTA barrier; uniform per CTA)
  const bool yfix = ty0 == 0 || ty0 + kTY + R > g.ny;
  const int64_t row_off = (int64_t)y * g.px + xl;
  constexpr int own = R * kRowW + 4;              // own cells of warp 0, lane 0 in a tile
  const int lo = warp * kRowW + 4 * lane;

  // ghost row this warp fills in y-boundary CTAs: tile row gt from row gs, sign gsg
  int gt = -1, gsrc = 0;
  float gsg = 0.f;
  if (yfix) {
    int k = 0;
    for (int tr = 0; tr < C::ROWS; ++tr) {
      const int yy = ty0 - R + tr;
      if ((yy >= 0 && yy < g.ny) || yy < -R || yy >= g.ny + R) continue;
      if (k++ == warp) {
        float sg;
        const int64_t ys = mirror_index(yy, g.ny, g.bc, &sg);
        gt = tr;
        gsrc = (int)ys - (ty0 - R);
        gsg = sg;
      }
    }
  }
  auto fill_ghost_rows = [&](int q, bool two) {
    if (gt >= 0) {
      for (int f = 0; f < (two ? 2 : 1); ++f) {
        float* t = tiles + (2 * (q % NB) + f) * C::STRIDE;
        for (int c = lane; c < kRowW / 4; c += 32) {
          float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
          if (gsg != 0.f) v = f4_scale(*reinterpret_cast<const float4*>(t + gsrc * kRowW + 4 * c), gsg);
          *reinterpret_cast<float4*>(t + gt * kRowW + 4 * c) = v;
        }
      }
      fence_async_smem();   // these writes before any later copy into the slot
    }
    __syncthreads();
  };

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
  // signs of the pass's tiles (planes z0 - r + q): bit q set = read negated
  uint32_t neg = 0;
  for (int q = 0; q < PP; ++q) {
    float sg;
    tile_source(z0 - R + q, g, R, &sg);
    if (sg < 0.f) neg |= 1u << q;
  }
  const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);

  // streaming operands of a plane: offset o (cells) of the row strip
  auto load_streams = [&](int p, int64_t o, float4& oa, float4& ob, float4& cf, float4& ac, float4& cp) {
    const bool two = 2 * p + 1 < b.nshots;
    oa = *reinterpret_cast<const float4*>(b.prev[2 * p] + o);
    if (two) ob = *reinterpret_cast<const float4*>(b.prev[2 * p + 1] + o);
    cf = __ldg(reinterpret_cast<const float4*>(a.coef + o));
    if (ACC != kAccNone) {
      ac = *reinterpret_cast<const float4*>(a.acc + o);
      if (ACC == kAccKahan) cp = *reinterpret_cast<const float4*>(a.comp + o);
    }
  };

  float4 oa = zero4, ob = zero4, cf = zero4, ac = zero4, cp = zero4;
  if (row_valid) load_streams(0, (int64_t)z0 * g.plane + row_off, oa, ob, cf, ac, cp);
  bool ok = true;

  // After a time-out (ok false) the loops run on without work, so every warp
  // passes the same CTA barriers and reaches the end.
  for (int p = 0; p < npass; ++p) {
    const bool two = 2 * p + 1 < b.nshots;
    float* const upA = b.prev[2 * p];
    float* const upB = b.prev[2 * p + (two ? 1 : 0)];
    const float fA = b.accf[2 * p], fB = two ? b.accf[2 * p + 1] : 0.f;
    const bool onA = ACC != kAccNone && ACC != kAccMix && fA != 0.f;
    const bool onB = ACC != kAccNone && (ACC == kAccMix ? two : fB != 0.f);
    const bool acc_on = onA || onB;
    const float scA = a.acc_scale * fA, scB = a.acc_scale * fB;

    // A z-block of one plane prefetched this pass's accumulator before the
    // previous pass stored it: read it again (the same thread stored it).
    if (ACC != kAccNone && nzb == 1 && p > 0 && row_valid && ok) {
      const int64_t o = (int64_t)z0 * g.plane + row_off;
      ac = *reinterpret_cast<const float4*>(a.acc + o);
      if (ACC == kAccKahan) cp = *reinterpret_cast<const float4*>(a.comp + o);
    }
    // ---- prologue: lower queues from tiles 0 .. r-1; tiles r .. 2r-1 landed
    float4 qa[R], qb[R];
#pragma unroll
    for (int q = 0; q < 2 * R; ++q) {
      ok = ok && bar_wait(&full[q % NB], (uint32_t)((q / NB) & 1), abort_flag, limit);
      if (q < R) {
        const float* tA = tiles + (2 * (q % NB)) * C::STRIDE + own + lo;
        qa[q] = zero4;
        qb[q] = zero4;
        if (ok) {
          const float sg = (neg >> q) & 1u ? -1.f : 1.f;
          qa[q] = f4_scale(*reinterpret_cast<const float4*>(tA), sg);
          if (two) qb[q] = f4_scale(*reinterpret_cast<const float4*>(tA + C::STRIDE), sg);
        }
        release(p, q);
      } else if (yfix) {
        if (__syncthreads_or(!ok)) ok = false;
        if (ok) fill_ghost_rows(q, two);
      }
    }

    int64_t off = (int64_t)z0 * g.plane + row_off;
#pragma unroll
    for (int i = 0; i < kZB; ++i) {
      const int qn = i + 2 * R;            // tile newly needed: plane z0 + i + r
      const int qc = i + R;                // centre tile: plane z0 + i
      ok = ok && bar_wait(&full[qn % NB], (uint32_t)((qn / NB) & 1), abort_flag, limit);
      if (yfix && qn < kZB + R) {          // a future centre tile: fill its ghost rows
        if (__syncthreads_or(!ok)) ok = false;
        if (ok) fill_ghost_rows(qn, two);
      }
      // streams of the next plane (or of the next pass's first plane)
      float4 n_oa = oa, n_ob = ob, n_cf = cf, n_ac = ac, n_cp = cp;
      if (row_valid && ok) {
        if (i + 1 < nzb) load_streams(p, off + g.plane, n_oa, n_ob, n_cf, n_ac, n_cp);
        else if (i + 1 == nzb && p + 1 < npass)   // (a one-plane block rereads acc at the pass start)
          load_streams(p + 1, (int64_t)z0 * g.plane + row_off, n_oa, n_ob, n_cf, n_ac, n_cp);
      }
      if (row_valid && i < nzb && ok) {
        const bool top = z0 + i + R >= g.nz;   // upper neighbours behind the z boundary
        float4 ua, una, ubv = zero4, unb = zero4;
#pragma unroll
        for (int f = 0; f < 2; ++f) {
          if (f == 1 && !two) break;
          float* tc = tiles + (2 * (qc % NB) + f) * C::STRIDE;
          float* srow = tc + (R + warp) * kRowW;
          float4 u = *reinterpret_cast<const float4*>(tc + own + lo);
          if (xfix) {
            const float val = (fx_pos >= 0 && fx_sgn != 0.f) ? fx_sgn * srow[fx_src] : 0.f;
            __syncwarp();
            if (fx_pos >= 0) srow[fx_pos] = val;
            __syncwarp();
            u = mask_row_padding(u, xl, g.nx);
          }
          float lap[4];
          x_terms<R>(srow, lane, lap, 3.f * cw<R>(0));
          float2 l01 = make_float2(lap[0], lap[1]), l23 = make_float2(lap[2], lap[3]);
#pragma unroll
          for (int j = 1; j <= R; ++j) {
            const float4 ym = *reinterpret_cast<const float4*>(tc + own + lo - j * kRowW);
            const float4 yp = *reinterpret_cast<const float4*>(tc + own + lo + j * kRowW);
            const float4 zm = f == 0 ? qa[(i - j + R) % R] : qb[(i - j + R) % R];
            float4 zp = *reinterpret_cast<const float4*>(tiles + (2 * ((qc + j) % NB) + f) * C::STRIDE + own + lo);
            if (top) zp = f4_scale(zp, (neg >> (qc + j)) & 1u ? -1.f : 1.f);
            const float2 c2 = make_float2(cw<R>(j), cw<R>(j));
            l01 = __ffma2_rn(c2, __fadd2_rn(__fadd2_rn(make_float2(ym.x, ym.y), make_float2(yp.x, yp.y)),
                                            __fadd2_rn(make_float2(zm.x, zm.y), make_float2(zp.x, zp.y))), l01);
            l23 = __ffma2_rn(c2, __fadd2_rn(__fadd2_rn(make_float2(ym.z, ym.w), make_float2(yp.z, yp.w)),
                                            __fadd2_rn(make_float2(zm.z, zm.w), make_float2(zp.z, zp.w))), l23);
          }
          const float4 uo = f == 0 ? oa : ob;
          const float2 tw = make_float2(2.f, 2.f);
          const float2 n01 = __ffma2_rn(make_float2(cf.x, cf.y), l01,
                                        __ffma2_rn(tw, make_float2(u.x, u.y), make_float2(-uo.x, -uo.y)));
          const float2 n23 = __ffma2_rn(make_float2(cf.z, cf.w), l23,
                                        __ffma2_rn(tw, make_float2(u.z, u.w), make_float2(-uo.z, -uo.w)));
          const float4 un = make_float4(n01.x, n01.y, n23.x, n23.y);
          if (f == 0) {
            ua = u;
            una = un;
          } else {
            ubv = u;
            unb = un;
          }
        }
        if (xfix) fence_async_smem();   // the ghost writes before the slot is refilled by a copy
        *reinterpret_cast<float4*>(upA + off) = una;
        if (two) *reinterpret_cast<float4*>(upB + off) = unb;
        if (ACC == kAccMix && acc_on) {
          // exact reverse-time mode: field A is u, field B is lambda (Eq.
          // kernel1 mixed term, same operand order as the one-field kernels)
          ac.x = fmaf(scB * (ubv.x - unb.x), ua.x - una.x, ac.x);
          ac.y = fmaf(scB * (ubv.y - unb.y), ua.y - una.y, ac.y);
          ac.z = fmaf(scB * (ubv.z - unb.z), ua.z - una.z, ac.z);
          ac.w = fmaf(scB * (ubv.w - unb.w), ua.w - una.w, ac.w);
          *reinterpret_cast<float4*>(a.acc + off) = ac;
        } else if (acc_on) {
          auto accumulate = [&](float sc, const float4& u, const float4& un) {
            const float d0 = un.x - u.x, d1 = un.y - u.y, d2 = un.z - u.z, d3 = un.w - u.w;
            if (ACC == kAccKahan) {
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
          if (onA) accumulate(scA, ua, una);
          if (onB) accumulate(scB, ubv, unb);
          *reinterpret_cast<float4*>(a.acc + off) = ac;
          if (ACC == kAccKahan) *reinterpret_cast<float4*>(a.comp + off) = cp;
        }
        qa[i % R] = ua;   // plane z enters the lower queues in place of plane z-r
        qb[i % R] = ubv;
      }
      release(p, qc);   // centre tile: last use
      oa = n_oa;
      ob = n_ob;
      cf = n_cf;
      ac = n_ac;
      cp = n_cp;
      off += g.plane;
    }
    // tiles of planes z0+8 .. z0+8+r-1 served as upper neighbours only
#pragma unroll
    for (int q = kZB + R; q < PP; ++q) release(p, q);
  }
  if (!ok) {
    if (lane == 0) atomicExch(b.err, 1);
    *abort_flag = 1;
  }
  // every warp gets here (waits are bounded); then the copies still in
  // flight are waited for (bounded) before the CTA's shared memory goes away
  __syncthreads();
  if (tid == 0 && *abort_flag) {
    for (int s = 0; s < NB; ++s) {
      if (nissued[s] == 0) continue;
      const long long t0 = clock64();
      while (!bar_test(&full[s], (uint32_t)((nissued[s] - 1) & 1)) && clock64() - t0 < limit) {
      }
    }
  }
}

// ---- host side: tensor maps ----------------------------------------------
typedef CUresult (*EncodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encoder() {
  static EncodeTiled fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(p);
  });
  return fn;
}

struct MapKey {
  const void* ptr;
  int64_t px, ny, nz;
  int rows;
  bool operator==(const MapKey& o) const {
    return ptr == o.ptr && px == o.px && ny == o.ny && nz == o.nz && rows == o.rows;
  }
};
struct MapKeyHash {
  size_t operator()(const MapKey& k) const {
    return std::hash<const void*>()(k.ptr) ^ (size_t)(k.px * 1000003 + k.ny * 10007 + k.nz * 101 + k.rows);
  }
};

// The tensor map of one pitched FP32 grid for tiles of `rows` rows: cached by
// (address, geometry); the buffers of a gradient call repeat every step.
cudaError_t tensor_map(const float* ptr, const Geom& g, int rows, CUtensorMap* out) {
  static std::mutex mu;
  static std::unordered_map<MapKey, CUtensorMap, MapKeyHash> cache;
  const MapKey key{ptr, g.px, g.ny, g.nz, rows};
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(key);
  if (it != cache.end()) {
    *out = it->second;
    return cudaSuccess;
  }
  EncodeTiled enc = encoder();
  if (!enc) return cudaErrorNotSupported;
  const cuuint64_t dims[3] = {(cuuint64_t)g.px, (cuuint64_t)g.ny, (cuuint64_t)g.nz};
  const cuuint64_t strides[2] = {(cuuint64_t)g.px * 4, (cuuint64_t)(g.px * g.ny) * 4};
  const cuuint32_t box[3] = {(cuuint32_t)kRowW, (cuuint32_t)rows, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  CUtensorMap m;
  const CUresult r = enc(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(ptr), dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  if (cache.size() > 4096) cache.clear();
  cache.emplace(key, m);
  *out = m;
  return cudaSuccess;
}

template <int R, int ACC>
cudaError_t launch_s(const StreamArgs& p, cudaStream_t s) {
  using C = SCfg<R>;
  cudaError_t e = set_smem_limit_once(reinterpret_cast<const void*>(step3d_velocity_stream_kernel<R, ACC>), (int)C::bytes());
  if (e != cudaSuccess) return e;
  const Geom& g = p.b.base.g;
  dim3 grid((unsigned)((g.nz + kZB - 1) / kZB), (unsigned)((g.nx + kStrip - 1) / kStrip),
            (unsigned)((g.ny + kTY - 1) / kTY));
  step3d_velocity_stream_kernel<R, ACC><<<grid, kThreads, C::bytes(), s>>>(p);
  count_launch();
  return cudaGetLastError();
}

template <int R>
cudaError_t launch_s_r(const StreamArgs& p, cudaStream_t s) {
  const BatchArgs& b = p.b;
  if (b.pair_mix) return launch_s<R, kAccMix>(p, s);
  bool any = false;
  for (int i = 0; i < b.nshots; ++i) any |= b.accf[i] != 0.f;
  if (!any || !b.base.acc) return launch_s<R, kAccNone>(p, s);
  if (b.base.comp) return launch_s<R, kAccKahan>(p, s);
  return launch_s<R, kAccSq>(p, s);
}

}  // namespace

// Whether the TMA-streamed kernel can take this launch: FP32 velocity form,
// 32-bit tile coordinates, a rows-of-128 pitch, an error word for its
// bounded waits, and no stored-history operands.
bool stream_supported(const BatchArgs& b) {
  const Geom& g = b.base.g;
  return b.nshots >= 1 && b.err != nullptr && !b.base.mix_a && !b.base.u_out && g.nz < (1 << 30) &&
         g.ny < (1 << 30) && g.px < (1 << 30) && (g.px % kStrip) == 0;
}

cudaError_t launch_step3d_stream(const BatchArgs& b, int order, cudaStream_t s) {
  const int R = order / 2;
  StreamArgs p;
  memset(&p, 0, sizeof(p));
  p.b = b;
  for (int i = 0; i < b.nshots; ++i) {
    cudaError_t e = tensor_map(b.cur[i], b.base.g, kTY + 2 * R, &p.map[i]);
    if (e != cudaSuccess) return e;
  }
  switch (order) {
    case 2: return launch_s_r<1>(p, s);
    case 4: return launch_s_r<2>(p, s);
    case 6: return launch_s_r<3>(p, s);
    case 8: return launch_s_r<4>(p, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace wave
