// 3D fused leapfrog step, FP32 storage, orders 2-8, batched launches: a CTA
// advances every shot of the launch over its tile, one after the other, with
// the sensitivity accumulator of its cells held in registers throughout and
// the u^n tiles arriving by TMA tensor copies.
//
// Arithmetic, element by element, is that of the other velocity pipelines
// (Eq. FDstencil1 in squared-slowness form; Algorithm 1's sensitivity
// increment of Eq. kernel1, the shots' increments added in launch order), so
// the results are bit-identical to theirs.  The mapping:
//
// * a CTA owns 16 rows x 128 cells (one warp per row, four cells per lane)
//   and a z-block of 8 planes; grid x runs over z-blocks fastest, so the CTAs
//   of neighbouring z-blocks run side by side and the halo planes one of them
//   stages the other reads at about the same time (an L2 hit);
// * each lane keeps the accumulator (and its Kahan compensation) of its 4 x 8
//   cells in registers: read once at the start, written once at the end of the
//   launch, whatever the number of shots -- the accumulator crosses HBM once
//   per step;
// * per shot the CTA needs the tiles of planes z0-r .. z0+8+r-1: 8 + 2r tiles of
//   16 + 2r rows x 136 cells (4 halo cells per side).  The shared-memory ring
//   holds exactly one shot's tiles, so tile q of shot s sits in slot q and the
//   copy of tile q of shot s+1 starts as soon as every warp is done with tile
//   q of shot s (the last warp to release a slot issues the copy): the next
//   shot's tiles stream in while the current shot is computed;
// * a warp keeps planes z-r .. z-1 of its row in a register queue, reads the x
//   and y neighbours from the tile of plane z and the upper z neighbours from
//   the tiles of planes z+1 .. z+r;
// * u^{n-1} and coef of the next plane (across a shot boundary, of the next
//   shot's first plane) are loaded into registers while a plane is computed;
// * ghost values: out-of-range tile rows and planes arrive as zeros (the
//   copy's out-of-bounds fill).  In CTAs at a y boundary the warps fill the
//   ghost rows of each centre tile from their mirror rows (then a CTA barrier);
//   planes behind a z boundary are copied from their mirror planes and read
//   with the mirror sign; the x ghosts of a warp's own row are written by that
//   warp;
// * every wait is bounded (wait_limit_cycles): on time-out the kernel sets the
//   device error word, the warps run their loops on without work, and the
//   copies in flight are waited for (bounded) before the CTA exits.
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
  static constexpr int STRIDE = (TILE + 31) / 32 * 32;   // floats between slots: 128-byte aligned copies
  static constexpr int PP = kZB + 2 * R;         // tiles per shot = ring slots
  static constexpr size_t BAR_OFF = (size_t)PP * STRIDE * 4;
  static constexpr size_t bytes() { return BAR_OFF + PP * sizeof(uint64_t) + 2 * PP * sizeof(int) + 16; }
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

enum { kAccNone = 0, kAccSq = 1, kAccKahan = 2 };

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
  constexpr int PP = C::PP;
  extern __shared__ __align__(128) float tiles[];   // [PP][STRIDE]
  uint64_t* full = reinterpret_cast<uint64_t*>(reinterpret_cast<char*>(tiles) + C::BAR_OFF);
  int* released = reinterpret_cast<int*>(full + PP);   // warps done with the slot's tile
  int* nissued = released + PP;                        // copies issued into the slot
  volatile int* abort_flag = nissued + PP;

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
  const int nsh = b.nshots;

  // Copy tile q (plane z0 - r + q) of shot s into slot q.
  auto issue = [&](int s, int q) {
    float sg;
    const int zsrc = tile_source(z0 - R + q, g, R, &sg);
    bar_expect(&full[q], (uint32_t)C::TILE_BYTES);
    tma_load_3d(tiles + q * C::STRIDE, &P.map[s], x0 - 4, ty0 - R, zsrc, &full[q]);
    nissued[q] += 1;
  };

  if (tid == 0) {
    for (int q = 0; q < PP; ++q) {
      bar_init(&full[q], 1);
      released[q] = 0;
      nissued[q] = 0;
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  if (tid == 0 && !b.debug_stall)
    for (int q = 0; q < PP; ++q) issue(0, q);

  // A warp is done with tile q of shot s: the last of the 16 warps to say so
  // copies tile q of the next shot into the slot.  The fences order the
  // warps' reads (and ghost writes) of the slot before the copy.
  auto release = [&](int s, int q) {
    __syncwarp();
    if (lane == 0) {
      __threadfence_block();
      if (atomicAdd(&released[q], 1) == kTY - 1) {
        released[q] = 0;
        __threadfence_block();
        fence_async_smem();
        if (s + 1 < nsh && !b.debug_stall && !*abort_flag) issue(s + 1, q);
      }
    }
  };

  const int y = ty0 + warp;
  const bool row_valid = y < g.ny;
  const int xl = x0 + 4 * lane;
  const bool xfix = (x0 == 0) || (x0 + kStrip + R > g.nx);
  const bool xfast = (g.nx % kStrip) == 0;   // row ends on strip boundaries: x ghosts in registers
  // rows behind a y boundary are filled from their mirror rows by the warps
  // once a centre tile has landed (then a CTA barrier; uniform per CTA)
  const bool yfix = ty0 == 0 || ty0 + kTY + R > g.ny;
  const int64_t row_off = (int64_t)y * g.px + xl;
  constexpr int own = R * kRowW + 4;              // own cells of warp 0, lane 0 in a tile
  const int lo = warp * kRowW + 4 * lane;

  // ghost row this warp fills in y-boundary CTAs: tile row gt from row gsrc, sign gsg
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
  auto fill_ghost_rows = [&](int q) {
    if (gt >= 0) {
      float* t = tiles + q * C::STRIDE;
      for (int c = lane; c < kRowW / 4; c += 32) {
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (gsg != 0.f) v = f4_scale(*reinterpret_cast<const float4*>(t + gsrc * kRowW + 4 * c), gsg);
        *reinterpret_cast<float4*>(t + gt * kRowW + 4 * c) = v;
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
  // signs of the tiles (planes z0 - r + q): bit q set = read negated
  uint32_t neg = 0;
  for (int q = 0; q < PP; ++q) {
    float sg;
    tile_source(z0 - R + q, g, R, &sg);
    if (sg < 0.f) neg |= 1u << q;
  }
  const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
  const int64_t off0 = (int64_t)z0 * g.plane + row_off;

  // the accumulator (and compensation) of the lane's cells in the z-block
  float4 acc[kZB], cmp[kZB];
#pragma unroll
  for (int i = 0; i < kZB; ++i) {
    acc[i] = zero4;
    cmp[i] = zero4;
    if (ACC != kAccNone && row_valid && i < nzb) {
      acc[i] = *reinterpret_cast<const float4*>(a.acc + off0 + (int64_t)i * g.plane);
      if (ACC == kAccKahan) cmp[i] = *reinterpret_cast<const float4*>(a.comp + off0 + (int64_t)i * g.plane);
    }
  }

  // u^{n-1} and coef of plane z0 + i of shot s
  float4 uo = zero4, cf = zero4;
  if (row_valid) {
    uo = *reinterpret_cast<const float4*>(b.prev[0] + off0);
    cf = __ldg(reinterpret_cast<const float4*>(a.coef + off0));
  }
  bool ok = true;

  // After a time-out (ok false) the loops run on without work, so every warp
  // passes the same CTA barriers and reaches the end.
  for (int s = 0; s < nsh; ++s) {
    const uint32_t par = (uint32_t)(s & 1);      // each slot completes once per shot
    float* const up = b.prev[s];
    const float sc = a.acc_scale * b.accf[s];
    const bool acc_on = ACC != kAccNone && b.accf[s] != 0.f;

    // ---- prologue: lower queue from tiles 0 .. r-1; tiles r .. 2r-1 landed
    float4 ql[R];
#pragma unroll
    for (int q = 0; q < 2 * R; ++q) {
      ok = ok && bar_wait(&full[q], par, abort_flag, limit);
      if (q < R) {
        ql[q] = zero4;
        if (ok) {
          const float sg = (neg >> q) & 1u ? -1.f : 1.f;
          ql[q] = f4_scale(*reinterpret_cast<const float4*>(tiles + q * C::STRIDE + own + lo), sg);
        }
        release(s, q);
      } else if (yfix) {
        if (__syncthreads_or(!ok)) ok = false;
        if (ok) fill_ghost_rows(q);
      }
    }

#pragma unroll
    for (int i = 0; i < kZB; ++i) {
      const int qn = i + 2 * R;            // tile newly needed: plane z0 + i + r
      const int qc = i + R;                // centre tile: plane z0 + i
      ok = ok && bar_wait(&full[qn], par, abort_flag, limit);
      if (yfix && qn < kZB + R) {          // a future centre tile: fill its ghost rows
        if (__syncthreads_or(!ok)) ok = false;
        if (ok) fill_ghost_rows(qn);
      }
      // streams of the next plane (or of the next shot's first plane)
      float4 n_uo = uo, n_cf = cf;
      if (row_valid && ok) {
        if (i + 1 < nzb) {
          n_uo = *reinterpret_cast<const float4*>(up + off0 + (int64_t)(i + 1) * g.plane);
          n_cf = __ldg(reinterpret_cast<const float4*>(a.coef + off0 + (int64_t)(i + 1) * g.plane));
        } else if (i + 1 == nzb && s + 1 < nsh) {
          n_uo = *reinterpret_cast<const float4*>(b.prev[s + 1] + off0);
          n_cf = __ldg(reinterpret_cast<const float4*>(a.coef + off0));
        }
      }
      if (row_valid && i < nzb && ok) {
        const bool top = z0 + i + R >= g.nz;   // upper neighbours behind the z boundary
        float* tc = tiles + qc * C::STRIDE;
        float* srow = tc + (R + warp) * kRowW;
        float4 u = *reinterpret_cast<const float4*>(tc + own + lo);
        float lap[4];
        if (xfix && !xfast) {   // ragged row end: ghosts written into the staged row
          const float val = (fx_pos >= 0 && fx_sgn != 0.f) ? fx_sgn * srow[fx_src] : 0.f;
          __syncwarp();
          if (fx_pos >= 0) srow[fx_pos] = val;
          __syncwarp();
          u = mask_row_padding(u, xl, g.nx);
          fence_async_smem();   // the ghost writes before the slot is refilled by a copy
          x_terms<R>(srow, lane, lap, 3.f * cw<R>(0));
        } else {
          float4 xa = *reinterpret_cast<const float4*>(srow + 4 * lane);
          float4 xc = *reinterpret_cast<const float4*>(srow + 8 + 4 * lane);
          if (xfix) {   // row ends on a strip boundary: ghosts from the lane's own cells
            if (lane == 0 && x0 == 0) xa = left_ghosts(u, g.bc);
            if (lane == 31 && x0 + kStrip == g.nx) xc = right_ghosts(u, g.bc);
          }
          x_terms_abc<R>(xa, u, xc, lap, 3.f * cw<R>(0));
        }
        float2 l01 = make_float2(lap[0], lap[1]), l23 = make_float2(lap[2], lap[3]);
#pragma unroll
        for (int j = 1; j <= R; ++j) {
          const float4 ym = *reinterpret_cast<const float4*>(tc + own + lo - j * kRowW);
          const float4 yp = *reinterpret_cast<const float4*>(tc + own + lo + j * kRowW);
          const float4 zm = ql[(i - j + R) % R];
          float4 zp = *reinterpret_cast<const float4*>(tiles + (qc + j) * C::STRIDE + own + lo);
          if (top) zp = f4_scale(zp, (neg >> (qc + j)) & 1u ? -1.f : 1.f);
          const float2 c2 = make_float2(cw<R>(j), cw<R>(j));
          l01 = __ffma2_rn(c2, __fadd2_rn(__fadd2_rn(make_float2(ym.x, ym.y), make_float2(yp.x, yp.y)),
                                          __fadd2_rn(make_float2(zm.x, zm.y), make_float2(zp.x, zp.y))), l01);
          l23 = __ffma2_rn(c2, __fadd2_rn(__fadd2_rn(make_float2(ym.z, ym.w), make_float2(yp.z, yp.w)),
                                          __fadd2_rn(make_float2(zm.z, zm.w), make_float2(zp.z, zp.w))), l23);
        }
        const float2 tw = make_float2(2.f, 2.f);
        const float2 n01 = __ffma2_rn(make_float2(cf.x, cf.y), l01,
                                      __ffma2_rn(tw, make_float2(u.x, u.y), make_float2(-uo.x, -uo.y)));
        const float2 n23 = __ffma2_rn(make_float2(cf.z, cf.w), l23,
                                      __ffma2_rn(tw, make_float2(u.z, u.w), make_float2(-uo.z, -uo.w)));
        const float4 un = make_float4(n01.x, n01.y, n23.x, n23.y);
        *reinterpret_cast<float4*>(up + off0 + (int64_t)i * g.plane) = un;
        if (acc_on) {
          const float d0 = un.x - u.x, d1 = un.y - u.y, d2 = un.z - u.z, d3 = un.w - u.w;
          if (ACC == kAccKahan) {
            kahan_add(acc[i].x, cmp[i].x, sc * d0 * d0);
            kahan_add(acc[i].y, cmp[i].y, sc * d1 * d1);
            kahan_add(acc[i].z, cmp[i].z, sc * d2 * d2);
            kahan_add(acc[i].w, cmp[i].w, sc * d3 * d3);
          } else {
            const float2 s2 = make_float2(sc, sc);
            const float2 e01 = make_float2(d0, d1), e23 = make_float2(d2, d3);
            const float2 r01 = __ffma2_rn(__fmul2_rn(s2, e01), e01, make_float2(acc[i].x, acc[i].y));
            const float2 r23 = __ffma2_rn(__fmul2_rn(s2, e23), e23, make_float2(acc[i].z, acc[i].w));
            acc[i] = make_float4(r01.x, r01.y, r23.x, r23.y);
          }
        }
        ql[i % R] = u;   // plane z enters the lower queue in place of plane z-r
      }
      release(s, qc);   // centre tile: last use
      uo = n_uo;
      cf = n_cf;
    }
    // tiles of planes z0+8 .. z0+8+r-1 served as upper neighbours only
#pragma unroll
    for (int q = kZB + R; q < PP; ++q) release(s, q);
  }
  // the accumulator crosses HBM once per launch
  if (ACC != kAccNone && row_valid && ok) {
#pragma unroll
    for (int i = 0; i < kZB; ++i) {
      if (i < nzb) {
        *reinterpret_cast<float4*>(a.acc + off0 + (int64_t)i * g.plane) = acc[i];
        if (ACC == kAccKahan) *reinterpret_cast<float4*>(a.comp + off0 + (int64_t)i * g.plane) = cmp[i];
      }
    }
  }
  if (!ok) {
    if (lane == 0) atomicExch(b.err, 1);
    *abort_flag = 1;
  }
  // every warp gets here (waits are bounded); then the copies still in
  // flight are waited for (bounded) before the CTA's shared memory goes away
  __syncthreads();
  if (tid == 0 && *abort_flag) {
    for (int q = 0; q < PP; ++q) {
      if (nissued[q] == 0) continue;
      const long long t0 = clock64();
      while (!bar_test(&full[q], (uint32_t)((nissued[q] - 1) & 1)) && clock64() - t0 < limit) {
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
  e = cudaGetLastError();
  if (e != cudaSuccess) note_error("step kernel launch", e);
  return e;
}

template <int R>
cudaError_t launch_s_r(const StreamArgs& p, cudaStream_t s) {
  const BatchArgs& b = p.b;
  bool any = false;
  for (int i = 0; i < b.nshots; ++i) any |= b.accf[i] != 0.f;
  if (!any || !b.base.acc) return launch_s<R, kAccNone>(p, s);
  if (b.base.comp) return launch_s<R, kAccKahan>(p, s);
  return launch_s<R, kAccSq>(p, s);
}

}  // namespace

// Whether the TMA-streamed kernel can take this launch: FP32 velocity form,
// 32-bit tile coordinates, a rows-of-128 pitch, an error word for its
// bounded waits, no stored-history operands and no mixed (u, lambda) term.
bool stream_supported(const BatchArgs& b) {
  const Geom& g = b.base.g;
  return b.nshots >= 1 && b.err != nullptr && !b.pair_mix && !b.base.mix_a && g.nz < (1 << 30) &&
         g.ny < (1 << 30) && g.px < (1 << 30) && (g.px % kStrip) == 0;
}

cudaError_t launch_step3d_stream(const BatchArgs& b, int order, cudaStream_t s) {
  const int R = order / 2;
  StreamArgs p;
  memset(&p, 0, sizeof(p));
  p.b = b;
  for (int i = 0; i < b.nshots; ++i) {
    cudaError_t e = tensor_map(b.cur[i], b.base.g, kTY + 2 * R, &p.map[i]);
    if (e != cudaSuccess) {
      note_error("cuTensorMapEncodeTiled", e);
      return e;
    }
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
