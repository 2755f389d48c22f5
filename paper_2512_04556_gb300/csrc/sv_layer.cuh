// One layer of the spatially varying cascade (Sec. 4.3 Eq. 9 + Sec. 3.2
// Eq. 3): the kernel template shared by the 1-D and 2-D translation units.
//
// Each CTA owns a 32 x 16 or 32 x 32 output tile (PIX = 2 or 4 vertically
// adjacent pixels of one column per thread; neighbouring pixels share the
// corner row between them when their integer offsets agree).  It stages the layer's source
// region (tile + the layer's halo, clamp-to-edge) into shared memory as FP32
// planes -- (r, g) pairs in one, b (or (b, a) pairs) in another -- converting
// FP16 sources once per staged pixel instead of once per tap and corner; a
// warp's 32 lanes (consecutive columns) read consecutive entries.  A planar
// FP32 intermediate is copied in by the tensor-memory accelerator; the
// caller's image goes through registers.  The layer's node taps are copied
// into shared memory beside the region.  Arithmetic and accumulation are FP32.
// When each thread's pixels sit in one kernel-space cell -- the common case,
// parameter maps being smooth -- the node taps of each tap index are fetched
// once per thread (128-bit shared-memory broadcasts) and blended for its
// pixels with each pixel's own weights; warps with a thread whose pixels
// straddle cells take the per-pixel path.
// The rotated variant (ROT) turns every pixel's blended tap offsets by that
// pixel's angle before sampling: the runtime form of the rotational and
// radial blur effects of Sec. 5.3, exact for the complex's impulse response.
#pragma once

#include <cuda.h>

#include <type_traits>

#include "sv_common.cuh"

namespace disk {

// Tile configurations: 32 columns x (8 warps x PIX rows); PIX pixels per
// thread.  PIX = 4 (32 x 32 tiles, 3 CTAs per SM) or PIX = 2 (32 x 16 tiles,
// 4 CTAs per SM); disk_sv_filter_autotune picks per frame shape.
constexpr int kSvTileW = 32, kSvThreads = 256;
constexpr int kSvWarps = kSvThreads / 32;
constexpr int kSvDefaultPix = 2;
__host__ __device__ constexpr int sv_tile_h(int pix) { return pix * kSvWarps; }
// Where a layer reads its node taps (B x T float4 (dx, dy, w, w)): a copy
// each block makes in shared memory, or global memory through L1 when that
// copy does not fit beside the staged region.
enum : int { kSvTapsGlobal = 0, kSvTapsShared = 1 };
constexpr int kSvMaxSmem = 232448;           // 227 KB opt-in shared memory per CTA

// Shared-memory bytes per staged pixel: FP32 (r, g) + b, or (r, g) + (b, a).
__host__ __device__ constexpr size_t sv_stage_bytes(int C) { return C == 4 ? 16 : 12; }

// Staged region of RN pixels: the (r, g) plane, then the b / (b, a) plane at
// a 128-byte boundary (the tensor copies' destination alignment), then the
// copy's mbarrier (8 bytes, in a 16-byte slot).
__host__ __device__ constexpr size_t sv_plane_b_offset(size_t RN) { return (RN * 8 + 127) & ~(size_t)127; }
__host__ __device__ constexpr size_t sv_smem_bytes(size_t RN, int C) {
  return ((sv_plane_b_offset(RN) + RN * (C == 4 ? 8 : 4) + 15) & ~(size_t)15) + 16;
}

// Iteration limit of the wait for a tile copy (each try_wait may also
// suspend the thread for a while); past it the kernel records
// DISK_ERR_TIMEOUT in *err and the block returns.
constexpr long long kSvMaxWaitIters = 1ll << 22;

struct SvLayerParams {
  // Tensor maps of the planar source's two planes (used when use_tma; the
  // type carries the 128-byte alignment the copies require).
  CUtensorMap tm_a;
  CUtensorMap tm_b;
  const void *src;
  long long src_pitch;   // bytes per row (plane A's rows for a planar source)
  long long src_plane_b; // planar source: byte offset of plane B
  void *dst;
  long long dst_pitch;
  long long dst_plane_b;
  const float *maps;
  const float2 *rot;    // [H][W] (cos, sin) of each pixel's angle, rotated variant only
  const float4 *gtaps;  // [B][T] taps of this layer: (dx, dy, w, w)
  int *err;             // device status word (DISK_ERR_TIMEOUT after a given-up wait)
  int H, W, C, T;
  int halo;             // rows staged above and below the tile
  int halo_x;           // columns staged left and right (>= halo; a multiple of 4 with TMA)
  int region_w;         // kSvTileW + 2 halo_x
  int use_tma;          // planar source copied by the tensor-memory accelerator
  int bt;               // B * T taps of this layer
  int tap_cap;          // nodes whose taps a block may copy into shared memory
  AxisNodes ax[2];
};

__device__ __forceinline__ unsigned smem_addr(const void *p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

// One 2-D tile of a tensor map into shared memory, completing on mbarrier
// bar (which expects the bytes beforehand).  x must be a multiple of 16
// bytes' worth of elements; out-of-range elements read as zero.
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y,
                                            unsigned bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];"
      :: "r"(smem_addr(dst)), "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y),
         "r"(bar)
      : "memory");
}

// Bounded wait for phase `parity` of mbarrier bar; false if it gave up.
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity,
                                          long long max_iters = kSvMaxWaitIters) {
  for (long long i = 0; i < max_iters; ++i) {
    unsigned ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;"
        " selp.u32 %0, 1, 0, p; }"
        : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
    if (ok) return true;
  }
  return false;
}

// Pixel weights of Eq. 9 broadcast into FP32 pairs for the packed
// (f32x2) arithmetic of sv_tap; built once per pixel.
struct CellPairs {
  float2 a00, a10, a01, a11;
};

__device__ __forceinline__ CellPairs cell_pairs(const Cell &c) {
  return {make_float2(c.a00, c.a00), make_float2(c.a10, c.a10), make_float2(c.a01, c.a01),
          make_float2(c.a11, c.a11)};
}

// Per-pixel accumulator: (r, g) as a packed pair, b and a scalar.
struct Acc {
  float2 rg;
  float b, a;
};

__device__ __forceinline__ float2 lo2(const float4 &v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(const float4 &v) { return make_float2(v.z, v.w); }

// The staged region: (r, g) pairs, then b (3 channels) or (b, a) pairs.
struct Staged {
  const float2 *rg;
  const float *b;     // CH == 3
  const float2 *ba;   // CH == 4
};

// Weighted corner e of the staged region into the accumulator.
template <int CH>
__device__ __forceinline__ void add_corner(const Staged &st, int e, const float2 &wb, Acc &acc) {
  acc.rg = __ffma2_rn(wb, st.rg[e], acc.rg);
  if (CH == 4) {
    const float2 ba = st.ba[e];
    acc.b = fmaf(wb.x, ba.x, acc.b);
    acc.a = fmaf(wb.x, ba.y, acc.a);
  } else {
    acc.b = fmaf(wb.x, st.b[e], acc.b);
  }
}

// Rotation of a pixel's offsets as two pairs: (cos, sin) and (-sin, cos).
struct RotPairs {
  float2 c, s;
};

// One tap of one pixel: the Eq. 9 blend of the node taps (dx, dy, w, w) with
// the pixel's weights, the optional rotation of the blended offset, the
// integer/fraction split of the offset, and the Eq. 2 bilinear sample from
// the staged region, all in packed FP32 pairs: (dx, dy) and the corner
// weights travel as pairs, colour as (r, g) + b.
template <int DIMS, int CH, bool ROT>
__device__ __forceinline__ void sv_tap(const float4 &q00, const float4 &q10, const float4 &q01,
                                       const float4 &q11, const CellPairs &a, const RotPairs &rot,
                                       const Staged &st, int base, int RW, Acc &acc) {
  float2 d = __fmul2_rn(a.a00, lo2(q00));
  float2 w = __fmul2_rn(a.a00, hi2(q00));
  d = __ffma2_rn(a.a10, lo2(q10), d);
  w = __ffma2_rn(a.a10, hi2(q10), w);
  if (DIMS == 2) {
    d = __ffma2_rn(a.a01, lo2(q01), d);
    w = __ffma2_rn(a.a01, hi2(q01), w);
    d = __ffma2_rn(a.a11, lo2(q11), d);
    w = __ffma2_rn(a.a11, hi2(q11), w);
  }
  // (dx, dy) -> (dx cos - dy sin, dx sin + dy cos)
  if (ROT) d = __ffma2_rn(make_float2(d.x, d.x), rot.c, __fmul2_rn(make_float2(d.y, d.y), rot.s));
  // integer part n = round-to-nearest(d - 1/2) (= floor(d) except at exact
  // integers, where bilinear sampling gives the same value either way) and
  // fraction f = d - n in [0, 1], for both axes at once; see split_offset.
  const float magic = 12582912.0f;
  const float2 r = __fadd2_rn(__fadd2_rn(d, make_float2(-0.5f, -0.5f)), make_float2(magic, magic));
  const float2 f = __ffma2_rn(__fadd2_rn(r, make_float2(-magic, -magic)), make_float2(-1.f, -1.f), d);
  // In bounds by construction: the Eq. 9 weights are non-negative and sum to
  // one within a few ulp (t is clamped to [0, 1] and p to the node range,
  // NaN to the first node), and every node tap satisfies |o| <= R, the layer
  // reach; so the blended |d| <= R (1 + 2^-21) and n = round(d - 1/2) lies in
  // [-ceil(R) - 1, ceil(R)] = [-halo, halo - 1], which with the corner n + 1
  // keeps every read inside the staged tile + halo region.  The rotated
  // variant takes R as the largest Euclidean tap length (the norm of a convex
  // blend is at most the largest node norm) and reads (cos, sin) normalised
  // to unit length by rotation_kernel, so each rotated component is within
  // R (1 + 2^-20): the same argument holds.
  const int nx = __float_as_int(r.x) - 0x4B400000;
  const int ny = __float_as_int(r.y) - 0x4B400000;
  const int e = base + ny * RW + nx;
  const float2 fx = make_float2(f.x, f.x), fy = make_float2(f.y, f.y);
  const float2 wy1 = __fmul2_rn(w, fy), wy0 = __ffma2_rn(wy1, make_float2(-1.f, -1.f), w);
  const float2 w11 = __fmul2_rn(wy1, fx), w10 = __ffma2_rn(w11, make_float2(-1.f, -1.f), wy1);
  const float2 w01 = __fmul2_rn(wy0, fx), w00 = __ffma2_rn(w01, make_float2(-1.f, -1.f), wy0);
  add_corner<CH>(st, e, w00, acc);
  add_corner<CH>(st, e + 1, w01, acc);
  add_corner<CH>(st, e + RW, w10, acc);
  add_corner<CH>(st, e + RW + 1, w11, acc);
}

// The thread's N vertically adjacent pixels and one tap, top to bottom.
// Neighbouring pixels' sample points usually have the same integer offset
// (the offsets vary slowly across pixels), and then a pixel's top corners
// are the previous pixel's bottom corners: they are kept in registers
// instead of being read from shared memory again.
template <int DIMS, int CH, bool ROT, int N>
__device__ __forceinline__ void sv_tap_column(const float4 &q00, const float4 &q10, const float4 &q01,
                                              const float4 &q11, const CellPairs *cp,
                                              const RotPairs *rp, const Staged &st, int base0,
                                              int RW, Acc *acc) {
  int eprev = 0;
  float2 prg0 = make_float2(0.f, 0.f), prg1 = prg0, pba0 = prg0, pba1 = prg0;
  auto accum = [&](Acc &a, const float2 &wb, const float2 &rg, const float2 &ba) {
    a.rg = __ffma2_rn(wb, rg, a.rg);
    a.b = fmaf(wb.x, ba.x, a.b);
    if (CH == 4) a.a = fmaf(wb.x, ba.y, a.a);
  };
  auto load_ba = [&](int e) -> float2 {
    return CH == 4 ? st.ba[e] : make_float2(st.b[e], 0.f);
  };
#pragma unroll
  for (int p = 0; p < N; ++p) {
    const CellPairs &a = cp[p];
    float2 d = __fmul2_rn(a.a00, lo2(q00));
    float2 w = __fmul2_rn(a.a00, hi2(q00));
    d = __ffma2_rn(a.a10, lo2(q10), d);
    w = __ffma2_rn(a.a10, hi2(q10), w);
    if (DIMS == 2) {
      d = __ffma2_rn(a.a01, lo2(q01), d);
      w = __ffma2_rn(a.a01, hi2(q01), w);
      d = __ffma2_rn(a.a11, lo2(q11), d);
      w = __ffma2_rn(a.a11, hi2(q11), w);
    }
    if (ROT) d = __ffma2_rn(make_float2(d.x, d.x), rp[p].c, __fmul2_rn(make_float2(d.y, d.y), rp[p].s));
    // split and bounds as in sv_tap
    const float magic = 12582912.0f;
    const float2 r = __fadd2_rn(__fadd2_rn(d, make_float2(-0.5f, -0.5f)), make_float2(magic, magic));
    const float2 f = __ffma2_rn(__fadd2_rn(r, make_float2(-magic, -magic)), make_float2(-1.f, -1.f), d);
    const int nx = __float_as_int(r.x) - 0x4B400000;
    const int ny = __float_as_int(r.y) - 0x4B400000;
    const int e = base0 + p * RW + ny * RW + nx;
    const float2 fx = make_float2(f.x, f.x), fy = make_float2(f.y, f.y);
    const float2 wy1 = __fmul2_rn(w, fy), wy0 = __ffma2_rn(wy1, make_float2(-1.f, -1.f), w);
    const float2 w11 = __fmul2_rn(wy1, fx), w10 = __ffma2_rn(w11, make_float2(-1.f, -1.f), wy1);
    const float2 w01 = __fmul2_rn(wy0, fx), w00 = __ffma2_rn(w01, make_float2(-1.f, -1.f), wy0);
    float2 t0, t1, tb0, tb1;
    if (p > 0 && e == eprev + RW) {
      t0 = prg0; t1 = prg1; tb0 = pba0; tb1 = pba1;
    } else {
      t0 = st.rg[e]; t1 = st.rg[e + 1]; tb0 = load_ba(e); tb1 = load_ba(e + 1);
    }
    prg0 = st.rg[e + RW]; prg1 = st.rg[e + RW + 1];
    pba0 = load_ba(e + RW); pba1 = load_ba(e + RW + 1);
    eprev = e;
    accum(acc[p], w00, t0, tb0);
    accum(acc[p], w01, t1, tb1);
    accum(acc[p], w10, prg0, pba0);
    accum(acc[p], w11, prg1, pba1);
  }
}

template <int DIMS, int SRC, int DST, int TAPS, int CH, int PIX, bool ROT>
__global__ void __launch_bounds__(kSvThreads, PIX == 2 ? 4 : 3)
sv_layer_kernel(const __grid_constant__ SvLayerParams P) {
  constexpr int kSvPix = PIX, kSvTileH = PIX * kSvWarps;
  extern __shared__ __align__(128) unsigned char sm_raw[];
  const int halo = P.halo, hx = P.halo_x, RW = P.region_w, RH = kSvTileH + 2 * halo, RN = RW * RH;
  float2 *s_rg = reinterpret_cast<float2 *>(sm_raw);
  float *s_b = reinterpret_cast<float *>(sm_raw + sv_plane_b_offset(RN));
  float2 *s_ba = reinterpret_cast<float2 *>(sm_raw + sv_plane_b_offset(RN));
  unsigned long long *s_bar = reinterpret_cast<unsigned long long *>(
      sm_raw + sv_smem_bytes(RN, CH) - 16);
  // The node taps the block needs, copied into shared memory after the
  // block's node range is known (see below); a warp's threads mostly fetch
  // the same tap, a broadcast.
  float4 *s_taps = reinterpret_cast<float4 *>(sm_raw + sv_smem_bytes(RN, CH));
  unsigned *s_range = reinterpret_cast<unsigned *>(s_bar + 1);  // lowest, highest node
  const int tx0 = blockIdx.x * kSvTileW, ty0 = blockIdx.y * kSvTileH;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // The tensor copies need a 128-byte aligned destination; a block whose
  // shared window is not (never seen) records an error and does nothing.
  const bool tma = SRC == PIX_PLANAR && P.use_tma;
  if (tma && (smem_addr(sm_raw) & 127u) != 0) {
    if (threadIdx.x == 0) atomicExch(P.err, DISK_ERR_UNSUPPORTED);
    return;
  }
  if (TAPS == kSvTapsShared && threadIdx.x == 0) {
    s_range[0] = 0xffffffffu;
    s_range[1] = 0u;
  }
  if (tma && threadIdx.x == 0) {
    // Both planes of the region [ty0 - halo, +RH) x [tx0 - hx, +RW) in one
    // phase of the barrier.  x offsets: 2 (tx0 - hx) floats for the pair
    // planes, tx0 - hx for a b plane; tx0 is a multiple of 32 and hx of 4,
    // so both start on 16-byte boundaries as the copy requires.
    const unsigned bar = smem_addr(s_bar);
    const unsigned bytes = (unsigned)RN * (CH == 4 ? 16u : 12u);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(bar), "r"(bytes)
                 : "memory");
    tma_load_2d(s_rg, &P.tm_a, 2 * (tx0 - hx), ty0 - halo, bar);
    tma_load_2d(s_b, &P.tm_b, CH == 4 ? 2 * (tx0 - hx) : tx0 - hx, ty0 - halo, bar);
  }

  const int x = tx0 + lane, xc = min(x, P.W - 1);
  const long long HW = (long long)P.H * P.W;
  const int T = P.T;
  // A table small enough for every block to hold whole is copied now,
  // overlapping the tile copy; larger ones are copied per node range below.
  const bool whole = TAPS == kSvTapsShared && P.tap_cap * T >= P.bt;
  if (whole)
    for (int i = threadIdx.x; i < P.bt; i += kSvThreads) s_taps[i] = __ldg(P.gtaps + i);
  // This thread's map values (and rotations), loaded before the staging so
  // their latency overlaps it; the cells are formed after it.
  float pv0[kSvPix], pv1[kSvPix];
  float2 rv[kSvPix];
#pragma unroll
  for (int j = 0; j < kSvPix; ++j) {
    const int yc = min(ty0 + warp * kSvPix + j, P.H - 1);
    const long long px = (long long)yc * P.W + xc;
    pv0[j] = __ldg(P.maps + px);
    pv1[j] = DIMS == 2 ? __ldg(P.maps + HW + px) : 0.f;
    rv[j] = ROT ? __ldg(P.rot + px) : make_float2(1.f, 0.f);
  }
  const bool ranged = TAPS == kSvTapsShared && !whole;
  if (tma || ranged) __syncthreads();  // the copy's mbarrier and the range slots are initialised
  if (tma) {
    const bool landed = mbar_wait(smem_addr(s_bar), 0);
    if (!__syncthreads_and(landed)) {
      // the copy did not land in time: record it; the whole block leaves
      // without reading the region
      if (threadIdx.x == 0) atomicExch(P.err, DISK_ERR_TIMEOUT);
      return;
    }
    // Clamp-to-edge for the parts of the region outside the image, which
    // the copy filled with zeros: rows first (whole rows from the nearest
    // image row, itself inside the region), then columns within each row.
    const int y0 = ty0 - halo, x0 = tx0 - hx;
    if (y0 < 0 || y0 + RH > P.H || x0 < 0 || x0 + RW > P.W) {
      for (int e = threadIdx.x; e < RN; e += kSvThreads) {
        const int ry = e / RW, rx = e - ry * RW;
        const int gy = y0 + ry, cy = min(max(gy, 0), P.H - 1);
        if (gy != cy) {
          const int f = (cy - y0) * RW + rx;
          s_rg[e] = s_rg[f];
          if (CH == 4) s_ba[e] = s_ba[f]; else s_b[e] = s_b[f];
        }
      }
      __syncthreads();
      for (int e = threadIdx.x; e < RN; e += kSvThreads) {
        const int ry = e / RW, rx = e - ry * RW;
        const int gx = x0 + rx, cx = min(max(gx, 0), P.W - 1);
        if (gx != cx) {
          const int f = ry * RW + (cx - x0);
          s_rg[e] = s_rg[f];
          if (CH == 4) s_ba[e] = s_ba[f]; else s_b[e] = s_b[f];
        }
      }
    }
  } else {
    // Stage the source region, clamping coordinates to the image (Eq. 3
    // read with clamp-to-edge).  Each warp takes rows warp, warp + 8, ...;
    // four of its rows are loaded before any is converted and stored, so
    // four global loads per thread are in flight instead of one.
    constexpr int kStageRows = 4;
    for (int rx = lane; rx < RW; rx += 32) {
      const int gx = min(max(tx0 - hx + rx, 0), P.W - 1);
      for (int ry0 = warp; ry0 < RH; ry0 += kSvWarps * kStageRows) {
        float4 v[kStageRows];
#pragma unroll
        for (int u = 0; u < kStageRows; ++u) {
          const int ry = ry0 + u * kSvWarps;
          const int gy = min(max(ty0 - halo + ry, 0), P.H - 1);
          if (ry < RH) {
            if (SRC == PIX_PLANAR)
              v[u] = load_planar(P.src, P.src_pitch, P.src_plane_b, CH, gy, gx);
            else
              v[u] = load_px<SRC == PIX_PLANAR ? PIX_F32 : SRC>(P.src, P.src_pitch, P.C, gy, gx);
          }
        }
#pragma unroll
        for (int u = 0; u < kStageRows; ++u) {
          const int ry = ry0 + u * kSvWarps;
          if (ry < RH) {
            const int e = ry * RW + rx;
            s_rg[e] = make_float2(v[u].x, v[u].y);
            if (CH == 4) s_ba[e] = make_float2(v[u].z, v[u].w);
            else s_b[e] = v[u].z;
          }
        }
      }
    }
  }
  Cell c[kSvPix];
  CellPairs cp[kSvPix];
  RotPairs rp[kSvPix];
  int base[kSvPix];
  Acc acc[kSvPix];
  bool same = true;
#pragma unroll
  for (int j = 0; j < kSvPix; ++j) {
    c[j] = make_cell_v<DIMS>(P.ax, pv0[j], pv1[j]);
    cp[j] = cell_pairs(c[j]);
    rp[j] = {rv[j], make_float2(-rv[j].y, rv[j].x)};
    base[j] = (warp * kSvPix + j + halo) * RW + (lane + hx);
    acc[j] = {make_float2(0.f, 0.f), 0.f, 0.f};
    same = same && (c[j].n00 == c[0].n00);
  }
  // Node range of the block (lowest n00, highest n11 over its pixels); when
  // it spans at most tap_cap nodes their taps are copied into shared memory,
  // else the block reads taps from global memory.  tap_base: index of the
  // first copied tap.
  bool shared_taps = whole;
  int tap_base = 0;
  if (ranged) {
    unsigned lo = 0xffffffffu, hi = 0u;
#pragma unroll
    for (int j = 0; j < kSvPix; ++j) {
      lo = min(lo, (unsigned)c[j].n00);
      hi = max(hi, (unsigned)c[j].n11);
    }
    lo = __reduce_min_sync(0xffffffffu, lo);
    hi = __reduce_max_sync(0xffffffffu, hi);
    if (lane == 0) {
      atomicMin(&s_range[0], lo);
      atomicMax(&s_range[1], hi);
    }
    __syncthreads();
    const int nlo = (int)s_range[0], nhi = (int)s_range[1];
    shared_taps = nhi - nlo < P.tap_cap;
    if (shared_taps) {
      tap_base = nlo * T;
      const int n = (nhi - nlo + 1) * T;
      for (int i = threadIdx.x; i < n; i += kSvThreads) s_taps[i] = __ldg(P.gtaps + tap_base + i);
    }
  }
  __syncthreads();
  const Staged st{s_rg, s_b, s_ba};

  // The tap loops, once per source of node taps (the choice is uniform over
  // the block).
  auto run_taps = [&](auto fetch) {
    if (__all_sync(0xffffffffu, same)) {
      // each thread's pixels share a cell: one node fetch per tap serves them
      const int b00 = c[0].n00 * T, b10 = c[0].n10 * T, b01 = c[0].n01 * T, b11 = c[0].n11 * T;
#pragma unroll 2
      for (int i = 0; i < T; ++i) {
        const float4 q00 = fetch(b00 + i), q10 = fetch(b10 + i);
        const float4 q01 = DIMS == 2 ? fetch(b01 + i) : q00;
        const float4 q11 = DIMS == 2 ? fetch(b11 + i) : q10;
        sv_tap_column<DIMS, CH, ROT, kSvPix>(q00, q10, q01, q11, cp, rp, st, base[0], RW, acc);
      }
    } else {
      // unrolled so the per-pixel arrays stay in registers
#pragma unroll
      for (int j = 0; j < kSvPix; ++j) {
        const int b00 = c[j].n00 * T, b10 = c[j].n10 * T, b01 = c[j].n01 * T, b11 = c[j].n11 * T;
#pragma unroll 1
        for (int i = 0; i < T; ++i) {
          const float4 q00 = fetch(b00 + i), q10 = fetch(b10 + i);
          const float4 q01 = DIMS == 2 ? fetch(b01 + i) : q00;
          const float4 q11 = DIMS == 2 ? fetch(b11 + i) : q10;
          sv_tap<DIMS, CH, ROT>(q00, q10, q01, q11, cp[j], rp[j], st, base[j], RW, acc[j]);
        }
      }
    }
  };
  if (TAPS == kSvTapsShared && shared_taps) {
    const float4 *t = s_taps - tap_base;
    run_taps([&](int idx) { return t[idx]; });
  } else {
    run_taps([&](int idx) { return __ldg(P.gtaps + idx); });
  }
  if (x < P.W) {
#pragma unroll
    for (int j = 0; j < kSvPix; ++j) {
      const int y = ty0 + warp * kSvPix + j;
      if (y < P.H) {
        const float4 v = make_float4(acc[j].rg.x, acc[j].rg.y, acc[j].b, acc[j].a);
        if (DST == PIX_PLANAR)
          store_planar(P.dst, P.dst_pitch, P.dst_plane_b, CH, y, x, v);
        else
          store_px<DST == PIX_PLANAR ? PIX_F32 : DST>(P.dst, P.dst_pitch, P.C, y, x, v);
      }
    }
  }
}

// (cos, sin) of every pixel's angle, once per filter call for all layers; a
// non-finite angle acts as 0; the pair is scaled to unit length.
__global__ void rotation_kernel(const float *__restrict__ angle, float2 *__restrict__ rot,
                                long long n);

template <int DIMS, int SRC, int DST, int TAPS, int CH, int PIX, bool ROT>
int launch_sv_layer_t(const SvLayerParams &P, cudaStream_t s) {
  auto k = sv_layer_kernel<DIMS, SRC, DST, TAPS, CH, PIX, ROT>;
  constexpr int kSvTileH = PIX * kSvWarps;
  const size_t smem = sv_smem_bytes((size_t)P.region_w * (kSvTileH + 2 * P.halo), CH) +
                      (TAPS == kSvTapsShared ? (size_t)P.tap_cap * P.T * sizeof(float4) : 0);
  static unsigned long long attr_set = 0;  // per instantiation, one bit per device
  int dev = 0;
  cudaGetDevice(&dev);
  if (!(attr_set & (1ull << (dev & 63)))) {
    DISK_TRY_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kSvMaxSmem),
                  "cudaFuncSetAttribute(sv_layer)");
    attr_set |= 1ull << (dev & 63);
  }
  dim3 grid((P.W + kSvTileW - 1) / kSvTileW, (P.H + kSvTileH - 1) / kSvTileH);
  k<<<grid, kSvThreads, smem, s>>>(P);
  DISK_TRY_CUDA(cudaGetLastError(), "launch sv_layer_kernel");
  return DISK_OK;
}

// Storage combination of one layer: (source kind, destination kind), tile
// configuration pix (2 or 4 pixels per thread); TAPS where the node taps are
// read; ROT selects the rotated variant (P.rot set).
template <int DIMS, int TAPS, bool ROT>
int launch_sv_layer(int src, int dst, int C, const SvLayerParams &P, cudaStream_t s, int pix);

// How many nodes' taps a block copies into shared memory (0: the layer reads
// them from global memory).  A block needs the nodes between the lowest and
// the highest index of its pixels' cells; with smooth maps a tile spans one
// or two cells per axis, i.e. at most 2 n1 + 4 consecutive indices of a 2-D
// basis (n1 nodes on axis 1).  Small tables are copied whole.
inline int sv_tap_cap(int dims, int n1, int B, int T, size_t region_smem) {
  int cap = (size_t)B * T * sizeof(float4) <= 8192 ? B : (dims == 1 ? 8 : 2 * n1 + 4);
  cap = cap < B ? cap : B;
  return region_smem + (size_t)cap * T * sizeof(float4) <= (size_t)kSvMaxSmem ? cap : 0;
}

// One layer of any variant: dims 1 or 2, taps in shared memory or global
// (defined with the filter's host code).
int launch_layer(int dims, bool shared_taps, bool rot, int src, int dst, int C,
                 const SvLayerParams &P, cudaStream_t s, int pix);

#define DISK_SV_CASE(DIMS, TAPS, ROT, S, D)                                                 \
  if (src == S && dst == D) {                                                               \
    if (pix == 4)                                                                           \
      return c4 ? launch_sv_layer_t<DIMS, S, D, TAPS, 4, 4, ROT>(P, s)                      \
                : launch_sv_layer_t<DIMS, S, D, TAPS, 3, 4, ROT>(P, s);                     \
    return c4 ? launch_sv_layer_t<DIMS, S, D, TAPS, 4, 2, ROT>(P, s)                        \
              : launch_sv_layer_t<DIMS, S, D, TAPS, 3, 2, ROT>(P, s);                       \
  }

// FP32 images: FP32 planes; FP16 images: FP16 planes (see intermediate_kind).
#define DISK_SV_INSTANTIATE(DIMS, TAPS, ROT)                                                \
  template <>                                                                               \
  int launch_sv_layer<DIMS, TAPS, ROT>(int src, int dst, int C, const SvLayerParams &P,       \
                                       cudaStream_t s, int pix) {                           \
    const bool c4 = C == 4;                                                                 \
    DISK_SV_CASE(DIMS, TAPS, ROT, PIX_F32, PIX_RGBA32)                                        \
    DISK_SV_CASE(DIMS, TAPS, ROT, PIX_RGBA32, PIX_RGBA32)                                     \
    DISK_SV_CASE(DIMS, TAPS, ROT, PIX_RGBA32, PIX_F32)                                        \
    DISK_SV_CASE(DIMS, TAPS, ROT, PIX_F32, PIX_F32)                                           \
    DISK_SV_CASE(DIMS, TAPS, ROT, PIX_F16, PIX_RGBA16)                                        \
    DISK_SV_CASE(DIMS, TAPS, ROT, PIX_RGBA16, PIX_RGBA16)                                     \
    DISK_SV_CASE(DIMS, TAPS, ROT, PIX_RGBA16, PIX_F16)                                        \
    DISK_SV_CASE(DIMS, TAPS, ROT, PIX_F16, PIX_F16)                                           \
    DISK_SV_CASE(DIMS, TAPS, ROT, PIX_F32, PIX_PLANAR)                                        \
    DISK_SV_CASE(DIMS, TAPS, ROT, PIX_F16, PIX_PLANAR)                                        \
    DISK_SV_CASE(DIMS, TAPS, ROT, PIX_PLANAR, PIX_PLANAR)                                     \
    DISK_SV_CASE(DIMS, TAPS, ROT, PIX_PLANAR, PIX_F32)                                        \
    DISK_SV_CASE(DIMS, TAPS, ROT, PIX_PLANAR, PIX_F16)                                        \
    return fail(DISK_ERR_INVALID_ARG, "unsupported layer storage combination");            \
  }

}  // namespace disk
