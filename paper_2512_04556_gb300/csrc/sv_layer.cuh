// One layer of the spatially varying cascade (Sec. 4.3 Eq. 9 + Sec. 3.2
// Eq. 3): the kernel template shared by the 1-D and 2-D translation units.
//
// Each CTA owns a 32 x 16 or 32 x 32 output tile (PIX = 2 or 4 vertically
// adjacent pixels of one column per thread; neighbouring pixels share the
// corner row between them when their integer offsets agree).  It stages the
// layer's source region (tile + the layer's halo, clamp-to-edge) into shared
// memory as FP32 pixels, C floats each, converting FP16 sources once per
// staged pixel instead of once per tap and corner; a warp's 32 lanes
// (consecutive columns) read consecutive pixels.  An FP32 intermediate
// (16-byte aligned rows) is copied in by the tensor-memory accelerator; the
// caller's image goes through registers.  The layer's node taps are copied
// into shared memory beside the region.  Arithmetic and accumulation are
// FP32.
// When each thread's pixels sit in one kernel-space cell -- the common case,
// parameter maps being smooth -- the node taps of each tap index are fetched
// once per thread (128-bit shared-memory broadcasts) and blended for its
// pixels with each pixel's own weights; warps with a thread whose pixels
// straddle cells take the per-pixel path.
// Three-channel images take the taps two at a time in packed FP32 pairs
// (lane 0: tap i, lane 1: tap i + 1), from a copy of the table that stores
// each pair's offsets and weights side by side: the blend, the floor split
// and the corner weights then need no broadcast operands, and each channel
// accumulates the even and the odd taps in the two lanes of one pair, summed
// at the end.  Four-channel images take one tap at a time with (r, g) and
// (b, a) as pairs.
// The rotated variant (ROT) turns every pixel's blended tap offsets by that
// pixel's angle before sampling: the runtime form of the rotational and
// radial blur effects of Sec. 5.3, exact for the complex's impulse response.
#pragma once

#include <cuda.h>

#include <type_traits>

#include "sv_common.cuh"

namespace disk {

// Tile configurations: 32 columns x (8 warps x PIX rows); PIX pixels per
// thread.  PIX = 2: 32 x 16 tiles, 4 CTAs per SM (64 registers); PIX = 4:
// 32 x 32 tiles, 3 CTAs per SM for four channels and 2 for three (whose tap
// pairs keep 128 registers busy); disk_sv_filter_autotune picks per layer
// and frame shape.
constexpr int kSvTileW = 32, kSvThreads = 256;
constexpr int kSvWarps = kSvThreads / 32;
constexpr int kSvDefaultPix = 2;
__host__ __device__ constexpr int sv_tile_h(int pix) { return pix * kSvWarps; }
constexpr int kSvMaxSmem = 232448;           // 227 KB opt-in shared memory per CTA

// Shared-memory bytes per staged pixel: C FP32 values.
__host__ __device__ constexpr size_t sv_stage_bytes(int C) { return (size_t)C * 4; }

// Staged region of RN pixels (C floats each, row-major, rows of region_w
// pixels), then a 16-byte slot with the tile copy's mbarrier and the block's
// node range.  The node taps follow.
__host__ __device__ constexpr size_t sv_smem_bytes(size_t RN, int C) {
  return ((RN * sv_stage_bytes(C) + 15) & ~(size_t)15) + 16;
}

// Iteration limit of the wait for a tile copy (each try_wait may also
// suspend the thread for a while); past it the kernel records
// DISK_ERR_TIMEOUT in *err and the block returns.
constexpr long long kSvMaxWaitIters = 1ll << 22;

struct SvLayerParams {
  // Tensor map of an FP32 source viewed as rows of 8-byte elements (used
  // when use_tma; the type carries the 128-byte alignment the copies
  // require).
  CUtensorMap tm;
  const void *src;
  long long src_pitch;   // bytes per row
  void *dst;
  long long dst_pitch;
  const float *maps;
  const float2 *rot;    // [H][W] (cos, sin) of each pixel's angle, rotated variant only
  // [B][T] taps of this layer: (dx, dy, w, w) per tap for 4 channels; for 3
  // channels the pair layout of sv_pair_slots (sv_layer_taps picks).
  const float4 *gtaps;
  int *err;             // device status word (DISK_ERR_TIMEOUT after a given-up wait)
  int H, W, C, T;
  int halo;             // rows staged above and below the tile
  int halo_x;           // columns staged left and right (>= halo; a multiple of 4 with TMA)
  int region_w;         // kSvTileW + 2 halo_x
  int use_tma;          // FP32 source copied by the tensor-memory accelerator
  int bt;               // B * T taps of this layer
  int tap_cap;          // nodes whose taps a block may copy into shared memory
  AxisNodes ax[2];
};

__device__ __forceinline__ unsigned smem_addr(const void *p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

// One 2-D tile of a tensor map into shared memory, completing on mbarrier
// bar (which expects the bytes beforehand).  x must be a multiple of 16
// bytes' worth of elements; out-of-range elements read as zero.  The source
// rows are viewed as 8-byte elements (no conversion: the copy moves bytes).
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

// Pixel weights of Eq. 9 broadcast into FP32 pairs for the packed (f32x2)
// arithmetic; built once per pixel.
struct CellPairs {
  float2 a00, a10, a01, a11;
};

__device__ __forceinline__ CellPairs cell_pairs(const Cell &c) {
  return {make_float2(c.a00, c.a00), make_float2(c.a10, c.a10), make_float2(c.a01, c.a01),
          make_float2(c.a11, c.a11)};
}

// Per-pixel accumulator, three FP32 pairs.  3 channels: r, g, b, each
// (even taps, odd taps); 4 channels: (r, g), (b, a) and an unused pair.
struct Acc {
  float2 p0, p1, p2;
};

template <int CH>
__device__ __forceinline__ float4 acc_value(const Acc &a) {
  if (CH == 3) return make_float4(a.p0.x + a.p0.y, a.p1.x + a.p1.y, a.p2.x + a.p2.y, 0.f);
  return make_float4(a.p0.x, a.p0.y, a.p1.x, a.p1.y);
}

__device__ __forceinline__ float2 lo2(const float4 &v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(const float4 &v) { return make_float2(v.z, v.w); }

// Floor split of an offset pair, both lanes at once: r = d + 1.5 * 2^23
// rounded toward minus infinity is exactly floor(d) + 1.5 * 2^23 (|d| < 2^22,
// where that sum's ulp is 1), so r's bit pattern minus kSvSplitBias is
// floor(d); the fraction f = d - floor(d) in [0, 1) is exact.
constexpr float kSvSplitMagic = 12582912.0f;  // 1.5 * 2^23
constexpr unsigned kSvSplitBias = 0x4B400000u; // bit pattern of kSvSplitMagic
__device__ __forceinline__ float2 sv_split_floor(const float2 &d, float2 &f) {
  const float2 r = __fadd2_rd(d, make_float2(kSvSplitMagic, kSvSplitMagic));
  f = __ffma2_rn(__fadd2_rn(r, make_float2(-kSvSplitMagic, -kSvSplitMagic)), make_float2(-1.f, -1.f), d);
  return r;
}

// A region index with the split's bias folded in: sv_biased(b, RW) +
// bits(ry) * RW + bits(rx) = b + floor(dy) * RW + floor(dx) (in wrapping
// 32-bit arithmetic; the result is a valid index).
__device__ __forceinline__ unsigned sv_biased(int base, int RW) {
  return (unsigned)base - kSvSplitBias * (unsigned)(RW + 1);
}
__device__ __forceinline__ int sv_index(unsigned biased, int RW, float rx, float ry) {
  return (int)(biased + (unsigned)__float_as_int(ry) * (unsigned)RW + (unsigned)__float_as_int(rx));
}

// Bilinear corner weights of a pair (per lane): w * (1 - fx) (1 - fy),
// w fx (1 - fy), w (1 - fx) fy, w fx fy.
struct CornerW {
  float2 w00, w01, w10, w11;
};
__device__ __forceinline__ CornerW corner_weights(const float2 &w, const float2 &fx, const float2 &fy) {
  const float2 m1 = make_float2(-1.f, -1.f);
  CornerW c;
  const float2 wy1 = __fmul2_rn(w, fy), wy0 = __ffma2_rn(wy1, m1, w);
  c.w11 = __fmul2_rn(wy1, fx);
  c.w10 = __ffma2_rn(c.w11, m1, wy1);
  c.w01 = __fmul2_rn(wy0, fx);
  c.w00 = __ffma2_rn(c.w01, m1, wy0);
  return c;
}

// In bounds by construction: the Eq. 9 weights are non-negative and sum to
// one within a few ulp (t is clamped to [0, 1] and p to the node range, NaN
// to the first node), and every node tap satisfies |o| <= R, the layer
// reach; so a blended |d| <= R (1 + 2^-21) and n = floor(d) lies in
// [-ceil(R) - 1, ceil(R)] = [-halo, halo - 1], which with the corner n + 1
// keeps every read inside the staged tile + halo region.  The rotated variant
// takes R as the largest Euclidean tap length (the norm of a convex blend is
// at most the largest node norm) and reads (cos, sin) normalised to unit
// length by rotation_kernel, so each rotated component is within
// R (1 + 2^-20): the same argument holds.

// v + the four weighted corners, in the order top left, top right, bottom
// left, bottom right.
__device__ __forceinline__ float2 corners_into(float2 v, const CornerW &cw, const float2 &tl,
                                               const float2 &tr, const float2 &bl, const float2 &br) {
  v = __ffma2_rn(cw.w00, tl, v);
  v = __ffma2_rn(cw.w01, tr, v);
  v = __ffma2_rn(cw.w10, bl, v);
  return __ffma2_rn(cw.w11, br, v);
}

// The pair layout of a node's T taps (3-channel images): for each
// j < T / 2, slot 2j holds (dx_2j, dx_2j+1, dy_2j, dy_2j+1) and slot 2j + 1
// holds (w_2j, w_2j+1) of the node and then of its successor on axis 0
// (node index + n1, or the node itself on the last row), so that one 16-byte
// fetch from a cell's n00 (n01) gives the weights of n00 and n10 (n01 and
// n11); an odd T's last slot holds its last tap as (dx, dy, w, w).

// Eq. 9 blend of a tap pair's (dx, dy, w) for one pixel: lane 0 tap 2j,
// lane 1 tap 2j + 1.
template <int DIMS>
__device__ __forceinline__ void blend_pair(const float4 (&A)[4], const float2 (&Wt)[4],
                                           const CellPairs &a, float2 &dx, float2 &dy, float2 &w) {
  dx = __fmul2_rn(a.a00, lo2(A[0]));
  dy = __fmul2_rn(a.a00, hi2(A[0]));
  w = __fmul2_rn(a.a00, Wt[0]);
  dx = __ffma2_rn(a.a10, lo2(A[1]), dx);
  dy = __ffma2_rn(a.a10, hi2(A[1]), dy);
  w = __ffma2_rn(a.a10, Wt[1], w);
  if (DIMS == 2) {
    dx = __ffma2_rn(a.a01, lo2(A[2]), dx);
    dy = __ffma2_rn(a.a01, hi2(A[2]), dy);
    w = __ffma2_rn(a.a01, Wt[2], w);
    dx = __ffma2_rn(a.a11, lo2(A[3]), dx);
    dy = __ffma2_rn(a.a11, hi2(A[3]), dy);
    w = __ffma2_rn(a.a11, Wt[3], w);
  }
}

// (dx, dy) -> (dx cos - dy sin, dx sin + dy cos) for both lanes; rv =
// (cos, sin) of the pixel.
__device__ __forceinline__ void rotate_pair(const float2 &rv, float2 &dx, float2 &dy) {
  const float2 c = make_float2(rv.x, rv.x), sn = make_float2(rv.y, rv.y);
  const float2 x = __ffma2_rn(dx, c, __fmul2_rn(dy, make_float2(-rv.y, -rv.y)));
  dy = __ffma2_rn(dx, sn, __fmul2_rn(dy, c));
  dx = x;
}

// A tap pair for the thread's N vertically adjacent pixels, top to bottom (3
// channels; px: staged region, 3 floats per pixel).  Neighbouring pixels'
// sample points usually have the same integer offset (the offsets vary
// slowly across pixels), and then a pixel's top corners are the previous
// pixel's bottom corners: they are kept in registers, per lane, instead of
// being read from shared memory again.  Per channel the pair accumulates
// corner by corner: top left, top right, bottom left, bottom right.
template <int DIMS, bool ROT, int N>
__device__ __forceinline__ void sv_pair_column(const float4 (&A)[4], const float2 (&Wt)[4],
                                               const CellPairs *cp, const float2 *rv,
                                               const float *px, int base0, int RW, Acc *acc) {
  const unsigned biased0 = sv_biased(base0, RW);
  int ep0 = 0, ep1 = 0;
  // previous pixel's bottom row: channel k of the left (l) and right (r)
  // corners, lanes (tap 2j, tap 2j + 1)
  float2 bl[3], br[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) bl[k] = br[k] = make_float2(0.f, 0.f);
#pragma unroll
  for (int p = 0; p < N; ++p) {
    float2 dx, dy, w;
    blend_pair<DIMS>(A, Wt, cp[p], dx, dy, w);
    if (ROT) rotate_pair(rv[p], dx, dy);
    float2 fx, fy;
    const float2 sx = sv_split_floor(dx, fx), sy = sv_split_floor(dy, fy);
    const unsigned bp = biased0 + (unsigned)(p * RW);
    const int e0 = sv_index(bp, RW, sx.x, sy.x), e1 = sv_index(bp, RW, sx.y, sy.y);
    const CornerW cw = corner_weights(w, fx, fy);
    const float *q0 = px + 3 * e0, *q1 = px + 3 * e1;
    float2 tl[3], tr[3];
    if (p > 0 && e0 == ep0 + RW) {
#pragma unroll
      for (int k = 0; k < 3; ++k) { tl[k].x = bl[k].x; tr[k].x = br[k].x; }
    } else {
#pragma unroll
      for (int k = 0; k < 3; ++k) { tl[k].x = q0[k]; tr[k].x = q0[3 + k]; }
    }
    if (p > 0 && e1 == ep1 + RW) {
#pragma unroll
      for (int k = 0; k < 3; ++k) { tl[k].y = bl[k].y; tr[k].y = br[k].y; }
    } else {
#pragma unroll
      for (int k = 0; k < 3; ++k) { tl[k].y = q1[k]; tr[k].y = q1[3 + k]; }
    }
    const float *u0 = q0 + 3 * RW, *u1 = q1 + 3 * RW;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      bl[k] = make_float2(u0[k], u1[k]);
      br[k] = make_float2(u0[3 + k], u1[3 + k]);
    }
    ep0 = e0;
    ep1 = e1;
    Acc &ac = acc[p];
    ac.p0 = corners_into(ac.p0, cw, tl[0], tr[0], bl[0], br[0]);
    ac.p1 = corners_into(ac.p1, cw, tl[1], tr[1], bl[1], br[1]);
    ac.p2 = corners_into(ac.p2, cw, tl[2], tr[2], bl[2], br[2]);
  }
}

// One tap (dx, dy, w, w blended from the four node taps q) for one pixel:
// the last tap of an odd T for 3 channels (added to lane 0 of each channel
// pair), or any tap for 4 channels ((r, g) and (b, a) pairs, px holding 4
// floats per pixel).  Corner order as in sv_pair_column.
template <int DIMS, int CH, bool ROT>
__device__ __forceinline__ void sv_tap(const float4 &q00, const float4 &q10, const float4 &q01,
                                       const float4 &q11, const CellPairs &a, const float2 &rv,
                                       const float *px, int base, int RW, Acc &acc) {
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
  if (ROT)
    d = __ffma2_rn(make_float2(d.x, d.x), rv, __fmul2_rn(make_float2(d.y, d.y), make_float2(-rv.y, rv.x)));
  float2 f;
  const float2 r = sv_split_floor(d, f);
  const int e = sv_index(sv_biased(base, RW), RW, r.x, r.y);
  const CornerW cw = corner_weights(w, make_float2(f.x, f.x), make_float2(f.y, f.y));
  const float2 wc[4] = {cw.w00, cw.w01, cw.w10, cw.w11};
  const int ec[4] = {e, e + 1, e + RW, e + RW + 1};
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    if (CH == 4) {
      const float4 v = reinterpret_cast<const float4 *>(px)[ec[c]];
      acc.p0 = __ffma2_rn(wc[c], lo2(v), acc.p0);
      acc.p1 = __ffma2_rn(wc[c], hi2(v), acc.p1);
    } else {
      const float *v = px + 3 * ec[c];
      acc.p0.x = fmaf(wc[c].x, v[0], acc.p0.x);
      acc.p1.x = fmaf(wc[c].x, v[1], acc.p1.x);
      acc.p2.x = fmaf(wc[c].x, v[2], acc.p2.x);
    }
  }
}

// One tap for the thread's N vertically adjacent pixels (4 channels), with
// the top-row reuse of sv_pair_column.
template <int DIMS, bool ROT, int N>
__device__ __forceinline__ void sv_tap_column4(const float4 &q00, const float4 &q10,
                                               const float4 &q01, const float4 &q11,
                                               const CellPairs *cp, const float2 *rv,
                                               const float *px, int base0, int RW, Acc *acc) {
  const float4 *pv = reinterpret_cast<const float4 *>(px);
  const unsigned biased0 = sv_biased(base0, RW);
  int eprev = 0;
  float4 bl = make_float4(0.f, 0.f, 0.f, 0.f), br = bl;
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
    if (ROT)
      d = __ffma2_rn(make_float2(d.x, d.x), rv[p],
                     __fmul2_rn(make_float2(d.y, d.y), make_float2(-rv[p].y, rv[p].x)));
    float2 f;
    const float2 r = sv_split_floor(d, f);
    const int e = sv_index(biased0 + (unsigned)(p * RW), RW, r.x, r.y);
    const CornerW cw = corner_weights(w, make_float2(f.x, f.x), make_float2(f.y, f.y));
    float4 tl, tr;
    if (p > 0 && e == eprev + RW) {
      tl = bl; tr = br;
    } else {
      tl = pv[e]; tr = pv[e + 1];
    }
    bl = pv[e + RW];
    br = pv[e + RW + 1];
    eprev = e;
    Acc &ac = acc[p];
    ac.p0 = __ffma2_rn(cw.w00, lo2(tl), ac.p0);
    ac.p1 = __ffma2_rn(cw.w00, hi2(tl), ac.p1);
    ac.p0 = __ffma2_rn(cw.w01, lo2(tr), ac.p0);
    ac.p1 = __ffma2_rn(cw.w01, hi2(tr), ac.p1);
    ac.p0 = __ffma2_rn(cw.w10, lo2(bl), ac.p0);
    ac.p1 = __ffma2_rn(cw.w10, hi2(bl), ac.p1);
    ac.p0 = __ffma2_rn(cw.w11, lo2(br), ac.p0);
    ac.p1 = __ffma2_rn(cw.w11, hi2(br), ac.p1);
  }
}

// The tap loops of one thread's PIX vertically adjacent pixels of one column
// (cells c, their weights cp, rotations rv, region indexes base; px: the
// staged region, rows of RW pixels): every tap of the layer, blended per
// pixel from the node taps, accumulated into acc.  fetch(i): slot i of the
// layer's node-tap table as a float4; same: the thread's pixels share a cell.
template <int DIMS, int CH, int PIX, bool ROT, class Fetch>
__device__ __forceinline__ void sv_run_taps(Fetch fetch, int T, const Cell (&c)[PIX],
                                            const CellPairs (&cp)[PIX], const float2 (&rv)[PIX],
                                            const float *px, const int (&base)[PIX], int RW,
                                            bool same, Acc (&acc)[PIX]) {
  constexpr int kSvPix = PIX;
  const int TP = CH == 3 ? (T & ~1) : 0;  // taps taken in pairs
  // the taps of one pixel group (one cell) from node slot bases b[4]
  auto pairs = [&](const int (&b)[4], auto column) {
#pragma unroll 1
    for (int i = 0; i < TP; i += 2) {
      float4 A[4];
      float2 Wt[4];
      A[0] = fetch(b[0] + i);
      A[1] = fetch(b[1] + i);
      // a weight slot holds the pair of its node and of the node next on
      // axis 0: n10 of an n00, n11 of an n01
      const float4 w0 = fetch(b[0] + i + 1);
      Wt[0] = lo2(w0);
      Wt[1] = hi2(w0);
      if (DIMS == 2) {
        A[2] = fetch(b[2] + i);
        A[3] = fetch(b[3] + i);
        const float4 w1 = fetch(b[2] + i + 1);
        Wt[2] = lo2(w1);
        Wt[3] = hi2(w1);
      } else {
        A[2] = A[0]; A[3] = A[1]; Wt[2] = Wt[0]; Wt[3] = Wt[1];
      }
      column(A, Wt);
    }
  };
  if (__all_sync(0xffffffffu, same)) {
    // each thread's pixels share a cell: one node fetch per tap serves them
    const int b[4] = {c[0].n00 * T, c[0].n10 * T, c[0].n01 * T, c[0].n11 * T};
    if (CH == 3) {
      pairs(b, [&](const float4 (&A)[4], const float2 (&Wt)[4]) {
        sv_pair_column<DIMS, ROT, kSvPix>(A, Wt, cp, rv, px, base[0], RW, acc);
      });
    }
#pragma unroll 2
    for (int i = TP; i < T; ++i) {
      const float4 q00 = fetch(b[0] + i), q10 = fetch(b[1] + i);
      const float4 q01 = DIMS == 2 ? fetch(b[2] + i) : q00;
      const float4 q11 = DIMS == 2 ? fetch(b[3] + i) : q10;
      if (CH == 4) {
        sv_tap_column4<DIMS, ROT, kSvPix>(q00, q10, q01, q11, cp, rv, px, base[0], RW, acc);
      } else {
#pragma unroll
        for (int j = 0; j < kSvPix; ++j)
          sv_tap<DIMS, CH, ROT>(q00, q10, q01, q11, cp[j], rv[j], px, base[j], RW, acc[j]);
      }
    }
  } else {
    // unrolled so the per-pixel arrays stay in registers
#pragma unroll
    for (int j = 0; j < kSvPix; ++j) {
      const int b[4] = {c[j].n00 * T, c[j].n10 * T, c[j].n01 * T, c[j].n11 * T};
      if (CH == 3) {
        pairs(b, [&](const float4 (&A)[4], const float2 (&Wt)[4]) {
          sv_pair_column<DIMS, ROT, 1>(A, Wt, &cp[j], &rv[j], px, base[j], RW, &acc[j]);
        });
      }
#pragma unroll 1
      for (int i = TP; i < T; ++i) {
        const float4 q00 = fetch(b[0] + i), q10 = fetch(b[1] + i);
        const float4 q01 = DIMS == 2 ? fetch(b[2] + i) : q00;
        const float4 q11 = DIMS == 2 ? fetch(b[3] + i) : q10;
        sv_tap<DIMS, CH, ROT>(q00, q10, q01, q11, cp[j], rv[j], px, base[j], RW, acc[j]);
      }
    }
  }
}

template <int DIMS, int SRC, int DST, int CH, int PIX, bool ROT>
__global__ void __launch_bounds__(kSvThreads, PIX == 2 ? 4 : (CH == 3 ? 2 : 3))
sv_layer_kernel(const __grid_constant__ SvLayerParams P) {
  constexpr int kSvPix = PIX, kSvTileH = PIX * kSvWarps;
  extern __shared__ __align__(128) unsigned char sm_raw[];
  const int halo = P.halo, hx = P.halo_x, RW = P.region_w, RH = kSvTileH + 2 * halo, RN = RW * RH;
  float *s_px = reinterpret_cast<float *>(sm_raw);
  unsigned long long *s_bar = reinterpret_cast<unsigned long long *>(
      sm_raw + sv_smem_bytes(RN, CH) - 16);
  // The node taps the block needs, copied into shared memory after the
  // block's node range is known (see below); a warp's threads mostly fetch
  // the same tap, a broadcast.
  float4 *s_taps = reinterpret_cast<float4 *>(sm_raw + sv_smem_bytes(RN, CH));
  unsigned *s_range = reinterpret_cast<unsigned *>(s_bar + 1);  // lowest, highest node
  const int tx0 = blockIdx.x * kSvTileW, ty0 = blockIdx.y * kSvTileH;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // The tensor copy needs a 128-byte aligned destination; a block whose
  // shared window is not (never seen) records an error and does nothing.
  const bool tma = SRC == PIX_F32 && P.use_tma;
  if (tma && (smem_addr(sm_raw) & 127u) != 0) {
    if (threadIdx.x == 0) atomicExch(P.err, DISK_ERR_UNSUPPORTED);
    return;
  }
  if (threadIdx.x == 0) {
    s_range[0] = 0xffffffffu;
    s_range[1] = 0u;
  }
  if (tma && threadIdx.x == 0) {
    // The region [ty0 - halo, +RH) x [tx0 - hx, +RW) in one copy: rows of
    // C * RW floats = C * RW / 2 eight-byte elements starting at element
    // C (tx0 - hx) / 2; tx0 is a multiple of 32 and hx of 4, so the start
    // is on a 16-byte boundary as the copy requires.
    const unsigned bar = smem_addr(s_bar);
    const unsigned bytes = (unsigned)RN * (unsigned)sv_stage_bytes(CH);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(bar), "r"(bytes)
                 : "memory");
    tma_load_2d(s_px, &P.tm, CH * (tx0 - hx) / 2, ty0 - halo, bar);
  }

  const int x = tx0 + lane, xc = min(x, P.W - 1);
  const long long HW = (long long)P.H * P.W;
  const int T = P.T;
  // A table small enough for every block to hold whole is copied now,
  // overlapping the tile copy; larger ones are copied per node range below.
  const bool whole = P.tap_cap * T >= P.bt;
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
  const bool ranged = !whole;
  if (tma || ranged) __syncthreads();  // the copy's mbarrier and the range slots are initialised
  // one staged pixel: C floats at s_px + C e
  auto put = [&](int e, const float4 &v) {
    if (CH == 4) {
      reinterpret_cast<float4 *>(s_px)[e] = v;
    } else {
      s_px[3 * e] = v.x;
      s_px[3 * e + 1] = v.y;
      s_px[3 * e + 2] = v.z;
    }
  };
  auto get = [&](int e) -> float4 {
    if (CH == 4) return reinterpret_cast<const float4 *>(s_px)[e];
    return make_float4(s_px[3 * e], s_px[3 * e + 1], s_px[3 * e + 2], 0.f);
  };
  if (tma) {
    const bool landed = mbar_wait(smem_addr(s_bar), 0);
    if (!__syncthreads_and(landed)) {
      // the copy did not land in time: record it; the whole block leaves
      // without reading the region
      if (threadIdx.x == 0) atomicExch(P.err, DISK_ERR_TIMEOUT);
      return;
    }
    // Clamp-to-edge for the parts of the region outside the image, which
    // the copy filled with zeros (or, right of the last column, with the
    // row's padding): rows first (whole rows from the nearest image row,
    // itself inside the region), then columns within each row.
    const int y0 = ty0 - halo, x0 = tx0 - hx;
    if (y0 < 0 || y0 + RH > P.H || x0 < 0 || x0 + RW > P.W) {
      for (int e = threadIdx.x; e < RN; e += kSvThreads) {
        const int ry = e / RW, rx = e - ry * RW;
        const int gy = y0 + ry, cy = min(max(gy, 0), P.H - 1);
        if (gy != cy) put(e, get((cy - y0) * RW + rx));
      }
      __syncthreads();
      for (int e = threadIdx.x; e < RN; e += kSvThreads) {
        const int ry = e / RW, rx = e - ry * RW;
        const int gx = x0 + rx, cx = min(max(gx, 0), P.W - 1);
        if (gx != cx) put(e, get(ry * RW + (cx - x0)));
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
          if (ry < RH) v[u] = load_px<SRC>(P.src, P.src_pitch, P.C, gy, gx);
        }
#pragma unroll
        for (int u = 0; u < kStageRows; ++u) {
          const int ry = ry0 + u * kSvWarps;
          if (ry < RH) put(ry * RW + rx, v[u]);
        }
      }
    }
  }
  Cell c[kSvPix];
  CellPairs cp[kSvPix];
  int base[kSvPix];
  Acc acc[kSvPix];
  bool same = true;
#pragma unroll
  for (int j = 0; j < kSvPix; ++j) {
    c[j] = make_cell_v<DIMS>(P.ax, pv0[j], pv1[j]);
    cp[j] = cell_pairs(c[j]);
    base[j] = (warp * kSvPix + j + halo) * RW + (lane + hx);
    acc[j] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
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
  const float *px = s_px;

  // The tap loops, once per source of node taps (the choice is uniform over
  // the block).
  if (shared_taps) {
    const float4 *t = s_taps - tap_base;
    sv_run_taps<DIMS, CH, kSvPix, ROT>([&](int idx) { return t[idx]; }, T, c, cp, rv, px, base,
                                       RW, same, acc);
  } else {
    sv_run_taps<DIMS, CH, kSvPix, ROT>([&](int idx) { return __ldg(P.gtaps + idx); }, T, c, cp,
                                       rv, px, base, RW, same, acc);
  }
  if (x < P.W) {
#pragma unroll
    for (int j = 0; j < kSvPix; ++j) {
      const int y = ty0 + warp * kSvPix + j;
      if (y < P.H) store_px<DST>(P.dst, P.dst_pitch, P.C, y, x, acc_value<CH>(acc[j]));
    }
  }
}

// (cos, sin) of every pixel's angle, once per filter call for all layers; a
// non-finite angle acts as 0; the pair is scaled to unit length.
__global__ void rotation_kernel(const float *__restrict__ angle, float2 *__restrict__ rot,
                                long long n);

template <int DIMS, int SRC, int DST, int CH, int PIX, bool ROT>
int launch_sv_layer_t(const SvLayerParams &P, cudaStream_t s) {
  auto k = sv_layer_kernel<DIMS, SRC, DST, CH, PIX, ROT>;
  constexpr int kSvTileH = PIX * kSvWarps;
  const size_t smem = sv_smem_bytes((size_t)P.region_w * (kSvTileH + 2 * P.halo), CH) +
                      (size_t)P.tap_cap * P.T * sizeof(float4);
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
// configuration pix (2 or 4 pixels per thread); ROT selects the rotated
// variant (P.rot set).
template <int DIMS, bool ROT>
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

// One layer of any variant: dims 1 or 2, rotated or not; the node taps come
// from shared memory when P.tap_cap allows, else from global memory (defined
// with the filter's host code).
int launch_layer(int dims, bool rot, int src, int dst, int C, const SvLayerParams &P,
                 cudaStream_t s, int pix);

#define DISK_SV_CASE(DIMS, ROT, S, D)                                                       \
  if (src == S && dst == D) {                                                               \
    if (pix == 4)                                                                           \
      return c4 ? launch_sv_layer_t<DIMS, S, D, 4, 4, ROT>(P, s)                            \
                : launch_sv_layer_t<DIMS, S, D, 3, 4, ROT>(P, s);                           \
    return c4 ? launch_sv_layer_t<DIMS, S, D, 4, 2, ROT>(P, s)                              \
              : launch_sv_layer_t<DIMS, S, D, 3, 2, ROT>(P, s);                             \
  }

// Storage combinations: the caller's FP32 or FP16 image in, FP32
// intermediates between layers (sv_filter), FP32 / FP16 RGBA intermediates
// (image adjoint's recomputation, no-allocation filter), the caller's
// image out.
#define DISK_SV_INSTANTIATE(DIMS, ROT)                                                      \
  template <>                                                                               \
  int launch_sv_layer<DIMS, ROT>(int src, int dst, int C, const SvLayerParams &P,           \
                                 cudaStream_t s, int pix) {                                 \
    const bool c4 = C == 4;                                                                 \
    DISK_SV_CASE(DIMS, ROT, PIX_F32, PIX_RGBA32)                                            \
    DISK_SV_CASE(DIMS, ROT, PIX_RGBA32, PIX_RGBA32)                                         \
    DISK_SV_CASE(DIMS, ROT, PIX_RGBA32, PIX_F32)                                            \
    DISK_SV_CASE(DIMS, ROT, PIX_F32, PIX_F32)                                               \
    DISK_SV_CASE(DIMS, ROT, PIX_F16, PIX_RGBA16)                                            \
    DISK_SV_CASE(DIMS, ROT, PIX_RGBA16, PIX_RGBA16)                                         \
    DISK_SV_CASE(DIMS, ROT, PIX_RGBA16, PIX_F16)                                            \
    DISK_SV_CASE(DIMS, ROT, PIX_F16, PIX_F16)                                               \
    DISK_SV_CASE(DIMS, ROT, PIX_F16, PIX_F32)                                               \
    DISK_SV_CASE(DIMS, ROT, PIX_F32, PIX_F16)                                               \
    return fail(DISK_ERR_INVALID_ARG, "unsupported layer storage combination");            \
  }

}  // namespace disk
