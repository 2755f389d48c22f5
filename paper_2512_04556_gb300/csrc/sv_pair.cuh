// Two adjacent layers of the spatially varying cascade (Sec. 4.3 Eq. 9 +
// Sec. 3.2 Eq. 3) fused into one launch: the layer-fused form of the filter,
// applied to a pair of layers l, l + 1.
//
// Each CTA owns a 32 x 16 output tile of layer l + 1.  It stages the source
// of layer l on the tile grown by both layers' halos (h0 + h1 rows, hxs >=
// h0 + h1 columns each side, clamp-to-edge) into shared memory -- one tensor
// copy when the source is an FP32 intermediate, else through registers --
// computes layer l on the tile grown by h1 (the part of it inside the
// image; the rest replicates the nearest edge pixel, which is what layer
// l + 1's clamp-to-edge reads there), keeps that intermediate in shared
// memory, and computes layer l + 1 on the tile from it.  The intermediate
// never goes to global memory; the price is layer l's work on the grown
// region (recomputed by the neighbouring tiles).  Taps, blends and
// accumulation are those of sv_layer_kernel (sv_run_taps), FP32 throughout.
#pragma once

#include "sv_layer.cuh"

namespace disk {

constexpr int kSvPairTileH = 16;  // 32 x 16 output tiles, 2 pixels per thread

struct SvPairParams {
  // Tensor map of an FP32 source viewed as rows of 8-byte elements (use_tma).
  CUtensorMap tm;
  const void *src;
  long long src_pitch;
  void *dst;
  long long dst_pitch;
  const float *maps;
  const float4 *gtaps0;  // node taps of layer l   (layout of layer_taps)
  const float4 *gtaps1;  // node taps of layer l + 1
  int *err;              // device status word
  int H, W, C, T;
  int h0, h1;            // halos of layers l and l + 1
  int hxs;               // staged columns each side of the tile (>= h0 + h1; a multiple of 4 with TMA)
  int use_tma;
  int bt;                // B * T taps per layer
  int taps_smem;         // both layers' tables copied whole into shared memory
  AxisNodes ax[2];
};

__host__ __device__ inline size_t sv_align16(size_t b) { return (b + 15) & ~(size_t)15; }

// Shared-memory layout: source region (SW x SH pixels of C floats), layer-l
// region (MW x MH), a 16-byte mbarrier slot, then (taps_smem) both tables.
struct SvPairGeom {
  int SW, SH, MW, MH;
  size_t src_bytes, mid_bytes, taps_off, total;
};

__host__ __device__ inline SvPairGeom sv_pair_geom(int h0, int h1, int hxs, int C, int bt,
                                                   bool taps_smem) {
  SvPairGeom g;
  g.SW = kSvTileW + 2 * hxs;
  g.SH = kSvPairTileH + 2 * (h0 + h1);
  g.MW = kSvTileW + 2 * h1;
  g.MH = kSvPairTileH + 2 * h1;
  g.src_bytes = sv_align16((size_t)g.SW * g.SH * C * 4);
  g.mid_bytes = sv_align16((size_t)g.MW * g.MH * C * 4);
  g.taps_off = g.src_bytes + g.mid_bytes + 16;
  g.total = g.taps_off + (taps_smem ? (size_t)2 * bt * sizeof(float4) : 0);
  return g;
}

template <int CH>
__device__ __forceinline__ void px_put(float *s, int e, const float4 &v) {
  if (CH == 4) {
    reinterpret_cast<float4 *>(s)[e] = v;
  } else {
    s[3 * e] = v.x;
    s[3 * e + 1] = v.y;
    s[3 * e + 2] = v.z;
  }
}

template <int CH>
__device__ __forceinline__ float4 px_get(const float *s, int e) {
  if (CH == 4) return reinterpret_cast<const float4 *>(s)[e];
  return make_float4(s[3 * e], s[3 * e + 1], s[3 * e + 2], 0.f);
}

// Clamp-to-edge inside a staged region of RW x RH pixels whose in-image
// part is rows [ylo, yhi) x columns [xlo, xhi): rows outside copy the
// nearest in-image row, then columns outside copy the nearest in-image
// column of their row.  Run by the whole block; ends synchronised.
template <int CH>
__device__ void sv_clamp_region(float *s, int RW, int RH, int ylo, int yhi, int xlo, int xhi) {
  if (ylo == 0 && yhi == RH && xlo == 0 && xhi == RW) return;
  const int RN = RW * RH;
  for (int e = threadIdx.x; e < RN; e += kSvThreads) {
    const int ry = e / RW, rx = e - ry * RW;
    const int cy = min(max(ry, ylo), yhi - 1);
    if (cy != ry) px_put<CH>(s, e, px_get<CH>(s, cy * RW + rx));
  }
  __syncthreads();
  for (int e = threadIdx.x; e < RN; e += kSvThreads) {
    const int ry = e / RW, rx = e - ry * RW;
    const int cx = min(max(rx, xlo), xhi - 1);
    if (cx != rx) px_put<CH>(s, e, px_get<CH>(s, ry * RW + cx));
  }
  __syncthreads();
}

template <int DIMS, int SRC, int DST, int CH>
__global__ void __launch_bounds__(kSvThreads, 2)
sv_pair_kernel(const __grid_constant__ SvPairParams P) {
  extern __shared__ __align__(128) unsigned char sm_raw[];
  const SvPairGeom g = sv_pair_geom(P.h0, P.h1, P.hxs, CH, P.bt, P.taps_smem);
  const int h0 = P.h0, h1 = P.h1, hxs = P.hxs, SW = g.SW, SH = g.SH, MW = g.MW, MH = g.MH;
  float *s_src = reinterpret_cast<float *>(sm_raw);
  float *s_mid = reinterpret_cast<float *>(sm_raw + g.src_bytes);
  unsigned long long *s_bar = reinterpret_cast<unsigned long long *>(sm_raw + g.src_bytes + g.mid_bytes);
  float4 *s_taps = reinterpret_cast<float4 *>(sm_raw + g.taps_off);
  const int tx0 = blockIdx.x * kSvTileW, ty0 = blockIdx.y * kSvPairTileH;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int sy0 = ty0 - h0 - h1, sx0 = tx0 - hxs;  // image coordinates of source (0, 0)
  const int my0 = ty0 - h1, mx0 = tx0 - h1;        // and of the layer-l region's (0, 0)
  const bool tma = SRC == PIX_F32 && P.use_tma;
  if (tma && (smem_addr(sm_raw) & 127u) != 0) {
    if (threadIdx.x == 0) atomicExch(P.err, DISK_ERR_UNSUPPORTED);
    return;
  }
  if (tma && threadIdx.x == 0) {
    // rows [sy0, +SH) x columns [sx0, +SW) in one copy: C * SW / 2 eight-byte
    // elements per row from element C * sx0 / 2 (tx0 a multiple of 32, hxs
    // of 4: a 16-byte boundary)
    const unsigned bar = smem_addr(s_bar);
    const unsigned bytes = (unsigned)(SW * SH * CH * 4);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(bar), "r"(bytes)
                 : "memory");
    tma_load_2d(s_src, &P.tm, CH * sx0 / 2, sy0, bar);
  }
  const int T = P.T;
  if (P.taps_smem)
    for (int i = threadIdx.x; i < P.bt; i += kSvThreads) {
      s_taps[i] = __ldg(P.gtaps0 + i);
      s_taps[P.bt + i] = __ldg(P.gtaps1 + i);
    }
  if (tma) {
    __syncthreads();  // the mbarrier is initialised
    const bool landed = mbar_wait(smem_addr(s_bar), 0);
    if (!__syncthreads_and(landed)) {
      if (threadIdx.x == 0) atomicExch(P.err, DISK_ERR_TIMEOUT);
      return;
    }
    sv_clamp_region<CH>(s_src, SW, SH, max(0, -sy0), min(SH, P.H - sy0), max(0, -sx0),
                        min(SW, P.W - sx0));
  } else {
    // clamped coordinates, four rows of loads in flight per thread
    constexpr int kStageRows = 4;
    for (int rx = lane; rx < SW; rx += 32) {
      const int gx = min(max(sx0 + rx, 0), P.W - 1);
      for (int ry0 = warp; ry0 < SH; ry0 += kSvWarps * kStageRows) {
        float4 v[kStageRows];
#pragma unroll
        for (int u = 0; u < kStageRows; ++u) {
          const int ry = ry0 + u * kSvWarps;
          const int gy = min(max(sy0 + ry, 0), P.H - 1);
          if (ry < SH) v[u] = load_px<SRC>(P.src, P.src_pitch, P.C, gy, gx);
        }
#pragma unroll
        for (int u = 0; u < kStageRows; ++u) {
          const int ry = ry0 + u * kSvWarps;
          if (ry < SH) px_put<CH>(s_src, ry * SW + rx, v[u]);
        }
      }
    }
    __syncthreads();
  }
  const long long HW = (long long)P.H * P.W;

  // Layer l on the in-image part of the grown region, one pixel per thread at
  // a time; a warp's lanes take consecutive pixels and the loop's trip count
  // is uniform over the warp (lanes past the end repeat the last pixel and
  // store nothing).
  {
    const int ylo = max(0, -my0), yhi = min(MH, P.H - my0);
    const int xlo = max(0, -mx0), xhi = min(MW, P.W - mx0);
    const int nx = xhi - xlo, n = nx * (yhi - ylo);
    const float2 rv[1] = {make_float2(1.f, 0.f)};
    for (int e0 = warp * 32; e0 < n; e0 += kSvThreads) {
      const int e = min(e0 + lane, n - 1);
      const int my = ylo + e / nx, mx = xlo + e % nx;
      const long long gp = (long long)(my0 + my) * P.W + (mx0 + mx);
      const Cell c[1] = {make_cell_v<DIMS>(P.ax, __ldg(P.maps + gp),
                                           DIMS == 2 ? __ldg(P.maps + HW + gp) : 0.f)};
      const CellPairs cp[1] = {cell_pairs(c[0])};
      const int base[1] = {(my + h0) * SW + (mx + hxs - h1)};
      Acc acc[1] = {{make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)}};
      if (P.taps_smem)
        sv_run_taps<DIMS, CH, 1, false>([&](int i) { return s_taps[i]; }, T, c, cp, rv, s_src,
                                        base, SW, true, acc);
      else
        sv_run_taps<DIMS, CH, 1, false>([&](int i) { return __ldg(P.gtaps0 + i); }, T, c, cp, rv,
                                        s_src, base, SW, true, acc);
      if (e0 + lane < n) px_put<CH>(s_mid, my * MW + mx, acc_value<CH>(acc[0]));
    }
    __syncthreads();
    sv_clamp_region<CH>(s_mid, MW, MH, ylo, yhi, xlo, xhi);
  }

  // Layer l + 1 on the tile from the layer-l region, two vertically adjacent
  // pixels per thread as in sv_layer_kernel.
  const int x = tx0 + lane, xc = min(x, P.W - 1);
  Cell c[2];
  CellPairs cp[2];
  int base[2];
  Acc acc[2];
  float2 rv[2];
  bool same = true;
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const int yc = min(ty0 + warp * 2 + j, P.H - 1);
    const long long gp = (long long)yc * P.W + xc;
    c[j] = make_cell_v<DIMS>(P.ax, __ldg(P.maps + gp), DIMS == 2 ? __ldg(P.maps + HW + gp) : 0.f);
    cp[j] = cell_pairs(c[j]);
    base[j] = (warp * 2 + j + h1) * MW + (lane + h1);
    acc[j] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    rv[j] = make_float2(1.f, 0.f);
    same = same && (c[j].n00 == c[0].n00);
  }
  if (P.taps_smem) {
    const float4 *t1 = s_taps + P.bt;
    sv_run_taps<DIMS, CH, 2, false>([&](int i) { return t1[i]; }, T, c, cp, rv, s_mid, base, MW,
                                    same, acc);
  } else {
    sv_run_taps<DIMS, CH, 2, false>([&](int i) { return __ldg(P.gtaps1 + i); }, T, c, cp, rv,
                                    s_mid, base, MW, same, acc);
  }
  if (x < P.W) {
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int y = ty0 + warp * 2 + j;
      if (y < P.H) store_px<DST>(P.dst, P.dst_pitch, P.C, y, x, acc_value<CH>(acc[j]));
    }
  }
}

template <int DIMS, int SRC, int DST, int CH>
int launch_sv_pair_t(const SvPairParams &P, cudaStream_t s) {
  auto k = sv_pair_kernel<DIMS, SRC, DST, CH>;
  const SvPairGeom g = sv_pair_geom(P.h0, P.h1, P.hxs, CH, P.bt, P.taps_smem);
  static unsigned long long attr_set = 0;  // per instantiation, one bit per device
  int dev = 0;
  cudaGetDevice(&dev);
  if (!(attr_set & (1ull << (dev & 63)))) {
    DISK_TRY_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kSvMaxSmem),
                  "cudaFuncSetAttribute(sv_pair)");
    attr_set |= 1ull << (dev & 63);
  }
  dim3 grid((P.W + kSvTileW - 1) / kSvTileW, (P.H + kSvPairTileH - 1) / kSvPairTileH);
  k<<<grid, kSvThreads, g.total, s>>>(P);
  DISK_TRY_CUDA(cudaGetLastError(), "launch sv_pair_kernel");
  return DISK_OK;
}

// A fused pair of layers with storage kinds (src, dst): the caller's image or
// an FP32 intermediate in, an FP32 intermediate or the caller's image out.
template <int DIMS>
int launch_sv_pair(int src, int dst, int C, const SvPairParams &P, cudaStream_t s);

#define DISK_PAIR_CASE(DIMS, S, D)                                                          \
  if (src == S && dst == D)                                                                 \
    return c4 ? launch_sv_pair_t<DIMS, S, D, 4>(P, s) : launch_sv_pair_t<DIMS, S, D, 3>(P, s);

#define DISK_PAIR_INSTANTIATE(DIMS)                                                         \
  template <>                                                                               \
  int launch_sv_pair<DIMS>(int src, int dst, int C, const SvPairParams &P, cudaStream_t s) { \
    const bool c4 = C == 4;                                                                 \
    DISK_PAIR_CASE(DIMS, PIX_F32, PIX_F32)                                                  \
    DISK_PAIR_CASE(DIMS, PIX_F16, PIX_F32)                                                  \
    DISK_PAIR_CASE(DIMS, PIX_F32, PIX_F16)                                                  \
    DISK_PAIR_CASE(DIMS, PIX_F16, PIX_F16)                                                  \
    return fail(DISK_ERR_INVALID_ARG, "unsupported pair storage combination");             \
  }

}  // namespace disk
