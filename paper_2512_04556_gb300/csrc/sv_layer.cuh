// One layer of the spatially varying cascade (Sec. 4.3 Eq. 9 + Sec. 3.2
// Eq. 3): the kernel template shared by the 1-D and 2-D translation units.
//
// Each CTA owns a 32 x 32 output tile.  It stages the layer's source region
// (tile + the layer's halo, clamp-to-edge) into shared memory as FP32 RGBA,
// one 16-byte entry per pixel, so each bilinear corner is one 16-byte shared
// load and a warp's 32 lanes (consecutive columns) read conflict-free.
// Every thread owns four pixels of one column (rows r, r+8, r+16, r+24).
// When all pixels of a warp sit in the same kernel-space cell -- the common
// case, parameter maps being smooth -- the node taps of each tap index are
// fetched once (warp-uniform constant-bank loads) and blended for the four
// pixels with each pixel's own weights; other warps take the per-pixel path.
#pragma once

#include "sv_common.cuh"

namespace disk {

constexpr int kSvTileW = 32, kSvTileH = 32, kSvThreads = 256;
constexpr int kSvWarps = kSvThreads / 32;
constexpr int kSvPix = kSvTileH / kSvWarps;  // pixels per thread
constexpr int kSvParamTaps = 1792;           // 28 KB of float4, inside the 32 KB parameter limit
constexpr int kSvMaxSmem = 232448;           // 227 KB opt-in shared memory per CTA

template <int NP>
struct SvLayerParams {
  const void *src;
  long long src_pitch;
  void *dst;
  long long dst_pitch;
  const float *maps;
  const float4 *gtaps;  // [B][T] of this layer when NP == 0
  int H, W, C, T, halo, region_w;
  AxisNodes ax[2];
  float4 taps[NP > 0 ? NP : 1];  // [B][T] of this layer when NP > 0
};

template <int NP>
__device__ __forceinline__ float4 node_tap(const SvLayerParams<NP> &P, int idx) {
  if (NP > 0) return P.taps[idx];
  return __ldg(P.gtaps + idx);
}

// One tap of one pixel: Eq. 9 blend of the node taps with the pixel's
// weights, then the Eq. 2 bilinear sample from the staged region.
template <int DIMS, int CH>
__device__ __forceinline__ void sv_tap(const float4 &q00, const float4 &q10, const float4 &q01,
                                       const float4 &q11, const Cell &c, const float4 *base,
                                       int RW, int halo, float4 &acc) {
  float dx = c.a00 * q00.x + c.a10 * q10.x;
  float dy = c.a00 * q00.y + c.a10 * q10.y;
  float w = c.a00 * q00.z + c.a10 * q10.z;
  if (DIMS == 2) {
    dx += c.a01 * q01.x + c.a11 * q11.x;
    dy += c.a01 * q01.y + c.a11 * q11.y;
    w += c.a01 * q01.z + c.a11 * q11.z;
  }
  // Convexity of Eq. 9 bounds every blended offset by the layer reach, so
  // nx, ny already lie in [-halo, halo - 1]; the clamp only guarantees that
  // shared memory is never read outside the staged region.
  float fx, fy;
  const int nx = min(max(split_offset(dx, fx), -halo), halo - 1);
  const int ny = min(max(split_offset(dy, fy), -halo), halo - 1);
  const float4 *q = base + ny * RW + nx;
  const float4 c00 = q[0], c01 = q[1], c10 = q[RW], c11 = q[RW + 1];
  const float wy1 = w * fy, wy0 = w - wy1;
  const float w11 = wy1 * fx, w10 = wy1 - w11, w01 = wy0 * fx, w00 = wy0 - w01;
  acc.x += w00 * c00.x + w01 * c01.x + w10 * c10.x + w11 * c11.x;
  acc.y += w00 * c00.y + w01 * c01.y + w10 * c10.y + w11 * c11.y;
  acc.z += w00 * c00.z + w01 * c01.z + w10 * c10.z + w11 * c11.z;
  if (CH == 4) acc.w += w00 * c00.w + w01 * c01.w + w10 * c10.w + w11 * c11.w;
}

template <int DIMS, int SRC, int DST, int NP, int CH>
__global__ void __launch_bounds__(kSvThreads, 2)
sv_layer_kernel(const __grid_constant__ SvLayerParams<NP> P) {
  extern __shared__ float4 sm[];
  const int halo = P.halo, RW = P.region_w, RH = kSvTileH + 2 * halo;
  const int tx0 = blockIdx.x * kSvTileW, ty0 = blockIdx.y * kSvTileH;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

  // Stage the source region, clamping coordinates to the image (Eq. 3 read
  // with clamp-to-edge).
  for (int ry = warp; ry < RH; ry += kSvWarps) {
    const int gy = min(max(ty0 - halo + ry, 0), P.H - 1);
    for (int rx = lane; rx < RW; rx += 32) {
      const int gx = min(max(tx0 - halo + rx, 0), P.W - 1);
      sm[ry * RW + rx] = load_px<SRC>(P.src, P.src_pitch, P.C, gy, gx);
    }
  }
  __syncthreads();

  const int x = tx0 + lane, xc = min(x, P.W - 1);
  const long long HW = (long long)P.H * P.W;
  const int T = P.T;
  Cell c[kSvPix];
  const float4 *base[kSvPix];
  float4 acc[kSvPix];
  bool same = true;
#pragma unroll
  for (int j = 0; j < kSvPix; ++j) {
    const int r = warp + kSvWarps * j;
    const int yc = min(ty0 + r, P.H - 1);
    c[j] = make_cell<DIMS>(P.ax, P.maps, HW, (long long)yc * P.W + xc);
    base[j] = sm + (r + halo) * RW + (lane + halo);
    acc[j] = make_float4(0.f, 0.f, 0.f, 0.f);
    same = same && (c[j].n00 == c[0].n00);
  }
  if (__all_sync(0xffffffffu, same)) {
    // one node fetch per tap serves the thread's four pixels
    const int b00 = c[0].n00 * T, b10 = c[0].n10 * T, b01 = c[0].n01 * T, b11 = c[0].n11 * T;
#pragma unroll 2
    for (int i = 0; i < T; ++i) {
      const float4 q00 = node_tap(P, b00 + i), q10 = node_tap(P, b10 + i);
      const float4 q01 = DIMS == 2 ? node_tap(P, b01 + i) : q00;
      const float4 q11 = DIMS == 2 ? node_tap(P, b11 + i) : q10;
#pragma unroll
      for (int j = 0; j < kSvPix; ++j) sv_tap<DIMS, CH>(q00, q10, q01, q11, c[j], base[j], RW, halo, acc[j]);
    }
  } else {
#pragma unroll 1
    for (int j = 0; j < kSvPix; ++j) {
      const int b00 = c[j].n00 * T, b10 = c[j].n10 * T, b01 = c[j].n01 * T, b11 = c[j].n11 * T;
#pragma unroll 2
      for (int i = 0; i < T; ++i) {
        const float4 q00 = node_tap(P, b00 + i), q10 = node_tap(P, b10 + i);
        const float4 q01 = DIMS == 2 ? node_tap(P, b01 + i) : q00;
        const float4 q11 = DIMS == 2 ? node_tap(P, b11 + i) : q10;
        sv_tap<DIMS, CH>(q00, q10, q01, q11, c[j], base[j], RW, halo, acc[j]);
      }
    }
  }
  if (x < P.W) {
#pragma unroll
    for (int j = 0; j < kSvPix; ++j) {
      const int y = ty0 + warp + kSvWarps * j;
      if (y < P.H) store_px<DST>(P.dst, P.dst_pitch, P.C, y, x, acc[j]);
    }
  }
}

template <int DIMS, int SRC, int DST, int NP, int CH>
int launch_sv_layer_t(const SvLayerParams<NP> &P, cudaStream_t s) {
  auto k = sv_layer_kernel<DIMS, SRC, DST, NP, CH>;
  const size_t smem = (size_t)P.region_w * (kSvTileH + 2 * P.halo) * sizeof(float4);
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

// Storage combination of one layer: (source kind, destination kind).
template <int DIMS, int NP>
int launch_sv_layer(int src, int dst, int C, const SvLayerParams<NP> &P, cudaStream_t s);

#define DISK_SV_INSTANTIATE(DIMS, NP)                                                         \
  template <>                                                                               \
  int launch_sv_layer<DIMS, NP>(int src, int dst, int C, const SvLayerParams<NP> &P,          \
                                cudaStream_t s) {                                           \
    const bool c4 = C == 4;                                                                 \
    if (src == PIX_F32 && dst == PIX_RGBA32)                                                \
      return c4 ? launch_sv_layer_t<DIMS, PIX_F32, PIX_RGBA32, NP, 4>(P, s)                 \
                : launch_sv_layer_t<DIMS, PIX_F32, PIX_RGBA32, NP, 3>(P, s);                \
    if (src == PIX_F16 && dst == PIX_RGBA32)                                                \
      return c4 ? launch_sv_layer_t<DIMS, PIX_F16, PIX_RGBA32, NP, 4>(P, s)                 \
                : launch_sv_layer_t<DIMS, PIX_F16, PIX_RGBA32, NP, 3>(P, s);                \
    if (src == PIX_RGBA32 && dst == PIX_RGBA32)                                             \
      return c4 ? launch_sv_layer_t<DIMS, PIX_RGBA32, PIX_RGBA32, NP, 4>(P, s)              \
                : launch_sv_layer_t<DIMS, PIX_RGBA32, PIX_RGBA32, NP, 3>(P, s);             \
    if (src == PIX_RGBA32 && dst == PIX_F32)                                                \
      return c4 ? launch_sv_layer_t<DIMS, PIX_RGBA32, PIX_F32, NP, 4>(P, s)                 \
                : launch_sv_layer_t<DIMS, PIX_RGBA32, PIX_F32, NP, 3>(P, s);                \
    if (src == PIX_RGBA32 && dst == PIX_F16)                                                \
      return c4 ? launch_sv_layer_t<DIMS, PIX_RGBA32, PIX_F16, NP, 4>(P, s)                 \
                : launch_sv_layer_t<DIMS, PIX_RGBA32, PIX_F16, NP, 3>(P, s);                \
    if (src == PIX_F32 && dst == PIX_F32)                                                   \
      return c4 ? launch_sv_layer_t<DIMS, PIX_F32, PIX_F32, NP, 4>(P, s)                    \
                : launch_sv_layer_t<DIMS, PIX_F32, PIX_F32, NP, 3>(P, s);                   \
    if (src == PIX_F16 && dst == PIX_F16)                                                   \
      return c4 ? launch_sv_layer_t<DIMS, PIX_F16, PIX_F16, NP, 4>(P, s)                    \
                : launch_sv_layer_t<DIMS, PIX_F16, PIX_F16, NP, 3>(P, s);                   \
    return fail(DISK_ERR_INVALID_ARG, "unsupported layer storage combination");            \
  }

}  // namespace disk
