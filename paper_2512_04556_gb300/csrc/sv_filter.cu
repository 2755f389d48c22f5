// Spatially varying filter with a sparse kernel complex (Sec. 4.3 Eq. 9 +
// Sec. 3.2 Eq. 3): one launch per layer.
//
// Each CTA owns a 32 x 32 output tile.  It stages the layer's source region
// (tile + the layer's halo, clamp-to-edge) into shared memory as FP32 RGBA,
// one 16-byte entry per pixel, so each bilinear corner is one 16-byte shared
// load.  Each warp then walks rows of the tile, one pixel per lane: it
// locates the pixel in kernel space (Eq. 9), and for every tap blends the
// node taps in registers, splits the offset into integer and fraction and
// accumulates the four weighted corners.  The tap table of the layer lives in
// the kernel's parameter space (constant bank) when it fits, so the mostly
// warp-uniform node reads go through the constant cache and leave the shared
// memory pipe to the corner loads.
#include <algorithm>

#include "sv_common.cuh"

namespace disk {
namespace {

constexpr int kTileW = 32, kTileH = 32, kThreads = 256;
constexpr int kParamTaps = 1792;  // 28 KB of float4, inside the 32 KB parameter limit

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

template <int DIMS, int SRC, int DST, int NP>
__global__ void __launch_bounds__(kThreads)
sv_layer_kernel(const __grid_constant__ SvLayerParams<NP> P) {
  extern __shared__ float4 sm[];
  const int halo = P.halo, RW = P.region_w, RH = kTileH + 2 * halo;
  const int tx0 = blockIdx.x * kTileW, ty0 = blockIdx.y * kTileH;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

  // Stage the source region, clamping coordinates to the image (Eq. 3 read
  // with clamp-to-edge).
  for (int ry = warp; ry < RH; ry += kThreads / 32) {
    const int gy = min(max(ty0 - halo + ry, 0), P.H - 1);
    for (int rx = lane; rx < RW; rx += 32) {
      const int gx = min(max(tx0 - halo + rx, 0), P.W - 1);
      sm[ry * RW + rx] = load_px<SRC>(P.src, P.src_pitch, P.C, gy, gx);
    }
  }
  __syncthreads();

  const int x = tx0 + lane;
  if (x >= P.W) return;
  const long long HW = (long long)P.H * P.W;
  const int T = P.T;
  for (int r = warp; r < kTileH; r += kThreads / 32) {
    const int y = ty0 + r;
    if (y >= P.H) break;
    const Cell cell = make_cell<DIMS>(P.ax, P.maps, HW, (long long)y * P.W + x);
    const int b00 = cell.n00 * T, b01 = cell.n01 * T, b10 = cell.n10 * T, b11 = cell.n11 * T;
    const float4 *base = sm + (r + halo) * RW + (lane + halo);
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 4
    for (int i = 0; i < T; ++i) {
      // Eq. 9: the pixel's tap is the alpha-weighted blend of the node taps.
      float dx, dy, w;
      {
        const float4 q00 = node_tap(P, b00 + i), q10 = node_tap(P, b10 + i);
        dx = cell.a00 * q00.x + cell.a10 * q10.x;
        dy = cell.a00 * q00.y + cell.a10 * q10.y;
        w = cell.a00 * q00.z + cell.a10 * q10.z;
        if (DIMS == 2) {
          const float4 q01 = node_tap(P, b01 + i), q11 = node_tap(P, b11 + i);
          dx += cell.a01 * q01.x + cell.a11 * q11.x;
          dy += cell.a01 * q01.y + cell.a11 * q11.y;
          w += cell.a01 * q01.z + cell.a11 * q11.z;
        }
      }
      // Eq. 2 tap at a fractional offset: bilinear from the staged region.
      // Convexity of Eq. 9 bounds every blended offset by the layer reach, so
      // nx, ny already lie in [-halo, halo - 1]; the clamp only guarantees
      // that shared memory is never read out of the staged region.
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
      acc.w += w00 * c00.w + w01 * c01.w + w10 * c10.w + w11 * c11.w;
    }
    store_px<DST>(P.dst, P.dst_pitch, P.C, y, x, acc);
  }
}

template <int DIMS, int SRC, int DST, int NP>
int launch_layer(const SvLayerParams<NP> &P, cudaStream_t s) {
  auto k = sv_layer_kernel<DIMS, SRC, DST, NP>;
  const int RH = kTileH + 2 * P.halo;
  const size_t smem = (size_t)P.region_w * RH * sizeof(float4);
  static unsigned long long attr_set = 0;  // per instantiation, one bit per device
  int dev = 0;
  cudaGetDevice(&dev);
  if (!(attr_set & (1ull << (dev & 63)))) {
    DISK_TRY_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448),
                  "cudaFuncSetAttribute(sv_layer)");
    attr_set |= 1ull << (dev & 63);
  }
  dim3 grid((P.W + kTileW - 1) / kTileW, (P.H + kTileH - 1) / kTileH);
  k<<<grid, kThreads, smem, s>>>(P);
  DISK_TRY_CUDA(cudaGetLastError(), "launch sv_layer_kernel");
  return DISK_OK;
}

template <int NP>
int dispatch_layer(int dims, int src, int dst, const SvLayerParams<NP> &P, cudaStream_t s) {
#define DISK_SV_CASE(D, S, O)                                   \
  if (dims == D && src == S && dst == O) return launch_layer<D, S, O, NP>(P, s);
#define DISK_SV_DIMS(D)                                         \
  DISK_SV_CASE(D, PIX_F32, PIX_RGBA32)                          \
  DISK_SV_CASE(D, PIX_F16, PIX_RGBA32)                          \
  DISK_SV_CASE(D, PIX_RGBA32, PIX_RGBA32)                       \
  DISK_SV_CASE(D, PIX_RGBA32, PIX_F32)                          \
  DISK_SV_CASE(D, PIX_RGBA32, PIX_F16)                          \
  DISK_SV_CASE(D, PIX_F32, PIX_F32)                             \
  DISK_SV_CASE(D, PIX_F16, PIX_F16)
  DISK_SV_DIMS(1)
  DISK_SV_DIMS(2)
#undef DISK_SV_DIMS
#undef DISK_SV_CASE
  return fail(DISK_ERR_INVALID_ARG, "unsupported layer storage combination");
}

template <int NP>
int run_filter(const disk_basis *b, const void *d_in, size_t in_pitch, void *d_out,
               size_t out_pitch, int H, int W, int C, int dtype, const float *d_maps,
               cudaStream_t s) {
  // The parameter block is large; keep it off the host stack.
  static thread_local SvLayerParams<NP> P;
  P.maps = d_maps;
  P.H = H; P.W = W; P.C = C; P.T = b->T;
  make_axes(b->dims, b->n_nodes, b->node_vals.data(), P.ax);
  const int user = dtype == DISK_F32 ? PIX_F32 : PIX_F16;
  const int L = b->L;
  float4 *bufs[2] = {nullptr, nullptr};
  const size_t plane = (size_t)H * W * sizeof(float4);
  const int nbuf = L >= 3 ? 2 : (L == 2 ? 1 : 0);
  for (int i = 0; i < nbuf; ++i) {
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&bufs[i]), plane, s);
    if (e != cudaSuccess) {
      if (i) cudaFreeAsync(bufs[0], s);
      return cuda_fail(e, "cudaMallocAsync(sv_filter scratch)");
    }
  }
  int rc = DISK_OK;
  for (int l = 0; l < L && rc == DISK_OK; ++l) {
    P.halo = halo_of(b->reach[l]);
    P.region_w = kTileW + 2 * P.halo;
    const int src = l == 0 ? user : PIX_RGBA32;
    const int dst = l == L - 1 ? user : PIX_RGBA32;
    P.src = l == 0 ? d_in : bufs[(l - 1) & 1];
    P.src_pitch = l == 0 ? (long long)in_pitch : (long long)W * sizeof(float4);
    P.dst = l == L - 1 ? d_out : bufs[l & 1];
    P.dst_pitch = l == L - 1 ? (long long)out_pitch : (long long)W * sizeof(float4);
    const float4 *layer_taps = b->d_taps + (size_t)l * b->B * b->T;
    P.gtaps = layer_taps;
    if (NP > 0) {
      // Tap table of this layer into the parameter block (host copy of the
      // same values the device copy holds).
      for (int k = 0; k < b->B; ++k)
        for (int i = 0; i < b->T; ++i) {
          const float *t = &b->theta[(((size_t)k * L + l) * b->T + i) * 3];
          P.taps[k * b->T + i] = make_float4(t[0], t[1], t[2], 0.f);
        }
    }
    rc = dispatch_layer<NP>(b->dims, src, dst, P, s);
  }
  for (int i = 0; i < nbuf; ++i) cudaFreeAsync(bufs[i], s);
  return rc;
}

}  // namespace
}  // namespace disk

using namespace disk;

extern "C" int disk_sv_filter(const disk_basis *b, const void *d_in, size_t in_pitch,
                              void *d_out, size_t out_pitch, int H, int W, int C, int dtype,
                              const float *d_maps, void *stream) {
  if (!b) return fail(DISK_ERR_INVALID_ARG, "null basis");
  int rc = validate_image_args(d_in, in_pitch, d_out, out_pitch, H, W, C, dtype, d_maps);
  if (rc) return rc;
  int dev = 0;
  DISK_TRY_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
  if (dev != b->device) return fail(DISK_ERR_INVALID_ARG, "basis lives on another device");
  for (int l = 0; l < b->L; ++l) {
    const int h = halo_of(b->reach[l]);
    const size_t smem = (size_t)(kTileW + 2 * h) * (kTileH + 2 * h) * sizeof(float4);
    if (smem > 232448) return fail(DISK_ERR_UNSUPPORTED, "layer halo exceeds shared memory");
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if ((size_t)b->B * b->T <= (size_t)kParamTaps)
    return run_filter<kParamTaps>(b, d_in, in_pitch, d_out, out_pitch, H, W, C, dtype, d_maps, s);
  return run_filter<0>(b, d_in, in_pitch, d_out, out_pitch, H, W, C, dtype, d_maps, s);
}
