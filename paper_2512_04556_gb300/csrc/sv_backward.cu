// Gradient of the spatially varying cascade with respect to its input image
// (the transpose of Sec. 3.2 Eq. 3 with the Sec. 4.3 Eq. 9 per-pixel
// complex): grad_in = A_1^T ... A_L^T grad_out.
//
// The filter is linear in the image, so no activation is needed -- only the
// per-pixel taps, recomputed from the maps exactly as the forward pass does.
// Each layer's transpose is a scatter (the taps belong to the output pixel):
// a CTA owns a 32 x 32 tile of output pixels x, zeroes a shared-memory
// accumulator covering the tile plus the layer halo, and for every tap adds
// w * beta_c * g[x] to the four corners x + n + c (coordinates clamped to the
// image, which is the transpose of the clamp-to-edge read).  The region is
// then added into the layer's FP32 RGBA gradient plane with vector global
// atomics (neighbouring tiles' regions overlap).  Summation order, and so the
// last bits, vary from run to run.
#include "sv_common.cuh"

namespace disk {
namespace {

constexpr int kBwTileW = 32, kBwTileH = 32, kBwThreads = 256;
constexpr int kBwWarps = kBwThreads / 32;
constexpr int kBwPix = kBwTileH / kBwWarps;
constexpr int kBwMaxSmem = 232448;

struct BwParams {
  const void *gsrc;     // gradient of this layer's output
  long long gsrc_pitch;
  float4 *gdst;         // gradient of this layer's input: FP32 RGBA plane, pre-zeroed
  const float *maps;
  const float4 *taps;   // [B][T] of this layer: (dx, dy, w, w)
  int H, W, C, T, halo, region_w;
  AxisNodes ax[2];
};

template <int DIMS, int GKIND, int CH>
__global__ void __launch_bounds__(kBwThreads)
sv_adjoint_layer_kernel(const __grid_constant__ BwParams P) {
  extern __shared__ float4 acc[];
  const int halo = P.halo, RW = P.region_w, RH = kBwTileH + 2 * halo;
  const int tx0 = blockIdx.x * kBwTileW, ty0 = blockIdx.y * kBwTileH;
  const int ox = tx0 - halo, oy = ty0 - halo;  // image coordinates of region (0, 0)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int j = threadIdx.x; j < RW * RH; j += kBwThreads) acc[j] = make_float4(0.f, 0.f, 0.f, 0.f);
  __syncthreads();

  // Tiles whose region crosses the image border clamp every corner; the
  // others cannot reach outside the image.
  const bool border = ox < 0 || oy < 0 || ox + RW > P.W || oy + RH > P.H;
  const int x = tx0 + lane;
  const long long HW = (long long)P.H * P.W;
  const int T = P.T;
  if (x < P.W) {
    for (int j = 0; j < kBwPix; ++j) {
      const int y = ty0 + warp + kBwWarps * j;
      if (y >= P.H) break;
      const float4 g = load_px<GKIND>(P.gsrc, P.gsrc_pitch, P.C, y, x);
      const Cell c = make_cell<DIMS>(P.ax, P.maps, HW, (long long)y * P.W + x);
      for (int i = 0; i < T; ++i) {
        const float4 q00 = __ldg(P.taps + c.n00 * T + i), q10 = __ldg(P.taps + c.n10 * T + i);
        float dx = c.a00 * q00.x + c.a10 * q10.x;
        float dy = c.a00 * q00.y + c.a10 * q10.y;
        float w = c.a00 * q00.z + c.a10 * q10.z;
        if (DIMS == 2) {
          const float4 q01 = __ldg(P.taps + c.n01 * T + i), q11 = __ldg(P.taps + c.n11 * T + i);
          dx += c.a01 * q01.x + c.a11 * q11.x;
          dy += c.a01 * q01.y + c.a11 * q11.y;
          w += c.a01 * q01.z + c.a11 * q11.z;
        }
        float fx, fy;
        const int nx = min(max(split_offset(dx, fx), -halo), halo - 1);
        const int ny = min(max(split_offset(dy, fy), -halo), halo - 1);
        const float wy1 = w * fy, wy0 = w - wy1;
        const float w11 = wy1 * fx, w10 = wy1 - w11, w01 = wy0 * fx, w00 = wy0 - w01;
        int lx0 = x + nx, lx1 = lx0 + 1, ly0 = y + ny, ly1 = ly0 + 1;
        if (border) {
          lx0 = min(max(lx0, 0), P.W - 1); lx1 = min(max(lx1, 0), P.W - 1);
          ly0 = min(max(ly0, 0), P.H - 1); ly1 = min(max(ly1, 0), P.H - 1);
        }
        lx0 -= ox; lx1 -= ox; ly0 -= oy; ly1 -= oy;
        float *c00 = &acc[ly0 * RW + lx0].x, *c01 = &acc[ly0 * RW + lx1].x;
        float *c10 = &acc[ly1 * RW + lx0].x, *c11 = &acc[ly1 * RW + lx1].x;
        atomicAdd(c00, w00 * g.x); atomicAdd(c00 + 1, w00 * g.y); atomicAdd(c00 + 2, w00 * g.z);
        atomicAdd(c01, w01 * g.x); atomicAdd(c01 + 1, w01 * g.y); atomicAdd(c01 + 2, w01 * g.z);
        atomicAdd(c10, w10 * g.x); atomicAdd(c10 + 1, w10 * g.y); atomicAdd(c10 + 2, w10 * g.z);
        atomicAdd(c11, w11 * g.x); atomicAdd(c11 + 1, w11 * g.y); atomicAdd(c11 + 2, w11 * g.z);
        if (CH == 4) {
          atomicAdd(c00 + 3, w00 * g.w); atomicAdd(c01 + 3, w01 * g.w);
          atomicAdd(c10 + 3, w10 * g.w); atomicAdd(c11 + 3, w11 * g.w);
        }
      }
    }
  }
  __syncthreads();
  // add the region into the plane (only image pixels: clamped corners landed inside)
  for (int ry = warp; ry < RH; ry += kBwWarps) {
    const int gy = oy + ry;
    if (gy < 0 || gy >= P.H) continue;
    for (int rx = lane; rx < RW; rx += 32) {
      const int gx = ox + rx;
      if (gx < 0 || gx >= P.W) continue;
      const float4 v = acc[ry * RW + rx];
      if (v.x != 0.f || v.y != 0.f || v.z != 0.f || v.w != 0.f)
        atomicAdd(P.gdst + (long long)gy * P.W + gx, v);
    }
  }
}

// FP32 RGBA plane -> caller's FP32 image with C channels.
__global__ void rgba_to_user_kernel(const float4 *src, float *dst, long long pitch, int H, int W,
                                    int C) {
  const long long n = (long long)H * W;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x) {
    const int y = (int)(p / W), x = (int)(p % W);
    const float4 v = src[p];
    float *o = reinterpret_cast<float *>(reinterpret_cast<char *>(dst) + y * pitch) + (long long)x * C;
    o[0] = v.x; o[1] = v.y; o[2] = v.z;
    if (C == 4) o[3] = v.w;
  }
}

template <int DIMS, int GKIND, int CH>
int launch_adjoint(const BwParams &P, cudaStream_t s) {
  auto k = sv_adjoint_layer_kernel<DIMS, GKIND, CH>;
  static unsigned long long attr_set = 0;
  int dev = 0;
  cudaGetDevice(&dev);
  if (!(attr_set & (1ull << (dev & 63)))) {
    DISK_TRY_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kBwMaxSmem),
                  "cudaFuncSetAttribute(sv_adjoint)");
    attr_set |= 1ull << (dev & 63);
  }
  const size_t smem = (size_t)P.region_w * (kBwTileH + 2 * P.halo) * sizeof(float4);
  dim3 grid((P.W + kBwTileW - 1) / kBwTileW, (P.H + kBwTileH - 1) / kBwTileH);
  k<<<grid, kBwThreads, smem, s>>>(P);
  DISK_TRY_CUDA(cudaGetLastError(), "launch sv_adjoint_layer_kernel");
  return DISK_OK;
}

template <int DIMS>
int dispatch_adjoint(int gkind, int C, const BwParams &P, cudaStream_t s) {
  const bool c4 = C == 4;
  if (gkind == PIX_F32) return c4 ? launch_adjoint<DIMS, PIX_F32, 4>(P, s) : launch_adjoint<DIMS, PIX_F32, 3>(P, s);
  if (gkind == PIX_F16) return c4 ? launch_adjoint<DIMS, PIX_F16, 4>(P, s) : launch_adjoint<DIMS, PIX_F16, 3>(P, s);
  return c4 ? launch_adjoint<DIMS, PIX_RGBA32, 4>(P, s) : launch_adjoint<DIMS, PIX_RGBA32, 3>(P, s);
}

}  // namespace
}  // namespace disk

using namespace disk;

extern "C" int disk_sv_filter_backward_image(const disk_basis *b, const void *d_grad_out,
                                             size_t gout_pitch, float *d_grad_in,
                                             size_t gin_pitch, int H, int W, int C, int dtype,
                                             const float *d_maps, void *stream) {
  if (!b) return fail(DISK_ERR_INVALID_ARG, "null basis");
  if (!d_grad_in) return fail(DISK_ERR_INVALID_ARG, "null grad_in");
  int rc = validate_image_args(d_grad_out, gout_pitch, d_grad_in, gin_pitch, H, W, C, dtype, d_maps);
  if (rc) return rc;
  if (gin_pitch < (size_t)W * C * 4 || gin_pitch % 4 || ((uintptr_t)d_grad_in % 4))
    return fail(DISK_ERR_INVALID_ARG, "grad_in is FP32: pitch must hold W * C floats");
  int dev = 0;
  DISK_TRY_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
  if (dev != b->device) return fail(DISK_ERR_INVALID_ARG, "basis lives on another device");
  for (int l = 0; l < b->L; ++l) {
    const int h = halo_of(b->reach[l]);
    if ((size_t)(kBwTileW + 2 * h) * (kBwTileH + 2 * h) * sizeof(float4) > (size_t)kBwMaxSmem)
      return fail(DISK_ERR_UNSUPPORTED, "layer halo exceeds shared memory");
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t plane = (size_t)H * W * sizeof(float4);
  float4 *bufs[2] = {nullptr, nullptr};
  const int nbuf = b->L >= 2 ? 2 : 1;
  for (int i = 0; i < nbuf; ++i) {
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&bufs[i]), plane, s);
    if (e != cudaSuccess) {
      if (i) cudaFreeAsync(bufs[0], s);
      return cuda_fail(e, "cudaMallocAsync(backward planes)");
    }
  }
  static thread_local BwParams P;
  P.maps = d_maps;
  P.H = H; P.W = W; P.C = C; P.T = b->T;
  make_axes(b->dims, b->n_nodes, b->node_vals.data(), P.ax);
  const int user = dtype == DISK_F32 ? PIX_F32 : PIX_F16;
  const float4 *src = nullptr;
  int k = 0;
  cudaError_t e = cudaSuccess;
  for (int l = b->L - 1; l >= 0 && rc == DISK_OK; --l) {
    float4 *dst = bufs[k];
    e = cudaMemsetAsync(dst, 0, plane, s);
    if (e != cudaSuccess) { rc = cuda_fail(e, "cudaMemsetAsync(backward plane)"); break; }
    P.halo = halo_of(b->reach[l]);
    P.region_w = kBwTileW + 2 * P.halo;
    P.taps = b->d_taps + (size_t)l * b->B * b->T;
    P.gdst = dst;
    const int gkind = l == b->L - 1 ? user : PIX_RGBA32;
    P.gsrc = l == b->L - 1 ? d_grad_out : static_cast<const void *>(src);
    P.gsrc_pitch = l == b->L - 1 ? (long long)gout_pitch : (long long)W * sizeof(float4);
    rc = b->dims == 1 ? dispatch_adjoint<1>(gkind, C, P, s) : dispatch_adjoint<2>(gkind, C, P, s);
    src = dst;
    k ^= 1;
  }
  if (rc == DISK_OK) {
    rgba_to_user_kernel<<<1216, 256, 0, s>>>(src, d_grad_in, (long long)gin_pitch, H, W, C);
    e = cudaGetLastError();
    if (e != cudaSuccess) rc = cuda_fail(e, "launch rgba_to_user_kernel");
  }
  for (int i = 0; i < nbuf; ++i) cudaFreeAsync(bufs[i], s);
  return rc;
}
