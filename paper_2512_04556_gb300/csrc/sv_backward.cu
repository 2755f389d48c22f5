// Gradient of the spatially varying cascade with respect to its input image
// (the transpose of Sec. 3.2 Eq. 3 with the Sec. 4.3 Eq. 9 per-pixel
// complex): grad_in = A_1^T ... A_L^T grad_out.
//
// The filter is linear in the image, so no activation is needed -- only the
// per-pixel taps, recomputed from the maps exactly as the forward pass does.
// Each layer's transpose is a scatter (the taps belong to the output pixel):
// a CTA owns a 32 x 32 tile of output pixels x, zeroes a shared-memory
// accumulator (one float plane per channel) covering the tile plus the layer
// halo, and for every tap adds
// w * beta_c * g[x] to the four corners x + n + c (coordinates clamped to the
// image, which is the transpose of the clamp-to-edge read).  The region is
// then added into the layer's FP32 RGBA gradient plane with vector global
// atomics (neighbouring tiles' regions overlap).  Summation order, and so the
// last bits, vary from run to run.
#include <type_traits>

#include "canvas.cuh"
#include "sv_layer.cuh"

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
  int H, W, C, T, halo;
  int halo_x;           // columns left and right of the tile: bw_halo_x(halo)
  int region_w;         // kBwTileW + 2 halo_x
  AxisNodes ax[2];
};

// Column halo of the image adjoint's region: the halo rounded up to 16
// pixels, so that region rows are a multiple of 32 floats and a warp whose
// lanes' corners straddle two rows adds to distinct banks.
inline int bw_halo_x(int halo) { return (halo + 15) & ~15; }

template <int DIMS, int GKIND, int CH>
__global__ void __launch_bounds__(kBwThreads)
sv_adjoint_layer_kernel(const __grid_constant__ BwParams P) {
  // One float plane per channel: consecutive lanes add to consecutive words,
  // so the shared-memory atomics of a warp spread over all banks.
  extern __shared__ float acc[];
  const int halo = P.halo, RW = P.region_w, RH = kBwTileH + 2 * halo, RN = RW * RH;
  const int tx0 = blockIdx.x * kBwTileW, ty0 = blockIdx.y * kBwTileH;
  const int ox = tx0 - P.halo_x, oy = ty0 - halo;  // image coordinates of region (0, 0)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int j = threadIdx.x; j < RN * CH; j += kBwThreads) acc[j] = 0.f;
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
        const int i00 = ly0 * RW + lx0, i01 = ly0 * RW + lx1, i10 = ly1 * RW + lx0, i11 = ly1 * RW + lx1;
#pragma unroll
        for (int ch = 0; ch < CH; ++ch) {
          const float gc = ch == 0 ? g.x : ch == 1 ? g.y : ch == 2 ? g.z : g.w;
          float *a = acc + ch * RN;
          atomicAdd(a + i00, w00 * gc);
          atomicAdd(a + i01, w01 * gc);
          atomicAdd(a + i10, w10 * gc);
          atomicAdd(a + i11, w11 * gc);
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
      const int e = ry * RW + rx;
      const float4 v = make_float4(acc[e], acc[RN + e], acc[2 * RN + e], CH == 4 ? acc[3 * RN + e] : 0.f);
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
  const size_t smem = (size_t)P.region_w * (kBwTileH + 2 * P.halo) * CH * sizeof(float);
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


// ---- gradient with respect to the basis taps ---------------------------------

struct TgParams {
  const void *src;        // this layer's input (activation recomputed by the forward kernels)
  long long src_pitch;
  const void *gsrc;       // gradient of this layer's output
  long long gsrc_pitch;
  float *gtheta;          // [B][L][T][3], accumulated
  const float *maps;
  const float4 *taps;     // [B][T] of this layer: (dx, dy, w, w)
  int H, W, C, T, B, L, layer, halo, region_w;
  AxisNodes ax[2];
};

__device__ __forceinline__ float tg_warp_sum(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Warp sums of N = 16 (or 8) values per lane by recursive halving: at each
// step a lane keeps half of its values and adds its partner's copies of that
// half, so the whole reduction takes N - 1 + (5 - log2 N) shuffles instead of
// 5 N.  On return lane l holds in v[0] the warp sum of value
// tg_scatter_index<N>(l) (lanes l and l ^ 1 hold the same one for N = 16).
template <int N>
__device__ __forceinline__ int tg_scatter_index(int lane) {
  return N == 16 ? (((lane >> 4) & 1) << 3) | (((lane >> 3) & 1) << 2) | (((lane >> 2) & 1) << 1) |
                       ((lane >> 1) & 1)
                 : (((lane >> 4) & 1) << 2) | (((lane >> 3) & 1) << 1) | ((lane >> 2) & 1);
}

template <int N>
__device__ __forceinline__ void tg_warp_reduce_scatter(float (&v)[N], int lane) {
#pragma unroll
  for (int n = N / 2, o = 16; n >= 1; n /= 2, o /= 2) {
    const bool upper = (lane & o) != 0;
#pragma unroll
    for (int k = 0; k < n; ++k) {
      const float keep = upper ? v[k + n] : v[k];
      const float give = upper ? v[k] : v[k + n];
      v[k] = keep + __shfl_xor_sync(0xffffffffu, give, o);
    }
  }
  // the offsets not used for halving sum the one remaining value
#pragma unroll
  for (int o = N == 16 ? 1 : 2; o >= 1; o /= 2) v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
}

__device__ __forceinline__ float4 tg_staged(const float4 &v) { return v; }
__device__ __forceinline__ float4 tg_staged(const uint2 &v) { return unpack_half4(v); }

// d/d(dx, dy, w) of <g, w * bilinear(I, x + o)> for one pixel and tap, from the
// staged layer input (floor convention: fraction in [0, 1)).
template <int CH, typename ST>
__device__ __forceinline__ float3 tap_grad(const ST *base, int RW, int halo, float dx, float dy,
                                           float w, const float4 &g) {
  float fx, fy;
  const int nx = min(max(split_floor(dx, fx), -halo), halo - 1);
  const int ny = min(max(split_floor(dy, fy), -halo), halo - 1);
  const ST *q = base + ny * RW + nx;
  const float4 a = tg_staged(q[0]), b = tg_staged(q[1]), c = tg_staged(q[RW]), d = tg_staged(q[RW + 1]);
  float gw = 0.f, gx = 0.f, gy = 0.f;
#define DISK_TG_CH(F, GC)                                                        \
  {                                                                              \
    const float top = a.F + fx * (b.F - a.F), bot = c.F + fx * (d.F - c.F);      \
    gw += GC * (top + fy * (bot - top));                                         \
    gx += GC * ((1.f - fy) * (b.F - a.F) + fy * (d.F - c.F));                    \
    gy += GC * (bot - top);                                                      \
  }
  DISK_TG_CH(x, g.x)
  DISK_TG_CH(y, g.y)
  DISK_TG_CH(z, g.z)
  if (CH == 4) DISK_TG_CH(w, g.w)
#undef DISK_TG_CH
  return make_float3(w * gx, w * gy, gw);
}

template <int DIMS, int SRC, int GKIND, int CH>
__global__ void __launch_bounds__(kBwThreads)
sv_theta_grad_kernel(const __grid_constant__ TgParams P) {
  constexpr bool kHalf = SRC == PIX_F16 || SRC == PIX_RGBA16;
  using ST = typename std::conditional<kHalf, uint2, float4>::type;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int halo = P.halo, RW = P.region_w, RH = kBwTileH + 2 * halo;
  ST *sm = reinterpret_cast<ST *>(sm_raw);
  float *gacc = reinterpret_cast<float *>(sm_raw + (((size_t)RW * RH * sizeof(ST) + 15) & ~(size_t)15));
  const int T = P.T, nacc = P.B * T * 3;
  const int tx0 = blockIdx.x * kBwTileW, ty0 = blockIdx.y * kBwTileH;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int j = threadIdx.x; j < nacc; j += kBwThreads) gacc[j] = 0.f;
  for (int ry = warp; ry < RH; ry += kBwWarps) {
    const int gy = min(max(ty0 - halo + ry, 0), P.H - 1);
    for (int rx = lane; rx < RW; rx += 32) {
      const int gx = min(max(tx0 - halo + rx, 0), P.W - 1);
      if constexpr (kHalf)
        sm[ry * RW + rx] = load_raw16<SRC>(P.src, P.src_pitch, P.C, gy, gx);
      else
        sm[ry * RW + rx] = load_px<SRC>(P.src, P.src_pitch, P.C, gy, gx);
    }
  }
  __syncthreads();

  const int x = tx0 + lane, xc = min(x, P.W - 1);
  const long long HW = (long long)P.H * P.W;
  Cell c[kBwPix];
  float4 g[kBwPix];
  const ST *base[kBwPix];
  bool same = true;
#pragma unroll
  for (int j = 0; j < kBwPix; ++j) {
    const int r = warp + kBwWarps * j, y = ty0 + r, yc = min(y, P.H - 1);
    c[j] = make_cell<DIMS>(P.ax, P.maps, HW, (long long)yc * P.W + xc);
    // pixels outside the image carry no gradient
    g[j] = (x < P.W && y < P.H) ? load_px<GKIND>(P.gsrc, P.gsrc_pitch, P.C, y, x)
                                : make_float4(0.f, 0.f, 0.f, 0.f);
    base[j] = sm + (r + halo) * RW + (lane + halo);
    same = same && (c[j].n00 == c[0].n00);
  }
  // The warp reduction below needs one cell for the whole warp, not only
  // per thread.  The shuffle is executed by every lane (it must not sit
  // behind a short-circuiting condition: a full-mask shuffle that some lanes
  // skip never completes).
  const int lead_cell = __shfl_sync(0xffffffffu, c[0].n00, 0);
  same = same && c[0].n00 == lead_cell;
  if (__all_sync(0xffffffffu, same)) {
    // nodes are warp-uniform: reduce each tap's node gradients over the
    // thread's pixels, then over the warp, and add them once
    const int n00 = c[0].n00, n10 = c[0].n10, n01 = c[0].n01, n11 = c[0].n11;
    for (int i = 0; i < T; ++i) {
      const float4 q00 = __ldg(P.taps + n00 * T + i), q10 = __ldg(P.taps + n10 * T + i);
      const float4 q01 = DIMS == 2 ? __ldg(P.taps + n01 * T + i) : q00;
      const float4 q11 = DIMS == 2 ? __ldg(P.taps + n11 * T + i) : q10;
      float v[12];
#pragma unroll
      for (int k = 0; k < 12; ++k) v[k] = 0.f;
#pragma unroll
      for (int j = 0; j < kBwPix; ++j) {
        const Cell &cj = c[j];
        float dx = cj.a00 * q00.x + cj.a10 * q10.x, dy = cj.a00 * q00.y + cj.a10 * q10.y;
        float w = cj.a00 * q00.z + cj.a10 * q10.z;
        if (DIMS == 2) {
          dx += cj.a01 * q01.x + cj.a11 * q11.x;
          dy += cj.a01 * q01.y + cj.a11 * q11.y;
          w += cj.a01 * q01.z + cj.a11 * q11.z;
        }
        const float3 t = tap_grad<CH, ST>(base[j], RW, halo, dx, dy, w, g[j]);
        v[0] += cj.a00 * t.x; v[1] += cj.a00 * t.y; v[2] += cj.a00 * t.z;
        v[3] += cj.a10 * t.x; v[4] += cj.a10 * t.y; v[5] += cj.a10 * t.z;
        if (DIMS == 2) {
          v[6] += cj.a01 * t.x; v[7] += cj.a01 * t.y; v[8] += cj.a01 * t.z;
          v[9] += cj.a11 * t.x; v[10] += cj.a11 * t.y; v[11] += cj.a11 * t.z;
        }
      }
      // reduce the 12 (2-D) or 6 (1-D) node-gradient values over the warp
      // in one reduce-scatter; one lane per value then adds it
      constexpr int NV = DIMS == 2 ? 16 : 8;
      float r[NV];
#pragma unroll
      for (int k = 0; k < NV; ++k) r[k] = k < (DIMS == 2 ? 12 : 6) ? v[k] : 0.f;
      tg_warp_reduce_scatter<NV>(r, lane);
      const int idx = tg_scatter_index<NV>(lane);
      const bool owner = NV == 16 ? (lane & 1) == 0 : (lane & 3) == 0;
      if (owner && idx < (DIMS == 2 ? 12 : 6)) {
        const int node = (idx / 3) == 0 ? n00 : (idx / 3) == 1 ? n10 : (idx / 3) == 2 ? n01 : n11;
        atomicAdd(gacc + (node * T + i) * 3 + idx % 3, r[0]);
      }
    }
  } else {
    // cells differ across the warp: per pixel slot, reduce one distinct cell
    // at a time (each round retires at least the leading lane, so at most 32
    // rounds); only lane 0 touches the shared accumulator.
#pragma unroll 1
    for (int j = 0; j < kBwPix; ++j) {
      const Cell &cj = c[j];
      for (int i = 0; i < T; ++i) {
        const float4 q00 = __ldg(P.taps + cj.n00 * T + i), q10 = __ldg(P.taps + cj.n10 * T + i);
        float dx = cj.a00 * q00.x + cj.a10 * q10.x, dy = cj.a00 * q00.y + cj.a10 * q10.y;
        float w = cj.a00 * q00.z + cj.a10 * q10.z;
        if (DIMS == 2) {
          const float4 q01 = __ldg(P.taps + cj.n01 * T + i), q11 = __ldg(P.taps + cj.n11 * T + i);
          dx += cj.a01 * q01.x + cj.a11 * q11.x;
          dy += cj.a01 * q01.y + cj.a11 * q11.y;
          w += cj.a01 * q01.z + cj.a11 * q11.z;
        }
        const float3 t = tap_grad<CH, ST>(base[j], RW, halo, dx, dy, w, g[j]);
        unsigned todo = 0xffffffffu;
        for (int round = 0; round < 32 && todo; ++round) {
          const int leader = __ffs(todo) - 1;
          const int cell = __shfl_sync(0xffffffffu, cj.n00, leader);
          const bool mine = ((todo >> lane) & 1u) && cj.n00 == cell;
          todo &= ~__ballot_sync(0xffffffffu, mine);
          const float m = mine ? 1.f : 0.f;
          float v[12] = {m * cj.a00 * t.x, m * cj.a00 * t.y, m * cj.a00 * t.z,
                         m * cj.a10 * t.x, m * cj.a10 * t.y, m * cj.a10 * t.z,
                         m * cj.a01 * t.x, m * cj.a01 * t.y, m * cj.a01 * t.z,
                         m * cj.a11 * t.x, m * cj.a11 * t.y, m * cj.a11 * t.z};
#pragma unroll
          for (int k = 0; k < (DIMS == 2 ? 12 : 6); ++k) v[k] = tg_warp_sum(v[k]);
          const int n10 = __shfl_sync(0xffffffffu, cj.n10, leader);
          const int n01 = __shfl_sync(0xffffffffu, cj.n01, leader);
          const int n11 = __shfl_sync(0xffffffffu, cj.n11, leader);
          if (lane == 0) {
            const int nodes[4] = {cell, n10, n01, n11};
#pragma unroll
            for (int k = 0; k < (DIMS == 2 ? 4 : 2); ++k) {
              float *dst = gacc + (nodes[k] * T + i) * 3;
              atomicAdd(dst, v[3 * k]); atomicAdd(dst + 1, v[3 * k + 1]); atomicAdd(dst + 2, v[3 * k + 2]);
            }
          }
        }
      }
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < nacc; j += kBwThreads) {
    const float v = gacc[j];
    if (v != 0.f) {
      const int k = j / (T * 3), r = j - k * T * 3;
      atomicAdd(P.gtheta + ((size_t)k * P.L + P.layer) * T * 3 + r, v);
    }
  }
}

template <int DIMS, int SRC, int GKIND, int CH>
int launch_theta_grad(const TgParams &P, cudaStream_t s) {
  auto k = sv_theta_grad_kernel<DIMS, SRC, GKIND, CH>;
  static unsigned long long attr_set = 0;
  int dev = 0;
  cudaGetDevice(&dev);
  if (!(attr_set & (1ull << (dev & 63)))) {
    DISK_TRY_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kBwMaxSmem),
                  "cudaFuncSetAttribute(sv_theta_grad)");
    attr_set |= 1ull << (dev & 63);
  }
  const size_t px = (SRC == PIX_F16 || SRC == PIX_RGBA16) ? 8 : 16;
  const size_t region = (((size_t)P.region_w * (kBwTileH + 2 * P.halo) * px) + 15) & ~(size_t)15;
  const size_t smem = region + (size_t)P.B * P.T * 3 * sizeof(float);
  if (smem > (size_t)kBwMaxSmem) return fail(DISK_ERR_UNSUPPORTED, "basis gradient exceeds shared memory");
  dim3 grid((P.W + kBwTileW - 1) / kBwTileW, (P.H + kBwTileH - 1) / kBwTileH);
  k<<<grid, kBwThreads, smem, s>>>(P);
  DISK_TRY_CUDA(cudaGetLastError(), "launch sv_theta_grad_kernel");
  return DISK_OK;
}

template <int DIMS>
int dispatch_theta_grad(int src, int gkind, int C, const TgParams &P, cudaStream_t s) {
  const bool c4 = C == 4;
#define DISK_TG_CASE(S, G)                                                                  \
  if (src == S && gkind == G)                                                               \
    return c4 ? launch_theta_grad<DIMS, S, G, 4>(P, s) : launch_theta_grad<DIMS, S, G, 3>(P, s);
  DISK_TG_CASE(PIX_F32, PIX_F32)
  DISK_TG_CASE(PIX_F32, PIX_RGBA32)
  DISK_TG_CASE(PIX_RGBA32, PIX_F32)
  DISK_TG_CASE(PIX_RGBA32, PIX_RGBA32)
  DISK_TG_CASE(PIX_F16, PIX_F16)
  DISK_TG_CASE(PIX_F16, PIX_RGBA32)
  DISK_TG_CASE(PIX_RGBA16, PIX_F16)
  DISK_TG_CASE(PIX_RGBA16, PIX_RGBA32)
#undef DISK_TG_CASE
  return fail(DISK_ERR_INVALID_ARG, "unsupported basis-gradient storage combination");
}

// Recompute the forward activations I_1 .. I_{L-1} (layer inputs) into
// planes with the forward kernels (nothing is kept from the forward call).
int recompute_activations(const disk_basis *b, const void *d_in, size_t in_pitch, int H, int W,
                          int C, int dtype, const float *d_maps, char *const *planes,
                          cudaStream_t s) {
  static thread_local SvLayerParams P;
  P.maps = d_maps;
  P.rot = nullptr;
  P.use_tma = 0;
  P.err = device_error_word();
  P.H = H; P.W = W; P.C = C; P.T = b->T;
  make_axes(b->dims, b->n_nodes, b->node_vals.data(), P.ax);
  const int user = dtype == DISK_F32 ? PIX_F32 : PIX_F16, mid = intermediate_kind(dtype);
  const size_t mid_bytes = kind_bytes(mid);
  for (int l = 0; l + 1 < b->L; ++l) {
    P.halo = P.halo_x = halo_of(b->reach[l]);
    P.region_w = kSvTileW + 2 * P.halo;
    P.src = l == 0 ? d_in : planes[l - 1];
    P.src_pitch = l == 0 ? (long long)in_pitch : (long long)(W * mid_bytes);
    P.dst = planes[l];
    P.dst_pitch = (long long)(W * mid_bytes);
    P.gtaps = layer_taps(b, l, C);
    P.bt = b->B * b->T;
    const size_t region = sv_smem_bytes((size_t)P.region_w * (sv_tile_h(kSvDefaultPix) + 2 * P.halo), C);
    P.tap_cap = sv_tap_cap(b->dims, b->n_nodes[1], b->B, b->T, region);
    const int rc = launch_layer(b->dims, false, l == 0 ? user : mid, mid, C, P, s, kSvDefaultPix);
    if (rc) return rc;
  }
  return DISK_OK;
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
    if ((size_t)(kBwTileW + 2 * bw_halo_x(h)) * (kBwTileH + 2 * h) * sizeof(float4) > (size_t)kBwMaxSmem)
      return fail(DISK_ERR_UNSUPPORTED, "layer halo exceeds shared memory");
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t plane = (size_t)H * W * sizeof(float4);
  float4 *bufs[2] = {nullptr, nullptr};
  const int nbuf = b->L >= 2 ? 2 : 1;
  for (int i = 0; i < nbuf; ++i) {
    cudaError_t e = scratch_alloc(reinterpret_cast<void **>(&bufs[i]), plane, s);
    if (e != cudaSuccess) {
      if (i) cudaFreeAsync(bufs[0], s);
      return cuda_fail(e, "scratch_alloc(backward planes)");
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
    P.halo_x = bw_halo_x(P.halo);
    P.region_w = kBwTileW + 2 * P.halo_x;
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

extern "C" int disk_sv_filter_backward(const disk_basis *b, const void *d_in, size_t in_pitch,
                                       const void *d_grad_out, size_t gout_pitch,
                                       float *d_grad_in, size_t gin_pitch, float *d_grad_theta,
                                       int H, int W, int C, int dtype, const float *d_maps,
                                       void *stream) {
  if (!b) return fail(DISK_ERR_INVALID_ARG, "null basis");
  if (!d_grad_in && !d_grad_theta) return fail(DISK_ERR_INVALID_ARG, "nothing to compute");
  int rc = validate_image_args(d_in, in_pitch, d_grad_out, gout_pitch, H, W, C, dtype, d_maps);
  if (rc) return rc;
  if (d_grad_in && (gin_pitch < (size_t)W * C * 4 || gin_pitch % 4 || ((uintptr_t)d_grad_in % 4)))
    return fail(DISK_ERR_INVALID_ARG, "grad_in is FP32: pitch must hold W * C floats");
  if (d_grad_theta && ((uintptr_t)d_grad_theta % 4))
    return fail(DISK_ERR_INVALID_ARG, "misaligned grad_theta");
  int dev = 0;
  DISK_TRY_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
  if (dev != b->device) return fail(DISK_ERR_INVALID_ARG, "basis lives on another device");
  const size_t stage_px = dtype == DISK_F32 ? 16 : 8;
  for (int l = 0; l < b->L; ++l) {
    const int h = halo_of(b->reach[l]);
    const size_t region = (size_t)(kBwTileW + 2 * h) * (kBwTileH + 2 * h);
    if ((size_t)(kBwTileW + 2 * bw_halo_x(h)) * (kBwTileH + 2 * h) * sizeof(float4) > (size_t)kBwMaxSmem ||
        ((region * stage_px + 15) & ~(size_t)15) + (size_t)b->B * b->T * 12 > (size_t)kBwMaxSmem)
      return fail(DISK_ERR_UNSUPPORTED, "layer halo or basis size exceeds shared memory");
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int L = b->L, mid = intermediate_kind(dtype), user = dtype == DISK_F32 ? PIX_F32 : PIX_F16;
  const size_t act_plane = (size_t)H * W * kind_bytes(mid), g_plane = (size_t)H * W * sizeof(float4);
  const size_t bytes = (size_t)(L - 1) * act_plane + 2 * g_plane;
  char *buf = nullptr;
  DISK_TRY_CUDA(scratch_alloc(reinterpret_cast<void **>(&buf), bytes, s), "scratch_alloc(backward)");
  char *acts[DISK_MAX_LAYERS];
  for (int l = 0; l + 1 < L; ++l) acts[l] = buf + (size_t)l * act_plane;
  float4 *gpl[2] = {reinterpret_cast<float4 *>(buf + (size_t)(L - 1) * act_plane),
                    reinterpret_cast<float4 *>(buf + (size_t)(L - 1) * act_plane + g_plane)};
  if (L > 1) {
    rc = recompute_activations(b, d_in, in_pitch, H, W, C, dtype, d_maps, acts, s);
  }
  cudaError_t e = cudaSuccess;
  if (rc == DISK_OK && d_grad_theta) {
    e = cudaMemsetAsync(d_grad_theta, 0, (size_t)b->B * L * b->T * 3 * sizeof(float), s);
    if (e != cudaSuccess) rc = cuda_fail(e, "cudaMemsetAsync(grad_theta)");
  }
  static thread_local TgParams TP;
  static thread_local BwParams BP;
  make_axes(b->dims, b->n_nodes, b->node_vals.data(), TP.ax);
  make_axes(b->dims, b->n_nodes, b->node_vals.data(), BP.ax);
  TP.maps = BP.maps = d_maps;
  TP.H = BP.H = H; TP.W = BP.W = W; TP.C = BP.C = C; TP.T = BP.T = b->T;
  TP.B = b->B; TP.L = L; TP.gtheta = d_grad_theta;
  const float4 *g_src = nullptr;
  int k = 0;
  for (int l = L - 1; l >= 0 && rc == DISK_OK; --l) {
    const int gkind = l == L - 1 ? user : PIX_RGBA32;
    const void *gptr = l == L - 1 ? d_grad_out : static_cast<const void *>(g_src);
    const long long gpitch = l == L - 1 ? (long long)gout_pitch : (long long)W * sizeof(float4);
    const float4 *ltaps = b->d_taps + (size_t)l * b->B * b->T;
    const int halo = halo_of(b->reach[l]);
    if (d_grad_theta) {
      TP.src = l == 0 ? d_in : acts[l - 1];
      TP.src_pitch = l == 0 ? (long long)in_pitch : (long long)(W * kind_bytes(mid));
      TP.gsrc = gptr; TP.gsrc_pitch = gpitch;
      TP.taps = ltaps; TP.layer = l; TP.halo = halo; TP.region_w = kBwTileW + 2 * halo;
      const int src = l == 0 ? user : mid;
      rc = b->dims == 1 ? dispatch_theta_grad<1>(src, gkind, C, TP, s)
                        : dispatch_theta_grad<2>(src, gkind, C, TP, s);
      if (rc) break;
    }
    if (l > 0 || d_grad_in) {
      float4 *dst = gpl[k];
      e = cudaMemsetAsync(dst, 0, g_plane, s);
      if (e != cudaSuccess) { rc = cuda_fail(e, "cudaMemsetAsync(backward plane)"); break; }
      BP.gsrc = gptr; BP.gsrc_pitch = gpitch; BP.gdst = dst; BP.taps = ltaps;
      BP.halo = halo; BP.halo_x = bw_halo_x(halo); BP.region_w = kBwTileW + 2 * BP.halo_x;
      rc = b->dims == 1 ? dispatch_adjoint<1>(gkind, C, BP, s) : dispatch_adjoint<2>(gkind, C, BP, s);
      g_src = dst;
      k ^= 1;
    }
  }
  if (rc == DISK_OK && d_grad_in) {
    rgba_to_user_kernel<<<1216, 256, 0, s>>>(g_src, d_grad_in, (long long)gin_pitch, H, W, C);
    e = cudaGetLastError();
    if (e != cudaSuccess) rc = cuda_fail(e, "launch rgba_to_user_kernel");
  }
  cudaFreeAsync(buf, s);
  return rc;
}
