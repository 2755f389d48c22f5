// Dense spatially varying convolution (Sec. 3.1 Eq. 1, one kernel per pixel
// blended from dense node kernels with the Eq. 9 weights): the reference
// DISK approximates and the speed baseline it is measured against.
//
// Same staging discipline as the sparse path so the comparison is fair: a
// 32 x 32 output tile plus the kernel half-width is staged in shared memory
// in the image's precision (FP16 RGBA for FP16 images, FP32 RGBA for FP32);
// each lane owns one pixel and walks the support box of its
// cell's node kernels (warp-uniform bound), reading the node kernels through
// L1 and the image from shared memory.
#include <type_traits>

#include "sv_common.cuh"

namespace disk {
namespace {

constexpr int kTileW = 32, kTileH = 32, kThreads = 256;

struct DenseParams {
  const void *src;
  long long src_pitch;
  void *dst;
  long long dst_pitch;
  const float *maps;
  const float *lut;     // [B][Kd][Kd]
  const int *node_hw;   // [B] half-width of each node kernel's non-zero box
  int H, W, C, Kd, hd, region_w;
  AxisNodes ax[2];
};

// Half-width of the smallest centred box holding every non-zero of node k.
__global__ void node_extent_kernel(const float *lut, int Kd, int *node_hw) {
  const int k = blockIdx.x, hd = (Kd - 1) / 2;
  const float *K = lut + (size_t)k * Kd * Kd;
  int m = 0;
  for (int j = threadIdx.x; j < Kd * Kd; j += blockDim.x)
    if (K[j] != 0.f) m = max(m, max(abs(j / Kd - hd), abs(j % Kd - hd)));
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  __shared__ int wm[32];
  if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    int r = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = max(r, wm[w]);
    node_hw[k] = r;
  }
}

__device__ __forceinline__ float4 dense_px(const float4 &v) { return v; }
__device__ __forceinline__ float4 dense_px(const uint2 &v) { return unpack_half4(v); }

template <int DIMS, int KIND>
__global__ void __launch_bounds__(kThreads) dense_sv_kernel(const __grid_constant__ DenseParams P) {
  // FP16 images are staged as FP16 (as the sparse filter does), FP32 as FP32.
  using ST = typename std::conditional<KIND == PIX_F16, uint2, float4>::type;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  ST *sm = reinterpret_cast<ST *>(sm_raw);
  const int hd = P.hd, RW = P.region_w, RH = kTileH + 2 * hd;
  const int tx0 = blockIdx.x * kTileW, ty0 = blockIdx.y * kTileH;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int ry = warp; ry < RH; ry += kThreads / 32) {
    const int gy = min(max(ty0 - hd + ry, 0), P.H - 1);
    for (int rx = lane; rx < RW; rx += 32) {
      const int gx = min(max(tx0 - hd + rx, 0), P.W - 1);
      if constexpr (KIND == PIX_F16)
        sm[ry * RW + rx] = load_raw16<KIND>(P.src, P.src_pitch, P.C, gy, gx);
      else
        sm[ry * RW + rx] = load_px<KIND>(P.src, P.src_pitch, P.C, gy, gx);
    }
  }
  __syncthreads();

  const int x = tx0 + lane;
  const bool xin = x < P.W;
  const long long HW = (long long)P.H * P.W;
  const int Kd = P.Kd, KK = Kd * Kd;
  for (int r = warp; r < kTileH; r += kThreads / 32) {
    const int y = ty0 + r;
    if (y >= P.H) break;
    Cell cell = make_cell<DIMS>(P.ax, P.maps, HW, (long long)y * P.W + (xin ? x : P.W - 1));
    int hb = max(__ldg(P.node_hw + cell.n00), __ldg(P.node_hw + cell.n10));
    if (DIMS == 2) hb = max(hb, max(__ldg(P.node_hw + cell.n01), __ldg(P.node_hw + cell.n11)));
    hb = __reduce_max_sync(0xffffffffu, hb);
    const float *k00 = P.lut + (size_t)cell.n00 * KK + hd * Kd + hd;
    const float *k10 = P.lut + (size_t)cell.n10 * KK + hd * Kd + hd;
    const float *k01 = P.lut + (size_t)cell.n01 * KK + hd * Kd + hd;
    const float *k11 = P.lut + (size_t)cell.n11 * KK + hd * Kd + hd;
    const ST *c = sm + (r + hd) * RW + (lane + hd);
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int my = -hb; my <= hb; ++my) {
      const ST *row = c - my * RW;
      const int ko = my * Kd;
#pragma unroll 4
      for (int mx = -hb; mx <= hb; ++mx) {
        float kw = cell.a00 * __ldg(k00 + ko + mx) + cell.a10 * __ldg(k10 + ko + mx);
        if (DIMS == 2) kw += cell.a01 * __ldg(k01 + ko + mx) + cell.a11 * __ldg(k11 + ko + mx);
        const float4 v = dense_px(row[-mx]);  // I[x - m]: true convolution
        acc.x += kw * v.x; acc.y += kw * v.y; acc.z += kw * v.z; acc.w += kw * v.w;
      }
    }
    if (xin) store_px<KIND>(P.dst, P.dst_pitch, P.C, y, x, acc);
  }
}

template <int DIMS, int KIND>
int launch_dense(const DenseParams &P, cudaStream_t s) {
  auto k = dense_sv_kernel<DIMS, KIND>;
  static unsigned long long attr_set = 0;
  int dev = 0;
  cudaGetDevice(&dev);
  if (!(attr_set & (1ull << (dev & 63)))) {
    DISK_TRY_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448),
                  "cudaFuncSetAttribute(dense_sv)");
    attr_set |= 1ull << (dev & 63);
  }
  const size_t smem = (size_t)P.region_w * (kTileH + 2 * P.hd) * (KIND == PIX_F16 ? 8 : 16);
  dim3 grid((P.W + kTileW - 1) / kTileW, (P.H + kTileH - 1) / kTileH);
  k<<<grid, kThreads, smem, s>>>(P);
  DISK_TRY_CUDA(cudaGetLastError(), "launch dense_sv_kernel");
  return DISK_OK;
}

}  // namespace
}  // namespace disk

using namespace disk;

extern "C" int disk_dense_sv(int dims, const int *n_nodes, const float *node_vals,
                             const float *d_lut, int Kd, const void *d_in, size_t in_pitch,
                             void *d_out, size_t out_pitch, int H, int W, int C, int dtype,
                             const float *d_maps, void *stream) {
  int rc = validate_nodes(dims, n_nodes, node_vals);
  if (rc) return rc;
  rc = validate_image_args(d_in, in_pitch, d_out, out_pitch, H, W, C, dtype, d_maps);
  if (rc) return rc;
  if (!d_lut || Kd < 1 || (Kd & 1) == 0 || Kd > 85)
    return fail(DISK_ERR_INVALID_ARG, "Kd must be odd and at most 85, and d_lut non-null");
  if ((uintptr_t)d_lut % 4) return fail(DISK_ERR_INVALID_ARG, "misaligned d_lut");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int B = dims == 1 ? n_nodes[0] : n_nodes[0] * n_nodes[1];
  static thread_local DenseParams P;
  P.src = d_in; P.src_pitch = (long long)in_pitch;
  P.dst = d_out; P.dst_pitch = (long long)out_pitch;
  P.maps = d_maps; P.lut = d_lut;
  P.H = H; P.W = W; P.C = C; P.Kd = Kd; P.hd = (Kd - 1) / 2;
  P.region_w = kTileW + 2 * P.hd;
  make_axes(dims, n_nodes, node_vals, P.ax);
  int *d_hw = nullptr;
  DISK_TRY_CUDA(scratch_alloc(reinterpret_cast<void **>(&d_hw), sizeof(int) * B, s),
                "scratch_alloc(dense extents)");
  node_extent_kernel<<<B, 256, 0, s>>>(d_lut, Kd, d_hw);
  rc = DISK_OK;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) rc = cuda_fail(e, "launch node_extent_kernel");
  P.node_hw = d_hw;
  if (rc == DISK_OK) {
    const int kind = dtype == DISK_F32 ? PIX_F32 : PIX_F16;
    if (dims == 1) rc = kind == PIX_F32 ? launch_dense<1, PIX_F32>(P, s) : launch_dense<1, PIX_F16>(P, s);
    else rc = kind == PIX_F32 ? launch_dense<2, PIX_F32>(P, s) : launch_dense<2, PIX_F16>(P, s);
  }
  cudaFreeAsync(d_hw, s);
  return rc;
}
