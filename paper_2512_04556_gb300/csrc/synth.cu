// Impulse-response synthesis, Sec. 4.4 Eq. 10: K_syn = F_theta(delta) for a
// batch of shift-invariant complexes, one CTA per complex.
//
// The CTA derives each layer's reach from its taps, then runs the cascade on
// two ping-pong canvases in global scratch (L2-resident at these sizes),
// computing layer l only on the box that can be non-zero and still matters
// for the K x K crop: b_l = min(S_l, (K-1)/2 + H_{l+1} + ... + H_L).  The
// frames beyond each computed box that the next layer reads are zeroed, so
// the canvas behaves as the zero-padded plane of Eq. 10.
#include <cmath>

#include "canvas.cuh"

namespace disk {
namespace {

constexpr int kSynthThreads = 512;

__global__ void __launch_bounds__(kSynthThreads)
synth_kernel(const float *theta, int L, int T, int K, float max_reach, int R, float *scratch,
             float *out) {
  extern __shared__ float4 taps[];  // [L][T]
  __shared__ LayerExtent ext[DISK_MAX_LAYERS];
  __shared__ PreparedTaps pt;
  __shared__ int bad;
  const int b = blockIdx.x, N = 2 * R + 1, hw = (K - 1) / 2;
  const float *th = theta + (size_t)b * L * T * 3;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int j = threadIdx.x; j < L * T; j += blockDim.x) {
    const float dx = th[3 * j], dy = th[3 * j + 1], w = th[3 * j + 2];
    if (!(fabsf(dx) <= max_reach) || !(fabsf(dy) <= max_reach) || !isfinite(w)) bad = 1;
    taps[j] = make_float4(dx, dy, w, 0.f);
  }
  __syncthreads();
  float *o = out + (size_t)b * K * K;
  if (bad) {  // a tap beyond the declared reach: the whole response is NaN
    for (int j = threadIdx.x; j < K * K; j += blockDim.x) o[j] = __int_as_float(0x7fc00000);
    return;
  }
  if (threadIdx.x < 32) {
    int S = 0;
    for (int l = 0; l < L; ++l) {
      float m = 0.f;
      for (int i = threadIdx.x; i < T; i += 32)
        m = fmaxf(m, fmaxf(fabsf(taps[l * T + i].x), fabsf(taps[l * T + i].y)));
      for (int s = 16; s > 0; s >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, s));
      const int H = (int)ceilf(m) + 1;
      S += H;
      if (threadIdx.x == 0) { ext[l].H = H; ext[l].S = S; }
    }
  }
  __syncthreads();
  float *pa = scratch + (size_t)b * 2 * N * N, *pb = pa + (size_t)N * N;
  // box b_l of each layer
  int bl[DISK_MAX_LAYERS];
  {
    int tail = 0;
    for (int l = L - 1; l >= 0; --l) {
      bl[l] = min(ext[l].S, hw + tail);
      tail += ext[l].H;
    }
  }
  // Impulse plane: zero the footprint layer 1 reads, then the unit impulse.
  zero_frame(pa, R, -1, bl[0] + ext[0].H);
  __syncthreads();
  if (threadIdx.x == 0) pa[R * N + R] = 1.f;
  __syncthreads();
  for (int l = 0; l < L; ++l) {
    prepare_taps(pt, taps + l * T, T, ext[l].H, 1.f, R);
    __syncthreads();
    canvas_layer(pa, pb, R, bl[l], pt, T);
    __syncthreads();
    if (l + 1 < L) {
      zero_frame(pb, R, bl[l], bl[l + 1] + ext[l + 1].H);
    } else {
      zero_frame(pb, R, bl[l], hw);
    }
    __syncthreads();
    float *t = pa; pa = pb; pb = t;
  }
  for (int j = threadIdx.x; j < K * K; j += blockDim.x) {
    const int v = j / K - hw, u = j % K - hw;
    o[j] = pa[(R + v) * N + (R + u)];
  }
}

}  // namespace
}  // namespace disk

using namespace disk;

extern "C" int disk_synth_kernel(const float *d_theta, int batch, int L, int T, int K,
                                 float max_reach, float *d_out, void *stream) {
  if (!d_theta || !d_out) return fail(DISK_ERR_INVALID_ARG, "null pointer");
  if (batch < 1 || L < 1 || L > DISK_MAX_LAYERS || T < 1 || T > DISK_MAX_TAPS)
    return fail(DISK_ERR_INVALID_ARG, "batch >= 1, L in [1, 16], T in [1, 64] required");
  if (K < 1 || K > 257 || (K & 1) == 0) return fail(DISK_ERR_INVALID_ARG, "K must be odd, <= 257");
  if (!(max_reach >= 0.f) || max_reach > 256.f)
    return fail(DISK_ERR_INVALID_ARG, "max_reach must be in [0, 256]");
  const int hw = (K - 1) / 2;
  const int R = hw + L * ((int)std::ceil(max_reach) + 1) + 1;
  const size_t N = 2 * (size_t)R + 1;
  const size_t bytes = (size_t)batch * 2 * N * N * sizeof(float);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  float *scratch = nullptr;
  DISK_TRY_CUDA(scratch_alloc(reinterpret_cast<void **>(&scratch), bytes, s),
                "scratch_alloc(synth canvases)");
  const size_t smem = (size_t)L * T * sizeof(float4);
  synth_kernel<<<batch, kSynthThreads, smem, s>>>(d_theta, L, T, K, max_reach, R, scratch, d_out);
  cudaError_t e = cudaGetLastError();
  cudaFreeAsync(scratch, s);
  if (e != cudaSuccess) return cuda_fail(e, "launch synth_kernel");
  return DISK_OK;
}
