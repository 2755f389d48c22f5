// disk_learned_init: the learned start of the Eq. 4 fit (a project addition
// to the Eq. 6 / Eq. 7 initialisations of Sec. 4.1-4.2), every step on the
// device: area-resample each target, run the network, turn its outputs into
// a complex in pixels (offsets clamped to the fit's box), build the Eq. 6
// start, evaluate the fitted loss of both, and keep per target the start
// with the lower loss (the network's on a tie).
#include <algorithm>
#include <vector>

#include "internal.h"

namespace disk {
namespace {

// Network units -> pixels: offsets clamped to [-1, 1] and scaled by the
// target's half-width s_b = max(1, (K_b - 1) / 2); weights divided by T.
__global__ void unscale_kernel(const float *__restrict__ y, const float *__restrict__ scale,
                               int per, float T, long long n, float *__restrict__ theta) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(i / per), c = (int)(i % per) % 3;
    const float v = y[i];
    theta[i] = c < 2 ? fminf(fmaxf(v, -1.f), 1.f) * scale[b] : v / T;
  }
}

// Per target, the network start where its loss is <= the Eq. 6 start's
// (a NaN loss compares false and keeps the Eq. 6 start).
__global__ void choose_kernel(const float *__restrict__ th_net, const float *__restrict__ th_ir,
                              const float *__restrict__ l_net, const float *__restrict__ l_ir,
                              int per, long long n, float *__restrict__ theta,
                              int *__restrict__ used) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(i / per);
    const bool net = l_net[b] <= l_ir[b];
    theta[i] = net ? th_net[i] : th_ir[i];
    if (used && i % per == 0) used[b] = net ? 1 : 0;
  }
}

int grid_for(long long n) { return (int)std::min<long long>((n + 255) / 256, 152LL * 8); }

}  // namespace
}  // namespace disk

using namespace disk;

extern "C" int disk_learned_init(const float *d_targets, const int *sizes, int batch, int L,
                                 int T, const float *d_params, int side, int hidden, int depth,
                                 int loss, float eps, float *d_theta_out, int *d_used_network,
                                 void *stream) {
  if (!d_targets || !sizes || !d_params || !d_theta_out)
    return fail(DISK_ERR_INVALID_ARG, "null pointer");
  if (batch < 1 || L < 1 || L > DISK_MAX_LAYERS || T < 1 || T > DISK_MAX_TAPS)
    return fail(DISK_ERR_INVALID_ARG, "batch >= 1, L in [1, 16], T in [1, 64] required");
  if (side < 1 || side > 1024) return fail(DISK_ERR_INVALID_ARG, "side in [1, 1024] required");
  const int per = L * T * 3, n_in = side * side;
  if (disk_mlp_param_count(n_in, hidden, depth, per) < 0)
    return fail(DISK_ERR_INVALID_ARG, "bad network shape");
  std::vector<float> scale(batch);
  for (int b = 0; b < batch; ++b) {
    if (sizes[b] < 1 || (sizes[b] & 1) == 0) return fail(DISK_ERR_INVALID_ARG, "target sizes must be odd");
    scale[b] = std::max(1.0f, (float)((sizes[b] - 1) / 2));
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // scratch: features, network outputs, both starts, their losses, one
  // gradient plane (the loss evaluation writes it), the scale table
  const size_t nB = (size_t)batch;
  const size_t floats = nB * n_in + 4 * nB * per + 2 * nB + nB;
  float *buf = nullptr;
  DISK_TRY_CUDA(scratch_alloc(&buf, floats * sizeof(float), s), "scratch_alloc(learned init)");
  float *X = buf, *Y = X + nB * n_in, *th_net = Y + nB * per, *th_ir = th_net + nB * per;
  float *grad = th_ir + nB * per, *l_net = grad + nB * per, *l_ir = l_net + nB;
  float *d_scale = l_ir + nB;
  int rc = disk_downsample_targets(d_targets, sizes, batch, side, X, stream);
  if (rc == DISK_OK) rc = disk_mlp_forward(d_params, n_in, hidden, depth, per, X, batch, Y, stream);
  if (rc == DISK_OK) {
    // small host table: a pageable copy returns once the data is staged
    cudaError_t e = cudaMemcpyAsync(d_scale, scale.data(), nB * sizeof(float),
                                    cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
      const long long n = (long long)nB * per;
      unscale_kernel<<<grid_for(n), 256, 0, s>>>(Y, d_scale, per, (float)T, n, th_net);
      e = cudaGetLastError();
    }
    if (e != cudaSuccess) rc = cuda_fail(e, "learned init: un-scaling");
  }
  if (rc == DISK_OK)
    rc = disk_fit(d_targets, sizes, batch, L, T, 0, 0.f, 0.f, DISK_INIT_IR, loss, eps, 0, th_ir,
                  nullptr, nullptr, stream);
  if (rc == DISK_OK)
    rc = disk_fit_loss_grad(d_targets, sizes, batch, L, T, loss, eps, th_net, l_net, grad, stream);
  if (rc == DISK_OK)
    rc = disk_fit_loss_grad(d_targets, sizes, batch, L, T, loss, eps, th_ir, l_ir, grad, stream);
  if (rc == DISK_OK) {
    const long long n = (long long)nB * per;
    choose_kernel<<<grid_for(n), 256, 0, s>>>(th_net, th_ir, l_net, l_ir, per, n, d_theta_out,
                                              d_used_network);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) rc = cuda_fail(e, "learned init: choice");
  }
  cudaFreeAsync(buf, s);
  return rc;
}
