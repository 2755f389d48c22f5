// Learned initializer of the fit: a multilayer perceptron from an area-
// resampled target kernel (side x side, scaled to a maximum of 1) to the
// L x T x 3 parameters of a complex (offsets in units of the target
// half-width, weights raw), with hand-written training and inference
// kernels.  The paper has no such network; it serves the fit of Sec. 4.1
// as a better starting point than the Eq. 6 / Eq. 7 initialisations.
//
// Parameters: for each layer, W [n_in][n_out] row-major then b [n_out];
// hidden layers ReLU, output linear.  Matrix products run in a tiled FP32
// SIMT GEMM (64 x 64 tile, 16-deep K slices in shared memory, 4 x 4 outputs
// per thread) whose epilogue adds the bias, applies ReLU, or multiplies by
// the ReLU mask of the backward pass; products whose tile grid cannot fill
// the GPU split K and sum the slices (in a fixed order) before the epilogue.
// Products of 2^24 multiply-adds and more (all of the benchmark network's)
// run on the tensor cores instead (tc_gemm.cuh: four TF32 products, FP32
// accuracy) with the same split-K reduction and epilogue.
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.h"
#include "tc_gemm.cuh"

namespace disk {
namespace {

constexpr int kBM = 64, kBN = 64, kBK = 16, kGemmThreads = 256;

enum Epi : int { EPI_NONE = 0, EPI_BIAS_RELU = 1, EPI_BIAS = 2, EPI_RELU_MASK = 3 };

// C[M][N] = op(A) op(B); op(A)[m][k] = TA ? A[k*lda + m] : A[m*lda + k],
// op(B)[k][n] = TB ? B[n*ldb + k] : B[k*ldb + n].
template <bool TA, bool TB, int EPI>
__global__ void __launch_bounds__(kGemmThreads)
gemm_kernel(const float *__restrict__ A, const float *__restrict__ B, float *__restrict__ C, int M,
            int N, int K, int lda, int ldb, int ldc, const float *__restrict__ bias,
            const float *__restrict__ mask, int ldm, int kchunk, long long cz) {
  __shared__ float As[kBK][kBM + 4];
  __shared__ float Bs[kBK][kBN + 4];
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * kBN;
  // split-K: blockIdx.z takes k in [kb, K') and writes its own slice of C
  const int kb = blockIdx.z * kchunk;
  K = min(K, kb + kchunk);
  C += blockIdx.z * cz;
  float acc[4][4] = {};
  for (int k0 = kb; k0 < K; k0 += kBK) {
    for (int e = tid; e < kBM * kBK; e += kGemmThreads) {
      int mm, kk;
      if (TA) { mm = e % kBM; kk = e / kBM; } else { kk = e % kBK; mm = e / kBK; }
      const int m = m0 + mm, k = k0 + kk;
      float v = 0.f;
      if (m < M && k < K) v = TA ? A[(long long)k * lda + m] : A[(long long)m * lda + k];
      As[kk][mm] = v;
    }
    for (int e = tid; e < kBN * kBK; e += kGemmThreads) {
      int nn, kk;
      if (TB) { kk = e % kBK; nn = e / kBK; } else { nn = e % kBN; kk = e / kBN; }
      const int n = n0 + nn, k = k0 + kk;
      float v = 0.f;
      if (n < N && k < K) v = TB ? B[(long long)n * ldb + k] : B[(long long)k * ldb + n];
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kBK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty * 4 + i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx * 4 + j;
      if (n >= N) continue;
      float v = acc[i][j];
      if (EPI == EPI_BIAS_RELU) v = fmaxf(v + bias[n], 0.f);
      if (EPI == EPI_BIAS) v += bias[n];
      if (EPI == EPI_RELU_MASK) v = mask[(long long)m * ldm + n] > 0.f ? v : 0.f;
      C[(long long)m * ldc + n] = v;
    }
  }
}

// Sum of the split-K slices ws[z * zs + m * ldw + n] in slice order, then
// the epilogue.
template <int EPI>
__global__ void splitk_reduce_kernel(const float *__restrict__ ws, int splits, long long zs,
                                     int ldw, int M, int N, float *__restrict__ C, int ldc,
                                     const float *__restrict__ bias,
                                     const float *__restrict__ mask, int ldm) {
  const long long MN = (long long)M * N;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < MN;
       i += (long long)gridDim.x * blockDim.x) {
    const int m = (int)(i / N), n = (int)(i % N);
    const long long w = (long long)m * ldw + n;
    float v = 0.f;
    for (int z = 0; z < splits; ++z) v += ws[z * zs + w];
    if (EPI == EPI_BIAS_RELU) v = fmaxf(v + bias[n], 0.f);
    if (EPI == EPI_BIAS) v += bias[n];
    if (EPI == EPI_RELU_MASK) v = mask[(long long)m * ldm + n] > 0.f ? v : 0.f;
    C[(long long)m * ldc + n] = v;
  }
}

constexpr int kGemmFillCtas = 2 * 152;  // about two waves of CTAs over the SMs

// Products of at least this many multiply-adds run on the tensor cores.
constexpr long long kTcMinMacs = 1ll << 24;

template <bool TA, bool TB, int EPI>
int gemm(const float *A, const float *B, float *C, int M, int N, int K, int lda, int ldb, int ldc,
         const float *bias, const float *mask, int ldm, cudaStream_t s) {
  if ((long long)M * N * K >= kTcMinMacs) {
    float *ws = nullptr;
    int Mp = 0, Np = 0, rc = DISK_OK;
    const int splits = tc::gemm_slices<TA, TB>(A, B, M, N, K, lda, ldb, &ws, &Mp, &Np, &rc, s);
    if (!splits) return rc;
    const long long MN = (long long)M * N;
    const int blocks = (int)std::min<long long>((MN + 255) / 256, 152LL * 8);
    splitk_reduce_kernel<EPI><<<blocks, 256, 0, s>>>(ws, splits, (long long)Mp * Np, Np, M, N, C,
                                                     ldc, bias, mask, ldm);
    const cudaError_t e = cudaGetLastError();
    cudaFreeAsync(ws, s);
    if (e != cudaSuccess) return cuda_fail(e, "launch tensor-core reduce");
    return DISK_OK;
  }
  dim3 grid((N + kBN - 1) / kBN, (M + kBM - 1) / kBM);
  // a tile grid too small to fill the GPU splits K (slices of >= 128) and
  // sums the slices in a second pass
  int splits = 1;
  while ((long long)grid.x * grid.y * splits < kGemmFillCtas && K / (2 * splits) >= 128) splits *= 2;
  if (splits == 1) {
    gemm_kernel<TA, TB, EPI><<<grid, kGemmThreads, 0, s>>>(A, B, C, M, N, K, lda, ldb, ldc, bias,
                                                           mask, ldm, K, 0);
    DISK_TRY_CUDA(cudaGetLastError(), "launch gemm_kernel");
    return DISK_OK;
  }
  const int kchunk = ((K + splits - 1) / splits + kBK - 1) / kBK * kBK;
  const long long MN = (long long)M * N;
  float *ws = nullptr;
  DISK_TRY_CUDA(scratch_alloc(&ws, (size_t)splits * MN * sizeof(float), s), "scratch_alloc(split-K)");
  grid.z = splits;
  gemm_kernel<TA, TB, EPI_NONE><<<grid, kGemmThreads, 0, s>>>(A, B, ws, M, N, K, lda, ldb, N,
                                                              nullptr, nullptr, 0, kchunk, MN);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) {
    const int blocks = (int)std::min<long long>((MN + 255) / 256, 152LL * 8);
    splitk_reduce_kernel<EPI><<<blocks, 256, 0, s>>>(ws, splits, MN, N, M, N, C, ldc, bias, mask,
                                                     ldm);
    e = cudaGetLastError();
  }
  cudaFreeAsync(ws, s);
  if (e != cudaSuccess) return cuda_fail(e, "launch split-K gemm");
  return DISK_OK;
}

// db[n] = sum_m D[m][n]
__global__ void colsum_kernel(const float *D, float *db, int M, int N) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float s = 0.f;
  for (int m = 0; m < M; ++m) s += D[(long long)m * N + n];
  db[n] = s;
}

// MSE over the batch and outputs: loss (stored to *loss) and
// dY = 2 (y - t) / (M N).  One block (launched with kMseThreads threads), so
// the sum is taken in a fixed order and the loss is reproducible bit for bit.
constexpr int kMseThreads = 1024;
__global__ void __launch_bounds__(kMseThreads) mse_kernel(const float *y, const float *t,
                                                          float *dy, long long n, float *loss) {
  __shared__ float red[32];
  float part = 0.f;
  const float inv = 1.f / (float)n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float d = y[i] - t[i];
    dy[i] = 2.f * d * inv;
    part += d * d * inv;
  }
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    *loss = s;
  }
}

// Adam (Kingma & Ba 2015), step counted from 1.
__global__ void adam_kernel(float *p, float *m, float *v, const float *g, long long n, float lr,
                            float c1, float c2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = 0.9f * m[i] + 0.1f * gi, vi = 0.999f * v[i] + 0.001f * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
  }
}

// He-uniform weights U(-sqrt(6/n_in), sqrt(6/n_in)) from SplitMix64 (Steele,
// Lea & Flood 2014) at counter seed + element index; zero biases.
__global__ void mlp_init_kernel(float *p, long long off, long long nw, long long nb, float lim,
                                unsigned long long seed) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nw + nb;
       i += (long long)gridDim.x * blockDim.x) {
    float v = 0.f;
    if (i < nw) {
      unsigned long long z = seed + (unsigned long long)(off + i + 1) * 0x9E3779B97F4A7C15ull;
      z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
      z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
      z ^= z >> 31;
      const double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);
      v = (float)((2.0 * u - 1.0) * lim);
    }
    p[off + i] = v;
  }
}

// Area resampling of target b (K x K) to side x side: each output cell
// [j s, (j+1) s) x [i s, (i+1) s), s = K / side, averages the input pixels
// it overlaps weighted by overlap area; then the block is scaled to a
// maximum of 1.
__global__ void downsample_kernel(const float *targets, const long long *offs, const int *sizes,
                                  int side, float *out) {
  __shared__ float red[32];
  const int b = blockIdx.x, K = sizes[b];
  const float *t = targets + offs[b];
  float *o = out + (long long)b * side * side;
  const float s = (float)K / side;
  float mx = 0.f;
  for (int e = threadIdx.x; e < side * side; e += blockDim.x) {
    const int j = e / side, i = e % side;
    const float y0 = j * s, y1 = (j + 1) * s, x0 = i * s, x1 = (i + 1) * s;
    float acc = 0.f;
    for (int p = (int)floorf(y0); p < min(K, (int)ceilf(y1)); ++p) {
      const float wy = fminf(y1, p + 1.f) - fmaxf(y0, (float)p);
      if (wy <= 0.f) continue;
      for (int q = (int)floorf(x0); q < min(K, (int)ceilf(x1)); ++q) {
        const float wx = fminf(x1, q + 1.f) - fmaxf(x0, (float)q);
        if (wx > 0.f) acc += wy * wx * t[p * K + q];
      }
    }
    acc /= s * s;
    o[e] = acc;
    mx = fmaxf(mx, acc);
  }
  for (int w = 16; w > 0; w >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, w));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  float m = 0.f;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, red[w]);
  if (m > 0.f)
    for (int e = threadIdx.x; e < side * side; e += blockDim.x) o[e] /= m;
}

struct Shape {
  int n_in, hidden, depth, n_out;
  int layers() const { return depth + 1; }
  int din(int i) const { return i == 0 ? n_in : hidden; }
  int dout(int i) const { return i == depth ? n_out : hidden; }
  long long count() const {
    long long c = 0;
    for (int i = 0; i < layers(); ++i) c += (long long)din(i) * dout(i) + dout(i);
    return c;
  }
  long long woff(int i) const {
    long long c = 0;
    for (int j = 0; j < i; ++j) c += (long long)din(j) * dout(j) + dout(j);
    return c;
  }
};

int check_shape(const Shape &sh) {
  if (sh.n_in < 1 || sh.hidden < 1 || sh.depth < 0 || sh.depth > 16 || sh.n_out < 1 ||
      sh.n_in > 65536 || sh.hidden > 16384 || sh.n_out > 16384)
    return fail(DISK_ERR_INVALID_ARG, "bad MLP shape");
  return DISK_OK;
}

// Forward pass; acts (may be null for inference) receives each layer's
// output: rows of hidden, ..., hidden, n_out for the batch.
int mlp_forward(const Shape &sh, const float *P, const float *x, int B, float *y, float *acts,
                float *ping, cudaStream_t s) {
  const float *h = x;
  for (int i = 0; i < sh.layers(); ++i) {
    const float *W = P + sh.woff(i), *b = W + (long long)sh.din(i) * sh.dout(i);
    float *dst;
    if (i == sh.depth) dst = y;
    else if (acts) dst = acts + (long long)i * B * sh.hidden;
    else dst = ping + (long long)(i & 1) * B * sh.hidden;
    const int rc = i == sh.depth
        ? gemm<false, false, EPI_BIAS>(h, W, dst, B, sh.dout(i), sh.din(i), sh.din(i), sh.dout(i), sh.dout(i), b, nullptr, 0, s)
        : gemm<false, false, EPI_BIAS_RELU>(h, W, dst, B, sh.dout(i), sh.din(i), sh.din(i), sh.dout(i), sh.dout(i), b, nullptr, 0, s);
    if (rc) return rc;
    h = dst;
  }
  return DISK_OK;
}

}  // namespace
}  // namespace disk

using namespace disk;

extern "C" long long disk_mlp_param_count(int n_in, int hidden, int depth, int n_out) {
  const Shape sh{n_in, hidden, depth, n_out};
  if (check_shape(sh)) return -1;
  return sh.count();
}

extern "C" int disk_mlp_init(float *d_params, int n_in, int hidden, int depth, int n_out,
                             uint64_t seed, void *stream) {
  const Shape sh{n_in, hidden, depth, n_out};
  int rc = check_shape(sh);
  if (rc) return rc;
  if (!d_params) return fail(DISK_ERR_INVALID_ARG, "null params");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  for (int i = 0; i < sh.layers(); ++i) {
    const long long nw = (long long)sh.din(i) * sh.dout(i);
    mlp_init_kernel<<<256, 256, 0, s>>>(d_params, sh.woff(i), nw, sh.dout(i),
                                        sqrtf(6.f / sh.din(i)), seed);
    DISK_TRY_CUDA(cudaGetLastError(), "launch mlp_init_kernel");
  }
  return DISK_OK;
}

extern "C" int disk_mlp_forward(const float *d_params, int n_in, int hidden, int depth, int n_out,
                                const float *d_x, int batch, float *d_y, void *stream) {
  const Shape sh{n_in, hidden, depth, n_out};
  int rc = check_shape(sh);
  if (rc) return rc;
  if (!d_params || !d_x || !d_y || batch < 1) return fail(DISK_ERR_INVALID_ARG, "bad arguments");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  float *ping = nullptr;
  if (sh.depth > 0)
    DISK_TRY_CUDA(scratch_alloc(reinterpret_cast<void **>(&ping), 2ull * batch * sh.hidden * sizeof(float), s),
                  "scratch_alloc(mlp forward)");
  rc = mlp_forward(sh, d_params, d_x, batch, d_y, nullptr, ping, s);
  if (ping) cudaFreeAsync(ping, s);
  return rc;
}

namespace disk {
namespace {

// Loss and gradient of one batch into grad (np floats); scratch from the pool.
int mlp_grad(const Shape &sh, const float *d_params, const float *d_x, const float *d_target,
             int batch, float *grad, float *d_loss, cudaStream_t s) {
  const long long nacts = (long long)batch * sh.hidden * sh.depth, ny = (long long)batch * sh.n_out;
  const long long wmax = std::max(sh.hidden, sh.n_out);
  const size_t bytes = sizeof(float) * (nacts + ny + 2 * batch * wmax);
  float *buf = nullptr;
  DISK_TRY_CUDA(scratch_alloc(reinterpret_cast<void **>(&buf), bytes, s), "scratch_alloc(mlp grad)");
  float *acts = buf, *y = acts + nacts, *d0 = y + ny, *d1 = d0 + batch * wmax;
  int rc = mlp_forward(sh, d_params, d_x, batch, y, acts, nullptr, s);
  cudaError_t e = cudaSuccess;
  if (rc == DISK_OK) {
    mse_kernel<<<1, kMseThreads, 0, s>>>(y, d_target, d0, ny, d_loss);
    e = cudaGetLastError();
    if (e != cudaSuccess) rc = cuda_fail(e, "mse");
  }
  // backward: d holds dL/d(output of layer i)
  float *d = d0, *dn = d1;
  for (int i = sh.depth; i >= 0 && rc == DISK_OK; --i) {
    const int ni = sh.din(i), no = sh.dout(i);
    const float *hin = i == 0 ? d_x : acts + (long long)(i - 1) * batch * sh.hidden;
    float *gW = grad + sh.woff(i), *gb = gW + (long long)ni * no;
    rc = gemm<true, false, EPI_NONE>(hin, d, gW, ni, no, batch, ni, no, no, nullptr, nullptr, 0, s);
    if (rc) break;
    colsum_kernel<<<(no + 255) / 256, 256, 0, s>>>(d, gb, batch, no);
    e = cudaGetLastError();
    if (e != cudaSuccess) { rc = cuda_fail(e, "colsum"); break; }
    if (i > 0) {
      const float *W = d_params + sh.woff(i);
      rc = gemm<false, true, EPI_RELU_MASK>(d, W, dn, batch, ni, no, no, no, ni, nullptr, hin, ni, s);
      float *t = d; d = dn; dn = t;
    }
  }
  cudaFreeAsync(buf, s);
  return rc;
}

int mlp_adam(long long np, float *d_params, float *d_m, float *d_v, const float *grad, int step,
             float lr, cudaStream_t s) {
  const float c1 = 1.f - powf(0.9f, (float)step), c2 = 1.f - powf(0.999f, (float)step);
  adam_kernel<<<1216, 256, 0, s>>>(d_params, d_m, d_v, grad, np, lr, c1, c2);
  DISK_TRY_CUDA(cudaGetLastError(), "adam");
  return DISK_OK;
}

}  // namespace
}  // namespace disk

extern "C" int disk_mlp_train_step(float *d_params, float *d_m, float *d_v, int step, float lr,
                                   int n_in, int hidden, int depth, int n_out, const float *d_x,
                                   const float *d_target, int batch, float *d_loss, void *stream) {
  const Shape sh{n_in, hidden, depth, n_out};
  int rc = check_shape(sh);
  if (rc) return rc;
  if (!d_params || !d_m || !d_v || !d_x || !d_target || !d_loss || batch < 1 || step < 1)
    return fail(DISK_ERR_INVALID_ARG, "bad arguments");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const long long np = sh.count();
  float *grad = nullptr;
  DISK_TRY_CUDA(scratch_alloc(reinterpret_cast<void **>(&grad), sizeof(float) * np, s),
                "scratch_alloc(mlp train)");
  rc = mlp_grad(sh, d_params, d_x, d_target, batch, grad, d_loss, s);
  if (rc == DISK_OK) rc = mlp_adam(np, d_params, d_m, d_v, grad, step, lr, s);
  cudaFreeAsync(grad, s);
  return rc;
}

extern "C" int disk_mlp_grad(const float *d_params, int n_in, int hidden, int depth, int n_out,
                             const float *d_x, const float *d_target, int batch, float *d_grad,
                             float *d_loss, void *stream) {
  const Shape sh{n_in, hidden, depth, n_out};
  int rc = check_shape(sh);
  if (rc) return rc;
  if (!d_params || !d_x || !d_target || !d_grad || !d_loss || batch < 1)
    return fail(DISK_ERR_INVALID_ARG, "bad arguments");
  return mlp_grad(sh, d_params, d_x, d_target, batch, d_grad, d_loss,
                  static_cast<cudaStream_t>(stream));
}

extern "C" int disk_mlp_adam(float *d_params, float *d_m, float *d_v, const float *d_grad,
                             int step, float lr, int n_in, int hidden, int depth, int n_out,
                             void *stream) {
  const Shape sh{n_in, hidden, depth, n_out};
  int rc = check_shape(sh);
  if (rc) return rc;
  if (!d_params || !d_m || !d_v || !d_grad || step < 1)
    return fail(DISK_ERR_INVALID_ARG, "bad arguments");
  return mlp_adam(sh.count(), d_params, d_m, d_v, d_grad, step, lr,
                  static_cast<cudaStream_t>(stream));
}

extern "C" int disk_downsample_targets(const float *d_targets, const int *sizes, int batch,
                                       int side, float *d_out, void *stream) {
  if (!d_targets || !sizes || !d_out || batch < 1 || side < 1 || side > 1024)
    return fail(DISK_ERR_INVALID_ARG, "bad arguments");
  std::vector<long long> offs(batch);
  long long o = 0;
  for (int b = 0; b < batch; ++b) {
    if (sizes[b] < 1 || sizes[b] > 4096) return fail(DISK_ERR_INVALID_ARG, "bad target size");
    offs[b] = o;
    o += (long long)sizes[b] * sizes[b];
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char *buf = nullptr;
  const size_t bytes = batch * (sizeof(long long) + sizeof(int));
  DISK_TRY_CUDA(scratch_alloc(reinterpret_cast<void **>(&buf), bytes, s), "scratch_alloc(downsample)");
  // small host tables: a pageable copy returns once the data is staged
  cudaError_t e = cudaMemcpyAsync(buf, offs.data(), batch * sizeof(long long), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(buf + batch * sizeof(long long), sizes, batch * sizeof(int), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    downsample_kernel<<<batch, 256, 0, s>>>(d_targets, reinterpret_cast<long long *>(buf),
                                            reinterpret_cast<int *>(buf + batch * sizeof(long long)), side,
                                            d_out);
    e = cudaGetLastError();
  }
  cudaFreeAsync(buf, s);
  if (e != cudaSuccess) return cuda_fail(e, "downsample");
  return DISK_OK;
}
