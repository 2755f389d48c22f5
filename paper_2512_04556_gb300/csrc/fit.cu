// Differentiable fit of sparse complexes to dense targets (Sec. 4.1 Eq. 4-6,
// Sec. 4.2 Eq. 7, Sec. 4.4 Eq. 10-11, schedule of Sec. 5.1), batched over
// targets of uneven size in one persistent launch.
//
// One CTA -- or one thread-block cluster of CL CTAs on CL SMs -- owns one
// target for all steps (targets ordered largest first, so the block
// scheduler runs them longest-processing-time first).  In a cluster every
// canvas sweep is split over the cluster's threads, the canvases stay in
// global memory, cluster barriers order the sweeps, and the loss and tap
// gradients are summed across the CTAs through distributed shared memory in a
// fixed order, so every CTA applies the same Adam update.  Per step:
//   forward   impulse on a zero-padded canvas, L shift-invariant layers, each
//             computed only on its support box S_l = H_1 + ... + H_l, with
//             H_l = ceil(max |o_l|) + 1 from the current taps; the first
//             layer in closed form (its output is T bilinear splats);
//   loss      MSE (or Charbonnier, Eq. 11) over the plane, target zero-padded;
//   backward  dL/dI_L, then per layer the tap gradients (one warp per pair
//             of taps, warp-shuffle reductions) and the adjoint plane, which on a
//             zero-bounded canvas is the same layer applied at -o (the
//             bilinear tent is symmetric) -- a gather, no atomics; the
//             first layer's tap gradients in closed form from the four pixels
//             per tap where its sums are non-zero, the second layer's as sums
//             over the first layer's <= 4T non-zero output pixels;
//   update    Adam with linearly decayed lr on offsets in units of the target
//             half-width s (clamped to |o/s| <= 1) and raw weights.
// All L+1 activations stay in a per-target scratch region (L2-resident for
// all but the largest targets); the canvas half-width bounds every support
// the clamp allows.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <tuple>
#include <vector>

#include <cooperative_groups.h>

#include "canvas.cuh"

namespace disk {
namespace {

constexpr int kFitThreads = 512;      // init kernel and default fit CTA size
constexpr int kFitWarps = kFitThreads / 32;
constexpr int kFitMaxWarps = 32;      // largest fit CTA: 1024 threads
constexpr int kFitMaxCluster = 4;     // CTAs per target

struct FitMeta {
  long long tgt_off;     // floats into the packed targets
  long long canvas_off;  // floats into scratch
  long long idx_off;     // ints into the index scratch (sparse-sampling init)
  int K, R;
  float s;               // offset scale: max(1, (K-1)/2)
};

struct FitArgs {
  const float *targets;
  const FitMeta *meta;
  const int *order;
  float *scratch;
  int *idx_scratch;
  float *theta;          // [batch][L][T][3], pixels
  float *loss_out;       // [batch] final loss (may be null)
  float *loss_hist;      // [batch][steps + 1] (may be null)
  float *grad_out;       // [batch][L][T][3] (loss-and-gradient mode only)
  float *state;          // [batch][3][L*T*3]: q, Adam m, Adam v (may be null)
  int batch, L, T, steps, loss_kind, mode;  // mode 0 = fit, 1 = loss and gradient
  int step0, total;      // this call runs steps step0 .. step0+steps-1 of total
  float eps, lr0, lr1;
};

// ---- block reductions ------------------------------------------------------

__device__ __forceinline__ float warp_sum(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ float block_sum(float v, float *red) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  float r = 0.f;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r += red[w];
  __syncthreads();
  return r;
}

__device__ double block_sum_d(double v, double *red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double r = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r += red[w];
  __syncthreads();
  return r;
}

// ---- SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) ------------------------

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long &st) {
  unsigned long long z = (st += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// ---- initialisation ---------------------------------------------------------

// Eq. 6 rings for layers l0..L-1: radius (l - l0 + 1) dr, angle 2 pi i / T
// (i = 1..T), weight 1/T.
__device__ void write_rings(float *th, int L, int T, int l0, double dr) {
  for (int j = threadIdx.x; j < (L - l0) * T; j += blockDim.x) {
    const int l = l0 + j / T, i = j % T;
    const double r = (l - l0 + 1) * dr;
    const double ang = 2.0 * M_PI * (double)(i + 1) / (double)T;
    float *t = th + ((size_t)l * T + i) * 3;
    t[0] = (float)(r * cos(ang));
    t[1] = (float)(r * sin(ang));
    t[2] = (float)(1.0 / T);
  }
}

__global__ void __launch_bounds__(kFitThreads)
fit_init_kernel(FitArgs A, int init, unsigned long long seed) {
  __shared__ double red[kFitWarps];
  __shared__ int scan[kFitThreads];
  __shared__ float acc_x[DISK_MAX_TAPS], acc_y[DISK_MAX_TAPS];
  __shared__ int total;
  const int b = blockIdx.x;
  const FitMeta m = A.meta[b];
  const int K = m.K, h = (K - 1) / 2, KK = K * K, L = A.L, T = A.T;
  const float *tgt = A.targets + m.tgt_off;
  float *th = A.theta + (size_t)b * L * T * 3;
  if (init == 0) return;  // given
  if (init == 3) {        // random: offsets uniform in [-h/L, h/L], weights 1/T
    if (threadIdx.x == 0) {
      unsigned long long st = seed;
      const double sc = ((K - 1) / 2.0) / L;
      for (int j = 0; j < L * T; ++j) {
        const double u0 = (double)(splitmix64(st) >> 11) * (1.0 / 9007199254740992.0);
        const double u1 = (double)(splitmix64(st) >> 11) * (1.0 / 9007199254740992.0);
        th[3 * j] = (float)((2.0 * u0 - 1.0) * sc);
        th[3 * j + 1] = (float)((2.0 * u1 - 1.0) * sc);
        th[3 * j + 2] = (float)(1.0 / T);
      }
    }
    return;
  }
  // Sparse sampling needs the non-zero pixels in row-major order: an ordered
  // compaction (per-thread contiguous chunks, exclusive scan of the counts).
  long long S = 0;
  if (init == 2) {
    const int per = (KK + blockDim.x - 1) / blockDim.x;
    const int j0 = min((int)threadIdx.x * per, KK), j1 = min(j0 + per, KK);
    int c = 0;
    for (int j = j0; j < j1; ++j) c += tgt[j] > 0.f;
    scan[threadIdx.x] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
      int run = 0;
      for (int t = 0; t < (int)blockDim.x; ++t) { const int v = scan[t]; scan[t] = run; run += v; }
      total = run;
    }
    __syncthreads();
    int pos = scan[threadIdx.x];
    int *idx = A.idx_scratch + m.idx_off;
    for (int j = j0; j < j1; ++j)
      if (tgt[j] > 0.f) idx[pos++] = j;
    __syncthreads();
    S = total;
  }
  if (init == 1 || S == 0) {
    // Eq. 6 step matching the target's per-axis second moment
    double s0 = 0, sx = 0, sy = 0;
    for (int j = threadIdx.x; j < KK; j += blockDim.x) {
      const double t = tgt[j];
      s0 += t; sx += t * (j % K); sy += t * (j / K);
    }
    s0 = block_sum_d(s0, red); sx = block_sum_d(sx, red); sy = block_sum_d(sy, red);
    double sig = 1.0;
    if (s0 > 0) {
      const double mx = sx / s0, my = sy / s0;
      double var = 0;
      for (int j = threadIdx.x; j < KK; j += blockDim.x) {
        const double t = tgt[j], dx = (j % K) - mx, dy = (j / K) - my;
        var += t * (dx * dx + dy * dy);
      }
      var = block_sum_d(var, red);
      sig = sqrt(var / (2.0 * s0));
    }
    write_rings(th, L, T, 0, sig * sqrt(12.0 / ((double)L * (L + 1) * (2 * L + 1))));
    return;
  }
  // Sec. 4.2 sparse sampling: dart throwing over the non-zero pixels with the
  // Eq. 7 radius, one thread, the same decisions as any exact implementation.
  const double r0sq = (double)S / ((double)T * M_PI);
  if (threadIdx.x == 0) {
    const int *idx = A.idx_scratch + m.idx_off;
    double r2 = r0sq;
    int acc = 0, fails = 0;
    unsigned long long st = seed;
    long long guard = 0;
    while (acc < T && guard < (1ll << 26)) {
      ++guard;
      const unsigned long long z = splitmix64(st);
      const int p = idx[z % (unsigned long long)S];
      const double qx = (double)(p % K - h), qy = (double)(p / K - h);
      bool ok = true;
      for (int a = 0; a < acc && ok; ++a) {
        const double ddx = qx - acc_x[a], ddy = qy - acc_y[a];
        if (ddx * ddx + ddy * ddy < r2) ok = false;
      }
      if (ok) { acc_x[acc] = (float)qx; acc_y[acc] = (float)qy; ++acc; fails = 0; }
      else if (++fails >= 30 * T) { r2 *= 0.81; fails = 0; if (r2 < 0.25) r2 = 0.0; }
    }
    for (; acc < T; ++acc) { acc_x[acc] = 0.f; acc_y[acc] = 0.f; }  // guard tripped
  }
  __syncthreads();
  for (int i = threadIdx.x; i < T; i += blockDim.x) {
    th[3 * i] = -acc_x[i];
    th[3 * i + 1] = -acc_y[i];
    th[3 * i + 2] = (float)(1.0 / T);
  }
  if (L > 1) {
    double sj = 0;
    for (int j = 1; j < L; ++j) sj += (double)j * j;
    write_rings(th, L, T, 1, sqrt(r0sq) / sqrt(2.0 * sj));
  }
}

// ---- the persistent fit ------------------------------------------------------

constexpr int kFitMaxTaps = 512;  // L * T limit of the fitter (static shared state)

struct FitShared {
  float4 taps[kFitMaxTaps];
  float q[kFitMaxTaps * 3];
  float mo[kFitMaxTaps * 3];
  float vo[kFitMaxTaps * 3];
  float g[kFitMaxTaps * 3];
  LayerExtent ext[DISK_MAX_LAYERS];
  PreparedTaps pt;  // the layer being swept
  float red[kFitMaxWarps];
  float closs;  // this CTA's share of the loss
  // the first layer's non-zero output pixels (closed form, rank 0 only)
  int splat_pix[4 * DISK_MAX_TAPS];
  float splat_val[4 * DISK_MAX_TAPS];
  int nsplat;
  // per-(chunk, tap) partial tap gradients of the warps of this CTA, two
  // buffers used by alternate layers
  static constexpr int kPart = 6 * (kFitMaxWarps * kFitMaxCluster > DISK_MAX_TAPS
                                        ? kFitMaxWarps * kFitMaxCluster
                                        : DISK_MAX_TAPS);
  float part[2 * kPart];
};

namespace cg = cooperative_groups;

// Barrier over the CTAs that share a target; a plain block barrier when
// CL == 1.  The cluster barrier's arrive has release and its wait acquire
// semantics at cluster scope, which orders the CTAs' global canvas writes
// before the other CTAs' reads with no separate fence.
template <int CL>
__device__ __forceinline__ void target_sync() {
  if (CL == 1) {
    __syncthreads();
  } else {
    cg::this_cluster().sync();
  }
}

template <int CL>
__device__ __forceinline__ unsigned target_rank() {
  if (CL == 1) return 0;
  return cg::this_cluster().block_rank();
}

// Address of *p in the shared memory of CTA r of the cluster.
template <int CL>
__device__ __forceinline__ const float *rank_ptr(const float *p, unsigned r) {
  if (CL == 1) return p;
  return cg::this_cluster().map_shared_rank(const_cast<float *>(p), r);
}

// taps (pixels) from normalised parameters; layer extents from the taps.
__device__ void make_taps(FitShared &sh, int L, int T, float s) {
  for (int j = threadIdx.x; j < L * T; j += blockDim.x)
    sh.taps[j] = make_float4(sh.q[3 * j] * s, sh.q[3 * j + 1] * s, sh.q[3 * j + 2], 0.f);
  __syncthreads();
  if (threadIdx.x < 32) {
    int S = 0;
    for (int l = 0; l < L; ++l) {
      float mx = 0.f;
      for (int i = threadIdx.x; i < T; i += 32)
        mx = fmaxf(mx, fmaxf(fabsf(sh.taps[l * T + i].x), fabsf(sh.taps[l * T + i].y)));
      for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      const int H = (int)ceilf(mx) + 1;
      S += H;
      if (threadIdx.x == 0) { sh.ext[l].H = H; sh.ext[l].S = S; }
    }
  }
  __syncthreads();
}

// The first layer of the cascade in closed form.  Its input is the unit
// impulse at the centre c, so the gather dst[p] = sum_i w_i bilinear(I_0,
// p + o_i) is non-zero only at the four pixels p = c - n_i - e of every tap
// (n_i the clamped floor of o_i, e in {0, 1}^2 the corner of the bilinear
// footprint that lands on c), where it receives the tap's corner weight; a
// pixel that several taps reach gets their sum in tap order, as the gather
// forms it.  The plane act[1] is therefore kept zero except at these <= 4T
// pixels: it is zeroed once when the fit starts, and every step clears the
// previous step's pixels before it writes the new ones.  Every CTA builds the
// list (entry k = 4i + e: pixel splat_pix[k], and in splat_val[k] the pixel's
// value at its first entry, 0 at repeated ones); only the CTA with `write`
// (the cluster's rank 0) writes the plane, which the caller's barrier
// publishes.  One entry per thread: every fit CTA has at least
// 4 * DISK_MAX_TAPS threads.
__device__ void splat_first_layer(FitShared &sh, float *dst, int R, int T, bool write) {
  const int N = 2 * R + 1, n = 4 * T, k = threadIdx.x;
  prepare_taps(sh.pt, sh.taps, T, sh.ext[0].H, 1.f, R);
  if (write)
    for (int j = threadIdx.x; j < sh.nsplat; j += blockDim.x) dst[sh.splat_pix[j]] = 0.f;
  __syncthreads();
  if (k < n) {
    const int i = k >> 2, ex = k & 1, ey = (k >> 1) & 1;
    const float4 w = sh.pt.w[i];
    sh.splat_pix[k] = R * N + R - sh.pt.off[i] - ey * N - ex;
    sh.splat_val[k] = ey ? (ex ? w.w : w.z) : (ex ? w.y : w.x);
  }
  __syncthreads();
  float acc = 0.f;
  bool first = false;
  if (k < n) {
    const int p = sh.splat_pix[k];
    first = true;
    for (int j = 0; j < k && first; ++j) first = sh.splat_pix[j] != p;
    if (first) {
      for (int j = k; j < n; ++j)
        if (sh.splat_pix[j] == p) acc += sh.splat_val[j];
      if (write) dst[p] = acc;
    }
  }
  __syncthreads();
  if (k < n) sh.splat_val[k] = first ? acc : 0.f;
  if (k == 0) sh.nsplat = n;
}

// Tap gradients of the first layer in closed form.  With the impulse as the
// layer's input, the terms of the tap-gradient sums over the layer's box
// vanish except at the four pixels p = c - n_i - e of the tap, where the
// bilinear corner values are 1 at e and 0 at the other three corners.  The
// sums' factor dL/dI_1 at those pixels is G itself when L = 1, else the
// adjoint of the second layer applied to G = dL/dI_2 (sh.pt holding that
// layer's taps prepared at -o), evaluated only there.  Every CTA of a cluster
// computes all of them (the same arithmetic on the same data) into sh.g.
__device__ void first_layer_grads(FitShared &sh, const float *G, int R, int T, bool adjoint) {
  const int N = 2 * R + 1, n = 4 * T, halo = sh.ext[0].H;
  const int lanes = (n + 31) & ~31;  // whole warps: the shuffles below
  for (int k = threadIdx.x; k < lanes; k += blockDim.x) {
    const bool valid = k < n;
    const int i = valid ? k >> 2 : 0, ex = k & 1, ey = (k >> 1) & 1;
    const float4 t = sh.taps[i];
    float fx, fy;
    const int nx = min(max(split_floor(t.x, fx), -halo), halo - 1);
    const int ny = min(max(split_floor(t.y, fy), -halo), halo - 1);
    const int p = (R - ny - ey) * N + (R - nx - ex);
    float g = 0.f;
    if (valid) {
      if (adjoint) {
        for (int j = 0; j < T; ++j) {
          const float4 w = sh.pt.w[j];
          const float *q = G + p + sh.pt.off[j];
          g += w.x * q[0] + w.y * q[1] + w.z * q[N] + w.w * q[N + 1];
        }
      } else {
        g = G[p];
      }
    }
    // the sweep's expressions with the corner values (a, b; c, d)
    const float a = (ex == 0 && ey == 0) ? 1.f : 0.f, b = (ex == 1 && ey == 0) ? 1.f : 0.f;
    const float c = (ex == 0 && ey == 1) ? 1.f : 0.f, d = (ex == 1 && ey == 1) ? 1.f : 0.f;
    const float top = a + fx * (b - a), bot = c + fx * (d - c);
    float gw = g * (top + fy * (bot - top));
    float gdx = g * ((1.f - fy) * (b - a) + fy * (d - c));
    float gdy = g * (bot - top);
    // the tap's four pixels are lanes 4i .. 4i+3: summed in a fixed order
    for (int o = 1; o <= 2; o <<= 1) {
      gw += __shfl_xor_sync(0xffffffffu, gw, o);
      gdx += __shfl_xor_sync(0xffffffffu, gdx, o);
      gdy += __shfl_xor_sync(0xffffffffu, gdy, o);
    }
    if (valid && (k & 3) == 0) {
      sh.g[i * 3] = gdx * t.z;
      sh.g[i * 3 + 1] = gdy * t.z;
      sh.g[i * 3 + 2] = gw;
    }
  }
}

// Tap gradients of the second layer from its sparse input.  I_1 is zero
// except at the first layer's splat pixels y (values v_y, sh.splat_val), and
// every term of the tap-gradient sums is linear in the four bilinear corners
// (a, b; c, d) it reads, so the sums over the layer's box regroup as sums
// over y of v_y times G at the four pixels that read y as a, b, c or d
// (y - n_j, y - n_j - 1, y - n_j - N, y - n_j - N - 1).  G = dL/dI_2.
// One warp per tap; every CTA of a cluster computes all of them into sh.g.
__device__ void second_layer_grads(FitShared &sh, const float *G, int R, int T) {
  const int N = 2 * R + 1, n = 4 * T, halo = sh.ext[1].H;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = warp; j < T; j += nw) {
    const float4 t = sh.taps[T + j];
    float fx, fy;
    const int nx = min(max(split_floor(t.x, fx), -halo), halo - 1);
    const int ny = min(max(split_floor(t.y, fy), -halo), halo - 1);
    const int off = ny * N + nx;
    const float gx = 1.f - fx, gy = 1.f - fy;
    float gw = 0.f, gdx = 0.f, gdy = 0.f;
    for (int k = lane; k < n; k += 32) {
      const float v = sh.splat_val[k];
      const float *q = G + (sh.splat_pix[k] - off);
      const float ga = q[0], gb = q[-1], gc = q[-N], gd = q[-N - 1];
      gw += v * (gy * (gx * ga + fx * gb) + fy * (gx * gc + fx * gd));
      gdx += v * (gy * (gb - ga) + fy * (gd - gc));
      gdy += v * (gx * (gc - ga) + fx * (gd - gb));
    }
    gw = warp_sum(gw); gdx = warp_sum(gdx); gdy = warp_sum(gdy);
    if (lane == 0) {
      sh.g[(T + j) * 3] = gdx * t.z;
      sh.g[(T + j) * 3 + 1] = gdy * t.z;
      sh.g[(T + j) * 3 + 2] = gw;
    }
  }
}

// Forward cascade on planes act[0..L]; returns the loss and leaves dL/dI_L in
// gL (box of half-width max(S_L, h)).  Sweeps are split over the CL CTAs.
template <int CL>
__device__ float forward_loss(FitShared &sh, const FitArgs &A, const FitMeta &m, float *const *act,
                              float *gL, const float *tgt, unsigned rank) {
  const int L = A.L, T = A.T, R = m.R, N = 2 * R + 1, K = m.K, h = (K - 1) / 2;
  const int tid = (int)rank * blockDim.x + threadIdx.x, nthr = blockDim.x * CL;
  splat_first_layer(sh, act[1], R, T, rank == 0);
  target_sync<CL>();
  for (int l = 1; l < L; ++l) {
    const int S = sh.ext[l].S;
    prepare_taps(sh.pt, sh.taps + l * T, T, sh.ext[l].H, 1.f, R);
    __syncthreads();
    canvas_layer(act[l], act[l + 1], R, S, sh.pt, T, tid, nthr);
    const int reach = (l + 1 < L) ? S + 2 * sh.ext[l + 1].H : max(S, h);
    zero_frame(act[l + 1], R, S, reach, tid, nthr);  // disjoint from the layer's box
    target_sync<CL>();
  }
  const int bx = max(sh.ext[L - 1].S, h);
  const float inv = 1.f / ((float)K * (float)K);
  const float *KL = act[L];
  float part = 0.f;
  const int side = 2 * bx + 1;
  for (int j = tid; j < side * side; j += nthr) {
    const int v = j / side - bx, u = j % side - bx;
    const float t = (abs(v) <= h && abs(u) <= h) ? tgt[(v + h) * K + (u + h)] : 0.f;
    const float d = KL[(R + v) * N + (R + u)] - t;
    float g;
    if (A.loss_kind == 0) {
      part += d * d * inv;
      g = 2.f * d * inv;
    } else {
      const float sq = sqrtf(d * d + A.eps * A.eps);
      part += (sq - A.eps) * inv;
      g = d / sq * inv;
    }
    gL[(R + v) * N + (R + u)] = g;
  }
  part = block_sum(part, sh.red);
  if (threadIdx.x == 0) sh.closs = part;
  target_sync<CL>();
  float loss = 0.f;
  for (unsigned r = 0; r < (unsigned)CL; ++r) loss += *rank_ptr<CL>(&sh.closs, r);
  return loss;
}

// Tap gradients of every layer into sh.g (pixel units); ga/gb are the two
// adjoint planes (ga holds dL/dI_L on entry).
template <int CL>
__device__ void backward(FitShared &sh, const FitArgs &A, const FitMeta &m, float *const *act,
                         float *ga, float *gb, unsigned rank) {
  const int L = A.L, T = A.T, R = m.R, N = 2 * R + 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int nwt = nw * CL, gwarp = (int)rank * nw + warp;
  const int tid = (int)rank * blockDim.x + threadIdx.x, nthr = blockDim.x * CL;
  float *G = ga, *Gn = gb;
  for (int l = L - 1; l >= 2; --l) {  // the first two layers: closed forms, below
    const int S = sh.ext[l].S, halo = sh.ext[l].H;
    const float *prev = act[l];
    // this layer's partial-sum buffer: the other one may still be read by
    // the cluster's CTAs summing the previous layer
    float *part = sh.part + (l & 1) * FitShared::kPart;
    // dL/dw, dL/do of every tap of layer l, taps in pairs (one read of G
    // serves both): `chunks` warps of the cluster per pair (every warp works
    // when the pairs are fewer than the warps), each over every chunks-th row
    // of the support box, lanes over its pixels.  Unit wi = c * T2 + p is
    // done by global warp wi mod nwt, which keeps its sums in its own CTA's
    // part[] slot wi; they are added in chunk order below.  An odd T's last
    // pair repeats its tap; the repeat's sums are not used.
    const int T2 = (T + 1) / 2;
    const int chunks = max(1, nwt / T2);
    for (int wi = gwarp; wi < T2 * chunks; wi += nwt) {
      const int ip = wi % T2, c = wi / T2;
      const int i0 = 2 * ip, i1 = min(2 * ip + 1, T - 1);
      const float4 t0 = sh.taps[l * T + i0], t1 = sh.taps[l * T + i1];
      float fx0, fy0, fx1, fy1;
      const int nx0 = min(max(split_floor(t0.x, fx0), -halo), halo - 1);
      const int ny0 = min(max(split_floor(t0.y, fy0), -halo), halo - 1);
      const int nx1 = min(max(split_floor(t1.x, fx1), -halo), halo - 1);
      const int ny1 = min(max(split_floor(t1.y, fy1), -halo), halo - 1);
      const int off0 = ny0 * N + nx0, off1 = ny1 * N + nx1;
      float gw0 = 0.f, gdx0 = 0.f, gdy0 = 0.f, gw1 = 0.f, gdx1 = 0.f, gdy1 = 0.f;
      // the box's pixels in row-major order, 32 per warp pass, every chunks-th
      // pass: no lane idles at a row's end; (u, v) advanced, not divided
      const int side = 2 * S + 1, npx = side * side, step = chunks * 32;
      const int dv = step / side, du = step - dv * side;
      int j = c * 32 + lane, v = j / side - S, u = j - (v + S) * side - S;
      for (; j < npx; j += step) {
        {
          const int p = (R + v) * N + (R + u);
          const float g = G[p];
          const float *q = prev + p + off0;
          const float a0 = q[0], b0 = q[1], c0 = q[N], d0 = q[N + 1];
          const float *r = prev + p + off1;
          const float a1 = r[0], b1 = r[1], c1 = r[N], d1 = r[N + 1];
          const float top0 = a0 + fx0 * (b0 - a0), bot0 = c0 + fx0 * (d0 - c0);
          gw0 += g * (top0 + fy0 * (bot0 - top0));
          gdx0 += g * ((1.f - fy0) * (b0 - a0) + fy0 * (d0 - c0));
          gdy0 += g * (bot0 - top0);
          const float top1 = a1 + fx1 * (b1 - a1), bot1 = c1 + fx1 * (d1 - c1);
          gw1 += g * (top1 + fy1 * (bot1 - top1));
          gdx1 += g * ((1.f - fy1) * (b1 - a1) + fy1 * (d1 - c1));
          gdy1 += g * (bot1 - top1);
        }
        u += du;
        v += dv;
        if (u > S) {
          u -= side;
          ++v;
        }
      }
      gw0 = warp_sum(gw0); gdx0 = warp_sum(gdx0); gdy0 = warp_sum(gdy0);
      gw1 = warp_sum(gw1); gdx1 = warp_sum(gdx1); gdy1 = warp_sum(gdy1);
      if (lane == 0) {
        float *pp = part + (size_t)wi * 6;
        pp[0] = gdx0 * t0.z; pp[1] = gdy0 * t0.z; pp[2] = gw0;
        pp[3] = gdx1 * t1.z; pp[4] = gdy1 * t1.z; pp[5] = gw1;
      }
    }
    // adjoint plane dL/dI_{l-1} on the support of I_{l-1}: gather at -o
    // (reads G like the tap gradients above, writes the other plane)
    prepare_taps(sh.pt, sh.taps + l * T, T, halo, -1.f, R);
    __syncthreads();
    canvas_layer(G, Gn, R, sh.ext[l - 1].S, sh.pt, T, tid, nthr);
    // the partial sums and the adjoint plane are complete everywhere
    target_sync<CL>();
    for (int j = threadIdx.x; j < T * 3; j += blockDim.x) {
      const int i = j / 3, k = j % 3, ip = i / 2, h = i % 2;
      auto val = [&](int c) {
        const int wi = c * T2 + ip;
        return rank_ptr<CL>(part, (unsigned)((wi % nwt) / nw))[(size_t)wi * 6 + h * 3 + k];
      };
      float acc = 0.f;
      int c = 0;
      for (; c + 4 <= chunks; c += 4) {  // four reads in flight, added in chunk order
        const float a0 = val(c), a1 = val(c + 1), a2 = val(c + 2), a3 = val(c + 3);
        acc += a0;
        acc += a1;
        acc += a2;
        acc += a3;
      }
      for (; c < chunks; ++c) acc += val(c);
      sh.g[(size_t)l * T * 3 + j] = acc;
    }
    float *t = G; G = Gn; Gn = t;
  }
  // G = dL/dI_min(L, 2), complete in every CTA's view: the first two layers'
  // gradients read it at a few pixels each, redundantly in every CTA, so they
  // need no exchange and no cluster barrier
  if (L >= 2) {
    prepare_taps(sh.pt, sh.taps + T, T, sh.ext[1].H, -1.f, R);
    __syncthreads();
    second_layer_grads(sh, G, R, T);
    first_layer_grads(sh, G, R, T, true);
  } else {
    first_layer_grads(sh, G, R, T, false);
  }
  __syncthreads();  // sh.g complete for the update
}

// 512-thread CTAs are held to 40 registers so that three fit on an SM: the
// sweeps are bound by the latency of their canvas reads, and the extra warps
// hide more of it than the few spilled values cost (225 against 233 ms for
// the 256-target batch at 4 CTAs per target).
template <int NT, int CL>
__global__ void __launch_bounds__(NT, NT == 512 ? 3 : 1) fit_kernel(FitArgs A) {
  static_assert(NT >= 4 * DISK_MAX_TAPS, "one splat entry per thread");
  __shared__ FitShared sh;
  const unsigned rank = target_rank<CL>();
  const int b = A.order[blockIdx.x / CL];
  const FitMeta m = A.meta[b];
  const int L = A.L, T = A.T, P = L * T * 3, N = 2 * m.R + 1;
  const size_t plane = (size_t)N * N;
  float *base = A.scratch + m.canvas_off;
  float *act[DISK_MAX_LAYERS + 1];
  for (int l = 0; l <= L; ++l) act[l] = base + l * plane;
  float *ga = base + (L + 1) * plane, *gb = base + (L + 2) * plane;
  const float *tgt = A.targets + m.tgt_off;
  float *th = A.theta + (size_t)b * P;
  const float s = m.s;
  float *st = A.state ? A.state + (size_t)b * 3 * P : nullptr;
  const bool resume = st && A.step0 > 0;
  for (int j = threadIdx.x; j < P; j += blockDim.x) {
    // a resumed state is clamped again: an identity on any state this kernel
    // wrote, and it keeps the taps of a corrupted one inside the canvases
    const float v = resume ? st[j] : th[j];
    sh.q[j] = (j % 3 == 2) ? v : fminf(fmaxf(resume ? v : v / s, -1.f), 1.f);
    sh.mo[j] = resume ? st[P + j] : 0.f;
    sh.vo[j] = resume ? st[2 * P + j] : 0.f;
  }
  // the first layer's output plane is kept zero away from its splat pixels
  for (long long j = (long long)rank * blockDim.x + threadIdx.x; j < (long long)plane;
       j += (long long)blockDim.x * CL)
    act[1][j] = 0.f;
  if (threadIdx.x == 0) sh.nsplat = 0;
  target_sync<CL>();
  const float b1 = 0.9f, b2 = 0.999f, aeps = 1e-8f;
  float b1t = 1.f, b2t = 1.f;
  for (int k = 0; k < A.step0; ++k) {  // the same products an unbroken run forms
    b1t *= b1;
    b2t *= b2;
  }
  for (int it = 0; it < A.steps || (A.mode == 1 && it == 0); ++it) {
    const int step = A.step0 + it;
    make_taps(sh, L, T, s);
    const float loss = forward_loss<CL>(sh, A, m, act, ga, tgt, rank);
    backward<CL>(sh, A, m, act, ga, gb, rank);
    if (A.mode == 1) {
      if (rank == 0) {
        for (int j = threadIdx.x; j < P; j += blockDim.x) A.grad_out[(size_t)b * P + j] = sh.g[j];
        if (threadIdx.x == 0 && A.loss_out) A.loss_out[b] = loss;
      }
      target_sync<CL>();  // no CTA leaves while another may read its shared memory
      return;
    }
    if (rank == 0 && threadIdx.x == 0 && A.loss_hist)
      A.loss_hist[(size_t)b * (A.steps + 1) + it] = loss;
    const float lr = A.total > 1 ? A.lr0 + (A.lr1 - A.lr0) * (float)step / (float)(A.total - 1) : A.lr0;
    b1t *= b1;
    b2t *= b2;
    for (int j = threadIdx.x; j < P; j += blockDim.x) {
      const float gj = (j % 3 == 2) ? sh.g[j] : sh.g[j] * s;
      const float mj = b1 * sh.mo[j] + (1.f - b1) * gj;
      const float vj = b2 * sh.vo[j] + (1.f - b2) * gj * gj;
      sh.mo[j] = mj;
      sh.vo[j] = vj;
      const float mh = mj / (1.f - b1t), vh = vj / (1.f - b2t);
      float qn = sh.q[j] - lr * mh / (sqrtf(vh) + aeps);
      if (j % 3 != 2) qn = fminf(fmaxf(qn, -1.f), 1.f);
      sh.q[j] = qn;
    }
    __syncthreads();
  }
  // final loss at the fitted parameters
  make_taps(sh, L, T, s);
  const float loss = forward_loss<CL>(sh, A, m, act, ga, tgt, rank);
  if (rank == 0) {
    if (threadIdx.x == 0) {
      if (A.loss_out) A.loss_out[b] = loss;
      if (A.loss_hist) A.loss_hist[(size_t)b * (A.steps + 1) + A.steps] = loss;
    }
    for (int j = threadIdx.x; j < P; j += blockDim.x) {
      th[j] = (j % 3 == 2) ? sh.q[j] : sh.q[j] * s;
      if (st) {
        st[j] = sh.q[j];
        st[P + j] = sh.mo[j];
        st[2 * P + j] = sh.vo[j];
      }
    }
  }
  target_sync<CL>();  // no CTA leaves while another may read its shared memory
}

// ---- host side -----------------------------------------------------------------

constexpr int kPlanChunk = 512;  // 512 * (40 + 4) bytes: inside the parameter limit

struct PlanChunk {
  int first, count;
  FitMeta meta[kPlanChunk];
  int order[kPlanChunk];
};

__global__ void plan_upload_kernel(const __grid_constant__ PlanChunk c, FitMeta *meta, int *order) {
  for (int j = threadIdx.x; j < c.count; j += blockDim.x) {
    meta[c.first + j] = c.meta[j];
    order[c.first + j] = c.order[j];
  }
}

struct FitPlan {
  std::vector<FitMeta> meta;
  std::vector<int> order;
  size_t scratch_floats = 0, idx_ints = 0, tgt_floats = 0;
  int kmax = 0;
};

int plan_fit(const int *sizes, int batch, int L, FitPlan &plan) {
  plan.meta.resize(batch);
  long long toff = 0, coff = 0, ioff = 0;
  for (int b = 0; b < batch; ++b) {
    const int K = sizes[b];
    if (K < 1 || K > 257 || (K & 1) == 0)
      return fail(DISK_ERR_INVALID_ARG, "target sizes must be odd and in [1, 257]");
    FitMeta &m = plan.meta[b];
    m.K = K;
    plan.kmax = std::max(plan.kmax, K);
    const int h = (K - 1) / 2;
    m.s = (float)std::max(1, h);
    const int Hmax = (int)std::ceil(m.s) + 1;
    // every read of the cascade stays within (L + 1) * Hmax of the centre
    m.R = std::max(h, (L + 1) * Hmax) + 1;
    m.tgt_off = toff;
    m.canvas_off = coff;
    m.idx_off = ioff;
    toff += (long long)K * K;
    coff += (long long)(L + 3) * (2 * m.R + 1) * (2 * m.R + 1);
    ioff += (long long)K * K;
  }
  plan.order.resize(batch);
  std::iota(plan.order.begin(), plan.order.end(), 0);
  std::stable_sort(plan.order.begin(), plan.order.end(),
                   [&](int a, int c) { return plan.meta[a].R > plan.meta[c].R; });
  plan.scratch_floats = coff;
  plan.idx_ints = ioff;
  plan.tgt_floats = toff;
  return DISK_OK;
}

// ---- launch-configuration autotuner ----------------------------------------------
// The launch configuration -- threads per CTA (256, 512, 1024) and CTAs per
// target (1, 2 or 4, a thread-block cluster) -- trades the parallelism of one
// target's canvas sweeps against how many targets share the GPU; the largest
// target of a batch sets the makespan when it runs on one SM.
// disk_fit_autotune times each on the caller's batch and records the fastest
// per (L, T, largest target size in 32-pixel buckets).
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int>, int> g_tune;

// A launch configuration is encoded as threads * 16 + CTAs per target.
int tuned_config(int L, int T, int kmax) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  auto it = g_tune.find(std::make_tuple(L, T, (kmax + 31) / 32));
  return it == g_tune.end() ? 512 * 16 + 1 : it->second;
}

template <int NT, int CL>
cudaError_t launch_fit(const FitArgs &A, cudaStream_t s) {
  if (CL == 1) {
    fit_kernel<NT, 1><<<A.batch, NT, 0, s>>>(A);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(A.batch * CL);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, fit_kernel<NT, CL>, A);
}

cudaError_t launch_fit_config(int config, const FitArgs &A, cudaStream_t s) {
  switch (config) {
    case 256 * 16 + 1: return launch_fit<256, 1>(A, s);
    case 1024 * 16 + 1: return launch_fit<1024, 1>(A, s);
    case 512 * 16 + 2: return launch_fit<512, 2>(A, s);
    case 1024 * 16 + 2: return launch_fit<1024, 2>(A, s);
    case 512 * 16 + 4: return launch_fit<512, 4>(A, s);
    case 1024 * 16 + 4: return launch_fit<1024, 4>(A, s);
    default: return launch_fit<512, 1>(A, s);
  }
}

constexpr int kFitConfigs[] = {256 * 16 + 1, 512 * 16 + 1, 1024 * 16 + 1, 512 * 16 + 2,
                               1024 * 16 + 2, 512 * 16 + 4, 1024 * 16 + 4};

int run_fit(const float *d_targets, const int *sizes, int batch, int L, int T, int steps,
            float lr0, float lr1, int init, int loss, float eps, unsigned long long seed,
            float *d_theta, float *d_loss, float *d_hist, float *d_grad, int mode,
            cudaStream_t s, int config = 0, float *d_state = nullptr, int step0 = 0,
            int total = -1) {
  if (!d_targets || !sizes || !d_theta) return fail(DISK_ERR_INVALID_ARG, "null pointer");
  if (batch < 1 || L < 1 || L > DISK_MAX_LAYERS || T < 1 || T > DISK_MAX_TAPS)
    return fail(DISK_ERR_INVALID_ARG, "batch >= 1, L in [1, 16], T in [1, 64] required");
  if (L * T > kFitMaxTaps) return fail(DISK_ERR_UNSUPPORTED, "the fitter supports L * T <= 512");
  if (steps < 0 || steps > 1000000) return fail(DISK_ERR_INVALID_ARG, "steps out of range");
  if (init < 0 || init > 3 || (loss != 0 && loss != 1))
    return fail(DISK_ERR_INVALID_ARG, "bad init or loss kind");
  if (loss == 1 && !(eps > 0.f)) return fail(DISK_ERR_INVALID_ARG, "Charbonnier needs eps > 0");
  if (!std::isfinite(lr0) || !std::isfinite(lr1)) return fail(DISK_ERR_INVALID_ARG, "bad lr");
  FitPlan plan;
  int rc = plan_fit(sizes, batch, L, plan);
  if (rc) return rc;
  const size_t meta_bytes = plan.meta.size() * sizeof(FitMeta);
  const size_t order_bytes = plan.order.size() * sizeof(int);
  const size_t head = ((meta_bytes + order_bytes + 255) / 256) * 256;
  const size_t bytes = head + plan.scratch_floats * sizeof(float) + plan.idx_ints * sizeof(int);
  char *buf = nullptr;
  DISK_TRY_CUDA(scratch_alloc(reinterpret_cast<void **>(&buf), bytes, s), "scratch_alloc(fit scratch)");
  // The plan rides in kernel parameters (no host staging buffer, no sync), so
  // the whole call can be captured in a CUDA graph.
  cudaError_t e = cudaSuccess;
  for (int first = 0; first < batch && e == cudaSuccess; first += kPlanChunk) {
    static thread_local PlanChunk chunk;
    chunk.first = first;
    chunk.count = std::min(kPlanChunk, batch - first);
    for (int j = 0; j < chunk.count; ++j) {
      chunk.meta[j] = plan.meta[first + j];
      chunk.order[j] = plan.order[first + j];
    }
    plan_upload_kernel<<<1, 256, 0, s>>>(chunk, reinterpret_cast<FitMeta *>(buf),
                                         reinterpret_cast<int *>(buf + meta_bytes));
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    cudaFreeAsync(buf, s);
    return cuda_fail(e, "upload fit plan");
  }
  FitArgs A;
  A.targets = d_targets;
  A.meta = reinterpret_cast<const FitMeta *>(buf);
  A.order = reinterpret_cast<const int *>(buf + meta_bytes);
  A.scratch = reinterpret_cast<float *>(buf + head);
  A.idx_scratch = reinterpret_cast<int *>(buf + head + plan.scratch_floats * sizeof(float));
  A.theta = d_theta;
  A.loss_out = d_loss;
  A.loss_hist = d_hist;
  A.grad_out = d_grad;
  A.state = d_state;
  A.step0 = step0;
  A.total = total < 0 ? steps : total;
  A.batch = batch; A.L = L; A.T = T; A.steps = steps; A.loss_kind = loss; A.mode = mode;
  A.eps = eps; A.lr0 = lr0; A.lr1 = lr1;
  if (mode == 0 && init != 0) fit_init_kernel<<<batch, kFitThreads, 0, s>>>(A, init, seed);
  e = cudaGetLastError();
  if (e == cudaSuccess) {
    e = launch_fit_config(config > 0 ? config : tuned_config(L, T, plan.kmax), A, s);
  }
  cudaFreeAsync(buf, s);
  if (e != cudaSuccess) return cuda_fail(e, "launch fit kernels");
  return DISK_OK;
}

}  // namespace
}  // namespace disk

using namespace disk;

extern "C" int disk_fit(const float *d_targets, const int *sizes, int batch, int L, int T,
                        int steps, float lr0, float lr1, int init, int loss, float eps,
                        uint64_t seed, float *d_theta_io, float *d_final_loss,
                        float *d_loss_hist, void *stream) {
  return run_fit(d_targets, sizes, batch, L, T, steps, lr0, lr1, init, loss, eps, seed,
                 d_theta_io, d_final_loss, d_loss_hist, nullptr, 0,
                 static_cast<cudaStream_t>(stream));
}

extern "C" int disk_fit_resume(const float *d_targets, const int *sizes, int batch, int L,
                               int T, int step0, int steps, int total_steps, float lr0,
                               float lr1, int init, int loss, float eps, uint64_t seed,
                               float *d_state, float *d_theta_io, float *d_final_loss,
                               float *d_loss_hist, void *stream) {
  if (!d_state) return fail(DISK_ERR_INVALID_ARG, "null optimiser state");
  if (step0 < 0 || steps < 0 || total_steps > 1000000 || steps > total_steps - step0)
    return fail(DISK_ERR_INVALID_ARG, "need 0 <= step0 <= step0 + steps <= total_steps <= 1e6");
  if (init < 0 || init > 3) return fail(DISK_ERR_INVALID_ARG, "bad init");
  return run_fit(d_targets, sizes, batch, L, T, steps, lr0, lr1,
                 step0 > 0 ? (int)DISK_INIT_GIVEN : init, loss, eps, seed,
                 d_theta_io, d_final_loss, d_loss_hist, nullptr, 0,
                 static_cast<cudaStream_t>(stream), 0, d_state, step0, total_steps);
}

extern "C" int disk_fit_loss_grad(const float *d_targets, const int *sizes, int batch, int L,
                                  int T, int loss, float eps, const float *d_theta,
                                  float *d_loss, float *d_grad, void *stream) {
  if (!d_grad || !d_loss) return fail(DISK_ERR_INVALID_ARG, "null output");
  return run_fit(d_targets, sizes, batch, L, T, 0, 0.f, 0.f, 0, loss, eps, 0,
                 const_cast<float *>(d_theta), d_loss, nullptr, d_grad, 1,
                 static_cast<cudaStream_t>(stream));
}

extern "C" int disk_fit_autotune(const float *d_targets, const int *sizes, int batch, int L, int T,
                                 int loss, float eps, int *chosen_config, void *stream) {
  if (!sizes || batch < 1) return fail(DISK_ERR_INVALID_ARG, "bad batch");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  float *theta = nullptr;
  const size_t tb = (size_t)batch * L * T * 3 * sizeof(float);
  DISK_TRY_CUDA(scratch_alloc(reinterpret_cast<void **>(&theta), tb, s), "scratch_alloc(autotune)");
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best_ms = 1e30f;
  int best = 512 * 16 + 1, rc = DISK_OK;
  int kmax = 0;
  for (int b = 0; b < batch; ++b) kmax = std::max(kmax, sizes[b]);
  for (int c = 0; c < (int)(sizeof(kFitConfigs) / sizeof(int)) && rc == DISK_OK; ++c) {
    // same start for every candidate: the sparse-sampling initialisation,
    // whose first layer spreads over the target's support as a fitted one
    // does, then 12 steps (enough for the ranking to follow a full fit's)
    rc = run_fit(d_targets, sizes, batch, L, T, 0, 1e-3f, 1e-4f, 2, loss, eps, 0, theta, nullptr,
                 nullptr, nullptr, 0, s, kFitConfigs[c]);
    if (rc) break;
    cudaEventRecord(e0, s);
    rc = run_fit(d_targets, sizes, batch, L, T, 12, 1e-3f, 1e-4f, 0, loss, eps, 0, theta, nullptr,
                 nullptr, nullptr, 0, s, kFitConfigs[c]);
    cudaEventRecord(e1, s);
    if (rc) break;
    cudaError_t e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) { rc = cuda_fail(e, "autotune timing"); break; }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best_ms) { best_ms = ms; best = kFitConfigs[c]; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(theta, s);
  if (rc) return rc;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune[std::make_tuple(L, T, (kmax + 31) / 32)] = best;
  }
  if (chosen_config) *chosen_config = best;
  return DISK_OK;
}

extern "C" int disk_fit_set_config(int L, int T, int kmax, int config) {
  bool known = false;
  for (int c : kFitConfigs) known = known || c == config;
  if (!known) return fail(DISK_ERR_INVALID_ARG, "unknown fit launch configuration");
  if (L < 1 || T < 1 || kmax < 1) return fail(DISK_ERR_INVALID_ARG, "bad L, T or kmax");
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune[std::make_tuple(L, T, (kmax + 31) / 32)] = config;
  return DISK_OK;
}
