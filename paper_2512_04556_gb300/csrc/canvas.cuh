// Device building blocks for shift-invariant complexes on a zero-padded
// square canvas (impulse synthesis, Sec. 4.4 Eq. 10, and its adjoint for the
// fit).  A canvas of half-width R is a dense (2R+1)^2 float plane centred on
// c = (R, R).  All routines are executed by every thread of one CTA, or of
// every CTA of a cluster that shares the canvas (tid, nthr: the thread's
// index among, and the number of, the threads that split the work).
#pragma once

#include <cuda_runtime.h>

#include "sv_common.cuh"

namespace disk {

// Per-layer bookkeeping derived from the current taps: H_l = ceil(reach)+1,
// support half-width S_l = H_1 + ... + H_l of the layer's output.
struct LayerExtent {
  int H;
  int S;
};

// Zero the square frame b_in < max(|dx|,|dy|) <= b_out of a canvas.
__device__ __forceinline__ void zero_frame(float *plane, int R, int b_in, int b_out,
                                           int tid = threadIdx.x, int nthr = blockDim.x) {
  b_out = min(b_out, R);
  if (b_out <= b_in) return;
  const int side = 2 * b_out + 1, N = 2 * R + 1;
  for (int j = tid; j < side * side; j += nthr) {
    const int v = j / side - b_out, u = j % side - b_out;
    if (max(abs(u), abs(v)) > b_in) plane[(R + v) * N + (R + u)] = 0.f;
  }
}

// floor split of an offset: d = n + f, n = floor(d), f in [0, 1).  The fit
// uses this exact convention (as the oracle does) because the one-sided
// derivative taken at integer offsets depends on it.
__device__ __forceinline__ int split_floor(float d, float &f) {
  const float fl = floorf(d);
  f = d - fl;
  return __float2int_rn(fl);
}

// One shift-invariant layer's taps prepared for a sweep: per tap the offset
// of its corner (0, 0) from the output pixel in canvas elements and the four
// bilinear corner weights times w, (w00, w01, w10, w11) -- the taps are the
// same at every pixel, so the split and the weights are taken once per layer.
struct PreparedTaps {
  float4 w[DISK_MAX_TAPS];
  int off[DISK_MAX_TAPS];
};

// Fills p from taps[T] (dx, dy, w) for a canvas of half-width R; sign = -1
// applies the taps at -o (the adjoint of a layer on a zero-bounded canvas,
// by the symmetry of the bilinear tent).  halo bounds every tap's reach as
// ceil(reach) + 1.  Run by the threads of one CTA; the caller synchronises
// the CTA before a sweep reads p.
__device__ __forceinline__ void prepare_taps(PreparedTaps &p, const float4 *taps, int T, int halo,
                                             float sign, int R) {
  const int N = 2 * R + 1;
  for (int i = threadIdx.x; i < T; i += blockDim.x) {
    const float4 t = taps[i];
    float fx, fy;
    const int nx = min(max(split_floor(sign * t.x, fx), -halo), halo - 1);
    const int ny = min(max(split_floor(sign * t.y, fy), -halo), halo - 1);
    const float wy1 = t.z * fy, wy0 = t.z - wy1;
    const float w11 = wy1 * fx, w10 = wy1 - w11, w01 = wy0 * fx, w00 = wy0 - w01;
    p.w[i] = make_float4(w00, w01, w10, w11);
    p.off[i] = ny * N + nx;
  }
}

// One shift-invariant layer (Eq. 3) with prepared taps p[T]:
// dst[p] = sum_i w_i * bilinear(src, p + o_i) for every p with
// max(|p - c|) <= b.  src must hold the true values (zeros outside the
// support) on the box of half-width b + halo.
__device__ __forceinline__ void canvas_layer(const float *src, float *dst, int R, int b,
                                             const PreparedTaps &p, int T,
                                             int tid = threadIdx.x, int nthr = blockDim.x) {
  const int side = 2 * b + 1, N = 2 * R + 1;
  for (int j = tid; j < side * side; j += nthr) {
    const int v = j / side - b, u = j % side - b;
    const float *base = src + (R + v) * N + (R + u);
    float acc = 0.f;
    for (int i = 0; i < T; ++i) {
      const float4 w = p.w[i];
      const float *q = base + p.off[i];
      acc += w.x * q[0] + w.y * q[1] + w.z * q[N] + w.w * q[N + 1];
    }
    dst[(R + v) * N + (R + u)] = acc;
  }
}

}  // namespace disk
