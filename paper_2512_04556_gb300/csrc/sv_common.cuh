// Device helpers shared by the spatially varying kernels (forward, dense
// baseline, image adjoint): pixel load/store in the storage types, kernel-
// space location (Eq. 9) and the integer/fraction split of an offset.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "internal.h"

namespace disk {

// Storage kinds of an image operand.
enum PixKind : int {
  PIX_RGBA32 = 0,  // library intermediate for FP32 images: float4 per pixel, dense rows
  PIX_F32 = 1,     // caller image: C floats per pixel
  PIX_F16 = 2,     // caller image: C halves per pixel
  PIX_RGBA16 = 3   // library intermediate for FP16 images: 4 halves per pixel, dense rows
};

// Row pitch of the forward filter's FP32 intermediates (any image
// precision): C floats per pixel (the PIX_F32 layout), rows padded to 16
// bytes.  The layout is the shared-memory staging layout of the layer
// kernel, so a tile of it is copied by the tensor-memory accelerator without
// conversion.
__host__ __device__ inline long long f32_mid_pitch(int W, int C) {
  return ((long long)W * C * 4 + 15) & ~15ll;
}

// Intermediate planes keep the caller's storage precision: FP32 RGBA for
// FP32 images, FP16 RGBA for FP16 images (arithmetic is FP32 either way).
__host__ __device__ inline int intermediate_kind(int dtype) {
  return dtype == DISK_F32 ? PIX_RGBA32 : PIX_RGBA16;
}
__host__ __device__ inline size_t kind_bytes(int kind) { return kind == PIX_RGBA32 ? 16 : 8; }

// Four halves <-> two 32-bit words (x holds channels 0,1; y holds 2,3).
__device__ __forceinline__ uint2 pack_half4(float4 v) {
  const __half2 a = __floats2half2_rn(v.x, v.y), b = __floats2half2_rn(v.z, v.w);
  return make_uint2(*reinterpret_cast<const unsigned *>(&a), *reinterpret_cast<const unsigned *>(&b));
}
__device__ __forceinline__ float4 unpack_half4(uint2 u) {
  const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&u.x));
  const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&u.y));
  return make_float4(a.x, a.y, b.x, b.y);
}

// Raw FP16 RGBA of one pixel of an FP16 source (no rounding: the values are
// already halves).
template <int KIND>
__device__ __forceinline__ uint2 load_raw16(const void *base, long long pitch, int C, int y, int x) {
  const char *row = static_cast<const char *>(base) + (long long)y * pitch;
  if (KIND == PIX_RGBA16) return __ldg(reinterpret_cast<const uint2 *>(row) + x);
  const unsigned short *p = reinterpret_cast<const unsigned short *>(row) + (long long)x * C;
  const unsigned a = __ldg(p), b = __ldg(p + 1), c = __ldg(p + 2), d = C == 4 ? __ldg(p + 3) : 0u;
  return make_uint2(a | (b << 16), c | (d << 16));
}

template <int KIND>
__device__ __forceinline__ float4 load_px(const void *base, long long pitch, int C, int y, int x) {
  const char *row = static_cast<const char *>(base) + (long long)y * pitch;
  if (KIND == PIX_RGBA32) {
    return __ldg(reinterpret_cast<const float4 *>(row) + x);
  } else if (KIND == PIX_RGBA16) {
    return unpack_half4(__ldg(reinterpret_cast<const uint2 *>(row) + x));
  } else if (KIND == PIX_F32) {
    const float *p = reinterpret_cast<const float *>(row) + (long long)x * C;
    return make_float4(__ldg(p), __ldg(p + 1), __ldg(p + 2), C == 4 ? __ldg(p + 3) : 0.f);
  } else {
    const __half *p = reinterpret_cast<const __half *>(row) + (long long)x * C;
    return make_float4(__half2float(p[0]), __half2float(p[1]), __half2float(p[2]),
                       C == 4 ? __half2float(p[3]) : 0.f);
  }
}

template <int KIND>
__device__ __forceinline__ void store_px(void *base, long long pitch, int C, int y, int x, float4 v) {
  char *row = static_cast<char *>(base) + (long long)y * pitch;
  if (KIND == PIX_RGBA32) {
    reinterpret_cast<float4 *>(row)[x] = v;
  } else if (KIND == PIX_RGBA16) {
    reinterpret_cast<uint2 *>(row)[x] = pack_half4(v);
  } else if (KIND == PIX_F32) {
    float *p = reinterpret_cast<float *>(row) + (long long)x * C;
    p[0] = v.x; p[1] = v.y; p[2] = v.z;
    if (C == 4) p[3] = v.w;
  } else {
    __half *p = reinterpret_cast<__half *>(row) + (long long)x * C;
    p[0] = __float2half_rn(v.x); p[1] = __float2half_rn(v.y); p[2] = __float2half_rn(v.z);
    if (C == 4) p[3] = __float2half_rn(v.w);
  }
}

// Eq. 9 on one axis: lower node k and blend t in [0, 1] for value p, clamped
// to the node range (fmaxf maps NaN to the first node).
__device__ __forceinline__ void locate(const AxisNodes &a, float p, int &k, float &t) {
  const int n = a.n;
  if (n <= 1) { k = 0; t = 0.f; return; }
  p = fminf(fmaxf(p, a.v[0]), a.v[n - 1]);
  int lo = 0, hi = n - 1;
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (p >= a.v[mid]) lo = mid; else hi = mid;
  }
  k = lo;
  t = fminf((p - a.v[lo]) * a.inv[lo], 1.f);
}

// Interpolation weights of a pixel: up to four (node index, weight) pairs.
struct Cell {
  int n00, n01, n10, n11;
  float a00, a01, a10, a11;
};

template <int DIMS>
__device__ __forceinline__ Cell make_cell_v(const AxisNodes *ax, float p0, float p1) {
  Cell c;
  int k0; float t0;
  locate(ax[0], p0, k0, t0);
  const int k0b = min(k0 + 1, ax[0].n - 1);
  if (DIMS == 1) {
    c.n00 = k0; c.n10 = k0b; c.n01 = k0; c.n11 = k0b;
    c.a00 = 1.f - t0; c.a10 = t0; c.a01 = 0.f; c.a11 = 0.f;
  } else {
    int k1; float t1;
    locate(ax[1], p1, k1, t1);
    const int k1b = min(k1 + 1, ax[1].n - 1), n1 = ax[1].n;
    c.n00 = k0 * n1 + k1;  c.n01 = k0 * n1 + k1b;
    c.n10 = k0b * n1 + k1; c.n11 = k0b * n1 + k1b;
    c.a00 = (1.f - t0) * (1.f - t1); c.a01 = (1.f - t0) * t1;
    c.a10 = t0 * (1.f - t1);         c.a11 = t0 * t1;
  }
  return c;
}

template <int DIMS>
__device__ __forceinline__ Cell make_cell(const AxisNodes *ax, const float *maps, long long HW,
                                          long long px) {
  return make_cell_v<DIMS>(ax, maps[px], DIMS == 2 ? maps[HW + px] : 0.f);
}

// Splits an offset d into an integer n and a fraction f = d - n in [0, 1]
// with n = round-to-nearest(d - 1/2).  n equals floor(d) except at exact
// integers, where it may be d - 1 with f = 1; bilinear sampling takes the
// same value either way.  The integer part is taken from d alone (never from
// pixel + d), so the fraction keeps full FP32 precision.  |d| < 2^21.
__device__ __forceinline__ int split_offset(float d, float &f) {
  const float magic = 12582912.0f;  // 1.5 * 2^23: adding it rounds to an integer
  const float r = __fadd_rn(__fadd_rn(d, -0.5f), magic);
  f = __fsub_rn(d, __fsub_rn(r, magic));
  return __float_as_int(r) - 0x4B400000;
}

}  // namespace disk
