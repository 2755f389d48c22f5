// Internal declarations shared by the translation units of libdisk.so.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "disk.h"

// Immutable basis of complexes (Sec. 4.3, Eq. 8) with its device copy.
struct disk_basis {
  int dims = 1;
  int n_nodes[2] = {1, 1};
  int L = 0, T = 0, B = 0;
  std::vector<float> node_vals;  // n_nodes[0] (+ n_nodes[1]) values
  std::vector<float> theta;      // [B][L][T][3] = (dx, dy, w), pixels
  std::vector<float> reach;      // [L]: max over nodes, taps of max(|dx|,|dy|)
  std::vector<float> reach_norm; // [L]: max over nodes, taps of sqrt(dx^2 + dy^2)
  int device = 0;
  float4 *d_taps = nullptr;      // [L][B][T] = (dx, dy, w, w)
  // the same taps in the pair layout of the 3-channel filter (same shape;
  // for each node, slot 2j = (dx_2j, dx_2j+1, dy_2j, dy_2j+1) and slot
  // 2j + 1 = (w_2j, w_2j+1) of the node, then of its successor on axis 0;
  // an odd T's last slot as above); it shares d_taps' allocation
  float4 *d_taps_pair = nullptr;
  // filter tile configuration (pixels per thread) of every layer, chosen by
  // disk_sv_filter_autotune per (H, W, C, dtype | rotated << 8); read by
  // disk_sv_filter and disk_sv_filter_rotated
  mutable std::mutex tune_mu;
  mutable std::map<std::tuple<int, int, int, int>, std::vector<int>> tune_pix;
};

namespace disk {

// Records a detail message for disk_last_error_message() and returns code.
int fail(int code, const std::string &msg);
// Maps a CUDA error to DISK_ERR_OOM / DISK_ERR_CUDA with a detail message.
int cuda_fail(cudaError_t e, const char *what);

// Stream-ordered scratch from the library's own memory pool on the current
// device.  The pool keeps freed memory mapped (release threshold: no limit),
// so a frame loop that synchronises between calls does not map and unmap its
// scratch every frame, as the default pool would at each synchronisation.
// Free with cudaFreeAsync.  Capturable into CUDA graphs.
cudaError_t scratch_alloc_raw(void **p, size_t bytes, cudaStream_t s);
template <class T>
inline cudaError_t scratch_alloc(T **p, size_t bytes, cudaStream_t s) {
  return scratch_alloc_raw(reinterpret_cast<void **>(p), bytes, s);
}

// Device status word of the current device (zero-initialised, one per
// device): kernels whose bounded waits give up store DISK_ERR_TIMEOUT there;
// disk_device_status reads and clears it.  nullptr if it cannot be allocated.
int *device_error_word();

inline int halo_of(float reach) {
  // Offsets with |o| <= reach touch pixels within ceil(reach) + 1 of the
  // output pixel (the +1 is the bilinear footprint).
  return static_cast<int>(__builtin_ceilf(reach)) + 1;
}

// Reach of layer l: per-axis for the plain filter; the Euclidean tap length
// when offsets are rotated at run time (a turned tap keeps its length).
inline float layer_reach(const disk_basis *b, int l, bool rotated) {
  return rotated ? b->reach_norm[l] : b->reach[l];
}

// Layer l's node-tap table as the filter kernel for C channels reads it
// (the pair layout for 3 channels).
inline const float4 *layer_taps(const disk_basis *b, int l, int C) {
  return (C == 3 ? b->d_taps_pair : b->d_taps) + (size_t)l * b->B * b->T;
}

// Kernel-space axis as the kernels see it: node values and inverse spacings.
struct AxisNodes {
  int n;
  float v[DISK_MAX_NODES_AXIS];
  float inv[DISK_MAX_NODES_AXIS];
};

void make_axes(int dims, const int *n_nodes, const float *node_vals, AxisNodes ax[2]);

int validate_image_args(const void *d_in, size_t in_pitch, const void *d_out,
                        size_t out_pitch, int H, int W, int C, int dtype,
                        const float *d_maps);
int validate_nodes(int dims, const int *n_nodes, const float *node_vals);

// disk_sv_filter with the two intermediate planes given by the caller
// (H * f32_mid_pitch(W, C) bytes each, 16-byte aligned; plane1 unused for
// L <= 2, both unused for L = 1): the same argument checks, tile choice,
// tensor copies and kernels, and no allocation.  Returns a DISK_* status.
int sv_filter_given_planes(const disk_basis *b, const void *d_in, size_t in_pitch, void *d_out,
                           size_t out_pitch, int H, int W, int C, int dtype,
                           const float *d_maps, void *plane0, void *plane1, cudaStream_t s);

}  // namespace disk

#define DISK_TRY_CUDA(expr, what)                   \
  do {                                              \
    cudaError_t e_ = (expr);                        \
    if (e_ != cudaSuccess) return disk::cuda_fail(e_, what); \
  } while (0)
