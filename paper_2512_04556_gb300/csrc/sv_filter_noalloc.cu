// disk_sv_filter_noalloc: the spatially varying filter for callers that may
// not allocate device memory.  It runs disk_sv_filter's own code path (the
// same checks, per-layer tile choice, tensor copies, kernels and FP32
// intermediate layout) with the two intermediate planes placed in a fixed
// array compiled into the library instead of memory taken from the pool, so
// its results equal disk_sv_filter's bit for bit.
#include <mutex>

#include "sv_layer.cuh"

namespace disk {
namespace {

constexpr long long kNoAllocMaxPixels = 1ll << 20;  // H * W limit: 1,048,576 pixels

// Two FP32 intermediate planes of up to kNoAllocMaxPixels pixels: a plane
// has rows of f32_mid_pitch(W, C) bytes, at most 16 W for C <= 4 (16 W is a
// multiple of 16 and at least 4 C W), so a plane needs at most 16 MiB and
// plane 1 starts at the array's half.  32 MiB that every device which loads
// the library holds until the process exits.  Every layer overwrites each
// pixel of its plane before the next layer reads it, so nothing needs
// clearing between calls.
static __device__ __align__(256) float4 g_noalloc_planes[2 * kNoAllocMaxPixels];

constexpr int kMaxDevices = 64;
std::mutex g_addr_mu;
float4 *g_addr[kMaxDevices] = {};

// Device address of the planes on device `dev` (the current device).  In
// host code the array's name is only a host-side stand-in, so the address is
// asked of the runtime once per device and cached.
int planes_address(int dev, float4 **out) {
  if (dev < 0 || dev >= kMaxDevices) return fail(DISK_ERR_UNSUPPORTED, "device index beyond 63");
  std::lock_guard<std::mutex> lock(g_addr_mu);
  if (!g_addr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_planes);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-alloc planes)");
    g_addr[dev] = static_cast<float4 *>(p);
  }
  *out = g_addr[dev];
  return DISK_OK;
}

}  // namespace
}  // namespace disk

using namespace disk;

extern "C" int disk_sv_filter_noalloc(const disk_basis *b, const void *d_in, size_t in_pitch,
                                      void *d_out, size_t out_pitch, int H, int W, int C,
                                      int dtype, const float *d_maps, void *stream) {
  if (!b) return fail(DISK_ERR_INVALID_ARG, "null basis");
  int rc = validate_image_args(d_in, in_pitch, d_out, out_pitch, H, W, C, dtype, d_maps);
  if (rc) return rc;
  if ((long long)H * W > kNoAllocMaxPixels)
    return fail(DISK_ERR_UNSUPPORTED, "disk_sv_filter_noalloc takes at most 1048576 pixels (H * W)");
  int dev = 0;
  DISK_TRY_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
  if (dev != b->device) return fail(DISK_ERR_INVALID_ARG, "basis lives on another device");
  float4 *planes = nullptr;
  rc = planes_address(dev, &planes);
  if (rc) return rc;
  // The device status word that the layer kernels report bounded-wait
  // timeouts in was allocated when the basis was created on this device, so
  // the call below allocates nothing.
  return sv_filter_given_planes(b, d_in, in_pitch, d_out, out_pitch, H, W, C, dtype, d_maps,
                                planes, planes + kNoAllocMaxPixels,
                                static_cast<cudaStream_t>(stream));
}
