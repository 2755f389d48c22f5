// disk_sv_filter_noalloc: the spatially varying filter for callers that may
// not allocate device memory.  Same kernels and results as disk_sv_filter;
// the intermediate layers live in a fixed array compiled into the library
// instead of memory taken from the stream's pool.
#include <mutex>

#include "sv_layer.cuh"

namespace disk {
namespace {

constexpr long long kNoAllocMaxPixels = 1ll << 20;  // H * W limit: 1,048,576 pixels

// Room for two FP32 RGBA intermediate planes of up to kNoAllocMaxPixels
// pixels each (FP16 images use FP16 planes and half of it): 32 MiB that every
// device which loads the library holds until the process exits.  Every layer overwrites each pixel of its plane before the next
// layer reads it, so nothing needs clearing between calls.
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

int run_noalloc(const disk_basis *b, const void *d_in, size_t in_pitch, void *d_out,
                size_t out_pitch, int H, int W, int C, int dtype, const float *d_maps,
                float4 *planes, cudaStream_t s) {
  static thread_local SvLayerParams P;
  P.maps = d_maps;
  P.rot = nullptr;
  P.use_tma = 0;
  P.err = device_error_word();
  P.H = H; P.W = W; P.C = C; P.T = b->T;
  make_axes(b->dims, b->n_nodes, b->node_vals.data(), P.ax);
  const int user = dtype == DISK_F32 ? PIX_F32 : PIX_F16;
  const int mid = intermediate_kind(dtype);
  const size_t mid_bytes = kind_bytes(mid);
  const int L = b->L;
  // plane 0 at the start of the array, plane 1 after H * W pixels of the
  // intermediate kind (both fit: the array holds two FP32 RGBA planes)
  char *bufs[2] = {reinterpret_cast<char *>(planes),
                   reinterpret_cast<char *>(planes) + (size_t)H * W * mid_bytes};
  int rc = DISK_OK;
  for (int l = 0; l < L && rc == DISK_OK; ++l) {
    P.halo = P.halo_x = halo_of(b->reach[l]);
    P.region_w = kSvTileW + 2 * P.halo;
    const int src = l == 0 ? user : mid;
    const int dst = l == L - 1 ? user : mid;
    P.src = l == 0 ? d_in : bufs[(l - 1) & 1];
    P.src_pitch = l == 0 ? (long long)in_pitch : (long long)(W * mid_bytes);
    P.dst = l == L - 1 ? d_out : bufs[l & 1];
    P.dst_pitch = l == L - 1 ? (long long)out_pitch : (long long)(W * mid_bytes);
    P.gtaps = layer_taps(b, l, C);
    P.bt = b->B * b->T;
    const size_t region = sv_smem_bytes((size_t)P.region_w * (sv_tile_h(kSvDefaultPix) + 2 * P.halo), C);
    P.tap_cap = sv_tap_cap(b->dims, b->n_nodes[1], b->B, b->T, region);
    rc = launch_layer(b->dims, false, src, dst, C, P, s, kSvDefaultPix);
  }
  return rc;
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
  for (int l = 0; l < b->L; ++l) {
    const int h = halo_of(b->reach[l]);
    const size_t smem = sv_smem_bytes((size_t)(kSvTileW + 2 * h) * (sv_tile_h(kSvDefaultPix) + 2 * h), C);
    if (smem > (size_t)kSvMaxSmem) return fail(DISK_ERR_UNSUPPORTED, "layer halo exceeds shared memory");
  }
  float4 *planes = nullptr;
  rc = planes_address(dev, &planes);
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return run_noalloc(b, d_in, in_pitch, d_out, out_pitch, H, W, C, dtype, d_maps, planes, s);
}
