// disk_sv_filter: the spatially varying cascade (Sec. 4.3 Eq. 9 + Sec. 3.2
// Eq. 3) as one shared-memory-staged launch per layer (kernel in
// sv_layer.cuh); disk_sv_filter_rotated: the same with every pixel's taps
// turned by a per-pixel angle (Sec. 5.3's rotational and radial blur).
// Intermediate layers live in FP32 buffers (C floats per pixel, rows
// padded to 16 bytes; f32_mid_pitch in sv_common.cuh) from the library's
// memory pool; the first layer reads the caller's image and the last writes
// the caller's output.  A layer that reads an intermediate has its source
// tile copied into shared memory by the tensor-memory accelerator (one 2-D
// copy, an mbarrier, a bounded wait).
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "sv_pair.cuh"

namespace disk {

__global__ void rotation_kernel(const float *__restrict__ angle, float2 *__restrict__ rot,
                                long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    float phi = angle[i];
    if (!isfinite(phi)) phi = 0.f;
    float sn, cs;
    sincosf(phi, &sn, &cs);
    const float inv = rsqrtf(fmaf(cs, cs, sn * sn));
    rot[i] = make_float2(cs * inv, sn * inv);
  }
}

int launch_layer(int dims, bool rot, int src, int dst, int C, const SvLayerParams &P,
                 cudaStream_t s, int pix) {
  if (dims == 1)
    return rot ? launch_sv_layer<1, true>(src, dst, C, P, s, pix)
               : launch_sv_layer<1, false>(src, dst, C, P, s, pix);
  return rot ? launch_sv_layer<2, true>(src, dst, C, P, s, pix)
             : launch_sv_layer<2, false>(src, dst, C, P, s, pix);
}

// Exercises the bounded wait of the tile copies: the block arms an
// mbarrier for 16 bytes that no copy will deliver, waits at most `iters`
// polls, and records DISK_ERR_TIMEOUT like a layer kernel whose copy did not
// land.  Nothing faults or hangs: the wait ends by its limit.
__global__ void wait_selftest_kernel(int *err, long long iters) {
  __shared__ __align__(8) unsigned long long bar;
  const unsigned b = smem_addr(&bar);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(b) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(b), "r"(16u)
                 : "memory");
  }
  __syncthreads();
  const bool landed = mbar_wait(b, 0, iters);
  if (!__syncthreads_and(landed) && threadIdx.x == 0) atomicExch(err, DISK_ERR_TIMEOUT);
}

namespace {

// Staging geometry of layer l: halo rows above and below the tile, halo_x
// columns left and right.  halo_x is the halo rounded up to a multiple of 16
// pixels, which makes the staged row length 32 + 2 halo_x a multiple of 32
// pixels: a warp whose lanes' integer offsets straddle two rows then reads
// them without shared-memory bank conflicts (pixel k of row r + 1 lies in
// the bank of pixel k of row r, and the lanes read distinct columns), and
// every tensor copy starts on a 16-byte boundary (tile origins are
// multiples of 32).  Where that region would not fit shared memory the halo
// is rounded up to 4 pixels only (tensor copies), or not at all (staging
// through registers).  Layers after the first read an FP32 intermediate,
// which the tensor-memory accelerator copies when the copy's box fits its
// 256-element limit (rows of C (32 + 2 halo_x) floats, copied as 8-byte
// elements: C (32 + 2 halo_x) / 2 <= 256).
struct LayerGeom {
  int halo, halo_x, tma;
};

LayerGeom layer_geom(const disk_basis *b, int C, int l, bool rot) {
  const int h = halo_of(layer_reach(b, l, rot));
  // a column halo whose region (with the smallest tile) fits shared memory;
  // the widest halos give up the rounding rather than the layer
  const size_t rows = (size_t)sv_tile_h(kSvDefaultPix) + 2 * h;
  auto fits = [&](int hx) { return sv_smem_bytes((kSvTileW + 2 * (size_t)hx) * rows, C) <= kSvMaxSmem; };
  const int hx16 = (h + 15) & ~15, hx4 = (h + 3) & ~3;
  if (l == 0) return {h, fits(hx16) ? hx16 : h, 0};
  for (const int hx : {hx16, hx4})
    if (C * (kSvTileW + 2 * hx) / 2 <= 256 && fits(hx)) return {h, hx, 1};
  return {h, h, 0};
}

// Layer choice code of the first layer of a fused pair (layers l and l + 1 in
// one launch); the second layer of the pair has code 0.
constexpr int kSvPairCode = 8;

// Geometry of the fused pair (l, l + 1): halos, staged columns, whether its
// source (an FP32 intermediate for l > 0) is copied by the tensor-memory
// accelerator (box of at most 256 elements per dimension), and whether both
// tap tables are copied into shared memory.  False if it does not fit.
struct PairGeom {
  int h0, h1, hxs, tma, taps;
};

bool pair_geom(const disk_basis *b, int C, int l, PairGeom &pg) {
  if (l + 1 >= b->L) return false;
  pg.h0 = halo_of(b->reach[l]);
  pg.h1 = halo_of(b->reach[l + 1]);
  const int hs = pg.h0 + pg.h1, hx4 = (hs + 3) & ~3;
  pg.tma = l > 0 && C * (kSvTileW + 2 * hx4) / 2 <= 256 && kSvPairTileH + 2 * hs <= 256;
  pg.hxs = pg.tma ? hx4 : hs;
  const int bt = b->B * b->T;
  for (const int taps : {1, 0}) {
    if (sv_pair_geom(pg.h0, pg.h1, pg.hxs, C, bt, taps).total <= (size_t)kSvMaxSmem) {
      pg.taps = taps;
      return true;
    }
  }
  return false;
}

bool fits_pair(const disk_basis *b, int C, int l) {
  PairGeom pg;
  return pair_geom(b, C, l, pg);
}

size_t layer_smem(const disk_basis *b, int C, int l, int pix, bool rot) {
  const LayerGeom g = layer_geom(b, C, l, rot);
  return sv_smem_bytes((size_t)(kSvTileW + 2 * g.halo_x) * (sv_tile_h(pix) + 2 * g.halo), C);
}

using EncodeTiled = PFN_cuTensorMapEncodeTiled_v12000;

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library); nullptr if the driver does not provide it.
EncodeTiled encode_tiled() {
  static std::once_flag once;
  static EncodeTiled fn = nullptr;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(p);
  });
  return fn;
}

// 2-D tensor map of an FP32 intermediate viewed as 8-byte elements (the
// copy moves bytes; a pixel's C floats stay in order): width elements per
// row, rows of pitch bytes, box_w x box_h elements per copy, zeros outside.
bool encode_rows(EncodeTiled fn, CUtensorMap *m, const void *base, long long width, int H,
                 long long pitch, int box_w, int box_h) {
  const cuuint64_t dims[2] = {(cuuint64_t)width, (cuuint64_t)H};
  const cuuint64_t strides[1] = {(cuuint64_t)pitch};
  const cuuint32_t box[2] = {(cuuint32_t)box_w, (cuuint32_t)box_h};
  const cuuint32_t es[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, const_cast<void *>(base), dims, strides, box,
            es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int run_filter(const disk_basis *b, const void *d_in, size_t in_pitch, void *d_out,
               size_t out_pitch, int H, int W, int C, int dtype, const float *d_maps,
               const float *d_angle, cudaStream_t s, const int *pix, cudaEvent_t *ev,
               void *const *given = nullptr) {
  // given (optional): two caller-owned intermediate planes of
  // H * f32_mid_pitch(W, C) bytes each, used instead of pool scratch.
  // The parameter block is large; keep it off the host stack.
  static thread_local SvLayerParams P;
  P.maps = d_maps;
  P.rot = nullptr;
  P.err = device_error_word();
  if (!P.err) return fail(DISK_ERR_CUDA, "device status word unavailable");
  P.H = H; P.W = W; P.C = C; P.T = b->T;
  make_axes(b->dims, b->n_nodes, b->node_vals.data(), P.ax);
  const int user = dtype == DISK_F32 ? PIX_F32 : PIX_F16;
  const int mid = PIX_F32;
  const long long mid_pitch = f32_mid_pitch(W, C);
  const int L = b->L;
  const bool rotated = d_angle != nullptr;
  const EncodeTiled encode = encode_tiled();
  void *bufs[2] = {nullptr, nullptr};
  const size_t plane = (size_t)H * mid_pitch;
  const int nbuf = given ? 0 : (L >= 3 ? 2 : (L == 2 ? 1 : 0));
  if (given) { bufs[0] = given[0]; bufs[1] = given[1]; }
  for (int i = 0; i < nbuf; ++i) {
    cudaError_t e = scratch_alloc(&bufs[i], plane, s);
    if (e != cudaSuccess) {
      if (i) cudaFreeAsync(bufs[0], s);
      return cuda_fail(e, "scratch_alloc(sv_filter scratch)");
    }
  }
  float2 *rot = nullptr;
  if (d_angle) {
    const long long n = (long long)H * W;
    cudaError_t e = scratch_alloc(&rot, (size_t)n * sizeof(float2), s);
    if (e != cudaSuccess) {
      for (int i = 0; i < nbuf; ++i) cudaFreeAsync(bufs[i], s);
      return cuda_fail(e, "scratch_alloc(rotation plane)");
    }
    const int blocks = (int)std::min<long long>((n + 255) / 256, 152LL * 16);
    rotation_kernel<<<blocks, 256, 0, s>>>(d_angle, rot, n);
    P.rot = rot;
  }
  int rc = DISK_OK;
  if (d_angle) {
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) rc = cuda_fail(e, "launch rotation_kernel");
  }
  // Each launch reads the previous launch's output (the caller's image first)
  // and writes the other intermediate plane (the caller's output last).
  const void *cur = d_in;
  for (int l = 0; l < L && rc == DISK_OK;) {
    const bool pair = !rotated && pix[l] == kSvPairCode && l + 1 < L;
    const int last = pair ? l + 1 : l;
    void *dst_ptr = last == L - 1 ? d_out : (cur == bufs[0] ? bufs[1] : bufs[0]);
    const int src = l == 0 ? user : mid;
    const int dst = last == L - 1 ? user : mid;
    const long long spitch = l == 0 ? (long long)in_pitch : mid_pitch;
    const long long dpitch = last == L - 1 ? (long long)out_pitch : mid_pitch;
    if (pair) {
      static thread_local SvPairParams Q;
      PairGeom pg;
      if (!pair_geom(b, C, l, pg)) { rc = fail(DISK_ERR_UNSUPPORTED, "fused pair exceeds shared memory"); break; }
      Q.src = cur; Q.src_pitch = spitch; Q.dst = dst_ptr; Q.dst_pitch = dpitch;
      Q.maps = d_maps; Q.err = P.err;
      Q.gtaps0 = layer_taps(b, l, C);
      Q.gtaps1 = layer_taps(b, l + 1, C);
      Q.H = H; Q.W = W; Q.C = C; Q.T = b->T;
      Q.h0 = pg.h0; Q.h1 = pg.h1; Q.hxs = pg.hxs;
      Q.bt = b->B * b->T;
      Q.taps_smem = pg.taps;
      Q.use_tma = 0;
      std::memcpy(Q.ax, P.ax, sizeof(Q.ax));
      if (pg.tma && encode) {
        const int SW = kSvTileW + 2 * pg.hxs, SH = kSvPairTileH + 2 * (pg.h0 + pg.h1);
        if (encode_rows(encode, &Q.tm, cur, ((long long)C * W + 1) / 2, H, mid_pitch, C * SW / 2, SH))
          Q.use_tma = 1;
      }
      if (!Q.use_tma) Q.hxs = pg.h0 + pg.h1;
      if (ev) { cudaEventRecord(ev[l], s); cudaEventRecord(ev[l + 1], s); }
      rc = b->dims == 1 ? launch_sv_pair<1>(src, dst, C, Q, s) : launch_sv_pair<2>(src, dst, C, Q, s);
      cur = dst_ptr;
      l += 2;
      continue;
    }
    const LayerGeom g = layer_geom(b, C, l, rotated);
    P.halo = g.halo;
    P.halo_x = g.halo_x;
    P.region_w = kSvTileW + 2 * g.halo_x;
    P.src = cur;
    P.src_pitch = spitch;
    P.dst = dst_ptr;
    P.dst_pitch = dpitch;
    P.use_tma = 0;
    if (g.tma && encode) {
      const int RW = P.region_w, RH = sv_tile_h(pix[l]) + 2 * g.halo;
      // rows of ceil(C W / 2) eight-byte elements (for odd C W the last
      // element's second half is row padding, inside the pitch)
      const bool ok = encode_rows(encode, &P.tm, P.src, ((long long)C * W + 1) / 2, H, mid_pitch,
                                  C * RW / 2, RH);
      if (ok) {
        P.use_tma = 1;
      } else {
        // without tensor maps the layer stages through registers, which needs
        // no rounding of the column halo
        P.halo_x = g.halo;
        P.region_w = kSvTileW + 2 * g.halo;
      }
    }
    P.gtaps = layer_taps(b, l, C);
    P.bt = b->B * b->T;
    if (ev) cudaEventRecord(ev[l], s);
    const size_t region = sv_smem_bytes((size_t)P.region_w * (sv_tile_h(pix[l]) + 2 * P.halo), C);
    P.tap_cap = sv_tap_cap(b->dims, b->n_nodes[1], b->B, b->T, region);
    rc = launch_layer(b->dims, rotated, src, dst, C, P, s, pix[l]);
    cur = dst_ptr;
    ++l;
  }
  if (ev && rc == DISK_OK) cudaEventRecord(ev[L], s);
  for (int i = 0; i < nbuf; ++i) cudaFreeAsync(bufs[i], s);
  if (rot) cudaFreeAsync(rot, s);
  return rc;
}

bool fits_layer(const disk_basis *b, int C, int l, int pix, bool rot) {
  return layer_smem(b, C, l, pix, rot) <= (size_t)kSvMaxSmem;
}

// Per-layer tile configuration for this frame shape: the recorded one, or
// the default, with any layer whose halo does not fit falling back to the
// smaller tile.
// Tuning key: the frame shape, the storage type and the variant.
std::tuple<int, int, int, int> tune_key(int H, int W, int C, int dtype, bool rot) {
  return std::make_tuple(H, W, C, dtype | (rot ? 0x100 : 0));
}

std::vector<int> layer_pix(const disk_basis *b, int H, int W, int C, int dtype, bool rot) {
  std::vector<int> pix(b->L, kSvDefaultPix);
  {
    std::lock_guard<std::mutex> lock(b->tune_mu);
    auto it = b->tune_pix.find(tune_key(H, W, C, dtype, rot));
    if (it != b->tune_pix.end() && (int)it->second.size() == b->L) pix = it->second;
  }
  // a recorded choice that no longer fits falls back to the smaller tile
  for (int l = 0; l < b->L; ++l) {
    if (pix[l] == kSvPairCode) {
      if (!rot && fits_pair(b, C, l) && pix[l + 1] == 0) { ++l; continue; }
      pix[l] = 2;
      if (l + 1 < b->L && pix[l + 1] == 0) pix[l + 1] = 2;
    }
    if (pix[l] == 0 || !fits_layer(b, C, l, pix[l], rot)) pix[l] = 2;
  }
  return pix;
}

int check_filter_args(const disk_basis *b, const void *d_in, size_t in_pitch, const void *d_out,
                      size_t out_pitch, int H, int W, int C, int dtype, const float *d_maps,
                      bool rot = false) {
  if (!b) return fail(DISK_ERR_INVALID_ARG, "null basis");
  int rc = validate_image_args(d_in, in_pitch, d_out, out_pitch, H, W, C, dtype, d_maps);
  if (rc) return rc;
  int dev = 0;
  DISK_TRY_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
  if (dev != b->device) return fail(DISK_ERR_INVALID_ARG, "basis lives on another device");
  for (int l = 0; l < b->L; ++l)
    if (!fits_layer(b, C, l, 2, rot))
      return fail(DISK_ERR_UNSUPPORTED, rot ? "layer halo (rotated: Euclidean tap length) exceeds shared memory"
                                            : "layer halo exceeds shared memory");
  return DISK_OK;
}

int filter_with(const disk_basis *b, const void *d_in, size_t in_pitch, void *d_out,
                size_t out_pitch, int H, int W, int C, int dtype, const float *d_maps,
                const float *d_angle, cudaStream_t s, const int *pix, cudaEvent_t *ev = nullptr) {
  return run_filter(b, d_in, in_pitch, d_out, out_pitch, H, W, C, dtype, d_maps, d_angle, s, pix,
                    ev);
}

// Times both tile configurations layer by layer (CUDA events, three passes
// each after a warm-up pass), then (plain filter) every adjacent pair of
// layers fused into one launch, and records the fastest cover of the layers
// by single layers and fused pairs.
int autotune(const disk_basis *b, const void *d_in, size_t in_pitch, void *d_out,
             size_t out_pitch, int H, int W, int C, int dtype, const float *d_maps,
             const float *d_angle, int *chosen, cudaStream_t s) {
  const bool rot = d_angle != nullptr;
  const int L = b->L;
  std::vector<cudaEvent_t> ev(L + 1);
  for (auto &e : ev) DISK_TRY_CUDA(cudaEventCreate(&e), "cudaEventCreate");
  std::vector<float> best_ms(L, 1e30f), pair_ms(L, 1e30f);
  std::vector<int> best(L, 2);
  int rc = DISK_OK;
  // times the configuration pix: per launch, the time from its first layer's
  // event to the next launch's
  auto trial = [&](const std::vector<int> &pix, auto record) {
    rc = filter_with(b, d_in, in_pitch, d_out, out_pitch, H, W, C, dtype, d_maps, d_angle, s,
                     pix.data());
    for (int r = 0; r < 3 && rc == DISK_OK; ++r) {
      rc = filter_with(b, d_in, in_pitch, d_out, out_pitch, H, W, C, dtype, d_maps, d_angle, s,
                       pix.data(), ev.data());
      cudaError_t e = cudaEventSynchronize(ev[L]);
      if (e != cudaSuccess) { rc = cuda_fail(e, "autotune timing"); break; }
      record();
    }
  };
  const int cand[2] = {2, 4};
  for (int c = 0; c < 2 && rc == DISK_OK; ++c) {
    std::vector<int> pix(L);
    for (int l = 0; l < L; ++l) pix[l] = fits_layer(b, C, l, cand[c], rot) ? cand[c] : 2;
    trial(pix, [&] {
      for (int l = 0; l < L; ++l) {
        if (pix[l] != cand[c]) continue;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev[l], ev[l + 1]);
        if (ms < best_ms[l]) { best_ms[l] = ms; best[l] = cand[c]; }
      }
    });
  }
  // fused pairs (l, l + 1), l even in one trial and odd in the other
  for (int parity = 0; parity < 2 && rc == DISK_OK && !rot; ++parity) {
    std::vector<int> pix = best;
    bool any = false;
    for (int l = parity; l + 1 < L; l += 2)
      if (fits_pair(b, C, l)) { pix[l] = kSvPairCode; pix[l + 1] = 0; any = true; }
    if (!any) continue;
    trial(pix, [&] {
      for (int l = 0; l + 1 < L; ++l) {
        if (pix[l] != kSvPairCode) continue;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev[l], ev[l + 2]);
        pair_ms[l] = std::min(pair_ms[l], ms);
      }
    });
  }
  for (auto &e : ev) cudaEventDestroy(e);
  if (rc) return rc;
  // cheapest cover: cost[l] = time of layers l..L-1
  std::vector<float> cost(L + 1, 0.f);
  std::vector<int> take_pair(L, 0);
  for (int l = L - 1; l >= 0; --l) {
    cost[l] = best_ms[l] + cost[l + 1];
    if (l + 1 < L && pair_ms[l] < 1e29f && pair_ms[l] + cost[l + 2] < cost[l]) {
      cost[l] = pair_ms[l] + cost[l + 2];
      take_pair[l] = 1;
    }
  }
  std::vector<int> pick(L);
  for (int l = 0; l < L;) {
    if (take_pair[l]) { pick[l] = kSvPairCode; pick[l + 1] = 0; l += 2; }
    else { pick[l] = best[l]; ++l; }
  }
  {
    std::lock_guard<std::mutex> lock(b->tune_mu);
    b->tune_pix[tune_key(H, W, C, dtype, rot)] = pick;
  }
  if (chosen) for (int l = 0; l < L; ++l) chosen[l] = pick[l];
  return DISK_OK;
}

}  // namespace

int sv_filter_given_planes(const disk_basis *b, const void *d_in, size_t in_pitch, void *d_out,
                           size_t out_pitch, int H, int W, int C, int dtype,
                           const float *d_maps, void *plane0, void *plane1, cudaStream_t s) {
  int rc = check_filter_args(b, d_in, in_pitch, d_out, out_pitch, H, W, C, dtype, d_maps);
  if (rc) return rc;
  const std::vector<int> pix = layer_pix(b, H, W, C, dtype, false);
  void *const planes[2] = {plane0, plane1};
  return run_filter(b, d_in, in_pitch, d_out, out_pitch, H, W, C, dtype, d_maps, nullptr, s,
                    pix.data(), nullptr, planes);
}

}  // namespace disk

using namespace disk;

extern "C" int disk_sv_filter(const disk_basis *b, const void *d_in, size_t in_pitch,
                              void *d_out, size_t out_pitch, int H, int W, int C, int dtype,
                              const float *d_maps, void *stream) {
  int rc = check_filter_args(b, d_in, in_pitch, d_out, out_pitch, H, W, C, dtype, d_maps);
  if (rc) return rc;
  const std::vector<int> pix = layer_pix(b, H, W, C, dtype, false);
  return filter_with(b, d_in, in_pitch, d_out, out_pitch, H, W, C, dtype, d_maps, nullptr,
                     static_cast<cudaStream_t>(stream), pix.data());
}

extern "C" int disk_sv_filter_autotune(const disk_basis *b, const void *d_in, size_t in_pitch,
                                       void *d_out, size_t out_pitch, int H, int W, int C,
                                       int dtype, const float *d_maps, int *chosen,
                                       void *stream) {
  int rc = check_filter_args(b, d_in, in_pitch, d_out, out_pitch, H, W, C, dtype, d_maps);
  if (rc) return rc;
  return autotune(b, d_in, in_pitch, d_out, out_pitch, H, W, C, dtype, d_maps, nullptr, chosen,
                  static_cast<cudaStream_t>(stream));
}

extern "C" int disk_sv_filter_rotated(const disk_basis *b, const void *d_in, size_t in_pitch,
                                      void *d_out, size_t out_pitch, int H, int W, int C,
                                      int dtype, const float *d_maps, const float *d_angle,
                                      void *stream) {
  if (!d_angle) return fail(DISK_ERR_INVALID_ARG, "null angle map");
  int rc = check_filter_args(b, d_in, in_pitch, d_out, out_pitch, H, W, C, dtype, d_maps, true);
  if (rc) return rc;
  const std::vector<int> pix = layer_pix(b, H, W, C, dtype, true);
  return filter_with(b, d_in, in_pitch, d_out, out_pitch, H, W, C, dtype, d_maps, d_angle,
                     static_cast<cudaStream_t>(stream), pix.data());
}

extern "C" int disk_sv_filter_rotated_autotune(const disk_basis *b, const void *d_in,
                                               size_t in_pitch, void *d_out, size_t out_pitch,
                                               int H, int W, int C, int dtype,
                                               const float *d_maps, const float *d_angle,
                                               int *chosen, void *stream) {
  if (!d_angle) return fail(DISK_ERR_INVALID_ARG, "null angle map");
  int rc = check_filter_args(b, d_in, in_pitch, d_out, out_pitch, H, W, C, dtype, d_maps, true);
  if (rc) return rc;
  return autotune(b, d_in, in_pitch, d_out, out_pitch, H, W, C, dtype, d_maps, d_angle, chosen,
                  static_cast<cudaStream_t>(stream));
}

extern "C" int disk_sv_filter_frames(const disk_basis *b, const void *const *h_in,
                                     void *const *h_out, const float *const *h_maps,
                                     int n_frames, int H, int W, int C, int dtype,
                                     void *stream) {
  if (!b) return fail(DISK_ERR_INVALID_ARG, "null basis");
  if (n_frames < 0) return fail(DISK_ERR_INVALID_ARG, "negative frame count");
  if (n_frames == 0) return DISK_OK;
  if (!h_in || !h_out || !h_maps) return fail(DISK_ERR_INVALID_ARG, "null frame array");
  for (int i = 0; i < n_frames; ++i)
    if (!h_in[i] || !h_out[i] || !h_maps[i])
      return fail(DISK_ERR_INVALID_ARG, "null host frame, output or map pointer");
  if (H < 1 || W < 1 || H > 32768 || W > 32768 || (C != 3 && C != 4) ||
      (dtype != DISK_F32 && dtype != DISK_F16))
    return fail(DISK_ERR_INVALID_ARG, "bad frame shape or dtype");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t row = (size_t)W * C * (dtype == DISK_F32 ? 4 : 2);
  const size_t img = row * H, map = (size_t)b->dims * H * W * sizeof(float);
  // Two slots (input, output, maps) alternate between frames.
  const int S = n_frames < 2 ? 1 : 2;
  const size_t a256 = 256, slot = ((img + a256 - 1) / a256 * a256) * 2 + (map + a256 - 1) / a256 * a256;
  char *buf = nullptr;
  DISK_TRY_CUDA(scratch_alloc(&buf, slot * S, s), "scratch_alloc(frame slots)");
  const void *d_in[2];
  void *d_out[2];
  const float *d_maps[2];
  for (int k = 0; k < S; ++k) {
    char *base = buf + slot * k;
    d_in[k] = base;
    d_out[k] = base + (img + a256 - 1) / a256 * a256;
    d_maps[k] = reinterpret_cast<const float *>(base + 2 * ((img + a256 - 1) / a256 * a256));
  }
  int rc = check_filter_args(b, d_in[0], row, d_out[0], row, H, W, C, dtype, d_maps[0]);
  cudaStream_t cin = nullptr, cout = nullptr;
  cudaEvent_t ev[7] = {};  // alloc, in_ready[2], comp_done[2], out_done[2]
  if (rc == DISK_OK) {
    cudaError_t e = cudaStreamCreateWithFlags(&cin, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cout, cudaStreamNonBlocking);
    for (int i = 0; i < 7 && e == cudaSuccess; ++i)
      e = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
    if (e != cudaSuccess) rc = cuda_fail(e, "frame streams and events");
  }
  if (rc == DISK_OK) {
    cudaEvent_t *in_ready = ev + 1, *comp_done = ev + 3, *out_done = ev + 5;
    const std::vector<int> pix = layer_pix(b, H, W, C, dtype, false);
    cudaEventRecord(ev[0], s);  // the slots exist on s from here on
    cudaStreamWaitEvent(cin, ev[0], 0);
    cudaStreamWaitEvent(cout, ev[0], 0);
    for (int i = 0; i < n_frames && rc == DISK_OK; ++i) {
      const int k = i % S;
      if (i >= S) cudaStreamWaitEvent(cin, comp_done[k], 0);  // slot input consumed
      cudaMemcpyAsync(const_cast<void *>(d_in[k]), h_in[i], img, cudaMemcpyHostToDevice, cin);
      cudaMemcpyAsync(const_cast<float *>(d_maps[k]), h_maps[i], map, cudaMemcpyHostToDevice, cin);
      cudaEventRecord(in_ready[k], cin);
      cudaStreamWaitEvent(s, in_ready[k], 0);
      if (i >= S) cudaStreamWaitEvent(s, out_done[k], 0);  // slot output read back
      rc = filter_with(b, d_in[k], row, d_out[k], row, H, W, C, dtype, d_maps[k], nullptr, s,
                       pix.data());
      cudaEventRecord(comp_done[k], s);
      cudaStreamWaitEvent(cout, comp_done[k], 0);
      cudaMemcpyAsync(h_out[i], d_out[k], img, cudaMemcpyDeviceToHost, cout);
      cudaEventRecord(out_done[k], cout);
    }
    for (int k = 0; k < S; ++k) cudaStreamWaitEvent(s, out_done[k], 0);
    const cudaError_t e = cudaGetLastError();
    if (rc == DISK_OK && e != cudaSuccess) rc = cuda_fail(e, "frame pipeline");
  }
  // Freed in stream order after the last read-back; streams and events are
  // released by the runtime once their work has completed.
  cudaFreeAsync(buf, s);
  for (auto &x : ev)
    if (x) cudaEventDestroy(x);
  if (cin) cudaStreamDestroy(cin);
  if (cout) cudaStreamDestroy(cout);
  return rc;
}

extern "C" int disk_sv_filter_set_tile(const disk_basis *b, int H, int W, int C, int dtype, int pix) {
  if (!b) return fail(DISK_ERR_INVALID_ARG, "null basis");
  if (pix != 2 && pix != 4) return fail(DISK_ERR_INVALID_ARG, "pixels per thread must be 2 or 4");
  for (int l = 0; l < b->L; ++l)
    if (!fits_layer(b, C, l, pix, false))
      return fail(DISK_ERR_UNSUPPORTED, "layer halo exceeds shared memory for this tile");
  std::lock_guard<std::mutex> lock(b->tune_mu);
  b->tune_pix[tune_key(H, W, C, dtype, false)] = std::vector<int>(b->L, pix);
  return DISK_OK;
}

extern "C" int disk_sv_filter_set_layers(const disk_basis *b, int H, int W, int C, int dtype,
                                         const int *choice) {
  if (!b || !choice) return fail(DISK_ERR_INVALID_ARG, "null basis or choice");
  std::vector<int> pick(choice, choice + b->L);
  for (int l = 0; l < b->L; ++l) {
    if (pick[l] == kSvPairCode) {
      if (l + 1 >= b->L || pick[l + 1] != 0)
        return fail(DISK_ERR_INVALID_ARG, "a fused pair needs code 0 on the layer after it");
      if (!fits_pair(b, C, l)) return fail(DISK_ERR_UNSUPPORTED, "fused pair exceeds shared memory");
      ++l;
      continue;
    }
    if (pick[l] != 2 && pick[l] != 4) return fail(DISK_ERR_INVALID_ARG, "layer codes are 2, 4, or 8 then 0");
    if (!fits_layer(b, C, l, pick[l], false))
      return fail(DISK_ERR_UNSUPPORTED, "layer halo exceeds shared memory for this tile");
  }
  std::lock_guard<std::mutex> lock(b->tune_mu);
  b->tune_pix[tune_key(H, W, C, dtype, false)] = pick;
  return DISK_OK;
}

extern "C" int disk_selftest_bounded_wait(long long iterations, void *stream) {
  if (iterations < 1 || iterations > (1ll << 24))
    return fail(DISK_ERR_INVALID_ARG, "iterations must be in [1, 2^24]");
  int *err = device_error_word();
  if (!err) return fail(DISK_ERR_CUDA, "device status word unavailable");
  wait_selftest_kernel<<<1, 64, 0, static_cast<cudaStream_t>(stream)>>>(err, iterations);
  DISK_TRY_CUDA(cudaGetLastError(), "launch wait_selftest_kernel");
  return DISK_OK;
}
