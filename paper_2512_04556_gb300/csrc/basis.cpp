// Basis handles (Sec. 4.3, Eq. 8): construction, validation, file I/O,
// error strings.  Host code only.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>

#include <mutex>

#include "internal.h"

namespace disk {

static thread_local std::string g_last_msg;

int fail(int code, const std::string &msg) {
  g_last_msg = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char *what) {
  cudaGetLastError();  // clear the sticky-free error state of the runtime
  std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" +
                  cudaGetErrorString(e) + ")";
  return fail(e == cudaErrorMemoryAllocation ? DISK_ERR_OOM : DISK_ERR_CUDA, m);
}

cudaError_t scratch_alloc_raw(void **p, size_t bytes, cudaStream_t s) {
  static std::mutex mu;
  static cudaMemPool_t pools[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  cudaMemPool_t pool;
  {
    std::lock_guard<std::mutex> lock(mu);
    if (!pools[dev]) {
      cudaMemPoolProps props = {};
      props.allocType = cudaMemAllocationTypePinned;
      props.location.type = cudaMemLocationTypeDevice;
      props.location.id = dev;
      cudaMemPool_t np;
      e = cudaMemPoolCreate(&np, &props);
      if (e != cudaSuccess) return e;
      unsigned long long keep = ~0ull;
      e = cudaMemPoolSetAttribute(np, cudaMemPoolAttrReleaseThreshold, &keep);
      if (e != cudaSuccess) {
        cudaMemPoolDestroy(np);
        return e;
      }
      pools[dev] = np;
    }
    pool = pools[dev];
  }
  return cudaMallocFromPoolAsync(p, bytes, pool, s);
}

int *device_error_word() {
  static std::mutex mu;
  static int *words[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (!words[dev]) {
    int *w = nullptr;
    if (cudaMalloc(&w, sizeof(int)) != cudaSuccess) return nullptr;
    if (cudaMemset(w, 0, sizeof(int)) != cudaSuccess) { cudaFree(w); return nullptr; }
    words[dev] = w;
  }
  return words[dev];
}

void make_axes(int dims, const int *n_nodes, const float *node_vals, AxisNodes ax[2]) {
  int off = 0;
  for (int a = 0; a < 2; ++a) {
    std::memset(&ax[a], 0, sizeof(AxisNodes));
    int n = (a < dims) ? n_nodes[a] : 1;
    ax[a].n = n;
    for (int i = 0; i < n; ++i) ax[a].v[i] = (a < dims) ? node_vals[off + i] : 0.f;
    for (int i = 0; i + 1 < n; ++i) ax[a].inv[i] = 1.0f / (ax[a].v[i + 1] - ax[a].v[i]);
    if (a < dims) off += n;
  }
}

int validate_nodes(int dims, const int *n_nodes, const float *node_vals) {
  if (dims != 1 && dims != 2) return fail(DISK_ERR_INVALID_ARG, "dims must be 1 or 2");
  if (!n_nodes || !node_vals) return fail(DISK_ERR_INVALID_ARG, "null node arrays");
  int off = 0;
  for (int a = 0; a < dims; ++a) {
    int n = n_nodes[a];
    if (n < 1 || n > DISK_MAX_NODES_AXIS)
      return fail(DISK_ERR_INVALID_ARG, "nodes per axis must be in [1, 64]");
    for (int i = 0; i < n; ++i) {
      float v = node_vals[off + i];
      if (!std::isfinite(v)) return fail(DISK_ERR_INVALID_ARG, "non-finite node value");
      if (i > 0 && !(v > node_vals[off + i - 1]))
        return fail(DISK_ERR_INVALID_ARG, "node values must increase strictly");
    }
    off += n;
  }
  return DISK_OK;
}

int validate_image_args(const void *d_in, size_t in_pitch, const void *d_out,
                        size_t out_pitch, int H, int W, int C, int dtype,
                        const float *d_maps) {
  if (!d_in || !d_out || !d_maps) return fail(DISK_ERR_INVALID_ARG, "null image or map pointer");
  if (H < 1 || W < 1 || H > 32768 || W > 32768)
    return fail(DISK_ERR_INVALID_ARG, "H and W must be in [1, 32768]");
  if (C != 3 && C != 4) return fail(DISK_ERR_INVALID_ARG, "C must be 3 or 4");
  if (dtype != DISK_F32 && dtype != DISK_F16) return fail(DISK_ERR_INVALID_ARG, "bad dtype");
  size_t es = dtype == DISK_F32 ? 4 : 2;
  size_t row = (size_t)W * C * es;
  if (in_pitch < row || out_pitch < row || in_pitch % es || out_pitch % es)
    return fail(DISK_ERR_INVALID_ARG, "pitch smaller than a row or not a multiple of the element size");
  if (((uintptr_t)d_in % es) || ((uintptr_t)d_out % es) || ((uintptr_t)d_maps % 4))
    return fail(DISK_ERR_INVALID_ARG, "misaligned image or map pointer");
  const char *a0 = (const char *)d_in, *a1 = a0 + in_pitch * (H - 1) + row;
  const char *b0 = (const char *)d_out, *b1 = b0 + out_pitch * (H - 1) + row;
  if (a0 < b1 && b0 < a1) return fail(DISK_ERR_INVALID_ARG, "input and output overlap");
  return DISK_OK;
}

}  // namespace disk

using disk::fail;

extern "C" int disk_version(void) { return 10000; }

extern "C" const char *disk_error_string(int status) {
  switch (status) {
    case DISK_OK: return "DISK_OK";
    case DISK_ERR_INVALID_ARG: return "DISK_ERR_INVALID_ARG";
    case DISK_ERR_BAD_FILE: return "DISK_ERR_BAD_FILE";
    case DISK_ERR_UNSUPPORTED: return "DISK_ERR_UNSUPPORTED";
    case DISK_ERR_CUDA: return "DISK_ERR_CUDA";
    case DISK_ERR_OOM: return "DISK_ERR_OOM";
    case DISK_ERR_TIMEOUT: return "DISK_ERR_TIMEOUT";
    default: return "DISK_ERR_UNKNOWN";
  }
}

extern "C" const char *disk_last_error_message(void) { return disk::g_last_msg.c_str(); }

extern "C" int disk_basis_from_arrays(int dims, const int *n_nodes, const float *node_vals,
                                      int L, int T, const float *theta, disk_basis **out) {
  if (!out) return fail(DISK_ERR_INVALID_ARG, "null out pointer");
  *out = nullptr;
  int rc = disk::validate_nodes(dims, n_nodes, node_vals);
  if (rc) return rc;
  if (L < 1 || L > DISK_MAX_LAYERS || T < 1 || T > DISK_MAX_TAPS)
    return fail(DISK_ERR_INVALID_ARG, "L must be in [1, 16] and T in [1, 64]");
  if (!theta) return fail(DISK_ERR_INVALID_ARG, "null theta");
  std::unique_ptr<disk_basis> b(new disk_basis());
  b->dims = dims;
  b->n_nodes[0] = n_nodes[0];
  b->n_nodes[1] = dims == 2 ? n_nodes[1] : 1;
  b->B = b->n_nodes[0] * b->n_nodes[1];
  b->L = L;
  b->T = T;
  b->node_vals.assign(node_vals, node_vals + n_nodes[0] + (dims == 2 ? n_nodes[1] : 0));
  size_t n = (size_t)b->B * L * T * 3;
  b->theta.assign(theta, theta + n);
  b->reach.assign(L, 0.f);
  b->reach_norm.assign(L, 0.f);
  std::vector<float4> taps((size_t)L * b->B * T);
  for (int k = 0; k < b->B; ++k)
    for (int l = 0; l < L; ++l)
      for (int i = 0; i < T; ++i) {
        const float *t = &b->theta[(((size_t)k * L + l) * T + i) * 3];
        if (!std::isfinite(t[0]) || !std::isfinite(t[1]) || !std::isfinite(t[2]))
          return fail(DISK_ERR_INVALID_ARG, "non-finite theta");
        float r = std::fmax(std::fabs(t[0]), std::fabs(t[1]));
        if (r > DISK_MAX_REACH)
          return fail(DISK_ERR_UNSUPPORTED, "tap offset beyond DISK_MAX_REACH");
        b->reach[l] = std::fmax(b->reach[l], r);
        b->reach_norm[l] = std::fmax(b->reach_norm[l], std::hypot(t[0], t[1]));
        taps[((size_t)l * b->B + k) * T + i] = make_float4(t[0], t[1], t[2], t[2]);
      }
  DISK_TRY_CUDA(cudaGetDevice(&b->device), "cudaGetDevice");
  // the device status word the filter kernels report to, allocated now so
  // that no later call (possibly inside a graph capture) has to
  if (!disk::device_error_word()) return fail(DISK_ERR_CUDA, "device status word allocation failed");
  // the pair layout of the 3-channel filter, after the plain table: per node
  // and tap pair (2j, 2j + 1), the offsets, then the weights of the node and
  // of its successor on axis 0 (the cell corner n10 of a corner n00)
  const size_t nt = taps.size();
  taps.resize(2 * nt);
  const int n1 = dims == 2 ? n_nodes[1] : 1;
  for (int l = 0; l < L; ++l)
    for (int k = 0; k < b->B; ++k) {
      const int k0 = k / n1, k1 = k % n1;
      const int succ = std::min(k0 + 1, n_nodes[0] - 1) * n1 + k1;
      const float4 *q = &taps[((size_t)l * b->B + k) * T];
      const float4 *qs = &taps[((size_t)l * b->B + succ) * T];
      float4 *o = &taps[nt + ((size_t)l * b->B + k) * T];
      for (int i = 0; i + 1 < T; i += 2) {
        o[i] = make_float4(q[i].x, q[i + 1].x, q[i].y, q[i + 1].y);
        o[i + 1] = make_float4(q[i].z, q[i + 1].z, qs[i].z, qs[i + 1].z);
      }
      if (T & 1) o[T - 1] = q[T - 1];
    }
  DISK_TRY_CUDA(cudaMalloc(&b->d_taps, taps.size() * sizeof(float4)), "cudaMalloc(basis)");
  b->d_taps_pair = b->d_taps + nt;
  cudaError_t e = cudaMemcpy(b->d_taps, taps.data(), taps.size() * sizeof(float4),
                             cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(b->d_taps);
    return disk::cuda_fail(e, "cudaMemcpy(basis)");
  }
  *out = b.release();
  return DISK_OK;
}

extern "C" void disk_basis_free(disk_basis *b) {
  if (!b) return;
  if (b->d_taps) {
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != b->device) cudaSetDevice(b->device);
    cudaFree(b->d_taps);
    if (cur != b->device) cudaSetDevice(cur);
  }
  delete b;
}

extern "C" int disk_basis_info(const disk_basis *b, int *dims, int *n_nodes2, int *L, int *T) {
  if (!b) return fail(DISK_ERR_INVALID_ARG, "null basis");
  if (dims) *dims = b->dims;
  if (n_nodes2) { n_nodes2[0] = b->n_nodes[0]; n_nodes2[1] = b->n_nodes[1]; }
  if (L) *L = b->L;
  if (T) *T = b->T;
  return DISK_OK;
}

// ---- file format ---------------------------------------------------------
// "DISKBAS1" | u32 version=1 | u32 dims | u32 L | u32 T | u32 n0 | u32 n1 |
// f32 node_vals[n0 (+ n1)] | f32 theta[B*L*T*3] | u64 FNV-1a of all above.

static uint64_t fnv1a64(const unsigned char *p, size_t n) {
  uint64_t h = 0xcbf29ce484222325ull;  // FNV offset basis
  for (size_t i = 0; i < n; ++i) {
    h ^= p[i];
    h *= 0x100000001b3ull;             // FNV prime
  }
  return h;
}

static void put_u32(std::vector<unsigned char> &v, uint32_t x) {
  for (int i = 0; i < 4; ++i) v.push_back((unsigned char)(x >> (8 * i)));
}
static uint32_t get_u32(const unsigned char *p) {
  return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}
static void put_f32(std::vector<unsigned char> &v, float f) {
  uint32_t x;
  std::memcpy(&x, &f, 4);
  put_u32(v, x);
}
static float get_f32(const unsigned char *p) {
  uint32_t x = get_u32(p);
  float f;
  std::memcpy(&f, &x, 4);
  return f;
}

extern "C" int disk_basis_save(const disk_basis *b, const char *path) {
  if (!b || !path) return fail(DISK_ERR_INVALID_ARG, "null basis or path");
  std::vector<unsigned char> buf;
  const char magic[8] = {'D', 'I', 'S', 'K', 'B', 'A', 'S', '1'};
  buf.insert(buf.end(), magic, magic + 8);
  put_u32(buf, 1);
  put_u32(buf, b->dims);
  put_u32(buf, b->L);
  put_u32(buf, b->T);
  put_u32(buf, b->n_nodes[0]);
  put_u32(buf, b->n_nodes[1]);
  for (float v : b->node_vals) put_f32(buf, v);
  for (float v : b->theta) put_f32(buf, v);
  uint64_t h = fnv1a64(buf.data(), buf.size());
  for (int i = 0; i < 8; ++i) buf.push_back((unsigned char)(h >> (8 * i)));
  FILE *f = std::fopen(path, "wb");
  if (!f) return fail(DISK_ERR_BAD_FILE, std::string("cannot open for writing: ") + path);
  size_t w = std::fwrite(buf.data(), 1, buf.size(), f);
  int cl = std::fclose(f);
  if (w != buf.size() || cl != 0) return fail(DISK_ERR_BAD_FILE, "short write");
  return DISK_OK;
}

extern "C" int disk_basis_load(const char *path, disk_basis **out) {
  if (!path || !out) return fail(DISK_ERR_INVALID_ARG, "null path or out pointer");
  *out = nullptr;
  FILE *f = std::fopen(path, "rb");
  if (!f) return fail(DISK_ERR_BAD_FILE, std::string("cannot open: ") + path);
  std::vector<unsigned char> buf;
  unsigned char tmp[65536];
  size_t r;
  while ((r = std::fread(tmp, 1, sizeof(tmp), f)) > 0) {
    buf.insert(buf.end(), tmp, tmp + r);
    if (buf.size() > (64u << 20)) { std::fclose(f); return fail(DISK_ERR_BAD_FILE, "file too large"); }
  }
  std::fclose(f);
  const size_t head = 8 + 6 * 4;
  if (buf.size() < head + 8) return fail(DISK_ERR_BAD_FILE, "truncated header");
  if (std::memcmp(buf.data(), "DISKBAS1", 8) != 0) return fail(DISK_ERR_BAD_FILE, "bad magic");
  const unsigned char *p = buf.data() + 8;
  uint32_t ver = get_u32(p), dims = get_u32(p + 4), L = get_u32(p + 8), T = get_u32(p + 12);
  uint32_t n0 = get_u32(p + 16), n1 = get_u32(p + 20);
  if (ver != 1) return fail(DISK_ERR_BAD_FILE, "unsupported version");
  if ((dims != 1 && dims != 2) || L < 1 || L > DISK_MAX_LAYERS || T < 1 || T > DISK_MAX_TAPS ||
      n0 < 1 || n0 > DISK_MAX_NODES_AXIS || n1 < 1 || n1 > DISK_MAX_NODES_AXIS ||
      (dims == 1 && n1 != 1))
    return fail(DISK_ERR_BAD_FILE, "header fields out of range");
  size_t nv = n0 + (dims == 2 ? n1 : 0), B = (size_t)n0 * n1, nt = B * L * T * 3;
  size_t need = head + 4 * (nv + nt) + 8;
  if (buf.size() != need) return fail(DISK_ERR_BAD_FILE, "file size does not match header");
  uint64_t h = 0;
  for (int i = 0; i < 8; ++i) h |= (uint64_t)buf[need - 8 + i] << (8 * i);
  if (h != fnv1a64(buf.data(), need - 8)) return fail(DISK_ERR_BAD_FILE, "checksum mismatch");
  std::vector<float> vals(nv), theta(nt);
  const unsigned char *q = buf.data() + head;
  for (size_t i = 0; i < nv; ++i) vals[i] = get_f32(q + 4 * i);
  q += 4 * nv;
  for (size_t i = 0; i < nt; ++i) theta[i] = get_f32(q + 4 * i);
  int nn[2] = {(int)n0, (int)n1};
  int rc = disk_basis_from_arrays((int)dims, nn, vals.data(), (int)L, (int)T, theta.data(), out);
  if (rc == DISK_ERR_INVALID_ARG) return fail(DISK_ERR_BAD_FILE, "invalid basis contents");
  return rc;
}

extern "C" int disk_device_status(void *stream) {
  int *w = disk::device_error_word();
  if (!w) return fail(DISK_ERR_CUDA, "device status word unavailable");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int h = 0;
  DISK_TRY_CUDA(cudaMemcpyAsync(&h, w, sizeof(int), cudaMemcpyDeviceToHost, s), "read device status");
  DISK_TRY_CUDA(cudaMemsetAsync(w, 0, sizeof(int), s), "clear device status");
  DISK_TRY_CUDA(cudaStreamSynchronize(s), "cudaStreamSynchronize(device status)");
  if (h == DISK_ERR_TIMEOUT) return fail(DISK_ERR_TIMEOUT, "a kernel gave up a bounded wait for a tile copy");
  return h ? fail(h, "device-side error") : DISK_OK;
}
