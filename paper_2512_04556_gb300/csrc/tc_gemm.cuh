// FP32 matrix product on the fifth-generation tensor cores (tcgen05) for the
// learned initializer's network: C = op(A) op(B) with near-FP32 accuracy
// from four TF32 products (each operand x = hi + lo, hi = x rounded to TF32,
// lo the FP32 remainder, |lo| <= 2^-12 |x|; C = A_hi B_hi + A_hi B_lo +
// A_lo B_hi + A_lo B_lo accumulated in FP32 in tensor memory), the TF32
// rounding of the lo parts being ~2^-23 of each product.
//
// A split pass writes both operands K-major and padded (rows to the tile,
// K to 32) as hi/lo planes.  Each CTA (128 threads) owns a 128 x 64 tile of
// C and a range of K: one thread issues tensor-memory-accelerator copies of
// 32-deep K slices (128-byte swizzled rows) of the four planes into a
// four-stage ring, one thread issues the tcgen05.mma instructions
// (M = 128, N = 64, K = 8) as slices land and returns ring slots through
// tcgen05.commit, and the four warps read the accumulator out of tensor
// memory (tcgen05.ld) into a split-K slice; a second pass sums the slices in
// a fixed order and applies the epilogue.  Every wait is bounded: past its
// limit the CTA records DISK_ERR_TIMEOUT in the device status word, stores
// nothing, waits (bounded) for its own copies, frees its tensor memory and
// returns.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "internal.h"

namespace disk {
namespace tc {

constexpr int kM = 128, kN = 64, kK = 32, kStages = 4, kThreads = 128;
constexpr unsigned kABytes = kM * kK * 4;                       // 16 KB
constexpr unsigned kBBytes = kN * kK * 4;                       // 8 KB
constexpr unsigned kStageBytes = 2 * kABytes + 2 * kBBytes;     // 48 KB
constexpr size_t kSmem = (size_t)kStages * kStageBytes + 1024;  // + 1024-byte alignment slack
constexpr int kTmemCols = kN;                                   // FP32 accumulator, one column each
constexpr long long kWaitIters = 1ll << 24;

struct Args {
  CUtensorMap a_hi, a_lo;  // [Mp][Kp] FP32, box {32, 128}, 128-byte swizzle
  CUtensorMap b_hi, b_lo;  // [Np][Kp] FP32, box {32, 64}, 128-byte swizzle
  float *ws;               // split-K slices [splits][Mp][Np]
  int Mp, Np, Kp, kb_per_split;
  int *err;
};

__device__ __forceinline__ unsigned saddr(const void *p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ bool wait_bar(unsigned bar, unsigned parity) {
  for (long long i = 0; i < kWaitIters; ++i) {
    unsigned ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;"
        " selp.u32 %0, 1, 0, p; }"
        : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
    if (ok) return true;
  }
  return false;
}

// Shared-memory matrix descriptor of a K-major tile of 128-byte swizzled
// rows (8-row groups 1024 bytes apart), starting at shared address a.
__device__ __forceinline__ unsigned long long sw128_desc(unsigned a) {
  unsigned long long d = (unsigned long long)((a & 0x3FFFFu) >> 4);  // start address / 16
  d |= 1ull << 16;                                                  // leading offset (unused)
  d |= (unsigned long long)(1024 >> 4) << 32;                       // stride offset / 16
  d |= 1ull << 46;                                                  // descriptor version
  d |= 2ull << 61;                                                  // 128-byte swizzle
  return d;
}

// Instruction descriptor: D FP32, A and B TF32, both K-major, M x N.
constexpr unsigned kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((unsigned)(kN >> 3) << 17) |
                            ((unsigned)(kM >> 4) << 24);

__device__ __forceinline__ void tma_2d(unsigned dst, const CUtensorMap *map, int x, int y,
                                       unsigned bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];"
      :: "r"(dst), "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void mma(unsigned tmem, unsigned long long ad, unsigned long long bd,
                                    unsigned acc) {
  asm volatile(
      "{ .reg .pred p; setp.ne.b32 p, %4, 0;"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p; }"
      :: "r"(tmem), "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc) : "memory");
}

__device__ __forceinline__ void commit(unsigned bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
               :: "r"(bar) : "memory");
}

__global__ void __launch_bounds__(kThreads, 1) gemm_kernel(const __grid_constant__ Args A) {
  extern __shared__ unsigned char raw[];
  __shared__ __align__(8) unsigned long long full[kStages], empty[kStages], done;
  __shared__ unsigned tmem_slot;
  const unsigned tiles = (saddr(raw) + 1023u) & ~1023u;  // swizzled tiles need 1024-byte alignment
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n0 = blockIdx.x * kN, m0 = blockIdx.y * kM;
  const int kb0 = blockIdx.z * A.kb_per_split;
  const int nkb = max(0, min(A.kb_per_split, A.Kp / kK - kb0));
  // shared addresses of slot s's four tiles
  auto a_hi = [&](int s) { return tiles + (unsigned)s * kStageBytes; };
  auto a_lo = [&](int s) { return tiles + (unsigned)s * kStageBytes + kABytes; };
  auto b_hi = [&](int s) { return tiles + (unsigned)s * kStageBytes + 2 * kABytes; };
  auto b_lo = [&](int s) { return tiles + (unsigned)s * kStageBytes + 2 * kABytes + kBBytes; };
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(saddr(&full[s])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(saddr(&empty[s])) : "memory");
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(saddr(&done)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(saddr(&tmem_slot)), "r"(kTmemCols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = tmem_slot;
  bool ok = true;
  if (warp == 0 && lane == 0) {
    // producer: the four planes' K slices into the ring
    int issued[kStages] = {0, 0, 0, 0};
    for (int i = 0; i < nkb && ok; ++i) {
      const int s = i % kStages;
      if (i >= kStages) ok = wait_bar(saddr(&empty[s]), ((i / kStages) - 1) & 1);
      if (!ok) break;
      const unsigned fb = saddr(&full[s]);
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                   :: "r"(fb), "r"(kStageBytes) : "memory");
      const int kx = (kb0 + i) * kK;
      tma_2d(a_hi(s), &A.a_hi, kx, m0, fb);
      tma_2d(a_lo(s), &A.a_lo, kx, m0, fb);
      tma_2d(b_hi(s), &A.b_hi, kx, n0, fb);
      tma_2d(b_lo(s), &A.b_lo, kx, n0, fb);
      ++issued[s];
    }
    if (!ok) {
      // copies this thread issued may still be landing: wait for each
      // slot's last one (bounded) before the CTA can leave
      for (int s = 0; s < kStages; ++s)
        if (issued[s]) wait_bar(saddr(&full[s]), (issued[s] - 1) & 1);
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer: the four hi/lo products for each 8-deep step
    for (int i = 0; i < nkb && ok; ++i) {
      const int s = i % kStages;
      ok = wait_bar(saddr(&full[s]), (i / kStages) & 1);
      if (!ok) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const unsigned ah = a_hi(s), al = a_lo(s), bh = b_hi(s), bl = b_lo(s);
#pragma unroll
      for (int j = 0; j < kK / 8; ++j) {
        const unsigned o = j * 32;  // 8 TF32 values = 32 bytes along the swizzled row
        mma(tmem, sw128_desc(ah + o), sw128_desc(bh + o), (i | j) != 0);
        mma(tmem, sw128_desc(ah + o), sw128_desc(bl + o), 1u);
        mma(tmem, sw128_desc(al + o), sw128_desc(bh + o), 1u);
        mma(tmem, sw128_desc(al + o), sw128_desc(bl + o), 1u);
      }
      commit(saddr(&empty[s]));  // the slot is free once these products are done
    }
    commit(saddr(&done));  // arrives when every product issued above has completed
  }
  __syncwarp();
  __syncthreads();  // both roles have finished issuing, the last commit included
  const bool landed = wait_bar(saddr(&done), 0);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const bool good = __syncthreads_and(ok && landed);
  if (good && nkb > 0) {
    // warp w reads tensor-memory lanes (rows) 32 w .. 32 w + 31
    const int row = m0 + warp * 32 + lane;
    float *dst = A.ws + (size_t)blockIdx.z * A.Mp * A.Np + (size_t)row * A.Np + n0;
#pragma unroll
    for (int c0 = 0; c0 < kN; c0 += 32) {
      unsigned r[32];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10,"
          " %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27,"
          " %28, %29, %30, %31}, [%32];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
            "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
            "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
            "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
            "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
            "=r"(r[31])
          : "r"(tmem + ((unsigned)(warp * 32) << 16) + (unsigned)c0));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int q = 0; q < 8; ++q)
        reinterpret_cast<float4 *>(dst + c0)[q] =
            make_float4(__uint_as_float(r[4 * q]), __uint_as_float(r[4 * q + 1]),
                        __uint_as_float(r[4 * q + 2]), __uint_as_float(r[4 * q + 3]));
    }
  } else if (good) {
    // an empty K range (not planned, kept exact): a zero slice
    const int row = m0 + warp * 32 + lane;
    float *dst = A.ws + (size_t)blockIdx.z * A.Mp * A.Np + (size_t)row * A.Np + n0;
    for (int c = 0; c < kN; ++c) dst[c] = 0.f;
  } else if (threadIdx.x == 0) {
    atomicExch(A.err, DISK_ERR_TIMEOUT);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                 :: "r"(tmem), "r"(kTmemCols) : "memory");
}

// hi/lo planes [Rp][Kp] of op(S) (element (r, k) = T ? S[k ld + r] :
// S[r ld + k], zero outside R x K): hi = the value rounded to the nearest
// TF32 number (10 fraction bits; ties away from zero), lo = value - hi
// (exact in FP32).  32 x 32 tiles through shared memory, so a transposed
// source is read along rows.
template <bool T>
__global__ void split_kernel(const float *__restrict__ S, int R, int K, int ld,
                             float *__restrict__ hi, float *__restrict__ lo, int Kp) {
  __shared__ float tile[32][33];
  const int r0 = blockIdx.y * 32, k0 = blockIdx.x * 32, tx = threadIdx.x, ty = threadIdx.y;
  auto put = [&](int r, int k, float v) {
    // adding half a TF32 unit to the magnitude's bits and truncating rounds
    // to nearest (a carry into the exponent is the correct result)
    const float h = __uint_as_float((__float_as_uint(v) + 0x1000u) & 0xFFFFE000u);
    hi[(size_t)r * Kp + k] = h;
    lo[(size_t)r * Kp + k] = v - h;
  };
  if (T) {
    for (int i = ty; i < 32; i += 8) {  // tile[k][r], read along r
      const int k = k0 + i, r = r0 + tx;
      tile[i][tx] = (r < R && k < K) ? S[(size_t)k * ld + r] : 0.f;
    }
    __syncthreads();
    for (int i = ty; i < 32; i += 8) put(r0 + i, k0 + tx, tile[tx][i]);
  } else {
    for (int i = ty; i < 32; i += 8) {
      const int r = r0 + i, k = k0 + tx;
      put(r, k, (r < R && k < K) ? S[(size_t)r * ld + k] : 0.f);
    }
  }
}

using EncodeTiled = PFN_cuTensorMapEncodeTiled_v12000;

inline EncodeTiled encoder() {
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

// Tensor map of an FP32 plane [rows][Kp] read in {32, box_rows} boxes of
// 128-byte swizzled rows.
inline bool encode_plane(EncodeTiled fn, CUtensorMap *m, const float *base, int rows, int Kp,
                         int box_rows) {
  const cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)Kp * 4};
  const cuuint32_t box[2] = {(cuuint32_t)kK, (cuuint32_t)box_rows};
  const cuuint32_t es[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

inline int round_up(int v, int m) { return (v + m - 1) / m * m; }

// C [M][N] (ld ldc) slices of op(A) op(B) into ws [splits][Mp][Np]; returns
// the number of slices (0 on error, with the status recorded).  ws and the
// hi/lo planes come from the library's memory pool; the caller frees *ws.
template <bool TA, bool TB>
int gemm_slices(const float *A, const float *B, int M, int N, int K, int lda, int ldb,
                float **ws, int *Mp_out, int *Np_out, int *rc, cudaStream_t s) {
  *rc = DISK_OK;
  const EncodeTiled fn = encoder();
  if (!fn) { *rc = fail(DISK_ERR_UNSUPPORTED, "cuTensorMapEncodeTiled unavailable"); return 0; }
  int *err = device_error_word();
  if (!err) { *rc = fail(DISK_ERR_CUDA, "device status word unavailable"); return 0; }
  const int Mp = round_up(M, kM), Np = round_up(N, kN), Kp = round_up(K, kK), kbs = Kp / kK;
  const int tiles = (Mp / kM) * (Np / kN);
  // enough K slices to give every SM a CTA, each at least two stages deep
  int per = std::max(2, (kbs * tiles + 151) / 152);
  per = std::min(per, kbs);
  const int splits = (kbs + per - 1) / per;
  const size_t a_el = (size_t)Mp * Kp, b_el = (size_t)Np * Kp, w_el = (size_t)splits * Mp * Np;
  float *buf = nullptr;
  cudaError_t e = scratch_alloc(&buf, (2 * a_el + 2 * b_el) * sizeof(float), s);
  if (e != cudaSuccess) { *rc = cuda_fail(e, "scratch_alloc(tensor-core operands)"); return 0; }
  e = scratch_alloc(ws, w_el * sizeof(float), s);
  if (e != cudaSuccess) {
    cudaFreeAsync(buf, s);
    *rc = cuda_fail(e, "scratch_alloc(tensor-core slices)");
    return 0;
  }
  float *a_hi = buf, *a_lo = a_hi + a_el, *b_hi = a_lo + a_el, *b_lo = b_hi + b_el;
  // A: rows m of op(A); B: rows n of op(B)^T, i.e. element (n, k) = op(B)(k, n)
  split_kernel<TA><<<dim3(Kp / 32, Mp / 32), dim3(32, 8), 0, s>>>(A, M, K, lda, a_hi, a_lo, Kp);
  split_kernel<!TB><<<dim3(Kp / 32, Np / 32), dim3(32, 8), 0, s>>>(B, N, K, ldb, b_hi, b_lo, Kp);
  e = cudaGetLastError();
  static thread_local Args args;
  bool enc = e == cudaSuccess && encode_plane(fn, &args.a_hi, a_hi, Mp, Kp, kM) &&
             encode_plane(fn, &args.a_lo, a_lo, Mp, Kp, kM) &&
             encode_plane(fn, &args.b_hi, b_hi, Np, Kp, kN) &&
             encode_plane(fn, &args.b_lo, b_lo, Np, Kp, kN);
  if (e == cudaSuccess && enc) {
    args.ws = *ws;
    args.Mp = Mp; args.Np = Np; args.Kp = Kp; args.kb_per_split = per;
    args.err = err;
    static int attr_dev = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (attr_dev != dev) {
      e = cudaFuncSetAttribute(gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
      if (e == cudaSuccess) attr_dev = dev;
    }
    if (e == cudaSuccess) {
      gemm_kernel<<<dim3(Np / kN, Mp / kM, splits), kThreads, kSmem, s>>>(args);
      e = cudaGetLastError();
    }
  }
  cudaFreeAsync(buf, s);  // stream order: freed after the product has read it
  if (e != cudaSuccess || !enc) {
    cudaFreeAsync(*ws, s);
    *rc = e != cudaSuccess ? cuda_fail(e, "launch tensor-core gemm")
                           : fail(DISK_ERR_CUDA, "tensor map encoding failed");
    return 0;
  }
  *Mp_out = Mp;
  *Np_out = Np;
  return splits;
}

}  // namespace tc
}  // namespace disk
