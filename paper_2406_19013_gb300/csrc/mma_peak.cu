// mma_peak.cu -- dense tcgen05 MMA throughput on the current GPU, for the
// roofline of the CMAC kernel (a measurement helper; the paper has no
// counterpart).
//
// Every SM runs one CTA that keeps a 128 x 128-byte A tile and a 256 x
// 128-byte B tile of E5M2 values in shared memory (128B-swizzled, K-major,
// the layout the CMAC kernel's operands use) and issues back-to-back
// tcgen05.mma.kind::f8f6f4 instructions (M = 128, N = n, K = 32) from one to
// four threads, each into its own fp32 accumulator in TMEM.  Optionally the A
// operand is read from TMEM instead.  Nothing but the MMAs runs in the timed
// loop, so the launch's duration gives the tensor pipe's dense fp8 rate with
// fp32 accumulation; the per-CTA cycle count gives the cycles per MMA.
#include <cuda_runtime.h>

#include "corr.h"
#include "ptx.cuh"
#include "xe_internal.h"

namespace xe {
namespace {

constexpr int kPeakThreads = 128;
constexpr int kPeakATile = 128 * 128;   // bytes
constexpr int kPeakBTile = 256 * 128;   // bytes
constexpr int kPeakACols = 32;          // TMEM columns of an A operand held in TMEM (4 K slices)
constexpr int kPeakSmem = 120 * 1024;   // more than half of an SM: one CTA per SM

// D[tmem] (+)= A[tmem] * B[smem]^T, kind::f8f6f4.
__device__ __forceinline__ void mma_f8_ts(uint32_t d_tmem, uint32_t a_tmem, uint32_t b_lo,
                                          uint32_t b_hi, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\n.reg .b64 db;\nsetp.ne.b32 p, %5, 0;\n"
      "mov.b64 db, {%2, %3};\n"
      "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], [%1], db, %4, p;\n}" ::"r"(d_tmem),
      "r"(a_tmem), "r"(b_lo), "r"(b_hi), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void tmem_st_32x32b_x8(uint32_t taddr, uint32_t v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %1, %1, %1, %1, %1, %1, %1};" ::"r"(taddr),
      "r"(v)
      : "memory");
}

__device__ __forceinline__ void tmem_st_wait() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// Four E5M2 codes of integers in [-7, 7] from a hash of the word index.
__device__ __forceinline__ uint32_t operand_word(uint32_t k, uint32_t salt) {
  uint32_t h = k * 0x9E3779B1u ^ salt * 0x85EBCA77u;
  h ^= h >> 15;
  h *= 0x2C1B3C6Du;
  h ^= h >> 12;
  // E5M2 codes of 0..7 (1 = 0x3C, 2 = 0x40, 3 = 0x42, 4..7 = 0x44..0x47)
  const uint32_t lo = 0x42403C00u, hi = 0x47464544u;
  uint32_t w = 0;
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const uint32_t nib = (h >> (8 * b)) & 7u, sgn = (h >> (8 * b + 3)) & 1u;
    const uint32_t code = __byte_perm(lo, hi, nib) & 0xFFu;
    w |= (code | (code ? sgn << 7 : 0u)) << (8 * b);
  }
  return w;
}

__global__ void __launch_bounds__(kPeakThreads, 1)
    mma_rate_kernel(int n, int issuers, int iters, int a_from_tmem, int *status,
                    long long *cycles, unsigned long long timeout_ns) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  uint8_t *a_s = smem;
  uint8_t *b_s = smem + kPeakATile;
  uint64_t *bars = reinterpret_cast<uint64_t *>(b_s + kPeakBTile);  // one per issuer
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 4);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  uint32_t *words = reinterpret_cast<uint32_t *>(smem);
  for (int k = threadIdx.x; k < (kPeakATile + kPeakBTile) / 4; k += kPeakThreads)
    words[k] = operand_word((uint32_t)k, blockIdx.x);
  if (threadIdx.x == 0) {
    for (int m = 0; m < 4; ++m) mbar_init(smem_u32(bars + m), 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  fence_proxy_async_smem();
  if (warp == 0) {
    tmem_alloc(smem_u32(tmem_slot), kTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t a_col = (uint32_t)(kTmemCols - kPeakACols);
  if (a_from_tmem) {
    // every warp fills its lane quarter of the A columns
    const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
    for (int c = 0; c < kPeakACols; c += 8)
      tmem_st_32x32b_x8(tmem + lane_base + a_col + (uint32_t)c,
                        operand_word((uint32_t)(threadIdx.x * 64 + c), 77u));
    tmem_st_wait();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();

  if (warp < issuers && lane == 0) {
    const uint32_t idesc = idesc_e5m2_f32(128, n);
    const uint32_t d = tmem + (uint32_t)(warp * n);
    const uint32_t a_lo = sdesc_sw128_lo(smem_u32(a_s)), b_lo = sdesc_sw128_lo(smem_u32(b_s));
    const uint32_t hi = sdesc_sw128_hi(1024u);
    const long long t0 = clock64();
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const uint32_t acc = (it | kk) ? 1u : 0u;
        if (a_from_tmem)
          mma_f8_ts(d, tmem + a_col + 8u * kk, b_lo + 2u * kk, hi, idesc, acc);
        else
          mma_f8_ss_w(d, a_lo + 2u * kk, hi, b_lo + 2u * kk, hi, idesc, acc);
      }
    }
    const uint32_t bar = smem_u32(bars + warp);
    mma_commit(bar);
    if (!mbar_wait(bar, 0, abort_flag, timeout_ns)) atomicOr(status, 1);
    if (warp == 0 && cycles) cycles[blockIdx.x] = clock64() - t0;
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    __syncwarp();
    tc_fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
}

}  // namespace
}  // namespace xe

extern "C" int corr_mma_rate(int n, int issuers, int iters, int a_from_tmem, int *d_status,
                             long long *d_cycles, void *stream) {
  if (n < 16 || n > 256 || n % 16 != 0 || issuers < 1 || issuers > 4 || iters < 1 ||
      iters > 10000000 || (a_from_tmem != 0 && a_from_tmem != 1) || !d_status)
    return CORR_EINVAL;
  if (issuers * n + (a_from_tmem ? xe::kPeakACols : 0) > xe::kTmemCols) return CORR_EINVAL;
  int dev = 0, n_sm = 0, major = 0, minor = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess)
    return CORR_ECUDA;
  if (major != 10 || minor != 3) return CORR_EARCH;
  if (cudaFuncSetAttribute(xe::mma_rate_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           xe::kPeakSmem) != cudaSuccess)
    return CORR_ECUDA;
  xe::mma_rate_kernel<<<n_sm, xe::kPeakThreads, xe::kPeakSmem, static_cast<cudaStream_t>(stream)>>>(
      n, issuers, iters, a_from_tmem, d_status, d_cycles, 2000000000ull);
  return cudaGetLastError() == cudaSuccess ? CORR_OK : CORR_ECUDA;
}
