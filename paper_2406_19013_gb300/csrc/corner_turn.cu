// corner_turn.cu -- device corner turn of a block of packed samples,
// uint8 [time][channel][input] -> uint8 [channel][input][time].
//
// The F-engines emit one spectrum per time step: every channel of every
// input for sample t.  The X-engine wants, per channel, each input's samples
// contiguous in time (Sec. 2.1: the Transpose module reorders the F-engine
// output into a layout suited to the correlation).  This kernel performs that
// reorder in HBM: one read and one write of every byte, nothing else.
//
// A CTA moves 128 x 128-byte tiles (128 inputs x 128 time samples of one
// channel), 256 threads:
//   1. thread (q, g) loads inputs 16 g .. 16 g + 15 of samples 4 q .. 4 q + 3
//      (four 16-byte loads; 8 threads cover a 128-byte source run);
//   2. four 4 x 4 byte blocks are transposed in registers (byte permutes),
//      giving 16 words of 4 samples of one input each;
//   3. the words go to a shared tile [128 inputs][8 chunks of 16 bytes] whose
//      chunk index is XOR-swizzled with bits of the input index, so that the
//      word writes of step 3 and the 16-byte row reads of step 4 are free of
//      bank conflicts;
//   4. 8 threads read one tile row (128 samples of one input) and store it as
//      128 contiguous destination bytes.
#include <cuda_runtime.h>

#include <cstdint>

#include "xe_internal.h"
#include "xe_unpack.cuh"

namespace xe {

namespace {

constexpr int kTile = 128;        // inputs and samples per tile
constexpr int kTileWords = 32;    // 4-byte words per tile row
constexpr int kCtThreads = 256;   // 8 warps

// 16 source bytes: inputs n..n+15 of one sample (row_off = start of the
// sample's row of N inputs).  Vector load when the whole run is in range and
// aligned, else bytes (zero past the end).
__device__ __forceinline__ uint4 load_src16(const uint8_t *src, long long row_off, int n, int N,
                                            bool vec) {
  if (vec) return __ldg(reinterpret_cast<const uint4 *>(src + row_off + n));
  uint32_t w[4] = {0u, 0u, 0u, 0u};
  for (int k = 0; k < 16; ++k)
    if (n + k < N) w[k >> 2] |= (uint32_t)__ldg(src + row_off + n + k) << (8 * (k & 3));
  return make_uint4(w[0], w[1], w[2], w[3]);
}


// Word w (4 samples) of tile row r: chunk (w / 4) is stored at chunk
// (w / 4) ^ ((r / 16) & 7).
__device__ __forceinline__ int tile_word(int r, int w) {
  return r * kTileWords + ((((w >> 2) ^ (r >> 4)) & 7) << 2) + (w & 3);
}

__global__ void __launch_bounds__(kCtThreads)
    corner_turn_kernel(const uint8_t *__restrict__ src, uint8_t *__restrict__ dst, int N, int C,
                       int T, int pitch) {
  __shared__ __align__(16) uint32_t tile[kTile * kTileWords];
  const int tid = threadIdx.x;
  const int g = tid & 7, q = tid >> 3;  // input group of 16, sample group of 4
  const int n_tiles_n = (N + kTile - 1) / kTile, n_tiles_t = (T + kTile - 1) / kTile;
  // Tiles are visited in blocks of kBlkC channels x kBlkT time tiles (time
  // fastest), so that the CTAs resident at one time read neighbouring
  // channels' rows of the same samples and write neighbouring 128-byte runs
  // of the same destination rows (DRAM page locality on both sides).  2 x 16
  // was the fastest of the shapes timed on a 192-input, 1024-channel block
  // (1 x 64, the plain order, was 13 % slower; 8 x 8 and 4 x 32, 10-16 %).
  constexpr int kBlkC = 2, kBlkT = 16;
  const int n_bc = (C + kBlkC - 1) / kBlkC, n_bt = (n_tiles_t + kBlkT - 1) / kBlkT;
  const long long n_tiles = (long long)n_bc * n_bt * n_tiles_n * kBlkC * kBlkT;
  const bool src_vec = (N & 15) == 0;
  const bool dst_vec = (pitch & 15) == 0;
  for (long long tl = blockIdx.x; tl < n_tiles; tl += gridDim.x) {
    const int tt_lo = (int)(tl % kBlkT);
    long long rest = tl / kBlkT;
    const int c_lo = (int)(rest % kBlkC);
    rest /= kBlkC;
    const int tn = (int)(rest % n_tiles_n);
    rest /= n_tiles_n;
    const int tt = (int)(rest % n_bt) * kBlkT + tt_lo;
    const int c = (int)(rest / n_bt) * kBlkC + c_lo;
    if (tt >= n_tiles_t || c >= C) continue;  // the blocks' ragged edges (uniform per CTA)
    const int n0 = tn * kTile, t0 = tt * kTile;
    // ---- steps 1-3
    const int n = n0 + 16 * g;
    if (n < N) {
      const bool vec = src_vec && n + 15 < N;
      uint4 v[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int t = t0 + 4 * q + k;
        v[k] = t < T ? load_src16(src, ((long long)t * C + c) * (long long)N, n, N, vec)
                     : make_uint4(0u, 0u, 0u, 0u);
      }
      const uint32_t *w0 = &v[0].x, *w1 = &v[1].x, *w2 = &v[2].x, *w3 = &v[3].x;
#pragma unroll
      for (int b = 0; b < 4; ++b) {  // inputs n + 4 b .. + 3
        uint32_t o[4];
        transpose4(w0[b], w1[b], w2[b], w3[b], o[0], o[1], o[2], o[3]);
#pragma unroll
        for (int j = 0; j < 4; ++j) tile[tile_word(16 * g + 4 * b + j, q)] = o[j];
      }
    }
    __syncthreads();
    // ---- step 4: 8 threads per row, 32 rows per pass
    for (int row = tid >> 3; row < kTile; row += kCtThreads / 8) {
      const int nn = n0 + row;
      if (nn >= N) break;
      const int ch = tid & 7;  // 16-byte chunk: samples 16 ch .. + 15
      const uint4 val = *reinterpret_cast<const uint4 *>(&tile[tile_word(row, 4 * ch)]);
      const int t = t0 + 16 * ch;
      uint8_t *out = dst + ((long long)c * N + nn) * (long long)pitch;
      if (dst_vec && t + 15 < T) {
        *reinterpret_cast<uint4 *>(out + t) = val;
      } else {
        const uint32_t vv[4] = {val.x, val.y, val.z, val.w};
        for (int k = 0; k < 16; ++k)
          if (t + k < T) out[t + k] = (uint8_t)(vv[k >> 2] >> (8 * (k & 3)));
      }
    }
    __syncthreads();
  }
}

}  // namespace

cudaError_t launch_corner_turn(const uint8_t *src, uint8_t *dst, int n_in, int n_chan,
                               int block_len, int dst_pitch, cudaStream_t stream, int grid) {
  corner_turn_kernel<<<grid, kCtThreads, 0, stream>>>(src, dst, n_in, n_chan, block_len,
                                                      dst_pitch);
  return cudaGetLastError();
}

}  // namespace xe
