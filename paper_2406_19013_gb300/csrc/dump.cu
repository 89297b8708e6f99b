// dump.cu -- end of integration: visibilities, full-Stokes, reset; and the
// pitch copy used when block_len is not a multiple of 16 bytes.
//
// Full-Stokes (abstract, Sec. 1) per antenna pair p >= q, inputs 2p+pol:
//   XX = V[2p][2q], YY = V[2p+1][2q+1], XY = V[2p][2q+1], YX = V[2p+1][2q]
//   (p == q: XY = conj(V[2p+1][2p]), the element above the diagonal)
//   I = XX + YY, Q = XX - YY, U = XY + YX, V = -j (XY - YX)
// Each lower-triangle element belongs to exactly one antenna pair, so one
// thread per pair reads its 3 or 4 elements, writes them to the visibility
// output, zeroes them in the integration buffer and writes the four Stokes
// products -- one pass over HBM with no cross-thread hazards.  Consecutive
// threads take consecutive q, so the 32-byte (XX, XY) and (YX, YY) element
// pairs they touch are contiguous across the warp.
#include <cmath>

#include "xe_internal.h"

namespace xe {

namespace {

__device__ __forceinline__ long long tri_row(long long a) {
  // largest p with p(p+1)/2 <= a
  long long p = (long long)((sqrt(8.0 * (double)a + 1.0) - 1.0) * 0.5);
  while ((p + 1) * (p + 2) / 2 <= a) ++p;
  while (p * (p + 1) / 2 > a) --p;
  return p;
}

__global__ void dump_dual_kernel(int64_t *__restrict__ acc, int64_t *__restrict__ vis,
                                 int64_t *__restrict__ stokes, int n_ant, int n_chan,
                                 int *status) {
  const long long n_in = 2LL * n_ant;
  const long long P = n_in * (n_in + 1) / 2;
  const long long A = (long long)n_ant * (n_ant + 1) / 2;
  const long long total = A * n_chan;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long c = idx / A, a = idx - c * A;
    const long long p = tri_row(a), q = a - p * (p + 1) / 2;
    const long long r0 = (2 * p) * (2 * p + 1) / 2, r1 = (2 * p + 1) * (2 * p + 2) / 2;
    const long long base = c * P;
    // element offsets (in pairs) of XX, XY (p > q only), YX, YY
    const long long e_xx = base + r0 + 2 * q, e_xy = base + r0 + 2 * q + 1;
    const long long e_yx = base + r1 + 2 * q, e_yy = base + r1 + 2 * q + 1;
#ifdef CORR_DEBUG
    // every element this thread touches lies in channel c's part of the buffer
    if (p >= n_ant || q > p || e_xx < base || e_yy >= base + P) {
      atomicOr(status, kStatusBounds);
      continue;
    }
#endif
    longlong2 *a2 = reinterpret_cast<longlong2 *>(acc);
    const longlong2 zero = make_longlong2(0, 0);
    const longlong2 xx = a2[e_xx], yx = a2[e_yx], yy = a2[e_yy];
    longlong2 xy;
    if (p > q) {
      xy = a2[e_xy];
    } else {
      xy = make_longlong2(yx.x, -yx.y);
    }
    if (vis) {
      longlong2 *v2 = reinterpret_cast<longlong2 *>(vis);
      v2[e_xx] = xx;
      v2[e_yx] = yx;
      v2[e_yy] = yy;
      if (p > q) v2[e_xy] = xy;
    }
    a2[e_xx] = zero;
    a2[e_yx] = zero;
    a2[e_yy] = zero;
    if (p > q) a2[e_xy] = zero;
    if (stokes) {
      longlong2 *s2 = reinterpret_cast<longlong2 *>(stokes) + idx * 4;
      s2[0] = make_longlong2(xx.x + yy.x, xx.y + yy.y);            // I
      s2[1] = make_longlong2(xx.x - yy.x, xx.y - yy.y);            // Q
      s2[2] = make_longlong2(xy.x + yx.x, xy.y + yx.y);            // U
      s2[3] = make_longlong2(xy.y - yx.y, -(xy.x - yx.x));         // V = -j (XY - YX)
    }
  }
}

__global__ void dump_single_kernel(int64_t *__restrict__ acc, int64_t *__restrict__ vis,
                                   long long n_elems2) {
  longlong2 *a2 = reinterpret_cast<longlong2 *>(acc);
  longlong2 *v2 = reinterpret_cast<longlong2 *>(vis);
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n_elems2;
       idx += (long long)gridDim.x * blockDim.x) {
    const longlong2 v = a2[idx];
    if (v2) v2[idx] = v;
    a2[idx] = make_longlong2(0, 0);
  }
}

// Debug builds: one block compares both guard bands with kGuardByte.
__global__ void guard_check_kernel(const unsigned char *__restrict__ before,
                                   const unsigned char *__restrict__ after, size_t bytes,
                                   int *status) {
  const uint32_t want = 0x01010101u * kGuardByte;
  bool bad = false;
  for (size_t w = threadIdx.x; w < bytes / 4; w += blockDim.x)
    bad |= reinterpret_cast<const uint32_t *>(before)[w] != want ||
           reinterpret_cast<const uint32_t *>(after)[w] != want;
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(status, kStatusBounds);
}

// dst[row][0..pitch) = src[row][0..T) followed by zeros
__global__ void pitch_kernel(const uint8_t *__restrict__ src, uint8_t *__restrict__ dst,
                             long long rows, int T, int pitch) {
  for (long long r = blockIdx.x; r < rows; r += gridDim.x) {
    const uint8_t *s = src + r * (long long)T;
    uint8_t *d = dst + r * (long long)pitch;
    for (int t = threadIdx.x; t < pitch; t += blockDim.x) d[t] = t < T ? s[t] : 0;
  }
}

}  // namespace

cudaError_t launch_dump(int64_t *acc, int64_t *vis, int64_t *stokes, int n_ant, int n_pol,
                        int n_chan, cudaStream_t stream, int grid, int *status) {
  if (n_pol == 2) {
    dump_dual_kernel<<<grid, 256, 0, stream>>>(acc, vis, stokes, n_ant, n_chan, status);
  } else {
    const long long n_in = n_ant;
    dump_single_kernel<<<grid, 256, 0, stream>>>(acc, vis, n_in * (n_in + 1) / 2 * n_chan);
  }
  return cudaGetLastError();
}

cudaError_t launch_guard_check(const unsigned char *before, const unsigned char *after,
                               size_t bytes, int *status, cudaStream_t stream) {
  guard_check_kernel<<<1, 256, 0, stream>>>(before, after, bytes, status);
  return cudaGetLastError();
}

cudaError_t launch_pitch(const uint8_t *src, uint8_t *dst, long long rows, int T, int pitch,
                         cudaStream_t stream, int grid) {
  pitch_kernel<<<grid, 256, 0, stream>>>(src, dst, rows, T, pitch);
  return cudaGetLastError();
}

}  // namespace xe
