// fengine.cu -- the F-engine on the GPU: polyphase filter bank (4 taps,
// 2048 points, Hamming-windowed sinc), 2048-point real FFT to 1024 channels,
// per-(input, channel) EQ gain and 4+4-bit requantisation, written in the
// X-engine's input order.
//
// Sec. 2.1 describes the ROACH2 F-engine: pfb_fir (PFB size 2^11, Hamming
// window, 4 taps), fft_biplex_real_2x (FFT size 2^11), EQ coefficients per
// input and channel, truncation to a 4-bit real and a 4-bit imaginary part,
// and the Transpose (corner turn) that orders the data for the X-engine.
// With x the 8-bit samples of one input and h the 8192-tap prototype filter,
// spectrum k of that input is
//     v_k[n] = sum_{j<4} h[2048 j + n] x[2048 (k + j) + n],   n < 2048,
//     X_k[c] = sum_n v_k[n] exp(-2 pi i n c / 2048),            c < 1024,
// and the output byte is (q(g Re X) << 4) | (q(g Im X) & 15) with q rounding
// half away from zero and clipping to [-7, 7].
//
// One CTA (256 threads) takes one input and a tile of kSpecTile consecutive
// spectra:
//   - the input's samples stream through a ring of 2048-byte segments in
//     shared memory, copied in with cp.async one batch ahead (each sample is
//     read from HBM once per tile, plus three segments of overlap at the
//     tile start);
//   - spectra go through in batches of kBatch, so that every barrier of the
//     FFT is shared by kBatch independent butterflies per thread;
//   - thread t owns samples 4 t .. 4 t + 3 and 1024 + 4 t .. + 3 of every
//     segment and filters a batch's spectra together: each of the batch's
//     kBatch + 3 segments is turned into fp32 once (a byte permute and an
//     exact subtraction) and feeds every spectrum of the batch whose taps
//     cover it, with the thread's 32 filter coefficients loaded once per
//     batch; it pairs the results as z[m] = v[2m] + i v[2m+1];
//   - a 1024-point complex FFT runs in three in-place passes over shared
//     memory, 1024 = 16 x 4 x 16 (each thread does a 16-point FFT in registers
//     in the first and last pass, four 4-point FFTs in the middle one);
//   - the standard split of the real FFT, X[c] = s_c Z[c] + (1 - s_c)
//     conj Z[N-c] with s_c = (1 - i W_2048^c) / 2, then the EQ gain and
//     requantisation; a thread takes a channel c and its mirror N - c, which
//     read the same two FFT outputs and whose split constants are conjugate,
//     so that one complex multiply-add gives both, and packs each one's codes
//     of the batch's 4 spectra into a word of a staging tile
//     [1024 channels][kSpecTile spectra];
//   - each channel's row of the staging tile is written out as one 32-byte run
//     of out[c][input][k0 ..].
// Floating point is fp32 (the host computes the filter and twiddles in
// double precision); the codes can differ from an exact computation only for
// values within the fp32 rounding error of a quantisation boundary.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "corr.h"
#include "trace.h"

namespace {

constexpr int kP = 2048;          // PFB / FFT points
constexpr int kTaps = 4;
constexpr int kHalf = kP / 2;     // channels; also the complex FFT size
constexpr int kThreads = 256;
constexpr int kSpecTile = 32;     // spectra per CTA tile
constexpr int kCtasPerSm = 2;     // resident CTAs per SM the kernel is built for

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Forward 4-point DFT in place: X[k] = sum_n a[n] (-i)^(n k).
// Complex sum and difference as one packed two-lane fp32 instruction each
// (round to nearest, the same results as two scalar operations).
__device__ __forceinline__ float2 cadd(float2 a, float2 b) {
  float2 d;
  asm("{\n.reg .b64 ra, rb, rd;\nmov.b64 ra, {%2, %3};\nmov.b64 rb, {%4, %5};\n"
      "add.rn.f32x2 rd, ra, rb;\nmov.b64 {%0, %1}, rd;\n}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ float2 csub(float2 a, float2 b) {
  float2 d;
  asm("{\n.reg .b64 ra, rb, rd;\nmov.b64 ra, {%2, %3};\nmov.b64 rb, {%4, %5};\n"
      "sub.rn.f32x2 rd, ra, rb;\nmov.b64 {%0, %1}, rd;\n}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}

// Two-lane products and fused multiply-adds (round to nearest, as fmaf).
__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
  float2 d;
  asm("{\n.reg .b64 ra, rb, rd;\nmov.b64 ra, {%2, %3};\nmov.b64 rb, {%4, %5};\n"
      "mul.rn.f32x2 rd, ra, rb;\nmov.b64 {%0, %1}, rd;\n}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
  float2 d;
  asm("{\n.reg .b64 ra, rb, rc, rd;\nmov.b64 ra, {%2, %3};\nmov.b64 rb, {%4, %5};\n"
      "mov.b64 rc, {%6, %7};\nfma.rn.f32x2 rd, ra, rb, rc;\nmov.b64 {%0, %1}, rd;\n}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
}

__device__ __forceinline__ void dft4(float2 &a0, float2 &a1, float2 &a2, float2 &a3) {
  const float2 s02 = cadd(a0, a2), d02 = csub(a0, a2);
  const float2 s13 = cadd(a1, a3), d13 = csub(a1, a3);
  a0 = cadd(s02, s13);
  a1 = make_float2(d02.x + d13.y, d02.y - d13.x);  // a0 - i a1 - a2 + i a3
  a2 = csub(s02, s13);
  a3 = make_float2(d02.x - d13.y, d02.y + d13.x);  // a0 + i a1 - a2 - i a3
}

// Forward 16-point DFT in place, natural order in and out:
// Y[ka + 4 kb] = sum_nb W4^(nb kb) W16^(nb ka) sum_na a[4 na + nb] W4^(na ka).
__device__ __forceinline__ void dft16(float2 (&a)[16]) {
  constexpr float c1 = 0.92387953251128674f, s1 = 0.38268343236508978f;  // cos, sin (pi/8)
  constexpr float r2 = 0.70710678118654752f;
#pragma unroll
  for (int nb = 0; nb < 4; ++nb) dft4(a[nb], a[4 + nb], a[8 + nb], a[12 + nb]);
  // a[4 ka + nb] now holds T[nb][ka]; twiddle by W16^(nb ka) (literal constants)
  a[5] = cmul(a[5], make_float2(c1, -s1));     // W16^1
  a[6] = cmul(a[6], make_float2(r2, -r2));     // W16^2
  a[7] = cmul(a[7], make_float2(s1, -c1));     // W16^3
  a[9] = cmul(a[9], make_float2(r2, -r2));     // W16^2
  a[10] = make_float2(a[10].y, -a[10].x);      // W16^4 = -i
  a[11] = cmul(a[11], make_float2(-r2, -r2));  // W16^6
  a[13] = cmul(a[13], make_float2(s1, -c1));   // W16^3
  a[14] = cmul(a[14], make_float2(-r2, -r2));  // W16^6
  a[15] = cmul(a[15], make_float2(-c1, s1));   // W16^9
  // 4-point DFTs over nb for each ka: outputs Y[ka + 4 kb] land in a[4 ka + kb]
#pragma unroll
  for (int ka = 0; ka < 4; ++ka) dft4(a[4 * ka], a[4 * ka + 1], a[4 * ka + 2], a[4 * ka + 3]);
  // transpose 4 x 4 so that a[k] = Y[k]
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = i + 1; j < 4; ++j) {
      const float2 t = a[4 * i + j];
      a[4 * i + j] = a[4 * j + i];
      a[4 * j + i] = t;
    }
}

// Round half away from zero, then clip to [-7, 7] (the clip bounds are
// integers, so clipping first gives the same code).  The half is added with
// rounding toward zero, so the sum never reaches the next integer unless the
// exact sum does, and the truncation then gives the rounded value exactly.
__device__ __forceinline__ int quant(float a) {
  const float y = fminf(fmaxf(a, -7.0f), 7.0f);
  return __float2int_rz(__fadd_rz(y, copysignf(0.5f, y)));
}

// Shared memory of one CTA (dynamic): the sample ring, the FFT buffers of a
// batch of spectra and, when quantising, the staging tile.
constexpr int kBatch = 4;                         // spectra per inner iteration
// Ring of sample segments: a batch reads kBatch + 3 of them while the next
// batch's kBatch newest ones are being copied in (cp.async), so the copies
// of HBM data overlap a whole batch of compute.
constexpr int kRing = 16;                         // ring slots (>= kTaps - 1 + 2 kBatch)
constexpr int kRingBytes = kRing * kP;            // 32 KB
// FFT buffers: element e of a spectrum sits at e + e / 64 (one pad element
// per 64).  That keeps the passes' runs of consecutive elements and their
// stride-64 gathers at the two shared-memory wavefronts a warp's float2
// access needs, and every unrolled access of a pass is its thread's base
// plus a constant offset.  The filter's output is the one exception: it is
// stored unpadded (element e at e), so that each thread's two consecutive
// elements leave as one aligned 16-byte store (padded, a warp's 8-byte stores
// 16 bytes apart took four wavefronts instead of two), and the first pass
// reads it from there; the first pass's reads all precede its padded writes.
constexpr int kBufElems = kHalf + kHalf / 64;
constexpr int kBufBytes = kBatch * kBufElems * 8;

// Staging tile: [channel][kSpecTile codes], rows kStagePitch bytes apart.
// 36 = 9 words, so the 4-byte stores and loads of 32 consecutive channels
// fall in 32 distinct banks.
constexpr int kStagePitch = kSpecTile + 4;
constexpr int kStageBytes = kHalf * kStagePitch;  // 36 KB

__device__ __forceinline__ int bpos(int e) { return e + (e >> 6); }

// 16-byte asynchronous copy global -> shared, cached in L2 only, so that the
// streamed samples do not evict the filter coefficients from L1; src_bytes 0
// writes zeros.
__device__ __forceinline__ void cp_async16(void *dst, const void *src, int src_bytes) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(src_bytes)
               : "memory");
}
// A 16-byte read-only load that the compiler keeps where it is written (it
// neither re-issues it at the use nor moves it across the barriers), so that
// the next batch's coefficients are in flight while the current batch ends.
__device__ __forceinline__ float4 ldg_keep(const float *p) {
  float4 v;
  asm volatile("ld.global.nc.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(p));
  return v;
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
static_assert(kSpecTile % kBatch == 0, "tile of whole batches");
static_assert(kRing >= kTaps - 1 + 2 * kBatch && (kRing & (kRing - 1)) == 0, "ring size");

// kQuant: 1 -> packed codes via the staging tile; 0 -> float2 g X straight to
// global (X-engine order, for tolerance checks).
template <int kQuant>
__global__ void __launch_bounds__(kThreads, kCtasPerSm)
    fengine_kernel(const int8_t *__restrict__ adc, const float *__restrict__ proto,
                   const float2 *__restrict__ tw_fft, const float2 *__restrict__ split,
                   const float *__restrict__ eq,
                   uint8_t *__restrict__ out_codes, float2 *__restrict__ out_spec, int n_in,
                   int n_spec) {
  extern __shared__ __align__(16) uint8_t fe_smem[];
  int8_t *ring = reinterpret_cast<int8_t *>(fe_smem);                      // [kRing][kP]
  float2 *buf = reinterpret_cast<float2 *>(fe_smem + kRingBytes);  // [kBatch][kBufElems]
  uint8_t *stage = fe_smem + kRingBytes + kBufBytes;               // [kHalf][kStagePitch]
  const int tid = threadIdx.x;
  // W64^j = W1024^(16 j), the first pass's twiddles, kept in shared memory
  __shared__ float2 tw64[64];
  if (tid < 64) tw64[tid] = __ldg(tw_fft + 16 * tid);
  __syncthreads();
  const int n_tiles = (n_spec + kSpecTile - 1) / kSpecTile;
  const int n_seg = n_spec + kTaps - 1;  // segments in one input's stream
  const long long stream_len = (long long)n_seg * kP;

  // starts the copy of 16-byte piece p of segment seg into its ring slot;
  // segments past the stream's end read as zero (they feed only spectra past
  // n_spec, which are computed and dropped)
  constexpr int kPieces = kP / 16;
  auto fetch_piece = [&](const int8_t *x, int seg, int p) {
    const bool in = seg < n_seg;
    cp_async16(&ring[(seg & (kRing - 1)) * kP + 16 * p],
               x + (in ? (long long)seg * kP + 16 * p : 0), in ? 16 : 0);
  };
  // the thread's 8 coefficients of each tap (samples 4 t .. 4 t + 3 and
  // 1024 + 4 t .. + 3), the same for every batch; loaded here for the first
  // batch and at the end of each batch for the next
  float4 hq[2 * kTaps];
  auto load_h = [&]() {
#pragma unroll
    for (int j = 0; j < kTaps; ++j) {
      hq[2 * j] = ldg_keep(proto + j * kP + 4 * tid);
      hq[2 * j + 1] = ldg_keep(proto + j * kP + kHalf + 4 * tid);
    }
  };
  load_h();

  for (long long w = blockIdx.x; w < (long long)n_in * n_tiles; w += gridDim.x) {
    const int in = (int)(w / n_tiles), tile = (int)(w % n_tiles);
    const int k0 = tile * kSpecTile;
    const int ns = min(kSpecTile, n_spec - k0);
    const int8_t *x = adc + (long long)in * stream_len;
    // the first batch's segments k0 .. k0 + kBatch + 2
    for (int i = tid; i < (kBatch + kTaps - 1) * kPieces; i += kThreads)
      fetch_piece(x, k0 + i / kPieces, i % kPieces);
    cp_async_commit();
    for (int s0 = 0; s0 < ns; s0 += kBatch) {
      const int nb = min(kBatch, ns - s0);  // spectra of this batch that are kept
      // the next batch's newest segments, while this batch computes
      if (s0 + kBatch < ns) {
#pragma unroll
        for (int i = tid; i < kBatch * kPieces; i += kThreads)
          fetch_piece(x, k0 + s0 + kBatch + kTaps - 1 + i / kPieces, i % kPieces);
      }
      cp_async_commit();
      cp_async_wait<1>();  // this batch's segments have landed (this thread's part)
      __syncthreads();     // ... and every thread's
      // ---- polyphase FIR of the batch's kBatch spectra.  Thread t owns
      // samples 4 t .. 4 t + 3 and 1024 + 4 t .. + 3 of every segment; segment
      // k0 + s0 + sg is tap j = sg - u of spectrum k0 + s0 + u, and the taps
      // of a spectrum are summed in the order j = 0, 1, 2, 3.
      {
        // the thread's 8 coefficients of each tap and its 8 samples of a
        // segment as 4 pairs, so that each filter step is 4 two-lane
        // fused multiply-adds
        float2 h[kTaps][4];
#pragma unroll
        for (int j = 0; j < kTaps; ++j) {
          h[j][0] = make_float2(hq[2 * j].x, hq[2 * j].y);
          h[j][1] = make_float2(hq[2 * j].z, hq[2 * j].w);
          h[j][2] = make_float2(hq[2 * j + 1].x, hq[2 * j + 1].y);
          h[j][3] = make_float2(hq[2 * j + 1].z, hq[2 * j + 1].w);
        }
        const float2 bias = make_float2(8388736.0f, 8388736.0f);
        float2 v[kBatch][4];
#pragma unroll
        for (int sg = 0; sg < kBatch + kTaps - 1; ++sg) {
          const int8_t *seg = &ring[((k0 + s0 + sg) & (kRing - 1)) * kP];
          // int8 -> fp32 without a conversion instruction: with the sign bit
          // flipped, byte b + 128 placed under the exponent of 2^23 is the
          // float 2^23 + b + 128, and subtracting 2^23 + 128 is exact
          const uint32_t wd[2] = {*reinterpret_cast<const uint32_t *>(seg + 4 * tid) ^ 0x80808080u,
                                  *reinterpret_cast<const uint32_t *>(seg + kHalf + 4 * tid) ^
                                      0x80808080u};
          float2 xs[4];
#pragma unroll
          for (int e = 0; e < 4; ++e)
            xs[e] = csub(make_float2(__uint_as_float(__byte_perm(wd[e >> 1], 0x4B000000u,
                                                                 0x7650 + 2 * (e & 1))),
                                     __uint_as_float(__byte_perm(wd[e >> 1], 0x4B000000u,
                                                                 0x7650 + 2 * (e & 1) + 1))),
                         bias);
#pragma unroll
          for (int u = 0; u < kBatch; ++u) {
            const int j = sg - u;
            if (j < 0 || j >= kTaps) continue;
#pragma unroll
            for (int e = 0; e < 4; ++e) v[u][e] = j == 0 ? mul2(h[0][e], xs[e]) : fma2(h[j][e], xs[e], v[u][e]);
          }
        }
        // z[2 tid], z[2 tid + 1] and z[512 + 2 tid], z[513 + 2 tid], unpadded:
        // one 16-byte store per pair, a warp's lanes contiguous
#pragma unroll
        for (int u = 0; u < kBatch; ++u)
#pragma unroll
          for (int hh = 0; hh < 2; ++hh)
            *reinterpret_cast<float4 *>(&buf[u * kBufElems + 512 * hh + 2 * tid]) =
                make_float4(v[u][2 * hh].x, v[u][2 * hh].y, v[u][2 * hh + 1].x, v[u][2 * hh + 1].y);
      }
      __syncthreads();
      // ---- 1024-point FFTs, 1024 = 16 x 4 x 16 (n = 64 m1 + 16 m2 + n2,
      // k = l1 + 16 l2 + 64 k2):
      //   pass 1: A[n2][m2][l1] = W64^(m2 l1) sum_m1 x[64 m1 + 16 m2 + n2] W16^(m1 l1)
      //   pass 2: B[n2][k1] = W1024^(n2 k1) sum_m2 A[n2][m2][l1] W4^(m2 l2),  k1 = l1 + 16 l2
      //   pass 3: X[k1 + 64 k2] = sum_n2 B[n2][k1] W16^(n2 k2)
      // A[n2][m2][l1] and B[n2][l1 + 16 l2] share element l1 + 16 m2 + 64 n2
      // (m2 <-> l2), and X[k1 + 64 k2] element k1 + 64 n2 (n2 <-> k2), so
      // passes 2 and 3 read and write the same elements of their thread.
      {
        // pass 1: thread t -> spectrum t / 64, (m2, n2) = (t % 64 / 16, t % 16)
        const int u = tid >> 6, r = tid & 63, m2 = r >> 4, n2 = r & 15;
        float2 *bu = buf + u * kBufElems;
        float2 a[16];
        const bool live = u < nb;
        if (live) {
#pragma unroll
          for (int m1 = 0; m1 < 16; ++m1) a[m1] = bu[64 * m1 + r];  // the filter's unpadded output
          dft16(a);
#pragma unroll
          for (int l1 = 1; l1 < 16; ++l1) a[l1] = cmul(a[l1], tw64[m2 * l1]);
        }
        __syncthreads();  // every thread has read its inputs
        if (live) {
#pragma unroll
          for (int l1 = 0; l1 < 16; ++l1) bu[bpos(l1 + 16 * m2 + 64 * n2)] = a[l1];
        }
      }
      __syncthreads();
      {
        // pass 2: thread t -> (n2, l1) = (t / 16, t % 16), every spectrum
        const int n2 = tid >> 4, l1 = tid & 15;
        float2 tw[4];
#pragma unroll
        for (int l2 = 0; l2 < 4; ++l2) tw[l2] = __ldg(tw_fft + ((n2 * (l1 + 16 * l2)) & (kHalf - 1)));
        // kept as a loop: unrolled, the four copies made the kernel 5 % slower
        // (a larger loop body for the instruction cache)
#pragma unroll 1
        for (int u = 0; u < kBatch; ++u) {
          if (u >= nb) break;
          float2 *bu = buf + u * kBufElems;
          float2 a0 = bu[bpos(l1 + 64 * n2)], a1 = bu[bpos(l1 + 16 + 64 * n2)];
          float2 a2 = bu[bpos(l1 + 32 + 64 * n2)], a3 = bu[bpos(l1 + 48 + 64 * n2)];
          dft4(a0, a1, a2, a3);
          bu[bpos(l1 + 64 * n2)] = cmul(a0, tw[0]);
          bu[bpos(l1 + 16 + 64 * n2)] = cmul(a1, tw[1]);
          bu[bpos(l1 + 32 + 64 * n2)] = cmul(a2, tw[2]);
          bu[bpos(l1 + 48 + 64 * n2)] = cmul(a3, tw[3]);
        }
      }
      __syncthreads();
      {
        // pass 3: thread t -> spectrum t / 64, k1 = t % 64
        const int u = tid >> 6, k1 = tid & 63;
        if (u < nb) {
          float2 *bu = buf + u * kBufElems;
          float2 a[16];
#pragma unroll
          for (int n2 = 0; n2 < 16; ++n2) a[n2] = bu[bpos(k1 + 64 * n2)];
          dft16(a);
#pragma unroll
          for (int k2 = 0; k2 < 16; ++k2) bu[bpos(k1 + 64 * k2)] = a[k2];
        }
      }
      __syncthreads();
      // ---- real-FFT split with the EQ gain, requantisation.  With
      // s_c = (1 - i W_2048^c) / 2 the split is X[c] = s_c Z[c] + (1 - s_c)
      // conj Z[N - c].  Channel c and its mirror m = N - c read the same two
      // FFT outputs P = Z[c] and R = Z[m], and since s_m = conj s_c,
      //   X[c] = U = conj R + s_c (P - conj R),
      //   X[m] = conj V,   V = P - s_c (P - conj R) = (P + conj R) - U,
      // so one thread takes both: c = tid + 256 e (e = 0, 1) and m = N - c,
      // except that thread 0 takes the self-mirrored N / 2 (as both c and m)
      // at e = 0, and channel 0 (also its own mirror) after the loop.
      const float2 k_mp = make_float2(-1.0f, 1.0f), k_pm = make_float2(1.0f, -1.0f);
#pragma unroll 1
      for (int e = 0; e < 2; ++e) {
        const int c = tid + kThreads * e == 0 ? kHalf / 2 : tid + kThreads * e;
        const int m = kHalf - c;
        const float gc = __ldg(eq + (long long)in * kHalf + c);  // EQ gains
        const float gm = __ldg(eq + (long long)in * kHalf + m);
        const float2 sc = __ldg(split + c);
        const float2 gcc = make_float2(gc, gc), gmm = make_float2(gm, -gm);
        uint32_t wc = 0, wm = 0;
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
          const float2 P = buf[u * kBufElems + bpos(c)];
          const float2 R = buf[u * kBufElems + bpos(m)];
          const float2 D = fma2(R, k_mp, P);  // P - conj R
          const float2 F = fma2(R, k_pm, P);  // P + conj R
          const float2 U = make_float2(fmaf(sc.x, D.x, fmaf(-sc.y, D.y, R.x)),
                                       fmaf(sc.x, D.y, fmaf(sc.y, D.x, -R.y)));
          const float2 xc = mul2(gcc, U);          // g X[c]
          const float2 xm = mul2(gmm, csub(F, U));  // g X[m] = g conj V
          if (kQuant) {
            wc |= (uint32_t)(((quant(xc.x) & 15) << 4) | (quant(xc.y) & 15)) << (8 * u);
            wm |= (uint32_t)(((quant(xm.x) & 15) << 4) | (quant(xm.y) & 15)) << (8 * u);
          } else if (u < nb) {
            out_spec[((long long)c * n_in + in) * n_spec + k0 + s0 + u] = xc;
            out_spec[((long long)m * n_in + in) * n_spec + k0 + s0 + u] = xm;
          }
        }
        if (kQuant) {
          *reinterpret_cast<uint32_t *>(&stage[c * kStagePitch + s0]) = wc;
          *reinterpret_cast<uint32_t *>(&stage[m * kStagePitch + s0]) = wm;
        }
      }
      if (tid == 0) {
        // channel 0: R = P = Z[0]
        const float g0 = __ldg(eq + (long long)in * kHalf);
        const float2 s_0 = __ldg(split);
        uint32_t w0 = 0;
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
          const float2 P = buf[u * kBufElems];
          const float2 D = fma2(P, k_mp, P);
          const float2 x0 = make_float2(g0 * fmaf(s_0.x, D.x, fmaf(-s_0.y, D.y, P.x)),
                                        g0 * fmaf(s_0.x, D.y, fmaf(s_0.y, D.x, -P.y)));
          if (kQuant) {
            w0 |= (uint32_t)(((quant(x0.x) & 15) << 4) | (quant(x0.y) & 15)) << (8 * u);
          } else if (u < nb) {
            out_spec[(long long)in * n_spec + k0 + s0 + u] = x0;
          }
        }
        if (kQuant) *reinterpret_cast<uint32_t *>(&stage[s0]) = w0;
      }
      load_h();         // the next batch's coefficients, in flight across the barrier
      __syncthreads();  // buf and the ring slots are reused by the next batch
    }
    if (kQuant) {
      // ---- staging tile -> out[c][in][k0 .. k0 + ns): thread per channel,
      // its row of the tile as eight words (conflict-free: rows 9 words apart)
      const bool vec = ns == kSpecTile && (n_spec & 15) == 0;
      static_assert(kSpecTile == 32, "two 16-byte stores per channel");
      for (int c = tid; c < kHalf; c += kThreads) {
        const uint32_t *row = reinterpret_cast<const uint32_t *>(&stage[c * kStagePitch]);
        uint8_t *dst = out_codes + ((long long)c * n_in + in) * n_spec + k0;
        if (vec) {
          reinterpret_cast<uint4 *>(dst)[0] = make_uint4(row[0], row[1], row[2], row[3]);
          reinterpret_cast<uint4 *>(dst)[1] = make_uint4(row[4], row[5], row[6], row[7]);
        } else {
          for (int b = 0; b < ns; ++b) dst[b] = stage[c * kStagePitch + b];
        }
      }
      __syncthreads();
    }
  }
}

constexpr int smem_bytes() { return kRingBytes + kBufBytes + kStageBytes; }

}  // namespace

struct corr_fengine {
  int n_in, n_spec, n_sm;
  float *d_proto;
  float2 *d_tw_fft, *d_split;
  float *d_eq;
};

namespace {

int cuda_err(cudaError_t e) {
  if (e == cudaSuccess) return CORR_OK;
  if (e == cudaErrorMemoryAllocation) return CORR_ENOMEM;
  return CORR_ECUDA;
}

void free_fengine(corr_fengine *f) {
  if (!f) return;
  cudaFree(f->d_proto);
  cudaFree(f->d_tw_fft);
  cudaFree(f->d_split);
  cudaFree(f->d_eq);
  delete f;
}

bool aligned(const void *p, unsigned a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

}  // namespace

extern "C" {

int corr_fengine_create(int n_in, int n_spectra, corr_fengine **out) {
  if (!out) return CORR_EINVAL;
  *out = nullptr;
  if (n_in <= 0 || n_spectra <= 0 || n_in > CORR_MAX_INPUTS) return CORR_EINVAL;
  int dev = 0;
  cudaDeviceProp prop;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess)
    return CORR_ECUDA;
  if (prop.major != 10 || prop.minor != 3) return CORR_EARCH;
  corr_fengine *f = new (std::nothrow) corr_fengine;
  if (!f) return CORR_ENOMEM;
  std::memset(f, 0, sizeof(*f));
  f->n_in = n_in;
  f->n_spec = n_spectra;
  f->n_sm = prop.multiProcessorCount;
  // prototype filter and twiddles in double precision, stored as fp32
  const int L = kTaps * kP;
  std::vector<float> proto(L), eq((size_t)n_in * kHalf, 1.0f);
  const double pi = 3.14159265358979323846;
  for (int m = 0; m < L; ++m) {
    const double w = 0.54 - 0.46 * std::cos(2.0 * pi * m / (L - 1));
    const double xx = (double)(m - L / 2) / kP;
    const double sinc = xx == 0.0 ? 1.0 : std::sin(pi * xx) / (pi * xx);
    proto[m] = (float)(w * sinc);
  }
  // FFT twiddles W_1024^k, and the real-FFT split's constant per channel:
  // with W = W_2048^c = cos t - i sin t (t = 2 pi c / 2048),
  // s_c = (1 - i W) / 2 = ((1 - sin t) / 2, -cos t / 2)
  std::vector<float2> tw_fft(kHalf), split(kHalf);
  for (int k = 0; k < kHalf; ++k) {
    tw_fft[k] = make_float2((float)std::cos(2.0 * pi * k / kHalf), (float)-std::sin(2.0 * pi * k / kHalf));
    const double t = 2.0 * pi * k / kP, ct = std::cos(t), st = std::sin(t);
    split[k] = make_float2((float)(0.5 * (1.0 - st)), (float)(-0.5 * ct));
  }
  int rc;
  if ((rc = cuda_err(cudaFuncSetAttribute(fengine_kernel<1>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          smem_bytes()))) != CORR_OK ||
      (rc = cuda_err(cudaFuncSetAttribute(fengine_kernel<0>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          smem_bytes()))) != CORR_OK ||
      (rc = cuda_err(cudaMalloc(&f->d_proto, L * sizeof(float)))) != CORR_OK ||
      (rc = cuda_err(cudaMalloc(&f->d_tw_fft, kHalf * sizeof(float2)))) != CORR_OK ||
      (rc = cuda_err(cudaMalloc(&f->d_split, kHalf * sizeof(float2)))) != CORR_OK ||
      (rc = cuda_err(cudaMalloc(&f->d_eq, eq.size() * sizeof(float)))) != CORR_OK ||
      (rc = cuda_err(cudaMemcpy(f->d_proto, proto.data(), L * sizeof(float),
                                cudaMemcpyHostToDevice))) != CORR_OK ||
      (rc = cuda_err(cudaMemcpy(f->d_tw_fft, tw_fft.data(), kHalf * sizeof(float2),
                                cudaMemcpyHostToDevice))) != CORR_OK ||
      (rc = cuda_err(cudaMemcpy(f->d_split, split.data(), kHalf * sizeof(float2),
                                cudaMemcpyHostToDevice))) != CORR_OK ||
      (rc = cuda_err(cudaMemcpy(f->d_eq, eq.data(), eq.size() * sizeof(float),
                                cudaMemcpyHostToDevice))) != CORR_OK) {
    free_fengine(f);
    return rc;
  }
  *out = f;
  return CORR_OK;
}

int corr_fengine_set_eq(corr_fengine *f, const float *h_eq) {
  if (!f || !h_eq) return CORR_EINVAL;
  return cuda_err(cudaMemcpy(f->d_eq, h_eq, (size_t)f->n_in * kHalf * sizeof(float),
                             cudaMemcpyHostToDevice));
}

int corr_fengine_run(corr_fengine *f, const int8_t *d_adc, uint8_t *d_out, void *stream) {
  CORR_TRACE("corr_fengine_run");
  if (!f || !d_adc || !d_out || !aligned(d_adc, 16) || !aligned(d_out, 16)) return CORR_EINVAL;
  const long long work = (long long)f->n_in * ((f->n_spec + kSpecTile - 1) / kSpecTile);
  const int grid = (int)std::min<long long>(work, (long long)f->n_sm * kCtasPerSm * 4);
  fengine_kernel<1><<<grid, kThreads, smem_bytes(), static_cast<cudaStream_t>(stream)>>>(
      d_adc, f->d_proto, f->d_tw_fft, f->d_split, f->d_eq, d_out, nullptr, f->n_in, f->n_spec);
  return cuda_err(cudaGetLastError());
}

int corr_fengine_spectra(corr_fengine *f, const int8_t *d_adc, float *d_spec, void *stream) {
  CORR_TRACE("corr_fengine_spectra");
  if (!f || !d_adc || !d_spec || !aligned(d_adc, 16) || !aligned(d_spec, 8)) return CORR_EINVAL;
  const long long work = (long long)f->n_in * ((f->n_spec + kSpecTile - 1) / kSpecTile);
  const int grid = (int)std::min<long long>(work, (long long)f->n_sm * kCtasPerSm * 4);
  fengine_kernel<0><<<grid, kThreads, smem_bytes(), static_cast<cudaStream_t>(stream)>>>(
      d_adc, f->d_proto, f->d_tw_fft, f->d_split, f->d_eq, nullptr,
      reinterpret_cast<float2 *>(d_spec), f->n_in, f->n_spec);
  return cuda_err(cudaGetLastError());
}

void corr_fengine_destroy(corr_fengine *f) { free_fengine(f); }

}  // extern "C"
