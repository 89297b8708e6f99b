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
//     shared memory (each sample is read from HBM once per tile, plus three
//     segments of overlap at the tile start);
//   - spectra go through in batches of kBatch, so that every barrier of the
//     FFT is shared by kBatch independent butterflies per thread;
//   - thread t filters samples 4 t .. 4 t + 3 and 1024 + 4 t .. + 3 (filter
//     coefficients read from L1 per tap, int8 samples turned into fp32 with a
//     byte permute and an exact subtraction), and pairs them as
//     z[m] = v[2m] + i v[2m+1];
//   - a 1024-point complex FFT runs in three in-place passes over shared
//     memory, 1024 = 16 x 4 x 16 (each thread does a 16-point FFT in registers
//     in the first and last pass, four 4-point FFTs in the middle one), then
//     the standard split gives the 2048-point real FFT's channels 0..1023;
//   - EQ and requantisation produce one byte per channel into a staging tile
//     [kSpecTile spectra][1024 channels], written out as 32-byte runs of
//     out[c][input][k0 ..].
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

namespace {

constexpr int kP = 2048;          // PFB / FFT points
constexpr int kTaps = 4;
constexpr int kHalf = kP / 2;     // channels; also the complex FFT size
constexpr int kThreads = 256;
constexpr int kSpecTile = 32;     // spectra per CTA tile

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Forward 4-point DFT in place: X[k] = sum_n a[n] (-i)^(n k).
__device__ __forceinline__ void dft4(float2 &a0, float2 &a1, float2 &a2, float2 &a3) {
  const float2 s02 = make_float2(a0.x + a2.x, a0.y + a2.y);
  const float2 d02 = make_float2(a0.x - a2.x, a0.y - a2.y);
  const float2 s13 = make_float2(a1.x + a3.x, a1.y + a3.y);
  const float2 d13 = make_float2(a1.x - a3.x, a1.y - a3.y);
  a0 = make_float2(s02.x + s13.x, s02.y + s13.y);
  a1 = make_float2(d02.x + d13.y, d02.y - d13.x);  // a0 - i a1 - a2 + i a3
  a2 = make_float2(s02.x - s13.x, s02.y - s13.y);
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

__device__ __forceinline__ int quant(float a) {
  const float r = roundf(a);  // half away from zero
  return (int)fminf(fmaxf(r, -7.0f), 7.0f);
}

// Shared memory of one CTA (dynamic): the sample ring, the FFT buffers of a
// batch of spectra and, when quantising, the staging tile.
constexpr int kBatch = 4;                         // spectra per inner iteration
constexpr int kRing = 8;                          // ring slots (>= kTaps - 1 + kBatch)
constexpr int kRingBytes = kRing * kP;            // 16 KB
// FFT buffers: element e of a spectrum sits at e + e / 64 (one pad element
// per 64).  That keeps the passes' runs of consecutive elements and their
// stride-64 gathers at the two shared-memory wavefronts a warp's float2
// access needs, and every unrolled access of a pass is its thread's base
// plus a constant offset.
constexpr int kBufElems = kHalf + kHalf / 64;
constexpr int kBufBytes = kBatch * kBufElems * 8;
constexpr int kStageBytes = kHalf * kSpecTile;    // 32 KB, [spectrum][channel]

__device__ __forceinline__ int bpos(int e) { return e + (e >> 6); }
static_assert(kSpecTile % kBatch == 0, "tile of whole batches");
static_assert(kRing >= kTaps - 1 + kBatch && (kRing & (kRing - 1)) == 0, "ring size");

// kQuant: 1 -> packed codes via the staging tile; 0 -> float2 g X straight to
// global (X-engine order, for tolerance checks).
template <int kQuant>
__global__ void __launch_bounds__(kThreads, 2)
    fengine_kernel(const int8_t *__restrict__ adc, const float *__restrict__ proto,
                   const float2 *__restrict__ tw_fft, const float2 *__restrict__ tw_split,
                   const float *__restrict__ eq, uint8_t *__restrict__ out_codes,
                   float2 *__restrict__ out_spec, int n_in, int n_spec) {
  extern __shared__ __align__(16) uint8_t fe_smem[];
  int8_t *ring = reinterpret_cast<int8_t *>(fe_smem);                      // [kRing][kP]
  float2 *buf = reinterpret_cast<float2 *>(fe_smem + kRingBytes);  // [kBatch][kBufElems]
  uint8_t *stage = fe_smem + kRingBytes + kBufBytes;               // [kSpecTile][kHalf]
  const int tid = threadIdx.x;
  // W64^j = W1024^(16 j), the first pass's twiddles, kept in shared memory
  __shared__ float2 tw64[64];
  if (tid < 64) tw64[tid] = __ldg(tw_fft + 16 * tid);
  __syncthreads();
  const int n_tiles = (n_spec + kSpecTile - 1) / kSpecTile;
  const long long stream_len = (long long)(n_spec + kTaps - 1) * kP;

  for (long long w = blockIdx.x; w < (long long)n_in * n_tiles; w += gridDim.x) {
    const int in = (int)(w / n_tiles), tile = (int)(w % n_tiles);
    const int k0 = tile * kSpecTile;
    const int ns = min(kSpecTile, n_spec - k0);
    const int8_t *x = adc + (long long)in * stream_len;
    // prime the ring with segments k0 .. k0 + 2
    for (int j = 0; j < kTaps - 1; ++j)
      *reinterpret_cast<uint2 *>(&ring[((k0 + j) & (kRing - 1)) * kP + 8 * tid]) =
          __ldg(reinterpret_cast<const uint2 *>(x + (long long)(k0 + j) * kP + 8 * tid));
    for (int s0 = 0; s0 < ns; s0 += kBatch) {
      const int nb = min(kBatch, ns - s0);  // spectra in this batch
      // newest segments k0 + s0 + 3 .. + nb + 2
      for (int u = 0; u < nb; ++u) {
        const int seg = k0 + s0 + u + kTaps - 1;
        *reinterpret_cast<uint2 *>(&ring[(seg & (kRing - 1)) * kP + 8 * tid]) =
            __ldg(reinterpret_cast<const uint2 *>(x + (long long)seg * kP + 8 * tid));
      }
      __syncthreads();
      // ---- polyphase FIR of each spectrum of the batch.  The filter
      // coefficients of this thread's 8 samples (4 tid .. + 3 and 1024 + 4 tid
      // .. + 3 of the 2048) are read from L1 per tap, so that they do not stay
      // live through the FFT passes.
#pragma unroll 1
      for (int u = 0; u < nb; ++u) {
        const int k = k0 + s0 + u;
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = 0.0f;
#pragma unroll
        for (int j = 0; j < kTaps; ++j) {
          const int8_t *seg = &ring[((k + j) & (kRing - 1)) * kP];
          const float4 h0 = __ldg(reinterpret_cast<const float4 *>(proto + j * kP + 4 * tid));
          const float4 h1 = __ldg(reinterpret_cast<const float4 *>(proto + j * kP + kHalf + 4 * tid));
          const float hc[8] = {h0.x, h0.y, h0.z, h0.w, h1.x, h1.y, h1.z, h1.w};
          // int8 -> fp32 without a conversion instruction: with the sign bit
          // flipped, byte b + 128 placed under the exponent of 2^23 is the
          // float 2^23 + b + 128, and subtracting 2^23 + 128 is exact
          const uint32_t wd[2] = {*reinterpret_cast<const uint32_t *>(seg + 4 * tid) ^ 0x80808080u,
                                  *reinterpret_cast<const uint32_t *>(seg + kHalf + 4 * tid) ^
                                      0x80808080u};
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const uint32_t f = __byte_perm(wd[e >> 2], 0x4B000000u, 0x7650 + (e & 3));
            const float xs = __uint_as_float(f) - 8388736.0f;
            v[e] = fmaf(hc[e], xs, v[e]);
          }
        }
        // z[2 tid], z[2 tid + 1] and z[512 + 2 tid], z[513 + 2 tid]
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          float2 *d = &buf[u * kBufElems + bpos(512 * h + 2 * tid)];
          d[0] = make_float2(v[4 * h], v[4 * h + 1]);
          d[1] = make_float2(v[4 * h + 2], v[4 * h + 3]);
        }
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
          for (int m1 = 0; m1 < 16; ++m1) a[m1] = bu[bpos(64 * m1 + r)];
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
#pragma unroll
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
      // ---- real-FFT split, EQ, requantisation: channels c = tid + 256 e
#pragma unroll 1
      for (int e = 0; e < 4; ++e) {
        const int c = tid + kThreads * e;
        const float2 tw = __ldg(tw_split + c);
        const float g = __ldg(eq + (long long)in * kHalf + c);  // EQ gain
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
          if (u >= nb) break;
          const float2 zc = buf[u * kBufElems + bpos(c)];
          const float2 zr = buf[u * kBufElems + bpos((kHalf - c) & (kHalf - 1))];
          // even part (Z[c] + conj Z[N-c]) / 2, odd part (Z[c] - conj Z[N-c]) / (2i)
          const float2 ev = make_float2(0.5f * (zc.x + zr.x), 0.5f * (zc.y - zr.y));
          const float2 od = make_float2(0.5f * (zc.y + zr.y), -0.5f * (zc.x - zr.x));
          const float2 t = cmul(tw, od);
          const float2 gX = make_float2(g * (ev.x + t.x), g * (ev.y + t.y));
          if (kQuant) {
            const int qr = quant(gX.x), qi = quant(gX.y);
            stage[(s0 + u) * kHalf + c] = (uint8_t)(((qr & 15) << 4) | (qi & 15));
          } else {
            out_spec[((long long)c * n_in + in) * n_spec + k0 + s0 + u] = gX;
          }
        }
      }
      __syncthreads();  // buf and the ring slots are reused by the next batch
    }
    if (kQuant) {
      // ---- staging tile -> out[c][in][k0 .. k0 + ns): thread per channel,
      // gathering its column of the tile (consecutive channels read
      // consecutive bytes, so the gathers are conflict-free)
      const bool vec = ns == kSpecTile && (n_spec & 15) == 0;
      static_assert(kSpecTile == 32, "two 16-byte stores per channel");
      for (int c = tid; c < kHalf; c += kThreads) {
        uint32_t wv[8];
#pragma unroll
        for (int b = 0; b < 8; ++b) {
          wv[b] = 0;
#pragma unroll
          for (int k = 0; k < 4; ++k) wv[b] |= (uint32_t)stage[(4 * b + k) * kHalf + c] << (8 * k);
        }
        uint8_t *dst = out_codes + ((long long)c * n_in + in) * n_spec + k0;
        if (vec) {
          reinterpret_cast<uint4 *>(dst)[0] = make_uint4(wv[0], wv[1], wv[2], wv[3]);
          reinterpret_cast<uint4 *>(dst)[1] = make_uint4(wv[4], wv[5], wv[6], wv[7]);
        } else {
          for (int b = 0; b < ns; ++b) dst[b] = stage[b * kHalf + c];
        }
      }
      __syncthreads();
    }
  }
}

constexpr int smem_bytes(int quant) { return kRingBytes + kBufBytes + (quant ? kStageBytes : 0); }

}  // namespace

struct corr_fengine {
  int n_in, n_spec, n_sm;
  float *d_proto;
  float2 *d_tw_fft, *d_tw_split;
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
  cudaFree(f->d_tw_split);
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
  std::vector<float2> tw_fft(kHalf), tw_split(kHalf);
  for (int k = 0; k < kHalf; ++k) {
    tw_fft[k] = make_float2((float)std::cos(2.0 * pi * k / kHalf), (float)-std::sin(2.0 * pi * k / kHalf));
    tw_split[k] = make_float2((float)std::cos(2.0 * pi * k / kP), (float)-std::sin(2.0 * pi * k / kP));
  }
  int rc;
  if ((rc = cuda_err(cudaFuncSetAttribute(fengine_kernel<1>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          smem_bytes(1)))) != CORR_OK ||
      (rc = cuda_err(cudaFuncSetAttribute(fengine_kernel<0>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          smem_bytes(0)))) != CORR_OK ||
      (rc = cuda_err(cudaMalloc(&f->d_proto, L * sizeof(float)))) != CORR_OK ||
      (rc = cuda_err(cudaMalloc(&f->d_tw_fft, kHalf * sizeof(float2)))) != CORR_OK ||
      (rc = cuda_err(cudaMalloc(&f->d_tw_split, kHalf * sizeof(float2)))) != CORR_OK ||
      (rc = cuda_err(cudaMalloc(&f->d_eq, eq.size() * sizeof(float)))) != CORR_OK ||
      (rc = cuda_err(cudaMemcpy(f->d_proto, proto.data(), L * sizeof(float),
                                cudaMemcpyHostToDevice))) != CORR_OK ||
      (rc = cuda_err(cudaMemcpy(f->d_tw_fft, tw_fft.data(), kHalf * sizeof(float2),
                                cudaMemcpyHostToDevice))) != CORR_OK ||
      (rc = cuda_err(cudaMemcpy(f->d_tw_split, tw_split.data(), kHalf * sizeof(float2),
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
  if (!f || !d_adc || !d_out || !aligned(d_adc, 8) || !aligned(d_out, 16)) return CORR_EINVAL;
  const long long work = (long long)f->n_in * ((f->n_spec + kSpecTile - 1) / kSpecTile);
  const int grid = (int)std::min<long long>(work, (long long)f->n_sm * 8);
  fengine_kernel<1><<<grid, kThreads, smem_bytes(1), static_cast<cudaStream_t>(stream)>>>(
      d_adc, f->d_proto, f->d_tw_fft, f->d_tw_split, f->d_eq, d_out, nullptr, f->n_in, f->n_spec);
  return cuda_err(cudaGetLastError());
}

int corr_fengine_spectra(corr_fengine *f, const int8_t *d_adc, float *d_spec, void *stream) {
  if (!f || !d_adc || !d_spec || !aligned(d_adc, 8) || !aligned(d_spec, 8)) return CORR_EINVAL;
  const long long work = (long long)f->n_in * ((f->n_spec + kSpecTile - 1) / kSpecTile);
  const int grid = (int)std::min<long long>(work, (long long)f->n_sm * 8);
  fengine_kernel<0><<<grid, kThreads, smem_bytes(0), static_cast<cudaStream_t>(stream)>>>(
      d_adc, f->d_proto, f->d_tw_fft, f->d_tw_split, f->d_eq, nullptr,
      reinterpret_cast<float2 *>(d_spec), f->n_in, f->n_spec);
  return cuda_err(cudaGetLastError());
}

void corr_fengine_destroy(corr_fengine *f) { free_fengine(f); }

}  // extern "C"
