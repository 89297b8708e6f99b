// xe_unpack.cuh -- on-chip unpack of 4+4-bit samples into E5M2 operand rows,
// shared-memory access helpers, shared by the CMAC kernels.
#pragma once
#include <cstdint>

namespace xe {

__device__ __forceinline__ uint32_t hfma2_bits(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm("fma.rn.f16x2 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}

// Four packed samples t0..t3 (bytes of w, earliest in the low byte) -> the
// 8-byte A-row and Q-row pieces of those samples in E5M2.  The K order inside
// a piece is [a0 a2 b0 b2 a1 a3 b1 b3] for the A row and
// [b0 b2 -a0 -a2 b1 b3 -a1 -a3] for the Q row: any fixed order of K gives the
// same dot products as long as every row uses it, and this one needs no
// per-sample shuffles.  A nibble n encodes n - 16 (n >= 8); with u = n ^ 8
// the value is u - 8.  fp16 0x6400 | k is 1024 + k, so
//   low nibble  in bits 0-3 :  (0x6400 | u)      - 1032        = u - 8
//   high nibble in bits 4-7 :  (0x6400 | 16 u) / 16 - 72       = u - 8
// (the XOR with 8 folds into the constant of the same logic op; every fp16
// step is exact on these small integers).  An integer of magnitude <= 8 has
// at most 3 significant bits, so its fp16 encoding has a zero low byte and
// its high byte is exactly its E5M2 encoding: one byte permute per four
// values converts.
__device__ __forceinline__ void decode_word(uint32_t w, uint2 &a, uint2 &q) {
  const uint32_t s16 = 0x2C002C00u, m72 = 0xD480D480u;    // (1/16, 1/16), (-72, -72)
  const uint32_t ns16 = 0xAC00AC00u, p72 = 0x54805480u;   // (-1/16, -1/16), (72, 72)
  const uint32_t one = 0x3C003C00u, m1032 = 0xE408E408u;  // (1, 1), (-1032, -1032)
  const uint32_t w8 = w >> 8;
  const uint32_t lo02 = (w & 0x000F000Fu) ^ 0x64086408u;   // samples 0, 2: 1024 + u_im
  const uint32_t hi02 = (w & 0x00F000F0u) ^ 0x64806480u;   //               1024 + 16 u_re
  const uint32_t lo13 = (w8 & 0x000F000Fu) ^ 0x64086408u;  // samples 1, 3
  const uint32_t hi13 = (w8 & 0x00F000F0u) ^ 0x64806480u;
  const uint32_t re02 = hfma2_bits(hi02, s16, m72), im02 = hfma2_bits(lo02, one, m1032);
  const uint32_t re13 = hfma2_bits(hi13, s16, m72), im13 = hfma2_bits(lo13, one, m1032);
  const uint32_t nre02 = hfma2_bits(hi02, ns16, p72), nre13 = hfma2_bits(hi13, ns16, p72);
  // high bytes of (x.lo, x.hi, y.lo, y.hi)
  a = make_uint2(__byte_perm(re02, im02, 0x7531), __byte_perm(re13, im13, 0x7531));
  q = make_uint2(__byte_perm(im02, nre02, 0x7531), __byte_perm(im13, nre13, 0x7531));
}

// As decode_word, the A-row piece only (for plain regions, whose inputs are
// only ever columns): the negations and the Q-row permutes are skipped.
__device__ __forceinline__ void decode_word_a(uint32_t w, uint2 &a) {
  const uint32_t s16 = 0x2C002C00u, m72 = 0xD480D480u;    // (1/16, 1/16), (-72, -72)
  const uint32_t one = 0x3C003C00u, m1032 = 0xE408E408u;  // (1, 1), (-1032, -1032)
  const uint32_t w8 = w >> 8;
  const uint32_t lo02 = (w & 0x000F000Fu) ^ 0x64086408u;
  const uint32_t hi02 = (w & 0x00F000F0u) ^ 0x64806480u;
  const uint32_t lo13 = (w8 & 0x000F000Fu) ^ 0x64086408u;
  const uint32_t hi13 = (w8 & 0x00F000F0u) ^ 0x64806480u;
  const uint32_t re02 = hfma2_bits(hi02, s16, m72), im02 = hfma2_bits(lo02, one, m1032);
  const uint32_t re13 = hfma2_bits(hi13, s16, m72), im13 = hfma2_bits(lo13, one, m1032);
  a = make_uint2(__byte_perm(re02, im02, 0x7531), __byte_perm(re13, im13, 0x7531));
}

// 16-byte shared-memory load and store on a 32-bit shared address.  The
// operand buffers are carved from the dynamic shared memory by integer
// alignment, so plain pointers into them would be generic pointers; these
// keep the unpack's accesses on the shared-memory path.
__device__ __forceinline__ uint4 lds128(uint32_t a) {
  uint4 v;
  asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "r"(a));
  return v;
}
__device__ __forceinline__ void sts128(uint32_t a, uint32_t x, uint32_t y, uint32_t z, uint32_t w) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(a), "r"(x), "r"(y), "r"(z), "r"(w));
}
__device__ __forceinline__ uint32_t lds32(uint32_t a) {
  uint32_t v;
  asm volatile("ld.shared.b32 %0, [%1];" : "=r"(v) : "r"(a));
  return v;
}
// As sts128, 1024 bytes (eight 128-byte operand rows) further on.
__device__ __forceinline__ void sts128_q(uint32_t a, uint32_t x, uint32_t y, uint32_t z,
                                        uint32_t w) {
  asm volatile("st.shared.v4.b32 [%0+1024], {%1, %2, %3, %4};" ::"r"(a), "r"(x), "r"(y), "r"(z),
               "r"(w));
}

// 4 x 4 byte transpose: out[j] byte k = in[k] byte j.
__device__ __forceinline__ void transpose4(uint32_t i0, uint32_t i1, uint32_t i2, uint32_t i3,
                                           uint32_t &o0, uint32_t &o1, uint32_t &o2,
                                           uint32_t &o3) {
  const uint32_t lo01 = __byte_perm(i0, i1, 0x5140);  // i0.b0 i1.b0 i0.b1 i1.b1
  const uint32_t hi01 = __byte_perm(i0, i1, 0x7362);  // i0.b2 i1.b2 i0.b3 i1.b3
  const uint32_t lo23 = __byte_perm(i2, i3, 0x5140);
  const uint32_t hi23 = __byte_perm(i2, i3, 0x7362);
  o0 = __byte_perm(lo01, lo23, 0x5410);
  o1 = __byte_perm(lo01, lo23, 0x7632);
  o2 = __byte_perm(hi01, hi23, 0x5410);
  o3 = __byte_perm(hi01, hi23, 0x7632);
}

}  // namespace xe
