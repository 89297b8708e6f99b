// xengine_tm.cu -- the X-engine CMAC kernel for windows of up to three row
// tiles (N <= 192 inputs, the paper's 96 dual-polarisation antennas), with
// the row operand of row tile 0 in tensor memory.
//
// The arithmetic is that of xengine.cu (Sec. 2.3, Eq. 1, Eq. 2): every input
// contributes an "A row" [a, b] and a "Q row" [b, -a] of E5M2 values along
// K = (sample, re/im); Re V_ij = <A_i, A_j> and Im V_ij = <Q_i, A_j>, so each
// 64-input row tile is one MMA per K slice of its 128 rows (A and Q rows of its
// inputs) against A rows of the inputs of its strip, fp32 in TMEM, folded into
// int64 once per item.
//
// What differs is where the operands live.  Shared-memory bandwidth binds the
// all-shared-memory kernel: per 64-sample chunk at 192 inputs it moves 168 KB
// through the SM's shared memory.  Here row tile 0's row operand is written
// straight into TMEM by the unpack warps (tcgen05.st, 16 lanes x 256 bits:
// lanes 16 b + l hold the A row of input 8 b + l and lanes 16 b + 8 + l its
// Q row) and read from there by its MMAs, which saves that tile's Q-row
// stores and its operand reads: 144 KB per chunk.  Tiles 1 and 2 keep their
// operands in shared memory, in the row order TmGeom describes, so that every
// tile's operands are contiguous rows (one MMA per tile per K slice).  At 192
// inputs the accumulators take 384 TMEM columns and the ring of tile-0 slots
// the other 128: four chunks of depth.
//
// Warp roles (24 warps, one CTA per SM, persistent over a balanced item list):
//   warps 0-15  unpack: warps 0-7 write one 8-input block of row tile 0 each
//               to TMEM (its A rows also to shared memory, the column
//               operand); the inputs of tiles 1 and 2 are unpacked into shared
//               memory, one 16-sample group of one input per thread
//   warps 16-19 epilogue: tcgen05.ld, re/im pairing, int64 red.add
//   warp 20     TMA producer
//   warps 21-23 MMA issuers, one per row tile
// Every wait is bounded; on expiry the kernel drains its copies and MMAs,
// frees TMEM and reports through *status.
#include <cuda.h>

#include "ptx.cuh"
#include "xe_internal.h"
#include "xe_unpack.cuh"

namespace xe {

namespace {

constexpr int kTmMmaWarps = 3;
constexpr int kTmWarpMma0 = kWarpTma + 1;
constexpr int kTmThreads = 32 * (kTmWarpMma0 + kTmMmaWarps);
static_assert(kTmThreads == 768, "24 warps");

struct TmBars {
  uint32_t pk_full, pk_empty, z_full, z_empty, acc_full, acc_empty, drain, never;
};

__device__ __forceinline__ XItem tm_item_at(const XParams &p, int it) {
  if (p.items) return p.items[it];
  XItem r;
  r.prob = 0;
  r.tpl = 0;
  r.chan = it;
  r.pk0 = 0;
  r.npk = p.implicit_npk;
  return r;
}

}  // namespace

__global__ void __launch_bounds__(kTmThreads, 1)
    xengine_cmac_tm_kernel(const __grid_constant__ XMaps maps, const XParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  uint8_t *z_buf = smem;
  uint8_t *pk_buf = z_buf + (size_t)p.z_stages * p.z_stage_bytes;
  uint64_t *bar_mem = reinterpret_cast<uint64_t *>(pk_buf + (size_t)p.pk_stages * p.pk_stage_bytes);
  uint32_t *misc = reinterpret_cast<uint32_t *>(bar_mem + 2 * p.pk_stages + 2 * p.z_stages + 2 +
                                                kTmMmaWarps + 1);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(misc + 1);
  const uint32_t bar0 = smem_u32(bar_mem);
  TmBars b;
  b.pk_full = bar0;
  b.pk_empty = bar0 + 8 * p.pk_stages;
  b.z_full = bar0 + 16 * p.pk_stages;
  b.z_empty = b.z_full + 8 * p.z_stages;
  b.acc_full = b.z_empty + 8 * p.z_stages;
  b.acc_empty = b.acc_full + 8;
  b.drain = b.acc_empty + 8;
  b.never = b.drain + 8 * kTmMmaWarps;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const TmGeom G = tm_geom(p.probs[0].n_in);

  if (threadIdx.x == 0) {
    for (int s = 0; s < p.pk_stages; ++s) {
      mbar_init(b.pk_full + 8 * s, 1);
      mbar_init(b.pk_empty + 8 * s, kUnpackWarps);
    }
    for (int s = 0; s < p.z_stages; ++s) {
      mbar_init(b.z_full + 8 * s, kUnpackWarps);
      mbar_init(b.z_empty + 8 * s, kTmMmaWarps);
    }
    mbar_init(b.acc_full, kTmMmaWarps);
    mbar_init(b.acc_empty, kEpiWarps);
    for (int m = 0; m < kTmMmaWarps; ++m) mbar_init(b.drain + 8 * m, 1);
    mbar_init(b.never, 1);  // nothing ever arrives here
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == kTmWarpMma0) {
    tmem_alloc(smem_u32(misc), kTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = misc[0];

  int it0, it1, it_step;
  if (p.items) {
    it0 = p.cta_first[blockIdx.x];
    it1 = p.cta_first[blockIdx.x + 1];
    it_step = 1;
  } else {
    it0 = blockIdx.x;
    it1 = p.implicit_n_chan;
    it_step = gridDim.x;
  }
  const uint64_t to = p.timeout_ns;
  const XProb pb = p.probs[0];
  const long long acc_elems = (long long)pb.n_chan * pb.n_pairs * 2;
  const int n_st = kTileInputs * G.n_rt;  // staged inputs

  if (warp == kWarpTma) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      int s = 0;
      uint32_t ph = 0;
      int armed[kMaxPkStages];
      uint32_t armed_ph[kMaxPkStages];
      for (int k = 0; k < kMaxPkStages; ++k) armed[k] = 0, armed_ph[k] = 0;
      bool ok = true;
      int last_map = -1;
      const uint32_t bytes = (uint32_t)(n_st * kPackedRowBytes);
      for (int it = it0; it < it1 && ok && !*abort_flag; it += it_step) {
        const XItem item = tm_item_at(p, it);
        for (int k = item.pk0; k < item.pk0 + item.npk; ++k) {
          const int blk = k / pb.pk_per_block, kc = k - blk * pb.pk_per_block;
          const int mi = pb.map0 + blk;
          const void *tmap = &maps.m[mi][0];
          if (mi != last_map) { prefetch_tmap(tmap); last_map = mi; }
          if (!mbar_wait(b.pk_empty + 8 * s, ph ^ 1u, abort_flag, to)) { ok = false; break; }
          const uint32_t full = b.pk_full + 8 * s;
          mbar_arrive_expect_tx(full, bytes);
          armed[s] = 1;
          armed_ph[s] = ph;
          const uint32_t dst0 = smem_u32(pk_buf + (size_t)s * p.pk_stage_bytes);
          for (int bx = 0; bx < n_st; bx += kTileInputs)
            tma_load_3d(dst0 + bx * kPackedRowBytes, tmap, full, kc * kPkSamples, bx, item.chan);
          if (++s == p.pk_stages) { s = 0; ph ^= 1u; }
        }
      }
      // every load this thread armed must have landed before the CTA exits
      int dummy = 0;
      for (int k = 0; k < p.pk_stages; ++k)
        if (armed[k]) mbar_wait(b.pk_full + 8 * k, armed_ph[k], &dummy, to);
    }
  } else if (warp >= kTmWarpMma0) {
    // ------------------------------------------------------------ MMA issuers
    // Issuer t runs row tile t's MMAs: tile 0 reads its row operand from the
    // TMEM ring, tiles 1 and 2 both operands from shared memory.
    const int t = warp - kTmWarpMma0;
    if (lane == 0) {
      const bool active = t < G.n_rt;
      const uint32_t d = tmem + (uint32_t)(active ? G.acc[t] : 0);
      const uint32_t idesc = idesc_e5m2_f32(128, active ? G.nt[t] : 16);
      const uint32_t z0 = smem_u32(z_buf), hi = sdesc_sw128_hi(1024u);
      // first rows of the row and column operands in the stage
      const int a_row = t == 1 ? G.row_q1 : G.row_a2;
      const int b_row = t == 0 ? G.row_a0 : G.row_a1;
      const uint32_t a_lo0 = sdesc_sw128_lo(z0 + (uint32_t)a_row * 128u);
      const uint32_t b_lo0 = sdesc_sw128_lo(z0 + (uint32_t)b_row * 128u);
      const uint32_t a_tm0 = tmem + (uint32_t)G.a_base;
      int zs = 0;
      uint32_t zph = 0;
      long long nu = 0;
      bool ok = true;
      for (int it = it0; it < it1 && ok && !*abort_flag; it += it_step, ++nu) {
        const XItem item = tm_item_at(p, it);
        if (nu > 0 && !mbar_wait(b.acc_empty, (uint32_t)((nu - 1) & 1), abort_flag, to)) break;
        tc_fence_after();
        uint32_t acc0 = 0;  // the item's first MMA overwrites the accumulator
        for (int k = item.pk0; k < item.pk0 + item.npk && ok; ++k) {
          const int kc = k % pb.pk_per_block;
          const int nch = min(kChunksPerPk, pb.chunks_per_block - kChunksPerPk * kc);
          for (int sub = 0; sub < nch; ++sub) {
            if (!mbar_wait(b.z_full + 8 * zs, zph, abort_flag, to)) { ok = false; break; }
            tc_fence_after();
            if (active) {
              const uint32_t zoff = ((uint32_t)zs * p.z_stage_bytes) >> 4;
              const uint32_t bl = b_lo0 + zoff;
              if (t == 0) {
                const uint32_t at = a_tm0 + (uint32_t)(zs * kTmSlotCols);
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)
                  mma_f8_ts_w(d, at + 8u * kk, bl + 2u * kk, hi, idesc, kk ? 1u : acc0);
              } else {
                const uint32_t al = a_lo0 + zoff;
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)
                  mma_f8_ss_w(d, al + 2u * kk, hi, bl + 2u * kk, hi, idesc, kk ? 1u : acc0);
              }
            }
            acc0 = 1;
            mma_commit(b.z_empty + 8 * zs);
            if (++zs == p.z_stages) { zs = 0; zph ^= 1u; }
          }
        }
        if (ok) mma_commit(b.acc_full);
      }
      // all MMAs this thread issued complete before TMEM is released
      mma_commit(b.drain + 8 * t);
      int dummy = 0;
      mbar_wait(b.drain + 8 * t, 0, &dummy, to);
    }
  } else if (warp < kUnpackWarps) {
    // ------------------------------------------------------------ unpack
    // TMEM item of warps 0-7 (lane quarter q = w % 4 may be written by warp
    // w): 8-input block bb = 2 q + w / 4 of row tile 0, TMEM lanes 16 bb ..
    // 16 bb + 15.  Thread (k8 = lane / 4, m = lane % 4) decodes input 8 bb + k8
    // at samples 16 r + 4 m .. + 3 (r = 0..3), the K bytes 32 r + 8 m .. + 7 of
    // the chunk, which the 16x256b.x4 store writes to its two lanes.  The A
    // row pieces also go to shared memory (tile 0's column operand): threads m
    // and m ^ 1 exchange pieces so that each writes two whole 16-byte chunks,
    // K slices m and m ^ 2, which keeps the eight threads of every store phase
    // on eight different bank groups.
    const int q = warp & 3, bb = 2 * q + ((warp >> 2) & 1);
    const bool tm_item = warp < 8;
    const int k8 = lane >> 2, m = lane & 3, h = m >> 1;
    const bool odd = (m & 1) != 0;
    const int in_tm = 8 * bb + k8;
    const int sw_tm = in_tm & 7;
    const uint32_t tm_addr = tmem + ((uint32_t)(32 * q + 16 * ((warp >> 2) & 1)) << 16) +
                             (uint32_t)G.a_base;
    const uint32_t ka = (uint32_t)(((2 * m + h) ^ sw_tm) << 4);        // K slice m
    const uint32_t kb = (uint32_t)(((2 * (m ^ 2) + h) ^ sw_tm) << 4);  // K slice m ^ 2
    const uint32_t a0_row = (uint32_t)(G.row_a0 + in_tm) * 128u;
    // shared-memory item: input 64 + i1 of tiles 1 and 2 (all 16 warps for
    // three row tiles, warps 8-15 for two), samples 16 g .. 16 g + 15
    const bool ss_item = G.n_rt == 3 || (G.n_rt == 2 && warp >= 8);
    const int i1 = (lane & 7) | ((G.n_rt == 3 ? warp : warp - 8) << 3);
    const int in_ss = kTileInputs + i1, g = (lane >> 3) & 3, sw = in_ss & 7;
    const bool in_t1 = in_ss < 2 * kTileInputs;
    const uint32_t ss_arow = (uint32_t)(in_t1 ? G.row_a1 + i1 : G.row_a2 + i1 - kTileInputs) * 128u;
    const uint32_t ss_qrow = (uint32_t)(in_t1 ? G.row_q1 + i1 : G.row_q2 + i1 - kTileInputs) * 128u;
    const uint32_t c0 = (uint32_t)(((2 * g) ^ sw) << 4), c1 = (uint32_t)(((2 * g + 1) ^ sw) << 4);
    const uint32_t pk_s0 = smem_u32(pk_buf), z_s0 = smem_u32(z_buf);
    int s = 0, zs = 0;
    uint32_t ph = 0, zph = 0;
    bool ok = true;
    for (int it = it0; it < it1 && ok && !*abort_flag; it += it_step) {
      const XItem item = tm_item_at(p, it);
      for (int k = item.pk0; k < item.pk0 + item.npk && ok; ++k) {
        const int kc = k % pb.pk_per_block;
        const int nch = min(kChunksPerPk, pb.chunks_per_block - kChunksPerPk * kc);
        if (!mbar_wait(b.pk_full + 8 * s, ph, abort_flag, to)) { ok = false; break; }
        const uint32_t pk_s = pk_s0 + (uint32_t)s * p.pk_stage_bytes;
#pragma unroll
        for (int sub = 0; sub < kChunksPerPk; ++sub) {
          if (sub >= nch) break;
          if (!mbar_wait(b.z_empty + 8 * zs, zph ^ 1u, abort_flag, to)) { ok = false; break; }
          tc_fence_after();
          const uint32_t z_s = z_s0 + (uint32_t)zs * p.z_stage_bytes;
          if (tm_item) {
            const uint32_t rowp = pk_s + (uint32_t)in_tm * kPackedRowBytes + 4u * (uint32_t)m;
            uint32_t w[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) w[r] = lds32(rowp + (uint32_t)((((sub << 2) + r) ^ sw_tm) << 4));
            uint2 a[4], qq[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) decode_word(w[r], a[r], qq[r]);
            uint32_t regs[16];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
              regs[4 * r] = a[r].x;
              regs[4 * r + 1] = a[r].y;
              regs[4 * r + 2] = qq[r].x;
              regs[4 * r + 3] = qq[r].y;
            }
            tmem_st_16x256b_x4(tm_addr + (uint32_t)(zs * kTmSlotCols), regs);
            // pieces for the partner: even m sends K slices 1, 3; odd m 0, 2
            const uint2 send0 = odd ? a[0] : a[1], send1 = odd ? a[2] : a[3];
            uint2 got0, got1;
            got0.x = __shfl_xor_sync(0xffffffffu, send0.x, 1);
            got0.y = __shfl_xor_sync(0xffffffffu, send0.y, 1);
            got1.x = __shfl_xor_sync(0xffffffffu, send1.x, 1);
            got1.y = __shfl_xor_sync(0xffffffffu, send1.y, 1);
            // K slice m (own a[m]) and K slice m ^ 2 (own a[m ^ 2])
            const uint2 own_a = h ? (odd ? a[3] : a[2]) : (odd ? a[1] : a[0]);
            const uint2 own_b = h ? (odd ? a[1] : a[0]) : (odd ? a[3] : a[2]);
            const uint2 got_a = h ? got1 : got0, got_b = h ? got0 : got1;
            const uint32_t arow = z_s + a0_row;
            if (odd) {
              sts128(arow + ka, got_a.x, got_a.y, own_a.x, own_a.y);
              sts128(arow + kb, got_b.x, got_b.y, own_b.x, own_b.y);
            } else {
              sts128(arow + ka, own_a.x, own_a.y, got_a.x, got_a.y);
              sts128(arow + kb, own_b.x, own_b.y, got_b.x, got_b.y);
            }
          }
          if (ss_item) {
            const uint4 in = lds128(pk_s + (uint32_t)in_ss * kPackedRowBytes +
                                    (uint32_t)((((sub << 2) + g) ^ sw) << 4));
            uint2 a0, q0, a1, q1, a2, q2, a3, q3;
            decode_word(in.x, a0, q0);
            decode_word(in.y, a1, q1);
            decode_word(in.z, a2, q2);
            decode_word(in.w, a3, q3);
            sts128(z_s + ss_arow + c0, a0.x, a0.y, a1.x, a1.y);
            sts128(z_s + ss_arow + c1, a2.x, a2.y, a3.x, a3.y);
            sts128(z_s + ss_qrow + c0, q0.x, q0.y, q1.x, q1.y);
            sts128(z_s + ss_qrow + c1, q2.x, q2.y, q3.x, q3.y);
          }
          if (tm_item) tmem_st_wait();
          tc_fence_before();
          fence_proxy_async_smem();
          __syncwarp();
          if (lane == 0) {
            mbar_arrive(b.z_full + 8 * zs);
            if (sub == nch - 1) mbar_arrive(b.pk_empty + 8 * s);
          }
          if (++zs == p.z_stages) { zs = 0; zph ^= 1u; }
        }
        if (++s == p.pk_stages) { s = 0; ph ^= 1u; }
      }
    }
  } else if (warp < kWarpTma) {
    // ------------------------------------------------------------ epilogue
    const int q = warp & 3;  // TMEM lane quarter this warp may access
    const int rho = 32 * q + lane;
    long long nu = 0;
    // failure-detection self-test: wait for a barrier that nothing completes
    if (p.selftest_never) mbar_wait(b.never, 0, abort_flag, to);
    for (int it = it0; it < it1; it += it_step, ++nu) {
      const XItem item = tm_item_at(p, it);
      const int c = item.chan;
      if (!mbar_wait(b.acc_full, (uint32_t)(nu & 1), abort_flag, to)) break;
      if (*abort_flag) break;
      tc_fence_after();
      int64_t *acc_c = pb.acc + (long long)c * pb.n_pairs * 2;
      // row tile 0 (TMEM operand): lane 16 g + l holds Re and lane 16 g + 8 + l
      // Im of input 8 g + l; the pair exchanges halves so each folds 8 columns
      {
        const int g = rho >> 4, is_im = (rho >> 3) & 1, l = rho & 7;
        const int i = 8 * g + l;
        const bool row_ok = i < pb.n_in;
        int64_t *arow = acc_c + (long long)i * (i + 1);
        for (int cb = 0; cb < G.nt[0]; cb += 16) {
          uint32_t v[16];
          __syncwarp();
          tmem_ld_32x32b_x16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(G.acc[0] + cb), v);
          tmem_ld_wait();
          int re[8], im[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const uint32_t send = is_im ? v[e] : v[8 + e];
            const uint32_t got = __shfl_xor_sync(0xffffffffu, send, 8);
            const int mine = __float2int_rn(__uint_as_float(is_im ? v[8 + e] : v[e]));
            const int other = __float2int_rn(__uint_as_float(got));
            re[e] = is_im ? other : mine;
            im[e] = is_im ? mine : other;
          }
          const int j0 = cb + (is_im ? 8 : 0);
          const int nvalid = row_ok ? min(8, i - j0 + 1) : 0;
          int64_t *ptr = arow + 2 * (long long)j0;
#pragma unroll
          for (int e = 0; e < 8; ++e)
            if (e < nvalid) {
              acc_add(pb.acc, acc_elems, p.status, ptr + 2 * e, re[e]);
              acc_add(pb.acc, acc_elems, p.status, ptr + 2 * e + 1, im[e]);
            }
        }
      }
      // row tiles 1 and 2 (shared-memory operands): tile 1's lanes 0-63 hold
      // Im (Q rows) and lanes 64-127 Re (A rows) of inputs 64..127, tile 2's
      // lanes 0-63 Re and 64-127 Im of inputs 128..191; each lane folds its
      // own component.  Column n is input 64 + n (n < 64), n - 64 (n < 128)
      // or n.
      for (int t = 1; t < G.n_rt; ++t) {
        const int i = kTileInputs * t + (rho & 63);
        const int comp = (t == 1) == (rho < 64) ? 1 : 0;
        const bool row_ok = i < pb.n_in;
        int64_t *arow = acc_c + (long long)i * (i + 1) + comp;
        const int ncols = t == 1 ? G.nt[1] : G.nt[2];
        const int col0 = t == 1 ? G.acc[1] : G.acc[2];
        for (int cb = 0; cb < ncols; cb += 16) {
          uint32_t v[16];
          __syncwarp();
          tmem_ld_32x32b_x16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(col0 + cb), v);
          tmem_ld_wait();
          const int j0 = cb < kTileInputs ? kTileInputs + cb : (cb < 2 * kTileInputs ? cb - kTileInputs : cb);
          const int nvalid = row_ok ? min(16, i - j0 + 1) : 0;
          int64_t *ptr = arow + 2 * (long long)j0;
#pragma unroll
          for (int e = 0; e < 16; ++e)
            if (e < nvalid)
              acc_add(pb.acc, acc_elems, p.status, ptr + 2 * e,
                      __float2int_rn(__uint_as_float(v[e])));
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(b.acc_empty);
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == kTmWarpMma0) {
    __syncwarp();
    tc_fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
  if (threadIdx.x == 0 && *abort_flag) atomicOr(p.status, 1);
}

cudaError_t cmac_tm_set_smem(int smem_bytes) {
  return cudaFuncSetAttribute(xengine_cmac_tm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              smem_bytes);
}

cudaError_t launch_cmac_tm(const XMaps &maps, const XParams &p, int grid, int smem_bytes,
                           cudaStream_t stream) {
  xengine_cmac_tm_kernel<<<grid, kTmThreads, smem_bytes, stream>>>(maps, p);
  return cudaGetLastError();
}

}  // namespace xe
