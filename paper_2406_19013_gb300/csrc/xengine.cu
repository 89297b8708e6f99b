// xengine.cu -- the X-engine CMAC kernel for sm_103a (tcgen05 + TMA + TMEM).
//
// For one channel, the X-engine (Sec. 2.3) forms V[i][j] = sum_t x_i conj(x_j)
// over the lower triangle (Eq. 1, Eq. 2).  With x = a + j b:
//   Re V_ij = sum_t a_i a_j + b_i b_j   = <[a_i, b_i], [a_j, b_j]>
//   Im V_ij = sum_t b_i a_j - a_i b_j   = <[b_i, -a_i], [a_j, b_j]>
// so with K running over (t, re/im) the whole channel is one real matrix
// product D = Arows * Brows^T, where every input contributes an "A row"
// [a, b] (used on both sides) and a "Q row" [b, -a] (row side only).  That is
// a dense rank-2T update, so it runs on the tensor cores: 8-bit float operands
// (E5M2: every integer in [-8, 8] is exact) and fp32 accumulators in TMEM.
// Each product is an integer of magnitude <= 64 and an item never spans more
// than 131071 samples, so its partial sums stay below 128 * 131071 < 2^24 and
// every fp32 accumulation is exact; each item's partials are folded into the
// int64 integration buffer when it ends.
//
// Kernel structure (persistent, one CTA per SM, 25 warps):
//   warp 20     TMA producer: packed bytes [channel][input][time] -> smem ring
//   warps 0-15  unpack: 4-bit nibbles -> E5M2 A/Q rows in the 128B-swizzled
//               K-major layout the MMA reads (the paper's CPU "fluff" step,
//               Sec. 2.3, moved on chip)
//   warps 21-24 MMA issuers: tcgen05.mma M=128 (64 inputs' A rows + Q rows),
//               N = columns of the triangle strip, K = 32 per instruction;
//               one issuing thread per accumulator, because a single thread
//               issues an MMA only every ~110-126 cycles in a loop with
//               waits and commits, too slow for the N = 64 strips alone
//   warps 16-19 epilogue: tcgen05.ld of the fp32 accumulators, exchange of
//               re/im between lanes, int64 red.add into the lower triangle
// A launch integrates up to kMaxBlocksPerLaunch blocks; the host cuts its
// items at fold windows of at most 131071 samples.
// A work unit is (problem, template, channel); a template names the inputs
// staged per chunk and the MMAs (row tile x column range) that cover its part
// of the triangle.  The host cuts the units into items (a unit over a range
// of 128-sample stages) and gives every CTA a contiguous run of items of
// about equal cost, so the last wave does not leave SMs idle; a launch may
// hold several independent problems (a batch of correlators).  All waits are
// bounded by a timeout; on expiry the kernel drains its own copies and MMAs,
// frees TMEM and reports through *status.
// The CTA-pair instance (PAIR) runs clusters of two CTAs on two SMs: each
// stages and unpacks two row tiles and half of a B operand of up to 256
// columns, the even CTA's two issuers run M = 256 MMAs (cta_group::2) over
// both halves and commit to both CTAs' barriers, one thread of the odd CTA
// forwards its unpack warps' stage arrivals to the even CTA, and each CTA
// folds its own 128 TMEM lanes.
#include <cuda.h>

#include <cstring>

#include "ptx.cuh"
#include "xe_internal.h"
#include "xe_unpack.cuh"

namespace xe {

namespace {

struct Bars {
  uint32_t pk_full, pk_empty, z_full, z_empty, acc_full, acc_empty, drain, never;
};

}  // namespace

// Item `it` of the launch (explicit list, or derived from the unit index).
__device__ __forceinline__ XItem item_at(const XParams &p, int it) {
  if (p.items) return p.items[it];
  XItem r;
  r.prob = 0;
  r.tpl = it / p.implicit_n_chan;
  r.chan = it - r.tpl * p.implicit_n_chan;
  r.pk0 = 0;
  r.npk = p.implicit_npk;
  return r;
}

// Chunks (of kChunkSamples) in packed stage kc of a block.
__device__ __forceinline__ int chunks_in_pk(const XProb &pb, int kc) {
  return min(kChunksPerPk, pb.chunks_per_block - kChunksPerPk * kc);
}

// kThreads = 32 * 25: warps 0-15 unpack, 16-19 epilogue, 20 TMA, 21-24 MMA.
// Every role walks the same item list, [cta_first[b], cta_first[b + 1]).
// TCN: the blocks are in F-engine order (XParams::tcn), staged and unpacked
// by the transposing path; a compile-time choice, so that the X-engine-order
// kernel carries none of that code.
// PAIR: the launch is clusters of two CTAs running pair units (XUnit::
// pair_rows): both CTAs stage and unpack their own rows, the even CTA's
// issuers run M = 256 MMAs over both, and both fold their own TMEM rows.
template <int M, bool TCN, bool PAIR>
__global__ void __launch_bounds__(kThreads, 1)
    xengine_cmac_kernel(const __grid_constant__ XMapsT<M> maps, const XParams p) {
  extern __shared__ uint8_t smem_raw[];
  // 1024-byte alignment for the swizzled operand atoms
  uint8_t *smem = reinterpret_cast<uint8_t *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  uint8_t *z_buf = smem;
  uint8_t *pk_buf = z_buf + (size_t)p.z_stages * p.z_stage_bytes;
  uint64_t *bar_mem = reinterpret_cast<uint64_t *>(pk_buf + (size_t)p.pk_stages * p.pk_stage_bytes);
  // [pk_full x S][pk_empty x S][z_full x Z][z_empty x Z][acc_full][acc_empty][drain x kMmaWarps]
  // [never]: the last is only waited on by the failure-detection self-test
  uint32_t *misc = reinterpret_cast<uint32_t *>(bar_mem + 2 * p.pk_stages + 2 * p.z_stages + 2 +
                                                kMmaWarps + 1);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(misc + 1);
  const uint32_t bar0 = smem_u32(bar_mem);
  Bars b;
  b.pk_full = bar0;
  b.pk_empty = bar0 + 8 * p.pk_stages;
  b.z_full = bar0 + 16 * p.pk_stages;
  b.z_empty = b.z_full + 8 * p.z_stages;
  b.acc_full = b.z_empty + 8 * p.z_stages;
  b.acc_empty = b.acc_full + 8;
  b.drain = b.acc_empty + 8;
  b.never = b.drain + 8 * kMmaWarps;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < p.pk_stages; ++s) {
      mbar_init(b.pk_full + 8 * s, 1);
      mbar_init(b.pk_empty + 8 * s, kUnpackWarps);
    }
    for (int s = 0; s < p.z_stages; ++s) {
      // a pair's even CTA also counts the odd CTA's forwarded arrive
      mbar_init(b.z_full + 8 * s, (PAIR && cluster_ctarank() == 0) ? kUnpackWarps + 1 : kUnpackWarps);
      mbar_init(b.z_empty + 8 * s, PAIR ? kPairIssuers : kMmaWarps);
    }
    mbar_init(b.acc_full, PAIR ? kPairIssuers : kMmaWarps);
    mbar_init(b.acc_empty, PAIR ? 2 * kEpiWarps : kEpiWarps);
    for (int m = 0; m < kMmaWarps; ++m) mbar_init(b.drain + 8 * m, 1);
    mbar_init(b.never, 1);  // nothing ever arrives here
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == kWarpMma0) {
    if (PAIR) {
      tmem_alloc_pair(smem_u32(misc), kTmemCols);
      tmem_relinquish_pair();
    } else {
      tmem_alloc(smem_u32(misc), kTmemCols);
      tmem_relinquish();
    }
  }
  tc_fence_before();
  __syncthreads();
  // a pair's CTAs arrive on each other's barriers: both must be initialised
  if (PAIR) cluster_sync();
  tc_fence_after();
  const uint32_t tmem = misc[0];
  // rank in the pair (the odd CTA stages its regions from in_lo1 and owns
  // its segments' rows from row_in1)
  const uint32_t rank = PAIR ? cluster_ctarank() : 0u;

  int it0, it1, it_step;
  if (p.items) {
    const int wkr = PAIR ? (int)(blockIdx.x >> 1) : (int)blockIdx.x;  // cluster or CTA
    it0 = p.cta_first[wkr];
    it1 = p.cta_first[wkr + 1];
    it_step = 1;
  } else {
    it0 = blockIdx.x;
    it1 = p.implicit_n_tpl * p.implicit_n_chan;
    it_step = gridDim.x;
  }
  const uint64_t to = p.timeout_ns;

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
      for (int it = it0; it < it1 && ok && !*abort_flag; it += it_step) {
        const XItem item = item_at(p, it);
        const XProb pb = p.probs[item.prob];
        const XUnit *u = pb.units + item.tpl;
        const int n_reg = u->n_reg;
        const uint32_t bytes = (uint32_t)u->pk_bytes;
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
          for (int r = 0; r < n_reg; ++r) {
            const int in_lo = rank ? u->reg[r].in_lo1 : u->reg[r].in_lo, n_in = u->reg[r].n_in;
            const int off = u->reg[r].pk_off;
            const int ch = item.chan + u->reg[r].chan_off;  // past the last: zero fill
            for (int bx = 0; bx < n_in; bx += kTileInputs) {
              if (TCN)  // (input, channel, time): a [128 samples][64 inputs] box
                tma_load_3d(dst0 + off + bx * kPackedRowBytes, tmap, full, in_lo + bx, ch,
                            kc * kPkSamples);
              else        // (time, input, channel): a [64 inputs][128 samples] box
                tma_load_3d(dst0 + off + bx * kPackedRowBytes, tmap, full, kc * kPkSamples,
                            in_lo + bx, ch);
            }
          }
          if (++s == p.pk_stages) { s = 0; ph ^= 1u; }
        }
      }
      // every load this thread armed must have landed before the CTA exits
      int dummy = 0;
      for (int k = 0; k < p.pk_stages; ++k)
        if (armed[k]) mbar_wait(b.pk_full + 8 * k, armed_ph[k], &dummy, to);
    }
  } else if (warp >= kWarpMma0) {
    // ------------------------------------------------------------ MMA issuers
    // Issuer m owns the accumulators of segments m, m + kMmaWarps, ...; one
    // thread per warp, so independent accumulators are fed by parallel
    // instruction streams.
    const int m = warp - kWarpMma0;
    // a pair's MMAs issue from its even CTA, one issuer per segment
    if (lane == 0 && (!PAIR || (rank == 0 && m < kPairIssuers))) {
      int zs = 0;
      uint32_t zph = 0;
      long long nu = 0;
      bool ok = true;
      for (int it = it0; it < it1 && ok && !*abort_flag; it += it_step, ++nu) {
        const XItem item = item_at(p, it);
        const XProb pb = p.probs[item.prob];
        const XUnit *u = pb.units + item.tpl;
        const int n_seg = u->n_seg;
        static_assert(kMaxSegs / kMmaWarps == 2, "two segments per issuer at most");
        // The (at most two) segments this issuer owns.  Their descriptors are
        // built once per item, for Z stage 0 and K slice 0, as 32-bit words:
        // a chunk in Z stage zs and K slice kk only adds (zs z_stage_bytes +
        // 32 kk) / 16 to the start-address field, so each MMA costs an add
        // or two and the instruction itself.  (One issuing thread shares its
        // SM sub-partition with four unpack warps; the fewer instructions it
        // needs per MMA, the sooner each MMA is issued.)
        const int n_mine = (m < n_seg) + (m + kMmaWarps < n_seg);
        uint32_t d_col[2], idesc[2], a_lo[2], b_lo[2], b_hi[2];
        const uint32_t z0 = smem_u32(z_buf), a_hi = sdesc_sw128_hi(1024u);
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const XSeg &sgm = u->seg[j < n_mine ? m + kMmaWarps * j : 0];
          d_col[j] = tmem + (uint32_t)sgm.tmem_col;
          idesc[j] = idesc_e5m2_f32(PAIR ? 256 : 128, sgm.n);
          a_lo[j] = sdesc_sw128_lo(z0 + (uint32_t)sgm.a_zrow * 128u);
          b_lo[j] = sdesc_sw128_lo(z0 + (uint32_t)sgm.b_zrow * 128u);
          b_hi[j] = sdesc_sw128_hi((uint32_t)sgm.b_sbo);
        }
        if (nu > 0 &&
            !(PAIR ? mbar_wait_cluster(b.acc_empty, (uint32_t)((nu - 1) & 1), abort_flag, to)
                   : mbar_wait(b.acc_empty, (uint32_t)((nu - 1) & 1), abort_flag, to)))
          break;
        tc_fence_after();
        uint32_t acc0 = 0;  // the item's first MMA of each accumulator overwrites it
        for (int k = item.pk0; k < item.pk0 + item.npk && ok; ++k) {
          const int nch = chunks_in_pk(pb, k % pb.pk_per_block);
          for (int sub = 0; sub < nch; ++sub) {
            if (!(PAIR ? mbar_wait_cluster(b.z_full + 8 * zs, zph, abort_flag, to)
                       : mbar_wait(b.z_full + 8 * zs, zph, abort_flag, to))) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t zoff = ((uint32_t)zs * p.z_stage_bytes) >> 4;
#pragma unroll
            for (int j = 0; j < 2; ++j) {
              if (j >= n_mine) break;
              const uint32_t al = a_lo[j] + zoff, bl = b_lo[j] + zoff;
#pragma unroll
              for (int kk = 0; kk < 4; ++kk) {
                if (PAIR)
                  mma_f8_ss_w_pair(d_col[j], al + 2u * kk, a_hi, bl + 2u * kk, b_hi[j], idesc[j],
                                   kk ? 1u : acc0);
                else
                  mma_f8_ss_w(d_col[j], al + 2u * kk, a_hi, bl + 2u * kk, b_hi[j], idesc[j],
                              kk ? 1u : acc0);
              }
            }
            acc0 = 1;
            if (PAIR)
              mma_commit_pair(b.z_empty + 8 * zs, 3);  // both CTAs' operand stages
            else
              mma_commit(b.z_empty + 8 * zs);
            if (++zs == p.z_stages) { zs = 0; zph ^= 1u; }
          }
        }
        if (ok) {
          if (PAIR)
            mma_commit_pair(b.acc_full, 3);
          else
            mma_commit(b.acc_full);
        }
      }
      // all MMAs this thread issued complete before TMEM is released
      if (PAIR)
        mma_commit_pair(b.drain + 8 * m, 1);
      else
        mma_commit(b.drain + 8 * m);
      int dummy = 0;
      mbar_wait(b.drain + 8 * m, 0, &dummy, to);
    }
    if (PAIR && rank != 0 && m == 0 && lane == 0) {
      // The odd CTA's operand stages are announced to the even CTA's
      // issuers by this one thread: it waits for the local unpack warps'
      // arrivals, then makes a single cluster-scope release-arrive on the
      // even CTA's z_full (one cluster fence per chunk instead of one per
      // unpack warp).
      int zs = 0;
      uint32_t zph = 0;
      bool ok = true;
      for (int it = it0; it < it1 && ok && !*abort_flag; it += it_step) {
        const XItem item = item_at(p, it);
        const XProb pb = p.probs[item.prob];
        for (int k = item.pk0; k < item.pk0 + item.npk && ok; ++k) {
          const int nch = chunks_in_pk(pb, k % pb.pk_per_block);
          for (int sub = 0; sub < nch; ++sub) {
            if (!mbar_wait(b.z_full + 8 * zs, zph, abort_flag, to)) { ok = false; break; }
            mbar_arrive_cluster(b.z_full + 8 * zs, 0);
            if (++zs == p.z_stages) { zs = 0; zph ^= 1u; }
          }
        }
      }
    }
  } else if (warp < kUnpackWarps) {
    // ------------------------------------------------------------ unpack
    // Thread tid owns rows row0 + R k of every staged region (R = 8 *
    // kUnpackWarps rows per pass) and the 16-sample group g of each chunk;
    // the 8 lanes of a quarter-warp share g and take 8 consecutive rows, so
    // their swizzled 16-byte accesses fall on 8 different bank groups.
    constexpr int R = 8 * kUnpackWarps;
    // a staged region holds at most 2 R rows, so a thread has at most two
    // items per chunk: both loads go out before either decode
    static_assert(2 * R >= kMaxRegionInputs, "two items per thread cover a region");
    const int tid = threadIdx.x;
    const int g = (tid >> 3) & 3, row0 = (tid & 7) | ((tid >> 5) << 3), sw = row0 & 7;
    // packed rows arrive 128B-swizzled: 16-byte chunk c of row r sits at
    // c ^ (r & 7); operand chunk `sub` of a stage is chunks 4 sub + g
    const uint32_t src_sub0 = (uint32_t)((g ^ sw) << 4), src_sub1 = (uint32_t)(((4 + g) ^ sw) << 4);
    const uint32_t off0 = (uint32_t)(((2 * g) ^ sw) << 4), off1 = (uint32_t)(((2 * g + 1) ^ sw) << 4);
    const uint32_t pk_s0 = smem_u32(pk_buf), z_s0 = smem_u32(z_buf);
    int s = 0, zs = 0;
    uint32_t ph = 0, zph = 0;
    bool ok = true;
    for (int it = it0; it < it1 && ok && !*abort_flag; it += it_step) {
      const XItem item = item_at(p, it);
      const XProb pb = p.probs[item.prob];
      const XUnit *u = pb.units + item.tpl;
      const int n_reg = u->n_reg;
      // per-region constants of this thread (at most two regions).  When
      // both regions together have at most R rows (a two-channel unit),
      // region 1's rows follow region 0's in the thread mapping, so every
      // unpack warp gets work; otherwise both start at row0.
      const int pack =
          n_reg == 2 && u->reg[0].n_in + u->reg[1].n_in <= R ? u->reg[0].n_in : 0;
      uint32_t src_off[2], dst_off[2], dst_step[2];
      int n_k[2], il[2];
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const XRegion rg = u->reg[r < n_reg ? r : 0];
        const int rr = r == 1 ? row0 - pack : row0;  // this thread's row of the region
        il[r] = rg.interleaved == 1;  // Q rows are decoded and stored
        const int rho0 = rg.interleaved ? (((rr >> 3) << 4) | sw) : rr;
        src_off[r] = (uint32_t)(rg.pk_off + rr * kPackedRowBytes);
        dst_off[r] = (uint32_t)(rg.z_row + rho0) * 128u;
        dst_step[r] = (uint32_t)((rg.interleaved ? 2 * R : R) * 128);  // R rows further on
        n_k[r] = r < n_reg && rr >= 0 && rr < rg.n_in ? (rg.n_in - rr + R - 1) / R : 0;
      }
      for (int k = item.pk0; k < item.pk0 + item.npk && ok; ++k) {
        const int nch = chunks_in_pk(pb, k % pb.pk_per_block);
        if (!mbar_wait(b.pk_full + 8 * s, ph, abort_flag, to)) { ok = false; break; }
        const uint32_t pk_s = pk_s0 + (uint32_t)s * p.pk_stage_bytes;
#pragma unroll
        for (int sub = 0; sub < kChunksPerPk; ++sub) {
          if (sub >= nch) break;
          if (!mbar_wait(b.z_empty + 8 * zs, zph ^ 1u, abort_flag, to)) { ok = false; break; }
          const uint32_t z_s = z_s0 + (uint32_t)zs * p.z_stage_bytes;
          if (TCN) {
            // F-engine order: each 64-input box is [128 samples][64 inputs].
            // Item (q, j) of a box: inputs 4 q .. 4 q + 3, samples 8 j ..
            // 8 j + 7 of the chunk; eight 4-byte loads (one sample of four
            // inputs each), two 4 x 4 byte transposes, and per input two
            // decoded words: 16 bytes of its A row (and Q row) at K bytes
            // 16 j .. 16 j + 15.  The half-warp of odd j loads its samples
            // rotated by one (the same rotation for every input, so a fixed
            // permutation of K), which puts the two half-warps' rows on
            // different bank halves.  Within every 8-input group of a region
            // the operand row of group position pos is (pos + group) % 8: the
            // eight threads of a store phase then hit eight bank groups.
#pragma unroll
            for (int r = 0; r < 2; ++r) {
              if (r >= n_reg) break;
              const XRegion rg = u->reg[r];
              const int u_it = tid;
              if (u_it < (rg.n_in / kTileInputs) * 128) {
                const int box = u_it >> 7, v = u_it & 127, qd = v & 15, j = v >> 4, jj = j & 1;
                const uint32_t src = pk_s + (uint32_t)rg.pk_off + (uint32_t)box * 8192u +
                                     (uint32_t)(64 * (kChunkSamples * sub + 8 * j)) + 4u * qd;
                uint32_t w[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) w[k] = lds32(src + 64u * (uint32_t)((k + jj) & 7));
                uint32_t lo[4], hi[4];
                transpose4(w[0], w[1], w[2], w[3], lo[0], lo[1], lo[2], lo[3]);
                transpose4(w[4], w[5], w[6], w[7], hi[0], hi[1], hi[2], hi[3]);
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                  uint2 al, ql, ah, qh;
                  decode_word(lo[e], al, ql);
                  decode_word(hi[e], ah, qh);
                  const int i_rel = kTileInputs * box + 4 * qd + e, grp = i_rel >> 3;
                  const int pos = ((i_rel & 7) + (grp & 3)) & 7;
                  const int zrow = rg.z_row + (rg.interleaved ? 16 * grp : 8 * grp) + pos;
                  const uint32_t d = z_s + (uint32_t)zrow * 128u + (uint32_t)((j ^ pos) << 4);
                  sts128(d, al.x, al.y, ah.x, ah.y);
                  if (rg.interleaved == 1) sts128_q(d, ql.x, ql.y, qh.x, qh.y);
                }
              }
            }
          } else {
          // operand chunk `sub` of the packed stage (64 of its 128 samples)
#pragma unroll
          for (int r = 0; r < 2; ++r) {
            if (r >= n_reg) break;
            const uint32_t src = pk_s + src_off[r] + (sub ? src_sub1 : src_sub0);
            const uint32_t dst = z_s + dst_off[r];
            uint4 in0 = make_uint4(0u, 0u, 0u, 0u), in1 = in0;
            if (n_k[r] > 0) in0 = lds128(src);
            if (n_k[r] > 1) in1 = lds128(src + R * kPackedRowBytes);
#pragma unroll
            for (int kr = 0; kr < 2; ++kr) {
              if (kr >= n_k[r]) break;
              const uint4 in = kr == 0 ? in0 : in1;
              const uint32_t d0 = dst + (kr ? dst_step[r] : 0u) + off0;
              const uint32_t d1 = dst + (kr ? dst_step[r] : 0u) + off1;
              if (il[r]) {
                uint2 a0, q0, a1, q1, a2, q2, a3, q3;
                decode_word(in.x, a0, q0);
                decode_word(in.y, a1, q1);
                decode_word(in.z, a2, q2);
                decode_word(in.w, a3, q3);
                sts128(d0, a0.x, a0.y, a1.x, a1.y);
                sts128(d1, a2.x, a2.y, a3.x, a3.y);
                // the Q rows follow 8 rows (1024 bytes) after the A rows
                sts128_q(d0, q0.x, q0.y, q1.x, q1.y);
                sts128_q(d1, q2.x, q2.y, q3.x, q3.y);
              } else {
                uint2 a0, a1, a2, a3;
                decode_word_a(in.x, a0);
                decode_word_a(in.y, a1);
                decode_word_a(in.z, a2);
                decode_word_a(in.w, a3);
                sts128(d0, a0.x, a0.y, a1.x, a1.y);
                sts128(d1, a2.x, a2.y, a3.x, a3.y);
              }
            }
          }
          }
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
    const int g = rho >> 4, is_im = (rho >> 3) & 1, l = rho & 7;
    long long nu = 0;
    // failure-detection self-test: wait for a barrier that nothing completes;
    // the bounded wait gives up, raises the abort flag and every role winds
    // down (nothing is folded)
    if (p.selftest_never) mbar_wait(b.never, 0, abort_flag, to);
    for (int it = it0; it < it1; it += it_step, ++nu) {
      const XItem item = item_at(p, it);
      const XProb pb = p.probs[item.prob];
      const XUnit *u = pb.units + item.tpl;
      if (!mbar_wait(b.acc_full, (uint32_t)(nu & 1), abort_flag, to)) break;
      // once the kernel is winding down nothing more is folded: the
      // integration is void and is reported as such
      if (*abort_flag) break;
      tc_fence_after();
      const int n_seg = u->n_seg;
      // in F-engine-order launches, lane 16 g + l holds the input at group
      // position (l - g) % 8 of its 8-input group, and column 8 G + e the one
      // at (e - G) % 8 (the groups of a row tile or column range start at
      // multiples of 64 inputs, so only g % 4 and G % 4 matter)
      const int l_in = TCN ? ((l - (g & 3)) & 7) : l;
      for (int sg = 0; sg < n_seg; ++sg) {
        const XSeg sgm = u->seg[sg];
        // a tile of several channels: this lane's row belongs to channel
        // block ci (the same for every lane of the warp, whose 16 rows lie in
        // one block of at least 16)
        const int rpc = sgm.ch_rows;
        const int il = (rank ? sgm.row_in1 : sgm.row_in0) + 8 * g + l_in;
        const int ci = rpc ? il / rpc : 0;
        const int c = item.chan + sgm.chan_off + ci;
        if (c >= pb.n_chan) continue;  // a multi-channel unit's missing last channels
        const int i = il - ci * rpc;
        const bool row_ok = i < pb.n_in;
        int64_t *arow = pb.acc + ((long long)c * pb.n_pairs + (long long)i * (i + 1) / 2) * 2;
        const long long acc_elems = (long long)pb.n_chan * pb.n_pairs * 2;
        for (int cb = 0; cb < sgm.n; cb += 16) {
          uint32_t v[16];
          __syncwarp();
          tmem_ld_32x32b_x16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(sgm.tmem_col + cb), v);
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
          const int cc = cb + (is_im ? 8 : 0);  // the 8 columns of this lane
          int j0 = sgm.col_blk[cc >> 6] + (cc & 63);
          bool blk_ok = true;  // the 8 columns lie in this row's channel block
          if (rpc) {
            blk_ok = j0 / rpc == ci;
            j0 -= (j0 / rpc) * rpc;
          }
          if (TCN) {
            const int rot = ((cb + (is_im ? 8 : 0)) >> 3) & 3;
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              const int jj = j0 + ((e - rot) & 7);
              if (row_ok && blk_ok && jj <= i) {
                acc_add(pb.acc, acc_elems, p.status, arow + 2 * (long long)jj, re[e]);
                acc_add(pb.acc, acc_elems, p.status, arow + 2 * (long long)jj + 1, im[e]);
              }
            }
          } else {
            const int nvalid = row_ok && blk_ok ? min(8, i - j0 + 1) : 0;
            int64_t *ptr = arow + 2 * (long long)j0;
#pragma unroll
            for (int e = 0; e < 8; ++e)
              if (e < nvalid) {
                acc_add(pb.acc, acc_elems, p.status, ptr + 2 * e, re[e]);
                acc_add(pb.acc, acc_elems, p.status, ptr + 2 * e + 1, im[e]);
              }
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        if (PAIR && rank != 0)
          mbar_arrive_cluster(b.acc_empty, 0);
        else
          mbar_arrive(b.acc_empty);
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  // a pair's even CTA reads the odd one's operands and the odd one arrives on
  // the even one's barriers: neither leaves before both are done
  if (PAIR) cluster_sync();
  if (warp == kWarpMma0) {
    __syncwarp();
    tc_fence_after();
    if (PAIR)
      tmem_dealloc_pair(tmem, kTmemCols);
    else
      tmem_dealloc(tmem, kTmemCols);
  }
  if (threadIdx.x == 0 && *abort_flag) atomicOr(p.status, 1);
}

cudaError_t cmac_set_smem(int smem_bytes) {
  cudaError_t e = cudaFuncSetAttribute(xengine_cmac_kernel<kMaxMaps, false, false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(xengine_cmac_kernel<kMaxMaps, true, false>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(xengine_cmac_kernel<kMaxMaps, false, true>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(xengine_cmac_kernel<kMaxBatchMaps, false, false>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
}

cudaError_t launch_cmac(const XMaps &maps, const XParams &p, int grid, int smem_bytes,
                        cudaStream_t stream) {
  if (p.tcn)
    xengine_cmac_kernel<kMaxMaps, true, false><<<grid, kThreads, smem_bytes, stream>>>(maps, p);
  else
    xengine_cmac_kernel<kMaxMaps, false, false><<<grid, kThreads, smem_bytes, stream>>>(maps, p);
  return cudaGetLastError();
}

namespace {
// Launch configuration of the pair instance: clusters of two CTAs.
struct PairConfig {
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  PairConfig(int clusters, int smem_bytes, cudaStream_t stream) {
    cfg = cudaLaunchConfig_t{};
    cfg.gridDim = dim3(2 * clusters);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = (size_t)smem_bytes;
    cfg.stream = stream;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
  }
};
}  // namespace

cudaError_t launch_cmac_pair(const XMaps &maps, const XParams &p, int clusters, int smem_bytes,
                             cudaStream_t stream) {
  PairConfig c(clusters, smem_bytes, stream);
  return cudaLaunchKernelEx(&c.cfg, xengine_cmac_kernel<kMaxMaps, false, true>, maps, p);
}

int cmac_pair_clusters(int smem_bytes) {
  PairConfig c(1, smem_bytes, nullptr);
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, xengine_cmac_kernel<kMaxMaps, false, true>, &c.cfg) !=
      cudaSuccess)
    return 0;
  return n;
}

cudaError_t launch_cmac_batch(const XBatchMaps &maps, const XParams &p, int grid, int smem_bytes,
                              cudaStream_t stream) {
  xengine_cmac_kernel<kMaxBatchMaps, false, false><<<grid, kThreads, smem_bytes, stream>>>(maps, p);
  return cudaGetLastError();
}

}  // namespace xe
