// xe_sched.cu -- triangle covers, shared-memory stage layout and the balanced
// split of a launch into per-CTA item runs (host code only).
#include "xe_sched.h"

#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

namespace xe {

namespace {

int round_up(int v, int m) { return (v + m - 1) / m * m; }

void add_seg(XUnit &u, int a_zrow, int b_zrow, int b_sbo, int n, int row_in0, int col_in0) {
  XSeg &s = u.seg[u.n_seg];
  int col = 0;
  for (int k = 0; k < u.n_seg; ++k) col += u.seg[k].n;
  s.a_zrow = a_zrow;
  s.b_zrow = b_zrow;
  s.b_sbo = b_sbo;
  s.n = n;
  s.tmem_col = col;
  s.row_in0 = row_in0;
  s.row_in1 = row_in0;
  for (int b = 0; b < 4; ++b) s.col_blk[b] = col_in0 + 64 * b;
  u.n_seg++;
  u.work += n;
}

void add_reg(XUnit &u, int in_lo, int n_in, int interleaved) {
  XRegion &r = u.reg[u.n_reg];
  r.in_lo = in_lo;
  r.in_lo1 = in_lo;
  r.n_in = n_in;
  r.interleaved = interleaved;
  r.z_row = u.z_rows;
  r.pk_off = u.pk_bytes;
  u.z_rows += interleaved ? 2 * n_in : n_in;
  u.pk_bytes += n_in * kPackedRowBytes;
  u.n_reg++;
}

XUnit empty_unit() {
  XUnit u;
  std::memset(&u, 0, sizeof(u));
  u.n_chan = 1;
  return u;
}

}  // namespace

// Tiles of 64 inputs (rows) cover the lower triangle strip by strip: row tile
// t needs columns [0, min(64 (t + 1), N)).  Within a unit, columns are staged
// once per chunk and shared by all its row tiles.
std::vector<XUnit> build_schedule(int N, int cover) {
  std::vector<XUnit> units;
  const int n16 = round_up(N, 16);
  const int n_rt = (N + kTileInputs - 1) / kTileInputs;
  if (N <= 32 && cover == kCoverWindow) {
    // 16 or 32 inputs at most: a 64-row tile holds 64 / n16 channels (the
    // TMA box brings that many channels' rows at once), and a unit two such
    // tiles; each tile's MMA also computes the cross-channel blocks, which
    // the epilogue skips
    XUnit u = empty_unit();
    const int cpt = kTileInputs / n16;
    u.n_chan = 2 * cpt;
    for (int r = 0; r < 2; ++r) {
      add_reg(u, 0, kTileInputs, 1);
      u.reg[r].chan_off = r * cpt;
    }
    for (int r = 0; r < 2; ++r) {
      add_seg(u, u.reg[r].z_row, u.reg[r].z_row, 2048, kTileInputs, 0, 0);
      u.seg[r].chan_off = r * cpt;
      u.seg[r].ch_rows = n16;
    }
    units.push_back(u);
  } else if (N <= 2 * kTileInputs && cover == kCoverWindow) {
    // one or two row tiles: a unit covers two channels (two staged regions,
    // one accumulator per row tile and channel, at most 2 x 192 TMEM
    // columns), so every chunk handed from the unpack to the MMA issuers
    // carries twice the work
    XUnit u = empty_unit();
    u.n_chan = 2;
    for (int r = 0; r < 2; ++r) {
      add_reg(u, 0, kTileInputs * n_rt, 1);
      u.reg[r].chan_off = r;
    }
    for (int r = 0; r < 2; ++r)
      for (int t = 0; t < n_rt; ++t) {
        add_seg(u, u.reg[r].z_row + 128 * t, u.reg[r].z_row, 2048,
                std::min(kTileInputs * (t + 1), n16), kTileInputs * t, 0);
        u.seg[u.n_seg - 1].chan_off = r;
      }
    units.push_back(u);
  } else if (N <= 256 && cover == kCoverWindow) {
    // units of consecutive row tiles, largest strip first, each as many as
    // fit 512 TMEM columns: a unit's lowest tile then bounds the inputs that
    // are only its columns, and those need no Q rows
    std::vector<std::vector<int>> bins;
    int used = kTmemCols + 1;
    for (int t = n_rt - 1; t >= 0; --t) {
      const int n = std::min(kTileInputs * (t + 1), n16);
      if (used + n > kTmemCols) {
        bins.push_back({});
        used = 0;
      }
      bins.back().push_back(t);
      used += n;
    }
    for (auto &bin : bins) {
      XUnit u = empty_unit();
      int t_max = 0, t_min = n_rt;
      for (int t : bin) t_max = std::max(t_max, t), t_min = std::min(t_min, t);
      // inputs below the unit's lowest row tile are only its columns: their
      // Q rows are neither decoded nor stored (same layout, so the B operand
      // still spans the window with one stride)
      if (t_min > 0) add_reg(u, 0, kTileInputs * t_min, 2);
      add_reg(u, kTileInputs * t_min, kTileInputs * (t_max + 1 - t_min), 1);
      for (int t : bin)
        add_seg(u, 128 * t, 0, 2048, std::min(kTileInputs * (t + 1), n16), kTileInputs * t, 0);
      units.push_back(u);
    }
  } else if (N <= 256 && cover == kCoverStrips) {
    for (int t = n_rt - 1; t >= 0; --t) {
      XUnit u = empty_unit();
      add_reg(u, 0, kTileInputs * (t + 1), 1);
      add_seg(u, 128 * t, 0, 2048, std::min(kTileInputs * (t + 1), n16), kTileInputs * t, 0);
      units.push_back(u);
    }
  } else if (N > 256 && cover == kCoverQuads) {
    // CTA pairs, blocks of 256 rows [R, R + 256) against 256 columns
    // [P, P + 256), P <= R, in four row tiles T0..T3 of 64 inputs.
    //  - Below the diagonal (P < R) the even CTA owns T0 and T1, the odd one
    //    T2 and T3; their B rows are a plain region, P .. P + 127 on the even
    //    CTA and P + 128 .. on the odd one.  Two N = 256 MMAs.
    //  - On the diagonal (P = R) the even CTA owns T0 and T3, the odd one T1
    //    and T2, and each CTA's own A rows are its B rows: the MMA of T0 and
    //    T1 (N = 128) takes the first 64 B rows of each CTA, columns T0 T1;
    //    that of T3 and T2 (N = 256) all of them, columns T0 T3 T1 T2.  That
    //    issues 3/4 of the work of two N = 256 MMAs over T0 T1 | T2 T3.
    for (int R = 0; R < N; R += 2 * kPairRows) {
      for (int P = 0; P <= R; P += 2 * kPairRows) {
        XUnit u = empty_unit();
        u.pair_rows = kPairRows;
        if (P < R) {
          add_reg(u, R, kPairRows, 1);
          u.reg[0].in_lo1 = R + kPairRows;
          add_reg(u, P, kPairRows, 0);
          u.reg[1].in_lo1 = P + kPairRows;
          const int bz = u.reg[1].z_row;
          for (int t = 0; t < 2; ++t) {
            add_seg(u, 128 * t, bz, 1024, 2 * kPairRows, R + kTileInputs * t, P);
            u.seg[t].row_in1 = R + kPairRows + kTileInputs * t;
          }
        } else {
          const int T = kTileInputs;
          add_reg(u, R, T, 1);  // even: T0, odd: T1
          u.reg[0].in_lo1 = R + T;
          add_reg(u, R + 3 * T, T, 1);  // even: T3, odd: T2
          u.reg[1].in_lo1 = R + 2 * T;
          add_seg(u, 0, 0, 2048, 2 * T, R, R);
          u.seg[0].row_in1 = R + T;
          u.seg[0].col_blk[1] = R + T;
          add_seg(u, 128, 0, 2048, 4 * T, R + 3 * T, R);
          u.seg[1].row_in1 = R + 2 * T;
          u.seg[1].col_blk[1] = R + 3 * T;
          u.seg[1].col_blk[2] = R + T;
          u.seg[1].col_blk[3] = R + 2 * T;
        }
        units.push_back(u);
      }
    }
  } else {
    // pairs of row tiles (2m, 2m+1) against 256-column pieces of their strip
    for (int m = 0; 2 * m < n_rt; ++m) {
      const int t0 = 2 * m;
      const bool two = t0 + 1 < n_rt;
      const int row_lo = kTileInputs * t0;
      const int kd = row_lo / 256;  // piece holding the diagonal
      for (int k = 0; k <= kd; ++k) {
        XUnit u = empty_unit();
        if (k < kd) {
          add_reg(u, row_lo, two ? 128 : 64, 1);
          add_reg(u, 256 * k, 256, 0);
          const int bz = u.reg[1].z_row;
          add_seg(u, 0, bz, 1024, 256, row_lo, 256 * k);
          if (two) add_seg(u, 128, bz, 1024, 256, row_lo + 64, 256 * k);
        } else {
          const int lo = 256 * k;
          const int hi = row_lo + (two ? 128 : 64);
          // inputs lo .. row_lo - 1 are only columns here: no Q rows
          if (row_lo > lo) add_reg(u, lo, row_lo - lo, 2);
          add_reg(u, row_lo, hi - row_lo, 1);
          const int a0 = 2 * (row_lo - lo);
          add_seg(u, a0, 0, 2048, std::min(row_lo + 64, n16) - lo, row_lo, lo);
          if (two) add_seg(u, a0 + 128, 0, 2048, std::min(row_lo + 128, n16) - lo, row_lo + 64, lo);
        }
        units.push_back(u);
      }
    }
  }
  std::stable_sort(units.begin(), units.end(),
                   [](const XUnit &a, const XUnit &b) { return a.work > b.work; });
  // the unpack handles regions of at most kMaxRegionInputs inputs (every
  // cover above satisfies this; an empty schedule reports a violation)
  for (const XUnit &u : units)
    for (int r = 0; r < u.n_reg; ++r)
      if (u.reg[r].n_in > kMaxRegionInputs) return {};
  return units;
}

int tile_ch_rows(const std::vector<XUnit> &units) {
  for (const XUnit &u : units)
    for (int s = 0; s < u.n_seg; ++s)
      if (u.seg[s].ch_rows) return u.seg[s].ch_rows;
  return kTileInputs;
}

bool stage_layout(const std::vector<const std::vector<XUnit> *> &unit_sets, int smem_optin,
                  int max_z, StageLayout *out) {
  int max_zr = 0, max_pk = 0;
  for (const auto *set : unit_sets)
    for (const XUnit &u : *set) {
      max_zr = std::max(max_zr, u.z_rows);
      max_pk = std::max(max_pk, u.pk_bytes);
    }
  StageLayout L;
  L.z_stage_bytes = (uint32_t)round_up(max_zr * 128, 1024);
  L.pk_stage_bytes = (uint32_t)round_up(max_pk, 1024);  // swizzled TMA destination
  const int fixed = 1024 /* alignment slack */ + kBarrierBytes;
  static_assert(8 * (2 * kMaxPkStages + 2 * kMaxZStages + 2 + kMmaWarps + 1) + 16 <= kBarrierBytes,
                "barrier area");
  const int avail = smem_optin - fixed;
  const int zb = (int)L.z_stage_bytes, pb = (int)L.pk_stage_bytes;
  const int zcap = std::min(max_z, kMaxZStages);
  // Operand stages first (three beside three packed stages, else three
  // beside two, else two beside three or two), then packed stages (bytes in
  // flight from HBM) up to six,
  // operand stages up to four, and both up to their caps while they fit.
  int zs, ps;
  if (3 * zb + 3 * pb <= avail && zcap >= 3) {
    zs = 3;
    ps = 3;
  } else if (3 * zb + 2 * pb <= avail && zcap >= 3) {
    // (the CTA-pair units: a third operand stage hides the peer's arrivals)
    zs = 3;
    ps = 2;
  } else if (2 * zb + 3 * pb <= avail) {
    zs = 2;
    ps = 3;
  } else if (2 * zb + 2 * pb <= avail) {
    zs = 2;
    ps = 2;
  } else {
    return false;
  }
  auto grow = [&](int &v, int cap, int bytes) {
    while (v < cap && zs * zb + ps * pb + bytes <= avail) ++v;
  };
  grow(ps, 6, pb);
  grow(zs, std::min(4, zcap), zb);
  grow(ps, kMaxPkStages, pb);
  grow(zs, zcap, zb);
  L.z_stages = zs;
  L.pk_stages = ps;
  L.smem_bytes = fixed + zs * zb + ps * pb;
  // one CTA per SM: the kernel holds all 512 TMEM columns
  L.smem_bytes = std::max(L.smem_bytes, smem_optin / 2 + 1024);
  L.smem_bytes = std::min(L.smem_bytes, smem_optin);
  *out = L;
  return true;
}

int build_items(const std::vector<ProbWork> &probs, int grid, std::vector<XItem> &items,
                std::vector<int> &cta_first, int min_split_pk, int max_item_pk) {
  items.clear();
  cta_first.clear();
  // Cost model, in operand-row chunks: unpacking one 64-sample chunk of one
  // operand row costs 1; the fold of a unit costs kFold per accumulator
  // column (its int64 atomic adds and the TMEM drain).
  constexpr long long kFold = 16;
  struct PW {
    int cpb, ppb, npk, nseg;  // nseg: fold-window segments of a unit's stages
  };
  if (max_item_pk < 1) max_item_pk = 1;
  std::vector<PW> pw(probs.size());
  long long total = 0;
  for (size_t p = 0; p < probs.size(); ++p) {
    const ProbWork &pr = probs[p];
    pw[p].cpb = (pr.block_len + kChunkSamples - 1) / kChunkSamples;
    pw[p].ppb = (pr.block_len + kPkSamples - 1) / kPkSamples;
    pw[p].npk = pw[p].ppb * pr.n_blocks;
    pw[p].nseg = (pw[p].npk + max_item_pk - 1) / max_item_pk;
    for (const XUnit &u : *pr.units)
      total += (long long)((pr.n_chan + u.n_chan - 1) / u.n_chan) *
               ((long long)pw[p].cpb * pr.n_blocks * u.z_rows + kFold * u.work * pw[p].nseg);
  }
  if (total == 0 || grid <= 0) {
    cta_first.push_back(0);
    return 0;
  }
  // cost of stages [a, b) of a unit with z_rows rows
  auto range_cost = [&](size_t p, int a, int b, int z_rows) {
    long long chunks = 0;
    for (int k = a; k < b; ++k) {
      const int kc = k % pw[p].ppb;
      chunks += std::min(kChunksPerPk, pw[p].cpb - kChunksPerPk * kc);
    }
    return chunks * z_rows;
  };
  long long remaining = total, load = 0;
  int cta = 0;
  long long target = (remaining + grid - 1) / grid;
  cta_first.push_back(0);
  auto close_cta = [&]() {
    remaining -= load;
    load = 0;
    ++cta;
    cta_first.push_back((int)items.size());
    if (cta < grid) target = (remaining + (grid - cta) - 1) / (grid - cta);
  };
  // deals the stages [pk, npk) of unit (p, t, c) over the CTAs
  auto deal = [&](size_t p, int t, int c, int pk, int npk) {
    const XUnit &u = (*probs[p].units)[t];
    const long long fold = kFold * u.work;
    while (pk < npk) {
      if (cta == grid - 1) {  // the last CTA takes everything left
        const long long cost = range_cost(p, pk, npk, u.z_rows) + fold;
        items.push_back({(int)p, t, c, pk, npk - pk});
        load += cost;
        pk = npk;
        continue;
      }
      const long long rest = range_cost(p, pk, npk, u.z_rows) + fold;
      if (load + rest <= target) {
        items.push_back({(int)p, t, c, pk, npk - pk});
        load += rest;
        pk = npk;
        if (load >= target) close_cta();
        continue;
      }
      // the rest overflows this CTA: take the stages that fit, if that
      // leaves pieces of at least min_split_pk stages on both sides
      int n = 0;
      const long long room = target - load - fold;
      if (room > 0) {
        const long long per = (long long)kChunksPerPk * u.z_rows;
        n = (int)std::min<long long>(npk - pk, room / per);
        while (n > 0 && range_cost(p, pk, pk + n, u.z_rows) > room) --n;
      }
      if (n >= min_split_pk && npk - pk - n >= min_split_pk) {
        items.push_back({(int)p, t, c, pk, n});
        load += range_cost(p, pk, pk + n, u.z_rows) + fold;
        remaining += fold;  // the rest of the unit is folded once more
        pk += n;
        close_cta();
      } else if (load == 0 || 2 * (load + rest - target) < rest) {
        // no useful split: the whole rest goes here when this CTA is
        // empty or when most of the rest fits
        items.push_back({(int)p, t, c, pk, npk - pk});
        load += rest;
        pk = npk;
        close_cta();
      } else {
        close_cta();
      }
    }
  };
  for (size_t p = 0; p < probs.size(); ++p) {
    const long long npk_total = pw[p].npk;
    const int nseg = pw[p].nseg;
    for (int t = 0; t < (int)probs[p].units->size(); ++t)
      for (int c = 0; c < probs[p].n_chan; c += std::max(1, (*probs[p].units)[t].n_chan))
        // fold-window segment sg: stages [npk sg / nseg, npk (sg + 1) / nseg)
        for (int sg = 0; sg < nseg; ++sg)
          deal(p, t, c, (int)(npk_total * sg / nseg), (int)(npk_total * (sg + 1) / nseg));
  }
  if (load > 0 || (int)cta_first.size() == 1) close_cta();
  // drop trailing empty CTAs
  while (cta_first.size() > 2 && cta_first[cta_first.size() - 2] == cta_first.back())
    cta_first.pop_back();
  return (int)cta_first.size() - 1;
}

namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn get_encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

}  // namespace

bool encode_block_map(const void *base, int block_len, int n_in, int n_chan, int pitch, void *map,
                      int ch_rows) {
  static_assert(sizeof(CUtensorMap) == 128, "tensor map size");
  EncodeTiledFn enc = get_encode_fn();
  if (!enc) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)block_len, (cuuint64_t)n_in, (cuuint64_t)n_chan};
  const cuuint64_t strides[2] = {(cuuint64_t)pitch, (cuuint64_t)pitch * (cuuint64_t)n_in};
  if (ch_rows != 16 && ch_rows != 32 && ch_rows != kTileInputs) return false;
  const cuuint32_t box[3] = {(cuuint32_t)kPkSamples, (cuuint32_t)ch_rows,
                             (cuuint32_t)(kTileInputs / ch_rows)};
  const cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(static_cast<CUtensorMap *>(map), CU_TENSOR_MAP_DATA_TYPE_UINT8, 3,
                   const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

bool encode_block_map_tcn(const void *base, int block_len, int n_in, int n_chan, void *map,
                          int ch_rows) {
  EncodeTiledFn enc = get_encode_fn();
  if (!enc || n_in % 16 != 0) return false;
  if (ch_rows != 16 && ch_rows != 32 && ch_rows != kTileInputs) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)n_in, (cuuint64_t)n_chan, (cuuint64_t)block_len};
  const cuuint64_t strides[2] = {(cuuint64_t)n_in, (cuuint64_t)n_in * (cuuint64_t)n_chan};
  // ch_rows inputs of 64 / ch_rows channels: each sample of the box is still
  // 64 bytes, channel-major, as the tile's rows are
  const cuuint32_t box[3] = {(cuuint32_t)ch_rows, (cuuint32_t)(kTileInputs / ch_rows),
                             (cuuint32_t)kPkSamples};
  const cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(static_cast<CUtensorMap *>(map), CU_TENSOR_MAP_DATA_TYPE_UINT8, 3,
                   const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace xe
