// xe_sched.h -- host-side scheduling of the CMAC kernel: the cover of the lower
// triangle by MMA tiles (templates) and the split of a launch's work into
// per-CTA runs of items of about equal cost.  Not part of the public ABI.
#pragma once
#include <cstdint>
#include <vector>

#include "xe_internal.h"

namespace xe {

// Cover variants of the triangle (the autotuner chooses between them).
enum Cover {
  // N <= 256: one staged window of all inputs per unit; the row tiles'
  // strips are packed first-fit into units of <= 512 TMEM columns.
  kCoverWindow = 0,
  // N <= 256: one unit per row tile t, staging inputs [0, 64 (t + 1)) only.
  kCoverStrips = 1,
  // any N: pairs of row tiles against 256-column pieces of their strip
  // (the only one-CTA cover for N > 256).
  kCoverPairs = 2,
  // N > 256, CTA pairs: blocks of 256 rows (four row tiles, two per CTA)
  // against 256-column pieces of their strip, each piece's B rows split
  // between the two CTAs (units with pair_rows = kPairRows).
  kCoverQuads = 3,
};

// Templates of the cover, heaviest first.  kCoverWindow and kCoverStrips
// fall back to kCoverPairs above 256 inputs.
std::vector<XUnit> build_schedule(int n_in, int cover = kCoverWindow);

// Shared-memory layout of a launch whose units are `units`.
struct StageLayout {
  int z_stages, pk_stages;
  uint32_t z_stage_bytes, pk_stage_bytes;
  int smem_bytes;
};
// Largest z_stages (<= max_z, >= 2) and pk_stages (3 if it leaves >= 2
// operand stages, else 2) that fit `smem_optin`.  Returns false if not even
// 2 + 2 stages fit.
bool stage_layout(const std::vector<const std::vector<XUnit> *> &unit_sets, int smem_optin,
                  int max_z, StageLayout *out);

// One problem as the item builder sees it.
struct ProbWork {
  const std::vector<XUnit> *units;
  int n_chan;
  int block_len;
  int n_blocks;  // blocks in the launch
};

// Packed stages one item may integrate before its fold: 1023 stages are at
// most 130944 samples, so every fp32 partial stays an integer below 2^24
// (128 per sample at most).
constexpr int kMaxFoldStages = 131071 / kPkSamples;

// Cuts every unit (problem, template, channel) into items and deals
// contiguous runs of them to at most `grid` CTAs.  Each CTA receives about
// the same modelled cost: the unpack work (operand rows x chunks) of its
// items plus a fixed fold cost per item.  A unit is split only at 128-sample
// stage boundaries and only into pieces of at least min_split_pk stages;
// first it is cut into equal segments of at most max_item_pk stages (the
// fold window), which every item stays inside.
// Fills items and cta_first (size used_grid + 1) and returns used_grid.
int build_items(const std::vector<ProbWork> &probs, int grid, std::vector<XItem> &items,
                std::vector<int> &cta_first, int min_split_pk = 16,
                int max_item_pk = kMaxFoldStages);

// The TMA descriptor of one block, uint8 [n_chan][n_in][row pitch], 3-D
// (time, input, channel) with boxes of 128 samples x ch_rows inputs x
// 64 / ch_rows channels (64 rows in all), 128B-swizzled.  ch_rows is 64
// except for schedules whose tiles hold several channels (16 or 32, see
// XSeg::ch_rows and tile_ch_rows).  `map` receives 128 bytes.  Returns false
// if the driver's encoder is unavailable or rejects the arguments.
bool encode_block_map(const void *base, int block_len, int n_in, int n_chan, int pitch, void *map,
                      int ch_rows = kTileInputs);

// Inputs per channel in a 64-row tile of a schedule's units: 16 or 32 when
// its tiles hold several channels, else 64.
int tile_ch_rows(const std::vector<XUnit> &units);

// The TMA descriptor of one block in F-engine order, uint8 [block_len][n_chan]
// [n_in], 3-D (input, channel, time) with 64-input x 1-channel x 128-sample
// boxes, no swizzle (each box lands as [128 samples][64 inputs]).  The
// channel and time strides must be multiples of 16 bytes: n_in % 16 == 0.
bool encode_block_map_tcn(const void *base, int block_len, int n_in, int n_chan, void *map,
                          int ch_rows = kTileInputs);

}  // namespace xe
