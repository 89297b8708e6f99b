// xe_internal.h -- structures shared by the host scheduler and the kernels.
// Not part of the public ABI (include/corr.h is).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace xe {

// Samples per pipeline chunk: one 128-byte operand row of fp8 (e5m2) values,
// two per sample (re, im), i.e. exactly one 128B-swizzle atom along K.
constexpr int kChunkSamples = 64;
// Inputs per row tile: the MMA A operand stacks 64 inputs' real-part rows and
// 64 inputs' imaginary-part rows (M = 128).
constexpr int kTileInputs = 64;
constexpr int kTmemCols = 512;
constexpr int kMaxSegs = 8;
constexpr int kMaxZRows = 512;
// Samples per TMA box row (one byte per complex sample): a packed stage holds
// kPkSamples samples of every staged input and feeds kPkSamples /
// kChunkSamples operand chunks.
constexpr int kPkSamples = 128;
constexpr int kPackedRowBytes = kPkSamples;
constexpr int kChunksPerPk = kPkSamples / kChunkSamples;
// Warp roles (see xengine.cu): unpack, epilogue (one per TMEM lane quarter),
// TMA producer, MMA issuers (one issue stream per accumulator).
constexpr int kUnpackWarps = 16;
constexpr int kEpiWarps = 4;
constexpr int kMmaWarps = 4;
constexpr int kWarpEpi0 = kUnpackWarps;
constexpr int kWarpTma = kWarpEpi0 + kEpiWarps;
constexpr int kWarpMma0 = kWarpTma + 1;
constexpr int kThreads = 32 * (kWarpMma0 + kMmaWarps);
// Largest region the unpack stages: each thread takes at most two rows of a
// region per chunk (rows row0 and row0 + 8 kUnpackWarps).
constexpr int kMaxRegionInputs = 2 * 8 * kUnpackWarps;
// Pipeline depth limits and the shared-memory area for the barriers (full and
// empty barrier per stage, accumulator full/empty, one drain barrier per MMA
// issuer) and the TMEM address / abort flag behind them.
constexpr int kMaxPkStages = 8;
constexpr int kMaxZStages = 6;
constexpr int kBarrierBytes = 512;
// Blocks integrated by one launch before the fold into int64.
constexpr int kMaxBlocksPerLaunch = 8;

// A contiguous range of inputs staged into the operand buffer ("Z") every
// chunk.  Interleaved regions store, per group of 8 inputs, 8 rows of
// [re, im] pairs (the "A rows") followed by 8 rows of [im, -re] pairs (the
// "Q rows"); plain regions store A rows only.
struct XRegion {
  int in_lo;        // first input
  int in_lo1;       // first input on the odd CTA of a pair (unused otherwise)
  int n_in;         // inputs staged (multiple of 64; rows past N read as zero)
  // 1: A and Q rows; 2: the interleaved layout with only the A rows written
  // (inputs that are only columns of the unit, next to interleaved rows, so
  // that one B operand spans both); 0: A rows only, packed (plain)
  int interleaved;
  int z_row;        // first row in the Z stage buffer (multiple of 8)
  int pk_off;       // byte offset in the packed stage buffer
  int chan_off;     // channel: the item's first channel + chan_off
};

// One MMA stream of the unit: D[128 x n] += A(tile) * B(cols)^T into TMEM.
struct XSeg {
  int a_zrow;    // Z row of the 128-row A operand (64 inputs, interleaved)
  int b_zrow;    // Z row of the first B row
  int b_sbo;     // byte stride between 8-row groups of B (2048 interleaved, 1024 plain)
  int n;         // B rows = output columns (multiple of 16, <= 256)
  int tmem_col;  // first TMEM column of the accumulator
  int row_in0;   // input index of the tile's first row
  int row_in1;   // the same on the odd CTA of a pair (unused otherwise)
  // input index of the first column of each 64-column block of the
  // accumulator (column c holds input col_blk[c / 64] + c % 64); one block
  // per 64 B rows, in the order the B operand takes them
  int col_blk[4];
  int chan_off;  // channel: the item's first channel + chan_off
  // 0: the tile's rows and columns are inputs of one channel.  Otherwise the
  // 64-row tile holds 64 / ch_rows channels of ch_rows inputs each (row and
  // column r: channel chan_off + r / ch_rows, input r % ch_rows); only the
  // diagonal blocks are folded
  int ch_rows;
};

struct XUnit {
  int n_reg, n_seg;
  int n_chan;    // channels one unit covers (its regions and segments name the offsets)
  // 0: one CTA runs the unit.  kPairRows: a CTA pair runs it with M = 256
  // MMAs; both CTAs stage the same layout of regions, the odd CTA from its
  // regions' in_lo1 and owning its segments' rows from row_in1; a segment's
  // column blocks are shared, since the pair's B operand is the even CTA's
  // N / 2 B rows followed by the odd one's
  int pair_rows;
  int z_rows;    // rows staged per chunk (sum over regions)
  int pk_bytes;  // packed bytes per chunk (sum over regions)
  int work;      // relative MMA work (sum of n), for ordering
  XRegion reg[2];
  XSeg seg[kMaxSegs];
};

// One correlator problem of a launch: its inputs, schedule and integration
// buffer.  A launch may carry several independent problems (a batch).
struct XProb {
  const XUnit *units;    // [n_tpl] templates
  int64_t *acc;          // [n_chan][n_pairs][2]
  long long n_pairs;     // N(N+1)/2
  int n_in;
  int n_chan;            // channels (a unit's channel past the last is skipped)
  int chunks_per_block;  // ceil(block_len / kChunkSamples)
  int pk_per_block;      // ceil(block_len / kPkSamples)
  int map0;              // the problem's first block map in the launch's map table
};

// One piece of work: template `tpl` of problem `prob` on channel `chan`,
// over packed stages [pk0, pk0 + npk) of the launch's blocks (stage k is
// stage k % pk_per_block of block k / pk_per_block).  A unit (problem,
// template, channel) may be split over several items, each folded on its
// own: the int64 fold is an atomic add, so the pieces sum exactly.
struct XItem {
  int prob, tpl, chan, pk0, npk;
};

// Inputs per CTA of a pair unit: two row tiles, and half of a 256-column
// B operand.
constexpr int kPairRows = 128;
// A pair unit has two segments (one per row tile of each CTA), each with
// its own issuing thread on the even CTA.
constexpr int kPairIssuers = 2;

// Bits of the device status word.
constexpr int kStatusTimeout = 1;  // a bounded wait ran out
constexpr int kStatusBounds = 2;   // debug builds: an address check or a guard band failed

// Atomic add into an int64 integration buffer of `elems` elements.  Debug
// builds (CORR_DEBUG) check the address first: one outside the buffer sets
// kStatusBounds and the add is skipped.  Release builds add unchecked.
__device__ __forceinline__ void acc_add(int64_t *base, long long elems, int *status, int64_t *ptr,
                                        long long v) {
#ifdef CORR_DEBUG
  const long long off = ptr - base;
  if (off < 0 || off >= elems) {
    atomicOr(status, kStatusBounds);
    return;
  }
#else
  (void)base;
  (void)elems;
  (void)status;
#endif
  asm volatile("red.global.add.u64 [%0], %1;" ::"l"(ptr), "l"((unsigned long long)v) : "memory");
}

struct XParams {
  const XProb *probs;
  // Explicit items: CTA b runs items [cta_first[b], cta_first[b + 1]).
  // With items == nullptr the launch holds problem 0 alone and CTA b runs the
  // whole units b, b + grid, ... of its n_tpl x n_chan units (unit w is
  // template w / n_chan on channel w % n_chan) over all npk stages.
  const XItem *items;
  const int *cta_first;
  int implicit_n_tpl, implicit_n_chan, implicit_npk;
  int *status;           // device status word (kStatusTimeout | kStatusBounds)
  unsigned long long timeout_ns;
  int z_stages, pk_stages;
  uint32_t z_stage_bytes, pk_stage_bytes;
  int selftest_never;  // failure-detection self-test (see corr_selftest_timeout)
  // 1: the blocks are in F-engine order, uint8 [time][channel][input], and
  // their maps are 3-D (input, channel, time) with 64-input x 128-sample
  // boxes (no swizzle); the unpack transposes them on chip, and operand rows
  // are rotated within every 8-input group (see xengine.cu)
  int tcn;
};

// TMA descriptors (CUtensorMap, 128 bytes each), one per (problem, block) of
// the launch, passed as a kernel parameter.
constexpr int kMaxMaps = 8;        // one problem, up to kMaxBlocksPerLaunch blocks
constexpr int kMaxBatchMaps = 128; // a batch: one block per problem
template <int M>
struct XMapsT {
  alignas(64) unsigned char m[M][128];
};
using XMaps = XMapsT<kMaxMaps>;
using XBatchMaps = XMapsT<kMaxBatchMaps>;

// Geometry of the TMEM-operand kernel (xengine_tm.cu) for one problem of
// n_in <= kTmMaxInputs inputs: one window unit of n_rt row tiles.  Row tile 0
// (inputs 0..63) reads its row operand from a TMEM ring of 32-column slots
// from column a_base; tiles 1 and 2 read theirs from shared memory.  Tile t
// has nt[t] columns and its accumulator at TMEM column acc[t] (the largest
// tile first).  The shared-memory operand stage holds, in units of 64 rows of
// 128 bytes (Q = [b, -a] rows, A = [a, b] rows):
//   n_rt = 1:  A(0..63)
//   n_rt = 2:  Q(64..127) A(64..127) A(0..63)
//   n_rt = 3:  Q(64..127) A(64..127) A(0..63) A(128..191) Q(128..191)
// so tile 1's row operand is [Q; A] of its inputs, tile 2's [A; Q], and the
// column operands of tiles 0, 1, 2 are the contiguous row ranges A(0..63),
// A(64..127) A(0..63) and A(64..127) A(0..63) A(128..191): one MMA per tile
// per K slice.  Column n of tiles 1 and 2 is input 64 + n for n < 64, n - 64
// for 64 <= n < 128, n above.
constexpr int kTmMaxInputs = 3 * kTileInputs;
struct TmGeom {
  int n_rt, n16;
  int nt[3], acc[3];
  int acc_cols, a_base;
  int z_rows, row_q1, row_a1, row_a0, row_a2, row_q2;  // operand-stage rows
};
__host__ __device__ inline TmGeom tm_geom(int n_in) {
  TmGeom g;
  g.n16 = (n_in + 15) / 16 * 16;
  g.n_rt = (n_in + kTileInputs - 1) / kTileInputs;
  g.nt[0] = g.n16 < kTileInputs ? g.n16 : kTileInputs;
  g.nt[1] = g.n_rt >= 2 ? 2 * kTileInputs : 0;
  g.nt[2] = g.n_rt >= 3 ? g.n16 : 0;
  g.acc[2] = 0;
  g.acc[1] = g.nt[2];
  g.acc[0] = g.nt[2] + g.nt[1];
  g.acc_cols = g.acc[0] + g.nt[0];
  g.a_base = (g.acc_cols + 31) / 32 * 32;
  const int T = kTileInputs;
  if (g.n_rt == 1) {
    g.row_a0 = 0;
    g.row_q1 = g.row_a1 = g.row_a2 = g.row_q2 = 0;
    g.z_rows = T;
  } else {
    g.row_q1 = 0;
    g.row_a1 = T;
    g.row_a0 = 2 * T;
    g.row_a2 = 3 * T;
    g.row_q2 = 4 * T;
    g.z_rows = g.n_rt == 2 ? 3 * T : 5 * T;
  }
  return g;
}
// TMEM columns of one ring slot: row tile 0's operand for one 64-sample chunk.
constexpr int kTmSlotCols = 32;

// Host-side launchers (defined in the .cu files).
cudaError_t launch_cmac(const XMaps &maps, const XParams &p, int grid, int smem_bytes,
                        cudaStream_t stream);
cudaError_t launch_cmac_batch(const XBatchMaps &maps, const XParams &p, int grid, int smem_bytes,
                              cudaStream_t stream);
cudaError_t cmac_set_smem(int smem_bytes);
// The CTA-pair instance for units with pair_rows != 0: `clusters` clusters
// of two CTAs, cluster w running items [cta_first[w], cta_first[w + 1]).
cudaError_t launch_cmac_pair(const XMaps &maps, const XParams &p, int clusters, int smem_bytes,
                             cudaStream_t stream);
// Clusters of two CTAs of the pair instance that can be resident at once
// (0 if the query fails).
int cmac_pair_clusters(int smem_bytes);
cudaError_t launch_cmac_tm(const XMaps &maps, const XParams &p, int grid, int smem_bytes,
                           cudaStream_t stream);
cudaError_t cmac_tm_set_smem(int smem_bytes);
// status: the owner's device status word (debug builds set kStatusBounds on a
// failed address check; release builds ignore it).
cudaError_t launch_dump(int64_t *acc, int64_t *vis, int64_t *stokes, int n_ant, int n_pol,
                        int n_chan, cudaStream_t stream, int grid, int *status);
// Debug builds: checks that the guard bands of `bytes` before and after a
// buffer still hold kGuardByte, else sets kStatusBounds.
constexpr unsigned char kGuardByte = 0xA5;
constexpr size_t kGuardBytes = 4096;
cudaError_t launch_guard_check(const unsigned char *before, const unsigned char *after,
                               size_t bytes, int *status, cudaStream_t stream);
cudaError_t launch_pitch(const uint8_t *src, uint8_t *dst, long long rows, int T, int pitch,
                         cudaStream_t stream, int grid);
cudaError_t launch_corner_turn(const uint8_t *src, uint8_t *dst, int n_in, int n_chan,
                               int block_len, int dst_pitch, cudaStream_t stream, int grid);

}  // namespace xe
