// corr.cu -- the C ABI declared in include/corr.h: context, schedule of the
// lower-triangle tiles, TMA descriptors and launches.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "corr.h"
#include "xe_sched.h"
#include "xe_internal.h"
#include "trace.h"

using xe::XParams;
using xe::XSeg;
using xe::XUnit;

// Device copy of a launch's item split (see sched.h), one per number of
// blocks per launch.
struct ItemPlan {
  xe::XItem *d_items;
  int *d_cta_first;
  int grid;
};

struct corr_ctx {
  int n_ant, n_pol, n_chan, block_len, n_in;
  long long n_pairs, n_apairs;
  int device, n_sm;
  int64_t *d_acc;
  unsigned char *acc_alloc;  // the allocation holding d_acc (with guard bands in debug builds)
  int *d_status;
  XUnit *d_units;
  xe::XProb *d_prob;
  int n_tpl;
  int per_launch;  // blocks per CMAC launch (<= kMaxBlocksPerLaunch)
  ItemPlan plans[xe::kMaxBlocksPerLaunch + 1];
  int smem_bytes, z_stages, pk_stages;
  uint32_t z_stage_bytes, pk_stage_bytes;
  int tm;  // 1: the TMEM-operand kernel (xengine_tm.cu) runs this context's launches
  int pair;  // 1: CTA pairs (the quad cover, M = 256 MMAs) run this context's launches
  int ch_rows;  // inputs per channel in the TMA box (64, or 16 / 32 for multi-channel tiles)
  int pitch;           // row pitch of the staged block (block_len rounded up to 16)
  uint8_t *d_pitched;  // [n_chan][n_in][pitch] when block_len % 16 != 0
  uint8_t *d_turned;   // [n_chan][n_in][pitch]: corner-turned blocks (allocated on first use)
  long long samples;        // samples per input in the integration in progress
  long long launches;
  long long blocks_pushed, samples_total, dumps;
  unsigned long long timeout_ns;
  // host-buffer variants
  uint8_t *d_stage[2];
  cudaEvent_t ev_free[2], ev_ready[2];
  cudaStream_t copy_stream;
  int next_slot;
  int64_t *d_vis_out, *d_stokes_out;
};

namespace {

#ifdef CORR_DEBUG
constexpr bool kDebug = true;
#else
constexpr bool kDebug = false;
#endif

int round_up(int v, int m) { return (v + m - 1) / m * m; }

int cuda_err(cudaError_t e) {
  if (e == cudaSuccess) return CORR_OK;
  if (e == cudaErrorMemoryAllocation) return CORR_ENOMEM;
  return CORR_ECUDA;
}

int encode_block_map(const corr_ctx *ctx, const void *base, CUtensorMap *m) {
  return xe::encode_block_map(base, ctx->block_len, ctx->n_in, ctx->n_chan, ctx->pitch, m,
                              ctx->ch_rows)
             ? CORR_OK
             : CORR_ECUDA;
}

int free_ctx(corr_ctx *ctx) {
  if (!ctx) return CORR_OK;
  cudaFree(ctx->acc_alloc);
  cudaFree(ctx->d_status);
  cudaFree(ctx->d_units);
  cudaFree(ctx->d_prob);
  for (auto &pl : ctx->plans) {
    cudaFree(pl.d_items);
    cudaFree(pl.d_cta_first);
  }
  cudaFree(ctx->d_pitched);
  cudaFree(ctx->d_turned);
  for (int k = 0; k < 2; ++k) {
    cudaFree(ctx->d_stage[k]);
    if (ctx->ev_free[k]) cudaEventDestroy(ctx->ev_free[k]);
    if (ctx->ev_ready[k]) cudaEventDestroy(ctx->ev_ready[k]);
  }
  if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
  cudaFree(ctx->d_vis_out);
  cudaFree(ctx->d_stokes_out);
  delete ctx;
  return CORR_OK;
}

// Whether the TMEM-operand kernel (xengine_tm.cu) runs a context of n_in
// inputs: only when CORR_CMAC_KERNEL=tm asks for it (up to three row tiles).
// The all-shared-memory kernel (xengine.cu) with two-channel units measured
// 1.25x faster at 80..128 inputs and the TMEM-operand kernel 9 % slower at
// 192 inputs.
bool use_tm_kernel(int n_in) {
  (void)n_in;
  const char *e = std::getenv("CORR_CMAC_KERNEL");
  return e && std::strcmp(e, "tm") == 0;
}

// Whether CTA pairs run a context of n_in inputs (more than 256 only).  The
// pair's shared B operand halves the inputs each SM unpacks per MMA, but on
// this part the pair kernel measured 5 % slower per issued MAC than one-CTA
// units at 512 to 2048 inputs, and its cover issues more padding on the
// diagonal: it runs only when CORR_CMAC_KERNEL=pair asks for it.
bool use_pair_kernel(int n_in) {
  if (n_in <= 256) return false;
  const char *e = std::getenv("CORR_CMAC_KERNEL");
  return e && std::strcmp(e, "pair") == 0;
}

// Shared-memory stages of the TMEM-operand kernel for n_in inputs: operand
// stages of G.z_rows rows (TmGeom), at most as many as the TMEM ring has
// slots, and packed stages of S = 64 n_rt rows of 128 bytes: three operand
// stages first, then packed stages up to eight, then operand stages while
// they fit.  Also returns the one window unit the item split models (its
// cost: operand rows written per chunk).  False above three row tiles or if
// two of each stage do not fit.
bool tm_stage_layout(int n_in, int smem_optin, xe::StageLayout *out, std::vector<XUnit> *units) {
  if (n_in > xe::kTmMaxInputs) return false;
  const xe::TmGeom G = xe::tm_geom(n_in);
  const int n_st = xe::kTileInputs * G.n_rt;
  const int zb = G.z_rows * 128, pb = n_st * xe::kPackedRowBytes;
  const int zmax = std::min(xe::kMaxZStages, (xe::kTmemCols - G.a_base) / xe::kTmSlotCols);
  const int avail = smem_optin - 1024 - xe::kBarrierBytes;
  if (zmax < 2 || 2 * zb + 2 * pb > avail) return false;
  int zs = std::min(zmax, 3);
  while (zs > 2 && zs * zb + 2 * pb > avail) --zs;
  const int ps = std::min(xe::kMaxPkStages, (avail - zs * zb) / pb);
  while (zs < zmax && (zs + 1) * zb + ps * pb <= avail) ++zs;
  xe::StageLayout L;
  L.z_stages = zs;
  L.pk_stages = ps;
  L.z_stage_bytes = (uint32_t)zb;
  L.pk_stage_bytes = (uint32_t)pb;
  L.smem_bytes = 1024 + xe::kBarrierBytes + zs * zb + ps * pb;
  // one CTA per SM: the kernel holds all 512 TMEM columns
  L.smem_bytes = std::min(std::max(L.smem_bytes, smem_optin / 2 + 1024), smem_optin);
  *out = L;
  XUnit u;
  std::memset(&u, 0, sizeof(u));
  u.n_chan = 1;
  u.z_rows = 2 * n_st;
  u.work = G.acc_cols;
  units->assign(1, u);
  return true;
}

size_t block_bytes(const corr_ctx *c) {
  return (size_t)c->n_chan * (size_t)c->n_in * (size_t)c->block_len;
}

}  // namespace

extern "C" {

const char *corr_strerror(int code) {
  switch (code) {
    case CORR_OK: return "ok";
    case CORR_EINVAL: return "invalid argument";
    case CORR_ENOMEM: return "out of memory";
    case CORR_ECUDA: return "CUDA call failed";
    case CORR_EARCH: return "device is not compute capability 10.3 (sm_103)";
    case CORR_ETIMEOUT: return "a device-side wait timed out";
    case CORR_ESTATE: return "call not valid in the current state";
    case CORR_EBOUNDS: return "an address check or a guard band failed (debug build)";
    default: return "unknown error";
  }
}

int corr_create(int n_ant, int n_pol, int n_chan, int block_len, corr_ctx **out) {
  CORR_TRACE("corr_create");
  if (!out) return CORR_EINVAL;
  *out = nullptr;
  if (n_ant <= 0 || n_chan <= 0 || block_len <= 0 || (n_pol != 1 && n_pol != 2))
    return CORR_EINVAL;
  if (block_len > CORR_MAX_BLOCK_LEN) return CORR_EINVAL;
  if ((long long)n_ant * n_pol > CORR_MAX_INPUTS) return CORR_EINVAL;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return CORR_ECUDA;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return CORR_ECUDA;
  if (prop.major != 10 || prop.minor != 3) return CORR_EARCH;
  int smem_optin = 0;
  if (cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
      cudaSuccess)
    return CORR_ECUDA;

  corr_ctx *ctx = new (std::nothrow) corr_ctx;
  if (!ctx) return CORR_ENOMEM;
  std::memset(ctx, 0, sizeof(*ctx));
  ctx->n_ant = n_ant;
  ctx->n_pol = n_pol;
  ctx->n_chan = n_chan;
  ctx->block_len = block_len;
  ctx->n_in = n_ant * n_pol;
  ctx->n_pairs = (long long)ctx->n_in * (ctx->n_in + 1) / 2;
  ctx->n_apairs = (long long)n_ant * (n_ant + 1) / 2;
  ctx->device = dev;
  ctx->n_sm = prop.multiProcessorCount;
  ctx->pitch = round_up(block_len, 16);
  ctx->timeout_ns = 2000000000ull;
  if (const char *s = std::getenv("CORR_TIMEOUT_MS")) {
    long long ms = std::atoll(s);
    if (ms > 0) ctx->timeout_ns = (unsigned long long)ms * 1000000ull;
  }

  ctx->pair = use_pair_kernel(ctx->n_in) ? 1 : 0;
  std::vector<XUnit> units =
      xe::build_schedule(ctx->n_in, ctx->pair ? xe::kCoverQuads : xe::kCoverWindow);
  if (units.empty()) {
    free_ctx(ctx);
    return CORR_EINVAL;
  }
  ctx->n_tpl = (int)units.size();
  xe::StageLayout L;
  if (!xe::stage_layout({&units}, smem_optin, xe::kMaxZStages, &L)) {
    free_ctx(ctx);
    return CORR_EINVAL;
  }
  ctx->z_stages = L.z_stages;
  ctx->pk_stages = L.pk_stages;
  ctx->z_stage_bytes = L.z_stage_bytes;
  ctx->pk_stage_bytes = L.pk_stage_bytes;
  ctx->smem_bytes = L.smem_bytes;
  // the TMEM-operand kernel where it is the faster one (up to three row
  // tiles); the item split then models its one window unit
  std::vector<XUnit> tm_units;
  xe::StageLayout TL;
  if (use_tm_kernel(ctx->n_in) && tm_stage_layout(ctx->n_in, smem_optin, &TL, &tm_units)) {
    ctx->tm = 1;
    ctx->z_stages = TL.z_stages;
    ctx->pk_stages = TL.pk_stages;
    ctx->z_stage_bytes = TL.z_stage_bytes;
    ctx->pk_stage_bytes = TL.pk_stage_bytes;
    ctx->smem_bytes = TL.smem_bytes;
  }
  const std::vector<XUnit> &plan_units = ctx->tm ? tm_units : units;
  ctx->ch_rows = ctx->tm ? xe::kTileInputs : xe::tile_ch_rows(units);
  // a fold must come before 2^24 / 128 samples have been accumulated in
  // fp32: launches of several blocks stay within that window, and the item
  // split cuts a longer block into pieces that each fold on their own
  ctx->per_launch = std::max(1, std::min(xe::kMaxBlocksPerLaunch, CORR_FOLD_SAMPLES / block_len));
  if (ctx->pitch != block_len) ctx->per_launch = 1;  // one pitched staging buffer

  int rc = CORR_OK;
  const size_t acc_bytes = (size_t)n_chan * (size_t)ctx->n_pairs * 16;
  // debug builds put a guard band of kGuardBytes on each side of the
  // integration buffer; corr_check verifies them
  const size_t guard = kDebug ? xe::kGuardBytes : 0;
  if ((rc = cuda_err(cudaMalloc(&ctx->acc_alloc, acc_bytes + 2 * guard))) != CORR_OK ||
      (rc = cuda_err(cudaMalloc(&ctx->d_status, sizeof(int)))) != CORR_OK ||
      (rc = cuda_err(cudaMalloc(&ctx->d_units, units.size() * sizeof(XUnit)))) != CORR_OK) {
    free_ctx(ctx);
    return rc;
  }
  ctx->d_acc = reinterpret_cast<int64_t *>(ctx->acc_alloc + guard);
  if (guard && ((rc = cuda_err(cudaMemset(ctx->acc_alloc, xe::kGuardByte, guard))) != CORR_OK ||
                (rc = cuda_err(cudaMemset(ctx->acc_alloc + guard + acc_bytes, xe::kGuardByte,
                                          guard))) != CORR_OK)) {
    free_ctx(ctx);
    return rc;
  }
  if (ctx->pitch != block_len) {
    if ((rc = cuda_err(cudaMalloc(&ctx->d_pitched, (size_t)n_chan * ctx->n_in * ctx->pitch))) !=
        CORR_OK) {
      free_ctx(ctx);
      return rc;
    }
  }
  // the problem descriptor and the balanced item split for every launch size
  xe::XProb prob;
  prob.units = ctx->d_units;
  prob.acc = ctx->d_acc;
  prob.n_pairs = ctx->n_pairs;
  prob.n_in = ctx->n_in;
  prob.n_chan = n_chan;
  prob.chunks_per_block = (block_len + xe::kChunkSamples - 1) / xe::kChunkSamples;
  prob.pk_per_block = (block_len + xe::kPkSamples - 1) / xe::kPkSamples;
  prob.map0 = 0;
  if ((rc = cuda_err(cudaMalloc(&ctx->d_prob, sizeof(prob)))) != CORR_OK ||
      (rc = cuda_err(cudaMemcpy(ctx->d_prob, &prob, sizeof(prob), cudaMemcpyHostToDevice))) !=
          CORR_OK) {
    free_ctx(ctx);
    return rc;
  }
  // workers: CTAs, or for CTA pairs the clusters that fit at once
  int workers = ctx->n_sm;
  if (ctx->pair) {
    if ((rc = cuda_err(xe::cmac_set_smem(smem_optin))) != CORR_OK) {
      free_ctx(ctx);
      return rc;
    }
    workers = std::min(ctx->n_sm / 2, xe::cmac_pair_clusters(ctx->smem_bytes));
    if (workers < 1) {
      free_ctx(ctx);
      return CORR_ECUDA;
    }
  }
  for (int nb = 1; nb <= ctx->per_launch; ++nb) {
    std::vector<xe::XItem> items;
    std::vector<int> first;
    ItemPlan &pl = ctx->plans[nb];
    pl.grid = xe::build_items({{&plan_units, n_chan, block_len, nb}}, workers, items, first);
    if ((rc = cuda_err(cudaMalloc(&pl.d_items, items.size() * sizeof(xe::XItem)))) != CORR_OK ||
        (rc = cuda_err(cudaMalloc(&pl.d_cta_first, first.size() * sizeof(int)))) != CORR_OK ||
        (rc = cuda_err(cudaMemcpy(pl.d_items, items.data(), items.size() * sizeof(xe::XItem),
                                  cudaMemcpyHostToDevice))) != CORR_OK ||
        (rc = cuda_err(cudaMemcpy(pl.d_cta_first, first.data(), first.size() * sizeof(int),
                                  cudaMemcpyHostToDevice))) != CORR_OK) {
      free_ctx(ctx);
      return rc;
    }
  }
  if ((rc = cuda_err(cudaMemset(ctx->d_acc, 0, acc_bytes))) != CORR_OK ||
      (rc = cuda_err(cudaMemset(ctx->d_status, 0, sizeof(int)))) != CORR_OK ||
      (rc = cuda_err(cudaMemcpy(ctx->d_units, units.data(), units.size() * sizeof(XUnit),
                                cudaMemcpyHostToDevice))) != CORR_OK ||
      (rc = cuda_err(xe::cmac_set_smem(smem_optin))) != CORR_OK ||
      (rc = cuda_err(xe::cmac_tm_set_smem(smem_optin))) != CORR_OK ||
      (rc = cuda_err(cudaDeviceSynchronize())) != CORR_OK) {
    free_ctx(ctx);
    return rc;
  }
  *out = ctx;
  return CORR_OK;
}

}  // extern "C"

namespace {

// One CMAC launch over nb (<= per_launch) blocks whose rows are already
// ctx->pitch bytes apart.  selftest_timeout_ns > 0 runs the failure-detection
// self-test instead (see corr_selftest_timeout).
int launch_staged(corr_ctx *ctx, const uint8_t *const *staged, int nb, cudaStream_t st,
                  unsigned long long selftest_timeout_ns = 0, bool tcn = false) {
  XParams p;
  std::memset(&p, 0, sizeof(p));
  p.probs = ctx->d_prob;
  p.status = ctx->d_status;
  p.timeout_ns = selftest_timeout_ns ? selftest_timeout_ns : ctx->timeout_ns;
  p.selftest_never = selftest_timeout_ns ? 1 : 0;
  p.z_stages = ctx->z_stages;
  p.pk_stages = ctx->pk_stages;
  p.z_stage_bytes = ctx->z_stage_bytes;
  p.pk_stage_bytes = ctx->pk_stage_bytes;
  xe::XMaps maps;
  std::memset(&maps, 0, sizeof(maps));
  int rc;
  p.tcn = tcn ? 1 : 0;
  for (int k = 0; k < nb; ++k) {
    if (tcn) {
      if (!xe::encode_block_map_tcn(staged[k], ctx->block_len, ctx->n_in, ctx->n_chan, maps.m[k],
                                    ctx->ch_rows))
        return CORR_ECUDA;
    } else if ((rc = encode_block_map(ctx, staged[k], reinterpret_cast<CUtensorMap *>(maps.m[k]))) !=
               CORR_OK) {
      return rc;
    }
  }
  const ItemPlan &pl = ctx->plans[nb];
  p.items = pl.d_items;
  p.cta_first = pl.d_cta_first;
  if ((rc = cuda_err(ctx->tm     ? xe::launch_cmac_tm(maps, p, pl.grid, ctx->smem_bytes, st)
                     : ctx->pair ? xe::launch_cmac_pair(maps, p, pl.grid, ctx->smem_bytes, st)
                                 : xe::launch_cmac(maps, p, pl.grid, ctx->smem_bytes, st))) !=
      CORR_OK)
    return rc;
  ctx->launches++;
  if (!selftest_timeout_ns) {
    ctx->samples += (long long)nb * ctx->block_len;
    ctx->samples_total += (long long)nb * ctx->block_len;
    ctx->blocks_pushed += nb;
  }
  return CORR_OK;
}

}  // namespace

extern "C" {

int corr_push_blocks(corr_ctx *ctx, const uint8_t *const *d_blocks, int n_blocks,
                     void *stream) {
  CORR_TRACE("corr_push_blocks");
  if (!ctx || !d_blocks || n_blocks <= 0) return CORR_EINVAL;
  for (int k = 0; k < n_blocks; ++k)
    if (!d_blocks[k] || (reinterpret_cast<uintptr_t>(d_blocks[k]) & 15u) != 0) return CORR_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  static_assert(sizeof(CUtensorMap) == sizeof(xe::XMaps::m[0]), "tensor map size");
  const int per = ctx->per_launch;
  int rc;
  for (int k0 = 0; k0 < n_blocks; k0 += per) {
    const int nb = std::min(per, n_blocks - k0);
    const uint8_t *staged[xe::kMaxBlocksPerLaunch];
    for (int k = 0; k < nb; ++k) {
      staged[k] = d_blocks[k0 + k];
      if (ctx->d_pitched) {
        if ((rc = cuda_err(xe::launch_pitch(staged[k], ctx->d_pitched,
                                            (long long)ctx->n_chan * ctx->n_in, ctx->block_len,
                                            ctx->pitch, st, ctx->n_sm * 8))) != CORR_OK)
          return rc;
        ctx->launches++;
        staged[k] = ctx->d_pitched;
      }
    }
    if ((rc = launch_staged(ctx, staged, nb, st)) != CORR_OK) return rc;
  }
  return CORR_OK;
}

int corr_corner_turn(const uint8_t *d_src, uint8_t *d_dst, int n_in, int n_chan, int block_len,
                     void *stream) {
  CORR_TRACE("corr_corner_turn");
  if (!d_src || !d_dst || n_in <= 0 || n_chan <= 0 || block_len <= 0) return CORR_EINVAL;
  if ((reinterpret_cast<uintptr_t>(d_src) & 3u) || (reinterpret_cast<uintptr_t>(d_dst) & 3u))
    return CORR_EINVAL;
  int dev = 0, n_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return CORR_ECUDA;
  return cuda_err(xe::launch_corner_turn(d_src, d_dst, n_in, n_chan, block_len, block_len,
                                         static_cast<cudaStream_t>(stream), n_sm * 8));
}

int corr_selftest_timeout(corr_ctx *ctx, const uint8_t *d_block, int timeout_ms, void *stream) {
  if (!ctx || !d_block || (reinterpret_cast<uintptr_t>(d_block) & 15u) || timeout_ms <= 0 ||
      timeout_ms > 10000)
    return CORR_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const uint8_t *staged = d_block;
  int rc;
  if (ctx->d_pitched) {
    if ((rc = cuda_err(xe::launch_pitch(d_block, ctx->d_pitched, (long long)ctx->n_chan * ctx->n_in,
                                        ctx->block_len, ctx->pitch, st, ctx->n_sm * 8))) !=
        CORR_OK)
      return rc;
    ctx->launches++;
    staged = ctx->d_pitched;
  }
  return launch_staged(ctx, &staged, 1, st, (unsigned long long)timeout_ms * 1000000ull);
}

int corr_push_block_tcn(corr_ctx *ctx, const uint8_t *d_src, void *stream) {
  CORR_TRACE("corr_push_block_tcn");
  if (!ctx || !d_src || (reinterpret_cast<uintptr_t>(d_src) & 3u)) return CORR_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // The shared-memory kernel stages F-engine-order blocks directly (TMA boxes
  // of [128 samples][64 inputs], transposed on chip) when the block's strides
  // allow a tensor map; otherwise the block is turned in HBM first.
  if (!ctx->tm && !ctx->pair && ctx->n_in % 16 == 0 &&
      (reinterpret_cast<uintptr_t>(d_src) & 15u) == 0)
    return launch_staged(ctx, &d_src, 1, st, 0, true);
  int rc;
  if (!ctx->d_turned &&
      (rc = cuda_err(cudaMalloc(&ctx->d_turned, (size_t)ctx->n_chan * ctx->n_in * ctx->pitch))) !=
          CORR_OK)
    return rc;
  if ((rc = cuda_err(xe::launch_corner_turn(d_src, ctx->d_turned, ctx->n_in, ctx->n_chan,
                                            ctx->block_len, ctx->pitch, st, ctx->n_sm * 8))) !=
      CORR_OK)
    return rc;
  ctx->launches++;
  const uint8_t *staged = ctx->d_turned;
  return launch_staged(ctx, &staged, 1, st);
}

int corr_push_block(corr_ctx *ctx, const uint8_t *d_block, void *stream) {
  if (!ctx || !d_block) return CORR_EINVAL;
  return corr_push_blocks(ctx, &d_block, 1, stream);
}

int corr_dump(corr_ctx *ctx, int64_t *d_vis, int64_t *d_stokes, void *stream) {
  CORR_TRACE("corr_dump");
  if (!ctx) return CORR_EINVAL;
  if (d_stokes && ctx->n_pol != 2) return CORR_EINVAL;
  if ((reinterpret_cast<uintptr_t>(d_vis) & 15u) || (reinterpret_cast<uintptr_t>(d_stokes) & 15u))
    return CORR_EINVAL;
  int rc = cuda_err(xe::launch_dump(ctx->d_acc, d_vis, d_stokes, ctx->n_ant, ctx->n_pol,
                                    ctx->n_chan, static_cast<cudaStream_t>(stream),
                                    ctx->n_sm * 8, ctx->d_status));
  if (rc != CORR_OK) return rc;
  ctx->launches++;
  ctx->dumps++;
  ctx->samples = 0;
  return CORR_OK;
}

int corr_push_block_host(corr_ctx *ctx, const uint8_t *h_block, void *stream) {
  CORR_TRACE("corr_push_block_host");
  if (!ctx || !h_block) return CORR_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t nb = block_bytes(ctx);
  int rc;
  if (!ctx->copy_stream) {
    if ((rc = cuda_err(cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking))) !=
        CORR_OK)
      return rc;
    for (int k = 0; k < 2; ++k) {
      if ((rc = cuda_err(cudaMalloc(&ctx->d_stage[k], nb))) != CORR_OK ||
          (rc = cuda_err(cudaEventCreateWithFlags(&ctx->ev_free[k], cudaEventDisableTiming))) !=
              CORR_OK ||
          (rc = cuda_err(cudaEventCreateWithFlags(&ctx->ev_ready[k], cudaEventDisableTiming))) !=
              CORR_OK)
        return rc;
    }
  }
  const int k = ctx->next_slot;
  ctx->next_slot ^= 1;
  // the slot is free once the push that last read it has run
  if ((rc = cuda_err(cudaStreamWaitEvent(ctx->copy_stream, ctx->ev_free[k], 0))) != CORR_OK ||
      (rc = cuda_err(cudaMemcpyAsync(ctx->d_stage[k], h_block, nb, cudaMemcpyHostToDevice,
                                     ctx->copy_stream))) != CORR_OK ||
      (rc = cuda_err(cudaEventRecord(ctx->ev_ready[k], ctx->copy_stream))) != CORR_OK ||
      (rc = cuda_err(cudaStreamWaitEvent(st, ctx->ev_ready[k], 0))) != CORR_OK)
    return rc;
  if ((rc = corr_push_block(ctx, ctx->d_stage[k], stream)) != CORR_OK) return rc;
  if ((rc = cuda_err(cudaEventRecord(ctx->ev_free[k], st))) != CORR_OK) return rc;
  // h_block may be reused once its copy is done
  return cuda_err(cudaEventSynchronize(ctx->ev_ready[k]));
}

int corr_dump_host(corr_ctx *ctx, int64_t *h_vis, int64_t *h_stokes, void *stream) {
  CORR_TRACE("corr_dump_host");
  if (!ctx) return CORR_EINVAL;
  if (h_stokes && ctx->n_pol != 2) return CORR_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t vis_bytes = (size_t)ctx->n_chan * ctx->n_pairs * 16;
  const size_t st_bytes = (size_t)ctx->n_chan * ctx->n_apairs * 64;
  int rc;
  if (h_vis && !ctx->d_vis_out && (rc = cuda_err(cudaMalloc(&ctx->d_vis_out, vis_bytes))) != CORR_OK)
    return rc;
  if (h_stokes && !ctx->d_stokes_out &&
      (rc = cuda_err(cudaMalloc(&ctx->d_stokes_out, st_bytes))) != CORR_OK)
    return rc;
  if ((rc = corr_dump(ctx, h_vis ? ctx->d_vis_out : nullptr, h_stokes ? ctx->d_stokes_out : nullptr,
                      stream)) != CORR_OK)
    return rc;
  if (h_vis && (rc = cuda_err(cudaMemcpyAsync(h_vis, ctx->d_vis_out, vis_bytes,
                                              cudaMemcpyDeviceToHost, st))) != CORR_OK)
    return rc;
  if (h_stokes && (rc = cuda_err(cudaMemcpyAsync(h_stokes, ctx->d_stokes_out, st_bytes,
                                                 cudaMemcpyDeviceToHost, st))) != CORR_OK)
    return rc;
  return cuda_err(cudaStreamSynchronize(st));
}

int corr_sizes(const corr_ctx *ctx, size_t *vis_elems, size_t *stokes_elems,
               long long *samples_integrated) {
  if (!ctx) return CORR_EINVAL;
  if (vis_elems) *vis_elems = (size_t)ctx->n_chan * ctx->n_pairs * 2;
  if (stokes_elems) *stokes_elems = ctx->n_pol == 2 ? (size_t)ctx->n_chan * ctx->n_apairs * 8 : 0;
  if (samples_integrated) *samples_integrated = ctx->samples;
  return CORR_OK;
}

int corr_check(corr_ctx *ctx, void *stream) {
  CORR_TRACE("corr_check");
  if (!ctx) return CORR_EINVAL;
  int rc;
  if (kDebug) {
    const size_t acc_bytes = (size_t)ctx->n_chan * ctx->n_pairs * 16;
    if ((rc = cuda_err(xe::launch_guard_check(ctx->acc_alloc,
                                              ctx->acc_alloc + xe::kGuardBytes + acc_bytes,
                                              xe::kGuardBytes, ctx->d_status,
                                              static_cast<cudaStream_t>(stream)))) != CORR_OK)
      return rc;
  }
  if ((rc = cuda_err(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)))) != CORR_OK)
    return rc;
  int status = 0;
  if ((rc = cuda_err(cudaMemcpy(&status, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost))) !=
      CORR_OK)
    return rc;
  if (status) {
    if ((rc = cuda_err(cudaMemset(ctx->d_status, 0, sizeof(int)))) != CORR_OK) return rc;
    return (status & xe::kStatusBounds) ? CORR_EBOUNDS : CORR_ETIMEOUT;
  }
  return CORR_OK;
}

int corr_plan(int n_in, uint8_t *cover, int *n_units, long long *issued_cmacs) {
  return corr_plan_cover(n_in, CORR_COVER_WINDOW, cover, n_units, issued_cmacs);
}

int corr_plan_items(int n_in, int n_chan, int block_len, int n_blocks, int cover, int grid,
                    int *items, int cap, int *n_items, int *cta_first, int *used_grid) {
  if (n_in <= 0 || n_in > CORR_MAX_INPUTS || n_chan <= 0 || block_len <= 0 ||
      block_len > CORR_MAX_BLOCK_LEN || n_blocks <= 0 || n_blocks > xe::kMaxBlocksPerLaunch ||
      grid <= 0 || cover < 0 || cover > 3)
    return CORR_EINVAL;
  // with CORR_COVER_QUADS, grid counts CTA pairs
  const std::vector<XUnit> units = xe::build_schedule(n_in, cover);
  if (units.empty()) return CORR_EINVAL;
  std::vector<xe::XItem> it;
  std::vector<int> first;
  const int used = xe::build_items({{&units, n_chan, block_len, n_blocks}}, grid, it, first);
  if (n_items) *n_items = (int)it.size();
  if (used_grid) *used_grid = used;
  if (cta_first)
    for (int k = 0; k <= used; ++k) cta_first[k] = first[k];
  if (items) {
    if (cap < (int)it.size()) return CORR_EINVAL;
    for (size_t k = 0; k < it.size(); ++k) {
      items[5 * k + 0] = it[k].prob;
      items[5 * k + 1] = it[k].tpl;
      items[5 * k + 2] = it[k].chan;
      items[5 * k + 3] = it[k].pk0;
      items[5 * k + 4] = it[k].npk;
    }
  }
  return CORR_OK;
}

int corr_plan_cover(int n_in, int cover_kind, uint8_t *cover, int *n_units,
                    long long *issued_cmacs) {
  if (n_in <= 0 || n_in > CORR_MAX_INPUTS || cover_kind < 0 || cover_kind > 3) return CORR_EINVAL;
  std::vector<XUnit> units = xe::build_schedule(n_in, cover_kind);
  if (units.empty()) return CORR_EINVAL;
  long long issued = 0;
  for (const XUnit &u : units) {
    // a unit of several channels repeats its cover once per channel: count
    // the first channel's segments
    // a pair unit covers its rows once per CTA of the pair, the odd CTA's
    // from row_in1
    for (int rank = 0; rank < (u.pair_rows ? 2 : 1); ++rank)
      for (int sg = 0; sg < u.n_seg; ++sg) {
        const XSeg &s = u.seg[sg];
        if (s.chan_off != 0) continue;
        // a multi-channel tile issues its MMAs for all its channels: count
        // the first channel's share, and only its diagonal block
        const int cpt = s.ch_rows ? xe::kTileInputs / s.ch_rows : 1;
        issued += 64LL * s.n / cpt;  // 128 accumulator rows = 64 inputs x (re, im)
        if (!cover) continue;
        // the epilogue's mapping: lane rho holds input row_in0 (row_in1 on the
        // odd CTA of a pair) + 8 (rho / 16) + rho % 8, real part when (rho / 8)
        // is even; column n holds input col_blk[n / 64] + n % 64
        for (int rho = 0; rho < 128; ++rho) {
          if ((rho >> 3) & 1) continue;
          const int i = (rank ? s.row_in1 : s.row_in0) + 8 * (rho >> 4) + (rho & 7);
          if (i >= n_in || (s.ch_rows && i >= s.ch_rows)) continue;
          for (int n = 0; n < s.n; ++n) {
            const int j = s.col_blk[n >> 6] + (n & 63);
            if (s.ch_rows && j >= s.ch_rows) continue;
            if (j <= i) cover[(size_t)i * n_in + j]++;
          }
        }
      }
  }
  if (n_units) *n_units = (int)units.size();
  if (issued_cmacs) *issued_cmacs = issued;
  return CORR_OK;
}

long long corr_launch_count(const corr_ctx *ctx) { return ctx ? ctx->launches : 0; }

int corr_debug_build(void) { return kDebug ? 1 : 0; }

int corr_debug_corrupt_guard(corr_ctx *ctx, int side) {
  if (!ctx || (side != 0 && side != 1)) return CORR_EINVAL;
  if (!kDebug) return CORR_ESTATE;
  const size_t acc_bytes = (size_t)ctx->n_chan * ctx->n_pairs * 16;
  unsigned char *at = side == 0 ? ctx->acc_alloc + xe::kGuardBytes / 2
                                : ctx->acc_alloc + xe::kGuardBytes + acc_bytes + xe::kGuardBytes / 2;
  return cuda_err(cudaMemset(at, 0, 1));
}

int corr_get_stats(const corr_ctx *ctx, corr_stats *out) {
  if (!ctx || !out) return CORR_EINVAL;
  out->blocks_pushed = ctx->blocks_pushed;
  out->samples_total = ctx->samples_total;
  out->samples_pending = ctx->samples;
  out->dumps = ctx->dumps;
  out->launches = ctx->launches;
  return CORR_OK;
}

int corr_snapshot(corr_ctx *ctx, int64_t *h_acc, long long *samples, void *stream) {
  if (!ctx || !h_acc || !samples) return CORR_EINVAL;
  CORR_TRACE("corr_snapshot");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t bytes = (size_t)ctx->n_chan * ctx->n_pairs * 16;
  int rc;
  if ((rc = cuda_err(cudaMemcpyAsync(h_acc, ctx->d_acc, bytes, cudaMemcpyDeviceToHost, st))) !=
          CORR_OK ||
      (rc = cuda_err(cudaStreamSynchronize(st))) != CORR_OK)
    return rc;
  *samples = ctx->samples;
  return CORR_OK;
}

int corr_restore(corr_ctx *ctx, const int64_t *h_acc, long long samples, void *stream) {
  if (!ctx || !h_acc || samples < 0) return CORR_EINVAL;
  CORR_TRACE("corr_restore");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t bytes = (size_t)ctx->n_chan * ctx->n_pairs * 16;
  int rc;
  if ((rc = cuda_err(cudaMemcpyAsync(ctx->d_acc, h_acc, bytes, cudaMemcpyHostToDevice, st))) !=
          CORR_OK ||
      (rc = cuda_err(cudaStreamSynchronize(st))) != CORR_OK)
    return rc;
  ctx->samples = samples;
  return CORR_OK;
}

void corr_destroy(corr_ctx *ctx) { free_ctx(ctx); }

}  // extern "C"
