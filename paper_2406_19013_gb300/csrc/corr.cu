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
#include "xe_internal.h"

using xe::XParams;
using xe::XRegion;
using xe::XSeg;
using xe::XUnit;

struct corr_ctx {
  int n_ant, n_pol, n_chan, block_len, n_in;
  long long n_pairs, n_apairs;
  int device, n_sm;
  int64_t *d_acc;
  int *d_status;
  XUnit *d_units;
  int n_tpl;
  int smem_bytes, z_stages, pk_stages;
  uint32_t z_stage_bytes, pk_stage_bytes;
  int pitch;           // row pitch of the staged block (block_len rounded up to 16)
  uint8_t *d_pitched;  // [n_chan][n_in][pitch] when block_len % 16 != 0
  long long samples;
  long long launches;
  unsigned long long timeout_ns;
  // host-buffer variants
  uint8_t *d_stage[2];
  cudaEvent_t ev_free[2], ev_ready[2];
  cudaStream_t copy_stream;
  int next_slot;
  int64_t *d_vis_out, *d_stokes_out;
};

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

int round_up(int v, int m) { return (v + m - 1) / m * m; }

// Tiles of 64 inputs (rows) cover the lower triangle strip by strip: row tile
// t needs columns [0, min(64(t+1), N)).  Columns are staged once per chunk
// and shared by all row tiles of a unit.
std::vector<XUnit> build_schedule(int N) {
  std::vector<XUnit> units;
  const int n16 = round_up(N, 16);
  const int n_rt = (N + xe::kTileInputs - 1) / xe::kTileInputs;
  auto add_seg = [](XUnit &u, int a_zrow, int b_zrow, int b_sbo, int n, int row_in0, int col_in0) {
    XSeg &s = u.seg[u.n_seg];
    int col = 0;
    for (int k = 0; k < u.n_seg; ++k) col += u.seg[k].n;
    s.a_zrow = a_zrow; s.b_zrow = b_zrow; s.b_sbo = b_sbo; s.n = n; s.tmem_col = col;
    s.row_in0 = row_in0; s.col_in0 = col_in0;
    u.n_seg++;
    u.work += n;
  };
  auto add_reg = [](XUnit &u, int in_lo, int n_in, int interleaved) {
    XRegion &r = u.reg[u.n_reg];
    r.in_lo = in_lo; r.n_in = n_in; r.interleaved = interleaved;
    r.z_row = u.z_rows; r.pk_off = u.pk_bytes;
    u.z_rows += interleaved ? 2 * n_in : n_in;
    u.pk_bytes += n_in * xe::kPackedRowBytes;
    u.n_reg++;
  };
  if (N <= 256) {
    // one staged window [0, 64 n_rt); strips packed first-fit into 512 TMEM columns
    std::vector<int> tiles(n_rt);
    for (int t = 0; t < n_rt; ++t) tiles[t] = t;
    std::sort(tiles.begin(), tiles.end(), [](int a, int b) { return a > b; });
    std::vector<std::vector<int>> bins;
    std::vector<int> used;
    for (int t : tiles) {
      const int n = std::min(xe::kTileInputs * (t + 1), n16);
      bool placed = false;
      for (size_t k = 0; k < bins.size(); ++k)
        if (used[k] + n <= xe::kTmemCols) { bins[k].push_back(t); used[k] += n; placed = true; break; }
      if (!placed) { bins.push_back({t}); used.push_back(n); }
    }
    for (auto &bin : bins) {
      XUnit u;
      std::memset(&u, 0, sizeof(u));
      int t_max = 0;
      for (int t : bin) t_max = std::max(t_max, t);
      add_reg(u, 0, xe::kTileInputs * (t_max + 1), 1);
      for (int t : bin)
        add_seg(u, 128 * t, 0, 2048, std::min(xe::kTileInputs * (t + 1), n16),
                xe::kTileInputs * t, 0);
      units.push_back(u);
    }
  } else {
    // pairs of row tiles (2m, 2m+1) against 256-column pieces of their strip
    for (int m = 0; 2 * m < n_rt; ++m) {
      const int t0 = 2 * m;
      const bool two = t0 + 1 < n_rt;
      const int row_lo = xe::kTileInputs * t0;
      const int kd = row_lo / 256;  // piece holding the diagonal
      for (int k = 0; k <= kd; ++k) {
        XUnit u;
        std::memset(&u, 0, sizeof(u));
        if (k < kd) {
          add_reg(u, row_lo, two ? 128 : 64, 1);
          add_reg(u, 256 * k, 256, 0);
          const int bz = u.reg[1].z_row;
          add_seg(u, 0, bz, 1024, 256, row_lo, 256 * k);
          if (two) add_seg(u, 128, bz, 1024, 256, row_lo + 64, 256 * k);
        } else {
          const int lo = 256 * k;
          const int hi = row_lo + (two ? 128 : 64);
          add_reg(u, lo, hi - lo, 1);
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
  return units;
}

int cuda_err(cudaError_t e) {
  if (e == cudaSuccess) return CORR_OK;
  if (e == cudaErrorMemoryAllocation) return CORR_ENOMEM;
  return CORR_ECUDA;
}

int encode_block_map(const corr_ctx *ctx, const void *base, CUtensorMap *m) {
  EncodeTiledFn enc = get_encode_fn();
  if (!enc) return CORR_ECUDA;
  const cuuint64_t dims[3] = {(cuuint64_t)ctx->block_len, (cuuint64_t)ctx->n_in,
                              (cuuint64_t)ctx->n_chan};
  const cuuint64_t strides[2] = {(cuuint64_t)ctx->pitch,
                                 (cuuint64_t)ctx->pitch * (cuuint64_t)ctx->n_in};
  const cuuint32_t box[3] = {(cuuint32_t)xe::kPkSamples, (cuuint32_t)xe::kTileInputs, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, const_cast<void *>(base), dims, strides,
                   box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? CORR_OK : CORR_ECUDA;
}

int free_ctx(corr_ctx *ctx) {
  if (!ctx) return CORR_OK;
  cudaFree(ctx->d_acc);
  cudaFree(ctx->d_status);
  cudaFree(ctx->d_units);
  cudaFree(ctx->d_pitched);
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
    default: return "unknown error";
  }
}

int corr_create(int n_ant, int n_pol, int n_chan, int block_len, corr_ctx **out) {
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

  std::vector<XUnit> units = build_schedule(ctx->n_in);
  ctx->n_tpl = (int)units.size();
  int max_z = 0, max_pk = 0;
  for (const XUnit &u : units) {
    max_z = std::max(max_z, u.z_rows);
    max_pk = std::max(max_pk, u.pk_bytes);
  }
  ctx->z_stage_bytes = (uint32_t)round_up(max_z * 128, 1024);
  ctx->pk_stage_bytes = (uint32_t)round_up(max_pk, 1024);  // swizzled TMA destination
  const int fixed = 1024 /* alignment slack */ + 256 /* barriers, TMEM address, flags */;
  static_assert(8 * (2 * 4 + 2 * 4 + 2 + xe::kMmaWarps) + 8 <= 256, "barrier area");
  // three packed stages (bytes in flight for HBM) if that leaves two or more
  // operand stages, else two
  int zs = 0;
  for (int ps = 3; ps >= 2 && zs < 2; --ps) {
    ctx->pk_stages = ps;
    zs = (smem_optin - fixed - ps * (int)ctx->pk_stage_bytes) / (int)ctx->z_stage_bytes;
  }
  zs = std::min(zs, 4);
  if (zs < 2) {
    free_ctx(ctx);
    return CORR_EINVAL;
  }
  ctx->z_stages = zs;
  ctx->smem_bytes = fixed + zs * (int)ctx->z_stage_bytes + ctx->pk_stages * (int)ctx->pk_stage_bytes;
  // one CTA per SM: the kernel holds all 512 TMEM columns
  ctx->smem_bytes = std::max(ctx->smem_bytes, smem_optin / 2 + 1024);
  ctx->smem_bytes = std::min(ctx->smem_bytes, smem_optin);

  int rc = CORR_OK;
  const size_t acc_bytes = (size_t)n_chan * (size_t)ctx->n_pairs * 16;
  if ((rc = cuda_err(cudaMalloc(&ctx->d_acc, acc_bytes))) != CORR_OK ||
      (rc = cuda_err(cudaMalloc(&ctx->d_status, sizeof(int)))) != CORR_OK ||
      (rc = cuda_err(cudaMalloc(&ctx->d_units, units.size() * sizeof(XUnit)))) != CORR_OK) {
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
  if ((rc = cuda_err(cudaMemset(ctx->d_acc, 0, acc_bytes))) != CORR_OK ||
      (rc = cuda_err(cudaMemset(ctx->d_status, 0, sizeof(int)))) != CORR_OK ||
      (rc = cuda_err(cudaMemcpy(ctx->d_units, units.data(), units.size() * sizeof(XUnit),
                                cudaMemcpyHostToDevice))) != CORR_OK ||
      (rc = cuda_err(xe::cmac_set_smem(ctx->smem_bytes))) != CORR_OK ||
      (rc = cuda_err(cudaDeviceSynchronize())) != CORR_OK) {
    free_ctx(ctx);
    return rc;
  }
  if (!get_encode_fn()) {
    free_ctx(ctx);
    return CORR_ECUDA;
  }
  *out = ctx;
  return CORR_OK;
}

int corr_push_blocks(corr_ctx *ctx, const uint8_t *const *d_blocks, int n_blocks,
                     void *stream) {
  if (!ctx || !d_blocks || n_blocks <= 0) return CORR_EINVAL;
  for (int k = 0; k < n_blocks; ++k)
    if (!d_blocks[k] || (reinterpret_cast<uintptr_t>(d_blocks[k]) & 15u) != 0) return CORR_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  static_assert(sizeof(CUtensorMap) == sizeof(xe::XMaps::m[0]), "tensor map size");
  // a fold must come before 2^24 / 128 samples have been accumulated in fp32
  int per = std::min(xe::kMaxBlocksPerLaunch, (CORR_MAX_BLOCK_LEN) / ctx->block_len);
  if (ctx->d_pitched) per = 1;  // one pitched staging buffer
  per = std::max(per, 1);
  XParams p;
  p.units = ctx->d_units;
  p.n_tpl = ctx->n_tpl;
  p.n_chan = ctx->n_chan;
  p.n_in = ctx->n_in;
  p.chunks_per_block = (ctx->block_len + xe::kChunkSamples - 1) / xe::kChunkSamples;
  p.pk_per_block = (ctx->block_len + xe::kPkSamples - 1) / xe::kPkSamples;
  p.n_pairs = ctx->n_pairs;
  p.acc = ctx->d_acc;
  p.status = ctx->d_status;
  p.timeout_ns = ctx->timeout_ns;
  p.z_stages = ctx->z_stages;
  p.pk_stages = ctx->pk_stages;
  p.z_stage_bytes = ctx->z_stage_bytes;
  p.pk_stage_bytes = ctx->pk_stage_bytes;
  const long long n_work = (long long)ctx->n_tpl * ctx->n_chan;
  const int grid = (int)std::min<long long>(n_work, ctx->n_sm);
  int rc;
  for (int k0 = 0; k0 < n_blocks; k0 += per) {
    const int nb = std::min(per, n_blocks - k0);
    xe::XMaps maps;
    std::memset(&maps, 0, sizeof(maps));
    for (int k = 0; k < nb; ++k) {
      const uint8_t *src = d_blocks[k0 + k];
      if (ctx->d_pitched) {
        if ((rc = cuda_err(xe::launch_pitch(src, ctx->d_pitched, (long long)ctx->n_chan * ctx->n_in,
                                            ctx->block_len, ctx->pitch, st, ctx->n_sm * 8))) !=
            CORR_OK)
          return rc;
        ctx->launches++;
        src = ctx->d_pitched;
      }
      if ((rc = encode_block_map(ctx, src, reinterpret_cast<CUtensorMap *>(maps.m[k]))) != CORR_OK)
        return rc;
    }
    p.n_blocks = nb;
    if ((rc = cuda_err(xe::launch_cmac(maps, p, grid, ctx->smem_bytes, st))) != CORR_OK) return rc;
    ctx->launches++;
    ctx->samples += (long long)nb * ctx->block_len;
  }
  return CORR_OK;
}

int corr_push_block(corr_ctx *ctx, const uint8_t *d_block, void *stream) {
  if (!ctx || !d_block) return CORR_EINVAL;
  return corr_push_blocks(ctx, &d_block, 1, stream);
}

int corr_dump(corr_ctx *ctx, int64_t *d_vis, int64_t *d_stokes, void *stream) {
  if (!ctx) return CORR_EINVAL;
  if (d_stokes && ctx->n_pol != 2) return CORR_EINVAL;
  if ((reinterpret_cast<uintptr_t>(d_vis) & 15u) || (reinterpret_cast<uintptr_t>(d_stokes) & 15u))
    return CORR_EINVAL;
  int rc = cuda_err(xe::launch_dump(ctx->d_acc, d_vis, d_stokes, ctx->n_ant, ctx->n_pol,
                                    ctx->n_chan, static_cast<cudaStream_t>(stream),
                                    ctx->n_sm * 8));
  if (rc != CORR_OK) return rc;
  ctx->launches++;
  ctx->samples = 0;
  return CORR_OK;
}

int corr_push_block_host(corr_ctx *ctx, const uint8_t *h_block, void *stream) {
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
  if (!ctx) return CORR_EINVAL;
  int rc;
  if ((rc = cuda_err(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)))) != CORR_OK)
    return rc;
  int status = 0;
  if ((rc = cuda_err(cudaMemcpy(&status, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost))) !=
      CORR_OK)
    return rc;
  if (status) {
    if ((rc = cuda_err(cudaMemset(ctx->d_status, 0, sizeof(int)))) != CORR_OK) return rc;
    return CORR_ETIMEOUT;
  }
  return CORR_OK;
}

int corr_plan(int n_in, uint8_t *cover, int *n_units, long long *issued_cmacs) {
  if (n_in <= 0 || n_in > CORR_MAX_INPUTS) return CORR_EINVAL;
  std::vector<XUnit> units = build_schedule(n_in);
  long long issued = 0;
  for (const XUnit &u : units) {
    for (int sg = 0; sg < u.n_seg; ++sg) {
      const XSeg &s = u.seg[sg];
      issued += 64LL * s.n;  // 128 accumulator rows = 64 inputs x (re, im)
      if (!cover) continue;
      // the epilogue's mapping: lane rho holds input row_in0 + 8 (rho / 16) + rho % 8,
      // real part when (rho / 8) is even; column n holds input col_in0 + n
      for (int rho = 0; rho < 128; ++rho) {
        if ((rho >> 3) & 1) continue;
        const int i = s.row_in0 + 8 * (rho >> 4) + (rho & 7);
        if (i >= n_in) continue;
        for (int n = 0; n < s.n; ++n) {
          const int j = s.col_in0 + n;
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

void corr_destroy(corr_ctx *ctx) { free_ctx(ctx); }

}  // extern "C"
