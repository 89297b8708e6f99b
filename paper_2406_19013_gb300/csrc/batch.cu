// batch.cu -- corr_batch_*: many independent correlators (different input
// counts, channel counts and block lengths) integrated by shared persistent
// launches of the CMAC kernel, plus the autotuner that picks each input
// count's triangle cover.
//
// The paper's system runs one X-engine per server and pipeline instance
// (Sec. 2.2-2.3), every one on its own fixed array.  On one GB300 a batch
// of such arrays, some with as few as 16 channels, cannot fill 152 SMs one
// launch at a time.  Here every instance's units (instance, template,
// channel) are cut into items and dealt to the SMs of one launch per
// shared-memory layout, so small instances fill the gaps of large ones.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <utility>
#include <vector>

#include "corr.h"
#include "xe_sched.h"
#include "xe_internal.h"
#include "trace.h"

namespace {

int cuda_err(cudaError_t e) {
  if (e == cudaSuccess) return CORR_OK;
  if (e == cudaErrorMemoryAllocation) return CORR_ENOMEM;
  return CORR_ECUDA;
}

int round_up(int v, int m) { return (v + m - 1) / m * m; }

struct BInst {
  int n_ant, n_pol, n_chan, block_len, n_in, pitch;
  long long n_pairs, n_apairs;
  size_t acc_off;      // element offset of this instance's buffer in d_acc
  uint8_t *d_pitched;  // [n_chan][n_in][pitch] when block_len % 16 != 0
  long long samples;
  int cover, group, slot;
};

struct BGroup {
  std::vector<int> members;
  std::vector<std::vector<xe::XUnit>> units;  // per member
  xe::StageLayout L;
  xe::XUnit *d_units;
  xe::XProb *d_probs;
  xe::XItem *d_items;
  int *d_cta_first;
  int grid;
};

// ---------------------------------------------------------------- autotuner
// Cover per (input count, block-length bucket), chosen by timing one launch
// of each candidate on a synthetic one-wave problem (best of five after a
// warm-up); a candidate replaces the default only when it is more than 3 %
// faster.  The kernel's time does
// not depend on the sample values, so the tuning input is all zeros.
std::mutex g_tune_mutex;
std::map<std::pair<int, int>, int> g_tune_cache;

int t_bucket(int T) {
  int b = 4;
  while ((1 << b) < T) ++b;
  return b;
}

std::vector<int> candidate_covers(int n_in) {
  if (n_in > 256) return {xe::kCoverPairs};
  return {xe::kCoverWindow, xe::kCoverStrips, xe::kCoverPairs};
}

// Milliseconds of one launch of `units` over C channels x T samples, or a
// negative value when the candidate cannot run.
float time_cover(const std::vector<xe::XUnit> &units, int n_in, int C, int T, int n_sm,
                 int smem_optin, uint8_t *d_x, int64_t *d_acc, int *d_status,
                 cudaStream_t st) {
  xe::StageLayout L;
  if (!xe::stage_layout({&units}, smem_optin, xe::kMaxZStages, &L)) return -1.0f;
  std::vector<xe::XItem> items;
  std::vector<int> first;
  const int grid = xe::build_items({{&units, C, T, 1}}, n_sm, items, first);
  xe::XUnit *d_units = nullptr;
  xe::XProb *d_prob = nullptr;
  xe::XItem *d_items = nullptr;
  int *d_first = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float best = -1.0f;
  xe::XProb prob;
  std::memset(&prob, 0, sizeof(prob));
  xe::XMaps maps;
  std::memset(&maps, 0, sizeof(maps));
  xe::XParams p;
  std::memset(&p, 0, sizeof(p));
  if (cudaMalloc(&d_units, units.size() * sizeof(xe::XUnit)) != cudaSuccess ||
      cudaMalloc(&d_prob, sizeof(xe::XProb)) != cudaSuccess ||
      cudaMalloc(&d_items, items.size() * sizeof(xe::XItem)) != cudaSuccess ||
      cudaMalloc(&d_first, first.size() * sizeof(int)) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    goto done;
  prob.units = d_units;
  prob.acc = d_acc;
  prob.n_pairs = (long long)n_in * (n_in + 1) / 2;
  prob.n_in = n_in;
  prob.n_chan = C;
  prob.chunks_per_block = (T + xe::kChunkSamples - 1) / xe::kChunkSamples;
  prob.pk_per_block = (T + xe::kPkSamples - 1) / xe::kPkSamples;
  prob.map0 = 0;
  if (cudaMemcpy(d_units, units.data(), units.size() * sizeof(xe::XUnit), cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      cudaMemcpy(d_prob, &prob, sizeof(prob), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(d_items, items.data(), items.size() * sizeof(xe::XItem),
                 cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(d_first, first.data(), first.size() * sizeof(int), cudaMemcpyHostToDevice) !=
          cudaSuccess)
    goto done;
  if (!xe::encode_block_map(d_x, T, n_in, C, T, maps.m[0], xe::tile_ch_rows(units))) goto done;
  p.probs = d_prob;
  p.items = d_items;
  p.cta_first = d_first;
  p.status = d_status;
  p.timeout_ns = 2000000000ull;
  p.z_stages = L.z_stages;
  p.pk_stages = L.pk_stages;
  p.z_stage_bytes = L.z_stage_bytes;
  p.pk_stage_bytes = L.pk_stage_bytes;
  for (int rep = 0; rep < 6; ++rep) {
    if (cudaEventRecord(e0, st) != cudaSuccess ||
        xe::launch_cmac(maps, p, grid, L.smem_bytes, st) != cudaSuccess ||
        cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
      best = -1.0f;
      goto done;
    }
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && (best < 0.0f || ms < best)) best = ms;  // the first launch warms up
  }
done:
  cudaFree(d_units);
  cudaFree(d_prob);
  cudaFree(d_items);
  cudaFree(d_first);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return best;
}

// The cover for (n_in, block_len): cached, else timed now.
int tuned_cover(int n_in, int block_len, int n_sm, int smem_optin, int *rc) {
  *rc = CORR_OK;
  const std::pair<int, int> key(n_in, t_bucket(block_len));
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  auto hit = g_tune_cache.find(key);
  if (hit != g_tune_cache.end()) return hit->second;
  const std::vector<int> cands = candidate_covers(n_in);
  if (cands.size() == 1) return g_tune_cache[key] = cands[0];
  const int T = std::min(1 << key.second, 8192);
  const int C = n_sm;
  const long long n_pairs = (long long)n_in * (n_in + 1) / 2;
  uint8_t *d_x = nullptr;
  int64_t *d_acc = nullptr;
  int *d_status = nullptr;
  cudaStream_t st = nullptr;
  int best_cover = cands[0];
  float best_ms = -1.0f;
  if ((*rc = cuda_err(cudaMalloc(&d_x, (size_t)C * n_in * T))) != CORR_OK ||
      (*rc = cuda_err(cudaMalloc(&d_acc, (size_t)C * n_pairs * 16))) != CORR_OK ||
      (*rc = cuda_err(cudaMalloc(&d_status, sizeof(int)))) != CORR_OK ||
      (*rc = cuda_err(cudaMemset(d_x, 0, (size_t)C * n_in * T))) != CORR_OK ||
      (*rc = cuda_err(cudaMemset(d_status, 0, sizeof(int)))) != CORR_OK ||
      (*rc = cuda_err(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking))) != CORR_OK)
    goto done;
  // the default cover (the first candidate) is kept unless another one is
  // faster by more than the run-to-run spread of a timing (3 %)
  for (int cv : cands) {
    const std::vector<xe::XUnit> units = xe::build_schedule(n_in, cv);
    if (units.empty()) continue;
    const float ms = time_cover(units, n_in, C, T, n_sm, smem_optin, d_x, d_acc, d_status, st);
    if (ms >= 0.0f && (best_ms < 0.0f || ms < 0.97f * best_ms)) {
      best_ms = ms;
      best_cover = cv;
    }
  }
  {
    int status = 0;
    if ((*rc = cuda_err(cudaMemcpy(&status, d_status, sizeof(int), cudaMemcpyDeviceToHost))) !=
        CORR_OK)
      goto done;
    if (status) *rc = CORR_ETIMEOUT;
  }
  if (best_ms < 0.0f && *rc == CORR_OK) *rc = CORR_ECUDA;
done:
  if (st) cudaStreamDestroy(st);
  cudaFree(d_x);
  cudaFree(d_acc);
  cudaFree(d_status);
  if (*rc != CORR_OK) return -1;
  return g_tune_cache[key] = best_cover;
}

}  // namespace

struct corr_batch {
  std::vector<BInst> inst;
  std::vector<BGroup> groups;
  // one stream per launch group after the first (which runs on the caller's
  // stream), so the tail of one group's launch overlaps the next; forked and
  // joined with events, so a push stays capturable in a CUDA graph
  std::vector<cudaStream_t> side;
  cudaEvent_t ev_fork = nullptr;
  std::vector<cudaEvent_t> ev_join;
  int64_t *d_acc;
  int *d_status;
  int device, n_sm, smem_optin;
  unsigned long long timeout_ns;
  long long launches;
};

namespace {

void free_batch(corr_batch *b) {
  if (!b) return;
  for (cudaStream_t st : b->side)
    if (st) cudaStreamDestroy(st);
  for (cudaEvent_t e : b->ev_join)
    if (e) cudaEventDestroy(e);
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  for (BGroup &g : b->groups) {
    cudaFree(g.d_units);
    cudaFree(g.d_probs);
    cudaFree(g.d_items);
    cudaFree(g.d_cta_first);
  }
  for (BInst &in : b->inst) cudaFree(in.d_pitched);
  cudaFree(b->d_acc);
  cudaFree(b->d_status);
  delete b;
}

// Uploads a group's templates, problem descriptors and item split.
int upload_group(corr_batch *b, BGroup &g) {
  std::vector<const std::vector<xe::XUnit> *> sets;
  for (auto &u : g.units) sets.push_back(&u);
  if (!xe::stage_layout(sets, b->smem_optin, xe::kMaxZStages, &g.L)) return CORR_EINVAL;
  std::vector<xe::XUnit> all;
  std::vector<size_t> first_unit;
  for (auto &u : g.units) {
    first_unit.push_back(all.size());
    all.insert(all.end(), u.begin(), u.end());
  }
  std::vector<xe::ProbWork> work;
  for (size_t k = 0; k < g.members.size(); ++k) {
    const BInst &in = b->inst[g.members[k]];
    work.push_back({&g.units[k], in.n_chan, in.block_len, 1});
  }
  std::vector<xe::XItem> items;
  std::vector<int> first;
  g.grid = xe::build_items(work, b->n_sm, items, first);
  int rc;
  if ((rc = cuda_err(cudaMalloc(&g.d_units, all.size() * sizeof(xe::XUnit)))) != CORR_OK ||
      (rc = cuda_err(cudaMalloc(&g.d_probs, g.members.size() * sizeof(xe::XProb)))) != CORR_OK ||
      (rc = cuda_err(cudaMalloc(&g.d_items, std::max<size_t>(1, items.size()) *
                                                sizeof(xe::XItem)))) != CORR_OK ||
      (rc = cuda_err(cudaMalloc(&g.d_cta_first, first.size() * sizeof(int)))) != CORR_OK)
    return rc;
  std::vector<xe::XProb> probs(g.members.size());
  for (size_t k = 0; k < g.members.size(); ++k) {
    const BInst &in = b->inst[g.members[k]];
    xe::XProb &p = probs[k];
    std::memset(&p, 0, sizeof(p));
    p.units = g.d_units + first_unit[k];
    p.acc = b->d_acc + in.acc_off;
    p.n_pairs = in.n_pairs;
    p.n_in = in.n_in;
    p.n_chan = in.n_chan;
    p.chunks_per_block = (in.block_len + xe::kChunkSamples - 1) / xe::kChunkSamples;
    p.pk_per_block = (in.block_len + xe::kPkSamples - 1) / xe::kPkSamples;
    p.map0 = (int)k;
  }
  if ((rc = cuda_err(cudaMemcpy(g.d_units, all.data(), all.size() * sizeof(xe::XUnit),
                                cudaMemcpyHostToDevice))) != CORR_OK ||
      (rc = cuda_err(cudaMemcpy(g.d_probs, probs.data(), probs.size() * sizeof(xe::XProb),
                                cudaMemcpyHostToDevice))) != CORR_OK ||
      (rc = cuda_err(cudaMemcpy(g.d_items, items.data(), items.size() * sizeof(xe::XItem),
                                cudaMemcpyHostToDevice))) != CORR_OK ||
      (rc = cuda_err(cudaMemcpy(g.d_cta_first, first.data(), first.size() * sizeof(int),
                                cudaMemcpyHostToDevice))) != CORR_OK)
    return rc;
  return CORR_OK;
}

}  // namespace

extern "C" {

int corr_batch_create(int n_inst, const int *n_ant, const int *n_pol, const int *n_chan,
                      const int *block_len, int flags, corr_batch **out) {
  CORR_TRACE("corr_batch_create");
  if (!out) return CORR_EINVAL;
  *out = nullptr;
  if (n_inst <= 0 || !n_ant || !n_pol || !n_chan || !block_len) return CORR_EINVAL;
  if (flags & ~CORR_BATCH_AUTOTUNE) return CORR_EINVAL;
  for (int k = 0; k < n_inst; ++k) {
    if (n_ant[k] <= 0 || n_chan[k] <= 0 || block_len[k] <= 0 || (n_pol[k] != 1 && n_pol[k] != 2))
      return CORR_EINVAL;
    if (block_len[k] > CORR_MAX_BLOCK_LEN) return CORR_EINVAL;
    if ((long long)n_ant[k] * n_pol[k] > CORR_MAX_INPUTS) return CORR_EINVAL;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return CORR_ECUDA;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return CORR_ECUDA;
  if (prop.major != 10 || prop.minor != 3) return CORR_EARCH;
  int optin = 0;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return CORR_ECUDA;

  corr_batch *b = new (std::nothrow) corr_batch;
  if (!b) return CORR_ENOMEM;
  b->d_acc = nullptr;
  b->d_status = nullptr;
  b->device = dev;
  b->n_sm = prop.multiProcessorCount;
  b->smem_optin = optin;
  b->launches = 0;
  b->timeout_ns = 2000000000ull;
  if (const char *s = std::getenv("CORR_TIMEOUT_MS")) {
    long long ms = std::atoll(s);
    if (ms > 0) b->timeout_ns = (unsigned long long)ms * 1000000ull;
  }
  int rc = CORR_OK;
  if ((rc = cuda_err(xe::cmac_set_smem(optin))) != CORR_OK) {
    free_batch(b);
    return rc;
  }
  size_t acc_elems = 0;
  b->inst.resize(n_inst);
  for (int k = 0; k < n_inst; ++k) {
    BInst &in = b->inst[k];
    std::memset(&in, 0, sizeof(in));
    in.n_ant = n_ant[k];
    in.n_pol = n_pol[k];
    in.n_chan = n_chan[k];
    in.block_len = block_len[k];
    in.n_in = n_ant[k] * n_pol[k];
    in.pitch = round_up(block_len[k], 16);
    in.n_pairs = (long long)in.n_in * (in.n_in + 1) / 2;
    in.n_apairs = (long long)in.n_ant * (in.n_ant + 1) / 2;
    in.acc_off = acc_elems;
    acc_elems += (size_t)in.n_chan * in.n_pairs * 2;
    in.cover = in.n_in <= 256 ? xe::kCoverWindow : xe::kCoverPairs;
    if (flags & CORR_BATCH_AUTOTUNE) {
      in.cover = tuned_cover(in.n_in, in.block_len, b->n_sm, optin, &rc);
      if (rc != CORR_OK) {
        free_batch(b);
        return rc;
      }
    }
  }
  if ((rc = cuda_err(cudaMalloc(&b->d_acc, acc_elems * sizeof(int64_t)))) != CORR_OK ||
      (rc = cuda_err(cudaMemset(b->d_acc, 0, acc_elems * sizeof(int64_t)))) != CORR_OK ||
      (rc = cuda_err(cudaMalloc(&b->d_status, sizeof(int)))) != CORR_OK ||
      (rc = cuda_err(cudaMemset(b->d_status, 0, sizeof(int)))) != CORR_OK) {
    free_batch(b);
    return rc;
  }
  for (BInst &in : b->inst)
    if (in.pitch != in.block_len &&
        (rc = cuda_err(cudaMalloc(&in.d_pitched, (size_t)in.n_chan * in.n_in * in.pitch))) !=
            CORR_OK) {
      free_batch(b);
      return rc;
    }

  // launch groups: instances whose templates need the same stage layout share
  // a launch (at most kMaxBatchMaps instances each, one block map apiece)
  std::vector<std::vector<xe::XUnit>> units(n_inst);
  std::map<std::pair<uint32_t, uint32_t>, std::vector<int>> by_layout;
  for (int k = 0; k < n_inst; ++k) {
    units[k] = xe::build_schedule(b->inst[k].n_in, b->inst[k].cover);
    xe::StageLayout L;
    if (units[k].empty() || !xe::stage_layout({&units[k]}, optin, xe::kMaxZStages, &L)) {
      free_batch(b);
      return CORR_EINVAL;
    }
    by_layout[{L.z_stage_bytes, L.pk_stage_bytes}].push_back(k);
  }
  for (auto &kv : by_layout) {
    const std::vector<int> &ks = kv.second;
    for (size_t a = 0; a < ks.size(); a += xe::kMaxBatchMaps) {
      BGroup g;
      g.d_units = nullptr;
      g.d_probs = nullptr;
      g.d_items = nullptr;
      g.d_cta_first = nullptr;
      g.grid = 0;
      for (size_t c = a; c < std::min(ks.size(), a + xe::kMaxBatchMaps); ++c) {
        b->inst[ks[c]].group = (int)b->groups.size();
        b->inst[ks[c]].slot = (int)g.members.size();
        g.members.push_back(ks[c]);
        g.units.push_back(units[ks[c]]);
      }
      b->groups.push_back(std::move(g));
      if ((rc = upload_group(b, b->groups.back())) != CORR_OK) {
        free_batch(b);
        return rc;
      }
    }
  }
  // largest groups first, so smaller ones fill in behind them
  std::stable_sort(b->groups.begin(), b->groups.end(), [b](const BGroup &x, const BGroup &y) {
    auto work = [b](const BGroup &g) {
      long long w = 0;
      for (size_t k = 0; k < g.members.size(); ++k)
        for (const xe::XUnit &u : g.units[k])
          w += (long long)b->inst[g.members[k]].n_chan * b->inst[g.members[k]].block_len * u.z_rows;
      return w;
    };
    return work(x) > work(y);
  });
  for (size_t gi = 0; gi < b->groups.size(); ++gi)
    for (int k : b->groups[gi].members) b->inst[k].group = (int)gi;
  if (b->groups.size() > 1) {
    if ((rc = cuda_err(cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming))) != CORR_OK) {
      free_batch(b);
      return rc;
    }
    for (size_t gi = 1; gi < b->groups.size(); ++gi) {
      cudaStream_t st = nullptr;
      cudaEvent_t ev = nullptr;
      rc = cuda_err(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
      if (rc == CORR_OK) rc = cuda_err(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
      b->side.push_back(st);
      b->ev_join.push_back(ev);
      if (rc != CORR_OK) {
        free_batch(b);
        return rc;
      }
    }
  }
  if ((rc = cuda_err(cudaDeviceSynchronize())) != CORR_OK) {
    free_batch(b);
    return rc;
  }
  *out = b;
  return CORR_OK;
}

int corr_batch_push(corr_batch *b, const uint8_t *const *d_blocks, void *stream) {
  CORR_TRACE("corr_batch_push");
  if (!b || !d_blocks) return CORR_EINVAL;
  for (size_t k = 0; k < b->inst.size(); ++k)
    if (!d_blocks[k] || (reinterpret_cast<uintptr_t>(d_blocks[k]) & 15u) != 0) return CORR_EINVAL;
  cudaStream_t user = static_cast<cudaStream_t>(stream);
  // one parameter block reused for every group (16 KB of tensor maps)
  static thread_local xe::XBatchMaps maps;
  int rc;
  if (!b->side.empty() && (rc = cuda_err(cudaEventRecord(b->ev_fork, user))) != CORR_OK) return rc;
  for (size_t gi = 0; gi < b->groups.size(); ++gi) {
    BGroup &g = b->groups[gi];
    cudaStream_t st = gi == 0 ? user : b->side[gi - 1];
    if (gi > 0 && (rc = cuda_err(cudaStreamWaitEvent(st, b->ev_fork, 0))) != CORR_OK) return rc;
    std::memset(&maps, 0, sizeof(maps));
    for (size_t s = 0; s < g.members.size(); ++s) {
      BInst &in = b->inst[g.members[s]];
      const uint8_t *src = d_blocks[g.members[s]];
      if (in.d_pitched) {
        if ((rc = cuda_err(xe::launch_pitch(src, in.d_pitched, (long long)in.n_chan * in.n_in,
                                            in.block_len, in.pitch, st, b->n_sm * 8))) != CORR_OK)
          return rc;
        b->launches++;
        src = in.d_pitched;
      }
      if (!xe::encode_block_map(src, in.block_len, in.n_in, in.n_chan, in.pitch, maps.m[s],
                                xe::tile_ch_rows(g.units[s])))
        return CORR_ECUDA;
    }
    xe::XParams p;
    std::memset(&p, 0, sizeof(p));
    p.probs = g.d_probs;
    p.items = g.d_items;
    p.cta_first = g.d_cta_first;
    p.status = b->d_status;
    p.timeout_ns = b->timeout_ns;
    p.z_stages = g.L.z_stages;
    p.pk_stages = g.L.pk_stages;
    p.z_stage_bytes = g.L.z_stage_bytes;
    p.pk_stage_bytes = g.L.pk_stage_bytes;
    if (g.grid > 0) {
      if ((rc = cuda_err(xe::launch_cmac_batch(maps, p, g.grid, g.L.smem_bytes, st))) != CORR_OK)
        return rc;
      b->launches++;
    }
    if (gi > 0 && (rc = cuda_err(cudaEventRecord(b->ev_join[gi - 1], st))) != CORR_OK) return rc;
  }
  for (size_t k = 0; k < b->ev_join.size(); ++k)
    if ((rc = cuda_err(cudaStreamWaitEvent(user, b->ev_join[k], 0))) != CORR_OK) return rc;
  for (BInst &in : b->inst) in.samples += in.block_len;
  return CORR_OK;
}

int corr_batch_dump(corr_batch *b, int inst, int64_t *d_vis, int64_t *d_stokes, void *stream) {
  CORR_TRACE("corr_batch_dump");
  if (!b || inst < 0 || inst >= (int)b->inst.size()) return CORR_EINVAL;
  BInst &in = b->inst[inst];
  if (d_stokes && in.n_pol != 2) return CORR_EINVAL;
  if ((reinterpret_cast<uintptr_t>(d_vis) & 15u) || (reinterpret_cast<uintptr_t>(d_stokes) & 15u))
    return CORR_EINVAL;
  int rc = cuda_err(xe::launch_dump(b->d_acc + in.acc_off, d_vis, d_stokes, in.n_ant, in.n_pol,
                                    in.n_chan, static_cast<cudaStream_t>(stream), b->n_sm * 8,
                                    b->d_status));
  if (rc != CORR_OK) return rc;
  b->launches++;
  in.samples = 0;
  return CORR_OK;
}

int corr_batch_sizes(const corr_batch *b, int inst, size_t *vis_elems, size_t *stokes_elems,
                     long long *samples_integrated) {
  if (!b || inst < 0 || inst >= (int)b->inst.size()) return CORR_EINVAL;
  const BInst &in = b->inst[inst];
  if (vis_elems) *vis_elems = (size_t)in.n_chan * in.n_pairs * 2;
  if (stokes_elems) *stokes_elems = in.n_pol == 2 ? (size_t)in.n_chan * in.n_apairs * 8 : 0;
  if (samples_integrated) *samples_integrated = in.samples;
  return CORR_OK;
}

int corr_batch_info(const corr_batch *b, int inst, int *cover, int *group, int *n_groups) {
  if (!b || inst < 0 || inst >= (int)b->inst.size()) return CORR_EINVAL;
  if (cover) *cover = b->inst[inst].cover;
  if (group) *group = b->inst[inst].group;
  if (n_groups) *n_groups = (int)b->groups.size();
  return CORR_OK;
}

int corr_batch_check(corr_batch *b, void *stream) {
  if (!b) return CORR_EINVAL;
  int rc;
  if ((rc = cuda_err(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)))) != CORR_OK)
    return rc;
  int status = 0;
  if ((rc = cuda_err(cudaMemcpy(&status, b->d_status, sizeof(int), cudaMemcpyDeviceToHost))) !=
      CORR_OK)
    return rc;
  if (status) {
    if ((rc = cuda_err(cudaMemset(b->d_status, 0, sizeof(int)))) != CORR_OK) return rc;
    return (status & xe::kStatusBounds) ? CORR_EBOUNDS : CORR_ETIMEOUT;
  }
  return CORR_OK;
}

long long corr_batch_launch_count(const corr_batch *b) { return b ? b->launches : 0; }

void corr_batch_destroy(corr_batch *b) { free_batch(b); }

int corr_tuned_cover(int n_in, int block_len) {
  if (n_in <= 0 || block_len <= 0) return CORR_EINVAL;
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  auto hit = g_tune_cache.find({n_in, t_bucket(block_len)});
  return hit == g_tune_cache.end() ? -1 : hit->second;
}

}  // extern "C"
