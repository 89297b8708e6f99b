// corr_static.cu -- corr_xcorr_static: one block's visibilities with no
// allocation at all.
//
// Some callers of this library cannot allocate device memory: code that runs
// inside a framework which owns the whole device memory pool (an allocation
// outside that pool can exceed its budget), and code on a real-time path where
// the implicit synchronisation of cudaMalloc/cudaFree would stall work already
// queued on the device.  For them this entry point runs the X-engine kernel on
// one block with every piece of scratch memory the kernel needs (its tile
// schedule and its status word) held in a file-scope device array of fixed
// size, and writes the visibilities straight into the caller's buffer.  It
// calls no cudaMalloc, cudaFree or other allocating routine, on the device or
// on the host.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "corr.h"
#include "xe_internal.h"

namespace {

// The scratch: [status word, padded to 256 bytes][problem descriptor,
// padded to 128 bytes][tile schedule].
static __device__ __align__(256) unsigned char g_static_scratch[CORR_STATIC_SCRATCH_BYTES];

constexpr int kStatusBytes = 256;
constexpr int kProbBytes = 128;
static_assert(sizeof(xe::XProb) <= kProbBytes, "problem descriptor slot");
constexpr int kMaxStaticUnits =
    (CORR_STATIC_SCRATCH_BYTES - kStatusBytes - kProbBytes) / (int)sizeof(xe::XUnit);
static_assert(kMaxStaticUnits >= 4, "scratch must hold the schedule of up to 256 inputs");

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned char *g_scratch_addr[kMaxDevices];  // device address of the array, per device
int g_smem_optin[kMaxDevices];
int g_n_sm[kMaxDevices];
unsigned long long g_timeout_ns = 2000000000ull;  // device-side wait limit (CORR_TIMEOUT_MS)

// The schedule and problem descriptor of one call, passed by value in the
// parameters of the set-up kernel below (so nothing is copied from host
// memory, which a captured copy would read again at replay).
constexpr int kMaxCallUnits = 4;
struct StaticPlan {
  xe::XProb prob;
  xe::XUnit units[kMaxCallUnits];
  int n_units;
};

// Writes the call's problem descriptor and schedule into the scratch array
// and clears the status word.  One block; the X-engine launch that follows on
// the same stream reads them.
__global__ void static_setup_kernel(const __grid_constant__ StaticPlan plan, xe::XProb *d_prob,
                                    xe::XUnit *d_units, int *d_status) {
  static_assert(sizeof(xe::XUnit) % 4 == 0 && sizeof(xe::XProb) % 4 == 0, "word copies");
  const uint32_t *src = reinterpret_cast<const uint32_t *>(plan.units);
  uint32_t *dst = reinterpret_cast<uint32_t *>(d_units);
  const int n_words = plan.n_units * (int)(sizeof(xe::XUnit) / 4);
  for (int k = threadIdx.x; k < n_words; k += blockDim.x) dst[k] = src[k];
  const uint32_t *ps = reinterpret_cast<const uint32_t *>(&plan.prob);
  uint32_t *pd = reinterpret_cast<uint32_t *>(d_prob);
  for (int k = threadIdx.x; k < (int)(sizeof(xe::XProb) / 4); k += blockDim.x) pd[k] = ps[k];
  if (threadIdx.x == 0) *d_status = 0;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn g_encode = nullptr;

int rc_of(cudaError_t e) { return e == cudaSuccess ? CORR_OK : CORR_ECUDA; }

// Once per device, with that device current: resolve the array's device
// address (in host code the array's name is only a host-side stand-in) and
// the limits the launch needs.
int setup_device(int dev) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (g_scratch_addr[dev]) return CORR_OK;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return CORR_ECUDA;
  if (prop.major != 10 || prop.minor != 3) return CORR_EARCH;
  int optin = 0;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return CORR_ECUDA;
  if (!g_encode) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return CORR_ECUDA;
    g_encode = reinterpret_cast<EncodeTiledFn>(p);
  }
  void *addr = nullptr;
  if (cudaGetSymbolAddress(&addr, g_static_scratch) != cudaSuccess || !addr) return CORR_ECUDA;
  if (const char *env = std::getenv("CORR_TIMEOUT_MS")) {
    const long long ms = std::atoll(env);
    if (ms > 0) g_timeout_ns = (unsigned long long)ms * 1000000ull;
  }
  g_smem_optin[dev] = optin;
  g_n_sm[dev] = prop.multiProcessorCount;
  g_scratch_addr[dev] = static_cast<unsigned char *>(addr);
  return CORR_OK;
}

// The single-window tile schedule (all inputs staged together; row tiles of
// 64 inputs packed into units of at most 512 accumulator columns), built in
// a fixed array.  Returns the number of units.
int plan_single_window(int N, xe::XUnit *units) {
  const int n16 = (N + 15) / 16 * 16;
  const int n_rt = (N + xe::kTileInputs - 1) / xe::kTileInputs;  // <= 4
  int bin_of[4], used[4] = {0, 0, 0, 0}, n_bins = 0;
  for (int t = n_rt - 1; t >= 0; --t) {  // largest strip first, first fit
    const int n = std::min(xe::kTileInputs * (t + 1), n16);
    int b = 0;
    while (b < n_bins && used[b] + n > xe::kTmemCols) ++b;
    if (b == n_bins) ++n_bins;
    used[b] += n;
    bin_of[t] = b;
  }
  for (int b = 0; b < n_bins; ++b) {
    xe::XUnit &u = units[b];
    std::memset(&u, 0, sizeof(u));
    u.n_chan = 1;
    int t_max = 0;
    for (int t = 0; t < n_rt; ++t)
      if (bin_of[t] == b) t_max = std::max(t_max, t);
    xe::XRegion &r = u.reg[0];
    r.in_lo = 0;
    r.in_lo1 = 0;
    r.n_in = xe::kTileInputs * (t_max + 1);
    r.interleaved = 1;
    r.z_row = 0;
    r.pk_off = 0;
    u.n_reg = 1;
    u.z_rows = 2 * r.n_in;
    u.pk_bytes = r.n_in * xe::kPackedRowBytes;
    for (int t = n_rt - 1; t >= 0; --t) {
      if (bin_of[t] != b) continue;
      xe::XSeg &s = u.seg[u.n_seg];
      s.a_zrow = 128 * t;
      s.b_zrow = 0;
      s.b_sbo = 2048;
      s.n = std::min(xe::kTileInputs * (t + 1), n16);
      s.tmem_col = u.work;
      s.row_in0 = xe::kTileInputs * t;
      s.row_in1 = s.row_in0;
      for (int c = 0; c < 4; ++c) s.col_blk[c] = 64 * c;  // columns 0, 1, 2, ...
      u.work += s.n;
      u.n_seg++;
    }
  }
  // heaviest unit first (at most four: an insertion sort)
  for (int i = 1; i < n_bins; ++i)
    for (int j = i; j > 0 && units[j - 1].work < units[j].work; --j) std::swap(units[j - 1], units[j]);
  return n_bins;
}

}  // namespace

extern "C" int corr_xcorr_static(const uint8_t *d_block, int n_ant, int n_pol, int n_chan,
                                 int block_len, int64_t *d_vis, void *stream) {
  if (!d_block || !d_vis || n_ant <= 0 || n_chan <= 0 || block_len <= 0 ||
      (n_pol != 1 && n_pol != 2))
    return CORR_EINVAL;
  const long long N = (long long)n_ant * n_pol;
  if (N > CORR_STATIC_MAX_INPUTS || block_len > CORR_STATIC_MAX_BLOCK_LEN || block_len % 16 != 0)
    return CORR_EINVAL;
  if ((reinterpret_cast<uintptr_t>(d_block) & 15u) || (reinterpret_cast<uintptr_t>(d_vis) & 15u))
    return CORR_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return CORR_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return CORR_EINVAL;
  int rc = setup_device(dev);
  if (rc != CORR_OK) return rc;

  StaticPlan plan;
  std::memset(&plan, 0, sizeof(plan));
  xe::XUnit *units = plan.units;
  const int n_tpl = plan_single_window((int)N, units);
  if (n_tpl > kMaxStaticUnits || n_tpl > kMaxCallUnits) return CORR_EINVAL;
  plan.n_units = n_tpl;
  int max_z = 0, max_pk = 0;
  for (int k = 0; k < n_tpl; ++k) {
    max_z = std::max(max_z, units[k].z_rows);
    max_pk = std::max(max_pk, units[k].pk_bytes);
  }
  // shared-memory stages, sized as for a context
  const int optin = g_smem_optin[dev];
  const int z_bytes = (max_z * 128 + 1023) / 1024 * 1024;
  const int pk_bytes = (max_pk + 1023) / 1024 * 1024;
  const int fixed = 1024 + xe::kBarrierBytes;
  int pk_stages = 3, z_stages = 0;
  for (int ps = 3; ps >= 2 && z_stages < 2; --ps) {
    pk_stages = ps;
    z_stages = (optin - fixed - ps * pk_bytes) / z_bytes;
  }
  z_stages = std::min(z_stages, 4);
  if (z_stages < 2) return CORR_EINVAL;
  int smem = fixed + z_stages * z_bytes + pk_stages * pk_bytes;
  smem = std::min(std::max(smem, optin / 2 + 1024), optin);

  cudaStream_t st = static_cast<cudaStream_t>(stream);
  unsigned char *scratch = g_scratch_addr[dev];
  int *d_status = reinterpret_cast<int *>(scratch);
  xe::XProb *d_prob = reinterpret_cast<xe::XProb *>(scratch + kStatusBytes);
  xe::XUnit *d_units = reinterpret_cast<xe::XUnit *>(scratch + kStatusBytes + kProbBytes);
  const size_t vis_bytes = (size_t)n_chan * (size_t)(N * (N + 1) / 2) * 16;
  xe::XProb &prob = plan.prob;
  prob.units = d_units;
  prob.acc = d_vis;
  prob.n_pairs = N * (N + 1) / 2;
  prob.n_in = (int)N;
  prob.n_chan = n_chan;
  prob.chunks_per_block = (block_len + xe::kChunkSamples - 1) / xe::kChunkSamples;
  prob.pk_per_block = (block_len + xe::kPkSamples - 1) / xe::kPkSamples;
  prob.map0 = 0;
  // the scratch keeps the previous call's contents: rewrite the schedule and
  // the problem and clear the status word (a set-up kernel that receives
  // them by value), and start the visibilities, which the X-engine
  // accumulates into, from zero
  if ((rc = rc_of(xe::cmac_set_smem(optin))) != CORR_OK) return rc;
  static_setup_kernel<<<1, 128, 0, st>>>(plan, d_prob, d_units, d_status);
  if ((rc = rc_of(cudaGetLastError())) != CORR_OK ||
      (rc = rc_of(cudaMemsetAsync(d_vis, 0, vis_bytes, st))) != CORR_OK)
    return rc;

  xe::XMaps maps;
  std::memset(&maps, 0, sizeof(maps));
  const cuuint64_t dims[3] = {(cuuint64_t)block_len, (cuuint64_t)N, (cuuint64_t)n_chan};
  const cuuint64_t strides[2] = {(cuuint64_t)block_len, (cuuint64_t)block_len * (cuuint64_t)N};
  const cuuint32_t box[3] = {(cuuint32_t)xe::kPkSamples, (cuuint32_t)xe::kTileInputs, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  if (g_encode(reinterpret_cast<CUtensorMap *>(maps.m[0]), CU_TENSOR_MAP_DATA_TYPE_UINT8, 3,
               const_cast<uint8_t *>(d_block), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
               CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return CORR_ECUDA;

  xe::XParams p;
  std::memset(&p, 0, sizeof(p));
  p.probs = d_prob;
  p.items = nullptr;  // whole units, dealt round-robin over the CTAs
  p.cta_first = nullptr;
  p.implicit_n_tpl = n_tpl;
  p.implicit_n_chan = n_chan;
  p.implicit_npk = prob.pk_per_block;
  p.status = d_status;
  p.timeout_ns = g_timeout_ns;
  p.z_stages = z_stages;
  p.pk_stages = pk_stages;
  p.z_stage_bytes = (uint32_t)z_bytes;
  p.pk_stage_bytes = (uint32_t)pk_bytes;
  const long long n_work = (long long)n_tpl * n_chan;
  const int grid = (int)std::min<long long>(n_work, g_n_sm[dev]);
  return rc_of(xe::launch_cmac(maps, p, grid, smem, st));
}
