// Device-side simulation object and the C ABI calls that touch the GPU.
//
// Internal layout: nodes in the order of padded_ordering (reverse Cuthill-McKee per connected
// component, SELL row sorting, every component padded to a multiple of 32 rows by dummy rows).
// perm[internal] = caller index or -1; every device node vector has n_int entries.  Dummy rows
// have no matrix entries and a zero Jacobi inverse, so their residual, direction and update stay
// zero and their potential stays at the resting value; they never reach the caller.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "ionic_tp06.cuh"
#include "kernels.cuh"
#include "mlp.cuh"
#include "surrogate.h"
#include "tc_internal.h"

using namespace tc;

namespace {

constexpr int kIonicThreads = 256;
constexpr int kGraphSteps = 30;   // steps per captured graph (a multiple of the 3-buffer cycle)

// Launch shape of the PCG kernel: 512 or 1024 threads per block, blocks per SM, and the SELL
// sorting window; TC_PCG_THREADS, TC_PCG_BLOCKS_PER_SM and TC_SELL_SIGMA override the defaults
// (tc_autotune picks the launch shape by measurement).
int env_int(const char* name, int dflt) {
  const char* v = std::getenv(name);
  return v && *v ? std::atoi(v) : dflt;
}

struct Dev {
  void* p = nullptr;
  size_t bytes = 0;
};

struct GraphCache {
  bool valid = false;
  int iv = -1;                      // buffer rotation phase the graph was captured for
  cudaGraphExec_t exec = nullptr;
};

}  // namespace

struct tc_sim {
  int device = 0;
  cudaStream_t stream = nullptr;
  int64_t n = 0, n_int = 0, nnz = 0, nslices = 0, padded = 0;
  int n_comp = 1;
  std::vector<int64_t> comp_rows;    // n_comp + 1 internal row offsets
  int precision = TC_FP64;
  size_t esz = 8;                    // bytes per matrix value / node-vector entry
  std::vector<int32_t> perm;         // perm[internal] = caller index or -1
  std::vector<int32_t> inv;          // inv[caller] = internal index
  int num_sms = 0, blocks_per_sm = 1, nblocks = 0, pcg_threads = 1024, sell_sigma = 1024;
  float l2_keep = 0.f;   // fraction of A and the index array kept in L2 by the PCG (FP64)
  // TP06 FP64: the four concentration logarithms of the states, [4][n_int], left by each ionic
  // launch for the next, and a device flag that says they match the states (set by the PCG
  // launch after every ionic launch, cleared whenever the states are written from outside)
  void* log_cache = nullptr;
  int* log_valid = nullptr;
  // device arrays (element type double for TC_FP64, float for TC_FP32)
  int32_t *slice_ptr = nullptr, *col = nullptr, *blk_slice = nullptr;
  // per SELL slice, the smallest and largest column it stores (padding included); per PCG block,
  // the window (lo, len) of z it stages in shared memory (len 0: gathers from global memory)
  std::vector<int32_t> slice_cmin, slice_cmax;
  int32_t* blk_win = nullptr;
  size_t pcg_dyn_smem = 0;     // dynamic shared memory of the PCG launch (the largest staged window)
  int pcg_stage = 0;           // stage windows when they fit (TC_PCG_STAGE=1, or chosen by tc_autotune)
  int fuse_ms = 1;             // Mitchell-Schaeffer update inside the PCG launch (TC_FUSE_IONIC=0: own kernel)
  int32_t win_staged = 0, win_max = 0;   // blocks staged, largest window (entries) of the partition
  int pcg_idx16 = 1;           // 16-bit column offsets when every window spans < 65536 (TC_PCG_IDX16=0: off)
  bool use16 = false;
  uint16_t* col16 = nullptr;   // column - lo of the entry's PCG block (padded entries)
  int32_t *comp_of_block = nullptr, *comp_block0 = nullptr;
  void *vM = nullptr, *vK = nullptr, *vA = nullptr, *dinv = nullptr;
  void* V[3] = {nullptr, nullptr, nullptr};
  int iv = 0;   // V[iv] = V^k, V[(iv+2)%3] = V^{k-1}, V[(iv+1)%3] = V^{k+1}
  void *state = nullptr, *g1 = nullptr, *g2 = nullptr;
  void *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr;
  double* act = nullptr;
  double *vpeak = nullptr, *rep90 = nullptr, *lrt = nullptr;
  double v_rest = 0.0, lrt_thr = -70.0;
  double *partA = nullptr, *partB = nullptr;
  GridBar* bar = nullptr;            // n_comp
  int* err = nullptr;
  DevStats* stats = nullptr;         // n_comp
  long long* k_dev = nullptr;        // device step index (start of the current launch group)
  int32_t *stim_off = nullptr, *stim_ids = nullptr;
  StimDev* stims = nullptr;
  std::vector<std::vector<int32_t>> stim_nodes;   // per stimulus, internal indices
  std::vector<StimDev> stim_host;
  // parameters
  double chi = 0, cm = 0, theta = 0, dt = 0;
  double atol = 0.0, rtol = 1e-10;
  int max_iter = 1000;
  double thr = 0.0;
  bool thr_locked = false;
  int model = -1;
  int n_states = 0;
  double ms[7] = {0};
  int cell = 0;
  long long k = 0;
  long long wait_limit = 1ll << 26;
  bool use_graphs = true;
  GraphCache graphs[3];
  // profiling
  bool prof = false;
  tc_profile prof_acc{};
  std::vector<cudaEvent_t> evpool;
  std::vector<Dev> allocs;
  double* pinned = nullptr;   // n_int doubles of page-locked staging for host reads/writes
  void* pinned_t = nullptr;   // n_int elements of the device type, page-locked
  // device-side reordering of host fields: perm (internal -> caller, -1 on padding rows), inv
  // (caller -> internal) and an n-double staging vector in caller order
  int32_t *perm_dev = nullptr, *inv_dev = nullptr;
  double* stage_dev = nullptr;
  // learned ionic surrogate (not owned)
  tc_mlp* sur = nullptr;
  int sur_window = 10;
  float sur_dv_max = 2.0f, sur_dvdt_max = 1.0f, sur_dv_nbr = 0.0f, sur_rest_band = 0.0f;
  uint8_t* sur_flag = nullptr;
  float *sur_iion = nullptr, *sur_raw = nullptr, *sur_zout = nullptr;
  __nv_bfloat16* sur_a0 = nullptr;
  int32_t* sur_idx = nullptr;
  int* sur_count = nullptr;
  unsigned long long* sur_rows = nullptr;   // profiling: candidate rows summed over windows
  unsigned long long* sur_counts = nullptr;
  int* sur_err = nullptr;
};

namespace {

tc_status cuda_fail(cudaError_t e, const char* what) {
  return fail(e == cudaErrorMemoryAllocation ? TC_ERR_NOMEM : TC_ERR_CUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

#define CUDA_TRY(x)                                   \
  do {                                                \
    cudaError_t e_ = (x);                             \
    if (e_ != cudaSuccess) return cuda_fail(e_, #x);  \
  } while (0)

#define TRY(x)                      \
  do {                              \
    tc_status st_ = (x);            \
    if (st_ != TC_OK) return st_;   \
  } while (0)

tc_status dalloc_bytes(tc_sim* s, void** out, size_t bytes) {
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, std::max<size_t>(bytes, 8));
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
  s->allocs.push_back({p, bytes});
  *out = p;
  return TC_OK;
}

template <class T>
tc_status dalloc(tc_sim* s, T** out, size_t count) {
  void* p = nullptr;
  TRY(dalloc_bytes(s, &p, count * sizeof(T)));
  *out = static_cast<T*>(p);
  return TC_OK;
}

void dfree(tc_sim* s, void* p) {
  if (!p) return;
  for (auto it = s->allocs.begin(); it != s->allocs.end(); ++it)
    if (it->p == p) {
      s->allocs.erase(it);
      break;
    }
  cudaFree(p);
}

void drop_graphs(tc_sim* s) {
  for (auto& g : s->graphs) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g = GraphCache{};
  }
}

int64_t round_half_even(double x) { return (int64_t)std::nearbyint(x); }

// Caller-order doubles (staged on the device) -> internal rows of a device field of type T; padding
// rows keep their values.
template <typename T>
__global__ void from_caller_kernel(int64_t n_int, const int32_t* perm, const double* stage, T* dst) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n_int && perm[i] >= 0) dst[i] = T(stage[perm[i]]);
}

// Internal rows of a device field of type T -> caller-order doubles in the staging vector.
template <typename T>
__global__ void to_caller_kernel(int64_t n, const int32_t* inv, const T* src, double* stage) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) stage[j] = double(src[inv[j]]);
}

// Host array in caller order (n doubles) -> device field (element type double when is_double,
// else the simulation's type): one copy into the staging vector, then a reordering kernel.
tc_status write_caller_field(tc_sim* s, void* dst, bool is_double, const double* host) {
  CUDA_TRY(cudaMemcpyAsync(s->stage_dev, host, s->n * sizeof(double), cudaMemcpyHostToDevice, s->stream));
  const unsigned blocks = (unsigned)((s->n_int + 255) / 256);
  if (is_double || s->precision == TC_FP64)
    from_caller_kernel<double><<<blocks, 256, 0, s->stream>>>(s->n_int, s->perm_dev, s->stage_dev,
                                                              static_cast<double*>(dst));
  else
    from_caller_kernel<float><<<blocks, 256, 0, s->stream>>>(s->n_int, s->perm_dev, s->stage_dev,
                                                             static_cast<float*>(dst));
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaStreamSynchronize(s->stream));
  return TC_OK;
}

// Device field -> host array in caller order (n doubles).
tc_status read_caller_field(const tc_sim* s, const void* src, bool is_double, double* host) {
  const unsigned blocks = (unsigned)((s->n + 255) / 256);
  if (is_double || s->precision == TC_FP64)
    to_caller_kernel<double><<<blocks, 256, 0, s->stream>>>(s->n, s->inv_dev, static_cast<const double*>(src),
                                                            s->stage_dev);
  else
    to_caller_kernel<float><<<blocks, 256, 0, s->stream>>>(s->n, s->inv_dev, static_cast<const float*>(src),
                                                           s->stage_dev);
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaMemcpyAsync(host, s->stage_dev, s->n * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  CUDA_TRY(cudaStreamSynchronize(s->stream));
  return TC_OK;
}

// Host doubles in internal order (n_int entries) -> device array of the simulation's type.
// With real_only, only the real rows of every component are written (dummy rows keep theirs).
tc_status upload_vec(tc_sim* s, void* dst, const double* src_internal, bool real_only) {
  CUDA_TRY(cudaStreamSynchronize(s->stream));
  const int64_t n = s->n_int;
  if (s->precision == TC_FP64) {
    std::memcpy(s->pinned_t, src_internal, n * sizeof(double));
  } else {
    float* f = static_cast<float*>(s->pinned_t);
    for (int64_t i = 0; i < n; ++i) f[i] = (float)src_internal[i];
  }
  if (!real_only) {
    CUDA_TRY(cudaMemcpyAsync(dst, s->pinned_t, n * s->esz, cudaMemcpyHostToDevice, s->stream));
  } else {
    for (int c = 0; c < s->n_comp; ++c) {
      const int64_t a = s->comp_rows[c];
      int64_t b = a;
      while (b < s->comp_rows[c + 1] && s->perm[b] >= 0) ++b;   // real rows come first
      if (b > a)
        CUDA_TRY(cudaMemcpyAsync(static_cast<char*>(dst) + a * s->esz,
                                 static_cast<char*>(s->pinned_t) + a * s->esz, (b - a) * s->esz,
                                 cudaMemcpyHostToDevice, s->stream));
    }
  }
  CUDA_TRY(cudaStreamSynchronize(s->stream));
  return TC_OK;
}

tc_status download_vec(const tc_sim* s, const void* src, double* dst_internal) {
  const int64_t n = s->n_int;
  CUDA_TRY(cudaMemcpyAsync(s->pinned_t, src, n * s->esz, cudaMemcpyDeviceToHost, s->stream));
  CUDA_TRY(cudaStreamSynchronize(s->stream));
  if (s->precision == TC_FP64) {
    std::memcpy(dst_internal, s->pinned_t, n * sizeof(double));
  } else {
    const float* f = static_cast<const float*>(s->pinned_t);
    for (int64_t i = 0; i < n; ++i) dst_internal[i] = (double)f[i];
  }
  return TC_OK;
}

// caller order -> internal order (dummy rows get `fill`)
void to_internal(const tc_sim* s, const double* host, double* out, double fill) {
  for (int64_t i = 0; i < s->n_int; ++i) out[i] = s->perm[i] >= 0 ? host[s->perm[i]] : fill;
}

void to_caller(const tc_sim* s, const double* internal, double* host) {
  for (int64_t i = 0; i < s->n_int; ++i)
    if (s->perm[i] >= 0) host[s->perm[i]] = internal[i];
}

tc_status upload_stimuli(tc_sim* s) {
  std::vector<std::vector<int32_t>> per_node(s->n_int);
  for (size_t sid = 0; sid < s->stim_nodes.size(); ++sid)
    for (int32_t i : s->stim_nodes[sid]) per_node[i].push_back((int32_t)sid);
  std::vector<int32_t> off(s->n_int + 1, 0), ids;
  for (int64_t i = 0; i < s->n_int; ++i) {
    off[i + 1] = off[i] + (int32_t)per_node[i].size();
    ids.insert(ids.end(), per_node[i].begin(), per_node[i].end());
  }
  dfree(s, s->stim_ids);
  dfree(s, s->stims);
  s->stim_ids = nullptr;
  s->stims = nullptr;
  TRY(dalloc(s, &s->stim_ids, std::max<size_t>(ids.size(), 1)));
  TRY(dalloc(s, &s->stims, std::max<size_t>(s->stim_host.size(), 1)));
  CUDA_TRY(cudaMemcpyAsync(s->stim_off, off.data(), off.size() * sizeof(int32_t),
                           cudaMemcpyHostToDevice, s->stream));
  if (!ids.empty())
    CUDA_TRY(cudaMemcpyAsync(s->stim_ids, ids.data(), ids.size() * sizeof(int32_t),
                             cudaMemcpyHostToDevice, s->stream));
  if (!s->stim_host.empty())
    CUDA_TRY(cudaMemcpyAsync(s->stims, s->stim_host.data(), s->stim_host.size() * sizeof(StimDev),
                             cudaMemcpyHostToDevice, s->stream));
  CUDA_TRY(cudaStreamSynchronize(s->stream));
  drop_graphs(s);   // graphs hold the old stimulus pointers
  return TC_OK;
}

template <typename T>
const void* pcg_kernel_ptr(int threads) {
  return threads == 1024 ? (const void*)pcg_step_kernel_1024<T>
                         : (const void*)pcg_step_kernel_512<T>;
}

const void* pcg_kernel(const tc_sim* s) {
  return s->precision == TC_FP64 ? pcg_kernel_ptr<double>(s->pcg_threads)
                                 : pcg_kernel_ptr<float>(s->pcg_threads);
}

// Blocks of the cooperative PCG launch: every component gets a contiguous range of blocks in
// proportion to its slices (at least one), and each block a contiguous range of its slices.
tc_status set_partition(tc_sim* s) {
  int bps = 0;
  CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, pcg_kernel(s), s->pcg_threads, 0));
  if (bps < 1) return fail(TC_ERR_CUDA, "PCG kernel cannot be resident on an SM");
  const int per_sm = std::min(bps, std::max(1, s->blocks_per_sm));
  const int64_t max_blocks = (int64_t)per_sm * s->num_sms;
  if (s->n_comp > max_blocks)
    return fail(TC_ERR_ARG, "mesh has " + std::to_string(s->n_comp) +
                                " connected components, more than the " +
                                std::to_string(max_blocks) + " co-resident PCG blocks");
  const int warps = s->pcg_threads / 32;
  std::vector<int64_t> cs(s->n_comp), want(s->n_comp);
  int64_t total_want = 0, total_slices = 0;
  for (int c = 0; c < s->n_comp; ++c) {
    cs[c] = (s->comp_rows[c + 1] - s->comp_rows[c]) / 32;
    want[c] = std::max<int64_t>(1, (cs[c] + warps - 1) / warps);   // >= one slice per warp
    total_want += want[c];
    total_slices += cs[c];
  }
  std::vector<int64_t> nbc(s->n_comp);
  if (total_want <= max_blocks) {
    nbc = want;
  } else {
    // share max_blocks in proportion to slices, at least one block per component
    int64_t used = 0;
    for (int c = 0; c < s->n_comp; ++c) {
      nbc[c] = std::max<int64_t>(1, std::min(want[c], (max_blocks * cs[c]) / std::max<int64_t>(total_slices, 1)));
      used += nbc[c];
    }
    while (used > max_blocks) {   // trim the largest shares
      const int c = (int)(std::max_element(nbc.begin(), nbc.end()) - nbc.begin());
      nbc[c] -= 1;
      used -= 1;
    }
    for (int c = 0; used < max_blocks; c = (c + 1) % s->n_comp) {   // hand out the rest
      if (nbc[c] < want[c]) {
        nbc[c] += 1;
        used += 1;
      }
      if (c == s->n_comp - 1) {
        bool any = false;
        for (int d = 0; d < s->n_comp; ++d) any |= nbc[d] < want[d];
        if (!any) break;
      }
    }
  }
  std::vector<int32_t> bs, cob, cb0(s->n_comp + 1, 0);
  for (int c = 0; c < s->n_comp; ++c) {
    const int64_t first_slice = s->comp_rows[c] / 32;
    for (int64_t b = 0; b < nbc[c]; ++b) {
      bs.push_back((int32_t)(first_slice + cs[c] * b / nbc[c]));
      cob.push_back(c);
    }
    cb0[c + 1] = cb0[c] + (int32_t)nbc[c];
  }
  bs.push_back((int32_t)(s->n_int / 32));
  s->nblocks = cb0[s->n_comp];
  // Shared-memory windows of z: a block's gathers touch the columns between the smallest and
  // largest column of its slices (under RCM a band about the block's rows).  The window is
  // aligned to 4 entries (16-byte vectors) and staged when it fits the shared memory left per
  // block at this launch shape; the dynamic shared memory of the launch is the largest staged one.
  std::vector<int32_t> win(2 * (size_t)s->nblocks, 0);
  size_t dyn = 0;
  int64_t span_max = INT64_MAX;   // widest column range of a block (16-bit offsets need < 65536)
  s->win_staged = 0;
  s->win_max = 0;
  if (!s->slice_cmin.empty()) {
    cudaFuncAttributes fa{};
    CUDA_TRY(cudaFuncGetAttributes(&fa, pcg_kernel(s)));
    int sm_per_sm = 0, sm_optin = 0;
    CUDA_TRY(cudaDeviceGetAttribute(&sm_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, s->device));
    CUDA_TRY(cudaDeviceGetAttribute(&sm_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, s->device));
    const int64_t per_block = std::min<int64_t>(sm_optin, sm_per_sm / per_sm - 1024) - (int64_t)fa.sharedSizeBytes;
    int64_t cap = per_block > 0 ? (per_block / (int64_t)s->esz) / 4 * 4 : 0;
    // TC_PCG_STAGE_CAP (entries) lowers the capacity, so that tests can mix staged and unstaged blocks
    const int env_cap = env_int("TC_PCG_STAGE_CAP", 0);
    if (env_cap > 0) cap = std::min<int64_t>(cap, env_cap);
    int64_t used = 0;
    span_max = 0;
    for (int b = 0; b < s->nblocks; ++b) {
      int32_t lo = INT32_MAX, hi = -1;
      for (int32_t sl = bs[b]; sl < bs[b + 1]; ++sl) {
        lo = std::min(lo, s->slice_cmin[sl]);
        hi = std::max(hi, s->slice_cmax[sl]);
      }
      if (hi < 0) continue;
      lo = lo / 4 * 4;
      const int64_t len = std::min<int64_t>(((int64_t)hi + 1 - lo + 3) / 4 * 4, s->n_int - lo);
      s->win_max = std::max<int32_t>(s->win_max, (int32_t)len);
      span_max = std::max<int64_t>(span_max, (int64_t)hi + 1 - lo);
      win[2 * b] = lo;
      if (s->pcg_stage && len <= cap) {
        win[2 * b + 1] = (int32_t)len;
        used = std::max(used, len);
        s->win_staged += 1;
      }
    }
    dyn = (size_t)used * s->esz;
    if (dyn > 0) {
      CUDA_TRY(cudaFuncSetAttribute(pcg_kernel(s), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
      int bps2 = 0;
      CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps2, pcg_kernel(s), s->pcg_threads, dyn));
      if (bps2 < per_sm) {   // cannot stay co-resident with the windows: gather from global memory
        for (int b = 0; b < s->nblocks; ++b) win[2 * b + 1] = 0;
        dyn = 0;
        s->win_staged = 0;
      }
    }
  }
  s->pcg_dyn_smem = dyn;
  for (void* p : {(void*)s->blk_slice, (void*)s->partA, (void*)s->partB, (void*)s->comp_of_block,
                  (void*)s->comp_block0, (void*)s->blk_win})
    dfree(s, p);
  TRY(dalloc(s, &s->blk_win, win.size()));
  CUDA_TRY(cudaMemcpy(s->blk_win, win.data(), win.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  TRY(dalloc(s, &s->blk_slice, bs.size()));
  TRY(dalloc(s, &s->comp_of_block, cob.size()));
  TRY(dalloc(s, &s->comp_block0, cb0.size()));
  TRY(dalloc(s, &s->partA, s->nblocks));
  TRY(dalloc(s, &s->partB, 2 * s->nblocks));
  CUDA_TRY(cudaMemcpy(s->blk_slice, bs.data(), bs.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(s->comp_of_block, cob.data(), cob.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(s->comp_block0, cb0.data(), cb0.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  // 16-bit column offsets from each block's window start (the index stream of the RHS pass and
  // the A-products at half the bytes), when every block's columns span fewer than 65,536 entries
  s->use16 = s->pcg_idx16 && span_max <= 65536 && s->padded > 0;
  if (s->use16) {
    if (!s->col16) TRY(dalloc(s, &s->col16, (size_t)s->padded));
    col16_kernel<<<s->nblocks, 256, 0, s->stream>>>(s->blk_slice, s->slice_ptr, s->col, s->blk_win, s->col16);
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaStreamSynchronize(s->stream));
  }
  drop_graphs(s);
  return TC_OK;
}

cudaEvent_t pooled_event(tc_sim* s, size_t idx) {
  while (s->evpool.size() <= idx) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    s->evpool.push_back(e);
  }
  return s->evpool[idx];
}

template <typename T>
tc_status upload_matrices(tc_sim* s, const Sell& sell, const std::vector<double>& mv,
                          const std::vector<double>& kv, const std::vector<double>& av,
                          const std::vector<double>& dinv) {
  std::vector<T> hM(sell.padded), hK(sell.padded), hA(sell.padded), hd(s->n_int);
  for (int64_t e = 0; e < sell.padded; ++e) {
    const int64_t q = sell.src[e];
    hM[e] = q >= 0 ? (T)mv[q] : T(0);
    hK[e] = q >= 0 ? (T)kv[q] : T(0);
    hA[e] = q >= 0 ? (T)av[q] : T(0);
  }
  for (int64_t i = 0; i < s->n_int; ++i) hd[i] = (T)dinv[i];
  CUDA_TRY(cudaMemcpy(s->vM, hM.data(), sell.padded * sizeof(T), cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(s->vK, hK.data(), sell.padded * sizeof(T), cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(s->vA, hA.data(), sell.padded * sizeof(T), cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(s->dinv, hd.data(), s->n_int * sizeof(T), cudaMemcpyHostToDevice));
  return TC_OK;
}

// Launch one time step (ionic kernel, then the cooperative PCG kernel) for the buffer phase
// `iv` and step offset `k_off` from the device step index.
template <typename T>
tc_status launch_step(tc_sim* s, int iv, int k_off, size_t* ev, std::vector<size_t>* marks) {
  T* Vc = static_cast<T*>(s->V[iv]);
  T* Vp = static_cast<T*>(s->V[(iv + 2) % 3]);
  T* Vn = static_cast<T*>(s->V[(iv + 1) % 3]);
  IonicArgs<T> ia;
  ia.n = s->n_int;
  ia.V = Vc;
  ia.Vp = Vp;
  ia.state = static_cast<T*>(s->state);
  ia.g1 = static_cast<T*>(s->g1);
  ia.g2 = static_cast<T*>(s->g2);
  ia.x0 = Vn;
  ia.stim_off = s->stim_off;
  ia.stim_ids = s->stim_ids;
  ia.stims = s->stims;
  ia.k_base = s->k_dev;
  ia.k_off = k_off;
  ia.chi = s->chi;
  ia.cm = s->cm;
  ia.dt = s->dt;
  ia.theta = s->theta;
  const double range = s->ms[6] - s->ms[5];
  ia.ms.vmin = s->ms[5];
  ia.ms.inv_range = range != 0.0 ? 1.0 / range : 0.0;
  ia.ms.range = range;
  ia.ms.vgate = s->ms[4];
  ia.ms.inv_tau_in = s->ms[0] != 0.0 ? 1.0 / s->ms[0] : 0.0;
  ia.ms.inv_tau_out = s->ms[1] != 0.0 ? 1.0 / s->ms[1] : 0.0;
  ia.ms.dec_open = s->ms[2] != 0.0 ? std::exp(-s->dt / s->ms[2]) : 0.0;
  ia.ms.dec_close = s->ms[3] != 0.0 ? std::exp(-s->dt / s->ms[3]) : 0.0;
  ia.cell = s->cell;
  ia.bar = s->bar;
  ia.n_bar = s->n_comp;
  ia.sur_flag = s->sur ? s->sur_flag : nullptr;
  ia.sur_iion = s->sur ? s->sur_iion : nullptr;
  ia.log_cache = s->model == TC_MODEL_TP06 && s->precision == TC_FP64 && s->log_cache
                     ? static_cast<T*>(s->log_cache)
                     : nullptr;
  ia.log_valid = s->log_valid;
  if (ev) {
    cudaEvent_t e = pooled_event(s, *ev);
    if (!e) return fail(TC_ERR_CUDA, "cudaEventCreate failed");
    CUDA_TRY(cudaEventRecord(e, s->stream));
    marks->push_back((*ev)++);
  }
  const int ion_blocks = (int)((s->n_int + kIonicThreads - 1) / kIonicThreads);
  const bool fused = s->model == TC_MODEL_MS && s->fuse_ms;
  if (fused) {
    // one launch per step: the update runs as the first phase of the PCG kernel below
  } else if (s->model == TC_MODEL_MS) {
    ionic_ms_kernel<T><<<ion_blocks, kIonicThreads, 0, s->stream>>>(ia);
  } else {
    const int tpb = Tp06Launch<T>::threads;
    ionic_tp06_kernel<T><<<(unsigned)((s->n_int + tpb - 1) / tpb), tpb, 0, s->stream>>>(ia);
  }
  CUDA_TRY(cudaGetLastError());
  PcgArgs<T> pa;
  pa.n = s->n_int;
  pa.slice_ptr = s->slice_ptr;
  pa.col = s->col;
  pa.vM = static_cast<const T*>(s->vM);
  pa.vK = static_cast<const T*>(s->vK);
  pa.vA = static_cast<const T*>(s->vA);
  pa.dinv = static_cast<const T*>(s->dinv);
  pa.blk_slice = s->blk_slice;
  pa.blk_win = s->blk_win;
  pa.col16 = s->use16 ? s->col16 : nullptr;
  pa.comp_of_block = s->comp_of_block;
  pa.comp_block0 = s->comp_block0;
  pa.g1 = static_cast<const T*>(s->g1);
  pa.g2 = static_cast<const T*>(s->g2);
  pa.x = Vn;
  pa.Vcur = Vc;
  pa.r = static_cast<T*>(s->r);
  pa.z = static_cast<T*>(s->z);
  pa.p = static_cast<T*>(s->p);
  pa.q = static_cast<T*>(s->q);
  pa.act = s->act;
  pa.vpeak = s->vpeak;
  pa.rep90 = s->rep90;
  pa.lrt = s->lrt;
  pa.v_rest = s->v_rest;
  pa.lrt_thr = s->lrt_thr;
  pa.partA = s->partA;
  pa.partB = s->partB;
  pa.bar = s->bar;
  pa.err = s->err;
  pa.stats = s->stats;
  pa.atol = s->atol;
  pa.rtol = s->rtol;
  pa.max_iter = s->max_iter;
  pa.wait_limit = s->wait_limit;
  pa.l2_keep = s->l2_keep;
  pa.log_valid = ia.log_cache ? s->log_valid : nullptr;
  pa.k_base = s->k_dev;
  pa.k_off = k_off;
  pa.dt = s->dt;
  pa.thr = s->thr;
  pa.fuse_ms = fused ? 1 : 0;
  pa.ion = ia;
  if (ev) {
    CUDA_TRY(cudaEventRecord(pooled_event(s, *ev), s->stream));
    (*ev)++;
  }
  void* args[] = {&pa};
  CUDA_TRY(cudaLaunchCooperativeKernel(pcg_kernel(s), s->nblocks, s->pcg_threads, args, s->pcg_dyn_smem,
                                       s->stream));
  if (ev) {
    CUDA_TRY(cudaEventRecord(pooled_event(s, *ev), s->stream));
    (*ev)++;
  }
  return TC_OK;
}

tc_status launch_step_any(tc_sim* s, int iv, int k_off, size_t* ev, std::vector<size_t>* marks) {
  return s->precision == TC_FP64 ? launch_step<double>(s, iv, k_off, ev, marks)
                                 : launch_step<float>(s, iv, k_off, ev, marks);
}

__global__ void add_count_kernel(const int* count, unsigned long long* acc) { *acc += (unsigned long long)*count; }

// Surrogate inference at the start of a window: step *k_dev + k_off at buffer phase iv.  With
// ev (profiling), four pooled events bracket the inference and its network; their first index is
// appended to marks.
tc_status launch_surrogate(tc_sim* s, int iv, int k_off, size_t* ev = nullptr,
                           std::vector<size_t>* marks = nullptr) {
  SurrogateStep q;
  if (ev) {
    for (int e = 0; e < 4; ++e)
      if (!pooled_event(s, *ev + e)) return fail(TC_ERR_CUDA, "cudaEventCreate failed");
    q.ev_mlp[0] = s->evpool[*ev + 1];
    q.ev_mlp[1] = s->evpool[*ev + 2];
    CUDA_TRY(cudaEventRecord(s->evpool[*ev], s->stream));
  }
  q.n = s->n_int;
  q.fp64 = s->precision == TC_FP64;
  q.state = s->state;
  q.V = s->V[iv];
  q.Vprev = s->V[(iv + 2) % 3];
  q.dinv = s->dinv;
  q.log_cache = q.fp64 && s->log_cache ? static_cast<double*>(s->log_cache) : nullptr;
  q.stim_off = s->stim_off;
  q.stim_ids = s->stim_ids;
  q.stims = s->stims;
  q.k_base = s->k_dev;
  q.k_off = k_off;
  q.win = s->sur_window;
  q.cm = s->cm;
  q.dt = s->dt;
  q.dv_max = s->sur_dv_max;
  q.dvdt_max = s->sur_dvdt_max;
  q.dv_nbr = s->sur_dv_nbr;
  q.v_rest = (float)s->v_rest;
  q.rest_band = s->sur_rest_band;
  q.slice_ptr = s->slice_ptr;
  q.col = s->col;
  q.a0 = s->sur_a0;
  q.idx = s->sur_idx;
  q.count = s->sur_count;
  q.raw = s->sur_raw;
  q.zout = s->sur_zout;
  q.flag = s->sur_flag;
  q.iion = s->sur_iion;
  q.counts = s->sur_counts;
  q.err = s->sur_err;
  TRY(surrogate_infer(s->sur, q, s->stream));
  if (ev) {
    add_count_kernel<<<1, 1, 0, s->stream>>>(s->sur_count, s->sur_rows);
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaEventRecord(s->evpool[*ev + 3], s->stream));
    marks->push_back(*ev);
    *ev += 4;
  }
  return TC_OK;
}

// Capture kGraphSteps steps starting at buffer phase iv, followed by the index advance.  With
// the surrogate attached the group starts on a window boundary and kGraphSteps is a multiple of
// the window, so the inference sits at fixed offsets inside the graph.
tc_status capture_graph(tc_sim* s, int iv, cudaGraphExec_t* out) {
  cudaStream_t cs;
  CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaStream_t saved = s->stream;
  s->stream = cs;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  tc_status st = TC_OK;
  if (e == cudaSuccess) {
    for (int j = 0; j < kGraphSteps && st == TC_OK; ++j) {
      if (s->sur && j % s->sur_window == 0) st = launch_surrogate(s, (iv + j) % 3, j);
      if (st == TC_OK) st = launch_step_any(s, (iv + j) % 3, j, nullptr, nullptr);
    }
    if (st == TC_OK) {
      tick_kernel<<<1, 1, 0, cs>>>(s->k_dev, kGraphSteps);
      e = cudaGetLastError();
    }
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(cs, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess && st == TC_OK) e = cudaGraphInstantiate(out, g, 0);
    if (g) cudaGraphDestroy(g);
  }
  s->stream = saved;
  cudaStreamDestroy(cs);
  if (st != TC_OK) return st;
  if (e != cudaSuccess) {
    cudaGetLastError();   // clear a sticky-free capture error
    return cuda_fail(e, "graph capture of the step loop");
  }
  return TC_OK;
}

struct Snapshot {
  std::vector<void*> bufs;
  long long k;
  int iv;
};

// ---- training pairs for the learned surrogate, drawn from the tissue's current state ----------

template <typename T>
struct SampleArgs {
  int64_t n;
  const T* state;               // [18][n]
  const T* V;                   // V^k
  const T* Vp;                  // V^{k-1}
  const T* dinv;                // 0 on padding rows
  const int32_t *stim_off, *stim_ids;
  const StimDev* stims;
  long long k0;
  int win, cell;
  double cm, dt, v_rest, rest_band, rest_keep, dv_keep, dvdt_keep;
  uint64_t seed;
  uint8_t* keep;                // [n] decision of the first pass
  uint32_t* blk_count;          // [blocks]
  const uint32_t* blk_off;      // [blocks + 1] exclusive offsets, total last
  float* x;                     // [capacity][20]
  float* y;                     // [capacity][19]
  int64_t base, capacity;
};

// Features of node i (18 states, V, stimulus averaged over the window in pA/pF) as the FP32
// values the network sees, and the exact cell's state after the window from them, in FP64.
template <typename T>
__device__ __forceinline__ void sample_window(const SampleArgs<T>& a, int64_t i, float* f, double* u, double& V) {
  const int64_t n = a.n;
  for (int j = 0; j < kTP06States; ++j) f[j] = (float)a.state[j * n + i];
  f[18] = (float)a.V[i];
  double is = 0.0;
  for (int s = 0; s < a.win; ++s) is += stimulus_at(a.stim_off, a.stim_ids, a.stims, i, a.k0 + s);
  f[19] = (float)(is / a.win / a.cm);
  for (int j = 0; j < kTP06States; ++j) u[j] = (double)f[j];
  V = (double)f[18];
  for (int s = 0; s < a.win; ++s) {
    const double iion = tp06_cell_step(V, u, a.cell, a.dt);
    V += a.dt * ((double)f[19] - iion);
  }
}

// A node is sampled unless it is a padding row, moved faster than dvdt_keep on the step before
// the window (when dvdt_keep > 0), or its exact window changes V by more than dv_keep (when
// dv_keep > 0) - the windows a deployed surrogate hands to the exact model anyway; a node within
// rest_band of the resting potential is kept only with probability rest_keep, by a counter-based
// draw (resting cells dominate a tissue and carry little information about the dynamics).
template <typename T>
__global__ void __launch_bounds__(256) sample_select_kernel(const SampleArgs<T> a) {
  exp2_table_init();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool keep = i < a.n && a.dinv[i] != T(0);
  if (keep && a.dvdt_keep > 0) keep = fabs((double)a.V[i] - (double)a.Vp[i]) <= a.dvdt_keep * a.dt;
  if (keep && fabs((double)a.V[i] - a.v_rest) <= a.rest_band) {
    uint64_t z = a.seed + (uint64_t)a.k0 * 0xD1B54A32D192ED03ull + (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    keep = (double)(z >> 11) * (1.0 / 9007199254740992.0) < a.rest_keep;
  }
  if (keep && a.dv_keep > 0) {
    float f[20];
    double u[kTP06States], V;
    sample_window(a, i, f, u, V);
    keep = fabs(V - (double)f[18]) <= a.dv_keep;
  }
  if (i < a.n) a.keep[i] = keep ? 1 : 0;
  const int c = __syncthreads_count(keep);
  if (threadIdx.x == 0) a.blk_count[blockIdx.x] = (uint32_t)c;
}

// Exclusive scan of the per-block counts (one block; fixed order).
__global__ void __launch_bounds__(1024) sample_scan_kernel(int nb, const uint32_t* cnt, uint32_t* off) {
  __shared__ uint32_t part[1024];
  const int t = threadIdx.x;
  const int per = (nb + 1023) / 1024;
  const int lo = min(nb, t * per), hi = min(nb, lo + per);
  uint32_t s = 0;
  for (int b = lo; b < hi; ++b) s += cnt[b];
  part[t] = s;
  __syncthreads();
  if (t == 0) {
    uint32_t run = 0;
    for (int j = 0; j < 1024; ++j) {
      const uint32_t v = part[j];
      part[j] = run;
      run += v;
    }
    off[nb] = run;
  }
  __syncthreads();
  uint32_t run = part[t];
  for (int b = lo; b < hi; ++b) {
    off[b] = run;
    run += cnt[b];
  }
}

// Kept nodes write their pair at base + (rank among kept nodes in internal order).
template <typename T>
__global__ void __launch_bounds__(256) sample_write_kernel(const SampleArgs<T> a) {
  exp2_table_init();
  __shared__ uint32_t warp_base[8];
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool keep = i < a.n && a.keep[i];
  const unsigned m = __ballot_sync(0xffffffffu, keep);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) warp_base[w] = __popc(m);
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t run = 0;
    for (int j = 0; j < 8; ++j) {
      const uint32_t v = warp_base[j];
      warp_base[j] = run;
      run += v;
    }
  }
  __syncthreads();
  if (!keep) return;
  const int64_t pos = a.base + a.blk_off[blockIdx.x] + warp_base[w] + __popc(m & ((1u << lane) - 1u));
  if (pos >= a.capacity) return;
  float f[20];
  double u[kTP06States], V;
  sample_window(a, i, f, u, V);
  float* xr = a.x + pos * 20;
  for (int j = 0; j < 20; ++j) xr[j] = f[j];
  float* yr = a.y + pos * 19;
  for (int j = 0; j < kTP06States; ++j) yr[j] = (float)u[j];
  yr[18] = (float)V;
}

template <typename T>
tc_status surrogate_sample_t(tc_sim* s, int win, double rest_band, double rest_keep, double dv_keep,
                             double dvdt_keep, uint64_t seed, float* x, float* y, int64_t capacity,
                             int64_t* count) {
  const int64_t n = s->n_int;
  const int nb = (int)((n + 255) / 256);
  uint32_t* cnt = nullptr;
  const size_t words = (size_t)(2 * nb + 1) + (size_t)(n + 3) / 4;
  CUDA_TRY(cudaMallocAsync(&cnt, words * sizeof(uint32_t), s->stream));
  SampleArgs<T> a{};
  a.n = n;
  a.state = static_cast<const T*>(s->state);
  a.V = static_cast<const T*>(s->V[s->iv]);
  a.Vp = static_cast<const T*>(s->V[(s->iv + 2) % 3]);
  a.dinv = static_cast<const T*>(s->dinv);
  a.stim_off = s->stim_off;
  a.stim_ids = s->stim_ids;
  a.stims = s->stims;
  a.k0 = s->k;
  a.win = win;
  a.cell = s->cell;
  a.cm = s->cm;
  a.dt = s->dt;
  a.v_rest = s->v_rest;
  a.rest_band = rest_band;
  a.rest_keep = rest_keep;
  a.dv_keep = dv_keep;
  a.dvdt_keep = dvdt_keep;
  a.seed = seed;
  a.blk_count = cnt;
  a.blk_off = cnt + nb;
  a.keep = reinterpret_cast<uint8_t*>(cnt + 2 * nb + 1);
  a.x = x;
  a.y = y;
  a.base = *count;
  a.capacity = capacity;
  sample_select_kernel<T><<<nb, 256, 0, s->stream>>>(a);
  sample_scan_kernel<<<1, 1024, 0, s->stream>>>(nb, cnt, cnt + nb);
  sample_write_kernel<T><<<nb, 256, 0, s->stream>>>(a);
  uint32_t total = 0;
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&total, cnt + 2 * nb, sizeof(uint32_t), cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaFreeAsync(cnt, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "surrogate sampling");
  *count = std::min<int64_t>(capacity, *count + (int64_t)total);
  return TC_OK;
}

}  // namespace

extern "C" {

tc_status tc_assemble(const tc_mesh* mesh, const double* sigma_l, const double* sigma_t,
                      int32_t n_regions, double chi, double cm, double theta, double dt,
                      int32_t precision, void* cuda_stream, tc_sim** out) {
  clear_error();
  if (!out) return fail(TC_ERR_ARG, "out must not be NULL");
  *out = nullptr;
  if (!mesh) return fail(TC_ERR_ARG, "mesh must not be NULL");
  if (!(chi > 0) || !(cm > 0) || !(dt > 0) || !(theta >= 0.0 && theta <= 1.0) ||
      !std::isfinite(chi) || !std::isfinite(cm) || !std::isfinite(dt))
    return fail(TC_ERR_ARG, "need chi > 0, cm > 0, dt > 0 and 0 <= theta <= 1");
  if (precision != TC_FP64 && precision != TC_FP32)
    return fail(TC_ERR_ARG, "precision must be TC_FP64 or TC_FP32, got " + std::to_string(precision));
  std::vector<double> mv, kv;
  try {
    TRY(assemble_mk(*mesh, sigma_l, sigma_t, n_regions, mv, kv));
  } catch (const std::bad_alloc&) {
    return fail(TC_ERR_NOMEM, "out of host memory");
  }
  tc_sim* s = new (std::nothrow) tc_sim();
  if (!s) return fail(TC_ERR_NOMEM, "out of host memory");
  auto bail = [&](tc_status st) {
    tc_sim_destroy(s);
    return st;
  };
  s->stream = static_cast<cudaStream_t>(cuda_stream);
  s->chi = chi;
  s->cm = cm;
  s->theta = theta;
  s->dt = dt;
  s->precision = precision;
  s->esz = precision == TC_FP64 ? sizeof(double) : sizeof(float);
  s->n = mesh->n;
  const Csr& pat = mesh->pattern;
  s->nnz = pat.row_ptr[mesh->n];
  s->pcg_threads = env_int("TC_PCG_THREADS", 1024) == 512 ? 512 : 1024;
  s->blocks_per_sm = std::max(1, env_int("TC_PCG_BLOCKS_PER_SM", s->pcg_threads == 1024 ? 1 : 2));
  s->sell_sigma = mesh->sell_sigma > 0 ? mesh->sell_sigma : std::max(1, env_int("TC_SELL_SIGMA", 1024));
  s->use_graphs = env_int("TC_GRAPHS", 1) != 0;
  Sell sell;
  std::vector<double> av, hdinv;
  try {
    padded_ordering(pat, s->sell_sigma, s->perm, s->comp_rows);
    s->n_int = (int64_t)s->perm.size();
    s->n_comp = (int)s->comp_rows.size() - 1;
    tc_status st = build_sell(pat, s->perm, sell);
    if (st != TC_OK) return bail(st);
    s->inv.assign(s->n, -1);
    for (int64_t i = 0; i < s->n_int; ++i)
      if (s->perm[i] >= 0) s->inv[s->perm[i]] = (int32_t)i;
    // A = chi Cm M + theta dt K, entry by entry (Eq. 3): two products, then the sum
    const double c1 = chi * cm, c2 = theta * dt;
    av.resize(s->nnz);
    for (int64_t q = 0; q < s->nnz; ++q) {
      volatile double t1 = c1 * mv[q];
      volatile double t2 = c2 * kv[q];
      av[q] = t1 + t2;
    }
    hdinv.assign(s->n_int, 0.0);   // dummy rows: zero inverse, so they never move
    for (int64_t i = 0; i < s->n_int; ++i) {
      const int32_t o = s->perm[i];
      if (o < 0) continue;
      const int32_t* cb = &pat.col[pat.row_ptr[o]];
      const int64_t len = pat.row_ptr[o + 1] - pat.row_ptr[o];
      const int64_t d = std::lower_bound(cb, cb + len, o) - cb;
      hdinv[i] = 1.0 / av[pat.row_ptr[o] + d];
    }
  } catch (const std::bad_alloc&) {
    return bail(fail(TC_ERR_NOMEM, "out of host memory"));
  }
  s->nslices = sell.nslices;
  s->padded = sell.padded;
  s->pcg_stage = env_int("TC_PCG_STAGE", 0) != 0;
  s->fuse_ms = env_int("TC_FUSE_IONIC", 1) != 0;
  s->pcg_idx16 = env_int("TC_PCG_IDX16", 1) != 0;
  try {
    s->slice_cmin.assign(sell.nslices, INT32_MAX);
    s->slice_cmax.assign(sell.nslices, -1);
    for (int64_t sl = 0; sl < sell.nslices; ++sl)
      for (int64_t e = sell.slice_ptr[sl]; e < sell.slice_ptr[sl + 1]; ++e) {
        s->slice_cmin[sl] = std::min(s->slice_cmin[sl], sell.col[e]);
        s->slice_cmax[sl] = std::max(s->slice_cmax[sl], sell.col[e]);
      }
  } catch (const std::bad_alloc&) {
    return bail(fail(TC_ERR_NOMEM, "out of host memory"));
  }
  cudaError_t ce = cudaGetDevice(&s->device);
  if (ce != cudaSuccess) return bail(cuda_fail(ce, "cudaGetDevice"));
  ce = cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, s->device);
  if (ce != cudaSuccess) return bail(cuda_fail(ce, "cudaDeviceGetAttribute"));
  {
    // FP64: the A-product streams A and the index array every iteration; keep about 35 % of L2
    // worth of their lines resident (evict-last) and let the rest pass (evict-first): 8 % faster
    // PCG on the 40x16x6 mm slab (half of its 89 MB).  FP32 keeps its whole working set in L2.
    int l2 = 0;
    cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, s->device);
    const double bytes = (double)sell.padded * (s->precision == TC_FP64 ? 12.0 : 8.0);
    s->l2_keep = s->precision == TC_FP64 && l2 > 0 ? (float)std::min(0.5, 0.35 * l2 / bytes) : 0.f;
  }
  int coop = 0;
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, s->device);
  if (!coop) return bail(fail(TC_ERR_CUDA, "device does not support cooperative launches"));
  tc_status st = TC_OK;
  const int64_t n = s->n_int;
  const size_t E = s->esz;
#define ALLOCB(ptr, bytes)                                 \
  do {                                                     \
    st = dalloc_bytes(s, (void**)&(ptr), (size_t)(bytes)); \
    if (st != TC_OK) return bail(st);                      \
  } while (0)
  ALLOCB(s->slice_ptr, (s->nslices + 1) * sizeof(int32_t));
  ALLOCB(s->col, sell.padded * sizeof(int32_t));
  ALLOCB(s->vM, sell.padded * E);
  ALLOCB(s->vK, sell.padded * E);
  ALLOCB(s->vA, sell.padded * E);
  ALLOCB(s->dinv, n * E);
  for (int j = 0; j < 3; ++j) ALLOCB(s->V[j], n * E);
  ALLOCB(s->g1, n * E);
  ALLOCB(s->g2, n * E);
  ALLOCB(s->r, n * E);
  ALLOCB(s->z, n * E);
  ALLOCB(s->p, n * E);
  ALLOCB(s->q, n * E);
  ALLOCB(s->act, n * sizeof(double));
  ALLOCB(s->vpeak, n * sizeof(double));
  ALLOCB(s->rep90, n * sizeof(double));
  ALLOCB(s->lrt, n * sizeof(double));
  ALLOCB(s->bar, s->n_comp * sizeof(GridBar));
  ALLOCB(s->err, sizeof(int));
  ALLOCB(s->stats, s->n_comp * sizeof(DevStats));
  ALLOCB(s->k_dev, sizeof(long long));
  ALLOCB(s->stim_off, (n + 1) * sizeof(int32_t));
#undef ALLOCB
  ce = cudaMemcpy(s->slice_ptr, sell.slice_ptr.data(), (s->nslices + 1) * sizeof(int32_t),
                  cudaMemcpyHostToDevice);
  if (ce == cudaSuccess)
    ce = cudaMemcpy(s->col, sell.col.data(), sell.padded * sizeof(int32_t), cudaMemcpyHostToDevice);
  if (ce != cudaSuccess) return bail(cuda_fail(ce, "cudaMemcpy"));
  st = precision == TC_FP64 ? upload_matrices<double>(s, sell, mv, kv, av, hdinv)
                            : upload_matrices<float>(s, sell, mv, kv, av, hdinv);
  if (st != TC_OK) return bail(st);
  ce = cudaMemset(s->bar, 0, s->n_comp * sizeof(GridBar));
  if (ce == cudaSuccess) ce = cudaMemset(s->err, 0, sizeof(int));
  if (ce == cudaSuccess) ce = cudaMemset(s->stats, 0, s->n_comp * sizeof(DevStats));
  if (ce == cudaSuccess) ce = cudaMemset(s->k_dev, 0, sizeof(long long));
  if (ce == cudaSuccess) ce = cudaMemset(s->stim_off, 0, (n + 1) * sizeof(int32_t));
  if (ce == cudaSuccess) ce = cudaMemset(s->act, 0, n * sizeof(double));
  if (ce != cudaSuccess) return bail(cuda_fail(ce, "cudaMemset"));
  ce = cudaMallocHost(&s->pinned, n * sizeof(double));
  if (ce == cudaSuccess) ce = cudaMallocHost(&s->pinned_t, n * sizeof(double));
  if (ce != cudaSuccess) return bail(cuda_fail(ce, "cudaMallocHost"));
  st = dalloc(s, &s->perm_dev, n);
  if (st == TC_OK) st = dalloc(s, &s->inv_dev, s->n);
  if (st == TC_OK) st = dalloc(s, &s->stage_dev, s->n);
  if (st != TC_OK) return bail(st);
  ce = cudaMemcpy(s->perm_dev, s->perm.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice);
  if (ce == cudaSuccess) ce = cudaMemcpy(s->inv_dev, s->inv.data(), s->n * sizeof(int32_t), cudaMemcpyHostToDevice);
  if (ce != cudaSuccess) return bail(cuda_fail(ce, "cudaMemcpy"));
  st = set_partition(s);
  if (st != TC_OK) return bail(st);
  st = upload_stimuli(s);
  if (st != TC_OK) return bail(st);
  *out = s;
  return TC_OK;
}

// The PCG marks part of A and the index array evict-last in L2 (FP64); after a tc_step call
// (and before the memory is freed) their lines go back to the normal priority so that they do
// not crowd out other work's data.
static cudaError_t l2_release(tc_sim* s) {
  if (!(s->l2_keep > 0.f)) return cudaSuccess;
  const int64_t lines_a = s->padded * 8 / 128, lines_c = s->padded * 4 / 128;
  l2_normal_priority_kernel<<<(unsigned)((lines_a + 255) / 256), 256, 0, s->stream>>>(
      static_cast<const char*>(s->vA), lines_a);
  l2_normal_priority_kernel<<<(unsigned)((lines_c + 255) / 256), 256, 0, s->stream>>>(
      reinterpret_cast<const char*>(s->col), lines_c);
  return cudaGetLastError();
}

void tc_sim_destroy(tc_sim* s) {
  if (!s) return;
  cudaSetDevice(s->device);
  l2_release(s);
  cudaStreamSynchronize(s->stream);
  drop_graphs(s);
  for (auto& d : s->allocs) cudaFree(d.p);
  for (cudaEvent_t e : s->evpool) cudaEventDestroy(e);
  if (s->pinned) cudaFreeHost(s->pinned);
  if (s->pinned_t) cudaFreeHost(s->pinned_t);
  delete s;
}

tc_status tc_sim_size(const tc_sim* s, int64_t* n_nodes, int64_t* nnz, int64_t* padded_nnz,
                      int32_t* n_blocks) {
  clear_error();
  if (!s) return fail(TC_ERR_ARG, "sim must not be NULL");
  if (n_nodes) *n_nodes = s->n;
  if (nnz) *nnz = s->nnz;
  if (padded_nnz) *padded_nnz = s->padded;
  if (n_blocks) *n_blocks = s->nblocks;
  return TC_OK;
}

tc_status tc_sim_layout(const tc_sim* s, int32_t* n_components, int64_t* n_internal,
                        int32_t* pcg_threads, int32_t* blocks_per_sm) {
  clear_error();
  if (!s) return fail(TC_ERR_ARG, "sim must not be NULL");
  if (n_components) *n_components = s->n_comp;
  if (n_internal) *n_internal = s->n_int;
  if (pcg_threads) *pcg_threads = s->pcg_threads;
  if (blocks_per_sm) *blocks_per_sm = s->blocks_per_sm;
  return TC_OK;
}

tc_status tc_sim_staging(const tc_sim* s, int32_t* blocks, int32_t* staged_blocks, int32_t* max_window,
                         int64_t* smem_bytes, int32_t* idx16) {
  clear_error();
  if (!s) return fail(TC_ERR_ARG, "sim must not be NULL");
  if (idx16) *idx16 = s->use16 ? 1 : 0;
  if (blocks) *blocks = s->nblocks;
  if (staged_blocks) *staged_blocks = s->win_staged;
  if (max_window) *max_window = s->win_max;
  if (smem_bytes) *smem_bytes = (int64_t)s->pcg_dyn_smem;
  return TC_OK;
}

tc_status tc_set_launch(tc_sim* s, int32_t pcg_threads, int32_t blocks_per_sm) {
  clear_error();
  if (!s || (pcg_threads != 512 && pcg_threads != 1024) || blocks_per_sm < 1)
    return fail(TC_ERR_ARG, "pcg_threads must be 512 or 1024 and blocks_per_sm >= 1");
  CUDA_TRY(cudaSetDevice(s->device));
  CUDA_TRY(cudaStreamSynchronize(s->stream));
  const int old_t = s->pcg_threads, old_b = s->blocks_per_sm;
  s->pcg_threads = pcg_threads;
  s->blocks_per_sm = blocks_per_sm;
  tc_status st = set_partition(s);
  if (st != TC_OK) {
    s->pcg_threads = old_t;
    s->blocks_per_sm = old_b;
    set_partition(s);
  }
  return st;
}

tc_status tc_set_graphs(tc_sim* s, int32_t on) {
  clear_error();
  if (!s) return fail(TC_ERR_ARG, "sim must not be NULL");
  s->use_graphs = on != 0;
  if (!s->use_graphs) drop_graphs(s);
  return TC_OK;
}

tc_status tc_set_ionic(tc_sim* s, int32_t model, const double* params, int32_t n_params,
                       const double* init_state) {
  clear_error();
  if (!s) return fail(TC_ERR_ARG, "sim must not be NULL");
  CUDA_TRY(cudaSetDevice(s->device));
  std::vector<double> rest;   // resting states (V excluded)
  double v0 = 0.0;
  if (model == TC_MODEL_MS) {
    if (!params || n_params != 7) return fail(TC_ERR_ARG, "Mitchell-Schaeffer needs 7 parameters");
    const double* p = params;
    if (!(p[0] > 0 && p[1] > 0 && p[2] > 0 && p[3] > 0 && p[6] > p[5]))
      return fail(TC_ERR_ARG, "Mitchell-Schaeffer needs positive time constants and v_max > v_min");
    std::copy(p, p + 7, s->ms);
    rest.assign(1, 1.0);
    v0 = p[5];
  } else if (model == TC_MODEL_TP06) {
    if (!params || n_params != 1) return fail(TC_ERR_ARG, "TP06 needs 1 parameter (cell type)");
    const int cell = (int)params[0];
    if (cell < 0 || cell > 2 || params[0] != (double)cell)
      return fail(TC_ERR_ARG, "TP06 cell type must be 0 (endo), 1 (mid) or 2 (epi)");
    s->cell = cell;
    rest.assign(kTP06States, 0.0);
    tp06_rest_state(cell, rest.data(), &v0);
  } else {
    return fail(TC_ERR_ARG, "unknown ionic model " + std::to_string(model));
  }
  CUDA_TRY(cudaStreamSynchronize(s->stream));
  const int ns = (int)rest.size();
  if (s->state && ns != s->n_states) {
    dfree(s, s->state);
    s->state = nullptr;
    drop_graphs(s);
  }
  if (!s->state) TRY(dalloc_bytes(s, &s->state, (size_t)ns * s->n_int * s->esz));
  if (model == TC_MODEL_TP06 && s->precision == TC_FP64 && !s->log_cache) {
    TRY(dalloc_bytes(s, &s->log_cache, (size_t)4 * s->n_int * sizeof(double)));
    void* flag = nullptr;
    TRY(dalloc_bytes(s, &flag, sizeof(int)));
    s->log_valid = static_cast<int*>(flag);
  }
  if (s->log_valid) CUDA_TRY(cudaMemsetAsync(s->log_valid, 0, sizeof(int), s->stream));
  s->model = model;
  s->n_states = ns;
  drop_graphs(s);   // model constants are baked into captured launches
  // the learned surrogate serves TP06 only; a re-initialised model starts exact
  if (model != TC_MODEL_TP06) s->sur = nullptr;
  if (s->sur_flag) CUDA_TRY(cudaMemset(s->sur_flag, 0, s->n_int));
  std::vector<double> col(s->n_int);
  for (int j = 0; j < ns; ++j) {
    if (init_state)
      to_internal(s, init_state + (size_t)j * s->n, col.data(), rest[j]);
    else
      std::fill(col.begin(), col.end(), rest[j]);
    TRY(upload_vec(s, static_cast<char*>(s->state) + (size_t)j * s->n_int * s->esz, col.data(), false));
  }
  std::fill(col.begin(), col.end(), v0);
  s->iv = 0;
  TRY(upload_vec(s, s->V[0], col.data(), false));
  TRY(upload_vec(s, s->V[2], col.data(), false));
  std::vector<double> a0(s->n_int, v0 >= s->thr ? 0.0 : -1.0), m1(s->n_int, -1.0);
  CUDA_TRY(cudaMemcpy(s->act, a0.data(), s->n_int * sizeof(double), cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(s->rep90, m1.data(), s->n_int * sizeof(double), cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(s->lrt, m1.data(), s->n_int * sizeof(double), cudaMemcpyHostToDevice));
  std::fill(m1.begin(), m1.end(), v0);
  CUDA_TRY(cudaMemcpy(s->vpeak, m1.data(), s->n_int * sizeof(double), cudaMemcpyHostToDevice));
  s->v_rest = v0;
  s->k = 0;
  return TC_OK;
}

tc_status tc_add_stimulus(tc_sim* s, const int32_t* nodes, int64_t n, double start_ms,
                          double duration_ms, double intensity) {
  clear_error();
  if (!s || (!nodes && n > 0) || n < 0) return fail(TC_ERR_ARG, "bad stimulus arguments");
  if (!(start_ms >= 0) || !(duration_ms >= 0) || !std::isfinite(intensity))
    return fail(TC_ERR_ARG, "stimulus start/duration must be >= 0 and intensity finite");
  std::vector<int32_t> in;
  in.reserve(n);
  for (int64_t i = 0; i < n; ++i) {
    if (nodes[i] < 0 || nodes[i] >= s->n)
      return fail(TC_ERR_ARG, "stimulus node index " + std::to_string(nodes[i]) + " out of range");
    in.push_back(s->inv[nodes[i]]);
  }
  std::sort(in.begin(), in.end());
  in.erase(std::unique(in.begin(), in.end()), in.end());
  StimDev d{};
  d.k0 = round_half_even(start_ms / s->dt);
  d.nk = round_half_even(duration_ms / s->dt);
  d.amp = intensity;
  s->stim_nodes.push_back(std::move(in));
  s->stim_host.push_back(d);
  CUDA_TRY(cudaSetDevice(s->device));
  return upload_stimuli(s);
}

tc_status tc_set_solver(tc_sim* s, double atol, double rtol, int32_t max_iter) {
  clear_error();
  if (!s) return fail(TC_ERR_ARG, "sim must not be NULL");
  if (!(atol >= 0) || !(rtol >= 0) || max_iter < 0)
    return fail(TC_ERR_ARG, "need atol >= 0, rtol >= 0, max_iter >= 0");
  s->atol = atol;
  s->rtol = rtol;
  s->max_iter = max_iter;
  drop_graphs(s);
  return TC_OK;
}

tc_status tc_set_activation_threshold(tc_sim* s, double v) {
  clear_error();
  if (!s || !std::isfinite(v)) return fail(TC_ERR_ARG, "bad threshold");
  if (s->thr_locked) return fail(TC_ERR_STATE, "threshold is fixed once stepping has started");
  s->thr = v;
  drop_graphs(s);
  if (s->model >= 0) {
    CUDA_TRY(cudaSetDevice(s->device));
    std::vector<double> vcur(s->n_int), a0(s->n_int);
    TRY(download_vec(s, s->V[s->iv], vcur.data()));
    for (int64_t i = 0; i < s->n_int; ++i) a0[i] = vcur[i] >= v ? 0.0 : -1.0;
    CUDA_TRY(cudaMemcpy(s->act, a0.data(), s->n_int * sizeof(double), cudaMemcpyHostToDevice));
  }
  return TC_OK;
}

tc_status tc_set_wait_limit(tc_sim* s, int64_t polls) {
  clear_error();
  if (!s || polls < 1) return fail(TC_ERR_ARG, "need polls >= 1");
  s->wait_limit = polls;
  drop_graphs(s);
  return TC_OK;
}

tc_status tc_step(tc_sim* s, int64_t n_steps, tc_step_stats* stats) {
  clear_error();
  if (!s || n_steps < 0) return fail(TC_ERR_ARG, "bad tc_step arguments");
  if (s->model < 0) return fail(TC_ERR_STATE, "tc_set_ionic must be called before tc_step");
  CUDA_TRY(cudaSetDevice(s->device));
  s->thr_locked = true;
  std::vector<DevStats> zero(s->n_comp);
  CUDA_TRY(cudaMemcpyAsync(s->stats, zero.data(), s->n_comp * sizeof(DevStats),
                           cudaMemcpyHostToDevice, s->stream));
  CUDA_TRY(cudaMemsetAsync(s->err, 0, sizeof(int), s->stream));
  CUDA_TRY(cudaMemsetAsync(s->bar, 0, s->n_comp * sizeof(GridBar), s->stream));
  const long long k0 = s->k;
  CUDA_TRY(cudaMemcpyAsync(s->k_dev, &k0, sizeof(long long), cudaMemcpyHostToDevice, s->stream));
  size_t ev = 0;
  std::vector<size_t> marks, sur_marks;
  int64_t done = 0, graph_steps = 0;
  // steps done .. done + cnt - 1 launched one by one, then the device index advanced
  auto single_steps = [&](int64_t cnt) -> tc_status {
    for (int64_t j = 0; j < cnt; ++j) {
      const int ivj = (int)((s->iv + done + j) % 3);
      const long long kj = s->k + done + j;
      if (s->sur && kj % s->sur_window == 0)
        TRY(launch_surrogate(s, ivj, (int)j, s->prof ? &ev : nullptr, &sur_marks));
      TRY(launch_step_any(s, ivj, (int)j, s->prof ? &ev : nullptr, &marks));
    }
    if (cnt > 0) {
      tick_kernel<<<1, 1, 0, s->stream>>>(s->k_dev, (int)cnt);
      CUDA_TRY(cudaGetLastError());
    }
    done += cnt;
    return TC_OK;
  };
  // whole groups of kGraphSteps steps replay a captured graph (not while profiling per launch;
  // with the surrogate only when the window divides the group, after steps up to a boundary)
  const bool graphs = s->use_graphs && !s->prof && (!s->sur || kGraphSteps % s->sur_window == 0);
  const int64_t lead = s->sur ? (s->sur_window - s->k % s->sur_window) % s->sur_window : 0;
  if (graphs && n_steps >= lead + kGraphSteps) {
    if (s->sur) TRY(surrogate_prepare(s->sur, s->n_int));
    TRY(single_steps(lead));
    const int iv0 = (int)((s->iv + done) % 3);
    GraphCache& g = s->graphs[iv0];
    if (!g.valid) {
      tc_status st = capture_graph(s, iv0, &g.exec);
      if (st == TC_OK) {
        g.valid = true;
        g.iv = iv0;
      } else {
        s->use_graphs = false;   // capture unsupported here: launch step by step instead
        clear_error();
      }
    }
    if (g.valid) {
      for (; done + kGraphSteps <= n_steps; done += kGraphSteps) {
        CUDA_TRY(cudaGraphLaunch(g.exec, s->stream));
        graph_steps += kGraphSteps;
      }
    }
  }
  TRY(single_steps(n_steps - done));
  CUDA_TRY(l2_release(s));
  s->iv = (int)((s->iv + n_steps) % 3);
  s->k += n_steps;
  std::vector<DevStats> ds(s->n_comp);
  int herr = 0;
  CUDA_TRY(cudaMemcpyAsync(ds.data(), s->stats, s->n_comp * sizeof(DevStats),
                           cudaMemcpyDeviceToHost, s->stream));
  CUDA_TRY(cudaMemcpyAsync(&herr, s->err, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
  CUDA_TRY(cudaStreamSynchronize(s->stream));
  long long iters = 0;
  int max_it = 0, not_conv = 0;
  double zn = 0.0, z0n = 0.0;
  for (const DevStats& d : ds) {
    iters += d.iters_total;
    max_it = std::max(max_it, d.max_iters);
    not_conv += d.not_conv;
    zn = std::max(zn, d.last_zn);
    z0n = std::max(z0n, d.last_z0n);
  }
  if (s->prof) {
    for (size_t m : marks) {
      float a = 0.f, b = 0.f;
      cudaEventElapsedTime(&a, s->evpool[m], s->evpool[m + 1]);
      cudaEventElapsedTime(&b, s->evpool[m + 1], s->evpool[m + 2]);
      s->prof_acc.ionic_ms += a;
      s->prof_acc.ionic_launches += s->model == TC_MODEL_MS && s->fuse_ms ? 0 : 1;
      s->prof_acc.pcg_ms += b;
      s->prof_acc.pcg_launches += 1;
    }
    s->prof_acc.pcg_iterations += iters;
    for (size_t m : sur_marks) {
      float a = 0.f, b = 0.f;
      cudaEventElapsedTime(&a, s->evpool[m], s->evpool[m + 3]);
      cudaEventElapsedTime(&b, s->evpool[m + 1], s->evpool[m + 2]);
      s->prof_acc.surrogate_ms += a;
      s->prof_acc.surrogate_windows += 1;
      s->prof_acc.mlp_ms += b;
    }
    if (!sur_marks.empty()) {
      unsigned long long rows = 0;
      CUDA_TRY(cudaMemcpy(&rows, s->sur_rows, sizeof(rows), cudaMemcpyDeviceToHost));
      CUDA_TRY(cudaMemset(s->sur_rows, 0, sizeof(rows)));
      s->prof_acc.surrogate_rows += (int64_t)rows;
    }
  }
  if (stats) {
    stats->steps = n_steps;
    stats->step_index = s->k;
    stats->cg_iterations = iters;
    stats->max_iterations = max_it;
    stats->not_converged = not_conv;
    stats->last_znorm = zn;
    stats->last_z0norm = z0n;
    stats->graph_steps = graph_steps;
  }
  if (herr & kErrTimeout) return fail(TC_ERR_TIMEOUT, "a grid barrier wait hit its limit");
  if (herr & kErrNan) return fail(TC_ERR_NAN, "non-finite value in the PCG solve");
  if (s->sur) {
    int serr = 0;
    CUDA_TRY(cudaMemcpy(&serr, s->sur_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (serr) return fail(TC_ERR_TIMEOUT, "a tensor-core wait of the surrogate hit its limit");
  }
  return TC_OK;
}

tc_status tc_set_surrogate(tc_sim* s, tc_mlp* mlp, int32_t window, double dv_max, double dvdt_max,
                           double dv_neighbour, double rest_band) {
  clear_error();
  if (!s) return fail(TC_ERR_ARG, "sim must not be NULL");
  if (!mlp) {
    if (s->sur) drop_graphs(s);   // captured groups hold the surrogate's launches
    s->sur = nullptr;
    return TC_OK;
  }
  if (s->model != TC_MODEL_TP06)
    return fail(TC_ERR_ARG, "the learned surrogate serves simulations of TP06");
  if (window < 1 || !(dv_max > 0) || !(dvdt_max > 0) || !(dv_neighbour >= 0) || !(rest_band >= 0))
    return fail(TC_ERR_ARG, "need window >= 1, dv_max > 0, dvdt_max > 0, dv_neighbour >= 0, rest_band >= 0");
  CUDA_TRY(cudaSetDevice(s->device));
  if (!s->sur_flag) {
    const int64_t n = s->n_int;
    TRY(dalloc(s, &s->sur_flag, n));
    TRY(dalloc(s, &s->sur_iion, n));
    TRY(dalloc(s, &s->sur_raw, 20 * n));
    TRY(dalloc(s, &s->sur_zout, 32 * n));
    TRY(dalloc(s, &s->sur_a0, (size_t)kMlpIn0 * n));
    TRY(dalloc(s, &s->sur_idx, n));
    TRY(dalloc(s, &s->sur_count, 1));
    TRY(dalloc(s, &s->sur_rows, 1));
    CUDA_TRY(cudaMemset(s->sur_rows, 0, sizeof(unsigned long long)));
    TRY(dalloc(s, &s->sur_counts, 2));
    TRY(dalloc(s, &s->sur_err, 1));
    CUDA_TRY(cudaMemset(s->sur_flag, 0, n));
  }
  CUDA_TRY(cudaMemset(s->sur_counts, 0, 2 * sizeof(unsigned long long)));
  CUDA_TRY(cudaMemset(s->sur_err, 0, sizeof(int)));
  s->sur = mlp;
  s->sur_window = window;
  s->sur_dv_max = (float)dv_max;
  s->sur_dvdt_max = (float)dvdt_max;
  s->sur_dv_nbr = (float)dv_neighbour;
  s->sur_rest_band = (float)rest_band;
  drop_graphs(s);
  return TC_OK;
}

tc_status tc_surrogate_sample(tc_sim* s, int32_t window, double rest_band, double rest_keep, double dv_keep,
                              double dvdt_keep, uint64_t seed, float* x_dev, float* y_dev, int64_t capacity,
                              int64_t* count) {
  clear_error();
  if (!s || !x_dev || !y_dev || !count) return fail(TC_ERR_ARG, "null argument");
  if (s->model != TC_MODEL_TP06) return fail(TC_ERR_STATE, "sampling needs the TP06 model");
  if (window < 1 || !(rest_band >= 0) || !(rest_keep >= 0 && rest_keep <= 1) || !(dv_keep >= 0) ||
      !(dvdt_keep >= 0) || capacity < 0 || *count < 0 || *count > capacity)
    return fail(TC_ERR_ARG, "bad sampling arguments");
  if (*count == capacity) return TC_OK;
  CUDA_TRY(cudaSetDevice(s->device));
  return s->precision == TC_FP64
             ? surrogate_sample_t<double>(s, window, rest_band, rest_keep, dv_keep, dvdt_keep, seed, x_dev, y_dev,
                                          capacity, count)
             : surrogate_sample_t<float>(s, window, rest_band, rest_keep, dv_keep, dvdt_keep, seed, x_dev, y_dev,
                                         capacity, count);
}

tc_status tc_surrogate_usage(const tc_sim* s, int64_t* surrogate_node_windows, int64_t* exact_node_windows) {
  clear_error();
  if (!s) return fail(TC_ERR_ARG, "sim must not be NULL");
  unsigned long long c[2] = {0, 0};
  if (s->sur_counts) CUDA_TRY(cudaMemcpy(c, s->sur_counts, sizeof(c), cudaMemcpyDeviceToHost));
  if (surrogate_node_windows) *surrogate_node_windows = (int64_t)c[0];
  if (exact_node_windows) *exact_node_windows = (int64_t)c[1];
  return TC_OK;
}

static void* field_ptr(const tc_sim* s, int32_t field) {
  if (field == TC_FIELD_V) return s->V[s->iv];
  if (field == TC_FIELD_V_PREV) return s->V[(s->iv + 2) % 3];
  if (field >= TC_FIELD_STATE && field < TC_FIELD_STATE + s->n_states)
    return static_cast<char*>(s->state) + (size_t)(field - TC_FIELD_STATE) * s->n_int * s->esz;
  return nullptr;
}

tc_status tc_read_state(const tc_sim* s, int32_t field, double* dst, int64_t n) {
  clear_error();
  if (!s || !dst) return fail(TC_ERR_ARG, "null argument");
  if (n != s->n) return fail(TC_ERR_ARG, "n must equal the node count");
  if (s->model < 0) return fail(TC_ERR_STATE, "no ionic model set");
  const void* src = field_ptr(s, field);
  if (!src) return fail(TC_ERR_ARG, "unknown field " + std::to_string(field));
  CUDA_TRY(cudaSetDevice(s->device));
  return read_caller_field(s, src, false, dst);
}

tc_status tc_write_state(tc_sim* s, int32_t field, const double* src, int64_t n) {
  clear_error();
  if (!s || !src) return fail(TC_ERR_ARG, "null argument");
  if (n != s->n) return fail(TC_ERR_ARG, "n must equal the node count");
  if (s->model < 0) return fail(TC_ERR_STATE, "no ionic model set");
  void* dst = field_ptr(s, field);
  if (!dst) return fail(TC_ERR_ARG, "unknown field " + std::to_string(field));
  CUDA_TRY(cudaSetDevice(s->device));
  CUDA_TRY(cudaStreamSynchronize(s->stream));   // the staging buffer may still feed a copy
  // nodes the learned surrogate holds for the current window restart on the exact model
  if (s->sur_flag) CUDA_TRY(cudaMemsetAsync(s->sur_flag, 0, s->n_int, s->stream));
  // the held-over concentration logarithms no longer match the states
  if (s->log_valid) CUDA_TRY(cudaMemsetAsync(s->log_valid, 0, sizeof(int), s->stream));
  return write_caller_field(s, dst, false, src);
}

tc_status tc_activation_times(const tc_sim* s, double v_threshold, double* dst, int64_t n) {
  clear_error();
  if (!s || !dst) return fail(TC_ERR_ARG, "null argument");
  if (n != s->n) return fail(TC_ERR_ARG, "n must equal the node count");
  if (v_threshold != s->thr)
    return fail(TC_ERR_STATE, "activation times were captured for another threshold");
  CUDA_TRY(cudaSetDevice(s->device));
  return read_caller_field(s, s->act, true, dst);
}

static tc_status read_double_field(const tc_sim* s, const double* src, double* dst, int64_t n) {
  if (!s || !dst) return fail(TC_ERR_ARG, "null argument");
  if (n != s->n) return fail(TC_ERR_ARG, "n must equal the node count");
  if (s->model < 0) return fail(TC_ERR_STATE, "no ionic model set");
  CUDA_TRY(cudaSetDevice(s->device));
  return read_caller_field(s, src, true, dst);
}

tc_status tc_set_repolarisation_threshold(tc_sim* s, double v) {
  clear_error();
  if (!s || !std::isfinite(v)) return fail(TC_ERR_ARG, "bad threshold");
  if (s->thr_locked) return fail(TC_ERR_STATE, "threshold is fixed once stepping has started");
  s->lrt_thr = v;
  drop_graphs(s);
  return TC_OK;
}

tc_status tc_repolarisation_times(const tc_sim* s, double* dst, int64_t n) {
  clear_error();
  return read_double_field(s, s ? s->lrt : nullptr, dst, n);
}

tc_status tc_apd90(const tc_sim* s, double* dst, int64_t n) {
  clear_error();
  TRY(read_double_field(s, s ? s->rep90 : nullptr, dst, n));
  std::vector<double> act(n);
  TRY(read_double_field(s, s->act, act.data(), n));
  for (int64_t i = 0; i < n; ++i) dst[i] = (dst[i] >= 0.0 && act[i] >= 0.0) ? dst[i] - act[i] : -1.0;
  return TC_OK;
}

tc_status tc_get_step_index(const tc_sim* s, int64_t* k) {
  clear_error();
  if (!s || !k) return fail(TC_ERR_ARG, "null argument");
  *k = s->k;
  return TC_OK;
}

tc_status tc_set_step_index(tc_sim* s, int64_t k) {
  clear_error();
  if (!s || k < 0) return fail(TC_ERR_ARG, "bad step index");
  s->k = k;
  if (s->sur_flag) {
    CUDA_TRY(cudaSetDevice(s->device));
    CUDA_TRY(cudaStreamSynchronize(s->stream));
    CUDA_TRY(cudaMemset(s->sur_flag, 0, s->n_int));
  }
  return TC_OK;
}

tc_status tc_autotune(tc_sim* s, int32_t trial_steps, int32_t* pcg_threads, int32_t* blocks_per_sm,
                      double* best_ms_per_step) {
  clear_error();
  if (!s || trial_steps < 1) return fail(TC_ERR_ARG, "need a simulation and trial_steps >= 1");
  if (s->model < 0) return fail(TC_ERR_STATE, "tc_set_ionic must be called before tc_autotune");
  CUDA_TRY(cudaSetDevice(s->device));
  CUDA_TRY(cudaStreamSynchronize(s->stream));
  // snapshot of everything a step changes, restored after every candidate
  struct Buf {
    void* dev;
    size_t bytes;
    void* copy;
  };
  std::vector<Buf> bufs;
  auto add = [&](void* p, size_t bytes) { bufs.push_back({p, bytes, nullptr}); };
  for (int j = 0; j < 3; ++j) add(s->V[j], s->n_int * s->esz);
  add(s->state, (size_t)s->n_states * s->n_int * s->esz);
  for (double* p : {s->act, s->vpeak, s->rep90, s->lrt}) add(p, s->n_int * sizeof(double));
  tc_status st = TC_OK;
  for (auto& b : bufs) {
    cudaError_t e = cudaMalloc(&b.copy, b.bytes);
    if (e == cudaSuccess) e = cudaMemcpy(b.copy, b.dev, b.bytes, cudaMemcpyDeviceToDevice);
    if (e != cudaSuccess) {
      st = cuda_fail(e, "autotune snapshot");
      break;
    }
  }
  const long long k0 = s->k;
  const int iv0 = s->iv;
  const bool thr_locked0 = s->thr_locked;
  const int t0 = s->pcg_threads, b0 = s->blocks_per_sm, g0 = s->pcg_stage;
  // launch shape (threads per block, blocks per SM) and whether the PCG stages its windows of z in
  // shared memory (it pays where the windows are small next to a block's rows)
  const int cand[][3] = {{1024, 1, 0}, {512, 1, 0}, {512, 2, 0}, {1024, 1, 1}, {512, 1, 1}, {512, 2, 1}};
  double best = 1e300;
  int best_t = t0, best_b = b0, best_g = g0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (st == TC_OK) {
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
  }
  for (const auto& c : cand) {
    if (st != TC_OK) break;
    s->pcg_threads = c[0];
    s->blocks_per_sm = c[1];
    s->pcg_stage = c[2];
    if (set_partition(s) != TC_OK) {
      clear_error();
      continue;
    }
    float ms = 0.f;
    cudaEventRecord(e0, s->stream);
    tc_status r = tc_step(s, trial_steps, nullptr);
    cudaEventRecord(e1, s->stream);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    if (r == TC_OK && ms < best) {
      best = ms;
      best_t = c[0];
      best_b = c[1];
      best_g = c[2];
    }
    clear_error();
    for (auto& b : bufs) cudaMemcpy(b.dev, b.copy, b.bytes, cudaMemcpyDeviceToDevice);
    if (s->log_valid) cudaMemsetAsync(s->log_valid, 0, sizeof(int), s->stream);   // the states went back
    s->k = k0;
    s->iv = iv0;
    s->thr_locked = thr_locked0;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  for (auto& b : bufs)
    if (b.copy) cudaFree(b.copy);
  s->pcg_threads = best_t;
  s->blocks_per_sm = best_b;
  s->pcg_stage = best_g;
  tc_status st2 = set_partition(s);
  if (st != TC_OK) return st;
  if (st2 != TC_OK) return st2;
  if (pcg_threads) *pcg_threads = best_t;
  if (blocks_per_sm) *blocks_per_sm = best_b;
  if (best_ms_per_step) *best_ms_per_step = best / trial_steps;
  return TC_OK;
}

static const void* op_values(const tc_sim* s, int32_t op) {
  return op == TC_OP_M ? s->vM : op == TC_OP_K ? s->vK : op == TC_OP_A ? s->vA : nullptr;
}

tc_status tc_apply_operator_dev(tc_sim* s, int32_t op, const void* x_dev, void* y_dev) {
  clear_error();
  if (!s || !x_dev || !y_dev) return fail(TC_ERR_ARG, "null argument");
  const void* val = op_values(s, op);
  if (!val) return fail(TC_ERR_ARG, "unknown operator");
  if (((uintptr_t)x_dev | (uintptr_t)y_dev) & 15) return fail(TC_ERR_ARG, "x/y must be 16-byte aligned");
  CUDA_TRY(cudaSetDevice(s->device));
  // two-warp blocks: the kernel strides over slices, one wave of resident blocks with no partial
  // second wave; small blocks spread the slices over the SMs more evenly (measured on the
  // 40x16x6 mm slab, FP64: 64 threads x 18 blocks per SM 22.8 us, 256 x 4 24.8 us)
  const int threads = 64;
  int occ = 1;
  if (s->precision == TC_FP64)
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, spmv_sell_kernel<double>, threads, 0));
  else
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, spmv_sell_kernel<float>, threads, 0));
  const int64_t blocks = std::min<int64_t>((s->nslices * 32 + threads - 1) / threads,
                                           (int64_t)s->num_sms * std::max(occ, 1));
  const int nb = (int)std::max<int64_t>(blocks, 1);
  if (s->precision == TC_FP64)
    spmv_sell_kernel<double><<<nb, threads, 0, s->stream>>>(
        s->n_int, s->nslices, s->slice_ptr, s->col, static_cast<const double*>(val),
        static_cast<const double*>(x_dev), static_cast<double*>(y_dev));
  else
    spmv_sell_kernel<float><<<nb, threads, 0, s->stream>>>(
        s->n_int, s->nslices, s->slice_ptr, s->col, static_cast<const float*>(val),
        static_cast<const float*>(x_dev), static_cast<float*>(y_dev));
  CUDA_TRY(cudaGetLastError());
  return TC_OK;
}

tc_status tc_apply_operator(tc_sim* s, int32_t op, const double* x, double* y, int64_t n) {
  clear_error();
  if (!s || !x || !y) return fail(TC_ERR_ARG, "null argument");
  if (n != s->n) return fail(TC_ERR_ARG, "n must equal the node count");
  if (!op_values(s, op)) return fail(TC_ERR_ARG, "unknown operator");
  CUDA_TRY(cudaSetDevice(s->device));
  void *dx = nullptr, *dy = nullptr;
  CUDA_TRY(cudaMalloc(&dx, s->n_int * s->esz));
  cudaError_t e = cudaMalloc(&dy, s->n_int * s->esz);
  if (e != cudaSuccess) {
    cudaFree(dx);
    return cuda_fail(e, "cudaMalloc");
  }
  to_internal(s, x, s->pinned, 0.0);
  tc_status st = upload_vec(s, dx, s->pinned, false);
  if (st == TC_OK) st = tc_apply_operator_dev(s, op, dx, dy);
  if (st == TC_OK) st = download_vec(s, dy, s->pinned);
  cudaFree(dx);
  cudaFree(dy);
  if (st != TC_OK) return st;
  to_caller(s, s->pinned, y);
  return TC_OK;
}

tc_status tc_set_profiling(tc_sim* s, int32_t on) {
  clear_error();
  if (!s) return fail(TC_ERR_ARG, "sim must not be NULL");
  s->prof = on != 0;
  return TC_OK;
}

tc_status tc_get_profile(const tc_sim* s, tc_profile* out) {
  clear_error();
  if (!s || !out) return fail(TC_ERR_ARG, "null argument");
  *out = s->prof_acc;
  return TC_OK;
}

tc_status tc_reset_profile(tc_sim* s) {
  clear_error();
  if (!s) return fail(TC_ERR_ARG, "sim must not be NULL");
  s->prof_acc = tc_profile{};
  return TC_OK;
}

static tc_status selftest_math(const double* x, double* y_fast, double* y_ref, int64_t n, int fn) {
  clear_error();
  if (!x || !y_fast || !y_ref || n < 1) return fail(TC_ERR_ARG, "bad self-test arguments");
  double* d = nullptr;
  CUDA_TRY(cudaMalloc(&d, 3 * n * sizeof(double)));
  cudaError_t e = cudaMemcpy(d, x, n * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    exp_selftest_kernel<<<(int)((n + 255) / 256), 256>>>(n, d, d + n, d + 2 * n, fn);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(y_fast, d + n, n * sizeof(double), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(y_ref, d + 2 * n, n * sizeof(double), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return cuda_fail(e, "math self-test");
  return TC_OK;
}

tc_status tc_selftest_exp(const double* x, double* y_fast, double* y_ref, int64_t n) {
  return selftest_math(x, y_fast, y_ref, n, 0);
}

tc_status tc_selftest_log(const double* x, double* y_fast, double* y_ref, int64_t n) {
  return selftest_math(x, y_fast, y_ref, n, 1);
}

tc_status tc_selftest_rcp(const double* x, double* y_fast, double* y_ref, int64_t n) {
  return selftest_math(x, y_fast, y_ref, n, 2);
}

tc_status tc_selftest_exp2(const double* x, double* y_fast, double* y_ref, int64_t n) {
  return selftest_math(x, y_fast, y_ref, n, 3);
}

const char* tc_version(void) { return "tc_b300 0.5 (sm_103a)"; }

// FP64 arithmetic rate of the current device: every thread runs eight independent chains of
// dependent FMAs (enough in flight to keep the FP64 pipe busy at full occupancy); the result is
// written only under a condition the data never meet, which keeps the work alive.
static __global__ void __launch_bounds__(256) fp64_rate_kernel(int iters, double* sink) {
  double a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = 1.0 + 1e-3 * (threadIdx.x + 32 * k);
  const double m = 1.0 - 1e-13, c = 1e-14;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = fma(a[k], m, c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k];
  if (s == -1.0) sink[blockIdx.x] = s;
}

tc_status tc_measure_fp64_rate(double* fma_per_s) {
  clear_error();
  if (!fma_per_s) return fail(TC_ERR_ARG, "fma_per_s must not be NULL");
  int dev = 0, sms = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = sms * 8, threads = 256, iters = 1 << 14;
  double* sink = nullptr;
  CUDA_TRY(cudaMalloc(&sink, blocks * sizeof(double)));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  fp64_rate_kernel<<<blocks, threads>>>(iters, sink);   // warm-up (clocks up)
  float best = 1e30f;
  for (int r = 0; r < 3; ++r) {
    cudaEventRecord(e0);
    fp64_rate_kernel<<<blocks, threads>>>(iters, sink);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    best = std::min(best, ms);
  }
  cudaError_t e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  if (e != cudaSuccess) return cuda_fail(e, "fp64 rate probe");
  *fma_per_s = (double)blocks * threads * 8.0 * iters / (best * 1e-3);
  return TC_OK;
}

}  // extern "C"

// ---- allocation-free operator application ------------------------------------------------
//
// tc_apply_operator stages x and y in device buffers that it allocates and frees on every
// call.  Some callers cannot do that: a process whose device memory is already reserved by
// another allocator (cudaMalloc would fail), or a caller that cannot afford the device-wide
// synchronisation cudaFree implies.  tc_apply_operator_static does the same work with its
// staging in the file-scope array below, which every GPU that loads this library holds until
// the process exits.  Calls share the array; calls that overlap on the GPU race.

namespace {

constexpr int64_t kStaticMaxNodes = 262144;   // x and y staging: 2 * 2 MiB
constexpr int kStaticMaxDevices = 128;

static __device__ __align__(256) double g_apply_scratch[2 * kStaticMaxNodes];

std::mutex g_apply_scratch_mu;
double* g_apply_scratch_addr[kStaticMaxDevices] = {nullptr};

// y = Op x with x read from, and y written to, the static staging array.
__global__ void __launch_bounds__(256) spmv_sell_static_kernel(
    int64_t n, int64_t nslices, const int32_t* __restrict__ slice_ptr,
    const int32_t* __restrict__ col, const double* __restrict__ val, double* scratch) {
  const double* x = scratch;
  double* y = scratch + kStaticMaxNodes;
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t s = gw; s < nslices; s += nw) {
    const int beg = slice_ptr[s] + lane;
    const int w = (slice_ptr[s + 1] - slice_ptr[s]) >> 5;
    const double acc = sell_dot<kSellChunk8>(col, val, beg, w, x);
    const int64_t row = s * 32 + lane;
    if (row < n) y[row] = acc;
  }
}

// Device address of the staging array on the current device, looked up once per device and kept
// for the life of that device's primary context (a cudaDeviceReset between calls may move the
// array; the header states that this is not supported).
tc_status static_scratch_address(int device, double** out) {
  if (device < 0 || device >= kStaticMaxDevices)
    return fail(TC_ERR_ARG, "device ordinal too large for the static staging table");
  std::lock_guard<std::mutex> lock(g_apply_scratch_mu);
  if (!g_apply_scratch_addr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_apply_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_apply_scratch)");
    g_apply_scratch_addr[device] = static_cast<double*>(p);
  }
  *out = g_apply_scratch_addr[device];
  return TC_OK;
}

}  // namespace

extern "C" tc_status tc_apply_operator_static(tc_sim* s, int32_t op, const double* x, double* y,
                                              int64_t n) {
  clear_error();
  if (!s || !x || !y) return fail(TC_ERR_ARG, "null argument");
  if (n != s->n) return fail(TC_ERR_ARG, "n must equal the node count");
  if (s->precision != TC_FP64)
    return fail(TC_ERR_ARG, "tc_apply_operator_static serves TC_FP64 simulations only");
  if (s->n_int > kStaticMaxNodes)
    return fail(TC_ERR_ARG, "tc_apply_operator_static handles at most " +
                                std::to_string(kStaticMaxNodes) + " rows of the padded device layout; this "
                                "simulation has " + std::to_string(s->n_int) + " (use tc_apply_operator)");
  const double* val = static_cast<const double*>(op_values(s, op));
  if (!val) return fail(TC_ERR_ARG, "unknown operator");
  CUDA_TRY(cudaSetDevice(s->device));
  double* scratch = nullptr;
  TRY(static_scratch_address(s->device, &scratch));
  // the simulation's page-locked staging buffer carries x in and y out
  CUDA_TRY(cudaStreamSynchronize(s->stream));
  double* h = s->pinned;
  to_internal(s, x, h, 0.0);
  CUDA_TRY(cudaMemcpyAsync(scratch, h, s->n_int * sizeof(double), cudaMemcpyHostToDevice, s->stream));
  const int threads = 64;   // two-warp blocks, one wave (as tc_apply_operator_dev)
  int occ = 1;
  CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, spmv_sell_static_kernel, threads, 0));
  const int64_t blocks = std::min<int64_t>((s->nslices * 32 + threads - 1) / threads,
                                           (int64_t)s->num_sms * std::max(occ, 1));
  spmv_sell_static_kernel<<<(int)std::max<int64_t>(blocks, 1), threads, 0, s->stream>>>(
      s->n_int, s->nslices, s->slice_ptr, s->col, val, scratch);
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaMemcpyAsync(h, scratch + kStaticMaxNodes, s->n_int * sizeof(double),
                           cudaMemcpyDeviceToHost, s->stream));
  CUDA_TRY(cudaStreamSynchronize(s->stream));
  to_caller(s, h, y);
  return TC_OK;
}
