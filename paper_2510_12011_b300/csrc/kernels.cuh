// Device kernels of the monodomain time step.
//
// Data layout (all in the internal node order: reverse Cuthill-McKee, then SELL-C-sigma row
// sorting): matrices in SELL-C-sigma with C = 32 (one warp per slice, one lane per row;
// entry j of the row in lane l of slice s sits at slice_ptr[s] + 32*j + l), one shared int32
// column array and one value array per matrix (M, K, A); node vectors are dense arrays.
//
// Every kernel is a template on the storage and arithmetic type T of the matrices and node
// vectors: T = double is the plain FP64 method; T = float is the precision form, in which the
// SpMVs, vector updates and the ionic model run in FP32 while the PCG reductions (block and
// grid sums), alpha, beta, the norms and the stopping test stay in FP64.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <type_traits>

namespace tc {

constexpr int kErrTimeout = 1;
constexpr int kErrNan = 2;

struct GridBar {
  unsigned count;
  unsigned gen;
};

struct DevStats {
  long long iters_total;
  long long steps;
  int max_iters;
  int not_conv;
  int last_iters;
  int pad;
  double last_zn;
  double last_z0n;
};

struct StimDev {
  long long k0;
  long long nk;
  double amp;
  double pad;
};

// Mitchell-Schaeffer constants prepared on the host.  dec_* = exp(-dt/tau_*).
struct MSConst {
  double vmin, inv_range, range, vgate, inv_tau_in, inv_tau_out, dec_open, dec_close;
};

// Per-node inputs of the right-hand side and the initial guess, written by the ionic kernels:
//   g1 = chi (Cm (V^{k-1} - V^k) + dt (I_stim - I_ion)),  g2 = dt (V^k + theta (V^k - V^{k-1})),
//   x0 = 2 V^k - V^{k-1}  (so that r0 = b - A x0 = M g1 - K g2).
template <typename T>
struct IonicArgs {
  int64_t n;
  const T* V;             // V^k
  const T* Vp;            // V^{k-1}
  T* state;               // [n_states][n] (in place)
  T* g1;
  T* g2;
  T* x0;                  // written into the V^{k+1} buffer
  const int32_t* stim_off;
  const int32_t* stim_ids;
  const StimDev* stims;
  const long long* k_base;   // step index of the first step of this launch group (device)
  int k_off;                 // this step = *k_base + k_off
  double chi, cm, dt, theta;
  MSConst ms;
  int cell;               // TP06 cell type
  GridBar* bar;           // per-component barrier words, zeroed here for the PCG launch that
  int n_bar;              // follows on the stream
  const uint8_t* sur_flag;   // learned-surrogate nodes of the current window (or null)
  const float* sur_iion;     // their effective ionic current over the window, pA/pF
  T* log_cache;              // TP06 FP64: [4][n] concentration logarithms of the states (or null)
  const int* log_valid;      // nonzero: log_cache holds the logarithms of the current states
};

template <typename T>
struct PcgArgs {
  int64_t n;
  const int32_t* slice_ptr;
  const int32_t* col;
  const T* vM;
  const T* vK;
  const T* vA;
  const T* dinv;
  const int32_t* blk_slice;   // gridDim.x + 1 slice boundaries
  const int32_t* comp_of_block;   // connected component (independent problem) of each block
  const int32_t* comp_block0;     // first block of each component, n_comp + 1 entries
  const int32_t* blk_win;         // per block (lo, len): the block's window of gathered columns,
                                  // staged in shared memory when len > 0 (lo set for every block)
  const uint16_t* col16;          // column - lo of the slice's block (or null: 32-bit columns only)
  const T* g1;
  const T* g2;
  T* x;                       // in: x0, out: V^{k+1}
  const T* Vcur;              // V^k (activation capture)
  T* r;
  T* z;
  T* p;
  T* q;
  double* act;
  double* vpeak;              // per-node maximum of V since activation
  double* rep90;              // time of the 90 % repolarisation crossing (APD90 = rep90 - act)
  double* lrt;                // repolarisation time: first downward crossing of lrt_thr
  double* partA;              // gridDim.x
  double* partB;              // 2*gridDim.x
  GridBar* bar;               // one per component
  int* err;
  DevStats* stats;            // one per component
  double atol, rtol;
  int max_iter;
  long long wait_limit;
  float l2_keep;              // fraction of A's and the index array's lines kept in L2 (0: none)
  int* log_valid;             // set once the preceding ionic kernel has refreshed its log cache
  const long long* k_base;
  int k_off;
  double dt, thr;
  double v_rest, lrt_thr;
  int fuse_ms;                // 1: the Mitchell-Schaeffer update of the step runs inside this launch
  IonicArgs<T> ion;           // its arguments (g1, g2 and x0 are the ones above)
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void red_release_add_u32(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid-wide barrier for a cooperative launch (all blocks co-resident).  The arrival counter
// only grows within a launch (it is zeroed by the kernel launched before on the same stream):
// barrier number e of the launch is passed once the counter reaches e * nblocks.  Arrival is a
// release reduction, the wait an acquire poll, so the block's writes before the barrier are
// visible to every block after it.  Every wait is bounded: after wait_limit polls the block
// records kErrTimeout and leaves.  The error word is read only every 64 polls (not on the path
// of a barrier that completes): a block that sees it set leaves too, so that after one block
// gives up every other block leaves at its next barrier instead of waiting out its own limit.
__device__ __forceinline__ bool grid_sync(GridBar* bar, unsigned nblocks, unsigned& epoch,
                                          long long wait_limit, int* err) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    epoch += 1;
    if (nblocks > 1) {
      const unsigned target = epoch * nblocks;
      red_release_add_u32(&bar->count, 1u);
      long long polls = 0;
      while (ld_acquire_u32(&bar->count) < target) {
        ++polls;
        if (polls > wait_limit) {
          atomicOr(err, kErrTimeout);
          ok = 0;
          break;
        }
        if ((polls & 63) == 0 && *(volatile int*)err) {
          ok = 0;
          break;
        }
        if (polls > 2048) __nanosleep(20);
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// The same barrier in two halves, so that a block can do work nobody else waits for between its
// arrival and its wait: grid_arrive (block barrier, then thread 0's release arrival) and
// grid_wait (thread 0's bounded acquire poll, then a block barrier).
__device__ __forceinline__ void grid_arrive(GridBar* bar, unsigned nblocks, unsigned& epoch) {
  __syncthreads();
  if (threadIdx.x == 0) {
    epoch += 1;
    if (nblocks > 1) red_release_add_u32(&bar->count, 1u);
  }
}

__device__ __forceinline__ bool grid_wait(GridBar* bar, unsigned nblocks, unsigned epoch, long long wait_limit,
                                          int* err) {
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    int ok = 1;
    if (nblocks > 1) {
      const unsigned target = epoch * nblocks;
      long long polls = 0;
      while (ld_acquire_u32(&bar->count) < target) {
        ++polls;
        if (polls > wait_limit) {
          atomicOr(err, kErrTimeout);
          ok = 0;
          break;
        }
        if ((polls & 63) == 0 && *(volatile int*)err) {
          ok = 0;
          break;
        }
        if (polls > 2048) __nanosleep(20);
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Fixed-order sums.  warp_sum: lane 0 gets the shfl_down tree sum.
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Block sum of NV values per thread through shared memory: every thread stores its partials,
// warp 0 adds them (lane l takes threads l, l+32, ...), then a shuffle tree; thread 0 holds the
// totals.  Only warp 0 issues FP64 adds, which matters on a GPU whose FP64 rate is low.
template <int THREADS, int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* sm) {
  const int tid = threadIdx.x, lane = tid & 31;
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; ++k) sm[k * THREADS + tid] = v[k];
  __syncthreads();
  if (tid < 32) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double s0 = 0.0, s1 = 0.0;
#pragma unroll 8
      for (int j = 0; j < THREADS / 32; j += 2) {
        s0 += sm[k * THREADS + j * 32 + lane];
        s1 += sm[k * THREADS + (j + 1) * 32 + lane];
      }
      v[k] = warp_sum(s0 + s1);
    }
  }
}

// Warp 0 of every block reduces the per-block partials in the same order; lane 0 of warp 0
// holds the totals.  Every block obtains bitwise the same totals.  Up to 160 partials (one wave
// of 148 blocks) every lane issues all its loads before adding them: one round trip to L2.
__device__ __forceinline__ void grid_sum_warp0(const double* part, int stride, unsigned nb,
                                               double& a, double& b, bool two) {
  const int lane = threadIdx.x & 31;
  double sa = 0.0, sb = 0.0;
  if (nb <= 160) {
    double va[5], vb[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      const unsigned i = lane + 32 * k;
      va[k] = i < nb ? __ldcg(&part[(size_t)i * stride]) : 0.0;
      vb[k] = two && i < nb ? __ldcg(&part[(size_t)i * stride + 1]) : 0.0;
    }
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      if (lane + 32 * k < nb) {
        sa += va[k];
        sb += vb[k];
      }
    }
  } else {
    unsigned i = lane;
    for (; i + 96 < nb; i += 128) {   // four loads in flight per lane
      const double a0 = __ldcg(&part[(size_t)i * stride]);
      const double a1 = __ldcg(&part[(size_t)(i + 32) * stride]);
      const double a2 = __ldcg(&part[(size_t)(i + 64) * stride]);
      const double a3 = __ldcg(&part[(size_t)(i + 96) * stride]);
      double b0 = 0.0, b1 = 0.0, b2 = 0.0, b3 = 0.0;
      if (two) {
        b0 = __ldcg(&part[(size_t)i * stride + 1]);
        b1 = __ldcg(&part[(size_t)(i + 32) * stride + 1]);
        b2 = __ldcg(&part[(size_t)(i + 64) * stride + 1]);
        b3 = __ldcg(&part[(size_t)(i + 96) * stride + 1]);
      }
      sa += a0;
      sa += a1;
      sa += a2;
      sa += a3;
      sb += b0;
      sb += b1;
      sb += b2;
      sb += b3;
    }
    for (; i < nb; i += 32) {
      sa += __ldcg(&part[(size_t)i * stride]);
      if (two) sb += __ldcg(&part[(size_t)i * stride + 1]);
    }
  }
  a = warp_sum(sa);
  b = two ? warp_sum(sb) : 0.0;
}

// L2 eviction policies for the matrix streams (createpolicy; hints only).  keep: a fixed fraction
// of the lines accessed is marked evict-last and the rest evict-first, so that the A-product's
// repeated passes find that fraction in L2 without the whole matrix displacing it; frac = 0 gives
// the normal policy.  stream: evict-first, for data read once per step (M, K in the RHS pass).
__device__ __forceinline__ uint64_t l2_policy_keep(float frac) {
  uint64_t pol;
  if (frac > 0.f)
    asm volatile("createpolicy.fractional.L2::evict_last.L2::evict_first.b64 %0, %1;" : "=l"(pol) : "f"(frac));
  else
    asm volatile("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ uint64_t l2_policy_stream() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ double ld_hint(const double* p, uint64_t pol) {
  double v;
  asm volatile("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ float ld_hint(const float* p, uint64_t pol) {
  float v;
  asm volatile("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ int ld_hint(const uint16_t* p, uint64_t pol) {
  unsigned short v;
  asm volatile("ld.global.nc.L2::cache_hint.u16 %0, [%1], %2;" : "=h"(v) : "l"(p), "l"(pol));
  return (int)v;
}
__device__ __forceinline__ int ld_hint(const int32_t* p, uint64_t pol) {
  int v;
  asm volatile("ld.global.nc.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
  return v;
}

// Back to the normal eviction priority for the 128-byte lines of [p, p + bytes) (the lines of
// the matrix marked evict-last would otherwise outlast the solve and crowd other work's data).
static __global__ void l2_normal_priority_kernel(const char* p, int64_t lines) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < lines) asm volatile("applypriority.global.L2::evict_normal [%0], 128;" ::"l"(p + 128 * i) : "memory");
}

__device__ __forceinline__ double fmaT(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fmaT(float a, float b, float c) { return fmaf(a, b, c); }

// Row products over one SELL slice, lane = row.  Even entries accumulate in acc0 and odd entries
// in acc1, each in entry order, so every shape below gives the same bits.  The product is bound by
// the latency of its rounds of dependent loads (index, then gathered vector entry); which shape
// hides that best depends on the launch (measured on the 40x16x6 mm slab):
//  kSellChunk8   predicated chunks of eight entries: indices and values of a chunk together, then
//                its gathers, then its FMAs - a 15-entry row is two rounds.  Standalone FP64
//                SpMV with 18 two-warp blocks per SM: 22.8 us against 28.0 us for kSellUnroll4;
//                also the FP32 PCG, whose working set stays in L2.
//  kSellUnroll4  four entries per round, then the last w mod 4 one at a time; fewer live
//                registers.  The FP64 PCG (1,024-thread blocks, 64 registers at most) runs 5 %
//                faster with it than with kSellChunk8, and 2 % faster than with predicated
//                rounds of four (a 15-entry row in four rounds, no entry loaded on its own).
// Entries past a row's width are neither loaded nor added; the predicates are uniform across the
// warp (one width per slice).
constexpr int kSellUnroll4 = 0;
constexpr int kSellChunk8 = 1;

template <int SHAPE, typename T, typename XF, typename I>
__device__ __forceinline__ T sell_dot_f(const I* __restrict__ col, const T* __restrict__ val,
                                        int beg, int w, XF xf, uint64_t pol = 0) {
  T acc0 = T(0), acc1 = T(0);
  if constexpr (SHAPE == kSellChunk8) {
    for (int j = 0; j < w; j += 8) {
      const int e = beg + 32 * j;
      int c[8];
      T v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        c[u] = j + u < w ? (int)__ldg(col + e + 32 * u) : 0;
        v[u] = j + u < w ? __ldg(val + e + 32 * u) : T(0);
      }
      T xv[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) xv[u] = j + u < w ? xf(c[u]) : T(0);
#pragma unroll
      for (int u = 0; u < 8; u += 2) {
        if (j + u < w) acc0 = fmaT(v[u], xv[u], acc0);
        if (j + u + 1 < w) acc1 = fmaT(v[u + 1], xv[u + 1], acc1);
      }
    }
  } else {
    int j = 0;
    // indices and values with the caller's L2 policy (pol)
    for (; j + 4 <= w; j += 4) {
      const int e = beg + 32 * j;
      const int c0 = ld_hint(col + e, pol), c1 = ld_hint(col + e + 32, pol), c2 = ld_hint(col + e + 64, pol),
                c3 = ld_hint(col + e + 96, pol);
      const T v0 = ld_hint(val + e, pol), v1 = ld_hint(val + e + 32, pol), v2 = ld_hint(val + e + 64, pol),
              v3 = ld_hint(val + e + 96, pol);
      const T x0 = xf(c0), x1 = xf(c1), x2 = xf(c2), x3 = xf(c3);
      acc0 = fmaT(v0, x0, acc0);
      acc1 = fmaT(v1, x1, acc1);
      acc0 = fmaT(v2, x2, acc0);
      acc1 = fmaT(v3, x3, acc1);
    }
    // the tail: one FMA each into acc0, then the two sums trade places so that the next entry
    // goes to the other one (a branch on the entry's parity was if-converted into both FMAs, a
    // fifth more FP64 work on a 15-entry row); the final sum is symmetric
    for (; j < w; ++j) {
      const int e = beg + 32 * j;
      acc0 = fmaT(ld_hint(val + e, pol), xf(ld_hint(col + e, pol)), acc0);
      const T t = acc0;
      acc0 = acc1;
      acc1 = t;
    }
  }
  return acc0 + acc1;
}

// The product gathering from a global vector x.
template <int SHAPE, typename T>
__device__ __forceinline__ T sell_dot(const int32_t* __restrict__ col, const T* __restrict__ val,
                                     int beg, int w, const T* x, uint64_t pol = 0) {
  return sell_dot_f<SHAPE>(col, val, beg, w, [x](int c) { return x[c]; }, pol);
}

// Copy x[lo, lo + len) into shared memory xs (lo and len multiples of 4, so every access is a
// 16-byte vector), bypassing L1: the vector was written by other blocks of the launch before
// the grid barrier that precedes this copy.  Four vectors per thread are loaded before they are
// stored, so that a thread has four loads in flight.
template <int THREADS, typename T>
__device__ __forceinline__ void stage_window(T* xs, const T* __restrict__ x, int lo, int len) {
  using V = typename std::conditional<sizeof(T) == 8, double2, float4>::type;
  constexpr int PER = 16 / sizeof(T);
  const V* src = reinterpret_cast<const V*>(x + lo);
  V* dst = reinterpret_cast<V*>(xs);
  const int nv = len / PER;
  int i = threadIdx.x;
  for (; i + 3 * THREADS < nv; i += 4 * THREADS) {
    const V a0 = __ldcg(src + i), a1 = __ldcg(src + i + THREADS), a2 = __ldcg(src + i + 2 * THREADS),
            a3 = __ldcg(src + i + 3 * THREADS);
    dst[i] = a0;
    dst[i + THREADS] = a1;
    dst[i + 2 * THREADS] = a2;
    dst[i + 3 * THREADS] = a3;
  }
  for (; i < nv; i += THREADS) dst[i] = __ldcg(src + i);
}

// The shape of the PCG's product per storage type (see above).
#ifndef TC_PCG_SELL_SHAPE_F64
#define TC_PCG_SELL_SHAPE_F64 kSellUnroll4
#endif
template <typename T>
__host__ __device__ constexpr int pcg_sell_shape() {
  return sizeof(T) == 8 ? TC_PCG_SELL_SHAPE_F64 : kSellChunk8;
}

// Two value streams over the same pattern: am = sum M_ij g1_j, ak = sum K_ij g2_j, each in entry
// order.  FP32: predicated chunks of eight entries (indices and values of a chunk first, then its
// gathers, then its FMAs: a 15-entry row takes two rounds of dependent loads; the predicates are
// uniform across the warp).  FP64: two entries per round (chunks of four spill at 64 registers).
template <typename T, typename I>
__device__ __forceinline__ void sell_dot2(const I* __restrict__ col, const T* __restrict__ vm,
                                          const T* __restrict__ vk, int beg, int w,
                                          const T* __restrict__ g1, const T* __restrict__ g2,
                                          T& am, T& ak) {
  am = T(0);
  ak = T(0);
  const uint64_t pol = l2_policy_stream();   // M and K are read once per step
  if constexpr (sizeof(T) == 4) {
    constexpr int CH = 8;
    for (int j = 0; j < w; j += CH) {
      const int e = beg + 32 * j;
      int c[CH];
      T m[CH], k[CH], ga[CH], gb[CH];
#pragma unroll
      for (int u = 0; u < CH; ++u) {
        c[u] = 0;
        m[u] = k[u] = T(0);
        if (j + u < w) {
          c[u] = (int)__ldg(col + e + 32 * u);
          m[u] = ld_hint(vm + e + 32 * u, pol);
          k[u] = ld_hint(vk + e + 32 * u, pol);
        }
      }
#pragma unroll
      for (int u = 0; u < CH; ++u) {
        ga[u] = gb[u] = T(0);
        if (j + u < w) {
          ga[u] = __ldg(g1 + c[u]);
          gb[u] = __ldg(g2 + c[u]);
        }
      }
#pragma unroll
      for (int u = 0; u < CH; ++u) {
        if (j + u < w) {
          am = fmaT(m[u], ga[u], am);
          ak = fmaT(k[u], gb[u], ak);
        }
      }
    }
  } else {
    int j = 0;
    for (; j + 2 <= w; j += 2) {
      const int e = beg + 32 * j;
      const int c0 = (int)__ldg(col + e), c1 = (int)__ldg(col + e + 32);
      const T m0 = ld_hint(vm + e, pol), m1 = ld_hint(vm + e + 32, pol);
      const T k0 = ld_hint(vk + e, pol), k1 = ld_hint(vk + e + 32, pol);
      const T a0 = __ldg(g1 + c0), a1 = __ldg(g1 + c1);
      const T b0 = __ldg(g2 + c0), b1 = __ldg(g2 + c1);
      am = fmaT(m0, a0, am);
      ak = fmaT(k0, b0, ak);
      am = fmaT(m1, a1, am);
      ak = fmaT(k1, b1, ak);
    }
    for (; j < w; ++j) {
      const int e = beg + 32 * j;
      const int c = (int)__ldg(col + e);
      am = fmaT(ld_hint(vm + e, pol), __ldg(g1 + c), am);
      ak = fmaT(ld_hint(vk + e, pol), __ldg(g2 + c), ak);
    }
  }
}

// Stimulus current of node i at step k (sum over the stimuli that list the node, in order).
__device__ __forceinline__ double stimulus_at(const int32_t* off, const int32_t* ids,
                                              const StimDev* stims, int64_t i, long long k) {
  double is = 0.0;
  for (int e = off[i]; e < off[i + 1]; ++e) {
    const StimDev s = stims[ids[e]];
    if (k >= s.k0 && k < s.k0 + s.nk) is += s.amp;
  }
  return is;
}

// Right-hand-side node vectors and initial guess from V^k, V^{k-1}, I_ion and I_stim.
template <typename T>
__device__ __forceinline__ void rhs_epilogue(const IonicArgs<T>& a, int64_t i, T V, T Vp, T iion,
                                             T is) {
  const T chi = T(a.chi), cm = T(a.cm), dt = T(a.dt), th = T(a.theta);
  a.g1[i] = chi * (cm * (Vp - V) + dt * (is - iion));
  a.g2[i] = dt * (V + th * (V - Vp));
  a.x0[i] = T(2) * V - Vp;
}

// (a1) Ionic update of node i, Mitchell-Schaeffer with a Rush-Larsen gate (state[0] = h), and
// the node's right-hand-side inputs.
template <typename T>
__device__ __forceinline__ void ms_node(const IonicArgs<T>& a, int64_t i) {
  const T V = a.V[i], Vp = a.Vp[i];
  const MSConst& c = a.ms;
  const T v = (V - T(c.vmin)) * T(c.inv_range);
  const bool closing = v >= T(c.vgate);
  const T hinf = closing ? T(0) : T(1);
  const T h = hinf + (a.state[i] - hinf) * (closing ? T(c.dec_close) : T(c.dec_open));
  a.state[i] = h;
  const T jin = h * v * v * (T(1) - v) * T(c.inv_tau_in);
  const T jout = -v * T(c.inv_tau_out);
  const T iion = -T(a.cm) * T(c.range) * (jin + jout);
  const T is = T(stimulus_at(a.stim_off, a.stim_ids, a.stims, i, *a.k_base + a.k_off));
  rhs_epilogue(a, i, V, Vp, iion, is);
}

template <typename T>
__global__ void __launch_bounds__(256) ionic_ms_kernel(const IonicArgs<T> a) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < a.n_bar) a.bar[i].count = 0u;
  if (i >= a.n) return;
  ms_node(a, i);
}

// Advances the device step index after a group of steps (the last node of a captured graph).
static __global__ void tick_kernel(long long* k_base, int add) { *k_base += add; }

// (a2)-(a5) in one cooperative launch: r0 = b - A x0 from the two value streams of M and K,
// the Jacobi-PCG loop of Algorithm 1 with the convergence decision taken identically by every
// block, and the activation-time capture.  Each block owns a contiguous range of slices (and
// so of rows); SpMV phases map one warp to one slice, vector phases stride threads over the
// block's rows.  Scalar FP64 work (sqrt, divisions, the stopping test) runs on thread 0 only:
// B300 issues FP64 at a small fraction of its FP32 rate.  A mesh made of several connected
// components is several independent problems: each component owns a contiguous range of
// blocks and runs its own PCG (own barrier, reductions, alpha, beta, stopping decision), so a
// batch of meshes advances in one launch without any instance waiting for another.
template <int THREADS, typename T>
__device__ __forceinline__ void pcg_step(const PcgArgs<T>& a) {
  constexpr int NW = THREADS / 32;
  __shared__ double s_red[2 * THREADS];
  __shared__ double s_sc[4];   // scalars computed by thread 0, then broadcast
  __shared__ int s_flag;       // 0 = iterate, 1 = converged, 2 = non-finite
  __shared__ T s_part[THREADS];   // partial row products of a split last round
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned b = blockIdx.x;
  const int comp = a.comp_of_block[b];
  const int cb0 = a.comp_block0[comp];
  const unsigned nb = (unsigned)(a.comp_block0[comp + 1] - cb0);
  GridBar* bar = a.bar + comp;
  const int s0 = a.blk_slice[b], s1 = a.blk_slice[b + 1];
  const int64_t r0 = (int64_t)s0 * 32;
  const int64_t r1 = min((int64_t)s1 * 32, a.n);
  unsigned epoch = 0;
  double rho = 0.0, z0n = 0.0, zn = 0.0;   // meaningful in thread 0
  const uint64_t pol_a = l2_policy_keep(a.l2_keep);
  // the ionic kernel launched before this one has left the logarithms of the new states
  if (a.log_valid && b == 0 && tid == 0) *a.log_valid = 1;
  int it = 0;

  // (a1) inside the launch (Mitchell-Schaeffer): every block updates its rows, then a barrier,
  // because the right-hand side gathers neighbours' g1 and g2
  if (a.fuse_ms) {
    for (int64_t i = r0 + tid; i < r1; i += THREADS) ms_node(a.ion, i);
    if (!grid_sync(bar, nb, epoch, a.wait_limit, a.err)) return;
  }
  // The block's window (blk_win: lo, len): its columns lie in [lo, lo + span); with col16 every
  // entry's column is stored as a 16-bit offset from lo (half the index stream).  len > 0 when the
  // window is staged in shared memory (see the loop below).
  const int win_lo = a.blk_win[2 * b], win_len = a.blk_win[2 * b + 1];
  const bool use16 = a.col16 != nullptr;
  // r0 = chi M (w - Cm x0) - dt K ((1-theta) V + theta x0) = M g1 - K g2
  T rho_t = T(0), zz_t = T(0);
  for (int s = s0 + warp; s < s1; s += NW) {
    const int beg = a.slice_ptr[s] + lane;
    const int w = (a.slice_ptr[s + 1] - a.slice_ptr[s]) >> 5;
    T am, ak;
    if (use16)
      sell_dot2(a.col16, a.vM, a.vK, beg, w, a.g1 + win_lo, a.g2 + win_lo, am, ak);
    else
      sell_dot2(a.col, a.vM, a.vK, beg, w, a.g1, a.g2, am, ak);
    const int64_t row = (int64_t)s * 32 + lane;
    if (row < a.n) {
      const T rr = am - ak;
      const T zv = __ldg(&a.dinv[row]) * rr;
      a.r[row] = rr;
      a.z[row] = zv;
      rho_t = fmaT(rr, zv, rho_t);
      zz_t = fmaT(zv, zv, zz_t);
    }
  }
  {
    double v2[2] = {double(rho_t), double(zz_t)};
    block_sum<THREADS, 2>(v2, s_red);
    if (tid == 0) {
      a.partB[2 * b] = v2[0];
      a.partB[2 * b + 1] = v2[1];
    }
  }
  if (!grid_sync(bar, nb, epoch, a.wait_limit, a.err)) return;
  if (warp == 0) {
    double t_rho, t_zz;
    grid_sum_warp0(a.partB + 2 * cb0, 2, nb, t_rho, t_zz, true);
    if (tid == 0) {
      rho = t_rho;
      z0n = sqrt(t_zz);
      zn = z0n;
      s_flag = !(z0n == z0n) ? 2 : (z0n == 0.0 || z0n < a.atol) ? 1 : 0;
    }
  }
  __syncthreads();
  int flag = s_flag;
  T beta = T(0);
  // The block's slices go to its warps in rounds of NW.  A short last round of R slices leaves
  // NW - R warps idle while the others take whole slices (3 1/3 slices per warp on the
  // 40x16x6 mm slab).  FP64: with R <= NW/2 each of those slices is split into G column ranges,
  // one warp each, whose partial products are added in range order through shared memory (PCG
  // launch 0.471 -> 0.462 ms on the slab).  FP32 keeps whole slices (the split was 2.6 % slower:
  // its cheaper product does not pay for the extra block barrier).
  const int n_sl = s1 - s0;
  const int tail_r = n_sl % NW;
  const int tail_g = tail_r == 0 ? 1 : min(NW / tail_r, 8);
  const bool split = sizeof(T) == 8 && tail_g >= 2;
  const int n_whole = split ? n_sl - tail_r : n_sl;
  // The block's window of z in shared memory (blk_win: lo, len; len = 0 when it does not fit):
  // the product's gathers then read shared memory instead of waiting on L2 for every entry.
  extern __shared__ __align__(16) unsigned char s_dyn[];
  T* s_x = reinterpret_cast<T*>(s_dyn);
  const bool staged = win_len > 0;
  while (flag == 0 && it < a.max_iter) {
    // p = z + beta p and q = A p, formed as q = A z + beta q (A p_k = A z_k + beta A p_{k-1}):
    // the product gathers z, complete since the last barrier, so p and q are updated row by row
    // without a barrier of their own; then p^T q
    T pq_t = T(0);
    auto load_row = [&](int64_t row, T& zr, T& pr, T& qr) {
      zr = a.z[row];
      if (it > 0) {
        pr = a.p[row];
        qr = a.q[row];
      }
    };
    auto store_row = [&](int64_t row, T acc, T zr, T pr, T qr) {
      T pn = zr, qn = acc;
      if (it > 0) {
        pn = fmaT(beta, pr, zr);
        qn = fmaT(beta, qr, acc);
      }
      a.p[row] = pn;
      a.q[row] = qn;
      pq_t = fmaT(pn, qn, pq_t);
    };
    if (staged) {
      stage_window<THREADS>(s_x, a.z, win_lo, win_len);
      __syncthreads();
    }
    // the product over the block's slices; `from_smem` selects the gather source and `idx16` the
    // index stream at compile time
    auto product = [&](auto from_smem, auto idx16) {
      constexpr bool kSmem = decltype(from_smem)::value;
      constexpr bool k16 = decltype(idx16)::value;
      auto xf = [&](int c) -> T {
        if constexpr (kSmem) {
          if constexpr (k16) return s_x[c];
          else return s_x[c - win_lo];
        } else {
          if constexpr (k16) return a.z[win_lo + c];
          else return a.z[c];
        }
      };
      const auto* colp = [&]() {
        if constexpr (k16) return a.col16;
        else return a.col;
      }();
      for (int s = s0 + warp; s < s0 + n_whole; s += NW) {
        const int beg = a.slice_ptr[s] + lane;
        const int w = (a.slice_ptr[s + 1] - a.slice_ptr[s]) >> 5;
        const int64_t row = (int64_t)s * 32 + lane;
        const bool real = row < a.n;
        // FP32: the row's own z, p, q are loaded before the product so that their latency
        // overlaps its loads (loaded after it they cost a round trip per slice: 15 % on the
        // 64-slab batch, about 35 slices per warp).  FP64: after it - holding them across the
        // product would spill at 1,024 threads.
        T zr = T(0), pr = T(0), qr = T(0);
        if constexpr (sizeof(T) == 4) {
          if (real) load_row(row, zr, pr, qr);
        }
        const T acc = sell_dot_f<pcg_sell_shape<T>()>(colp, a.vA, beg, w, xf, pol_a);
        if constexpr (sizeof(T) == 8) {
          if (real) load_row(row, zr, pr, qr);
        }
        if (real) store_row(row, acc, zr, pr, qr);
      }
      if (split) {
        const int t = warp / tail_g, c = warp - t * tail_g;
        const int s = s0 + n_whole + t;
        const int64_t row = (int64_t)s * 32 + lane;
        const bool real = t < tail_r && row < a.n;
        T zr = T(0), pr = T(0), qr = T(0);
        if (t < tail_r) {
          const int beg = a.slice_ptr[s] + lane;
          const int w = (a.slice_ptr[s + 1] - a.slice_ptr[s]) >> 5;
          const int per = (w + tail_g - 1) / tail_g;
          const int j0 = min(w, c * per), j1 = min(w, j0 + per);
          if constexpr (sizeof(T) == 4) {
            if (c == 0 && real) load_row(row, zr, pr, qr);
          }
          s_part[warp * 32 + lane] = sell_dot_f<pcg_sell_shape<T>()>(colp, a.vA, beg + 32 * j0, j1 - j0, xf, pol_a);
        }
        __syncthreads();
        if (c == 0 && real) {
          T acc = s_part[warp * 32 + lane];
          for (int k = 1; k < tail_g; ++k) acc += s_part[(warp + k) * 32 + lane];
          if constexpr (sizeof(T) == 8) load_row(row, zr, pr, qr);
          store_row(row, acc, zr, pr, qr);
        }
      }
    };
    if (staged) {
      if (use16) product(std::true_type{}, std::true_type{});
      else product(std::true_type{}, std::false_type{});
    } else {
      if (use16) product(std::false_type{}, std::true_type{});
      else product(std::false_type{}, std::false_type{});
    }
    {
      double v1[1] = {double(pq_t)};
      block_sum<THREADS, 1>(v1, s_red);
      if (tid == 0) a.partA[b] = v1[0];
    }
    if (!grid_sync(bar, nb, epoch, a.wait_limit, a.err)) return;
    if (warp == 0) {
      double pq, unused;
      grid_sum_warp0(a.partA + cb0, 1, nb, pq, unused, false);
      if (tid == 0) {
        s_sc[0] = rho / pq;
        s_sc[1] = pq;
      }
    }
    __syncthreads();
    const T alpha = T(s_sc[0]);
    // x += alpha p, r -= alpha q, z = D^-1 r, rho' = r^T z, ||z||^2.  Each thread takes rows
    // i, i + THREADS, ... in that order (the same sums either way).  FP64 and 1,024-thread FP32:
    // the loads for four rows are issued before their arithmetic (FP64 PCG 2.4 %, FP32 1.6 %
    // faster on the 40x16x6 mm slab); 512-thread FP32 (the batched form's shape): two rows per
    // round (the four-row form was 10 % slower there).  FP64 updates x after this block's arrival
    // at the barrier below, while the other blocks arrive (no other block reads x): FP64 PCG
    // 0.485 -> 0.472 ms on the slab; FP32 was slower that way (1.9 % slab, 11 % 64-slab batch).
    constexpr bool kLateX = sizeof(T) == 8;
    rho_t = T(0);
    zz_t = T(0);
    if constexpr (sizeof(T) == 8 || THREADS == 1024) {
      for (int64_t i = r0 + tid; i < r1; i += 4 * THREADS) {
        T pv[4], qv[4], xv[4], rv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int64_t iu = i + (int64_t)u * THREADS;
          const bool ok = iu < r1;
          if constexpr (!kLateX) {
            pv[u] = ok ? a.p[iu] : T(0);
            xv[u] = ok ? a.x[iu] : T(0);
          }
          qv[u] = ok ? a.q[iu] : T(0);
          rv[u] = ok ? a.r[iu] : T(0);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int64_t iu = i + (int64_t)u * THREADS;
          if (iu < r1) {
            if constexpr (!kLateX) a.x[iu] = fmaT(alpha, pv[u], xv[u]);
            const T ri = fmaT(-alpha, qv[u], rv[u]);
            a.r[iu] = ri;
            const T zi = __ldg(&a.dinv[iu]) * ri;
            a.z[iu] = zi;
            rho_t = fmaT(ri, zi, rho_t);
            zz_t = fmaT(zi, zi, zz_t);
          }
        }
      }
    } else {
      for (int64_t i = r0 + tid; i < r1; i += 2 * THREADS) {
        const int64_t i2 = i + THREADS;
        const bool two = i2 < r1;
        const T p0 = a.p[i], q0 = a.q[i], x0 = a.x[i], rr0 = a.r[i], d0 = __ldg(&a.dinv[i]);
        T p1 = T(0), q1 = T(0), x1 = T(0), rr1 = T(0), d1 = T(0);
        if (two) {
          p1 = a.p[i2];
          q1 = a.q[i2];
          x1 = a.x[i2];
          rr1 = a.r[i2];
          d1 = __ldg(&a.dinv[i2]);
        }
        a.x[i] = fmaT(alpha, p0, x0);
        const T ri = fmaT(-alpha, q0, rr0);
        a.r[i] = ri;
        const T zi = d0 * ri;
        a.z[i] = zi;
        rho_t = fmaT(ri, zi, rho_t);
        zz_t = fmaT(zi, zi, zz_t);
        if (two) {
          a.x[i2] = fmaT(alpha, p1, x1);
          const T rj = fmaT(-alpha, q1, rr1);
          a.r[i2] = rj;
          const T zj = d1 * rj;
          a.z[i2] = zj;
          rho_t = fmaT(rj, zj, rho_t);
          zz_t = fmaT(zj, zj, zz_t);
        }
      }
    }
    {
      double v2[2] = {double(rho_t), double(zz_t)};
      block_sum<THREADS, 2>(v2, s_red);
      if (tid == 0) {
        a.partB[2 * b] = v2[0];
        a.partB[2 * b + 1] = v2[1];
      }
    }
    if constexpr (kLateX) {
      grid_arrive(bar, nb, epoch);
      // x += alpha p while the other blocks arrive
      for (int64_t i = r0 + tid; i < r1; i += 2 * THREADS) {
        const int64_t i2 = i + THREADS;
        const T p0 = a.p[i], x0 = a.x[i];
        T p1 = T(0), x1 = T(0);
        if (i2 < r1) {
          p1 = a.p[i2];
          x1 = a.x[i2];
        }
        a.x[i] = fmaT(alpha, p0, x0);
        if (i2 < r1) a.x[i2] = fmaT(alpha, p1, x1);
      }
      if (!grid_wait(bar, nb, epoch, a.wait_limit, a.err)) return;
    } else {
      if (!grid_sync(bar, nb, epoch, a.wait_limit, a.err)) return;
    }
    ++it;
    if (warp == 0) {
      double rho_new, zz;
      grid_sum_warp0(a.partB + 2 * cb0, 2, nb, rho_new, zz, true);
      if (tid == 0) {
        zn = sqrt(zz);
        const double pq = s_sc[1];
        int f = 0;
        if (!(zn == zn) || !(pq == pq)) f = 2;
        else if (zn < a.atol || zn / z0n < a.rtol) f = 1;
        s_sc[2] = rho_new / rho;   // beta
        rho = rho_new;
        s_flag = f;
      }
    }
    __syncthreads();
    flag = s_flag;
    beta = T(s_sc[2]);
  }
  // activation capture (first upward crossing of thr) and, after activation, the peak, the
  // 90 % repolarisation crossing and the LRT crossing, each interpolated inside the step
  const double t_k = (double)(*a.k_base + a.k_off) * a.dt;
  for (int64_t i = r0 + tid; i < r1; i += THREADS) {
    const double vo = double(a.Vcur[i]), vn = double(a.x[i]);
    if (a.act[i] < 0.0) {
      if (vo < a.thr && vn >= a.thr) {
        a.act[i] = t_k + a.dt * (a.thr - vo) / (vn - vo);
        a.vpeak[i] = vn;
      }
    } else if (a.rep90[i] < 0.0 || a.lrt[i] < 0.0) {
      const double vp = fmax(a.vpeak[i], vn);
      a.vpeak[i] = vp;
      const double t90 = a.v_rest + 0.1 * (vp - a.v_rest);
      if (a.rep90[i] < 0.0 && vo >= t90 && vn < t90)
        a.rep90[i] = t_k + a.dt * (vo - t90) / (vo - vn);
      if (a.lrt[i] < 0.0 && vo >= a.lrt_thr && vn < a.lrt_thr)
        a.lrt[i] = t_k + a.dt * (vo - a.lrt_thr) / (vo - vn);
    }
  }
  // the last block of the component to get here (every block is past its last barrier wait)
  // returns the barrier words to zero for the next launch on the stream
  if (tid == 0 && nb > 1) {
    if (atomicAdd(&bar->gen, 1u) == nb - 1) {
      bar->count = 0u;
      bar->gen = 0u;
    }
  }
  if (b == (unsigned)cb0 && tid == 0) {
    DevStats* st = a.stats + comp;
    st->iters_total += it;
    st->steps += 1;
    if (it > st->max_iters) st->max_iters = it;
    if (flag != 1) st->not_conv += 1;
    st->last_iters = it;
    st->last_zn = zn;
    st->last_z0n = z0n;
    if (flag == 2) atomicOr(a.err, kErrNan);
  }
}

// The launch entry points, one per block size, because their launch bounds differ (measured
// against one template with either form for both): 1,024 threads with one block per SM stated
// (64 registers; the FP32 PCG 3 % faster on the 40x16x6 mm slab than without the block count,
// FP64 within 0.2 %), 512 threads with none (64 registers by the compiler's choice; the 64-slab
// batch steps 9 % faster than with two blocks per SM stated, at the same register count).
template <typename T>
__global__ void __launch_bounds__(1024, 1) pcg_step_kernel_1024(const PcgArgs<T> a) {
  pcg_step<1024, T>(a);
}
template <typename T>
__global__ void __maxnreg__(64) pcg_step_kernel_512(const PcgArgs<T> a) {
  pcg_step<512, T>(a);
}

// col16[e] = col[e] - lo of the PCG block that owns entry e's slice (one CTA per PCG block; every
// column of the block's slices lies in [lo, lo + 65536), checked on the host).
static __global__ void col16_kernel(const int32_t* __restrict__ blk_slice, const int32_t* __restrict__ slice_ptr,
                                    const int32_t* __restrict__ col, const int32_t* __restrict__ blk_win,
                                    uint16_t* __restrict__ col16) {
  const int b = blockIdx.x;
  const int lo = blk_win[2 * b];
  const int e0 = slice_ptr[blk_slice[b]], e1 = slice_ptr[blk_slice[b + 1]];
  for (int e = e0 + (int)threadIdx.x; e < e1; e += blockDim.x) col16[e] = (uint16_t)(col[e] - lo);
}

// Standalone y = Op x (the SpMV of Algorithm 1) for operator checks and bandwidth runs.
template <typename T>
__global__ void __launch_bounds__(256) spmv_sell_kernel(int64_t n, int64_t nslices,
                                                        const int32_t* __restrict__ slice_ptr,
                                                        const int32_t* __restrict__ col,
                                                        const T* __restrict__ val,
                                                        const T* __restrict__ x,
                                                        T* __restrict__ y) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t s = gw; s < nslices; s += nw) {
    const int beg = slice_ptr[s] + lane;
    const int w = (slice_ptr[s + 1] - slice_ptr[s]) >> 5;
    const T acc = sell_dot<kSellChunk8>(col, val, beg, w, x);
    const int64_t row = s * 32 + lane;
    if (row < n) y[row] = acc;
  }
}

}  // namespace tc
