// Device kernels of the monodomain time step (FP64 path).
//
// Data layout (all in the internal node order: reverse Cuthill-McKee, then SELL-C-sigma row
// sorting): matrices in SELL-C-sigma with C = 32 (one warp per slice, one lane per row;
// entry j of the row in lane l of slice s sits at slice_ptr[s] + 32*j + l), one shared int32
// column array and one value array per matrix (M, K, A); node vectors are dense arrays.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

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

struct IonicArgs {
  int64_t n;
  const double* V;        // V^k
  const double* Vp;       // V^{k-1}
  double* h;              // gate (in place)
  double* g1;             // chi (Cm (V^{k-1} - V^k) + dt (I_stim - I_ion))
  double* g2;             // dt (V^k + theta (V^k - V^{k-1}))
  double* x0;             // 2 V^k - V^{k-1}: PCG initial guess, written into the V^{k+1} buffer
  const int32_t* stim_off;
  const int32_t* stim_ids;
  const StimDev* stims;
  long long k;
  double chi, cm, dt, theta;
  MSConst ms;
};

struct PcgArgs {
  int64_t n;
  const int32_t* slice_ptr;
  const int32_t* col;
  const double* vM;
  const double* vK;
  const double* vA;
  const double* dinv;
  const int32_t* blk_slice;   // gridDim.x + 1 slice boundaries
  const double* g1;
  const double* g2;
  double* x;                  // in: x0, out: V^{k+1}
  const double* Vcur;         // V^k (activation capture)
  double* r;
  double* z;
  double* p;
  double* q;
  double* act;
  double* partA;              // gridDim.x
  double* partB;              // 2*gridDim.x
  GridBar* bar;
  int* err;
  DevStats* stats;
  double atol, rtol;
  int max_iter;
  long long wait_limit;
  double t_k, dt, thr;
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid-wide barrier for a cooperative launch (all blocks co-resident).  Every wait is bounded:
// after wait_limit polls the block records kErrTimeout and leaves; a block that sees any error
// flag returns false so that the kernel can exit without further waits.
__device__ __forceinline__ bool grid_sync(GridBar* bar, unsigned nblocks, long long wait_limit,
                                          int* err) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = *(volatile int*)err ? 0 : 1;   // after an error, leave without waiting
    if (ok && nblocks > 1) {
      const unsigned g = ld_acquire_u32(&bar->gen);
      __threadfence();
      const unsigned prev = atomicAdd(&bar->count, 1u);
      if (prev == nblocks - 1) {
        atomicExch(&bar->count, 0u);
        __threadfence();
        atomicAdd(&bar->gen, 1u);
      } else {
        long long polls = 0;
        while (ld_acquire_u32(&bar->gen) == g) {
          if (++polls > wait_limit) {
            atomicOr(err, kErrTimeout);
            ok = 0;
            break;
          }
          if (polls > 256) __nanosleep(32);
        }
      }
      __threadfence();
    }
    if (ok && *(volatile int*)err) ok = 0;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Fixed-order sums: lane 0 of a warp gets the shfl_down tree sum; warp sums are added in warp
// order.  The result is a pure function of the inputs' placement, so runs are bitwise equal.
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

template <int NW>
__device__ __forceinline__ void block_sum2(double& a, double& b, double* sm) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  a = warp_sum(a);
  b = warp_sum(b);
  __syncthreads();
  if (lane == 0) {
    sm[warp] = a;
    sm[NW + warp] = b;
  }
  __syncthreads();
  if (warp == 0) {
    a = lane < NW ? sm[lane] : 0.0;
    b = lane < NW ? sm[NW + lane] : 0.0;
    a = warp_sum(a);
    b = warp_sum(b);
  }
}

// Every block reduces the per-block partials in the same order and broadcasts the result.
template <int NW>
__device__ __forceinline__ void grid_sum2(const double* part, int stride, unsigned nb, double& a,
                                          double& b, double* bc, bool two) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (warp == 0) {
    double sa = 0.0, sb = 0.0;
    for (unsigned i = lane; i < nb; i += 32) {
      sa += __ldcg(&part[(size_t)i * stride]);
      if (two) sb += __ldcg(&part[(size_t)i * stride + 1]);
    }
    sa = warp_sum(sa);
    sb = warp_sum(sb);
    if (lane == 0) {
      bc[0] = sa;
      bc[1] = sb;
    }
  }
  __syncthreads();
  a = bc[0];
  b = bc[1];
}

// (a1) Ionic update, Mitchell-Schaeffer with a Rush-Larsen gate, plus the per-node vectors of
// the right-hand side and the extrapolated initial guess.
__global__ void __launch_bounds__(256) ionic_ms_kernel(const IonicArgs a) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const double V = a.V[i], Vp = a.Vp[i];
  const MSConst& c = a.ms;
  const double v = (V - c.vmin) * c.inv_range;
  const bool closing = v >= c.vgate;
  const double hinf = closing ? 0.0 : 1.0;
  const double h = hinf + (a.h[i] - hinf) * (closing ? c.dec_close : c.dec_open);
  a.h[i] = h;
  const double jin = h * v * v * (1.0 - v) * c.inv_tau_in;
  const double jout = -v * c.inv_tau_out;
  const double iion = -a.cm * c.range * (jin + jout);
  double is = 0.0;
  for (int e = a.stim_off[i]; e < a.stim_off[i + 1]; ++e) {
    const StimDev s = a.stims[a.stim_ids[e]];
    if (a.k >= s.k0 && a.k < s.k0 + s.nk) is += s.amp;
  }
  a.g1[i] = a.chi * (a.cm * (Vp - V) + a.dt * (is - iion));
  a.g2[i] = a.dt * (V + a.theta * (V - Vp));
  a.x0[i] = 2.0 * V - Vp;
}

// (a2)-(a5) in one cooperative launch: r0 = b - A x0 from the two value streams of M and K,
// the Jacobi-PCG loop of Algorithm 1 with the convergence decision taken identically by every
// block, and the activation-time capture.  Each block owns a contiguous range of slices (and
// so of rows); SpMV phases map one warp to one slice, vector phases stride threads over the
// block's rows.
template <int THREADS>
__global__ void __launch_bounds__(THREADS) pcg_step_kernel(const PcgArgs a) {
  constexpr int NW = THREADS / 32;
  __shared__ double s_red[2 * NW];
  __shared__ double s_bc[2];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned nb = gridDim.x, b = blockIdx.x;
  const int s0 = a.blk_slice[b], s1 = a.blk_slice[b + 1];
  const int64_t r0 = (int64_t)s0 * 32;
  const int64_t r1 = min((int64_t)s1 * 32, a.n);

  // r0 = chi M (w - Cm x0) - dt K ((1-theta) V + theta x0) = M g1 - K g2
  double rho_l = 0.0, zz_l = 0.0;
  for (int s = s0 + warp; s < s1; s += NW) {
    const int beg = a.slice_ptr[s] + lane;
    const int w = (a.slice_ptr[s + 1] - a.slice_ptr[s]) >> 5;
    double am = 0.0, ak = 0.0;
    for (int j = 0; j < w; ++j) {
      const int e = beg + 32 * j;
      const int c = __ldg(&a.col[e]);
      am = fma(__ldg(&a.vM[e]), __ldg(&a.g1[c]), am);
      ak = fma(__ldg(&a.vK[e]), __ldg(&a.g2[c]), ak);
    }
    const int64_t row = (int64_t)s * 32 + lane;
    if (row < a.n) {
      const double rr = am - ak;
      const double zv = __ldg(&a.dinv[row]) * rr;
      a.r[row] = rr;
      a.z[row] = zv;
      a.p[row] = zv;
      rho_l = fma(rr, zv, rho_l);
      zz_l = fma(zv, zv, zz_l);
    }
  }
  block_sum2<NW>(rho_l, zz_l, s_red);
  if (tid == 0) {
    a.partB[2 * b] = rho_l;
    a.partB[2 * b + 1] = zz_l;
  }
  if (!grid_sync(a.bar, nb, a.wait_limit, a.err)) return;
  double rho, zz0;
  grid_sum2<NW>(a.partB, 2, nb, rho, zz0, s_bc, true);
  const double z0n = sqrt(zz0);
  double zn = z0n;
  int it = 0;
  bool conv = false, bad = !(z0n == z0n);
  if (!bad && (z0n == 0.0 || z0n < a.atol)) conv = true;
  while (!conv && !bad && it < a.max_iter) {
    // q = A p, p^T q
    double pq_l = 0.0, dummy = 0.0;
    for (int s = s0 + warp; s < s1; s += NW) {
      const int beg = a.slice_ptr[s] + lane;
      const int w = (a.slice_ptr[s + 1] - a.slice_ptr[s]) >> 5;
      double acc = 0.0;
      for (int j = 0; j < w; ++j) {
        const int e = beg + 32 * j;
        acc = fma(__ldg(&a.vA[e]), a.p[__ldg(&a.col[e])], acc);
      }
      const int64_t row = (int64_t)s * 32 + lane;
      if (row < a.n) {
        a.q[row] = acc;
        pq_l = fma(a.p[row], acc, pq_l);
      }
    }
    block_sum2<NW>(pq_l, dummy, s_red);
    if (tid == 0) a.partA[b] = pq_l;
    if (!grid_sync(a.bar, nb, a.wait_limit, a.err)) return;
    double pq, unused;
    grid_sum2<NW>(a.partA, 1, nb, pq, unused, s_bc, false);
    const double alpha = rho / pq;
    // x += alpha p, r -= alpha q, z = D^-1 r, rho' = r^T z, ||z||^2
    rho_l = 0.0;
    zz_l = 0.0;
    for (int64_t i = r0 + tid; i < r1; i += THREADS) {
      a.x[i] = fma(alpha, a.p[i], a.x[i]);
      const double ri = fma(-alpha, a.q[i], a.r[i]);
      a.r[i] = ri;
      const double zi = __ldg(&a.dinv[i]) * ri;
      a.z[i] = zi;
      rho_l = fma(ri, zi, rho_l);
      zz_l = fma(zi, zi, zz_l);
    }
    block_sum2<NW>(rho_l, zz_l, s_red);
    if (tid == 0) {
      a.partB[2 * b] = rho_l;
      a.partB[2 * b + 1] = zz_l;
    }
    if (!grid_sync(a.bar, nb, a.wait_limit, a.err)) return;
    double rho_new, zz;
    grid_sum2<NW>(a.partB, 2, nb, rho_new, zz, s_bc, true);
    ++it;
    zn = sqrt(zz);
    if (!(zn == zn) || !(pq == pq)) {
      bad = true;
      break;
    }
    if (zn < a.atol || zn / z0n < a.rtol) {
      conv = true;
      break;
    }
    const double beta = rho_new / rho;
    rho = rho_new;
    for (int64_t i = r0 + tid; i < r1; i += THREADS) a.p[i] = fma(beta, a.p[i], a.z[i]);
    if (!grid_sync(a.bar, nb, a.wait_limit, a.err)) return;
  }
  // activation capture: first upward crossing of thr, interpolated inside the step
  for (int64_t i = r0 + tid; i < r1; i += THREADS) {
    if (a.act[i] < 0.0) {
      const double vo = a.Vcur[i], vn = a.x[i];
      if (vo < a.thr && vn >= a.thr) a.act[i] = a.t_k + a.dt * (a.thr - vo) / (vn - vo);
    }
  }
  if (b == 0 && tid == 0) {
    DevStats* st = a.stats;
    st->iters_total += it;
    st->steps += 1;
    if (it > st->max_iters) st->max_iters = it;
    if (!conv) st->not_conv += 1;
    st->last_iters = it;
    st->last_zn = zn;
    st->last_z0n = z0n;
    if (bad) atomicOr(a.err, kErrNan);
  }
}

// Standalone y = Op x (the SpMV of Algorithm 1) for operator checks and bandwidth runs.
__global__ void __launch_bounds__(256) spmv_sell_kernel(int64_t n, int64_t nslices,
                                                        const int32_t* __restrict__ slice_ptr,
                                                        const int32_t* __restrict__ col,
                                                        const double* __restrict__ val,
                                                        const double* __restrict__ x,
                                                        double* __restrict__ y) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t s = gw; s < nslices; s += nw) {
    const int beg = slice_ptr[s] + lane;
    const int w = (slice_ptr[s + 1] - slice_ptr[s]) >> 5;
    double acc = 0.0;
    for (int j = 0; j < w; ++j) {
      const int e = beg + 32 * j;
      acc = fma(val[e], x[col[e]], acc);
    }
    const int64_t row = s * 32 + lane;
    if (row < n) y[row] = acc;
  }
}

}  // namespace tc
