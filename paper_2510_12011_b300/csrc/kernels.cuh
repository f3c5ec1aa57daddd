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
  GridBar* bar;           // zeroed here for the PCG launch that follows on the stream
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

__device__ __forceinline__ void red_release_add_u32(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid-wide barrier for a cooperative launch (all blocks co-resident).  The arrival counter
// only grows within a launch (it is zeroed by the kernel launched before on the same stream):
// barrier number e of the launch is passed once the counter reaches e * nblocks.  Arrival is a
// release reduction, the wait an acquire poll, so the block's writes before the barrier are
// visible to every block after it.  Every wait is bounded: after wait_limit polls the block
// records kErrTimeout and leaves; a block that sees any error flag returns false so that the
// kernel can exit without further waits.
__device__ __forceinline__ bool grid_sync(GridBar* bar, unsigned nblocks, unsigned& epoch,
                                          long long wait_limit, int* err) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = *(volatile int*)err ? 0 : 1;   // after an error, leave without waiting
    epoch += 1;
    if (ok && nblocks > 1) {
      const unsigned target = epoch * nblocks;
      red_release_add_u32(&bar->count, 1u);
      long long polls = 0;
      while (ld_acquire_u32(&bar->count) < target) {
        if (++polls > wait_limit) {
          atomicOr(err, kErrTimeout);
          ok = 0;
          break;
        }
        if (polls > 2048) __nanosleep(20);
      }
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

// Warp 0 of every block reduces the per-block partials in the same order; lane 0 of warp 0
// holds the totals.  Every block obtains bitwise the same totals.
__device__ __forceinline__ void grid_sum_warp0(const double* part, int stride, unsigned nb,
                                               double& a, double& b, bool two) {
  const int lane = threadIdx.x & 31;
  double sa = 0.0, sb = 0.0;
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
  a = warp_sum(sa);
  b = two ? warp_sum(sb) : 0.0;
}

// Row products over one SELL slice, lane = row.  Four entries are fetched (indices, values,
// gathered vector entries) before their four FMAs, which keeps four gathers in flight per lane
// while the FMAs still accumulate in entry order.
__device__ __forceinline__ double sell_dot(const int32_t* __restrict__ col,
                                          const double* __restrict__ val, int beg, int w,
                                          const double* x) {
  double acc0 = 0.0, acc1 = 0.0;   // even / odd entries: two independent FMA chains
  int j = 0;
  for (; j + 4 <= w; j += 4) {
    const int e = beg + 32 * j;
    const int c0 = __ldg(col + e), c1 = __ldg(col + e + 32), c2 = __ldg(col + e + 64),
              c3 = __ldg(col + e + 96);
    const double v0 = __ldg(val + e), v1 = __ldg(val + e + 32), v2 = __ldg(val + e + 64),
                 v3 = __ldg(val + e + 96);
    const double x0 = x[c0], x1 = x[c1], x2 = x[c2], x3 = x[c3];
    acc0 = fma(v0, x0, acc0);
    acc1 = fma(v1, x1, acc1);
    acc0 = fma(v2, x2, acc0);
    acc1 = fma(v3, x3, acc1);
  }
  for (; j < w; ++j) {
    const int e = beg + 32 * j;
    const double v = __ldg(val + e), xv = x[__ldg(col + e)];
    if (j & 1)
      acc1 = fma(v, xv, acc1);
    else
      acc0 = fma(v, xv, acc0);
  }
  return acc0 + acc1;
}

// Two value streams over the same pattern: am = sum M_ij g1_j, ak = sum K_ij g2_j.
__device__ __forceinline__ void sell_dot2(const int32_t* __restrict__ col,
                                          const double* __restrict__ vm,
                                          const double* __restrict__ vk, int beg, int w,
                                          const double* __restrict__ g1,
                                          const double* __restrict__ g2, double& am,
                                          double& ak) {
  am = 0.0;
  ak = 0.0;
  int j = 0;
  for (; j + 2 <= w; j += 2) {
    const int e = beg + 32 * j;
    const int c0 = __ldg(col + e), c1 = __ldg(col + e + 32);
    const double m0 = __ldg(vm + e), m1 = __ldg(vm + e + 32);
    const double k0 = __ldg(vk + e), k1 = __ldg(vk + e + 32);
    const double a0 = __ldg(g1 + c0), a1 = __ldg(g1 + c1);
    const double b0 = __ldg(g2 + c0), b1 = __ldg(g2 + c1);
    am = fma(m0, a0, am);
    ak = fma(k0, b0, ak);
    am = fma(m1, a1, am);
    ak = fma(k1, b1, ak);
  }
  for (; j < w; ++j) {
    const int e = beg + 32 * j;
    const int c = __ldg(col + e);
    am = fma(__ldg(vm + e), __ldg(g1 + c), am);
    ak = fma(__ldg(vk + e), __ldg(g2 + c), ak);
  }
}

// (a1) Ionic update, Mitchell-Schaeffer with a Rush-Larsen gate, plus the per-node vectors of
// the right-hand side and the extrapolated initial guess.
__global__ void __launch_bounds__(256) ionic_ms_kernel(const IonicArgs a) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) a.bar->count = 0u;
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
  __shared__ double s_sc[4];   // scalars computed once per block by thread 0, then broadcast
  __shared__ int s_flag;       // 0 = iterate, 1 = converged, 2 = non-finite
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned nb = gridDim.x, b = blockIdx.x;
  const int s0 = a.blk_slice[b], s1 = a.blk_slice[b + 1];
  const int64_t r0 = (int64_t)s0 * 32;
  const int64_t r1 = min((int64_t)s1 * 32, a.n);
  unsigned epoch = 0;
  // Scalar FP64 work (sqrt, divisions, the stopping test) runs on thread 0 only: B300 issues
  // FP64 at a small fraction of its FP32 rate, so replicating it over every thread is costly.
  double rho = 0.0, z0n = 0.0, zn = 0.0;   // meaningful in thread 0
  int it = 0;

  // r0 = chi M (w - Cm x0) - dt K ((1-theta) V + theta x0) = M g1 - K g2
  double rho_l = 0.0, zz_l = 0.0;
  for (int s = s0 + warp; s < s1; s += NW) {
    const int beg = a.slice_ptr[s] + lane;
    const int w = (a.slice_ptr[s + 1] - a.slice_ptr[s]) >> 5;
    double am, ak;
    sell_dot2(a.col, a.vM, a.vK, beg, w, a.g1, a.g2, am, ak);
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
  if (!grid_sync(a.bar, nb, epoch, a.wait_limit, a.err)) return;
  if (warp == 0) {
    double t_rho, t_zz;
    grid_sum_warp0(a.partB, 2, nb, t_rho, t_zz, true);
    if (tid == 0) {
      rho = t_rho;
      z0n = sqrt(t_zz);
      zn = z0n;
      s_flag = !(z0n == z0n) ? 2 : (z0n == 0.0 || z0n < a.atol) ? 1 : 0;
    }
  }
  __syncthreads();
  int flag = s_flag;
  while (flag == 0 && it < a.max_iter) {
    // q = A p, p^T q
    double pq_l = 0.0, dummy = 0.0;
    for (int s = s0 + warp; s < s1; s += NW) {
      const int beg = a.slice_ptr[s] + lane;
      const int w = (a.slice_ptr[s + 1] - a.slice_ptr[s]) >> 5;
      const double acc = sell_dot(a.col, a.vA, beg, w, a.p);
      const int64_t row = (int64_t)s * 32 + lane;
      if (row < a.n) {
        a.q[row] = acc;
        pq_l = fma(a.p[row], acc, pq_l);
      }
    }
    block_sum2<NW>(pq_l, dummy, s_red);
    if (tid == 0) a.partA[b] = pq_l;
    if (!grid_sync(a.bar, nb, epoch, a.wait_limit, a.err)) return;
    if (warp == 0) {
      double pq, unused;
      grid_sum_warp0(a.partA, 1, nb, pq, unused, false);
      if (tid == 0) {
        s_sc[0] = rho / pq;
        s_sc[1] = pq;
      }
    }
    __syncthreads();
    const double alpha = s_sc[0];
    // x += alpha p, r -= alpha q, z = D^-1 r, rho' = r^T z, ||z||^2
    rho_l = 0.0;
    zz_l = 0.0;
    for (int64_t i = r0 + tid; i < r1; i += 2 * THREADS) {
      const int64_t i2 = i + THREADS;
      const bool two = i2 < r1;
      const double p0 = a.p[i], q0 = a.q[i], x0 = a.x[i], rr0 = a.r[i], d0 = __ldg(&a.dinv[i]);
      double p1 = 0.0, q1 = 0.0, x1 = 0.0, rr1 = 0.0, d1 = 0.0;
      if (two) {
        p1 = a.p[i2];
        q1 = a.q[i2];
        x1 = a.x[i2];
        rr1 = a.r[i2];
        d1 = __ldg(&a.dinv[i2]);
      }
      a.x[i] = fma(alpha, p0, x0);
      const double ri = fma(-alpha, q0, rr0);
      a.r[i] = ri;
      const double zi = d0 * ri;
      a.z[i] = zi;
      rho_l = fma(ri, zi, rho_l);
      zz_l = fma(zi, zi, zz_l);
      if (two) {
        a.x[i2] = fma(alpha, p1, x1);
        const double rj = fma(-alpha, q1, rr1);
        a.r[i2] = rj;
        const double zj = d1 * rj;
        a.z[i2] = zj;
        rho_l = fma(rj, zj, rho_l);
        zz_l = fma(zj, zj, zz_l);
      }
    }
    block_sum2<NW>(rho_l, zz_l, s_red);
    if (tid == 0) {
      a.partB[2 * b] = rho_l;
      a.partB[2 * b + 1] = zz_l;
    }
    if (!grid_sync(a.bar, nb, epoch, a.wait_limit, a.err)) return;
    ++it;
    if (warp == 0) {
      double rho_new, zz;
      grid_sum_warp0(a.partB, 2, nb, rho_new, zz, true);
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
    if (flag != 0) break;
    const double beta = s_sc[2];
    for (int64_t i = r0 + tid; i < r1; i += 2 * THREADS) {
      const int64_t i2 = i + THREADS;
      const double p0 = a.p[i], z0 = a.z[i];
      if (i2 < r1) {
        const double p1 = a.p[i2], z1 = a.z[i2];
        a.p[i2] = fma(beta, p1, z1);
      }
      a.p[i] = fma(beta, p0, z0);
    }
    if (!grid_sync(a.bar, nb, epoch, a.wait_limit, a.err)) return;
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
    if (flag != 1) st->not_conv += 1;
    st->last_iters = it;
    st->last_zn = zn;
    st->last_z0n = z0n;
    if (flag == 2) atomicOr(a.err, kErrNan);
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
    const double acc = sell_dot(col, val, beg, w, x);
    const int64_t row = s * 32 + lane;
    if (row < n) y[row] = acc;
  }
}

}  // namespace tc
