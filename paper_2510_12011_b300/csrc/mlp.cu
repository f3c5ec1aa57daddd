// Learned ionic surrogate: network storage, training and inference kernels, and the C ABI.
//
// GEMM forms used (row-major matrices, FP32 accumulation):
//   NT  C[M][N] = A[M][K] . B[N][K]^T     forward Z = A W^T and surrogate inference
//   NN  C[M][N] = A[M][K] . B[K][N]       backward dA = dZ W^T-matrix  (B = W^T as stored)
//   TN  C[M][N] = A[K][M]^T . B[K][N]     backward dW^T = dZ^T A
// The NT form runs on the tensor cores (tcgen05, gemm_tc.cuh); all three forms also have a
// SIMT implementation used as the reference the tensor-core path is checked against.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <cstdlib>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "../../include/tc.h"
#include "gemm_tc.cuh"
#include "ionic_tp06.cuh"
#include "kernels.cuh"
#include "mlp.cuh"
#include "surrogate.h"
#include "tc_internal.h"

using namespace tc;

struct tc_mlp {
  int device = 0;
  MlpDims d{};
  float* params = nullptr;           // FP32 master weights and biases
  float* grads = nullptr;
  float* adam_m = nullptr;
  float* adam_v = nullptr;
  __nv_bfloat16* wt = nullptr;       // BF16 copies of the weights W_l^T (same offsets, biases unused)
  __nv_bfloat16* wt0d = nullptr;     // layer-0 BF16 weights duplicated for the split input, [256][64]
  uint8_t* img = nullptr;            // swizzled tensor-core images of the BF16 weights
  uint32_t img_off[kMlpLayers] = {0}, img_bytes[kMlpLayers] = {0};
  int num_sms = 0;
  float* norm = nullptr;             // device: in_mean[20], in_scale[20], out_mean[19], out_scale[19]
  std::vector<float> norm_host;
  int64_t adam_t = 0;
  int gemm = kGemmTcgen05;
  int fused_kernel = 2;   // forward kernel: 2 = two pipelined tiles per CTA, 1 = one tile (TC_MLP_KERNEL)
  // training workspace (sized for the largest batch seen)
  int64_t ws_rows = 0;
  __nv_bfloat16* act[kMlpLayers] = {nullptr};   // A_l, [rows][op_in_l] (layer 0: split input)
  float* z[kMlpLayers] = {nullptr};             // Z_l, [rows][out_l]
  float* dz = nullptr;                          // [rows][256]
  float* da = nullptr;                          // [rows][256]
  float* tgt = nullptr;                         // [rows][32] normalized targets
  int32_t* idx = nullptr;                       // batch row indices
  float* loss = nullptr;                        // device scalar
  float* splitk = nullptr;                      // split-K partial products (kMaxSplits x 256 x 256)
  float* gw0d = nullptr;                        // gradient of the duplicated layer-0 weights [256][64]
  // tensor-core backward pass: K-major BF16 copies of dZ^T, A_l^T, dZ and the weights W_l [in][out]
  __nv_bfloat16 *dzT = nullptr, *actT = nullptr, *dzb = nullptr, *wT = nullptr;
  int* gemm_err = nullptr;                      // wait failures of the GEMM kernel
  int* counters = nullptr;                      // device: [0] batch index in the epoch, [1] Adam steps
};

namespace {

inline unsigned blocks_for(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

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

__device__ __forceinline__ float to_f(float x) { return x; }
__device__ __forceinline__ float to_f(__nv_bfloat16 x) { return __bfloat162float(x); }

// ---- SIMT GEMMs (reference path) --------------------------------------------------------
// 64x64 output tile per 256-thread block, 4x4 outputs per thread, K in steps of 16 through
// shared memory.  FORM: 0 = NT, 1 = NN, 2 = TN (see the file header).  blockIdx.z selects a
// slice [z kchunk, (z+1) kchunk) of the reduction (split K); its partial product goes to
// C + z M N, and the slices are summed in order afterwards.
template <int FORM, typename TA, typename TB>
__global__ void __launch_bounds__(256) gemm_simt_kernel(int M, int N, int K, int kchunk, const TA* __restrict__ A,
                                                        const TB* __restrict__ B, float* __restrict__ C) {
  __shared__ float As[16][64 + 1];
  __shared__ float Bs[16][64 + 1];
  const int tid = threadIdx.x;
  const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  const int tm = (tid / 16) * 4, tn = (tid % 16) * 4;
  const int kb = blockIdx.z * kchunk, ke = min(K, kb + kchunk);
  C += (int64_t)blockIdx.z * M * N;
  float acc[4][4] = {};
  for (int k0 = kb; k0 < ke; k0 += 16) {
    for (int e = tid; e < 16 * 64; e += 256) {
      const int kk = e / 64, mm = e % 64;
      const int m = m0 + mm, k = k0 + kk;
      float av = 0.f;
      if (m < M && k < ke) av = FORM == 2 ? to_f(A[(int64_t)k * M + m]) : to_f(A[(int64_t)m * K + k]);
      As[kk][mm] = av;
      const int n = n0 + mm;
      float bv = 0.f;
      if (n < N && k < ke) bv = FORM == 0 ? to_f(B[(int64_t)n * K + k]) : to_f(B[(int64_t)k * N + n]);
      Bs[kk][mm] = bv;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][tm + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tn + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int m = m0 + tm + i, n = n0 + tn + j;
      if (m < M && n < N) C[(int64_t)m * N + n] = acc[i][j];
    }
}

__global__ void sum_splits_kernel(int64_t mn, int splits, const float* __restrict__ part, float* __restrict__ C) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= mn) return;
  float s = part[e];
  for (int z = 1; z < splits; ++z) s += part[z * mn + e];
  C[e] = s;
}

constexpr int kMaxSplits = 32;

// C = op(A) op(B); with ws (kMaxSplits M N floats) and a long reduction, K is split so that the
// grid covers the GPU (the weight gradients have few output tiles and K = batch rows).
template <int FORM, typename TA, typename TB>
tc_status gemm_simt(int M, int N, int K, const TA* A, const TB* B, float* C, cudaStream_t st,
                    float* ws = nullptr) {
  const int tiles = ((N + 63) / 64) * ((M + 63) / 64);
  int splits = 1;
  if (ws) splits = std::max(1, std::min({kMaxSplits, K / 128, (296 + tiles - 1) / tiles}));
  const int kchunk = ((K + splits - 1) / splits + 15) / 16 * 16;
  splits = (K + kchunk - 1) / kchunk;
  dim3 grid((N + 63) / 64, (M + 63) / 64, splits);
  gemm_simt_kernel<FORM, TA, TB><<<grid, 256, 0, st>>>(M, N, K, kchunk, A, B, splits > 1 ? ws : C);
  if (splits > 1) {
    const int64_t mn = (int64_t)M * N;
    sum_splits_kernel<<<blocks_for(mn), 256, 0, st>>>(mn, splits, ws, C);
  }
  CUDA_TRY(cudaGetLastError());
  return TC_OK;
}

// out[c][r] = bf16(in[r][c]) for r < rows_out (zero where r >= rows), c < cols; 32 x 32 tiles.
template <typename TI>
__global__ void transpose_bf16_kernel(int rows, int rows_out, int cols, const TI* __restrict__ in, int64_t ld_in,
                                      __nv_bfloat16* __restrict__ out, int64_t ld_out) {
  __shared__ float t[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int r = r0 + j, c = c0 + threadIdx.x;
    t[j][threadIdx.x] = (r < rows && c < cols) ? to_f(in[(int64_t)r * ld_in + c]) : 0.f;
  }
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int c = c0 + j, r = r0 + threadIdx.x;
    if (c < cols && r < rows_out) out[(int64_t)c * ld_out + r] = __float2bfloat16(t[threadIdx.x][j]);
  }
}

template <typename TI>
tc_status transpose_bf16(int rows, int rows_out, int cols, const TI* in, int64_t ld_in, __nv_bfloat16* out,
                         int64_t ld_out, cudaStream_t st) {
  dim3 grid((cols + 31) / 32, (rows_out + 31) / 32);
  transpose_bf16_kernel<TI><<<grid, dim3(32, 8), 0, st>>>(rows, rows_out, cols, in, ld_in, out, ld_out);
  CUDA_TRY(cudaGetLastError());
  return TC_OK;
}

// FP32 [rows][cols] -> BF16 (same layout)
__global__ void to_bf16_kernel(int64_t n, const float* in, __nv_bfloat16* out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) out[e] = __float2bfloat16(in[e]);
}

// C = A . B^T on the tensor cores (gemm_nt_kernel): A [M][K], B [N][K] BF16, C [M][N] FP32 with
// row strides lda, ldb, ldc.  With ws (kMaxSplits M N floats) and a long K, K is split across
// CTAs and the partial products summed in a fixed order.
tc_status gemm_nt(int M, int N, int K, const __nv_bfloat16* A, int64_t lda, const __nv_bfloat16* B,
                  int64_t ldb, float* C, int64_t ldc, cudaStream_t st, float* ws, int* err) {
  if (M < 1 || N < 1 || K < 8 || (K & 7) || (lda & 7) || (ldb & 7)) return fail(TC_ERR_ARG, "bad GEMM shape");
  const int nt = N <= 32 ? 32 : N <= 64 ? 64 : N <= 128 ? 128 : 256;
  const int tiles = ((N + nt - 1) / nt) * ((M + 127) / 128);
  int splits = 1;
  if (ws) splits = std::max(1, std::min({kMaxSplits, K / 128, (148 + tiles - 1) / tiles}));
  int kchunk = ((K + splits - 1) / splits + 63) / 64 * 64;
  splits = (K + kchunk - 1) / kchunk;
  GemmNTArgs a{};
  a.M = M;
  a.N = N;
  a.K = K;
  a.n_tile = nt;
  a.kchunk = kchunk;
  a.A = A;
  a.lda = lda;
  a.B = B;
  a.ldb = ldb;
  a.C = splits > 1 ? ws : C;
  a.ldc = splits > 1 ? N : ldc;
  a.split_stride = (int64_t)M * N;
  a.err = err;
  dim3 grid((N + nt - 1) / nt, (M + 127) / 128, splits);
  gemm_nt_kernel<<<grid, kGemmThreads, gemm_nt_smem_bytes(nt), st>>>(a);
  CUDA_TRY(cudaGetLastError());
  if (splits > 1) {
    const int64_t mn = (int64_t)M * N;
    if (ldc == N) {
      sum_splits_kernel<<<blocks_for(mn), 256, 0, st>>>(mn, splits, ws, C);
    } else {
      return fail(TC_ERR_ARG, "split-K output must be dense");
    }
    CUDA_TRY(cudaGetLastError());
  }
  return TC_OK;
}

// ---- elementwise kernels ----------------------------------------------------------------

__device__ __forceinline__ float silu(float z) { return z / (1.f + __expf(-z)); }
__device__ __forceinline__ float silu_grad(float z) {
  const float s = 1.f / (1.f + __expf(-z));
  return s * (1.f + z * (1.f - s));
}

// Z += bias (in place); hidden layers also write A_next = SiLU(Z) as BF16.
__global__ void bias_act_kernel(int64_t rows, int out, float* z, const float* bias,
                                __nv_bfloat16* a_next, int silu_on) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= rows * out) return;
  const float v = z[e] + bias[e % out];
  z[e] = v;
  if (silu_on) a_next[e] = __float2bfloat16(silu(v));
}

// dZ = (Yhat - T) * 2 / (rows * kMlpOut) over the real outputs; loss accumulated in FP32.
__global__ void loss_grad_kernel(int64_t rows, const float* y, const float* t, float* dz, float* loss) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  float l = 0.f;
  if (e < rows * kMlpPad) {
    const int c = (int)(e % kMlpPad);
    float g = 0.f;
    if (c < kMlpOut) {
      const float d = y[e] - t[e];
      g = 2.f * d / (float)(rows * kMlpOut);
      l = d * d / (float)(rows * kMlpOut);
    }
    dz[e] = g;
  }
  for (int o = 16; o > 0; o >>= 1) l += __shfl_down_sync(0xffffffffu, l, o);
  if ((threadIdx.x & 31) == 0 && l != 0.f) atomicAdd(loss, l);
}

// db[c] = sum_r dZ[r][c]  (one block per column group, fixed order inside a block)
__global__ void colsum_kernel(int64_t rows, int cols, const float* dz, float* db) {
  const int c = blockIdx.x;
  float s = 0.f;
  for (int64_t r = threadIdx.x; r < rows; r += blockDim.x) s += dz[r * cols + c];
  __shared__ float sm[256];
  sm[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) db[c] = sm[0];
}

// dZ_prev = dA * SiLU'(Z_prev)
__global__ void silu_back_kernel(int64_t n, const float* da, const float* zprev, float* dz) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) dz[e] = da[e] * silu_grad(zprev[e]);
}

__global__ void accumulate_kernel(float* sum, const float* v) { *sum += *v; }

// Adam (Kingma & Ba 2015) on the FP32 master parameters, then the BF16 weight copies; the step
// count t = counters[1] + 1 is read on the device (bias corrections 1 - b^t), so that one captured
// training step serves every batch.
__global__ void adam_kernel(int64_t n, float* p, const float* g, float* m, float* v, __nv_bfloat16* wt,
                                 float lr, float b1, float b2, float eps, const int* counters) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float t = (float)(counters[1] + 1);
  const float c1 = 1.f - powf(b1, t), c2 = 1.f - powf(b2, t);
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  p[i] = pi;
  wt[i] = __float2bfloat16(pi);
}

// End of a training step: next batch of the epoch, one more Adam step.
__global__ void train_tick_kernel(int* counters) {
  counters[0] += 1;
  counters[1] += 1;
}

__global__ void cast_kernel(int64_t n, const float* p, __nv_bfloat16* wt) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) wt[i] = __float2bfloat16(p[i]);
}

// Layer-0 weights for the split input: W0d[o][c] = W0d[o][32 + c] = bf16(W0[o][c]).
__global__ void dup_w0_kernel(const float* w0, __nv_bfloat16* wt0d) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= kMlpHidden * kMlpIn0) return;
  const int o = e / kMlpIn0, c = e % kMlpIn0;
  wt0d[e] = __float2bfloat16(w0[o * kMlpPad + (c % kMlpPad)]);
}

// Gradient of the tied layer-0 weights: dW0[o][c] = dW0d[o][c] + dW0d[o][32 + c].
__global__ void fold_w0_kernel(const float* gw0d, float* g0) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= kMlpHidden * kMlpPad) return;
  const int o = e / kMlpPad, c = e % kMlpPad;
  g0[e] = gw0d[o * kMlpIn0 + c] + gw0d[o * kMlpIn0 + kMlpPad + c];
}

// Zero the weights that connect padding columns, so padded widths stay exact zeros.
__global__ void mask_padding_kernel(float* p, int64_t w0_off, int64_t w4_off, int64_t b4_off) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  // layer 0: W^T [256][32], input columns >= 20 are padding
  if (i < 256 * kMlpPad && (i % kMlpPad) >= kMlpIn) p[w0_off + i] = 0.f;
  // layer 4: W^T [32][256], output rows >= 19 are padding
  if (i < kMlpPad * 256 && (i / 256) >= kMlpOut) p[w4_off + i] = 0.f;
  if (i < kMlpPad && i >= kMlpOut) p[b4_off + i] = 0.f;
}

// Deterministic initialisation: uniform(-a, a) from SplitMix64 counters, a = sqrt(6/(fan_in+fan_out))
__global__ void init_kernel(int64_t n, float* p, uint64_t seed, const int64_t* off, const int* fin,
                            const int* fout) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int l = 0;
  while (l + 1 < kMlpLayers && i >= off[2 * (l + 1)]) ++l;
  const bool is_bias = i >= off[2 * l + 1];
  if (is_bias) {
    p[i] = 0.f;
    return;
  }
  uint64_t z = seed + (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  const double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);
  const int fi = fin[l] == kMlpPad && l == 0 ? kMlpIn : fin[l];
  const int fo = fout[l] == kMlpPad && l == kMlpLayers - 1 ? kMlpOut : fout[l];
  const double a = sqrt(6.0 / (fi + fo)) * (l == kMlpLayers - 1 ? 0.1 : 1.0);
  p[i] = (float)((2.0 * u - 1.0) * a);
}

// Rows of the training set -> normalized split-BF16 inputs and FP32 targets of one batch.
// x: [n][20] raw features; y: [n][19] raw next state; targets are normalized deltas.
__global__ void gather_batch_kernel(int64_t rows, const int32_t* idx, const int* batch_index, const float* x,
                                    const float* y, const float* norm, __nv_bfloat16* a0, float* tgt) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= rows * kMlpPad) return;
  const int64_t r = e / kMlpPad;
  const int c = (int)(e % kMlpPad);
  const int64_t s = idx ? idx[(batch_index ? (int64_t)*batch_index * rows : 0) + r] : r;
  const float* in_mean = norm;
  const float* in_scale = norm + kMlpIn;
  const float* out_mean = norm + 2 * kMlpIn;
  const float* out_scale = norm + 2 * kMlpIn + kMlpOut;
  float xin = 0.f, t = 0.f;
  if (c < kMlpIn) xin = (x[s * kMlpIn + c] - in_mean[c]) / in_scale[c];
  if (c < kMlpOut && y) t = ((y[s * kMlpOut + c] - x[s * kMlpIn + c]) - out_mean[c]) / out_scale[c];
  const __nv_bfloat16 hi = __float2bfloat16(xin);
  a0[r * kMlpIn0 + c] = hi;
  a0[r * kMlpIn0 + kMlpPad + c] = __float2bfloat16(xin - __bfloat162float(hi));
  if (tgt) tgt[e] = t;
}

// Column statistics of the training set for the normalization: column c < 20 is input
// feature c of x [n][20]; column 20 + c is the change y[.][c] - x[.][c] of output c.  One block
// per column, FP64 sums in a fixed order; pass 0 writes the means, pass 1 the standard deviations.
__global__ void __launch_bounds__(1024) column_stats_kernel(int64_t n, const float* x, const float* y, int pass,
                                                            double* mean, double* sdev) {
  const int c = blockIdx.x;
  const double mu = pass ? mean[c] : 0.0;
  double s = 0.0;
  for (int64_t r = threadIdx.x; r < n; r += blockDim.x) {
    const double v = c < kMlpIn ? (double)x[r * kMlpIn + c]
                                : (double)y[r * kMlpOut + (c - kMlpIn)] - (double)x[r * kMlpIn + (c - kMlpIn)];
    s += pass ? (v - mu) * (v - mu) : v;
  }
  __shared__ double sm[1024];
  sm[threadIdx.x] = s;
  __syncthreads();
  for (int o = 512; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (pass) sdev[c] = sqrt(sm[0] / (double)n);
    else mean[c] = sm[0] / (double)n;
  }
}

tc_status rebuild_images(tc_mlp* m, cudaStream_t st) {
  dup_w0_kernel<<<blocks_for(kMlpHidden * kMlpIn0), 256, 0, st>>>(m->params + m->d.w_off[0], m->wt0d);
  for (int l = 0; l < kMlpLayers; ++l) {
    const int64_t chunks = (int64_t)((m->d.op_in[l] + 63) / 64) * m->d.out[l] * 8;
    const __nv_bfloat16* w = l == 0 ? m->wt0d : m->wt + m->d.w_off[l];
    weight_image_kernel<<<(unsigned)((chunks + 255) / 256), 256, 0, st>>>(w, m->d.out[l], m->d.op_in[l],
                                                                        m->img + m->img_off[l]);
  }
  // W_l as [in][out] (K-major operand of dA = dZ W) for the hidden and output layers
  for (int l = 1; l < kMlpLayers; ++l)
    TRY((transpose_bf16<__nv_bfloat16>(m->d.out[l], m->d.out[l], m->d.in[l], m->wt + m->d.w_off[l], m->d.in[l],
                                       m->wT + m->d.w_off[l], m->d.out[l], st)));
  CUDA_TRY(cudaGetLastError());
  return TC_OK;
}

// Tensor-core forward of act0 (M x 32 BF16) through all layers; y (M x 32 FP32) gets the
// output, and with store_hidden Z_l and the activations go to the training workspace.
tc_status forward_tc(tc_mlp* m, int64_t M, const __nv_bfloat16* act0, float* y, bool store_hidden,
                     int* err, cudaStream_t st, const int* M_dev = nullptr) {
  MlpFusedArgs a{};
  a.M = M;
  a.M_dev = M_dev;
  a.a0 = act0;
  for (int l = 0; l < kMlpLayers; ++l) {
    a.img[l] = m->img + m->img_off[l];
    a.img_bytes[l] = m->img_bytes[l];
    a.bias[l] = m->params + m->d.b_off[l];
    a.in[l] = m->d.op_in[l];
    a.out[l] = m->d.out[l];
    a.z[l] = store_hidden && l + 1 < kMlpLayers ? m->z[l] : nullptr;
    a.act[l] = store_hidden ? m->act[l] : nullptr;
  }
  a.y = y;
  a.err = err;
  const int64_t tiles = (M + kTcRows - 1) / kTcRows;
  if (m->fused_kernel == 2) {
    // two tiles per CTA (pipelined roles)
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((tiles + 1) / 2, m->num_sms));
    if (store_hidden)
      mlp_fused2_kernel<true><<<grid, kT2Threads, kT2SmemBytes, st>>>(a);
    else
      mlp_fused2_kernel<false><<<grid, kT2Threads, kT2SmemBytes, st>>>(a);
  } else {
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, m->num_sms));
    if (store_hidden)
      mlp_fused_kernel<true><<<grid, kTcThreads, kTcSmemBytes, st>>>(a);
    else
      mlp_fused_kernel<false><<<grid, kTcThreads, kTcSmemBytes, st>>>(a);
  }
  CUDA_TRY(cudaGetLastError());
  return TC_OK;
}

tc_status ensure_workspace(tc_mlp* m, int64_t rows) {
  if (rows <= m->ws_rows) return TC_OK;
  for (int l = 0; l < kMlpLayers; ++l) {
    cudaFree(m->act[l]);
    cudaFree(m->z[l]);
    m->act[l] = nullptr;
    m->z[l] = nullptr;
  }
  cudaFree(m->dz);
  cudaFree(m->da);
  cudaFree(m->tgt);
  cudaFree(m->idx);
  m->dz = m->da = m->tgt = nullptr;
  m->idx = nullptr;
  m->ws_rows = 0;
  const int64_t r = (rows + 127) / 128 * 128;
  for (int l = 0; l < kMlpLayers; ++l) {
    CUDA_TRY(cudaMalloc(&m->act[l], r * m->d.op_in[l] * sizeof(__nv_bfloat16)));
    CUDA_TRY(cudaMalloc(&m->z[l], r * m->d.out[l] * sizeof(float)));
  }
  CUDA_TRY(cudaMalloc(&m->dz, r * kMlpHidden * sizeof(float)));
  CUDA_TRY(cudaMalloc(&m->da, r * kMlpHidden * sizeof(float)));
  CUDA_TRY(cudaMalloc(&m->tgt, r * kMlpPad * sizeof(float)));
  CUDA_TRY(cudaMalloc(&m->idx, r * sizeof(int32_t)));
  if (!m->splitk) CUDA_TRY(cudaMalloc(&m->splitk, (size_t)kMaxSplits * kMlpHidden * kMlpHidden * sizeof(float)));
  if (!m->gw0d) CUDA_TRY(cudaMalloc(&m->gw0d, (size_t)kMlpHidden * kMlpIn0 * sizeof(float)));
  cudaFree(m->dzT);
  cudaFree(m->actT);
  cudaFree(m->dzb);
  m->dzT = m->actT = m->dzb = nullptr;
  CUDA_TRY(cudaMalloc(&m->dzT, r * kMlpHidden * sizeof(__nv_bfloat16)));
  CUDA_TRY(cudaMalloc(&m->actT, r * kMlpHidden * sizeof(__nv_bfloat16)));
  CUDA_TRY(cudaMalloc(&m->dzb, r * kMlpHidden * sizeof(__nv_bfloat16)));
  m->ws_rows = r;
  return TC_OK;
}

// Forward pass on act[0] (rows x 32): fills z[l], act[l+1]; output in z[4].
tc_status forward(tc_mlp* m, int64_t rows, cudaStream_t st) {
  if (m->gemm == kGemmTcgen05) {
    int* err = reinterpret_cast<int*>(m->loss) + 1;   // the word after the loss scalar (callers reset it)
    TRY(forward_tc(m, rows, m->act[0], m->z[kMlpLayers - 1], true, err, st));
    return TC_OK;
  }
  for (int l = 0; l < kMlpLayers; ++l) {
    const int in = m->d.op_in[l], out = m->d.out[l];
    TRY(gemm_simt<0>((int)rows, out, in, m->act[l], l == 0 ? m->wt0d : m->wt + m->d.w_off[l], m->z[l], st));
    const bool hidden = l + 1 < kMlpLayers;
    bias_act_kernel<<<blocks_for(rows * out), 256, 0, st>>>(
        rows, out, m->z[l], m->params + m->d.b_off[l], hidden ? m->act[l + 1] : nullptr, hidden);
    CUDA_TRY(cudaGetLastError());
  }
  return TC_OK;
}

// Backward pass on the tensor cores: per layer the weight gradient dW^T = dZ^T A (K = batch
// rows, split across CTAs) and the input gradient dA = dZ W (K = layer width), both as NT GEMMs on
// K-major BF16 copies (dZ^T, A^T, dZ, W as [in][out]); FP32 accumulation, FP32 dZ kept for the
// bias gradient and the SiLU derivative.
tc_status backward_tc(tc_mlp* m, int64_t rows, cudaStream_t st) {
  const int R = (int)((rows + 127) / 128 * 128);   // K of the weight gradients, zero-padded rows
  CUDA_TRY(cudaMemsetAsync(m->loss, 0, sizeof(float), st));
  loss_grad_kernel<<<blocks_for(rows * kMlpPad), 256, 0, st>>>(rows, m->z[kMlpLayers - 1], m->tgt, m->dz,
                                                                m->loss);
  CUDA_TRY(cudaGetLastError());
  for (int l = kMlpLayers - 1; l >= 0; --l) {
    const int in = m->d.op_in[l], out = m->d.out[l];
    TRY((transpose_bf16<float>((int)rows, R, out, m->dz, out, m->dzT, R, st)));
    TRY((transpose_bf16<__nv_bfloat16>((int)rows, R, in, m->act[l], in, m->actT, R, st)));
    TRY(gemm_nt(out, in, R, m->dzT, R, m->actT, R, l == 0 ? m->gw0d : m->grads + m->d.w_off[l], in, st,
                m->splitk, m->gemm_err));
    if (l == 0)
      fold_w0_kernel<<<blocks_for(kMlpHidden * kMlpPad), 256, 0, st>>>(m->gw0d, m->grads + m->d.w_off[0]);
    colsum_kernel<<<out, 256, 0, st>>>(rows, out, m->dz, m->grads + m->d.b_off[l]);
    CUDA_TRY(cudaGetLastError());
    if (l == 0) break;
    to_bf16_kernel<<<blocks_for(rows * out), 256, 0, st>>>(rows * out, m->dz, m->dzb);
    TRY(gemm_nt((int)rows, m->d.in[l], out, m->dzb, out, m->wT + m->d.w_off[l], out, m->da, m->d.in[l], st,
                nullptr, m->gemm_err));
    silu_back_kernel<<<blocks_for(rows * m->d.in[l]), 256, 0, st>>>(rows * m->d.in[l], m->da, m->z[l - 1], m->dz);
    CUDA_TRY(cudaGetLastError());
  }
  mask_padding_kernel<<<blocks_for(256 * kMlpPad), 256, 0, st>>>(m->grads, m->d.w_off[0],
                                                                 m->d.w_off[kMlpLayers - 1],
                                                                 m->d.b_off[kMlpLayers - 1]);
  CUDA_TRY(cudaGetLastError());
  return TC_OK;
}

// Backward pass from the loss of z[4] against tgt: fills grads (weights as W^T).
tc_status backward(tc_mlp* m, int64_t rows, cudaStream_t st) {
  if (m->gemm == kGemmTcgen05) return backward_tc(m, rows, st);
  CUDA_TRY(cudaMemsetAsync(m->loss, 0, sizeof(float), st));
  loss_grad_kernel<<<blocks_for(rows * kMlpPad), 256, 0, st>>>(rows, m->z[kMlpLayers - 1], m->tgt, m->dz,
                                                                m->loss);
  CUDA_TRY(cudaGetLastError());
  for (int l = kMlpLayers - 1; l >= 0; --l) {
    const int in = m->d.in[l], out = m->d.out[l];
    // dW_l^T[out][in] = dZ^T A_l  (layer 0: over the split operand, then the tied halves summed)
    if (l == 0) {
      TRY((gemm_simt<2, float, __nv_bfloat16>(out, kMlpIn0, (int)rows, m->dz, m->act[0], m->gw0d, st,
                                              m->splitk)));
      fold_w0_kernel<<<blocks_for(kMlpHidden * kMlpPad), 256, 0, st>>>(m->gw0d, m->grads + m->d.w_off[0]);
    } else {
      TRY((gemm_simt<2, float, __nv_bfloat16>(out, in, (int)rows, m->dz, m->act[l],
                                              m->grads + m->d.w_off[l], st, m->splitk)));
    }
    colsum_kernel<<<out, 256, 0, st>>>(rows, out, m->dz, m->grads + m->d.b_off[l]);
    CUDA_TRY(cudaGetLastError());
    if (l == 0) break;
    // dA_l[rows][in] = dZ W_l^T-matrix  (B stored as [out][in] = K x N)
    TRY((gemm_simt<1, float, __nv_bfloat16>((int)rows, in, out, m->dz, m->wt + m->d.w_off[l], m->da, st)));
    silu_back_kernel<<<blocks_for(rows * in), 256, 0, st>>>(rows * in, m->da, m->z[l - 1], m->dz);
    CUDA_TRY(cudaGetLastError());
  }
  // keep the padding weights at zero
  mask_padding_kernel<<<blocks_for(256 * kMlpPad), 256, 0, st>>>(m->grads, m->d.w_off[0],
                                                                 m->d.w_off[kMlpLayers - 1],
                                                                 m->d.b_off[kMlpLayers - 1]);
  CUDA_TRY(cudaGetLastError());
  return TC_OK;
}

}  // namespace

extern "C" {

tc_status tc_mlp_create(uint64_t seed, tc_mlp** out) {
  clear_error();
  if (!out) return fail(TC_ERR_ARG, "out must not be NULL");
  *out = nullptr;
  tc_mlp* m = new (std::nothrow) tc_mlp();
  if (!m) return fail(TC_ERR_NOMEM, "out of host memory");
  cudaGetDevice(&m->device);
  m->d = mlp_dims();
  const int64_t n = m->d.n_params;
  auto bail = [&](tc_status st) {
    tc_mlp_destroy(m);
    return st;
  };
  cudaError_t e = cudaMalloc(&m->params, n * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&m->grads, n * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&m->adam_m, n * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&m->adam_v, n * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&m->wt, n * sizeof(__nv_bfloat16));
  if (e == cudaSuccess) e = cudaMalloc(&m->wt0d, kMlpHidden * kMlpIn0 * sizeof(__nv_bfloat16));
  if (e == cudaSuccess) e = cudaMalloc(&m->wT, n * sizeof(__nv_bfloat16));
  if (e == cudaSuccess) e = cudaMalloc(&m->gemm_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&m->counters, 2 * sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(m->gemm_err, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&m->norm, (2 * kMlpIn + 2 * kMlpOut) * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&m->loss, 4 * sizeof(float));   // loss, error word, epoch sum
  uint32_t img_total = 0;
  for (int l = 0; l < kMlpLayers; ++l) {
    m->img_off[l] = img_total;
    m->img_bytes[l] = weight_image_bytes(m->d.out[l], m->d.op_in[l]);
    img_total += m->img_bytes[l];
  }
  if (e == cudaSuccess) e = cudaMalloc(&m->img, img_total);
  cudaDeviceGetAttribute(&m->num_sms, cudaDevAttrMultiProcessorCount, m->device);
  {
    const char* k = std::getenv("TC_MLP_KERNEL");
    m->fused_kernel = k && std::atoi(k) == 1 ? 1 : 2;
  }
  if (e != cudaSuccess) return bail(cuda_fail(e, "cudaMalloc"));
  e = cudaFuncSetAttribute(mlp_fused_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmemBytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(mlp_fused_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmemBytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(mlp_fused2_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kT2SmemBytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(mlp_fused2_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kT2SmemBytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(gemm_nt_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gemm_nt_smem_bytes(256));
  if (e != cudaSuccess) return bail(cuda_fail(e, "cudaFuncSetAttribute"));
  cudaMemset(m->adam_m, 0, n * sizeof(float));
  cudaMemset(m->adam_v, 0, n * sizeof(float));
  std::vector<int64_t> off(2 * kMlpLayers);
  std::vector<int> fin(kMlpLayers), fout(kMlpLayers);
  for (int l = 0; l < kMlpLayers; ++l) {
    off[2 * l] = m->d.w_off[l];
    off[2 * l + 1] = m->d.b_off[l];
    fin[l] = m->d.in[l];
    fout[l] = m->d.out[l];
  }
  int64_t* doff = nullptr;
  int *dfin = nullptr, *dfout = nullptr;
  e = cudaMalloc(&doff, off.size() * sizeof(int64_t));
  if (e == cudaSuccess) e = cudaMalloc(&dfin, kMlpLayers * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&dfout, kMlpLayers * sizeof(int));
  if (e == cudaSuccess) e = cudaMemcpy(doff, off.data(), off.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dfin, fin.data(), kMlpLayers * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dfout, fout.data(), kMlpLayers * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    init_kernel<<<blocks_for(n), 256>>>(n, m->params, seed, doff, dfin, dfout);
    mask_padding_kernel<<<blocks_for(256 * kMlpPad), 256>>>(m->params, m->d.w_off[0],
                                                            m->d.w_off[kMlpLayers - 1],
                                                            m->d.b_off[kMlpLayers - 1]);
    cast_kernel<<<blocks_for(n), 256>>>(n, m->params, m->wt);
    e = cudaGetLastError();
    if (e == cudaSuccess && rebuild_images(m, 0) != TC_OK) e = cudaErrorUnknown;
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
  }
  cudaFree(doff);
  cudaFree(dfin);
  cudaFree(dfout);
  if (e != cudaSuccess) return bail(cuda_fail(e, "network initialisation"));
  m->norm_host.assign(2 * kMlpIn + 2 * kMlpOut, 0.f);
  for (int j = 0; j < kMlpIn; ++j) m->norm_host[kMlpIn + j] = 1.f;
  for (int j = 0; j < kMlpOut; ++j) m->norm_host[2 * kMlpIn + kMlpOut + j] = 1.f;
  e = cudaMemcpy(m->norm, m->norm_host.data(), m->norm_host.size() * sizeof(float), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return bail(cuda_fail(e, "cudaMemcpy"));
  *out = m;
  return TC_OK;
}

void tc_mlp_destroy(tc_mlp* m) {
  if (!m) return;
  cudaSetDevice(m->device);
  cudaDeviceSynchronize();
  for (void* p : {(void*)m->params, (void*)m->grads, (void*)m->adam_m, (void*)m->adam_v, (void*)m->wt,
                  (void*)m->norm, (void*)m->dz, (void*)m->da, (void*)m->tgt, (void*)m->idx,
                  (void*)m->loss, (void*)m->img, (void*)m->splitk, (void*)m->gw0d, (void*)m->wt0d,
                  (void*)m->dzT, (void*)m->actT, (void*)m->dzb, (void*)m->wT, (void*)m->gemm_err,
                  (void*)m->counters})
    cudaFree(p);
  for (int l = 0; l < kMlpLayers; ++l) {
    cudaFree(m->act[l]);
    cudaFree(m->z[l]);
  }
  delete m;
}

tc_status tc_mlp_n_params(const tc_mlp* m, int64_t* n) {
  clear_error();
  if (!m || !n) return fail(TC_ERR_ARG, "null argument");
  *n = m->d.n_params;
  return TC_OK;
}

tc_status tc_mlp_get_params(const tc_mlp* m, float* host, int64_t n) {
  clear_error();
  if (!m || !host || n != m->d.n_params) return fail(TC_ERR_ARG, "bad arguments");
  CUDA_TRY(cudaSetDevice(m->device));
  CUDA_TRY(cudaMemcpy(host, m->params, n * sizeof(float), cudaMemcpyDeviceToHost));
  return TC_OK;
}

tc_status tc_mlp_set_params(tc_mlp* m, const float* host, int64_t n) {
  clear_error();
  if (!m || !host || n != m->d.n_params) return fail(TC_ERR_ARG, "bad arguments");
  CUDA_TRY(cudaSetDevice(m->device));
  CUDA_TRY(cudaMemcpy(m->params, host, n * sizeof(float), cudaMemcpyHostToDevice));
  mask_padding_kernel<<<blocks_for(256 * kMlpPad), 256>>>(m->params, m->d.w_off[0], m->d.w_off[kMlpLayers - 1],
                                                          m->d.b_off[kMlpLayers - 1]);
  cast_kernel<<<blocks_for(n), 256>>>(n, m->params, m->wt);
  TRY(rebuild_images(m, 0));
  CUDA_TRY(cudaDeviceSynchronize());
  return TC_OK;
}

tc_status tc_mlp_set_normalization(tc_mlp* m, const float* host, int64_t n) {
  clear_error();
  if (!m || !host || n != 2 * kMlpIn + 2 * kMlpOut) return fail(TC_ERR_ARG, "bad normalization");
  for (int64_t j = 0; j < n; ++j)
    if (!std::isfinite(host[j])) return fail(TC_ERR_ARG, "non-finite normalization");
  for (int j = 0; j < kMlpIn; ++j)
    if (!(host[kMlpIn + j] > 0.f)) return fail(TC_ERR_ARG, "input scales must be > 0");
  for (int j = 0; j < kMlpOut; ++j)
    if (!(host[2 * kMlpIn + kMlpOut + j] > 0.f)) return fail(TC_ERR_ARG, "output scales must be > 0");
  m->norm_host.assign(host, host + n);
  CUDA_TRY(cudaSetDevice(m->device));
  CUDA_TRY(cudaMemcpy(m->norm, host, n * sizeof(float), cudaMemcpyHostToDevice));
  return TC_OK;
}

// Fit the normalization to a device training set (x [n][20] features, y [n][19] next states):
// feature and output-change means, and standard deviations as scales (1 where a column is
// constant, so that it passes through unscaled).
tc_status tc_mlp_fit_normalization(tc_mlp* m, const float* x_dev, const float* y_dev, int64_t n) {
  clear_error();
  if (!m || !x_dev || !y_dev || n < 2) return fail(TC_ERR_ARG, "bad arguments");
  CUDA_TRY(cudaSetDevice(m->device));
  constexpr int C = kMlpIn + kMlpOut;
  double* d = nullptr;
  CUDA_TRY(cudaMalloc(&d, 2 * C * sizeof(double)));
  column_stats_kernel<<<C, 1024>>>(n, x_dev, y_dev, 0, d, d + C);
  column_stats_kernel<<<C, 1024>>>(n, x_dev, y_dev, 1, d, d + C);
  double h[2 * C];
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return cuda_fail(e, "normalization statistics");
  std::vector<float> norm(2 * kMlpIn + 2 * kMlpOut);
  for (int c = 0; c < C; ++c) {
    const double mu = h[c], sd = h[C + c];
    const bool flat = !(sd > 1e-12 * std::max(1.0, std::fabs(mu)));
    if (c < kMlpIn) {
      norm[c] = (float)mu;
      norm[kMlpIn + c] = flat ? 1.f : (float)sd;
    } else {
      norm[2 * kMlpIn + (c - kMlpIn)] = (float)mu;
      norm[2 * kMlpIn + kMlpOut + (c - kMlpIn)] = flat ? 1.f : (float)sd;
    }
  }
  return tc_mlp_set_normalization(m, norm.data(), (int64_t)norm.size());
}

tc_status tc_mlp_get_normalization(const tc_mlp* m, float* host, int64_t n) {
  clear_error();
  if (!m || !host || n != (int64_t)m->norm_host.size()) return fail(TC_ERR_ARG, "bad arguments");
  std::copy(m->norm_host.begin(), m->norm_host.end(), host);
  return TC_OK;
}

tc_status tc_mlp_set_gemm(tc_mlp* m, int32_t impl) {
  clear_error();
  if (!m || (impl != kGemmTcgen05 && impl != kGemmSimt)) return fail(TC_ERR_ARG, "bad GEMM choice");
  m->gemm = impl;
  return TC_OK;
}

// Forward pass of already-normalized inputs: x [n][20] -> y [n][19] normalized outputs (host).
tc_status tc_mlp_forward(tc_mlp* m, const float* x, int64_t n, float* y) {
  clear_error();
  if (!m || !x || !y || n < 1) return fail(TC_ERR_ARG, "bad arguments");
  CUDA_TRY(cudaSetDevice(m->device));
  TRY(ensure_workspace(m, n));
  std::vector<__nv_bfloat16> a0(n * kMlpIn0);
  for (int64_t r = 0; r < n; ++r) mlp_split_input(x + r * kMlpIn, a0.data() + r * kMlpIn0);
  CUDA_TRY(cudaMemcpy(m->act[0], a0.data(), a0.size() * sizeof(__nv_bfloat16), cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemset(reinterpret_cast<int*>(m->loss) + 1, 0, sizeof(int)));
  TRY(forward(m, n, 0));
  int err = 0;
  CUDA_TRY(cudaMemcpy(&err, reinterpret_cast<int*>(m->loss) + 1, sizeof(int), cudaMemcpyDeviceToHost));
  if (m->gemm == kGemmTcgen05 && err) return fail(TC_ERR_TIMEOUT, "tensor-core MLP wait hit its limit");
  std::vector<float> z(n * kMlpPad);
  CUDA_TRY(cudaMemcpy(z.data(), m->z[kMlpLayers - 1], z.size() * sizeof(float), cudaMemcpyDeviceToHost));
  for (int64_t r = 0; r < n; ++r)
    for (int c = 0; c < kMlpOut; ++c) y[r * kMlpOut + c] = z[r * kMlpPad + c];
  return TC_OK;
}

// Loss and gradients for normalized inputs x [n][20] and normalized targets t [n][19] (host):
// the mean squared error over the real outputs and its gradient with respect to every
// parameter (weights as W^T [out][in], then biases), as the training step computes them.
tc_status tc_mlp_gradients(tc_mlp* m, const float* x, const float* t, int64_t n, float* grads,
                           float* loss) {
  clear_error();
  if (!m || !x || !t || !grads || !loss || n < 1) return fail(TC_ERR_ARG, "bad arguments");
  CUDA_TRY(cudaSetDevice(m->device));
  TRY(ensure_workspace(m, n));
  std::vector<__nv_bfloat16> a0(n * kMlpIn0);
  std::vector<float> tg(n * kMlpPad, 0.f);
  for (int64_t r = 0; r < n; ++r) {
    mlp_split_input(x + r * kMlpIn, a0.data() + r * kMlpIn0);
    for (int c = 0; c < kMlpOut; ++c) tg[r * kMlpPad + c] = t[r * kMlpOut + c];
  }
  CUDA_TRY(cudaMemcpy(m->act[0], a0.data(), a0.size() * sizeof(__nv_bfloat16), cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(m->tgt, tg.data(), tg.size() * sizeof(float), cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemset(m->gemm_err, 0, sizeof(int)));
  CUDA_TRY(cudaMemset(reinterpret_cast<int*>(m->loss) + 1, 0, sizeof(int)));
  TRY(forward(m, n, 0));
  TRY(backward(m, n, 0));
  CUDA_TRY(cudaMemcpy(grads, m->grads, m->d.n_params * sizeof(float), cudaMemcpyDeviceToHost));
  CUDA_TRY(cudaMemcpy(loss, m->loss, sizeof(float), cudaMemcpyDeviceToHost));
  int err[2] = {0, 0};
  CUDA_TRY(cudaMemcpy(&err[0], reinterpret_cast<int*>(m->loss) + 1, sizeof(int), cudaMemcpyDeviceToHost));
  CUDA_TRY(cudaMemcpy(&err[1], m->gemm_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (m->gemm == kGemmTcgen05 && (err[0] || err[1])) return fail(TC_ERR_TIMEOUT, "a tensor-core wait hit its limit");
  return TC_OK;
}

// Train on a device data set: x [n][20] raw features, y [n][19] raw next states (FP32, device).
// Mini-batches drawn by a seeded shuffle per epoch; Adam.  loss_history[epoch] = mean batch loss.
tc_status tc_mlp_train(tc_mlp* m, const float* x_dev, const float* y_dev, int64_t n, int32_t epochs,
                       int32_t batch, float lr, uint64_t seed, void* stream, float* loss_history) {
  clear_error();
  if (!m || !x_dev || !y_dev || n < batch || epochs < 1 || batch < 32 || !(lr > 0.f))
    return fail(TC_ERR_ARG, "bad training arguments");
  CUDA_TRY(cudaSetDevice(m->device));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  TRY(ensure_workspace(m, batch));
  const int64_t nb = n / batch;
  std::vector<int32_t> order(n);
  for (int64_t i = 0; i < n; ++i) order[i] = (int32_t)i;
  int32_t* d_order = nullptr;
  CUDA_TRY(cudaMalloc(&d_order, n * sizeof(int32_t)));
  uint64_t rng = seed;
  auto next = [&]() {
    rng += 0x9E3779B97F4A7C15ull;
    uint64_t z = rng;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  };
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  float* d_sum = m->loss + 2;
  int* d_err = reinterpret_cast<int*>(m->loss) + 1;
  // One training step: gather the batch (its index in the epoch from counters[0]), forward,
  // backward, Adam (step count from counters[1]), weight images, advance the counters.  Captured
  // once per call as a CUDA graph and replayed for every batch; launched directly if capture fails.
  auto record_step = [&](cudaStream_t cs) -> tc_status {
    gather_batch_kernel<<<blocks_for((int64_t)batch * kMlpPad), 256, 0, cs>>>(
        batch, d_order, m->counters, x_dev, y_dev, m->norm, m->act[0], m->tgt);
    TRY(forward(m, batch, cs));
    TRY(backward(m, batch, cs));
    accumulate_kernel<<<1, 1, 0, cs>>>(d_sum, m->loss);
    adam_kernel<<<blocks_for(m->d.n_params), 256, 0, cs>>>(m->d.n_params, m->params, m->grads, m->adam_m,
                                                           m->adam_v, m->wt, lr, b1, b2, eps, m->counters);
    TRY(rebuild_images(m, cs));   // duplicated layer-0 weights and tensor-core images
    train_tick_kernel<<<1, 1, 0, cs>>>(m->counters);
    CUDA_TRY(cudaGetLastError());
    return TC_OK;
  };
  cudaGraphExec_t exec = nullptr;
  {
    cudaStream_t cs;
    CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    tc_status rs = e == cudaSuccess ? record_step(cs) : TC_ERR_CUDA;
    if (e == cudaSuccess) {
      cudaError_t e2 = cudaStreamEndCapture(cs, &g);
      if (rs == TC_OK && e2 == cudaSuccess && cudaGraphInstantiate(&exec, g, 0) != cudaSuccess) exec = nullptr;
      if (g) cudaGraphDestroy(g);
    }
    cudaStreamDestroy(cs);
    cudaGetLastError();   // a failed capture leaves no sticky error; launch step by step then
    clear_error();
  }
  int h_counters[2] = {0, (int)m->adam_t};
  tc_status status = TC_OK;
  for (int ep = 0; ep < epochs && status == TC_OK; ++ep) {
    for (int64_t i = n - 1; i > 0; --i) std::swap(order[i], order[next() % (uint64_t)(i + 1)]);
    h_counters[0] = 0;
    cudaError_t e = cudaMemcpyAsync(d_order, order.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(m->counters, h_counters, 2 * sizeof(int), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_sum, 0, sizeof(float), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_err, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->gemm_err, 0, sizeof(int), st);
    if (e != cudaSuccess) {
      status = cuda_fail(e, "training epoch set-up");
      break;
    }
    for (int64_t bi = 0; bi < nb && status == TC_OK; ++bi) {
      if (exec) {
        e = cudaGraphLaunch(exec, st);
        if (e != cudaSuccess) status = cuda_fail(e, "training step");
      } else {
        status = record_step(st);
      }
    }
    if (status != TC_OK) break;
    float sums[2] = {0.f, 0.f};
    cudaMemcpyAsync(sums, d_sum, sizeof(float), cudaMemcpyDeviceToHost, st);
    int err = 0, gerr = 0;
    cudaMemcpyAsync(&err, d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(&gerr, m->gemm_err, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaError_t e2 = cudaStreamSynchronize(st);
    if (e2 != cudaSuccess) {
      status = cuda_fail(e2, "training epoch");
      break;
    }
    h_counters[1] += (int)nb;
    m->adam_t = h_counters[1];
    if (m->gemm == kGemmTcgen05 && (err || gerr)) status = fail(TC_ERR_TIMEOUT, "tensor-core MLP wait hit its limit");
    const float mean = sums[0] / (float)nb;
    if (loss_history) loss_history[ep] = mean;
    if (!std::isfinite(mean)) status = fail(TC_ERR_NAN, "training loss is not finite");
  }
  if (exec) cudaGraphExecDestroy(exec);
  cudaFree(d_order);
  cudaStreamSynchronize(st);
  return status;
}

// Exact single-cell windows (the training targets and the reference the surrogate is checked against):
// in [19][n] (18 states then V), istim [n] pA/pF or NULL, out [19][n]; device arrays, FP32
// storage, arithmetic in FP64 (precision = TC_FP64) or FP32.
tc_status tc_tp06_window(const float* in_dev, const float* istim_dev, int64_t n, double dt, int32_t nsub,
                         int32_t cell, int32_t precision, float* out_dev, void* stream) {
  clear_error();
  if (!in_dev || !out_dev || n < 1 || !(dt > 0) || nsub < 1 || cell < 0 || cell > 2)
    return fail(TC_ERR_ARG, "bad window arguments");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (precision == TC_FP64)
    tp06_window_kernel<double><<<blocks_for(n), 256, 0, st>>>(n, in_dev, istim_dev, out_dev, cell, dt, nsub);
  else
    tp06_window_kernel<float><<<blocks_for(n), 256, 0, st>>>(n, in_dev, istim_dev, out_dev, cell, dt, nsub);
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaStreamSynchronize(st));
  return TC_OK;
}

// C [M][N] (FP32) = A [M][K] . B [N][K]^T with BF16 A, B on the device (row-major, K
// contiguous); the tensor-core GEMM of the training pass, exposed for direct checks.
tc_status tc_gemm_bf16_nt(const void* a_dev, const void* b_dev, float* c_dev, int32_t M, int32_t N, int32_t K,
                          void* stream) {
  clear_error();
  if (!a_dev || !b_dev || !c_dev || M < 1 || N < 1 || K < 8 || (K & 7)) return fail(TC_ERR_ARG, "bad GEMM arguments");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  static int* d_err = nullptr;
  static bool attr = false;
  if (!d_err) CUDA_TRY(cudaMalloc(&d_err, sizeof(int)));
  if (!attr) {
    CUDA_TRY(cudaFuncSetAttribute(gemm_nt_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)gemm_nt_smem_bytes(256)));
    attr = true;
  }
  CUDA_TRY(cudaMemsetAsync(d_err, 0, sizeof(int), st));
  TRY(gemm_nt(M, N, K, static_cast<const __nv_bfloat16*>(a_dev), K, static_cast<const __nv_bfloat16*>(b_dev), K,
              c_dev, N, st, nullptr, d_err));
  int err = 0;
  CUDA_TRY(cudaMemcpyAsync(&err, d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  if (err) return fail(TC_ERR_TIMEOUT, "a tensor-core GEMM wait hit its limit");
  return TC_OK;
}

tc_status tc_mlp_diagnostics(const tc_mlp* m, tc_mlp_diag* out) {
  clear_error();
  if (!m || !out) return fail(TC_ERR_ARG, "null argument");
  out->gemm = m->gemm;
  out->n_params = m->d.n_params;
  out->adam_steps = m->adam_t;
  return TC_OK;
}

}  // extern "C"

// ---- surrogate inference inside the time step ---------------------------------------------

namespace tc {

// Window start, every node: the checks that need no prediction decide whether the node is a
// candidate for the network this window - a real row, no stimulus during the window, |dV/dt| on
// the step before within dvdt_max, V outside the resting band (a resting cell's tiny gate values
// and slow drift are below the network's resolution, and errors there would change the tissue's
// excitability ahead of the next wave), and, with dv_nbr > 0, no matrix-row neighbour differing
// from it by more than dv_nbr mV (a front next to it could cross the window; the network sees one
// cell, not the diffusion that drives the front).  Candidates get a compacted input row (18
// states, V, window-mean stimulus; normalized, split BF16) at a position taken from *count, and
// idx[pos] = node; everyone else stays with the exact model (flag 0) and is counted as such.
template <typename T>
__global__ void sur_features_kernel(int64_t n, const T* state, const T* V, const T* Vprev,
                                    const T* dinv, const int32_t* stim_off, const int32_t* stim_ids,
                                    const StimDev* stims, const long long* k_base, int k_off, int win, double cm,
                                    double dt, float dvdt_max, float v_rest, float rest_band, float dv_nbr,
                                    const int32_t* slice_ptr, const int32_t* col, const float* norm,
                                    __nv_bfloat16* a0, float* raw, int32_t* idx, int* count, uint8_t* flag,
                                    unsigned long long* counts) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool real = i < n && dinv[i] != T(0);
  bool cand = real;
  float vi = 0.f, is = 0.f;
  if (cand) {
    vi = (float)V[i];
    const long long k0 = *k_base + k_off;
    double acc = 0.0;
    for (int s = 0; s < win; ++s) acc += stimulus_at(stim_off, stim_ids, stims, i, k0 + s);
    is = (float)(acc / win / cm);   // uA/mm^2 -> pA/pF
    cand = is == 0.f && fabsf(vi - (float)Vprev[i]) <= dvdt_max * (float)dt &&
           !(rest_band > 0.f && fabsf(vi - v_rest) <= rest_band);
  }
  if (cand && dv_nbr > 0.f) {
    const int64_t s = i >> 5;
    const int beg = slice_ptr[s] + (int)(i & 31);
    const int w = (slice_ptr[s + 1] - slice_ptr[s]) >> 5;
    // chunks of eight entries: the column indices first, then the gathers (two rounds of
    // dependent loads for a 15-entry row instead of fifteen); the maximum is order-free
    float d = 0.f;
    for (int j = 0; j < w; j += 8) {
      int c[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) c[u] = j + u < w ? __ldg(col + beg + 32 * (j + u)) : -1;
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (c[u] >= 0) d = fmaxf(d, fabsf((float)V[c[u]] - vi));
    }
    cand = d <= dv_nbr;
  }
  if (i < n) flag[i] = 0;
  // one atomic per block (256 threads): the warps' candidate counts are laid out in warp order
  // behind the block's base
  const unsigned cm_ = __ballot_sync(0xffffffffu, cand);
  const unsigned rm = __ballot_sync(0xffffffffu, real && !cand);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __shared__ int s_wc[8], s_rc[8], s_base;
  if (lane == 0) {
    s_wc[warp] = __popc(cm_);
    s_rc[warp] = __popc(rm);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int tot = 0, rtot = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      const int c = s_wc[w];
      s_wc[w] = tot;
      tot += c;
      rtot += s_rc[w];
    }
    s_base = tot ? atomicAdd(count, tot) : 0;
    if (rtot) atomicAdd(&counts[1], (unsigned long long)rtot);
  }
  __syncthreads();
  const int base = s_base + s_wc[warp];
  if (!cand) return;
  const int pos = base + __popc(cm_ & ((1u << lane) - 1u));
  idx[pos] = (int32_t)i;
  float f[kMlpIn];
#pragma unroll
  for (int j = 0; j < 18; ++j) f[j] = (float)state[j * n + i];
  f[18] = vi;
  f[19] = is;
  float xn[kMlpIn];
#pragma unroll
  for (int j = 0; j < kMlpIn; ++j) {
    raw[j * n + i] = f[j];
    xn[j] = (f[j] - norm[j]) / norm[kMlpIn + j];
  }
  __align__(16) __nv_bfloat16 h[kMlpIn0];
  mlp_split_input(xn, h);
#pragma unroll
  for (int u = 0; u < kMlpIn0 / 8; ++u)
    reinterpret_cast<uint4*>(a0 + (int64_t)pos * kMlpIn0)[u] = reinterpret_cast<const uint4*>(h)[u];
}

// Candidates: decode the prediction (row pos, node idx[pos]), check it (finite, concentrations
// positive, gates inside [0, 1] up to a small margin, |V' - V| <= dv_max) and commit: states <-
// prediction, flag, the window's effective current.
template <typename T>
__global__ void sur_commit_kernel(const int* count, int64_t n, const int32_t* idx, const float* zout,
                                  const float* raw, const float* norm, double dt, int win, float dv_max,
                                  T* state, uint8_t* flag, float* iion, unsigned long long* counts,
                                  double* log_cache) {
  const int64_t pos = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool have = pos < *count;
  bool ok = false;
  if (have) {
    const int64_t i = idx[pos];
    const float* out_mean = norm + 2 * kMlpIn;
    const float* out_scale = norm + 2 * kMlpIn + kMlpOut;
    float y[kMlpOut];
    ok = true;
#pragma unroll
    for (int j = 0; j < kMlpOut; ++j) {
      y[j] = raw[j * n + i] + out_mean[j] + out_scale[j] * zout[pos * kMlpPad + j];
      ok = ok && isfinite(y[j]);
    }
#pragma unroll
    for (int j = 0; j < 5; ++j) ok = ok && y[j] > 0.f;
#pragma unroll
    for (int j = 5; j < 18; ++j) ok = ok && y[j] > -0.01f && y[j] < 1.01f;
    const float dv = y[18] - raw[18 * n + i];
    ok = ok && fabsf(dv) <= dv_max;
    flag[i] = ok ? 1 : 0;
    if (ok) {
#pragma unroll
      for (int j = 0; j < 18; ++j) state[j * n + i] = T(j >= 5 ? fminf(fmaxf(y[j], 0.f), 1.f) : y[j]);
      // the held logarithms no longer describe the states: the node's next exact step takes them anew
      if (log_cache) log_cache[i] = __longlong_as_double(0x7ff8000000000000ll);
      // single cell: dV/dt = -I_ion + I_stim over the window (no stimulus here)
      iion[i] = raw[19 * n + i] - dv / (float)(win * dt);
    }
  }
  // one pair of atomics per block (256 threads)
  const unsigned okm = __ballot_sync(0xffffffffu, ok);
  const unsigned hm = __ballot_sync(0xffffffffu, have);
  __shared__ int s_ok[8], s_have[8];
  const int warp = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    s_ok[warp] = __popc(okm);
    s_have[warp] = __popc(hm);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int o = 0, h = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      o += s_ok[w];
      h += s_have[w];
    }
    if (h) {
      atomicAdd(&counts[0], (unsigned long long)o);
      atomicAdd(&counts[1], (unsigned long long)(h - o));
    }
  }
}

tc_status surrogate_prepare(tc_mlp* m, int64_t n) {
  CUDA_TRY(cudaSetDevice(m->device));
  return m->gemm == kGemmTcgen05 ? TC_OK : ensure_workspace(m, n);
}

tc_status surrogate_infer(tc_mlp* m, const SurrogateStep& q, cudaStream_t st) {
  CUDA_TRY(cudaMemsetAsync(q.count, 0, sizeof(int), st));
  if (q.fp64)
    sur_features_kernel<double><<<blocks_for(q.n), 256, 0, st>>>(
        q.n, static_cast<const double*>(q.state), static_cast<const double*>(q.V),
        static_cast<const double*>(q.Vprev), static_cast<const double*>(q.dinv), q.stim_off, q.stim_ids, q.stims,
        q.k_base, q.k_off, q.win, q.cm, q.dt, q.dvdt_max, q.v_rest, q.rest_band, q.dv_nbr, q.slice_ptr, q.col,
        m->norm, q.a0, q.raw, q.idx, q.count, q.flag, q.counts);
  else
    sur_features_kernel<float><<<blocks_for(q.n), 256, 0, st>>>(
        q.n, static_cast<const float*>(q.state), static_cast<const float*>(q.V), static_cast<const float*>(q.Vprev),
        static_cast<const float*>(q.dinv), q.stim_off, q.stim_ids, q.stims, q.k_base, q.k_off, q.win, q.cm, q.dt,
        q.dvdt_max, q.v_rest, q.rest_band, q.dv_nbr, q.slice_ptr, q.col, m->norm, q.a0, q.raw, q.idx, q.count,
        q.flag, q.counts);
  CUDA_TRY(cudaGetLastError());
  if (q.ev_mlp[0]) CUDA_TRY(cudaEventRecord(q.ev_mlp[0], st));
  if (m->gemm == kGemmTcgen05) {
    TRY(forward_tc(m, q.n, q.a0, q.zout, false, q.err, st, q.count));
  } else {
    TRY(ensure_workspace(m, q.n));
    CUDA_TRY(cudaMemcpyAsync(m->act[0], q.a0, q.n * kMlpIn0 * sizeof(__nv_bfloat16), cudaMemcpyDeviceToDevice, st));
    TRY(forward(m, q.n, st));
    CUDA_TRY(cudaMemcpyAsync(q.zout, m->z[kMlpLayers - 1], q.n * kMlpPad * sizeof(float), cudaMemcpyDeviceToDevice, st));
  }
  if (q.ev_mlp[1]) CUDA_TRY(cudaEventRecord(q.ev_mlp[1], st));
  if (q.fp64)
    sur_commit_kernel<double><<<blocks_for(q.n), 256, 0, st>>>(q.count, q.n, q.idx, q.zout, q.raw, m->norm, q.dt,
                                                               q.win, q.dv_max, static_cast<double*>(q.state),
                                                               q.flag, q.iion, q.counts, q.log_cache);
  else
    sur_commit_kernel<float><<<blocks_for(q.n), 256, 0, st>>>(q.count, q.n, q.idx, q.zout, q.raw, m->norm, q.dt,
                                                              q.win, q.dv_max, static_cast<float*>(q.state), q.flag,
                                                              q.iion, q.counts, nullptr);
  CUDA_TRY(cudaGetLastError());
  return TC_OK;
}

}  // namespace tc
