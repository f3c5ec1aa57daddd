// Fused MLP forward on the 5th-generation tensor cores (tcgen05, sm_100-family).
//
// One CTA (512 threads) owns 128 rows at a time.  For each layer:
//   * the layer's weights W^T [N][K] arrive in shared memory as a pre-swizzled image through
//     bulk asynchronous copies (cp.async.bulk, completion counted on an mbarrier); the copy of
//     the next layer's image is issued as soon as this layer's MMAs have finished reading, so
//     it overlaps the epilogue;
//   * thread 0 issues tcgen05.mma (kind::f16, BF16 x BF16 -> FP32) over K in steps of 16,
//     accumulating the 128 x N tile in tensor memory, and commits to a second mbarrier;
//   * sixteen warps (four per tensor-memory lane quarter, each on a quarter of the columns)
//     read the accumulator back (tcgen05.ld), add the bias (staged in shared memory once per
//     CTA), apply SiLU and write the BF16 result straight into the swizzled shared-memory
//     operand of the next layer (optionally also Z and the activation to global memory for the
//     backward pass).
// Activations therefore never leave the chip between layers.
//
// Shared-memory operand layout (K-major, 128-byte swizzle): K is cut into panels of 64
// elements (128 bytes per row); inside a panel, rows are grouped in atoms of 8 rows x 128 B
// (1024 B, 1024-aligned) and 16-byte chunk c of row r sits at chunk position c ^ (r % 8).  The
// matrix descriptor for a K-step of 16 elements points at the panel plus 32 B per step, with a
// stride of 1024 B between 8-row groups.  Every wait on an mbarrier is bounded; on expiry the
// CTA records an error, frees its tensor memory and leaves.
#pragma once

#include <cstdint>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "mlp.cuh"

namespace tc {

constexpr int kTcThreads = 512;
constexpr int kTcBias = 4 * kMlpHidden + kMlpPad;      // all biases, staged in shared memory
constexpr int kTcRows = 128;
constexpr uint32_t kTcSmemA = 4 * 128 * 128;            // 128 rows x 256 K, BF16
constexpr uint32_t kTcSmemW = 4 * 256 * 128;            // 256 rows x 256 K, BF16
constexpr uint32_t kTcSmemBytes = kTcSmemA + kTcSmemW + 1024 + kTcBias * 4;
constexpr long long kTcWaitLimit = 1ll << 24;

struct MlpFusedArgs {
  int64_t M;                               // rows (an upper bound when M_dev is set)
  const int* M_dev;                        // optional device row count (read by every CTA)
  const __nv_bfloat16* a0;                 // [M][64] split-BF16 inputs (normalized; hi | lo)
  const uint8_t* img[kMlpLayers];          // swizzled weight images
  uint32_t img_bytes[kMlpLayers];
  const float* bias[kMlpLayers];
  int in[kMlpLayers], out[kMlpLayers];
  float* z[kMlpLayers];                    // optional [M][out] pre-activations
  __nv_bfloat16* act[kMlpLayers];          // optional act[l] = input of layer l, [M][in]
  float* y;                                // [M][32] output of the last layer (FP32)
  int* err;
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (long long it = 0; it < kTcWaitLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 1024 B between 8-row
// groups (fields: start >> 4 at bit 0, leading offset (unused for this layout, 1) at bit 16,
// stride >> 4 at bit 32, descriptor version 1 at bit 46, layout 2 = 128-byte swizzle at bit 61).
__device__ __forceinline__ uint64_t umma_desc_sw128(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor of kind::f16: FP32 accumulator (bit 4), A and B BF16 (bits 7, 10),
// both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_addr(bar))
               : "memory");
}

// 32 consecutive FP32 columns of this thread's tensor-memory lane, as raw words; the values
// are valid only after tmem_wait_ld().
__device__ __forceinline__ void tmem_ld32_nowait(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// 16 consecutive FP32 columns of this thread's tensor-memory lane (valid after tmem_wait_ld16).
__device__ __forceinline__ void tmem_ld16_nowait(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}

// Wait for this thread's tensor-memory loads, with the 16 registers of the latest load tied to
// the wait so that no use of them is scheduled above it.
__device__ __forceinline__ void tmem_wait_ld16(uint32_t* r) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]),
                 "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]),
                 "+r"(r[14]), "+r"(r[15])
               :
               : "memory");
}

// Byte offset of 16-byte chunk `chunk` (0..7 inside a 64-element K panel) of row r in a
// swizzled operand with `rows` rows per panel.
__host__ __device__ __forceinline__ uint32_t sw128_offset(int panel, int rows, int r, int chunk) {
  return (uint32_t)panel * rows * 128u + (uint32_t)(r >> 3) * 1024u + (uint32_t)(r & 7) * 128u +
         (uint32_t)((chunk ^ (r & 7)) * 16);
}

__device__ __forceinline__ float tanh_approx(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
// SiLU z sigmoid(z) with sigmoid(z) = (1 + tanh(z/2)) / 2, as h + h tanh(h) with h = z/2: one
// special-function operation and two FP32 instructions.
__device__ __forceinline__ float silu_fast(float z) {
  const float h = 0.5f * z;
  return fmaf(h, tanh_approx(h), h);
}

// Issue the bulk copies of one layer's weight image into sW (thread 0).
__device__ __forceinline__ void load_weights(uint8_t* sW, const uint8_t* img, uint32_t bytes, uint64_t* bar) {
  mbar_expect_tx(bar, bytes);
  for (uint32_t off = 0; off < bytes; off += 32768u) {
    const uint32_t nb = bytes - off < 32768u ? bytes - off : 32768u;
    bulk_copy_g2s(sW + off, img + off, nb, bar);
  }
}

template <bool STORE>
__global__ void __launch_bounds__(kTcThreads, 1) mlp_fused_kernel(const MlpFusedArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;
  uint8_t* sW = smem + kTcSmemA;
  float* sBias = reinterpret_cast<float*>(sW + kTcSmemW);
  __shared__ uint64_t bar_w, bar_mma;
  __shared__ uint32_t s_tmem;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t M = a.M_dev ? (a.M < (int64_t)*a.M_dev ? a.M : (int64_t)*a.M_dev) : a.M;
  const int64_t ntiles = (M + kTcRows - 1) / kTcRows;
  if (tid == 0) {
    mbar_init(&bar_w, 1);
    mbar_init(&bar_mma, 1);
  }
  {
    int off = 0;
    for (int l = 0; l < kMlpLayers; ++l) {
      for (int c = tid; c < a.out[l]; c += kTcThreads) sBias[off + c] = a.bias[l][c];
      off += a.out[l];
    }
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&s_tmem)),
                 "r"(256)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  // Work thread 0 has outstanding on the two barriers (a weight copy, an MMA group) and the
  // phase each completes; on a failure it waits for them before the CTA frees its memory.
  bool pend_w = false, pend_m = false;
  uint32_t pend_w_ph = 0, pend_m_ph = 0;
  uint32_t ph_w = 0, ph_m = 0;
  bool bad = false;               // this thread saw a wait give up (sticky)
  bool any_bad = false;           // some thread of the CTA did (uniform, from __syncthreads_or)
  if (tid == 0 && (int64_t)blockIdx.x < ntiles) {
    load_weights(sW, a.img[0], a.img_bytes[0], &bar_w);   // layer 0 of the first tile
    pend_w = true;
    pend_w_ph = ph_w;
  }
  const int q = warp & 3;        // tensor-memory lane quarter of this warp
  const int cg = warp >> 2;      // column quarter handled by this warp
  const int row = 32 * q + lane;
  for (int64_t tile = blockIdx.x; tile < ntiles && !any_bad; tile += gridDim.x) {
    const int64_t row0 = tile * kTcRows;
    // inputs: 128 rows x 64 BF16 (one 128-byte panel row each) into panel 0
    for (int e = tid; e < kTcRows * 8; e += kTcThreads) {
      const int r = e >> 3, c = e & 7;
      const int64_t gr = row0 + r;
      uint4 v = make_uint4(0, 0, 0, 0);
      if (gr < M) v = *reinterpret_cast<const uint4*>(a.a0 + gr * kMlpIn0 + c * 8);
      *reinterpret_cast<uint4*>(sA + sw128_offset(0, kTcRows, r, c)) = v;
    }
    fence_proxy_async_smem();
    int boff = 0;
    for (int l = 0; l < kMlpLayers; ++l) {
      const int K = a.in[l], N = a.out[l];
      if (mbar_wait(&bar_w, ph_w)) {
        if (tid == 0) pend_w = false;
      } else {
        bad = true;
      }
      ph_w ^= 1u;
      any_bad = __syncthreads_or(bad);
      if (any_bad) break;
      tc_fence_after();
      if (tid == 0) {
        const uint32_t idesc = umma_idesc_bf16(kTcRows, N);
        for (int ks = 0; ks < K / 16; ++ks) {
          const int panel = ks >> 2;
          const uint32_t koff = (uint32_t)(ks & 3) * 32u;
          const uint64_t ad = umma_desc_sw128(smem_addr(sA + panel * kTcRows * 128) + koff);
          const uint64_t bd = umma_desc_sw128(smem_addr(sW + panel * N * 128) + koff);
          umma_bf16(tmem, ad, bd, idesc, ks > 0 ? 1u : 0u);
        }
        umma_commit(&bar_mma);
        pend_m = true;
        pend_m_ph = ph_m;
      }
      if (mbar_wait(&bar_mma, ph_m)) {
        if (tid == 0) pend_m = false;
      } else {
        bad = true;
      }
      ph_m ^= 1u;
      tc_fence_after();
      // the MMAs have read sW: start the next image (next layer, or layer 0 of the next tile)
      if (tid == 0 && !bad) {
        const bool more = l + 1 < kMlpLayers || tile + gridDim.x < ntiles;
        if (more) {
          const int nl = l + 1 < kMlpLayers ? l + 1 : 0;
          load_weights(sW, a.img[nl], a.img_bytes[nl], &bar_w);
          pend_w = true;
          pend_w_ph = ph_w;
        }
      }
      any_bad = __syncthreads_or(bad);
      if (any_bad) break;
      // epilogue: warp (q, cg) handles lanes 32q..32q+31 and a quarter of the columns
      const int cols = N / 4 >= 32 ? N / 4 : 32;
      const int cbeg = cg * cols;
      const int64_t grow = row0 + row;
      const bool valid = grow < M;
      if (cbeg < N) {
        const int nch = cols / 32;   // 1 or 2 chunks of 32 columns (uniform in the warp)
        uint32_t raw[2][32];
#pragma unroll
        for (int ch = 0; ch < 2; ++ch)
          if (ch < nch) tmem_ld32_nowait(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(cbeg + 32 * ch), raw[ch]);
        tmem_wait_ld();
#pragma unroll
        for (int ch = 0; ch < 2; ++ch) {
          if (ch >= nch) break;
          const int c0 = cbeg + 32 * ch;
          float v[32];
          const float4* b4 = reinterpret_cast<const float4*>(sBias + boff + c0);   // 16-byte aligned
#pragma unroll
          for (int j = 0; j < 32; j += 4) {
            const float4 bb = b4[j >> 2];
            v[j] = __uint_as_float(raw[ch][j]) + bb.x;
            v[j + 1] = __uint_as_float(raw[ch][j + 1]) + bb.y;
            v[j + 2] = __uint_as_float(raw[ch][j + 2]) + bb.z;
            v[j + 3] = __uint_as_float(raw[ch][j + 3]) + bb.w;
          }
          if (l + 1 < kMlpLayers) {
            if (STORE && valid && a.z[l]) {
              float* zp = a.z[l] + grow * N + c0;
#pragma unroll
              for (int j = 0; j < 32; j += 4) *reinterpret_cast<float4*>(zp + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
            }
            __align__(16) __nv_bfloat162 h[16];   // column pairs, one conversion each
#pragma unroll
            for (int j = 0; j < 16; ++j) h[j] = __floats2bfloat162_rn(silu_fast(v[2 * j]), silu_fast(v[2 * j + 1]));
            const int panel = c0 >> 6, chunk0 = (c0 & 63) >> 3;
#pragma unroll
            for (int u = 0; u < 4; ++u)
              *reinterpret_cast<uint4*>(sA + sw128_offset(panel, kTcRows, row, chunk0 + u)) =
                  reinterpret_cast<const uint4*>(h)[u];
            if (STORE && valid && a.act[l + 1]) {
              __nv_bfloat16* ap = a.act[l + 1] + grow * N + c0;
#pragma unroll
              for (int u = 0; u < 4; ++u) reinterpret_cast<uint4*>(ap)[u] = reinterpret_cast<const uint4*>(h)[u];
            }
          } else if (valid) {
            float* yp = a.y + grow * kMlpPad + c0;
#pragma unroll
            for (int j = 0; j < 32; j += 4) *reinterpret_cast<float4*>(yp + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
            if (STORE && a.z[l]) {
              float* zp = a.z[l] + grow * N + c0;
#pragma unroll
              for (int j = 0; j < 32; j += 4) *reinterpret_cast<float4*>(zp + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
            }
          }
        }
      }
      boff += N;
      fence_proxy_async_smem();
      tc_fence_before();
      __syncthreads();
    }
  }
  // after a failure: let thread 0's outstanding copy and MMA group land (bounded) before the
  // shared and tensor memory go away
  if (tid == 0 && any_bad) {
    atomicOr(a.err, 1);
    if (pend_m) mbar_wait(&bar_mma, pend_m_ph);
    if (pend_w) mbar_wait(&bar_w, pend_w_ph);
  }
  __syncthreads();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256) : "memory");
}

// ---- the pipelined forward: two row tiles per CTA, warp-specialised roles -------------------
//
// The kernel above runs a layer's MMAs and then its epilogue, so the tensor pipe idles while the
// sixteen epilogue warps read the accumulator back.  This one keeps two 128-row tiles (slots A
// and B) in flight with their accumulators in the two halves of tensor memory (2 x 256 columns):
// while the epilogue warps finish layer l of one slot, the tensor cores run the next job of the
// other.  Roles:
//   * warp 16, lane 0 (producer): streams the weight images as 64-wide K-panels (one contiguous
//     bulk copy each, <= 32 KB) through a two-stage ring, in the order the MMAs consume them;
//   * warp 17, lane 0 (MMA issuer): per job (slot, layer) waits for the slot's operand, then per
//     panel for its stage, issues the panel's four K-steps and commits to the stage's "empty"
//     barrier; after the last panel it commits to the slot's "accumulator full" barrier;
//   * warps 0-15 (epilogue): per job read the accumulator (tcgen05.ld), add the bias, apply SiLU
//     and write the next layer's BF16 operand into the slot (or the output), then signal the
//     slot's "operand ready" barrier; after a tile's last layer they load the next tile's inputs.
// Job order per CTA: tile pairs (2i, 2i + 1) for i = blockIdx.x, blockIdx.x + gridDim.x, ...;
// per pair layers 0..4, per layer slot A then slot B (B absent when the tile count is odd).
// The epilogue warps do not wait for one another: each arrives on the slot's operand barrier
// (16 arrivals per phase) when its columns of the next operand are written and its tensor-memory
// reads are done, and goes on to the other slot's job. A warp is never more than one phase ahead
// of the slowest, since the MMAs behind its next job need every warp's arrival.
// Every wait is bounded; a wait that gives up sets a shared abort flag that every role polls, so
// all roles leave their loops, and the CTA frees its tensor memory after the others have left.
constexpr int kT2EpiThreads = 512;
constexpr int kT2Threads = kT2EpiThreads + 64;
constexpr uint32_t kT2Panel = 256u * 128u;                                  // one K-panel, 256 rows
constexpr uint32_t kT2SmemBytes = 2 * kTcSmemA + 2 * kT2Panel + 1024 + kTcBias * 4;

__device__ __forceinline__ bool mbar_wait_abort(uint64_t* bar, uint32_t parity, volatile int* abort) {
  for (long long it = 0; it < kTcWaitLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    if (done) return true;
    if ((it & 255) == 255 && *abort) return false;
  }
  return false;
}

// One epilogue warp's arrival on a slot's operand barrier: every lane's shared-memory writes are
// made visible to the tensor cores' (async) proxy and its tensor-memory loads are ordered before
// the arrival.
__device__ __forceinline__ void epi_warp_arrive(uint64_t* bar, int lane) {
  fence_proxy_async_smem();
  tc_fence_before();
  __syncwarp();
  if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

template <bool STORE>
__global__ void __launch_bounds__(kT2Threads, 1) mlp_fused2_kernel(const MlpFusedArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* const sAct0 = smem;                       // slot A operand, 128 rows x 256 K
  uint8_t* const sW0 = smem + 2 * kTcSmemA;          // weight ring, two panels
  float* sBias = reinterpret_cast<float*>(sW0 + 2 * kT2Panel);
  __shared__ uint64_t full_b[2], empty_b[2], acc_b[2], act_b[2];
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort;
  volatile int* abort = &s_abort;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t M = a.M_dev ? (a.M < (int64_t)*a.M_dev ? a.M : (int64_t)*a.M_dev) : a.M;
  const int64_t ntiles = (M + kTcRows - 1) / kTcRows;
  const int64_t npairs = (ntiles + 1) / 2;
  if (tid == 0) {
    for (int i = 0; i < 2; ++i) {
      mbar_init(&full_b[i], 1);
      mbar_init(&empty_b[i], 1);
      mbar_init(&acc_b[i], 1);
      mbar_init(&act_b[i], kT2EpiThreads / 32);
    }
    s_abort = 0;
  }
  {
    // hidden layers keep half their bias: h = z/2 = fma(acc, 1/2, b/2) is the rounded (acc + b)/2
    // (halving is exact), so the SiLU's argument costs one instruction
    int off = 0;
    for (int l = 0; l < kMlpLayers; ++l) {
      const float f = l + 1 < kMlpLayers ? 0.5f : 1.0f;
      for (int c = tid; c < a.out[l]; c += kT2Threads) sBias[off + c] = f * a.bias[l][c];
      off += a.out[l];
    }
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&s_tmem)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  auto tile_exists = [&](int64_t pi, int x) { return 2 * pi + x < ntiles; };

  if (warp == kT2EpiThreads / 32) {
    // ---- producer: weight panels in consumption order ----
    if (lane == 0) {
      uint32_t g = 0;
      bool ok = true;
      for (int64_t pi = blockIdx.x; pi < npairs && ok; pi += gridDim.x)
        for (int l = 0; l < kMlpLayers && ok; ++l)
          for (int x = 0; x < 2 && ok; ++x) {
            if (!tile_exists(pi, x)) continue;
            const int np = (a.in[l] + 63) / 64;
            const uint32_t pbytes = (uint32_t)a.out[l] * 128u;
            for (int pp = 0; pp < np; ++pp, ++g) {
              const int st = g & 1;
              if (g >= 2 && !mbar_wait_abort(&empty_b[st], ((g >> 1) - 1) & 1, abort)) {
                ok = false;
                *abort = 1;
                break;
              }
              mbar_expect_tx(&full_b[st], pbytes);
              bulk_copy_g2s(sW0 + st * kT2Panel, a.img[l] + (size_t)pp * pbytes, pbytes, &full_b[st]);
            }
          }
      // the copies in flight land before the CTA's shared memory goes away
      for (uint32_t k = g > 2 ? g - 2 : 0; k < g; ++k) mbar_wait(&full_b[k & 1], (k >> 1) & 1);
    }
  } else if (warp == kT2EpiThreads / 32 + 1) {
    // ---- MMA issuer ----
    if (lane == 0) {
      uint32_t g = 0, nact[2] = {0, 0};
      bool ok = true;
      for (int64_t pi = blockIdx.x; pi < npairs && ok; pi += gridDim.x)
        for (int l = 0; l < kMlpLayers && ok; ++l)
          for (int x = 0; x < 2 && ok; ++x) {
            if (!tile_exists(pi, x)) continue;
            if (!mbar_wait_abort(&act_b[x], nact[x] & 1, abort)) {
              ok = false;
              *abort = 1;
              break;
            }
            ++nact[x];
            tc_fence_after();
            const int np = (a.in[l] + 63) / 64;
            const uint32_t idesc = umma_idesc_bf16(kTcRows, a.out[l]);
            const uint32_t tm = tmem + (uint32_t)(x * 256);
            uint8_t* sAct = sAct0 + x * kTcSmemA;
            for (int pp = 0; pp < np; ++pp, ++g) {
              const int st = g & 1;
              if (!mbar_wait_abort(&full_b[st], (g >> 1) & 1, abort)) {
                ok = false;
                *abort = 1;
                break;
              }
              tc_fence_after();
              for (int kk = 0; kk < 4; ++kk) {
                const uint64_t ad = umma_desc_sw128(smem_addr(sAct + pp * kTcRows * 128) + kk * 32u);
                const uint64_t bd = umma_desc_sw128(smem_addr(sW0 + st * kT2Panel) + kk * 32u);
                umma_bf16(tm, ad, bd, idesc, (pp > 0 || kk > 0) ? 1u : 0u);
              }
              umma_commit(&empty_b[st]);
            }
            if (ok) umma_commit(&acc_b[x]);
          }
      // the MMAs issued complete before tensor memory is freed
      if (g > 0) mbar_wait(&empty_b[(g - 1) & 1], ((g - 1) >> 1) & 1);
    }
  } else {
    // ---- epilogue warps ----
    const int q = warp & 3;        // tensor-memory lane quarter of this warp
    const int cg = warp >> 2;      // column quarter handled by this warp
    const int row = 32 * q + lane;
    uint32_t nacc[2] = {0, 0};
    // this warp's eight rows of a tile's layer-0 operand (16-byte chunks, coalesced), then its arrival
    auto load_inputs = [&](int64_t tile, int x) {
      uint8_t* sAct = sAct0 + x * kTcSmemA;
      const int64_t row0 = tile * kTcRows;
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int e = warp * 64 + j * 32 + lane;
        const int r = e >> 3, c = e & 7;
        const int64_t gr = row0 + r;
        uint4 v = make_uint4(0, 0, 0, 0);
        if (gr < M) v = *reinterpret_cast<const uint4*>(a.a0 + gr * kMlpIn0 + c * 8);
        *reinterpret_cast<uint4*>(sAct + sw128_offset(0, kTcRows, r, c)) = v;
      }
      epi_warp_arrive(&act_b[x], lane);
    };
    // The last layer's accumulator is 32 columns wide and read by warps 0-3; warps 8-15 fetch the
    // slot's next tile inputs into registers before that job's wait (16 rows each, hiding the
    // global-load latency behind the last layer's MMAs) and store them once its MMAs are done.
    uint4 pre[4];
    auto prefetch_inputs = [&](int64_t tile) {
      const int64_t row0 = tile * kTcRows;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int e = (warp - 8) * 128 + j * 32 + lane;
        const int64_t gr = row0 + (e >> 3);
        pre[j] = make_uint4(0, 0, 0, 0);
        if (gr < M) pre[j] = __ldg(reinterpret_cast<const uint4*>(a.a0 + gr * kMlpIn0 + (e & 7) * 8));
      }
    };
    auto store_prefetched = [&](int x) {
      uint8_t* sAct = sAct0 + x * kTcSmemA;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int e = (warp - 8) * 128 + j * 32 + lane;
        *reinterpret_cast<uint4*>(sAct + sw128_offset(0, kTcRows, e >> 3, e & 7)) = pre[j];
      }
    };
    bool stop = false;
    if ((int64_t)blockIdx.x < npairs) {
      for (int x = 0; x < 2; ++x)
        if (tile_exists(blockIdx.x, x)) load_inputs(2 * (int64_t)blockIdx.x + x, x);
    }
    for (int64_t pi = blockIdx.x; pi < npairs && !stop; pi += gridDim.x) {
      int boff = 0;
      for (int l = 0; l < kMlpLayers && !stop; ++l) {
        const int N = a.out[l];
        for (int x = 0; x < 2 && !stop; ++x) {
          if (!tile_exists(pi, x)) continue;
          const int64_t npi = pi + gridDim.x;
          const bool next = l + 1 == kMlpLayers && npi < npairs && tile_exists(npi, x);
          if (l + 1 == kMlpLayers && warp >= 8) {
            // no accumulator columns here: move the slot's next inputs
            if (next) prefetch_inputs(2 * npi + x);
            const bool ok = __all_sync(0xffffffffu, mbar_wait_abort(&acc_b[x], nacc[x] & 1, abort));
            ++nacc[x];
            if (!ok) {
              *abort = 1;
              stop = true;
              break;
            }
            if (next) {
              store_prefetched(x);
              epi_warp_arrive(&act_b[x], lane);
            }
            continue;
          }
          const bool ok = __all_sync(0xffffffffu, mbar_wait_abort(&acc_b[x], nacc[x] & 1, abort));
          ++nacc[x];
          if (!ok) {
            *abort = 1;
            stop = true;
            break;
          }
          tc_fence_after();
          uint8_t* sAct = sAct0 + x * kTcSmemA;
          const int64_t grow = (2 * pi + x) * kTcRows + row;
          const bool valid = grow < M;
          const int cols = N / 4 >= 32 ? N / 4 : 32;
          const int cbeg = cg * cols;
          if (cbeg < N) {
            // 16-column pieces, double-buffered: the next piece's tensor-memory load is in flight
            // while this one is converted
            auto piece = [&](const uint32_t* raw, int c0) {
              const float4* b4 = reinterpret_cast<const float4*>(sBias + boff + c0);
              if (l + 1 < kMlpLayers) {
                __align__(16) __nv_bfloat162 h[8];
#pragma unroll
                for (int j = 0; j < 16; j += 4) {
                  const float4 hb = b4[j >> 2];
                  float z[4] = {__uint_as_float(raw[j]), __uint_as_float(raw[j + 1]), __uint_as_float(raw[j + 2]),
                                __uint_as_float(raw[j + 3])};
                  if (STORE && valid && a.z[l])
                    *reinterpret_cast<float4*>(a.z[l] + grow * N + c0 + j) =
                        make_float4(fmaf(hb.x, 2.0f, z[0]), fmaf(hb.y, 2.0f, z[1]), fmaf(hb.z, 2.0f, z[2]),
                                    fmaf(hb.w, 2.0f, z[3]));
                  const float h0 = fmaf(z[0], 0.5f, hb.x), h1 = fmaf(z[1], 0.5f, hb.y);
                  const float h2 = fmaf(z[2], 0.5f, hb.z), h3 = fmaf(z[3], 0.5f, hb.w);
                  h[j >> 1] = __floats2bfloat162_rn(fmaf(h0, tanh_approx(h0), h0), fmaf(h1, tanh_approx(h1), h1));
                  h[(j >> 1) + 1] = __floats2bfloat162_rn(fmaf(h2, tanh_approx(h2), h2), fmaf(h3, tanh_approx(h3), h3));
                }
                const int panel = c0 >> 6, chunk0 = (c0 & 63) >> 3;
#pragma unroll
                for (int u = 0; u < 2; ++u)
                  *reinterpret_cast<uint4*>(sAct + sw128_offset(panel, kTcRows, row, chunk0 + u)) =
                      reinterpret_cast<const uint4*>(h)[u];
                if (STORE && valid && a.act[l + 1]) {
                  __nv_bfloat16* ap = a.act[l + 1] + grow * N + c0;
#pragma unroll
                  for (int u = 0; u < 2; ++u) reinterpret_cast<uint4*>(ap)[u] = reinterpret_cast<const uint4*>(h)[u];
                }
              } else if (valid) {
                float v[16];
#pragma unroll
                for (int j = 0; j < 16; j += 4) {
                  const float4 bb = b4[j >> 2];
                  v[j] = __uint_as_float(raw[j]) + bb.x;
                  v[j + 1] = __uint_as_float(raw[j + 1]) + bb.y;
                  v[j + 2] = __uint_as_float(raw[j + 2]) + bb.z;
                  v[j + 3] = __uint_as_float(raw[j + 3]) + bb.w;
                }
                float* yp = a.y + grow * kMlpPad + c0;
#pragma unroll
                for (int j = 0; j < 16; j += 4)
                  *reinterpret_cast<float4*>(yp + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
                if (STORE && a.z[l]) {
                  float* zp = a.z[l] + grow * N + c0;
#pragma unroll
                  for (int j = 0; j < 16; j += 4)
                    *reinterpret_cast<float4*>(zp + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
                }
              }
            };
            const int npc = cols / 16;   // 4 (hidden layers) or 2 (last layer): even
            const uint32_t tb = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(x * 256 + cbeg);
            uint32_t r0[16], r1[16];
            tmem_ld16_nowait(tb, r0);
            tmem_wait_ld16(r0);
            for (int pc = 0; pc < npc; pc += 2) {
              tmem_ld16_nowait(tb + 16u * (pc + 1), r1);
              piece(r0, cbeg + 16 * pc);
              tmem_wait_ld16(r1);
              if (pc + 2 < npc) tmem_ld16_nowait(tb + 16u * (pc + 2), r0);
              piece(r1, cbeg + 16 * (pc + 1));
              if (pc + 2 < npc) tmem_wait_ld16(r0);
            }
          }
          // this warp's part of the accumulator has been read and (below the last layer) its columns
          // of the next operand written
          if (l + 1 < kMlpLayers) {
            epi_warp_arrive(&act_b[x], lane);
          } else if (next) {
            // the slot's last MMAs have completed; the next tile's MMAs also wait for this warp's
            // tensor-memory reads of this layer
            epi_warp_arrive(&act_b[x], lane);
          }
        }
        boff += N;
      }
    }
  }
  __syncthreads();
  if (tid == 0 && *abort) atomicOr(a.err, 1);
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
}

// Weight image of one layer: W^T [N][Kin] BF16 (row-major) -> swizzled K-major panels of 64
// (Kin < 64 is zero-padded inside its panel).
static __global__ void weight_image_kernel(const __nv_bfloat16* wt, int N, int Kin, uint8_t* img) {
  const int panels = (Kin + 63) / 64;
  const int64_t total = (int64_t)panels * N * 8;   // 16-byte chunks
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= total) return;
  const int chunk = (int)(e % 8);
  const int n = (int)((e / 8) % N);
  const int p = (int)(e / (8 * (int64_t)N));
  __align__(16) __nv_bfloat16 h[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int k = p * 64 + chunk * 8 + j;
    h[j] = k < Kin ? wt[(int64_t)n * Kin + k] : __float2bfloat16(0.f);
  }
  *reinterpret_cast<uint4*>(img + sw128_offset(p, N, n, chunk)) = *reinterpret_cast<const uint4*>(h);
}

inline uint32_t weight_image_bytes(int N, int Kin) { return (uint32_t)((Kin + 63) / 64) * N * 128u; }

}  // namespace tc

namespace tc {

// ---- generic NT GEMM on the tensor cores (the training pass) -------------------------------
//
// C[M][N] (FP32, row stride ldc) = A[M][K] . B[N][K]^T, A and B BF16 with K contiguous (row
// strides lda, ldb in elements, multiples of 8), K a multiple of 8.  One CTA (128 threads) per
// 128 x n_tile output tile (n_tile in {32, 64, 128, 256}); K in panels of 64 staged in shared
// memory (128-byte swizzle, as above) through a two-stage cp.async pipeline, one elected thread
// issuing the MMAs of a panel and committing them to that stage's mbarrier, which releases the
// stage for the panel after next.  Rows, columns and K beyond the matrix are zero-filled.  With
// blockIdx.z > 0 the CTA takes the z-th slice of K (kchunk, a multiple of 64) and writes its
// partial product to C + z * split_stride.

constexpr int kGemmThreads = 128;
constexpr long long kGemmWaitLimit = 1ll << 24;

struct GemmNTArgs {
  int M, N, K, n_tile, kchunk;
  const __nv_bfloat16* A;
  int64_t lda;
  const __nv_bfloat16* B;
  int64_t ldb;
  float* C;
  int64_t ldc, split_stride;
  int* err;
};

__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_addr(dst)), "l"(src),
               "r"(valid ? 16 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__device__ __forceinline__ bool mbar_wait_limit(uint64_t* bar, uint32_t parity, long long limit) {
  for (long long it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Stage one 64-wide K panel (rows [r0, r0 + rows) of X, K range [k0, k0 + 64)) into a swizzled
// operand of `rows` rows; entries outside rows_max x k_end are zero.
__device__ __forceinline__ void stage_panel(uint8_t* dst, const __nv_bfloat16* X, int64_t ld, int r0, int rows,
                                            int rows_max, int k0, int k_end) {
  for (int e = threadIdx.x; e < rows * 8; e += kGemmThreads) {
    const int r = e >> 3, c = e & 7;
    const int gr = r0 + r, gk = k0 + 8 * c;
    const bool ok = gr < rows_max && gk < k_end;
    const __nv_bfloat16* src = ok ? X + (int64_t)gr * ld + gk : X;
    cp_async16(dst + sw128_offset(0, rows, r, c), src, ok);
  }
}

__global__ void __launch_bounds__(kGemmThreads, 1) gemm_nt_kernel(const GemmNTArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int nt = a.n_tile;
  const uint32_t a_bytes = 128u * 128u, b_bytes = (uint32_t)nt * 128u;
  const uint32_t stage_bytes = a_bytes + b_bytes;   // stage s: A at s * stage_bytes, B after it
  __shared__ uint64_t bar[2];
  __shared__ uint32_t s_tmem;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * 128, n0 = blockIdx.x * nt;
  const int kb = blockIdx.z * a.kchunk, ke = min(a.K, kb + a.kchunk);
  const int np = (ke - kb + 63) / 64;
  float* C = a.C + (int64_t)blockIdx.z * a.split_stride;
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&s_tmem)),
                 "r"(nt)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  const uint32_t idesc = umma_idesc_bf16(128, nt);
  bool bad = false, any_bad = false;
  uint32_t committed = 0;   // panels whose MMAs thread 0 has committed
  uint32_t waited0 = 0, waited1 = 0;   // completed phases waited for, per stage
  stage_panel(smem, a.A, a.lda, m0, 128, a.M, kb, ke);
  stage_panel(smem + a_bytes, a.B, a.ldb, n0, nt, a.N, kb, ke);
  cp_async_commit();
  for (int p = 0; p < np; ++p) {
    const int s = p & 1;
    if (p + 1 < np) {
      const int s1 = (p + 1) & 1;
      // the stage of panel p+1 held panel p-1: its MMAs must have finished reading it
      if (p >= 1) {
        uint32_t& w = s1 ? waited1 : waited0;
        if (!mbar_wait_limit(&bar[s1], w & 1u, kGemmWaitLimit)) bad = true;
        ++w;
      }
      if (!bad) {
        uint8_t* st = smem + s1 * stage_bytes;
        stage_panel(st, a.A, a.lda, m0, 128, a.M, kb + 64 * (p + 1), ke);
        stage_panel(st + a_bytes, a.B, a.ldb, n0, nt, a.N, kb + 64 * (p + 1), ke);
      }
      cp_async_commit();
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    fence_proxy_async_smem();
    any_bad = __syncthreads_or(bad);
    if (any_bad) break;
    tc_fence_after();
    if (tid == 0) {
      const uint32_t sa = smem_addr(smem + s * stage_bytes);
      for (int ks = 0; ks < 4; ++ks) {
        const uint64_t ad = umma_desc_sw128(sa + 32u * ks);
        const uint64_t bd = umma_desc_sw128(sa + a_bytes + 32u * ks);
        umma_bf16(tmem, ad, bd, idesc, (p > 0 || ks > 0) ? 1u : 0u);
      }
      umma_commit(&bar[s]);
      committed++;
    }
  }
  cp_async_wait<0>();
  // every committed MMA group must complete before the accumulator is read or freed
  if (tid == 0) {
    for (uint32_t p = 0; p < committed; ++p) {
      const int s = p & 1;
      if ((p >> 1) < (s ? waited1 : waited0)) continue;   // already waited for
      if (!mbar_wait_limit(&bar[s], (p >> 1) & 1u, kGemmWaitLimit)) bad = true;
    }
  }
  any_bad = __syncthreads_or(bad) || any_bad;
  tc_fence_after();
  if (!any_bad && np > 0) {
    const int row = m0 + 32 * warp + lane;
    for (int c0 = 0; c0 < nt; c0 += 32) {
      uint32_t r[32];
      tmem_ld32_nowait(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, r);
      tmem_wait_ld();
      if (row < a.M) {
        float* cp = C + (int64_t)row * a.ldc + n0 + c0;
        const int lim = min(32, a.N - (n0 + c0));
        if (lim == 32 && (((uintptr_t)cp) & 15) == 0) {
#pragma unroll
          for (int j = 0; j < 32; j += 4)
            *reinterpret_cast<float4*>(cp + j) = make_float4(__uint_as_float(r[j]), __uint_as_float(r[j + 1]),
                                                             __uint_as_float(r[j + 2]), __uint_as_float(r[j + 3]));
        } else {
#pragma unroll
          for (int j = 0; j < 32; ++j)
            if (j < lim) cp[j] = __uint_as_float(r[j]);
        }
      }
    }
  } else if (np == 0 && a.N > n0) {
    // an empty K slice contributes zeros
    const int row = m0 + 32 * warp + lane;
    if (row < a.M)
      for (int j = 0; j < nt && n0 + j < a.N; ++j) C[(int64_t)row * a.ldc + n0 + j] = 0.f;
  }
  if (any_bad && tid == 0) atomicOr(a.err, 1);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(nt) : "memory");
}

inline uint32_t gemm_nt_smem_bytes(int n_tile) { return 2u * (128u * 128u + (uint32_t)n_tile * 128u) + 1024u; }

}  // namespace tc
