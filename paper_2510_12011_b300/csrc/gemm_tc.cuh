// Fused MLP forward on the 5th-generation tensor cores (tcgen05, sm_100-family).
//
// One CTA (256 threads) owns 128 rows at a time.  For each layer:
//   * the layer's weights W^T [N][K] arrive in shared memory as a pre-swizzled image through
//     bulk asynchronous copies (cp.async.bulk, completion counted on an mbarrier);
//   * thread 0 issues tcgen05.mma (kind::f16, BF16 x BF16 -> FP32) over K in steps of 16,
//     accumulating the 128 x N tile in tensor memory, and commits to a second mbarrier;
//   * eight warps read the accumulator back (tcgen05.ld), add the bias, apply SiLU and write
//     the BF16 result straight into the swizzled shared-memory operand of the next layer
//     (optionally also Z and the activation to global memory for the backward pass).
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

constexpr int kTcThreads = 256;
constexpr int kTcRows = 128;
constexpr uint32_t kTcSmemA = 4 * 128 * 128;            // 128 rows x 256 K, BF16
constexpr uint32_t kTcSmemW = 4 * 256 * 128;            // 256 rows x 256 K, BF16
constexpr uint32_t kTcSmemBytes = kTcSmemA + kTcSmemW + 1024;
constexpr long long kTcWaitLimit = 1ll << 24;

struct MlpFusedArgs {
  int64_t M;
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

// 32 consecutive FP32 columns of this thread's tensor-memory lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
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
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Byte offset of 16-byte chunk `chunk` (0..7 inside a 64-element K panel) of row r in a
// swizzled operand with `rows` rows per panel.
__host__ __device__ __forceinline__ uint32_t sw128_offset(int panel, int rows, int r, int chunk) {
  return (uint32_t)panel * rows * 128u + (uint32_t)(r >> 3) * 1024u + (uint32_t)(r & 7) * 128u +
         (uint32_t)((chunk ^ (r & 7)) * 16);
}

__device__ __forceinline__ float silu_fast(float z) { return __fdividef(z, 1.f + __expf(-z)); }

template <bool STORE>
__global__ void __launch_bounds__(kTcThreads, 1) mlp_fused_kernel(const MlpFusedArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;
  uint8_t* sW = smem + kTcSmemA;
  __shared__ uint64_t bar_w, bar_mma;
  __shared__ uint32_t s_tmem;
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    mbar_init(&bar_w, 1);
    mbar_init(&bar_mma, 1);
    s_fail = 0;
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
  uint32_t ph_w = 0, ph_m = 0;
  const int64_t ntiles = (a.M + kTcRows - 1) / kTcRows;
  const int q = warp & 3;        // tensor-memory lane quarter of this warp
  const int half = warp >> 2;    // column half handled by this warp
  const int row = 32 * q + lane;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t row0 = tile * kTcRows;
    // inputs: 128 rows x 64 BF16 (one 128-byte panel row each) into panel 0
    {
      const int r = tid >> 1, c0 = (tid & 1) * 4;
      const int64_t gr = row0 + r;
      for (int c = c0; c < c0 + 4; ++c) {
        uint4 v = make_uint4(0, 0, 0, 0);
        if (gr < a.M) v = *reinterpret_cast<const uint4*>(a.a0 + gr * kMlpIn0 + c * 8);
        *reinterpret_cast<uint4*>(sA + sw128_offset(0, kTcRows, r, c)) = v;
      }
    }
    fence_proxy_async_smem();
    for (int l = 0; l < kMlpLayers; ++l) {
      const int K = a.in[l], N = a.out[l];
      if (tid == 0) {
        mbar_expect_tx(&bar_w, a.img_bytes[l]);
        for (uint32_t off = 0; off < a.img_bytes[l]; off += 32768u) {
          const uint32_t nb = a.img_bytes[l] - off < 32768u ? a.img_bytes[l] - off : 32768u;
          bulk_copy_g2s(sW + off, a.img[l] + off, nb, &bar_w);
        }
      }
      if (!mbar_wait(&bar_w, ph_w)) atomicOr(&s_fail, 1);
      ph_w ^= 1u;
      __syncthreads();
      if (s_fail) break;
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
      }
      if (!mbar_wait(&bar_mma, ph_m)) atomicOr(&s_fail, 1);
      ph_m ^= 1u;
      tc_fence_after();
      __syncthreads();
      if (s_fail) break;
      // epilogue: warp (q, half) handles lanes 32q..32q+31 and columns [half*N/2, (half+1)*N/2)
      const int cols = N / 2 >= 32 ? N / 2 : 32;
      const int cbeg = half * cols;
      const int64_t grow = row0 + row;
      const bool valid = grow < a.M;
      if (cbeg < N) {
        for (int c0 = cbeg; c0 < cbeg + cols && c0 < N; c0 += 32) {
          float v[32];
          tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)c0, v);
          const float* b = a.bias[l] + c0;
#pragma unroll
          for (int j = 0; j < 32; ++j) v[j] += b[j];
          if (l + 1 < kMlpLayers) {
            if (STORE && valid && a.z[l]) {
              float* zp = a.z[l] + grow * N + c0;
#pragma unroll
              for (int j = 0; j < 32; j += 4) *reinterpret_cast<float4*>(zp + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
            }
            __align__(16) __nv_bfloat16 h[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) h[j] = __float2bfloat16(silu_fast(v[j]));
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
      fence_proxy_async_smem();
      tc_fence_before();
      __syncthreads();
    }
    if (s_fail) break;
  }
  __syncthreads();
  if (s_fail && tid == 0) atomicOr(a.err, 1);
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256) : "memory");
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
