// Learned ionic surrogate: a multilayer perceptron that maps a cell's state to its state a
// window of W ionic substeps later (BF16 weights and activations, FP32 accumulation).
//
// Layout: layer l computes Z_l = A_l W_l^T + b_l with A_l [rows][in_l] BF16 (row-major) and
// W_l^T [out_l][in_l] BF16 (row-major: every weight row is contiguous along the reduction
// index, which is what the tensor-core operands want); hidden layers apply SiLU,
// A_{l+1} = Z_l * sigmoid(Z_l), stored as BF16; the last layer is linear.  Widths are padded
// to multiples of 32 (20 inputs -> 32, 19 outputs -> 32) with zero weights.
//
// Split-BF16 input: a normalized feature x enters layer 0 as two BF16 numbers, hi = bf16(x) and
// lo = bf16(x - hi), in columns c and 32 + c of a 64-wide operand whose weight columns c and
// 32 + c are the same BF16 weight.  The tensor cores then see x to about 16 significant bits
// (one BF16 alone resolves a membrane potential only to about 0.3 mV, and a slowly moving
// input would repeat the same rounding error window after window).
#pragma once

#include <cstdint>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace tc {

constexpr int kMlpLayers = 5;     // 20 -> 256 -> 256 -> 256 -> 256 -> 19
constexpr int kMlpIn = 20;        // 18 states, V, window-mean stimulus current
constexpr int kMlpOut = 19;       // 18 states, V after the window
constexpr int kMlpHidden = 256;
constexpr int kMlpPad = 32;
constexpr int kMlpIn0 = 64;       // width of the layer-0 operand: hi in 0..31, lo in 32..63

struct MlpDims {
  int in[kMlpLayers];    // padded input width of every layer (parameter layout)
  int op_in[kMlpLayers]; // width of the BF16 operand the GEMM reads (kMlpIn0 for layer 0)
  int out[kMlpLayers];   // padded output width
  int64_t w_off[kMlpLayers], b_off[kMlpLayers];   // offsets into the parameter vector
  int64_t n_params;
};

inline MlpDims mlp_dims() {
  MlpDims d{};
  const int widths[kMlpLayers + 1] = {kMlpPad, kMlpHidden, kMlpHidden, kMlpHidden, kMlpHidden, kMlpPad};
  int64_t off = 0;
  for (int l = 0; l < kMlpLayers; ++l) {
    d.in[l] = widths[l];
    d.op_in[l] = l == 0 ? kMlpIn0 : widths[l];
    d.out[l] = widths[l + 1];
    d.w_off[l] = off;
    off += (int64_t)d.in[l] * d.out[l];
    d.b_off[l] = off;
    off += d.out[l];
  }
  d.n_params = off;
  return d;
}

// Which GEMM implementation the network uses (tensor cores, or the SIMT reference).
enum GemmImpl { kGemmTcgen05 = 0, kGemmSimt = 1 };

// The split-BF16 layer-0 operand of one normalized input row (xn[0..19]) -> a0[0..63].
__host__ __device__ inline void mlp_split_input(const float* xn, __nv_bfloat16* a0) {
  for (int c = 0; c < kMlpPad; ++c) {
    const float x = c < kMlpIn ? xn[c] : 0.f;
    const __nv_bfloat16 hi = __float2bfloat16(x);
    a0[c] = hi;
    a0[kMlpPad + c] = __float2bfloat16(x - __bfloat162float(hi));
  }
}

}  // namespace tc
