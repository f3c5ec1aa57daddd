// Internal interface between the simulation (sim.cu) and the learned surrogate (mlp.cu).
#pragma once

#include <cstdint>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "../../include/tc.h"
#include "kernels.cuh"

namespace tc {

// One window start of the surrogate inside a TP06 simulation (FP32 or FP64 tissue).
struct SurrogateStep {
  int64_t n;                    // internal rows
  int fp64;                     // element type of state, V, Vprev, dinv: double when set, else float
  void* state;                  // [18][n] TP06 states (written for nodes that pass the check)
  const void* V;                // V^k
  const void* Vprev;            // V^{k-1}
  const void* dinv;             // 0 on padding rows (neither flagged nor counted)
  double* log_cache;            // FP64 tissue: [4][n] held concentration logarithms (or null); a
                                // committed node's entry is marked stale (NaN in row 0)
  const int32_t* stim_off;
  const int32_t* stim_ids;
  const StimDev* stims;
  const long long* k_base;      // device step index of the launch group
  int k_off;                    // first step of the window = *k_base + k_off
  int win;                      // steps per window
  double cm, dt;
  float dv_max, dvdt_max;       // the check: |V' - V| over the window, |dV/dt| before it
  float dv_nbr;                 // and max |V_j - V_i| over the node's matrix row (0 = off)
  float v_rest, rest_band;      // and |V - v_rest| > rest_band (0 = off)
  const int32_t* slice_ptr;     // SELL-C-32 pattern of the system matrix
  const int32_t* col;
  __nv_bfloat16* a0;            // [n][64] scratch: compacted split-BF16 inputs of the candidates
  int32_t* idx;                 // [n] node of each compacted row
  int* count;                   // number of candidates (device)
  float* raw;                   // [20][n] scratch
  float* zout;                  // [n][32] scratch
  uint8_t* flag;                // [n] 1 = surrogate node for this window
  float* iion;                  // [n] effective ionic current over the window, pA/pF
  unsigned long long* counts;   // [2] surrogate / exact node-windows
  int* err;                     // tensor-core wait failures
  cudaEvent_t ev_mlp[2] = {nullptr, nullptr};   // recorded around the network when profiling
};

tc_status surrogate_infer(tc_mlp* m, const SurrogateStep& q, cudaStream_t st);

// Everything surrogate_infer needs that must not happen inside a stream capture (workspace
// allocation, kernel attributes), done ahead for n rows.
tc_status surrogate_prepare(tc_mlp* m, int64_t n);

}  // namespace tc
