/*
 * tc.h - C ABI of the B300 monodomain hot path (TorchCor, arXiv 2510.12011).
 *
 * The library advances the operator-split monodomain P1-FEM scheme of Section 2.2:
 *   per step k -> k+1
 *     (a1) ionic update u^{k+1} = f(V^k, u^k), I_ion(V^k, u^{k+1})            Eq. 2, row 1
 *     (a2) b = chi M (Cm V^k - dt I_ion + dt I_stim) - (1 - theta) dt K V^k     after Eq. 3
 *     (a3,a4) Jacobi-PCG solve of (chi Cm M + theta dt K) V^{k+1} = b           Algorithm 1
 *          from the extrapolated guess 2 V^k - V^{k-1}                         end of Sec. 2.2
 *     (a5) activation time: first upward crossing of a threshold (LAT)         Section 2.1
 * on one GPU with hand-written sm_103a kernels.  Units follow Table 1: mm, ms, mV,
 * uA/mm^2 (currents), uF/mm^2 (Cm), 1/mm (chi), S/m (conductivities); with these units the
 * diffusion term needs no conversion factor.
 *
 * Conventions for every call
 *   - Every call returns tc_status; TC_OK is 0, errors are negative.  On error,
 *     tc_last_error() returns a message for the calling thread; no call aborts the process.
 *   - Input arrays are host pointers unless a name says "dev"; they are copied before the
 *     call returns, and the caller keeps ownership of them.
 *   - Handles are owned by the library and released only by *_destroy; destroying NULL is
 *     a no-op.  A handle may be used by one thread at a time.
 *   - Node numbering in and out of the library is the caller's.  The library reorders nodes
 *     internally (reverse Cuthill-McKee, then SELL-C-sigma row sorting, Section 2.2: "RCM")
 *     and undoes the order on every read.
 */
#ifndef TC_H
#define TC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TC_OK = 0,
  TC_ERR_ARG = -1,      /* null pointer, size out of range, bad enum value            */
  TC_ERR_MESH = -2,     /* degenerate tetrahedron, node index out of range             */
  TC_ERR_STATE = -3,    /* call made in the wrong order / on a mismatched object       */
  TC_ERR_CUDA = -4,     /* a CUDA runtime call failed (message has the CUDA error)     */
  TC_ERR_NOMEM = -5,    /* host or device allocation failed                            */
  TC_ERR_TIMEOUT = -6,  /* a device-side wait hit its iteration limit                  */
  TC_ERR_NAN = -7       /* a non-finite value appeared in the solver                   */
} tc_status;

typedef enum { TC_MODEL_MS = 0, TC_MODEL_TP06 = 1 } tc_model;
typedef enum { TC_FP64 = 0, TC_FP32 = 1 } tc_precision;
typedef enum { TC_OP_M = 0, TC_OP_K = 1, TC_OP_A = 2 } tc_operator;
/* Fields for tc_read_state / tc_write_state.  TC_FIELD_STATE + j is ionic state j. */
typedef enum { TC_FIELD_V = 0, TC_FIELD_V_PREV = 1, TC_FIELD_STATE = 16 } tc_field;

typedef struct tc_mesh tc_mesh;
typedef struct tc_sim tc_sim;

/* Statistics of one tc_step call (filled when the pointer is not NULL). */
typedef struct {
  int64_t steps;          /* time steps made by this call                               */
  int64_t step_index;     /* index k of the next step after the call                    */
  int64_t cg_iterations;  /* A-products made inside the PCG loops, summed over the steps  */
  int32_t max_iterations; /* largest PCG iteration count of one step                    */
  int32_t not_converged;  /* steps whose PCG stopped at max_iter (Algorithm 1 just stops) */
  double last_znorm;      /* ||z|| when the last step's PCG stopped                      */
  double last_z0norm;     /* ||z_0|| of the last step's PCG                              */
  int64_t graph_steps;    /* steps of this call replayed from captured CUDA graphs       */
} tc_step_stats;

/* Accumulated device time per kernel while profiling is on (tc_set_profiling). */
typedef struct {
  double ionic_ms;        int64_t ionic_launches;
  double pcg_ms;          int64_t pcg_launches;
  int64_t pcg_iterations; /* iterations inside the profiled PCG launches                */
  double surrogate_ms;    int64_t surrogate_windows;   /* learned-surrogate inference (features,
                                                          network, check), one per window     */
  double mlp_ms;          /* of which the network's fused tensor-core forward pass          */
  int64_t surrogate_rows; /* node rows the network evaluated (the candidates of each window) */
} tc_profile;

/* ---- mesh ------------------------------------------------------------------------- */

/* tc_mesh_create: copy a tetrahedral mesh (Section 2.1: points, connectivity, fibres).
 *   xyz     [n_nodes][3] node coordinates in mm
 *   tets    [n_tets][4]  0-based node indices; either orientation is accepted
 *   fibres  [n_tets][3]  fibre direction per element (normalised here), or NULL for (1,0,0)
 *   region  [n_tets]     region id per element in [0, n_regions), or NULL for all 0
 * Errors: TC_ERR_ARG (null/size), TC_ERR_MESH (index out of range, zero-length fibre,
 * |det J| <= 1e-12 * (longest edge)^3, i.e. a degenerate element). */
tc_status tc_mesh_create(const double* xyz, int64_t n_nodes, const int32_t* tets, int64_t n_tets,
                         const double* fibres, const int32_t* region, tc_mesh** out);
/* tc_mesh_destroy: release a mesh (simulations assembled from it stay valid: they hold their own
 * copies).  NULL is a no-op. */
void tc_mesh_destroy(tc_mesh* mesh);

/* Number of stored entries of M, K and A (one shared pattern: every node pair of an element). */
tc_status tc_mesh_nnz(const tc_mesh* mesh, int64_t* nnz);

/* tc_mesh_matrices: host-side P1 assembly, returned in the caller's node order as CSR with
 * sorted column indices (Section 2.2: "M and K ... are sparse").  Per element:
 *   M_e[i][j] = vol (1 + delta_ij) / 20,  K_e[i][j] = vol grad(l_i)^T sigma_e grad(l_j),
 *   sigma_e = sigma_t I + (sigma_l - sigma_t) f f^T  (Section 2.1, conductivity from fibres).
 * sigma_l, sigma_t: [n_regions] conductivities in S/m.  Outputs (caller-allocated):
 * row_ptr [n+1], col [nnz], m_val [nnz], k_val [nnz]; any of the four may be NULL.
 * Runs on the host only; needs no GPU. */
tc_status tc_mesh_matrices(const tc_mesh* mesh, const double* sigma_l, const double* sigma_t,
                           int32_t n_regions, int64_t* row_ptr, int32_t* col, double* m_val,
                           double* k_val);

/* tc_monodomain_conductivity: per region, the monodomain conductivity of each direction from the
 * intracellular (il, it) and extracellular (el, et) ones of the bidomain description used to set
 * regions up (Listing 1 of the paper): sigma = sigma_i sigma_e / (sigma_i + sigma_e), the
 * harmonic combination, for the longitudinal and the transverse direction.  Host arrays of
 * n_regions entries (S/m); every input must be > 0 (TC_ERR_ARG otherwise).  No GPU needed. */
tc_status tc_monodomain_conductivity(const double* il, const double* it, const double* el, const double* et,
                                     int32_t n_regions, double* sigma_l, double* sigma_t);

/* tc_mesh_layout_size: number of connected components of the mesh and the internal row count
 * of the device layout (every component padded to a multiple of 32 rows).  Host only.
 * Each connected component is an independent problem: the PCG runs per component (its own
 * alpha, beta and stopping test), which is how many meshes are batched into one simulation. */
tc_status tc_mesh_layout_size(const tc_mesh* mesh, int32_t* n_components, int64_t* n_internal);

/* tc_mesh_set_sell_sigma: the SELL-C-32 row-sorting window (rows sorted by length inside windows
 * of sell_sigma rows of the RCM order, never across components) of simulations assembled from this
 * mesh afterwards; default 1024.  sell_sigma >= 1. */
tc_status tc_mesh_set_sell_sigma(tc_mesh* mesh, int32_t sell_sigma);

/* tc_mesh_ordering: the internal node order the device path uses (host only).
 * perm[k] = caller index of the k-th real row (n_nodes entries, dummy rows left out);
 * slice_width (if not NULL) receives n_internal/32 SELL slice widths. */
tc_status tc_mesh_ordering(const tc_mesh* mesh, int32_t sell_sigma, int32_t* perm,
                           int32_t* slice_width);

/* ---- simulation ------------------------------------------------------------------- */

/* tc_assemble: assemble M, K and A = chi Cm M + theta dt K (Eq. 3), build the Jacobi
 * preconditioner diag(A) (Section 2.2), reorder and upload everything to the current CUDA
 * device, and allocate the state.  The simulation starts at step 0 with the ionic model's
 * resting state (set by tc_set_ionic) and V^{-1} = V^0.
 *   sigma_l, sigma_t [n_regions] S/m; chi 1/mm; cm uF/mm^2; theta in [0,1]; dt ms > 0
 *   precision: TC_FP64 (all arithmetic in double) or TC_FP32 (matrix/ionic in float, PCG
 *   dot products and alpha/beta recurrences in double)
 *   cuda_stream: a cudaStream_t to run on, or NULL for the legacy default stream.
 * Errors: TC_ERR_ARG, TC_ERR_MESH, TC_ERR_CUDA, TC_ERR_NOMEM. */
tc_status tc_assemble(const tc_mesh* mesh, const double* sigma_l, const double* sigma_t,
                      int32_t n_regions, double chi, double cm, double theta, double dt,
                      int32_t precision, void* cuda_stream, tc_sim** out);
/* tc_sim_destroy: release the simulation's device and host memory (after waiting for its stream);
 * the mesh it was assembled from is not touched.  NULL is a no-op. */
void tc_sim_destroy(tc_sim* sim);

tc_status tc_sim_size(const tc_sim* sim, int64_t* n_nodes, int64_t* nnz, int64_t* padded_nnz,
                      int32_t* n_blocks);

/* tc_sim_layout: connected components (independent problems solved side by side), internal
 * row count of the device layout, and the PCG launch shape in use.  Any pointer may be NULL. */
tc_status tc_sim_layout(const tc_sim* sim, int32_t* n_components, int64_t* n_internal,
                        int32_t* pcg_threads, int32_t* blocks_per_sm);

/* tc_sim_staging: how the PCG launch gathers the vector of its A-products (Algorithm 1's q = A p).
 * Each block of the cooperative launch owns a contiguous range of SELL slices; under the RCM
 * order the columns those rows touch form a band (the block's window).  When the window fits the
 * shared memory left per block at the launch shape, the block copies it into shared memory after
 * each grid barrier and its gathers read shared memory; otherwise they read global memory.  The
 * results are bitwise the same either way.  When every block's columns span fewer than 65,536
 * entries, the column indices of the RHS pass and the A-products are also read as 16-bit offsets
 * from the block's window start (half the index stream; again bitwise the same results).  Reports
 * the number of blocks, how many stage their window, the largest window (entries), the launch's
 * dynamic shared memory (bytes) and whether the 16-bit offsets are in use; any pointer may be
 * NULL.  Staging is off unless the environment variable TC_PCG_STAGE=1 (read at tc_assemble) asks
 * for it or tc_autotune picks it (measured on B300 it pays only where the windows are small next
 * to a block's rows: the gathers mostly hit L1 otherwise); TC_PCG_IDX16=0 turns the offsets off. */
tc_status tc_sim_staging(const tc_sim* sim, int32_t* blocks, int32_t* staged_blocks, int32_t* max_window,
                         int64_t* smem_bytes, int32_t* idx16);

/* tc_set_launch: PCG launch shape (512 or 1024 threads per block, blocks per SM, capped by the
 * occupancy of the cooperative launch).  Errors: TC_ERR_ARG (shape or too many components). */
tc_status tc_set_launch(tc_sim* sim, int32_t pcg_threads, int32_t blocks_per_sm);

/* tc_autotune: time trial_steps steps with every candidate launch shape (1024x1, 512x1, 512x2),
 * each with and without the PCG's shared-memory windows (tc_sim_staging), restoring the state
 * after each trial, and keep the fastest.  Reports the launch shape and its time per step (any
 * pointer may be NULL; the staging choice through tc_sim_staging).  The state and step index are
 * unchanged on return. */
tc_status tc_autotune(tc_sim* sim, int32_t trial_steps, int32_t* pcg_threads,
                      int32_t* blocks_per_sm, double* best_ms_per_step);

/* tc_set_graphs: when on (default), tc_step runs whole groups of 30 steps by replaying a CUDA
 * graph of the step loop (captured on first use, one per buffer phase; the step index lives on
 * the device).  Off: every step is launched from the host.  Per-launch profiling always launches
 * from the host. */
tc_status tc_set_graphs(tc_sim* sim, int32_t on);

/* tc_set_ionic: choose the ionic model and reset the state to init_state (NULL = the model's
 * resting state; otherwise [n_states][n_nodes] in caller order, V excluded).
 * TC_MODEL_MS (Mitchell-Schaeffer in mV; 1 state h): params = {tau_in, tau_out, tau_open,
 *   tau_close, v_gate, v_min, v_max} (ms, ms, ms, ms, -, mV, mV); n_params = 7.
 *   v = (V - v_min)/(v_max - v_min); I_ion = -Cm (v_max - v_min)(h v^2 (1-v)/tau_in - v/tau_out);
 *   gate by Rush-Larsen: v < v_gate -> (h_inf, tau) = (1, tau_open), else (0, tau_close).
 * TC_MODEL_TP06 (ten Tusscher-Panfilov 2006; 18 states): params = {cell type} with
 *   0 = endo, 1 = mid-myocardial, 2 = epi; n_params = 1.
 * Sets V^0 = V^{-1} = the model's resting potential, resets activation times and the step
 * index to 0.  Must be called before tc_step.  Errors: TC_ERR_ARG, TC_ERR_CUDA. */
tc_status tc_set_ionic(tc_sim* sim, int32_t model, const double* params, int32_t n_params,
                       const double* init_state);

/* tc_add_stimulus: any number of stimuli (Section 2.1).  The nodes receive I_stim += intensity
 * (uA/mm^2) during steps k with k0 <= k < k0 + nk, k0 = round(start/dt), nk = round(duration/dt)
 * (round half to even); I_stim enters b as chi M dt I_stim.  Errors: TC_ERR_ARG (index range). */
tc_status tc_add_stimulus(tc_sim* sim, const int32_t* nodes, int64_t n, double start_ms,
                          double duration_ms, double intensity);

/* tc_set_solver: PCG tolerances (Algorithm 1): stop when ||z|| < atol or ||z||/||z_0|| < rtol,
 * z = D^{-1} r, 2-norms; at most max_iter iterations (reaching it is not an error). */
tc_status tc_set_solver(tc_sim* sim, double atol, double rtol, int32_t max_iter);

/* tc_set_activation_threshold: threshold (mV) of the activation-time capture; default 0 mV
 * (LAT: "first becomes positive").  Only before the first step. */
tc_status tc_set_activation_threshold(tc_sim* sim, double v_threshold);

/* tc_step: advance n_steps >= 0 time steps on the simulation's stream and wait for them.
 * One step k -> k+1 is the operator-split scheme of Section 2.2:
 *   the ionic update u^{k+1} = f(V^k, u^k) and I_ion(V^k, u^{k+1})       (Eq. 2, first row),
 *   b = chi M (Cm V^k - dt I_ion + dt I_stim) - (1 - theta) dt K V^k      (definition after Eq. 3),
 *   A V^{k+1} = b, A = chi Cm M + theta dt K, solved by Jacobi-PCG           (Eq. 3, Algorithm 1)
 *     from the extrapolated guess 2 V^k - V^{k-1}                          (end of Section 2.2),
 *   then the activation (LAT) and repolarisation (LRT) capture             (Section 2.1).
 * Errors: TC_ERR_STATE (no ionic model), TC_ERR_TIMEOUT (a device wait hit its limit; the
 * state is then undefined), TC_ERR_NAN, TC_ERR_CUDA. */
tc_status tc_step(tc_sim* sim, int64_t n_steps, tc_step_stats* stats);

/* tc_read_state / tc_write_state: the solution output of Section 2.1 (the transmembrane
 * potential written every plot interval) and its inverse, for checkpoint/restart.  Copy one field
 * to/from a host array of n = n_nodes doubles in caller node order (TC_FIELD_V = V^k,
 * TC_FIELD_V_PREV = V^{k-1}, the second history level of the extrapolated guess at the end of
 * Section 2.2; TC_FIELD_STATE + j = ionic state j of Eq. 2's u).  Errors: TC_ERR_ARG (null
 * pointer, n != n_nodes, unknown field), TC_ERR_CUDA.  tc_write_state returns nodes held by the
 * learned surrogate to the exact model. */
tc_status tc_read_state(const tc_sim* sim, int32_t field, double* host_dst, int64_t n);
tc_status tc_write_state(tc_sim* sim, int32_t field, const double* host_src, int64_t n);

/* tc_activation_times: the local activation times (LAT) of Section 2.1 - per node, the first
 * time (ms) V crossed v_threshold upwards (0 mV by default: "first becomes positive"), linearly
 * interpolated within the step; 0 if V^0 >= threshold; -1 if never.  host_dst: n = n_nodes
 * doubles, caller order.  v_threshold must equal the capture threshold (TC_ERR_STATE
 * otherwise); TC_ERR_ARG on a null pointer or n != n_nodes. */
tc_status tc_activation_times(const tc_sim* sim, double v_threshold, double* host_dst, int64_t n);

/* Repolarisation (Section 2.1, LRT: V returns below -70 mV with a negative time derivative).
 * tc_set_repolarisation_threshold: the LRT threshold (default -70 mV); only before stepping.
 * tc_repolarisation_times: per node, the first downward crossing of that threshold after
 *   activation, linearly interpolated within the step; -1 if none yet.
 * tc_apd90: per node, APD90 = t90 - activation time, where t90 is the first downward crossing
 *   of V_rest + 0.1 (V_peak - V_rest) after activation (V_peak: maximum of V since activation,
 *   V_rest: the model's resting potential set by tc_set_ionic); -1 where undefined.
 * Arrays: host, [n_nodes], caller order. */
tc_status tc_set_repolarisation_threshold(tc_sim* sim, double v_threshold);
tc_status tc_repolarisation_times(const tc_sim* sim, double* host_dst, int64_t n);
tc_status tc_apd90(const tc_sim* sim, double* host_dst, int64_t n);

/* tc_get_step_index / tc_set_step_index: the step counter k (for checkpoint/restart). */
tc_status tc_get_step_index(const tc_sim* sim, int64_t* k);
tc_status tc_set_step_index(tc_sim* sim, int64_t k);

/* tc_apply_operator: y = Op x with Op in {M, K, A} using the device SELL-C-sigma kernel
 * (the SpMV of Algorithm 1).  x, y: host arrays [n_nodes] in caller order. */
tc_status tc_apply_operator(tc_sim* sim, int32_t op, const double* x, double* y, int64_t n);

/* tc_apply_operator_dev: the same on device arrays in the INTERNAL node order (no copies,
 * asynchronous on the simulation's stream).  x_dev, y_dev: n_nodes doubles (TC_FP64) or
 * floats (TC_FP32), 16-byte aligned. */
tc_status tc_apply_operator_dev(tc_sim* sim, int32_t op, const void* x_dev, void* y_dev);

/* tc_apply_operator_static: the same result as tc_apply_operator, for callers that must not
 * allocate device memory while they run (a process whose device memory is reserved by another
 * allocator, so cudaMalloc would fail, or a caller that cannot afford the device-wide
 * synchronisation cudaFree implies).  The paper has no counterpart; it is a library facility.
 * TC_FP64 simulations only (others get TC_ERR_ARG).  x and y are host arrays [n_nodes] in caller
 * order (n != n_nodes gives TC_ERR_ARG).  Device staging for x and y is a static 4 MiB array
 * inside the library (2 x 262,144 doubles) that every GPU loading the library holds until the
 * process exits; a simulation whose padded device layout has more than 262,144 rows (each
 * connected component is padded to a multiple of 32 rows, so up to 31 more rows than nodes per
 * component) is rejected with TC_ERR_ARG.  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress) and keeps it for the life of the device's primary
 * context (a cudaDeviceReset between calls is not supported); make that first call before any
 * stream capture.  All calls share the array: calls that overlap on the GPU (e.g. from two
 * threads or two streams) race.  Allocates nothing; waits for the simulation's stream before and
 * after the copy. */
tc_status tc_apply_operator_static(tc_sim* sim, int32_t op, const double* x, double* y, int64_t n);

/* Profiling: when on, tc_step records CUDA events around every launch on the simulation's
 * stream and accumulates their durations; tc_get_profile reads and tc_reset_profile clears. */
tc_status tc_set_profiling(tc_sim* sim, int32_t on);
tc_status tc_get_profile(const tc_sim* sim, tc_profile* out);
tc_status tc_reset_profile(tc_sim* sim);

/* tc_set_wait_limit: iteration limit of every device-side wait of the PCG kernel's grid
 * barrier (default 1<<26 polls).  A tiny limit makes the barrier give up and tc_step return
 * TC_ERR_TIMEOUT with the GPU context intact (used to test the timeout path). */
tc_status tc_set_wait_limit(tc_sim* sim, int64_t polls);

/* tc_selftest_exp: evaluate, on the current device, the FP64 exponential the ionic kernels use
 * (table-driven, Tang 1989) and the CUDA library exp at the host inputs x[n]; y_fast[n] and
 * y_ref[n] receive the two results (host arrays).  Diagnostics; allocates 24 n bytes. */
tc_status tc_selftest_exp(const double* x, double* y_fast, double* y_ref, int64_t n);
/* tc_selftest_log: the same for the FP64 natural logarithm of the ionic kernels (table-driven,
 * Tang 1990) against the CUDA library log. */
tc_status tc_selftest_log(const double* x, double* y_fast, double* y_ref, int64_t n);
/* tc_selftest_rcp: the same for the FP64 reciprocal of the ionic kernels (hardware estimate and
 * two Newton-Raphson steps) against the IEEE division 1.0 / x.  x finite, nonzero and normal. */
tc_status tc_selftest_rcp(const double* x, double* y_fast, double* y_ref, int64_t n);
/* tc_selftest_exp2: the same for the base-2 FP64 exponential of the ionic kernels (table-driven,
 * 2^y) against the CUDA library exp2. */
tc_status tc_selftest_exp2(const double* x, double* y_fast, double* y_ref, int64_t n);

/* tc_measure_fp64_rate: FP64 FMA instructions per second (thread level) that the current device
 * sustains in a probe kernel with eight independent FMA chains per thread at full occupancy; the
 * measured ceiling of kernels bound by B300's FP64 pipe (the TP06 FP64 ionic update).  Allocates
 * a few KB of device memory; about 40 ms. */
tc_status tc_measure_fp64_rate(double* fma_per_s);

/* ---- learned ionic surrogate --------------------------------------------------------
 * A multilayer perceptron (20 -> 4 x 256 SiLU -> 19; BF16 weights and activations, FP32
 * accumulation, FP32 master weights) that maps a TP06 cell's (18 states, V, window-mean
 * stimulus current in pA/pF) to its 18 states and V after a window of ionic steps.  Inputs are
 * normalized as (x - in_mean)/in_scale; the network predicts the normalized change
 * ((y - x) - out_mean)/out_scale.  Forward passes run on the tensor cores (tcgen05, all layers
 * fused in one kernel); training runs that forward pass, a backward pass and Adam on the GPU.
 * Parameter vector: per layer W^T [out][in] (row-major, widths padded to 32/256) then the bias. */
typedef struct tc_mlp tc_mlp;
typedef struct { int32_t gemm; int64_t n_params; int64_t adam_steps; } tc_mlp_diag;

tc_status tc_mlp_create(uint64_t seed, tc_mlp** out);
void tc_mlp_destroy(tc_mlp* mlp);
tc_status tc_mlp_n_params(const tc_mlp* mlp, int64_t* n);
tc_status tc_mlp_get_params(const tc_mlp* mlp, float* host, int64_t n);
tc_status tc_mlp_set_params(tc_mlp* mlp, const float* host, int64_t n);
/* normalization: in_mean[20], in_scale[20], out_mean[19], out_scale[19] (n = 78) */
tc_status tc_mlp_set_normalization(tc_mlp* mlp, const float* host, int64_t n);
/* tc_mlp_fit_normalization: set the normalization from a device training set (x [n][20]
 * features, y [n][19] next states, FP32): means and standard deviations of the features and of
 * the changes y - x[:19]; a constant column gets scale 1.  tc_mlp_get_normalization copies the
 * current 78 values out. */
tc_status tc_mlp_fit_normalization(tc_mlp* mlp, const float* x_dev, const float* y_dev, int64_t n);
tc_status tc_mlp_get_normalization(const tc_mlp* mlp, float* host, int64_t n);
/* 0 = tensor cores (tcgen05, default), 1 = SIMT reference kernels */
tc_status tc_mlp_set_gemm(tc_mlp* mlp, int32_t impl);
/* forward pass of normalized inputs x [n][20] -> normalized outputs y [n][19] (host arrays) */
tc_status tc_mlp_forward(tc_mlp* mlp, const float* x, int64_t n, float* y);
/* mean squared error over the 19 outputs of normalized targets t [n][19], and its gradient
 * with respect to every parameter (host arrays), as one training step computes them */
tc_status tc_mlp_gradients(tc_mlp* mlp, const float* x, const float* t, int64_t n, float* grads, float* loss);
/* train on device arrays x [n][20] (raw features) and y [n][19] (raw next states): epochs of
 * shuffled mini-batches, Adam (beta 0.9/0.999); loss_history[epochs] receives the mean batch loss */
tc_status tc_mlp_train(tc_mlp* mlp, const float* x_dev, const float* y_dev, int64_t n, int32_t epochs,
                       int32_t batch, float lr, uint64_t seed, void* cuda_stream, float* loss_history);
tc_status tc_mlp_diagnostics(const tc_mlp* mlp, tc_mlp_diag* out);

/* tc_gemm_bf16_nt: c [M][N] (FP32) = a [M][K] . b [N][K]^T on the tensor cores (tcgen05), a and b
 * BF16 device arrays, row-major with K contiguous (K a multiple of 8); the GEMM the network's
 * training pass is built from (weight and input gradients), exposed for direct checks.
 * Synchronous on `cuda_stream`; TC_ERR_TIMEOUT if a device wait gave up. */
tc_status tc_gemm_bf16_nt(const void* a_dev, const void* b_dev, float* c_dev, int32_t M, int32_t N, int32_t K,
                          void* cuda_stream);

/* tc_tp06_window: the exact model over a window, for data generation and as the reference the
 * surrogate is measured against: from in [19][n] (18 states then V, device FP32) and a constant stimulus istim [n]
 * (pA/pF, or NULL), nsub split steps of the single cell (Eq. 2 with V advanced by forward Euler);
 * out [19][n].  precision TC_FP64 or TC_FP32 arithmetic. */
tc_status tc_tp06_window(const float* in_dev, const float* istim_dev, int64_t n, double dt, int32_t nsub,
                         int32_t cell, int32_t precision, float* out_dev, void* cuda_stream);

/* tc_set_surrogate: attach (mlp != NULL) or detach the surrogate to a TP06 simulation (TC_FP32 or
 * TC_FP64 tissue; the network itself computes in BF16 with FP32 accumulation).
 * Every `window` steps each node's surrogate prediction is checked (finite, concentrations > 0,
 * gates in [0,1] within 0.01, |V' - V| <= dv_max over the window, |dV/dt| <= dvdt_max on the
 * step before, no stimulus during the window, and - with dv_neighbour > 0 - no neighbour in the
 * node's matrix row differing from it by more than dv_neighbour mV, i.e. no activation or
 * repolarisation front next to it), and - with rest_band > 0 - V farther than rest_band mV from
 * the model's resting potential (a resting cell stays with the exact model: its slow drift and
 * tiny gate values are below the network's resolution); nodes that pass take the predicted
 * states at
 * once and use the window's effective ionic current I_stim - (V' - V)/(window dt) in every step
 * of the window; all other nodes take the exact model step by step.  The network is not owned; keep it alive.  While a
 * node is held by the network its states read back as the window's end values; tc_write_state,
 * tc_set_step_index and tc_set_ionic return every node to the exact model until the next window
 * boundary, and tc_set_ionic with a model other than TP06 detaches the surrogate. */
tc_status tc_set_surrogate(tc_sim* sim, tc_mlp* mlp, int32_t window, double dv_max, double dvdt_max,
                           double dv_neighbour, double rest_band);
/* tc_surrogate_sample: append training pairs drawn from the simulation's current state (TP06,
 * either precision) to device arrays x_dev [capacity][20] and y_dev [capacity][19].  For a
 * sampled node, x = (18 states, V, stimulus current averaged over the next `window` steps in
 * pA/pF) as FP32 and y = the exact single cell's 18 states and V after `window` steps from x,
 * computed in FP64.  A real node is sampled unless |V^k - V^{k-1}| > dvdt_keep dt (when
 * dvdt_keep > 0) or its exact window changes V by more than dv_keep mV (when dv_keep > 0); a
 * node within rest_band mV of the resting potential is kept only with probability rest_keep (a
 * counter-based draw from seed, the step index and the node).  Pairs are written in internal
 * node order from *count on; *count is advanced and stops at capacity. */
tc_status tc_surrogate_sample(tc_sim* sim, int32_t window, double rest_band, double rest_keep, double dv_keep,
                              double dvdt_keep, uint64_t seed, float* x_dev, float* y_dev, int64_t capacity,
                              int64_t* count);
/* node-windows handled by the surrogate and by the exact fallback since tc_set_surrogate */
tc_status tc_surrogate_usage(const tc_sim* sim, int64_t* surrogate_node_windows, int64_t* exact_node_windows);

/* Thread-local message of the last error ("" if none). */
const char* tc_last_error(void);
/* Library version string. */
const char* tc_version(void);

#ifdef __cplusplus
}
#endif
#endif /* TC_H */
