#!/usr/bin/env python
"""Benchmark of the monodomain hot path: node-steps/s of the plain FP64 method on one B300,
with the FP32 precision form and the FP32 form with the learned ionic surrogate timed on the same
steps, and their errors against the FP64 result.

One step = ionic update + RHS + Jacobi-PCG solve + activation capture for every node of the
workload (one time step k -> k+1 of the operator-split scheme).  The default workload is the
40x16x6 mm slab at h = 0.2 mm (504,711 nodes, 2,880,000 tets) with the ten Tusscher-Panfilov
2006 epicardial model, dt = 0.02 ms.  Every form steps 40 ms from rest (the corner stimulus's wave
is then crossing the slab), W warm-up steps, then K timed steps.  A second leg runs the
2,136,691-node truncated ellipsoid for 300 ms in all three forms (FP64, FP32, FP32 + surrogate)
with activation-time and APD90 errors against the FP64 run.  The network also runs in FP64
tissue, on the same timed steps and from rest over the first 120 ms (what it gains at the same
precision).  Inputs are synthetic and seeded.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  With N > 1 (torchrun), every rank steps its own replica of
the workload (independent problems, no data-path collective: weak scaling).
"""
import argparse
import json
import os

# the CPU baseline reports one thread: keep BLAS single-threaded before numpy loads
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2510_12011_b300 import inputs as I  # noqa: E402

METRIC = ("node-steps/s (plain FP64 monodomain step: ionic + RHS + Jacobi-PCG + activation "
          "capture); FP32 precision form alongside")
# FP64 pipe work of one ionic_tp06_kernel<double> launch per node, from the ncu capture in
# profiles/ (sm__inst_executed_pipe_fp64 of peak x 2 per clock x 148 SMs x cycles / nodes); used to
# turn the live launch time into an achieved FP64 instruction rate.
TP06_FP64_INSTR_PER_NODE = 914.0
TP06_FP64_DRAM_BYTES_PER_LAUNCH = 142.57e6   # dram read + write of the same capture
# dram read + write of one pcg_step_kernel_1024<double> launch on the large slab (ncu capture in
# profiles/ of the autotuned launch - windows staged, 16-bit column offsets - near the end of the
# 40 ms pre-roll: 11 CG iterations)
PCG_FP64_DRAM_BYTES_PER_LAUNCH = 0.549e9
PCG_FP64_CAPTURE_ITERATIONS = 11.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["large_tp06", "large_ms", "small_ms", "ellipsoid_tp06"],
                    default="large_tp06")
    ap.add_argument("--no-fp32", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-surrogate", action="store_true")
    ap.add_argument("--no-prior-art", action="store_true",
                    help="skip the PyTorch version of the paper's own design (context line)")
    ap.add_argument("--no-surrogate-apd", action="store_true",
                    help="skip the surrogate's 400 ms APD90 check on the unseen slab")
    ap.add_argument("--fp64-beat-ms", type=float, default=120.0,
                    help="simulated ms of the FP64-tissue network run from rest against FP64 exact "
                         "(0 skips it)")
    ap.add_argument("--batched-steps", type=int, default=600)
    ap.add_argument("--e2e-steps", type=int, default=30)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-cpu-all-cores", action="store_true",
                    help="skip the oracle timed as independent processes on every host core")
    ap.add_argument("--preroll-ms", type=float, default=40.0,
                    help="simulated time stepped (untimed) before the warm-up and the timed steps, "
                         "so that the timed window sees a propagating wave rather than rest")
    ap.add_argument("--no-ellipsoid", action="store_true",
                    help="skip the ellipsoid leg (FP64, FP32 and FP32 + surrogate over 300 ms)")
    ap.add_argument("--ellipsoid-ms", type=float, default=300.0)
    return ap.parse_args()


def workload(name):
    if name == "large_tp06":
        return I.slab_large("tp06")
    if name == "ellipsoid_tp06":
        return I.ellipsoid_tp06()
    if name == "large_ms":
        return I.slab_large("ms")
    return I.slab_small_ms()


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6400.0), "measured"
    return 6400.0, "fallback"


# FP64 pipe of B300: 2 thread-level FP64 instructions (DFMA/DADD/DMUL) per clock per SM
# (ncu: sm__sass_thread_inst_executed_op_dfma_pred_on peak_sustained = 2 inst/cycle/SM).
SMS = 148


def fp64_instr_peak(sm_mhz):
    return 2.0 * SMS * (sm_mhz or 2032.0) * 1e6


# ---- algorithmic bytes (FP64 values, int32 indices; SELL padding not counted) -------------
def pcg_launch_bytes(n, nnz, nslices, iters, vb=8):
    """Bytes one PCG launch must move (vb = bytes per matrix value and node-vector entry: 8 for
    FP64, 4 for the FP32 form; indices int32; activation times FP64): RHS pass (M, K values,
    indices, g1/g2, dinv in; r, z out), per iteration the A-product (A values, indices, z gather;
    p, q out, and p, q in on all but the first iteration, where p = z and q = A z) and the vector
    phase (x, r r/w; p, q, dinv in; z out), and the activation capture (act, V^k, V^{k+1})."""
    rhs = (2 * vb + 4) * nnz + 4 * (nslices + 1) + 2 * vb * n + vb * n + 2 * vb * n
    spmv = (vb + 4) * nnz + 4 * (nslices + 1) + vb * n + 2 * vb * n
    vec = 8 * vb * n
    pq_in = 2 * vb * n
    cap = (8 + 2 * vb) * n
    return rhs + iters * (spmv + vec) + max(iters - 1.0, 0.0) * pq_in + cap


def pcg_launch_bytes_minimum(n, nnz, iters):
    """The minimum bytes of one FP64 PCG launch by the plan's count: the RHS pass 20 nnz + 4 (n + 1)
    + 24 n + 16 n, and per iteration the matrix 12 nnz + 4 n plus about 72 n of node vectors."""
    return 20 * nnz + 4 * (n + 1) + 40 * n + iters * (12 * nnz + 4 * n + 72 * n)


def pcg_fp64_ops(n, nnz, iters):
    """FP64 multiply-adds of one PCG launch by Algorithm 1's count (padding and reductions' own
    adds not counted): the RHS r0 = M g1 - K g2 (2 nnz), z0 = D^-1 r0, rho0, |z0| and the
    extrapolated guess (4 n); per iteration q = A p (nnz) and p.q, x += a p, r -= a q, z = D^-1 r,
    |z|, r.z, p = z + b p (7 n)."""
    return 2 * nnz + 4 * n + iters * (nnz + 7 * n)


def spmv_bytes(n, nnz, value_bytes=8):
    """CSR-equivalent algorithmic bytes of one y = A x: values + column indices + row pointers +
    x read once + y written once (value_bytes 8 for FP64, 4 for FP32)."""
    return (value_bytes + 4) * nnz + 4 * (n + 1) + 2 * value_bytes * n


def spmv_cold(sim, n, dtype, stream, torch, tc, reps=30):
    """Mean device time (ms) of one y = A x launch that starts with the matrix out of L2: `reps`
    pairs (a 512 MB read that evicts L2, then the SpMV) back to back between two events, minus
    `reps` of the read alone timed the same way; the median of three such differences.  One SpMV
    spans only about a dozen ticks of the event clock (about 2 us each), so single launches are
    not timed on their own.  Returns (ms, reps)."""
    dev = torch.device("cuda", torch.cuda.current_device())
    x = torch.randn(n, dtype=dtype, device=dev)
    y = torch.empty_like(x)
    flush = torch.ones(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def seq(with_spmv):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            flush.sum()   # reading 512 MB evicts the matrix without leaving dirty lines
            if with_spmv:
                sim.apply_dev(tc.TC_OP_A, x.data_ptr(), y.data_ptr())
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b)
    seq(True)
    diffs = sorted((seq(True) - seq(False)) / reps for _ in range(3))
    return float(diffs[1]), reps


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.15)
        self.proc.terminate()
        self.proc.wait()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) == 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[j] for r in rows for j in range(4) if r[5 + j] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def cpu_baseline(w, seconds):
    """Time the FP64 oracle, as it stands, on a bounded number of steps of the same workload."""
    from oracle.monodomain import Monodomain
    sim = Monodomain(w)        # assembly: not timed
    t0 = time.perf_counter()
    sim.step()
    first = time.perf_counter() - t0
    extra = max(0, int(seconds / max(first, 1e-6)) - 1)
    t0 = time.perf_counter()
    for _ in range(extra):
        sim.step()
    el = time.perf_counter() - t0
    steps, total = (extra, el) if extra > 0 else (1, first)
    model = None
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    return {"value": w.mesh.n_nodes * steps / total, "unit": "node-steps/s", "cores": 1,
            "host_cores": os.cpu_count(), "cpu_model": model, "kind": "oracle",
            "sample": f"{steps} time steps (steps 2..{steps + 1}) of {w.name}, "
                      f"{w.mesh.n_nodes} nodes, numpy/scipy FP64, 1 thread"}


def _oracle_process(name, seconds, barrier, queue):
    """One oracle process of the all-cores baseline: assemble (untimed), wait for the others, then
    step the workload for `seconds` and report (steps, elapsed)."""
    from oracle.monodomain import Monodomain
    w = workload(name)
    sim = Monodomain(w)
    sim.step()
    barrier.wait()
    t0 = time.perf_counter()
    steps = 0
    while time.perf_counter() - t0 < seconds:
        sim.step()
        steps += 1
    queue.put((steps, time.perf_counter() - t0, w.mesh.n_nodes))


def cpu_baseline_all_cores(name, seconds):
    """The oracle, as it stands, on every host core: one independent single-threaded process per
    core (capped by the memory each needs), each stepping its own copy of the workload over the
    same wall-clock window - the way independent cases share a CPU.  Throughput = the sum of the
    processes' node-steps/s.  Processes are spawned (not forked: the parent holds a CUDA context)."""
    import multiprocessing as mp
    need_gb = 3.0 if "large" in name or "slab40" in name or "ellipsoid" in name else 0.5
    avail_gb = None
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemAvailable"):
                avail_gb = int(line.split()[1]) / 1e6
    except OSError:
        pass
    cores = os.cpu_count() or 1
    procs_n = max(1, min(cores, int(avail_gb // need_gb) if avail_gb else cores))
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(procs_n)
    queue = ctx.Queue()
    procs = [ctx.Process(target=_oracle_process, args=(name, seconds, barrier, queue)) for _ in range(procs_n)]
    for p_ in procs:
        p_.start()
    res = [queue.get() for _ in procs]
    for p_ in procs:
        p_.join()
    value = sum(n * st / el for st, el, n in res)
    return {"value": value, "unit": "node-steps/s", "cores": procs_n, "host_cores": cores,
            "kind": "oracle", "processes": procs_n,
            "sample": f"{procs_n} independent single-threaded oracle processes, each stepping its own "
                      f"copy of {name} for {seconds:g} s ({sum(r[0] for r in res)} steps in total)",
            "mem_available_gb": avail_gb}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = workload(args.workload)
    budget = max(5.0, min(60.0, args.cpu_seconds * 2))
    cb = cpu_baseline(w, budget)
    steps = int(cb["sample"].split()[0])
    # the oracle takes about a second per step of the full workload on one core: it times the
    # steps that fit the CPU budget (reported as steps/warmup) rather than the K requested
    out = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": "node-steps/s",
           "n_gpus": args.gpus, "steps": steps, "warmup": 1,
           "requested_steps": args.steps, "requested_warmup": args.warmup,
           "ms_per_step": 1e3 * w.mesh.n_nodes / cb["value"], "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": w.name, "n_nodes": w.mesh.n_nodes, "dt_ms": w.dt,
                      "parallelism": "1 CPU thread (oracle)"},
           "cpu_baseline": cb,
           "e2e": {"value": cb["value"], "unit": "node-steps/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def timed_steps(sim, w, K, W, stream, torch, preroll=0, usage=False):
    """`preroll` steps from rest (a stimulated wave starts to cross the tissue), W warm-up steps,
    then K steps timed with CUDA events on the simulation's stream (per-launch events inside
    tc_step give the per-kernel split).  The timed window therefore starts at step preroll + W,
    the same window for every form.  With usage, also the surrogate's node-window counts of the
    timed steps alone."""
    sim.step(preroll + W)
    u0 = sim.surrogate_usage() if usage else None
    sim.set_profiling(True)
    sim.reset_profile()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    stats = sim.step(K)
    e1.record(stream)
    torch.cuda.synchronize()
    prof = sim.profile()
    sim.set_profiling(False)
    if usage:
        u1 = sim.surrogate_usage()
        stats = dict(stats, usage_timed={k: u1[k] - u0[k] for k in u1})
    return e0.elapsed_time(e1), stats, prof


def apd90_same_run(apd_ref, apd, act_ref, act):
    """APD90 and activation-time errors of a run against the FP64 run of the same workload, when
    the timed steps cover a full beat (nodes that repolarise in both)."""
    ok = (apd_ref > 0) & (apd > 0)
    if not ok.any():
        return None
    rel = np.abs(apd[ok] - apd_ref[ok]) / apd_ref[ok]
    both = (act_ref >= 0) & (act >= 0)
    return {"nodes_repolarised_both": int(ok.sum()), "repolarised_fp64": int((apd_ref > 0).sum()),
            "repolarised": int((apd > 0).sum()), "apd90_fp64_ms_mean": float(apd_ref[ok].mean()),
            "apd90_err_pct_max": float(100 * rel.max()), "apd90_err_pct_mean": float(100 * rel.mean()),
            "act_err_ms_max": float(np.abs(act[both] - act_ref[both]).max())}


def apd90_check(w_big, torch):
    """APD90 error of the FP32 form against the FP64 path over one full beat (400 ms) of the
    10x4x2 mm slab with the same ionic model (the timed workload ends before repolarisation)."""
    from paper_2510_12011_b300 import tc
    w = I.slab_small_ms()
    w.model, w.tp06_cell, w.dt, w.t_end = w_big.model, w_big.tp06_cell, w_big.dt, 400.0
    w.rtol, w.atol, w.max_iter = w_big.rtol, w_big.atol, w_big.max_iter
    out = {}
    for prec in (tc.TC_FP64, tc.TC_FP32):
        g = tc.from_workload(w, precision=prec)
        g.step(w.n_steps)
        out[prec] = (g.apd90(), g.activation_times())
        g.close()
    a64, a32 = out[tc.TC_FP64][0], out[tc.TC_FP32][0]
    ok = (a64 > 0) & (a32 > 0)
    rel = np.abs(a32[ok] - a64[ok]) / a64[ok]
    return {"workload": f"slab10x4x2_h0.5_{w.model}, {w.t_end:g} ms (one beat)",
            "nodes_repolarised": int(ok.sum()), "nodes": int(a64.size),
            "apd90_fp64_ms_mean": float(a64[ok].mean()) if ok.any() else None,
            "apd90_err_pct_max": float(100 * rel.max()) if ok.any() else None,
            "act_err_ms_max": float(np.abs(out[tc.TC_FP32][1] - out[tc.TC_FP64][1]).max())}


# FLOPs of one network evaluation per row: 20 -> 256 -> 256 -> 256 -> 256 -> 19 (2 per MAC)
MLP_FLOP_PER_ROW = 2 * (20 * 256 + 3 * 256 * 256 + 256 * 19)


def mlp_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return json.load(open(p)).get("bf16_tflops_sustained", 1400.0), "measured"
    return 1400.0, "fallback"


def mlp_roofline(prof):
    """Tensor-pipe roofline of the fused network from the per-window events of a profiled run."""
    mlp_ms = prof["mlp_ms"] / max(prof["surrogate_windows"], 1)
    rows_per_launch = prof["surrogate_rows"] / max(prof["surrogate_windows"], 1)
    flops = MLP_FLOP_PER_ROW * rows_per_launch
    peak, kind = mlp_peak()
    ach = flops / (mlp_ms * 1e-3) / 1e12 if mlp_ms > 0 else 0.0
    return {"kernel": "mlp_fused2_kernel", "bound": "tensor", "achieved": ach, "peak": peak,
            "unit": "TFLOP/s", "frac": ach / peak, "flop_per_launch": flops,
            "rows_per_launch": rows_per_launch, "avg_launch_ms": mlp_ms,
            "peak_source": f"{kind} bf16_tflops_sustained (kernel timed inside the step loop)"}


SURROGATE_CHECK = (10, 2.0, 1.0, 0.3, 0.5)   # window, dv_max, dvdt_max, dv_neighbour, rest_band


def fp64_tissue_run(w, m, t_ms, W, stream, torch):
    """FP64 exact against FP64 tissue with the network, both from rest over t_ms of the slab
    (stimulus, upstroke and the plateau the network takes), graphs on, W untimed steps first:
    ms per step of each, their ratio, the network's share of the node-windows and the activation
    times' largest difference."""
    from paper_2510_12011_b300 import tc
    steps = int(round(t_ms / w.dt))
    res = {}
    for name, net in (("exact", False), ("network", True)):
        sim = tc.from_workload(w, stream=stream.cuda_stream, precision=tc.TC_FP64)
        if net:
            sim.set_surrogate(m, *SURROGATE_CHECK)
        sim.step(W)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = sim.step(steps - W)
        e1.record(stream)
        torch.cuda.synchronize()
        u = sim.surrogate_usage() if net else None
        res[name] = (e0.elapsed_time(e1) / (steps - W), sim.activation_times(), u, st["not_converged"])
        sim.close()
    (ms_e, act_e, _, nc_e), (ms_n, act_n, u, nc_n) = res["exact"], res["network"]
    both = (act_e >= 0) & (act_n >= 0)
    return {"simulated_ms": [0.0, t_ms], "timed_steps": steps - W, "ms_per_step_exact": ms_e,
            "ms_per_step_network": ms_n, "speedup": ms_e / ms_n,
            "network_share": u["surrogate"] / max(1, u["surrogate"] + u["exact"]),
            "activated_both": int(both.sum()),
            "act_err_ms_max": float(np.abs(act_n[both] - act_e[both]).max()) if both.any() else None,
            "not_converged": nc_e + nc_n}


def surrogate_form(w, K, W, preroll, ms64, ms32, act64, stream, torch, apd=True, apd64=None, beat_ms=0.0):
    """FP32 + the learned TP06 surrogate (the network stored with the package) on the same
    workload and the same timed window as the FP64 and FP32 runs (after the pre-roll, so that the
    wave is propagating and the network takes the plateau and recovery windows): node-steps/s,
    the network's share of the timed node-windows, activation-time error against the FP64 run, the
    fused tensor-core kernel's throughput, and APD90 over one beat of the 20x8x3 mm slab the
    network never saw (against the FP64 exact model)."""
    from paper_2510_12011_b300 import surrogate as S, tc
    m = S.load(S.DEFAULT_WEIGHTS)
    sim = tc.from_workload(w, stream=stream.cuda_stream, precision=tc.TC_FP32)
    sim.set_surrogate(m, *SURROGATE_CHECK)
    ms, st, prof = timed_steps(sim, w, K, W, stream, torch, preroll=preroll, usage=True)
    use = sim.surrogate_usage()   # pre-roll, warm-up and timed steps
    ut = st["usage_timed"]
    act = sim.activation_times()
    apd_run = apd90_same_run(apd64, sim.apd90(), act64, act) if apd64 is not None else None
    sim.close()
    both = (act >= 0) & (act64 >= 0)
    n = w.mesh.n_nodes
    apd90 = None
    if apd:
        t = I.surrogate_test_slab(t_end=400.0)
        ref = S.run(t, tc.TC_FP64)
        got = S.run(t, tc.TC_FP32, mlp=m)
        c = S.compare(ref, got)
        u = got["usage"]
        apd90 = {"workload": f"{t.name}, {t.t_end:g} ms, {t.mesh.n_nodes} nodes (not in the training set)",
                 "act_err_ms_max": c["act_err_max_ms"], "apd90_err_pct_max": 100 * c["apd_rel_err_max"],
                 "apd90_err_pct_mean": 100 * c["apd_rel_err_mean"], "nodes_repolarised": c["apd_nodes"],
                 "nodes": t.mesh.n_nodes,
                 "network_share": u["surrogate"] / max(1, u["surrogate"] + u["exact"]),
                 "seconds_fp64": ref["seconds"], "seconds_fp32_surrogate": got["seconds"]}
    # the same network in FP64 tissue: what it gains at the same precision as the exact FP64 run
    sim = tc.from_workload(w, stream=stream.cuda_stream, precision=tc.TC_FP64)
    sim.set_surrogate(m, *SURROGATE_CHECK)
    ms_d, st_d, prof_d = timed_steps(sim, w, K, W, stream, torch, preroll=preroll, usage=True)
    act_d = sim.activation_times()
    sim.close()
    ut_d = st_d["usage_timed"]
    both_d = (act_d >= 0) & (act64 >= 0)
    fp64_tissue = {"value": n * K / (ms_d * 1e-3), "unit": "node-steps/s", "ms_per_step": ms_d / K,
                   "speedup_vs_fp64_exact": ms64 / ms_d, "dtype": "f64 tissue, bf16 network (fp32 accumulate)",
                   "network_share": ut_d["surrogate"] / max(1, ut_d["surrogate"] + ut_d["exact"]),
                   "act_err_ms_max": float(np.abs(act_d[both_d] - act64[both_d]).max()) if both_d.any() else None,
                   "kernels": {"ionic_ms": prof_d["ionic_ms"], "pcg_ms": prof_d["pcg_ms"],
                               "surrogate_ms": prof_d["surrogate_ms"], "mlp_ms": prof_d["mlp_ms"]}}
    if beat_ms > 0:
        fp64_tissue["from_rest"] = fp64_tissue_run(w, m, beat_ms, W, stream, torch)
    return {"value": n * K / (ms * 1e-3), "unit": "node-steps/s", "ms_per_step": ms / K,
            "speedup_vs_fp64": ms64 / ms, "speedup_vs_fp32": ms32 / ms if ms32 else None,
            "fp64_tissue": fp64_tissue,
            "dtype": "f32 tissue, bf16 network (fp32 accumulate)",
            "timed_window_ms": [(preroll + W) * w.dt, (preroll + W + K) * w.dt],
            "window_steps": SURROGATE_CHECK[0],
            "check": {"dv_max_mV": SURROGATE_CHECK[1], "dvdt_max_mV_per_ms": SURROGATE_CHECK[2],
                      "dv_neighbour_mV": SURROGATE_CHECK[3], "rest_band_mV": SURROGATE_CHECK[4]},
            "network_node_windows": ut["surrogate"], "exact_node_windows": ut["exact"],
            "network_share": ut["surrogate"] / max(1, ut["surrogate"] + ut["exact"]),
            "network_share_whole_run": use["surrogate"] / max(1, use["surrogate"] + use["exact"]),
            "act_err_ms_max": float(np.abs(act[both] - act64[both]).max()) if both.any() else None,
            "activated_fp64": int((act64 >= 0).sum()), "activated": int((act >= 0).sum()),
            "mean_cg_iterations": st["cg_iterations"] / max(K, 1),
            "kernels": {"ionic_ms": prof["ionic_ms"], "pcg_ms": prof["pcg_ms"],
                        "surrogate_ms": prof["surrogate_ms"], "mlp_ms": prof["mlp_ms"],
                        "windows": prof["surrogate_windows"]},
            "roofline_mlp": mlp_roofline(prof),
            "apd90": apd90, "apd90_this_run": apd_run}


def ellipsoid_forms(t_end, W, stream, torch):
    """The ellipsoid workloads (the precision form's mesh and the surrogate's): the truncated
    prolate-ellipsoid shell (2,136,691 nodes, TP06 epicardial, dt = 0.02 ms, 5 endocardial
    stimulus sites) run for t_end ms in each of the three forms - plain FP64, FP32, and FP32 with
    the learned surrogate - with CUDA-graph replay.  Each form steps W warm-up steps and is timed
    over the remaining steps of the run; activation times and APD90 of the FP32 forms are compared
    with the FP64 run (nodes that activate / repolarise in both)."""
    from paper_2510_12011_b300 import surrogate as S, tc
    t0 = time.perf_counter()
    w = I.ellipsoid_tp06(t_end=t_end)
    mesh = tc.Mesh.from_inputs(w.mesh)
    gen_s = time.perf_counter() - t0
    n, steps = w.mesh.n_nodes, w.n_steps
    K = steps - W
    m = S.load(S.DEFAULT_WEIGHTS)
    out = {"workload": w.name, "n_nodes": n, "n_tets": w.mesh.n_tets, "dt_ms": w.dt, "simulated_ms": t_end,
           "steps": steps, "warmup": W, "timed_steps": K, "mesh_seconds": gen_s}
    ref = None
    for name, prec, sur in (("fp64", tc.TC_FP64, False), ("fp32", tc.TC_FP32, False),
                            ("fp32_surrogate", tc.TC_FP32, True)):
        sim = tc.from_workload(w, stream=stream.cuda_stream, precision=prec, mesh=mesh)
        if sur:
            sim.set_surrogate(m, *SURROGATE_CHECK)
        sim.step(W)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = sim.step(K)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        act, apd = sim.activation_times(), sim.apd90()
        r = {"value": n * K / (ms * 1e-3), "unit": "node-steps/s", "ms_per_step": ms / K,
             "mean_cg_iterations": st["cg_iterations"] / K, "not_converged": st["not_converged"],
             "graph_steps": st["graph_steps"], "activated": int((act >= 0).sum()),
             "repolarised": int((apd > 0).sum())}
        if sur:
            u = sim.surrogate_usage()
            r["network_share"] = u["surrogate"] / max(1, u["surrogate"] + u["exact"])
            r["network_node_windows"] = u["surrogate"]
        sim.close()
        if ref is None:
            ref = (act, apd, ms)
        else:
            a64, p64, ms64 = ref
            both = (act >= 0) & (a64 >= 0)
            rep = (apd > 0) & (p64 > 0)
            rel = np.abs(apd[rep] - p64[rep]) / p64[rep]
            r.update({"speedup_vs_fp64": ms64 / ms,
                      "act_err_ms_max": float(np.abs(act[both] - a64[both]).max()) if both.any() else None,
                      "act_err_ms_mean": float(np.abs(act[both] - a64[both]).mean()) if both.any() else None,
                      "activated_only_one": int(((act >= 0) ^ (a64 >= 0)).sum()),
                      "apd90_err_pct_max": float(100 * rel.max()) if rep.any() else None,
                      "apd90_err_pct_mean": float(100 * rel.mean()) if rep.any() else None,
                      "apd90_nodes_both": int(rep.sum()), "repolarised_only_one": int(((apd > 0) ^ (p64 > 0)).sum())})
            r["meets_bar"] = bool(r["act_err_ms_max"] is not None and r["act_err_ms_max"] <= 1.0 and
                                  r["apd90_err_pct_max"] is not None and r["apd90_err_pct_max"] <= 2.0)
        out[name] = r
    out["value_fp64"] = out["fp64"]["value"]
    out["value_fp32_surrogate"] = out["fp32_surrogate"]["value"]
    return out


def prior_art_torch(steps, warmup, stream, torch):
    """The paper's own GPU design on the same B300, as prior-art context (not a baseline this
    library is checked against): PyTorch FP64 sparse CSR products and elementwise ops, the
    Mitchell-Schaeffer update as torch expressions, Algorithm 1 driven from the host with its
    stopping test read back every iteration.  Workload: the 504,711-node slab with the
    Mitchell-Schaeffer model (the step is then SpMV/PCG work), timed beside this library's FP64
    step on the same workload and steps.  Matrices come from the library's host assembly."""
    import warnings
    from paper_2510_12011_b300 import tc
    warnings.filterwarnings("ignore", message="Sparse")
    w = I.slab_large("ms")
    n = w.mesh.n_nodes
    mesh = tc.Mesh.from_inputs(w.mesh)
    rp, col, mv, kv = mesh.matrices(w.sigma_l, w.sigma_t)
    dev = torch.device("cuda", torch.cuda.current_device())
    crow = torch.from_numpy(rp).to(dev)
    cidx = torch.from_numpy(col.astype(np.int64)).to(dev)
    Mt = torch.sparse_csr_tensor(crow, cidx, torch.from_numpy(mv).to(dev), size=(n, n))
    Kt = torch.sparse_csr_tensor(crow, cidx, torch.from_numpy(kv).to(dev), size=(n, n))
    av = w.chi * w.cm * mv + w.theta * w.dt * kv
    At = torch.sparse_csr_tensor(crow, cidx, torch.from_numpy(av).to(dev), size=(n, n))
    rows = np.repeat(np.arange(n), np.diff(rp))
    diag = torch.from_numpy(av[rows == col]).to(dev)
    p_ = w.ms
    span = p_.v_max - p_.v_min
    stim = torch.zeros(n, dtype=torch.float64, device=dev)
    st = w.stimuli[0]
    stim[torch.from_numpy(np.asarray(st.nodes, dtype=np.int64)).to(dev)] = st.intensity
    k0, nk = int(round(st.start / w.dt)), int(round(st.duration / w.dt))

    def run(nsteps):
        V = torch.full((n,), p_.v_min, dtype=torch.float64, device=dev)
        Vp = V.clone()
        h = torch.ones(n, dtype=torch.float64, device=dev)
        iters = 0
        for k in range(nsteps):
            v = (V - p_.v_min) / span
            opening = v < p_.v_gate
            hinf = opening.to(torch.float64)
            tau = torch.where(opening, torch.full_like(v, p_.tau_open), torch.full_like(v, p_.tau_close))
            h = hinf + (h - hinf) * torch.exp(-w.dt / tau)
            iion = -w.cm * span * (h * v * v * (1 - v) / p_.tau_in - v / p_.tau_out)
            ist = stim if k0 <= k < k0 + nk else torch.zeros_like(stim)
            b = w.chi * (Mt @ (w.cm * V - w.dt * iion + w.dt * ist)) - (1 - w.theta) * w.dt * (Kt @ V)
            x = 2 * V - Vp
            r = b - At @ x
            z = r / diag
            pvec = z.clone()
            rho = torch.dot(r, z)
            z0 = torch.linalg.vector_norm(z).item()
            if z0 > w.atol:
                for it in range(w.max_iter):
                    q = At @ pvec
                    alpha = rho / torch.dot(pvec, q)
                    x = x + alpha * pvec
                    r = r - alpha * q
                    z = r / diag
                    zn = torch.linalg.vector_norm(z).item()
                    iters += 1
                    if zn < w.atol or zn / z0 < w.rtol:
                        break
                    rho_n = torch.dot(r, z)
                    pvec = z + (rho_n / rho) * pvec
                    rho = rho_n
            Vp, V = V, x
        return iters

    run(warmup)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    it_t = run(steps)
    torch.cuda.synchronize()
    t_torch = time.perf_counter() - t0
    sim = tc.from_workload(w, stream=stream.cuda_stream)
    sim.step(warmup)
    tc.set_model(sim, w)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st_ours = sim.step(steps)
    torch.cuda.synchronize()
    t_ours = time.perf_counter() - t0
    sim.close()
    return {"workload": w.name, "n_nodes": n, "steps": steps, "dtype": "f64",
            "what": "PyTorch sparse CSR + elementwise ops, Algorithm 1 with a host-read stopping test "
                    "per iteration (the paper's design), same GPU",
            "torch": {"value": n * steps / t_torch, "unit": "node-steps/s", "ms_per_step": 1e3 * t_torch / steps,
                      "mean_cg_iterations": it_t / steps},
            "this_library": {"value": n * steps / t_ours, "unit": "node-steps/s", "ms_per_step": 1e3 * t_ours / steps,
                             "mean_cg_iterations": st_ours["cg_iterations"] / steps},
            "speedup": t_torch / t_ours}


def batched_form(steps, stream, torch):
    """The batched form: 64 uneven slabs (5.3 M nodes) as independent problems in one
    simulation, FP32, launch shape by the autotuner, step loop by CUDA-graph replay (also timed
    with host launches for comparison)."""
    from paper_2510_12011_b300 import tc
    b = I.batched_slabs()
    w = b.workload
    t0 = time.perf_counter()
    sim = tc.from_workload(w, stream=stream.cuda_stream, precision=tc.TC_FP32)
    setup_s = time.perf_counter() - t0
    tune = sim.autotune(20)
    out = {"workload": w.name, "instances": len(b.instances), "n_nodes": w.mesh.n_nodes,
           "instance_nodes_min": int(min(x.mesh.n_nodes for x in b.instances)),
           "instance_nodes_max": int(max(x.mesh.n_nodes for x in b.instances)),
           "dtype": "f32 (FP64 reductions)", "dt_ms": w.dt, "autotune": tune,
           "setup_s": setup_s}
    for graphs in (True, False):
        sim.set_graphs(graphs)
        tc.set_model(sim, w)
        sim.step(30)
        tc.set_model(sim, w)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = sim.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        key = "graph" if graphs else "host_launches"
        out[key] = {"value": w.mesh.n_nodes * steps / (ms * 1e-3), "unit": "node-steps/s",
                    "ms_per_step": ms / steps, "steps": steps,
                    "mean_cg_iterations_per_instance": st["cg_iterations"] / steps / len(b.instances),
                    "not_converged": st["not_converged"]}
    out["value"] = out["graph"]["value"]
    # per-launch split and the PCG launch's roofline from a short profiled run (host launches)
    tc.set_model(sim, w)
    sim.step(60)
    sim.set_profiling(True)
    sim.reset_profile()
    st = sim.step(30)
    prof = sim.profile()
    sim.set_profiling(False)
    size = sim.size()
    n_int = sim.layout()["n_internal"]
    it_mean = st["cg_iterations"] / 30 / len(b.instances)
    pcg_ms = prof["pcg_ms"] / max(prof["pcg_launches"], 1)
    by = pcg_launch_bytes(w.mesh.n_nodes, size["nnz"], n_int // 32, it_mean, vb=4)
    peak, kind = measured_peaks()
    out["kernels"] = {"ionic_ms_per_launch": prof["ionic_ms"] / max(prof["ionic_launches"], 1),
                      "pcg_ms_per_launch": pcg_ms,
                      "launches_per_step": (prof["ionic_launches"] + prof["pcg_launches"]) / 30.0,
                      "note": "the Mitchell-Schaeffer update runs inside the PCG launch (one persistent "
                              "launch per time step)" if prof["ionic_launches"] == 0 else None}
    by += 7 * 4 * w.mesh.n_nodes if prof["ionic_launches"] == 0 else 0   # fused update: V, V^{k-1}, h in; h, g1, g2, x0 out
    out["roofline_pcg"] = {"kernel": "pcg_step_kernel_512<float>", "bound": "hbm",
                           "achieved": by / (pcg_ms * 1e-3) / 1e9, "peak": peak, "unit": "GB/s",
                           "frac": by / (pcg_ms * 1e-3) / 1e9 / peak, "bytes_per_launch": by,
                           "bytes_note": "FP32 values, int32 indices; mean CG iterations per instance "
                                         f"({it_mean:.2f}) times the whole batch's per-iteration bytes",
                           "peak_source": f"{kind} hbm_gbs", "avg_launch_ms": pcg_ms}
    sim.close()
    return out


def replica_throughput(ms_local, n_nodes, steps, world, device):
    """Whole-job node-steps/s of `world` independent replicas (weak scaling): the slowest rank's
    time (max over ranks) bounds the job; every rank stepped n_nodes for `steps` steps."""
    ms = ms_local
    if world > 1:
        import torch
        t = torch.tensor([ms_local], dtype=torch.float64, device=device)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    return ms, n_nodes * steps * world / (ms * 1e-3)


def run_ours(args):
    import torch
    from paper_2510_12011_b300 import tc

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    w = workload(args.workload)
    K = args.steps if args.steps is not None else w.n_steps
    W = max(3, args.warmup)
    P = max(0, int(round(args.preroll_ms / w.dt)))
    n = w.mesh.n_nodes

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    sim = tc.from_workload(w, stream=stream.cuda_stream)
    # the library's autotuner picks the PCG launch shape and whether to stage z windows in
    # shared memory (trial steps from rest; the state is restored afterwards)
    tune64 = dict(sim.autotune(10), staging=sim.staging())
    size = sim.size()
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    ms, stats, prof = timed_steps(sim, w, K, W, stream, torch, preroll=P)
    barrier()
    clk = clocks.stop()
    v64, act64, apd64 = sim.read(), sim.activation_times(), sim.apd90()
    ms, value = replica_throughput(ms, n, K, world, dev)

    # roofline of the dominant kernel (by accumulated device time)
    peak, peak_kind = measured_peaks()
    pcg_launch_ms = prof["pcg_ms"] / max(prof["pcg_launches"], 1)
    ion_launch_ms = prof["ionic_ms"] / max(prof["ionic_launches"], 1)
    iters = prof["pcg_iterations"] / max(prof["pcg_launches"], 1)
    bytes_launch = pcg_launch_bytes(n, size["nnz"], (n + 31) // 32, iters)
    pcg_gbs = bytes_launch / (pcg_launch_ms * 1e-3) / 1e9
    cap = w.name == "slab40x16x6_h0.2_tp06"
    roof_pcg = {"kernel": "pcg_step_kernel", "bound": "hbm", "achieved": pcg_gbs, "peak": peak,
                "unit": "GB/s", "frac": pcg_gbs / peak,
                "traffic": PCG_FP64_DRAM_BYTES_PER_LAUNCH if cap else None,
                "traffic_note": (f"ncu dram bytes of one launch in a run averaging {PCG_FP64_CAPTURE_ITERATIONS} CG iterations "
                                 f"(this run averages {iters:.2f}); about half of A and its index array stays in the "
                                 "132.6 MB L2 across iterations (evict-last fraction), the rest and M, K stream from DRAM") if cap else None,
                "peak_source": f"{peak_kind} hbm_gbs", "bytes_per_launch": bytes_launch,
                "avg_launch_ms": pcg_launch_ms}
    by_min = pcg_launch_bytes_minimum(n, size["nnz"], iters)
    roof_pcg["bytes_minimum_per_launch"] = by_min
    roof_pcg["frac_of_minimum_bytes"] = by_min / (pcg_launch_ms * 1e-3) / 1e9 / peak
    # B300's FP64 pipe binds this launch as much as HBM does: the same launch against the measured
    # FP64 multiply-add rate
    rate = tc.measure_fp64_rate()
    ops = pcg_fp64_ops(n, size["nnz"], iters)
    roof_pcg["fp64"] = {"ops_per_launch": ops, "achieved": ops / (pcg_launch_ms * 1e-3) / 1e12,
                        "peak_measured": rate / 1e12, "unit": "T FP64 FMA/s",
                        "frac_of_measured": ops / (pcg_launch_ms * 1e-3) / rate,
                        "count": "Algorithm 1: RHS 2 nnz + 4 n, per iteration nnz + 7 n"}
    if prof["ionic_ms"] > prof["pcg_ms"] and w.model == "tp06" and TP06_FP64_INSTR_PER_NODE:
        ach = TP06_FP64_INSTR_PER_NODE * n / (ion_launch_ms * 1e-3)
        pk = fp64_instr_peak(clk.get("sm_mhz"))
        roofline = {"kernel": "ionic_tp06_kernel<double>", "bound": "alu", "achieved": ach / 1e12,
                    "peak": pk / 1e12, "unit": "T FP64 thread-instr/s", "frac": ach / pk,
                    "peak_measured": rate / 1e12, "frac_of_measured": ach / rate,
                    "peak_measured_source": "tc_measure_fp64_rate: FMA chains, eight per thread, full occupancy",
                    "traffic": TP06_FP64_DRAM_BYTES_PER_LAUNCH * n / 504711,
                    "traffic_unit": "bytes per launch (ncu dram read + write)",
                    "peak_source": "FP64 pipe: 2 instr/clk/SM x 148 SMs x median SM clock of the run",
                    "fp64_instr_per_node": TP06_FP64_INSTR_PER_NODE, "avg_launch_ms": ion_launch_ms}
    else:
        roofline = roof_pcg

    # SpMV HBM GB/s: y = A x alone, L2 flushed before every launch
    spmv_ms, spmv_reps = spmv_cold(sim, n, torch.float64, stream, torch, tc)
    spmv_gbs = spmv_bytes(n, size["nnz"]) / (spmv_ms * 1e-3) / 1e9

    # end to end through the C ABI with host buffers: each step uploads V^k, V^{k-1} and every
    # ionic state from page-locked host memory, steps once and reads V^{k+1} and the states back
    Ke = max(1, min(args.e2e_steps, K))
    tc.set_model(sim, w)
    n_states = 1 if w.model == "ms" else 18
    fields = [tc.TC_FIELD_V, tc.TC_FIELD_V_PREV] + [tc.TC_FIELD_STATE + j for j in range(n_states)]
    host = {f: torch.empty(n, dtype=torch.float64, pin_memory=True).numpy() for f in fields}
    for f in fields:
        host[f][:] = sim.read(f)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(Ke):
        for f in fields:
            sim.write(f, host[f])
        sim.step(1)
        host[tc.TC_FIELD_V_PREV][:] = host[tc.TC_FIELD_V]
        for f in fields:
            if f != tc.TC_FIELD_V_PREV:
                sim.read(f, out=host[f])
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    barrier()
    e2e = {"value": n * Ke * world / e2e_s, "unit": "node-steps/s",
           "h2d_bytes_per_step": len(fields) * 8 * n, "d2h_bytes_per_step": (len(fields) - 1) * 8 * n,
           "steps": Ke,
           "what": "per step: tc_write_state of V^k, V^{k-1} and every ionic state from pinned host "
                   "arrays, tc_step(1), tc_read_state of V^{k+1} and the states"}
    # the same with the state left resident: per step tc_step(1) and tc_read_state of V^{k+1}
    tc.set_model(sim, w)
    vbuf = torch.empty(n, dtype=torch.float64, pin_memory=True).numpy()
    sim.step(1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(Ke):
        sim.step(1)
        sim.read(tc.TC_FIELD_V, out=vbuf)
    e2e_v_s = time.perf_counter() - t0
    e2e["v_only"] = {"value": n * Ke * world / e2e_v_s, "unit": "node-steps/s", "h2d_bytes_per_step": 0,
                     "d2h_bytes_per_step": 8 * n, "steps": Ke,
                     "what": "state resident on the device; per step tc_step(1) and tc_read_state of V^{k+1}"}
    sim.close()

    # FP32 precision form on the same workload and steps, and its error against FP64
    fp32 = None
    if not args.no_fp32:
        sim32 = tc.from_workload(w, stream=stream.cuda_stream, precision=tc.TC_FP32)
        tune32 = dict(sim32.autotune(10), staging=sim32.staging())
        ms32, st32, prof32 = timed_steps(sim32, w, K, W, stream, torch, preroll=P)
        v32, act32, apd32 = sim32.read(), sim32.activation_times(), sim32.apd90()
        both = (act32 >= 0) & (act64 >= 0)
        fp32 = {"value": n * K * world / (ms32 * 1e-3), "unit": "node-steps/s",
                "ms_per_step": ms32 / K, "dtype": "f32 (FP64 reductions, alpha, beta)",
                "speedup_vs_fp64": ms / ms32,
                "act_err_ms_max": float(np.abs(act32[both] - act64[both]).max()) if both.any() else None,
                "activated_fp64": int((act64 >= 0).sum()), "activated_fp32": int((act32 >= 0).sum()),
                "v_err_mv_max": float(np.abs(v32 - v64).max()),
                "mean_cg_iterations": st32["cg_iterations"] / max(K, 1), "autotune": tune32,
                "kernels": {"ionic_ms": prof32["ionic_ms"], "pcg_ms": prof32["pcg_ms"]}}
        pcg32_ms = prof32["pcg_ms"] / max(prof32["pcg_launches"], 1)
        it32 = prof32["pcg_iterations"] / max(prof32["pcg_launches"], 1)
        by32 = pcg_launch_bytes(n, size["nnz"], (n + 31) // 32, it32, vb=4)
        fp32["roofline_pcg"] = {"kernel": "pcg_step_kernel_1024<float>", "bound": "hbm",
                                "achieved": by32 / (pcg32_ms * 1e-3) / 1e9, "peak": peak, "unit": "GB/s",
                                "frac": by32 / (pcg32_ms * 1e-3) / 1e9 / peak, "bytes_per_launch": by32,
                                "avg_launch_ms": pcg32_ms, "iterations_per_launch": it32,
                                "us_per_iteration": 1e3 * pcg32_ms / max(it32, 1e-9),
                                "note": "the FP32 matrices (59 MB) stay in the 132.6 MB L2 across iterations: "
                                        "the launch is latency- and barrier-bound, not HBM-bound"}
        ms_sp, reps = spmv_cold(sim32, n, torch.float32, stream, torch, tc)
        by = spmv_bytes(n, size["nnz"], 4)
        fp32["spmv"] = {"value": by / (ms_sp * 1e-3) / 1e9, "unit": "GB/s", "ms": ms_sp, "bytes": by,
                        "frac": by / (ms_sp * 1e-3) / 1e9 / peak, "launches": reps,
                        "statistic": "median of 3 (sequence of flush + SpMV minus sequence of flush) / launches",
                        "l2": "flushed (512 MB read) before every launch"}
        sim32.close()
        if w.model == "tp06":
            fp32["apd90_this_run"] = apd90_same_run(apd64, apd32, act64, act32)
            if fp32["apd90_this_run"] is None:
                fp32["apd90"] = apd90_check(w, torch)

    sur = None
    if not args.no_surrogate and w.model == "tp06":
        sur = surrogate_form(w, K, W, P, ms, ms32 if fp32 else None, act64, stream, torch,
                             apd=not args.no_surrogate_apd, apd64=apd64, beat_ms=args.fp64_beat_ms)

    prior = None
    if not args.no_prior_art and world == 1:
        prior = prior_art_torch(300, 5, stream, torch)

    batched = None
    if not args.no_batched:
        batched = batched_form(min(args.batched_steps, max(K, 30)), stream, torch)

    ell = None
    if not args.no_ellipsoid and world == 1 and w.model == "tp06":
        ell = ellipsoid_forms(args.ellipsoid_ms, W, stream, torch)

    if rank != 0:
        return
    out = {
        "metric": METRIC, "value": value, "unit": "node-steps/s", "n_gpus": world, "steps": K,
        "warmup": W, "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "n_nodes": n, "n_tets": w.mesh.n_tets, "nnz": size["nnz"],
                   "padded_nnz": size["padded_nnz"], "pcg_blocks": size["n_blocks"],
                   "dt_ms": w.dt, "simulated_ms": K * w.dt, "ionic_model": w.model,
                   "timed_window_ms": [(P + W) * w.dt, (P + W + K) * w.dt],
                   "preroll": f"{P} steps ({P * w.dt:g} ms) from rest before the {W} warm-up steps: the "
                              "corner stimulus's wave is crossing the slab during the timed steps",
                   "tp06_cell": w.tp06_cell if w.model == "tp06" else None,
                   "pcg": {"atol": w.atol, "rtol": w.rtol, "max_iter": w.max_iter},
                   "l2": "inputs larger than L2: one step streams M, K, A values and indices "
                         f"({size['padded_nnz'] * 28 / 1e6:.0f} MB) plus node vectors vs 132.6 MB L2",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "autotune": tune64},
        "stats": {"cg_iterations": stats["cg_iterations"],
                  "mean_cg_iterations": stats["cg_iterations"] / max(K, 1),
                  "max_cg_iterations": stats["max_iterations"],
                  "not_converged": stats["not_converged"]},
        "kernels": {"ionic": {"launches": prof["ionic_launches"], "ms": prof["ionic_ms"]},
                    "pcg_step_kernel": {"launches": prof["pcg_launches"], "ms": prof["pcg_ms"],
                                        "iterations": prof["pcg_iterations"]}},
        "roofline": roofline,
        "roofline_pcg": roof_pcg,
        "spmv": {"value": spmv_gbs, "unit": "GB/s", "ms": spmv_ms, "bytes": spmv_bytes(n, size["nnz"]),
                 "frac": spmv_gbs / peak, "l2": "flushed (512 MB read) before every launch",
                 "launches": spmv_reps, "statistic": "median of 3 (sequence of flush + SpMV minus sequence of flush) / launches"},
        "fp32_form": fp32,
        "surrogate_form": sur,
        "batched_form": batched,
        "ellipsoid_forms": ell,
        "prior_art_torch": prior,
        "e2e": e2e,
        "gpu_launches": prof["ionic_launches"] + prof["pcg_launches"],
        "clocks": clk,
    }
    if not args.no_cpu_baseline and world == 1:
        out["cpu_baseline"] = cpu_baseline(w, args.cpu_seconds)
        if not args.no_cpu_all_cores:
            out["cpu_baseline_all_cores"] = cpu_baseline_all_cores(args.workload, args.cpu_seconds)
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
