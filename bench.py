#!/usr/bin/env python
"""Benchmark of the monodomain hot path: node-steps/s of the plain FP64 method on one B300.

One step = ionic update + RHS + Jacobi-PCG solve + activation capture for every node of the
workload (one time step k -> k+1 of the operator-split scheme).  The default workload is the
40x16x6 mm slab at h = 0.2 mm (504,711 nodes, 2,880,000 tets, dt = 0.02 ms, 5000 steps =
100 ms).  Inputs are synthetic and seeded.

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

METRIC = "node-steps/s (plain FP64 monodomain step: ionic + RHS + Jacobi-PCG + activation capture)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["large_ms", "small_ms"], default="large_ms")
    ap.add_argument("--e2e-steps", type=int, default=30)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def workload(name):
    if name == "large_ms":
        return I.slab_large("ms")
    return I.slab_small_ms()


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6400.0), "measured"
    return 6400.0, "fallback"


# ---- algorithmic bytes (FP64 values, int32 indices; SELL padding not counted) -------------
def pcg_launch_bytes(n, nnz, nslices, iters):
    """Bytes one PCG launch must move: RHS pass (M, K values, indices, g1/g2, dinv in; r, z, p
    out), per iteration the A-product (A values, indices, p gather, q out) and the vector
    phases (x, r r/w; p, q, dinv in; z out), the direction update on all but the last
    iteration (z in, p r/w), and the activation capture (act, V^k, V^{k+1})."""
    rhs = 20 * nnz + 4 * (nslices + 1) + 16 * n + 8 * n + 24 * n
    spmv = 12 * nnz + 4 * (nslices + 1) + 16 * n
    vec = 64 * n
    pupd = 24 * n
    cap = 24 * n
    return rhs + iters * (spmv + vec) + max(iters - 1.0, 0.0) * pupd + cap


def spmv_bytes(n, nnz):
    """CSR-equivalent algorithmic bytes of one y = A x: values + column indices + row pointers +
    x read once + y written once."""
    return 12 * nnz + 4 * (n + 1) + 8 * n + 8 * n


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
    if True:
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
    return {"value": w.mesh.n_nodes * steps / total, "unit": "node-steps/s", "cores": 1,
            "kind": "oracle",
            "sample": f"{steps} time steps (steps 2..{steps + 1}) of {w.name}, "
                      f"{w.mesh.n_nodes} nodes, numpy/scipy FP64, 1 thread"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = workload(args.workload)
    budget = max(5.0, min(60.0, args.cpu_seconds * 2))
    cb = cpu_baseline(w, budget)
    steps = int(cb["sample"].split()[0])
    out = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": "node-steps/s",
           "n_gpus": args.gpus, "steps": steps, "warmup": 1,
           "ms_per_step": 1e3 * w.mesh.n_nodes / cb["value"], "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": w.name, "n_nodes": w.mesh.n_nodes, "dt_ms": w.dt,
                      "parallelism": "1 CPU thread (oracle)"},
           "cpu_baseline": cb,
           "e2e": {"value": cb["value"], "unit": "node-steps/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


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
    n = w.mesh.n_nodes

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    sim = tc.from_workload(w, stream=stream.cuda_stream)
    size = sim.size()
    sim.step(W)
    sim.set_ionic(tc.TC_MODEL_MS, w.ms.as_array())     # back to rest, step 0
    sim.set_profiling(True)
    sim.reset_profile()
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    stats = sim.step(K)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    prof = sim.profile()
    sim.set_profiling(False)
    if world > 1:
        t = torch.tensor([ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    value = n * K * world / (ms * 1e-3)

    # roofline of the dominant kernel (by accumulated device time)
    peak, peak_kind = measured_peaks()
    pcg_launch_ms = prof["pcg_ms"] / max(prof["pcg_launches"], 1)
    iters = prof["pcg_iterations"] / max(prof["pcg_launches"], 1)
    bytes_launch = pcg_launch_bytes(n, size["nnz"], (n + 31) // 32, iters)
    achieved = bytes_launch / (pcg_launch_ms * 1e-3) / 1e9
    dominant = "pcg_step_kernel" if prof["pcg_ms"] >= prof["ionic_ms"] else "ionic_ms_kernel"

    # SpMV HBM GB/s: y = A x alone, L2 flushed before every launch
    x = torch.randn(n, dtype=torch.float64, device=dev)
    y = torch.empty_like(x)
    flush = torch.ones(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    times = []
    for rep in range(12):
        flush_sum = flush.sum()   # reading 512 MB evicts the matrix without leaving dirty lines
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sim.apply_dev(tc.TC_OP_A, x.data_ptr(), y.data_ptr())
        b.record(stream)
        torch.cuda.synchronize()
        if rep >= 2:
            times.append(a.elapsed_time(b))
    spmv_ms = float(np.median(times))
    spmv_gbs = spmv_bytes(n, size["nnz"]) / (spmv_ms * 1e-3) / 1e9
    del flush

    # end to end through the C ABI with host buffers: each step uploads V^k, V^{k-1} and the
    # ionic state from page-locked host memory, steps once and reads V^{k+1} back
    Ke = max(1, min(args.e2e_steps, K))
    sim.set_ionic(tc.TC_MODEL_MS, w.ms.as_array())
    hv = torch.empty(n, dtype=torch.float64, pin_memory=True).numpy()
    hp = torch.empty(n, dtype=torch.float64, pin_memory=True).numpy()
    hh = torch.empty(n, dtype=torch.float64, pin_memory=True).numpy()
    hv[:] = w.ms.v_min
    hp[:] = w.ms.v_min
    hh[:] = 1.0
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(Ke):
        sim.write(tc.TC_FIELD_V, hv)
        sim.write(tc.TC_FIELD_V_PREV, hp)
        sim.write(tc.TC_FIELD_STATE, hh)
        sim.step(1)
        hp[:] = hv
        hv[:] = sim.read(tc.TC_FIELD_V)
        hh[:] = sim.read(tc.TC_FIELD_STATE)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    barrier()
    e2e = {"value": n * Ke * world / e2e_s, "unit": "node-steps/s", "h2d_bytes_per_step": 3 * 8 * n,
           "d2h_bytes_per_step": 2 * 8 * n, "steps": Ke,
           "what": "per step: tc_write_state(V^k, V^{k-1}, gate) from pinned host arrays, "
                   "tc_step(1), tc_read_state(V^{k+1}, gate) to host"}

    if rank != 0:
        return
    out = {
        "metric": METRIC, "value": value, "unit": "node-steps/s", "n_gpus": world, "steps": K,
        "warmup": W, "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "n_nodes": n, "n_tets": w.mesh.n_tets, "nnz": size["nnz"],
                   "padded_nnz": size["padded_nnz"], "pcg_blocks": size["n_blocks"],
                   "dt_ms": w.dt, "simulated_ms": K * w.dt, "ionic_model": w.model,
                   "pcg": {"atol": w.atol, "rtol": w.rtol, "max_iter": w.max_iter},
                   "l2": "inputs larger than L2: one step streams M, K, A values and indices "
                         f"({size['padded_nnz'] * 28 / 1e6:.0f} MB) plus node vectors vs 132.6 MB L2",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "stats": {"cg_iterations": stats["cg_iterations"],
                  "mean_cg_iterations": stats["cg_iterations"] / max(K, 1),
                  "max_cg_iterations": stats["max_iterations"],
                  "not_converged": stats["not_converged"]},
        "kernels": {"ionic_ms_kernel": {"launches": prof["ionic_launches"], "ms": prof["ionic_ms"]},
                    "pcg_step_kernel": {"launches": prof["pcg_launches"], "ms": prof["pcg_ms"],
                                        "iterations": prof["pcg_iterations"]}},
        "roofline": {"kernel": dominant, "bound": "hbm", "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak, "traffic": None,
                     "peak_source": f"{peak_kind} hbm_gbs",
                     "bytes_per_launch": bytes_launch, "avg_launch_ms": pcg_launch_ms},
        "spmv": {"value": spmv_gbs, "unit": "GB/s", "ms": spmv_ms, "bytes": spmv_bytes(n, size["nnz"]),
                 "frac": spmv_gbs / peak, "l2": "flushed (512 MB read) before every launch"},
        "e2e": e2e,
        "gpu_launches": prof["ionic_launches"] + prof["pcg_launches"],
        "clocks": clk,
    }
    if not args.no_cpu_baseline and world == 1:
        out["cpu_baseline"] = cpu_baseline(w, args.cpu_seconds)
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
