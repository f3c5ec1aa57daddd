"""N-version benchmark study (Section 3.1.2, Table 3): activation times along the diagonal from
P1 to P8 of the 20x7x3 mm slab at spacings 0.5, 0.2 and 0.1 mm (dt = 0.005 ms), FP64.

No gold-standard data ships with this package, so the study reports self-convergence: the
differences between successive spacings, which shrink as the mesh is refined.  All arithmetic
runs in the library's kernels; this module schedules the runs.

    python -m paper_2510_12011_b300.nversion [--h 0.5 0.2 0.1] [--t-end 100]
"""
import argparse
import json
import time

import numpy as np

from . import inputs, tc


def run(h, t_end=100.0, precision=tc.TC_FP64, points=11):
    """One spacing: activation times (ms) at `points` nodes along the P1-P8 diagonal, the
    positions of those nodes, and the wall time."""
    w = inputs.nversion_slab(h, t_end)
    sim = tc.from_workload(w, precision=precision)
    try:
        t0 = time.perf_counter()
        st = sim.step(w.n_steps)
        wall = time.perf_counter() - t0
        act = sim.activation_times(w.v_threshold)
    finally:
        sim.close()
    d = inputs.diagonal_nodes(w.mesh, points)
    return {"h": h, "n_nodes": w.mesh.n_nodes, "steps": w.n_steps, "seconds": wall,
            "mean_cg_iterations": st["cg_iterations"] / max(1, w.n_steps),
            "diagonal_mm": w.mesh.xyz[d].tolist(), "act_ms": act[d].tolist(),
            "all_activated": bool((act >= 0).all())}


def study(hs=(0.5, 0.2, 0.1), t_end=100.0):
    out = [run(h, t_end) for h in hs]
    for a, b in zip(out, out[1:]):
        da = np.abs(np.asarray(a["act_ms"]) - np.asarray(b["act_ms"]))
        b["diff_to_coarser_ms_max"] = float(da.max())
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--h", type=float, nargs="+", default=[0.5, 0.2, 0.1])
    ap.add_argument("--t-end", type=float, default=100.0)
    a = ap.parse_args(argv)
    for r in study(a.h, a.t_end):
        print(json.dumps(r), flush=True)


if __name__ == "__main__":
    main()
