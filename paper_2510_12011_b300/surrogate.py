"""Learned ionic surrogate: training-data generation from tissue runs, training, and the check
of a trained network inside the monodomain step against the exact TP06 model.

All arithmetic runs in the library's kernels (tissue steps, FP64 exact windows, the tensor-core
network and its training); this module only schedules those calls and holds device buffers.
"""
import os
import time

import numpy as np

from . import tc


def generate(workloads, capacity, window=10, every=10, rest_band=1.0, rest_keep=0.05, dv_keep=4.0,
             dvdt_keep=2.0, seed=0, device="cuda"):
    """Run every workload (TP06, FP32 form) and sample training pairs at every `every`-th window
    start; returns device tensors x [count][20], y [count][19] (views of the first `count` rows)
    and the count.  Capacity bounds the memory: sampling stops when it is full.  dv_keep and
    dvdt_keep leave out the windows a deployed surrogate's check (set at half these bounds)
    hands to the exact model, so that the network's output scale resolves the slow phases."""
    import torch
    x = torch.empty((capacity, tc.Mlp.N_IN), dtype=torch.float32, device=device)
    y = torch.empty((capacity, tc.Mlp.N_OUT), dtype=torch.float32, device=device)
    count = 0
    for wi, w in enumerate(workloads):
        sim = tc.from_workload(w, precision=tc.TC_FP32)
        try:
            n_steps = w.n_steps
            k = 0
            while k < n_steps and count < capacity:
                count = sim.surrogate_sample(x.data_ptr(), y.data_ptr(), capacity, count, window, rest_band,
                                             rest_keep, dv_keep, dvdt_keep, seed + 1000003 * wi)
                adv = min(window * every, n_steps - k)
                sim.step(adv)
                k += adv
        finally:
            sim.close()
    return x[:count], y[:count], count


def train(x, y, count, epochs=20, batch=2048, lr=1e-3, lr_end=1e-5, v_weight=9.0, seed=1, mlp=None):
    """Fit the normalization to (x, y) and train a network with Adam, the step size decaying
    geometrically from lr to lr_end over the epochs; returns (network, mean loss per epoch).
    v_weight multiplies the loss weight of the membrane potential's change (its output scale is
    divided by sqrt(v_weight)): the potential is the output the tissue sees directly, through
    the window's effective current."""
    m = mlp or tc.Mlp(seed=seed)
    m.fit_normalization(x.data_ptr(), y.data_ptr(), count)
    if v_weight != 1.0:
        nm = m.normalization()
        nm[2 * tc.Mlp.N_IN + tc.Mlp.N_OUT + 18] /= np.sqrt(v_weight)
        m.set_normalization(nm[:20], nm[20:40], nm[40:59], nm[59:78])
    hist = []
    for e in range(epochs):
        lr_e = lr * (lr_end / lr) ** (e / max(1, epochs - 1))
        hist.append(float(m.train(x.data_ptr(), y.data_ptr(), count, 1, batch, lr_e, seed=seed + e)[0]))
    return m, np.array(hist)


def run(w, precision, mlp=None, window=10, dv_max=2.0, dvdt_max=1.0, dv_neighbour=0.3, rest_band=0.5,
        graphs=True):
    """One full run of workload w; returns activation times, APD90, wall time and (with a
    network) the surrogate's usage counts."""
    import torch
    sim = tc.from_workload(w, precision=precision)
    try:
        sim.set_graphs(graphs)
        if mlp is not None:
            sim.set_surrogate(mlp, window, dv_max, dvdt_max, dv_neighbour, rest_band)
        sim.step(min(50, w.n_steps))    # warm-up (graph capture, tensor-map set-up)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = sim.step(w.n_steps - min(50, w.n_steps))
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        out = {"act": sim.activation_times(w.v_threshold), "apd90": sim.apd90(), "seconds": wall,
               "timed_steps": w.n_steps - min(50, w.n_steps), "n": w.mesh.n_nodes,
               "graph_steps": st["graph_steps"]}
        if mlp is not None:
            out["usage"] = sim.surrogate_usage()
        return out
    finally:
        sim.close()


def compare(ref, got):
    """Activation-time and APD90 errors of `got` against `ref` (nodes that activate / repolarise
    in both runs), and the coverage of each."""
    a0, a1 = ref["act"], got["act"]
    both = (a0 >= 0) & (a1 >= 0)
    p0, p1 = ref["apd90"], got["apd90"]
    rep = (p0 > 0) & (p1 > 0)
    rel = np.abs(p1[rep] - p0[rep]) / p0[rep]
    return {
        "act_nodes": int(both.sum()), "act_only_one": int(((a0 >= 0) ^ (a1 >= 0)).sum()),
        "act_err_max_ms": float(np.abs(a1[both] - a0[both]).max()) if both.any() else float("nan"),
        "act_err_mean_ms": float(np.abs(a1[both] - a0[both]).mean()) if both.any() else float("nan"),
        "apd_nodes": int(rep.sum()), "apd_only_one": int(((p0 > 0) ^ (p1 > 0)).sum()),
        "apd_rel_err_max": float(rel.max()) if rep.any() else float("nan"),
        "apd_rel_err_mean": float(rel.mean()) if rep.any() else float("nan"),
    }


def save(m, path):
    """Write a trained network (parameters and normalization) to an .npz file."""
    np.savez(path, params=m.params(), norm=m.normalization())


def load(path, seed=0):
    """A network with the parameters and normalization stored by save()."""
    d = np.load(path)
    m = tc.Mlp(seed=seed)
    m.set_params(d["params"])
    nm = d["norm"]
    m.set_normalization(nm[:20], nm[20:40], nm[40:59], nm[59:78])
    return m


DEFAULT_WEIGHTS = os.path.join(os.path.dirname(__file__), "data", "tp06_epi_surrogate.npz")


def main(argv=None):
    """Train the TP06 (epicardial) surrogate from the four seeded training slabs and store it."""
    import argparse
    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("--out", default=DEFAULT_WEIGHTS)
    ap.add_argument("--slabs", type=int, default=4)
    ap.add_argument("--epochs", type=int, default=20)
    a = ap.parse_args(argv)
    from . import inputs
    t0 = time.time()
    x, y, cnt = generate(inputs.surrogate_training_slabs(count=a.slabs, t_end=500.0), capacity=40_000_000)
    t1 = time.time()
    m, hist = train(x, y, cnt, epochs=a.epochs)
    t2 = time.time()
    os.makedirs(os.path.dirname(a.out), exist_ok=True)
    save(m, a.out)
    print(f"{cnt} pairs in {t1 - t0:.1f} s; {a.epochs} epochs in {t2 - t1:.1f} s; loss {hist[0]:.3e} -> "
          f"{hist[-1]:.3e}; saved {a.out}")


if __name__ == "__main__":
    main()
