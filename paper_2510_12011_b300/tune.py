"""Layout autotuner: the SELL-C-32 row-sorting window sigma and the launch shape of a workload,
chosen by timing.

For each candidate window a simulation is assembled from the same mesh; tc_autotune then times
trial steps for each launch shape (threads per block, blocks per SM, and with them the CTAs each
component gets) and keeps the fastest; the window whose tuned step is fastest wins.  The slice
height C stays 32: a slice is one warp instruction wide.  All timing runs in the library."""
from . import tc


def autotune_layout(w, precision=tc.TC_FP32, sigmas=(256, 1024, 4096), trial_steps=20, stream=None):
    """Returns {'sell_sigma', 'pcg_threads', 'blocks_per_sm', 'ms_per_step', 'trials', 'mesh'}:
    the fastest candidate, every candidate's tuned result, and a Mesh set to the chosen window
    (pass it to tc.from_workload(..., mesh=...) to assemble the tuned simulation)."""
    mesh = tc.Mesh.from_inputs(w.mesh)
    trials = []
    for sg in sigmas:
        mesh.set_sell_sigma(sg)
        sim = tc.from_workload(w, stream=stream, precision=precision, mesh=mesh)
        try:
            r = sim.autotune(trial_steps)
            trials.append({"sell_sigma": int(sg), "padded_nnz": sim.size()["padded_nnz"], **r})
        finally:
            sim.close()
    best = min(trials, key=lambda t: t["ms_per_step"])
    mesh.set_sell_sigma(best["sell_sigma"])
    return {**best, "trials": trials, "mesh": mesh}
