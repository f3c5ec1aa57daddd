"""Shared-memory staging of the PCG's gathers: every block of the cooperative launch copies its
window of z (the band of columns its rows touch under the RCM order) into shared memory when it
fits (when staging is asked for, or picked by the autotuner), and gathers from global memory
otherwise; column indices are read as 16-bit offsets from the window's start when every window
spans fewer than 65,536 entries (the default).  Both paths sum the same products in the same
order, so a run with every block staged, with none, and with a mix (a lowered capacity) must give
the same bits; the staged default is the path every other parity test exercises."""
import os

import numpy as np
import pytest

from oracle.monodomain import Monodomain
from paper_2510_12011_b300 import inputs as I
from paper_2510_12011_b300 import tc

pytestmark = pytest.mark.gpu


def _run(w, steps, precision, env):
    old = {k: os.environ.get(k) for k in env}
    os.environ.update({k: str(v) for k, v in env.items()})
    try:
        g = tc.from_workload(w, precision=precision)
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    info = g.staging()
    g.step(steps)
    out = (g.read(), g.activation_times(), info)
    g.close()
    return out


@pytest.mark.parametrize("precision", [tc.TC_FP64, tc.TC_FP32])
def test_staged_unstaged_and_mixed_windows_agree_bitwise(precision):
    # 20x8x3 mm at h = 0.25 (34,749 nodes): about 34 blocks of 1,024 threads
    w = I.slab_custom(20.0, 8.0, 3.0, 0.25, jitter=0.15, seed=9, fibre="rotating", dt=0.02, model="ms",
                      t_end=4.0)
    v1, a1, i1 = _run(w, 300, precision, {"TC_PCG_STAGE": 1})
    assert i1["staged_blocks"] == i1["blocks"] > 8 and i1["smem_bytes"] > 0 and i1["idx16"]
    v0, a0, i0 = _run(w, 300, precision, {})     # the default: no staging, 16-bit offsets
    assert i0["staged_blocks"] == 0 and i0["smem_bytes"] == 0 and i0["idx16"]
    # staged windows with 32-bit column indices, and neither
    v2, a2, i2 = _run(w, 300, precision, {"TC_PCG_STAGE": 1, "TC_PCG_IDX16": 0})
    assert i2["staged_blocks"] == i2["blocks"] and not i2["idx16"]
    v3, a3, i3 = _run(w, 300, precision, {"TC_PCG_IDX16": 0})
    assert i3["staged_blocks"] == 0 and not i3["idx16"]
    assert np.array_equal(v1, v2) and np.array_equal(a1, a2)
    assert np.array_equal(v1, v3) and np.array_equal(a1, a3)
    # a capacity of three quarters of the largest window: some blocks fit, some do not
    vm, am, im = _run(w, 300, precision, {"TC_PCG_STAGE": 1,
                                          "TC_PCG_STAGE_CAP": max(4, (i1["max_window"] * 3 // 4) // 4 * 4)})
    assert 0 < im["staged_blocks"] < im["blocks"] and im["idx16"]   # 16-bit offsets, some from global z
    assert np.array_equal(v1, v0) and np.array_equal(v1, vm)
    assert np.array_equal(a1, a0) and np.array_equal(a1, am)
    assert (a1 >= 0).sum() > 200


def test_staged_pcg_against_oracle_on_a_jittered_slab():
    """The staged path against the oracle on a mesh with several blocks (the small parity slab is
    a single block): 300 steps, parity mode."""
    w = I.slab_custom(12.0, 6.0, 3.0, 0.25, jitter=0.15, seed=5, fibre="rotating", dt=0.01, model="ms",
                      t_end=3.0)
    w.rtol, w.atol, w.max_iter = 1e-10, 0.0, 1000
    old = os.environ.get("TC_PCG_STAGE")
    os.environ["TC_PCG_STAGE"] = "1"
    try:
        g = tc.from_workload(w)
    finally:
        if old is None:
            os.environ.pop("TC_PCG_STAGE", None)
        else:
            os.environ["TC_PCG_STAGE"] = old
    info = g.staging()
    assert info["blocks"] > 4 and info["staged_blocks"] == info["blocks"]
    g.step(300)
    o = Monodomain(w).run(300)
    assert np.abs(g.read() - o.V).max() <= 1e-8
    assert np.array_equal(g.activation_times() >= 0, o.act >= 0)
    assert np.abs(g.activation_times() - o.act).max() <= 1e-6
