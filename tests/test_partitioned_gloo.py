"""Multi-GPU design check on host ranks: the row-partitioned PCG (halo exchange before every
A-product, all-reduced inner products) reproduces the single-partition solve of the small
slab's system to 1e-13, with the same iteration count, for 2 and 3 ranks (gloo, CPU)."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _system():
    from oracle import fem
    from paper_2510_12011_b300 import inputs
    w = inputs.slab_small_ms()
    M, K = fem.mass_stiffness(w.mesh.xyz, w.mesh.tets, w.mesh.fibres, w.sigma_l, w.sigma_t)
    A = fem.system_matrix(M, K, w.chi, w.cm, w.theta, w.dt)
    n = A.shape[0]
    rng = np.random.default_rng(8)
    x_true = rng.normal(size=n)
    return A, A @ x_true, rng.normal(size=n), A.diagonal()


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import partitioned
    A, b, x0, d = _system()
    offs = partitioned.row_blocks(A.shape[0], world)
    x, it, zn, ok = partitioned.pcg_rank(A, b, x0, d, 0.0, 1e-12, 500, offs)
    out[rank] = (x, it, ok)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_partitioned_pcg_matches_single_partition(world):
    from oracle.pcg import pcg
    A, b, x0, d = _system()
    x_ref, it_ref, _, ok_ref = pcg(A, b, x0, d, 0.0, 1e-12, 500)
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    x = np.concatenate([out[r][0] for r in range(world)])
    assert all(out[r][1] == it_ref and out[r][2] for r in range(world)) and ok_ref
    assert np.max(np.abs(x - x_ref)) <= 1e-13 * np.max(np.abs(x_ref))


def test_halo_is_the_off_block_columns():
    import scipy.sparse as sp
    from oracle import partitioned
    A = sp.diags([np.ones(9), np.ones(10), np.ones(9)], [-1, 0, 1], format="csr")
    offs = partitioned.row_blocks(10, 2)
    assert list(offs) == [0, 5, 10]
    assert list(partitioned.halo(A[0:5], 0, 5)) == [5]
    assert list(partitioned.halo(A[5:10], 5, 10)) == [4]
