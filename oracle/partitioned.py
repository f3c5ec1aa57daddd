"""Row-partitioned Jacobi-PCG over cooperating ranks (oracle side of the multi-GPU design check;
test infrastructure only).

The hot path shards by rows: rank k owns a contiguous block of rows of A (after the node
ordering), its slices of x, r, z, p, q and of the Jacobi diagonal.  One CG iteration of
Algorithm 1 (Section 2.2) then needs two communication steps:
  * before q = A p, the entries of p in the columns a rank's rows reference outside its own
    block (its halo) - fetched here by an all-gather of every rank's p block;
  * each inner product (p^T q, r^T z, z^T z) is a local partial sum followed by an all-reduce.
Everything else is local.  With torch.distributed initialised (gloo on the host), `pcg_rank`
returns this rank's block of the solution; the single-partition `oracle.pcg.pcg` is the
reference it must reproduce up to the order of the dot-product additions.
"""
import numpy as np
import scipy.sparse as sp
import torch
import torch.distributed as dist


def row_blocks(n, parts):
    """Contiguous, near-equal row blocks: offsets[k] .. offsets[k+1] belong to rank k."""
    return np.linspace(0, n, parts + 1).round().astype(np.int64)


def halo(A_rows, lo, hi):
    """Columns referenced by a block of rows outside its own range [lo, hi)."""
    cols = np.unique(A_rows.indices)
    return cols[(cols < lo) | (cols >= hi)]


def _allreduce(v):
    t = torch.tensor([v], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def _gather_full(block, offsets):
    """The full vector from every rank's block (the halo exchange, done as an all-gather of
    blocks padded to the largest block's length)."""
    sizes = np.diff(offsets)
    m = int(sizes.max())
    mine = torch.zeros(m, dtype=torch.float64)
    mine[:block.size] = torch.from_numpy(np.ascontiguousarray(block))
    parts = [torch.zeros(m, dtype=torch.float64) for _ in sizes]
    dist.all_gather(parts, mine)
    return torch.cat([t[:int(sz)] for t, sz in zip(parts, sizes)]).numpy()


def pcg_rank(A, b, x0, diag, atol, rtol, max_iter, offsets):
    """This rank's share of Algorithm 1 (same readings as oracle.pcg): returns (x block,
    iterations, final ||z||, converged)."""
    k = dist.get_rank()
    lo, hi = int(offsets[k]), int(offsets[k + 1])
    A_rows = sp.csr_matrix(A)[lo:hi]
    d = diag[lo:hi]
    x_full = x0.copy()
    x = x0[lo:hi].copy()
    r = b[lo:hi] - A_rows @ x_full
    z = r / d
    p = z.copy()
    rho = _allreduce(float(r @ z))
    z0_norm = np.sqrt(_allreduce(float(z @ z)))
    if z0_norm == 0.0 or z0_norm < atol:
        return x, 0, z0_norm, True
    z_norm = z0_norm
    for it in range(max_iter):
        q = A_rows @ _gather_full(p, offsets)
        alpha = rho / _allreduce(float(p @ q))
        x = x + alpha * p
        r = r - alpha * q
        z = r / d
        z_norm = np.sqrt(_allreduce(float(z @ z)))
        if z_norm < atol or z_norm / z0_norm < rtol:
            return x, it + 1, z_norm, True
        rho_next = _allreduce(float(r @ z))
        beta = rho_next / rho
        p = z + beta * p
        rho = rho_next
    return x, max_iter, z_norm, False
