"""FP64 reference of the ionic surrogate's multilayer perceptron (test infrastructure only).

The paper motivates learned and physics-based models side by side (Section 4, Section 5) but
specifies no network; the surrogate's network (20 -> 4 x 256 SiLU -> 19) is stated in the
package.  This module computes its forward pass, mean-squared-error loss and gradients by the
chain rule in FP64, with the parameter layout of the library (per layer W^T [out][in], then the
bias; widths padded 20 -> 32 and 19 -> 32).  With bf16=True it rounds where the GPU stores BF16
(weights, hidden activations, and the input as the sum of two BF16 numbers hi = bf16(x) and
lo = bf16(x - hi), the split the library feeds its first layer) so that the two can be compared
closely."""
import numpy as np

WIDTHS = [32, 256, 256, 256, 256, 32]
N_IN, N_OUT = 20, 19


def layout():
    offs, off = [], 0
    for l in range(5):
        w = off
        off += WIDTHS[l] * WIDTHS[l + 1]
        b = off
        off += WIDTHS[l + 1]
        offs.append((w, b))
    return offs, off


def bf16(x):
    """Round to bfloat16 (round to nearest even), returned as float64."""
    f = np.asarray(x, dtype=np.float32).copy()
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _unpack(params, round_w):
    offs, _ = layout()
    Ws, bs = [], []
    for l, (w, b) in enumerate(offs):
        W = params[w:b].astype(np.float64).reshape(WIDTHS[l + 1], WIDTHS[l])
        Ws.append(bf16(W) if round_w else W)
        bs.append(params[b:b + WIDTHS[l + 1]].astype(np.float64))
    return Ws, bs


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(params, x, bf=True):
    """x [n][20] normalized inputs -> (outputs [n][19], cache)."""
    Ws, bs = _unpack(params, bf)
    a = np.zeros((x.shape[0], WIDTHS[0]))
    a[:, :N_IN] = np.asarray(x, dtype=np.float32)
    if bf:
        hi = bf16(a)
        a = hi + bf16(a - hi)
    acts, zs = [a], []
    for l in range(5):
        z = acts[-1] @ Ws[l].T + bs[l]
        zs.append(z)
        if l < 4:
            h = silu(z)
            acts.append(bf16(h) if bf else h)
    return zs[-1][:, :N_OUT], (Ws, acts, zs)


def loss_and_grads(params, x, t, bf=True):
    """Mean squared error over the 19 outputs and its gradient (library layout)."""
    y, (Ws, acts, zs) = forward(params, x, bf)
    n = x.shape[0]
    d = y - t
    loss = float(np.mean(d * d))
    dz = np.zeros((n, WIDTHS[-1]))
    dz[:, :N_OUT] = 2.0 * d / (n * N_OUT)
    offs, total = layout()
    g = np.zeros(total)
    for l in range(4, -1, -1):
        w, b = offs[l]
        g[w:b] = (dz.T @ acts[l]).ravel()
        g[b:b + WIDTHS[l + 1]] = dz.sum(axis=0)
        if l == 0:
            break
        da = dz @ Ws[l]
        dz = da * silu_grad(zs[l - 1])
    # padding weights are held at zero by the library
    w0, _ = offs[0]
    g[w0:w0 + WIDTHS[1] * WIDTHS[0]].reshape(WIDTHS[1], WIDTHS[0])[:, N_IN:] = 0.0
    w4, b4 = offs[4]
    g[w4:b4].reshape(WIDTHS[5], WIDTHS[4])[N_OUT:, :] = 0.0
    g[b4 + N_OUT:b4 + WIDTHS[5]] = 0.0
    return loss, g


def window(u, V, istim, dt, nsub, cell):
    """Exact single-cell window (the targets): nsub split steps of TP06 with V advanced by
    forward Euler, dV/dt = -I_ion + I_stim (pA/pF)."""
    from . import tp06
    u = u.copy()
    V = V.copy()
    for _ in range(nsub):
        u, i_ion = tp06.step(V, u, dt, cell)
        V = V + dt * (istim - i_ion)
    return u, V
