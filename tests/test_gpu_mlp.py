"""The surrogate's network on the GPU: the tensor-core (tcgen05) forward pass against the SIMT
reference, forward values and gradients against the FP64 oracle with the same BF16 rounding
points, the exact single-cell window against the oracle, and a short training run."""
import numpy as np
import pytest

from oracle import mlp as omlp
from oracle import tp06 as otp06
from paper_2510_12011_b300 import tc

pytestmark = pytest.mark.gpu


def _params(seed=0):
    rng = np.random.default_rng(seed)
    offs, total = omlp.layout()
    p = np.zeros(total)
    for l, (w, b) in enumerate(offs):
        fan = omlp.WIDTHS[l] + omlp.WIDTHS[l + 1]
        W = rng.uniform(-1, 1, (omlp.WIDTHS[l + 1], omlp.WIDTHS[l])) * np.sqrt(6.0 / fan)
        if l == 0:
            W[:, omlp.N_IN:] = 0.0
        if l == 4:
            W[omlp.N_OUT:, :] = 0.0
        p[w:b] = W.ravel()
        bias = rng.normal(0, 0.1, omlp.WIDTHS[l + 1])
        if l == 4:
            bias[omlp.N_OUT:] = 0.0
        p[b:b + omlp.WIDTHS[l + 1]] = bias
    return p.astype(np.float32)


@pytest.fixture(scope="module")
def net():
    m = tc.Mlp(seed=3)
    m.set_params(_params())
    return m


# Element-wise bounds of the GPU network against the oracle.  The oracle rounds to BF16 where the
# library stores BF16 (weights, hidden activations, the split input), so what is left between the
# two is rounding inside the last contraction and rounding carried into it: FP32 instead of FP64
# sums, the hardware tanh in the fused kernel's SiLU, a BF16 rounding of an activation that falls
# on the other side, and the BF16 copy of dZ that the tensor-core GEMMs read.  Each is a fraction
# of one BF16 unit (2^-8) of the terms it touches, and the errors that reach a result from
# earlier layers enter it through the same terms and partly cancel, so every output and every
# gradient entry is held to one BF16 unit of the sum of the absolute values of its terms:
#   |y_j - y_o,j| <= 2^-8 (sum_k |W_jk a_k| + |b_j|)   (last layer),
#   |g_ij - g_o,ij| <= 2^-8 sum_n |dz_ni a_nj|,   |g_i - g_o,i| <= 2^-8 sum_n |dz_ni|   (biases).
# A CPU emulation of the GPU's rounding points (FP32 sums, BF16 copies) stays below a quarter of
# these bounds; a wrong column, tile or sign is far outside them.
def _elementwise_bounds(p, x, t):
    y, (Ws, acts, zs) = omlp.forward(p, x, bf=True)
    offs, total = omlp.layout()
    b4 = p[offs[4][1]:offs[4][1] + omlp.WIDTHS[5]]
    by = 2.0 ** -8 * (np.abs(acts[4]) @ np.abs(Ws[4]).T + np.abs(b4))[:, :omlp.N_OUT]
    n = x.shape[0]
    dz = np.zeros((n, omlp.WIDTHS[-1]))
    dz[:, :omlp.N_OUT] = 2.0 * (y - t) / (n * omlp.N_OUT)
    bg = np.zeros(total)
    for l in range(4, -1, -1):
        w, b = offs[l]
        bg[w:b] = 2.0 ** -8 * (np.abs(dz).T @ np.abs(acts[l])).ravel()
        bg[b:b + omlp.WIDTHS[l + 1]] = 2.0 ** -8 * np.abs(dz).sum(axis=0)
        if l == 0:
            break
        dz = (dz @ Ws[l]) * omlp.silu_grad(zs[l - 1])
    return y, by, bg


def test_tensor_core_forward_matches_simt(net):
    rng = np.random.default_rng(5)
    x = rng.normal(size=(1000, 20)).astype(np.float32)    # 7 full 128-row tiles and a tail
    net.set_gemm(tc.Mlp.GEMM_SIMT)
    y_ref = net.forward(x)
    net.set_gemm(tc.Mlp.GEMM_TC)
    y_tc = net.forward(x)
    # each within the oracle's element-wise bound, so within twice of it of each other
    _, by, _ = _elementwise_bounds(net.params().astype(np.float64), x.astype(np.float64),
                                   np.zeros((1000, 19)))
    assert np.all(np.abs(y_tc - y_ref) <= 2.0 * by), np.max(np.abs(y_tc - y_ref) / by)


def test_forward_and_gradients_match_oracle(net):
    """Every output and every parameter gradient within its element-wise bound (above), for the
    tensor-core and the SIMT kernels (1000 rows: 7 full 128-row tiles and a ragged tail)."""
    rng = np.random.default_rng(6)
    x = rng.normal(size=(1000, 20)).astype(np.float32)
    t = rng.normal(size=(1000, 19)).astype(np.float32)
    p = net.params().astype(np.float64)
    y_o, by, bg = _elementwise_bounds(p, x.astype(np.float64), t.astype(np.float64))
    loss_o, g_o = omlp.loss_and_grads(p, x.astype(np.float64), t.astype(np.float64), bf=True)
    # the bounds are tight enough to matter: flipping the sign of most gradient entries breaks them
    assert (np.abs(g_o) > bg).mean() > 0.5
    for impl in (tc.Mlp.GEMM_TC, tc.Mlp.GEMM_SIMT):
        net.set_gemm(impl)
        y = net.forward(x)
        assert np.all(np.abs(y - y_o) <= by), (impl, np.max(np.abs(y - y_o) / by))
        loss, g = net.gradients(x, t)
        assert abs(loss - loss_o) <= 1e-3 * loss_o
        ok = np.abs(g - g_o) <= bg
        assert ok.all(), (impl, np.max(np.abs(g - g_o) / (bg + 1e-300)), int((~ok).sum()))
    net.set_gemm(tc.Mlp.GEMM_TC)


def test_window_matches_oracle():
    import torch
    n = 64
    V, u = otp06.rest(n)
    V = np.linspace(-86.0, 30.0, n)
    istim = np.where(np.arange(n) % 4 == 0, 20.0, 0.0)
    # [19][n] row-major: the entry point reads raw pointers, so the layout must be C order
    inp = np.ascontiguousarray(np.concatenate([u.T, V[None, :]], axis=0), dtype=np.float32)
    x = torch.tensor(inp, device="cuda")
    assert x.is_contiguous()
    s = torch.tensor(istim.astype(np.float32), device="cuda")
    out = torch.empty_like(x)
    tc.tp06_window(x.data_ptr(), s.data_ptr(), n, 0.02, 10, 2, tc.TC_FP64, out.data_ptr())
    got = out.cpu().numpy().astype(np.float64)
    uw, Vw = omlp.window(inp[:18].T.astype(np.float64), inp[18].astype(np.float64),
                         istim.astype(np.float32).astype(np.float64), 0.02, 10, 2)
    assert np.allclose(got[18], Vw, rtol=1e-6, atol=1e-5)
    assert np.allclose(got[:18].T, uw, rtol=1e-6, atol=1e-9)


def test_window_with_fast_concentration_changes_matches_oracle():
    """States whose Ki and Nai are small enough that a step changes them by more than 2^-20 of
    their value take the full log and I_K1 evaluation at u^{k+1} (the FP64 step otherwise carries
    the logarithms over from the evaluation at u^k); both kinds of node against the oracle."""
    import torch
    n = 96
    V, u = otp06.rest(n)
    V = np.linspace(-86.0, 20.0, n)
    small = np.arange(n) % 2 == 1
    u = u.copy()
    u[small, 0] = 0.5 + 0.01 * np.arange(small.sum())     # Ki, mM
    u[small, 1] = 0.05 + 0.001 * np.arange(small.sum())   # Nai, mM
    inp = np.ascontiguousarray(np.concatenate([u.T, V[None, :]], axis=0), dtype=np.float32)
    x = torch.tensor(inp, device="cuda")
    out = torch.empty_like(x)
    tc.tp06_window(x.data_ptr(), None, n, 0.02, 10, 2, tc.TC_FP64, out.data_ptr())
    got = out.cpu().numpy().astype(np.float64)
    uw, Vw = omlp.window(inp[:18].T.astype(np.float64), inp[18].astype(np.float64), np.zeros(n), 0.02, 10, 2)
    # the small-Ki nodes do move fast: more than 2^-20 relative per step on Ki or Nai
    rel = np.abs(uw[:, :2] - inp[:2].T) / inp[:2].T / 10
    assert np.all(rel[small].max(axis=1) > 2.0 ** -20) and np.all(rel[~small, 0] < 2.0 ** -20)
    assert np.allclose(got[18], Vw, rtol=1e-6, atol=1e-5)
    assert np.allclose(got[:18].T, uw, rtol=1e-6, atol=1e-9)


def test_short_training_reduces_loss():
    import torch
    rng = np.random.default_rng(7)
    n = 20000
    x = rng.normal(size=(n, 20)).astype(np.float32)
    y = (x[:, :19] + 0.1 * np.tanh(x[:, :19] * x[:, 1:20])).astype(np.float32)   # a smooth map
    xd = torch.tensor(x, device="cuda")
    yd = torch.tensor(y, device="cuda")
    m = tc.Mlp(seed=11)
    m.set_normalization(np.zeros(20), np.ones(20), np.zeros(19), 0.1 * np.ones(19))
    hist = m.train(xd.data_ptr(), yd.data_ptr(), n, epochs=6, batch=512, lr=2e-3)
    assert np.all(np.isfinite(hist)) and hist[-1] < 0.3 * hist[0], hist


@pytest.mark.parametrize("M,N,K", [(128, 256, 2048), (300, 64, 256), (256, 32, 4096), (1000, 256, 32), (7, 40, 200)])
def test_tensor_core_gemm_matches_fp32_reference(M, N, K):
    """The training pass's tcgen05 GEMM against a plain FP32 product of the same BF16 operands
    (several tiles, ragged M, N and K, K below one 64-wide panel, split-free)."""
    import torch
    g = torch.Generator().manual_seed(M * 7 + N * 3 + K)
    a = torch.randn(M, K, generator=g).to(torch.bfloat16)
    b = torch.randn(N, K, generator=g).to(torch.bfloat16)
    ref = (a.double() @ b.double().T).float()
    ad, bd = a.cuda(), b.cuda()
    c = torch.full((M, N), float("nan"), device="cuda")
    tc.gemm_bf16_nt(ad.data_ptr(), bd.data_ptr(), c.data_ptr(), M, N, K)
    got = c.cpu()
    assert torch.isfinite(got).all()
    tol = 1e-5 * K ** 0.5 * (a.float().abs().max() * b.float().abs().max()).item()
    assert (got - ref).abs().max().item() <= max(tol, 1e-4), (got - ref).abs().max().item()



def test_pipelined_forward_equals_single_tile_forward():
    """The forward kernel that keeps two row tiles in flight per CTA (warp-specialised producer,
    MMA and epilogue roles) issues the same MMAs in the same K order and the same epilogue as the
    one-tile kernel: bitwise the same outputs, for tile counts that are odd, even, a single ragged
    tile, and more than one pair per CTA; and the same gradients (the training forward stores
    the hidden layers)."""
    import os
    p = _params(seed=9)
    old = os.environ.get("TC_MLP_KERNEL")
    try:
        os.environ["TC_MLP_KERNEL"] = "1"
        m1 = tc.Mlp(seed=3)
    finally:
        if old is None:
            os.environ.pop("TC_MLP_KERNEL", None)
        else:
            os.environ["TC_MLP_KERNEL"] = old
    m2 = tc.Mlp(seed=3)
    m1.set_params(p)
    m2.set_params(p)
    rng = np.random.default_rng(12)
    for rows in (1, 127, 128, 129, 3 * 128 + 5, 148 * 2 * 128 * 2 + 77):
        x = rng.normal(size=(rows, 20)).astype(np.float32)
        assert np.array_equal(m1.forward(x), m2.forward(x)), rows
    x = rng.normal(size=(777, 20)).astype(np.float32)
    t = rng.normal(size=(777, 19)).astype(np.float32)
    l1, g1 = m1.gradients(x, t)
    l2, g2 = m2.gradients(x, t)
    # the loss is summed with FP32 atomics (its order varies run to run); the gradients are not
    assert abs(l1 - l2) <= 1e-6 * abs(l1) and np.array_equal(g1, g2)
