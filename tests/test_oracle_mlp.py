"""Pins of the oracle MLP: gradients against central finite differences (FP64, no rounding),
the BF16 rounding helper against exactly representable values, and the single-cell window
against the split step it is made of."""
import numpy as np

from oracle import mlp, tp06


def _params(seed=0):
    rng = np.random.default_rng(seed)
    offs, total = mlp.layout()
    p = np.zeros(total)
    for l, (w, b) in enumerate(offs):
        fan = mlp.WIDTHS[l] + mlp.WIDTHS[l + 1]
        p[w:b] = rng.uniform(-1, 1, b - w) * np.sqrt(6.0 / fan)
        p[b:b + mlp.WIDTHS[l + 1]] = rng.normal(0, 0.1, mlp.WIDTHS[l + 1])
    return p


def test_gradients_match_finite_differences():
    p = _params()
    rng = np.random.default_rng(1)
    x = rng.normal(size=(7, mlp.N_IN))
    t = rng.normal(size=(7, mlp.N_OUT))
    loss, g = mlp.loss_and_grads(p, x, t, bf=False)
    offs, _ = mlp.layout()
    picks = []
    for l, (w, b) in enumerate(offs):
        W = mlp.WIDTHS[l]
        picks += [w + 3 * W + 5, w + 17 * W + 1 if l < 4 else w + 2 * W + 9, b + 2]
    for i in picks:
        h = 1e-6
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (mlp.loss_and_grads(pp, x, t, bf=False)[0] - mlp.loss_and_grads(pm, x, t, bf=False)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_bf16_rounding():
    v = np.array([1.0, 1.0 + 2.0 ** -7, 1.0 + 2.0 ** -9, 1.0 + 3 * 2.0 ** -8, -2.5, 0.0])
    r = mlp.bf16(v)
    assert r[0] == 1.0 and r[1] == 1.0 + 2.0 ** -7 and r[4] == -2.5 and r[5] == 0.0
    assert r[2] == 1.0                       # below half an ulp rounds down
    assert r[3] == 1.0 + 2 * 2.0 ** -7       # a tie rounds to even


def test_window_is_repeated_split_step():
    V, u = tp06.rest(2)
    V[1] = -20.0
    istim = np.array([0.0, 10.0])
    uw, Vw = mlp.window(u, V, istim, 0.02, 10, 2)
    u2, V2 = u.copy(), V.copy()
    for _ in range(10):
        u2, i = tp06.step(V2, u2, 0.02, 2)
        V2 = V2 + 0.02 * (istim - i)
    assert np.array_equal(uw, u2) and np.array_equal(Vw, V2)


def test_split_input_resolves_sixteen_bits():
    """The two-BF16 input carries x to 16 significant bits: |hi + lo - x| <= 2^-16 |x|, where a
    single BF16 is off by up to 2^-9 |x| (values that are exact in FP32)."""
    x = np.random.default_rng(3).normal(size=20000).astype(np.float32).astype(np.float64)
    hi = mlp.bf16(x)
    lo = mlp.bf16(x - hi)
    assert np.all(np.abs(hi + lo - x) <= 2.0 ** -16 * np.abs(x))
    assert np.max(np.abs(hi - x) / np.abs(x)) > 2.0 ** -10
    p = _params()
    y, (_, acts, _) = mlp.forward(p, x[:20 * 50].reshape(50, 20), bf=True)
    assert np.array_equal(acts[0][:, :20], (hi + lo)[:1000].reshape(50, 20))

