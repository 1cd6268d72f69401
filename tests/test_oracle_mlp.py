"""Pins of the FP64 reference of the learned sampler (oracle/mlp.py): its
backpropagation against central finite differences, the GELU identities, its
bfloat16 rounding against torch's independent conversion, and Adam's first
step against its closed form."""
import math

import numpy as np
import pytest

from oracle import mlp


def _theta(seed=0, scale=0.3):
    r = np.random.default_rng(seed)
    return r.normal(0.0, scale, mlp.NPARAM)


def test_backprop_matches_finite_differences():
    r = np.random.default_rng(1)
    theta = _theta(1)
    X = r.uniform(-1, 1, (40, 2))
    t = r.normal(size=40)
    _, g = mlp.loss_and_grad(theta, X, t, round_bf16=False)
    idx = np.concatenate([r.choice(mlp.NPARAM - 1, 60, replace=False), [mlp.NPARAM - 1, 0, 128, 192, 4288]])
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        lp, _ = mlp.loss_and_grad(tp, X, t, round_bf16=False)
        lm, _ = mlp.loss_and_grad(tm, X, t, round_bf16=False)
        fd = (lp - lm) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-5, abs=1e-9), i


def test_gelu_identities_and_derivative():
    x = np.linspace(-6, 6, 101)
    assert np.allclose(mlp.gelu(x) - mlp.gelu(-x), x, atol=1e-14)  # tanh is odd
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    assert mlp.gelu(np.array([30.0]))[0] == pytest.approx(30.0)
    h = 1e-6
    fd = (mlp.gelu(x + h) - mlp.gelu(x - h)) / (2 * h)
    assert np.allclose(mlp.gelu_grad(x), fd, atol=1e-8)


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    r = np.random.default_rng(2)
    v = np.concatenate([r.normal(0, 3, 5000), [1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, -1 - 2 ** -8, 0.0, 65504.0]])
    ref = torch.tensor(v.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16(v), ref)
    assert mlp.bf16(np.array([1 + 2 ** -8]))[0] == 1.0          # tie to even
    assert mlp.bf16(np.array([1 + 3 * 2 ** -8]))[0] == 1 + 2 ** -6


def test_adam_first_step_is_signed_lr():
    theta = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    new, m, v = mlp.adam(theta, np.zeros(3), np.zeros(3), g, 1, 0.01)
    # bias-corrected first step: m/(sqrt(v)+eps) = g/|g| up to eps
    assert np.allclose(new, theta - 0.01 * np.sign(g), atol=1e-7)


def test_output_maps():
    u = np.array([1e-6, 0.3, 0.7, 0.999])
    y = np.array([0.2, -1.0, 0.4, 0.0])
    chi = np.array([1e-4, 1.0, 3.0, 5e3])  # the first and last outside [1e-3, 1e3]: clamped
    qs = mlp.output(0, y, chi, u, 1e-3, 1e3)
    L = np.log(np.clip(chi, 1e-3, 1e3) / (1 + np.clip(chi, 1e-3, 1e3)))
    assert L[1] == pytest.approx(-math.log(2.0)) and L[0] == pytest.approx(math.log(1e-3 / 1.001))
    assert np.all(qs < 1.0) and np.allclose(np.log(qs / (1 - qs)), y + 3 * np.log(u) + L)
    # the map inverts the targets
    t = mlp.targets(0, chi, u, qs, 1e-3, 1e3)
    assert np.allclose(t, y)
    # BW: w(chi) -> sqrt(3 chi / 64) for small chi, 1/2 for large
    w = mlp.centre_scale(1, np.array([1e-6, 1e9]), 1e-6, 1e9)
    assert w[0] == pytest.approx(math.sqrt(3e-6 / 64), rel=1e-6) and w[1] == pytest.approx(0.5, rel=1e-8)
    chib = np.array([0.02, 1.0, 16.0 / 3.0, 1e3])
    yb = np.array([0.2, 0.7, -0.1, 3.0])
    bw = mlp.output(1, yb, chib, u, 0.02, 1e3)
    wb = 0.5 * np.sqrt(chib / (chib + 16.0 / 3.0))
    assert wb[2] == pytest.approx(0.5 / math.sqrt(2.0))
    # the logit of the folded split is 4 w y; y < 0 clamps at 1/2
    assert bw[2] == 0.5 and np.all(bw <= 0.5)
    k = [0, 1, 3]
    assert np.allclose(np.log((1 - bw[k]) / bw[k]), 4 * wb[k] * yb[k], rtol=1e-12)
    # near 1/2 the map is 1/2 - w y to first order (the linear map of a narrow split)
    eps = 1e-4
    near = mlp.output(1, np.array([eps]), np.array([0.1]), np.array([0.3]), 0.02, 1e3)[0]
    w01 = 0.5 * math.sqrt(0.1 / (0.1 + 16.0 / 3.0))
    assert abs(near - (0.5 - w01 * eps)) < 1e-3 * w01 * eps
    # at large chi it resolves the crowded small splits: y = ln((1 - xi_s) / xi_s) / (4 w)
    assert bw[3] == pytest.approx(1.0 / (1.0 + math.exp(4 * wb[3] * 3.0)), rel=1e-12) and bw[3] < 3e-3
    # targets take the electron's fraction and fold it by U, and invert the map
    xe = np.where(u <= 0.5, bw, 1 - bw)
    tb = mlp.targets(1, chib, u, xe, 0.02, 1e3)
    assert np.allclose(tb[k], yb[k], rtol=1e-9) and tb[2] == 0.0
    X = mlp.features(1, [1e-5, 1.0, 1e9], [0.2, 0.9, 0.5], 0.02, 1e3)
    assert X[0, 0] == -1.0 and X[2, 0] == 1.0
    assert np.allclose(X[:, 1], [2 * 0.4 - 1, 2 * 0.2 - 1, 1.0])
