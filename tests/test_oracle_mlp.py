"""Pins of the FP64 ranker-network reference: analytic gradients against central
finite differences, bf16 rounding against torch's bfloat16 conversion, the loss in
closed-form special cases, and Adam's first step."""
import math

import numpy as np
import pytest

from oracle import mlp_oracle as M


def batch(n=37, seed=3):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((n, M.D_IN))
    y = (rng.uniform(size=n) < 0.5).astype(float)
    ell = rng.uniform(-1.0, 2.0, size=n)
    return x, y, ell


def test_gradients_match_finite_differences():
    p = M.init_params(1)
    for k in ["b1", "b2", "b3"]:
        p[k] = np.random.default_rng(7).normal(0, 0.1, size=M.SHAPES[k])
    x, y, ell = batch()
    _, g = M.loss_and_grads(p, x, y, ell)
    flat = M.flatten(p)
    gflat = M.flatten(g)
    rng = np.random.default_rng(11)
    idx = rng.choice(flat.size, size=80, replace=False)
    h = 1e-6
    for i in idx:
        a, b = flat.copy(), flat.copy()
        a[i] += h
        b[i] -= h
        fd = (M.loss_and_grads(M.unflatten(a), x, y, ell)[0] - M.loss_and_grads(M.unflatten(b), x, y, ell)[0]) / (2 * h)
        assert abs(fd - gflat[i]) <= 1e-7 + 1e-5 * abs(fd), (i, fd, gflat[i])


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    v = np.random.default_rng(0).standard_normal(4096) * 10.0 ** np.random.default_rng(1).integers(-8, 8, 4096)
    v = np.concatenate([v, [0.0, -0.0, 1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, 65504.0, 3e38]])
    ref = torch.tensor(v.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(M.bf16(v), ref)


def test_loss_special_cases():
    p = {k: np.zeros(M.SHAPES[k]) for k in M.ORDER}
    p["b3"] = np.array([0.0, math.log(10.0)])     # z = (0, log T) for every row
    x = np.ones((4, M.D_IN))
    y = np.array([1.0, 0.0, 1.0, 0.0])
    ell = np.array([math.log(10.0), 0.0, math.log(10.0) - 1.0, 5.0])
    loss, _ = M.loss_and_grads(p, x, y, ell, T=10.0)
    # BCE at z0 = 0 is log 2 for every row; squared errors 0, 0 (censored, z1 = log T), 1, 0
    assert abs(loss - (math.log(2.0) + 1.0 / 4)) < 1e-15


def test_adam_first_step_is_a_signed_learning_rate_step():
    p = M.init_params(2)
    g = {k: np.random.default_rng(5).standard_normal(M.SHAPES[k]) for k in M.ORDER}
    q = M.adam_step({k: v.copy() for k, v in p.items()}, g, {}, lr=1e-3)
    for k in M.ORDER:
        step = p[k] - q[k]
        assert np.allclose(step, 1e-3 * g[k] / (np.abs(g[k]) + 1e-8), rtol=1e-12, atol=1e-18)


def test_bf16_points_change_the_forward_only_at_bf16_level():
    p = M.init_params(4)
    x, _, _ = batch(64, 9)
    z, _ = M.forward(p, x)
    zb, _ = M.forward(p, x, bf16_points=True)
    assert np.abs(z - zb).max() <= 0.05 * np.abs(z).max()
