"""Ranker network on the GPU against the FP64 reference (oracle/mlp_oracle.py): forward,
gradients (the reference rounds to bf16 at the points the kernels store bf16), one
Adam step, a training run on a separable rule, and the Gaussian shell features."""
import numpy as np
import pytest

from oracle import mlp_oracle as M

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build_library()
    from paper_1501_04552_gb300 import kg as K
    yield K
    K.kg_mlp_finalize()


def params32(seed):
    p = M.init_params(seed)
    rng = np.random.default_rng(seed + 100)
    for k in ("b1", "b2", "b3"):
        p[k] = rng.normal(0.0, 0.05, size=M.SHAPES[k])
    flat = M.flatten(p).astype(np.float32)
    return flat, M.unflatten(flat.astype(np.float64))


def data(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, M.D_IN)).astype(np.float32)
    y = (rng.uniform(size=n) < 0.4).astype(np.float32)
    ell = rng.uniform(-0.5, 2.0, size=n).astype(np.float32)
    return X, y, ell


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, float) - np.asarray(b, float)) / max(np.linalg.norm(b), 1e-300))


def test_param_count(kg):
    assert kg.kg_mlp_param_count() == M.N_PARAMS


@pytest.mark.parametrize("n", [1, 127, 300, 1024])
def test_forward_matches_reference(kg, n):
    flat, p = params32(1)
    kg.kg_mlp_set_params(flat)
    X, _, _ = data(n, 2)
    prob, logt = kg.kg_mlp_predict(X)
    z, _ = M.forward(p, X.astype(np.float64), bf16_points=True)
    assert rel(logt, z[:, 1]) <= 5e-3
    assert np.abs(prob - M.sigmoid(z[:, 0])).max() <= 5e-3


def test_gradients_match_reference(kg):
    flat, p = params32(3)
    kg.kg_mlp_set_params(flat)
    X, y, ell = data(513, 4)
    loss, g = kg.kg_mlp_grad(X, y, ell, T=10.0)
    rl, rg = M.loss_and_grads(p, X.astype(np.float64), y, ell, T=10.0, bf16_points=True)
    assert abs(loss - rl) <= 1e-3 * abs(rl)
    gd = M.unflatten(g.astype(np.float64))
    for k in M.ORDER:
        assert rel(gd[k], rg[k]) <= 2e-2, (k, rel(gd[k], rg[k]))


# bf16 keeps 8 significant bits: each rounding to bf16 changes a value by at most
# u = 2^-8 relative.  The kernels round at 7 kinds of points (inputs, weights, h1, h2, dz,
# dh2, dh1); the longest chain from the inputs to a gradient -- forward through three
# layers, backward through two -- passes through at most 14 of them, and to first order
# the relative errors of a chain add.  FP32 accumulation adds nothing at this scale.
BF16_GRAD_BOUND = 14 * 2.0 ** -8


def test_gradients_against_unrounded_network(kg):
    """the GPU gradients against the FP64 network with no bf16 rounding anywhere (an oracle
    that does not mirror the kernels' rounding points), per tensor, to the bf16 bound"""
    flat, p = params32(3)
    kg.kg_mlp_set_params(flat)
    X, y, ell = data(513, 4)
    loss, g = kg.kg_mlp_grad(X, y, ell, T=10.0)
    rl64, rg64 = M.loss_and_grads(p, X.astype(np.float64), y, ell, T=10.0, bf16_points=False)
    assert abs(loss - rl64) <= BF16_GRAD_BOUND * abs(rl64)
    gd = M.unflatten(g.astype(np.float64))
    for k in M.ORDER:
        assert rel(gd[k], rg64[k]) <= BF16_GRAD_BOUND, (k, rel(gd[k], rg64[k]))
    assert rel(M.flatten(gd), M.flatten(rg64)) <= BF16_GRAD_BOUND


def test_adam_step_matches_reference(kg):
    flat, p = params32(5)
    kg.kg_mlp_set_params(flat)
    g = np.random.default_rng(6).standard_normal(M.N_PARAMS).astype(np.float32)
    for _ in range(3):
        kg.kg_mlp_adam_step(g, lr=2e-3)
    got = kg.kg_mlp_get_params()
    st = {}
    q = M.unflatten(flat.astype(np.float64))
    gd = M.unflatten(g.astype(np.float64))
    for _ in range(3):
        q = M.adam_step(q, gd, st, lr=2e-3)
    assert np.abs(got - M.flatten(q)).max() <= 1e-6


def test_training_learns_a_separable_rule(kg):
    rng = np.random.default_rng(7)
    n = 4096
    X = rng.uniform(-1.5, 1.5, size=(n, M.D_IN)).astype(np.float32)
    y = (X[:, 0] + 0.5 * X[:, 1] > 0.2).astype(np.float32)
    ell = (0.5 + 0.3 * X[:, 0]).astype(np.float32)
    flat, _ = params32(8)
    kg.kg_mlp_set_params(flat)
    l0, _ = kg.kg_mlp_grad(X, y, ell)
    final = kg.kg_mlp_train(X, y, ell, epochs=60, batch=256, lr=3e-3, T=10.0, seed=3)
    assert final < 0.3 * l0
    Xt = rng.uniform(-1.5, 1.5, size=(2048, M.D_IN)).astype(np.float32)
    yt = Xt[:, 0] + 0.5 * Xt[:, 1] > 0.2
    p, logt = kg.kg_mlp_predict(Xt)
    assert np.mean((p > 0.5) == yt) > 0.97
    assert np.abs(logt[yt] - (0.5 + 0.3 * Xt[yt, 0])).mean() < 0.1


def test_gaussian_features_match_oracle_and_instances(kg):
    from oracle import oracle as O
    from paper_1501_04552_gb300 import inputs as I
    A = np.array([0.7, 2.5, 3.9])
    s = np.array([0.6, 1.3, 1.95])
    f = kg.kg_gaussian_features(64, 32.0, A, s)
    for i in range(3):
        ref = O.shell_energies(I.gaussian(64, 32.0, A[i], s[i]), 32.0)
        assert np.allclose(f[i], ref, rtol=1e-11, atol=0), (i, f[i], ref)
