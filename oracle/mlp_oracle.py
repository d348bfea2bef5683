"""FP64 reference of the blow-up ranker network (TEST INFRASTRUCTURE).

Only the test suite and the benchmark's CPU leg use this module.  It is the plain
definition of the network the GPU kernels train, written in numpy float64 with the
backward pass derived by hand (checked against finite differences in the tests).

Network (a builder's choice: the paper has no learned component; it motivates
parametric blow-up studies in section 1):
    h1 = relu(x W1 + b1)       x: 6 features, W1: 6 x 128
    h2 = relu(h1 W2 + b2)      W2: 128 x 128
    z  = h2 W3 + b3            W3: 128 x 2; z0 = blow-up logit, z1 = predicted log t_b
Loss, mean over the batch of n rows, with y in {0, 1} the solver's blow-up flag,
l = log t_b of the blown-up runs and the censoring time T:
    BCE(z0, y) + y (z1 - l)^2 + (1 - y) relu(log T - z1)^2
(runs that did not blow up only say t_b > T, hence the one-sided term).
Adam: m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2, w -= lr m^ / (sqrt(v^) + eps)
with bias-corrected m^, v^.

bf16=True rounds to bfloat16 (round to nearest even) at the points where the GPU
kernels store bf16 values: the inputs, the weights, h1, h2, dz, dh2 and dh1.
"""
import numpy as np

D_IN, D_H, D_OUT = 6, 128, 2
SHAPES = {"W1": (D_IN, D_H), "b1": (D_H,), "W2": (D_H, D_H), "b2": (D_H,), "W3": (D_H, D_OUT), "b3": (D_OUT,)}
ORDER = ["W1", "b1", "W2", "b2", "W3", "b3"]


def bf16(a):
    """round float64 values to bfloat16 through float32, round to nearest even"""
    f = np.ascontiguousarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    nan = np.isnan(f)
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    out[nan] = np.nan
    return out.reshape(np.shape(a))


def init_params(seed=0):
    """He-style uniform initialisation from a seeded generator"""
    rng = np.random.default_rng(seed)
    p = {}
    for name in ORDER:
        shp = SHAPES[name]
        if name.startswith("W"):
            bound = np.sqrt(6.0 / shp[0])
            p[name] = rng.uniform(-bound, bound, size=shp)
        else:
            p[name] = np.zeros(shp)
    return p


def _r(a, on):
    return bf16(a) if on else a


def forward(p, x, bf16_points=False):
    x = _r(np.asarray(x, dtype=np.float64), bf16_points)
    W1, W2, W3 = (_r(p[k], bf16_points) for k in ("W1", "W2", "W3"))
    a1 = x @ W1 + p["b1"]
    h1 = _r(np.maximum(a1, 0.0), bf16_points)
    a2 = h1 @ W2 + p["b2"]
    h2 = _r(np.maximum(a2, 0.0), bf16_points)
    z = h2 @ W3 + p["b3"]
    return z, {"x": x, "h1": h1, "h2": h2, "a1": a1, "a2": a2, "W1": W1, "W2": W2, "W3": W3}


def sigmoid(t):
    return 0.5 * (1.0 + np.tanh(0.5 * t))


def loss_and_grads(p, x, y, ell, T=10.0, bf16_points=False):
    y = np.asarray(y, dtype=np.float64)
    ell = np.asarray(ell, dtype=np.float64)
    n = x.shape[0]
    z, c = forward(p, x, bf16_points)
    z0, z1 = z[:, 0], z[:, 1]
    logT = np.log(T)
    # BCE(z0, y) = softplus(z0) - y z0, written stably
    bce = np.maximum(z0, 0.0) - y * z0 + np.log1p(np.exp(-np.abs(z0)))
    cens = np.maximum(logT - z1, 0.0)
    loss = np.mean(bce + y * (z1 - ell) ** 2 + (1.0 - y) * cens ** 2)
    dz = np.empty_like(z)
    dz[:, 0] = (sigmoid(z0) - y) / n
    dz[:, 1] = (2.0 * y * (z1 - ell) - 2.0 * (1.0 - y) * cens) / n
    dz = _r(dz, bf16_points)
    g = {}
    g["W3"] = c["h2"].T @ dz
    g["b3"] = dz.sum(axis=0)
    dh2 = _r((dz @ c["W3"].T) * (c["a2"] > 0), bf16_points)
    g["W2"] = c["h1"].T @ dh2
    g["b2"] = dh2.sum(axis=0)
    dh1 = _r((dh2 @ c["W2"].T) * (c["a1"] > 0), bf16_points)
    g["W1"] = c["x"].T @ dh1
    g["b1"] = dh1.sum(axis=0)
    return loss, g


def adam_step(p, g, state, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k in ORDER:
        m = state.setdefault("m_" + k, np.zeros_like(p[k]))
        v = state.setdefault("v_" + k, np.zeros_like(p[k]))
        m[:] = b1 * m + (1 - b1) * g[k]
        v[:] = b2 * v + (1 - b2) * g[k] ** 2
        mh = m / (1 - b1 ** t)
        vh = v / (1 - b2 ** t)
        p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)
    return p


def flatten(p):
    return np.concatenate([np.asarray(p[k], dtype=np.float64).ravel() for k in ORDER])


def unflatten(v):
    out, o = {}, 0
    for k in ORDER:
        n = int(np.prod(SHAPES[k]))
        out[k] = np.asarray(v[o:o + n], dtype=np.float64).reshape(SHAPES[k])
        o += n
    return out


N_PARAMS = sum(int(np.prod(s)) for s in SHAPES.values())
