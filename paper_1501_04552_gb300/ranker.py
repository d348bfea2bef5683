"""Learned blow-up ranker: spend the solver near the blow-up boundary of (A, s).

The paper motivates parametric studies of blow-up in the cubic Klein-Gordon equation
(section 1: which initial data blow up is not understood, and parametric runs are the
way to map it).  This driver does such a study on 64^3 grids with initial data
u0 = A exp(-|x|^2/s^2), v0 = 0:

1. label runs with the solver (the batched ensemble of libkg.so): blow-up flag and
   blow-up time t_b (first level whose max|u| exceeds the threshold, times dt),
   censored at T;
2. train the network of kg_mlp_* on features (A, s, log of four low-mode shell
   energies at t = 0);
3. rank a Sobol sweep of (A, s) by |p - 1/2| and re-solve the top points with the
   solver, which judges every label the network predicts;
4. measure what the network gains: the share of judged points within a band of the
   solver's boundary A*(s) against the same number of uniform Sobol points, and the
   solver runs needed to bracket A*(s) to a given width with and without the network.

Every solver run, every network step and the feature extraction run on the GPU
through the C ABI; this module only orchestrates and scores.
"""
import time

import numpy as np

from . import inputs as I


class _LazyKg:
    """the C-ABI binding, loaded on first use (so the pure helpers import without it)"""

    def __getattr__(self, name):
        from . import kg as _k
        return getattr(_k, name)


kg = _LazyKg()

A_RANGE = (0.5, 4.0)
S_RANGE = (0.5, 2.0)
L_BOX = 32.0


# ---------------------------------------------------------------------------
# Sobol points, dimensions 1 and 2 (Bratley & Fox 1988; Joe & Kuo 2003): direction
# numbers v_k = m_k / 2^k with m_k = 1 for dimension 1 (van der Corput, base 2) and,
# for dimension 2 (primitive polynomial x + 1), m_1 = 1, m_k = 2 m_{k-1} xor m_{k-1};
# points in Gray-code order: x_n = x_{n-1} xor v_c, c = position of the lowest zero
# bit of n - 1.
# ---------------------------------------------------------------------------
def sobol2(n, skip=0):
    bits = 32
    v1 = [1 << (bits - k) for k in range(1, bits + 1)]
    m = [1]
    for _ in range(1, bits):
        m.append((2 * m[-1]) ^ m[-1])
    v2 = [m[k - 1] << (bits - k) for k in range(1, bits + 1)]
    out = np.empty((n, 2), dtype=np.float64)
    x1 = x2 = 0
    total = n + skip
    for i in range(total):
        if i > 0:
            c, j = 0, i - 1
            while j & 1:
                j >>= 1
                c += 1
            x1 ^= v1[c]
            x2 ^= v2[c]
        if i >= skip:
            out[i - skip, 0] = x1 / 2.0 ** bits
            out[i - skip, 1] = x2 / 2.0 ** bits
    return out


def to_params(u):
    A = A_RANGE[0] + (A_RANGE[1] - A_RANGE[0]) * u[:, 0]
    s = S_RANGE[0] + (S_RANGE[1] - S_RANGE[0]) * u[:, 1]
    return A, s


# ---------------------------------------------------------------------------
# solver runs
# ---------------------------------------------------------------------------
def solve(A, s, T, dt=0.005, N=64, threshold=1e3, chunk=1024, precision="df64"):
    """blow-up flags and times of the runs (A[i], s[i]) on N^3, by batched ensembles"""
    A = np.asarray(A, dtype=np.float64)
    s = np.asarray(s, dtype=np.float64)
    flags = np.zeros(A.size, dtype=bool)
    tb = np.full(A.size, np.inf)
    feats = np.empty((A.size, 4))
    steps = int(round(T / dt))
    kg.kg_set_options(precision=precision)
    inst_steps = 0
    t0 = time.perf_counter()
    for b in range(0, A.size, chunk):
        sl = slice(b, min(A.size, b + chunk))
        n = sl.stop - sl.start
        kg.kg_ens_init(np.full(n, N, dtype=np.int32), L_BOX, dt, A[sl], s[sl])
        kg.kg_ens_run(steps, threshold)
        r = kg.kg_ens_results()
        feats[sl] = kg.kg_ens_features()
        flags[sl] = r["frozen"]
        tb[sl] = np.where(r["frozen"], r["blowup_level"] * dt, np.inf)
        inst_steps += int(r["level"].sum())
    kg.kg_ens_finalize()
    return {"flag": flags, "tb": tb, "features": feats, "seconds": time.perf_counter() - t0,
            "instance_steps": inst_steps}


def features(A, s, shells):
    return np.column_stack([A, s, np.log(np.maximum(shells, 1e-300))])


class Standardizer:
    def __init__(self, X):
        self.mu = X.mean(axis=0)
        self.sd = X.std(axis=0) + 1e-12

    def __call__(self, X):
        return ((X - self.mu) / self.sd).astype(np.float32)


def auc(scores, labels):
    """area under the ROC curve by the rank statistic (ties averaged)"""
    labels = np.asarray(labels, dtype=bool)
    order = np.argsort(scores, kind="mergesort")
    ranks = np.empty(len(scores), dtype=np.float64)
    sorted_scores = np.asarray(scores)[order]
    i = 0
    while i < len(scores):
        j = i
        while j + 1 < len(scores) and sorted_scores[j + 1] == sorted_scores[i]:
            j += 1
        ranks[order[i:j + 1]] = 0.5 * (i + j) + 1
        i = j + 1
    npos, nneg = labels.sum(), (~labels).sum()
    if npos == 0 or nneg == 0:
        return float("nan")
    return float((ranks[labels].sum() - npos * (npos + 1) / 2) / (npos * nneg))


def init_params(seed):
    """He-uniform weights, zero biases, in the layout kg_mlp_* uses"""
    rng = np.random.default_rng(seed)
    shapes = [(6, 128), (128,), (128, 128), (128,), (128, 2), (2,)]
    out = []
    for shp in shapes:
        if len(shp) == 2:
            bound = np.sqrt(6.0 / shp[0])
            out.append(rng.uniform(-bound, bound, size=shp).ravel())
        else:
            out.append(np.zeros(shp))
    return np.concatenate(out).astype(np.float32)


def boundary_bisect(svals, T, width, lo=None, hi=None, dt=0.005, N=64, threshold=1e3, precision="df64"):
    """A*(s) to the given bracket width at every s, bisecting all s together (one batched
    solver call per round).  A bracket [lo, hi] means 'lo does not blow up by T, hi does'.
    A guessed bracket is checked first: if its lower end blows up the boundary lies in
    [A_min, lo]; if its upper end does not, it lies in [hi, A_max].  Without a guess the
    bracket is the whole range.  Returns (midpoints, solver runs used)."""
    svals = np.asarray(svals, dtype=np.float64)
    k = svals.size
    runs = 0
    if lo is None:
        lo = np.full(k, A_RANGE[0])
        hi = np.full(k, A_RANGE[1])
    else:
        lo = np.clip(np.asarray(lo, float), *A_RANGE)
        hi = np.clip(np.asarray(hi, float), *A_RANGE)
        r = solve(np.concatenate([lo, hi]), np.concatenate([svals, svals]), T, dt, N, threshold, precision=precision)
        runs += 2 * k
        lo_blows = r["flag"][:k]
        hi_quiet = ~r["flag"][k:]
        new_lo = np.where(lo_blows, A_RANGE[0], np.where(hi_quiet, hi, lo))
        new_hi = np.where(lo_blows, lo, np.where(hi_quiet, A_RANGE[1], hi))
        lo, hi = new_lo, new_hi
    while np.any(hi - lo > width):
        act = hi - lo > width
        mid = 0.5 * (lo + hi)
        r = solve(mid[act], svals[act], T, dt, N, threshold, precision=precision)
        runs += int(act.sum())
        blown = np.zeros(k, dtype=bool)
        blown[act] = r["flag"]
        hi = np.where(act & blown, mid, hi)
        lo = np.where(act & ~blown, mid, lo)
    return 0.5 * (lo + hi), runs


def predicted_boundary(std, svals, n_grid=701):
    """the smallest A on a fine grid where the network's p(A, s) reaches 1/2, per s"""
    Ag = np.linspace(A_RANGE[0], A_RANGE[1], n_grid)
    A = np.repeat(Ag[None, :], len(svals), axis=0).ravel()
    s = np.repeat(np.asarray(svals)[:, None], n_grid, axis=1).ravel()
    shells = kg.kg_gaussian_features(64, L_BOX, A, s)
    p, _ = kg.kg_mlp_predict(std(features(A, s, shells)))
    p = p.reshape(len(svals), n_grid)
    idx = np.argmax(p >= 0.5, axis=1)
    none = ~(p >= 0.5).any(axis=1)
    return np.where(none, A_RANGE[1], Ag[idx])


def run(n_train=4096, n_sweep=65536, n_judge=1024, T=10.0, dt=0.005, epochs=150, batch=256, lr=2e-3, seed=5,
        n_s=32, width=0.04, guess=0.1, band=0.1, precision="df64", held_out=0.2, log=None):
    """the whole study; returns a dict of measurements"""
    say = log or (lambda *a: None)
    out = {"n_train": n_train, "n_sweep": n_sweep, "n_judge": n_judge, "T": T, "dt": dt, "precision": precision}
    # 1. solver-labelled training runs, (A, s) uniform from a seeded stream
    u = I.uniform(seed, 2 * n_train).reshape(n_train, 2)
    A, s = to_params(u)
    lab = solve(A, s, T, dt, precision=precision)
    out["label_seconds"] = lab["seconds"]
    out["label_instance_steps"] = lab["instance_steps"]
    out["blowup_fraction"] = float(lab["flag"].mean())
    say("labelled %d runs in %.1f s, %.1f%% blew up" % (n_train, lab["seconds"], 100 * lab["flag"].mean()))
    X = features(A, s, lab["features"])
    y = lab["flag"].astype(np.float32)
    ell = np.where(lab["flag"], np.log(np.where(lab["flag"], lab["tb"], 1.0)), 0.0).astype(np.float32)
    n_hold = int(held_out * n_train)
    tr, ho = slice(n_hold, n_train), slice(0, n_hold)
    std = Standardizer(X[tr])
    kg.kg_mlp_set_params(init_params(seed))
    t0 = time.perf_counter()
    out["final_train_loss"] = kg.kg_mlp_train(std(X[tr]), y[tr], ell[tr], epochs=epochs, batch=batch, lr=lr, T=T,
                                              seed=seed)
    out["train_seconds"] = time.perf_counter() - t0
    p_ho, lt_ho = kg.kg_mlp_predict(std(X[ho]))
    out["heldout_auc"] = auc(p_ho, y[ho])
    out["heldout_accuracy"] = float(np.mean((p_ho > 0.5) == (y[ho] > 0.5)))
    blown = y[ho] > 0.5
    out["heldout_logt_mae"] = float(np.mean(np.abs(lt_ho[blown] - ell[ho][blown]))) if blown.any() else None
    say("held-out AUC %.4f, accuracy %.4f" % (out["heldout_auc"], out["heldout_accuracy"]))
    # 2. Sobol sweep ranked by closeness of p to 1/2
    us = sobol2(n_sweep, skip=1)
    As, ss = to_params(us)
    t0 = time.perf_counter()
    shells = kg.kg_gaussian_features(64, L_BOX, As, ss)
    ps, _ = kg.kg_mlp_predict(std(features(As, ss, shells)))
    out["sweep_infer_seconds"] = time.perf_counter() - t0
    top = np.argsort(np.abs(ps - 0.5), kind="mergesort")[:n_judge]
    uni = np.arange(n_judge)
    # 3. the solver judges every label the network predicts
    jt = solve(As[top], ss[top], T, dt, precision=precision)
    ju = solve(As[uni], ss[uni], T, dt, precision=precision)
    out["judged_label_accuracy_top"] = float(np.mean((ps[top] > 0.5) == jt["flag"]))
    out["judged_label_accuracy_uniform"] = float(np.mean((ps[uni] > 0.5) == ju["flag"]))
    # 4. the solver's boundary, and what the network saves in locating it
    svals = np.linspace(S_RANGE[0], S_RANGE[1], n_s)
    Astar, runs_plain = boundary_bisect(svals, T, width, dt=dt, precision=precision)
    Ahat = predicted_boundary(std, svals)
    Astar2, runs_mlp = boundary_bisect(svals, T, width, lo=Ahat - guess, hi=Ahat + guess, dt=dt,
                                       precision=precision)
    out["boundary_runs_plain"] = runs_plain
    out["boundary_runs_guided"] = runs_mlp
    out["boundary_max_disagreement"] = float(np.abs(Astar - Astar2).max())
    out["boundary_pred_mae"] = float(np.mean(np.abs(Ahat - Astar)))
    Ab = np.interp(ss, svals, Astar)
    near_top = np.abs(As[top] - Ab[top]) < band
    near_uni = np.abs(As[uni] - Ab[uni]) < band
    out["band"] = band
    out["near_boundary_fraction_top"] = float(near_top.mean())
    out["near_boundary_fraction_uniform"] = float(near_uni.mean())
    out["near_boundary_gain"] = float(near_top.mean() / max(near_uni.mean(), 1e-12))
    out["mixed_label_fraction_top"] = float(np.mean(jt["flag"]))
    say("near-boundary share: network %.3f vs uniform %.3f; boundary runs %d guided vs %d plain"
        % (near_top.mean(), near_uni.mean(), runs_mlp, runs_plain))
    return out


if __name__ == "__main__":
    import argparse
    import json
    import sys

    ap = argparse.ArgumentParser(description="learned blow-up ranker study on the GPU")
    ap.add_argument("--train", type=int, default=4096)
    ap.add_argument("--sweep", type=int, default=65536)
    ap.add_argument("--judge", type=int, default=1024)
    ap.add_argument("--T", type=float, default=10.0)
    ap.add_argument("--epochs", type=int, default=150)
    ap.add_argument("--precision", default="df64")
    a = ap.parse_args()
    res = run(n_train=a.train, n_sweep=a.sweep, n_judge=a.judge, T=a.T, epochs=a.epochs, precision=a.precision,
              log=lambda *m: print(*m, file=sys.stderr, flush=True))
    print(json.dumps(res), flush=True)
