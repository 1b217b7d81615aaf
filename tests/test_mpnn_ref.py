"""Pins of the FP64 reference of the learned surrogate (oracle/mpnn.py).

The network is not in the paper; its reference is pinned by properties that
hold for any correct implementation of its definition: central finite
differences of the loss for every parameter tensor, the adjoint identity of
the neighbour aggregation, a closed form when the message-passing weights
vanish, relabelling equivariance, translation invariance of the features and
the Shepard identity that ties the first edge weight to the colour (Eq. 14).
"""
import numpy as np
import pytest

from paper_1603_02421_gb300 import workloads as wl


@pytest.fixture(scope="module")
def mp():
    from oracle import mpnn
    return mpnn


def _graph(seed, n=14, deg=5):
    rng = np.random.default_rng(seed)
    a, b = [], []
    for i in range(n):
        for j in rng.choice(n - 1, size=deg, replace=False):
            a.append(i)
            b.append(j if j < i else j + 1)
    a = np.array(a)
    b = np.array(b)
    w = rng.normal(0.0, 0.5, (len(a), 4))
    x = rng.normal(0.0, 1.0, (n, 4))
    t = rng.normal(0.0, 1.0, (n, 2))
    return x, a, b, w, t


def _params(seed):
    prm = wl.mpnn_init(seed)
    rng = np.random.default_rng(seed + 100)
    for k, v in prm.items():
        if v.ndim == 1:
            prm[k] = rng.normal(0.0, 0.1, v.shape)
    return prm


def test_gradients_match_finite_differences(mp):
    x, a, b, w, t = _graph(3)
    prm = _params(4)
    y, cache = mp.forward(prm, x, a, b, w)
    L0, dy = mp.loss(y, t)
    grads = mp.backward(prm, cache, dy, a, b, w)
    rng = np.random.default_rng(5)
    eps = 1e-6
    for name, g in grads.items():
        flat = prm[name].reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            keep = flat[idx]
            flat[idx] = keep + eps
            lp, _ = mp.loss(mp.forward(prm, x, a, b, w)[0], t)
            flat[idx] = keep - eps
            lm, _ = mp.loss(mp.forward(prm, x, a, b, w)[0], t)
            flat[idx] = keep
            fd = (lp - lm) / (2 * eps)
            an = g.reshape(-1)[idx]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (name, idx, fd, an)


def test_aggregation_adjoint(mp):
    x, a, b, w, t = _graph(7, n=20)
    rng = np.random.default_rng(8)
    z = rng.normal(size=(20, 32))
    dg = rng.normal(size=(20, 128))
    lhs = np.sum(mp.aggregate(z, a, b, w, 20) * dg)
    rhs = np.sum(z * mp.aggregate_T(dg, a, b, w, 20))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_no_message_passing_closed_form(mp):
    x, a, b, w, t = _graph(9)
    prm = _params(10)
    for l in range(mp.L):
        prm["U%d" % l][:] = 0.0
        prm["c%d" % l][:] = 0.0
    y, _ = mp.forward(prm, x, a, b, w)
    ref = np.maximum(x @ prm["W_in"] + prm["b_in"], 0.0) @ prm["D"] + prm["d"]
    assert np.allclose(y, ref, rtol=0, atol=1e-13)


def test_relabelling_equivariance(mp):
    x, a, b, w, t = _graph(11)
    prm = _params(12)
    y, _ = mp.forward(prm, x, a, b, w)
    perm = np.random.default_rng(13).permutation(len(x))
    inv = np.argsort(perm)
    y2, _ = mp.forward(prm, x[perm], inv[a], inv[b], w)
    assert np.allclose(y2, y[perm], rtol=0, atol=1e-12)


@pytest.fixture(scope="module")
def drop(orc):
    st = wl.disc(R=0.4, dx=0.02)
    rng = np.random.default_rng(2)
    st["u"] = rng.normal(0, 0.05, len(st["x"]))
    st["v"] = rng.normal(0, 0.05, len(st["x"]))
    st["rho"] = st["rho"] * (1 + rng.uniform(-0.002, 0.002, len(st["x"])))
    p = wl.test_params(dx=0.02, sigma=0.05)
    d = orc.derive(p)
    return d, st


def test_features_translation_invariant(mp, orc, drop):
    d, st = drop
    ev = orc.evaluate(d, st)
    x1, a1, b1, w1 = mp.features(d, st, ev, 1.0)
    st2 = dict(st, x=st["x"] + 0.3125, y=st["y"] - 0.1875)
    ev2 = orc.evaluate(d, st2)
    x2, a2, b2, w2 = mp.features(d, st2, ev2, 1.0)
    assert np.array_equal(a1, a2) and np.array_equal(b1, b2)
    assert np.allclose(w1, w2, rtol=0, atol=1e-9)
    assert np.allclose(x1, x2, rtol=0, atol=1e-9)


def test_first_edge_weight_is_colour_without_self(mp, orc, drop):
    d, st = drop
    ev = orc.evaluate(d, st)
    x, a, b, w = mp.features(d, st, ev, 1.0)
    s = np.bincount(a, weights=w[:, 0], minlength=len(st["x"]))
    Va = st["m"] / st["rho"]
    W0 = orc.W(d.kernel, 0.0, d.h)
    assert np.allclose(s + Va * W0, ev["C"], rtol=1e-12, atol=1e-12)
    assert np.allclose(x[:, 2], ev["C"])
