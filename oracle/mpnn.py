"""FP64 CPU reference of the learned surrogate network (message passing on
the SPH neighbour graph).

TEST INFRASTRUCTURE ONLY.  Only the test suite may import this module; the
product path (the CUDA library and its binding) never imports or runs it,
and the two share no code.

The paper has no learned part; this network is the surrogate of the build
(a 3-layer message-passing network of width 128 that predicts a particle's
mean acceleration over the next k substeps).  Its definition, which the
CUDA kernels implement:

  node inputs   x_a = [100 (rho_a/rho0 - 1), N_a (Eq. 20 flag), C_a (Eq. 14),
                       h |n_a| (Eq. 18)]
  edge weights  over ordered pairs a != b with r_ab < 2h (Sec. 2-7), with
                V_b = m_b / rho_b, W and F = (1/r) dW/dr of Eqs. 27-28:
                  w0 = V_b W_ab
                  w1 = V_b F_ab (x_a - x_b) h
                  w2 = V_b F_ab (y_a - y_b) h
                  w3 = V_b F_ab ((u_a - u_b).(r_a - r_b)) h / U_ref
  layers        h0 = relu(x W_in + b_in)
                for l = 0, 1, 2:
                  z = h Pi_l                                   (N x 32)
                  g_a[32k + j] = sum_b w_k,ab z_b[j], k = 0..3  (N x 128)
                  h = h + relu([h, g] U_l + c_l)
                y = h D + d                                    (N x 2)
  loss          L = (1/N) sum_a |y_a - t_a|^2

All arithmetic here is float64 numpy with no blocking or reordering beyond
the definitions above.
"""
from __future__ import annotations

import math

import numpy as np

from . import oracle as orc

H, P, L = 128, 32, 3


def relu(v):
    return np.maximum(v, 0.0)


def features(d, st, ev, U_ref):
    """Node inputs and edge weights from an oracle state and its evaluation.

    Returns (x[N,4], a[E], b[E], w[E,4]) with the pairs in the order of the
    oracle's neighbour lists (ascending a, then ascending b)."""
    n = len(st["x"])
    h = d.h
    x = np.zeros((n, 4))
    x[:, 0] = 100.0 * (st["rho"] / d.rho0 - 1.0)
    x[:, 1] = ev["N"].astype(np.float64)
    x[:, 2] = ev["C"]
    x[:, 3] = h * np.hypot(ev["nx"], ev["ny"])
    start, lst = orc.neighbours(st["x"], st["y"], 2.0 * h)
    a = np.repeat(np.arange(n), np.diff(start))
    b = lst.astype(np.int64)
    rx = st["x"][a] - st["x"][b]
    ry = st["y"][a] - st["y"][b]
    r = np.sqrt(rx * rx + ry * ry)
    Vb = st["m"][b] / st["rho"][b]
    Wv = np.array([orc.W(d.kernel, ri, h) for ri in r])
    Fv = np.array([orc.dWdr(d.kernel, ri, h) / ri if ri > 0 else 0.0 for ri in r])
    du = st["u"][a] - st["u"][b]
    dv = st["v"][a] - st["v"][b]
    w = np.zeros((len(a), 4))
    w[:, 0] = Vb * Wv
    w[:, 1] = Vb * Fv * rx * h
    w[:, 2] = Vb * Fv * ry * h
    w[:, 3] = Vb * Fv * (du * rx + dv * ry) * h / U_ref
    return x, a, b, w


def aggregate(z, a, b, w, n):
    """g_a[32k + j] = sum over pairs (a, b) of w_k,ab z_b[j]."""
    g = np.zeros((n, 4, z.shape[1]))
    for k in range(4):
        np.add.at(g[:, k, :], a, w[:, k:k + 1] * z[b])
    return g.reshape(n, 4 * z.shape[1])


def aggregate_T(dg, a, b, w, n):
    """Adjoint of aggregate: dz_b[j] = sum over pairs (a, b) of
    sum_k w_k,ab dg_a[32k + j]."""
    p = dg.shape[1] // 4
    dg4 = dg.reshape(n, 4, p)
    dz = np.zeros((n, p))
    for k in range(4):
        np.add.at(dz, b, w[:, k:k + 1] * dg4[a, k, :])
    return dz


def forward(prm, x, a, b, w):
    n = x.shape[0]
    cache = {"x": x}
    pre0 = x @ prm["W_in"] + prm["b_in"]
    h = relu(pre0)
    cache["pre_in"] = pre0
    hs = [h]
    for l in range(L):
        z = h @ prm["Pi%d" % l]
        g = aggregate(z, a, b, w, n)
        cat = np.concatenate([h, g], axis=1)
        pre = cat @ prm["U%d" % l] + prm["c%d" % l]
        h = h + relu(pre)
        cache["z%d" % l] = z
        cache["cat%d" % l] = cat
        cache["pre%d" % l] = pre
        hs.append(h)
    cache["h"] = hs
    y = h @ prm["D"] + prm["d"]
    return y, cache


def loss(y, t):
    n = y.shape[0]
    diff = y - t
    return float(np.sum(diff * diff) / n), 2.0 * diff / n


def backward(prm, cache, dy, a, b, w):
    n = dy.shape[0]
    grads = {}
    hs = cache["h"]
    grads["D"] = hs[L].T @ dy
    grads["d"] = dy.sum(axis=0)
    dh = dy @ prm["D"].T
    for l in reversed(range(L)):
        pre = cache["pre%d" % l]
        dpre = dh * (pre > 0.0)
        grads["U%d" % l] = cache["cat%d" % l].T @ dpre
        grads["c%d" % l] = dpre.sum(axis=0)
        dcat = dpre @ prm["U%d" % l].T
        dh_prev = dh + dcat[:, :H]
        dg = dcat[:, H:]
        dz = aggregate_T(dg, a, b, w, n)
        grads["Pi%d" % l] = hs[l].T @ dz
        dh = dh_prev + dz @ prm["Pi%d" % l].T
    dpre0 = dh * (cache["pre_in"] > 0.0)
    grads["W_in"] = cache["x"].T @ dpre0
    grads["b_in"] = dpre0.sum(axis=0)
    return grads
