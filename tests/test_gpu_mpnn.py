"""Learned surrogate on the GPU (sph_mpnn_*) against the FP64 reference
(oracle/mpnn.py).

* inputs: the node inputs and edge weights the CUDA path builds from a
  context's evaluation equal the reference's, built from the oracle's own
  evaluation of the same state (FP32 against FP64);
* forward: on the GPU's own inputs, the FP32 network equals the FP64
  reference to rel-L2 1e-5; the BF16 tensor-core path (8-bit mantissa
  operands, FP32 accumulation, about seven roundings deep) to 2e-2;
* backward: loss and every parameter gradient of the FP32 pass equal the
  FP64 reference's to rel-L2 1e-4;
* training: Adam on the GPU lowers the loss on a fixed state.
"""
import numpy as np
import pytest

from paper_1603_02421_gb300 import workloads as wl
from tests.helpers import ambiguous_mask, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sph():
    from paper_1603_02421_gb300 import binding, build
    build.build()
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    return binding


@pytest.fixture(scope="module")
def mp():
    from oracle import mpnn
    return mpnn


def _drop(seed=2):
    st = wl.disc(R=0.4, dx=0.02)
    rng = np.random.default_rng(seed)
    st["u"] = rng.normal(0, 0.05, len(st["x"]))
    st["v"] = rng.normal(0, 0.05, len(st["x"]))
    st["rho"] = st["rho"] * (1 + rng.uniform(-0.002, 0.002, len(st["x"])))
    p = wl.test_params(dx=0.02, sigma=0.05)
    p["capacity"] = len(st["x"]) + 64
    return p, st


@pytest.fixture(scope="module")
def evaluated(sph):
    p, st = _drop()
    sim = sph.Simulation({"params": p, "fluid": st, "boundary": None, "inflow": None})
    sim.evaluate()
    net = sph.Mpnn(capacity=len(st["x"]) + 64)
    yield p, st, sim, net
    net.close()
    sim.close()


def _params(seed):
    prm = wl.mpnn_init(seed)
    rng = np.random.default_rng(seed + 50)
    for k, v in prm.items():
        if v.ndim == 1:
            prm[k] = rng.normal(0.0, 0.05, v.shape)
    return prm


def _as_f32(prm):
    return {k: np.asarray(v, np.float32).astype(np.float64) for k, v in prm.items()}


def _gpu_inputs(sph, net, sim, n):
    ids, x, ea, eb, w = sph.sph_mpnn_features(net.net, sim.ctx, 1.0, n + 64, 64 * n)
    return ids, x.astype(np.float64), ea.astype(np.int64), eb.astype(np.int64), w.astype(np.float64)


def test_inputs_match_oracle(sph, mp, orc, evaluated):
    p, st, sim, net = evaluated
    n = len(st["x"])
    ids, x, ea, eb, w = _gpu_inputs(sph, net, sim, n)
    d = orc.derive(p)
    ev = orc.evaluate(d, st)
    xo, ao, bo, wo = mp.features(d, st, ev, 1.0)
    # the same ordered pairs
    ga, gb = ids[ea].astype(np.int64), ids[eb].astype(np.int64)
    key_g = ga * n + gb
    key_o = ao * n + bo
    og, oo = np.argsort(key_g), np.argsort(key_o)
    assert np.array_equal(key_g[og], key_o[oo])
    wg = w[og]
    wr = wo[oo]
    for c in range(4):
        assert rel_l2(wg[:, c], wr[:, c]) < 1e-5, c
    xg = np.zeros_like(x)
    xg[ids] = x
    keep = ~ambiguous_mask(orc, d, st, ev)
    assert rel_l2(xg[:, 0], xo[:, 0]) < 1e-4            # FP32 rho near rho0
    assert np.array_equal(xg[keep, 1], xo[keep, 1])     # Eq. 20 flags
    assert rel_l2(xg[:, 2], xo[:, 2]) < 1e-6
    assert rel_l2(xg[keep, 3], xo[keep, 3]) < 1e-5


@pytest.mark.parametrize("bf16,tol", [(False, 1e-5), (True, 2e-2)])
def test_forward_matches_reference(sph, mp, evaluated, bf16, tol):
    p, st, sim, net = evaluated
    n = len(st["x"])
    prm = _as_f32(_params(3))
    net.set_params(prm)
    ids, x, ea, eb, w = _gpu_inputs(sph, net, sim, n)
    ids2, y = sph.sph_mpnn_forward(net.net, sim.ctx, 1.0, bf16, n + 64)
    assert np.array_equal(ids, ids2)
    yr, _ = mp.forward(prm, x, ea, eb, w)
    assert np.abs(yr).max() > 0
    assert rel_l2(y[:, 0], yr[:, 0]) < tol and rel_l2(y[:, 1], yr[:, 1]) < tol


def test_gradients_match_reference(sph, mp, evaluated):
    p, st, sim, net = evaluated
    n = len(st["x"])
    prm = _as_f32(_params(4))
    net.set_params(prm)
    ids, x, ea, eb, w = _gpu_inputs(sph, net, sim, n)
    t = np.random.default_rng(6).normal(0.0, 1.0, (n, 2)).astype(np.float32)
    loss = sph.sph_mpnn_backward(net.net, sim.ctx, 1.0, t)
    g = net.grads()
    yr, cache = mp.forward(prm, x, ea, eb, w)
    lr_, dy = mp.loss(yr, t.astype(np.float64))
    gr = mp.backward(prm, cache, dy, ea, eb, w)
    assert abs(loss - lr_) <= 1e-5 * lr_
    for k in gr:
        assert rel_l2(g[k], gr[k]) < 1e-4, k


def test_training_lowers_the_loss(sph, evaluated):
    p, st, sim, net = evaluated
    n = len(st["x"])
    net.set_params(_params(7))
    s = sim.state()
    ids, _ = sph.sph_mpnn_forward(net.net, sim.ctx, 1.0, False, n + 64)
    a = np.stack([s["ax"], s["ay"]], 1)
    a_ref = a.std()
    order = np.argsort(s["id"])
    t = (a[order][ids] / a_ref).astype(np.float32)       # targets in cell order
    losses = []
    for _ in range(150):
        losses.append(sph.sph_mpnn_backward(net.net, sim.ctx, 1.0, t))
        sph.sph_mpnn_adam(net.net, 2e-3)
    assert losses[-1] < 0.3 * losses[0]


def test_layer_kernel_waits_are_bounded(sph):
    # the stall hook issues no operand loads, so every mbarrier wait of the
    # tensor-core layer kernels runs out (about a second each): the kernels
    # record ERR_TIMEOUT, free their tensor memory and return, the call
    # reports SPH_ERR_TIMEOUT, and the GPU stays usable
    import time
    p, st = _drop(5)
    n = len(st["x"])
    sim = sph.Simulation({"params": p, "fluid": st, "boundary": None, "inflow": None})
    sim.evaluate()
    net = sph.Mpnn(capacity=n + 64)
    net.set_params(_params(13))
    sph.sph_mpnn_inject_stall(net.net, 1)
    t0 = time.time()
    with pytest.raises(sph.SphError) as e:
        sph.sph_mpnn_forward(net.net, sim.ctx, 1.0, True, n + 64)
    assert e.value.status == -6
    assert time.time() - t0 < 60
    sph.sph_mpnn_inject_stall(net.net, 0)
    sim.close()
    fresh = sph.Simulation({"params": p, "fluid": st, "boundary": None, "inflow": None})
    fresh.evaluate()
    ids, y = sph.sph_mpnn_forward(net.net, fresh.ctx, 1.0, True, n + 64)
    assert len(ids) == n and np.all(np.isfinite(y))
    net.close()
    fresh.close()


def test_needs_an_evaluated_state(sph):
    p, st = _drop(5)
    sim = sph.Simulation({"params": p, "fluid": st, "boundary": None, "inflow": None})
    net = sph.Mpnn(capacity=len(st["x"]) + 64)
    with pytest.raises(sph.SphError) as ei:
        sph.sph_mpnn_forward(net.net, sim.ctx, 1.0, False, len(st["x"]) + 64)
    assert ei.value.status == sph.SPH_ERR_STATE
    sim.evaluate()
    sph.sph_mpnn_forward(net.net, sim.ctx, 1.0, False, len(st["x"]) + 64)
    sim.step()
    with pytest.raises(sph.SphError):
        sph.sph_mpnn_forward(net.net, sim.ctx, 1.0, False, len(st["x"]) + 64)
    net.close()
    sim.close()


# ---------------------------------------------------------------------------
# surrogate step (plain SPH as judge and fallback)
# ---------------------------------------------------------------------------
def _patch_case(seed):
    st = wl.jittered_patch(seed=seed, nx=40, ny=30, dx=0.02, vel=0.05, drho=0.002)
    p = wl.test_params(dx=0.02, sigma=0.05, box=(-0.5, -0.5, 1.3, 1.1))
    p["capacity"] = len(st["x"]) + 64
    p["skin_over_h"] = 0.3
    return {"params": p, "fluid": st, "boundary": None, "inflow": None}


def test_accepted_surrogate_step_applies_the_prediction(sph):
    case = _patch_case(3)
    sim = sph.Simulation(case)
    dt = sim.step()
    n = len(case["fluid"]["x"])
    net = sph.Mpnn(capacity=n + 64)
    net.set_params(_params(8))
    sim.evaluate()
    before = sim.state()
    t0 = sim.time()["t"]
    ids, y = sph.sph_mpnn_forward(net.net, sim.ctx, 1.0, True, n + 64)
    a_ref, k = 0.5, 4
    acc, rm, rd = sph.sph_surrogate_step(sim.ctx, net.net, k, 1.0, a_ref, 1e30, True)
    assert acc and rm > 0
    after = sim.state()
    dT = sim.time()["t"] - t0           # k times the Eq. 32 step at this state
    assert abs(dT - k * dt) < 0.05 * k * dt
    yb = np.zeros_like(y, dtype=np.float64)
    yb[ids] = y
    # the correction less its mass-weighted mean over the fluid
    fl = before["type"] == sph.FLUID
    ym = (before["m"][fl, None] * yb[fl]).sum(0) / before["m"][fl].sum()
    assert np.abs(ym).max() > 1e-3            # the removal is seen
    ax = before["ax"] + a_ref * (yb[:, 0] - ym[0])   # a_n + the network's correction
    ay = before["ay"] + a_ref * (yb[:, 1] - ym[1])
    u1 = before["u"] + dT * ax
    v1 = before["v"] + dT * ay
    x1 = before["x"] + dT * (before["u"] + 0.5 * dT * ax)
    y1 = before["y"] + dT * (before["v"] + 0.5 * dT * ay)
    rho1 = before["rho"] + dT * before["drho"]
    assert np.array_equal(after["id"], before["id"])
    assert np.allclose(after["x"], x1, rtol=0, atol=1e-9)
    assert np.allclose(after["y"], y1, rtol=0, atol=1e-9)
    assert rel_l2(after["u"], u1) < 1e-6 and rel_l2(after["v"], v1) < 1e-6
    assert np.allclose(after["rho"], rho1, rtol=1e-6, atol=0)
    net.close()
    sim.close()


def test_rejected_surrogate_step_equals_plain_steps(sph):
    case = _patch_case(4)
    a = sph.Simulation(case)
    b = sph.Simulation(case)
    a.step()
    b.step()
    n = len(case["fluid"]["x"])
    net = sph.Mpnn(capacity=n + 64)
    net.set_params(_params(9))
    acc, rm, rd = sph.sph_surrogate_step(a.ctx, net.net, 3, 1.0, 1.0, 1e-30, True)
    assert not acc
    b.run(3)
    assert a.time() == b.time()
    sa, sb = a.state(), b.state()
    for key in ("x", "y", "u", "v", "rho", "id"):
        assert np.array_equal(sa[key], sb[key]), key
    net.close()
    a.close()
    b.close()


def test_surrogate_steps_on_a_jet(sph):
    case = wl.jet(seed=2, dx=1.0 / 20, length=6.0, Re=200, We=20)
    case["params"]["skin_over_h"] = 0.3
    sim = sph.Simulation(case)
    sim.run(2)
    net = sph.Mpnn(capacity=case["params"]["capacity"])
    net.set_params(_params(10))
    t0 = sim.time()["t"]
    for _ in range(6):
        acc, rm, rd = sph.sph_surrogate_step(sim.ctx, net.net, 4, 1.0, 0.1, 1e30, True)
        assert acc
    assert sim.time()["t"] > t0
    sim.run(3)                      # plain steps continue from the surrogate's state
    s = sim.state()
    assert np.all(np.isfinite(s["x"])) and len(np.unique(s["id"])) == len(s["id"])
    net.close()
    sim.close()


def _by_id(st):
    o = np.argsort(st["id"])
    return {k: v[o] for k, v in st.items()}


def test_accepted_steps_reuse_the_end_evaluation(sph):
    # an accepted surrogate step's end evaluation starts the next one (no cell
    # build in between) and gives what a fresh start on rebuilt lists gives,
    # up to the FP32 order of the pair sums
    case = wl.jet(seed=3, dx=1.0 / 20, length=6.0, Re=200, We=20)
    case["params"]["skin_over_h"] = 0.3
    a, b = sph.Simulation(case), sph.Simulation(case)
    for sim in (a, b):
        sim.set_tuning(2, 8)
        sim.run(2)
    net = sph.Mpnn(capacity=case["params"]["capacity"])
    net.set_params(_params(11))
    builds = []
    for _ in range(3):
        acc, rm, rd = sph.sph_surrogate_step(a.ctx, net.net, 4, 1.0, 0.1, 1e30, True)
        assert acc
        builds.append(sph.sph_get_rebuild_stats(a.ctx)[0])
        sph.sph_request_rebuild(b.ctx)
        acc, rm, rd = sph.sph_surrogate_step(b.ctx, net.net, 4, 1.0, 0.1, 1e30, True)
        assert acc
    assert builds[2] == builds[0], builds     # steps 2 and 3 started from the reuse
    assert sph.sph_get_rebuild_stats(b.ctx)[0] >= builds[0] + 2
    assert a.time()["t"] == pytest.approx(b.time()["t"], rel=1e-6)
    sa, sb = _by_id(a.state()), _by_id(b.state())
    assert np.array_equal(sa["id"], sb["id"])
    assert np.max(np.abs(sa["x"] - sb["x"])) < 1e-7 and np.max(np.abs(sa["y"] - sb["y"])) < 1e-7
    assert rel_l2(sa["u"], sb["u"]) < 1e-4 and rel_l2(sa["v"], sb["v"]) < 1e-4
    assert rel_l2(sa["rho"] - case["params"]["rho0"], sb["rho"] - case["params"]["rho0"]) < 1e-3
    net.close()
    a.close()
    b.close()


def test_batched_steps_equal_single_steps(sph):
    # sph_surrogate_batch on two jets (one threshold rejecting, one
    # accepting) does what sph_surrogate_step does on each alone; the
    # FP64 sums of the mean removal and the residuals may differ in their
    # last bits (atomics), nothing more
    def jet(seed):
        c = wl.jet(seed=seed, dx=1.0 / 20, length=6.0, Re=200, We=20)
        c["params"]["skin_over_h"] = 0.3
        return c

    cases = [jet(6), jet(7)]
    single = [sph.Simulation(c) for c in cases]
    batch = [sph.Simulation(c) for c in cases]
    for sim in single + batch:
        sim.set_tuning(2, 8)
        sim.run(2)
    net = sph.Mpnn(capacity=max(c["params"]["capacity"] for c in cases))
    net.set_params(_params(12))
    for it, thr in enumerate((1e30, 1e30, 1e-30, 1e30)):
        acc, rm, rd, rf = sph.sph_surrogate_batch([s.ctx for s in batch], net.net, 4, 1.0, 0.1, thr)
        for i, sim in enumerate(single):
            a1, m1, d1, f1 = sph.sph_surrogate_step(sim.ctx, net.net, 4, 1.0, 0.1, thr, True,
                                                   field=True)
            assert a1 == acc[i], (it, i)
            assert m1 == pytest.approx(rm[i], rel=1e-6, abs=1e-12)
            assert d1 == pytest.approx(rd[i], rel=1e-6, abs=1e-15)
            assert f1 == pytest.approx(rf[i], rel=1e-6)
    for a, b in zip(single, batch):
        assert a.time()["t"] == b.time()["t"]
        sa, sb = _by_id(a.state()), _by_id(b.state())
        assert np.array_equal(sa["id"], sb["id"])
        assert np.max(np.abs(sa["x"] - sb["x"])) < 1e-9
        assert rel_l2(sa["u"], sb["u"]) < 1e-6 and rel_l2(sa["v"], sb["v"]) < 1e-6
    net.close()
    for sim in single + batch:
        sim.close()


def test_ensemble_surrogate_step_and_plain_steps_after_it(sph):
    # the ensemble's batched surrogate form: sph_ensemble_surrogate_step on
    # two members equals sph_surrogate_batch on twin contexts, and plain
    # ensemble steps continue from the surrogate's states (rebuilding first)
    def jet(seed):
        c = wl.jet(seed=seed, dx=1.0 / 20, length=6.0, Re=200, We=20)
        c["params"]["skin_over_h"] = 0.3
        return c

    cases = [jet(14), jet(15)]
    ens_sims = [sph.Simulation(c) for c in cases]
    twins = [sph.Simulation(c) for c in cases]
    for sim in ens_sims + twins:
        sim.set_tuning(2, 8)
    ens = sph.Ensemble(ens_sims)
    ens.run(2)
    for sim in twins:
        sim.run(2)
    net = sph.Mpnn(capacity=max(c["params"]["capacity"] for c in cases))
    net.set_params(_params(16))
    acc, rm, rd, rf = ens.surrogate_step(net.net, 4, 1.0, 0.1, 1e30)
    acc2, rm2, rd2, rf2 = sph.sph_surrogate_batch([s.ctx for s in twins], net.net, 4, 1.0, 0.1,
                                                   1e30)
    assert acc.all() and acc2.all()
    assert np.allclose(rm, rm2, rtol=1e-6) and np.allclose(rd, rd2, rtol=1e-6, atol=1e-15)
    ens.run(3)
    for sim in twins:
        sim.run(3)
    for a, b in zip(ens_sims, twins):
        assert a.time()["t"] == pytest.approx(b.time()["t"], rel=1e-12)
        sa, sb = _by_id(a.state()), _by_id(b.state())
        assert np.array_equal(sa["id"], sb["id"])
        assert np.all(np.isfinite(sa["u"]))
        assert np.max(np.abs(sa["x"] - sb["x"])) < 1e-9
        assert rel_l2(sa["u"], sb["u"]) < 1e-6
    ens.close()
    net.close()
    for sim in ens_sims + twins:
        sim.close()


def test_batch_names_the_failing_member(sph):
    # an FP64 context cannot take a surrogate step: the batch reports
    # SPH_ERR_ARG and names it before it touches any member
    case = wl.jet(seed=17, dx=1.0 / 20, length=6.0, Re=200, We=20)
    a = sph.Simulation(case)
    b = sph.Simulation(wl.jet(seed=18, dx=1.0 / 20, length=6.0, Re=200, We=20, prec="fp64"))
    a.run(2)
    b.run(2)
    net = sph.Mpnn(capacity=case["params"]["capacity"])
    net.set_params(_params(19))
    t0 = a.time()["t"]
    with pytest.raises(sph.SphError) as e:
        sph.sph_surrogate_batch([a.ctx, b.ctx], net.net, 4, 1.0, 0.1, 1e30)
    assert e.value.status == -1 and "member 1" in str(e.value)
    assert a.time()["t"] == t0
    net.close()
    a.close()
    b.close()


def test_trained_network_beats_the_instantaneous_acceleration(sph):
    # what the network gains: the k-step mean acceleration it predicts on
    # jets with (Re, We) it was not trained on is closer to the truth (k plain
    # steps) than the SPH acceleration at the step start alone
    from paper_1603_02421_gb300 import surrogate as sg

    def case(Re, We, seed):
        c = wl.jet(seed=seed, Re=Re, We=We, dx=1.0 / 20, length=8.0)
        c["params"]["skin_over_h"] = 0.3
        return c

    train = [case(200, 20, 0), case(400, 10, 1), case(100, 40, 2), case(700, 15, 3)]
    held = [case(300, 30, 4), case(150, 12, 5)]
    data = [(ci, s) for ci, c in enumerate(train) for s in sg.collect(c, 8, every=10)]
    test = [(ci, s) for ci, c in enumerate(held) for s in sg.collect(c, 4, every=10)]
    a_ref = sg.a_scale([s for _, s in data])
    cap = max(c["params"]["capacity"] for c in train + held)
    tr = sg.Trainer(train, cap)
    tr.train(data, a_ref, epochs=300, lr=1e-3)
    ev = sg.Trainer(held, cap)
    ev.net.set_params(tr.net.params())
    e_net, e_an = ev.prediction_errors(test, a_ref)
    assert e_net < 0.5 * e_an, (e_net, e_an)
    tr.close()
    ev.close()
