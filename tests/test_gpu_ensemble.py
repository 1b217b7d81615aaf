"""Ensembles (sph_ensemble_*): several jets with different dx, Re, We, seeds
and particle counts advanced by one CUDA graph launch per ensemble step.

Each member runs the kernels a solo run of the same case runs, in the same
order on the same data, so after any number of ensemble steps its state is
bit-identical to the solo run's; the solo runs are themselves held to the
oracle by the parity tests, and one member is also compared with the oracle
directly here.
"""
import numpy as np
import pytest

from paper_1603_02421_gb300 import workloads as wl
from tests.helpers import oracle_sim, rel_l2, rel_l2_vec

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sph():
    from paper_1603_02421_gb300 import binding, build
    build.build()
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    return binding


# (seed, Re, We, dx, length, lanes, cadence, start form): uneven sizes, mixed
# tunings, both ways of picking a step's start on the device
MEMBERS = [
    (0, 100, 10, 1.0 / 12, 10.0, 4, 1, 0),
    (1, 200, 20, 1.0 / 20, 6.0, 2, 8, 1),
    (2, 400, 40, 1.0 / 16, 12.0, 8, 4, 0),
    (3, 700, 5, 1.0 / 24, 5.0, 1, 2, 1),
]


def _case(seed, Re, We, dx, length):
    case = wl.jet(seed=seed, Re=Re, We=We, dx=dx, length=length)
    case["params"]["skin_over_h"] = 0.3
    return case


def _make(sph, spec):
    seed, Re, We, dx, length, lanes, cadence, form = spec
    sim = sph.Simulation(_case(seed, Re, We, dx, length))
    sim.set_tuning(lanes, cadence)
    sim.set_start_form(form)
    return sim


def _same(a, b):
    for k in ("x", "y", "u", "v", "rho", "id", "type"):
        if not np.array_equal(a[k], b[k]):
            return False
    return True


def test_members_match_solo_runs_bit_for_bit(sph):
    sims = [_make(sph, m) for m in MEMBERS]
    sizes = [len(s.state()["x"]) for s in sims]
    assert len(set(sizes)) == len(sizes)           # uneven particle counts
    ens = sph.Ensemble(sims)
    ens.run(60)
    for spec, sim in zip(MEMBERS, sims):
        solo = _make(sph, spec)
        solo.run(60)
        assert sim.time() == solo.time()
        assert _same(sim.state(), solo.state()), spec
        solo.close()
    # a second batch after a member was stepped on its own (host and device
    # step bookkeeping stay consistent across the two paths)
    sims[1].run(5)
    ens.run(20)
    solo = _make(sph, MEMBERS[1])
    solo.run(85)
    assert _same(sims[1].state(), solo.state())
    ens.close()


def test_member_against_oracle(sph, orc):
    # one member held to the FP64 oracle directly (fixed dt, so the step
    # sequence is the same on both sides)
    cases = [_case(5, 200, 20, 1.0 / 20, 6.0), _case(6, 100, 10, 1.0 / 14, 8.0)]
    cases[0]["params"]["dt_fixed"] = 1e-3
    sims = [sph.Simulation(c) for c in cases]
    sims[0].set_tuning(2, 4)
    ens = sph.Ensemble(sims)
    ens.run(100)
    osim = oracle_sim(orc, cases[0])
    osim.run(100)
    g = sims[0].state()
    st = osim.st
    assert np.array_equal(g["id"], st["id"].astype(np.uint32))
    assert rel_l2_vec(g["x"], g["y"], st["x"], st["y"]) < 1e-4
    assert rel_l2_vec(g["u"], g["v"], st["u"], st["v"]) < 1e-4
    assert rel_l2(g["rho"], st["rho"]) < 1e-4
    ens.close()


def test_retuned_member_is_recaptured(sph):
    sims = [_make(sph, m) for m in MEMBERS[:2]]
    ens = sph.Ensemble(sims)
    ens.run(10)
    sims[0].set_tuning(2, 4)          # changes the captured step of member 0
    sims[1].set_start_form(sph.START_GATED)   # and the start form of member 1
    ens.run(30)
    b0 = sims[0].rebuild_stats()[0]
    ens.run(16)
    assert sims[0].rebuild_stats()[0] - b0 < 16   # cadence 4 now reuses builds
    solo = _make(sph, MEMBERS[0])
    solo.run(10)
    solo.set_tuning(2, 4)
    solo.run(46)
    assert _same(sims[0].state(), solo.state())
    solo = _make(sph, MEMBERS[1])
    solo.run(10)
    solo.set_start_form(sph.START_GATED)
    solo.run(46)
    assert _same(sims[1].state(), solo.state())
    ens.close()


def test_error_names_the_member(sph):
    sims = [_make(sph, m) for m in MEMBERS[:3]]
    bad = _case(9, 200, 20, 1.0 / 20, 6.0)
    probe = sph.Simulation(bad)
    n0 = probe.time()["n"]                # fluid + inflow buffer layers
    probe.close()
    # no room for another inflow layer: the first spawn raises a capacity error
    bad["params"]["capacity"] = n0
    sims.insert(2, sph.Simulation(bad))
    ens = sph.Ensemble(sims)
    with pytest.raises(sph.SphError) as ei:
        ens.run(120)
    assert ei.value.member == 2
    assert ei.value.status == sph.SPH_ERR_CAPACITY
    ens.close()


def test_autotune_restores_states(sph):
    sims = [_make(sph, m) for m in MEMBERS[:3]]
    ens = sph.Ensemble(sims)
    ens.run(4)
    before = [s.state() for s in sims]
    t_before = [s.time() for s in sims]
    lanes, cadence, ms = ens.autotune(trial_steps=8)
    assert lanes in (1, 2, 4, 8) and cadence in (1, 2, 4, 8, 16, 32) and ms > 0
    assert len({s.start_form() for s in sims}) == 1
    for s, b, t in zip(sims, before, t_before):
        assert s.time() == t
        assert _same(s.state(), b)
        assert s.tuning() == (lanes, cadence)
    ens.run(8)
    ens.close()


def test_rejects_bad_arguments(sph):
    sim = _make(sph, MEMBERS[0])
    with pytest.raises(sph.SphError):
        sph.Ensemble([])
    with pytest.raises(sph.SphError):
        sph.Ensemble([sim, sim])
    ens = sph.Ensemble([sim])
    with pytest.raises(sph.SphError):
        ens.run_async(-1)
    ens.close()
