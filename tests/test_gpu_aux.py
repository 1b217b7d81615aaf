"""Checkpoint / resume and run statistics through the C ABI on a GPU.

* A context that runs on from a checkpoint and a new context loaded from it
  give bit-identical states after the same steps (the cell order after a
  rebuild depends only on positions and ids; the checkpoint carries the
  density compensation carries and the clocks).
* sph_stats' FP64 sums equal the same sums over the state read back with
  sph_get_state, and match the oracle's state after the same steps.
"""
import math

import numpy as np
import pytest

from paper_1603_02421_gb300 import workloads as wl
from tests.helpers import oracle_sim

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sph():
    from paper_1603_02421_gb300 import binding, build
    build.build()
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    return binding


def _jet():
    case = wl.jet(seed=5, dx=1.0 / 20, length=6.0, Re=200, We=20)
    case["params"]["skin_over_h"] = 0.3
    return case


@pytest.mark.parametrize("lanes,cadence", [(2, 8), (4, 1)])
def test_checkpoint_resume_is_bit_identical(sph, lanes, cadence):
    case = _jet()
    a = sph.Simulation(case)
    a.set_tuning(lanes, cadence)
    a.run(37)
    blob = sph.sph_checkpoint_save(a.ctx)
    ta = a.time()
    b = sph.Simulation(case)
    b.set_tuning(lanes, cadence)
    sph.sph_checkpoint_load(b.ctx, blob)
    tb = b.time()
    assert tb == ta
    # the running context rebuilds at the step the loaded one starts with
    sph.sph_request_rebuild(a.ctx)
    a.run(45)
    b.run(45)
    sa, sb = a.state(), b.state()
    assert a.time() == b.time()
    for k in ("x", "y", "u", "v", "rho", "m", "id", "type"):
        assert np.array_equal(sa[k], sb[k]), k
    # and a checkpoint of each is the same bytes
    assert sph.sph_checkpoint_save(a.ctx) == sph.sph_checkpoint_save(b.ctx)
    a.close()
    b.close()


def test_checkpoint_rejects_foreign_buffers(sph):
    case = _jet()
    a = sph.Simulation(case)
    blob = sph.sph_checkpoint_save(a.ctx)
    for bad in (b"", blob[:40], b"X" + blob[1:], blob + b"\0"):
        with pytest.raises(sph.SphError) as e:
            sph.sph_checkpoint_load(a.ctx, bad)
        assert e.value.status == -1
    c64 = sph.Simulation(case, prec="fp64")
    with pytest.raises(sph.SphError) as e:
        sph.sph_checkpoint_load(c64.ctx, blob)
    assert e.value.status == -1
    a.close()
    c64.close()


def _sums(st, p, fluid):
    """The statistics of sph_stats over a state dict, in numpy FP64."""
    m = st["m"][fluid] if "m" in st else st["mass"][fluid]
    u, v = st["u"][fluid], st["v"][fluid]
    x, y = st["x"][fluid], st["y"][fluid]
    rho0, c0, gamma = p["rho0"], p["c0"], p.get("gamma", 7.0)
    B = rho0 * c0 * c0 / gamma
    d = (st["rho"][fluid] - rho0) / rho0
    e = B / rho0 * (np.expm1((gamma - 1.0) * np.log1p(d)) / (gamma - 1.0) - d / (1.0 + d))
    return {"mass": m.sum(), "momentum_x": (m * u).sum(), "momentum_y": (m * v).sum(),
            "kinetic": (0.5 * m * (u * u + v * v)).sum(),
            "potential": -(m * (p.get("gx", 0.0) * x + p.get("gy", 0.0) * y)).sum(),
            "elastic": (m * e).sum(), "max_rel_density": np.abs(d).max()}


def test_stats_match_the_state_and_the_oracle(sph, orc):
    case = wl.dam_break(seed=2, dx=0.02, prec="fp32")
    sim = sph.Simulation(case)
    osim = oracle_sim(orc, case)
    sim.run(60)
    osim.run(60)
    s = sph.sph_stats(sim.ctx)
    g = sim.state()
    p = case["params"]
    fluid = g["type"] == 0
    ref = _sums(g, p, fluid)
    assert s["n_fluid"] == int(fluid.sum()) and s["n_buffer"] == 0
    assert s["n_boundary"] == len(case["boundary"]["x"])
    assert s["step"] == 60 and s["t"] == pytest.approx(osim.t, rel=1e-12)
    for k, v in ref.items():
        # the state read back rounds rho - rho0 to FP32 without its carry
        tol = 1e-6 if k in ("elastic", "max_rel_density") else 1e-10
        assert s[k] == pytest.approx(v, rel=tol, abs=1e-12 * abs(ref["kinetic"])), k
    # mass is exactly that of the particles added (Sec. 2-2: constant masses)
    assert s["mass"] == pytest.approx(float(np.sum(case["fluid"]["m"])), rel=1e-7)
    ofl = osim.st["type"] == 0
    oref = _sums(osim.st, p, ofl)
    for k in ("mass", "kinetic", "potential", "elastic"):
        assert s[k] == pytest.approx(oref[k], rel=1e-4), k
    # total energy of the collapsing column: the same as the oracle's, and
    # nearly constant over the first 6 ms (the wall factors of Eq. 29 and the
    # start from a hydrostatic lattice move it by about 1 %)
    s0 = sph.Simulation(case)
    e0 = sph.sph_stats(s0.ctx)
    s0.close()
    E0 = e0["kinetic"] + e0["potential"] + e0["elastic"]
    E1 = s["kinetic"] + s["potential"] + s["elastic"]
    assert E1 == pytest.approx(oref["kinetic"] + oref["potential"] + oref["elastic"], rel=1e-4)
    assert abs(E1 - E0) <= 0.02 * abs(E0)
    assert math.isfinite(s["max_rel_density"]) and s["max_rel_density"] < 0.05
    sim.close()


def test_state_round_trip_count_query_and_first_bad_particle(sph):
    """sph_set_state -> sph_get_state returns the state unchanged (FP32
    velocities and density offsets round-trip exactly through their FP64
    host form); a call with too small a cap returns SPH_ERR_CAPACITY with the
    full count; set_state names the first invalid particle.  The jet has more
    than 2^16 particles, so the host loops run split over threads."""
    import ctypes
    case = wl.jet(seed=3, dx=1.0 / 40, length=42.0, Re=200, We=20)
    a = sph.Simulation(case)
    a.run(3)
    st = a.state()
    n = len(st["x"])
    assert n > (1 << 16)
    assert np.all(np.diff(st["id"].astype(np.int64)) > 0)
    cnt = ctypes.c_longlong()
    status = sph.lib().sph_get_state(a.ctx, 10, ctypes.byref(cnt), *([None] * 11))
    assert status == -3 and cnt.value == n
    b = sph.Simulation(case)
    b.set_state(st)
    sb = b.state()
    for k in ("x", "y", "u", "v", "rho", "m", "id", "type"):
        assert np.array_equal(st[k], sb[k]), k
    # the first invalid particle is the one reported, whichever chunk of the
    # threaded check finds it
    bad = {k: v.copy() for k, v in st.items()}
    bad["x"][n - 7] = case["params"]["xmax"] + 1.0
    bad["type"][40001] = 9
    with pytest.raises(sph.SphError) as e:
        b.set_state(bad)
    assert e.value.status == -1 and "particle 40001:" in str(e.value)
    bad["type"][40001] = st["type"][40001]
    with pytest.raises(sph.SphError) as e:
        b.set_state(bad)
    assert e.value.status == -1 and ("particle %d lies outside" % (n - 7)) in str(e.value)
    # repeated ids, found by the threaded marking: the smallest one is named
    dup = {k: v.copy() for k, v in st.items()}
    ids = dup["id"]
    dup["id"][n - 3] = ids[50000]
    dup["id"][9] = ids[20000]
    with pytest.raises(sph.SphError) as e:
        b.set_state(dup)
    assert e.value.status == -1
    assert ("duplicate id %d" % min(ids[50000], ids[20000])) in str(e.value)
    # the context still holds the state set before the failed calls
    sb = b.state()
    assert np.array_equal(sb["id"], st["id"]) and np.array_equal(sb["x"], st["x"])
    a.close()
    b.close()
