"""The seeded synthetic inputs against the configurations they stand in for.

The workloads are geometries, not datasets: a dam break with an obstacle
(Sec. 3-1) and planar jets issuing from an inflow (Sec. 3-2), at the sizes of
the five benchmark configurations -- the 2.4k-particle dam break, the 96k and
1M-particle jets, the 64-jet ensemble on a Re x We grid with uneven particle
counts, and the 16 held-out surrogate jets.  Checked here on the CPU: counts,
spacings, extents, physical parameters and the seeded draws.
"""
import math

import numpy as np
import pytest

import bench
from paper_1603_02421_gb300 import workloads as wl


def test_dam_break_recipe():
    case = wl.dam_break(seed=3, dx=0.01)
    p, f, b = case["params"], case["fluid"], case["boundary"]
    dx = 0.01
    # water column 0.4 m x 0.6 m at the left wall on a dx lattice: 2400 particles
    assert len(f["x"]) == 40 * 60
    lx = np.round(f["x"] / dx - 0.5)
    ly = np.round(f["y"] / dx - 0.5)
    assert lx.min() == 0 and lx.max() == 39 and ly.min() == 0 and ly.max() == 59
    # seeded uniform jitter of at most +-0.01 dx, reproducible, seed-dependent
    jx = f["x"] - (lx + 0.5) * dx
    jy = f["y"] - (ly + 0.5) * dx
    assert np.abs(jx).max() <= 0.01 * dx and np.abs(jy).max() <= 0.01 * dx
    assert np.abs(jx).max() > 0.009 * dx
    again = wl.dam_break(seed=3, dx=0.01)["fluid"]
    other = wl.dam_break(seed=4, dx=0.01)["fluid"]
    assert np.array_equal(again["x"], f["x"]) and not np.array_equal(other["x"], f["x"])
    # hydrostatic start: the Tait pressure of each particle is rho0 g (H - y)
    B = p["rho0"] * p["c0"] ** 2 / p["gamma"]
    P = B * ((f["rho"] / p["rho0"]) ** p["gamma"] - 1.0)
    assert np.allclose(P, p["rho0"] * 9.81 * (0.6 - f["y"]), rtol=1e-9, atol=1e-6)
    # physical parameters of the configuration
    assert p["kernel"] == "cubic" and p["prec"] == "fp64" and p["h_over_dx"] == 1.3
    assert p["gamma"] == 7.0 and p["rho0"] == 1000.0 and p["alpha"] == 0.01
    assert p["c0"] == pytest.approx(10.0 * math.sqrt(9.81 * 0.6))
    assert p["dt_fixed"] == 1e-4 and p["gy"] == -9.81 and p["sigma"] == 0.0
    # tank 1.6 m x 0.8 m and a 0.12 m square obstacle 0.9 m from the left
    # wall, wall particles at dx/2 with unit normals into the fluid
    assert b["x"].min() == 0.0 and b["x"].max() == pytest.approx(1.6)
    assert b["y"].min() == 0.0 and b["y"].max() == pytest.approx(0.8)
    assert np.allclose(np.hypot(b["nx"], b["ny"]), 1.0)
    ob = (b["x"] >= 0.9 - 1e-12) & (b["x"] <= 1.02 + 1e-12) & (b["y"] > 1e-12)
    assert b["y"][ob].max() == pytest.approx(0.12)
    on_floor = np.abs(b["y"]) < 1e-12
    gaps = np.diff(np.sort(b["x"][on_floor]))
    assert np.allclose(gaps[gaps < 0.02], 0.5 * dx)
    assert 650 <= len(b["x"]) <= 850


@pytest.mark.parametrize("name,n,dx,length,re,we", [("jet_c2", 96000, 1 / 40, 60.0, 200.0, 20.0),
                                                    ("jet_c3", 1000000, 1 / 100, 100.0, 100.0,
                                                     10.0)])
def test_planar_jet_recipe(name, n, dx, length, re, we):
    case, desc = bench.workload(name, seed=2)
    p, f, inf = case["params"], case["fluid"], case["inflow"]
    # a strip [0, L) x [-D/2, D/2) on a dx lattice
    assert len(f["x"]) == n
    assert p["dx"] == pytest.approx(dx) and p["h_over_dx"] == 1.3
    assert f["x"].min() == pytest.approx(0.5 * dx) and f["x"].max() < length
    assert f["y"].min() == pytest.approx(-0.5 + 0.5 * dx)
    assert f["y"].max() == pytest.approx(0.5 - 0.5 * dx)
    # D = U = 1, rho = 1000: sigma = rho U^2 D / We; alpha reproduces
    # nu = U D / Re through nu = alpha h c0 / 8 (the configurations' mapping)
    h = 1.3 * dx
    assert p["sigma"] == pytest.approx(1000.0 / we)
    assert p["alpha"] * h * p["c0"] / 8.0 == pytest.approx(1.0 / re)
    assert p["kernel"] == "wendland" and p["prec"] == "fp32" and p["dt_fixed"] == 0.0
    # the inflow: 1 % sinusoidal velocity perturbation at a seeded wavenumber
    # in [0.5, 1] / D, and the prefilled strip carries the same profile
    assert inf["amp"] == 0.01 and 0.5 <= inf["k"] <= 1.0
    assert np.allclose(f["u"], 1.0 + 0.01 * np.sin(-inf["k"] * f["x"]))
    ks = {bench.workload(name, seed=s)[0]["inflow"]["k"] for s in (0, 1, 2)}
    assert len(ks) == 3


def test_ensemble_recipe():
    members = bench.ensemble_members()
    assert len(members) == 64
    assert sorted({m[1] for m in members}) == [100, 200, 400, 700, 1000, 1500, 2000, 3000]
    assert sorted({m[2] for m in members}) == [5, 10, 15, 20, 30, 40, 50, 60]
    assert len({(m[1], m[2]) for m in members}) == 64
    dxs = [m[3] for m in members]
    assert max(dxs) == pytest.approx(1 / 30) and min(dxs) == pytest.approx(1 / 80)
    # uneven particle counts from 20k to 400k: the smallest and the largest member
    for m in (members[0], members[-1]):
        case = bench.ensemble_case(*m, skin=0.15)
        target = 20000.0 * 20.0 ** (m[0] / 63.0)
        assert abs(len(case["fluid"]["x"]) - target) <= 0.02 * target
    # each member has its own seed, hence its own inflow perturbation
    ks = [bench.ensemble_case(*m, skin=0.15)["inflow"]["k"] for m in members[:4]]
    assert len(set(ks)) == 4


def test_surrogate_held_out_recipe():
    held = [(re, we) for re in bench.SUR_HELD_RE for we in bench.SUR_HELD_WE]
    grid = {(m[1], m[2]) for m in bench.ensemble_members()}
    assert len(held) == 16 and not (set(held) & grid)
    assert set(bench.SUR_TRAIN) <= grid
    dx = 1.0 / 60
    case = wl.jet(seed=201, Re=300, We=7.5, dx=dx, length=200000 * dx * dx)
    assert abs(len(case["fluid"]["x"]) - 200000) <= 0.01 * 200000
