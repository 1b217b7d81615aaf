"""Host-side helpers of the learned surrogate (paper_1603_02421_gb300/surrogate.py):
the correction scale and the residual floor, on hand-made samples (no GPU)."""
import numpy as np

from paper_1603_02421_gb300 import surrogate as sg


def _sample(abar, a_n, a_end, valid):
    abar = np.asarray(abar, float)
    a_n = np.asarray(a_n, float)
    return {"abar": abar, "corr": abar - a_n, "a_end": np.asarray(a_end, float),
            "valid": np.asarray(valid, bool)}


def test_residual_floor_is_zero_when_the_mean_is_the_trapezoid():
    rng = np.random.default_rng(0)
    a_n = rng.normal(size=(50, 2))
    a_end = rng.normal(size=(50, 2))
    abar = 0.5 * (a_n + a_end)
    (r,) = sg.residual_floor([_sample(abar, a_n, a_end, np.ones(50))])
    assert r < 1e-14             # a_n is recovered as abar - (abar - a_n): rounding only


def test_residual_floor_closed_form():
    # a_n = (1, 0), a_end = (3, 0): trapezoid (2, 0); abar = (2, 1) misses it by
    # |(0, 1)| on every particle, so the residual is 1 / 2
    n = 8
    a_n = np.tile([1.0, 0.0], (n, 1))
    a_end = np.tile([3.0, 0.0], (n, 1))
    abar = np.tile([2.0, 1.0], (n, 1))
    (r,) = sg.residual_floor([_sample(abar, a_n, a_end, np.ones(n))])
    assert abs(r - 0.5) < 1e-15


def test_residual_floor_ignores_invalid_particles_and_is_scale_free():
    n = 6
    a_n = np.tile([1.0, 0.0], (n, 1))
    a_end = np.tile([3.0, 0.0], (n, 1))
    abar = np.tile([2.0, 1.0], (n, 1))
    valid = np.ones(n, bool)
    abar_bad = abar.copy()
    abar_bad[0] = [1e9, -1e9]        # a particle without a target
    valid_bad = valid.copy()
    valid_bad[0] = False
    r_all = sg.residual_floor([_sample(abar, a_n, a_end, valid)])[0]
    r_masked = sg.residual_floor([_sample(abar_bad, a_n, a_end, valid_bad)])[0]
    r_scaled = sg.residual_floor([_sample(7.0 * abar, 7.0 * a_n, 7.0 * a_end, valid)])[0]
    assert abs(r_all - r_masked) < 1e-15
    assert abs(r_all - r_scaled) < 1e-15


def test_momentum_floor_closed_form_and_balance():
    # trapezoid (2, 0) on every particle; abar misses it by (0, 1) on all:
    # the imbalance is sum m (0, 1) = (0, n) against sum m |(2, 0)| = 2n
    n = 8
    a_n = np.tile([1.0, 0.0], (n, 1))
    a_end = np.tile([3.0, 0.0], (n, 1))
    abar = np.tile([2.0, 1.0], (n, 1))
    smp = _sample(abar, a_n, a_end, np.ones(n))
    assert abs(sg.momentum_floor([smp])[0] - 0.5) < 1e-15
    # errors of opposite sign on equal masses balance: no momentum residual,
    # though every particle misses the trapezoid
    abar2 = abar.copy()
    abar2[::2, 1] = -1.0
    smp2 = _sample(abar2, a_n, a_end, np.ones(n))
    assert sg.momentum_floor([smp2])[0] < 1e-15
    assert sg.residual_floor([smp2])[0] == sg.residual_floor([smp])[0]
    # masses weight the balance
    smp3 = dict(smp2, state={"m": np.where(np.arange(n) % 2 == 0, 3.0, 1.0)})
    # (0, 1) on the odd (m = 1) and (0, -1) on the even (m = 3) particles:
    # |4 (1 - 3)| / (2 * (4 * 3 + 4 * 1)) = 8 / 32
    assert abs(sg.momentum_floor([smp3])[0] - 0.25) < 1e-15


def test_a_scale_is_the_per_component_rms_of_valid_corrections():
    corr = np.array([[3.0, 4.0], [0.0, 0.0], [100.0, 100.0]])
    valid = np.array([True, True, False])
    smp = {"corr": corr, "valid": valid}
    # valid components: 3, 4, 0, 0 -> rms = sqrt(25 / 4)
    assert abs(sg.a_scale([smp]) - 2.5) < 1e-15


def test_density_floor_closed_form():
    # the continuity rate changes by (+2, -2) on alternate valid particles
    # over dT = 0.5: (0.5 / 2) * rms(2) / rho0
    n = 10
    smp = {"valid": np.ones(n, bool), "drho": np.zeros(n),
           "drho_end": np.where(np.arange(n) % 2 == 0, 2.0, -2.0), "dT": 0.5}
    assert abs(sg.density_floor([smp], 1000.0)[0] - 0.25 * 2.0 / 1000.0) < 1e-18
    # invalid particles do not count
    smp2 = dict(smp, valid=np.arange(n) < 4, drho_end=np.where(np.arange(n) < 4, smp["drho_end"], 1e6))
    assert abs(sg.density_floor([smp2], 1000.0)[0] - 0.25 * 2.0 / 1000.0) < 1e-18
