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


def test_a_scale_is_the_per_component_rms_of_valid_corrections():
    corr = np.array([[3.0, 4.0], [0.0, 0.0], [100.0, 100.0]])
    valid = np.array([True, True, False])
    smp = {"corr": corr, "valid": valid}
    # valid components: 3, 4, 0, 0 -> rms = sqrt(25 / 4)
    assert abs(sg.a_scale([smp]) - 2.5) < 1e-15
