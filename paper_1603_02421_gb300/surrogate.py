"""Training and evaluation of the learned surrogate (sph_mpnn_*,
sph_surrogate_step) from plain SPH trajectories.

A sample is a state s_n of a jet together with what the network must
predict there: the correction y* = (abar - a_n) / a_ref, where abar =
(u_{n+k} - u_n) / (t_{n+k} - t_n) is the mean acceleration of a particle over
the next k plain steps and a_n its SPH acceleration at s_n (Eq. 25).  Only
fluid particles present at both ends carry a target; the others get y* = 0.
The surrogate step then advances with abar = a_n + a_ref (y - ybar), ybar
the mass-weighted mean of y over the fluid (plain SPH judges it and takes
over when its residuals exceed the threshold).

Everything runs through the C ABI of libsph (binding.py); nothing here
computes SPH or network arithmetic itself.
"""
from __future__ import annotations

import time

import numpy as np

from . import binding

STATE_KEYS = ("x", "y", "u", "v", "rho", "m", "type", "id")


def collect(case, nsamples, every=20, k=4, warm=20, lanes_cadence=(2, 8), end_accel=False):
    """Samples from one jet: warm-up steps, then every `every` steps a state
    with the k-step targets.  Returns a list of dicts (state arrays sorted by
    id, the correction abar - a_n and abar per particle, the validity mask;
    with end_accel also a_end and drho_end, the SPH acceleration and
    continuity rate at the end of the k steps, drho at the start and the span
    dT, for the residual floors)."""
    sim = binding.Simulation(case)
    sim.set_tuning(*lanes_cadence)
    out = []
    try:
        sim.run(warm)
        for _ in range(nsamples):
            sim.evaluate()
            s0 = sim.state()
            t0 = sim.time()["t"]
            sim.run(k)
            if end_accel:
                sim.evaluate()
            s1 = sim.state()
            t1 = sim.time()["t"]
            common, i0, i1 = np.intersect1d(s0["id"], s1["id"], return_indices=True)
            n0 = len(s0["id"])
            abar = np.zeros((n0, 2))
            abar[i0, 0] = (s1["u"][i1] - s0["u"][i0]) / (t1 - t0)
            abar[i0, 1] = (s1["v"][i1] - s0["v"][i0]) / (t1 - t0)
            valid = np.zeros(n0, bool)
            valid[i0] = (s0["type"][i0] == binding.FLUID) & (s1["type"][i1] == binding.FLUID)
            a_n = np.stack([s0["ax"], s0["ay"]], 1)
            corr = np.where(valid[:, None], abar - a_n, 0.0)
            out.append({"state": {key: s0[key] for key in STATE_KEYS}, "corr": corr,
                        "abar": np.where(valid[:, None], abar, 0.0), "valid": valid})
            if end_accel:
                a_end = np.zeros((n0, 2))
                a_end[i0, 0] = s1["ax"][i1]
                a_end[i0, 1] = s1["ay"][i1]
                out[-1]["a_end"] = np.where(valid[:, None], a_end, 0.0)
                dr_end = np.zeros(n0)
                dr_end[i0] = s1["drho"][i1]
                out[-1]["drho"] = np.where(valid, s0["drho"], 0.0)
                out[-1]["drho_end"] = np.where(valid, dr_end, 0.0)
                out[-1]["dT"] = t1 - t0
            sim.run(max(every - k, 0))
    finally:
        sim.close()
    return out


def residual_floor(samples):
    """The acceleration-field residual sqrt(sum |abar - (a_n + a_k)/2|^2 /
    sum |(a_n + a_k)/2|^2) over the valid particles, evaluated with the true
    k-step mean abar of plain SPH and the SPH accelerations a_n, a_k at both
    ends of those k steps: what a perfect predictor would score.  One value
    per sample (samples collected with end_accel=True).  The step-to-step
    acoustic noise of WCSPH accelerations keeps it near 0.1, which is why
    the judge does not use it."""
    out = []
    for smp in samples:
        v = smp["valid"]
        abar = smp["abar"][v]
        a_n = abar - smp["corr"][v]
        trap = 0.5 * (a_n + smp["a_end"][v])
        den = float(np.sum(trap ** 2))
        out.append(float(np.sqrt(np.sum((abar - trap) ** 2) / den)) if den > 0 else 0.0)
    return out


def momentum_floor(samples):
    """The judge's momentum-balance residual |sum m (abar - (a_n + a_k)/2)|
    / sum m |(a_n + a_k)/2| over the valid particles, with the true k-step
    mean abar of plain SPH: what a perfect predictor would score.  The
    internal pair forces cancel in the sums, so the step-to-step noise of
    single particles does not enter.  One value per sample (samples with
    end_accel=True; masses from the sample's state, unit masses without
    one)."""
    out = []
    for smp in samples:
        v = smp["valid"]
        m = np.asarray(smp["state"]["m"], float)[v] if "state" in smp else np.ones(int(v.sum()))
        abar = smp["abar"][v]
        a_n = abar - smp["corr"][v]
        trap = 0.5 * (a_n + smp["a_end"][v])
        den = float(np.sum(m * np.hypot(trap[:, 0], trap[:, 1])))
        num = np.sum(m[:, None] * (abar - trap), axis=0)
        out.append(float(np.hypot(num[0], num[1]) / den) if den > 0 else 0.0)
    return out


def density_floor(samples, rho0):
    """The judge's density residual (dT/2) rms(drho/dt_k - drho/dt_n) / rho0
    over the valid particles of each sample (end_accel=True), dT the span of
    its k plain steps: the change of the continuity rate over k plain steps,
    which the surrogate step's end evaluation also sees."""
    out = []
    for smp in samples:
        v = smp["valid"]
        d = smp["drho_end"][v] - smp["drho"][v]
        out.append(float(0.5 * smp["dT"] * np.sqrt(np.mean(d * d)) / rho0) if d.size else 0.0)
    return out


def a_scale(samples):
    """RMS (per component) of the correction over the valid particles."""
    num = sum(float(np.sum(s["corr"][s["valid"]] ** 2)) for s in samples)
    cnt = sum(int(np.sum(s["valid"])) for s in samples)
    return float(np.sqrt(num / max(cnt, 1) / 2.0)) or 1.0


class Trainer:
    """One evaluation context per case (the samples of a case share its
    parameters); the network is trained on the GPU with its own forward,
    backward and Adam kernels."""

    def __init__(self, cases, capacity, u_ref=1.0, seed=0, device=0):
        from .workloads import mpnn_init
        self.sims = [binding.Simulation(c) for c in cases]
        self.net = binding.Mpnn(capacity, device)
        prm = mpnn_init(seed)
        prm["D"][:] = 0.0          # start from the zero correction (steps with a_n)
        self.net.set_params(prm)
        self.u_ref = u_ref
        self.capacity = capacity

    def _load(self, ci, sample):
        sim = self.sims[ci]
        binding.sph_set_state(sim.ctx, sample["state"])
        sim.evaluate()
        return sim

    def _order(self, sim, sample):
        """Positions, in the sample's id-sorted arrays, of the context's
        particles in cell order."""
        ids, _ = binding.sph_mpnn_forward(self.net.net, sim.ctx, self.u_ref, False, self.capacity)
        return np.searchsorted(sample["state"]["id"], ids)

    def train(self, data, a_ref, epochs=None, seconds=None, lr=1e-3, seed=0):
        """data: list of (case index, sample).  Stops after `epochs` passes or
        `seconds` of wall time.  Returns the mean loss of each pass."""
        rng = np.random.default_rng(seed)
        losses = []
        t_start = time.perf_counter()
        while True:
            tot = 0.0
            for j in rng.permutation(len(data)):
                ci, smp = data[j]
                sim = self._load(ci, smp)
                pos = self._order(sim, smp)
                t = (smp["corr"][pos] / a_ref).astype(np.float32)
                tot += binding.sph_mpnn_backward(self.net.net, sim.ctx, self.u_ref, t)
                binding.sph_mpnn_adam(self.net.net, lr)
            losses.append(tot / len(data))
            if epochs is not None and len(losses) >= epochs:
                break
            if seconds is not None and time.perf_counter() - t_start >= seconds:
                break
        return losses

    def prediction_errors(self, data, a_ref, bf16=True):
        """Relative L2 errors, over the valid particles of all samples, of the
        predicted mean acceleration a_n + a_ref (y - ybar) against the true
        k-step mean, and of a_n alone (the method without the network); ybar
        is the mass-weighted mean of y over the fluid, which the surrogate
        step removes (sph_surrogate_step)."""
        num_net = num_zero = den = 0.0
        for ci, smp in data:
            sim = self._load(ci, smp)
            ids, y = binding.sph_mpnn_forward(self.net.net, sim.ctx, self.u_ref, bf16,
                                              self.capacity)
            pos = np.searchsorted(smp["state"]["id"], ids)
            y = y.astype(np.float64)
            fl = smp["state"]["type"][pos] == binding.FLUID
            m = smp["state"]["m"][pos][fl]
            if m.sum() > 0:
                y = y - (m[:, None] * y[fl]).sum(0) / m.sum()
            v = smp["valid"][pos]
            corr = smp["corr"][pos][v]
            pred = a_ref * y[v]
            num_net += float(np.sum((pred - corr) ** 2))
            num_zero += float(np.sum(corr ** 2))
            den += float(np.sum(smp["abar"][pos][v] ** 2))
        return float(np.sqrt(num_net / den)), float(np.sqrt(num_zero / den))

    def close(self):
        self.net.close()
        for s in self.sims:
            s.close()
