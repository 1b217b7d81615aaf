"""Shared helpers of the test suite (comparison metrics, case builders)."""
import numpy as np


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (den if den > 0 else 1.0))


def rel_l2_vec(ax, ay, bx, by):
    num = np.sqrt(np.sum((np.asarray(ax) - bx) ** 2 + (np.asarray(ay) - by) ** 2))
    den = np.sqrt(np.sum(np.asarray(bx) ** 2 + np.asarray(by) ** 2))
    return float(num / (den if den > 0 else 1.0))


def oracle_sim(orc, case, use_cells=True):
    sim = orc.OracleSim(case["params"], case["fluid"], case.get("boundary"),
                        use_cells=use_cells)
    inf = case.get("inflow")
    if inf is not None:
        sim.add_inflow(inf["x_exit"], inf["y0"], inf["y1"], inf["U"], inf["amp"], inf["k"],
                       inf["phase"], inf["layers"])
    return sim


def ambiguous_mask(orc, d, st, ev, band=1e-4):
    """Particles whose CSF filter decision (Eq. 20) is within `band` of the
    threshold, plus every particle within 2h of one: their curvature term can
    legitimately differ between FP32 and FP64."""
    mag = np.hypot(ev["nx"], ev["ny"])
    amb = np.abs(mag / d.eps_n - 1.0) < band
    if not amb.any():
        return amb
    start, lst = orc.neighbours(st["x"], st["y"], 2.0 * d.h)
    out = amb.copy()
    for a in np.nonzero(amb)[0]:
        out[lst[start[a]:start[a + 1]]] = True
    return out
