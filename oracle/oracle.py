"""FP64 CPU oracle for the 2D WCSPH jet-breakup method (arXiv 1603.02421).

TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and
the benchmark's CPU-baseline leg may import this module.  The product path
(the CUDA library and its binding) never imports, links or runs it, and the
two share no code.

The heavy per-evaluation sums live in ``sph_oracle.c`` (plain C, double
precision, no fused multiply-add); this module loads it with ctypes and
restates the time loop of the method around it:

* ``evaluate``: one evaluation of Eqs. 7, 9-10, 14, 18, 20-26, 29-31.
* ``OracleSim.step``: the predictor-corrector step of Sec. 2-8 with the
  adaptive step of Eqs. 30-32 (or a fixed step), followed by inflow and
  outflow handling.
* ``breakup_length``: the Sec. 3-2 criterion (links shorter than 1.5 h).
* ``correlation_LD``: the empirical breakup correlation of Eq. 37.

Readings taken where the paper is silent (predictor-corrector formulas,
sound speed, inflow) are stated at each function.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sph_oracle.c")
_HDR = os.path.join(_HERE, "sph_oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")

FLUID, BOUNDARY, BUFFER = 0, 1, 2
CUBIC, WENDLAND = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle's C file into ``oracle/liboracle.so`` with gcc
    (with OpenMP where the compiler has it; the particle loops then run on
    ``set_threads`` threads, 1 by default, with identical results)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + ".tmp%d" % os.getpid()
        base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        if subprocess.call(base[:1] + ["-fopenmp"] + base[1:],
                           stderr=subprocess.DEVNULL) != 0:
            subprocess.check_call(base)
        os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int), ("use_cells", ctypes.c_int),
                ("h", ctypes.c_double), ("rho0", ctypes.c_double),
                ("c0", ctypes.c_double), ("gamma", ctypes.c_double),
                ("alpha", ctypes.c_double), ("eta2", ctypes.c_double),
                ("sigma", ctypes.c_double), ("eps_n", ctypes.c_double),
                ("gx", ctypes.c_double), ("gy", ctypes.c_double),
                ("wall_A", ctypes.c_double), ("wall_db", ctypes.c_double),
                ("wall_h0", ctypes.c_double)]


_dp = ctypes.POINTER(ctypes.c_double)
_up = ctypes.POINTER(ctypes.c_ubyte)


class _State(ctypes.Structure):
    _fields_ = [("n", ctypes.c_longlong),
                ("x", _dp), ("y", _dp), ("u", _dp), ("v", _dp), ("rho", _dp), ("m", _dp),
                ("type", _up),
                ("nb", ctypes.c_longlong),
                ("bx", _dp), ("by", _dp), ("bnx", _dp), ("bny", _dp)]


class _Out(ctypes.Structure):
    _fields_ = [("ax", _dp), ("ay", _dp), ("drho", _dp),
                ("C", _dp), ("nx", _dp), ("ny", _dp), ("kappa", _dp),
                ("Nflag", _up), ("dt_f", _dp), ("dt_cv", _dp)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _lib.orc_kernel_norm.restype = ctypes.c_double
        _lib.orc_kernel_norm.argtypes = [ctypes.c_int]
        for f in (_lib.orc_W, _lib.orc_dWdr):
            f.restype = ctypes.c_double
            f.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double]
        for f in (_lib.orc_pressure, _lib.orc_sound_speed):
            f.restype = ctypes.c_double
            f.argtypes = [ctypes.c_double] * 4
        _lib.orc_neighbours.restype = ctypes.c_longlong
        _lib.orc_neighbours.argtypes = [
            ctypes.c_longlong, _dp, _dp, _up, ctypes.c_double, ctypes.c_int,
            ctypes.POINTER(ctypes.POINTER(ctypes.c_longlong)),
            ctypes.POINTER(ctypes.POINTER(ctypes.c_int))]
        _lib.orc_free.restype = None
        _lib.orc_free.argtypes = [ctypes.c_void_p]
        _lib.orc_evaluate.restype = ctypes.c_int
        _lib.orc_evaluate.argtypes = [ctypes.POINTER(_Params), ctypes.POINTER(_State),
                                      ctypes.POINTER(_Out)]
        _lib.orc_summation_density.restype = ctypes.c_int
        _lib.orc_summation_density.argtypes = [ctypes.POINTER(_Params), ctypes.POINTER(_State),
                                               _dp]
        _lib.orc_set_threads.restype = None
        _lib.orc_set_threads.argtypes = [ctypes.c_int]
        _lib.orc_max_threads.restype = ctypes.c_int
        _lib.orc_max_threads.argtypes = []
        _lib.orc_components.restype = ctypes.c_longlong
        _lib.orc_components.argtypes = [ctypes.c_longlong, _dp, _dp, ctypes.c_double,
                                        ctypes.c_int, ctypes.POINTER(ctypes.c_longlong)]
    return _lib


def set_threads(n: int) -> None:
    """Threads of the oracle's particle loops (results do not depend on it)."""
    lib().orc_set_threads(int(n))


def max_threads() -> int:
    """The host's OpenMP thread count (1 when built without OpenMP)."""
    return int(lib().orc_max_threads())


def _d(a):
    return a.ctypes.data_as(_dp)


def _u8(a):
    return a.ctypes.data_as(_up)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# --------------------------------------------------------------------------
# scalar functions (Sec. 2-4, 2-5)
# --------------------------------------------------------------------------
def kernel_id(name) -> int:
    if isinstance(name, int):
        return name
    return {"cubic": CUBIC, "wendland": WENDLAND}[name]


def W(kernel, r, h):
    """Eq. 27 / Eq. 28 (2D, unit-integral normalisation)."""
    return lib().orc_W(kernel_id(kernel), float(r), float(h))


def dWdr(kernel, r, h):
    return lib().orc_dWdr(kernel_id(kernel), float(r), float(h))


def kernel_norm(kernel):
    return lib().orc_kernel_norm(kernel_id(kernel))


def pressure(rho, rho0, c0, gamma=7.0):
    """Eq. 26: Tait equation of state."""
    return lib().orc_pressure(float(rho), float(rho0), float(c0), float(gamma))


def sound_speed(rho, rho0, c0, gamma=7.0):
    return lib().orc_sound_speed(float(rho), float(rho0), float(c0), float(gamma))


def correlation_LD(We: float, Re: float) -> float:
    """Eq. 37: L/D0 = 13 sqrt(We) (1 + 3 Oh), Oh = sqrt(We)/Re (Eq. 35).

    The printed "(1 + 30h)" is read as "(1 + 3 Oh)"; Table 1's last column
    follows from that reading.  We and Re use the orifice radius (Eqs. 33-34).
    """
    Oh = math.sqrt(We) / Re
    return 13.0 * math.sqrt(We) * (1.0 + 3.0 * Oh)


# --------------------------------------------------------------------------
# neighbour lists (Sec. 2-7)
# --------------------------------------------------------------------------
def neighbours(x, y, radius, use_cells=True, active=None):
    """All ordered pairs (a, b), a != b, with |r_a - r_b|^2 < radius^2.

    Returns (start[n+1], list) with each list ascending in b.
    """
    x = _f64(x)
    y = _f64(y)
    n = len(x)
    act = None
    if active is not None:
        act = np.ascontiguousarray(active, dtype=np.uint8)
    start_p = ctypes.POINTER(ctypes.c_longlong)()
    list_p = ctypes.POINTER(ctypes.c_int)()
    tot = lib().orc_neighbours(n, _d(x), _d(y), _u8(act) if act is not None else None,
                               float(radius), int(bool(use_cells)),
                               ctypes.byref(start_p), ctypes.byref(list_p))
    if tot < 0:
        raise MemoryError("oracle neighbour search failed")
    start = np.ctypeslib.as_array(start_p, shape=(n + 1,)).copy()
    lst = (np.ctypeslib.as_array(list_p, shape=(tot,)).copy() if tot > 0
           else np.zeros(0, np.int32))
    lib().orc_free(ctypes.cast(start_p, ctypes.c_void_p))
    lib().orc_free(ctypes.cast(list_p, ctypes.c_void_p))
    return start, lst


def pair_set(x, y, radius, use_cells=True):
    """Set of ordered pairs as an (npairs, 2) int64 array, lexicographically sorted."""
    start, lst = neighbours(x, y, radius, use_cells)
    a = np.repeat(np.arange(len(x), dtype=np.int64), np.diff(start))
    return np.stack([a, lst.astype(np.int64)], axis=1)


# --------------------------------------------------------------------------
# parameters
# --------------------------------------------------------------------------
@dataclass
class Derived:
    kernel: int
    h: float
    H2: float
    rho0: float
    c0: float
    gamma: float
    alpha: float
    eta2: float
    sigma: float
    eps_n: float
    gx: float
    gy: float
    courant: float
    dt_fixed: float
    xmin: float
    ymin: float
    xmax: float
    ymax: float
    wall_A: float
    wall_db: float
    wall_h0: float
    summation: bool


def derive(params: dict) -> Derived:
    """Map the configuration dictionary to the quantities of the method.

    h = h_over_dx * dx (Sec. 2-2, 1.3 dx); eta^2 = 0.01 h^2 (Eq. 10);
    eps = 0.01 / h (Eq. 20); wall A = coef * c0^2 / h; boundary spacing
    db = wall_db_over_dx * dx.
    """
    dx = float(params["dx"])
    h = float(params.get("h_over_dx", 1.3)) * dx
    H = 2.0 * h
    c0 = float(params["c0"])
    return Derived(
        kernel=kernel_id(params.get("kernel", "wendland")), h=h, H2=H * H,
        rho0=float(params.get("rho0", 1000.0)), c0=c0,
        gamma=float(params.get("gamma", 7.0)), alpha=float(params.get("alpha", 0.0)),
        eta2=float(params.get("eta2_over_h2", 0.01)) * h * h,
        sigma=float(params.get("sigma", 0.0)),
        eps_n=float(params.get("eps_n_times_h", 0.01)) / h,
        gx=float(params.get("gx", 0.0)), gy=float(params.get("gy", 0.0)),
        courant=float(params.get("courant", 0.2)),
        dt_fixed=float(params.get("dt_fixed", 0.0)),
        xmin=float(params["xmin"]), ymin=float(params["ymin"]),
        xmax=float(params["xmax"]), ymax=float(params["ymax"]),
        wall_A=float(params.get("wall_A_coef", 0.01)) * c0 * c0 / h,
        wall_db=float(params.get("wall_db_over_dx", 0.5)) * dx,
        wall_h0=float(params.get("wall_h0", 0.0)),
        summation=params.get("density", "continuity") == "summation")


def _cparams(d: Derived, use_cells: bool) -> _Params:
    return _Params(kernel=d.kernel, use_cells=int(bool(use_cells)), h=d.h, rho0=d.rho0,
                   c0=d.c0, gamma=d.gamma, alpha=d.alpha, eta2=d.eta2, sigma=d.sigma,
                   eps_n=d.eps_n, gx=d.gx, gy=d.gy, wall_A=d.wall_A, wall_db=d.wall_db,
                   wall_h0=d.wall_h0)


# --------------------------------------------------------------------------
# one evaluation
# --------------------------------------------------------------------------
def evaluate(d: Derived, st: dict, boundary: dict | None = None, use_cells=True) -> dict:
    """Right-hand sides at state ``st`` (arrays x, y, u, v, rho, m, type).

    Returns du/dt (Eq. 25 incl. g and walls), drho/dt (Eq. 7), the CSF
    intermediates C (Eq. 14), n (Eq. 18), N (Eq. 20), kappa (Eq. 23) and the
    per-particle time-step terms of Eqs. 30-31.
    """
    n = len(st["x"])
    cols = {k: _f64(st[k]) for k in ("x", "y", "u", "v", "rho", "m")}
    typ = np.ascontiguousarray(st["type"], dtype=np.uint8)
    if boundary is not None and len(boundary["x"]) > 0:
        b = {k: _f64(boundary[k]) for k in ("x", "y", "nx", "ny")}
        nbd = len(b["x"])
    else:
        b = {k: np.zeros(1) for k in ("x", "y", "nx", "ny")}
        nbd = 0
    s = _State(n=n, x=_d(cols["x"]), y=_d(cols["y"]), u=_d(cols["u"]), v=_d(cols["v"]),
               rho=_d(cols["rho"]), m=_d(cols["m"]), type=_u8(typ), nb=nbd,
               bx=_d(b["x"]), by=_d(b["y"]), bnx=_d(b["nx"]), bny=_d(b["ny"]))
    m = max(n, 1)
    out = {k: np.zeros(m) for k in ("ax", "ay", "drho", "C", "nx", "ny", "kappa",
                                     "dt_f", "dt_cv")}
    out["N"] = np.zeros(m, np.uint8)
    o = _Out(ax=_d(out["ax"]), ay=_d(out["ay"]), drho=_d(out["drho"]), C=_d(out["C"]),
             nx=_d(out["nx"]), ny=_d(out["ny"]), kappa=_d(out["kappa"]),
             Nflag=_u8(out["N"]), dt_f=_d(out["dt_f"]), dt_cv=_d(out["dt_cv"]))
    cp = _cparams(d, use_cells)
    if lib().orc_evaluate(ctypes.byref(cp), ctypes.byref(s), ctypes.byref(o)) != 0:
        raise MemoryError("oracle evaluation failed")
    return {k: v[:n] for k, v in out.items()}


def summation_density(d: Derived, st: dict, use_cells=True) -> np.ndarray:
    """Eq. 6: rho_a = sum_b m_b W_ab over the fluid and buffer particles
    within 2h, the particle itself included."""
    n = len(st["x"])
    cols = {k: _f64(st[k]) for k in ("x", "y", "u", "v", "rho", "m")}
    typ = np.ascontiguousarray(st["type"], dtype=np.uint8)
    z = np.zeros(1)
    s = _State(n=n, x=_d(cols["x"]), y=_d(cols["y"]), u=_d(cols["u"]), v=_d(cols["v"]),
               rho=_d(cols["rho"]), m=_d(cols["m"]), type=_u8(typ), nb=0,
               bx=_d(z), by=_d(z), bnx=_d(z), bny=_d(z))
    out = np.zeros(max(n, 1))
    cp = _cparams(d, use_cells)
    if lib().orc_summation_density(ctypes.byref(cp), ctypes.byref(s), _d(out)) != 0:
        raise MemoryError("oracle summation density failed")
    return out[:n]


# --------------------------------------------------------------------------
# breakup (Sec. 3-2)
# --------------------------------------------------------------------------
def components(x, y, radius, use_cells=True):
    x = _f64(x)
    y = _f64(y)
    lab = np.zeros(max(len(x), 1), np.int64)
    nc = lib().orc_components(len(x), _d(x), _d(y), float(radius), int(bool(use_cells)),
                              lab.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)))
    if nc < 0:
        raise MemoryError("oracle components failed")
    return nc, lab[:len(x)]


def breakup_length(st: dict, h: float, x_exit: float, D: float, use_cells=True):
    """Breakup length L/D (Sec. 3-2).

    Particles closer than 1.5 h are linked; the jet is the union of the
    connected components that contain an inflow-buffer particle, and L is the
    largest streamwise distance of a jet particle from the orifice, in units
    of D.  Returns (L/D, broken) where ``broken`` is True when some particle
    lies outside those components.
    """
    x = _f64(st["x"])
    y = _f64(st["y"])
    _, lab = components(x, y, 1.5 * h, use_cells)
    roots = np.unique(lab[np.asarray(st["type"]) == BUFFER])
    if len(roots) == 0:
        raise ValueError("breakup length needs inflow-buffer particles")
    attached = np.isin(lab, roots)
    L = (x[attached].max() - x_exit) / D
    return float(L), bool((~attached).any())


# --------------------------------------------------------------------------
# time integration (Sec. 2-8) with inflow / outflow
# --------------------------------------------------------------------------
@dataclass
class Inflow:
    """Inflow buffer of the planar jet.

    The paper feeds its jet from a tank; this reading replaces the tank by
    ``layers`` buffer layers of spacing dx across [y0, y1] that move with the
    prescribed velocity u_in(t) = U (1 + amp sin(k U t + phase)) and turn into
    fluid when they cross x_exit.  A new layer is laid upstream whenever the
    upstream-most layer has advanced one spacing.
    """
    x_exit: float
    y0: float
    y1: float
    U: float
    amp: float
    k: float
    phase: float
    layers: int
    dx: float
    x_up: float = 0.0

    def u_in(self, t: float) -> float:
        return self.U * (1.0 + self.amp * math.sin(self.k * self.U * t + self.phase))

    def layer_y(self):
        ny = int(round((self.y1 - self.y0) / self.dx))
        return np.array([self.y0 + (j + 0.5) * self.dx for j in range(ny)])


class OracleSim:
    """Plain FP64 time stepping of the method, state kept in particle-id order."""

    def __init__(self, params: dict, fluid: dict, boundary: dict | None = None,
                 use_cells: bool = True):
        self.p = dict(params)
        self.d = derive(params)
        self.use_cells = use_cells
        n = len(fluid["x"])
        self.st = {
            "x": _f64(fluid["x"]).copy(), "y": _f64(fluid["y"]).copy(),
            "u": _f64(fluid["u"]).copy(), "v": _f64(fluid["v"]).copy(),
            "rho": _f64(fluid["rho"]).copy(), "m": _f64(fluid["m"]).copy(),
            "type": np.asarray(fluid.get("type", np.zeros(n)), dtype=np.uint8).copy(),
            "id": np.arange(n, dtype=np.int64),
        }
        self.next_id = n
        self.boundary = boundary
        self.inflow: Inflow | None = None
        self.t = 0.0
        self.nstep = 0
        self.deleted = 0
        self.last_dt = 0.0
        self.last_eval = None

    # -- inflow set-up ------------------------------------------------------
    def add_inflow(self, x_exit, y0, y1, U, amp, k, phase, layers=3):
        dx = float(self.p["dx"])
        inf = Inflow(x_exit, y0, y1, U, amp, k, phase, int(layers), dx)
        ys = inf.layer_y()
        u0 = inf.u_in(self.t)
        for j in range(inf.layers):
            xj = x_exit - (j + 0.5) * dx
            self._append(np.full(len(ys), xj), ys, u0)
        inf.x_up = x_exit - (inf.layers - 0.5) * dx
        self.inflow = inf

    def _append(self, xs, ys, u0):
        k = len(xs)
        d = self.d
        dxv = float(self.p["dx"])
        m_layer = d.rho0 * (dxv * dxv)
        new = {"x": xs, "y": ys, "u": np.full(k, u0), "v": np.zeros(k),
               "rho": np.full(k, d.rho0), "m": np.full(k, m_layer),
               "type": np.full(k, BUFFER, np.uint8),
               "id": np.arange(self.next_id, self.next_id + k, dtype=np.int64)}
        self.next_id += k
        for key in self.st:
            self.st[key] = np.concatenate([self.st[key], new[key].astype(self.st[key].dtype)])

    # -- one step -------------------------------------------------------------
    def evaluate(self, st=None):
        return evaluate(self.d, self.st if st is None else st, self.boundary, self.use_cells)

    def step(self) -> float:
        """Advance one step; returns the dt used.

        Predictor-corrector of Sec. 2-8 (the scheme of the paper's ref. [48],
        whose formulas the paper does not print), read as Monaghan's form:
          evaluate at n;  X^{1/2} = X^n + dt/2 Xdot^n;
          evaluate at n+1/2;  X* = X^n + dt/2 Xdot^{1/2} (positions with u*);
          X^{n+1} = 2 X* - X^n,   for X in {r, u, rho}.
        dt is the fixed step, or Cr min(dt_f, dt_cv) of Eqs. 30-32 taken
        from the evaluation at n over the fluid particles.
        Buffer particles follow the prescribed inflow velocity through the
        same position update and keep rho = rho0.
        With params["density"] == "summation" the fluid density of each
        evaluation is Eq. 6 at that evaluation's positions instead of the
        integrated Eq. 7, and the state keeps the density of the last
        evaluation (the half step).
        """
        d = self.d
        st = self.st
        fl = st["type"] == FLUID
        bf = st["type"] == BUFFER
        if d.summation:
            # Eq. 6 in place of Eq. 7: each evaluation takes the fluid density
            # from the positions; it is not integrated
            st = dict(st)
            st["rho"] = np.where(fl, summation_density(d, st, self.use_cells), st["rho"])
        ev = self.evaluate(st)
        self.last_eval = ev
        if d.dt_fixed > 0.0:
            dt = d.dt_fixed
        else:
            if not fl.any():
                raise ValueError("adaptive dt needs fluid particles")
            dt = d.courant * min(ev["dt_f"][fl].min(), ev["dt_cv"][fl].min())
        half = 0.5 * dt
        t = self.t
        uin_half = self.inflow.u_in(t + half) if self.inflow else 0.0
        uin_new = self.inflow.u_in(t + dt) if self.inflow else 0.0

        # predictor
        mid = dict(st)
        mid["x"] = st["x"] + half * st["u"]
        mid["y"] = st["y"] + half * st["v"]
        mid["u"] = np.where(fl, st["u"] + half * ev["ax"], st["u"])
        mid["v"] = np.where(fl, st["v"] + half * ev["ay"], st["v"])
        mid["rho"] = np.where(fl, st["rho"] + half * ev["drho"], st["rho"])
        if bf.any():
            mid["u"] = np.where(bf, uin_half, mid["u"])
            mid["v"] = np.where(bf, 0.0, mid["v"])
        if d.summation:
            mid["rho"] = np.where(fl, summation_density(d, mid, self.use_cells), st["rho"])
        ev2 = self.evaluate(mid)

        # corrector
        us = np.where(fl, st["u"] + half * ev2["ax"], mid["u"])
        vs = np.where(fl, st["v"] + half * ev2["ay"], mid["v"])
        rs = np.where(fl, st["rho"] + half * ev2["drho"], st["rho"])
        xs = st["x"] + half * us
        ys = st["y"] + half * vs
        new = dict(st)
        new["x"] = 2.0 * xs - st["x"]
        new["y"] = 2.0 * ys - st["y"]
        new["u"] = 2.0 * us - st["u"]
        new["v"] = 2.0 * vs - st["v"]
        new["rho"] = 2.0 * rs - st["rho"]
        if d.summation:
            new["rho"] = mid["rho"]         # the density of the last evaluation
        if bf.any():
            new["u"] = np.where(bf, uin_new, new["u"])
            new["v"] = np.where(bf, 0.0, new["v"])
            new["rho"] = np.where(bf, st["rho"], new["rho"])
        self.st = new
        self.t = t + dt
        self.nstep += 1
        self.last_dt = dt
        self._inflow_outflow(dt, uin_half, uin_new)
        return dt

    def _inflow_outflow(self, dt, uin_half, uin_new):
        """Buffer-to-fluid conversion, outflow deletion and layer spawning.

        Order: (1) buffer particles with x >= x_exit become fluid; (2) fluid
        particles outside [xmin, xmax) x [ymin, ymax) are deleted; (3) the
        upstream-most layer position advances like a buffer particle, and a
        new layer is laid one spacing upstream of it once it has moved past
        its initial slot x_exit - (layers - 0.5) dx, so that at least ``layers``
        buffer layers (and at most one more) always lie upstream of x_exit.
        """
        d = self.d
        st = self.st
        if self.inflow is not None:
            inf = self.inflow
            conv = (st["type"] == BUFFER) & (st["x"] >= inf.x_exit)
            st["type"][conv] = FLUID
        fl = st["type"] == FLUID
        out = fl & ((st["x"] < d.xmin) | (st["x"] >= d.xmax) |
                    (st["y"] < d.ymin) | (st["y"] >= d.ymax))
        if out.any():
            keep = ~out
            self.deleted += int(out.sum())
            for key in st:
                st[key] = st[key][keep]
        if self.inflow is not None:
            inf = self.inflow
            half = 0.5 * dt
            xs = inf.x_up + half * uin_half
            inf.x_up = 2.0 * xs - inf.x_up
            if inf.x_up >= inf.x_exit - (inf.layers - 0.5) * inf.dx:
                xn = inf.x_up - inf.dx
                ys = inf.layer_y()
                self._append(np.full(len(ys), xn), ys, uin_new)
                inf.x_up = xn

    def run(self, nsteps: int):
        for _ in range(nsteps):
            self.step()

    def breakup_length(self, D: float = 1.0):
        if self.inflow is None:
            raise ValueError("breakup length needs an inflow")
        return breakup_length(self.st, self.d.h, self.inflow.x_exit, D, self.use_cells)
