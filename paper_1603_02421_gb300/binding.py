"""Python binding of libsph (include/sph.h): argument marshalling only.

Every function below has the name of the C entry point it calls and does no
computation of its own: all steps of the method run in the CUDA kernels
behind the C ABI.  There is no fallback: if ``libsph.so`` has not been built
(``paper_1603_02421_gb300.build.build()``) or no GPU is present, the calls
raise.

Arrays are numpy arrays on the host; the library copies inputs and fills
caller-allocated outputs, exactly as the C ABI specifies.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsph.so")

SPH_OK = 0
SPH_ERR_ARG, SPH_ERR_OOM, SPH_ERR_CAPACITY, SPH_ERR_CUDA = -1, -2, -3, -4
SPH_ERR_NONFINITE, SPH_ERR_TIMEOUT, SPH_ERR_STATE, SPH_ERR_SKIN = -5, -6, -7, -8
STATUS = {0: "SPH_OK", -1: "SPH_ERR_ARG", -2: "SPH_ERR_OOM", -3: "SPH_ERR_CAPACITY",
          -4: "SPH_ERR_CUDA", -5: "SPH_ERR_NONFINITE", -6: "SPH_ERR_TIMEOUT",
          -7: "SPH_ERR_STATE", -8: "SPH_ERR_SKIN"}
FLUID, BOUNDARY, BUFFER = 0, 1, 2
START_GATED, START_CONDITIONAL = 0, 1       # sph_start_form
KERNELS = {"cubic": 0, "wendland": 1}
PRECISIONS = {"fp32": 0, "fp64": 1}


class SphError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


class sph_params(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int), ("precision", ctypes.c_int),
                ("dx", ctypes.c_double), ("h_over_dx", ctypes.c_double),
                ("rho0", ctypes.c_double), ("c0", ctypes.c_double), ("gamma", ctypes.c_double),
                ("alpha", ctypes.c_double), ("eta2_over_h2", ctypes.c_double),
                ("sigma", ctypes.c_double), ("eps_n_times_h", ctypes.c_double),
                ("gx", ctypes.c_double), ("gy", ctypes.c_double),
                ("courant", ctypes.c_double), ("dt_fixed", ctypes.c_double),
                ("xmin", ctypes.c_double), ("ymin", ctypes.c_double),
                ("xmax", ctypes.c_double), ("ymax", ctypes.c_double),
                ("skin_over_h", ctypes.c_double), ("wall_A_coef", ctypes.c_double),
                ("wall_h0", ctypes.c_double), ("wall_db_over_dx", ctypes.c_double),
                ("u_frame_x", ctypes.c_double), ("u_frame_y", ctypes.c_double),
                ("capacity", ctypes.c_longlong), ("boundary_capacity", ctypes.c_longlong),
                ("cuda_stream", ctypes.c_void_p), ("device", ctypes.c_int),
                ("density", ctypes.c_int)]


_D = ctypes.POINTER(ctypes.c_double)
_U8 = ctypes.POINTER(ctypes.c_ubyte)
_U32 = ctypes.POINTER(ctypes.c_uint)
_LL = ctypes.POINTER(ctypes.c_longlong)
_CTX = ctypes.c_void_p
_F32 = ctypes.POINTER(ctypes.c_float)
_I32 = ctypes.POINTER(ctypes.c_int)

_SIGS = {
    "sph_init": ([ctypes.POINTER(sph_params), ctypes.POINTER(_CTX)], ctypes.c_int),
    "sph_destroy": ([_CTX], None),
    "sph_last_error": ([_CTX], ctypes.c_char_p),
    "sph_add_particles": ([_CTX, ctypes.c_longlong, _D, _D, _D, _D, _D, _D, _U8, _D, _D],
                          ctypes.c_int),
    "sph_inflow": ([_CTX] + [ctypes.c_double] * 7 + [ctypes.c_int], ctypes.c_int),
    "sph_step": ([_CTX, _D], ctypes.c_int),
    "sph_run": ([_CTX, ctypes.c_longlong, ctypes.c_int, ctypes.c_double, _D, _LL],
                ctypes.c_int),
    "sph_breakup_length": ([_CTX, ctypes.c_double, _D, ctypes.POINTER(ctypes.c_int)],
                           ctypes.c_int),
    "sph_evaluate": ([_CTX], ctypes.c_int),
    "sph_get_state": ([_CTX, ctypes.c_longlong, _LL, _D, _D, _D, _D, _D, _D, _U8, _U32, _D,
                       _D, _D], ctypes.c_int),
    "sph_set_state": ([_CTX, ctypes.c_longlong, _D, _D, _D, _D, _D, _D, _U8, _U32],
                      ctypes.c_int),
    "sph_get_csf": ([_CTX, ctypes.c_longlong, _LL, _U32, _D, _D, _D], ctypes.c_int),
    "sph_get_pairs": ([_CTX, ctypes.c_longlong, _U32, _U32, _LL], ctypes.c_int),
    "sph_get_time": ([_CTX, _D, _LL, _LL, _LL], ctypes.c_int),
    "sph_kernel_counts": ([_CTX, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                           ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "sph_get_rebuild_stats": ([_CTX, _LL, _D, _D], ctypes.c_int),
    "sph_request_rebuild": ([_CTX], ctypes.c_int),
    "sph_checkpoint_size": ([_CTX, ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "sph_checkpoint_save": ([_CTX, ctypes.c_void_p, ctypes.c_size_t,
                             ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "sph_checkpoint_load": ([_CTX, ctypes.c_void_p, ctypes.c_size_t], ctypes.c_int),
    "sph_stats": ([_CTX, ctypes.c_void_p], ctypes.c_int),
    "sph_fma_peak": ([ctypes.c_int, ctypes.c_int, _D, _D], ctypes.c_int),
    "sph_ensemble_create": ([ctypes.POINTER(_CTX), ctypes.c_int, ctypes.c_void_p,
                             ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
    "sph_ensemble_run": ([ctypes.c_void_p, ctypes.c_longlong], ctypes.c_int),
    "sph_ensemble_sync": ([ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "sph_ensemble_surrogate_step": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_int, ctypes.POINTER(ctypes.c_int), _D, _D, _D,
                                     ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "sph_ensemble_autotune": ([ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                               ctypes.POINTER(ctypes.c_int), _D], ctypes.c_int),
    "sph_ensemble_destroy": ([ctypes.c_void_p], None),
    "sph_ensemble_last_error": ([ctypes.c_void_p], ctypes.c_char_p),
    "sph_mpnn_param_count": ([], ctypes.c_longlong),
    "sph_mpnn_create": ([ctypes.c_int, ctypes.c_longlong, ctypes.POINTER(ctypes.c_void_p)],
                        ctypes.c_int),
    "sph_mpnn_destroy": ([ctypes.c_void_p], None),
    "sph_mpnn_last_error": ([ctypes.c_void_p], ctypes.c_char_p),
    "sph_mpnn_set_params": ([ctypes.c_void_p, _F32, ctypes.c_longlong], ctypes.c_int),
    "sph_mpnn_get_params": ([ctypes.c_void_p, _F32, ctypes.c_longlong], ctypes.c_int),
    "sph_mpnn_get_grads": ([ctypes.c_void_p, _F32, ctypes.c_longlong], ctypes.c_int),
    "sph_mpnn_features": ([ctypes.c_void_p, _CTX, ctypes.c_double, ctypes.c_longlong, _LL, _U32,
                           _F32, ctypes.c_longlong, _LL, _I32, _I32, _F32], ctypes.c_int),
    "sph_mpnn_forward": ([ctypes.c_void_p, _CTX, ctypes.c_double, ctypes.c_int,
                          ctypes.c_longlong, _LL, _U32, _F32], ctypes.c_int),
    "sph_mpnn_backward": ([ctypes.c_void_p, _CTX, ctypes.c_double, _F32, ctypes.c_longlong, _D],
                          ctypes.c_int),
    "sph_mpnn_adam": ([ctypes.c_void_p, ctypes.c_double], ctypes.c_int),
    "sph_mpnn_inject_stall": ([ctypes.c_void_p, ctypes.c_int], ctypes.c_int),
    "sph_surrogate_step": ([_CTX, ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                            ctypes.c_double, ctypes.c_int, ctypes.POINTER(ctypes.c_int), _D, _D,
                            _D], ctypes.c_int),
    "sph_surrogate_batch": ([ctypes.POINTER(_CTX), ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                             ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                             ctypes.POINTER(ctypes.c_int), _D, _D, _D,
                             ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "sph_run_async": ([_CTX, ctypes.c_longlong], ctypes.c_int),
    "sph_set_tuning": ([_CTX, ctypes.c_int, ctypes.c_int], ctypes.c_int),
    "sph_set_start_form": ([_CTX, ctypes.c_int], ctypes.c_int),
    "sph_get_start_form": ([_CTX, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "sph_get_tuning": ([_CTX, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)],
                       ctypes.c_int),
    "sph_autotune": ([_CTX, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                      ctypes.POINTER(ctypes.c_int), _D], ctypes.c_int),
    "sph_pairs_noalloc": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_longlong] +
                          [ctypes.c_double] * 5 + [ctypes.c_void_p, ctypes.c_void_p,
                                                   ctypes.c_longlong, _LL, ctypes.c_void_p],
                          ctypes.c_int),
    "sph_sync": ([_CTX], ctypes.c_int),
    "sph_profile": ([_CTX, ctypes.c_int], ctypes.c_int),
    "sph_profile_report": ([_CTX, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                            ctypes.POINTER(ctypes.c_char_p), _D, _LL], ctypes.c_int),
}

_lib = None


def lib():
    """Load libsph.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise OSError("libsph.so not built: run paper_1603_02421_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _check(ctx, st):
    if st != SPH_OK:
        raise SphError(st, lib().sph_last_error(ctx).decode(errors="replace"))


def _d(a):
    return None if a is None else a.ctypes.data_as(_D)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def make_params(p: dict, capacity=None, boundary_capacity=0, stream=None, device=0):
    """sph_params from a configuration dict (see workloads.py)."""
    cap = int(capacity if capacity is not None else p.get("capacity", 0))
    return sph_params(
        kernel=KERNELS[p.get("kernel", "wendland")],
        precision=PRECISIONS[p.get("prec", "fp32")],
        dx=p["dx"], h_over_dx=p.get("h_over_dx", 1.3), rho0=p.get("rho0", 1000.0),
        c0=p["c0"], gamma=p.get("gamma", 7.0), alpha=p.get("alpha", 0.0),
        eta2_over_h2=p.get("eta2_over_h2", 0.01), sigma=p.get("sigma", 0.0),
        eps_n_times_h=p.get("eps_n_times_h", 0.01), gx=p.get("gx", 0.0),
        gy=p.get("gy", 0.0), courant=p.get("courant", 0.2), dt_fixed=p.get("dt_fixed", 0.0),
        xmin=p["xmin"], ymin=p["ymin"], xmax=p["xmax"], ymax=p["ymax"],
        skin_over_h=p.get("skin_over_h", 0.2), wall_A_coef=p.get("wall_A_coef", 0.01),
        wall_h0=p.get("wall_h0", 0.0), wall_db_over_dx=p.get("wall_db_over_dx", 0.5),
        u_frame_x=p.get("u_frame_x", 0.0), u_frame_y=p.get("u_frame_y", 0.0),
        capacity=cap, boundary_capacity=int(boundary_capacity),
        cuda_stream=stream, device=int(device),
        density=1 if p.get("density", "continuity") == "summation" else 0)


# ---------------------------------------------------------------------------
# entry points
# ---------------------------------------------------------------------------
def sph_init(params: sph_params):
    ctx = _CTX()
    st = lib().sph_init(ctypes.byref(params), ctypes.byref(ctx))
    _check(None, st)
    return ctx


def sph_destroy(ctx):
    lib().sph_destroy(ctx)


def sph_add_particles(ctx, x, y, u=None, v=None, rho=None, mass=None, type=None, nx=None,
                      ny=None):
    x, y = _f64(x), _f64(y)
    n = len(x)
    u, v, rho, mass, nx, ny = (_f64(a) for a in (u, v, rho, mass, nx, ny))
    t = np.ascontiguousarray(type if type is not None else np.zeros(n), dtype=np.uint8)
    _check(ctx, lib().sph_add_particles(ctx, n, _d(x), _d(y), _d(u), _d(v), _d(rho), _d(mass),
                                        t.ctypes.data_as(_U8), _d(nx), _d(ny)))


def sph_inflow(ctx, x_exit, y0, y1, U, amp, k, phase, layers):
    _check(ctx, lib().sph_inflow(ctx, x_exit, y0, y1, U, amp, k, phase, int(layers)))


def sph_step(ctx) -> float:
    dt = ctypes.c_double()
    _check(ctx, lib().sph_step(ctx, ctypes.byref(dt)))
    return dt.value


def sph_run(ctx, nsteps, breakup_every=0, D=1.0):
    cnt = nsteps // breakup_every if breakup_every > 0 else 0
    L = np.zeros(max(cnt, 1))
    nL = ctypes.c_longlong()
    _check(ctx, lib().sph_run(ctx, int(nsteps), int(breakup_every), float(D),
                              _d(L) if breakup_every > 0 else None,
                              ctypes.byref(nL) if breakup_every > 0 else None))
    return L[:nL.value]


def sph_breakup_length(ctx, D=1.0):
    L = ctypes.c_double()
    b = ctypes.c_int()
    _check(ctx, lib().sph_breakup_length(ctx, float(D), ctypes.byref(L), ctypes.byref(b)))
    return L.value, bool(b.value)


def sph_evaluate(ctx):
    _check(ctx, lib().sph_evaluate(ctx))


def sph_get_state(ctx, cap=None) -> dict:
    if cap is None:
        n = ctypes.c_longlong()
        st = lib().sph_get_state(ctx, 0, ctypes.byref(n), *([None] * 11))
        if st not in (SPH_OK, -3):
            _check(ctx, st)
        cap = n.value
    out = {k: np.zeros(max(cap, 1)) for k in ("x", "y", "u", "v", "rho", "m", "ax", "ay",
                                                "drho")}
    out["type"] = np.zeros(max(cap, 1), np.uint8)
    out["id"] = np.zeros(max(cap, 1), np.uint32)
    n = ctypes.c_longlong()
    _check(ctx, lib().sph_get_state(ctx, cap, ctypes.byref(n), _d(out["x"]), _d(out["y"]),
                                    _d(out["u"]), _d(out["v"]), _d(out["rho"]), _d(out["m"]),
                                    out["type"].ctypes.data_as(_U8),
                                    out["id"].ctypes.data_as(_U32), _d(out["ax"]),
                                    _d(out["ay"]), _d(out["drho"])))
    return {k: a[:n.value] for k, a in out.items()}


def sph_set_state(ctx, st: dict):
    x = _f64(st["x"])
    n = len(x)
    ids = np.ascontiguousarray(st["id"], dtype=np.uint32)
    t = np.ascontiguousarray(st["type"], dtype=np.uint8)
    _check(ctx, lib().sph_set_state(ctx, n, _d(x), _d(_f64(st["y"])), _d(_f64(st["u"])),
                                    _d(_f64(st["v"])), _d(_f64(st["rho"])),
                                    _d(_f64(st["m"])), t.ctypes.data_as(_U8),
                                    ids.ctypes.data_as(_U32)))


def sph_get_csf(ctx, cap) -> dict:
    out = {"C": np.zeros(max(cap, 1)), "nx": np.zeros(max(cap, 1)), "ny": np.zeros(max(cap, 1)),
           "id": np.zeros(max(cap, 1), np.uint32)}
    n = ctypes.c_longlong()
    _check(ctx, lib().sph_get_csf(ctx, cap, ctypes.byref(n), out["id"].ctypes.data_as(_U32),
                                  _d(out["C"]), _d(out["nx"]), _d(out["ny"])))
    return {k: a[:n.value] for k, a in out.items()}


def sph_get_pairs(ctx, cap):
    a = np.zeros(max(cap, 1), np.uint32)
    b = np.zeros(max(cap, 1), np.uint32)
    n = ctypes.c_longlong()
    _check(ctx, lib().sph_get_pairs(ctx, cap, a.ctypes.data_as(_U32), b.ctypes.data_as(_U32),
                                    ctypes.byref(n)))
    return a[:n.value], b[:n.value]


def sph_get_time(ctx):
    t = ctypes.c_double()
    s, n, d = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_longlong()
    _check(ctx, lib().sph_get_time(ctx, ctypes.byref(t), ctypes.byref(s), ctypes.byref(n),
                                   ctypes.byref(d)))
    return {"t": t.value, "steps": s.value, "n": n.value, "deleted": d.value}


def sph_kernel_counts(ctx):
    """(kernels of a rebuilding step, of a step reusing the build, of a
    breakup-length evaluation)."""
    a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(ctx, lib().sph_kernel_counts(ctx, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return a.value, b.value, c.value


def sph_get_rebuild_stats(ctx):
    """(cell builds so far, largest displacement since the build, largest move
    of the last step) as seen by the last step's rebuild decision."""
    b, d, m = ctypes.c_longlong(), ctypes.c_double(), ctypes.c_double()
    _check(ctx, lib().sph_get_rebuild_stats(ctx, ctypes.byref(b), ctypes.byref(d),
                                            ctypes.byref(m)))
    return b.value, d.value, m.value


class sph_stats_t(ctypes.Structure):
    _fields_ = [("n_fluid", ctypes.c_longlong), ("n_buffer", ctypes.c_longlong),
                ("n_boundary", ctypes.c_longlong), ("n_deleted", ctypes.c_longlong),
                ("step", ctypes.c_longlong), ("t", ctypes.c_double), ("dt", ctypes.c_double),
                ("mass", ctypes.c_double), ("momentum_x", ctypes.c_double),
                ("momentum_y", ctypes.c_double), ("kinetic", ctypes.c_double),
                ("potential", ctypes.c_double), ("elastic", ctypes.c_double),
                ("max_rel_density", ctypes.c_double)]


def sph_stats(ctx) -> dict:
    """Run statistics of the current state (see include/sph.h)."""
    st = sph_stats_t()
    _check(ctx, lib().sph_stats(ctx, ctypes.byref(st)))
    return {name: getattr(st, name) for name, _ in sph_stats_t._fields_}


def sph_checkpoint_size(ctx) -> int:
    n = ctypes.c_size_t()
    _check(ctx, lib().sph_checkpoint_size(ctx, ctypes.byref(n)))
    return n.value


def sph_checkpoint_save(ctx) -> bytes:
    """The context's checkpoint as bytes."""
    cap = sph_checkpoint_size(ctx)
    buf = ctypes.create_string_buffer(max(cap, 1))
    n = ctypes.c_size_t()
    _check(ctx, lib().sph_checkpoint_save(ctx, buf, cap, ctypes.byref(n)))
    return buf.raw[:n.value]


def sph_checkpoint_load(ctx, data: bytes):
    buf = ctypes.create_string_buffer(data, len(data))
    _check(ctx, lib().sph_checkpoint_load(ctx, buf, len(data)))


def sph_request_rebuild(ctx):
    """The next step rebuilds the cells and neighbour lists."""
    _check(ctx, lib().sph_request_rebuild(ctx))


def sph_fma_peak(device=0, precision=0):
    """(TFLOP/s, ms of the best launch) of the device's FMA pipes in FP32
    (precision 0) or FP64 (1)."""
    t, ms = ctypes.c_double(), ctypes.c_double()
    st = lib().sph_fma_peak(int(device), int(precision), ctypes.byref(t), ctypes.byref(ms))
    if st != SPH_OK:
        raise SphError(st, "sph_fma_peak failed")
    return t.value, ms.value


def sph_set_tuning(ctx, lanes, cadence):
    _check(ctx, lib().sph_set_tuning(ctx, int(lanes), int(cadence)))


def sph_get_tuning(ctx):
    a, b = ctypes.c_int(), ctypes.c_int()
    _check(ctx, lib().sph_get_tuning(ctx, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def sph_set_start_form(ctx, form):
    """form: START_GATED or START_CONDITIONAL (how a step at cadence > 1 picks
    its start on the device; the results are identical)."""
    _check(ctx, lib().sph_set_start_form(ctx, int(form)))


def sph_get_start_form(ctx):
    f = ctypes.c_int()
    _check(ctx, lib().sph_get_start_form(ctx, ctypes.byref(f)))
    return f.value


def sph_autotune(ctx, trial_steps=20):
    a, b, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    _check(ctx, lib().sph_autotune(ctx, int(trial_steps), ctypes.byref(a), ctypes.byref(b),
                                   ctypes.byref(ms)))
    return a.value, b.value, ms.value


def sph_run_async(ctx, nsteps):
    _check(ctx, lib().sph_run_async(ctx, int(nsteps)))


def sph_sync(ctx):
    _check(ctx, lib().sph_sync(ctx))


def sph_profile(ctx, enable):
    _check(ctx, lib().sph_profile(ctx, int(bool(enable))))


def sph_profile_report(ctx, cap=64) -> dict:
    n = ctypes.c_int()
    names = (ctypes.c_char_p * cap)()
    ms = np.zeros(cap)
    cnt = np.zeros(cap, np.int64)
    _check(ctx, lib().sph_profile_report(ctx, cap, ctypes.byref(n), names, _d(ms),
                                         cnt.ctypes.data_as(_LL)))
    return {names[k].decode(): (float(ms[k]), int(cnt[k])) for k in range(n.value)}


def sph_pairs_noalloc(x_ptr, y_ptr, n, h, box, a_ptr, b_ptr, cap, stream=None):
    """Neighbour pairs on caller-owned device buffers (raw device pointers as
    ints, e.g. torch tensors' data_ptr()); allocates no device memory.
    Returns the pair count."""
    npairs = ctypes.c_longlong()
    st = lib().sph_pairs_noalloc(x_ptr, y_ptr, int(n), float(h), float(box[0]), float(box[1]),
                                 float(box[2]), float(box[3]), a_ptr, b_ptr, int(cap),
                                 ctypes.byref(npairs), stream)
    if st != SPH_OK:
        err = SphError(st, "sph_pairs_noalloc failed (%d pairs found)" % npairs.value)
        err.count = npairs.value
        raise err
    return npairs.value


# ---------------------------------------------------------------------------
# convenience: a context built from a workload case
# ---------------------------------------------------------------------------
class Simulation:
    """A libsph context for a case dict of ``workloads`` (owns the context)."""

    def __init__(self, case: dict, capacity=None, stream=None, device=0, prec=None):
        p = dict(case["params"])
        if prec is not None:
            p["prec"] = prec
        fl = case["fluid"]
        bd = case.get("boundary")
        nb = 0 if bd is None else len(bd["x"])
        cap = capacity or p.get("capacity") or (len(fl["x"]) + 64)
        self.params = make_params(p, capacity=cap, boundary_capacity=nb, stream=stream,
                                  device=device)
        self.ctx = sph_init(self.params)
        try:
            sph_add_particles(self.ctx, fl["x"], fl["y"], fl["u"], fl["v"], fl["rho"], fl["m"],
                              fl["type"])
            if nb:
                z = np.zeros(nb)
                sph_add_particles(self.ctx, bd["x"], bd["y"], z, z, np.full(nb, p["rho0"]),
                                  np.ones(nb), np.full(nb, BOUNDARY, np.uint8), bd["nx"],
                                  bd["ny"])
            inf = case.get("inflow")
            if inf is not None:
                sph_inflow(self.ctx, inf["x_exit"], inf["y0"], inf["y1"], inf["U"], inf["amp"],
                           inf["k"], inf["phase"], inf["layers"])
        except Exception:
            sph_destroy(self.ctx)
            self.ctx = None
            raise

    def close(self):
        if self.ctx is not None:
            sph_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self):
        return sph_step(self.ctx)

    def run(self, nsteps, breakup_every=0, D=1.0):
        return sph_run(self.ctx, nsteps, breakup_every, D)

    def evaluate(self):
        sph_evaluate(self.ctx)

    def state(self):
        return sph_get_state(self.ctx)

    def set_state(self, st):
        sph_set_state(self.ctx, st)

    def csf(self, cap):
        return sph_get_csf(self.ctx, cap)

    def pairs(self, cap):
        return sph_get_pairs(self.ctx, cap)

    def breakup_length(self, D=1.0):
        return sph_breakup_length(self.ctx, D)

    def time(self):
        return sph_get_time(self.ctx)

    def set_tuning(self, lanes, cadence):
        sph_set_tuning(self.ctx, lanes, cadence)

    def tuning(self):
        return sph_get_tuning(self.ctx)

    def set_start_form(self, form):
        sph_set_start_form(self.ctx, form)

    def start_form(self):
        return sph_get_start_form(self.ctx)

    def autotune(self, trial_steps=20):
        return sph_autotune(self.ctx, trial_steps)

    def rebuild_stats(self):
        return sph_get_rebuild_stats(self.ctx)

    def kernels_per_step(self):
        return sph_kernel_counts(self.ctx)[0]


def _ens_check(ens, st, bad=None):
    if st != SPH_OK:
        err = SphError(st, lib().sph_ensemble_last_error(ens).decode(errors="replace"))
        err.member = bad
        raise err


def sph_ensemble_last_error(ens=None):
    return lib().sph_ensemble_last_error(ens).decode(errors="replace")


def sph_ensemble_create(ctxs, stream=None):
    arr = (_CTX * len(ctxs))(*ctxs)
    out = ctypes.c_void_p()
    _ens_check(None, lib().sph_ensemble_create(arr, len(ctxs), stream, ctypes.byref(out)))
    return out.value


def sph_ensemble_run(ens, nsteps):
    _ens_check(ens, lib().sph_ensemble_run(ens, int(nsteps)))


def sph_ensemble_sync(ens):
    """Raises SphError with .member = index of the failing member."""
    bad = ctypes.c_int(-1)
    st = lib().sph_ensemble_sync(ens, ctypes.byref(bad))
    _ens_check(ens, st, bad.value)


def sph_ensemble_surrogate_step(ens, m, net, k, u_ref, a_ref, threshold, bf16=True):
    """One surrogate step of each of the m members (sph_surrogate_batch over
    the ensemble); returns (accepted, momentum, density, field residuals) as
    numpy arrays of m."""
    acc = (ctypes.c_int * max(m, 1))()
    rm, rd, rf = (np.zeros(max(m, 1)) for _ in range(3))
    bad = ctypes.c_int(-1)
    st = lib().sph_ensemble_surrogate_step(ens, net, int(k), float(u_ref), float(a_ref),
                                           float(threshold), int(bool(bf16)), acc, _d(rm),
                                           _d(rd), _d(rf), ctypes.byref(bad))
    _ens_check(ens, st, bad.value)
    return (np.array([bool(acc[i]) for i in range(m)]), rm[:m], rd[:m], rf[:m])


def sph_ensemble_autotune(ens, trial_steps=16):
    a, b, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    _ens_check(ens, lib().sph_ensemble_autotune(ens, int(trial_steps), ctypes.byref(a),
                                                ctypes.byref(b), ctypes.byref(ms)))
    return a.value, b.value, ms.value


def sph_ensemble_destroy(ens):
    lib().sph_ensemble_destroy(ens)


class Ensemble:
    """Several Simulations advanced together, one CUDA graph launch per
    ensemble step (sph_ensemble_*).  The Simulations stay owned by the
    caller and must outlive the Ensemble."""

    def __init__(self, sims, stream=None):
        self.sims = list(sims)
        self.ens = None
        self.ens = sph_ensemble_create([s.ctx for s in self.sims], stream)

    def run_async(self, nsteps):
        sph_ensemble_run(self.ens, nsteps)

    def sync(self):
        sph_ensemble_sync(self.ens)

    def run(self, nsteps):
        self.run_async(nsteps)
        self.sync()

    def autotune(self, trial_steps=16):
        return sph_ensemble_autotune(self.ens, trial_steps)

    def surrogate_step(self, net, k, u_ref, a_ref, threshold, bf16=True):
        """One surrogate step of every member; (accepted, residuals...)."""
        return sph_ensemble_surrogate_step(self.ens, len(self.sims), net, k, u_ref, a_ref,
                                           threshold, bf16)

    def close(self):
        if getattr(self, "ens", None):
            sph_ensemble_destroy(self.ens)
            self.ens = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# learned surrogate
# ---------------------------------------------------------------------------
def _mp_check(net, st):
    if st != SPH_OK:
        raise SphError(st, lib().sph_mpnn_last_error(net).decode(errors="replace"))


def _f32p(a):
    return a.ctypes.data_as(_F32)


def sph_mpnn_param_count():
    return int(lib().sph_mpnn_param_count())


def sph_mpnn_last_error(net=None):
    return lib().sph_mpnn_last_error(net).decode(errors="replace")


def sph_mpnn_create(capacity, device=0):
    out = ctypes.c_void_p()
    _mp_check(None, lib().sph_mpnn_create(int(device), int(capacity), ctypes.byref(out)))
    return out.value


def sph_mpnn_destroy(net):
    lib().sph_mpnn_destroy(net)


def sph_mpnn_set_params(net, flat):
    a = np.ascontiguousarray(flat, dtype=np.float32)
    _mp_check(net, lib().sph_mpnn_set_params(net, _f32p(a), a.size))


def sph_mpnn_get_params(net):
    a = np.zeros(sph_mpnn_param_count(), np.float32)
    _mp_check(net, lib().sph_mpnn_get_params(net, _f32p(a), a.size))
    return a


def sph_mpnn_get_grads(net):
    a = np.zeros(sph_mpnn_param_count(), np.float32)
    _mp_check(net, lib().sph_mpnn_get_grads(net, _f32p(a), a.size))
    return a


def sph_mpnn_features(net, ctx, u_ref, cap, ecap):
    """(ids, x[n,4], ea, eb, w[ne,4]) in the context's cell order."""
    n, ne = ctypes.c_longlong(), ctypes.c_longlong()
    ids = np.zeros(cap, np.uint32)
    x = np.zeros((cap, 4), np.float32)
    ea = np.zeros(ecap, np.int32)
    eb = np.zeros(ecap, np.int32)
    w = np.zeros((ecap, 4), np.float32)
    _mp_check(net, lib().sph_mpnn_features(net, ctx, float(u_ref), int(cap), ctypes.byref(n),
                                           ids.ctypes.data_as(_U32), _f32p(x), int(ecap),
                                           ctypes.byref(ne), ea.ctypes.data_as(_I32),
                                           eb.ctypes.data_as(_I32), _f32p(w)))
    k, m = n.value, ne.value
    return ids[:k], x[:k], ea[:m], eb[:m], w[:m]


def sph_mpnn_forward(net, ctx, u_ref, bf16, cap):
    """(ids, y[n,2]) in the context's cell order."""
    n = ctypes.c_longlong()
    ids = np.zeros(cap, np.uint32)
    y = np.zeros((cap, 2), np.float32)
    _mp_check(net, lib().sph_mpnn_forward(net, ctx, float(u_ref), int(bool(bf16)), int(cap),
                                          ctypes.byref(n), ids.ctypes.data_as(_U32), _f32p(y)))
    return ids[:n.value], y[:n.value]


def sph_mpnn_backward(net, ctx, u_ref, target):
    t = np.ascontiguousarray(target, dtype=np.float32)
    loss = ctypes.c_double()
    _mp_check(net, lib().sph_mpnn_backward(net, ctx, float(u_ref), _f32p(t), len(t),
                                           ctypes.byref(loss)))
    return loss.value


def sph_mpnn_adam(net, lr):
    _mp_check(net, lib().sph_mpnn_adam(net, float(lr)))


def sph_mpnn_inject_stall(net, on):
    """Test hook: the following inference passes issue no operand loads, so
    their bounded waits run out and the calls report SPH_ERR_TIMEOUT."""
    _mp_check(net, lib().sph_mpnn_inject_stall(net, int(bool(on))))


def sph_surrogate_batch(ctxs, net, k, u_ref, a_ref, threshold, bf16=True):
    """One surrogate step on each context of the list, sharing the host
    synchronisations; returns (accepted, momentum, density, field residuals)
    as numpy arrays of len(ctxs)."""
    m = len(ctxs)
    arr = (_CTX * max(m, 1))(*ctxs)
    acc = (ctypes.c_int * max(m, 1))()
    rm, rd, rf = (np.zeros(max(m, 1)) for _ in range(3))
    bad = ctypes.c_int(-1)
    st = lib().sph_surrogate_batch(arr, m, net, int(k), float(u_ref), float(a_ref),
                                   float(threshold), int(bool(bf16)), acc, _d(rm), _d(rd), _d(rf),
                                   ctypes.byref(bad))
    if st != SPH_OK:
        i = bad.value
        msg = lib().sph_last_error(ctxs[i]).decode(errors="replace") if 0 <= i < m else ""
        raise SphError(st, "member %d: %s" % (i, msg))
    return (np.array([bool(acc[i]) for i in range(m)]), rm[:m], rd[:m], rf[:m])


def sph_surrogate_step(ctx, net, k, u_ref, a_ref, threshold, bf16=True, field=False):
    """One surrogate step with plain SPH as judge and fallback; returns
    (accepted, momentum residual, density residual), with field=True also
    the acceleration-field residual."""
    acc = ctypes.c_int()
    rm, rd, rf = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(ctx, lib().sph_surrogate_step(ctx, net, int(k), float(u_ref), float(a_ref),
                                         float(threshold), int(bool(bf16)), ctypes.byref(acc),
                                         ctypes.byref(rm), ctypes.byref(rd), ctypes.byref(rf)))
    if field:
        return bool(acc.value), rm.value, rd.value, rf.value
    return bool(acc.value), rm.value, rd.value


class Mpnn:
    """The learned surrogate (sph_mpnn_*): parameters as a dict of float64
    arrays in the shapes of workloads.mpnn_shapes()."""

    def __init__(self, capacity, device=0):
        self.net = None
        self.net = sph_mpnn_create(capacity, device)

    @staticmethod
    def pack(prm):
        from .workloads import mpnn_shapes
        return np.concatenate([np.asarray(prm[k], np.float64).reshape(-1) for k, _ in mpnn_shapes()])

    @staticmethod
    def unpack(flat):
        from .workloads import mpnn_shapes
        out, o = {}, 0
        for k, shp in mpnn_shapes():
            size = int(np.prod(shp))
            out[k] = np.asarray(flat[o:o + size], np.float64).reshape(shp)
            o += size
        return out

    def set_params(self, prm):
        sph_mpnn_set_params(self.net, self.pack(prm))

    def params(self):
        return self.unpack(sph_mpnn_get_params(self.net))

    def grads(self):
        return self.unpack(sph_mpnn_get_grads(self.net))

    def close(self):
        if getattr(self, "net", None):
            sph_mpnn_destroy(self.net)
            self.net = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
