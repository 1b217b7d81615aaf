"""Seeded synthetic inputs shaped like the paper's workloads.

This module only lays particles out and fills in configuration numbers; it
contains none of the SPH method's arithmetic (no kernel, force, equation of
state or integrator).  Both the CUDA library's tests and benchmark and the
CPU oracle take their inputs from here, so that the two always see
identical, reproducible states.

A *case* is a dict with

* ``params``  -- configuration numbers (kernel, dx, rho0, c0, alpha, sigma, g,
  dt, domain box, precision, ...);
* ``fluid``   -- float64 arrays x, y, u, v, rho, m and uint8 type
  (0 fluid, 2 inflow buffer);
* ``boundary`` -- float64 arrays x, y, nx, ny of fixed wall particles, or None;
* ``inflow``  -- dict(x_exit, y0, y1, U, amp, k, phase, layers) or None.

Workloads (Sec. 3 of the paper; sizes as configured here):

* ``dam_break``: 0.4 m x 0.6 m water column in a 1.6 m x 0.8 m tank with a
  0.12 m square obstacle 0.9 m from the left wall (Sec. 3-1, Fig. 2 scaled),
  dx = 0.01 m, hydrostatic initial density, seed-driven +-0.01 dx jitter.
* ``jet``: single-phase planar jet in nondimensional units (Sec. 3-2),
  nozzle width D, speed U, strip of fluid prefilled over the domain length,
  inflow buffer with a 1 % sinusoidal velocity perturbation whose wavenumber
  is drawn from U[0.5, 1.0]/D by the seed.
"""
from __future__ import annotations

import math

import numpy as np

FLUID, BOUNDARY, BUFFER = 0, 1, 2


def lattice(x0, y0, nx, ny, dx):
    """Cell-centred square lattice of nx*ny points, row-major in y then x."""
    i = np.arange(nx)
    j = np.arange(ny)
    X, Y = np.meshgrid(x0 + (i + 0.5) * dx, y0 + (j + 0.5) * dx)
    return X.ravel().astype(np.float64), Y.ravel().astype(np.float64)


def _fluid(x, y, u=None, v=None, rho=None, m=None, rho0=1000.0, dx=0.01, typ=None):
    n = len(x)
    return {
        "x": np.asarray(x, np.float64), "y": np.asarray(y, np.float64),
        "u": np.zeros(n) if u is None else np.asarray(u, np.float64),
        "v": np.zeros(n) if v is None else np.asarray(v, np.float64),
        "rho": np.full(n, rho0) if rho is None else np.asarray(rho, np.float64),
        "m": np.full(n, rho0 * (dx * dx)) if m is None else np.asarray(m, np.float64),
        "type": np.zeros(n, np.uint8) if typ is None else np.asarray(typ, np.uint8),
    }


# --------------------------------------------------------------------------
# dam break with obstacle
# --------------------------------------------------------------------------
def _segment(p0, p1, spacing, normal, include_end=True):
    L = math.hypot(p1[0] - p0[0], p1[1] - p0[1])
    k = int(round(L / spacing))
    ts = np.arange(k + (1 if include_end else 0)) / max(k, 1)
    xs = p0[0] + ts * (p1[0] - p0[0])
    ys = p0[1] + ts * (p1[1] - p0[1])
    nx = np.full(len(xs), normal[0])
    ny = np.full(len(xs), normal[1])
    return xs, ys, nx, ny


def dam_break_boundary(dx=0.01, tank=(1.6, 0.8), obstacle=(0.9, 0.12, 0.12)):
    """Fixed wall particles at spacing dx/2 with unit normals into the fluid.

    Tank floor and side walls plus the three exposed faces of the obstacle;
    convex and concave corners carry diagonal normals.
    """
    db = 0.5 * dx
    W, H = tank
    ox, ow, oh = obstacle
    s2 = 1.0 / math.sqrt(2.0)
    pts = []
    # floor, left part, right part (excluding the obstacle footprint)
    pts.append(_segment((db, 0.0), (ox - db, 0.0), db, (0.0, 1.0)))
    pts.append(_segment((ox + ow + db, 0.0), (W - db, 0.0), db, (0.0, 1.0)))
    # side walls
    pts.append(_segment((0.0, db), (0.0, H), db, (1.0, 0.0)))
    pts.append(_segment((W, db), (W, H), db, (-1.0, 0.0)))
    # obstacle faces
    pts.append(_segment((ox, db), (ox, oh - db), db, (-1.0, 0.0)))
    pts.append(_segment((ox + db, oh), (ox + ow - db, oh), db, (0.0, 1.0)))
    pts.append(_segment((ox + ow, db), (ox + ow, oh - db), db, (1.0, 0.0)))
    # corners
    corners = [((0.0, 0.0), (s2, s2)), ((W, 0.0), (-s2, s2)),
               ((ox, 0.0), (-s2, s2)), ((ox + ow, 0.0), (s2, s2)),
               ((ox, oh), (-s2, s2)), ((ox + ow, oh), (s2, s2))]
    for (cx, cy), (nx, ny) in corners:
        pts.append((np.array([cx]), np.array([cy]), np.array([nx]), np.array([ny])))
    x = np.concatenate([p[0] for p in pts])
    y = np.concatenate([p[1] for p in pts])
    nx = np.concatenate([p[2] for p in pts])
    ny = np.concatenate([p[3] for p in pts])
    return {"x": x, "y": y, "nx": nx, "ny": ny}


def dam_break(seed=0, dx=0.01, kernel="cubic", prec="fp64", column=(0.4, 0.6),
              alpha=0.01, dt=1e-4, jitter=0.01):
    """2D dam break with an obstacle (Sec. 3-1), configuration of the paper's
    validation case at dx = 0.01 m: ~2.4k fluid and ~0.7k wall particles."""
    rng = np.random.default_rng(seed)
    g = 9.81
    rho0 = 1000.0
    Hc = column[1]
    c0 = 10.0 * math.sqrt(g * Hc)
    gamma = 7.0
    nx = int(round(column[0] / dx))
    ny = int(round(column[1] / dx))
    x, y = lattice(0.0, 0.0, nx, ny, dx)
    x = x + rng.uniform(-jitter * dx, jitter * dx, len(x))
    y = y + rng.uniform(-jitter * dx, jitter * dx, len(y))
    # hydrostatic initial density (inverse of the Tait relation for p = rho0 g (H - y))
    B = rho0 * c0 * c0 / gamma
    rho = rho0 * np.power(1.0 + rho0 * g * (Hc - y) / B, 1.0 / gamma)
    params = dict(kernel=kernel, prec=prec, dx=dx, h_over_dx=1.3, rho0=rho0, c0=c0,
                  gamma=gamma, alpha=alpha, eta2_over_h2=0.01, sigma=0.0,
                  eps_n_times_h=0.01, gx=0.0, gy=-g, courant=0.2, dt_fixed=dt,
                  xmin=-0.1, ymin=-0.1, xmax=1.7, ymax=1.3, skin_over_h=0.1,
                  wall_A_coef=0.01, wall_h0=Hc, wall_db_over_dx=0.5,
                  capacity=len(x) + 64)
    return {"name": "dam_break", "params": params,
            "fluid": _fluid(x, y, rho=rho, rho0=rho0, dx=dx),
            "boundary": dam_break_boundary(dx), "inflow": None}


# --------------------------------------------------------------------------
# planar jet
# --------------------------------------------------------------------------
def jet_params(Re, We, D=1.0, U=1.0, rho0=1000.0, dx=None, kernel="wendland",
               prec="fp32", length=60.0, half_width=5.0, layers=3):
    """Configuration numbers of the nondimensional planar jet.

    sigma = rho U^2 D / We and nu = U D / Re (D-based groups); the artificial
    viscosity coefficient reproduces nu through the 2D relation
    nu = alpha h c0 / 8, i.e. alpha = 8 U D / (Re h c0); c0 = 10 U.
    """
    dx = D / 40.0 if dx is None else dx
    h = 1.3 * dx
    c0 = 10.0 * U
    alpha = 8.0 * U * D / (Re * h * c0)
    sigma = rho0 * U * U * D / We
    return dict(kernel=kernel, prec=prec, dx=dx, h_over_dx=1.3, rho0=rho0, c0=c0,
                gamma=7.0, alpha=alpha, eta2_over_h2=0.01, sigma=sigma,
                eps_n_times_h=0.01, gx=0.0, gy=0.0, courant=0.2, dt_fixed=0.0,
                xmin=-(layers + 5) * dx, ymin=-half_width * D, xmax=length * D,
                ymax=half_width * D, skin_over_h=0.1, wall_A_coef=0.01, wall_h0=0.0,
                wall_db_over_dx=0.5, u_frame_x=U, u_frame_y=0.0)


def jet(seed=0, Re=200.0, We=20.0, D=1.0, U=1.0, rho0=1000.0, dx=None,
        length=60.0, kernel="wendland", prec="fp32", amp=0.01, layers=3,
        fill=None, capacity_factor=1.3, Fr=None, drho=0.0, nozzle=0.0, tank=0.0):
    """Planar jet of width D issuing at x = 0 along +x (Sec. 3-2 setting,
    inflow buffer in place of the paper's tank).  The strip [0, fill*D) is
    prefilled on a dx lattice with u = u_in(-x/U), the velocity the inflow
    had when that fluid left the orifice.  Fr = U / sqrt(g D) (Eq. 36)
    adds gravity along the jet axis (the paper's jets fall from a tank);
    None means no gravity.  drho > 0 adds a seeded uniform density
    perturbation of relative amplitude drho (the density fluctuations of a
    running weakly-compressible flow; 0 gives the uniform start state).
    nozzle > 0 adds a nozzle of that length (in D) upstream of x = 0: walls of
    repulsive boundary particles (Eq. 29) at y = +-D/2, spacing dx/2, normals
    into the channel; the inflow buffer then enters at the nozzle inlet
    x = -nozzle D and the channel is prefilled like the strip (the paper's
    jets leave a tank through a nozzle of aspect ratio 15).  tank > 1 (with
    nozzle > 0) widens that channel into a reservoir of width tank D closed
    by an orifice plate at x = 0 with an opening of width D (Sec. 3-2: the
    jet leaves a particle-filled tank through an orifice; aspect ratio =
    tank height / orifice width): side walls at y = +-tank D/2, the plate's
    two parts facing upstream, diagonal normals at the inner corners and at
    the orifice edges; the inflow then spans the tank width at U / tank (the
    orifice's mass flux) and the tank is prefilled at that speed."""
    rng = np.random.default_rng(seed)
    p = jet_params(Re, We, D=D, U=U, rho0=rho0, dx=dx, kernel=kernel, prec=prec,
                   length=length, layers=layers)
    dx = p["dx"]
    if Fr is not None:
        p["gx"] = U * U / (Fr * Fr * D)
    fill = length if fill is None else fill
    k = rng.uniform(0.5, 1.0) / D
    phase = 0.0
    x0 = -nozzle * D
    if nozzle > 0:
        p["xmin"] = x0 - (layers + 5) * dx
    W = tank * D if (tank > 1.0 and nozzle > 0) else D
    if W > D:
        p["ymin"] = min(p["ymin"], -0.5 * W - 5 * dx)
        p["ymax"] = max(p["ymax"], 0.5 * W + 5 * dx)
    # whole lattice columns inside [x0, fill): the last column centre stays
    # below the box end even when fill is not a whole number of spacings
    nyp = int(round(D / dx))
    if W > D:
        # the tank [x0, 0) x [-W/2, W/2) at U D / W, then the strip [0, fill)
        nxt = int(math.floor(-x0 / dx + 1e-6))
        nyt = int(round(W / dx))
        xt, yt = lattice(x0, -0.5 * W, nxt, nyt, dx)
        nxs = int(math.floor(fill * D / dx + 1e-6))
        xs_, ys_ = lattice(x0 + nxt * dx, -0.5 * D, nxs, nyp, dx)
        x, y = np.concatenate([xt, xs_]), np.concatenate([yt, ys_])
        u = np.concatenate([np.full(len(xt), U * D / W),
                            U * (1.0 + amp * np.sin(k * U * (-xs_ / U) + phase))])
        n_layer = nyt
    else:
        nxp = int(math.floor((fill * D - x0) / dx + 1e-6))
        x, y = lattice(x0, -0.5 * D, nxp, nyp, dx)
        u = U * (1.0 + amp * np.sin(k * U * (-x / U) + phase))
        n_layer = nyp
    rho = rho0 * (1.0 + rng.uniform(-drho, drho, len(x))) if drho > 0 else None
    fluid = _fluid(x, y, u=u, rho=rho, rho0=rho0, dx=dx)
    p["capacity"] = int(capacity_factor * (len(x) + layers * n_layer)) + 1024
    inflow = dict(x_exit=x0, y0=-0.5 * W, y1=0.5 * W, U=U * D / W, amp=amp, k=k, phase=phase,
                  layers=layers)
    boundary = None
    if W > D:
        db = 0.5 * dx
        s2 = 1.0 / math.sqrt(2.0)
        pts = [_segment((x0, 0.5 * W), (-db, 0.5 * W), db, (0.0, -1.0)),       # side walls
               _segment((x0, -0.5 * W), (-db, -0.5 * W), db, (0.0, 1.0)),
               _segment((0.0, 0.5 * D + db), (0.0, 0.5 * W - db), db, (-1.0, 0.0)),   # plate
               _segment((0.0, -0.5 * W + db), (0.0, -0.5 * D - db), db, (-1.0, 0.0))]
        corners = [((0.0, 0.5 * W), (-s2, -s2)), ((0.0, -0.5 * W), (-s2, s2)),   # inner corners
                   ((0.0, 0.5 * D), (-s2, -s2)), ((0.0, -0.5 * D), (-s2, s2))]   # orifice edges
        for (cx, cy), (nx_, ny_) in corners:
            pts.append((np.array([cx]), np.array([cy]), np.array([nx_]), np.array([ny_])))
        boundary = {"x": np.concatenate([q[0] for q in pts]), "y": np.concatenate([q[1] for q in pts]),
                    "nx": np.concatenate([q[2] for q in pts]), "ny": np.concatenate([q[3] for q in pts])}
    elif nozzle > 0:
        db = 0.5 * dx
        top = _segment((x0, 0.5 * D), (0.0, 0.5 * D), db, (0.0, -1.0))
        bot = _segment((x0, -0.5 * D), (0.0, -0.5 * D), db, (0.0, 1.0))
        boundary = {"x": np.concatenate([top[0], bot[0]]), "y": np.concatenate([top[1], bot[1]]),
                    "nx": np.concatenate([top[2], bot[2]]), "ny": np.concatenate([top[3], bot[3]])}
    return {"name": "jet", "params": p, "fluid": fluid, "boundary": boundary, "inflow": inflow,
            "D": D, "nozzle": nozzle * D, "tank": W}


# --------------------------------------------------------------------------
# small test states
# --------------------------------------------------------------------------
def random_cloud(seed=0, n=500, box=(1.0, 1.0), dx=0.05, vel=0.1, drho=0.01, rho0=1000.0):
    """Particles at uniform random positions with random velocity and density."""
    rng = np.random.default_rng(seed)
    x = rng.uniform(0.0, box[0], n)
    y = rng.uniform(0.0, box[1], n)
    u = rng.normal(0.0, vel, n)
    v = rng.normal(0.0, vel, n)
    rho = rho0 * (1.0 + rng.uniform(-drho, drho, n))
    return _fluid(x, y, u, v, rho, rho0=rho0, dx=dx)


def jittered_patch(seed=0, nx=40, ny=30, dx=0.02, jitter=0.05, vel=0.05, drho=0.005,
                   rho0=1000.0, x0=0.0, y0=0.0):
    """Lattice patch with seeded position jitter, velocities and densities."""
    rng = np.random.default_rng(seed)
    x, y = lattice(x0, y0, nx, ny, dx)
    x = x + rng.uniform(-jitter * dx, jitter * dx, len(x))
    y = y + rng.uniform(-jitter * dx, jitter * dx, len(y))
    u = rng.normal(0.0, vel, len(x))
    v = rng.normal(0.0, vel, len(x))
    rho = rho0 * (1.0 + rng.uniform(-drho, drho, len(x)))
    return _fluid(x, y, u, v, rho, rho0=rho0, dx=dx)


def disc(R=1.0, dx=0.05, rho0=1000.0, cx=0.0, cy=0.0):
    """Lattice points inside a circle of radius R (a 2D drop)."""
    n = int(math.ceil(2 * R / dx)) + 2
    x, y = lattice(cx - n * dx / 2, cy - n * dx / 2, n, n, dx)
    keep = (x - cx) ** 2 + (y - cy) ** 2 < R * R
    return _fluid(x[keep], y[keep], rho0=rho0, dx=dx)


def test_params(kernel="wendland", dx=0.02, sigma=0.0, alpha=0.1, c0=10.0, g=0.0,
                box=(-1.0, -1.0, 2.0, 2.0), prec="fp32", dt_fixed=0.0, rho0=1000.0):
    """A parameter set for small test states."""
    return dict(kernel=kernel, prec=prec, dx=dx, h_over_dx=1.3, rho0=rho0, c0=c0,
                gamma=7.0, alpha=alpha, eta2_over_h2=0.01, sigma=sigma,
                eps_n_times_h=0.01, gx=0.0, gy=-g, courant=0.2, dt_fixed=dt_fixed,
                xmin=box[0], ymin=box[1], xmax=box[2], ymax=box[3], skin_over_h=0.1,
                wall_A_coef=0.01, wall_h0=0.0, wall_db_over_dx=0.5, capacity=0)


# ---------------------------------------------------------------------------
# Learned surrogate: shapes and seeded initial weights (random draws only;
# the network's arithmetic lives in the CUDA library and, for tests, in the
# oracle's reference).
# ---------------------------------------------------------------------------
MPNN_IN, MPNN_H, MPNN_P, MPNN_L, MPNN_OUT = 4, 128, 32, 3, 2


def mpnn_shapes():
    """Parameter tensors in their packed order: (name, shape)."""
    shp = [("W_in", (MPNN_IN, MPNN_H)), ("b_in", (MPNN_H,))]
    for l in range(MPNN_L):
        shp += [("Pi%d" % l, (MPNN_H, MPNN_P)), ("U%d" % l, (MPNN_H + 4 * MPNN_P, MPNN_H)),
                ("c%d" % l, (MPNN_H,))]
    shp += [("D", (MPNN_H, MPNN_OUT)), ("d", (MPNN_OUT,))]
    return shp


def mpnn_init(seed=0, scale=1.0):
    """Seeded initial weights: normal(0, scale/sqrt(fan_in)) matrices, zero
    biases; returned as a dict of float64 arrays."""
    rng = np.random.default_rng(seed)
    out = {}
    for name, shp in mpnn_shapes():
        if len(shp) == 1:
            out[name] = np.zeros(shp)
        else:
            out[name] = rng.normal(0.0, scale / math.sqrt(shp[0]), shp)
    return out
