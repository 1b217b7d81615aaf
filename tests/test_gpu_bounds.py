"""The bounds-check build (libsph_bounds.so, SPH_BOUNDS_CHECK) on small cases.

Every particle index the neighbour walks and the network's gathers meet is
checked against the capacity there; an index out of range would set
ERR_BOUNDS and fail the call with SPH_ERR_STATE.  Each case runs in its own
process with the checked library and with the product library: the checked
run must report no error and give the same results (the checks add integer
compares only; FP32 results to rounding, see the test).
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_SCRIPT = r'''
import json, sys
import numpy as np
sys.path.insert(0, sys.argv[2])
from paper_1603_02421_gb300 import binding, workloads as wl
binding.LIB_PATH = sys.argv[1]
import torch
out = {}
# a jet with the inflow, reused lists and cell rebuilds
jet = wl.jet(seed=4, dx=1.0 / 20, length=6.0, Re=200, We=20)
jet["params"]["skin_over_h"] = 0.3
sim = binding.Simulation(jet)
sim.set_tuning(2, 8)
sim.run(24)
st = sim.state()
o = np.argsort(st["id"])
out["jet"] = [st[k][o].tolist() for k in ("x", "y", "u", "v", "rho")]
L = binding.sph_breakup_length(sim.ctx)
out["jet_L"] = [float(L[0])]
# the network and a surrogate step on it
net = binding.Mpnn(jet["params"]["capacity"], 0)
net.set_params(wl.mpnn_init(3))
sim.evaluate()
ids, y = binding.sph_mpnn_forward(net.net, sim.ctx, 1.0, True, jet["params"]["capacity"])
out["mpnn"] = y[np.argsort(ids)].astype(float).ravel().tolist()
acc, rm, rd = binding.sph_surrogate_step(sim.ctx, net.net, 4, 1.0, 0.05, 1e30, True)
st = sim.state()
o = np.argsort(st["id"])
out["surrogate"] = [st[k][o].tolist() for k in ("x", "u")]
net.close()
sim.close()
# the dam break with walls, FP64
dam = wl.dam_break(seed=1, dx=0.02, prec="fp64")
sim = binding.Simulation(dam)
sim.run(20)
st = sim.state()
o = np.argsort(st["id"])
out["dam"] = [st[k][o].tolist() for k in ("x", "y", "u", "v", "rho")]
sim.close()
# the allocation-free pair search
rng = np.random.default_rng(7)
xy = rng.uniform(0.0, 1.0, (2, 3000))
dev = torch.device("cuda", 0)
x = torch.tensor(xy[0], device=dev)
yy = torch.tensor(xy[1], device=dev)
a = torch.zeros(400000, dtype=torch.int32, device=dev)
b = torch.zeros(400000, dtype=torch.int32, device=dev)
npairs = binding.sph_pairs_noalloc(x.data_ptr(), yy.data_ptr(), 3000, 0.01, (0.0, 0.0, 1.0, 1.0),
                                   a.data_ptr(), b.data_ptr(), 400000)
pa, pb = a[:npairs].cpu().numpy(), b[:npairs].cpu().numpy()
out["pairs"] = sorted(zip(pa.tolist(), pb.tolist()))
print(json.dumps(out))
'''


def _run(lib):
    r = subprocess.run([sys.executable, "-c", _SCRIPT, lib, ROOT], capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def _rel(xa, xb):
    return float(np.linalg.norm(xa - xb) / max(np.linalg.norm(xb), 1e-300))


def test_bounds_checked_library_matches_and_reports_nothing():
    """The checks change no arithmetic, but the compiler may fuse multiply-adds
    differently around the extra compares, so FP32 results agree to rounding
    (an index out of range, a skipped or a wrong neighbour would differ by
    orders of magnitude more); the integer pair search agrees exactly and the
    FP64 dam break to 1e-10."""
    from paper_1603_02421_gb300 import build
    checked = build.build(bounds_check=True)
    product = build.build()
    a, b = _run(checked), _run(product)
    assert a["pairs"] == b["pairs"]
    assert a["jet_L"][0] == pytest.approx(b["jet_L"][0], rel=1e-7)
    for key in ("jet", "mpnn", "surrogate", "dam"):
        assert np.asarray(a[key]).shape == np.asarray(b[key]).shape, key
    ja, jb = np.asarray(a["jet"], float), np.asarray(b["jet"], float)
    for f, name in enumerate(("x", "y", "u", "v")):
        assert _rel(ja[f], jb[f]) < 1e-6, ("jet", name, _rel(ja[f], jb[f]))
    assert _rel(ja[4] - 1000.0, jb[4] - 1000.0) < 1e-4, ("jet", "rho - rho0")
    # BF16 activations: an input change in the last FP32 bit can flip a rounding
    assert _rel(np.asarray(a["mpnn"], float), np.asarray(b["mpnn"], float)) < 1e-3
    sa, sb = np.asarray(a["surrogate"], float), np.asarray(b["surrogate"], float)
    assert _rel(sa[0], sb[0]) < 1e-6 and _rel(sa[1], sb[1]) < 1e-4, "surrogate"
    da, db = np.asarray(a["dam"], float), np.asarray(b["dam"], float)
    assert np.allclose(da, db, rtol=1e-10, atol=1e-12), "dam"
