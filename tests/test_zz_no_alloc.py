"""The allocation-free pair search (sph_pairs_noalloc) against the context
entry point sph_get_pairs and against the FP64 oracle, through the C ABI on a
GPU.

Callers that cannot call cudaMalloc -- code inside another framework's memory
pool, an application with a fixed device footprint, a plugin that only gets
device buffers -- hand the library device buffers they own; the entry point
keeps its scratch in a static device array.  Its pair set must equal the
context's and the oracle's exactly (integer output: bit-exact), on two calls
in a row (the second reuses the scratch left by the first).  The status codes
decided on the device (a particle outside the box, an output buffer that is
too short) must still report the pairs found.  This file runs last so that a
failure here cannot hide the other tests.
"""
import numpy as np
import pytest

from paper_1603_02421_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

BOX = (-0.1, -0.1, 2.1, 1.6)
DX = 0.02
H = 1.3 * DX


def _setup():
    from paper_1603_02421_gb300 import binding, build
    build.build()
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    return binding, torch, torch.device("cuda", 0)


def _call(binding, torch, x, y, n, cap, dev):
    out_a = torch.full((max(cap, 1),), -1, dtype=torch.int32, device=dev)
    out_b = torch.full((max(cap, 1),), -1, dtype=torch.int32, device=dev)
    torch.cuda.synchronize()
    try:
        cnt = binding.sph_pairs_noalloc(x.data_ptr(), y.data_ptr(), n, H, BOX,
                                        out_a.data_ptr(), out_b.data_ptr(), cap)
        status = 0
    except binding.SphError as e:
        cnt, status = e.count, e.status
    k = min(cnt, cap)
    got = np.stack([out_a[:k].cpu().numpy(), out_b[:k].cpu().numpy()], 1).astype(np.int64)
    return status, cnt, got


def test_noalloc_pairs_match_context_and_oracle_pairs(orc):
    binding, torch, dev = _setup()
    p = wl.test_params(dx=DX, box=BOX)
    p["capacity"] = 8000
    st = wl.random_cloud(seed=12, n=6000, box=(2.0, 1.5), dx=DX)
    sim = binding.Simulation({"params": p, "fluid": st, "boundary": None, "inflow": None},
                             device=0)
    a, b = sim.pairs(300000)
    ref = np.unique(np.stack([a, b], 1).astype(np.int64), axis=0)
    sim.close()
    # the oracle's FP64 pair set (ids = input indices here)
    assert np.array_equal(ref, orc.pair_set(st["x"], st["y"], 2.0 * H))
    x = torch.tensor(st["x"], dtype=torch.float64, device=dev)
    y = torch.tensor(st["y"], dtype=torch.float64, device=dev)
    for call in range(2):
        status, n, got = _call(binding, torch, x, y, len(st["x"]), 300000, dev)
        assert status == 0
        got_u = np.unique(got, axis=0)
        assert len(got_u) == n, "call %d: duplicate pairs" % call
        assert np.array_equal(got_u, ref), "call %d differs from sph_get_pairs" % call


def test_noalloc_reports_particles_outside_the_box(orc):
    # SPH_ERR_ARG from the device, with the pairs of the particles inside the
    # box still exact: one particle just past xmax, one with a NaN coordinate
    binding, torch, dev = _setup()
    st = wl.random_cloud(seed=13, n=3000, box=(2.0, 1.5), dx=DX)
    xs, ys = st["x"].copy(), st["y"].copy()
    bad = [17, 2222]
    xs[bad[0]] = BOX[2] + 1e-9
    ys[bad[1]] = np.nan
    keep = np.setdiff1d(np.arange(len(xs)), bad)
    ref = orc.pair_set(xs[keep], ys[keep], 2.0 * H)
    ref = np.stack([keep[ref[:, 0]], keep[ref[:, 1]]], 1)
    ref = ref[np.lexsort((ref[:, 1], ref[:, 0]))]
    x = torch.tensor(xs, dtype=torch.float64, device=dev)
    y = torch.tensor(ys, dtype=torch.float64, device=dev)
    status, n, got = _call(binding, torch, x, y, len(xs), 200000, dev)
    assert status == -1
    assert n == len(ref)
    assert np.array_equal(np.unique(got, axis=0), ref)


def test_noalloc_short_output_reports_the_full_count(orc):
    # SPH_ERR_CAPACITY from the device: the first cap slots hold valid,
    # distinct pairs and the count is the full one
    binding, torch, dev = _setup()
    st = wl.random_cloud(seed=14, n=2000, box=(2.0, 1.5), dx=DX)
    ref = orc.pair_set(st["x"], st["y"], 2.0 * H)
    x = torch.tensor(st["x"], dtype=torch.float64, device=dev)
    y = torch.tensor(st["y"], dtype=torch.float64, device=dev)
    cap = len(ref) // 3
    status, n, got = _call(binding, torch, x, y, len(st["x"]), cap, dev)
    assert status == -3
    assert n == len(ref)
    assert len(got) == cap and len(np.unique(got, axis=0)) == cap
    refset = set(map(tuple, ref.tolist()))
    assert all(tuple(r) in refset for r in got.tolist())


def test_noalloc_rejects_oversize_inputs():
    binding, torch, dev = _setup()
    x = torch.zeros(4, dtype=torch.float64, device=dev)
    with pytest.raises(binding.SphError) as e:
        binding.sph_pairs_noalloc(x.data_ptr(), x.data_ptr(), (1 << 18) + 1, 0.01,
                                  (0.0, 0.0, 1.0, 1.0), x.data_ptr(), x.data_ptr(), 0)
    assert e.value.status == -3
    with pytest.raises(binding.SphError) as e:      # grid beyond the fixed cell limit
        binding.sph_pairs_noalloc(x.data_ptr(), x.data_ptr(), 4, 1e-4,
                                  (0.0, 0.0, 1.0, 1.0), x.data_ptr(), x.data_ptr(), 0)
    assert e.value.status == -3


def test_noalloc_refuses_a_capturing_stream():
    # the call synchronises, which a capture cannot hold: it returns
    # SPH_ERR_ARG before enqueuing anything, and the caller's capture stays
    # valid
    binding, torch, dev = _setup()
    x = torch.zeros(16, dtype=torch.float64, device=dev)
    a = torch.zeros(16, dtype=torch.int32, device=dev)
    s = torch.cuda.Stream(device=dev)
    g = torch.cuda.CUDAGraph()
    torch.cuda.synchronize(dev)
    status = None
    with torch.cuda.stream(s):
        g.capture_begin()
        y = x + 1.0
        try:
            binding.sph_pairs_noalloc(x.data_ptr(), x.data_ptr(), 4, 0.1, (0.0, 0.0, 1.0, 1.0),
                                      a.data_ptr(), a.data_ptr(), 4, stream=s.cuda_stream)
        except binding.SphError as e:
            status = e.status
        finally:
            g.capture_end()
    assert status == -1
    g.replay()
    torch.cuda.synchronize(dev)
    assert float(y[0]) == 1.0
