"""The allocation-free pair search (sph_pairs_noalloc) against the context
entry point sph_get_pairs, through the C ABI on a GPU.

Callers that cannot call cudaMalloc hand the library device buffers they own;
the entry point keeps its scratch in a static device array.  Its pair set must
equal the context's exactly (integer output: bit-exact), on two calls in a
row (the second reuses the scratch left by the first).  This file runs last
so that a failure here cannot hide the other tests.
"""
import numpy as np
import pytest

from paper_1603_02421_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def test_noalloc_pairs_match_context_pairs():
    from paper_1603_02421_gb300 import binding, build
    build.build()
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    dev = torch.device("cuda", 0)
    box = (-0.1, -0.1, 2.1, 1.6)
    p = wl.test_params(dx=0.02, box=box)
    p["capacity"] = 8000
    st = wl.random_cloud(seed=12, n=6000, box=(2.0, 1.5), dx=0.02)
    sim = binding.Simulation({"params": p, "fluid": st, "boundary": None, "inflow": None},
                             device=0)
    a, b = sim.pairs(300000)
    ref = np.unique(np.stack([a, b], 1).astype(np.int64), axis=0)
    sim.close()
    h = 1.3 * 0.02
    x = torch.tensor(st["x"], dtype=torch.float64, device=dev)
    y = torch.tensor(st["y"], dtype=torch.float64, device=dev)
    cap = 300000
    out_a = torch.zeros(cap, dtype=torch.int32, device=dev)
    out_b = torch.zeros(cap, dtype=torch.int32, device=dev)
    for call in range(2):
        out_a.fill_(-1)
        out_b.fill_(-1)
        torch.cuda.synchronize()
        n = binding.sph_pairs_noalloc(x.data_ptr(), y.data_ptr(), len(st["x"]), h, box,
                                      out_a.data_ptr(), out_b.data_ptr(), cap)
        got = np.stack([out_a[:n].cpu().numpy(), out_b[:n].cpu().numpy()], 1).astype(np.int64)
        got = np.unique(got, axis=0)
        assert len(got) == n, "call %d: duplicate pairs" % call
        assert np.array_equal(got, ref), "call %d differs from sph_get_pairs" % call


def test_noalloc_rejects_oversize_inputs():
    from paper_1603_02421_gb300 import binding, build
    build.build()
    import torch
    dev = torch.device("cuda", 0)
    x = torch.zeros(4, dtype=torch.float64, device=dev)
    with pytest.raises(binding.SphError) as e:
        binding.sph_pairs_noalloc(x.data_ptr(), x.data_ptr(), (1 << 18) + 1, 0.01,
                                  (0.0, 0.0, 1.0, 1.0), x.data_ptr(), x.data_ptr(), 0)
    assert e.value.status == -3
    with pytest.raises(binding.SphError) as e:      # grid beyond the fixed cell limit
        binding.sph_pairs_noalloc(x.data_ptr(), x.data_ptr(), 4, 1e-4,
                                  (0.0, 0.0, 1.0, 1.0), x.data_ptr(), x.data_ptr(), 0)
    assert e.value.status == -3
