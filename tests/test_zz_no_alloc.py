"""The allocation-free inversion entry point (afm_invert_noalloc) against
the workspace one (afm_invert): same inputs, same result within the
inversion tolerances of the other tests (misfit 1e-4, FP64 re-evaluation
1e-9, parameters 0.5 %), on two calls in a row -- the second call reuses
the library's static scratch left over by the first.

Some callers cannot allocate device memory (a real-time feedback loop that
forbids allocator calls after start-up, a plug-in whose host owns the
device-memory budget); this entry point serves them.  This file is
collected last so that a run stopping at its first failure has already run
every other test."""
import ctypes as C

import numpy as np
import pytest

from paper_1109_0334_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def afm():
    from paper_1109_0334_gb300 import build
    build.build()
    from paper_1109_0334_gb300 import afminv
    assert torch.cuda.is_available()
    return afminv


def _record(afm, spec):
    N = W.n_steps(spec)
    prob = afm.make_problem(spec)
    off = torch.tensor([0, N], dtype=torch.int64, device="cuda")
    xt = torch.full((len(spec["free"]), 1), 0.4, dtype=torch.float64, device="cuda")
    return prob, afm.synth_records(prob, xt, off, spec["record_sub"], spec["sigma"], spec["seed"], 0)


def _same(r, ref, D):
    assert r["status"] == 0 and r["nonfinite"] == 0
    assert abs(r["S"] - ref["S"]) <= 1e-4 * ref["S"]
    assert abs(r["S_f64"] - ref["S_f64"]) <= 1e-9 * ref["S_f64"]
    th, th_ref = np.array(r["theta"]), np.array(ref["theta"])
    nz = th_ref != 0
    assert np.all(np.abs(th[nz] / th_ref[nz] - 1) <= 0.005)
    assert np.all(np.abs(np.array(r["x"][:D]) - np.array(ref["x"][:D])) <= 1e-6)
    # the FP64 re-evaluation ran by multiple shooting here as well
    assert r["segments"] == ref["segments"] > 0


@pytest.mark.parametrize("name,iters", [("c1", 50), ("c2", 10)])
def test_invert_noalloc_matches_invert_twice(afm, name, iters):
    spec = W.get(name, iters=iters)
    D = len(spec["free"])
    prob, U = _record(afm, spec)
    cfg = afm.make_pso(spec)
    res_ref, hist_ref = afm.invert(prob, U, cfg)
    torch.cuda.synchronize()
    ref = afm.decode_result(res_ref)
    for _ in range(2):
        res = torch.zeros(afm.result_dtype_size(), dtype=torch.uint8, device="cuda")
        hist = torch.empty(spec["iters"] + 1, dtype=torch.float32, device="cuda")
        afm.invert_noalloc(prob, U, cfg, res, hist)
        torch.cuda.synchronize()
        _same(afm.decode_result(res), ref, D)
        np.testing.assert_allclose(hist.cpu().numpy(), hist_ref.cpu().numpy(), rtol=1e-4)


def test_invert_noalloc_rejects_oversized_swarm(afm):
    spec = W.get("c2", P=300000, iters=1)
    prob, U = _record(afm, W.get("c2"))
    cfg = afm.make_pso(spec)
    res = torch.zeros(afm.result_dtype_size(), dtype=torch.uint8, device="cuda")
    with pytest.raises(afm.AfmError) as ei:
        afm.invert_noalloc(prob, U, cfg, res)
    assert ei.value.status == afm.ERR_INVALID_ARG
    assert b"static scratch" in afm.lib().afm_last_error()
