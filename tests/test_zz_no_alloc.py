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


def test_invert_noalloc_sequential_fallback(afm):
    """A swarm that fills most of the scratch (58 000 particles x 4
    parameters: 3.9 of 4 MiB) leaves no room for the ~0.35 MB of
    multiple-shooting segments of a 25 600-step record: the winner is
    re-evaluated by the one-thread sequential FP64 pass instead (segments =
    0), which agrees with afm_invert's multiple-shooting value to rounding."""
    spec = W.get("c2", P=58000, iters=1)
    D = len(spec["free"])
    prob, U = _record(afm, spec)
    cfg = afm.make_pso(spec)
    res_ref, _ = afm.invert(prob, U, cfg)
    torch.cuda.synchronize()
    ref = afm.decode_result(res_ref)
    assert ref["segments"] > 0
    for _ in range(2):
        res = torch.zeros(afm.result_dtype_size(), dtype=torch.uint8, device="cuda")
        afm.invert_noalloc(prob, U, cfg, res)
        torch.cuda.synchronize()
        r = afm.decode_result(res)
        assert r["status"] == 0 and r["nonfinite"] == 0
        assert r["segments"] == 0
        assert r["winner"] == ref["winner"] and r["S"] == ref["S"]
        assert np.array_equal(r["x"][:D], ref["x"][:D])
        assert np.array_equal(r["theta"], ref["theta"])
        assert abs(r["S_f64"] - ref["S_f64"]) <= 1e-9 * ref["S_f64"]


def test_invert_noalloc_lanes_profile_and_error(afm):
    """The entry point honours the context's lanes choice (every variant is
    bit-identical), its iteration launches are seen by the profiling
    counters (iters + 1 per call), and a successful call clears the message
    an earlier failed call left behind."""
    spec = W.get("c2", iters=4)
    prob, U = _record(afm, spec)
    cfg = afm.make_pso(spec)
    bad = afm.make_pso(W.get("c2", P=300000, iters=1))
    out = {}
    try:
        for lanes in ("one", "modes3", "auto"):
            afm.set_lanes(lanes)
            afm.profile_enable(True)
            afm.profile_read()
            res = torch.zeros(afm.result_dtype_size(), dtype=torch.uint8, device="cuda")
            with pytest.raises(afm.AfmError):     # leaves a message behind
                afm.invert_noalloc(prob, U, bad, res)
            assert afm.lib().afm_last_error() != b""
            afm.invert_noalloc(prob, U, cfg, res)
            assert afm.lib().afm_last_error() == b""
            torch.cuda.synchronize()
            ms, n = afm.profile_read()
            assert n == spec["iters"] + 1 and ms > 0
            out[lanes] = afm.decode_result(res)
    finally:
        afm.profile_enable(False)
        afm.set_lanes("auto")
    for lanes in ("one", "modes3"):
        assert out[lanes]["S"] == out["auto"]["S"]
        assert np.array_equal(out[lanes]["x"], out["auto"]["x"])


def test_invert_noalloc_rejects_oversized_swarm(afm):
    spec = W.get("c2", P=300000, iters=1)
    prob, U = _record(afm, W.get("c2"))
    cfg = afm.make_pso(spec)
    res = torch.zeros(afm.result_dtype_size(), dtype=torch.uint8, device="cuda")
    with pytest.raises(afm.AfmError) as ei:
        afm.invert_noalloc(prob, U, cfg, res)
    assert ei.value.status == afm.ERR_INVALID_ARG
    assert b"static scratch" in afm.lib().afm_last_error()
