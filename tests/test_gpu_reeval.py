"""The FP64 re-evaluation of an inversion's winner by multiple shooting in
time: segments of 32 RK4 steps integrated concurrently in FP64, their start
states made consistent by Newton's method on the matching conditions.  Its
misfit must equal the oracle's FP64 misfit (Eq. 5) at the winner and the
GPU's sequential FP64 forward solve, for each force law and mode count it
serves; records too short for two segments use the sequential run."""
import math

import numpy as np
import pytest

from paper_1109_0334_gb300 import workloads as W
from common import NM, oracle_record

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def afm():
    from paper_1109_0334_gb300 import build
    build.build()
    from paper_1109_0334_gb300 import afminv
    assert torch.cuda.is_available()
    return afminv


CASES = [
    ("c1", dict(P=48, iters=4)),
    ("c2", dict(P=64, iters=3, cycles=40)),
    ("c4", dict(P=64, iters=3, cycles=40)),
    ("c2", dict(P=32, iters=2, cycles=30, force="linear_spring", fixed=[0.0] * 5,
                free=[(0, 2.0, 20.0, False), (1, 10e-9, 20e-9, False)])),
    ("c2", dict(P=32, iters=2, cycles=30, force="hooke", fixed=[0.0] * 5,
                free=[(0, 0.5, 8.0, True), (1, -2e-9, 4e-9, False)])),
    ("c2", dict(P=32, iters=2, cycles=30, force="spring_damper", fixed=[0.0] * 5,
                free=[(0, 0.5, 8.0, True), (1, -2e-9, 4e-9, False), (2, 0.0, 2e-7, False)])),
    ("f2_hooke", dict(P=64, iters=3, cycles=4)),
    ("f2_spring_damper", dict(P=64, iters=3, cycles=4)),
    ("c2", dict(P=32, iters=2, cycles=20, n_modes=5, spc=512)),
]


def _invert(afm, spec, U32, n=None):
    prob = afm.make_problem(spec, n_steps=n)
    res, _ = afm.invert(prob, torch.from_numpy(U32).cuda(), afm.make_pso(spec))
    torch.cuda.synchronize()
    return prob, afm.decode_result(res)


@pytest.mark.parametrize("name,over", CASES, ids=["c1-dmt", "c2-dmt", "c4-kv", "linear", "hooke",
                                                  "spring-damper", "8-modes-hooke",
                                                  "8-modes-spring-damper", "5-modes-padded"])
def test_multiple_shooting_matches_oracle_and_sequential(orc, afm, name, over):
    spec = W.get(name, **over)
    U32, U_m, _ = oracle_record(orc, spec)
    N = len(U32)
    prob, r = _invert(afm, spec, U32)
    D = len(spec["free"])
    assert r["status"] == 0
    assert r["segments"] == math.ceil(N / 32), r
    assert 0.0 <= r["defect"] <= 1e-9
    x = r["x"][:D].reshape(D, 1)
    c, pm = orc.make_case(spec), orc.make_pmap(spec)
    S_orc = orc.misfit_batch(c, pm, x, U_m)[0] / NM ** 2
    assert abs(r["S_f64"] - S_orc) <= 1e-9 * S_orc
    _, S_seq = afm.forward_batch_f64(prob, torch.from_numpy(x).cuda(),
                                     torch.from_numpy(U32.astype(np.float64)).cuda(), want_defl=False)
    torch.cuda.synchronize()
    S_seq = float(S_seq.cpu().numpy()[0])
    assert abs(r["S_f64"] - S_seq) <= 1e-11 * S_seq
    # J_rel = sqrt(S / sum U^2) from the same FP64 sum
    assert abs(r["J_rel"] - math.sqrt(r["S_f64"] / float(np.sum(U32.astype(np.float64) ** 2)))) <= 1e-12


def test_short_record_uses_the_sequential_run(orc, afm):
    spec = W.get("c1", P=16, iters=2)
    n = 50
    U32, U_m, _ = oracle_record(orc, spec, n=n)
    _, r = _invert(afm, spec, U32, n=n)
    assert r["status"] == 0 and r["segments"] == 0 and r["defect"] == 0.0
    x = r["x"][:2].reshape(2, 1)
    c, pm = orc.make_case(spec), orc.make_pmap(spec)
    S_orc = orc.misfit_batch(c, pm, x, U_m)[0] / NM ** 2
    assert abs(r["S_f64"] - S_orc) <= 1e-9 * S_orc
