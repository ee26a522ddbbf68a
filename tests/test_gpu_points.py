"""Deflection records at several points along the cantilever (the paper's
n_dp points, Sec. 3.2; reading R19): GPU forward solves against the oracle
in FP32 and FP64, a single tip point against the tip-only path, and an
inversion against the oracle's inversion of the same three-point record."""
import numpy as np
import pytest

from paper_1109_0334_gb300 import workloads as W
from common import NM, assert_determined, identifiable_check, oracle_defl_nm, oracle_record, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def afm():
    from paper_1109_0334_gb300 import build
    build.build()
    from paper_1109_0334_gb300 import afminv
    assert torch.cuda.is_available()
    return afminv


@pytest.mark.parametrize("modes,points", [(3, (1 / 3, 2 / 3, 1.0)), (5, (0.25, 0.5, 0.75, 1.0)),
                                          (1, (0.5,))])
def test_points_forward_parity(orc, afm, modes, points):
    spec = W.get("f4_points", cycles=12, n_modes=modes, points=points,
                 spc=512 if modes > 3 else 256)
    D = len(spec["free"])
    x = W.sample_x(D, 29, seed=modes)
    U32, _, _ = oracle_record(orc, spec)
    prob = afm.make_problem(spec)
    xg, Ug = torch.from_numpy(x).cuda(), torch.from_numpy(U32).cuda()
    defl, S = afm.forward_batch(prob, xg, Ug)
    d64, _ = afm.forward_batch_f64(prob, xg.double(), Ug.double())
    torch.cuda.synchronize()
    ref = oracle_defl_nm(orc, spec, x)
    assert defl.shape[0] == W.n_steps(spec) * len(points)
    assert rel_l2(defl.cpu().numpy(), ref, axis=0).max() <= 1e-5
    assert rel_l2(d64.cpu().numpy(), ref, axis=0).max() <= 1e-9
    c, pm = orc.make_case(spec), orc.make_pmap(spec)
    S_ref = orc.misfit_batch(c, pm, x.astype(np.float64), U32.astype(np.float64) * NM) / NM ** 2
    assert np.max(np.abs(S.cpu().numpy() - S_ref) / S_ref) <= 1e-4


def test_single_tip_point_equals_the_tip_path(orc, afm):
    spec = W.get("c2", cycles=10)
    x = torch.from_numpy(W.sample_x(4, 40, seed=3)).cuda()
    U32, _, _ = oracle_record(orc, spec)
    Ug = torch.from_numpy(U32).cuda()
    d0, S0 = afm.forward_batch(afm.make_problem(spec), x, Ug)
    d1, S1 = afm.forward_batch(afm.make_problem(dict(spec, points=(1.0,))), x, Ug)
    torch.cuda.synchronize()
    assert torch.equal(d0, d1) and torch.equal(S0, S1)


def test_points_inversion(orc, afm):
    spec = W.get("f4_points", cycles=20, P=256, iters=30)
    c, pm = orc.make_case(spec), orc.make_pmap(spec)
    U32, U_m, _ = oracle_record(orc, spec)
    x_o, S_o, _ = orc.invert(c, pm, U_m, spec["P"], spec["iters"], spec["w"], spec["c1"],
                             spec["c2"], spec["seed"])
    prob = afm.make_problem(spec)
    res, _ = afm.invert(prob, torch.from_numpy(U32).cuda(), afm.make_pso(spec))
    torch.cuda.synchronize()
    r = afm.decode_result(res)
    err, n_id, S_g, widths = identifiable_check(orc, spec, U_m, x_o, S_o, r["x"][:pm.D])
    assert r["status"] == 0 and n_id == 1
    assert err <= 0.005, (err, widths)
    assert_determined(orc, spec, U_m, x_o, r["x"][:pm.D], 1, [])
    assert S_g <= S_o * (1 + 1e-4)
    assert abs(r["S"] - S_g / NM ** 2) <= 1e-4 * S_g / NM ** 2
    assert abs(r["S_f64"] - S_g / NM ** 2) <= 1e-9 * S_g / NM ** 2
    # the FP64 re-evaluation over the points ran as multiple shooting
    assert r["segments"] == -(-W.n_steps(spec) // 32) and r["defect"] <= 1e-9


@pytest.mark.parametrize("over", [
    dict(),
    dict(points=(0.25, 0.5, 0.75, 1.0)),
    dict(n_modes=2, points=(0.5, 1.0), force="linear_spring", fixed=[0.0] * 5,
         free=[(0, 2.0, 20.0, False), (1, 10e-9, 20e-9, False)]),
    dict(force="hooke", fixed=[0.0] * 5, free=[(0, 0.5, 8.0, True), (1, -2e-9, 4e-9, False)]),
])
def test_points_inversion_one_mode_per_lane_is_bit_identical(orc, afm, over):
    """The points iteration with one mode per lane (2 or 3 modes, rate-free
    laws) against the one-lane kernel: the same swarm, bit for bit, on a
    ragged swarm (77 particles: the last warp part-filled)."""
    spec = W.get("f4_points", cycles=8, P=77, iters=6, **over)
    U32, _, _ = oracle_record(orc, spec)
    prob = afm.make_problem(spec)
    cfg = afm.make_pso(spec)
    Ut = torch.from_numpy(U32).cuda()
    out = {}
    for lanes in ("one", "auto"):
        afm.set_lanes(lanes)
        try:
            r, h = afm.invert(prob, Ut, cfg)
            torch.cuda.synchronize()
        finally:
            afm.set_lanes("auto")
        out[lanes] = (afm.decode_result(r), h.cpu().numpy())
    (a, ha), (b, hb) = out["one"], out["auto"]
    assert a["status"] == 0 and b["status"] == 0
    assert a["winner"] == b["winner"] and a["S"] == b["S"] and a["S_f64"] == b["S_f64"]
    np.testing.assert_array_equal(a["x"], b["x"])
    np.testing.assert_array_equal(ha, hb)
