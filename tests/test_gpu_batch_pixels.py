"""Batched inversions whose pixels differ in their problem (one afm_problem
per pixel: the set-point, free amplitude and cantilever calibration of an
image scan drift from pixel to pixel; the inverse problem of Sec. 2.3 per
pixel).  Each pixel must equal the single-pixel inversion on its own
problem bit for bit, agree with the oracle's inversion of its own record,
and a list of identical problems must equal the shared-problem batch."""
import numpy as np
import pytest

from paper_1109_0334_gb300 import workloads as W
from common import NM, identifiable_check

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# per-pixel departures from the workload's cantilever and set-point
VARIANTS = [dict(), dict(Zc=14e-9), dict(A0=18e-9), dict(f1_hz=310e3, k=35.0), dict(Q=300.0),
            dict(Zc=15e-9, A0=22e-9)]


@pytest.fixture(scope="module")
def afm():
    from paper_1109_0334_gb300 import build
    build.build()
    from paper_1109_0334_gb300 import afminv
    assert torch.cuda.is_available()
    return afminv


def _records(orc, base, variants, cyc_div):
    """Oracle records of each pixel's truth under its own problem."""
    specs, recs = [], []
    for p, var in enumerate(variants):
        sp = dict(base, **var)
        c, pm = orc.make_case(sp), orc.make_pmap(sp)
        cyc = max(2, orc.cycles(sp["seed"], p, 20, 200) // cyc_div)
        xt = orc.truth_x(pm.D, sp["seed"], p)
        U = orc.record(c, pm, xt, cyc * sp["spc"], sp["record_sub"], sp["sigma"], sp["seed"], p)
        specs.append(dict(sp, cycles=cyc))
        recs.append((U / NM).astype(np.float32))
    off = np.concatenate([[0], np.cumsum([len(r) for r in recs])]).astype(np.int64)
    return specs, np.concatenate(recs), off, recs


def _batch_probs(afm, specs, off):
    n_max = int(max(np.diff(off)))
    return [afm.make_problem(sp, n_steps=n_max) for sp in specs]


@pytest.mark.parametrize("kp", [1, 2, 4])
def test_per_pixel_problems_equal_single_pixel_inversions(orc, afm, kp):
    base = W.get("c3", P=96, iters=12)
    specs, U_cat, off, recs = _records(orc, base, VARIANTS, cyc_div=20)
    probs = _batch_probs(afm, specs, off)
    cfg = afm.make_pso(base)
    res, used = afm.invert_batch(probs, torch.from_numpy(U_cat).cuda(), torch.from_numpy(off).cuda(),
                                 cfg, particles_per_thread=kp)
    torch.cuda.synchronize()
    assert used == kp
    batch = afm.decode_results(res)
    for i, U in enumerate(recs):
        prob_i = afm.make_problem(specs[i], n_steps=len(U))
        r1, _ = afm.invert(prob_i, torch.from_numpy(U).cuda(), afm.make_pso(base, pixel=i))
        torch.cuda.synchronize()
        single = afm.decode_result(r1)
        b = batch[i]
        assert b["status"] == 0
        assert b["winner"] == single["winner"] and b["S"] == single["S"]
        np.testing.assert_array_equal(b["x"], single["x"])
        np.testing.assert_array_equal(b["theta"], single["theta"])
        assert abs(b["S_f64"] - single["S_f64"]) <= 1e-11 * single["S_f64"]
        assert b["segments"] == -(-len(U) // 32)


def test_identical_problem_list_equals_shared_problem(orc, afm):
    base = W.get("c3", P=64, iters=6)
    specs, U_cat, off, _ = _records(orc, base, [dict()] * 5, cyc_div=20)
    probs = _batch_probs(afm, specs, off)
    Ug, og = torch.from_numpy(U_cat).cuda(), torch.from_numpy(off).cuda()
    cfg = afm.make_pso(base)
    r_shared, _ = afm.invert_batch(probs[0], Ug, og, cfg, particles_per_thread=2)
    r_list, _ = afm.invert_batch(probs, Ug, og, cfg, particles_per_thread=2)
    torch.cuda.synchronize()
    assert torch.equal(r_shared, r_list)


def test_per_pixel_problems_oracle_parity(orc, afm):
    """Two set-points (16 and 14 nm) and two calibrations in one batch, full
    swarm (256 particles x 60 updates), each pixel against the oracle's
    inversion of its own record under its own problem."""
    base = W.get("c3")
    variants = [dict(), dict(Zc=14e-9), dict(f1_hz=310e3, k=35.0)]
    specs, U_cat, off, recs = _records(orc, base, variants, cyc_div=10)
    probs = _batch_probs(afm, specs, off)
    res, _ = afm.invert_batch(probs, torch.from_numpy(U_cat).cuda(), torch.from_numpy(off).cuda(),
                              afm.make_pso(base))
    torch.cuda.synchronize()
    batch = afm.decode_results(res)
    for i, sp in enumerate(specs):
        c, pm = orc.make_case(sp), orc.make_pmap(sp)
        U_m = recs[i].astype(np.float64) * NM
        x_o, S_o, _ = orc.invert(c, pm, U_m, sp["P"], sp["iters"], sp["w"], sp["c1"], sp["c2"],
                                 sp["seed"], i)
        r = batch[i]
        err, n_id, S_g, widths = identifiable_check(orc, sp, U_m, x_o, S_o, r["x"][:pm.D])
        assert r["status"] == 0 and n_id >= 1
        assert err <= 0.005, (err, widths)
        assert S_g <= S_o * (1 + 1e-4)
        assert abs(r["S"] - S_g / NM ** 2) <= 1e-4 * S_g / NM ** 2
        assert abs(r["S_f64"] - S_g / NM ** 2) <= 1e-9 * S_g / NM ** 2


def test_per_pixel_problems_polished(orc, afm):
    """The Levenberg-Marquardt polished batch with per-pixel problems equals
    afm_invert_polished on each pixel's own problem bit for bit; the
    steepest-descent polish is refused for per-pixel problems."""
    base = W.get("c3", P=96, iters=6)
    specs, U_cat, off, recs = _records(orc, base, VARIANTS[:4], cyc_div=20)
    probs = _batch_probs(afm, specs, off)
    Ug, og = torch.from_numpy(U_cat).cuda(), torch.from_numpy(off).cuda()
    cfg = afm.make_pso(base)
    Kc, steps, J = 4, 3, 8
    res, _ = afm.invert_batch_polished(probs, Ug, og, cfg, polish_k=Kc, polish_steps=steps,
                                       n_cand=J, method="lm")
    torch.cuda.synchronize()
    batch = afm.decode_results(res)
    for i, U in enumerate(recs):
        prob_i = afm.make_problem(specs[i], n_steps=len(U))
        r1, _ = afm.invert_polished(prob_i, torch.from_numpy(U).cuda(), afm.make_pso(base, pixel=i),
                                    polish_k=Kc, polish_steps=steps, n_cand=J, method="lm")
        torch.cuda.synchronize()
        single = afm.decode_result(r1)
        b = batch[i]
        assert b["status"] == 0
        assert b["winner"] == single["winner"] and b["S"] == single["S"]
        np.testing.assert_array_equal(b["x"], single["x"])
        assert abs(b["S_f64"] - single["S_f64"]) <= 1e-11 * single["S_f64"]
    with pytest.raises(afm.AfmError) as ei:
        afm.invert_batch_polished(probs, Ug, og, cfg, polish_k=Kc, polish_steps=1, n_cand=J,
                                  method="steepest")
    assert ei.value.status == afm.ERR_UNSUPPORTED
