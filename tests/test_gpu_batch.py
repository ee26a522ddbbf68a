"""GPU parity of the batched pixel inversion (one persistent, graph-captured
launch for many independent inversions) against the single-pixel inversion
and the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

from paper_1109_0334_gb300 import workloads as W
from common import NM, assert_determined, identifiable_check

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def afm():
    from paper_1109_0334_gb300 import build
    build.build()
    from paper_1109_0334_gb300 import afminv
    assert torch.cuda.is_available()
    return afminv


def _oracle_records(orc, spec, pixels, cyc_div=10, min_cycles=2):
    """Oracle records of each pixel's truth, lengths from the workload's
    20..200-cycle draw divided by cyc_div."""
    c, pm = orc.make_case(spec), orc.make_pmap(spec)
    recs, xts = [], []
    for p in pixels:
        cyc = max(min_cycles, orc.cycles(spec["seed"], p, 20, 200) // cyc_div)
        n = cyc * spec["spc"]
        xt = orc.truth_x(pm.D, spec["seed"], p)
        U = orc.record(c, pm, xt, n, spec["record_sub"], spec["sigma"], spec["seed"], p)
        recs.append((U / NM).astype(np.float32))
        xts.append(xt)
    off = np.concatenate([[0], np.cumsum([len(r) for r in recs])]).astype(np.int64)
    return np.concatenate(recs), off, recs, xts


@pytest.mark.parametrize("kp", [1, 2, 4])
def test_batch_equals_single_pixel_inversions(orc, afm, kp):
    """Each pixel of the batch runs the same swarm, with the same arithmetic,
    as afm_invert with cfg.pixel = pixel0 + i: identical winners."""
    spec = W.get("c3", P=96, iters=12)
    pixels = list(range(7))
    U_cat, off, recs, _ = _oracle_records(orc, spec, pixels, cyc_div=20)
    prob = afm.make_problem(spec, n_steps=int(max(np.diff(off))))
    cfg = afm.make_pso(spec)
    res, used = afm.invert_batch(prob, torch.from_numpy(U_cat).cuda(), torch.from_numpy(off).cuda(),
                                 cfg, pixel0=0, particles_per_thread=kp)
    torch.cuda.synchronize()
    assert used == kp
    batch = afm.decode_results(res)
    for i, U in enumerate(recs):
        prob_i = afm.make_problem(spec, n_steps=len(U))
        cfg_i = afm.make_pso(spec, pixel=i)
        r1, _ = afm.invert(prob_i, torch.from_numpy(U).cuda(), cfg_i)
        torch.cuda.synchronize()
        single = afm.decode_result(r1)
        b = batch[i]
        assert b["status"] == 0
        assert b["winner"] == single["winner"]
        assert b["S"] == single["S"]
        np.testing.assert_array_equal(b["x"], single["x"])
        # FP64 re-evaluations: sequential per pixel in the batch, multiple
        # shooting in afm_invert (different FP64 rounding, same trajectory)
        assert abs(b["S_f64"] - single["S_f64"]) <= 1e-11 * single["S_f64"]


def test_batch_oracle_parity_and_autotune(orc, afm):
    """Full swarm (256 particles x 60 updates) on three pixels with
    shortened records, against the oracle's inversion of each pixel."""
    spec = W.get("c3")
    pixels = [0, 1, 2]
    U_cat, off, recs, xts = _oracle_records(orc, spec, pixels, cyc_div=10)
    prob = afm.make_problem(spec, n_steps=int(max(np.diff(off))))
    cfg = afm.make_pso(spec)
    res, kp = afm.invert_batch(prob, torch.from_numpy(U_cat).cuda(), torch.from_numpy(off).cuda(), cfg)
    torch.cuda.synchronize()
    assert kp in (1, 2, 4)
    batch = afm.decode_results(res)
    c, pm = orc.make_case(spec), orc.make_pmap(spec)
    for i, p in enumerate(pixels):
        U_m = recs[i].astype(np.float64) * NM
        sp = dict(spec, cycles=len(recs[i]) // spec["spc"])
        cp = orc.make_case(sp)
        x_o, S_o, _ = orc.invert(cp, pm, U_m, spec["P"], spec["iters"], spec["w"], spec["c1"],
                                 spec["c2"], spec["seed"], p)
        r = batch[i]
        D = pm.D
        err, n_id, S_g, _ = identifiable_check(orc, sp, U_m, x_o, S_o, r["x"][:D])
        assert err <= 0.005 and n_id == 1
        assert_determined(orc, sp, U_m, x_o, r["x"][:D], 1, [])
        assert S_g <= S_o * (1 + 1e-4)
        assert abs(r["S"] - S_g / NM ** 2) <= 1e-4 * S_g / NM ** 2
        assert abs(r["S_f64"] - S_g / NM ** 2) <= 1e-9 * S_g / NM ** 2
        assert abs(r["J_rel"] - np.sqrt(S_g / np.sum(U_m ** 2))) <= 1e-9
        # the FP64 value came from multiple shooting over 32-step segments
        assert r["segments"] == -(-len(U_m) // 32) and r["defect"] <= 1e-9


def test_batch_edge_cases(orc, afm):
    """One pixel; a one-step record; a swarm that is not a multiple of 32;
    graph replay of identical arguments gives identical results."""
    spec = W.get("c3", P=50, iters=3)
    U_cat, off, recs, _ = _oracle_records(orc, spec, [5, 6], cyc_div=100, min_cycles=1)
    U_cat = np.concatenate([U_cat, U_cat[:1]])
    off = np.concatenate([off, [off[-1] + 1]]).astype(np.int64)
    prob = afm.make_problem(spec, n_steps=int(max(np.diff(off))))
    cfg = afm.make_pso(spec)
    Ut, ot = torch.from_numpy(U_cat).cuda(), torch.from_numpy(off).cuda()
    r1, _ = afm.invert_batch(prob, Ut, ot, cfg, pixel0=5)
    r2, _ = afm.invert_batch(prob, Ut, ot, cfg, pixel0=5)
    torch.cuda.synchronize()
    assert torch.equal(r1, r2)
    out = afm.decode_results(r1)
    assert len(out) == 3 and all(o["status"] == 0 for o in out)
    assert out[2]["winner"] < 50
    one, _ = afm.invert_batch(prob, Ut, ot[:2].contiguous(), cfg, pixel0=5)
    torch.cuda.synchronize()
    assert afm.decode_results(one)[0]["S"] == out[0]["S"]
