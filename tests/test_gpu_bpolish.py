"""GPU parity of the polished batched inversion (afm_invert_batch_polished:
batched swarms, then the adjoint-gradient polish of every pixel's best
particles, all pixels' candidates in each launch) against the single-pixel
polished inversion and the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

from paper_1109_0334_gb300 import workloads as W
from common import NM

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def afm():
    from paper_1109_0334_gb300 import build
    build.build()
    from paper_1109_0334_gb300 import afminv
    assert torch.cuda.is_available()
    return afminv


def _records(orc, spec, pixels, cyc_div):
    c, pm = orc.make_case(spec), orc.make_pmap(spec)
    recs = []
    for p in pixels:
        cyc = max(2, orc.cycles(spec["seed"], p, 20, 200) // cyc_div)
        xt = orc.truth_x(pm.D, spec["seed"], p)
        U = orc.record(c, pm, xt, cyc * spec["spc"], spec["record_sub"], spec["sigma"],
                       spec["seed"], p)
        recs.append((U / NM).astype(np.float32))
    off = np.concatenate([[0], np.cumsum([len(r) for r in recs])]).astype(np.int64)
    return np.concatenate(recs), off, recs


@pytest.mark.parametrize("name,kp,method", [("c3", 1, "steepest"), ("c3", 2, "steepest"),
                                            ("c4", 0, "steepest"), ("c3", 0, "lm"),
                                            ("c4", 1, "lm")])
def test_batch_polished_equals_single_pixel_polished(orc, afm, name, kp, method):
    """Each pixel's candidates follow the arithmetic of afm_invert_polished
    on that pixel alone: identical winners, FP32 misfits and parameters; the
    FP64 re-evaluations (sequential in the batch, multiple shooting alone)
    agree to 1e-11."""
    spec = W.get(name, P=96, iters=8)
    pixels = [0, 1, 2, 3, 4]
    U_cat, off, recs = _records(orc, spec, pixels, cyc_div=20)
    prob = afm.make_problem(spec, n_steps=int(max(np.diff(off))))
    cfg = afm.make_pso(spec)
    Kc, steps, J = 4, 3, 8
    res, used = afm.invert_batch_polished(prob, torch.from_numpy(U_cat).cuda(),
                                          torch.from_numpy(off).cuda(), cfg, polish_k=Kc,
                                          polish_steps=steps, n_cand=J, particles_per_thread=kp,
                                          method=method)
    torch.cuda.synchronize()
    assert kp == 0 or used == kp
    batch = afm.decode_results(res)
    for i, U in enumerate(recs):
        prob_i = afm.make_problem(spec, n_steps=len(U))
        r1, _ = afm.invert_polished(prob_i, torch.from_numpy(U).cuda(), afm.make_pso(spec, pixel=i),
                                    polish_k=Kc, polish_steps=steps, n_cand=J, method=method)
        torch.cuda.synchronize()
        single = afm.decode_result(r1)
        b = batch[i]
        assert b["status"] == 0 and single["status"] == 0
        assert b["winner"] == single["winner"]
        assert b["S"] == single["S"]
        np.testing.assert_array_equal(b["x"], single["x"])
        assert abs(b["S_f64"] - single["S_f64"]) <= 1e-11 * single["S_f64"]


@pytest.mark.parametrize("method", ["steepest", "lm"])
def test_batch_polished_oracle_and_descent(orc, afm, method):
    """Against the oracle: each winner's FP64 misfit is the oracle's misfit at
    that point (1e-9) and the polish never raises a pixel's misfit above its
    plain batched swarm winner's."""
    spec = W.get("c3", P=128, iters=10)
    pixels = [7, 8, 9]
    U_cat, off, recs = _records(orc, spec, pixels, cyc_div=10)
    prob = afm.make_problem(spec, n_steps=int(max(np.diff(off))))
    cfg = afm.make_pso(spec)
    Ut, ot = torch.from_numpy(U_cat).cuda(), torch.from_numpy(off).cuda()
    rp, _ = afm.invert_batch_polished(prob, Ut, ot, cfg, polish_k=4, polish_steps=5, n_cand=8,
                                      pixel0=7, method=method)
    rb, _ = afm.invert_batch(prob, Ut, ot, cfg, pixel0=7)
    torch.cuda.synchronize()
    pol, plain = afm.decode_results(rp), afm.decode_results(rb)
    c, pm = orc.make_case(spec), orc.make_pmap(spec)
    for i, U in enumerate(recs):
        U_m = U.astype(np.float64) * NM
        sp = dict(spec, cycles=len(U) // spec["spc"])
        cp = orc.make_case(sp)
        x = pol[i]["x"][:pm.D].reshape(-1, 1)
        S_orc = orc.misfit_batch(cp, pm, x, U_m)[0] / NM ** 2
        assert pol[i]["status"] == 0
        assert abs(pol[i]["S_f64"] - S_orc) <= 1e-9 * S_orc
        assert abs(pol[i]["S"] - S_orc) <= 1e-4 * S_orc
        assert pol[i]["S_f64"] <= plain[i]["S_f64"] * (1 + 1e-9)


def test_batch_polished_record_beyond_n_steps_keeps_swarm_winner(orc, afm):
    """A record longer than prob.n_steps (which sizes the adjoint
    checkpoints) is not polished: its result is the plain batched one."""
    spec = W.get("c3", P=64, iters=4)
    U_cat, off, recs = _records(orc, spec, [0, 1, 2], cyc_div=20)
    lens = np.diff(off)
    n_short = int(np.min(lens))
    assert np.max(lens) > n_short
    prob = afm.make_problem(spec, n_steps=n_short)
    cfg = afm.make_pso(spec)
    Ut, ot = torch.from_numpy(U_cat).cuda(), torch.from_numpy(off).cuda()
    rp, _ = afm.invert_batch_polished(prob, Ut, ot, cfg, polish_k=2, polish_steps=2, n_cand=4)
    rb, _ = afm.invert_batch(prob, Ut, ot, cfg)
    torch.cuda.synchronize()
    pol, plain = afm.decode_results(rp), afm.decode_results(rb)
    for i in range(3):
        if lens[i] > n_short:
            assert pol[i]["winner"] == plain[i]["winner"]
            assert pol[i]["S"] == plain[i]["S"]
            np.testing.assert_array_equal(pol[i]["x"], plain[i]["x"])
        assert pol[i]["S_f64"] <= plain[i]["S_f64"] * (1 + 1e-9)


def test_paired_trial_point_forward_matches_smaller_batches(orc, afm):
    """512 pixels x 32 candidates x 4 damping values = 65 536 trial points per
    Levenberg-Marquardt step take the paired-instruction forward (two
    candidates of one pixel per thread); batches of 64 pixels (8 192 trial
    points) take the one-candidate-per-thread kernel.  Every pixel's result
    must be the same bit for bit."""
    spec = W.get("c3", P=64, iters=2)
    n_pix, sub = 512, 64
    pixels = list(range(n_pix))
    U_cat, off, recs = _records(orc, spec, pixels, cyc_div=100)
    prob = afm.make_problem(spec, n_steps=int(max(np.diff(off))))
    cfg = afm.make_pso(spec)
    Kc, steps, J = 32, 2, 4
    res, _ = afm.invert_batch_polished(prob, torch.from_numpy(U_cat).cuda(),
                                       torch.from_numpy(off).cuda(), cfg, polish_k=Kc,
                                       polish_steps=steps, n_cand=J, method="lm")
    torch.cuda.synchronize()
    full = afm.decode_results(res)
    for b0 in range(0, n_pix, sub):
        o = off[b0:b0 + sub + 1]
        Ub = np.concatenate(recs[b0:b0 + sub])
        rb, _ = afm.invert_batch_polished(prob, torch.from_numpy(Ub).cuda(),
                                          torch.from_numpy(o - o[0]).cuda(), cfg, polish_k=Kc,
                                          polish_steps=steps, n_cand=J, pixel0=b0, method="lm")
        torch.cuda.synchronize()
        for i, r in enumerate(afm.decode_results(rb)):
            f = full[b0 + i]
            assert r["status"] == 0 and f["status"] == 0
            assert r["winner"] == f["winner"] and r["S"] == f["S"]
            np.testing.assert_array_equal(r["x"], f["x"])
