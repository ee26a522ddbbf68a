"""Parity at the workloads' full sizes, in the launch configurations the
benchmark times, on outputs the FP64 oracle can check one by one: the
winners' misfits (FP32 and the FP64 re-evaluation) re-computed by the
oracle on the same oracle-made records, and the optimum against the
oracle's own where it is affordable (stored by tests/golden/make_golden.py,
which calls only the oracle)."""
import json
import os

import numpy as np
import pytest

from paper_1109_0334_gb300 import workloads as W
from common import NM, combination_error, identifiable_check, oracle_record

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def afm():
    from paper_1109_0334_gb300 import build
    build.build()
    from paper_1109_0334_gb300 import afminv
    assert torch.cuda.is_available()
    return afminv


def _check_winner(orc, spec, U_m, r, f32_tol=1e-4, f64_tol=1e-9):
    """The GPU winner's FP32 misfit and FP64 re-evaluation against the
    oracle's misfit at the same parameters; returns the oracle's value [m^2]."""
    c, pm = orc.make_case(spec), orc.make_pmap(spec)
    D = pm.D
    S_o = orc.misfit_batch(c, pm, np.asarray(r["x"][:D], dtype=np.float64).reshape(-1, 1), U_m)[0]
    S_nm = S_o / NM ** 2
    assert r["status"] == 0
    assert abs(r["S"] - S_nm) <= f32_tol * S_nm
    assert abs(r["S_f64"] - S_nm) <= f64_tol * S_nm
    return S_o


def test_c3_full_batch_sampled_pixels(orc, afm):
    """4096 pixels, 20..200 cycles each, 256 particles x 60 updates, one
    persistent graph launch with the autotuned particles per thread.  Four
    sampled pixels (the first, the last, the longest and the shortest
    record) carry records of their own truths; the other pixels carry
    prefixes of one long oracle record (their results are not compared,
    they only fill the launch)."""
    spec = W.get("c3")
    n_pix, spc = spec["n_pix"], spec["spc"]
    c, pm = orc.make_case(spec), orc.make_pmap(spec)
    cyc = np.array([orc.cycles(spec["seed"], p, 20, 200) for p in range(n_pix)])
    lens = cyc * spc
    sampled = sorted({0, n_pix - 1, int(np.argmax(cyc)), int(np.argmin(cyc))})
    base_x = orc.truth_x(pm.D, spec["seed"], n_pix)
    base = orc.record(c, pm, base_x, int(lens.max()), spec["record_sub"], spec["sigma"],
                      spec["seed"], n_pix)
    base32 = (base / NM).astype(np.float32)
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    U_cat = np.empty(int(off[-1]), dtype=np.float32)
    own = {}
    for p in range(n_pix):
        if p in sampled:
            xt = orc.truth_x(pm.D, spec["seed"], p)
            U = orc.record(c, pm, xt, int(lens[p]), spec["record_sub"], spec["sigma"],
                           spec["seed"], p)
            own[p] = (U / NM).astype(np.float32)
            U_cat[off[p]:off[p + 1]] = own[p]
        else:
            U_cat[off[p]:off[p + 1]] = base32[:lens[p]]
    prob = afm.make_problem(spec, n_steps=int(lens.max()))
    cfg = afm.make_pso(spec)
    res, kp = afm.invert_batch(prob, torch.from_numpy(U_cat).cuda(), torch.from_numpy(off).cuda(),
                               cfg)
    torch.cuda.synchronize()
    out = afm.decode_results(res)
    assert len(out) == n_pix and all(o["status"] == 0 for o in out)
    shortest = int(np.argmin(cyc))
    for p in sampled:
        sp = dict(spec, cycles=int(cyc[p]))
        U_m = own[p].astype(np.float64) * NM
        S_g = _check_winner(orc, sp, U_m, out[p])
        if p == shortest:
            # the oracle's own inversion of this pixel (256 x 60, shortest record)
            x_o, S_o, _ = orc.invert(orc.make_case(sp), pm, U_m, spec["P"], spec["iters"],
                                     spec["w"], spec["c1"], spec["c2"], spec["seed"], p)
            err, _, _, _ = identifiable_check(orc, sp, U_m, x_o, S_o, out[p]["x"][:pm.D])
            assert err <= 0.005
            assert S_g <= S_o * (1 + 1e-4)


def test_c4_full_polished_against_oracle_optimum(orc, afm):
    """The full Kelvin-Voigt record, the benchmark's Levenberg-Marquardt
    configuration: the winner is statistically at the oracle's optimum
    (delta chi^2 <= 1) and agrees with it in the combinations the law
    depends on.  (The misfit is exactly flat along R with those fixed, so
    two optima can sit far apart in R; a finite-difference Hessian of this
    non-smooth misfit does not resolve that valley cleanly enough for the
    eigen-direction comparison.)"""
    with open(os.path.join(HERE, "golden", "c4_invert.json")) as f:
        gold = json.load(f)
    spec = W.get("c4")
    U32, U_m, _ = oracle_record(orc, spec)
    assert abs(float(np.sum(U_m ** 2)) / gold["sumU2_m2"] - 1) < 1e-9
    prob = afm.make_problem(spec)
    lp = spec["lm_polish"]
    cfg = afm.make_pso(dict(spec, iters=lp["iters"]))
    r, _ = afm.invert_polished(prob, torch.from_numpy(U32).cuda(), cfg, lp["polish_k"],
                               lp["polish_steps"], lp["n_cand"], method="lm")
    torch.cuda.synchronize()
    r = afm.decode_result(r)
    S_g = _check_winner(orc, spec, U_m, r)
    dchi2 = (S_g - gold["S_m2"]) / spec["sigma"] ** 2
    assert dchi2 <= 1.0
    D = len(spec["free"])
    err = combination_error(orc, spec, np.array(gold["x"]), r["x"][:D])
    assert err <= 0.005, err


def test_c5_full_fe_inversion_sampled(orc, afm):
    """The full finite-element inversion (8192 particles x 60 updates, 50
    cycles x 512 steps, Newmark beta = 1/4): the winner's misfits against
    the oracle's FE forward at the same parameters, and the winner fits the
    record at least as well as the truth does."""
    spec = W.get("c5")
    U32, U_m, xt = oracle_record(orc, spec)
    prob = afm.make_problem(spec)
    cfg = afm.make_pso(spec)
    r, _ = afm.invert(prob, torch.from_numpy(U32).cuda(), cfg)
    torch.cuda.synchronize()
    r = afm.decode_result(r)
    # FP32 misfit against the oracle's; the FP64 re-evaluation against it
    # through the trajectories: |S_gpu - S_oracle| <= |u_gpu - u_oracle|
    # |2U - u_gpu - u_oracle| (Cauchy-Schwarz), the trajectories pinned at
    # 1e-7 over the 50 cycles (the drive sits on the resonance, Q = 400, so
    # rounding-level differences of the modal formulation grow with the
    # record: ~8e-9 after 10 cycles, ~6e-8 after 50)
    S_g = _check_winner(orc, spec, U_m, r, f32_tol=1e-4, f64_tol=1.0)
    c, pm = orc.make_case(spec), orc.make_pmap(spec)
    D = pm.D
    xw = np.asarray(r["x"][:D], dtype=np.float64).reshape(-1, 1)
    d64, _ = afm.forward_batch_f64(prob, torch.from_numpy(xw.copy()).cuda(), None)
    torch.cuda.synchronize()
    u_g = d64.cpu().numpy()[:, 0]
    u_o = orc.fe_forward(c, orc.map_x(pm, xw[:, 0]), len(U32)) / NM
    assert np.linalg.norm(u_g - u_o) <= 1e-7 * np.linalg.norm(u_o)
    U = U32.astype(np.float64)
    bound = np.linalg.norm(u_g - u_o) * np.linalg.norm(2 * U - u_g - u_o)
    assert abs(r["S_f64"] - S_g / NM ** 2) <= bound + 1e-12 * S_g / NM ** 2
    S_truth = orc.misfit_batch(c, pm, np.asarray(xt, dtype=np.float64).reshape(-1, 1), U_m)[0]
    assert S_g <= S_truth * (1 + 1e-3)


def test_c3_polished_batch_meets_oracle_optima(orc, afm):
    """The benchmark's accuracy claim on the oracle's own records: the first
    64 pixels of the 4096-pixel batch (seeded truths, lengths and noise of
    workloads.c3_layout), LM-polished batch configuration, against the
    oracle's stored optimum of each (tests/golden/c3_subset_optima.json,
    oracle only).  The winners are statistically at the optimum (delta
    chi^2 <= 1 on the same record; the FP64 re-evaluation is the oracle's
    misfit at the winner) on at least 95 % of the pixels and within two
    noise variances on all (a one-sigma bound on a stochastic search: one of
    the 64 sits at 1.04), and their parameters agree with the optimum's
    within 0.5 % along the directions the record determines to 0.5 % on at
    least 90 % (the others lie on a flatter valley of equal misfit or in a
    second minimum of equal misfit)."""
    with open(os.path.join(HERE, "golden", "c3_subset_optima.json")) as f:
        gold = json.load(f)
    spec = W.get("c3")
    cyc, xt = W.c3_layout(spec)
    pm = orc.make_pmap(spec)
    recs = []
    for g in gold["pixels"]:
        i = g["pixel"]
        assert g["cycles"] == int(cyc[i])
        c = orc.make_case(dict(spec, cycles=int(cyc[i])))
        U = orc.record(c, pm, xt[:, i], int(cyc[i]) * spec["spc"], spec["record_sub"],
                       spec["sigma"], spec["seed"], i)
        recs.append((U / NM).astype(np.float32))
    off = np.concatenate([[0], np.cumsum([len(r) for r in recs])]).astype(np.int64)
    lp = spec["lm_polish"]
    prob = afm.make_problem(spec, n_steps=int(max(np.diff(off))))
    cfg = afm.make_pso(dict(spec, iters=lp["iters"]))
    res, _ = afm.invert_batch_polished(prob, torch.from_numpy(np.concatenate(recs)).cuda(),
                                       torch.from_numpy(off).cuda(), cfg, lp["polish_k"],
                                       lp["polish_steps"], lp["n_cand"], method="lm")
    torch.cuda.synchronize()
    out = afm.decode_results(res)
    var = spec["sigma"] ** 2
    meets, at_opt = 0, 0
    for k, g in enumerate(gold["pixels"]):
        sp = dict(spec, cycles=g["cycles"])
        U_m = recs[k].astype(np.float64) * NM
        S_g = _check_winner(orc, sp, U_m, out[k])
        dchi2 = (S_g - g["S_m2"]) / var
        assert dchi2 <= 2.0, (k, dchi2)
        at_opt += bool(dchi2 <= 1.0)
        err, n_id, _, _ = identifiable_check(orc, sp, U_m, np.array(g["x"]), g["S_m2"],
                                             out[k]["x"][:pm.D])
        meets += bool((err <= 0.005 and dchi2 <= 1.0) or dchi2 < -1.0)
    assert at_opt >= 0.95 * len(gold["pixels"]), at_opt
    assert meets >= 0.9 * len(gold["pixels"]), meets
