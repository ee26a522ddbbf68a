"""Image scans with cross-pixel warm start (reading R17): the batched swarm
on a subset of pixels, inside per-pixel boxes with seed particles, against
the full batch and the oracle's boxed swarm; the two-pass image inversion
against its own passes and a cold inversion of every pixel."""
import numpy as np
import pytest

from paper_1109_0334_gb300 import workloads as W
from common import NM, identifiable_check

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def afm():
    from paper_1109_0334_gb300 import build
    build.build()
    from paper_1109_0334_gb300 import afminv
    assert torch.cuda.is_available()
    return afminv


def _records(orc, spec, xts, cycles):
    c, pm = orc.make_case(dict(spec, cycles=cycles)), orc.make_pmap(spec)
    n = cycles * spec["spc"]
    recs = [(orc.record(c, pm, xts[:, k], n, spec["record_sub"], spec["sigma"], spec["seed"], k)
             / NM).astype(np.float32) for k in range(xts.shape[1])]
    off = np.concatenate([[0], np.cumsum([len(r) for r in recs])]).astype(np.int64)
    return np.concatenate(recs), off, recs


def test_subset_equals_full_batch(orc, afm):
    spec = W.get("c3", P=64, iters=4)
    xts = W.image_truth(4, 3, 2, spec["seed"])
    U, off, recs = _records(orc, spec, xts, 4)
    prob = afm.make_problem(spec, n_steps=int(np.max(np.diff(off))))
    cfg = afm.make_pso(spec)
    Ut, ot = torch.from_numpy(U).cuda(), torch.from_numpy(off).cuda()
    full, _ = afm.invert_batch_polished(prob, Ut, ot, cfg, 4, 3, 8, method="lm")
    pix = torch.tensor([4, 1, 3], dtype=torch.int32, device="cuda")
    sub, _ = afm.invert_batch_polished(prob, Ut, ot, cfg, 4, 3, 8, method="lm", pixels=pix)
    torch.cuda.synchronize()
    a, b = afm.decode_results(full), afm.decode_results(sub)
    for k in (4, 1, 3):
        assert b[k]["winner"] == a[k]["winner"] and b[k]["S"] == a[k]["S"]
        np.testing.assert_array_equal(b[k]["x"], a[k]["x"])
    for k in (0, 2, 5):
        assert b[k]["status"] == 0 and b[k]["iters"] == 0 and b[k]["S"] == 0.0   # untouched


def test_boxed_seeded_swarm_matches_oracle(orc, afm):
    """Boxes of +-0.1 around each truth and two seed particles; no polish:
    each winner against the oracle's boxed swarm (identifiable 0.5 %, misfit
    1e-4), inside its box."""
    spec = W.get("c3", P=96, iters=10)
    D = 4
    xts = W.image_truth(D, 3, 1, spec["seed"] + 1)
    U, off, recs = _records(orc, spec, xts, 8)
    prob = afm.make_problem(spec, n_steps=int(np.max(np.diff(off))))
    cfg = afm.make_pso(spec)
    xr = np.ascontiguousarray(xts.T)                   # [pixel][D]
    lo = np.clip(xr - 0.1, 0, 1).astype(np.float32)
    hi = np.clip(xr + 0.1, 0, 1).astype(np.float32)
    seeds = np.ascontiguousarray(np.stack([np.clip(xr + 0.03, 0, 1), np.clip(xr - 0.05, 0, 1)],
                                          axis=1).astype(np.float32))
    pix = torch.arange(3, dtype=torch.int32, device="cuda")
    res, _ = afm.invert_batch_polished(prob, torch.from_numpy(U).cuda(), torch.from_numpy(off).cuda(),
                                       cfg, 1, 0, 1, method="lm", pixels=pix,
                                       box_lo=torch.from_numpy(lo).cuda(),
                                       box_hi=torch.from_numpy(hi).cuda(),
                                       seeds=torch.from_numpy(seeds).cuda())
    torch.cuda.synchronize()
    out = afm.decode_results(res)
    pm = orc.make_pmap(spec)
    for k in range(3):
        sp = dict(spec, cycles=8)
        c = orc.make_case(sp)
        U_m = recs[k].astype(np.float64) * NM
        xo, So = orc.invert_boxed(c, pm, U_m, spec["P"], spec["iters"], spec["w"], spec["c1"],
                                  spec["c2"], spec["seed"], lo[k].astype(np.float64),
                                  hi[k].astype(np.float64), seeds[k].astype(np.float64), pixel=k)
        r = out[k]
        xg = r["x"][:D]
        assert np.all(xg >= lo[k] - 1e-6) and np.all(xg <= hi[k] + 1e-6)
        err, n_id, S_g, widths = identifiable_check(orc, sp, U_m, xo, So, xg)
        assert S_g <= So * (1 + 1e-4)
        assert err <= 0.005, (err, widths)
        assert abs(r["S"] - S_g / NM ** 2) <= 1e-4 * S_g / NM ** 2


def test_image_warm_start(orc, afm):
    """A 9 x 5 image (coarse grid every 4th pixel: 6 coarse, 39 fine) of the
    image workload's records (40 cycles): the coarse pass equals a subset
    batch with the coarse swarm bit for bit; the fine pixels, searched
    inside their neighbours' box, reach the misfit of a cold inversion of
    every pixel (delta chi^2 <= 1) on at least 90 % of pixels.  (On 10- or
    20-cycle records only ~80 % do against this cold configuration: the
    flatter misfit of a short record puts the optimum outside the box more
    often.)"""
    spec = W.get("f1_image", width=9, height=5)
    Wd, Hd = spec["width"], spec["height"]
    # the 9 x 5 corner of a 64 x 64 image: truths as smooth on the coarse grid
    # as in the full-size scan
    big = W.image_truth(4, 64, 64, spec["seed"]).reshape(4, 64, 64)
    xts = np.ascontiguousarray(big[:, :Hd, :Wd].reshape(4, -1))
    U, off, recs = _records(orc, spec, xts, spec["cycles"])
    prob = afm.make_problem(spec, n_steps=int(np.max(np.diff(off))))
    coarse = afm.make_pso(spec)
    fine = afm.make_pso(dict(spec, **{k: spec["fine"][k] for k in ("P", "iters")}))
    icfg = afm.make_image_cfg(Wd, Hd, spec["stride"], spec["margin"], coarse, fine,
                              coarse_polish=(spec["polish_k"], spec["polish_steps"]),
                              fine_polish=(spec["fine"]["polish_k"], spec["fine"]["polish_steps"]),
                              n_cand=spec["n_cand"], method="lm")
    Ut, ot = torch.from_numpy(U).cuda(), torch.from_numpy(off).cuda()
    res = afm.invert_image(prob, Ut, ot, icfg)
    cpix = [j * Wd + i for j in range(0, Hd, 4) for i in range(0, Wd, 4)]
    ref, _ = afm.invert_batch_polished(prob, Ut, ot, coarse, spec["polish_k"], spec["polish_steps"],
                                       spec["n_cand"], method="lm",
                                       pixels=torch.tensor(cpix, dtype=torch.int32, device="cuda"))
    cold, _ = afm.invert_batch_polished(prob, Ut, ot, coarse, spec["polish_k"], spec["polish_steps"],
                                        spec["n_cand"], method="lm")
    torch.cuda.synchronize()
    img, r_c, r_cold = afm.decode_results(res), afm.decode_results(ref), afm.decode_results(cold)
    for k in cpix:
        assert img[k]["winner"] == r_c[k]["winner"] and img[k]["S"] == r_c[k]["S"]
    var = (spec["sigma"] / NM) ** 2
    fine_pix = [k for k in range(Wd * Hd) if k not in cpix]
    assert all(img[k]["status"] == 0 for k in range(Wd * Hd))
    ok = [img[k]["S_f64"] - r_cold[k]["S_f64"] <= var for k in fine_pix]
    assert np.mean(ok) >= 0.9, np.mean(ok)
