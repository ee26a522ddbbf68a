"""GPU parity of the particle swarm (Sec. 3.4, Eq. 8) and of the fused
inversion (IP, Sec. 2.3) against the FP64 oracle, through the C ABI.

Swarm initialisation is bit-exact (24-bit uniforms are exact in FP32).  One
swarm step agrees to FP32 rounding.  Whole inversions follow the same
seeded swarm but may part ways after near-ties of FP32 and FP64 misfits, so
they are compared on what is unique: the optimum misfit (within 1e-4) and
the parameter combinations the record determines (within 0.5 %); along
valleys the record does not resolve, the GPU's point must reach the
oracle's misfit.
"""
import json
import os

import numpy as np
import pytest

from paper_1109_0334_gb300 import workloads as W
from common import NM, assert_determined, identifiable_check, oracle_record

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def afm():
    from paper_1109_0334_gb300 import build
    build.build()
    from paper_1109_0334_gb300 import afminv
    assert torch.cuda.is_available()
    return afminv


def test_pso_init_bit_exact(orc, afm):
    for D, P in ((2, 64), (4, 1024), (5, 37)):
        cfg = afm.PsoCfg(P=P, iters=10, w=0.7, c1=1.5, c2=1.5, seed=1109033402, pixel=7)
        sw = afm.pso_init(cfg, D)
        torch.cuda.synchronize()
        x_ref, v_ref = orc.pso_init(P, D, cfg.seed, cfg.pixel)
        assert np.array_equal(sw.x.cpu().numpy().astype(np.float64), x_ref)
        assert np.array_equal(sw.v.cpu().numpy().astype(np.float64), v_ref)
        assert np.all(np.isinf(sw.pbest_S.cpu().numpy()))


def test_pso_step_matches_oracle(orc, afm):
    """P9: from identical (x, v, pbest, S) the GPU step equals the Eq. 8
    update of the oracle to FP32 rounding; personal and global bests are
    exact, ties going to the lowest index."""
    D, P, it = 4, 301, 5
    cfg = afm.PsoCfg(P=P, iters=10, w=0.7, c1=1.5, c2=1.5, seed=99, pixel=3)
    sw = afm.pso_init(cfg, D)
    rng = np.random.default_rng(0)
    x = rng.uniform(0, 1, (D, P)).astype(np.float32)
    v = rng.uniform(-0.3, 0.3, (D, P)).astype(np.float32)
    pbx = rng.uniform(0, 1, (D, P)).astype(np.float32)
    pbS = rng.uniform(1, 2, P).astype(np.float32)
    S = rng.uniform(0.5, 2.5, P).astype(np.float32)
    S[[17, 40, 200]] = 0.25          # a three-way tie for the global best
    S[55] = np.nan                   # a diverged candidate never becomes a best
    for t, a in ((sw.x, x), (sw.v, v), (sw.pbest_x, pbx), (sw.pbest_S, pbS)):
        t.copy_(torch.from_numpy(a))
    sw.gbest.fill_(-1)
    afm.pso_step(cfg, sw, torch.from_numpy(S).cuda(), it)
    torch.cuda.synchronize()
    # expected bests from the definition
    Sd = np.where(np.isnan(S), np.inf, S).astype(np.float64)
    better = Sd < pbS
    pb_exp = np.where(better[None, :], x, pbx)
    pbS_exp = np.where(better, Sd, pbS)
    g = int(np.argmin(pbS_exp))
    assert g == 17
    assert np.array_equal(sw.pbest_S.cpu().numpy(), pbS_exp.astype(np.float32))
    assert np.array_equal(sw.pbest_x.cpu().numpy(), pb_exp)
    key = int(sw.gbest.cpu().numpy().view(np.uint64)[0])
    assert key & 0xFFFFFFFF == 17
    x_ref, v_ref = orc.pso_update(it + 1, cfg.seed, cfg.pixel, cfg.w, cfg.c1, cfg.c2,
                                  x.astype(np.float64), v.astype(np.float64),
                                  pb_exp.astype(np.float64), pb_exp[:, g].astype(np.float64))
    xg, vg = sw.x.cpu().numpy(), sw.v.cpu().numpy()
    assert np.max(np.abs(vg - v_ref)) <= 4 * np.finfo(np.float32).eps
    assert np.max(np.abs(xg - x_ref)) <= 4 * np.finfo(np.float32).eps
    # clamped coordinates sit on the bound with zero velocity on both sides
    on_bound = (x_ref == 0.0) | (x_ref == 1.0)
    assert np.all(vg[on_bound] == 0.0)


def _gpu_invert(afm, spec, U32):
    prob = afm.make_problem(spec)
    cfg = afm.make_pso(spec)
    res, hist = afm.invert(prob, torch.from_numpy(U32).cuda(), cfg)
    torch.cuda.synchronize()
    return afm.decode_result(res), hist.cpu().numpy()


def _check_inversion(orc, spec, U_m, r, x_o, S_o_m, hist, n_id_expected, names):
    D = len(spec["free"])
    x_g = r["x"][:D]
    err, n_id, S_g_orc, widths = identifiable_check(orc, spec, U_m, x_o, S_o_m, x_g)
    S_o = S_o_m / NM ** 2
    assert n_id == n_id_expected, widths
    assert err <= 0.005, (err, widths)
    # the named combinations the record determines, compared by name
    assert_determined(orc, spec, U_m, x_o, x_g, n_id_expected, names)
    # the GPU's optimum is as good as the oracle's
    assert S_g_orc / NM ** 2 <= S_o * (1 + 1e-4)
    # FP32 misfit of the winner and its FP64 re-evaluation on the GPU
    assert abs(r["S"] - S_g_orc / NM ** 2) <= 1e-4 * S_o
    assert abs(r["S_f64"] - S_g_orc / NM ** 2) <= 1e-9 * S_o
    assert np.all(np.diff(hist) <= 0)
    assert r["status"] == 0 and r["nonfinite"] == 0
    # the FP64 re-evaluation ran as multiple shooting over 32-step segments
    assert r["segments"] == -(-len(U_m) // 32) and r["defect"] <= 1e-9


def test_invert_c1_parity(orc, afm):
    spec = W.get("c1")
    U32, U_m, xt = oracle_record(orc, spec)
    r, hist = _gpu_invert(afm, spec, U32)
    x_o, S_o, _ = orc.invert(orc.make_case(spec), orc.make_pmap(spec), U_m, spec["P"],
                             spec["iters"], spec["w"], spec["c1"], spec["c2"], spec["seed"])
    _check_inversion(orc, spec, U_m, r, x_o, S_o, hist, 1, [])
    assert r["iters"] == spec["iters"] and len(hist) == spec["iters"] + 1


def test_invert_c2_full_size_parity(orc, afm):
    """The 1024 x 100 inversion of the 3-mode cantilever (25 600 steps)
    against the oracle's own inversion of the same record, stored by
    tests/golden/make_golden.py (oracle only)."""
    with open(os.path.join(GOLDEN, "c2_invert.json")) as f:
        gold = json.load(f)
    spec = W.get("c2")
    U32, U_m, xt = oracle_record(orc, spec)
    assert abs(float(np.sum(U_m ** 2)) / gold["sumU2_m2"] - 1) < 1e-9
    r, hist = _gpu_invert(afm, spec, U32)
    _check_inversion(orc, spec, U_m, r, np.array(gold["x"]), gold["S_m2"], hist, 2,
                     ["E* sqrt(R)"])


@pytest.mark.parametrize("lanes", ["auto", "one", "stages", "modes2", "modes3", "modes4"])
@pytest.mark.parametrize("name,over", [
    ("c2", dict(cycles=12)),
    ("c1", dict(cycles=12)),
    ("c2", dict(cycles=12, n_modes=2)),
    ("c2", dict(cycles=12, force="linear_spring", fixed=[0.0] * 5,
                free=[(0, 2.0, 20.0, False), (1, 10e-9, 20e-9, False)])),
    ("c2", dict(cycles=12, n_modes=2, force="linear_spring", fixed=[0.0] * 5,
                free=[(0, 2.0, 20.0, False), (1, 10e-9, 20e-9, False)])),
    ("c2", dict(cycles=12, force="hooke", fixed=[0.0] * 5,
                free=[(0, 0.5, 8.0, True), (1, -2e-9, 4e-9, False)])),
])
def test_multi_lane_iteration_is_bit_identical(orc, afm, name, over, lanes):
    """Small swarms of rate-free laws run several lanes per particle (RK4
    stage forces or modes split between the lanes); every variant must be
    bit-identical to the one-lane arithmetic of the batched-pixel kernel on
    the same pixel."""
    spec = W.get(name, P=77, iters=6, **over)
    U32, _, _ = oracle_record(orc, spec)
    prob = afm.make_problem(spec)
    cfg = afm.make_pso(spec)
    Ut = torch.from_numpy(U32).cuda()
    afm.set_lanes(lanes)
    try:
        r1, h1 = afm.invert(prob, Ut, cfg)
        torch.cuda.synchronize()
    finally:
        afm.set_lanes("auto")
    off = torch.tensor([0, len(U32)], dtype=torch.int64, device="cuda")
    rb, _ = afm.invert_batch(prob, Ut, off, cfg, particles_per_thread=1)
    torch.cuda.synchronize()
    a, b = afm.decode_result(r1), afm.decode_results(rb)[0]
    assert a["winner"] == b["winner"] and a["S"] == b["S"]
    np.testing.assert_array_equal(a["x"], b["x"])
    assert np.all(np.diff(h1.cpu().numpy()) <= 0)


def _stepwise(afm, prob, cfg, U, sw, first, last):
    """Swarm evaluations first..last through the boundary's separate steps:
    afm_forward_batch for the misfits, afm_pso_step for bests and move."""
    for it in range(first, last + 1):
        _, S = afm.forward_batch(prob, sw.x, U, want_defl=False)
        afm.pso_step(cfg, sw, S, it)
    return sw


@pytest.mark.parametrize("name", ["c1", "c2"])
def test_checkpoint_resume_is_bitwise(orc, afm, name):
    """The swarm state (x, v, personal bests, global best key) is the whole
    state of an inversion: copied to the host after evaluation k and
    restored into fresh device buffers, the run continues bit for bit as an
    uninterrupted one (Philox draws are keyed by particle, iteration and
    pixel, so nothing else carries over).  The composed steps also give the
    fused inversion's winner and misfit."""
    spec = W.get(name, cycles=6, P=96, iters=9)
    D = len(spec["free"])
    U32, _, _ = oracle_record(orc, spec)
    prob = afm.make_problem(spec)
    cfg = afm.make_pso(spec)
    U = torch.from_numpy(U32).cuda()
    full = _stepwise(afm, prob, cfg, U, afm.pso_init(cfg, D), 0, spec["iters"])
    part = _stepwise(afm, prob, cfg, U, afm.pso_init(cfg, D), 0, 4)
    torch.cuda.synchronize()
    saved = {k: getattr(part, k).cpu().clone() for k in ("x", "v", "pbest_x", "pbest_S", "gbest")}
    del part
    resumed = afm.SwarmState(**{k: t.cuda() for k, t in saved.items()})
    resumed = _stepwise(afm, prob, cfg, U, resumed, 5, spec["iters"])
    torch.cuda.synchronize()
    for k in ("x", "v", "pbest_x", "pbest_S", "gbest"):
        assert torch.equal(getattr(full, k), getattr(resumed, k)), k
    # the fused inversion is the composition of the same steps
    r, _ = afm.invert(prob, U, cfg)
    torch.cuda.synchronize()
    r = afm.decode_result(r)
    key = int(full.gbest.cpu().numpy().view(np.uint64)[0])
    g = key & 0xFFFFFFFF
    assert r["winner"] == g
    assert np.float32(r["S"]) == full.pbest_S.cpu().numpy()[g]
    np.testing.assert_array_equal(np.float32(r["x"][:D]), full.pbest_x.cpu().numpy()[:, g])


@pytest.mark.parametrize("P", [1, 2, 31, 33])
def test_degenerate_and_ragged_swarm_sizes(orc, afm, P):
    """Swarms of one particle, and sizes that leave the last lane group or
    warp partly empty: the automatic multi-lane iteration equals the
    one-lane arithmetic of the batched-pixel kernel bit for bit, and the
    history never rises."""
    spec = W.get("c2", cycles=8, P=P, iters=4)
    U32, _, _ = oracle_record(orc, spec)
    prob = afm.make_problem(spec)
    cfg = afm.make_pso(spec)
    Ut = torch.from_numpy(U32).cuda()
    r1, h1 = afm.invert(prob, Ut, cfg)
    off = torch.tensor([0, len(U32)], dtype=torch.int64, device="cuda")
    rb, _ = afm.invert_batch(prob, Ut, off, cfg, particles_per_thread=1)
    torch.cuda.synchronize()
    a, b = afm.decode_result(r1), afm.decode_results(rb)[0]
    assert a["status"] == 0 and 0 <= a["winner"] < P
    assert a["winner"] == b["winner"] and a["S"] == b["S"]
    np.testing.assert_array_equal(a["x"], b["x"])
    assert np.all(np.diff(h1.cpu().numpy()) <= 0)
