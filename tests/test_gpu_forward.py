"""GPU parity of the forward problem (Eq. 2 + RK4), the misfit (Eq. 5) and
the synthetic-record generator against the FP64 oracle, through the C ABI.

Tolerances (stated for the FP32 path): forward deflection relative L2 error
<= 1e-5 per particle; misfit relative error <= 1e-4; FP64 path <= 1e-10.
"""
import numpy as np
import pytest

from paper_1109_0334_gb300 import workloads as W
from common import NM, oracle_defl_nm, oracle_record, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FWD_TOL = 1e-5
MIS_TOL = 1e-4


@pytest.fixture(scope="module")
def afm():
    from paper_1109_0334_gb300 import build
    build.build()
    from paper_1109_0334_gb300 import afminv
    assert torch.cuda.is_available()
    return afminv


def _gpu_forward(afm, spec, x_dp, U32=None, n=None):
    prob = afm.make_problem(spec, n_steps=n)
    x = torch.from_numpy(np.ascontiguousarray(x_dp, dtype=np.float32)).cuda()
    U = None if U32 is None else torch.from_numpy(U32).cuda()
    defl, S = afm.forward_batch(prob, x, U)
    torch.cuda.synchronize()
    return defl.cpu().numpy(), (None if S is None else S.cpu().numpy())


@pytest.mark.parametrize("name,P,cycles", [("c1", 100, 20), ("c2", 70, 100), ("c4", 45, 100)])
def test_forward_and_misfit_parity(orc, afm, name, P, cycles):
    """Full record length; P not a multiple of the warp (ragged tail)."""
    spec = W.get(name, cycles=cycles)
    D = len(spec["free"])
    x = W.sample_x(D, P, seed=11 + P)
    U32, U_m, _ = oracle_record(orc, spec)
    defl, S = _gpu_forward(afm, spec, x, U32)
    ref = oracle_defl_nm(orc, spec, x)
    err = rel_l2(defl, ref, axis=0)
    assert err.max() <= FWD_TOL, (err.max(), np.argmax(err))
    c, pm = orc.make_case(spec), orc.make_pmap(spec)
    S_ref = orc.misfit_batch(c, pm, x.astype(np.float64), U_m) / NM ** 2
    assert np.max(np.abs(S - S_ref) / S_ref) <= MIS_TOL


@pytest.mark.parametrize("force,th", [
    ("linear_spring", [(0, 2.0, 20.0, False), (1, 10e-9, 20e-9, False)]),
    ("hooke", [(0, 0.5, 8.0, True), (1, -2e-9, 4e-9, False)]),
    ("spring_damper", [(0, 0.5, 8.0, True), (1, -2e-9, 4e-9, False), (2, 0.0, 2e-7, False)]),
])
def test_other_force_laws(orc, afm, force, th):
    spec = W.get("c2", force=force, cycles=30, free=th, fixed=[0.0, 0.0, 0.0, 0.0, 0.0])
    x = W.sample_x(len(th), 37, seed=5)
    defl, _ = _gpu_forward(afm, spec, x)
    ref = oracle_defl_nm(orc, spec, x)
    assert rel_l2(defl, ref, axis=0).max() <= FWD_TOL


@pytest.mark.parametrize("n_modes", [2, 5, 8])
def test_padded_mode_counts(orc, afm, n_modes):
    """Mode counts without a specialised kernel run in the 8-mode kernel with
    zero padding."""
    spec = W.get("c2", n_modes=n_modes, cycles=20, spc=512 if n_modes > 4 else 256)
    x = W.sample_x(4, 33, seed=n_modes)
    defl, _ = _gpu_forward(afm, spec, x)
    ref = oracle_defl_nm(orc, spec, x)
    assert rel_l2(defl, ref, axis=0).max() <= FWD_TOL


def test_forward_f64_parity(orc, afm):
    spec = W.get("c2", cycles=40)
    x = W.sample_x(4, 20, seed=3).astype(np.float64)
    U32, U_m, _ = oracle_record(orc, spec)
    prob = afm.make_problem(spec)
    xt = torch.from_numpy(x).cuda()
    U = torch.from_numpy(U32.astype(np.float64)).cuda()
    defl, S = afm.forward_batch_f64(prob, xt, U)
    torch.cuda.synchronize()
    ref = oracle_defl_nm(orc, spec, x)
    assert rel_l2(defl.cpu().numpy(), ref, axis=0).max() <= 1e-10
    c, pm = orc.make_case(spec), orc.make_pmap(spec)
    S_ref = orc.misfit_batch(c, pm, x, U_m) / NM ** 2
    np.testing.assert_allclose(S.cpu().numpy(), S_ref, rtol=1e-9)


def test_single_particle_and_single_step(orc, afm):
    spec = W.get("c1", cycles=1)
    x = W.sample_x(2, 1, seed=1)
    defl, _ = _gpu_forward(afm, spec, x, n=1)
    ref = oracle_defl_nm(orc, spec, x, n=1)
    assert defl.shape == (1, 1)
    assert abs(defl[0, 0] - ref[0, 0]) <= 1e-6 * abs(ref[0, 0])


@pytest.mark.parametrize("N,P", [(25600, 1024), (4001, 77), (1, 1), (63, 33)])
def test_misfit_kernel(orc, afm, N, P):
    rng = np.random.default_rng(N + P)
    defl = rng.normal(0, 20, size=(N, P)).astype(np.float32)
    U = rng.normal(0, 20, size=N).astype(np.float32)
    S = afm.misfit(torch.from_numpy(defl).cuda(), torch.from_numpy(U).cuda())
    torch.cuda.synchronize()
    ref = np.array([orc.misfit(U.astype(np.float64), defl[:, p].astype(np.float64)) for p in range(P)])
    np.testing.assert_allclose(S.cpu().numpy(), ref, rtol=MIS_TOL / 10)


def test_diverging_candidate_gives_infinite_misfit(afm):
    """A linear spring of large negative stiffness is unstable: its misfit is
    reported as +inf, the other candidates are unaffected."""
    spec = W.get("c1", force="linear_spring", cycles=20,
                 free=[(0, -5000.0, 10.0, False), (1, 0.0, 20e-9, False)], fixed=[0.0] * 5)
    x = np.array([[0.0, 0.999], [0.5, 0.5]], dtype=np.float32)
    U = np.zeros(W.n_steps(spec), dtype=np.float32)
    _, S = _gpu_forward(afm, spec, x, U)
    assert np.isinf(S[0]) and np.isfinite(S[1])


def test_synth_records_match_oracle(orc, afm):
    """Records made on the GPU (FP32 at dt/4 + Philox/Box-Muller noise) match
    the oracle's records of the same truth and seed."""
    spec = W.get("c3")
    pixels = [0, 1, 2, 3, 4, 5]
    lens = [orc.cycles(spec["seed"], p, 20, 200) * spec["spc"] // 10 for p in pixels]
    xt = np.stack([orc.truth_x(4, spec["seed"], p) for p in pixels], axis=1)
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    prob = afm.make_problem(spec, n_steps=max(lens))
    U = afm.synth_records(prob, torch.from_numpy(xt).cuda(), torch.from_numpy(off).cuda(),
                          spec["record_sub"], spec["sigma"], spec["seed"], 0)
    torch.cuda.synchronize()
    U = U.cpu().numpy()
    c, pm = orc.make_case(spec), orc.make_pmap(spec)
    for i, p in enumerate(pixels):
        ref = orc.record(c, pm, xt[:, i], lens[i], spec["record_sub"], spec["sigma"],
                         spec["seed"], p) / NM
        got = U[off[i]:off[i + 1]]
        assert rel_l2(got, ref) <= FWD_TOL


@pytest.mark.parametrize("name,P", [("c2", 65537), ("c1", 65536)])
def test_paired_particle_forward_is_bit_identical(orc, afm, name, P):
    """Large FP32 DMT batches run two particles per thread in paired FP32
    instructions: deflections and misfits equal the one-particle-per-thread
    kernel's bit for bit (an odd batch ends in a half-filled pair), and a
    sample of them matches the oracle."""
    spec = W.get(name, cycles=2)
    D = len(spec["free"])
    x = torch.from_numpy(W.sample_x(D, P, seed=P)).cuda()
    U32, _, _ = oracle_record(orc, spec)
    Ug = torch.from_numpy(U32).cuda()
    prob = afm.make_problem(spec)
    out = {}
    for lanes in ("one", "auto"):
        afm.set_lanes(lanes)
        try:
            out[lanes] = afm.forward_batch(prob, x, Ug)
            torch.cuda.synchronize()
        finally:
            afm.set_lanes("auto")
    (d1, S1), (d2, S2) = out["one"], out["auto"]
    assert torch.equal(d1, d2) and torch.equal(S1, S2)
    idx = np.array([0, 1, P // 2, P - 2, P - 1])
    ref = oracle_defl_nm(orc, spec, x.cpu().numpy()[:, idx])
    assert rel_l2(d2.cpu().numpy()[:, idx], ref, axis=0).max() <= 1e-5
