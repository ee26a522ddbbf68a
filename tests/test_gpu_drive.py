"""Base-motion inversion (Sec. 4.1; drive mode 1, reading R18): the base
moves as a sin(2 pi (f t + g t^2)) with per-particle (a, f, g), the
cantilever starts at rest.  GPU forward solves against the oracle in FP32
and FP64; the paper's three experiments (amplitude, amplitude + frequency,
chirp) inverted on the GPU against the oracle's inversion of the same
records and the paper's truths."""
import numpy as np
import pytest

from paper_1109_0334_gb300 import workloads as W
from common import NM, assert_determined, identifiable_check, oracle_defl_nm, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def afm():
    from paper_1109_0334_gb300 import build
    build.build()
    from paper_1109_0334_gb300 import afminv
    assert torch.cuda.is_available()
    return afminv


@pytest.mark.parametrize("name,modes", [("f3_chirp", 8), ("f3_chirp", 3), ("f3_amp_freq", 8),
                                        ("f3_amp_freq", 1)])
def test_drive_forward_parity(orc, afm, name, modes):
    over = dict(n_modes=modes) if modes > 1 else dict(model="point_mass", n_modes=1)
    spec = W.get(name, n_steps=3000, **over)
    D = len(spec["free"])
    x = W.sample_x(D, 37, seed=17)
    prob = afm.make_problem(spec)
    defl, _ = afm.forward_batch(prob, torch.from_numpy(x).cuda(), None)
    d64, _ = afm.forward_batch_f64(prob, torch.from_numpy(x.astype(np.float64)).cuda(), None)
    torch.cuda.synchronize()
    ref = oracle_defl_nm(orc, spec, x)
    assert rel_l2(defl.cpu().numpy(), ref, axis=0).max() <= 1e-5
    assert rel_l2(d64.cpu().numpy(), ref, axis=0).max() <= 1e-9


@pytest.mark.parametrize("name,named", [("f3_amp", ["a"]), ("f3_amp_freq", ["a", "f"]),
                                        ("f3_chirp", ["a", "f", "g"])])
def test_drive_inversion(orc, afm, name, named):
    spec = W.get(name)
    c, pm = orc.make_case(spec), orc.make_pmap(spec)
    n = W.n_steps(spec)
    xt = np.array(spec["x_truth"])
    U_m = orc.record(c, pm, xt, n, spec["record_sub"], spec["sigma"], spec["seed"], 0)
    U32 = (U_m / NM).astype(np.float32)
    U_m = U32.astype(np.float64) * NM
    x_o, S_o, _ = orc.invert(c, pm, U_m, spec["P"], spec["iters"], spec["w"], spec["c1"],
                             spec["c2"], spec["seed"])
    prob = afm.make_problem(spec)
    res, _ = afm.invert(prob, torch.from_numpy(U32).cuda(), afm.make_pso(spec))
    torch.cuda.synchronize()
    r = afm.decode_result(res)
    D = pm.D
    err, n_id, S_g, widths = identifiable_check(orc, spec, U_m, x_o, S_o, r["x"][:D])
    assert r["status"] == 0 and n_id == len(named)
    assert err <= 0.005, (err, widths)
    assert_determined(orc, spec, U_m, x_o, r["x"][:D], len(named), named)
    assert S_g <= S_o * (1 + 1e-4)
    assert abs(r["S"] - S_g / NM ** 2) <= 1e-4 * S_g / NM ** 2
    assert abs(r["S_f64"] - S_g / NM ** 2) <= 1e-9 * S_g / NM ** 2
    th = orc.map_x(pm, r["x"][:D])
    np.testing.assert_allclose(r["drive"], th[5:8], rtol=1e-12)
    err_t, _, _, _ = identifiable_check(orc, spec, U_m, x_o, S_o, xt)
    assert err_t <= 0.01


def test_drive_mode_is_rejected_where_unsupported(afm):
    spec = W.get("f3_amp")
    prob = afm.make_problem(spec)
    x = torch.full((1, 4), 0.5, device="cuda")
    U = torch.zeros(W.n_steps(spec), device="cuda")
    with pytest.raises(afm.AfmError) as e:
        afm.adjoint(prob, x, U)
    assert e.value.status == 5          # AFM_ERR_UNSUPPORTED
