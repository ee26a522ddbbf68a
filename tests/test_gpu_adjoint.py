"""GPU parity of the discrete adjoint (gradient of the misfit with respect
to the normalised force parameters) against the FP64 oracle's complex-step
gradient and against central differences, through the C ABI and the
torch.autograd binding.

Tolerance: each gradient component within 1e-3 of the gradient's largest
component (FP32 recurrence over up to 25 600 steps)."""
import numpy as np
import pytest

from paper_1109_0334_gb300 import workloads as W
from common import NM, oracle_record

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-3


@pytest.fixture(scope="module")
def afm():
    from paper_1109_0334_gb300 import build
    build.build()
    from paper_1109_0334_gb300 import afminv
    assert torch.cuda.is_available()
    return afminv


def _setup(orc, name, cycles, P, seed):
    spec = W.get(name, cycles=cycles)
    U32, U_m, xt = oracle_record(orc, spec)
    D = len(spec["free"])
    x = np.clip(xt[:, None] + W.sample_x(D, P, seed=seed, lo=-0.15, hi=0.15), 0.02, 0.98)
    return spec, U32, U_m, x.astype(np.float32)


@pytest.mark.parametrize("name,cycles,P", [("c4", 20, 6), ("c4", 100, 4), ("c2", 100, 4), ("c1", 20, 5)])
def test_adjoint_vs_oracle_complex_step(orc, afm, name, cycles, P):
    spec, U32, U_m, x = _setup(orc, name, cycles, P, seed=cycles + P)
    prob = afm.make_problem(spec)
    xt = torch.from_numpy(x).cuda()
    Ut = torch.from_numpy(U32).cuda()
    S, G = afm.adjoint(prob, xt, Ut)
    _, S_fwd = afm.forward_batch(prob, xt, Ut, want_defl=False)
    torch.cuda.synchronize()
    # the adjoint integrates with every mode compensated, the forward kernel
    # the lowest mode only: the two misfits agree within the misfit
    # tolerance, and the adjoint's is the oracle's to the same bound
    torch.testing.assert_close(S, S_fwd, rtol=1e-4, atol=0)
    G = G.cpu().numpy()
    c, pm = orc.make_case(spec), orc.make_pmap(spec)
    for p in range(P):
        S_o, g_o = orc.grad_cs(c, pm, x[:, p].astype(np.float64), U_m)
        assert abs(float(S[p]) - S_o / NM ** 2) <= 1e-4 * S_o / NM ** 2
        g_o = g_o / NM ** 2
        scale = np.max(np.abs(g_o))
        assert np.max(np.abs(G[:, p] - g_o)) <= GRAD_TOL * scale, (p, G[:, p], g_o)


def test_adjoint_vs_central_differences(orc, afm):
    """Central differences of the FP64 misfit.  With the prescribed relative
    step 1e-4 the differences straddle contact-switch events (the misfit
    bends on that scale in the stiff directions) and can be off by a few
    percent from the exact derivative; with a relative step of 1e-6 they
    converge to it (they agree with the complex-step derivative to ~2e-4).
    The adjoint must match the 1e-6 differences; its agreement with the 1e-4
    differences is checked where those agree with the complex step."""
    spec, U32, U_m, x = _setup(orc, "c4", 40, 3, seed=9)
    prob = afm.make_problem(spec)
    S, G = afm.adjoint(prob, torch.from_numpy(x).cuda(), torch.from_numpy(U32).cuda())
    torch.cuda.synchronize()
    G = G.cpu().numpy()
    c, pm = orc.make_case(spec), orc.make_pmap(spec)
    D = pm.D

    def fd(p, d, rel):
        h = rel * float(x[d, p])
        xp = x[:, p].astype(np.float64).copy()
        xm = xp.copy()
        xp[d] += h
        xm[d] -= h
        Sv = orc.misfit_batch(c, pm, np.stack([xp, xm], axis=1), U_m) / NM ** 2
        return (Sv[0] - Sv[1]) / (2 * h)

    for p in range(x.shape[1]):
        f6 = np.array([fd(p, d, 1e-6) for d in range(D)])
        scale = np.max(np.abs(f6))
        assert np.max(np.abs(G[:, p] - f6)) <= 2 * GRAD_TOL * scale, (G[:, p], f6)
        f4 = np.array([fd(p, d, 1e-4) for d in range(D)])
        _, g_cs = orc.grad_cs(c, pm, x[:, p].astype(np.float64), U_m)
        g_cs = g_cs / NM ** 2
        ok = np.abs(f4 - g_cs) <= GRAD_TOL * scale
        assert np.all(np.abs(G[ok, p] - f4[ok]) <= 2 * GRAD_TOL * scale)


def test_autograd_function(afm):
    spec = W.get("c2", cycles=10)
    N = W.n_steps(spec)
    prob = afm.make_problem(spec)
    U = torch.zeros(N, dtype=torch.float32, device="cuda")
    x = torch.tensor(W.sample_x(4, 8, seed=4), device="cuda", requires_grad=True)
    S = afm.misfit_autograd(prob, x, U)
    w = torch.arange(1, 9, dtype=torch.float32, device="cuda")
    (S * w).sum().backward()
    S2, G = afm.adjoint(prob, x.detach(), U)
    torch.cuda.synchronize()
    assert torch.equal(S.detach(), S2)
    assert torch.allclose(x.grad, G * w[None, :], rtol=0, atol=0)
