"""Why the FE beam runs in its modal basis rather than as a dense
propagator product on the tensor cores: the physical-coordinate Newmark
recursion (the oracle's three-term form, tip force left out) applied with
the dense propagator at reduced precision, against FP64, on the FE
model's own matrices.  The propagator mixes the resonant mode with stiff
element modes (condition ~3e4), so FP32 already loses ~1e-3 of the
resonant response over 10 cycles and TF32 operands (10 mantissa bits)
lose it entirely."""
import math

import numpy as np

from paper_1109_0334_gb300 import workloads as W


def _tf32(x):
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    return ((b + 0x1000) & 0xFFFFE000).astype(np.uint32).view(np.float32)


def test_dense_fe_propagator_loses_the_resonant_response(orc):
    spec = W.get("c5", cycles=10)
    c = orc.make_case(spec)
    M, K, Cm, _ = orc.fe_matrices(c)
    n = M.shape[0]
    tip = n - 2
    _, setup = orc.fe_forward(c, orc.map_x(orc.make_pmap(spec), np.full(4, 0.5)), 1,
                              want_setup=True)
    w1, a, psi, h = (float(setup[i]) for i in (0, 4, 5, 6))
    r = np.zeros(n)
    r[0::2] = 1.0
    Mr = M @ r
    X = np.linalg.solve(K - w1 * w1 * M + 1j * w1 * Cm, Mr.astype(complex))
    u0 = (a * w1 * w1 * X * np.exp(1j * psi)).imag
    um = (a * w1 * w1 * X * np.exp(1j * (psi - w1 * h))).imag
    q = h * h / 4
    Si = np.linalg.inv(M + h / 2 * Cm + q * K)
    A1 = Si @ (2 * M - h * h / 2 * K)
    A2 = -Si @ (M - h / 2 * Cm + q * K)
    bG = q * (Si @ Mr)
    spc, N = c.spc, W.n_steps(spec)

    def run(mode):
        u, v = u0.copy(), um.copy()
        A1m, A2m = A1, A2
        if mode != "f64":
            A1m, A2m = A1.astype(np.float32), A2.astype(np.float32)
            if mode == "tf32":
                A1m, A2m = _tf32(A1m), _tf32(A2m)
            u, v = u.astype(np.float32), v.astype(np.float32)
        out = np.zeros(N)
        for s in range(N):
            G = a * w1 * w1 * (math.sin(w1 * h * ((s + 1) % spc) + psi)
                               + 2 * math.sin(w1 * h * (s % spc) + psi)
                               + math.sin(w1 * h * ((s - 1) % spc) + psi))
            if mode == "f64":
                up = A1m @ u + A2m @ v + bG * G
            else:
                uu, vv = (_tf32(u), _tf32(v)) if mode == "tf32" else (u, v)
                up = (A1m @ uu + A2m @ vv + (bG * G).astype(np.float32)).astype(np.float32)
            v, u = u, up
            out[s] = float(u[tip])
        return out

    ref = run("f64")
    # the FP64 dense recursion is the oracle's FE solve with a zero tip force
    c0 = orc.make_case(dict(spec, force="linear_spring", fixed=[0.0] * 5))
    u_or = orc.fe_forward(c0, np.zeros(8), N)
    assert np.linalg.norm(u_or - ref) <= 1e-7 * np.linalg.norm(ref)
    e32 = np.linalg.norm(run("f32") - ref) / np.linalg.norm(ref)
    etf = np.linalg.norm(run("tf32") - ref) / np.linalg.norm(ref)
    assert 1e-4 < e32 < 1e-2
    assert etf > 0.1
