"""Shared helpers of the test suite: workload conversion for the oracle and
for the CUDA library, oracle-made records, and the identifiable-parameter
comparison used for inversion parity."""
from __future__ import annotations

import math

import numpy as np

from paper_1109_0334_gb300 import workloads as W

NM = 1e-9


def oracle_case(orc, spec):
    return orc.make_case(spec), orc.make_pmap(spec)


def oracle_record(orc, spec, pixel: int = 0, n: int | None = None):
    """Record of the workload's seeded truth, made by the oracle (FP64,
    finer step, noise).  Returns (U_nm float32, U_m float64 of the same
    float32 values, truth x)."""
    c, pm = oracle_case(orc, spec)
    n = W.n_steps(spec) if n is None else n
    xt = orc.truth_x(pm.D, spec["seed"], pixel)
    U = orc.record(c, pm, xt, n, spec["record_sub"], spec["sigma"], spec["seed"], pixel)
    U32 = (U / NM).astype(np.float32)
    return U32, U32.astype(np.float64) * NM, xt


def oracle_defl_nm(orc, spec, x_dp, n: int | None = None):
    """Oracle deflection [n * values per step][P] in nm (the tip, or the
    workload's deflection points) for coordinates x [D][P]."""
    c, pm = oracle_case(orc, spec)
    n = W.n_steps(spec) if n is None else n
    x_dp = np.asarray(x_dp, dtype=np.float64)
    out = np.empty((n * orc.n_values(c), x_dp.shape[1]))
    for p in range(x_dp.shape[1]):
        th = orc.map_x(pm, x_dp[:, p])
        out[:, p] = orc.forward(c, th, n) / NM
    return out


def rel_l2(a, b, axis=0):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b, axis=axis) / np.linalg.norm(b, axis=axis)


def hessian_x(orc, c, pm, U_m, x0, h=1e-3):
    """Misfit Hessian in normalised coordinates by central differences."""
    D = len(x0)
    pts, idx = [], {}
    for a in range(D):
        for b in range(a, D):
            for sa in (1, -1):
                for sb in (1, -1):
                    xx = np.array(x0, dtype=np.float64)
                    xx[a] += sa * h
                    xx[b] += sb * h
                    idx[(a, b, sa, sb)] = len(pts)
                    pts.append(xx)
    S = orc.misfit_batch(c, pm, np.array(pts).T.copy(), U_m)
    H = np.zeros((D, D))
    for a in range(D):
        for b in range(a, D):
            H[a, b] = H[b, a] = (S[idx[(a, b, 1, 1)]] - S[idx[(a, b, 1, -1)]]
                                 - S[idx[(a, b, -1, 1)]] + S[idx[(a, b, -1, -1)]]) / (4 * h * h)
    return H


def _rel_scale(spec, d):
    """Fixed scale for relative errors of free dimension d (workload key
    rel_scale), or None: relative to the parameter's own value."""
    rs = spec.get("rel_scale")
    return None if rs is None else rs[d]


def log_jacobian(spec, x):
    """d ln(theta_d) / d x_d for each free dimension at x (for a dimension
    with a fixed relative scale s: d (theta_d / s) / d x_d)."""
    J = np.empty(len(spec["free"]))
    for d, (slot, lo, hi, lg) in enumerate(spec["free"]):
        sc = _rel_scale(spec, d)
        if lg:
            J[d] = math.log(10.0) * (math.log10(hi) - math.log10(lo))
        elif sc is not None:
            J[d] = (hi - lo) / sc
        else:
            th = lo + x[d] * (hi - lo)
            J[d] = (hi - lo) / th if th > 0 else np.inf
    return J


def identifiable_check(orc, spec, U_m, x_ref, S_ref, x_test, rel_param=0.005):
    """Parameters are compared where the record determines them: the
    eigen-directions of the misfit Hessian (in log-parameter coordinates, at
    the reference optimum) whose one-sigma statistical half-width (noise
    sigma) is below `rel_param`.  Returns (max projected relative error over
    those directions, number of identifiable directions, S_oracle(x_test))."""
    c, pm = oracle_case(orc, spec)
    H = hessian_x(orc, c, pm, U_m, x_ref)
    J = log_jacobian(spec, x_ref)
    Jinv = np.diag(1.0 / J)
    Hr = Jinv @ H @ Jinv
    lam, V = np.linalg.eigh(Hr)
    sig2 = spec["sigma"] ** 2
    widths = np.sqrt(2 * sig2 / np.maximum(lam, 1e-300))
    ident = widths <= rel_param
    th_ref = orc.map_x(pm, x_ref)
    th_t = orc.map_x(pm, x_test)
    drho = np.array([(th_t[s] - th_ref[s]) / _rel_scale(spec, d) if _rel_scale(spec, d) is not None
                     else math.log(th_t[s] / th_ref[s]) for d, (s, *_r) in enumerate(spec["free"])])
    proj = np.abs(V.T @ drho)
    err = float(proj[ident].max()) if ident.any() else 0.0
    S_t = orc.misfit_batch(c, pm, np.asarray(x_test, dtype=np.float64).reshape(-1, 1), U_m)[0]
    return err, int(ident.sum()), float(S_t), widths


def law_combinations(orc, spec, x):
    """The parameter combinations a DMT-family law depends on (Sec. 3.3 force
    law: van der Waals -H R / (6 d^2), Hertz (4/3) E* sqrt(R) (a0 - d)^1.5,
    Kelvin-Voigt eta sqrt(R) sqrt(a0 - d) d'): H R, E* sqrt(R), a0 and, with
    contact damping, eta sqrt(R).  Along R with these fixed the force, and
    so the misfit, is exactly constant: R alone is not determined."""
    pm = orc.make_pmap(spec)
    th = orc.map_x(pm, np.asarray(x, dtype=np.float64))
    comb = [th[1] * th[2], th[0] * math.sqrt(th[2]), th[3]]
    if spec["force"] == "dmt_kv":
        comb.append(th[4] * math.sqrt(th[2]))
    return np.array(comb)


def combination_error(orc, spec, x_ref, x_test):
    """Largest relative difference of the law's combinations."""
    a, b = law_combinations(orc, spec, x_ref), law_combinations(orc, spec, x_test)
    return float(np.max(np.abs(b / a - 1)))
