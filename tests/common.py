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


def _gauss_newton_ok(spec) -> bool:
    """The oracle's complex-step residual sensitivities cover the force-law
    slots of the steady drive on tip records."""
    return (spec.get("drive") is None and not spec.get("points")
            and all(f[0] < 5 for f in spec["free"]))


def rho_eigen(orc, spec, U_m, x_ref, rel_param=0.005):
    """Eigen-decomposition of the misfit Hessian in the relative coordinates
    rho (log-parameters; a dimension with a fixed relative scale s: theta /
    s) at x_ref: eigenvalues, eigenvectors (columns) and their one-sigma
    statistical half-widths sqrt(2 sigma^2 / lambda) for noise sigma.  The
    Hessian is the Gauss-Newton matrix 2 sum_n a_n a_n^T of the oracle's
    complex-step residual sensitivities where it has them (exact to
    rounding, so a direction the misfit does not see has a zero eigenvalue),
    else central differences of the misfit."""
    c, pm = oracle_case(orc, spec)
    x_ref = np.asarray(x_ref, dtype=np.float64)
    if _gauss_newton_ok(spec):
        _S, Hgn, _b = orc.normal_eq(c, pm, x_ref.reshape(-1, 1).copy(), U_m)
        H = 2.0 * np.asarray(Hgn)
    else:
        H = hessian_x(orc, c, pm, U_m, x_ref)
    J = log_jacobian(spec, x_ref)
    Hr = H / np.outer(J, J)
    lam, V = np.linalg.eigh(Hr)
    widths = np.sqrt(2 * spec["sigma"] ** 2 / np.maximum(lam, 1e-300))
    return lam, V, widths


def _drho(orc, spec, x_ref, x_test):
    pm = orc.make_pmap(spec)
    th_ref = orc.map_x(pm, np.asarray(x_ref, dtype=np.float64))
    th_t = orc.map_x(pm, np.asarray(x_test, dtype=np.float64))
    return np.array([(th_t[s] - th_ref[s]) / _rel_scale(spec, d) if _rel_scale(spec, d) is not None
                     else math.log(th_t[s] / th_ref[s]) for d, (s, *_r) in enumerate(spec["free"])])


def identifiable_check(orc, spec, U_m, x_ref, S_ref, x_test, rel_param=0.005):
    """Parameters are compared where the record determines them: the
    eigen-directions of the misfit Hessian (rho_eigen, at the reference
    optimum) whose one-sigma statistical half-width (noise sigma) is below
    `rel_param`.  Returns (max projected relative error over those
    directions, number of identifiable directions, S_oracle(x_test),
    widths)."""
    c, pm = oracle_case(orc, spec)
    lam, V, widths = rho_eigen(orc, spec, U_m, x_ref)
    ident = widths <= rel_param
    proj = np.abs(V.T @ _drho(orc, spec, x_ref, x_test))
    err = float(proj[ident].max()) if ident.any() else 0.0
    S_t = orc.misfit_batch(c, pm, np.asarray(x_test, dtype=np.float64).reshape(-1, 1), U_m)[0]
    return err, int(ident.sum()), float(S_t), widths


def named_combinations(spec):
    """The parameter combinations the force law depends on, each as
    (name, {slot: exponent}): a DMT-family law sees H and R only through
    H R (van der Waals -H R / (6 d^2)), E* and R only through E* sqrt(R)
    (Hertz), and, with contact damping, eta only through eta sqrt(R); a0
    enters alone.  Combinations whose slots are all fixed are left out.
    Other laws (Hooke, spring-damper, base motion): the free parameters
    themselves."""
    free_slots = [f[0] for f in spec["free"]]
    if spec["force"] in ("dmt", "dmt_kv"):
        cands = [("H R", {1: 1.0, 2: 1.0}), ("E* sqrt(R)", {0: 1.0, 2: 0.5}), ("a0", {3: 1.0})]
        if spec["force"] == "dmt_kv":
            cands.append(("eta sqrt(R)", {4: 1.0, 2: 0.5}))
        return [(n, e) for n, e in cands if any(sl in free_slots for sl in e)]
    names = {0: "k", 1: "h", 2: "zeta_s", 5: "a", 6: "f", 7: "g"}
    return [(names.get(sl, f"slot {sl}"), {sl: 1.0}) for sl in free_slots]


def named_check(orc, spec, U_m, x_ref, x_test, rel_param=0.005):
    """The named combinations (named_combinations) against the determined
    subspace (the span of the Hessian eigen-directions of rho_eigen whose
    half-width is <= rel_param): for combination k with gradient g_k in rho
    (log c_k = sum_s e_s rho_s), the fraction |P g_k|^2 / |g_k|^2 of it that
    lies in that subspace (1: fully determined; the rest of it runs along
    directions the record resolves worse than rel_param), and the relative
    difference of c_k between x_test and x_ref.  Returns (n_id, {name:
    (fraction, relative difference)})."""
    lam, V, widths = rho_eigen(orc, spec, U_m, x_ref)
    ident = V[:, widths <= rel_param]
    d_of = {slot: d for d, (slot, *_r) in enumerate(spec["free"])}
    drho = _drho(orc, spec, x_ref, x_test)
    out = {}
    for name, expo in named_combinations(spec):
        g = np.zeros(len(spec["free"]))
        for sl, e in expo.items():
            if sl in d_of:
                g[d_of[sl]] = e
        pg = ident @ (ident.T @ g)
        frac = float(pg @ pg / (g @ g))
        lr = float(g @ drho)
        sl0 = next(iter(expo))
        err = abs(lr) if (len(expo) == 1 and _rel_scale(spec, d_of[sl0]) is not None) \
            else abs(math.expm1(lr))
        out[name] = (frac, err)
    return int(ident.shape[1]), out


def inside(named, min_frac=0.99):
    """Names of the combinations that lie (to min_frac of their squared
    length, i.e. within ~6 degrees) in the determined subspace.  (A
    combination further out can move along a statistically flat direction:
    on the full-size 3-mode record a0 lies 95 % inside, and two optima of
    equal misfit differ in a0 by 1.4 %.)"""
    return sorted(n for n, (f, _e) in named.items() if f >= min_frac)


def assert_determined(orc, spec, U_m, x_ref, x_test, n_id, names, rel_param=0.005):
    """The inversion-parity statement made explicit: the record determines
    exactly n_id eigen-directions to rel_param; the named combinations
    `names` (and no others) lie in their span; x_test agrees with x_ref on
    each of those combinations within rel_param."""
    n, named = named_check(orc, spec, U_m, x_ref, x_test, rel_param)
    assert n == n_id, (n, named)
    assert inside(named) == sorted(names), named
    for k in names:
        assert named[k][1] <= rel_param, (k, named[k])
    return named


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
