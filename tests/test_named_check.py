"""CPU checks of the inversion-parity helpers (tests/common.py) on oracle
records: the Gauss-Newton Hessian agrees with central differences where the
record determines the parameters, a point moved along the DMT law's exact
valley (R changed with H R, E* sqrt(R) and a0 held) has the same misfit and
zero error on every named combination, and the determined subspace of the
full-size 3-mode record holds E* sqrt(R), most of a0 and little of H R."""
import json
import math
import os

import numpy as np

from paper_1109_0334_gb300 import workloads as W
from common import (NM, hessian_x, identifiable_check, inside, log_jacobian, named_check,
                    oracle_record, rho_eigen)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _c2_gold(orc):
    with open(os.path.join(GOLDEN, "c2_invert.json")) as f:
        gold = json.load(f)
    spec = W.get("c2")
    _, U_m, _ = oracle_record(orc, spec)
    return spec, U_m, np.array(gold["x"]), gold["S_m2"]


def test_gauss_newton_matches_finite_differences(orc):
    spec, U_m, x0, _ = _c2_gold(orc)
    lam, V, widths = rho_eigen(orc, spec, U_m, x0)
    c, pm = orc.make_case(spec), orc.make_pmap(spec)
    H = hessian_x(orc, c, pm, U_m, x0)
    J = log_jacobian(spec, x0)
    Hr = H / np.outer(J, J)
    # the curvature along each determined direction, both ways
    for k in np.nonzero(widths <= 0.005)[0]:
        v = V[:, k]
        assert abs(v @ Hr @ v / lam[k] - 1) <= 0.05
    # the exact valley direction (rho_E, rho_H, rho_R, rho_a0) ~ (1/2, 1, -1, 0)
    null = np.array([0.5, 1.0, -1.0, 0.0]) / 1.5
    assert abs(null @ V[:, 0]) >= 1 - 1e-6 and widths[0] > 1e3


def test_valley_point_has_zero_named_error(orc):
    spec, U_m, x0, S0 = _c2_gold(orc)
    pm = orc.make_pmap(spec)
    th = orc.map_x(pm, x0)
    # R -> 1.3 R with H R, E* sqrt(R), a0 held: back to normalised coordinates
    R1 = 1.3 * th[2]
    th1 = [th[0] * math.sqrt(th[2] / R1), th[1] * th[2] / R1, R1, th[3]]
    x1 = np.empty(4)
    for d, (slot, lo, hi, lg) in enumerate(spec["free"]):
        x1[d] = (math.log10(th1[slot]) - math.log10(lo)) / (math.log10(hi) - math.log10(lo)) \
            if lg else (th1[slot] - lo) / (hi - lo)
    c = orc.make_case(spec)
    S1 = orc.misfit_batch(c, pm, x1.reshape(-1, 1), U_m)[0]
    assert abs(S1 / S0 - 1) <= 1e-10
    n_id, named = named_check(orc, spec, U_m, x0, x1)
    assert n_id == 2
    assert all(e <= 1e-9 for _f, e in named.values()), named
    err, n2, _S, _w = identifiable_check(orc, spec, U_m, x0, S0, x1)
    assert n2 == 2 and err <= 1e-9


def test_named_subspace_of_the_full_size_record(orc):
    spec, U_m, x0, _ = _c2_gold(orc)
    n_id, named = named_check(orc, spec, U_m, x0, x0)
    assert n_id == 2
    assert inside(named) == ["E* sqrt(R)"]
    assert named["E* sqrt(R)"][0] >= 0.999 and 0.9 <= named["a0"][0] < 0.99
    assert named["H R"][0] <= 0.3
