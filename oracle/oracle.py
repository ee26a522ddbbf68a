"""ctypes binding of the FP64 CPU oracle (``afm_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the
CPU-baseline leg of the benchmark are the only callers.  The CUDA library
never imports this module and shares no code with it.

All quantities here are SI double precision.  Arrays of swarm coordinates
are dimension-major ``[D][P]`` like the CUDA side's, but nothing else is
shared.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

MAXM = 8
NSLOT = 8       # parameter slots: 0..4 force law, 5..7 base motion (a, f, g)
POINT_MASS, MODAL_EB, FE_HERMITE = 0, 1, 2
F_LINEAR, F_DMT, F_DMT_KV, F_HOOKE, F_SPRING_DAMPER = 0, 1, 2, 3, 4


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP, no fast-math)."""
    src = [os.path.join(_HERE, "afm_oracle.c")]
    hdr = os.path.join(_HERE, "afm_oracle.h")
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(p) for p in src + [hdr])
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= newest:
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-Wall",
           "-o", tmp] + src + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class Case(C.Structure):
    _fields_ = [("model", C.c_int), ("n_modes", C.c_int), ("f1", C.c_double),
                ("k", C.c_double), ("Q", C.c_double * MAXM), ("A0", C.c_double),
                ("Zc", C.c_double), ("spc", C.c_int), ("force", C.c_int),
                ("n_elem", C.c_int), ("L", C.c_double), ("E", C.c_double),
                ("rho", C.c_double), ("fe_k", C.c_double), ("fe_f1", C.c_double),
                ("fe_Q", C.c_double), ("nm_beta", C.c_double), ("drive", C.c_int),
                ("dt", C.c_double), ("n_points", C.c_int), ("point_xi", C.c_double * 4)]


class Modal(C.Structure):
    _fields_ = [("m", C.c_int), ("w", C.c_double * MAXM), ("gam", C.c_double * MAXM),
                ("mass", C.c_double), ("wd", C.c_double), ("a", C.c_double),
                ("psi", C.c_double), ("eta0", C.c_double * MAXM),
                ("etad0", C.c_double * MAXM), ("dt", C.c_double)]


class Pmap(C.Structure):
    _fields_ = [("D", C.c_int), ("slot", C.c_int * 5), ("lo", C.c_double * 5),
                ("hi", C.c_double * 5), ("logs", C.c_int * 5), ("fixed", C.c_double * NSLOT)]


class Pso(C.Structure):
    _fields_ = [("P", C.c_int), ("iters", C.c_int), ("w", C.c_double), ("c1", C.c_double),
                ("c2", C.c_double), ("seed", C.c_uint64), ("pixel", C.c_uint32)]


_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_u32p = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            L.orc_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
            L.orc_uniform.argtypes = [C.c_uint32]
            L.orc_uniform.restype = C.c_double
            L.orc_draw.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32,
                                   C.c_uint32, C.c_uint32, C.c_int]
            L.orc_draw.restype = C.c_double
            L.orc_beam_root.argtypes = [C.c_int]
            L.orc_beam_root.restype = C.c_double
            L.orc_mode_shape.argtypes = [C.c_double, C.c_double]
            L.orc_mode_shape.restype = C.c_double
            L.orc_modal_factors.argtypes = [C.c_int, C.c_int, _dp, _dp, _dp, _dp]
            L.orc_setup.argtypes = [C.POINTER(Case), C.POINTER(Modal)]
            L.orc_drive_half.argtypes = [C.POINTER(Modal), C.c_int, C.c_long]
            L.orc_drive_half.restype = C.c_double
            L.orc_force.argtypes = [C.c_int, _dp, C.c_double, C.c_double]
            L.orc_force.restype = C.c_double
            L.orc_forward.argtypes = [C.POINTER(Case), _dp, C.c_int, C.c_int, _dp, C.c_void_p]
            L.orc_misfit.argtypes = [_dp, _dp, C.c_int]
            L.orc_misfit.restype = C.c_double
            L.orc_map.argtypes = [C.POINTER(Pmap), _dp, _dp]
            L.orc_drive_chirp.restype = C.c_double
            L.orc_drive_chirp.argtypes = [_dp, C.c_double]
            L.orc_misfit_batch.argtypes = [C.POINTER(Case), C.POINTER(Pmap), _dp, C.c_int,
                                           _dp, C.c_int, _dp]
            L.orc_pso_init.argtypes = [C.c_int, C.c_int, C.c_uint64, C.c_uint32, _dp, _dp]
            L.orc_pso_init_slice.argtypes = [C.c_int, C.c_int, C.c_int, C.c_uint64, C.c_uint32,
                                             _dp, _dp]
            L.orc_pso_update_slice.argtypes = [C.c_int, C.c_int, C.c_int, C.c_uint32, C.c_uint64,
                                               C.c_uint32, C.c_double, C.c_double, C.c_double,
                                               _dp, _dp, _dp, _dp]
            L.orc_pso_update.argtypes = [C.c_int, C.c_int, C.c_uint32, C.c_uint64, C.c_uint32,
                                         C.c_double, C.c_double, C.c_double, _dp, _dp, _dp, _dp]
            L.orc_invert.argtypes = [C.POINTER(Case), C.POINTER(Pmap), _dp, C.c_int,
                                     C.POINTER(Pso), _dp, C.POINTER(C.c_double), _dp]
            L.orc_truth_x.argtypes = [C.c_int, C.c_uint64, C.c_uint32, _dp]
            L.orc_cycles.argtypes = [C.c_uint64, C.c_uint32, C.c_int, C.c_int]
            L.orc_record.argtypes = [C.POINTER(Case), C.POINTER(Pmap), _dp, C.c_int, C.c_int,
                                     C.c_double, C.c_uint64, C.c_uint32, _dp]
            L.orc_grad_cs.argtypes = [C.POINTER(Case), C.POINTER(Pmap), _dp, _dp, C.c_int,
                                      C.POINTER(C.c_double), _dp]
            L.orc_polish.argtypes = [C.POINTER(Case), C.POINTER(Pmap), _dp, C.c_int, _dp, C.c_int,
                                     C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, _dp]
            L.orc_normal_eq.argtypes = [C.POINTER(Case), C.POINTER(Pmap), _dp, _dp, C.c_int,
                                        C.POINTER(C.c_double), _dp, _dp]
            L.orc_lm_polish.argtypes = [C.POINTER(Case), C.POINTER(Pmap), _dp, C.c_int, _dp,
                                        C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, _dp]
            L.orc_invert_boxed.argtypes = [C.POINTER(Case), C.POINTER(Pmap), _dp, C.c_int,
                                           C.POINTER(Pso), _dp, _dp, _dp, C.c_int, _dp,
                                           C.POINTER(C.c_double)]
            L.orc_fe_dofs.argtypes = [C.POINTER(Case)]
            L.orc_fe_matrices.argtypes = [C.POINTER(Case), C.c_void_p, C.c_void_p, C.c_void_p,
                                          C.c_void_p, C.c_void_p]
            L.orc_fe_forward.argtypes = [C.POINTER(Case), _dp, C.c_int, C.c_int, _dp, C.c_void_p]
            L.orc_set_threads.argtypes = [C.c_int]
            L.orc_get_threads.restype = C.c_int
            _lib = L
    return _lib


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def get_threads() -> int:
    return int(lib().orc_get_threads())


# --------------------------------------------------------------------------
# Builders from plain workload descriptions (dicts of SI values)
# --------------------------------------------------------------------------
_MODEL = {"point_mass": POINT_MASS, "modal_eb": MODAL_EB, "fe_hermite": FE_HERMITE}
_FORCE = {"linear_spring": F_LINEAR, "dmt": F_DMT, "dmt_kv": F_DMT_KV, "hooke": F_HOOKE,
          "spring_damper": F_SPRING_DAMPER}


def make_case(spec: dict) -> Case:
    c = Case()
    c.model = _MODEL[spec["model"]]
    c.n_modes = int(spec.get("n_modes", 1))
    c.f1 = float(spec.get("f1_hz", 0.0))
    c.k = float(spec.get("k", 0.0))
    q = spec.get("Q", 400.0)
    qs = list(q) if hasattr(q, "__len__") else [q] * MAXM
    for i in range(MAXM):
        c.Q[i] = float(qs[i] if i < len(qs) else qs[-1])
    c.A0 = float(spec.get("A0", 0.0))
    c.Zc = float(spec.get("Zc", 0.0))
    c.spc = int(spec["spc"])
    c.force = _FORCE[spec["force"]]
    c.n_elem = int(spec.get("n_elem", 0))
    c.L = float(spec.get("L", 0.0))
    c.E = float(spec.get("E", 0.0))
    c.rho = float(spec.get("rho", 0.0))
    c.fe_k = float(spec.get("k", 0.0))
    c.fe_f1 = float(spec.get("f1_hz", 0.0))
    c.fe_Q = float(qs[0])
    c.nm_beta = float(spec.get("newmark_beta", 0.25))
    c.drive = 1 if spec.get("drive") == "chirp" else 0
    c.dt = float(spec.get("dt", 0.0))
    pts = spec.get("points", ())
    c.n_points = len(pts)
    for k, xi in enumerate(pts):
        c.point_xi[k] = float(xi)
    return c


def n_values(case: Case) -> int:
    """Record values per step: the deflection points, else the tip."""
    return max(int(case.n_points), 1)


def make_pmap(spec: dict) -> Pmap:
    """spec["free"]: list of (slot, lo, hi, log); spec["fixed"]: 5 slot values."""
    pm = Pmap()
    free = spec["free"]
    pm.D = len(free)
    for d, (slot, lo, hi, lg) in enumerate(free):
        pm.slot[d] = int(slot)
        pm.lo[d] = float(lo)
        pm.hi[d] = float(hi)
        pm.logs[d] = int(bool(lg))
    for s in range(5):
        pm.fixed[s] = float(spec["fixed"][s])
    for s, v in enumerate(spec.get("drive_params", (0.0, 0.0, 0.0))):   # slots 5..7: a, f, g
        pm.fixed[5 + s] = float(v)
    return pm


# --------------------------------------------------------------------------
# Thin wrappers
# --------------------------------------------------------------------------
def philox(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(c, k, out)
    return out


def beam_root(i: int) -> float:
    return lib().orc_beam_root(int(i))


def mode_shape(bL: float, xi: float) -> float:
    return lib().orc_mode_shape(float(bL), float(xi))


def modal_factors(n_modes: int, n_points: int = 501):
    bL, gam, i2, tip = (np.zeros(n_modes) for _ in range(4))
    rc = lib().orc_modal_factors(n_modes, n_points, bL, gam, i2, tip)
    if rc:
        raise ValueError("orc_modal_factors failed")
    return bL, gam, i2, tip


def setup(case: Case) -> Modal:
    md = Modal()
    if lib().orc_setup(C.byref(case), C.byref(md)):
        raise ValueError("orc_setup failed")
    return md


def drive_half(md: Modal, spc: int, j: int) -> float:
    return lib().orc_drive_half(C.byref(md), int(spc), int(j))


def force(kind: int, th, d: float, ddot: float = 0.0) -> float:
    return lib().orc_force(int(kind), np.ascontiguousarray(th, dtype=np.float64),
                           float(d), float(ddot))


def forward(case: Case, th, n_steps: int, sub: int = 1, want_state: bool = False):
    th = np.ascontiguousarray(th, dtype=np.float64)
    u = np.zeros(n_steps * n_values(case))
    m = 1 if case.model == POINT_MASS else case.n_modes
    st = np.zeros((n_steps + 1, 2 * m)) if want_state else None
    rc = lib().orc_forward(C.byref(case), th, int(n_steps), int(sub), u,
                           st.ctypes.data if want_state else None)
    if rc:
        raise ValueError("orc_forward failed")
    return (u, st) if want_state else u


def misfit(U, u) -> float:
    U = np.ascontiguousarray(U, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    return lib().orc_misfit(U, u, len(U))


def map_x(pm: Pmap, x) -> np.ndarray:
    th = np.zeros(NSLOT)
    lib().orc_map(C.byref(pm), np.ascontiguousarray(x, dtype=np.float64), th)
    return th


def misfit_batch(case: Case, pm: Pmap, x_dp, U) -> np.ndarray:
    x = np.ascontiguousarray(x_dp, dtype=np.float64)
    D, P = x.shape
    assert D == pm.D
    U = np.ascontiguousarray(U, dtype=np.float64)
    S = np.zeros(P)
    lib().orc_misfit_batch(C.byref(case), C.byref(pm), x, P, U, len(U) // n_values(case), S)
    return S


def pso_init(P: int, D: int, seed: int, pixel: int = 0, p0: int = 0):
    """Initial positions and velocities [D][P] of particles p0 .. p0 + P - 1."""
    x = np.zeros((D, P))
    v = np.zeros((D, P))
    lib().orc_pso_init_slice(P, p0, D, seed, pixel, x, v)
    return x, v


def pso_update(it: int, seed: int, pixel: int, w: float, c1: float, c2: float,
               x, v, pbest_x, gbest_x, p0: int = 0):
    """Eq. 8 move of particles p0 .. p0 + P - 1 (columns of x, v [D][P])."""
    x = np.array(x, dtype=np.float64, order="C")
    v = np.array(v, dtype=np.float64, order="C")
    D, P = x.shape
    lib().orc_pso_update_slice(P, p0, D, it, seed, pixel, w, c1, c2, x, v,
                               np.ascontiguousarray(pbest_x, dtype=np.float64),
                               np.ascontiguousarray(gbest_x, dtype=np.float64))
    return x, v


def invert(case: Case, pm: Pmap, U, P: int, iters: int, w: float, c1: float, c2: float,
           seed: int, pixel: int = 0):
    cfg = Pso(P=P, iters=iters, w=w, c1=c1, c2=c2, seed=seed, pixel=pixel)
    U = np.ascontiguousarray(U, dtype=np.float64)
    bx = np.zeros(pm.D)
    bS = C.c_double()
    hist = np.zeros(iters + 1)
    lib().orc_invert(C.byref(case), C.byref(pm), U, len(U) // n_values(case), C.byref(cfg), bx,
                     C.byref(bS), hist)
    return bx, bS.value, hist


def invert_boxed(case: Case, pm: Pmap, U, P: int, iters: int, w: float, c1: float, c2: float,
                 seed: int, lo, hi, seeds=None, pixel: int = 0):
    """The swarm searching the box [lo, hi] with seed particles [n_seed][D]
    (reading R17); returns (best x in the cube, best S)."""
    cfg = Pso(P=P, iters=iters, w=w, c1=c1, c2=c2, seed=seed, pixel=pixel)
    U = np.ascontiguousarray(U, dtype=np.float64)
    sd = np.zeros((0, pm.D)) if seeds is None else np.asarray(seeds, dtype=np.float64)
    sd = np.ascontiguousarray(sd.reshape(-1, pm.D))
    bx = np.zeros(pm.D)
    bS = C.c_double()
    rc = lib().orc_invert_boxed(C.byref(case), C.byref(pm), U, len(U) // n_values(case), C.byref(cfg),
                                np.ascontiguousarray(lo, dtype=np.float64),
                                np.ascontiguousarray(hi, dtype=np.float64),
                                sd if len(sd) else np.zeros(pm.D), len(sd), bx, C.byref(bS))
    if rc:
        raise ValueError("orc_invert_boxed failed")
    return bx, bS.value


def truth_x(D: int, seed: int, pixel: int = 0) -> np.ndarray:
    x = np.zeros(D)
    lib().orc_truth_x(D, seed, pixel, x)
    return x


def cycles(seed: int, pixel: int, lo: int, hi: int) -> int:
    return int(lib().orc_cycles(seed, pixel, lo, hi))


def record(case: Case, pm: Pmap, x, n: int, sub: int, sigma: float, seed: int,
           pixel: int = 0) -> np.ndarray:
    U = np.zeros(n * n_values(case))
    rc = lib().orc_record(C.byref(case), C.byref(pm), np.ascontiguousarray(x, dtype=np.float64),
                          n, sub, sigma, seed, pixel, U)
    if rc:
        raise ValueError("orc_record failed")
    return U


def grad_cs(case: Case, pm: Pmap, x, U):
    g = np.zeros(pm.D)
    S = C.c_double()
    U = np.ascontiguousarray(U, dtype=np.float64)
    lib().orc_grad_cs(C.byref(case), C.byref(pm), np.ascontiguousarray(x, dtype=np.float64),
                      U, len(U), C.byref(S), g)
    return S.value, g


def normal_eq(case: Case, pm: Pmap, x, U):
    """(S, H [D][D], b [D]) of the misfit at x: residual sensitivities by the
    complex step on the whole trajectory (reading R15)."""
    D = pm.D
    H = np.zeros(D * D)
    b = np.zeros(D)
    S = C.c_double()
    U = np.ascontiguousarray(U, dtype=np.float64)
    rc = lib().orc_normal_eq(C.byref(case), C.byref(pm), np.ascontiguousarray(x, dtype=np.float64),
                             U, len(U), C.byref(S), H, b)
    if rc:
        raise ValueError("orc_normal_eq failed")
    return S.value, H.reshape(D, D), b


def lm_polish(case: Case, pm: Pmap, U, x_dk, steps: int, n_lambda: int = 8, lam0: float = 1e-7,
              lam_ratio: float = 10.0):
    """Levenberg-Marquardt polish with a ladder of n_lambda damping values
    (reading R15); returns (x [D][K], S [K])."""
    x = np.array(x_dk, dtype=np.float64, order="C")
    D, K = x.shape
    S = np.zeros(K)
    U = np.ascontiguousarray(U, dtype=np.float64)
    rc = lib().orc_lm_polish(C.byref(case), C.byref(pm), U, len(U), x, K, steps, n_lambda, lam0,
                             lam_ratio, S)
    if rc:
        raise ValueError("orc_lm_polish failed")
    return x, S


def refine_optimum(case: Case, pm: Pmap, U, x, max_iter: int = 3000, rtol: float = 1e-14):
    """The minimiser of the cost functional (Eq. 5) over the parameter box
    [0, 1]^D near x (the inverse problem of Sec. 2.3: the parameters whose
    misfit no other admissible parameters undercut), by Marquardt's damped
    Gauss-Newton method with an active set, run to convergence.  Each
    iteration takes the misfit's Gauss-Newton system (normal_eq); holds at
    its bound every coordinate that sits on a bound with the gradient
    pointing out of the box; solves the damped system (H + lam diag H) dx =
    b of the other coordinates; and keeps the step (projected onto the box)
    if it lowers the misfit, dividing lam by 10, else multiplies lam by 10.
    It stops when a step with lam <= 1e-4 lowers the misfit by no more than
    rtol of itself, when lam exceeds 1e12 (no step lowers it), or after
    max_iter iterations (a valley of nearly equal misfit can take that many).
    Returns (x [D], S).

    Pinned by the tests on a 2-parameter case: its result lies at or below
    the minimum of a brute-force grid of the misfit and of a fine local grid
    around it, satisfies the first-order (KKT) conditions of the box, and,
    with the truth placed outside the box, ends on the bound the truth lies
    beyond."""
    x = np.clip(np.asarray(x, dtype=np.float64).ravel().copy(), 0.0, 1.0)
    U = np.ascontiguousarray(U, dtype=np.float64)
    S, H, b = normal_eq(case, pm, x, U)
    lam = 1e-3
    for _ in range(max_iter):
        g = -2.0 * b                                  # gradient of S
        held = ((x <= 0.0) & (g > 0.0)) | ((x >= 1.0) & (g < 0.0))
        free = ~held
        if not free.any():
            break
        Hf = H[np.ix_(free, free)]
        dg = np.diag(Hf)
        dg = np.maximum(dg, 1e-12 * max(dg.max(), 1e-300))
        step = np.zeros_like(x)
        try:
            step[free] = np.linalg.solve(Hf + lam * np.diag(dg), b[free])
        except np.linalg.LinAlgError:
            step[:] = 0.0
        xn = np.clip(x + step, 0.0, 1.0)
        Sn = float(misfit_batch(case, pm, xn.reshape(-1, 1), U)[0])
        if Sn < S:
            small = S - Sn <= rtol * S
            x = xn
            S, H, b = normal_eq(case, pm, x, U)
            if small and lam <= 1e-4:
                break
            lam = max(lam / 10.0, 1e-12)
        else:
            lam *= 10.0
            if lam > 1e12:
                break
    return x, S


def polish(case: Case, pm: Pmap, U, x_dk, steps: int, n_cand: int = 16, alpha0: float = 0.05,
           shrink: float = 0.5, sigma: float = 1e-4):
    """Projected-gradient polish with batched Armijo candidates; returns (x, S)."""
    x = np.array(x_dk, dtype=np.float64, order="C")
    D, K = x.shape
    S = np.zeros(K)
    U = np.ascontiguousarray(U, dtype=np.float64)
    rc = lib().orc_polish(C.byref(case), C.byref(pm), U, len(U), x, K, steps, n_cand, alpha0,
                          shrink, sigma, S)
    if rc:
        raise ValueError("orc_polish failed")
    return x, S


def fe_matrices(case: Case):
    """(M, K, C, geom) of the FE model; geom = thickness, width, mu, w1, w2,
    alpha, beta."""
    n = int(lib().orc_fe_dofs(C.byref(case)))
    M, K, Cm = (np.zeros((n, n)) for _ in range(3))
    geom = np.zeros(7)
    rc = lib().orc_fe_matrices(C.byref(case), M.ctypes.data, K.ctypes.data, Cm.ctypes.data, None,
                               geom.ctypes.data)
    if rc:
        raise ValueError("orc_fe_matrices failed")
    return M, K, Cm, geom


def fe_forward(case: Case, th, n_steps: int, sub: int = 1, want_setup: bool = False):
    u = np.zeros(n_steps)
    st = np.zeros(8)
    rc = lib().orc_fe_forward(C.byref(case), np.ascontiguousarray(th, dtype=np.float64),
                              int(n_steps), int(sub), u, st.ctypes.data)
    if rc:
        raise ValueError("orc_fe_forward failed")
    return (u, st) if want_setup else u
