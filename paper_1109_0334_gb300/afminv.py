"""Python binding of libafminv (ctypes).  Argument marshalling only: every
step of the computation runs in the library's CUDA kernels.  PyTorch supplies
device memory and streams.

The names follow the C ABI in ``include/afminv.h``:
``forward_batch``, ``forward_batch_f64``, ``misfit``, ``pso_init``,
``pso_step``, ``invert``, ``synth_records``.

If the shared library is missing this module raises on first use; there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libafminv.so")

MAX_MODES, MAX_PARAMS, MAX_POINTS = 8, 5, 4
POINT_MASS, MODAL_EB, FE_HERMITE = 0, 1, 2
LINEAR_SPRING, DMT, DMT_KV, HOOKE, SPRING_DAMPER = 0, 1, 2, 3, 4
OK, ERR_INVALID_ARG, ERR_CUDA, ERR_NONFINITE, ERR_TIMEOUT, ERR_UNSUPPORTED = range(6)

_MODEL = {"point_mass": POINT_MASS, "modal_eb": MODAL_EB, "fe_hermite": FE_HERMITE}
_FORCE = {"linear_spring": LINEAR_SPRING, "dmt": DMT, "dmt_kv": DMT_KV, "hooke": HOOKE,
          "spring_damper": SPRING_DAMPER}


class Problem(C.Structure):
    _fields_ = [("model", C.c_int), ("n_modes", C.c_int), ("f1_hz", C.c_double),
                ("k_N_per_m", C.c_double), ("Q", C.c_double * MAX_MODES),
                ("n_elem", C.c_int), ("L_m", C.c_double), ("E_Pa", C.c_double),
                ("rho_kg_m3", C.c_double), ("newmark_beta", C.c_double),
                ("A0_m", C.c_double), ("Zc_m", C.c_double), ("steps_per_cycle", C.c_int),
                ("n_steps", C.c_int), ("force", C.c_int), ("fixed", C.c_double * MAX_PARAMS),
                ("n_free", C.c_int), ("slot", C.c_int * MAX_PARAMS),
                ("lo", C.c_double * MAX_PARAMS), ("hi", C.c_double * MAX_PARAMS),
                ("log_scale", C.c_int * MAX_PARAMS), ("drive_mode", C.c_int),
                ("dt_s", C.c_double), ("drive_a_m", C.c_double), ("drive_f_hz", C.c_double),
                ("drive_g_hz_s", C.c_double), ("n_points", C.c_int),
                ("point_xi", C.c_double * MAX_POINTS)]


class PsoCfg(C.Structure):
    _fields_ = [("P", C.c_int), ("iters", C.c_int), ("w", C.c_double), ("c1", C.c_double),
                ("c2", C.c_double), ("seed", C.c_uint64), ("pixel", C.c_uint32)]


class BatchSelect(C.Structure):
    _fields_ = [("pixels", C.c_void_p), ("n_run", C.c_int), ("box_lo", C.c_void_p),
                ("box_hi", C.c_void_p), ("seeds", C.c_void_p), ("n_seed", C.c_int)]


class ImageCfg(C.Structure):
    _fields_ = [("width", C.c_int), ("height", C.c_int), ("stride", C.c_int),
                ("margin", C.c_double), ("coarse", PsoCfg), ("fine", PsoCfg),
                ("coarse_polish_k", C.c_int), ("coarse_polish_steps", C.c_int),
                ("fine_polish_k", C.c_int), ("fine_polish_steps", C.c_int),
                ("n_cand", C.c_int), ("method", C.c_int)]


class Swarm(C.Structure):
    _fields_ = [("P", C.c_int), ("D", C.c_int), ("x", C.c_void_p), ("v", C.c_void_p),
                ("pbest_x", C.c_void_p), ("pbest_S", C.c_void_p), ("gbest", C.c_void_p)]


class Result(C.Structure):
    _fields_ = [("x", C.c_double * MAX_PARAMS), ("theta", C.c_double * MAX_PARAMS),
                ("S", C.c_double), ("S_f64", C.c_double), ("J_rel", C.c_double),
                ("iters", C.c_int32), ("winner", C.c_int32), ("nonfinite", C.c_int32),
                ("status", C.c_int32), ("defect", C.c_double), ("segments", C.c_int32),
                ("reserved", C.c_int32), ("drive", C.c_double * 3)]


class AfmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


_lock = threading.Lock()
_lib = None
_ctx = {}


def lib():
    """Load libafminv.so (built by ``paper_1109_0334_gb300.build``)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libafminv is not built ({LIB_PATH} missing); run "
                                   "paper_1109_0334_gb300.build.build() first")
            L = C.CDLL(LIB_PATH)
            vp, i, u32, u64, d = C.c_void_p, C.c_int, C.c_uint32, C.c_uint64, C.c_double
            L.afm_ctx_create.argtypes = [i, C.POINTER(vp)]
            L.afm_ctx_destroy.argtypes = [vp]
            L.afm_last_error.restype = C.c_char_p
            L.afm_status_string.restype = C.c_char_p
            L.afm_status_string.argtypes = [i]
            L.afm_profile_enable.argtypes = [vp, i]
            L.afm_set_lanes.argtypes = [vp, i]
            L.afm_profile_read.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_int)]
            L.afm_forward_batch.argtypes = [vp, C.POINTER(Problem), vp, i, vp, vp, vp, vp]
            L.afm_forward_batch_f64.argtypes = [vp, C.POINTER(Problem), vp, i, vp, vp, vp, vp]
            L.afm_misfit.argtypes = [vp, vp, vp, i, i, vp, vp]
            L.afm_pso_init.argtypes = [vp, C.POINTER(PsoCfg), C.POINTER(Swarm), vp]
            L.afm_pso_step.argtypes = [vp, C.POINTER(PsoCfg), C.POINTER(Swarm), vp, u32, vp]
            L.afm_pso_init_slice.argtypes = [vp, C.POINTER(PsoCfg), i, C.POINTER(Swarm), vp]
            L.afm_pso_best_slice.argtypes = [vp, C.POINTER(PsoCfg), i, C.POINTER(Swarm), vp, u32,
                                             vp]
            L.afm_pso_move_slice.argtypes = [vp, C.POINTER(PsoCfg), i, C.POINTER(Swarm), vp, u32,
                                             vp]
            L.afm_invert_workspace_size.argtypes = [C.POINTER(Problem), C.POINTER(PsoCfg),
                                                    C.POINTER(C.c_size_t)]
            L.afm_invert.argtypes = [vp, C.POINTER(Problem), vp, C.POINTER(PsoCfg), vp,
                                     C.c_size_t, vp, vp, vp]
            L.afm_adjoint_workspace_size.argtypes = [C.POINTER(Problem), i, C.POINTER(C.c_size_t)]
            L.afm_adjoint.argtypes = [vp, C.POINTER(Problem), vp, i, vp, vp, vp, vp, C.c_size_t, vp]
            L.afm_normal_equations.argtypes = [vp, C.POINTER(Problem), vp, i, vp, vp, vp, vp, vp]
            L.afm_polish_workspace_size.argtypes = [C.POINTER(Problem), i, i, i,
                                                    C.POINTER(C.c_size_t)]
            L.afm_polish.argtypes = [vp, C.POINTER(Problem), vp, vp, vp, i, i, i, i, vp, C.c_size_t,
                                     vp]
            L.afm_invert_polished_workspace_size.argtypes = [C.POINTER(Problem), C.POINTER(PsoCfg),
                                                             i, i, i, C.POINTER(C.c_size_t)]
            L.afm_invert_polished.argtypes = [vp, C.POINTER(Problem), vp, C.POINTER(PsoCfg), i, i,
                                              i, i, vp, C.c_size_t, vp, vp, vp]
            L.afm_invert_batch_workspace_size.argtypes = [C.POINTER(Problem), i, i,
                                                          C.POINTER(C.c_size_t)]
            L.afm_invert_batch.argtypes = [vp, C.POINTER(Problem), i, vp, vp, i, u32,
                                           C.POINTER(PsoCfg), vp, C.c_size_t, vp,
                                           C.POINTER(C.c_int), vp]
            L.afm_invert_batch_polished_workspace_size.argtypes = [
                C.POINTER(Problem), i, C.POINTER(PsoCfg), i, i, i, i, C.POINTER(C.c_size_t)]
            L.afm_invert_batch_polished.argtypes = [vp, C.POINTER(Problem), i, vp, vp, i, u32,
                                                    C.POINTER(PsoCfg), i, i, i, i,
                                                    C.POINTER(BatchSelect), vp, C.c_size_t,
                                                    vp, C.POINTER(C.c_int), vp]
            L.afm_invert_image_workspace_size.argtypes = [C.POINTER(Problem), C.POINTER(ImageCfg),
                                                          C.POINTER(C.c_size_t)]
            L.afm_invert_image.argtypes = [vp, C.POINTER(Problem), vp, vp, u32, C.POINTER(ImageCfg),
                                           vp, C.c_size_t, vp, vp]
            L.afm_invert_noalloc.argtypes = [vp, C.POINTER(Problem), vp, C.POINTER(PsoCfg), vp,
                                             vp, vp]
            L.afm_synth_records.argtypes = [vp, C.POINTER(Problem), vp, i, vp, i, d, u64, u32,
                                            vp, vp]
            _lib = L
    return _lib


def _check(st: int):
    if st != OK:
        raise AfmError(st, lib().afm_last_error().decode())


def context(device: int | None = None):
    import torch
    dev = torch.cuda.current_device() if device is None else int(device)
    with _lock:
        c = _ctx.get(dev)
    if c is None:
        h = C.c_void_p()
        _check(lib().afm_ctx_create(dev, C.byref(h)))
        with _lock:
            _ctx[dev] = h
        c = h
    return c


def profile_enable(on: bool = True, device=None) -> None:
    """Bracket the hot kernels with CUDA events (see afm_profile_enable)."""
    _check(lib().afm_profile_enable(context(device), int(bool(on))))


LANES = {"auto": 0, "one": 1, "stages": 2, "modes2": 3, "modes4": 4, "modes3": 5}


def set_lanes(lanes: str = "auto", device=None) -> None:
    """Lanes per particle of the fused inversion iteration (see afm_set_lanes):
    'auto', 'one', 'stages', 'modes2', 'modes3' or 'modes4'; all are
    bit-identical."""
    _check(lib().afm_set_lanes(context(device), LANES[lanes]))


def profile_read(device=None):
    """(summed device ms, launches) of the timed kernels since the last read."""
    ms, n = C.c_double(), C.c_int()
    _check(lib().afm_profile_read(context(device), C.byref(ms), C.byref(n)))
    return ms.value, n.value


def _stream(stream=None):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


# --------------------------------------------------------------------------
# Problem / swarm descriptors from workload dicts (SI)
# --------------------------------------------------------------------------
def make_problem(spec: dict, n_steps: int | None = None) -> Problem:
    p = Problem()
    p.model = _MODEL[spec["model"]]
    p.n_modes = int(spec.get("n_modes", 1))
    p.f1_hz = float(spec["f1_hz"])
    p.k_N_per_m = float(spec["k"])
    q = spec.get("Q", 400.0)
    qs = list(q) if hasattr(q, "__len__") else [q] * MAX_MODES
    for k in range(MAX_MODES):
        p.Q[k] = float(qs[k] if k < len(qs) else qs[-1])
    p.n_elem = int(spec.get("n_elem", 0))
    p.L_m = float(spec.get("L", 0.0))
    p.E_Pa = float(spec.get("E", 0.0))
    p.rho_kg_m3 = float(spec.get("rho", 0.0))
    p.newmark_beta = float(spec.get("newmark_beta", 0.25))
    p.A0_m = float(spec["A0"])
    p.Zc_m = float(spec["Zc"])
    p.steps_per_cycle = int(spec.get("spc", 0))
    if n_steps is None:
        n_steps = int(spec["n_steps"]) if "n_steps" in spec else int(spec["cycles"]) * int(spec["spc"])
    p.n_steps = int(n_steps)
    p.force = _FORCE[spec["force"]]
    for s in range(MAX_PARAMS):
        p.fixed[s] = float(spec["fixed"][s])
    free = spec["free"]
    p.n_free = len(free)
    for dd, (slot, lo, hi, lg) in enumerate(free):
        p.slot[dd] = int(slot)
        p.lo[dd] = float(lo)
        p.hi[dd] = float(hi)
        p.log_scale[dd] = int(bool(lg))
    if spec.get("drive") == "chirp":          # base-motion inversion from rest
        p.drive_mode = 1
        p.dt_s = float(spec["dt"])
        p.drive_a_m, p.drive_f_hz, p.drive_g_hz_s = (float(v) for v in spec["drive_params"])
    pts = spec.get("points", ())                # deflection points x / L along the cantilever
    p.n_points = len(pts)
    for k, xi in enumerate(pts):
        p.point_xi[k] = float(xi)
    return p


def n_values(prob: Problem) -> int:
    """Record values per step: the deflection points, else the tip."""
    return max(int(prob.n_points), 1)


def make_pso(spec: dict, pixel: int = 0) -> PsoCfg:
    return PsoCfg(P=int(spec["P"]), iters=int(spec["iters"]), w=float(spec["w"]),
                  c1=float(spec["c1"]), c2=float(spec["c2"]), seed=int(spec["seed"]),
                  pixel=int(pixel))


# --------------------------------------------------------------------------
# Entry points
# --------------------------------------------------------------------------
def forward_batch(prob: Problem, x, U=None, want_defl: bool = True, want_S: bool = True,
                  stream=None):
    """FP for P candidates.  x: float32 CUDA tensor [D, P].  Returns (defl, S):
    defl [n_steps, P] or None, S [P] or None (needs U [n_steps])."""
    import torch
    P = int(x.shape[1]) if x.dim() == 2 else int(x.shape[0])
    dev = x.device
    defl = torch.empty((prob.n_steps * n_values(prob), P), dtype=torch.float32, device=dev) \
        if want_defl else None
    S = torch.empty(P, dtype=torch.float32, device=dev) if (want_S and U is not None) else None
    _check(lib().afm_forward_batch(context(dev.index), C.byref(prob), _ptr(x), P, _ptr(defl),
                                   _ptr(U), _ptr(S), _stream(stream)))
    return defl, S


def forward_batch_f64(prob: Problem, x, U=None, want_defl: bool = True, want_S: bool = True,
                      stream=None):
    import torch
    P = int(x.shape[1]) if x.dim() == 2 else int(x.shape[0])
    dev = x.device
    defl = torch.empty((prob.n_steps * n_values(prob), P), dtype=torch.float64, device=dev) \
        if want_defl else None
    S = torch.empty(P, dtype=torch.float64, device=dev) if (want_S and U is not None) else None
    _check(lib().afm_forward_batch_f64(context(dev.index), C.byref(prob), _ptr(x), P, _ptr(defl),
                                       _ptr(U), _ptr(S), _stream(stream)))
    return defl, S


def misfit(defl, U, stream=None):
    import torch
    N, P = int(defl.shape[0]), int(defl.shape[1])
    S = torch.empty(P, dtype=torch.float32, device=defl.device)
    _check(lib().afm_misfit(context(defl.device.index), _ptr(defl), _ptr(U), N, P, _ptr(S),
                            _stream(stream)))
    return S


@dataclass
class SwarmState:
    x: object
    v: object
    pbest_x: object
    pbest_S: object
    gbest: object

    def c_struct(self) -> Swarm:
        D, P = self.x.shape
        return Swarm(P=P, D=D, x=self.x.data_ptr(), v=self.v.data_ptr(),
                     pbest_x=self.pbest_x.data_ptr(), pbest_S=self.pbest_S.data_ptr(),
                     gbest=self.gbest.data_ptr())


def pso_init(cfg: PsoCfg, D: int, device=None, stream=None) -> SwarmState:
    import torch
    dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
    P = cfg.P
    sw = SwarmState(x=torch.empty((D, P), dtype=torch.float32, device=dev),
                    v=torch.empty((D, P), dtype=torch.float32, device=dev),
                    pbest_x=torch.empty((D, P), dtype=torch.float32, device=dev),
                    pbest_S=torch.empty(P, dtype=torch.float32, device=dev),
                    gbest=torch.empty(1, dtype=torch.int64, device=dev))
    cs = sw.c_struct()
    _check(lib().afm_pso_init(context(dev.index), C.byref(cfg), C.byref(cs), _stream(stream)))
    return sw


def pso_step(cfg: PsoCfg, sw: SwarmState, S_new, it: int, stream=None) -> None:
    cs = sw.c_struct()
    _check(lib().afm_pso_step(context(sw.x.device.index), C.byref(cfg), C.byref(cs),
                              _ptr(S_new), int(it), _stream(stream)))


def pso_init_slice(cfg: PsoCfg, p0: int, n: int, D: int, device=None, stream=None) -> SwarmState:
    """Particles p0 .. p0 + n - 1 of a swarm of cfg.P split across processes
    (afm_pso_init_slice)."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
    sw = SwarmState(x=torch.empty((D, n), dtype=torch.float32, device=dev),
                    v=torch.empty((D, n), dtype=torch.float32, device=dev),
                    pbest_x=torch.empty((D, n), dtype=torch.float32, device=dev),
                    pbest_S=torch.empty(n, dtype=torch.float32, device=dev),
                    gbest=torch.empty(1, dtype=torch.int64, device=dev))
    cs = sw.c_struct()
    _check(lib().afm_pso_init_slice(context(dev.index), C.byref(cfg), int(p0), C.byref(cs),
                                    _stream(stream)))
    return sw


def pso_best_slice(cfg: PsoCfg, p0: int, sw: SwarmState, S_new, it: int, stream=None) -> None:
    """Personal bests of the slice and its best key in sw.gbest."""
    cs = sw.c_struct()
    _check(lib().afm_pso_best_slice(context(sw.x.device.index), C.byref(cfg), int(p0), C.byref(cs),
                                    _ptr(S_new), int(it), _stream(stream)))


def pso_move_slice(cfg: PsoCfg, p0: int, sw: SwarmState, gbest_x, it: int, stream=None) -> None:
    """Eq. 8 move of the slice for generation it + 1 with the swarm's global
    best position gbest_x (float32 CUDA [D])."""
    cs = sw.c_struct()
    _check(lib().afm_pso_move_slice(context(sw.x.device.index), C.byref(cfg), int(p0), C.byref(cs),
                                    _ptr(gbest_x), int(it), _stream(stream)))


def invert_workspace_size(prob: Problem, cfg: PsoCfg) -> int:
    n = C.c_size_t()
    _check(lib().afm_invert_workspace_size(C.byref(prob), C.byref(cfg), C.byref(n)))
    return int(n.value)


def result_dtype_size() -> int:
    return C.sizeof(Result)


def invert(prob: Problem, U, cfg: PsoCfg, workspace=None, result=None, history=None,
           stream=None):
    """IP: one fused inversion on the GPU.  U: float32 CUDA tensor [n_steps].
    Returns (result_tensor_uint8, history) left on the device; decode the
    result with ``decode_result``."""
    import torch
    dev = U.device
    nbytes = invert_workspace_size(prob, cfg)
    if workspace is None or workspace.numel() < nbytes:
        workspace = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    if result is None:
        result = torch.zeros(C.sizeof(Result), dtype=torch.uint8, device=dev)
    if history is None:
        history = torch.empty(cfg.iters + 1, dtype=torch.float32, device=dev)
    _check(lib().afm_invert(context(dev.index), C.byref(prob), _ptr(U), C.byref(cfg),
                            _ptr(workspace), C.c_size_t(workspace.numel()), _ptr(result),
                            _ptr(history), _stream(stream)))
    return result, history


def adjoint_workspace_size(prob: Problem, P: int) -> int:
    n = C.c_size_t()
    _check(lib().afm_adjoint_workspace_size(C.byref(prob), int(P), C.byref(n)))
    return int(n.value)


def adjoint(prob: Problem, x, U, workspace=None, stream=None):
    """Misfit S [P] and its gradient dS/dx [D, P] for x float32 CUDA [D, P]
    (discrete adjoint of the FP32 RK4 + compensated misfit)."""
    import torch
    D, P = int(x.shape[0]), int(x.shape[1])
    dev = x.device
    nbytes = adjoint_workspace_size(prob, P)
    if workspace is None or workspace.numel() < nbytes:
        workspace = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    S = torch.empty(P, dtype=torch.float32, device=dev)
    G = torch.empty((D, P), dtype=torch.float32, device=dev)
    _check(lib().afm_adjoint(context(dev.index), C.byref(prob), _ptr(x), P, _ptr(U), _ptr(S),
                             _ptr(G), _ptr(workspace), C.c_size_t(workspace.numel()),
                             _stream(stream)))
    return S, G


def _misfit_function():
    import torch

    class Misfit(torch.autograd.Function):
        """S(x) with the adjoint gradient: forward runs afm_adjoint (misfit and
        gradient in one pass), backward scales the stored gradient."""

        @staticmethod
        def forward(ctx, x, prob, U):
            S, G = adjoint(prob, x.detach().contiguous(), U)
            ctx.save_for_backward(G)
            return S

        @staticmethod
        def backward(ctx, gS):
            (G,) = ctx.saved_tensors
            return G * gS.unsqueeze(0), None, None

    return Misfit


_MISFIT = None


def misfit_autograd(prob: Problem, x, U):
    """Differentiable misfit S(x) [P] for x [D, P] (torch.autograd)."""
    global _MISFIT
    if _MISFIT is None:
        _MISFIT = _misfit_function()
    return _MISFIT.apply(x, prob, U)


POLISH_STEEPEST, POLISH_LM = 0, 1
_METHOD = {"steepest": POLISH_STEEPEST, "lm": POLISH_LM}


def _method(m) -> int:
    return _METHOD[m] if isinstance(m, str) else int(m)


def normal_equations(prob: Problem, x, U, stream=None):
    """Misfit S [P] and its normal equations H [P, D, D], b [P, D] (FP64) from
    the tangent-linear sensitivities, for x float32 CUDA [D, P]."""
    import torch
    D, P = int(x.shape[0]), int(x.shape[1])
    S = torch.empty(P, dtype=torch.float32, device=x.device)
    H = torch.empty((P, D, D), dtype=torch.float64, device=x.device)
    b = torch.empty((P, D), dtype=torch.float64, device=x.device)
    _check(lib().afm_normal_equations(context(x.device.index), C.byref(prob), _ptr(x), P, _ptr(U),
                                      _ptr(S), _ptr(H), _ptr(b), _stream(stream)))
    return S, H, b


def polish_workspace_size(prob: Problem, K: int, n_cand: int = 16, method="steepest") -> int:
    n = C.c_size_t()
    _check(lib().afm_polish_workspace_size(C.byref(prob), int(K), int(n_cand), _method(method),
                                           C.byref(n)))
    return int(n.value)


def invert_polished_workspace_size(prob: Problem, cfg: PsoCfg, polish_k: int = 32,
                                   n_cand: int = 16, method="steepest") -> int:
    n = C.c_size_t()
    _check(lib().afm_invert_polished_workspace_size(C.byref(prob), C.byref(cfg), int(polish_k),
                                                    int(n_cand), _method(method), C.byref(n)))
    return int(n.value)


def polish(prob: Problem, U, x, steps: int, n_cand: int = 16, method="steepest", stream=None):
    """Projected-gradient polish of candidates x float32 CUDA [D, K] (in
    place); returns their misfits S [K]."""
    import torch
    D, K = int(x.shape[0]), int(x.shape[1])
    n = C.c_size_t()
    _check(lib().afm_polish_workspace_size(C.byref(prob), K, int(n_cand), _method(method),
                                           C.byref(n)))
    ws = torch.empty(int(n.value), dtype=torch.uint8, device=x.device)
    S = torch.empty(K, dtype=torch.float32, device=x.device)
    _check(lib().afm_polish(context(x.device.index), C.byref(prob), _ptr(U), _ptr(x), _ptr(S), K,
                            int(steps), int(n_cand), _method(method), _ptr(ws),
                            C.c_size_t(ws.numel()),
                            _stream(stream)))
    return S


def invert_polished(prob: Problem, U, cfg: PsoCfg, polish_k: int = 32, polish_steps: int = 20,
                    n_cand: int = 16, workspace=None, result=None, history=None, stream=None,
                    method="steepest"):
    """PSO (cfg) then gradient polish of the best polish_k particles; returns
    (result uint8 tensor, history)."""
    import torch
    dev = U.device
    n = C.c_size_t()
    _check(lib().afm_invert_polished_workspace_size(C.byref(prob), C.byref(cfg), int(polish_k),
                                                    int(n_cand), _method(method), C.byref(n)))
    if workspace is None or workspace.numel() < n.value:
        workspace = torch.empty(int(n.value), dtype=torch.uint8, device=dev)
    if result is None:
        result = torch.zeros(C.sizeof(Result), dtype=torch.uint8, device=dev)
    if history is None:
        history = torch.empty(cfg.iters + 1, dtype=torch.float32, device=dev)
    _check(lib().afm_invert_polished(context(dev.index), C.byref(prob), _ptr(U), C.byref(cfg),
                                     int(polish_k), int(polish_steps), int(n_cand),
                                     _method(method), _ptr(workspace),
                                     C.c_size_t(workspace.numel()), _ptr(result),
                                     _ptr(history), _stream(stream)))
    return result, history


def _problems(prob):
    """(pointer to the first of an afm_problem array, count) for one Problem
    (shared by every pixel) or a sequence of them (one per pixel)."""
    if isinstance(prob, Problem):
        return C.byref(prob), 1
    arr = (Problem * len(prob))(*prob)
    return arr, len(prob)


def invert_batch_workspace_size(prob, n_pix: int) -> int:
    n = C.c_size_t()
    pp, n_prob = _problems(prob)
    _check(lib().afm_invert_batch_workspace_size(pp, n_prob, int(n_pix), C.byref(n)))
    return int(n.value)


def invert_batch(prob, U_cat, off, cfg: PsoCfg, pixel0: int = 0,
                 particles_per_thread: int = 0, workspace=None, results=None, stream=None):
    """Many pixel inversions in one graph launch.  prob: one Problem for all
    pixels or a sequence of n_pix (one per pixel).  U_cat float32 CUDA [sum
    n_i], off int64 CUDA [n_pix + 1].  Returns (results uint8 [n_pix,
    sizeof(afm_result)], particles per thread used)."""
    import torch
    dev = U_cat.device
    n_pix = int(off.shape[0]) - 1
    nbytes = invert_batch_workspace_size(prob, n_pix)
    if workspace is None or workspace.numel() < nbytes:
        workspace = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    if results is None:
        results = torch.zeros((n_pix, C.sizeof(Result)), dtype=torch.uint8, device=dev)
    kp = C.c_int(int(particles_per_thread))
    pp, n_prob = _problems(prob)
    _check(lib().afm_invert_batch(context(dev.index), pp, n_prob, _ptr(U_cat), _ptr(off), n_pix,
                                  int(pixel0), C.byref(cfg), _ptr(workspace),
                                  C.c_size_t(workspace.numel()), _ptr(results), C.byref(kp),
                                  _stream(stream)))
    return results, kp.value


def invert_batch_polished_workspace_size(prob, cfg: PsoCfg, n_pix: int, polish_k: int,
                                         n_cand: int = 16, method="steepest") -> int:
    n = C.c_size_t()
    pp, n_prob = _problems(prob)
    _check(lib().afm_invert_batch_polished_workspace_size(pp, n_prob, C.byref(cfg), int(n_pix),
                                                          int(polish_k), int(n_cand),
                                                          _method(method), C.byref(n)))
    return int(n.value)


def invert_batch_polished(prob, U_cat, off, cfg: PsoCfg, polish_k: int, polish_steps: int,
                          n_cand: int = 16, pixel0: int = 0, particles_per_thread: int = 0,
                          workspace=None, results=None, stream=None, method="steepest",
                          pixels=None, box_lo=None, box_hi=None, seeds=None):
    """Many pixel inversions, each followed by the gradient polish of its
    polish_k best particles (afm_invert_batch_polished).  prob: one Problem
    or one per pixel (as invert_batch); n_steps must bound the record
    lengths.  Optional selection and prior (CUDA tensors):
    pixels int32 [n_run], box_lo / box_hi float32 [n_run, D], seeds float32
    [n_run, n_seed, D].  Returns (results, particles per thread used)."""
    import torch
    dev = U_cat.device
    n_pix = int(off.shape[0]) - 1
    sel = None
    if pixels is not None:
        # row-major device arrays, as the C API reads them
        pixels = pixels.to(torch.int32).contiguous()
        box_lo = None if box_lo is None else box_lo.to(torch.float32).contiguous()
        box_hi = None if box_hi is None else box_hi.to(torch.float32).contiguous()
        seeds = None if seeds is None else seeds.to(torch.float32).contiguous()
        sel = BatchSelect(pixels=C.c_void_p(pixels.data_ptr()), n_run=int(pixels.numel()),
                          box_lo=_ptr(box_lo), box_hi=_ptr(box_hi), seeds=_ptr(seeds),
                          n_seed=0 if seeds is None else int(seeds.shape[1]))
    n_run = n_pix if sel is None else sel.n_run
    nbytes = invert_batch_polished_workspace_size(prob, cfg, n_run, polish_k, n_cand, method)
    if workspace is None or workspace.numel() < nbytes:
        workspace = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    if results is None:
        results = torch.zeros((n_pix, C.sizeof(Result)), dtype=torch.uint8, device=dev)
    kp = C.c_int(int(particles_per_thread))
    pp, n_prob = _problems(prob)
    _check(lib().afm_invert_batch_polished(context(dev.index), pp, n_prob, _ptr(U_cat), _ptr(off),
                                           n_pix, int(pixel0), C.byref(cfg), int(polish_k),
                                           int(polish_steps), int(n_cand), _method(method),
                                           None if sel is None else C.byref(sel), _ptr(workspace),
                                           C.c_size_t(workspace.numel()), _ptr(results),
                                           C.byref(kp), _stream(stream)))
    return results, kp.value


def make_image_cfg(width: int, height: int, stride: int, margin: float, coarse: PsoCfg,
                   fine: PsoCfg, coarse_polish=(8, 12), fine_polish=(4, 6), n_cand: int = 8,
                   method="lm") -> ImageCfg:
    return ImageCfg(width=int(width), height=int(height), stride=int(stride), margin=float(margin),
                    coarse=coarse, fine=fine, coarse_polish_k=int(coarse_polish[0]),
                    coarse_polish_steps=int(coarse_polish[1]), fine_polish_k=int(fine_polish[0]),
                    fine_polish_steps=int(fine_polish[1]), n_cand=int(n_cand),
                    method=_method(method))


def invert_image_workspace_size(prob: Problem, icfg: ImageCfg) -> int:
    n = C.c_size_t()
    _check(lib().afm_invert_image_workspace_size(C.byref(prob), C.byref(icfg), C.byref(n)))
    return int(n.value)


def invert_image(prob: Problem, U_cat, off, icfg: ImageCfg, pixel0: int = 0, workspace=None,
                 results=None, stream=None):
    """Image scan with cross-pixel warm start (afm_invert_image); returns the
    results [width * height, sizeof(afm_result)] (uint8, device)."""
    import torch
    dev = U_cat.device
    nbytes = invert_image_workspace_size(prob, icfg)
    if workspace is None or workspace.numel() < nbytes:
        workspace = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    if results is None:
        results = torch.zeros((icfg.width * icfg.height, C.sizeof(Result)), dtype=torch.uint8,
                              device=dev)
    _check(lib().afm_invert_image(context(dev.index), C.byref(prob), _ptr(U_cat), _ptr(off),
                                  int(pixel0), C.byref(icfg), _ptr(workspace),
                                  C.c_size_t(workspace.numel()), _ptr(results), _stream(stream)))
    return results


def decode_results(results) -> list:
    """Host copies of an [n_pix] array of afm_result (uint8 tensor)."""
    raw = results.cpu().numpy().reshape(-1, C.sizeof(Result))
    return [decode_result(bytes(r.tobytes())) for r in raw]


def invert_noalloc(prob: Problem, U, cfg: PsoCfg, result, history=None, stream=None):
    """IP without a workspace: the swarm state lives in the library's fixed
    device scratch (see afm_invert_noalloc), so this call allocates nothing.
    The caller provides `result` (uint8 CUDA tensor of sizeof(afm_result)
    bytes) and optionally `history` (float32 [iters + 1])."""
    _check(lib().afm_invert_noalloc(context(U.device.index), C.byref(prob), _ptr(U), C.byref(cfg),
                                    _ptr(result), _ptr(history), _stream(stream)))
    return result, history


def decode_result(result_bytes) -> dict:
    """Host copy of an afm_result (uint8 tensor or bytes) as a dict."""
    raw = bytes(result_bytes.cpu().numpy().tobytes()) if hasattr(result_bytes, "cpu") else bytes(result_bytes)
    r = Result.from_buffer_copy(raw[:C.sizeof(Result)])
    return dict(x=np.array(r.x[:]), theta=np.array(r.theta[:]), S=r.S, S_f64=r.S_f64,
                J_rel=r.J_rel, iters=r.iters, winner=r.winner, nonfinite=r.nonfinite,
                status=r.status, defect=r.defect, segments=r.segments, drive=np.array(r.drive[:]))


def synth_records(prob: Problem, x_truth, off, sub: int, sigma_m: float, seed: int,
                  pixel0: int = 0, stream=None):
    """Synthetic records (FP32 at dt/sub, sampled every sub steps, plus
    Philox/Box-Muller noise).  x_truth: float64 CUDA [D, n_pix]; off: int64
    CUDA [n_pix + 1].  Returns U_cat float32 [off[-1]]."""
    import torch
    n_pix = int(off.shape[0]) - 1
    total = int(off[-1].item())
    U = torch.empty(total, dtype=torch.float32, device=off.device)
    _check(lib().afm_synth_records(context(off.device.index), C.byref(prob), _ptr(x_truth),
                                   n_pix, _ptr(off), int(sub), float(sigma_m), int(seed),
                                   int(pixel0), _ptr(U), _stream(stream)))
    return U
