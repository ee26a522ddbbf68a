#!/usr/bin/env python
"""Benchmark of the fused inversion hot path on GB300.

One step = one batched inversion of 4096 independent pixels (each its own
seeded truth and record of 20..200 cycles x 256 steps of the 3-mode
Euler-Bernoulli cantilever with the DMT law; 256 particles x (60 + 1)
evaluations of the fused forward + misfit + swarm update per pixel; every
winner re-evaluated in FP64), as one persistent CUDA-graph launch of
afm_invert_batch on records made on the GPU.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0): particle-timesteps/s of the whole job, the
swarm kernel's roofline, the end-to-end rate through the C ABI with host
buffers, the accuracy of the winners against the oracle's stored optima,
the LM-polished batch (ms per pixel at that accuracy), the FP64 oracle on
the host cores, and the other workloads as extra keys.  Under torchrun each
rank inverts its own share of a (N x 4096)-pixel image (independent
problems: weak scaling, no data-path collective); the timing is the
maximum over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import glob
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle·timesteps/s forward+misfit; ms per inversion at ≤0.5% param error"
UNIT = "particle·timesteps/s"
PROBE_WORKLOAD = "c2"      # default workload of the --probe captures


# ---------------------------------------------------------------------------
# FP32 operation count of the fused kernel per particle and RK4 step
# ---------------------------------------------------------------------------
def fp32_ops_per_step(m: int, force: str) -> int:
    """FP32 instructions (add/mul/fma/min/max) per particle per RK4 step of
    the fused forward + misfit kernel, counted from its source:
    accel(): tip sum (m-1), gap (1), force law, per mode 4 (+1 for mode 1's
    low word); RK4 stage states and slope sums 12m; state update 8 for the
    lowest mode (compensated) and 2 for each other mode (plain sums);
    tip deflection (m-1); compensated misfit 5."""
    force_ops = {"dmt": 7, "dmt_kv": 9 + (m - 1), "linear_spring": 2, "hooke": 3,
                 "spring_damper": 4 + (m - 1)}[force]
    accel = (m - 1) + 1 + force_ops + 4 * m + 1
    return 4 * accel + 12 * m + 8 + 2 * (m - 1) + (m - 1) + 5


def algo_ops_per_step(m: int) -> int:
    """The method's FP32 lane-operations per particle and RK4 step (the
    roofline's numerator): 4 RK4 stages x [(m - 1) adds for the tip
    deflection, 1 for the gap, ~5 for the DMT law with one hardware
    reciprocal square root, 4m for the modal accelerations of Eq. 2, 2m
    stage-state and 2m slope-accumulation FMAs] plus the misfit of Eq. 5
    with its compensated sum: 36m + 24 (132 for 3 modes, 60 for 1).  The
    library issues more (fp32_ops_per_step: the resonant mode's compensated
    state update and low word are precision devices of this implementation,
    not work of the method), so a fraction on this count is the
    conservative one."""
    return 36 * m + 24


def fe_algo_ops_per_step(n: int = 64) -> int:
    """The method's FP32 operations per particle and Newmark step of the FE
    cantilever run in its modal basis (the roofline's numerator), with each
    mode carried scaled by its tip displacement (w = phi(tip) z): per mode
    delta + increment = (1 + d2) delta + b1 w + g G + f Fo (1 mul + 3 fma),
    the predicted coordinate w + that sum and its term of the tip sum (2
    adds), the update delta' = that sum + f F (1 fma) and w' = w + delta' (1
    add): 8; per particle Fo = 2 F_n + F_{n-1} (1), one Newton step of the DMT
    law with the final force evaluation (2 x 8 for gap and law, 4 for residual
    and update), the tip deflection (1) and the compensated misfit (5): 27.
    539 for 64 modes.  The kernel issues more (fe_fp32_ops_per_step): the
    increment form with compensated updates for the lowest modes and the
    group's redundant Newton solve and tip sum."""
    return 8 * n + 27


def fe_fp32_ops_per_step() -> int:
    """FP32 add/mul/fma instructions per particle per step of the FP32 FE
    kernel (DMT law, 64 modes on 8 lanes of 8 mode slots), counted from its
    source.  Per lane: the force history term 1; slot 0 (compensated): the
    increment 5 (drive and past-force terms 2, state terms 2, b1's low word
    1), the predicted coordinate 3, the update 1 + 8 (two Kahan sums); slots
    1-7: delta + increment 4, the predicted coordinate 1, the update 2; the
    lane's tip tree 7 and the group's sum 3; one Newton step 15 (gap 1 + law
    4.5, residual 2, update 2, gap 1 + law 4.5; the law's constant products
    hoisted, contact and free branches 5 and 4).  Lane 0 alone: the tip
    deflection and the compensated misfit 6."""
    slot0 = 5 + 3 + 1 + 8
    slot_plain = 4 + 1 + 2
    per_lane = 1 + slot0 + 7 * slot_plain + 7 + 3 + 15
    return 8 * per_lane + 6


# ---------------------------------------------------------------------------
# nvidia-smi clock sampler (runs during the timed region)
# ---------------------------------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f)
    return {}


# The device code of each kernel: its own source and the device headers.
# (afm_launch.h, the host-side launcher declarations, is left out: adding a
# declaration there does not change a kernel.)
KERNEL_SOURCES = {
    "invert_iter_kernel": ["afm_device.cuh", "afm_internal.h", "kern_invert.cu"],
    "invert_pair_kernel": ["afm_device.cuh", "afm_internal.h", "kern_pair.cu"],
    "invert_modes_kernel": ["afm_device.cuh", "afm_internal.h", "kern_modes.cu"],
    "fwd_kernel": ["afm_device.cuh", "afm_internal.h", "kern_forward.cu"],
    "fwd_x2_kernel": ["afm_device.cuh", "afm_internal.h", "afm_f32x2.cuh", "kern_forward.cu"],
    "batch_kernel": ["afm_device.cuh", "afm_internal.h", "afm_f32x2.cuh", "kern_batch.cuh", "kern_batch.cu",
                     "kern_batch_dmt.cu"],
    "fe_modal_kernel": ["afm_device.cuh", "afm_internal.h", "kern_fe.cu"],
}


def kernel_source_hash(kernel: str) -> str:
    """Hash of the sources a kernel is compiled from (first 16 hex digits)."""
    h = hashlib.sha256()
    for name in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_1109_0334_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str, workload: str):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current kernel sources (profiles/*.md lines 'traffic: <kernel>
    <workload> <bytes> <source-hash>')."""
    want = kernel_source_hash(kernel)
    for f in glob.glob(os.path.join(ROOT, "profiles", "*.md")):
        for line in open(f):
            parts = line.strip().strip("`").split()
            if len(parts) == 5 and parts[0] == "traffic:" and parts[1] == kernel \
                    and parts[2] == workload and parts[4] == want:
                return float(parts[3])
    return None


# ---------------------------------------------------------------------------
# Distributed plumbing
# ---------------------------------------------------------------------------
def dist_setup(backend: str | None = None):
    """Rank, world size and local rank from the torchrun environment; joins the
    process group for N > 1 (NCCL on GPUs, gloo where none is visible)."""
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if backend is None:
        backend = "nccl" if torch.cuda.is_available() else "gloo"
    if world > 1:
        import torch.distributed as dist
        if backend == "nccl":
            torch.cuda.set_device(local)
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:
            dist.init_process_group(backend)
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def all_max(val: float, world: int) -> float:
    """Maximum of a per-rank value over all ranks (the job's wall time is the
    slowest rank's)."""
    if world == 1:
        return val
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([val], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_slice(n: int, rank: int, world: int):
    """Contiguous share [lo, hi) of n independent units (pixels) for a rank;
    the shares partition range(n) and differ in size by at most one."""
    q, r = divmod(n, world)
    lo = rank * q + min(rank, r)
    return lo, lo + q + (1 if rank < r else 0)


def job_rate(units_per_rank: float, steps: int, max_ms: float, world: int) -> float:
    """Whole-job throughput under weak scaling: every rank processes
    units_per_rank per step; the job takes the slowest rank's time."""
    return world * units_per_rank * steps / (max_ms / 1e3)


# ---------------------------------------------------------------------------
# Batched pixel inversions (4096 independent inversions, one graph launch)
# ---------------------------------------------------------------------------
def c3_inputs(A, W, dev, n_pix=None, cycles_div=1, pixel_lo=0, n_total=None):
    """Seeded truths and record lengths (20..200 cycles) of the batched
    workload (an image of n_total pixels, this call's share starting at
    pixel_lo), records made on the GPU (FP32 at dt/4 + noise keyed by the
    global pixel index)."""
    import numpy as np
    import torch
    spec = W.get("c3")
    n_total = spec["n_pix"] if n_total is None else n_total
    cyc_all, xt_all = W.c3_layout(spec, n_total, cycles_div)
    n_pix = n_total - pixel_lo if n_pix is None else n_pix
    cyc = cyc_all[pixel_lo:pixel_lo + n_pix]
    xt = np.ascontiguousarray(xt_all[:, pixel_lo:pixel_lo + n_pix])
    lens = cyc * spec["spc"]
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    prob = A.make_problem(spec, n_steps=int(lens.max()))
    off_d = torch.from_numpy(off).to(dev)
    U = A.synth_records(prob, torch.from_numpy(xt).to(dev), off_d, spec["record_sub"],
                        spec["sigma"], spec["seed"], pixel_lo)
    return spec, prob, U, off_d, int(lens.sum()), xt, lens


def c3_config(spec, world: int = 1) -> dict:
    """The benchmark's workload description, shared by both arms."""
    return {"workload": "c3: 4096 independent pixel inversions in one persistent CUDA-graph "
                        "launch, 3-mode Euler-Bernoulli cantilever, DMT 4 unknowns, records "
                        "20..200 cycles x 256 steps, 256 particles x 60 updates per pixel",
            "pixels": spec["n_pix"], "particles": spec["P"], "updates": spec["iters"],
            "modes": spec["n_modes"], "force": spec["force"], "steps_per_cycle": spec["spc"],
            "cycles": list(spec["cycles"]),
            "per_rank": f"{spec['n_pix']} pixels of a {spec['n_pix'] * world}-pixel image",
            "l2": "inputs larger than L2 (0.46 GB of records) and a 256 MiB write between steps"}


def _theta_of(spec, xn):
    """SI parameter slots (5 force-law slots, then base a, f, g) of
    normalised coordinates xn [D] (truth draws)."""
    th = [0.0] * 8
    for s5, v in enumerate(spec["fixed"]):
        th[s5] = v
    for k, v in enumerate(spec.get("drive_params", (0.0, 0.0, 0.0))):
        th[5 + k] = v
    for d, (slot, lo, hi, lg) in enumerate(spec["free"]):
        th[slot] = 10 ** (math.log10(lo) + xn[d] * (math.log10(hi) - math.log10(lo))) if lg \
            else lo + xn[d] * (hi - lo)
    return th


def _dmt_comb(th):
    """The combinations a DMT record determines: H R, E* sqrt(R), a0."""
    return [th[1] * th[2], th[0] * math.sqrt(th[2]), th[3]]


def _comb_err(a, b):
    return max(abs(x / y - 1) for x, y in zip(_dmt_comb(a), _dmt_comb(b)))


GOLDEN_C3 = os.path.join(ROOT, "tests", "golden", "c3_subset_optima.json")
GOLDEN_C2 = os.path.join(ROOT, "tests", "golden", "c2_invert.json")


def _dchi2_and_comb(A, spec, prob_n, U_pix, r, x_ref):
    """Delta chi^2 of result r against the stored optimum x_ref, both on the
    same record (the optimum's FP64 misfit computed by the library's FP64
    forward on that record), and the relative differences of H R, E* sqrt(R)
    and a0."""
    import torch
    D = len(spec["free"])
    xo = torch.tensor(x_ref, dtype=torch.float64, device=U_pix.device).reshape(D, 1)
    _, S_ref = A.forward_batch_f64(prob_n, xo, U_pix.double(), want_defl=False)
    S_ref = float(S_ref.item())
    var = (spec["sigma"] / 1e-9) ** 2
    ca, cb = _dmt_comb(list(r["theta"])), _dmt_comb(_theta_of(spec, x_ref))
    return (r["S_f64"] - S_ref) / var, [abs(a / b - 1) for a, b in zip(ca, cb)], S_ref


def determined_error(A, spec, prob_n, U_pix, x_ref, x_test, rel=0.005):
    """Relative parameter error of x_test against x_ref along the directions
    the record determines: the misfit's Gauss-Newton Hessian at x_ref (the
    library's tangent-linear normal equations), in log-parameter coordinates,
    has eigen-directions of one-sigma half-width sqrt(2 sigma^2 / lambda)
    for noise sigma; over those of half-width <= rel, the largest projection
    of the log-parameter difference.  Returns (error, number of such
    directions)."""
    import numpy as np
    import torch
    D = len(spec["free"])
    xo = torch.tensor(x_ref, dtype=torch.float32, device=U_pix.device).reshape(D, 1)
    _, H, _ = A.normal_equations(prob_n, xo, U_pix.contiguous())
    Hs = 2.0 * H[0].cpu().numpy()                        # Hessian of S [nm^2]
    th_r, th_t = _theta_of(spec, x_ref), _theta_of(spec, x_test)
    J, drho = np.empty(D), np.empty(D)
    for d, (slot, lo, hi, lg) in enumerate(spec["free"]):
        J[d] = math.log(10.0) * (math.log10(hi) - math.log10(lo)) if lg else (hi - lo) / th_r[slot]
        drho[d] = math.log(th_t[slot] / th_r[slot])
    lam, V = np.linalg.eigh(Hs / np.outer(J, J))
    widths = np.sqrt(2 * (spec["sigma"] / 1e-9) ** 2 / np.maximum(lam, 1e-300))
    ident = widths <= rel
    proj = np.abs(V.T @ drho)
    return (float(proj[ident].max()) if ident.any() else 0.0), int(ident.sum())


def accuracy_vs_oracle(A, spec, U, off, results, golden=GOLDEN_C3):
    """Each result of the first pixels against the oracle's stored optimum of
    the same pixel (tests/golden/c3_subset_optima.json, written by the
    oracle alone on records with the same truths, lengths and noise):
    delta chi^2 = (S - S_opt) / sigma^2 on this record (<= 1: statistically
    at the optimum), the parameter error along the directions the record
    determines to 0.5 % (determined_error), and, for information, the
    combinations H R, E* sqrt(R), a0 (only some of which a record
    determines) against the optimum's.  A point more than one noise variance
    below the stored optimum counts as meeting the parameter criterion (it is
    a better optimum than the stored one)."""
    import numpy as np
    with open(golden) as f:
        gold = json.load(f)
    off_h = off.cpu().numpy()
    rows = []
    for g in gold["pixels"]:
        i = g["pixel"]
        n = int(off_h[i + 1] - off_h[i])
        assert n == g["cycles"] * spec["spc"], "golden subset and bench records differ"
        prob_n = A.make_problem(spec, n_steps=n)
        U_pix = U[int(off_h[i]):int(off_h[i + 1])]
        d, comb, _ = _dchi2_and_comb(A, spec, prob_n, U_pix, results[i], g["x"])
        e, n_id = determined_error(A, spec, prob_n, U_pix, g["x"], list(results[i]["x"][:len(g["x"])]))
        rows.append((d, comb, e, n_id))
    dchi = np.array([r[0] for r in rows])
    comb = np.array([r[1] for r in rows])
    err = np.array([r[2] for r in rows])
    # a point more than one noise variance below the stored optimum is a
    # better optimum than the oracle's: the parameter comparison is void there
    ok, ok_p = dchi <= 1.0, (err <= 0.005) | (dchi < -1.0)
    return {"pixels": len(rows),
            "reference": "oracle optimum per pixel (own 256 x 60 swarm, then 12 LM steps from "
                         "its winner and from the seeded truth; the best of the three refined "
                         "to convergence in the box by Marquardt's method), FP64 misfit "
                         "re-evaluated on this run's record",
            "frac_dchi2_le_1": float(ok.mean()),
            "frac_param_err_le_0.5pct_determined": float(ok_p.mean()),
            "frac_meeting_both": float((ok & ok_p).mean()),
            "median_dchi2": float(np.median(dchi)), "max_dchi2": float(dchi.max()),
            "median_determined_directions": float(np.median([r[3] for r in rows])),
            "frac_combinations_within_0.5pct": {
                "H R": float((comb[:, 0] <= 0.005).mean()),
                "E* sqrt(R)": float((comb[:, 1] <= 0.005).mean()),
                "a0": float((comb[:, 2] <= 0.005).mean())}}


def run_c3_per_pixel(A, spec, U, off, flush, shared_ms):
    """The same 4096-pixel batch with one problem per pixel (the set-point
    drifting by up to +-1 nm and the free amplitude by +-5 % across the
    image, as in a real scan): the cost of the per-pixel path, timed over one
    call after an untimed one (timing only: the records are the shared
    problem's)."""
    import numpy as np
    import torch
    n_pix = int(off.shape[0]) - 1
    n_max = int((off[1:] - off[:-1]).max().item())
    k = np.arange(n_pix)
    probs = [A.make_problem(dict(spec, Zc=spec["Zc"] + 1e-9 * np.sin(0.013 * i),
                                 A0=spec["A0"] * (1 + 0.05 * np.cos(0.007 * i))), n_steps=n_max)
             for i in k]
    cfg = A.make_pso(spec)
    ws = torch.empty(A.invert_batch_workspace_size(probs, n_pix), dtype=torch.uint8, device=U.device)
    res = torch.zeros((n_pix, A.result_dtype_size()), dtype=torch.uint8, device=U.device)
    A.invert_batch(probs, U, off, cfg, workspace=ws, results=res)
    torch.cuda.synchronize()
    flush.zero_()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    _, kp = A.invert_batch(probs, U, off, cfg, workspace=ws, results=res)
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    ok = sum(1 for r in A.decode_results(res) if r["status"] == 0)
    return {"config": "the headline batch with one afm_problem per pixel (Zc +-1 nm, A0 +-5 % "
                      "across pixels; constants uploaded from host memory each call)",
            "ms": ms, "ms_per_pixel_inversion": ms / n_pix, "particles_per_thread": kp,
            "pixels_ok": ok, "slowdown_vs_shared_problem": ms / shared_ms}


def run_c3_polished(A, spec, prob, U, off, pixel0, flush, steps=3):
    """The same pixels by a short swarm plus Levenberg-Marquardt polish of
    each pixel's best particles (the configuration that meets the accuracy
    target), timed over `steps` calls after one untimed call."""
    import torch
    lp = spec["lm_polish"]
    cfg = A.make_pso(dict(spec, iters=lp["iters"]))
    n_pix = int(off.shape[0]) - 1
    nbytes = A.invert_batch_polished_workspace_size(prob, cfg, n_pix, lp["polish_k"], lp["n_cand"], "lm")
    ws = torch.empty(nbytes, dtype=torch.uint8, device=U.device)

    def call(results=None):
        return A.invert_batch_polished(prob, U, off, cfg, lp["polish_k"], lp["polish_steps"],
                                       lp["n_cand"], method="lm", workspace=ws, results=results,
                                       pixel0=pixel0)
    res, _ = call()
    torch.cuda.synchronize()
    ms = []
    for _ in range(steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        res, kp = call(res)
        e1.record()
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    return res, float(statistics.median(ms)), kp, {
        "config": f"{spec['P']} particles x {lp['iters']} updates, then {lp['polish_steps']} "
                  f"Levenberg-Marquardt steps on each pixel's best {lp['polish_k']} "
                  f"({lp['n_cand']} damping values per step)", "timed_calls": steps}


# ---------------------------------------------------------------------------
# Gradient-polished inversion against plain PSO (Kelvin-Voigt workload)
# ---------------------------------------------------------------------------
def ident_errors(theta, truth):
    """Relative errors of the combinations the DMT(+KV) law depends on:
    H R, E* sqrt(R), a0, eta sqrt(R)."""
    import math

    def comb(t):
        return [t[1] * t[2], t[0] * math.sqrt(t[2]), t[3], t[4] * math.sqrt(t[2])]
    a, b = comb(theta), comb(truth)
    return [abs(x / y - 1) if y else abs(x) for x, y in zip(a, b)]


def run_c4(A, W, dev, flush):
    import numpy as np
    import torch
    spec = W.get("c4")
    D = len(spec["free"])
    N = W.n_steps(spec)
    rng = np.random.default_rng(spec["seed"])
    xt = rng.uniform(0.1, 0.9, size=(D, 1))
    prob = A.make_problem(spec)
    off = torch.tensor([0, N], dtype=torch.int64, device=dev)
    U = A.synth_records(prob, torch.from_numpy(xt).to(dev), off, spec["record_sub"], spec["sigma"],
                        spec["seed"], 0)
    th_true = [0.0] * 5
    for d, (slot, lo, hi, lg) in enumerate(spec["free"]):
        th_true[slot] = 10 ** (np.log10(lo) + xt[d, 0] * (np.log10(hi) - np.log10(lo))) if lg \
            else lo + xt[d, 0] * (hi - lo)

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        r = fn()
        e1.record()
        e1.synchronize()
        return e0.elapsed_time(e1), A.decode_result(r[0])

    cfg = A.make_pso(spec)
    ms_pol, r_pol = timed(lambda: A.invert_polished(prob, U, cfg, spec["polish_k"],
                                                    spec["polish_steps"]))
    plain = A.make_pso(dict(spec, iters=100))
    ms_pso, r_pso = timed(lambda: A.invert(prob, U, plain))
    lp = spec["lm_polish"]
    cfg_lm = A.make_pso(dict(spec, iters=lp["iters"]))
    ms_lm, r_lm = timed(lambda: A.invert_polished(prob, U, cfg_lm, lp["polish_k"], lp["polish_steps"],
                                                  lp["n_cand"], method="lm"))
    var = (spec["sigma"] / 1e-9) ** 2
    S_best = min(r_pol["S_f64"], r_pso["S_f64"], r_lm["S_f64"])
    return {"workload": "c4: 3-mode DMT + Kelvin-Voigt, 5 unknowns, 100 cycles x 256 steps",
            "lm_polished": {"config": f"1024 particles x {lp['iters']} updates + {lp['polish_steps']} "
                                      f"Levenberg-Marquardt steps on the best {lp['polish_k']} "
                                      f"({lp['n_cand']} damping values per step)",
                            "ms_per_inversion": ms_lm, "S_f64_nm2": r_lm["S_f64"],
                            "dchi2_vs_best": (r_lm["S_f64"] - S_best) / var,
                            "ident_rel_err_vs_truth": ident_errors(list(r_lm["theta"]), th_true)},
            "polished": {"config": "1024 particles x 40 updates + 20 adjoint-gradient polish "
                                   "steps on the best 32 (16 Armijo candidates per step)",
                         "ms_per_inversion": ms_pol, "S_f64_nm2": r_pol["S_f64"],
                         "dchi2_vs_best": (r_pol["S_f64"] - S_best) / var,
                         "ident_rel_err_vs_truth": ident_errors(list(r_pol["theta"]), th_true)},
            "plain_pso": {"config": "1024 particles x 100 updates",
                          "ms_per_inversion": ms_pso, "S_f64_nm2": r_pso["S_f64"],
                          "dchi2_vs_best": (r_pso["S_f64"] - S_best) / var,
                          "ident_rel_err_vs_truth": ident_errors(list(r_pso["theta"]), th_true)},
            "ident": "H R, E* sqrt(R), a0, eta sqrt(R)",
            "records_16": lm_vs_plain(A, W, "c4", U.device, flush)}


def lm_vs_plain(A, W, name, dev, flush, n_rec=16, plain_iters=100):
    """Plain swarm (plain_iters updates) against short swarm + LM polish
    on n_rec seeded records (pixels 0..n_rec-1): median ms per inversion and
    the fraction of records at delta chi^2 <= 1 against the better of the
    two (statistically at the optimum)."""
    import numpy as np
    import torch
    spec = W.get(name)
    D, N = len(spec["free"]), W.n_steps(spec)
    prob = A.make_problem(spec)
    lp = spec["lm_polish"]
    var = (spec["sigma"] / 1e-9) ** 2
    off = torch.tensor([0, N], dtype=torch.int64, device=dev)
    rows = []
    for pix in range(n_rec):
        rng = np.random.default_rng(spec["seed"] + 1000 * pix)
        xt = rng.uniform(0.1, 0.9, size=(D, 1))
        U = A.synth_records(prob, torch.from_numpy(xt).to(dev), off, spec["record_sub"],
                            spec["sigma"], spec["seed"], pix)
        cfg_p = A.make_pso(dict(spec, iters=plain_iters), pixel=pix)
        cfg_l = A.make_pso(dict(spec, iters=lp["iters"]), pixel=pix)
        runs = {"plain_pso": lambda: A.invert(prob, U, cfg_p),
                "lm_polished": lambda: A.invert_polished(prob, U, cfg_l, lp["polish_k"],
                                                         lp["polish_steps"], lp["n_cand"],
                                                         method="lm")}
        row = {}
        for key, fn in runs.items():
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            r = fn()
            e1.record()
            e1.synchronize()
            row[key] = (e0.elapsed_time(e1), A.decode_result(r[0])["S_f64"])
        rows.append(row)
    out = {"records": n_rec, "plain_config": f"{spec['P']} particles x {plain_iters} updates",
           "lm_config": f"{spec['P']} particles x {lp['iters']} updates + {lp['polish_steps']} "
                        f"Levenberg-Marquardt steps on the best {lp['polish_k']} "
                        f"({lp['n_cand']} damping values per step)"}
    for key in ("plain_pso", "lm_polished"):
        d = np.array([(row[key][1] - min(v[1] for v in row.values())) / var for row in rows])
        out[key] = {"median_ms_per_inversion": float(np.median([row[key][0] for row in rows])),
                    "frac_dchi2_le_1": float(np.mean(d <= 1.0)), "max_dchi2": float(d.max())}
    return out


# ---------------------------------------------------------------------------
# Finite-element cantilever inversion (32 Hermite elements, Newmark)
# ---------------------------------------------------------------------------
def run_c5(A, W, dev, peak_ops, flush, iters=None):
    """One full FE inversion (8192 particles x 61 evaluations x 25 600 steps).
    The record is the library's FE forward of a seeded truth at dt/4, sampled
    every 4th step, plus seeded Gaussian noise (input generation only)."""
    import numpy as np
    import torch
    spec = W.get("c5") if iters is None else W.get("c5", iters=iters)
    D = len(spec["free"])
    N = W.n_steps(spec)
    rng = np.random.default_rng(spec["seed"])
    xt = rng.uniform(0.1, 0.9, size=(D, 1)).astype(np.float32)
    fine = A.make_problem(dict(spec, spc=spec["spc"] * 4), n_steps=N * 4)
    defl, _ = A.forward_batch(fine, torch.from_numpy(xt).to(dev), None)
    gen = torch.Generator(device=dev).manual_seed(spec["seed"])
    U = (defl[3::4, 0] + (spec["sigma"] / 1e-9) * torch.randn(N, device=dev, generator=gen)).contiguous()
    prob = A.make_problem(spec)
    cfg = A.make_pso(spec)
    A.invert(prob, U, A.make_pso(dict(spec, iters=1)))     # warm-up
    torch.cuda.synchronize()
    flush.zero_()
    A.profile_enable(True)
    A.profile_read()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    res, _ = A.invert(prob, U, cfg)
    e1.record()
    e1.synchronize()
    kms, kn = A.profile_read()
    A.profile_enable(False)
    ms = e0.elapsed_time(e1)
    r = A.decode_result(res)
    units = spec["P"] * (spec["iters"] + 1) * N
    ops_ps = fe_algo_ops_per_step()
    ach = spec["P"] * N * ops_ps / ((kms / max(kn, 1)) / 1e3)
    return {"workload": "c5: 32-element Hermite FE cantilever, Newmark beta=1/4, DMT 4 unknowns, "
                        "8192 particles x 60 updates, 50 cycles x 512 steps",
            "ms_per_inversion": ms, "value": units / (ms / 1e3), "unit": UNIT,
            "kernel_ms_per_launch": kms / max(kn, 1), "launches": kn,
            "S_f64_nm2": r["S_f64"], "J_rel": r["J_rel"], "status": r["status"],
            "roofline": {"bound": "alu", "achieved": ach / 1e12, "peak": peak_ops / 1e12,
                         "unit": "T FP32 lane-ops/s", "frac": ach / peak_ops,
                         "ops_per_particle_step": ops_ps,
                         "issued_ops_per_particle_step": fe_fp32_ops_per_step(),
                         "kernel": "fe_modal_kernel<float,DMT,invert iteration>",
                         "traffic": ncu_traffic("fe_modal_kernel", "c5"),
                         "note": "modal-basis Newmark kernel (no dense propagator)"}}


# ---------------------------------------------------------------------------
# Image scan with cross-pixel warm start
# ---------------------------------------------------------------------------
def run_image(A, W, dev, flush):
    """64 x 64 image of smoothly varying truths: every pixel cold (short
    swarm + LM polish, the polished-batch configuration) against the two-pass
    warm start (coarse grid cold, the rest inside their neighbours' box);
    accuracy against the better of the two per pixel."""
    import numpy as np
    import torch
    spec = W.get("f1_image")
    Wd, Hd = spec["width"], spec["height"]
    n_pix = Wd * Hd
    D = len(spec["free"])
    N = W.n_steps(spec)
    xt = W.image_truth(D, Wd, Hd, spec["seed"])
    prob = A.make_problem(spec)
    off = torch.arange(0, (n_pix + 1) * N, N, dtype=torch.int64, device=dev)
    U = A.synth_records(prob, torch.from_numpy(xt).to(dev), off, spec["record_sub"], spec["sigma"],
                        spec["seed"], 0)
    coarse = A.make_pso(spec)
    fine = A.make_pso(dict(spec, P=spec["fine"]["P"], iters=spec["fine"]["iters"]))
    icfg = A.make_image_cfg(Wd, Hd, spec["stride"], spec["margin"], coarse, fine,
                            coarse_polish=(spec["polish_k"], spec["polish_steps"]),
                            fine_polish=(spec["fine"]["polish_k"], spec["fine"]["polish_steps"]),
                            n_cand=spec["n_cand"], method="lm")

    def timed(fn):
        r = fn()
        torch.cuda.synchronize()
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        r = fn()
        e1.record()
        e1.synchronize()
        return e0.elapsed_time(e1), A.decode_results(r[0] if isinstance(r, tuple) else r)

    ms_cold, cold = timed(lambda: A.invert_batch_polished(prob, U, off, coarse, spec["polish_k"],
                                                          spec["polish_steps"], spec["n_cand"],
                                                          method="lm"))
    ms_warm, warm = timed(lambda: A.invert_image(prob, U, off, icfg))
    var = (spec["sigma"] / 1e-9) ** 2
    truth = [_theta_of(spec, xt[:, i]) for i in range(n_pix)]

    def stats(res):
        dchi, eb, et = [], [], []
        for i in range(n_pix):
            best = min((cold[i], warm[i]), key=lambda r: r["S_f64"])
            dchi.append((res[i]["S_f64"] - best["S_f64"]) / var)
            eb.append(_comb_err(list(res[i]["theta"]), list(best["theta"])))
            et.append(_comb_err(list(res[i]["theta"]), truth[i]))
        dchi, eb, et = map(np.array, (dchi, eb, et))
        return {"frac_dchi2_le_1": float(np.mean(dchi <= 1.0)),
                "frac_ident_within_0.5pct": float(np.mean(eb <= 0.005)),
                "median_ident_err_vs_truth": float(np.median(et))}
    return {"workload": f"{Wd} x {Hd} image, 3-mode DMT, {spec['cycles']} cycles x {spec['spc']} "
                        f"steps per pixel, truths smooth over the image",
            "cold": {"config": f"every pixel: {spec['P']} particles x {spec['iters']} updates + "
                               f"{spec['polish_steps']} LM steps on the best {spec['polish_k']}",
                     "ms": ms_cold, "ms_per_pixel": ms_cold / n_pix, **stats(cold)},
            "warm_start": {"config": f"coarse grid (every {spec['stride']}th row and column) as cold; "
                                     f"the rest {spec['fine']['P']} particles x {spec['fine']['iters']} "
                                     f"updates inside the box of the 4 coarse neighbours' winners "
                                     f"(+-{spec['margin']}), seeded with them, + "
                                     f"{spec['fine']['polish_steps']} LM steps on the best "
                                     f"{spec['fine']['polish_k']}",
                           "ms": ms_warm, "ms_per_pixel": ms_warm / n_pix, **stats(warm)},
            "speedup": ms_cold / ms_warm}


# ---------------------------------------------------------------------------
# Deflection points along the cantilever (the paper's n_dp = 3)
# ---------------------------------------------------------------------------
def run_points(A, W, dev, flush):
    """The same seeded cantilever and truth inverted from the tip record and
    from records at L/3, 2L/3 and L (records: FP64 forward at dt/4, every
    4th sample, plus noise)."""
    import numpy as np
    import torch
    spec = W.get("f4_points")
    D, N, npt = len(spec["free"]), W.n_steps(spec), len(spec["points"])
    rng = np.random.default_rng(spec["seed"])
    xt = rng.uniform(0.1, 0.9, size=(D, 1))
    fine = A.make_problem(dict(spec, spc=spec["spc"] * 4), n_steps=4 * N)
    d, _ = A.forward_batch_f64(fine, torch.from_numpy(xt).to(dev), None)
    gen = torch.Generator(device=dev).manual_seed(spec["seed"])
    rec = d.reshape(4 * N, npt)[3::4].float()
    rec = (rec + (spec["sigma"] / 1e-9) * torch.randn(rec.shape, device=dev, generator=gen)).contiguous()
    th_t = _theta_of(spec, xt[:, 0])
    out = {"workload": spec["name"]}
    for label, sp, U in (("tip_only", dict(spec, points=()), rec[:, -1].contiguous()),
                         ("three_points", spec, rec.reshape(-1))):
        prob = A.make_problem(sp)
        cfg = A.make_pso(sp)
        A.invert(prob, U, cfg)
        torch.cuda.synchronize()
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        res, _ = A.invert(prob, U, cfg)
        e1.record()
        e1.synchronize()
        r = A.decode_result(res)
        out[label] = {"ms_per_inversion": e0.elapsed_time(e1), "record_values": int(U.numel()),
                      "ident_rel_err_vs_truth": ident_errors(list(r["theta"]), th_t)[:3],
                      "S_f64_nm2": r["S_f64"], "status": r["status"]}
    # the same three-point inversion on the one-lane kernel (bit-identical)
    prob, cfg, U = A.make_problem(spec), A.make_pso(spec), rec.reshape(-1)
    A.set_lanes("one")
    try:
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        res, _ = A.invert(prob, U, cfg)
        e1.record()
        e1.synchronize()
    finally:
        A.set_lanes("auto")
    r = A.decode_result(res)
    out["three_points_one_lane"] = {"ms_per_inversion": e0.elapsed_time(e1),
                                    "same_result": r["S_f64"] == out["three_points"]["S_f64_nm2"]}
    out["ident"] = "H R, E* sqrt(R), a0"
    return out


# ---------------------------------------------------------------------------
# The paper's own experiments (App. A cantilever, 8 modes)
# ---------------------------------------------------------------------------
def run_paper_laws(A, W, dev, flush):
    """Hooke contact (k, h) and spring-damper (k, zeta_s) inversions (Sec. 4.2,
    4.3) and the base-motion inversions (Sec. 4.1: amplitude, amplitude and
    frequency, chirp) with the paper's truth values; records made on the GPU
    at dt/4 plus noise."""
    import torch
    out = {}
    for name in ("f2_hooke", "f2_spring_damper", "f3_amp", "f3_amp_freq", "f3_chirp"):
        spec = W.get(name)
        N = W.n_steps(spec)
        prob = A.make_problem(spec)
        xt = torch.tensor(spec["x_truth"], dtype=torch.float64, device=dev).reshape(-1, 1)
        if spec.get("drive") == "chirp":
            # record: the library's forward at dt/4 (every 4th sample) plus noise
            fine = A.make_problem(dict(spec, dt=spec["dt"] / 4, n_steps=4 * N))
            d, _ = A.forward_batch_f64(fine, xt, None)
            gen = torch.Generator(device=dev).manual_seed(spec["seed"])
            U = (d[3::4, 0].float() + (spec["sigma"] / 1e-9) *
                 torch.randn(N, device=dev, generator=gen)).contiguous()
        else:
            off = torch.tensor([0, N], dtype=torch.int64, device=dev)
            U = A.synth_records(prob, xt, off, spec["record_sub"], spec["sigma"], spec["seed"], 0)
        cfg = A.make_pso(spec)
        A.invert(prob, U, cfg)
        torch.cuda.synchronize()
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        res, _ = A.invert(prob, U, cfg)
        e1.record()
        e1.synchronize()
        r = A.decode_result(res)
        th_t = _theta_of(spec, spec["x_truth"])
        slots = [f[0] for f in spec["free"]]
        val = list(r["theta"]) + list(r["drive"])
        out[name] = {"workload": spec["name"], "ms_per_inversion": e0.elapsed_time(e1),
                     "record_steps": N, "theta_free": [val[s] for s in slots],
                     "theta_truth": [th_t[s] for s in slots], "S_f64_nm2": r["S_f64"],
                     "J_rel": r["J_rel"], "status": r["status"]}
    return out


# ---------------------------------------------------------------------------
# Single inversion (C2): plain swarm, LM-polished, accuracy, wide forward
# ---------------------------------------------------------------------------
def run_c2(A, W, dev, flush, peak_ops, steps=3):
    """One 1024 x 100 inversion of the 3-mode cantilever on the record of
    the stored truth (tests/golden/c2_invert.json; record made on the GPU),
    its LM-polished counterpart, both against the oracle's converged optimum
    of that record (x_opt; delta chi^2 on this record), the 16-record
    comparison,
    the fused iteration kernel's roofline, and the wide forward + misfit
    launch (262 144 particles) of the same record."""
    import numpy as np
    import torch
    spec = W.get("c2")
    with open(GOLDEN_C2) as f:
        gold = json.load(f)
    N, D, P, iters = W.n_steps(spec), len(spec["free"]), spec["P"], spec["iters"]
    m = spec["n_modes"]
    prob = A.make_problem(spec)
    off = torch.tensor([0, N], dtype=torch.int64, device=dev)
    xt = torch.tensor(gold["truth_x"], dtype=torch.float64, device=dev).reshape(D, 1)
    U = A.synth_records(prob, xt, off, spec["record_sub"], spec["sigma"], spec["seed"], 0)
    cfg = A.make_pso(spec)
    ws = torch.empty(A.invert_workspace_size(prob, cfg), dtype=torch.uint8, device=dev)
    res = torch.zeros(A.result_dtype_size(), dtype=torch.uint8, device=dev)
    hist = torch.empty(iters + 1, dtype=torch.float32, device=dev)
    A.invert(prob, U, cfg, workspace=ws, result=res, history=hist)
    torch.cuda.synchronize()
    A.profile_enable(True)
    A.profile_read()
    ms = []
    for _ in range(steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        A.invert(prob, U, cfg, workspace=ws, result=res, history=hist)
        e1.record()
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    kms, kn = A.profile_read()
    A.profile_enable(False)
    r = A.decode_result(res)
    lp = spec["lm_polish"]
    cfg_lm = A.make_pso(dict(spec, iters=lp["iters"]))
    A.invert_polished(prob, U, cfg_lm, lp["polish_k"], lp["polish_steps"], lp["n_cand"], method="lm")
    lm_ms = []
    for _ in range(steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        r_lm = A.invert_polished(prob, U, cfg_lm, lp["polish_k"], lp["polish_steps"], lp["n_cand"],
                                 method="lm")
        e1.record()
        e1.synchronize()
        lm_ms.append(e0.elapsed_time(e1))
    r_lm = A.decode_result(r_lm[0])

    def acc(rr):
        d, comb, S_ref = _dchi2_and_comb(A, spec, prob, U, rr, gold["x_opt"])
        e, n_id = determined_error(A, spec, prob, U, gold["x_opt"], list(rr["x"][:D]))
        return {"dchi2_vs_oracle_optimum": d, "param_err_determined": e,
                "determined_directions": n_id,
                "combinations_rel_err_vs_oracle": dict(zip(("H R", "E* sqrt(R)", "a0"), comb)),
                "meets_0.5pct": bool(d <= 1.0 and (e <= 0.005 or d < -1.0))}
    units = P * (iters + 1) * N
    ops_launch = P * N * algo_ops_per_step(m)
    avg_s = (kms / max(kn, 1)) / 1e3
    out = {"workload": "c2: 3-mode Euler-Bernoulli cantilever, DMT 4 unknowns, 1024 particles x "
                       "100 updates, 100 cycles x 256 steps (one inversion)",
           "plain_pso": dict(acc(r), ms_per_inversion=float(statistics.median(ms)),
                             value=units / (statistics.median(ms) / 1e3), unit=UNIT,
                             S_f64_nm2=r["S_f64"], S_f64_segments=r["segments"]),
           "lm_polished": dict(acc(r_lm), ms_per_inversion=float(statistics.median(lm_ms)),
                               config=f"{P} particles x {lp['iters']} updates + "
                                      f"{lp['polish_steps']} Levenberg-Marquardt steps on the best "
                                      f"{lp['polish_k']} ({lp['n_cand']} damping values per step)"),
           "ident": "H R, E* sqrt(R), a0 (the combinations a DMT record determines)",
           "roofline": {"bound": "alu", "achieved": ops_launch / avg_s / 1e12,
                        "peak": peak_ops / 1e12, "unit": "T FP32 lane-ops/s",
                        "frac": ops_launch / avg_s / peak_ops,
                        "kernel": "invert_modes_kernel<3,DMT,3> (one lane per mode of a particle)",
                        "ops_per_particle_step": algo_ops_per_step(m),
                        "issued_ops_per_particle_step": fp32_ops_per_step(m, spec["force"]),
                        "avg_launch_ms": avg_s * 1e3, "launches_timed": kn,
                        "traffic": ncu_traffic("invert_modes_kernel", "c2")},
           "records_16": lm_vs_plain(A, W, "c2", dev, flush)}
    # throughput regime: one wide forward + misfit launch (262 144 particles)
    Pb = 256 * 1024
    xb = torch.rand((D, Pb), dtype=torch.float32, device=dev,
                    generator=torch.Generator(device=dev).manual_seed(7))
    A.forward_batch(prob, xb, U, want_defl=False)
    torch.cuda.synchronize()
    A.profile_enable(True)
    A.profile_read()
    for _ in range(2):
        flush.zero_()
        A.forward_batch(prob, xb, U, want_defl=False)
    ms_b, n_b = A.profile_read()
    A.profile_enable(False)
    ach_b = Pb * N * algo_ops_per_step(m) / ((ms_b / n_b) / 1e3)
    out["batched_forward"] = {
        "particles": Pb, "steps": N, "ms_per_launch": ms_b / n_b,
        "value": Pb * N / ((ms_b / n_b) / 1e3), "unit": UNIT,
        "roofline": {"bound": "alu", "achieved": ach_b / 1e12, "peak": peak_ops / 1e12,
                     "unit": "T FP32 lane-ops/s", "frac": ach_b / peak_ops,
                     "ops_per_particle_step": algo_ops_per_step(m),
                     "kernel": "fwd_x2_kernel<3,DMT> (two particles per thread, paired FP32 "
                               "instructions)",
                     "traffic": ncu_traffic("fwd_x2_kernel", "c2_batched")}}
    return out


# ---------------------------------------------------------------------------
# Our arm: the 4096-pixel batched inversion
# ---------------------------------------------------------------------------
def all_sum(val: float, world: int) -> float:
    """Sum of a per-rank value over all ranks."""
    if world == 1:
        return val
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([val], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def run_ours(args):
    import torch

    from paper_1109_0334_gb300 import build as B
    B.build()
    from paper_1109_0334_gb300 import afminv as A
    from paper_1109_0334_gb300 import workloads as W

    rank, world, local = dist_setup()
    dev = torch.device("cuda", torch.cuda.current_device())
    spec0 = W.get("c3")
    # an image of world x 4096 pixels; each rank inverts its contiguous share
    # (independent problems: no data-path collective, weak scaling)
    n_total = spec0["n_pix"] * world
    lo, hi = rank_slice(n_total, rank, world)
    spec, prob, U, off, total_steps, xt, lens = c3_inputs(A, W, dev, n_pix=hi - lo, pixel_lo=lo,
                                                          n_total=n_total)
    n_pix = hi - lo
    P, iters, m = spec["P"], spec["iters"], spec["n_modes"]
    cfg = A.make_pso(spec)
    ws = torch.empty(A.invert_batch_workspace_size(prob, n_pix), dtype=torch.uint8, device=dev)
    res = torch.zeros((n_pix, A.result_dtype_size()), dtype=torch.uint8, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MiB > L2
    stream = torch.cuda.current_stream()
    kp = {}

    def step():
        _, kp["kp"] = A.invert_batch(prob, U, off, cfg, pixel0=lo, workspace=ws, results=res)

    for _ in range(args.warmup):          # the first call tunes and captures the graph
        step()
    torch.cuda.synchronize()

    A.profile_enable(True)
    A.profile_read()
    clocks = Clocks(local)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    step_ms = []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    kern_ms, kern_n = A.profile_read()
    A.profile_enable(False)
    T_ms = all_max(sum(step_ms), world)
    units_rank = P * (iters + 1) * total_steps            # particle-steps per step, this rank
    units_job = all_sum(units_rank, world)
    value = units_job * args.steps / (T_ms / 1e3)
    out_res = A.decode_results(res)

    # end to end through the public API with host buffers: records and offsets
    # copied in from pinned memory, every pixel's result copied out
    U_host = U.cpu().pin_memory()
    off_host = off.cpu().pin_memory()
    res_host = torch.empty_like(res, device="cpu").pin_memory()
    U_dev, off_dev = torch.empty_like(U), torch.empty_like(off)
    U_dev.copy_(U)
    off_dev.copy_(off)
    A.invert_batch(prob, U_dev, off_dev, cfg, pixel0=lo, workspace=ws, results=res)  # own graph
    torch.cuda.synchronize()
    e2e_steps = min(args.steps, 3)
    e2e_ms = []
    barrier(world)
    for _ in range(e2e_steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        U_dev.copy_(U_host, non_blocking=True)
        off_dev.copy_(off_host, non_blocking=True)
        A.invert_batch(prob, U_dev, off_dev, cfg, pixel0=lo, workspace=ws, results=res)
        res_host.copy_(res, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
    E_ms = all_max(sum(e2e_ms), world)
    e2e = {"value": units_job * e2e_steps / (E_ms / 1e3), "unit": UNIT,
           "h2d_bytes_per_step": int(U.numel() * 4 + off.numel() * 8),
           "d2h_bytes_per_step": int(res.numel()), "steps": e2e_steps,
           "ms_per_batch": E_ms / e2e_steps,
           "api": "afm_invert_batch (U_cat, off from pinned host memory; results to host)"}

    # roofline of the swarm kernel, its device time measured by event nodes
    # around it inside the launch graph
    props = torch.cuda.get_device_properties(dev)
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak_ops = props.multi_processor_count * 128 * sm_max * 1e6
    ops_launch = units_rank * algo_ops_per_step(m)
    avg_launch_s = (kern_ms / max(kern_n, 1)) / 1e3
    achieved = ops_launch / avg_launch_s
    roof = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_ops / 1e12,
            "unit": "T FP32 lane-ops/s", "frac": achieved / peak_ops,
            "traffic": ncu_traffic("batch_kernel", "c3"),
            "kernel": f"batch_kernel<3,DMT,{kp.get('kp')},false> (persistent swarm kernel, "
                      f"{kp.get('kp')} particles per thread)",
            "ops_per_particle_step": algo_ops_per_step(m),
            "ops_basis": "the method's count 36m + 24 (4 RK4 stages: tip sum, gap, DMT law, "
                         "modal accelerations, stage and slope FMAs; compensated misfit)",
            "issued_ops_per_particle_step": fp32_ops_per_step(m, spec["force"]),
            "particle_steps_per_launch": units_rank,
            "launches_timed": kern_n, "avg_launch_ms": avg_launch_s * 1e3,
            "kernel_share_of_step": kern_ms / sum(step_ms),
            "peak_basis": f"{props.multi_processor_count} SMs x 128 FP32 lanes x {sm_max:.0f} MHz"
                          + (" (sm_max_mhz of measured)" if peaks else " (nominal max clock)")}

    accuracy = polished = None
    if world == 1 and not args.no_accuracy:
        accuracy = accuracy_vs_oracle(A, spec, U, off, out_res)
        res_p, ms_p, kp_p, desc = run_c3_polished(A, spec, prob, U, off, lo, flush)
        pol = A.decode_results(res_p)
        polished = dict(desc, ms=ms_p, ms_per_pixel_inversion=ms_p / n_pix,
                        speedup_vs_plain_pso=(T_ms / args.steps) / ms_p, particles_per_thread=kp_p,
                        pixels_ok=sum(1 for r in pol if r["status"] == 0),
                        accuracy_vs_oracle=accuracy_vs_oracle(A, spec, U, off, pol))

    extras = {}
    if rank == 0 and world == 1 and not args.no_accuracy:
        extras["batch_per_pixel_problems"] = run_c3_per_pixel(A, spec, U, off, flush,
                                                              T_ms / args.steps)
    if rank == 0 and world == 1:
        if not args.no_c2:
            extras["single_inversion_c2"] = run_c2(A, W, dev, flush, peak_ops)
        if not args.no_c4:
            extras["polished_inversion_c4"] = run_c4(A, W, dev, flush)
        if not args.no_c5:
            extras["fe_inversion_c5"] = run_c5(A, W, dev, peak_ops, flush)
        if not args.no_f2:
            extras["paper_experiments"] = run_paper_laws(A, W, dev, flush)
        if not args.no_image:
            extras["image_warm_start"] = run_image(A, W, dev, flush)
        if not args.no_points:
            extras["deflection_points"] = run_points(A, W, dev, flush)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        rate, threads, desc, _ = oracle_c3_sample(spec)
        cpu = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": desc,
               "extrapolated_ms_per_batch": units_rank / rate * 1e3}
        if not args.no_c2:
            cpu["other_workloads"] = oracle_per_config(W, threads)

    if rank == 0:
        ok = sum(1 for r in out_res if r["status"] == 0)
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": T_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded truths and record lengths per pixel, GPU-made records at "
                    "dt/4 + 0.5% A0 noise)",
            "config": c3_config(spec, world),
            "ms_per_pixel_inversion": T_ms / args.steps / n_pix,
            # per step: queue reset, sort, swarm kernel, FP64 re-evaluation (guess, 2 x
            # (segment pass + join correction), final pass, result)
            "gpu_launches": 9 * args.steps,
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
            "result": {"pixels": n_pix, "pixels_ok": ok, "particles_per_thread": kp.get("kp"),
                       "particle_steps_per_step": units_rank,
                       "record_steps_total": total_steps},
            "accuracy_vs_oracle": accuracy,
            "ms_per_inversion_at_0.5pct": None if polished is None else {
                "config": "LM-polished batch: " + polished["config"],
                "ms_per_pixel_inversion": polished["ms_per_pixel_inversion"],
                "frac_pixels_meeting": polished["accuracy_vs_oracle"]["frac_meeting_both"],
                "criterion": "delta chi^2 <= 1 against the oracle's optimum and <= 0.5 % "
                             "parameter error along every direction the record determines to "
                             f"0.5 % ({polished['accuracy_vs_oracle']['pixels']}-pixel subset)"},
            "lm_polished_batch": polished,
        }
        out.update(extras)
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# CPU baseline and reference arm: the FP64 oracle on the host cores
# ---------------------------------------------------------------------------
def oracle_c3_setup(spec, pixels):
    """The oracle's own records of the given batch pixels (same truths,
    lengths and noise as the GPU's) and an initial swarm per pixel."""
    import numpy as np
    from oracle import oracle as O
    from paper_1109_0334_gb300 import workloads as W
    O.build()
    cyc, xt = W.c3_layout(spec, max(pixels) + 1)
    pm = O.make_pmap(spec)
    cases = []
    for i in pixels:
        sp = dict(spec, cycles=int(cyc[i]))
        c = O.make_case(sp)
        n = int(cyc[i]) * spec["spc"]
        U = O.record(c, pm, xt[:, i], n, spec["record_sub"], spec["sigma"], spec["seed"], i)
        U = (U / 1e-9).astype(np.float32).astype(np.float64) * 1e-9
        x, _ = O.pso_init(spec["P"], pm.D, spec["seed"], i)
        cases.append((c, U, np.ascontiguousarray(x)))
    return O, pm, cases


def oracle_c3_sample(spec, n_sub: int = 32):
    """One whole-swarm evaluation (256 particles: forward + misfit) of each of
    pixels 0..n_sub-1 by the oracle on all host cores; returns (particle-steps
    /s, threads, description, wall s)."""
    O, pm, cases = oracle_c3_setup(spec, list(range(n_sub)))
    threads = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    O.set_threads(threads)
    units, t0 = 0, time.perf_counter()
    for c, U, x in cases:
        O.misfit_batch(c, pm, x, U)
        units += x.shape[1] * len(U)
    wall = time.perf_counter() - t0
    desc = (f"one whole-swarm evaluation ({spec['P']} particles, FP64 oracle, OpenMP over "
            f"particles) of each of pixels 0..{n_sub - 1} on its own record "
            f"({units // spec['P']} record steps), {wall:.2f} s wall; the batch time beside it "
            f"is extrapolated from this rate to all {spec['n_pix']} pixels x "
            f"{spec['iters'] + 1} evaluations")
    return units / wall, threads, desc, wall


def oracle_per_config(W, threads: int) -> dict:
    """The oracle beside the GPU numbers of the other workloads, each on a
    bounded sample timed on the host cores (OpenMP over particles) and
    extrapolated where stated: C1 the full inversion; C2 one whole-swarm
    evaluation, extrapolated to its 101; C4 one whole-swarm evaluation and
    the complex-step gradients of the 32 particles its polish takes; C5 one
    swarm pass of 64 of the 8192 particles, extrapolated to 8192 x 61.
    Records are the oracle's own (seeded truths, dt/4 integration, noise)."""
    import numpy as np
    from oracle import oracle as O
    O.build()
    O.set_threads(threads)

    def setup(name):
        spec = W.get(name)
        c, pm = O.make_case(spec), O.make_pmap(spec)
        n = W.n_steps(spec)
        xt = O.truth_x(pm.D, spec["seed"])
        U = O.record(c, pm, xt, n, spec["record_sub"], spec["sigma"], spec["seed"])
        U = (U / 1e-9).astype(np.float32).astype(np.float64) * 1e-9
        x, _ = O.pso_init(spec["P"], pm.D, spec["seed"], 0)
        return spec, c, pm, n, U, np.ascontiguousarray(x)

    out = {}
    spec, c, pm, n, U, x = setup("c1")
    t0 = time.perf_counter()
    O.invert(c, pm, U, spec["P"], spec["iters"], spec["w"], spec["c1"], spec["c2"], spec["seed"])
    wall = time.perf_counter() - t0
    units = spec["P"] * (spec["iters"] + 1) * n
    out["c1"] = {"value": units / wall, "unit": UNIT, "ms_per_inversion": wall * 1e3,
                 "sample": f"the full inversion ({spec['P']} particles x {spec['iters']} "
                           f"updates, {n} steps)"}
    for name in ("c2", "c4"):
        spec, c, pm, n, U, x = setup(name)
        t0 = time.perf_counter()
        O.misfit_batch(c, pm, x, U)
        wall = time.perf_counter() - t0
        rate = x.shape[1] * n / wall
        iters = 100 if name == "c4" else spec["iters"]
        out[name] = {"value": rate, "unit": UNIT,
                     "extrapolated_ms_per_plain_inversion": x.shape[1] * (iters + 1) * n / rate * 1e3,
                     "sample": f"one whole-swarm evaluation ({x.shape[1]} particles, {n} steps), "
                               f"{wall:.2f} s wall, extrapolated to {iters + 1} evaluations"}
        if name == "c4":
            t0 = time.perf_counter()
            for p in range(32):
                O.grad_cs(c, pm, x[:, p].copy(), U)
            g_wall = time.perf_counter() - t0
            out[name]["ms_per_gradient"] = g_wall / 32 * 1e3
            out[name]["sample"] += (f"; complex-step gradients of 32 particles, {g_wall:.2f} s "
                                    f"wall (one particle at a time)")
    spec, c, pm, n, U, x = setup("c5")
    xs = np.ascontiguousarray(x[:, :64])
    t0 = time.perf_counter()
    O.misfit_batch(c, pm, xs, U)
    wall = time.perf_counter() - t0
    rate = xs.shape[1] * n / wall
    out["c5"] = {"value": rate, "unit": UNIT,
                 "extrapolated_ms_per_inversion": spec["P"] * (spec["iters"] + 1) * n / rate * 1e3,
                 "sample": f"one swarm pass of 64 of the {spec['P']} particles ({n} steps), "
                           f"{wall:.2f} s wall, extrapolated to {spec['P']} particles x "
                           f"{spec['iters'] + 1} evaluations"}
    return out


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_1109_0334_gb300 import workloads as W
    spec = W.get("c3")
    n_sub = 8
    O, pm, cases = oracle_c3_setup(spec, list(range(n_sub)))
    threads = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    O.set_threads(threads)

    def one():
        t0 = time.perf_counter()
        for c, U, x in cases:
            O.misfit_batch(c, pm, x, U)
        return time.perf_counter() - t0
    for _ in range(args.warmup):
        one()
    walls = [one() for _ in range(args.steps)]
    units = sum(x.shape[1] * len(U) for _c, U, x in cases)
    T = sum(walls)
    value = units * args.steps / T
    desc = (f"per step: one whole-swarm evaluation ({spec['P']} particles, FP64 oracle, OpenMP "
            f"over particles) of each of pixels 0..{n_sub - 1} of the batch on its own record "
            f"({units // spec['P']} record steps)")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
           "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * T / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": c3_config(spec, int(os.environ.get("WORLD_SIZE", "1"))),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                            "sample": desc},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


# ---------------------------------------------------------------------------
# Small untimed cases for profiler captures
# ---------------------------------------------------------------------------
# ---------------------------------------------------------------------------
# Configuration sweeps behind the workloads' polish settings (--sweep)
# ---------------------------------------------------------------------------
def _timed_results(A, fn):
    """One untimed call, then one timed call; (ms, decoded results)."""
    import torch
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    r = fn()
    e1.record()
    e1.synchronize()
    return e0.elapsed_time(e1), A.decode_results(r[0] if isinstance(r, tuple) else r)


def sweep_lm(A, W, dev, name):
    """Swarm updates x LM steps of the single-inversion polish (64
    candidates, 8 damping values) on 16 seeded records: median ms and the
    records within one noise variance of the best point any run found
    (a 100-update plain swarm and a 6 x 12 polish included)."""
    import numpy as np
    import torch
    spec = W.get(name)
    D, N = len(spec["free"]), W.n_steps(spec)
    prob = A.make_problem(spec)
    var = (spec["sigma"] / 1e-9) ** 2
    off = torch.tensor([0, N], dtype=torch.int64, device=dev)
    configs = [(3, 6), (3, 5), (2, 5), (3, 4), (4, 4), (2, 6)]
    runs = {c: [] for c in configs}
    best = []
    for pix in range(16):
        rng = np.random.default_rng(spec["seed"] + 1000 * pix)
        xt = rng.uniform(0.1, 0.9, size=(D, 1))
        U = A.synth_records(prob, torch.from_numpy(xt).to(dev), off, spec["record_sub"],
                            spec["sigma"], spec["seed"], pix)
        Ss = [A.decode_result(A.invert(prob, U, A.make_pso(dict(spec, iters=100), pixel=pix))[0])["S_f64"],
              A.decode_result(A.invert_polished(prob, U, A.make_pso(dict(spec, iters=6), pixel=pix),
                                                64, 12, 8, method="lm")[0])["S_f64"]]
        for (it, st) in configs:
            cfg = A.make_pso(dict(spec, iters=it), pixel=pix)
            ms, r = _timed_results(A, lambda: A.invert_polished(prob, U, cfg, 64, st, 8, method="lm"))
            runs[(it, st)].append((ms, r[0]["S_f64"]))
            Ss.append(r[0]["S_f64"])
        best.append(min(Ss))
    for c in configs:
        d = np.array([(s - b) / var for (_, s), b in zip(runs[c], best)])
        print(json.dumps({"workload": name, "updates": c[0], "lm_steps": c[1],
                          "median_ms": float(np.median([m for m, _ in runs[c]])),
                          "records_at_best": int((d <= 1.0).sum()), "max_dchi2": float(d.max())}))


def sweep_polish(A, W, dev):
    """Swarm updates x best K x LM steps (4 damping values) of the polished
    4096-pixel batch: ms, the pixels within one noise variance of the better
    of it and the plain batch, and the accuracy against the oracle's stored
    optima (accuracy_vs_oracle)."""
    import numpy as np
    import torch
    spec, prob, U, off, _, _, _ = c3_inputs(A, W, dev)
    var = (spec["sigma"] / 1e-9) ** 2
    _, plain = _timed_results(A, lambda: A.invert_batch(prob, U, off, A.make_pso(spec)))
    Sp = np.array([r["S_f64"] for r in plain])
    for it, k, st in ((2, 32, 5), (2, 32, 4), (2, 32, 3), (2, 16, 5), (1, 32, 5), (1, 32, 4),
                      (1, 32, 3), (1, 24, 4), (0, 32, 5)):
        cfg = A.make_pso(dict(spec, iters=it))
        ms, rs = _timed_results(A, lambda: A.invert_batch_polished(prob, U, off, cfg, k, st, 4,
                                                                  method="lm"))
        S = np.array([r["S_f64"] for r in rs])
        acc = accuracy_vs_oracle(A, spec, U, off, rs)
        print(json.dumps({"updates": it, "best_k": k, "lm_steps": st, "ms": ms,
                          "frac_dchi2_le_1_vs_plain": float(np.mean((S - np.minimum(S, Sp)) / var <= 1.0)),
                          "oracle_pixels": acc["pixels"], "frac_meeting_both": acc["frac_meeting_both"]}))


def sweep_image(A, W, dev):
    """Cold and warm-start configurations of the 64 x 64 image scan: ms and
    the pixels within one noise variance of the best of all runs."""
    import numpy as np
    import torch
    spec = W.get("f1_image")
    Wd, Hd = spec["width"], spec["height"]
    n_pix, D, N = Wd * Hd, len(spec["free"]), W.n_steps(spec)
    xt = W.image_truth(D, Wd, Hd, spec["seed"])
    prob = A.make_problem(spec)
    off = torch.arange(0, (n_pix + 1) * N, N, dtype=torch.int64, device=dev)
    U = A.synth_records(prob, torch.from_numpy(xt).to(dev), off, spec["record_sub"], spec["sigma"],
                        spec["seed"], 0)
    var = (spec["sigma"] / 1e-9) ** 2
    runs = {}
    for c in ((5, 8, 12, 8), (1, 32, 4, 4), (2, 32, 4, 4), (1, 32, 5, 4), (1, 16, 4, 4)):
        cfg = A.make_pso(dict(spec, iters=c[0]))
        runs[("cold",) + c] = _timed_results(
            A, lambda: A.invert_batch_polished(prob, U, off, cfg, c[1], c[2], c[3], method="lm"))
    for c, f in (((5, 8, 12, 8), (0, 4, 6)), ((1, 32, 4, 4), (0, 4, 6)), ((1, 32, 4, 4), (0, 8, 4)),
                 ((1, 32, 4, 4), (0, 4, 4)), ((5, 8, 12, 8), (0, 8, 4))):
        coarse = A.make_pso(dict(spec, iters=c[0]))
        fine = A.make_pso(dict(spec, P=spec["fine"]["P"], iters=f[0]))
        icfg = A.make_image_cfg(Wd, Hd, spec["stride"], spec["margin"], coarse, fine,
                                coarse_polish=(c[1], c[2]), fine_polish=(f[1], f[2]), n_cand=c[3],
                                method="lm")
        runs[("warm",) + c + f] = _timed_results(A, lambda: A.invert_image(prob, U, off, icfg))
    S = {k: np.array([r["S_f64"] for r in v[1]]) for k, v in runs.items()}
    best = np.min(np.array(list(S.values())), axis=0)
    for k, (ms, _) in runs.items():
        print(json.dumps({"run": list(k), "ms": ms,
                          "frac_dchi2_le_1_vs_best": float(np.mean((S[k] - best) / var <= 1.0))}))


def run_probe(args):
    """--probe invert: one inversion of the workload with --probe-iters
    updates; --probe forward: two forward + misfit launches over
    --probe-particles particles.  Prints the result; no timing."""
    import torch

    from paper_1109_0334_gb300 import build as B
    B.build()
    from paper_1109_0334_gb300 import afminv as A
    from paper_1109_0334_gb300 import workloads as W

    if args.probe == "batch":
        # one full wave of resident pixels (8 per SM: the occupancy of the
        # 4-particles-per-thread kernel) with records shortened tenfold,
        # --probe-iters updates
        props = torch.cuda.get_device_properties(0)
        spec, prob, U, off, total, _, _ = c3_inputs(A, W, torch.device("cuda"),
                                                 n_pix=props.multi_processor_count * 8,
                                                 cycles_div=10)
        cfg = A.make_pso(dict(spec, iters=args.probe_iters))
        res, kp = A.invert_batch(prob, U, off, cfg, particles_per_thread=args.probe_kp or 0)
        torch.cuda.synchronize()
        out = A.decode_results(res)
        print(json.dumps({"pixels": len(out), "kp": kp, "ok": sum(r["status"] == 0 for r in out)}))
        return
    if args.probe == "fe":
        # one FE swarm evaluation (8192 particles) of a 10-cycle record
        spec = W.get("c5", cycles=10)
        D, N = len(spec["free"]), W.n_steps(spec)
        prob = A.make_problem(spec)
        g = torch.Generator(device="cuda").manual_seed(7)
        x = torch.rand((D, spec["P"]), dtype=torch.float32, device="cuda", generator=g)
        U = torch.zeros(N, dtype=torch.float32, device="cuda")
        for _ in range(2):
            _, S = A.forward_batch(prob, x, U, want_defl=False)
        torch.cuda.synchronize()
        print(json.dumps({"S_mean": float(S.mean())}))
        return
    if args.probe == "adjoint":
        # gradient of 32 particles of the Kelvin-Voigt workload (one polish step's adjoint)
        spec = W.get("c4")
        D, N = len(spec["free"]), W.n_steps(spec)
        prob = A.make_problem(spec)
        off = torch.tensor([0, N], dtype=torch.int64, device="cuda")
        xt = torch.full((D, 1), 0.5, dtype=torch.float64, device="cuda")
        U = A.synth_records(prob, xt, off, spec["record_sub"], spec["sigma"], spec["seed"], 0)
        g = torch.Generator(device="cuda").manual_seed(7)
        x = torch.rand((D, 32), dtype=torch.float32, device="cuda", generator=g)
        for _ in range(2):
            S, G = A.adjoint(prob, x, U)
        torch.cuda.synchronize()
        print(json.dumps({"S_mean": float(S.mean()), "G_absmax": float(G.abs().max())}))
        return
    if args.probe == "polish_full":
        # the full 4096-pixel LM-polished batch, twice (the second after tuning)
        spec, prob, U, off, total, _, _ = c3_inputs(A, W, torch.device("cuda"))
        lp = spec["lm_polish"]
        cfg = A.make_pso(dict(spec, iters=lp["iters"]))
        for _ in range(2):
            res, kp = A.invert_batch_polished(prob, U, off, cfg, lp["polish_k"], lp["polish_steps"],
                                              lp["n_cand"], method="lm")
        torch.cuda.synchronize()
        out = A.decode_results(res)
        print(json.dumps({"pixels": len(out), "kp": kp, "ok": sum(r["status"] == 0 for r in out)}))
        return
    if args.probe == "polish":
        # one pixel wave of the LM-polished batch (records shortened tenfold)
        props = torch.cuda.get_device_properties(0)
        spec, prob, U, off, total, _, _ = c3_inputs(A, W, torch.device("cuda"),
                                                 n_pix=props.multi_processor_count * 4,
                                                 cycles_div=10)
        lp = spec["lm_polish"]
        cfg = A.make_pso(dict(spec, iters=lp["iters"]))
        res, kp = A.invert_batch_polished(prob, U, off, cfg, lp["polish_k"], 2, lp["n_cand"],
                                          method="lm")
        torch.cuda.synchronize()
        out = A.decode_results(res)
        print(json.dumps({"pixels": len(out), "kp": kp, "ok": sum(r["status"] == 0 for r in out)}))
        return
    spec = W.get(args.workload, iters=args.probe_iters)
    D = len(spec["free"])
    N = W.n_steps(spec)
    prob = A.make_problem(spec)
    off = torch.tensor([0, N], dtype=torch.int64, device="cuda")
    xt = torch.full((D, 1), 0.5, dtype=torch.float64, device="cuda")
    U = A.synth_records(prob, xt, off, spec["record_sub"], spec["sigma"], spec["seed"], 0)
    if args.probe == "invert":
        res, _ = A.invert(prob, U, A.make_pso(spec))
        torch.cuda.synchronize()
        print(json.dumps({k: (v.tolist() if hasattr(v, "tolist") else v)
                          for k, v in A.decode_result(res).items()}))
    elif args.probe == "sens":
        # normal equations of --probe-particles candidates (throughput regime)
        g = torch.Generator(device="cuda").manual_seed(7)
        x = torch.rand((D, args.probe_particles), dtype=torch.float32, device="cuda", generator=g)
        for _ in range(2):
            S, H, b = A.normal_equations(prob, x, U)
        torch.cuda.synchronize()
        print(json.dumps({"particles": args.probe_particles, "S_mean": float(S.mean())}))
    else:
        g = torch.Generator(device="cuda").manual_seed(7)
        x = torch.rand((D, args.probe_particles), dtype=torch.float32, device="cuda", generator=g)
        for _ in range(2):
            _, S = A.forward_batch(prob, x, U, want_defl=False)
        torch.cuda.synchronize()
        print(json.dumps({"particles": args.probe_particles, "S_mean": float(S.mean())}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=PROBE_WORKLOAD, help="workload of --probe invert/forward/sens")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--no-accuracy", action="store_true",
                    help="skip the accuracy check against the oracle's optima and the polished batch")
    ap.add_argument("--no-c2", action="store_true",
                    help="skip the single-inversion comparisons (plain / polished, 16 records, wide forward)")
    ap.add_argument("--no-c4", action="store_true", help="skip the polished-inversion comparison")
    ap.add_argument("--no-c5", action="store_true", help="skip the finite-element inversion")
    ap.add_argument("--no-f2", action="store_true", help="skip the paper's own experiments (tip-sample laws, base motion)")
    ap.add_argument("--no-image", action="store_true", help="skip the image warm-start comparison")
    ap.add_argument("--no-points", action="store_true", help="skip the deflection-points inversion")
    ap.add_argument("--probe", choices=["invert", "forward", "batch", "adjoint", "fe", "sens", "polish",
                                        "polish_full"],
                    default=None,
                    help="run one small untimed case for a profiler capture and exit")
    ap.add_argument("--sweep", choices=["lm_c2", "lm_c4", "polish", "image"], default=None,
                    help="run the configuration sweep behind a workload's polish settings and exit")
    ap.add_argument("--probe-iters", type=int, default=2)
    ap.add_argument("--probe-kp", type=int, default=None,
                    help="particles per thread of the batch probe (default: autotuned)")
    ap.add_argument("--probe-particles", type=int, default=32768)
    args = ap.parse_args()
    if args.probe:
        run_probe(args)
    elif args.sweep is not None:
        import torch
        from paper_1109_0334_gb300 import build as B
        B.build()
        from paper_1109_0334_gb300 import afminv as A
        from paper_1109_0334_gb300 import workloads as W
        dev = torch.device("cuda", 0)
        if args.sweep.startswith("lm_"):
            sweep_lm(A, W, dev, args.sweep[3:])
        elif args.sweep == "polish":
            sweep_polish(A, W, dev)
        else:
            sweep_image(A, W, dev)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
