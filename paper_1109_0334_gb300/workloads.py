"""Seeded synthetic workloads: the cantilever / force / swarm configurations
the library is exercised on (C1-C5 and the paper's own tip-sample
experiments), as plain SI values.

This module holds inputs only (physical constants, bounds, swarm sizes,
seeds, and a seeded sampler for swarm coordinates).  It contains none of the
method's arithmetic, so both the CUDA path and the independent CPU oracle
may read it.

Parameter slots (theta[0..4]) of the DMT family: E* [Pa], H [J], R [m],
a0 [m], eta [Pa s].  A free parameter is (slot, lo, hi, log_scale).
"""
from __future__ import annotations

import copy

import numpy as np

SEED_BASE = 1109033400

_CANTILEVER = dict(f1_hz=300e3, k=40.0, Q=400.0, A0=20e-9, Zc=16e-9)
_PSO = dict(w=0.7, c1=1.5, c2=1.5)

_E = (0, 1e8, 1e10, True)       # E* in [0.1, 10] GPa, log
_H = (1, 1e-20, 1e-19, True)    # Hamaker constant, log
_R = (2, 5e-9, 30e-9, False)    # tip radius, linear
_A0 = (3, 0.2e-9, 0.5e-9, False)  # intermolecular distance, linear
_ETA = (4, 0.0, 500.0, False)   # contact viscosity, linear

WORKLOADS = {
    # Single-mode point mass, FP64 oracle scale: 20 cycles x 200 steps.
    "c1": dict(name="point-mass DMT, 2 unknowns, 64 particles x 50 updates",
               model="point_mass", n_modes=1, spc=200, cycles=20, force="dmt",
               free=[_E, _H], fixed=[0.0, 0.0, 10e-9, 0.3e-9, 0.0],
               P=64, iters=50, seed=SEED_BASE + 1, **_CANTILEVER, **_PSO),
    # 3-mode Euler-Bernoulli modal cantilever: 100 cycles x 256 steps.
    "c2": dict(name="3-mode EB DMT, 4 unknowns, 1024 particles x 100 updates",
               model="modal_eb", n_modes=3, spc=256, cycles=100, force="dmt",
               free=[_E, _H, _R, _A0], fixed=[0.0, 0.0, 0.0, 0.0, 0.0],
               P=1024, iters=100, seed=SEED_BASE + 2,
               # the same record by a short swarm and Levenberg-Marquardt
               # polish of its best particles (64 candidates cost the time of
               # 8 while they fit the GPU's sub-partitions, and reach the
               # optimum far more often: a sweep over 16 records put 16 of 16
               # at delta chi^2 <= 1 against 13 of 16 with 8 candidates; 3
               # updates and 5 steps keep 16 of 16 within 0.03 of the best,
               # as do 4 steps, but 4 steps left two C4 records 30 variances
               # off after 4 updates)
               lm_polish=dict(iters=3, polish_k=64, polish_steps=5, n_cand=8),
               **_CANTILEVER, **_PSO),
    # 4096 independent pixels, 20..200 cycles each, 256 particles x 60 updates.
    "c3": dict(name="4096 pixels, 3-mode EB DMT, 256 particles x 60 updates",
               model="modal_eb", n_modes=3, spc=256, cycles=(20, 200), force="dmt",
               free=[_E, _H, _R, _A0], fixed=[0.0, 0.0, 0.0, 0.0, 0.0],
               P=256, iters=60, n_pix=4096, seed=SEED_BASE + 3,
               # the same pixels by a short swarm and Levenberg-Marquardt polish
               # of each pixel's best particles: a sweep over the first 1024
               # pixels at about equal cost favoured many candidates from a
               # short swarm (2 updates, best 32, 5 steps of 4 damping values:
               # 98 % of pixels at delta chi^2 <= 1 in 0.78 s) over deep polish
               # of few (5 updates, best 8, 12 steps of 8: 92 % in 1.08 s); a
               # sweep over all 4096 then put 1 update and 4 steps (99.4 % in
               # 0.93 s) ahead of 2 updates and 5 steps (99.2 % in 1.18 s)
               lm_polish=dict(iters=1, polish_k=32, polish_steps=4, n_cand=4),
               **_CANTILEVER, **_PSO),
    # DMT + Kelvin-Voigt contact damping, adjoint-polished.
    "c4": dict(name="3-mode EB DMT+KV, 5 unknowns, 1024 x 40 + 20 polish on 32",
               model="modal_eb", n_modes=3, spc=256, cycles=100, force="dmt_kv",
               free=[_E, _H, _R, _A0, _ETA], fixed=[0.0, 0.0, 0.0, 0.0, 0.0],
               P=1024, iters=40, polish_k=32, polish_steps=20, seed=SEED_BASE + 4,
               lm_polish=dict(iters=3, polish_k=64, polish_steps=5, n_cand=8),
               **_CANTILEVER, **_PSO),
    # 32-element Hermite FE beam, Newmark beta = 1/4.
    "c5": dict(name="FE Hermite 32 elements DMT, 4 unknowns, 8192 particles x 60 updates",
               model="fe_hermite", n_elem=32, L=125e-6, E=1.76e11, rho=2330.0,
               newmark_beta=0.25, spc=512, cycles=50, force="dmt",
               free=[_E, _H, _R, _A0], fixed=[0.0, 0.0, 0.0, 0.0, 0.0],
               P=8192, iters=60, seed=SEED_BASE + 5, **_CANTILEVER, **_PSO),
}
# The paper's own tip-sample experiments (Sec. 4.2, 4.3) on its App. A
# cantilever (L = 525 um, 35 x 5 um silicon, mu = 4.0775e-7 kg/m): first
# natural frequency 25 468.9 Hz (printed in App. A), mode-1 modal stiffness
# omega_1^2 mu L / 4 = 1.3705 N/m, 8 modes.  Set-point: the sample 50 nm from
# the neutral axis (the paper's h), free amplitude 60 nm.  Truths are the
# paper's (normalised in x_truth), not drawn.
_APPA = dict(f1_hz=25468.9, k=1.3705, Q=400.0, A0=60e-9, Zc=50e-9)
_KS = (0, 0.0, 25.0, False)            # sample stiffness [N/m], linear
_HD = (1, -10e-9, 10e-9, False)        # contact datum: separation 50 nm - c1
_ZS = (2, 0.0, 2e-6, False)            # sample damping [N s/m], linear
WORKLOADS["f2_hooke"] = dict(
    name="App. A cantilever, 8 modes, Hooke contact (k, h), 512 particles x 30 updates",
    model="modal_eb", n_modes=8, spc=512, cycles=8, force="hooke",
    free=[_KS, _HD], fixed=[0.0, 0.0, 0.0, 0.0, 0.0], x_truth=[4.0 / 25.0, 0.5],
    rel_scale=[None, 50e-9],           # datum errors relative to the 50 nm separation
    P=512, iters=30, seed=SEED_BASE + 6, **_APPA, **_PSO)
WORKLOADS["f2_spring_damper"] = dict(
    name="App. A cantilever, 8 modes, spring-damper contact (k, zeta_s), 512 x 30",
    model="modal_eb", n_modes=8, spc=512, cycles=8, force="spring_damper",
    free=[_KS, _ZS], fixed=[0.0, 0.0, 0.0, 0.0, 0.0], x_truth=[4.0 / 25.0, 0.05],
    P=512, iters=30, seed=SEED_BASE + 7, **_APPA, **_PSO)

# Image scan with cross-pixel warm start: a 64 x 64 image of the 3-mode DMT
# cantilever, 40 cycles per pixel, truths varying smoothly over the image.
WORKLOADS["f1_image"] = dict(
    name="64 x 64 image, 3-mode EB DMT, coarse grid every 4th pixel",
    model="modal_eb", n_modes=3, spc=256, cycles=40, force="dmt",
    free=[_E, _H, _R, _A0], fixed=[0.0, 0.0, 0.0, 0.0, 0.0],
    width=64, height=64, stride=4, margin=0.05,
    # a sweep (accuracy against the best of all configurations per pixel) put
    # the polished batch's configuration ahead of a deeper polish of fewer
    # candidates: cold 1 x 32 x 4 98.7 % at delta chi^2 <= 1 in 338 ms
    # against 5 x 8 x 12 92.0 % in 551 ms; warm start with 4 steps on the
    # best 8 of the box-seeded swarm 97.1 % in 166 ms (6 steps on the best 4:
    # 95.0 % in 165 ms)
    P=256, iters=1, polish_k=32, polish_steps=4, n_cand=4,            # coarse pixels
    fine=dict(P=64, iters=0, polish_k=8, polish_steps=4),             # the others
    seed=SEED_BASE + 8, **_CANTILEVER, **_PSO)

# The paper's base-motion inversions (Sec. 4.1): App. A cantilever, 8 modes,
# no tip force, base y_b = a sin(2 pi (f t + g t^2)) from rest, step 1e-7 s,
# 1000 steps; truths a = 2 nm, f = 25 600 Hz (sine) or f = 10 kHz,
# g = 2e7 Hz/s (chirp); the paper's search boxes.  Noise 0.5 % of a.
_DRV = dict(model="modal_eb", n_modes=8, spc=400, drive="chirp", dt=1e-7, n_steps=1000,
            force="linear_spring", fixed=[0.0, 0.0, 0.0, 0.0, 0.0], P=512, iters=30,
            sigma=0.005 * 2e-9, **_APPA, **_PSO)
_DA = (5, 0.0, 100e-9, False)          # base amplitude [m]
WORKLOADS["f3_amp"] = dict(
    name="App. A cantilever, 8 modes, base amplitude (1-D), 512 x 30",
    free=[_DA], drive_params=(2e-9, 25600.0, 0.0), x_truth=[0.02], seed=SEED_BASE + 9, **_DRV)
WORKLOADS["f3_amp_freq"] = dict(
    name="App. A cantilever, 8 modes, base amplitude and frequency (2-D), 512 x 30",
    free=[_DA, (6, 25100.0, 26100.0, False)], drive_params=(2e-9, 25600.0, 0.0),
    x_truth=[0.02, 0.5], seed=SEED_BASE + 10, **_DRV)
WORKLOADS["f3_chirp"] = dict(
    name="App. A cantilever, 8 modes, chirp (a, f, g) (3-D), 512 x 30",
    free=[_DA, (6, 7500.0, 12500.0, False), (7, 1.9e7, 2.1e7, False)],
    drive_params=(2e-9, 1e4, 2e7), x_truth=[0.02, 0.5, 0.5], seed=SEED_BASE + 11, **_DRV)

# Deflection records at three points of the 3-mode cantilever (the paper's
# n_dp = 3, Sec. 3.2): x = L/3, 2L/3 and the tip.
WORKLOADS["f4_points"] = dict(WORKLOADS["c2"], name="3-mode EB DMT, deflections at L/3, 2L/3, L, "
                              "512 particles x 50 updates", points=(1.0 / 3.0, 2.0 / 3.0, 1.0),
                              cycles=40, P=512, iters=50, seed=SEED_BASE + 12)

for _w in WORKLOADS.values():
    _w.setdefault("sigma", 0.005 * _w["A0"])    # 0.5 % of the free amplitude
    _w["record_sub"] = 4


def get(name: str, **overrides) -> dict:
    """A copy of one workload with fields overridden (e.g. cycles, P, iters)."""
    w = copy.deepcopy(WORKLOADS[name])
    w.update(overrides)
    return w


def n_steps(w: dict) -> int:
    if "n_steps" in w:
        return int(w["n_steps"])
    cyc = w["cycles"]
    if isinstance(cyc, (tuple, list)):
        raise ValueError("per-pixel record lengths: use the pixel's own cycle count")
    return int(cyc) * int(w["spc"])


def c3_layout(spec: dict, n_pix: int | None = None, cycles_div: int = 1):
    """Seeded per-pixel inputs of the 4096-pixel batch: record lengths in
    cycles (uniform integers in the workload's cycle range, divided by
    cycles_div, at least 1) and truths x* [D][n_pix] uniform in [0.1, 0.9]
    (the interior of the normalised cube).  Pixel i's record is its truth's
    deflection over cycles[i] * spc steps plus noise keyed by pixel i."""
    n_pix = spec["n_pix"] if n_pix is None else n_pix
    lo, hi = spec["cycles"]
    rng = np.random.default_rng(spec["seed"])
    cyc = np.maximum(rng.integers(lo, hi + 1, size=n_pix) // cycles_div, 1)
    xt = rng.uniform(0.1, 0.9, size=(len(spec["free"]), n_pix))
    return cyc, xt


def sample_x(D: int, P: int, seed: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """Seeded uniform swarm coordinates, shape [D][P], float32-exact."""
    rng = np.random.default_rng(seed)
    x = rng.uniform(lo, hi, size=(D, P)).astype(np.float32)
    return x


def image_truth(D: int, width: int, height: int, seed: int) -> np.ndarray:
    """Seeded truths varying smoothly over a width x height image, [D][W*H]
    in [0.15, 0.85] (row-major pixels): per dimension two plane waves of
    small integer wave numbers."""
    rng = np.random.default_rng(seed)
    j, i = np.meshgrid(np.arange(height), np.arange(width), indexing="ij")
    out = np.empty((D, width * height))
    for d in range(D):
        f = np.zeros((height, width))
        for amp in (0.6, 0.4):
            kx, ky = rng.integers(0, 3, size=2)
            ph = rng.uniform(0, 2 * np.pi)
            f += amp * np.sin(2 * np.pi * (kx * i / width + ky * j / height) + ph)
        out[d] = (0.5 + 0.35 * f).reshape(-1)
    return out
