"""The C-ABI library builds, loads and exports every entry point that
include/*.h declares; host-side argument validation needs no GPU."""
import ctypes as C
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libafm():
    from paper_1109_0334_gb300 import build
    build.build()
    from paper_1109_0334_gb300 import afminv
    return afminv


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names.update(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(afm_\w+)\s*\(", txt, flags=re.M))
    return sorted(names)


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("afm_forward_batch", "afm_misfit", "afm_pso_step", "afm_invert"):
        assert n in names


def test_library_exports_every_declared_symbol(libafm):
    L = libafm.lib()
    missing = [n for n in _declared() if not hasattr(L, n)]
    assert not missing, missing


def test_python_binding_names_follow_the_abi(libafm):
    for n in _declared():
        short = n[len("afm_"):]
        if short in ("ctx_create", "ctx_destroy", "last_error", "status_string", "version",
                     "invert_workspace_size"):
            continue
        assert hasattr(libafm, short), short


def _c1_problem(libafm, **kw):
    from paper_1109_0334_gb300 import workloads as W
    return libafm.make_problem(W.get("c1", **kw))


def test_invalid_arguments_rejected_before_any_launch(libafm):
    L = libafm.lib()
    p = _c1_problem(libafm)
    # NULL problem
    assert L.afm_forward_batch(None, None, None, 1, None, None, None, None) == libafm.ERR_INVALID_ARG
    # lo >= hi
    bad = _c1_problem(libafm)
    bad.hi[0] = bad.lo[0]
    assert L.afm_forward_batch(None, C.byref(bad), None, 1, None, None, None, None) == libafm.ERR_INVALID_ARG
    assert b"lo < hi" in L.afm_last_error()
    # too many modes
    bad = _c1_problem(libafm, model="modal_eb", n_modes=9)
    assert L.afm_forward_batch(None, C.byref(bad), None, 1, None, None, None, None) == libafm.ERR_INVALID_ARG
    # log scale with lo <= 0
    bad = _c1_problem(libafm)
    bad.lo[0] = 0.0
    assert L.afm_forward_batch(None, C.byref(bad), None, 1, None, None, None, None) == libafm.ERR_INVALID_ARG
    # steps per cycle out of range, n_steps < 1
    bad = _c1_problem(libafm, spc=3)
    assert L.afm_forward_batch(None, C.byref(bad), None, 1, None, None, None, None) == libafm.ERR_INVALID_ARG
    bad = _c1_problem(libafm)
    bad.n_steps = 0
    assert L.afm_forward_batch(None, C.byref(bad), None, 1, None, None, None, None) == libafm.ERR_INVALID_ARG
    # repeated slot
    bad = _c1_problem(libafm)
    bad.slot[1] = bad.slot[0]
    assert L.afm_forward_batch(None, C.byref(bad), None, 1, None, None, None, None) == libafm.ERR_INVALID_ARG
    # DMT needs R, a0 > 0
    bad = _c1_problem(libafm)
    bad.fixed[2] = 0.0
    assert L.afm_forward_batch(None, C.byref(bad), None, 1, None, None, None, None) == libafm.ERR_INVALID_ARG
    # valid problem but NULL context
    assert L.afm_forward_batch(None, C.byref(p), None, 1, None, None, None, None) == libafm.ERR_INVALID_ARG
    assert b"context" in L.afm_last_error()


def test_workspace_size_and_pso_cfg_validation(libafm):
    from paper_1109_0334_gb300 import workloads as W
    p = _c1_problem(libafm)
    cfg = libafm.make_pso(W.get("c1"))
    n = libafm.invert_workspace_size(p, cfg)
    # x, v, two personal-best buffers (each D*P floats, 256-aligned) + pbest_S + keys + flags
    assert n >= 4 * 2 * 64 * 4 + 64 * 4 + 16
    assert n % 256 == 0
    cfg.P = 0
    with pytest.raises(libafm.AfmError):
        libafm.invert_workspace_size(p, cfg)


def test_status_strings(libafm):
    L = libafm.lib()
    assert L.afm_status_string(0) == b"AFM_OK"
    assert L.afm_status_string(3) == b"AFM_ERR_NONFINITE"
    assert L.afm_version() >= 100


def test_batch_problem_array_validation(libafm):
    """One problem for every pixel, or one per pixel: the workspace grows by
    the per-pixel constants; other counts and problems that differ in more
    than the cantilever, drive and set-point are rejected."""
    from paper_1109_0334_gb300 import workloads as W
    spec = W.get("c3", P=64, iters=2)
    p0 = libafm.make_problem(spec, n_steps=2560)
    p1 = libafm.make_problem(dict(spec, Zc=14e-9, A0=18e-9, f1_hz=310e3), n_steps=2048)
    n1 = libafm.invert_batch_workspace_size(p0, 2)
    n2 = libafm.invert_batch_workspace_size([p0, p1], 2)
    assert n2 > n1 and n2 % 256 == 0
    with pytest.raises(libafm.AfmError) as ei:
        libafm.invert_batch_workspace_size([p0, p1], 3)
    assert ei.value.status == libafm.ERR_INVALID_ARG
    bad = libafm.make_problem(dict(spec, spc=128), n_steps=2048)
    with pytest.raises(libafm.AfmError) as ei:
        libafm.invert_batch_workspace_size([p0, bad], 2)
    assert ei.value.status == libafm.ERR_INVALID_ARG
    assert b"differs from problem 0" in libafm.lib().afm_last_error()
    bad = libafm.make_problem(spec, n_steps=2048)
    bad.hi[2] = 40e-9
    with pytest.raises(libafm.AfmError):
        libafm.invert_batch_workspace_size([p0, bad], 2)
    # the largest n_steps sizes the FP64 re-evaluation
    assert libafm.invert_batch_workspace_size([p1, p0], 2) == n2
