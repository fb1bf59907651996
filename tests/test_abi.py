"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/scg.h declares; host-side argument checks reject bad input
before any CUDA call (CPU only, no compute)."""
import ctypes
import os
import re

import pytest
import torch

from paper_1709_04912_gb300 import build as scg_build
from paper_1709_04912_gb300 import scg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(scg_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    scg_build.build()
    return scg.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("scg_solve", "scg_project", "scg_backproject", "scg_tv", "scg_tv_grad"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_strerror_and_defaults(lib):
    assert lib.scg_strerror(0) == b"ok"
    assert b"invalid" in lib.scg_strerror(-1)
    p = scg.default_params()
    assert p["a"] == 0.975 and p["max_trials"] == 31 and p["K"] == 2 and p["max_iter"] == 100


def test_workspace_queries(lib):
    g = scg.geometry(512, 720, 725)
    b32 = lib.scg_solve_workspace_bytes(ctypes.byref(g), 2, scg.F32)
    b64 = lib.scg_solve_workspace_bytes(ctypes.byref(g), 2, scg.F64)
    assert b32 > 0 and b64 > b32
    assert lib.scg_solve_workspace_bytes(ctypes.byref(g), 5, scg.F32) > b32   # filter buffers
    bad = scg.geometry(1, 720, 725)
    assert lib.scg_solve_workspace_bytes(ctypes.byref(bad), 2, scg.F32) == 0
    assert lib.scg_op_workspace_bytes(ctypes.byref(g), 7) == 0


def test_invalid_arguments_rejected_before_any_launch(lib):
    g = scg.geometry(64, 90, 95)
    fake = ctypes.c_void_p(256)
    assert lib.scg_project(ctypes.byref(g), scg.F32, None, fake, fake, 1 << 20, None) == -1
    bad = scg.geometry(0, 90, 95)
    assert lib.scg_project(ctypes.byref(bad), scg.F32, fake, fake, fake, 1 << 20, None) == -1
    assert lib.scg_project(ctypes.byref(g), 9, fake, fake, fake, 1 << 20, None) == -5
    p = scg._params(scg.default_params())
    res = scg.Result()
    # eps <= 0, bad variant, bad a
    assert lib.scg_solve(ctypes.byref(g), 2, scg.F32, ctypes.byref(p), 0.0, fake, None, fake, fake,
                         1 << 30, ctypes.byref(res), None, 0, None, None, None) == -1
    assert lib.scg_solve(ctypes.byref(g), 11, scg.F32, ctypes.byref(p), 1.0, fake, None, fake, fake,
                         1 << 30, ctypes.byref(res), None, 0, None, None, None) == -1
    p2 = scg._params(scg.default_params(a=1.5))
    assert lib.scg_solve(ctypes.byref(g), 2, scg.F32, ctypes.byref(p2), 1.0, fake, None, fake, fake,
                         1 << 30, ctypes.byref(res), None, 0, None, None, None) == -1


def test_batch_workspace_query_and_validation(lib):
    shapes = [(64, 90, 95), (77, 33, 110), (130, 181, 185)]
    b = scg.batch_workspace_bytes(shapes, "S-CG", torch.float32)
    # at least the sum of the solo workspaces (plus descriptors and item lists)
    solo = sum(lib.scg_solve_workspace_bytes(ctypes.byref(scg.geometry(*s)), 2, scg.F32) for s in shapes)
    assert b >= solo
    assert scg.batch_workspace_bytes(shapes + [(1, 90, 95)], "S-CG", torch.float32) == 0
    arr = (scg.Problem * 2)()
    for q in range(2):
        arr[q].geometry = scg.geometry(64, 90, 95)
        arr[q].eps = 1.0
        arr[q].y = 256
        arr[q].x_out = 512
    assert lib.scg_batch_workspace_bytes(arr, 0, 2, scg.F32) == 0
    assert lib.scg_batch_workspace_bytes(arr, 2, 9, scg.F32) == 0
    p = scg._params(scg.default_params())
    res = (scg.Result * 2)()
    fake = ctypes.c_void_p(256)
    assert lib.scg_solve_batch(arr, 0, 2, scg.F32, ctypes.byref(p), fake, 1 << 30, res, None) == -1
    arr[1].eps = 0.0
    assert lib.scg_solve_batch(arr, 2, 2, scg.F32, ctypes.byref(p), fake, 1 << 30, res, None) == -1
    arr[1].eps = 1.0
    arr[1].y = None
    assert lib.scg_solve_batch(arr, 2, 2, scg.F32, ctypes.byref(p), fake, 1 << 30, res, None) == -1
    arr[1].y = 256
    hl = scg._params(scg.default_params(host_loop=1))
    assert lib.scg_solve_batch(arr, 2, 2, scg.F32, ctypes.byref(hl), fake, 1 << 30, res, None) == -5
