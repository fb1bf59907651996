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
    assert p["a"] == 0.975 and p["max_trials"] == 32 and p["K"] == 2 and p["max_iter"] == 100


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


def test_eta_rule_needs_a_positive_eta0(lib):
    g = scg.geometry(64, 90, 95)
    fake = ctypes.c_void_p(256)
    res = scg.Result()
    for e0 in (0.0, -1.0, float("inf")):
        p = scg._params(scg.default_params(perturb="eta", eta0=e0))
        assert lib.scg_solve(ctypes.byref(g), scg.VARIANTS["S-CG"], scg.F32, ctypes.byref(p), 1.0, fake, None,
                             fake, fake, 1 << 40, ctypes.byref(res), None, 0, None, None, None) == -1
    p = scg._params(scg.default_params(perturb="eta", eta0=0.0))
    pr = (scg.Problem * 1)()
    pr[0].geometry = g
    pr[0].eps = 1.0
    pr[0].y = fake
    pr[0].x_out = fake
    assert lib.scg_solve_batch(pr, 1, scg.VARIANTS["S-CG"], scg.F32, ctypes.byref(p), fake, 1 << 40,
                               (scg.Result * 1)(), None) == -1


def test_filter_length_limit_rejected_before_any_launch(lib):
    # the row filter holds a padded row pair's FFT in shared memory: n_bins above
    # 8192 (FP32 arithmetic) or 4096 (FP64) is refused by every entry point that
    # filters, before any device work
    fake = ctypes.c_void_p(256)
    big32, big64 = scg.geometry(64, 10, 8193), scg.geometry(64, 10, 4097)
    assert lib.scg_filter(ctypes.byref(big32), scg.F32, 0.0, 1.0, fake, fake, fake, 1 << 40, None) == -5
    assert lib.scg_filter(ctypes.byref(big32), scg.F16, 0.0, 1.0, fake, fake, fake, 1 << 40, None) == -5
    assert lib.scg_filter(ctypes.byref(big64), scg.F64, 0.0, 1.0, fake, fake, fake, 1 << 40, None) == -5
    assert lib.scg_fbp(ctypes.byref(big32), scg.F32, fake, fake, fake, 1 << 40, None) == -5
    p = scg._params(scg.default_params())
    res = scg.Result()
    assert lib.scg_solve(ctypes.byref(big32), scg.VARIANTS["S-PCG"], scg.F32, ctypes.byref(p), 1.0, fake, None,
                         fake, fake, 1 << 40, ctypes.byref(res), None, 0, None, None, None) == -5
    # and bad filter parameters
    g = scg.geometry(64, 10, 95)
    assert lib.scg_filter(ctypes.byref(g), scg.F32, 0.0, 0.0, fake, fake, fake, 1 << 40, None) == -1


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


def test_server_host_side(lib):
    # create / submit / pending / destroy touch no device memory until the first step
    fp = scg.server_footprint(64, 90, 95, "S-CG", torch.float32)
    assert fp >= lib.scg_solve_workspace_bytes(ctypes.byref(scg.geometry(64, 90, 95)), 2, scg.F32)
    assert scg.server_footprint(64, 90, 95, "S-PCG", torch.float32) > fp     # filter buffers
    assert scg.server_footprint(1, 90, 95) == 0
    p = scg._params(scg.default_params())
    cfg = scg.ServerConfig(2, scg.F32, p, 1 << 20, 3 * fp, 4, 1)
    h = ctypes.c_void_p()
    assert lib.scg_server_create(ctypes.byref(cfg), ctypes.byref(h)) == 0
    arr = (scg.Problem * 1)()
    arr[0].geometry = scg.geometry(64, 90, 95)
    arr[0].eps = 1.0
    arr[0].y = 256
    arr[0].x_out = 512
    assert lib.scg_server_submit(h, arr, 7) == 0
    assert lib.scg_server_submit(h, arr, 8) == 0
    big = (scg.Problem * 1)()
    big[0].geometry = scg.geometry(1024, 1440, 1449)
    big[0].eps = 1.0
    big[0].y = 256
    big[0].x_out = 512
    assert lib.scg_server_submit(h, big, 9) == -3           # can never fit this pool
    arr[0].eps = -1.0
    assert lib.scg_server_submit(h, arr, 10) == -1
    q, a = ctypes.c_int(), ctypes.c_int()
    assert lib.scg_server_pending(h, ctypes.byref(q), ctypes.byref(a)) == 0
    assert (q.value, a.value) == (2, 0)
    assert lib.scg_server_destroy(h) == 0
    # invalid configurations
    for bad in (scg.ServerConfig(2, scg.F32, p, 1 << 20, 3 * fp, 0, 1),
                scg.ServerConfig(2, scg.F32, p, 1 << 20, 3 * fp, 4, 0),
                scg.ServerConfig(9, scg.F32, p, 1 << 20, 3 * fp, 4, 1),
                scg.ServerConfig(2, scg.F32, p, None, 3 * fp, 4, 1),
                scg.ServerConfig(2, scg.F32, p, 1 << 20, 64, 4, 1)):
        assert lib.scg_server_create(ctypes.byref(bad), ctypes.byref(h)) in (-1, -3)


def test_reduced_storage_workspaces(lib):
    g = scg.geometry(512, 720, 725)
    b32 = lib.scg_solve_workspace_bytes(ctypes.byref(g), 2, scg.F32)
    b16 = lib.scg_solve_workspace_bytes(ctypes.byref(g), 2, scg.F16)
    bb16 = lib.scg_solve_workspace_bytes(ctypes.byref(g), 2, scg.BF16)
    assert 0 < b16 == bb16 < 0.6 * b32                 # vectors and views at 2 bytes
    for v in (0, 1):                                   # CG, PCG: recursive updates, FP32/FP64 only
        assert lib.scg_solve_workspace_bytes(ctypes.byref(g), v, scg.F16) == 0
        assert lib.scg_solve_workspace_bytes(ctypes.byref(g), v, scg.BF16) == 0
    assert lib.scg_op_workspace_bytes(ctypes.byref(g), scg.F16) > 0
    assert lib.scg_solve_workspace_bytes(ctypes.byref(g), 2, 4) == 0


def test_operator_rejects_bad_arguments_without_device_work(lib):
    h = ctypes.c_void_p()
    fake = ctypes.c_void_p(256)
    bad = scg.geometry(1, 90, 95)
    assert lib.scg_operator_create(ctypes.byref(bad), scg.F32, fake, 1 << 20, None, ctypes.byref(h)) == -1
    g = scg.geometry(64, 90, 95)
    assert lib.scg_operator_create(ctypes.byref(g), 7, fake, 1 << 20, None, ctypes.byref(h)) == -5
    assert lib.scg_operator_project(None, fake, fake, None) == -1
    assert lib.scg_operator_destroy(None) == -1
    assert lib.scg_operator_timing(None, 1) == -1


def test_release_with_nothing_cached(lib):
    assert lib.scg_release() == 0
