"""scg_tv_static: the TV norm for callers that cannot allocate device memory.

Such callers (a plug-in inside a host program whose memory pool owns the
device, a real-time loop that forbids allocator calls, a fixed memory budget)
cannot provide the workspace scg_tv needs, so this entry point keeps its
scratch in a fixed device array inside the library.  The test calls it through
the C ABI and checks it against scg_tv and against the FP64 oracle's TV,
within the same tolerances as the other TV tests, on two calls in a row (the
second call must not see the first one's leftovers); after scg_release() (which
makes the next call look up the scratch address again) it must still agree;
and sizes beyond its limit are refused.  This file is
collected last so that a run stopping at its first failure has run every other
test already.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_1709_04912_gb300 import inputs, scg

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _entry():
    lib = scg.load()
    fn = lib.scg_tv_static
    fn.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    return fn


def _image(n, seed):
    x = inputs.ellipse_phantom(n, 8, seed)
    return x + 0.1 * inputs.normal(seed, "img", n * n).reshape(n, n)


@pytest.mark.parametrize("dtype,n,tol", [(torch.float32, 64, 1e-6), (torch.float32, 1024, 1e-6),
                                         (torch.float64, 200, 1e-12)])
def test_static_scratch_tv_matches_workspace_tv_twice(dtype, n, tol):
    fn = _entry()
    prec = scg.F64 if dtype == torch.float64 else scg.F32
    stream = torch.cuda.current_stream().cuda_stream
    for call, seed in enumerate((1, 2, 3)):       # two calls in a row, different images ...
        if call == 2:
            scg.release()                         # ... then one after the address was forgotten
        img = _image(n, seed + n)
        x = torch.tensor(img, dtype=dtype, device=DEV)
        ref = float(scg.scg_tv(x))
        out = torch.full((), -1.0, dtype=torch.float64, device=DEV)
        rc = fn(n, prec, x.data_ptr(), out.data_ptr(), stream)
        assert rc == 0, (call, rc)
        torch.cuda.synchronize()
        got = float(out)
        assert abs(got - ref) <= tol * abs(ref), (call, got, ref)
        # the oracle's TV of the same stored image
        orc = oracle.tv(x.double().cpu().numpy())
        assert abs(got - orc) <= tol * abs(orc), (call, got, orc)


def test_static_scratch_refuses_oversize():
    fn = _entry()
    x = torch.zeros((1025, 1025), dtype=torch.float32, device=DEV)
    out = torch.zeros((), dtype=torch.float64, device=DEV)
    rc = fn(1025, scg.F32, x.data_ptr(), out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert rc == -5          # SCG_ERR_UNSUPPORTED
