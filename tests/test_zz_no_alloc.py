"""The allocation-free entry point lc_direct_static, called through the C ABI.

Some callers cannot allocate device memory (their host application's pool
owns the device, or an allocation's implicit synchronisation is not
acceptable where they run).  lc_direct_static keeps its scratch in a static
device array instead.  Its output must match lc_execute's (the plan-based
path) within the tolerance of the other parity tests (E_2 <= 1e-13), on two
calls in a row that leave different tables in the shared array.  This file is
collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import workloads
from gpu_util import rel_errors

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lc():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2411_00033_gb300 as m
    return m


def _static_call(lib, direction, x, out):
    f = lib.lc_direct_static
    f.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p]
    f.restype = ctypes.c_int
    batch, n = x.shape
    return f(direction, n, batch, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()),
             x.stride(0), x.stride(1), out.stride(0), out.stride(1),
             ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_static_scratch_matches_plan_execute(lc):
    lib = lc.binding.load()
    dev = torch.device("cuda", 0)
    cases = [("l2c", lc.LC_L2C, 5000, 2), ("c2l", lc.LC_C2L, 3001, 1)]
    for direction, code, n, batch in cases:  # two calls in a row on the shared array
        x = torch.as_tensor(np.stack([workloads.decaying_vector(n, seed=60 + b, r=0.5) for b in range(batch)]),
                            device=dev)
        out = torch.full_like(x, float("nan"))
        assert _static_call(lib, code, x, out) == 0
        ref = lc.Plan(n, direction, batch, "f64", dev)(x if batch > 1 else x[0])
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        want = ref.cpu().numpy().reshape(batch, n)
        for b in range(batch):
            e2, einf = rel_errors(got[b], want[b])
            assert e2 <= 1e-13, (direction, b, e2, einf)


def test_static_scratch_rejects_oversize(lc):
    lib = lc.binding.load()
    dev = torch.device("cuda", 0)
    limit = 16384
    x = torch.zeros((1, limit + 1), dtype=torch.float64, device=dev)
    out = torch.zeros_like(x)
    assert _static_call(lib, lc.LC_L2C, x, out) == 1      # LC_ERR_INVALID_ARG, nothing launched
    x2 = torch.zeros((1, limit), dtype=torch.float64, device=dev)
    assert _static_call(lib, lc.LC_C2L, x2, torch.zeros_like(x2)) == 0
    torch.cuda.synchronize()
