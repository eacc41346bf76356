"""The allocation-free entry point lc_direct_static, called through the C ABI.

Some callers cannot allocate device memory: their host application's memory
pool owns the device, or an allocation's implicit synchronisation is not
acceptable where they run.  lc_direct_static keeps its scratch in a static
device array instead.  Its output must match the plan-based lc_execute (the
existing entry point) and the CPU oracle within the tolerance of the other
parity tests (E_2 <= 1e-13), on two calls in a row that leave different
tables in the shared array, and at the largest size the array allows.  This
file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import oracle
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


def _static_call(lib, direction, x, out, ob=None, oe=None):
    f = lib.lc_direct_static
    f.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p]
    f.restype = ctypes.c_int
    batch, n = x.shape
    return f(direction, n, batch, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()),
             x.stride(0), x.stride(1), out.stride(0) if ob is None else ob, out.stride(1) if oe is None else oe,
             ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def _check_against_execute_and_oracle(lc, direction, code, X, got):
    dev = torch.device("cuda", 0)
    batch, n = X.shape
    xt = torch.as_tensor(X, device=dev)
    ref = lc.Plan(n, direction, batch, "f64", dev)(xt if batch > 1 else xt[0])
    torch.cuda.synchronize()
    want = ref.cpu().numpy().reshape(batch, n)
    for b in range(batch):
        e2, einf = rel_errors(got[b], want[b])
        assert e2 <= 1e-13, ("vs lc_execute", direction, n, b, e2, einf)
        e2, einf = rel_errors(got[b], oracle.apply(code, X[b]))
        assert e2 <= 1e-13, ("vs oracle", direction, n, b, e2, einf)


def test_static_scratch_matches_execute_and_oracle(lc):
    lib = lc.binding.load()
    dev = torch.device("cuda", 0)
    cases = [("l2c", lc.LC_L2C, oracle.L2C, 5000, 2), ("c2l", lc.LC_C2L, oracle.C2L, 3001, 1)]
    for direction, lcode, ocode, n, batch in cases:  # two calls in a row on the shared array
        X = np.stack([workloads.decaying_vector(n, seed=60 + b, r=0.5) for b in range(batch)])
        x = torch.as_tensor(X, device=dev)
        out = torch.full_like(x, float("nan"))
        assert _static_call(lib, lcode, x, out) == 0
        torch.cuda.synchronize()
        _check_against_execute_and_oracle(lc, direction, ocode, X, out.cpu().numpy())


def test_static_scratch_at_the_size_limit(lc):
    lib = lc.binding.load()
    dev = torch.device("cuda", 0)
    n = lc.binding.LC_STATIC_MAX_N
    X = workloads.decaying_vector(n, seed=61, r=0.5)[None, :]
    x = torch.as_tensor(X, device=dev)
    for direction, lcode, ocode in (("c2l", lc.LC_C2L, oracle.C2L), ("l2c", lc.LC_L2C, oracle.L2C)):
        out = torch.full_like(x, float("nan"))
        assert _static_call(lib, lcode, x, out) == 0
        torch.cuda.synchronize()
        _check_against_execute_and_oracle(lc, direction, ocode, X, out.cpu().numpy())


def test_static_scratch_rejects_bad_sizes_and_strides(lc):
    lib = lc.binding.load()
    dev = torch.device("cuda", 0)
    limit = lc.binding.LC_STATIC_MAX_N
    x = torch.zeros((1, limit + 1), dtype=torch.float64, device=dev)
    out = torch.full_like(x, 5.0)
    assert _static_call(lib, lc.LC_L2C, x, out) == 1      # LC_ERR_INVALID_ARG, nothing launched
    x2 = torch.ones((2, 100), dtype=torch.float64, device=dev)
    out2 = torch.full_like(x2, 5.0)
    assert _static_call(lib, lc.LC_L2C, x2, out2, oe=0) == 1  # every row of a vector on one address
    assert _static_call(lib, lc.LC_C2L, x2, out2, ob=0) == 1  # both vectors on one row
    torch.cuda.synchronize()
    assert bool((out == 5.0).all()) and bool((out2 == 5.0).all())
