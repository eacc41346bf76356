"""Tensor-product transforms of 3-D arrays along each axis, one call per axis.

Axes 0 and 2 of a C-order array take one batch stride (lc_execute); the
middle axis takes the two-level batch of lc_execute_ex (inner index stride 1,
outer index stride n*Q).  Every fibre is checked against the CPU oracle:
E_2 <= 1e-13 for the FP64-output tiers, 2e-6 for the FP32 tier (against the
oracle on the FP32-rounded input).
"""
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


def _array(shape, seed):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(shape)
    for ax, m in enumerate(shape):  # N(0,1) / ((i+1)(j+1)(k+1)), as the 512^3 workload
        w = 1.0 / np.arange(1, m + 1, dtype=np.float64)
        x *= w.reshape([-1 if a == ax else 1 for a in range(3)])
    return x


@pytest.mark.parametrize("shape", [(32, 32, 32), (20, 300, 12)])
@pytest.mark.parametrize("adjoint", [False, True])
@pytest.mark.parametrize("tier", ["f64", "f64_df", "f64_split", "f32"])
def test_every_axis_one_call(lc, tier, adjoint, shape):
    x = _array(shape, seed=4)
    dev = torch.device("cuda", 0)
    dt = torch.float32 if tier == "f32" else torch.float64
    xt = torch.as_tensor(x, device=dev, dtype=dt).contiguous()
    xr = xt.double().cpu().numpy()  # the values the transform sees
    tol = 2e-6 if tier == "f32" else 1e-13
    for direction, code in (("l2c", oracle.L2C), ("c2l", oracle.C2L)):
        for axis in range(3):
            n = shape[axis]
            batch = int(np.prod(shape)) // n
            plan = lc.Plan(n, direction, batch, tier, dev)
            z = plan.along_axis(xt, axis, adjoint=adjoint).double().cpu().numpy()
            zf = np.moveaxis(z, axis, -1).reshape(-1, n)
            xf = np.moveaxis(xr, axis, -1).reshape(-1, n)
            worst = 0.0
            for b in range(batch):
                e2, _ = rel_errors(zf[b], oracle.apply(code, xf[b], adjoint=adjoint))
                worst = max(worst, e2)
            assert worst <= tol, (tier, direction, axis, adjoint, worst)


def test_two_level_batch_validation(lc):
    dev = torch.device("cuda", 0)
    plan = lc.Plan(64, "l2c", 12, "f64", dev)
    x = torch.zeros(12 * 64, dtype=torch.float64, device=dev)
    out = torch.zeros_like(x)
    bad = [((1, 4, 256), (1, 4, 256), 0),    # batch_inner < 1
           ((1, 4, 256), (1, 4, 256), 13),   # batch_inner > batch
           ((1, 4, 256), (1, 4, 0), 4),      # outer output stride 0 with 3 groups
           ((1, 4, 256), (0, 4, 256), 4),    # inner output stride 0 with 4 per group
           ((1, 4, 256), (1, 0, 256), 4),    # element output stride 0
           ((-1, 4, 256), (1, 4, 256), 4)]   # negative stride
    for si, so, inner in bad:
        with pytest.raises(lc.LegChebError) as e:
            plan.execute_strided2(x, out, si, so, inner)
        assert e.value.status == 1, (si, so, inner)
    # batch_inner equal to the batch is the one-stride layout
    X = torch.as_tensor(workloads.decaying_vector(64, seed=3, batch=12), device=dev)
    a = plan(X)
    b = torch.empty_like(X)
    plan.execute_strided2(X, b, (64, 1, 0), (64, 1, 0), batch_inner=12)
    assert torch.equal(a, b)
