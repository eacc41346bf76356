"""Differentiation through the hand-written adjoint (torch.autograd.Function).

Least-squares fit loss = ||leg2cheb(x) - y||^2 (the configuration of a
differentiable transform inside training): the gradient 2 A^T C^-1 (Ax - y)
is checked against the oracle's explicit transpose and against central
finite differences along random directions.
"""
import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lc():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2411_00033_gb300 as m
    return m


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-12), ("f64_df", 1e-12), ("f64_split", 1e-12)])
@pytest.mark.parametrize("fn,code", [("leg2cheb", oracle.L2C), ("cheb2leg", oracle.C2L)])
def test_fit_gradient_against_oracle_transpose(lc, dtype, tol, fn, code):
    n, batch = 4096, 8
    x, y = workloads.fit_pair(n, batch)
    dev = torch.device("cuda", 0)
    xt = torch.as_tensor(x, device=dev).requires_grad_(True)
    yt = torch.as_tensor(y, device=dev)
    z = getattr(lc, fn)(xt, dtype=dtype)
    loss = ((z - yt) ** 2).sum()
    loss.backward()
    g = xt.grad.cpu().numpy()
    for b in range(batch):
        r = 2.0 * (oracle.apply(code, x[b]) - y[b])
        want = oracle.apply(code, r, adjoint=True)
        err = np.linalg.norm(g[b] - want) / np.linalg.norm(want)
        assert err <= tol, (b, err)


def test_fit_gradient_finite_differences(lc):
    n, batch = 2048, 4
    x, y = workloads.fit_pair(n, batch)
    dev = torch.device("cuda", 0)
    xt = torch.as_tensor(x, device=dev).requires_grad_(True)
    yt = torch.as_tensor(y, device=dev)

    def loss_of(v):
        return ((lc.leg2cheb(v) - yt) ** 2).sum()

    loss = loss_of(xt)
    loss.backward()
    g = xt.grad.detach()
    rng = np.random.default_rng(4)
    eps = 1e-6
    for _ in range(16):
        d = torch.as_tensor(rng.standard_normal((batch, n)), device=dev)
        with torch.no_grad():
            fd = (loss_of(xt + eps * d) - loss_of(xt - eps * d)) / (2 * eps)
        an = (g * d).sum()
        assert abs(float(fd - an)) <= 1e-6 * max(1.0, abs(float(an))), (float(fd), float(an))


def test_fp32_fit_gradient(lc):
    n, batch = 65536, 4
    x, y = workloads.fit_pair(n, batch)
    dev = torch.device("cuda", 0)
    xt = torch.as_tensor(x, device=dev, dtype=torch.float32).requires_grad_(True)
    yt = torch.as_tensor(y, device=dev, dtype=torch.float32)
    loss = ((lc.leg2cheb(xt) - yt) ** 2).sum()
    loss.backward()
    g = xt.grad.double().cpu().numpy()
    rows = workloads.sample_rows(n, 256)
    for b in range(batch):
        r = 2.0 * (oracle.apply(oracle.L2C, x[b].astype(np.float32).astype(np.float64)) - y[b].astype(np.float32))
        want = oracle.apply(oracle.L2C, r, rows=rows, adjoint=True)
        err = np.linalg.norm(g[b][rows] - want) / np.linalg.norm(want)
        assert err <= 2e-5, (b, err)
