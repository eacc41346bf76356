"""The nodal variant (eq:AijLag, plan option `nodal`) against the oracle.

The nodal far field represents each block by the kernel's values at the
M x M Chebyshev-Gauss node pairs with Lagrange bases, the method of Alpert
and Rokhlin that the paper's modal method replaces.  Both interpolate the
kernel at the same nodes, so they are the same approximation: the nodal
plans must meet the same gates as the modal ones, and their block matrices
must be the modal ones before the 2-D DCT of eq:aklmore.
"""
import numpy as np
import pytest

import oracle
import workloads
from gpu_util import rel_errors

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

M = 18
DIRS = [("l2c", oracle.L2C), ("c2l", oracle.C2L)]


@pytest.fixture(scope="module")
def lc():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2411_00033_gb300 as m
    return m


def _dev():
    return torch.device("cuda", 0)


def _nodes():
    return np.cos((np.arange(M) + 0.5) * np.pi / M)


def _cheb(j, X):
    return np.cos(j * np.arccos(np.clip(X, -1, 1)))


def test_leaf_matrix_reproduces_polynomials(lc):
    # T(sigma)_{mk} = l_k(X_m): sum_k p(X_k) l_k(X) = p(X) for every p of degree < M
    plan = lc.Plan(5000, "l2c", 1, "f64", _dev(), nodal=True)
    s = plan.info["s"]
    T = plan.table(1).reshape(2, s, M)
    Xn = _nodes()
    for sigma in (0, 1):
        X = -1 + (2 * np.arange(s) + sigma) / s
        assert np.abs(T[sigma].sum(axis=1) - 1.0).max() < 1e-14
        for j in (1, 5, 11, M - 1):
            assert np.abs(T[sigma] @ _cheb(j, Xn) - _cheb(j, X)).max() < 1e-13, (sigma, j)


def test_level_maps_reproduce_polynomials(lc):
    # P(l)_{kj} = l_k((X_j + 2l - 1)/2): the parent's basis at child l's nodes
    plan = lc.Plan(5000, "l2c", 1, "f64", _dev(), nodal=True)
    P = plan.table(2).reshape(2, M, M)
    Xn = _nodes()
    for l in (0, 1):
        Y = 0.5 * (Xn + 2 * l - 1)
        for j in (0, 1, 7, M - 1):
            # sum_k p(X_k) l_k(Y_j) = p(Y_j)
            assert np.abs(_cheb(j, Xn) @ P[l] - _cheb(j, Y)).max() < 1e-13, (l, j)


@pytest.mark.parametrize("direction", ["l2c", "c2l"])
@pytest.mark.parametrize("alpha", [None, 0.25])
def test_blocks_are_the_modal_blocks_before_the_dct(lc, direction, alpha):
    # eq:aklmore: modal A-hat = 4/(c_k c_l M^2) C S C^T with S the nodal block
    # (the kernel at the node pairs) and C_km = cos(k (m+1/2) pi/M)
    n = 20000
    opts = {} if alpha is None else {"alpha": alpha}
    nod = lc.Plan(n, direction, 1, "f64", _dev(), nodal=True, **opts)
    mod = lc.Plan(n, direction, 1, "f64", _dev(), **opts)
    nc = nod.info["n_c"]
    S = nod.table(3).reshape(nc, M, M)
    A = mod.table(3).reshape(nc, M, M)
    C = np.cos(np.outer(np.arange(M), np.arange(M) + 0.5) * np.pi / M)
    w = np.full(M, 1.0)
    w[0] = 0.5
    scale = 4.0 / M ** 2 * np.outer(w, w)
    got = scale * np.einsum("km,bmn,ln->bkl", C, S, C)
    big = np.abs(A).reshape(nc, -1).max(axis=1)
    err = (np.abs(got - A).reshape(nc, -1).max(axis=1) / big).max()
    assert err < 1e-14, err


@pytest.mark.parametrize("direction,code", DIRS)
@pytest.mark.parametrize("n", [1, 100, 129, 1000, 4097, 33333])
def test_f64_matches_oracle(lc, n, direction, code):
    x = workloads.decaying_vector(n, seed=n + 3, r=0.5)
    z = lc.Plan(n, direction, 1, "f64", _dev(), nodal=True)(torch.as_tensor(x, device=_dev())).cpu().numpy()
    e2, einf = rel_errors(z, oracle.apply(code, x))
    assert e2 <= 1e-13, (n, direction, e2, einf)


@pytest.mark.parametrize("direction,code", DIRS)
def test_adjoint_and_batch(lc, direction, code):
    n, batch = 5000, 3
    X = workloads.decaying_vector(n, seed=9, r=0.5, batch=batch)
    xt = torch.as_tensor(X, device=_dev())
    plan = lc.Plan(n, direction, batch, "f64", _dev(), nodal=True)
    Z = plan(xt).cpu().numpy()
    G = plan.execute(xt, adjoint=True).cpu().numpy()
    for b in range(batch):
        e2, _ = rel_errors(Z[b], oracle.apply(code, X[b]))
        assert e2 <= 1e-13, (b, e2)
        e2, _ = rel_errors(G[b], oracle.apply(code, X[b], adjoint=True))
        assert e2 <= 1e-13, (b, e2)


@pytest.mark.parametrize("direction,code", DIRS)
def test_f32_tier(lc, direction, code):
    n = 40000
    x = workloads.decaying_vector(n, seed=4, r=0.5)
    z = lc.Plan(n, direction, 1, "f32", _dev(), nodal=True)(
        torch.as_tensor(x, device=_dev(), dtype=torch.float32)).double().cpu().numpy()
    e2, _ = rel_errors(z, oracle.apply(code, x))
    assert e2 <= 2e-6, e2


@pytest.mark.parametrize("direction,code", DIRS)
def test_gegenbauer_nodal(lc, direction, code):
    n, a = 7000, 1.6
    x = workloads.decaying_vector(n, seed=5, r=1.0)
    z = lc.Plan(n, direction, 1, "f64", _dev(), nodal=True, alpha=a)(torch.as_tensor(x, device=_dev())).cpu().numpy()
    e2, _ = rel_errors(z, oracle.apply(code, x, alpha=a))
    assert e2 <= 1e-13, e2


def test_nodal_and_modal_agree(lc):
    n = 300000
    x = torch.as_tensor(workloads.decaying_vector(n, seed=6, r=1.0), device=_dev())
    for d in ("l2c", "c2l"):
        a = lc.Plan(n, d, 1, "f64", _dev(), nodal=True)(x).cpu().numpy()
        b = lc.Plan(n, d, 1, "f64", _dev())(x).cpu().numpy()
        e2, _ = rel_errors(a, b)
        assert e2 <= 1e-14, (d, e2)


@pytest.mark.parametrize("dtype", ["f64_df", "f64_split"])
def test_other_tiers_unsupported(lc, dtype):
    with pytest.raises(Exception):
        lc.Plan(1000, "l2c", 2, dtype, _dev(), nodal=True)
