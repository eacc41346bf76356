"""Pins for the oracle's Gegenbauer maps (the generalisation the Conclusions
name: transforms between Gegenbauer bases C_j^(a), with Legendre at a = 1/2).

Each check comes from outside the oracle's own recursions:

* Point values: sum_j f_j C_j^(a)(x_m) (mpmath's Gegenbauer polynomials at 50
  digits) against the Chebyshev series sum_k z_k T_k(x_m) at the n
  Chebyshev-Gauss nodes, which fixes a polynomial of degree < n.  Both
  directions: L2C gives z from f; C2L gives f from z.
* a = 1: C^(1) = U, so Gegenbauer -> Chebyshev is U_j = sum of T's with
  weights 2/c_i (1 on the last), and T_j = (U_j - U_{j-2})/2.
* a = 1/2 is the Legendre map, which the oracle computes by another route
  (Lambda recursion, eq:Lxymod) and which has its own pins.
* Round trip C2L(L2C(f)) = f.
"""
import numpy as np
import pytest

import oracle
from oracle import L2C, C2L

mp = pytest.importorskip("mpmath")

ALPHAS = [-0.3, 0.25, 0.75, 1.0, 1.6, 2.0]


def _nodes(n):
    return [mp.cos((m + mp.mpf(1) / 2) * mp.pi / n) for m in range(n)]


def _geg_values(f, a, n):
    with mp.workdps(50):
        aa = mp.mpf(a)
        return [mp.fsum(mp.mpf(f[j]) * mp.gegenbauer(j, aa, x) for j in range(len(f))) for x in _nodes(n)]


def _cheb_values(z, n):
    with mp.workdps(50):
        return [mp.fsum(mp.mpf(z[k]) * mp.chebyt(k, x) for k in range(len(z))) for x in _nodes(n)]


@pytest.mark.parametrize("a", ALPHAS)
@pytest.mark.parametrize("n", [1, 2, 5, 16, 33])
def test_l2c_point_values(a, n):
    f = np.random.default_rng(700 + n).uniform(-1, 1, n)
    z = oracle.apply(L2C, f, alpha=a)
    want = np.array([float(v) for v in _geg_values(f, a, n)])
    got = np.array([float(v) for v in _cheb_values(z, n)])
    scale = max(np.abs(want).max(), 1e-300)
    assert np.abs(got - want).max() <= 1e-14 * scale, (a, n, np.abs(got - want).max() / scale)


@pytest.mark.parametrize("a", ALPHAS)
@pytest.mark.parametrize("n", [1, 2, 6, 17, 32])
def test_c2l_point_values(a, n):
    c = np.random.default_rng(800 + n).uniform(-1, 1, n)
    f = oracle.apply(C2L, c, alpha=a)
    want = np.array([float(v) for v in _cheb_values(c, n)])
    got = np.array([float(v) for v in _geg_values(f, a, n)])
    scale = max(np.abs(want).max(), 1e-300)
    assert np.abs(got - want).max() <= 1e-14 * scale, (a, n, np.abs(got - want).max() / scale)


def test_second_kind_closed_forms():
    # C^(1)_j = U_j = 2 sum_{i <= j, j-i even} T_i, with T_0 counted once
    n = 40
    f = np.random.default_rng(3).standard_normal(n)
    z = oracle.apply(L2C, f, alpha=1.0)
    want = np.array([(1.0 if i == 0 else 2.0) * f[i::2].sum() for i in range(n)])
    assert np.abs(z - want).max() <= 4e-15 * np.abs(want).max()
    # T_0 = U_0, T_1 = U_1 / 2, T_j = (U_j - U_{j-2})/2: coefficient of U_i is
    # c_i/2 - c_{i+2}/2 (i >= 1), c_0 - c_2/2 (i = 0)
    c = np.random.default_rng(4).standard_normal(n)
    g = oracle.apply(C2L, c, alpha=1.0)
    cp = np.concatenate([c, [0.0, 0.0]])
    want = np.array([(cp[i] if i == 0 else 0.5 * cp[i]) - 0.5 * cp[i + 2] for i in range(n)])
    assert np.abs(g - want).max() <= 4e-15 * np.abs(want).max()


@pytest.mark.parametrize("d", [L2C, C2L])
def test_half_is_legendre(d):
    x = np.random.default_rng(5).standard_normal(777)
    a = oracle.apply(d, x)
    b = oracle.apply(d, x, alpha=0.5)
    assert np.abs(a - b).max() <= 4e-16 * np.abs(a).max()
    for (i, j) in [(0, 0), (0, 2), (3, 9), (100, 500)]:
        e0, e1 = oracle.entry(d, 600, i, j), oracle.entry_geg(d, 0.5, 600, i, j)
        assert abs(e0 - e1) <= 4e-16 * max(abs(e0), 1e-300)


@pytest.mark.parametrize("a", [-0.3, 0.25, 1.6])
def test_entries_against_gamma_ratios(a):
    # the closed forms through Gamma functions (50 digits), a route without
    # the ratio recursions: L2C (2/c_i) G(l+a)G(m+a)/(G(a)^2 l! m!);
    # C2L (2i+2a) j G(a) G(l-a) G(m) / (4 G(-a) l! G(m+a+1))
    n = 400
    with mp.workdps(50):
        A = mp.mpf(a)
        for (i, j) in [(0, 2), (1, 7), (10, 10), (12, 300), (0, 398)]:
            l, m = (j - i) // 2, (j + i) // 2
            want = (1 if i == 0 else 2) * mp.gamma(l + A) * mp.gamma(m + A) / (
                mp.gamma(A) ** 2 * mp.factorial(l) * mp.factorial(m))
            got = oracle.entry_geg(L2C, a, n, i, j)
            assert abs(got - float(want)) <= 3e-16 * abs(float(want)), (i, j)
            want = (2 * i + 2 * A) * j * mp.gamma(A) * mp.gamma(l - A) * mp.gamma(m) / (
                4 * mp.gamma(-A) * mp.factorial(l) * mp.gamma(m + A + 1))
            got = oracle.entry_geg(C2L, a, n, i, j)
            assert abs(got - float(want)) <= 3e-16 * abs(float(want)), (i, j)


@pytest.mark.parametrize("a", [-0.3, 0.25, 1.5])
def test_round_trip(a):
    n = 1500
    f = np.random.default_rng(6).standard_normal(n) / np.arange(1, n + 1)
    g = oracle.apply(C2L, oracle.apply(L2C, f, alpha=a), alpha=a)
    assert np.abs(g - f).max() <= 1e-13 * np.abs(f).max()


def test_adjoint_is_transpose():
    n = 60
    for d in (L2C, C2L):
        M = oracle.dense_matrix(d, n, alpha=0.3)
        r = np.random.default_rng(7).standard_normal(n)
        assert np.abs(oracle.apply(d, r, adjoint=True, alpha=0.3) - M.T @ r).max() <= 1e-14 * np.abs(M.T @ r).max()


def test_planted_mistakes_fail_the_point_values():
    # plausible slips in the Gegenbauer entries must fail the node pin
    a, n = 0.3, 12
    f = np.random.default_rng(8).uniform(-1, 1, n)
    want = np.array([float(v) for v in _geg_values(f, a, n)])
    M = oracle.dense_matrix(L2C, n, alpha=a)
    Mleg = oracle.dense_matrix(L2C, n)
    mistakes = {
        "row 0 doubled": M @ f + np.where(np.arange(n) == 0, (M @ f)[0], 0.0),
        "transposed": M.T @ f,
        "Legendre entries": Mleg @ f,
        "alpha sign": oracle.dense_matrix(L2C, n, alpha=-a) @ f,
    }
    for name, z in mistakes.items():
        got = np.array([float(v) for v in _cheb_values(z, n)])
        assert np.abs(got - want).max() > 1e-6 * np.abs(want).max(), name
    c = np.random.default_rng(9).uniform(-1, 1, n)
    C = oracle.dense_matrix(C2L, n, alpha=a)
    wantc = np.array([float(v) for v in _cheb_values(c, n)])
    for name, g in {"(2i+1) kept": np.diag((2 * np.arange(n) + 1) / (2 * np.arange(n) + 2 * a)) @ C @ c,
                    "transposed": C.T @ c}.items():
        got = np.array([float(v) for v in _geg_values(g, a, n)])
        assert np.abs(got - wantc).max() > 1e-6 * np.abs(wantc).max(), name
