"""Pins for the CPU oracle: each check comes from outside the oracle itself.

* Brute force through a different route (Sec. 1, eq:fx): evaluate the
  Legendre series at the n Chebyshev-Gauss nodes in 50-digit arithmetic and
  take the discrete Chebyshev transform, which is exact for degree < n.
* Textbook Legendre expansions (P_2, P_3, P_4 in the Chebyshev basis).
* Structure of A (eq:aij, eq:hik, eq:matH): upper triangular, zero on odd
  diagonals, diagonal-wise product form.
* Lambda against 50-digit Gamma ratios (eq:Lambda).
* C2L as the inverse map: A^{-1}C from a 50-digit solve (eq:directmv), and
  the round trip leg -> cheb -> leg (Sec. 5.1).
* Adjoint: dot test and explicit transpose.
"""
import numpy as np
import pytest

import oracle
from oracle import L2C, C2L
import workloads

mp = pytest.importorskip("mpmath")


def _brute_l2c(f, dps=50):
    """f^cheb from f^leg via values at Chebyshev-Gauss nodes (exact for deg < n)."""
    n = len(f)
    with mp.workdps(dps):
        xs = [mp.cos((m + mp.mpf(1) / 2) * mp.pi / n) for m in range(n)]
        vals = []
        for x in xs:
            # Legendre three-term recurrence (Bonnet)
            p0, p1 = mp.mpf(1), x
            acc = mp.mpf(f[0]) * p0
            if n > 1:
                acc += mp.mpf(f[1]) * p1
            for j in range(1, n - 1):
                p0, p1 = p1, ((2 * j + 1) * x * p1 - j * p0) / (j + 1)
                acc += mp.mpf(f[j + 1]) * p1
            vals.append(acc)
        out = []
        for k in range(n):
            s = mp.fsum(vals[m] * mp.cos(k * (m + mp.mpf(1) / 2) * mp.pi / n) for m in range(n))
            ck = 2 if k == 0 else 1
            out.append(float(2 * s / (ck * n)))
    return np.array(out)


def _mp_A(n):
    """A (eq:aij) as an mpmath matrix, from Gamma directly."""
    A = mp.zeros(n, n)
    for i in range(n):
        for j in range(i, n, 2):
            a = mp.gamma(mp.mpf(j - i) / 2 + mp.mpf(1) / 2) / mp.gamma(mp.mpf(j - i) / 2 + 1)
            b = mp.gamma(mp.mpf(j + i) / 2 + mp.mpf(1) / 2) / mp.gamma(mp.mpf(j + i) / 2 + 1)
            A[i, j] = a * b
    return A


@pytest.mark.parametrize("n", [1, 2, 3, 8, 17, 40])
def test_l2c_matches_gauss_node_bruteforce(n):
    f = np.random.default_rng(100 + n).uniform(-1, 1, n)
    want = _brute_l2c(f)
    got = oracle.apply(L2C, f)
    scale = max(np.abs(want).max(), 1e-300)
    assert np.abs(got - want).max() <= 4e-16 * scale


def test_textbook_legendre_expansions():
    # P2 = T0/4 + 3 T2/4 ; P3 = 3 T1/8 + 5 T3/8 ; P4 = 9 T0/64 + 5 T2/16 + 35 T4/64
    cases = {2: {0: 1 / 4, 2: 3 / 4}, 3: {1: 3 / 8, 3: 5 / 8}, 4: {0: 9 / 64, 2: 5 / 16, 4: 35 / 64}}
    for j, coeffs in cases.items():
        e = np.zeros(6)
        e[j] = 1.0
        z = oracle.apply(L2C, e)
        want = np.zeros(6)
        for k, v in coeffs.items():
            want[k] = v
        assert np.abs(z - want).max() <= 2e-16, (j, z)


def test_structure_of_A():
    n = 23
    for d in (L2C, C2L):
        M = oracle.dense_matrix(d, n)
        for i in range(n):
            for j in range(n):
                if j < i or (j - i) % 2:
                    assert M[i, j] == 0.0
                else:
                    assert M[i, j] != 0.0


@pytest.mark.parametrize("i,k", [(0, 0), (1, 0), (0, 5), (7, 3), (1000, 17), (123456, 40), (999000, 499)])
def test_diagonal_product_form(i, k):
    # (C^{-1}A)_{i,i+2k} = 2/(c_i pi) Lambda(k) Lambda(i+k)   (eq:hik)
    n = i + 2 * k + 1
    got = oracle.entry(L2C, n, i, i + 2 * k)
    lam = lambda z: mp.gamma(z + mp.mpf(1) / 2) / mp.gamma(z + 1)
    with mp.workdps(40):
        want = lam(k) * lam(i + k) * (1 if i == 0 else 2) / mp.pi
    assert abs(got - float(want)) <= 2.3e-16 * abs(float(want))


@pytest.mark.parametrize("k", list(range(0, 65)) + [1000, 100000, 999999])
def test_lambda_against_gamma(k):
    hi, lo = oracle.lambda_table(k + 1)
    with mp.workdps(40):
        want = mp.gamma(k + mp.mpf(1) / 2) / mp.gamma(k + 1)
        err = abs((mp.mpf(hi[k]) + mp.mpf(lo[k])) - want) / want
    assert float(err) < 1e-28
    assert abs(hi[k] - float(want)) <= 0.5000001 * np.spacing(float(want))


def test_c2l_is_inverse_map_mpmath():
    # A^{-1} C computed by a 50-digit solve equals the oracle's C2L matrix.
    n = 24
    with mp.workdps(50):
        A = _mp_A(n)
        C = mp.diag([mp.pi if i == 0 else mp.pi / 2 for i in range(n)])
        X = mp.inverse(A) * C
        want = np.array([[float(X[i, j]) for j in range(n)] for i in range(n)])
    got = oracle.dense_matrix(C2L, n)
    assert np.abs(got - want).max() <= 4e-16 * np.abs(want).max()
    assert got[0, 0] == 1.0


@pytest.mark.parametrize("n,r", [(1, 0.0), (2, 0.0), (5, 0.5), (1024, 0.0), (4096, 0.5)])
def test_round_trip(n, r):
    x = np.random.default_rng(7).uniform(0, 1, n) * np.arange(1, n + 1) ** (-r)
    back = oracle.apply(C2L, oracle.apply(L2C, x))
    assert np.abs(back - x).max() <= 4e-15 * np.abs(x).max()


@pytest.mark.parametrize("d", [L2C, C2L])
def test_adjoint_dot_and_transpose(d):
    n = 301
    rng = np.random.default_rng(11)
    x, y = rng.standard_normal(n), rng.standard_normal(n)
    Mx = oracle.apply(d, x)
    Mty = oracle.apply(d, y, adjoint=True)
    lhs, rhs = float(Mx @ y), float(x @ Mty)
    assert abs(lhs - rhs) <= 1e-13 * max(abs(lhs), np.abs(Mx).max() * np.abs(y).sum())
    M = oracle.dense_matrix(d, 64)
    yy = rng.standard_normal(64)
    assert np.abs(oracle.apply(d, yy, adjoint=True) - M.T @ yy).max() <= 1e-14 * np.abs(M.T @ yy).max()


def test_sampled_rows_equal_full_rows():
    n = 5000
    x = workloads.decaying_vector(n, seed=1)
    rows = workloads.sample_rows(n, count=64)
    for d in (L2C, C2L):
        full = oracle.apply(d, x)
        part = oracle.apply(d, x, rows=rows)
        assert np.array_equal(full[rows], part)
        fullT = oracle.apply(d, x, adjoint=True)
        partT = oracle.apply(d, x, rows=rows, adjoint=True)
        assert np.array_equal(fullT[rows], partT)


def test_planted_mistakes_fail_the_pins():
    # A pin is only useful if plausible mistakes fail it.  Apply mistakes to
    # the oracle's own output and check that the brute force rejects them.
    n = 17
    f = np.random.default_rng(5).uniform(-1, 1, n)
    want = _brute_l2c(f)
    good = oracle.apply(L2C, f)
    M = oracle.dense_matrix(L2C, n)
    mistakes = {
        "row0 C^-1 dropped": good * np.where(np.arange(n) == 0, np.pi, 1.0) / 1.0,
        "C applied instead of C^-1": good * np.where(np.arange(n) == 0, np.pi ** 2, (np.pi / 2) ** 2),
        "transposed operand": M.T @ f,
        "odd diagonal kept": good + np.roll(good, 1) * 1e-3,
    }
    for name, bad in mistakes.items():
        assert np.abs(bad - want).max() > 1e-6 * np.abs(want).max(), name
