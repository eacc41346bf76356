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


# ---- values at Chebyshev points (the synthesis and its inverse)
def _mp_values(f, dps=50):
    """p(x_m) for p = sum_j f_j P_j at the n Chebyshev-Gauss nodes, 50 digits,
    exact nodes, Bonnet's recurrence: a route that never forms C^{-1}A or a
    cosine sum."""
    n = len(f)
    with mp.workdps(dps):
        out = []
        for m in range(n):
            x = mp.cos((m + mp.mpf(1) / 2) * mp.pi / n)
            p0, p1 = mp.mpf(1), x
            acc = mp.mpf(f[0])
            if n > 1:
                acc += mp.mpf(f[1]) * p1
            for j in range(1, n - 1):
                p0, p1 = p1, ((2 * j + 1) * x * p1 - j * p0) / (j + 1)
                acc += mp.mpf(f[j + 1]) * p1
            out.append(float(acc))
    return np.array(out)


@pytest.mark.parametrize("n", [1, 2, 3, 8, 16, 33, 64])
def test_synthesis_matches_node_evaluation(n):
    f = np.random.default_rng(300 + n).uniform(-1, 1, n)
    want = _mp_values(f)
    got = oracle.synthesis(f)
    scale = max(np.abs(want).max(), 1e-300)
    assert np.abs(got - want).max() <= 1e-15 * scale, (n, np.abs(got - want).max() / scale)


def test_chebyshev_values_closed_forms():
    # T_0 is 1 at every node, T_1 is the node itself, T_k(x_m) = cos(k (m+1/2) pi/n),
    # and at k = n the nodes are the zeros of T_n (so T_n would vanish, not tested: k < n)
    def cheb_at_nodes(k, n):
        with mp.workdps(50):
            return np.array([float(mp.cos(k * (m + mp.mpf(1) / 2) * mp.pi / n)) for m in range(n)])
    for n in (1, 2, 7, 64, 1000):
        nodes = cheb_at_nodes(1, n)
        e = np.zeros(n)
        e[0] = 1.0
        assert np.abs(oracle.dct(0, e) - 1.0).max() == 0.0
        if n > 1:
            e[:] = 0.0
            e[1] = 1.0
            assert np.abs(oracle.dct(0, e) - nodes).max() <= 2.3e-16
            k = n - 1
            e[:] = 0.0
            e[k] = 1.0
            assert np.abs(oracle.dct(0, e) - cheb_at_nodes(k, n)).max() <= 2.3e-16


@pytest.mark.parametrize("n", [1, 5, 64, 500])
def test_values_round_trip_and_inverse(n):
    # discrete orthogonality makes kind 1 the exact inverse of kind 0 for degree < n;
    # analysis(synthesis(f)) returns the Legendre coefficients
    rng = np.random.default_rng(400 + n)
    c = rng.standard_normal(n)
    assert np.abs(oracle.dct(1, oracle.dct(0, c)) - c).max() <= 4e-15 * max(1.0, np.abs(c).max())
    f = rng.standard_normal(n) / np.arange(1, n + 1) ** 0.5
    assert np.abs(oracle.analysis(oracle.synthesis(f)) - f).max() <= 4e-14 * np.abs(f).max()


def test_values_planted_mistakes_fail():
    # a dropped half-node offset or a missing k = 0 weight would not match the node evaluation
    n = 16
    f = np.random.default_rng(9).uniform(-1, 1, n)
    want = _mp_values(f)
    c = oracle.apply(L2C, f)
    m = np.arange(n)[:, None]
    k = np.arange(n)[None, :]
    wrong_nodes = np.cos(k * m * np.pi / n) @ c
    assert np.abs(wrong_nodes - want).max() > 1e-3
    ca = oracle.dct(1, want)
    ca_bad = ca.copy()
    ca_bad[0] *= 2
    assert np.abs(oracle.apply(C2L, ca_bad) - f).max() > 1e-3


def test_dct_sampled_rows_equal_full_rows():
    x = np.random.default_rng(410).standard_normal(700)
    rows = np.array([0, 1, 5, 349, 698, 699], np.int64)
    for kind in (0, 1):
        assert np.array_equal(oracle.dct(kind, x)[rows], oracle.dct(kind, x, rows=rows))
