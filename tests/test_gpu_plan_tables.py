"""GPU plan tables against what the paper fixes.

* B(0), B(1): first rows printed in Appendix A.1 (eq:appT), and every entry
  equal (bitwise) to the exact rational W^{-1} V(0) W of Appendix A.3.
* lambda: the tau-series/recursion table of Sec. 4.3 within the paper's
  stated accuracy (relative error < 1e-15) of the oracle's double-double table.
* T(sigma): Chebyshev polynomials at X = -1 + (2m+sigma)/s (eq:Xs).
* A-hat: per submatrix, T A-hat T^T against the exact entries of the block
  (eq:Aoverline), block-relative error ~1e-14 for A (M = 18, Sec. 3.2).
"""
from fractions import Fraction
from math import comb
from pathlib import Path

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
GOLDEN = Path(__file__).resolve().parent / "golden"
M = 18


@pytest.fixture(scope="module")
def lc():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2411_00033_gb300 as m
    return m


def _exact_B0():
    """W^{-1} V(0) W in exact rationals (Appendix A.3)."""
    W = [[Fraction(0)] * M for _ in range(M)]
    Wi = [[Fraction(0)] * M for _ in range(M)]
    V = [[Fraction(0)] * M for _ in range(M)]
    for n in range(M):
        for j in range(n + 1):
            if (n - j) % 2 == 0:
                cj = 2 if j == 0 else 1
                W[n][j] = Fraction(2, cj * 2 ** n) * comb(n, (n - j) // 2)
                if n == 0:
                    Wi[n][j] = Fraction(1)
                else:
                    Wi[n][j] = Fraction(n * (-1) ** ((n - j) // 2) * 2 ** j, n + j) * comb((n + j) // 2, (n - j) // 2)
            V[n][j] = Fraction(comb(n, n - j) * (-1) ** (n - j), 2 ** n)
    def mul(a, b):
        return [[sum(a[i][k] * b[k][j] for k in range(M)) for j in range(M)] for i in range(M)]
    return mul(mul(Wi, V), W)


def _golden_rows():
    rows = {"B0": {}, "B1": {}}
    for line in (GOLDEN / "B_first_rows.txt").read_text().splitlines():
        if not line or line.startswith("#"):
            continue
        parts = line.split()
        rows[parts[0]][int(parts[1])] = [Fraction(p) for p in parts[2:]]
    return rows


def test_B_exact(lc):
    plan = lc.Plan(1024, "l2c", 1, "f64", torch.device("cuda", 0))
    B = plan.table(2).reshape(M, M)
    exact = _exact_B0()
    for i in range(M):
        for j in range(M):
            assert Fraction(B[i, j]) == exact[i][j], (i, j)
    gold = _golden_rows()
    for n, row in gold["B0"].items():
        assert [Fraction(v) for v in B[n, :n + 1]] == row
    B1 = np.array([[B[k, j] * (-1) ** (k - j) for j in range(M)] for k in range(M)])
    for n, row in gold["B1"].items():
        assert [Fraction(v) for v in B1[n, :n + 1]] == row


def test_lambda_accuracy(lc):
    n = 1 << 20
    plan = lc.Plan(n, "l2c", 1, "f64", torch.device("cuda", 0))
    lam = plan.table(0)
    hi, lo = oracle.lambda_table(plan.info["N"])
    rel = np.abs((lam - hi) - lo) / hi
    assert rel.max() < 1e-15, rel.max()
    ulp = np.abs(lam - hi) / np.spacing(hi)
    assert ulp.max() <= 5


def test_c2l_near_field_tables(lc):
    # u_k = Lambda(k)/(1 - 2k) and v_m = 1/(2m(2m+1) Lambda(m)), the factors of
    # L(i, i+2k) = (2i+1)(i+2k) u_k v_(i+k) (eq:Lxymod), against the oracle's
    # double-double lambda: lambda's own error (up to 5 ulp, test above) and
    # the four roundings of the table kernel, below 2e-15 relative
    n = 1 << 20
    plan = lc.Plan(n, "c2l", 1, "f64", torch.device("cuda", 0))
    N = plan.info["N"]
    u, v = plan.table(4), plan.table(5)
    hi, lo = oracle.lambda_table(N)
    k = np.arange(N, dtype=np.float64)
    lam = hi + lo
    u_ref = lam / (1.0 - 2.0 * k)
    ru = np.abs(u - u_ref) / np.abs(u_ref)
    assert ru.max() < 2e-15, ru.max()
    assert v[0] == 0.0
    v_ref = 1.0 / (2.0 * k[1:] * (2.0 * k[1:] + 1.0) * lam[1:])
    rv = np.abs(v[1:] - v_ref) / v_ref
    assert rv.max() < 2e-15, rv.max()


def test_T_matrix(lc):
    plan = lc.Plan(1000, "l2c", 1, "f64", torch.device("cuda", 0))
    s = plan.info["s"]
    T = plan.table(1).reshape(2, s, M)
    for sigma in range(2):
        X = -1 + (2 * np.arange(s) + sigma) / s
        ref = np.cos(np.outer(np.arccos(np.clip(X, -1, 1)), np.arange(M)))
        assert np.abs(T[sigma] - ref).max() < 1e-13


def _exact_block(code, lam, i0, j0, h, sigma):
    rows = i0 + 2 * np.arange(h) + sigma
    cols = j0 + 2 * np.arange(h) + sigma
    I, J = np.meshgrid(rows, cols, indexing="ij")
    k = (J - I) // 2
    if code == oracle.L2C:
        return lam[k] * lam[I + k]
    # L(i, j) of eq:Lxymod written out at x = i, y = j
    return (2 * I + 1) * J / ((I + J) * (I + J + 1.0) * (I - J + 1.0)) * lam[k] / lam[I + k]


@pytest.mark.parametrize("direction,code,tol", [("l2c", oracle.L2C, 3e-14), ("c2l", oracle.C2L, 1e-12)])
def test_ahat_block_approximation(lc, direction, code, tol):
    n = 4096
    plan = lc.Plan(n, direction, 1, "f64", torch.device("cuda", 0))
    L, s, nc = plan.info["L"], plan.info["s"], plan.info["n_c"]
    Ah = plan.table(3).reshape(nc, M, M)
    hi, lo = oracle.lambda_table(plan.info["N"])
    lam = hi
    worst = 0.0
    aoff = lambda g: 3 * ((1 << (g + 1)) - 2 - g)
    for gamma in range(L):
        h = s << (L - gamma - 1)
        nb = (1 << (gamma + 1)) - 1
        for b in sorted({0, nb // 2, nb - 1}):
            for r, (p, q) in enumerate([(0, 0), (0, 1), (1, 1)]):
                i0, j0 = 2 * h * (2 * b + p), 2 * h * (2 * b + q + 2)
                for sigma in (0, 1):
                    X = -1 + (2 * np.arange(h) + sigma) / h
                    T = np.cos(np.outer(np.arccos(np.clip(X, -1, 1)), np.arange(M)))
                    approx = T @ Ah[aoff(gamma) + 3 * b + r] @ T.T
                    exact = _exact_block(code, lam, i0, j0, h, sigma)
                    worst = max(worst, np.abs(approx - exact).max() / np.abs(exact).max())
    assert worst <= tol, worst


@pytest.mark.parametrize("direction,head", [("l2c", 13), ("c2l", 16)])
@pytest.mark.parametrize("n", [200, 3000, 16385, 65536, 300000])
def test_ahat_tail_below_compact_head(lc, n, direction, head):
    """The double-float tier keeps trailing words only for the entries of
    A-hat with k + l <= head.  That rests on the entries, the 2-D Chebyshev
    coefficients of a kernel smooth across well-separated blocks, falling
    off geometrically in k + l: past the head every entry of every matrix is
    below 2e-9 of the matrix's largest, so its FP32 leading word alone
    carries it to 1e-16 of the matrix.  These n give leaf sizes s from 17 to 32."""
    plan = lc.Plan(n, direction, 1, "f64", torch.device("cuda", 0))
    nc = plan.info["n_c"]
    assert nc > 0
    Ah = np.abs(plan.table(3).reshape(nc, M, M))
    tail = np.add.outer(np.arange(M), np.arange(M)) > head
    peak = Ah.reshape(nc, -1).max(axis=1)
    assert (peak > 0).all()
    worst = (Ah[:, tail].max(axis=1) / peak).max()
    assert worst <= 2e-9, (plan.info["s"], worst)


@pytest.mark.parametrize("direction,head", [("l2c", 13), ("c2l", 16)])
@pytest.mark.parametrize("s", [4, 5, 6, 8, 11, 12, 16, 24, 40, 48, 63, 64])
def test_ahat_tail_below_compact_head_every_leaf_size(lc, s, direction, head):
    """The same property for leaf sizes s across the whole range the plan
    options accept (4..64), each with six levels, so that the double-float
    tier's compact A-hat is covered for every s it can be asked to use.  The
    smallest blocks (s = 4, C2L) reach 2.35e-9; the bound here, 4e-9, still
    keeps each tail entry's FP32 leading word within 2.4e-16 of its matrix."""
    plan = lc.Plan(s * 2 ** 8 - 1, direction, 1, "f64", torch.device("cuda", 0), fixed_s=s)
    assert plan.info["s"] == s and plan.info["L"] == 6
    nc = plan.info["n_c"]
    Ah = np.abs(plan.table(3).reshape(nc, M, M))
    tail = np.add.outer(np.arange(M), np.arange(M)) > head
    peak = Ah.reshape(nc, -1).max(axis=1)
    assert (peak > 0).all()
    worst = (Ah[:, tail].max(axis=1) / peak).max()
    assert worst <= (4e-9 if s == 4 else 2e-9), (s, worst)


def _compact_values(words, nc, direction):
    """Entries of the compact double-float A-hat (raw FP32 words): hi + lo where a
    trailing word is kept (k + l <= head), hi alone elsewhere."""
    head, per = (13, 436) if direction == "l2c" else (16, 484)
    w = words.view(np.float32)[: nc * per].reshape(nc, per).astype(np.float64)
    out = w[:, : M * M].reshape(nc, M, M).copy()
    pos = M * M
    for k in range(head + 1):
        cnt = head + 1 - k
        out[:, k, :cnt] += w[:, pos:pos + cnt]
        pos += cnt
    return out


@pytest.mark.parametrize("direction", ["l2c", "c2l"])
@pytest.mark.parametrize("n", [3000, 65536, 1000000])
def test_double_float_plan_matches_fp64_plan(lc, n, direction):
    # the double-float tier's compact A-hat built in double-float arithmetic
    # (default) against the one converted from the FP64 plan (fp64_plan=1):
    # within a few units of 2^-48 (3.6e-15) of each matrix's largest entry
    dev = torch.device("cuda", 0)
    fast = lc.Plan(n, direction, 1, "f64_df", dev)
    ref = lc.Plan(n, direction, 1, "f64_df", dev, fp64_plan=True)
    nc = fast.info["n_c"]
    a = _compact_values(fast.table(6), nc, direction)
    b = _compact_values(ref.table(6), nc, direction)
    peak = np.abs(b).reshape(nc, -1).max(axis=1)
    err = (np.abs(a - b).reshape(nc, -1).max(axis=1) / peak).max()
    assert err <= 2e-14, (n, direction, err)
    with pytest.raises(lc.LegChebError):
        fast.table(3)  # no FP64 A-hat behind the fast plan
