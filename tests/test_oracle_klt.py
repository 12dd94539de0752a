"""Pins of the oracle's setup-time math (Sec. 2 and Sec. 3 of the paper) against
facts fixed outside the oracle: the paper's Table 1, a library eigensolver, the
eigen-equation itself, and the rounding rule's definition."""
import numpy as np
import pytest

import golden_io

RHOS = [0.1, 0.2, 0.3, 0.4, 0.5, 0.6, 0.7, 0.8, 0.9, 0.95]


def markov(n, rho):
    i = np.arange(n)
    return rho ** np.abs(i[:, None] - i[None, :])


@pytest.mark.parametrize("n", [4, 8, 16, 32])
@pytest.mark.parametrize("rho", [0.1, 0.5, 0.8, 0.95])
def test_closed_form_matches_jacobi(orc, n, rho):
    """Two independent routes to the exact KLT agree (Sec. 2.1 closed form, Sec. 3 numeric)."""
    Kc, lc = orc.klt_closed_form(n, rho)
    Kj, lj = orc.klt_jacobi(n, rho)
    assert np.max(np.abs(Kc - Kj)) < 1e-12
    assert np.max(np.abs(lc - lj)) < 1e-12


@pytest.mark.parametrize("n", [4, 8, 16, 32])
@pytest.mark.parametrize("rho", [0.3, 0.9])
def test_closed_form_is_eigenbasis(orc, n, rho):
    """Each closed-form row k_i satisfies R k_i = lambda_i k_i; rows orthonormal;
    lambda strictly decreasing; sign rule K[i, 0] > 0; matches numpy's eigh."""
    K, lam = orc.klt_closed_form(n, rho)
    R = markov(n, rho)
    assert np.max(np.abs(R @ K.T - K.T * lam[None, :])) < 1e-12
    assert np.max(np.abs(K @ K.T - np.eye(n))) < 1e-12
    assert np.all(np.diff(lam) < 0)
    assert np.all(K[:, 0] > 0)
    w, V = np.linalg.eigh(R)
    assert np.max(np.abs(w[::-1] - lam)) < 1e-12
    V = V[:, ::-1].T
    V = V * np.sign(V[:, :1])
    assert np.max(np.abs(V - K)) < 1e-10


@pytest.mark.parametrize("n", [4, 8, 16, 32])
def test_klt_row_parity(orc, n):
    """R is centrosymmetric, so basis row i is symmetric for even i and antisymmetric
    for odd i: K[i, N-1-j] = (-1)^i K[i, j]."""
    K, _ = orc.klt_closed_form(n, 0.7)
    sgn = (-1.0) ** np.arange(n)
    assert np.max(np.abs(K[:, ::-1] - sgn[:, None] * K)) < 1e-13


@pytest.mark.parametrize("route", ["closed", "jacobi"])
def test_table1_matrices(orc, route):
    """Table 1: round(2 K^(rho)) for rho = 0.1 .. 0.9 gives T1 (0.1-0.3), T2 (0.4-0.6),
    T3 (0.7) and T4 (0.8, 0.9), with the printed S diagonals."""
    t1 = golden_io.table1()
    expect = {0.1: "T1", 0.2: "T1", 0.3: "T1", 0.4: "T2", 0.5: "T2", 0.6: "T2",
              0.7: "T3", 0.8: "T4", 0.9: "T4"}
    for rho, name in expect.items():
        p = orc.Plan(8, rho, 2.0, route=route)
        assert np.array_equal(p.T, t1[name]["T"]), (rho, name)
        assert np.allclose(p.s, t1[name]["s"], rtol=0, atol=1e-15)
        assert t1[name]["rho_lo"] <= rho < t1[name]["rho_hi"]


def test_table1_orthogonality_flags(orc):
    """T1 and T4 have diagonal T T^T; T2 and T3 do not (Eq. 1's two branches)."""
    t1 = golden_io.table1()
    for name, orth in (("T1", True), ("T2", False), ("T3", False), ("T4", True)):
        s, o = orc.normalisation(t1[name]["T"].astype(np.int32))
        assert o == orth
        TT = t1[name]["T"] @ t1[name]["T"].T
        assert (np.count_nonzero(TT - np.diag(np.diag(TT))) == 0) == orth
        assert np.allclose(s, 1 / np.sqrt(np.diag(TT)))


def test_algorithm1_sweep(orc):
    """Algorithm 1 with N = 8, alpha = 2, step 0.1 collects exactly T1, T2, T3, T4, in order."""
    t1 = golden_io.table1()
    found, prev = [], np.zeros((8, 8), np.int32)
    for k in range(1, 10):
        p = orc.Plan(8, k / 10, 2.0)
        if not np.array_equal(p.T, prev):
            found.append(p.T.copy())
            prev = p.T
    assert len(found) == 4
    for got, name in zip(found, ["T1", "T2", "T3", "T4"]):
        assert np.array_equal(got, t1[name]["T"])


def test_rounding_rule_definition(orc):
    """round(x) = floor(x + 1/2) elementwise (Sec. 2.3): halves go up, also below zero."""
    K = np.array([[0.25, -0.25], [0.7499, -0.7501]])
    T, margin, ok = orc.round_alpha(K, 2.0)
    assert T.tolist() == [[1, 0], [1, -2]]
    assert not ok                       # -2 is outside {0, +1, -1}
    assert margin == pytest.approx(0.0)
    T, margin, ok = orc.round_alpha(np.array([[0.1, -0.3], [0.2, 0.0]]), 2.0)
    assert ok and T.tolist() == [[0, -1], [0, 0]]
    assert margin == pytest.approx(0.1)


def test_alpha_range_rule(orc):
    """Sec. 2.3 / Sec. 3: alpha is admissible up to 3/(2 gamma), gamma = max |K|; for
    N = 8 the paper quotes about 3.07, which lies inside the span over rho."""
    his = []
    for rho in RHOS:
        K, _ = orc.klt_closed_form(8, rho)
        gamma = np.max(np.abs(K))
        hi = 3 / (2 * gamma)
        his.append(hi)
        _, _, ok = orc.round_alpha(K, hi * 0.999)
        assert ok
        _, _, ok = orc.round_alpha(K, hi * 1.001)
        assert not ok
    assert min(his) < 3.07 < max(his) and max(his) - min(his) < 0.3


@pytest.mark.parametrize("n", [4, 8, 16, 32])
def test_default_alpha_gives_full_rank(orc, n):
    """alpha_N = 2 sqrt(N/8) gives {0, +-1} full-rank matrices away from rounding ties
    for every rho used by the workloads; plain alpha = 2 at N = 32 gives all zeros."""
    for rho in RHOS:
        p = orc.Plan(n, rho)
        assert set(np.unique(p.T)) <= {-1, 0, 1}
        assert np.linalg.matrix_rank(p.T) == n
        assert p.tie_margin > 1e-6
    K, _ = orc.klt_closed_form(32, 0.95)
    T, _, ok = orc.round_alpha(K, 2.0)
    assert ok and not T.any()


def test_orthogonality_by_size(orc):
    """Diagonal T T^T: the N = 4 matrices are; the N = 16 and N = 32 ones at rho = 0.95 are not."""
    assert orc.Plan(4, 0.95).orthogonal
    assert orc.Plan(8, 0.95).orthogonal
    assert not orc.Plan(16, 0.95).orthogonal
    assert not orc.Plan(32, 0.95).orthogonal
