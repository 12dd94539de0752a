"""Algorithm 1 and the figures of merit as library services (host FP64, no GPU):
against the paper's Table 1 / Table 2 and against the independent oracle."""
import numpy as np
import pytest

import golden_io


@pytest.fixture(scope="module")
def rk():
    import paper_2111_14239_gb300 as rk
    return rk


def test_algorithm1_reproduces_table1(rk):
    """N = 8, alpha = 2, rho = 0.1 .. 0.9 in steps of 0.1 (Sec. 3) gives exactly the
    four matrices of Table 1, in order, with rho ranges inside the printed intervals."""
    out = rk.rklt_design_sweep(8, 2.0, 0.1)
    t1 = golden_io.table1()
    assert len(out) == 4
    for (T, lo, hi), name in zip(out, ("T1", "T2", "T3", "T4")):
        assert np.array_equal(T, t1[name]["T"])
        assert t1[name]["rho_lo"] - 1e-9 <= lo <= hi < t1[name]["rho_hi"] + 1e-9


def test_algorithm1_fine_grid_matches_the_oracle(rk, orc):
    """Step 1e-3: every returned matrix is the oracle's round(alpha K) at its first rho,
    and consecutive matrices differ."""
    out = rk.rklt_design_sweep(8, 2.0, 1e-3)
    for k, (T, lo, hi) in enumerate(out):
        K, _ = orc.klt_closed_form(8, lo)
        Tref, _, _ = orc.round_alpha(K, 2.0)
        assert np.array_equal(T, Tref)
        if k:
            assert not np.array_equal(T, out[k - 1][0])


def test_algorithm1_budget(rk):
    with pytest.raises(rk.RklTError) as e:
        rk.rklt_design_sweep(8, 2.0, 1e-3, max_out=2)
    assert e.value.status == 6


@pytest.mark.parametrize("rho", [0.5, 0.95])
def test_figures_match_the_oracle(rk, orc, rho):
    for n in (8, 16):
        plan = rk.rklt_make(n, rho)
        p = orc.Plan(n, rho)
        f = rk.rklt_figures(plan, rho)
        assert f["cg"] == pytest.approx(orc.coding_gain(p.That, rho), abs=1e-10)
        assert f["eta"] == pytest.approx(orc.transform_efficiency(p.That, rho), abs=1e-10)
        assert f["mse"] == pytest.approx(orc.mse_to_klt(p.K, p.That, rho), abs=1e-12)
        assert f["eps"] == pytest.approx(orc.total_error_energy(p.K, p.That), abs=1e-12)


def test_figures_of_the_exact_klt(rk):
    """The exact KLT has zero distance to itself and an efficiency of 100 (Table 2, K)."""
    f = rk.rklt_figures(rk.rklt_make_klt(8, 0.95), 0.95)
    assert f["mse"] == pytest.approx(0.0, abs=1e-24) and f["eps"] == pytest.approx(0.0, abs=1e-24)
    assert f["eta"] == pytest.approx(100.0, abs=1e-9)
