"""Pins of the oracle's comparison transforms (Sec. 4.1): the orthonormal DCT-II and
the exact KLT run through the same per-block path as the RKLT."""
import numpy as np
import pytest

import golden_io
import synth_inputs as si


@pytest.mark.parametrize("n", [4, 8, 16, 32])
def test_dct_matches_library_routine(orc, n):
    """The oracle's DCT-II equals scipy's orthonormal DCT-II and is orthonormal."""
    fft = pytest.importorskip("scipy.fft")
    M = orc.dct_matrix(n)
    ref = fft.dct(np.eye(n), type=2, norm="ortho", axis=0)
    assert np.max(np.abs(M - ref)) < 1e-14
    assert np.max(np.abs(M @ M.T - np.eye(n))) < 1e-14


def test_dct_textbook_entries(orc):
    M = orc.dct_matrix(8)
    assert np.allclose(M[0], 1 / np.sqrt(8), atol=1e-15)
    assert M[1, 0] == pytest.approx(0.5 * np.cos(np.pi / 16), abs=1e-15)     # 0.4904
    assert M[2, 1] == pytest.approx(0.5 * np.cos(3 * np.pi / 8), abs=1e-15)  # 0.1913
    # row parity used by the kernels' butterflies: M[k][N-1-j] = (-1)^k M[k][j]
    for k in range(8):
        assert np.allclose(M[k, ::-1], (-1) ** k * M[k], atol=1e-15)


def test_rounded_dct_is_table1_t4(orc):
    """Sec. 3: rounding 2 C (C the 8-point DCT) gives the paper's matrix T4."""
    T4 = golden_io.table1()["T4"]["T"]
    assert np.array_equal(np.floor(2 * orc.dct_matrix(8) + 0.5).astype(int), T4)


@pytest.mark.parametrize("n", [4, 8])
def test_exact_transforms_reconstruct_at_full_r(orc, n):
    """Keeping every coefficient of an orthonormal transform reconstructs the image."""
    img = si.ar1_image(8 * n, 16 * n, 0.9, 77)
    for M in (orc.dct_matrix(n), orc.klt_closed_form(n, 0.95)[0]):
        sse, _, rec = orc.pipeline(n, M, img, n * n, want_recon=True)
        assert sse < 1e-18 * img.size * 255 ** 2
        assert np.max(np.abs(rec - img)) < 1e-10


def test_exact_transforms_bound_the_rklt_on_ar1(orc):
    """On a ρ = 0.95 AR(1) field the exact KLT and the DCT give nearly the same PSNR
    (within 0.5 dB) and both beat the rounded KLT, which trades a little quality for
    a multiplication-free transform (the comparison of Sec. 4.1)."""
    img = si.ar1_image(256, 256, 0.95, 5)
    K, _ = orc.klt_closed_form(8, 0.95)
    p = orc.Plan(8, 0.95)
    for r in (6, 10, 15):
        s_k = orc.pipeline(8, K, img, r)[0]
        s_d = orc.pipeline(8, orc.dct_matrix(8), img, r)[0]
        s_r = orc.pipeline(8, p.That, img, r)[0]
        assert abs(10 * np.log10(s_k / s_d)) < 0.5
        assert s_r > max(s_k, s_d)
