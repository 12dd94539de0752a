"""Pins of the oracle's JPEG-like quantisation with S absorbed (Appendix):
Bbar = round(B / Q) = round(C / Qtilde), Qtilde = Q / (s s^T), round(x) = floor(x + 1/2)."""
import numpy as np
import pytest

import synth_inputs as si


def _zz(orc, n, X):
    zr, zc = orc.zigzag(n)
    return X[..., zr, zc]


@pytest.mark.parametrize("n", [4, 8])
def test_q_equal_to_r_reduces_to_the_zonal_path(orc, n):
    """Q = s s^T makes Qtilde = 1: Bbar is the exact integer C and the reconstruction is
    the plain zonal pipeline's."""
    p = orc.Plan(n, 0.95)
    Q = np.outer(p.s, p.s)
    img = si.ar1_image(8 * n, 12 * n, 0.9, 11)
    for r in (1, n * n // 2, n * n):
        sse_q, qc, rec_q = orc.quant_pipeline(n, p.T, p.s, Q, img, r, want_coef=True, want_recon=True)
        C = orc.int_stage(n, p.T, img)
        assert np.array_equal(qc, _zz(orc, n, C)[:, :r])
        sse, _, rec = orc.pipeline(n, p.That, img, r, want_recon=True)
        assert np.max(np.abs(rec_q - rec)) < 1e-9 and sse_q == pytest.approx(sse, rel=1e-12, abs=1e-9)


def test_s_absorption_identity(orc):
    """round(B / Q) on B = That A That^T (FP64, the left side of the Appendix identity)
    equals the oracle's round(C / Qtilde) wherever B / Q is not within binary32 error of
    a rounding tie."""
    n = 8
    p = orc.Plan(n, 0.95)
    rng = np.random.default_rng(3)
    Q = rng.uniform(1.0, 40.0, (n, n))
    img = si.ar1_image(64, 96, 0.9, 12)
    _, qc, _ = orc.quant_pipeline(n, p.T, p.s, Q, img, n * n, want_coef=True)
    B = orc.forward(n, p.That, img)                  # [nblk][N*N] zig-zag order
    ratio = B / _zz(orc, n, Q)[None, :]
    direct = np.floor(ratio + 0.5)
    frac = ratio + 0.5 - np.floor(ratio + 0.5)
    near_tie = np.minimum(frac, 1 - frac) < 1e-5 * np.maximum(np.abs(ratio), 1.0)
    assert np.array_equal(qc[~near_tie], direct[~near_tie].astype(np.int32))
    assert near_tie.mean() < 0.01


def test_hand_worked_constant_block(orc):
    """A constant 4 x 4 block of 10 with Q = 16: for the N = 4 plan (first row of T all
    ones, s_0 = 1/2) C_00 = 10 * 4 * 4 = 160 and B_00 = 160 / 4 = 40; 40 / 16 = 2.5 is a
    tie and rounds up to 3 (floor(x + 1/2)); every other coefficient is 0 (the other
    rows of T sum to 0).  Decoding: B'_00 = 48, so A' = 48 / 4 = 12 everywhere and the
    SSE is 16 * 2^2 = 64."""
    p = orc.Plan(4, 0.95)
    assert np.array_equal(p.T[0], [1, 1, 1, 1]) and np.all(p.T[1:].sum(axis=1) == 0)
    img = np.full((4, 4), 10, np.uint8)
    sse, qc, rec = orc.quant_pipeline(4, p.T, p.s, np.full((4, 4), 16.0), img, 16, want_coef=True,
                                      want_recon=True)
    assert qc[0, 0] == 3 and np.all(qc[0, 1:] == 0)
    assert np.allclose(rec, 12.0, atol=1e-12) and sse == pytest.approx(64.0, abs=1e-9)


def test_bad_quantiser_is_rejected(orc):
    p = orc.Plan(8, 0.95)
    with pytest.raises(ValueError):
        orc.quant_pipeline(8, p.T, p.s, np.zeros((8, 8)), np.zeros((8, 8), np.uint8), 10)
