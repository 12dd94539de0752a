"""Pins of the oracle's per-image path (Sec. 4.1 and the Appendix): zig-zag order
against the JPEG table, the 2-D transforms against Kronecker brute force, exact
reconstruction, Parseval, the S-independence of the reconstruction, PSNR closed
forms and Table 3's MSE/PSNR pairs."""
import math

import numpy as np
import pytest

import golden_io
import synth_inputs as si


def test_zigzag_is_jpeg_order(orc):
    zr, zc = orc.zigzag(8)
    table = golden_io.jpeg_zigzag()
    for k in range(64):
        assert table[zr[k], zc[k]] == k


@pytest.mark.parametrize("n", [2, 4, 8, 16, 32])
def test_zigzag_walk_properties(orc, n):
    """A permutation of the block; anti-diagonals visited in order; consecutive
    positions are neighbours (king moves) except at diagonal turns."""
    zr, zc = orc.zigzag(n)
    assert len(set(zip(zr.tolist(), zc.tolist()))) == n * n
    d = zr + zc
    assert np.all(np.diff(d) >= 0) and np.all(np.diff(d) <= 1)
    steps = np.abs(np.diff(zr)) + np.abs(np.diff(zc))
    assert np.all((steps == 1) | (steps == 2))
    assert (zr[1], zc[1]) == (0, 1)


def kron_block_transform(M, A):
    """vec(M A M^T) = (M kron M) vec(A) for row-major vec."""
    n = M.shape[0]
    return (np.kron(M, M) @ A.reshape(-1)).reshape(n, n)


def blocks(img, n):
    H, W = img.shape
    return img.reshape(H // n, n, W // n, n).transpose(0, 2, 1, 3).reshape(-1, n, n)


@pytest.mark.parametrize("n,rho", [(4, 0.95), (8, 0.2), (8, 0.5), (8, 0.7), (8, 0.95), (16, 0.95), (32, 0.95)])
@pytest.mark.parametrize("kind", ["random", "full", "checker", "impulse"])
def test_int_stage_kronecker(orc, n, rho, kind):
    """C = T A T^T, exact, against an integer Kronecker product."""
    H, W = 2 * n, 3 * n
    img = si.uniform_image(H, W, 7) if kind == "random" else si.pattern_image(kind, H, W)
    p = orc.Plan(n, rho)
    C = orc.int_stage(n, p.T, img)
    T = p.T.astype(np.int64)
    for b, A in enumerate(blocks(img, n)):
        ref = kron_block_transform(T, A.astype(np.int64))
        assert np.array_equal(C[b], ref)


@pytest.mark.parametrize("n,rho", [(4, 0.95), (8, 0.5), (8, 0.95), (16, 0.95), (32, 0.95)])
def test_forward_kronecker_and_scaling(orc, n, rho):
    """B = That A That^T in zig-zag order equals (That kron That) vec(A), and equals
    (s s^T) o (T A T^T): the Appendix's separation of S from the integer stage."""
    img = si.ar1_image(2 * n, 2 * n, 0.9, 3)
    p = orc.Plan(n, rho)
    B = orc.forward(n, p.That, img)
    C = orc.int_stage(n, p.T, img)
    zr, zc = orc.zigzag(n)
    S2 = np.outer(p.s, p.s)
    for b, A in enumerate(blocks(img, n)):
        ref = kron_block_transform(p.That, A.astype(np.float64))
        assert np.max(np.abs(B[b] - ref[zr, zc])) < 1e-9 * max(1.0, np.abs(ref).max())
        assert np.max(np.abs(B[b] - (S2 * C[b])[zr, zc])) < 1e-9 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("n,rho", [(4, 0.95), (8, 0.2), (8, 0.5), (8, 0.7), (8, 0.95), (16, 0.95), (32, 0.95)])
def test_full_retention_reconstructs(orc, n, rho):
    """r = N^2: the inverse undoes the forward (up to FP64 rounding)."""
    img = si.uniform_image(2 * n, 2 * n, 11)
    p = orc.Plan(n, rho)
    B = orc.forward(n, p.That, img)
    rec = orc.inverse(n, p.That, B, n * n, 2 * n, 2 * n)
    assert np.max(np.abs(rec - img)) < 1e-9


@pytest.mark.parametrize("rho", [0.2, 0.95])
def test_parseval_orthogonal(orc, rho):
    """Orthogonal That (T1, T4): block energy is preserved and the squared error
    of keeping r coefficients is the energy of the discarded ones."""
    n = 8
    img = si.ar1_image(16, 24, 0.9, 5)
    p = orc.Plan(n, rho, 2.0)
    assert p.orthogonal
    B = orc.forward(n, p.That, img)
    assert np.sum(B ** 2) == pytest.approx(np.sum(img.astype(np.float64) ** 2), rel=1e-12)
    for r in (1, 10, 37, 64):
        sse, _, _ = orc.pipeline(n, p.That, img, r)
        assert sse == pytest.approx(np.sum(B[:, r:] ** 2), rel=1e-9, abs=1e-6)


@pytest.mark.parametrize("n,rho", [(4, 0.3), (4, 0.95), (8, 0.2), (8, 0.95)])
def test_parseval_retained_integer_form(orc, n, rho):
    """T T^T = diag(d): T^-1 = T^T diag(1/d), so the error of keeping r coefficients
    is the block energy less the retained C_ij^2 / (d_i d_j).  With m = lcm(d) every
    m^2 / (d_i d_j) is an integer and the sum is exact in integers; the oracle's FP64
    reconstruction error must agree.  (The no-reconstruction kernels use this form.)"""
    import fractions
    p = orc.Plan(n, rho)
    assert p.orthogonal
    d = [int(x) for x in np.sum(p.T.astype(np.int64) ** 2, axis=1)]
    m = math.lcm(*d)
    assert all((m * m) % (di * dj) == 0 for di in d for dj in d)
    img = si.ar1_image(3 * n, 5 * n, 0.9, 17)
    C = orc.int_stage(n, p.T, img)
    zr, zc = orc.zigzag(n)
    blocks = img.reshape(3, n, 5, n).transpose(0, 2, 1, 3).reshape(-1, n, n).astype(np.int64)
    energy = int(np.sum(blocks ** 2))
    for r in (0, 1, 2, n * n // 8, n * n // 2 + 1, n * n - 1, n * n):
        kept = sum(int(Cb[zr[k], zc[k]]) ** 2 * (m * m // (d[zr[k]] * d[zc[k]])) for Cb in C for k in range(r))
        exact = fractions.Fraction(m * m * energy - kept, m * m)
        assert exact >= 0
        if r == 0:
            assert exact == energy
            continue
        sse, _, _ = orc.pipeline(n, p.That, img, r)
        if r == n * n:
            assert exact == 0 and sse < 1e-12 * energy
        else:
            assert sse == pytest.approx(float(exact), rel=1e-10)


@pytest.mark.parametrize("n,rho", [(8, 0.5), (8, 0.7), (16, 0.95)])
def test_gram_error_non_orthogonal(orc, n, rho):
    """Non-orthogonal T: A - A' = T^-1 E T^-T with E the discarded integer
    coefficients, so SSE = sum_{k,l discarded} c_k c_l H[i_k, i_l] H[j_k, j_l],
    H = (T T^T)^-1 (computed here with numpy)."""
    img = si.ar1_image(2 * n, 2 * n, 0.9, 9)
    p = orc.Plan(n, rho)
    assert not p.orthogonal
    C = orc.int_stage(n, p.T, img).astype(np.float64)
    H = np.linalg.inv(p.T.astype(np.float64) @ p.T.T)
    zr, zc = orc.zigzag(n)
    for r in (1, 5, n * n // 2):
        ref = 0.0
        for Cb in C:
            c = Cb[zr, zc][r:]
            i, j = zr[r:], zc[r:]
            ref += c @ (H[np.ix_(i, i)] * H[np.ix_(j, j)]) @ c
        sse, _, _ = orc.pipeline(n, p.That, img, r)
        assert sse == pytest.approx(ref, rel=1e-9)


@pytest.mark.parametrize("n,rho", [(8, 0.5), (8, 0.95), (16, 0.95)])
def test_reconstruction_independent_of_s(orc, n, rho):
    """The diagonal S cancels between forward and inverse: reconstructing with
    That or with the bare T gives the same image."""
    img = si.ar1_image(2 * n, 2 * n, 0.9, 13)
    p = orc.Plan(n, rho)
    Tf = p.T.astype(np.float64)
    for r in (3, 10):
        _, _, rec_hat = orc.pipeline(n, p.That, img, r, want_recon=True)
        _, _, rec_t = orc.pipeline(n, Tf, img, r, want_recon=True)
        assert np.max(np.abs(rec_hat - rec_t)) < 1e-9


def test_zonal_and_zero_retention(orc):
    n = 8
    img = si.ar1_image(16, 16, 0.9, 2)
    p = orc.Plan(n, 0.95)
    B = orc.forward(n, p.That, img)
    Z = orc.zonal(n, B, 10)
    assert Z.shape == (4, 10) and np.array_equal(Z, B[:, :10])
    rec = orc.inverse(n, p.That, orc.zonal(n, B, 0), 0, 16, 16)
    assert not rec.any()
    sse, _, _ = orc.pipeline(n, p.That, img, 0)
    assert sse == pytest.approx(np.sum(img.astype(np.float64) ** 2))


def test_pipeline_composition_and_threads(orc):
    """pipeline == forward -> zonal -> inverse -> sse, and does not depend on the thread count."""
    n, r = 8, 10
    img = si.ar1_image(64, 48, 0.95, 4)
    p = orc.Plan(n, 0.95)
    B = orc.forward(n, p.That, img)
    Z = orc.zonal(n, B, r)
    rec = orc.inverse(n, p.That, Z, r, 64, 48)
    ref = orc.sse(img, rec)
    s1, z1, r1 = orc.pipeline(n, p.That, img, r, True, True, nthreads=1)
    s4, z4, r4 = orc.pipeline(n, p.That, img, r, True, True, nthreads=4)
    assert s1 == s4 and np.array_equal(z1, z4) and np.array_equal(r1, r4)
    assert s1 == pytest.approx(ref, rel=1e-12)
    assert np.array_equal(z1, Z)
    assert np.max(np.abs(r1 - rec)) < 1e-12


def test_psnr_closed_forms(orc):
    """One pixel off by e in an H x W image: SSE = e^2, PSNR = 10 log10(255^2 H W / e^2)."""
    H, W = 16, 24
    img = np.full((H, W), 100, np.uint8)
    rec = img.astype(np.float64)
    rec[3, 5] += 2.5
    s = orc.sse(img, rec)
    assert s == 6.25
    assert orc.psnr(s, H, W) == pytest.approx(10 * math.log10(255 ** 2 * H * W / 6.25), rel=1e-14)
    assert orc.psnr(0.0, H, W) == math.inf
    # MSE = 255^2 -> 0 dB
    assert orc.psnr(255.0 ** 2 * H * W, H, W) == pytest.approx(0.0, abs=1e-12)


def test_table3_psnr_definition(orc):
    """Table 3's MSE/PSNR pairs: PSNR = 10 log10(255^2 / MSE) to the printed decimals."""
    for row in golden_io.table3():
        got = orc.psnr(row["mse"] * 512 * 512, 512, 512)
        assert abs(got - row["psnr"]) <= 0.0015, row


def test_recon_u8_rounding(orc):
    """clip(floor(x + 1/2), 0, 255)."""
    x = np.array([[-3.2, -0.5, 0.49, 0.5, 2.4999, 2.5, 254.5, 255.49, 300.0, 127.5]])
    assert orc.recon_u8(x).tolist() == [[0, 0, 0, 1, 2, 3, 255, 255, 255, 128]]


def test_table3_qualitative_shape(orc):
    """On a synthetic AR(1) image at r = 15: That_1 is far worse than the others
    (the paper reports ~13 dB against ~23-31 dB), That_2 ~ That_3, and the rounded
    transforms stay within a few dB of the exact KLT at the matching rho."""
    img = si.ar1_image(256, 256, 0.95, 0)
    H, W = img.shape
    ps = {}
    for name, rho in (("T1", 0.3), ("T2", 0.4), ("T3", 0.7), ("T4", 0.8)):
        p = orc.Plan(8, rho, 2.0)
        sse, _, _ = orc.pipeline(8, p.That, img, 15)
        ps[name] = orc.psnr(sse, H, W)
        K, _ = orc.klt_closed_form(8, rho)
        sse_k, _, _ = orc.pipeline(8, K, img, 15)
        ps["K" + name] = orc.psnr(sse_k, H, W)
    assert ps["T1"] < 20 and ps["T2"] > 25 and ps["T3"] > 25 and ps["T4"] > 25
    assert abs(ps["T2"] - ps["T3"]) < 1.0
    assert ps["T4"] < ps["KT4"] + 0.5
