"""The comparison transforms (exact KLT and orthonormal DCT-II, Sec. 4.1) through the
fused pipeline and the split path, against the FP64 oracle.

These plans are real-valued, so the kernels run them in FP32 (no exact integer
stage).  The bounds are derived from that arithmetic, per block, with u = 2^-24:
  coefficient (i, j):  |b - b_ref| <= 4 (2N) u (|M| |A| |M|^T)_ij
  reconstruction px:   |a' - a'_ref| <= sum_ij |M_iy| (t_ij + 4 (2N) u |b_ij|) |M_jx|
                       (t = the coefficient bound, kept entries only)
  SSE:                 |SSE - SSE_ref| <= sum_px (2 |e_px| d_px + d_px^2)
  8-bit output:        exact except within d_px of a rounding boundary (then +-1)
"""
import math

import numpy as np
import pytest

import synth_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U = 2.0 ** -24
SHAPES = {4: (196, 548), 8: (200, 552), 16: (208, 560), 32: (224, 576)}


@pytest.fixture(scope="module")
def rk():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2111_14239_gb300 as rk
    rk.rklt_set_transport(0)
    return rk


def blocks(img, n):
    H, W = img.shape
    return img.astype(np.float64).reshape(H // n, n, W // n, n).transpose(0, 2, 1, 3).reshape(-1, n, n)


def unblocks(b, H, W, n):
    return b.reshape(H // n, W // n, n, n).transpose(0, 2, 1, 3).reshape(H, W)


def bounds(M, img, n, r, zz):
    """Per-coefficient and per-pixel bounds of the FP32 kernels (module docstring)."""
    A = blocks(img, n)
    Ma = np.abs(M)
    absterms = np.einsum("ik,bkl,jl->bij", Ma, A, Ma)
    tcoef = 4 * (2 * n) * U * absterms
    B = np.einsum("ik,bkl,jl->bij", M, A, M)
    keep = np.zeros((n, n), bool)
    for z in range(r):
        keep[zz[0][z], zz[1][z]] = True
    t = np.where(keep, tcoef + 4 * (2 * n) * U * np.abs(B), 0.0)
    dpx = np.einsum("iy,bij,jx->byx", Ma, t, Ma)
    return tcoef, dpx


@pytest.mark.parametrize("n", [4, 8, 16, 32])
@pytest.mark.parametrize("kind", ["klt", "dct"])
def test_fused_exact_transforms(rk, orc, n, kind):
    H, W = SHAPES[n]
    img = si.ar1_image(H, W, 0.95, 50 + n)
    plan = rk.rklt_make_klt(n, 0.95) if kind == "klt" else rk.rklt_make_dct(n)
    M = orc.klt_closed_form(n, 0.95)[0] if kind == "klt" else orc.dct_matrix(n)
    assert plan.kind == (1 if kind == "klt" else 2)
    assert np.max(np.abs(plan.matrix() - M)) < 1e-12
    zz = orc.zigzag(n)
    d = torch.from_numpy(img).cuda()
    nblk = (H // n) * (W // n)
    # r = 15 at N = 8 is the largest support of the register path (diagonals 0..4)
    for r in sorted({1, max(1, n * n // 8), min(15, n * n), n * n // 2, n * n}):
        for transport in (0, 1):
            zc = torch.full((nblk, r), float("nan"), device="cuda")
            rec = torch.zeros_like(d)
            sse = torch.zeros(1, dtype=torch.float64, device="cuda")
            ps = torch.zeros(1, dtype=torch.float32, device="cuda")
            rk.rklt_set_transport(transport)
            try:
                rk.rklt_fused(plan, d, r, sse, ps, zcoef=zc, recon=rec)
                torch.cuda.synchronize()
            finally:
                rk.rklt_set_transport(0)
            rk.rklt_device_status()
            sse_ref, zc_ref, rec_ref = orc.pipeline(n, M, img, r, want_coef=True, want_recon=True)
            tcoef, dpx = bounds(M, img, n, r, zz)
            tz = np.stack([tcoef[:, zz[0][z], zz[1][z]] for z in range(r)], axis=1)
            got = zc.cpu().numpy().astype(np.float64)
            assert np.all(np.abs(got - zc_ref) <= tz), f"coef err {np.max(np.abs(got - zc_ref) - tz)}"
            d_img = unblocks(dpx, H, W, n)
            e = img.astype(np.float64) - rec_ref
            assert abs(sse.item() - sse_ref) <= np.sum(2 * np.abs(e) * d_img + d_img ** 2)
            u8 = rec.cpu().numpy().astype(np.int64)
            ref = np.clip(np.floor(rec_ref + 0.5), 0, 255).astype(np.int64)
            frac = rec_ref + 0.5 - np.floor(rec_ref + 0.5)
            near = np.minimum(frac, 1 - frac) <= d_img
            assert np.all(np.abs(u8 - ref) <= 1) and np.all(u8[~near] == ref[~near])
            if sse_ref > 0 and sse.item() > 0:
                assert ps.item() == pytest.approx(10 * math.log10(255 ** 2 * H * W / sse.item()), abs=1e-4)


@pytest.mark.parametrize("n", [8, 16])
def test_split_path_exact_transforms(rk, orc, n):
    H, W = SHAPES[n]
    img = si.ar1_image(H, W, 0.9, 60 + n)
    plan = rk.rklt_make_dct(n)
    M = orc.dct_matrix(n)
    zz = orc.zigzag(n)
    d = torch.from_numpy(img).cuda()
    nblk = (H // n) * (W // n)
    coef = torch.zeros((nblk, n * n), device="cuda")
    rk.rklt_forward(plan, d, coef)
    torch.cuda.synchronize()
    tcoef, _ = bounds(M, img, n, n * n, zz)
    tz = np.stack([tcoef[:, zz[0][z], zz[1][z]] for z in range(n * n)], axis=1)
    ref = orc.forward(n, M, img)
    assert np.all(np.abs(coef.cpu().numpy() - ref) <= tz)


def test_integer_only_entry_points_reject_real_plans(rk):
    plan = rk.rklt_make_klt(8, 0.95)
    d = torch.zeros((16, 16), dtype=torch.uint8, device="cuda")
    C = torch.zeros((4, 8, 8), dtype=torch.int32, device="cuda")
    with pytest.raises(rk.RklTError) as e:
        rk.rklt_forward_int(plan, d, C)
    assert e.value.status == 8
    s = torch.zeros(1, dtype=torch.float64, device="cuda")
    p = torch.zeros(1, device="cuda")
    with pytest.raises(rk.RklTError) as e:
        rk.rklt_fused_items(rk.make_items([(d, 0, 8, None, None)]), [plan], s, p)
    assert e.value.status == 8
