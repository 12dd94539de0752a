"""MSSIM (Sec. 4.1 quality measure) on the GPU against the FP64 oracle.

Bound (from the FP32 arithmetic of the kernel): each window sum of the centred
second moments is rounded along 22 steps, so sigma_x^2 + sigma_y^2 and sigma_xy carry errors
below 22 u (E[(x-128)^2] + E[(y-128)^2]), u = 2^-24, and its SSIM below four such
terms over C2.  Averaged over the positions this is bounded by
4 * 22 u * (mean (x-128)^2 + mean (y-128)^2) / C2 (the window weights sum to 1);
the means add FP32 rounding of order 1e-7 relative."""
import numpy as np
import pytest

import synth_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U = 2.0 ** -24
C2 = (0.03 * 255) ** 2


@pytest.fixture(scope="module")
def rk():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2111_14239_gb300 as rk
    return rk


def bound(x, y):
    m = np.mean((x.astype(np.float64) - 128) ** 2) + np.mean((y.astype(np.float64) - 128) ** 2)
    return 4 * 22 * U * m / C2 + 1e-6


def gpu_mssim(rk, x, y):
    dx, dy = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    n = 1 if dx.dim() == 2 else dx.shape[0]
    out = torch.zeros(n, dtype=torch.float64, device="cuda")
    rk.rklt_mssim(dx, dy, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("shape", [(64, 64), (200, 552), (11, 11), (37, 300), (600, 129)])
def test_mssim_reconstruction_against_oracle(rk, orc, shape):
    H, W = shape
    Hb, Wb = (H // 8) * 8, (W // 8) * 8
    x = si.ar1_image(H, W, 0.95, 90)
    y = x.copy()
    if Hb and Wb:  # decoded 8-bit image of the fused pass (N = 8, r = 10) where blocks fit
        plan = rk.rklt_make(8, 0.95)
        d = torch.from_numpy(np.ascontiguousarray(x[:Hb, :Wb])).cuda()
        rec = torch.zeros_like(d)
        s = torch.zeros(1, dtype=torch.float64, device="cuda")
        p = torch.zeros(1, device="cuda")
        rk.rklt_fused(plan, d, 10, s, p, recon=rec)
        torch.cuda.synchronize()
        y[:Hb, :Wb] = rec.cpu().numpy()
    got = gpu_mssim(rk, x, y)[0]
    ref, _ = orc.mssim(x, y)
    assert abs(got - ref) <= bound(x, y), (got, ref)


def test_mssim_identical_images_and_batches(rk, orc):
    xs = np.stack([si.ar1_image(96, 160, 0.9, 91 + i) for i in range(3)])
    ys = np.stack([np.clip(xs[i].astype(int) + (i * 7) % 13 - 6, 0, 255).astype(np.uint8) for i in range(3)])
    same = gpu_mssim(rk, xs, xs)
    assert np.all(same == 1.0)
    got = gpu_mssim(rk, xs, ys)
    for i in range(3):
        assert got[i] == gpu_mssim(rk, xs[i], ys[i])[0]            # batch-invariant
        assert abs(got[i] - orc.mssim(xs[i], ys[i])[0]) <= bound(xs[i], ys[i])


def test_mssim_too_small_is_nan(rk):
    out = gpu_mssim(rk, np.zeros((10, 64), np.uint8), np.zeros((10, 64), np.uint8))
    assert np.isnan(out[0])


def test_mssim_tma_and_plain_transport_agree(rk, orc):
    """16-byte aligned rows (TMA chunk loads, several units in both directions, ragged
    edges) against the oracle, and bit-identical to the plain-load transport."""
    H, W = 1100, 608
    x = si.ar1_image(H, W, 0.95, 95)
    y = np.clip(x.astype(int) + si.ar1_image(H, W, 0.5, 96).astype(int) // 16 - 8, 0, 255).astype(np.uint8)
    out = []
    for transport in (0, 1):
        rk.rklt_set_transport(transport)
        try:
            out.append(gpu_mssim(rk, x, y)[0])
        finally:
            rk.rklt_set_transport(0)
    assert out[0] == out[1]
    ref, _ = orc.mssim(x, y)
    assert abs(out[0] - ref) <= bound(x, y), (out[0], ref)
