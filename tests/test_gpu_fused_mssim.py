"""The fused pass with MSSIM (Sec. 4.1: PSNR and SSIM of the reconstruction) on the GPU.

What the one-launch form must give, for the register-path plans (N = 4; N = 8 with
r <= 15 and T T^T diagonal):
  - coefficients, 8-bit reconstruction, SSE and PSNR bit-identical to
    rklt_fused_batched (the same block code);
  - MSSIM within 1e-6 of rklt_mssim on that reconstruction (the SSIM of every window
    position is computed in the same order; only the grouping of the FP32 partial
    sums differs), and within the MSSIM bound of the FP64 oracle;
  - the same MSSIM with and without the reconstruction written out, with TMA and
    with plain loads, alone and in a batch.
Other plans take the two-pass form, which must equal the two calls exactly."""
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


def oracle_bound(x, y):
    m = np.mean((x.astype(np.float64) - 128) ** 2) + np.mean((y.astype(np.float64) - 128) ** 2)
    return 4 * 22 * U * m / C2 + 1e-6


def two_pass(rk, plan, d, r, n):
    nimg, H, W = d.shape
    rec = torch.zeros_like(d)
    zc = torch.zeros(max(nimg * (H // n) * (W // n) * r, 1), device="cuda")
    s = torch.zeros(nimg, dtype=torch.float64, device="cuda")
    p = torch.zeros(nimg, device="cuda")
    rk.rklt_fused_batched(plan, d, r, s, p, zcoef=zc, recon=rec)
    ms = torch.zeros(nimg, dtype=torch.float64, device="cuda")
    rk.rklt_mssim(d, rec, ms)
    torch.cuda.synchronize()
    return zc.cpu().numpy(), rec.cpu().numpy(), s.cpu().numpy(), p.cpu().numpy(), ms.cpu().numpy()


def fused(rk, plan, d, r, n, want_recon=True, want_coef=True):
    nimg, H, W = d.shape
    rec = torch.zeros_like(d) if want_recon else None
    zc = torch.zeros(max(nimg * (H // n) * (W // n) * r, 1), device="cuda") if want_coef else None
    s = torch.zeros(nimg, dtype=torch.float64, device="cuda")
    p = torch.zeros(nimg, device="cuda")
    ms = torch.zeros(nimg, dtype=torch.float64, device="cuda")
    rk.rklt_fused_mssim(plan, d, r, s, p, ms, zcoef=zc, recon=rec)
    torch.cuda.synchronize()
    rk.rklt_device_status()
    return (zc.cpu().numpy() if zc is not None else None, rec.cpu().numpy() if rec is not None else None,
            s.cpu().numpy(), p.cpu().numpy(), ms.cpu().numpy())


def images(nimg, H, W, seed):
    return np.stack([si.ar1_image(H, W, 0.95, seed + i) for i in range(nimg)])


# shapes: several 256-column strips with a ragged last one, several row segments
# (heights above 8 x 88 rows), images narrower than one strip, the 11-pixel edge
SHAPES = [(64, 64), (176, 264), (1000, 520), (720, 1000), (16, 16), (88, 96), (1416, 264), (512, 512)]


@pytest.mark.parametrize("n,rho,r", [(8, 0.95, 10), (8, 0.95, 1), (8, 0.95, 15), (4, 0.95, 5), (4, 0.9, 16),
                                     (8, 0.2, 6)])
@pytest.mark.parametrize("shape", SHAPES)
def test_fused_mssim_matches_two_passes(rk, n, rho, r, shape):
    H, W = shape
    x = images(1, H, W, 300 + H + W)
    d = torch.from_numpy(x).cuda()
    plan = rk.rklt_make(n, rho)
    zc0, rec0, s0, p0, ms0 = two_pass(rk, plan, d, r, n)
    zc1, rec1, s1, p1, ms1 = fused(rk, plan, d, r, n)
    assert np.array_equal(rec0, rec1)
    assert np.array_equal(zc0.view(np.uint32), zc1.view(np.uint32))
    assert np.array_equal(s0, s1) and np.array_equal(p0.view(np.uint32), p1.view(np.uint32))
    if H < 11 or W < 11:
        assert np.isnan(ms1[0])
    else:
        assert abs(ms1[0] - ms0[0]) <= 1e-6, (ms1, ms0)


def test_fused_mssim_against_oracle(rk, orc):
    H, W = 600, 776
    x = images(1, H, W, 410)
    d = torch.from_numpy(x).cuda()
    plan = rk.rklt_make(8, 0.95)
    _, rec, s, p, ms = fused(rk, plan, d, 10, 8)
    ref, _ = orc.mssim(x[0], rec[0])
    assert abs(ms[0] - ref) <= oracle_bound(x[0], rec[0]), (ms[0], ref)


def test_fused_mssim_without_outputs_and_batched(rk):
    """No reconstruction and no coefficients written: the same scalars; a batch of
    three equals each image alone."""
    x = images(3, 704, 520, 420)
    d = torch.from_numpy(x).cuda()
    plan = rk.rklt_make(8, 0.95)
    _, _, s_all, p_all, ms_all = fused(rk, plan, d, 8, 8)
    _, _, s_b, p_b, ms_b = fused(rk, plan, d, 8, 8, want_recon=False, want_coef=False)
    assert np.array_equal(s_all, s_b) and np.array_equal(ms_all, ms_b) and np.array_equal(p_all, p_b)
    for i in range(3):
        _, _, s1, p1, ms1 = fused(rk, plan, d[i:i + 1], 8, 8, want_recon=False, want_coef=False)
        assert s1[0] == s_all[i] and ms1[0] == ms_all[i] and p1[0] == p_all[i]


def test_fused_mssim_tma_and_plain_agree(rk):
    x = images(2, 1416, 600, 430)
    d = torch.from_numpy(x).cuda()
    plan = rk.rklt_make(8, 0.95)
    out = []
    for transport in (0, 1):
        rk.rklt_set_transport(transport)
        try:
            out.append(fused(rk, plan, d, 12, 8))
        finally:
            rk.rklt_set_transport(0)
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)


def test_fused_mssim_unaligned_pitch(rk):
    """Rows 8-byte but not 16-byte aligned: the plain-load path."""
    H, W = 400, 520
    base = torch.from_numpy(images(1, H, W + 8, 440)[0]).cuda()
    d = base[:, 8:W + 8].unsqueeze(0)     # pitch 528, start 8 bytes in: not 16-byte aligned
    plan = rk.rklt_make(8, 0.95)
    dc = d.contiguous()
    zc0, rec0, s0, p0, ms0 = two_pass(rk, plan, dc, 10, 8)
    zc1, rec1, s1, p1, ms1 = fused(rk, plan, d, 10, 8)
    assert np.array_equal(rec0, rec1) and np.array_equal(s0, s1)
    assert abs(ms0[0] - ms1[0]) <= 1e-6


@pytest.mark.parametrize("n,rho,r", [(8, 0.5, 10), (8, 0.95, 40), (16, 0.95, 32)])
def test_fused_mssim_two_pass_plans(rk, n, rho, r):
    """Plans outside the register path: exactly the two calls."""
    x = images(2, 256, 320, 450)
    d = torch.from_numpy(x).cuda()
    plan = rk.rklt_make(n, rho)
    zc0, rec0, s0, p0, ms0 = two_pass(rk, plan, d, r, n)
    zc1, rec1, s1, p1, ms1 = fused(rk, plan, d, r, n)
    assert np.array_equal(rec0, rec1) and np.array_equal(s0, s1) and np.array_equal(ms0, ms1)
    _, _, s2, _, ms2 = fused(rk, plan, d, r, n, want_recon=False)
    assert np.array_equal(s0, s2) and np.array_equal(ms0, ms2)


def test_fused_mssim_rejects(rk):
    plan = rk.rklt_make(8, 0.95)
    d = torch.zeros((1, 64, 60), dtype=torch.uint8, device="cuda")
    s = torch.zeros(1, dtype=torch.float64, device="cuda")
    p = torch.zeros(1, device="cuda")
    ms = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(RuntimeError):
        rk.rklt_fused_mssim(plan, d, 10, s, p, ms)
