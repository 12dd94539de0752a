"""Limits of the batched fused call: the largest image count it accepts (65535) and one
past it, and extreme aspect ratios (one block-row 262144 pixels wide, one block-column
262144 pixels tall), against the FP64 oracle."""
import math

import numpy as np
import pytest

import synth_inputs as si
from test_gpu_parity import check_coef, check_recon_u8, check_sse

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rk():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2111_14239_gb300 as rk
    rk.rklt_set_transport(0)
    return rk


def test_largest_image_count(rk, orc):
    n, r, nimg, H, W = 8, 10, 65535, 8, 16
    g = np.random.default_rng(5)
    imgs = g.integers(0, 256, (nimg, H, W), dtype=np.uint8)
    plan = rk.rklt_make(n, 0.95)
    p = orc.Plan(n, 0.95)
    d = torch.from_numpy(imgs).cuda()
    zc = torch.empty(nimg * 2 * r, device="cuda")
    rec = torch.empty_like(d)
    sse = torch.empty(nimg, dtype=torch.float64, device="cuda")
    ps = torch.empty(nimg, device="cuda")
    rk.rklt_fused_batched(plan, d, r, sse, ps, zcoef=zc, recon=rec)
    torch.cuda.synchronize()
    rk.rklt_device_status()
    sse_h, ps_h = sse.cpu().numpy(), ps.cpu().numpy()
    assert np.all(np.isfinite(ps_h)) and np.all(sse_h > 0)
    zcv = zc.view(nimg, 2, r).cpu().numpy()
    for i in (0, 1, 32767, nimg - 2, nimg - 1):
        ref, zref, rref = orc.pipeline(n, p.That, imgs[i], r, want_coef=True, want_recon=True)
        check_sse(sse_h[i], ref, H, W, n)
        check_coef(zcv[i], zref)
        check_recon_u8(rec[i].cpu().numpy(), rref, n)
    with pytest.raises(rk.RklTError) as e:
        rk.rklt_fused_batched(plan, torch.zeros((nimg + 1, H, W), dtype=torch.uint8, device="cuda"), r,
                              torch.empty(nimg + 1, dtype=torch.float64, device="cuda"),
                              torch.empty(nimg + 1, device="cuda"))
    assert e.value.status == 1


@pytest.mark.parametrize("n", [8, 32])
@pytest.mark.parametrize("shape", [(32, 262144), (262144, 32)])
def test_extreme_aspect_ratios(rk, orc, n, shape):
    H, W = shape
    img = si.ar1_image(H, W, 0.9, 77)
    r = n * n // 8
    plan = rk.rklt_make(n, 0.95)
    p = orc.Plan(n, 0.95)
    d = torch.from_numpy(img).cuda()
    zc = torch.empty((H // n) * (W // n) * r, device="cuda")
    rec = torch.empty_like(d)
    sse = torch.empty(1, dtype=torch.float64, device="cuda")
    ps = torch.empty(1, device="cuda")
    rk.rklt_fused(plan, d, r, sse, ps, zcoef=zc, recon=rec)
    torch.cuda.synchronize()
    rk.rklt_device_status()
    ref, zref, rref = orc.pipeline(n, p.That, img, r, want_coef=True, want_recon=True)
    check_sse(float(sse.item()), ref, H, W, n)
    assert abs(float(ps.item()) - 10 * math.log10(255 ** 2 * H * W / ref)) <= 1e-3
    check_coef(zc.view(-1, r).cpu().numpy(), zref)
    check_recon_u8(rec.cpu().numpy(), rref, n)
