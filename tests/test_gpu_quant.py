"""JPEG-like quantisation with S absorbed (Appendix) through the C ABI against the
FP64 oracle: the quantised coefficients Bbar are integers and must match bit for bit
(both sides take the rounding decision in binary32 the same way); the reconstruction
is the FP32 inverse of the dequantised coefficients, within the FP32 bounds of the
fused path."""
import math

import numpy as np
import pytest

import synth_inputs as si
from test_gpu_parity import RECON_TOL, check_recon_u8, check_sse

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rk():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2111_14239_gb300 as rk
    return rk


def quantisers(n):
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    rng = np.random.default_rng(n)
    return {
        "ramp": 2.0 + 3.0 * (i + j),                 # coarser at high frequency
        "flat16": np.full((n, n), 16.0),
        "random": rng.uniform(0.5, 60.0, (n, n)),
    }


def run(rk, plan, img, r, Q, nimg_axis=False):
    n = plan.N
    d = torch.from_numpy(img).cuda()
    if d.dim() == 2:
        d = d.unsqueeze(0)
    nimg, H, W = d.shape
    nblk = (H // n) * (W // n)
    qc = torch.full((nimg * nblk * max(r, 1),), -7, dtype=torch.int32, device="cuda")
    rec = torch.zeros_like(d)
    sse = torch.zeros(nimg, dtype=torch.float64, device="cuda")
    ps = torch.zeros(nimg, dtype=torch.float32, device="cuda")
    rk.rklt_fused_quant(plan, d, r, Q, sse, ps, qcoef=qc if r else None, recon=rec)
    torch.cuda.synchronize()
    return (qc.cpu().numpy()[:nimg * nblk * r].reshape(nimg, nblk, r), rec.cpu().numpy(), sse.cpu().numpy(),
            ps.cpu().numpy())


SHAPES = {4: (196, 548), 8: (200, 552), 16: (208, 560), 32: (224, 576)}


@pytest.mark.parametrize("n,rho", [(8, 0.95), (8, 0.5), (4, 0.95), (16, 0.95), (32, 0.95), (16, 0.5)])
def test_quant_against_oracle(rk, orc, n, rho):
    """Bbar bit-exact against the oracle; for N = 16, 32 r = N^2/8 runs on the tensor
    cores and r = N^2/4, N^2 on the cooperative path."""
    H, W = SHAPES[n]
    img = si.ar1_image(H, W, 0.95, 70 + n)
    plan = rk.rklt_make(n, rho)
    p = orc.Plan(n, rho)
    for qname, Q in quantisers(n).items():
        for r in sorted({1, n * n // 8, n * n // 4, n * n}):
            qc, rec, sse, ps = run(rk, plan, img, r, Q)
            sse_ref, qc_ref, rec_ref = orc.quant_pipeline(n, p.T, p.s, Q, img, r, want_coef=True, want_recon=True)
            assert np.array_equal(qc[0], qc_ref), f"{qname} r={r}: {np.count_nonzero(qc[0] != qc_ref)} differ"
            check_sse(sse[0], sse_ref, H, W, n)
            check_recon_u8(rec[0], rec_ref, n)
            if sse_ref > 0:
                assert ps[0] == pytest.approx(10 * math.log10(255 ** 2 * H * W / sse[0]), abs=1e-4)


def test_quant_batched_equals_single(rk):
    n = 8
    imgs = np.stack([si.ar1_image(64, 256, 0.9, 80 + i) for i in range(3)])
    plan = rk.rklt_make(n, 0.95)
    Q = quantisers(n)["ramp"]
    qc, rec, sse, ps = run(rk, plan, imgs, 20, Q)
    for i in range(3):
        q1, r1, s1, p1 = run(rk, plan, imgs[i], 20, Q)
        assert np.array_equal(qc[i], q1[0]) and np.array_equal(rec[i], r1[0])
        assert sse[i] == s1[0] and ps[i] == p1[0]


def test_quant_q_equal_r_matches_the_zonal_fused_pass(rk, orc):
    """Q = s s^T: Bbar is the exact integer C, so the reconstruction is the fused pass's
    (same plan and r), within the FP32 bound."""
    n = 8
    img = si.ar1_image(64, 256, 0.9, 90)
    plan = rk.rklt_make(n, 0.95)
    p = orc.Plan(n, 0.95)
    qc, rec, sse, _ = run(rk, plan, img, 10, np.outer(p.s, p.s))
    C = orc.int_stage(n, p.T, img)
    zr, zc = orc.zigzag(n)
    assert np.array_equal(qc[0], C[:, zr, zc][:, :10])
    sse_ref, _, rec_ref = orc.pipeline(n, p.That, img, 10, want_recon=True)
    check_recon_u8(rec[0], rec_ref, n)
    check_sse(sse[0], sse_ref, 64, 256, n)


def test_quant_rejects(rk):
    d = torch.zeros((16, 16), dtype=torch.uint8, device="cuda")
    s = torch.zeros(1, dtype=torch.float64, device="cuda")
    ps = torch.zeros(1, device="cuda")
    for plan, Q, status in ((rk.rklt_make_dct(8), np.ones((8, 8)), 8),
                            (rk.rklt_make_klt(16, 0.95), np.ones((16, 16)), 8),
                            (rk.rklt_make(8, 0.95), np.zeros((8, 8)), 1)):
        with pytest.raises(rk.RklTError) as e:
            rk.rklt_fused_quant(plan, d, 10, Q, s, ps)
        assert e.value.status == status


@pytest.mark.parametrize("n", [4, 8, 16, 32])
def test_quant_tma_ragged_and_plain_transport(rk, orc, n):
    """16-byte aligned rows (TMA tiles) with ragged edges in both directions, against the
    oracle, and bit-identical to the plain-load transport of the same call."""
    H, W = {4: (196, 1040), 8: (200, 1040), 16: (208, 1040), 32: (224, 1056)}[n]
    img = si.ar1_image(H, W, 0.9, 110 + n)
    plan = rk.rklt_make(n, 0.95)
    p = orc.Plan(n, 0.95)
    Q = quantisers(n)["random"]
    for r in (3, n * n // 2 + 1, n * n):
        out = []
        for transport in (0, 1):
            rk.rklt_set_transport(transport)
            try:
                out.append(run(rk, plan, img, r, Q))
            finally:
                rk.rklt_set_transport(0)
        sse_ref, qc_ref, rec_ref = orc.quant_pipeline(n, p.T, p.s, Q, img, r, want_coef=True, want_recon=True)
        qc, rec, sse, _ = out[0]
        assert np.array_equal(qc[0], qc_ref)
        check_sse(sse[0], sse_ref, H, W, n)
        check_recon_u8(rec[0], rec_ref, n)
        for a, b in zip(out[0], out[1]):
            assert np.array_equal(a, b)
