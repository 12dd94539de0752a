"""The tcgen05 / tensor-memory engine for 32 x 32 blocks (rklt_set_tensor_engine(1),
retained support inside i + j < 16): parity against the FP64 oracle, both transports
bit-identical, batched equal to single, and the coefficients bit-identical to the
default warp-level engine (both form the exact integer C and scale it by the same
FP32 s_i s_j)."""
import math

import numpy as np
import pytest

import synth_inputs as si
from test_gpu_parity import check_coef, check_recon_u8, check_sse, run_fused

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N = 32
SHAPE = (224, 800)          # 7 x 25 blocks: the last 256-column tile holds one block


@pytest.fixture(scope="module")
def rk():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2111_14239_gb300 as rk
    rk.rklt_set_transport(0)
    yield rk
    rk.rklt_set_tensor_engine(0)


def _engine(rk, mode, fn):
    rk.rklt_set_tensor_engine(mode)
    try:
        return fn()
    finally:
        rk.rklt_set_tensor_engine(0)


@pytest.mark.parametrize("rho", [0.95, 0.6])
@pytest.mark.parametrize("transport", [0, 1])
def test_tmem_engine_against_oracle(rk, orc, rho, transport):
    H, W = SHAPE
    img = si.ar1_image(H, W, 0.95, 21)
    plan = rk.rklt_make(N, rho)
    p = orc.Plan(N, rho)
    pitch = ((W + 15) // 16) * 16
    for r in (1, 10, 32, 128, 136):
        zc, rec, sse, ps = _engine(rk, 1, lambda: run_fused(rk, plan, img, r, pitch=pitch, transport=transport))
        sse_ref, zc_ref, rec_ref = orc.pipeline(N, p.That, img, r, want_coef=True, want_recon=True)
        check_coef(zc, zc_ref)
        check_sse(sse, sse_ref, H, W, N)
        check_recon_u8(rec, rec_ref, N)
        assert ps == pytest.approx(10 * math.log10(255 ** 2 * H * W / sse), abs=1e-4)
        # the default engine gives the same coefficients bit for bit
        zc0, _, _, _ = run_fused(rk, plan, img, r, pitch=pitch, transport=transport)
        assert np.array_equal(zc, zc0)


def test_tmem_engine_transports_identical(rk):
    H, W = SHAPE
    img = si.ar1_image(H, W, 0.9, 22)
    plan = rk.rklt_make(N, 0.95)
    pitch = ((W + 15) // 16) * 16
    a = _engine(rk, 1, lambda: run_fused(rk, plan, img, 128, pitch=pitch, transport=0))
    b = _engine(rk, 1, lambda: run_fused(rk, plan, img, 128, pitch=pitch, transport=1))
    c = _engine(rk, 1, lambda: run_fused(rk, plan, img, 128, pitch=None, transport=0))
    for x, y in ((a, b), (a, c)):
        assert np.array_equal(x[0], y[0]) and np.array_equal(x[1], y[1])
        assert x[2] == y[2] and x[3] == y[3]


def test_tmem_engine_batched_equals_single(rk):
    H, W = 128, 512
    imgs = np.stack([si.ar1_image(H, W, 0.9, 30 + i) for i in range(3)])
    plan = rk.rklt_make(N, 0.95)
    r = 128
    nblk = (H // N) * (W // N)

    def batched():
        d = torch.from_numpy(imgs).cuda()
        zc = torch.zeros((3, nblk, r), device="cuda")
        rec = torch.zeros_like(d)
        sse = torch.zeros(3, dtype=torch.float64, device="cuda")
        ps = torch.zeros(3, dtype=torch.float32, device="cuda")
        rk.rklt_fused_batched(plan, d, r, sse, ps, zcoef=zc, recon=rec)
        torch.cuda.synchronize()
        return zc.cpu().numpy(), rec.cpu().numpy(), sse.cpu().numpy(), ps.cpu().numpy()

    zc, rec, sse, ps = _engine(rk, 1, batched)
    for i in range(3):
        z1, r1, s1, p1 = _engine(rk, 1, lambda: run_fused(rk, plan, imgs[i], r))
        assert np.array_equal(zc[i], z1) and np.array_equal(rec[i], r1)
        assert sse[i] == s1 and ps[i] == p1


def test_tmem_engine_leaves_other_sizes_alone(rk):
    """r > 136 at N = 32 and every other N run the default kernels under either setting."""
    img = si.ar1_image(128, 256, 0.9, 40)
    for n, r in ((32, 200), (16, 32), (8, 10)):
        plan = rk.rklt_make(n, 0.95)
        a = run_fused(rk, plan, img, r)
        b = _engine(rk, 1, lambda: run_fused(rk, plan, img, r))
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and a[2] == b[2]
