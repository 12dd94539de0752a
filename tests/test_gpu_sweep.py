"""r-sweep through the C ABI against the oracle's literal per-r reconstruction
(forward, keep the first r zig-zag coefficients, inverse, squared error)."""
import math

import numpy as np
import pytest

import synth_inputs as si
from test_gpu_parity import check_sse

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rk():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2111_14239_gb300 as rk
    return rk


@pytest.mark.parametrize("N,rhos", [(8, (0.2, 0.5, 0.7, 0.95, 0.9)), (4, (0.5, 0.95))])
def test_rsweep_against_oracle(rk, orc, N, rhos):
    H, W, nimg = 64, 96, 3
    imgs = np.stack([si.ar1_image(H, W, 0.85 + 0.04 * i, 800 + i) for i in range(nimg)])
    plans = [rk.rklt_make(N, rho) for rho in rhos]
    K = N * N
    d = torch.from_numpy(imgs).cuda()
    sse = torch.zeros((nimg, len(plans), K), dtype=torch.float64, device="cuda")
    ps = torch.zeros((nimg, len(plans), K), dtype=torch.float32, device="cuda")
    rk.rklt_rsweep(plans, d, sse, ps)
    torch.cuda.synchronize()
    rk.rklt_device_status()
    sse, ps = sse.cpu().numpy(), ps.cpu().numpy()
    for p, rho in enumerate(rhos):
        op = orc.Plan(N, rho)
        for i in range(nimg):
            for r in range(1, K + 1):
                ref, _, _ = orc.pipeline(N, op.That, imgs[i], r)
                got = sse[i, p, r - 1]
                if r == K:
                    assert got == 0.0 and ps[i, p, r - 1] == math.inf
                    continue
                check_sse(got, ref, H, W, N)
                assert ps[i, p, r - 1] == pytest.approx(10 * math.log10(255 ** 2 * H * W / got), abs=1e-4)
    # identical matrices (rho 0.9 and 0.95 both give T4) give identical rows
    if N == 8:
        assert np.array_equal(sse[:, 3], sse[:, 4])


def test_rsweep_batch_invariance(rk):
    """An image's sweep is the same alone and inside a larger batch."""
    N = 8
    imgs = np.stack([si.ar1_image(128, 128, 0.9, 900 + i) for i in range(5)])
    plans = [rk.rklt_make(N, 0.5), rk.rklt_make(N, 0.95)]
    d = torch.from_numpy(imgs).cuda()
    full = torch.zeros((5, 2, 64), dtype=torch.float32, device="cuda")
    rk.rklt_rsweep(plans, d, None, full)
    one = torch.zeros((1, 2, 64), dtype=torch.float32, device="cuda")
    rk.rklt_rsweep(plans, d[3:4], None, one)
    torch.cuda.synchronize()
    assert np.array_equal(full[3].cpu().numpy(), one[0].cpu().numpy())
