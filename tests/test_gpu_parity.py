"""GPU parity of the CUDA path (through the C ABI) against the FP64 oracle.

Bars (see the tolerance section of the design notes):
  integer stage        bit-exact
  coefficients         |b - b_ref| <= 1e-5 * max(|b_ref|, 1)
  FP32 reconstruction  |a' - a'_ref| <= RECON_TOL[N]
  SSE / PSNR           |SSE - SSE_ref| <= 2.3e-4 * SSE_ref (1e-3 dB) while the
                       oracle PSNR is below 60 dB; otherwise the MSE difference is
                       bounded by the FP32 reconstruction error
  8-bit reconstruction equal to clip(floor(a'_ref + 1/2), 0, 255) except where a'_ref
                       lies within RECON_TOL[N] of a rounding boundary (then off by <= 1)
"""
import math

import numpy as np
import pytest

import synth_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# FP32 reconstruction bound: |error| <= gamma_m * sum |terms| with m ~ 2N terms of
# magnitude up to ~|C| |T^-1| ~ 255 * N / 8 and gamma_m = m 2^-24; stated per N
# with a 4x margin over that estimate.
RECON_TOL = {4: 2e-4, 8: 5e-4, 16: 2e-3, 32: 8e-3}
SSE_REL = 2.3e-4          # 10 log10(1 + 2.3e-4) = 1.0e-3 dB
COEF_REL = 1e-5

SHAPES = {4: (196, 548), 8: (200, 552), 16: (208, 560), 32: (224, 576)}
CASES = [(4, 0.95), (8, 0.2), (8, 0.5), (8, 0.7), (8, 0.95), (16, 0.95), (32, 0.95), (16, 0.5), (32, 0.6)]


@pytest.fixture(scope="module")
def rk():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2111_14239_gb300 as rk
    rk.rklt_set_transport(0)
    return rk


def dev(a, pitch=None):
    """Copy a 2-D uint8 array to the GPU, optionally with a padded row pitch."""
    H, W = a.shape
    if pitch is None or pitch == W:
        return torch.from_numpy(np.ascontiguousarray(a)).cuda()
    buf = torch.zeros((H, pitch), dtype=torch.uint8, device="cuda")
    buf[:, :W] = torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return buf[:, :W]


def run_fused(rk, plan, img_np, r, pitch=None, want_coef=True, want_recon=True, transport=0):
    n = plan.N
    H, W = img_np.shape
    d = dev(img_np, pitch)
    nblk = (H // n) * (W // n)
    zc = torch.full((max(nblk * r, 1),), float("nan"), device="cuda") if want_coef else None
    rec = dev(np.zeros((H, W), np.uint8), pitch) if want_recon else None
    sse = torch.zeros(1, dtype=torch.float64, device="cuda")
    ps = torch.zeros(1, dtype=torch.float32, device="cuda")
    rk.rklt_set_transport(transport)
    try:
        rk.rklt_fused(plan, d, r, sse, ps, zcoef=zc, recon=rec)
        torch.cuda.synchronize()
    finally:
        rk.rklt_set_transport(0)
    rk.rklt_device_status()
    return (zc[:nblk * r].view(nblk, r).cpu().numpy() if want_coef else None,
            rec.cpu().numpy() if want_recon else None, float(sse.item()), float(ps.item()))


def check_coef(got, ref):
    err = np.abs(got.astype(np.float64) - ref)
    bound = COEF_REL * np.maximum(np.abs(ref), 1.0)
    assert np.all(err <= bound), f"max coef err {np.max(err - bound)}"


def check_sse(sse, ref, H, W, n):
    if ref == 0:
        assert sse <= H * W * RECON_TOL[n] ** 2
        return
    psnr_ref = 10 * math.log10(255 ** 2 * H * W / ref)
    if psnr_ref < 60:
        assert abs(sse - ref) <= SSE_REL * ref, (sse, ref)
    else:
        mse, mse_ref = sse / (H * W), ref / (H * W)
        d = RECON_TOL[n]
        assert abs(mse - mse_ref) <= 2 * math.sqrt(mse_ref) * d + d * d, (sse, ref)


def check_recon_u8(got, ref_f, n):
    ref = np.clip(np.floor(ref_f + 0.5), 0, 255)
    diff = np.abs(got.astype(np.int64) - ref.astype(np.int64))
    frac = ref_f + 0.5 - np.floor(ref_f + 0.5)   # distance above the rounding boundary
    near = (np.minimum(frac, 1 - frac) <= RECON_TOL[n])
    assert np.all(diff <= 1)
    assert np.all(diff[~near] == 0), f"{np.count_nonzero(diff[~near])} pixels differ away from a boundary"


@pytest.mark.parametrize("n,rho", CASES)
def test_forward_int_bit_exact(rk, orc, n, rho):
    H, W = SHAPES[n]
    for img in (si.ar1_image(H, W, 0.9, 1), si.uniform_image(H, W, 2), si.pattern_image("checker", H, W)):
        plan = rk.rklt_make(n, rho)
        C = torch.zeros(((H // n) * (W // n), n, n), dtype=torch.int32, device="cuda")
        rk.rklt_forward_int(plan, dev(img), C)
        ref = orc.int_stage(n, orc.Plan(n, rho).T, img)
        assert np.array_equal(C.cpu().numpy().astype(np.int64), ref)


@pytest.mark.parametrize("n,rho", CASES)
def test_split_path(rk, orc, n, rho):
    """forward -> zonal -> inverse -> psnr, each against the oracle."""
    H, W = SHAPES[n]
    img = si.ar1_image(H, W, 0.9, 3)
    plan = rk.rklt_make(n, rho)
    p = orc.Plan(n, rho)
    nblk = (H // n) * (W // n)
    coef = torch.zeros((nblk, n * n), device="cuda")
    rk.rklt_forward(plan, dev(img), coef)
    Bref = orc.forward(n, p.That, img)
    check_coef(coef.cpu().numpy(), Bref)
    for r in (1, n * n // 8, n * n // 2 + 3, n * n):
        z = torch.zeros((nblk, r), device="cuda")
        rk.rklt_zonal(plan, coef, nblk, r, z)
        assert np.array_equal(z.cpu().numpy(), coef.cpu().numpy()[:, :r])
        rec = torch.zeros((H, W), device="cuda")
        rk.rklt_inverse(plan, z, r, H, W, rec)
        rec_ref = orc.inverse(n, p.That, orc.zonal(n, Bref, r), r, H, W)
        assert np.max(np.abs(rec.cpu().numpy() - rec_ref)) <= RECON_TOL[n]
        sse = torch.zeros(1, dtype=torch.float64, device="cuda")
        ps = torch.zeros(1, dtype=torch.float32, device="cuda")
        rk.rklt_psnr(dev(img), rec, sse, ps)
        # the PSNR kernel itself is FP64: against the oracle's SSE of the same FP32 image
        # (only the summation order differs)
        ref_same = orc.sse(img, rec.cpu().numpy().astype(np.float64))
        assert sse.item() == pytest.approx(ref_same, rel=1e-10, abs=1e-9)
        check_sse(sse.item(), orc.sse(img, rec_ref), H, W, n)


@pytest.mark.parametrize("n,rho", CASES)
@pytest.mark.parametrize("transport", [0, 1])
def test_fused_against_oracle(rk, orc, n, rho, transport):
    H, W = SHAPES[n]
    img = si.ar1_image(H, W, 0.95, 4)
    plan = rk.rklt_make(n, rho)
    p = orc.Plan(n, rho)
    for r in sorted({1, max(1, n * n // 8), 10 if n == 8 else n, n * n // 2, n * n - 1}):
        zc, rec, sse, ps = run_fused(rk, plan, img, r, pitch=((W + 15) // 16) * 16, transport=transport)
        sse_ref, zc_ref, rec_ref = orc.pipeline(n, p.That, img, r, want_coef=True, want_recon=True)
        check_coef(zc, zc_ref)
        check_sse(sse, sse_ref, H, W, n)
        check_recon_u8(rec, rec_ref, n)
        if sse_ref > 0:
            assert ps == pytest.approx(10 * math.log10(255 ** 2 * H * W / sse), abs=1e-4)


@pytest.mark.parametrize("n", [4, 8, 16, 32])
def test_transports_identical(rk, n):
    """TMA ring and plain loads give bit-identical results (same arithmetic, same order)."""
    H, W = SHAPES[n]
    img = si.ar1_image(H, W, 0.9, 5)
    plan = rk.rklt_make(n, 0.95)
    r = max(1, n * n // 8)
    pitch = ((W + 15) // 16) * 16
    a = run_fused(rk, plan, img, r, pitch=pitch, transport=0)
    b = run_fused(rk, plan, img, r, pitch=pitch, transport=1)
    c = run_fused(rk, plan, img, r, pitch=None, transport=0)   # unaligned pitch: plain loads
    for x, y in ((a, b), (a, c)):
        assert np.array_equal(x[0], y[0]) and np.array_equal(x[1], y[1])
        assert x[2] == y[2] and x[3] == y[3]


@pytest.mark.parametrize("n", [4, 8, 16, 32])
def test_batched_equals_single(rk, n):
    """Each image's result is identical alone and inside a batch."""
    H, W = 128, 512
    imgs = np.stack([si.ar1_image(H, W, 0.9, 10 + i) for i in range(3)])
    plan = rk.rklt_make(n, 0.95)
    r = max(1, n * n // 8)
    d = torch.from_numpy(imgs).cuda()
    nblk = (H // n) * (W // n)
    zc = torch.zeros((3, nblk, r), device="cuda")
    rec = torch.zeros_like(d)
    sse = torch.zeros(3, dtype=torch.float64, device="cuda")
    ps = torch.zeros(3, dtype=torch.float32, device="cuda")
    rk.rklt_fused_batched(plan, d, r, sse, ps, zcoef=zc, recon=rec)
    torch.cuda.synchronize()
    for i in range(3):
        z1, r1, s1, p1 = run_fused(rk, plan, imgs[i], r)
        assert np.array_equal(zc[i].cpu().numpy(), z1)
        assert np.array_equal(rec[i].cpu().numpy(), r1)
        assert sse[i].item() == s1 and ps[i].item() == p1
    # PSNR only (the Parseval copy for N = 4, 8): also identical alone and in the batch
    rk.rklt_fused_batched(plan, d, r, sse, ps)
    torch.cuda.synchronize()
    for i in range(3):
        _, _, s1, p1 = run_fused(rk, plan, imgs[i], r, want_coef=False, want_recon=False)
        assert sse[i].item() == s1 and ps[i].item() == p1


def test_edge_cases(rk, orc):
    plan = rk.rklt_make(8, 0.95)
    p = orc.Plan(8, 0.95)
    # one block, r = 0 (nothing kept: reconstruction 0, SSE = sum of squares)
    img = si.uniform_image(8, 8, 9)
    zc, rec, sse, ps = run_fused(rk, plan, img, 0, want_coef=False)
    assert not rec.any() and sse == float(np.sum(img.astype(np.float64) ** 2))
    # r = N^2 on extremes: lossless up to FP32 noise
    for kind in ("zeros", "full", "checker", "impulse"):
        img = si.pattern_image(kind, 64, 64)
        _, rec, sse, ps = run_fused(rk, plan, img, 64)
        assert np.array_equal(rec, img)
        assert sse <= 64 * 64 * RECON_TOL[8] ** 2
    # constant image: PSNR is +inf only when the SSE is exactly zero
    img = np.zeros((16, 16), np.uint8)
    _, _, sse, ps = run_fused(rk, plan, img, 1)
    assert sse == 0.0 and ps == math.inf
    # empty image: SSE 0, PSNR NaN, nothing launched on pixels
    d = torch.zeros((0, 64), dtype=torch.uint8, device="cuda")
    s = torch.full((1,), 7.0, dtype=torch.float64, device="cuda")
    q = torch.zeros(1, device="cuda")
    rk.rklt_fused(plan, d, 10, s, q)
    torch.cuda.synchronize()
    assert s.item() == 0.0 and math.isnan(q.item())
    # pitch larger than W and a single-row-of-blocks image
    img = si.ar1_image(8, 1024, 0.9, 6)
    zc, rec, sse, _ = run_fused(rk, plan, img, 10, pitch=1040)
    sse_ref, zc_ref, rec_ref = orc.pipeline(8, p.That, img, 10, want_coef=True, want_recon=True)
    check_coef(zc, zc_ref)
    check_sse(sse, sse_ref, 8, 1024, 8)
    check_recon_u8(rec, rec_ref, 8)


def test_paper_matrices_via_from_matrix(rk, orc):
    """The printed Table 1 matrices run through the fused path like the derived plans."""
    import golden_io
    img = si.ar1_image(64, 256, 0.9, 8)
    for name in ("T1", "T2", "T3", "T4"):
        T = golden_io.table1()[name]["T"]
        plan = rk.rklt_make_from_matrix(8, T)
        s, _ = orc.normalisation(T.astype(np.int32))
        M = orc.that(T.astype(np.int32), s)
        zc, rec, sse, _ = run_fused(rk, plan, img, 15)
        sse_ref, zc_ref, rec_ref = orc.pipeline(8, M, img, 15, want_coef=True, want_recon=True)
        check_coef(zc, zc_ref)
        check_sse(sse, sse_ref, 64, 256, 8)


def test_bounded_wait_gives_up(rk):
    """Fault injection: the TMA producer issues no loads, the consumers' bounded waits
    run out, the kernel returns early and the host reads RKLT_ERR_TIMEOUT; the
    context stays usable afterwards."""
    plan = rk.rklt_make(8, 0.95)
    img = torch.zeros((256, 1024), dtype=torch.uint8, device="cuda")
    sse = torch.zeros(1, dtype=torch.float64, device="cuda")
    ps = torch.zeros(1, device="cuda")
    rk.rklt_set_wait_timeout_us(20000)
    rk.rklt_debug_inject_stall(True)
    try:
        rk.rklt_fused(plan, img, 10, sse, ps)
        with pytest.raises(rk.RklTError) as e:
            rk.rklt_device_status()
        assert e.value.status == 7
    finally:
        rk.rklt_debug_inject_stall(False)
        rk.rklt_set_wait_timeout_us(0)
    rk.rklt_fused(plan, img, 10, sse, ps)
    rk.rklt_device_status()
    assert sse.item() == 0.0


def zz_diagonals(n, r):
    """Anti-diagonals i + j < D touched by the first r zig-zag positions."""
    D, cnt = 0, 0
    while cnt < r:
        cnt += min(D, 2 * n - 2 - D) + 1
        D += 1
    return D


def parseval_path(plan, r):
    """Whether a call takes the integer-Parseval register path: a rounded plan with
    T T^T diagonal on the register path (N = 4; N = 8 with D <= 5)."""
    return plan.kind == 0 and plan.orthogonal and (plan.N == 4 or (plan.N == 8 and zz_diagonals(8, r) <= 5))


@pytest.mark.parametrize("n", [4, 8, 16, 32])
def test_output_subsets_agree(rk, orc, n):
    """Every subset of the optional outputs (coefficients, 8-bit reconstruction) gives
    the same coefficients / reconstruction as the full call, and the same SSE / PSNR
    bit for bit: the kernels take separate code paths for the full set and the
    others.  Plans with T T^T diagonal on the register path take the error from
    Parseval's identity in integers with or without a reconstruction (exact integers,
    so every subset agrees bit for bit); that SSE is also checked against the oracle."""
    H, W = SHAPES[n]
    img = si.ar1_image(H, W, 0.9, 31 + n)
    plan = rk.rklt_make(n, 0.95)
    r = n * n // 8
    full = run_fused(rk, plan, img, r, pitch=((W + 15) // 16) * 16)
    ref = orc.pipeline(n, orc.Plan(n, 0.95).That, img, r)[0]
    for want_coef, want_recon in ((True, False), (False, True), (False, False)):
        zc, rec, sse, ps = run_fused(rk, plan, img, r, pitch=((W + 15) // 16) * 16, want_coef=want_coef,
                                     want_recon=want_recon)
        if parseval_path(plan, r):
            check_sse(sse, ref, H, W, n)
        assert sse == full[2] and ps == full[3]
        if want_coef:
            assert np.array_equal(zc, full[0])
        if want_recon:
            assert np.array_equal(rec, full[1])


@pytest.mark.parametrize("n,rho", [(4, 0.3), (4, 0.95), (8, 0.2), (8, 0.95)])
def test_parseval_no_recon(rk, orc, n, rho):
    """Calls without a reconstruction on plans with T T^T diagonal: the SSE is the
    block energy less the retained C^2 / (d_i d_j), in integers.  Against the oracle
    over every r the register path serves, on a ragged image in both transports;
    r = N^2 must give exactly 0 and r = 0 the image energy; the coefficients are
    bit-identical to the full call's."""
    H, W = SHAPES[n]
    img = si.ar1_image(H, W, 0.9, 41 + n)
    plan = rk.rklt_make(n, rho)
    assert plan.orthogonal
    p = orc.Plan(n, rho)
    energy = float(np.sum(img.astype(np.float64) ** 2))
    pitch = ((W + 15) // 16) * 16      # aligned: the TMA ring (transport 0) and plain loads (1)
    for r in ([0, 1, 2, 3, 5, 8, 11, 15, 16] if n == 4 else [0, 1, 3, 6, 8, 10, 13, 15]):
        assert parseval_path(plan, r)
        for transport in (0, 1):
            zc, _, sse, ps = run_fused(rk, plan, img, r, pitch=pitch, want_recon=False, transport=transport)
            if r == 0:
                assert sse == pytest.approx(energy, rel=1e-6)   # FP32 sums of exact block energies
                continue
            ref, zref, _ = orc.pipeline(n, p.That, img, r, want_coef=True)
            if r == n * n:
                assert sse == 0.0 and ps == math.inf
            else:
                check_sse(sse, ref, H, W, n)
                assert abs(ps - 10 * math.log10(255 ** 2 * H * W / ref)) <= 1e-3
            check_coef(zc, zref)
            full = run_fused(rk, plan, img, r, pitch=pitch, transport=transport)
            assert np.array_equal(zc, full[0])
    # a constant image at r = 1: where the oracle's error is zero (every AC row of T
    # sums to zero) the integer form gives exactly zero and PSNR +inf
    flat = np.full((H, W), 77, np.uint8)
    _, _, sse, ps = run_fused(rk, plan, flat, 1, want_recon=False)
    ref = orc.pipeline(n, p.That, flat, 1)[0]
    if ref <= 1e-9 * float(np.sum(flat.astype(np.float64) ** 2)):
        assert sse == 0.0 and ps == math.inf
    else:
        check_sse(sse, ref, H, W, n)
