"""Batched form (uneven sizes, per-image plan and r) through the C ABI, against
the FP64 oracle; each image's result must be identical alone and in the mix, and
the graph-replayed batch must equal the immediate launch."""
import math

import numpy as np
import pytest

import synth_inputs as si
from test_gpu_parity import RECON_TOL, check_coef, check_recon_u8, check_sse

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RHOS = (0.2, 0.5, 0.7, 0.95)   # T1, T2, T3, T4


@pytest.fixture(scope="module")
def rk():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2111_14239_gb300 as rk
    return rk


def _mixed(n, seed, N=8):
    g = np.random.Generator(np.random.PCG64(seed))
    specs = []
    for i in range(n):
        H = int(g.integers(1, 40)) * N
        W = int(g.integers(1, 90)) * N
        plan = int(g.integers(0, len(RHOS)))
        r = int(g.integers(0, N * N + 1)) if i % 5 else min(N * N, [0, 1, N * N, 10, 37][i // 5 % 5])
        specs.append((H, W, plan, r, 7000 + i))
    return specs


def _alloc(specs, N):
    """Device images packed in one buffer (8-byte aligned rows), outputs per item."""
    imgs, entries, host = [], [], []
    for (H, W, plan, r, seed) in specs:
        img = si.ar1_image(H, W, 0.9, seed)
        host.append(img)
        ld = ((W + 7) // 8) * 8 + 8 * (seed % 3)   # uneven pitches
        d = torch.zeros((H, ld), dtype=torch.uint8, device="cuda")
        d[:, :W] = torch.from_numpy(img).cuda()
        rec = torch.zeros((H, ld + 8), dtype=torch.uint8, device="cuda")
        nblk = (H // N) * (W // N)
        zc = torch.full((max(nblk * r, 1),), float("nan"), device="cuda")
        imgs.append((d[:, :W], rec[:, :W], zc))
        entries.append((d[:, :W], plan, r, zc, rec[:, :W]))
    return host, imgs, entries


def _results(imgs, specs, sse, ps, N):
    out = []
    for (d, rec, zc), (H, W, plan, r, _) in zip(imgs, specs):
        nblk = (H // N) * (W // N)
        out.append((zc[:nblk * r].view(nblk, r).cpu().numpy(), rec.cpu().numpy(), sse, ps))
    return out


@pytest.mark.parametrize("N", [8, 4])
def test_items_against_oracle_and_alone(rk, orc, N):
    specs = _mixed(30, 11 if N == 8 else 12, N)
    plans = [rk.rklt_make(N, rho) for rho in RHOS]
    host, imgs, entries = _alloc(specs, N)
    items = rk.make_items(entries)
    sse = torch.zeros(len(specs), dtype=torch.float64, device="cuda")
    ps = torch.zeros(len(specs), dtype=torch.float32, device="cuda")
    rk.rklt_fused_items(items, plans, sse, ps)
    torch.cuda.synchronize()
    sse_h, ps_h = sse.cpu().numpy(), ps.cpu().numpy()
    mix = [(zc[: (H // N) * (W // N) * r].cpu().numpy().copy(), rec.cpu().numpy().copy())
           for (d, rec, zc), (H, W, _, r, _) in zip(imgs, specs)]
    for i, (H, W, plan, r, seed) in enumerate(specs):
        p = orc.Plan(N, RHOS[plan])
        sref, zref, rref = orc.pipeline(N, p.That, host[i], r, want_coef=True, want_recon=True)
        zc = mix[i][0].reshape(-1, r) if r else np.zeros((0, 0))
        if r:
            check_coef(zc, zref)
        check_sse(sse_h[i], sref, H, W, N)
        check_recon_u8(mix[i][1], rref, N)
        if sref > 0 and sse_h[i] > 0:
            assert ps_h[i] == pytest.approx(10 * math.log10(255 ** 2 * H * W / sse_h[i]), abs=1e-4)
    # alone: a batch of one item gives bit-identical outputs (the mix, with more than
    # three (plan, support) groups, ran as one queue launch; one item runs as one group)
    for i in (0, 3, 17, 29):
        one = rk.make_items([entries[i]])
        s1 = torch.zeros(1, dtype=torch.float64, device="cuda")
        p1 = torch.zeros(1, dtype=torch.float32, device="cuda")
        rk.rklt_fused_items(one, plans, s1, p1)
        torch.cuda.synchronize()
        H, W, _, r, _ = specs[i]
        assert s1.item() == sse_h[i] and (p1.item() == ps_h[i] or (math.isnan(p1.item()) and math.isnan(ps_h[i])))
        d, rec, zc = imgs[i]
        assert np.array_equal(rec.cpu().numpy(), mix[i][1])
        assert np.array_equal(zc[: (H // N) * (W // N) * r].cpu().numpy(), mix[i][0])


def test_graph_batch_matches_immediate(rk):
    N = 8
    specs = _mixed(24, 13, N)
    plans = [rk.rklt_make(N, rho) for rho in RHOS]
    host, imgs, entries = _alloc(specs, N)
    items = rk.make_items(entries)
    s0 = torch.zeros(len(specs), dtype=torch.float64, device="cuda")
    p0 = torch.zeros(len(specs), dtype=torch.float32, device="cuda")
    rk.rklt_fused_items(items, plans, s0, p0)
    torch.cuda.synchronize()
    rec0 = [rec.cpu().numpy().copy() for (_, rec, _) in imgs]
    s1 = torch.zeros(len(specs), dtype=torch.float64, device="cuda")
    p1 = torch.zeros(len(specs), dtype=torch.float32, device="cuda")
    b = rk.rklt_batch_create(items, plans, s1, p1, autotune=True)
    info = b.info()
    assert info["threads"] in (128, 256) and info["groups"] >= 4 and info["tuned_us"] > 0
    for (_, rec, _) in imgs:
        rec.zero_()
    s1.zero_()
    for _ in range(3):
        b.run()
    torch.cuda.synchronize()
    assert np.array_equal(s1.cpu().numpy(), s0.cpu().numpy())
    assert np.array_equal(p1.cpu().numpy(), p0.cpu().numpy(), equal_nan=True)
    for k, (_, rec, _) in enumerate(imgs):
        assert np.array_equal(rec.cpu().numpy(), rec0[k])
    b.close()
    rk.rklt_device_status()


def test_batch_rejects_bad_items(rk):
    plans = [rk.rklt_make(16, 0.95)]
    d = torch.zeros((16, 16), dtype=torch.uint8, device="cuda")
    s = torch.zeros(1, dtype=torch.float64, device="cuda")
    p = torch.zeros(1, device="cuda")
    with pytest.raises(rk.RklTError) as e:
        rk.rklt_fused_items(rk.make_items([(d, 0, 8, None, None)]), plans, s, p)
    assert e.value.status == 8     # N = 16 is not batched
    plans = [rk.rklt_make(8, 0.95)]
    with pytest.raises(rk.RklTError) as e:
        rk.rklt_fused_items(rk.make_items([(d[:, 1:9], 0, 8, None, None)]), plans, s, p)
    assert e.value.status == 8     # misaligned rows
    with pytest.raises(rk.RklTError) as e:
        rk.rklt_fused_items(rk.make_items([(d, 1, 8, None, None)]), plans, s, p)
    assert e.value.status == 1     # plan index out of range
