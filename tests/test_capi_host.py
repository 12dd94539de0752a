"""Host-side tests of the C-ABI library (no GPU needed): it loads, exports every
entry point declared in include/rklt.h, and builds plans (host FP64) identical
to the oracle's; bad arguments return the documented status codes."""
import ctypes

import numpy as np
import pytest

import golden_io

rk = pytest.importorskip("paper_2111_14239_gb300")

RHOS = [0.1, 0.2, 0.3, 0.4, 0.5, 0.6, 0.7, 0.8, 0.9, 0.95, 0.99]


def test_exports_every_header_symbol():
    names = rk.header_symbols()
    assert len(names) >= 18
    for name in names:
        assert hasattr(rk.lib, name), name
        getattr(rk.lib, name)  # resolves through dlsym


@pytest.mark.parametrize("n", [4, 8, 16, 32])
def test_plans_match_oracle(orc, n):
    for rho in RHOS:
        plan = rk.rklt_make(n, rho)
        T, s, orth = plan.info()
        ref = orc.Plan(n, rho)
        assert np.array_equal(T.astype(np.int32), ref.T), (n, rho)
        assert np.max(np.abs(s - ref.s)) < 1e-15
        assert orth == ref.orthogonal
        assert plan.N == n and plan.alpha == pytest.approx(rk.default_alpha(n))


def test_plans_reproduce_table1():
    t1 = golden_io.table1()
    for rho, name in ((0.2, "T1"), (0.5, "T2"), (0.7, "T3"), (0.85, "T4")):
        T, s, _ = rk.rklt_make(8, rho).info()
        assert np.array_equal(T.astype(np.int64), t1[name]["T"])
        assert np.allclose(s, t1[name]["s"], atol=1e-15, rtol=0)
        T2, s2, _ = rk.rklt_make_from_matrix(8, t1[name]["T"]).info()
        assert np.array_equal(T2, T) and np.array_equal(s2, s)


def test_status_codes():
    h = ctypes.c_void_p()
    assert rk.lib.rklt_make(5, 0.5, ctypes.byref(h)) == 1
    assert rk.lib.rklt_make(8, 0.0, ctypes.byref(h)) == 1
    assert rk.lib.rklt_make(8, 1.0, ctypes.byref(h)) == 1
    assert rk.lib.rklt_make(8, 0.5, None) == 1
    # alpha past 3/(2 gamma) rounds some entry to 2
    assert rk.lib.rklt_make_alpha(8, 0.5, 4.0, ctypes.byref(h)) == 3
    assert b"outside" in rk.lib.rklt_last_error()
    # alpha = 2 at N = 32 rounds everything to zero
    assert rk.lib.rklt_make_alpha(32, 0.95, 2.0, ctypes.byref(h)) == 3
    # a matrix without the KLT row parity
    bad = np.eye(8, dtype=np.int8)
    assert rk.lib.rklt_make_from_matrix(8, bad.ctypes.data, ctypes.byref(h)) == 3
    # singular: repeated row
    T = golden_io.table1()["T4"]["T"].astype(np.int8).copy()
    T[2] = T[0]
    assert rk.lib.rklt_make_from_matrix(8, T.ctypes.data, ctypes.byref(h)) == 3
    assert rk.lib.rklt_status_string(7) == b"RKLT_ERR_TIMEOUT"


def test_argument_checks_without_gpu():
    """Shape and argument errors are caught on the host before any launch."""
    plan = rk.rklt_make(8, 0.95)
    d = ctypes.c_void_p(16)  # never dereferenced: validation fails first
    assert rk.lib.rklt_fused(plan.handle, d, 12, 16, 16, 10, None, None, 0, d, d, None) == 2   # H % 8
    assert rk.lib.rklt_fused(plan.handle, d, 16, 16, 8, 10, None, None, 0, d, d, None) == 2    # ld < W
    assert rk.lib.rklt_fused(plan.handle, d, 16, 16, 16, 65, None, None, 0, d, d, None) == 1   # r > 64
    assert rk.lib.rklt_fused(plan.handle, d, 16, 16, 16, 10, None, None, 0, None, d, None) == 1
    assert rk.lib.rklt_zonal(plan.handle, d, 4, 10, d, None) == 1                           # aliasing, r < 64
    assert rk.lib.rklt_fused_batched(plan.handle, d, 2, 16, 16, 16, 100, 10, None, None, 0, 0, d, d, None) == 2


def test_quality_and_quantiser_argument_checks_without_gpu():
    """The MSSIM, fused-MSSIM and quantiser entry points reject bad arguments on the
    host, before any launch (documented status codes: 1 argument, 2 shape,
    8 unsupported)."""
    plan = rk.rklt_make(8, 0.95)
    d = ctypes.c_void_p(16)  # never dereferenced: validation fails first
    fm = rk.lib.rklt_fused_mssim
    assert fm(plan.handle, d, 1, 12, 16, 16, 0, 10, None, None, 0, 0, d, d, d, None) == 2    # H % 8
    assert fm(plan.handle, d, 1, 16, 16, 8, 0, 10, None, None, 0, 0, d, d, d, None) == 2     # ld < W
    assert fm(plan.handle, d, 1, 16, 16, 16, 0, 65, None, None, 0, 0, d, d, d, None) == 1    # r > 64
    assert fm(plan.handle, d, 1, 16, 16, 16, 0, 10, None, None, 0, 0, d, d, None, None) == 1  # no mssim
    assert fm(plan.handle, d, 0, 16, 16, 16, 0, 10, None, None, 0, 0, d, d, d, None) == 1    # nimg 0
    assert fm(plan.handle, d, 2, 16, 16, 16, 100, 10, None, None, 0, 0, d, d, d, None) == 2  # image stride
    assert fm(None, d, 1, 16, 16, 16, 0, 10, None, None, 0, 0, d, d, d, None) == 1          # no plan
    ms = rk.lib.rklt_mssim
    assert ms(d, d, 1, 16, 16, 8, 0, 16, 0, d, None) == 2       # ldx < W
    assert ms(d, d, 1, 16, 16, 16, 0, 16, 0, None, None) == 1   # no output
    assert ms(d, d, 0, 16, 16, 16, 0, 16, 0, d, None) == 1      # nimg 0
    q = rk.lib.rklt_fused_quant
    good = np.full(64, 4.0)
    bad = good.copy()
    bad[5] = 0.0
    assert q(plan.handle, d, 1, 16, 16, 16, 0, 10, bad.ctypes.data, None, None, 0, 0, d, d, None) == 1   # Q <= 0
    assert q(plan.handle, d, 1, 16, 16, 16, 0, 10, None, None, None, 0, 0, d, d, None) == 1              # no Q
    assert q(plan.handle, d, 1, 12, 16, 16, 0, 10, good.ctypes.data, None, None, 0, 0, d, d, None) == 2   # H % 8
    dct = rk.rklt_make_dct(8)
    assert q(dct.handle, d, 1, 16, 16, 16, 0, 10, good.ctypes.data, None, None, 0, 0, d, d, None) == 8    # real plan


def test_batch_item_checks_without_gpu():
    """Uneven-batch items are validated on the host before anything is queued: plan
    index, r, shape, pitch, and the N-byte row alignment the batch kernels read with."""
    plans8 = [rk.rklt_make(8, 0.95), rk.rklt_make(8, 0.5)]
    arr8 = rk._plan_array(plans8)
    d = ctypes.c_void_p(16)

    def item(**kw):
        it = rk.RklTItem()
        it.d_img, it.H, it.W, it.ld, it.plan, it.r = 4096, 64, 64, 64, 0, 10
        it.d_zcoef, it.d_recon, it.ld_recon = None, None, 0
        for k, v in kw.items():
            setattr(it, k, v)
        return (rk.RklTItem * 1)(it)

    def call(items, arr=arr8, nplans=2):
        return rk.lib.rklt_fused_items(items, 1, ctypes.cast(arr, ctypes.c_void_p), nplans, d, d, None)

    assert call(item(plan=2)) == 1            # plan index out of range
    assert call(item(r=65)) == 1              # r > 64
    assert call(item(H=60)) == 2              # H % 8
    assert call(item(ld=32)) == 2             # ld < W
    assert call(item(d_img=4100)) == 8        # rows not 8-byte aligned
    assert call(item(d_img=None)) == 1        # no image
    assert call(item(d_recon=4096, ld_recon=32)) == 2
    plans16 = [rk.rklt_make(16, 0.95)]
    assert call(item(), rk._plan_array(plans16), 1) == 8   # N = 16: not a batch size
    mixed = [rk.rklt_make(8, 0.95), rk.rklt_make(4, 0.95)]
    assert call(item(), rk._plan_array(mixed), 2) == 1     # plans of different N
