"""Host logic of the serving loop (no GPU): the native loop's first-fit arena and the
request sizes its admission uses."""
import pytest

rk = pytest.importorskip("paper_2111_14239_gb300")
serve = pytest.importorskip("paper_2111_14239_gb300.serve")


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_native_copy_pool_stages_every_row(seed):
    """The request loop's staging workers: many rounds in a row (each round hands the
    workers a new set of chunks), every row copied exactly, padding untouched."""
    st = rk.lib.rklt_copypool_selftest(seed, 300)
    assert st == 0, rk.lib.rklt_last_error()


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_native_arena_never_overlaps_and_coalesces(seed):
    st = rk.lib.rklt_arena_selftest(seed, 5000)
    assert st == 0, rk.lib.rklt_last_error()


def test_request_sizes():
    # rows padded to 16 bytes; coefficients [blocks][r] FP32
    assert serve.bytes_needed(64, 72, 10) == (64 * 80, 64 * 80, 8 * 9 * 10 * 4)
    assert serve.bytes_needed(8, 16, 0) == (128, 128, 0)
    assert serve._align(1) == 256 and serve._align(256) == 256 and serve._align(257) == 512


def test_server_create_argument_checks_without_gpu():
    """The request loop's configuration is checked before anything is allocated."""
    import ctypes
    plans = [rk.rklt_make(8, 0.95)]
    arr = rk._plan_array(plans)
    out = ctypes.c_void_p()
    create = rk.lib.rklt_server_create
    P = lambda a: ctypes.cast(a, ctypes.c_void_p)
    assert create(P(arr), 1, 1024, 4, 64, ctypes.byref(out)) == 1          # budget below 4 KB
    assert create(P(arr), 1, 1 << 20, 0, 64, ctypes.byref(out)) == 1       # no stream
    assert create(P(arr), 1, 1 << 20, 4, 5000, ctypes.byref(out)) == 1     # batch above 4096
    assert create(P(arr), 0, 1 << 20, 4, 64, ctypes.byref(out)) == 1       # no plan
    mixed = rk._plan_array([rk.rklt_make(8, 0.95), rk.rklt_make(4, 0.95)])
    assert create(P(mixed), 2, 1 << 20, 4, 64, ctypes.byref(out)) == 1     # two block sizes
    n16 = rk._plan_array([rk.rklt_make(16, 0.95)])
    assert create(P(n16), 1, 1 << 20, 4, 64, ctypes.byref(out)) == 8       # N = 16
    assert out.value is None
