"""Host logic of the serving loop (no GPU): the first-fit arena allocator and the
frozen-heap scope around request loops."""
import random

import pytest

serve = pytest.importorskip("paper_2111_14239_gb300.serve")


def test_arena_first_fit_and_coalescing():
    a = serve.Arena(1 << 20)
    offs = [a.alloc(1000) for _ in range(10)]
    assert all(o is not None and o % 256 == 0 for o in offs)
    assert len(set(offs)) == 10
    for o in offs[::2]:
        a.release(o, 1000)
    for o in offs[1::2]:
        a.release(o, 1000)
    assert a.free == [(0, 1 << 20)] and a.used == 0


def test_arena_random_churn_never_overlaps():
    rng = random.Random(1)
    a = serve.Arena(1 << 16)
    live = {}
    for step in range(2000):
        if live and rng.random() < 0.5:
            o = rng.choice(list(live))
            a.release(o, live.pop(o))
        else:
            n = rng.randint(1, 4000)
            o = a.alloc(n)
            if o is not None:
                for p, m in live.items():
                    assert o + serve._align(n) <= p or p + serve._align(m) <= o
                live[o] = n
    for o, n in list(live.items()):
        a.release(o, n)
    assert a.free == [(0, 1 << 16)]


def test_frozen_heap_scope():
    import gc
    saved = gc.get_freeze_count()
    gc.unfreeze()
    try:
        keep = [[i] for i in range(1000)]
        with serve.frozen_heap():
            assert gc.get_freeze_count() >= len(keep)
            assert gc.isenabled()
        assert gc.get_freeze_count() == 0
        with pytest.raises(RuntimeError):
            with serve.frozen_heap():
                raise RuntimeError("the heap is unfrozen on the way out")
        assert gc.get_freeze_count() == 0
        # a heap frozen by someone else stays frozen
        gc.freeze()
        with serve.frozen_heap():
            pass
        assert gc.get_freeze_count() > 0
    finally:
        gc.unfreeze()
        if saved:
            gc.freeze()
