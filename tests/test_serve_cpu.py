"""Host logic of the serving loop that needs no GPU: the budget allocator."""
from __future__ import annotations

import numpy as np

from paper_2304_07342_gb300.serve import Arena


def test_arena_first_fit_merge_and_budget():
    a = Arena(4096)
    x = a.alloc(1000)   # 1024
    y = a.alloc(1000)   # 1024
    z = a.alloc(2048)
    assert (x, y, z) == (0, 1024, 2048)
    assert a.alloc(1) == -1          # budget exhausted
    a.release(y, 1000)
    assert a.alloc(2000) == -1       # a 1024 hole only
    a.release(x, 1000)               # merges into 2048 at 0
    assert a.alloc(2000) == 0
    a.release(0, 2000)
    a.release(z, 2048)
    assert a.free == [(0, 4096)]


def test_arena_random_never_overlaps():
    rng = np.random.default_rng(0)
    a = Arena(1 << 20)
    live = {}
    for step in range(3000):
        if live and rng.random() < 0.45:
            k = list(live)[int(rng.integers(0, len(live)))]
            a.release(k, live.pop(k))
        else:
            n = int(rng.integers(1, 40_000))
            o = a.alloc(n)
            if o >= 0:
                live[o] = n
        spans = sorted((o, o + Arena._round(n)) for o, n in live.items())
        for (a0, a1), (b0, b1) in zip(spans, spans[1:]):
            assert a1 <= b0
        assert all(0 <= s0 and s1 <= 1 << 20 for s0, s1 in spans)


def test_request_larger_than_budget_is_refused():
    import pytest

    from paper_2304_07342_gb300.serve import Request, Trace, check_budget
    ok = Request(0, 0.0, True, 0, 1000, None, 1000, 1000)
    big = Request(1, 0.001, True, 0, 5000, None, 4097, 4097)
    check_budget(Trace([ok]), 4096)  # fits
    with pytest.raises(ValueError):
        check_budget(Trace([ok, big]), 4096)  # 4097 rounds to 4352 > 4096
    check_budget(Trace([ok, big]), 4352)
