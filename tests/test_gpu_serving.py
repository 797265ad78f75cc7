"""Serving loop: every request's result in the continuous-batching mix (and
in the plain per-request mode) is identical to the request run alone; the
loop finishes under a tight HBM budget."""
from __future__ import annotations

import numpy as np
import pytest
import torch

from paper_2304_07342_gb300 import lz, serve
from tests import gpu_util as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def codec():
    c = G.codec()
    yield c
    c.close()


@pytest.fixture(scope="module")
def trace(codec):
    return serve.build_trace(torch, codec, rate=2000.0, duration=0.3, seed=3,
                             pool_bytes=32 << 20, median_bytes=64 << 10, sigma=1.2,
                             cap_bytes=4 << 20)


def _alone(codec, r):
    if r.compress:
        out = torch.empty(r.n_out_max, dtype=torch.uint8, device="cuda")
        nb = torch.zeros(1, dtype=torch.int64, device="cuda")
        lz.lz_compress(codec.ctx, r.d_in, r.n_in, r.params, out.data_ptr(), r.n_out_max,
                       nb.data_ptr())
    else:
        out = torch.empty(max(r.n_out_max, 1), dtype=torch.uint8, device="cuda")
        nb = torch.zeros(1, dtype=torch.int64, device="cuda")
        lz.lz_decompress(codec.ctx, r.d_in, r.n_in, out.data_ptr(), r.n_out_max, nb.data_ptr())
    assert codec.sync() == lz.LZ_OK
    return out[: int(nb.item())].clone()


@pytest.mark.parametrize("budget", [40 << 30, 24 << 20])
def test_batched_results_equal_alone(codec, trace, budget):
    ref = {r.rid: _alone(codec, r) for r in trace.requests}
    seen = []

    def check(r, got, size):
        assert size == ref[r.rid].numel(), r.rid
        assert torch.equal(got, ref[r.rid]), r.rid
        seen.append(r.rid)

    stats = serve.run_batched(torch, codec, trace, budget_bytes=budget, on_done=check)
    assert sorted(seen) == [r.rid for r in trace.requests]
    assert stats["requests"] == len(trace.requests)
    assert np.isfinite(stats["p99_ms"]) and stats["p99_ms"] >= stats["p50_ms"] > 0
    assert stats["groups"] <= len(trace.requests)


def test_plain_results_equal_alone(codec, trace):
    ref = {r.rid: _alone(codec, r) for r in trace.requests[:200]}

    def check(r, got, size):
        if r.rid in ref:
            assert torch.equal(got, ref[r.rid]), r.rid

    stats = serve.run_plain(torch, codec, trace, budget_bytes=24 << 20, on_done=check)
    assert stats["requests"] == len(trace.requests)
