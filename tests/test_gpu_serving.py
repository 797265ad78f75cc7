"""Serving loop: every request's result in the continuous-batching mix (and
in the plain per-request mode) is checked against the CPU oracle -- a
compress request's stream byte for byte against the oracle's stream of the
same input and parameters, a decompress request's output against the
original input -- with a generous and a tight HBM budget, over requests of
1-, 2- and 4-byte symbols.  Requests are independent (chunks are, section
3.3.1), so a request's result may not depend on what it was batched with."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
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
                             pool_bytes=32 << 20, median_bytes=32 << 10, sigma=1.2,
                             cap_bytes=2 << 20)


@pytest.fixture(scope="module")
def expected(trace):
    """Oracle result of every request: the stream for a compress request, the
    original bytes for a decompress request."""
    out = {}
    for r in trace.requests:
        src = r.source.cpu().numpy()
        if r.compress:
            out[r.rid] = oracle.compress(src, oracle.Params(*(r.params.S, r.params.C, r.params.W,
                                                             r.params.m, r.params.M)))
        else:
            out[r.rid] = src
    return out


def test_trace_covers_every_kind(trace):
    kinds = {(r.compress, r.params.S) for r in trace.requests}
    assert kinds == {(c, S) for c in (True, False) for S in (1, 2, 4)}


@pytest.mark.parametrize("budget", [40 << 30, 24 << 20])
def test_batched_results_equal_oracle(codec, trace, expected, budget):
    seen = []

    def check(r, got, size):
        ref = expected[r.rid]
        assert size == ref.size, r.rid
        assert np.array_equal(got.cpu().numpy(), ref), r.rid
        seen.append(r.rid)

    stats = serve.run_batched(torch, codec, trace, budget_bytes=budget, on_done=check)
    assert sorted(seen) == [r.rid for r in trace.requests]
    assert stats["requests"] == len(trace.requests)
    assert np.isfinite(stats["p99_ms"]) and stats["p99_ms"] >= stats["p50_ms"] > 0
    assert stats["groups"] <= len(trace.requests)


def test_plain_results_equal_oracle(codec, trace, expected):
    seen = []

    def check(r, got, size):
        ref = expected[r.rid]
        assert size == ref.size, r.rid
        assert np.array_equal(got.cpu().numpy(), ref), r.rid
        seen.append(r.rid)

    stats = serve.run_plain(torch, codec, trace, budget_bytes=24 << 20, on_done=check)
    assert sorted(seen) == [r.rid for r in trace.requests]
    assert stats["requests"] == len(trace.requests)


def test_batched_groups_form_under_load(codec):
    """At an arrival rate the GPU cannot keep up with one request at a time,
    requests queue and groups of several form; every result still matches
    the oracle."""
    tr = serve.build_trace(torch, codec, rate=200000.0, duration=0.004, seed=11,
                           pool_bytes=16 << 20, median_bytes=16 << 10, sigma=1.0,
                           cap_bytes=1 << 20)
    exp = {}
    for r in tr.requests:
        src = r.source.cpu().numpy()
        exp[r.rid] = (oracle.compress(src, oracle.Params(r.params.S, r.params.C, r.params.W,
                                                         r.params.m, r.params.M))
                      if r.compress else src)
    bad = []

    def check(r, got, size):
        ref = exp[r.rid]
        if size != ref.size or not np.array_equal(got.cpu().numpy(), ref):
            bad.append(r.rid)

    stats = serve.run_batched(torch, codec, tr, budget_bytes=1 << 30, on_done=check)
    assert not bad
    assert stats["mean_group"] > 2, stats


def test_oversize_request_is_refused(codec, trace):
    with pytest.raises(ValueError):
        serve.run_batched(torch, codec, trace, budget_bytes=4096)
    with pytest.raises(ValueError):
        serve.run_plain(torch, codec, trace, budget_bytes=4096)
