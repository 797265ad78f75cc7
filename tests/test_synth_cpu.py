"""Seeded generators: shapes, ranges, determinism and edge sizes (CPU)."""
from __future__ import annotations

import numpy as np
import pytest

from paper_2304_07342_gb300 import synth


@pytest.mark.parametrize("n", [0, 1, 2, 31, 1000])
def test_edge_sizes(n):
    assert synth.quant_codes_laplace(n).shape == (n,)
    assert synth.markov_codes(n).shape == (n,)
    assert synth.sorted_indices(n).shape == (n,)
    assert synth.uniform_bytes(n).shape == (n,)


def test_block_boundaries_are_continuous():
    n = synth._BLOCK + 17
    m = synth.markov_codes(n, seed=4)
    assert m.min() >= 0 and m.max() <= 1023
    idx = synth.sorted_indices(n, seed=4)
    assert np.all(np.diff(idx.astype(np.int64)) >= 1)  # strictly increasing across blocks
    q = synth.quant_codes_laplace(n, seed=4)
    assert q.min() >= 0 and q.max() <= 1023


def test_deterministic_and_seed_sensitive():
    a = synth.quant_codes_laplace(5000, seed=1)
    assert np.array_equal(a, synth.quant_codes_laplace(5000, seed=1))
    assert not np.array_equal(a, synth.quant_codes_laplace(5000, seed=2))
    g = synth.gaussian_field((4, 8, 16), seed=0)
    assert g.dtype == np.float32 and g.shape == (4, 8, 16)
    assert np.array_equal(g, synth.gaussian_field((4, 8, 16), seed=0))


def test_quant_codes_shape_of_distribution():
    x = synth.workload_small()
    assert x.dtype == np.uint16 and x.size == 524_288
    runs = np.mean(x[1:] == x[:-1])
    assert 0.3 < runs < 0.5  # 30% copies plus equal Laplace draws
    assert abs(np.median(x.astype(np.int64)) - 512) <= 1


def test_batch_and_serving_recipes():
    sizes, kinds = synth.batch_buffers(1000, seed=0)
    assert sizes.min() >= 16 and sizes.max() <= 16 << 20 and np.all(sizes % 16 == 0)
    assert set(np.unique(kinds)) <= {0, 1, 2, 3}
    t, comp, sz, sym = synth.serving_trace(rate=100, duration=2.0, seed=0)
    assert np.all(np.diff(t) >= 0) and np.all(sz % sym == 0) and np.all(sz <= 64 << 20)
