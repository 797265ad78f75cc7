"""The compressor's literal pre-check (a Bloom filter over symbol keys that
lets a chunk without repeats skip the hash chains) must never change the
stream: streams stay byte-identical to the oracle's.

The inputs are random symbols (no repeats, so the pre-check is taken) with
one planted repeat of m or more symbols, placed where the exactness
argument is delicate: source and target in one 32-position slab (either
order of the atomic unit), in adjacent slabs, in one group of 8 slabs or
across two, at offsets just inside and
just outside the window, shorter than m, overlapping (offset < m), and at
the very end of the chunk.  Random data with many near-duplicate keys (small
alphabets in the high bytes) exercises the exact check of flagged
positions.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from oracle import Params
from tests import gpu_util as G

pytestmark = pytest.mark.gpu

DT = {1: np.uint8, 2: np.uint16, 4: np.uint32}


@pytest.fixture(scope="module")
def codec():
    c = G.codec()
    yield c
    c.close()


def distinct_random(n_sym: int, S: int, seed: int) -> np.ndarray:
    """Random symbols with no value repeated (S = 2: a shuffled range)."""
    rng = np.random.default_rng(seed)
    if S == 2:
        return rng.permutation(1 << 16)[:n_sym].astype(np.uint16)
    return (rng.permutation(n_sym).astype(np.uint64) * 2654435761 + 12345).astype(np.uint32)


def check(codec, x: np.ndarray, P: Params):
    ref = oracle.compress(x, P)
    got = G.gpu_compress(codec, x, P)
    assert np.array_equal(got, ref), G.first_difference(got, ref)
    assert np.array_equal(G.gpu_decompress(codec, got), x.view(np.uint8))


CASES = []
for S, C, W, m in ((4, 8192, 256, 2), (4, 4096, 128, 1), (4, 8192, 256, 3),
                   (2, 4096, 128, 3), (2, 2048, 64, 2)):
    k = C // S
    for tgt, d, ln in ((40, 5, m), (37, 3, m + 2), (70, 40, m), (64, 1, 4), (63, 2, 4),
                       (300, W, m), (300, W + 1, m), (500, W - 1, m + 1),
                       (k - m, 17, m), (k - m, W, m), (100, 9, max(1, m - 1)),
                       (33, 31, m), (95, 31, m), (31, 30, m),
                       # farther apart inside the first 8 slabs, and across
                       # their end
                       (200, 100, m), (255, 200, m), (250, 60, m + 1), (260, 10, m),
                       (290, 250, m), (511, 255, m)):
        CASES.append((S, C, W, m, tgt, d, ln))


@pytest.mark.parametrize("S,C,W,m,tgt,d,ln", CASES)
def test_planted_repeat(codec, S, C, W, m, tgt, d, ln):
    """Chunk 1 of 3 carries one repeat: symbols [tgt, tgt+ln) copy
    [tgt-d, tgt-d+ln); chunks 0 and 2 have none."""
    k = C // S
    x = distinct_random(3 * k, S, seed=tgt * 7 + d)
    base = k  # chunk 1
    if tgt - d >= 0 and tgt + ln <= k:
        x[base + tgt: base + tgt + ln] = x[base + tgt - d: base + tgt - d + ln].copy()
    check(codec, x, Params(S, C, W, m, 255))


@pytest.mark.parametrize("S,m", [(4, 2), (4, 1), (2, 3), (2, 1)])
def test_near_duplicate_keys(codec, S, m):
    """Symbols from an alphabet of k/2 values, each recurring about a dozen
    times at random places: many flagged positions, some true repeats
    inside the window and many beyond it."""
    rng = np.random.default_rng(S * 10 + m)
    k = 8192 // S
    n = 6 * k
    # each of k/2 values recurs about twelve times, at random places
    x = (rng.permutation(n) % (k // 2)).astype(DT[S])
    check(codec, x, Params(S, 8192, 64, m, 255))
    # and the same with a few values repeated within the window
    y = x.copy()
    y[100::997] = y[90::997][: y[100::997].size]
    check(codec, y, Params(S, 8192, 64, m, 255))
