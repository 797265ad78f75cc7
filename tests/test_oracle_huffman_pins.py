"""Pins for the Huffman-stage oracle (huffref.c), by things other than itself:

* the textbook worked example of Huffman coding (six symbols with counts
  45/13/12/16/9/5, optimal cost 224);
* a heap-based Huffman written here (a different algorithm from
  package-merge) giving the same optimal cost whenever no length exceeds
  the limit;
* brute force over every length vector on tiny alphabets for the
  length-limited optimum;
* the canonical-code worked example of the DEFLATE specification (RFC 1951
  section 3.2.2: lengths 3,3,3,3,3,2,4,4 give codes 010 011 100 101 110 00
  1110 1111);
* stream invariants: round trip, the size identity, the sub-block offsets,
  and rejection of corrupt streams.
"""
from __future__ import annotations

import heapq
import itertools
import struct

import numpy as np
import pytest

import oracle


def huffman_cost_heap(counts):
    """Optimal (unlimited) prefix-code cost by the textbook heap merge."""
    h = [c for c in counts if c > 0]
    if len(h) <= 1:
        return sum(h)  # one symbol: one bit each
    heapq.heapify(h)
    cost = 0
    while len(h) > 1:
        a, b = heapq.heappop(h), heapq.heappop(h)
        cost += a + b
        heapq.heappush(h, a + b)
    return cost


def hist_of(counts: dict) -> np.ndarray:
    h = np.zeros(256, np.uint64)
    for s, c in counts.items():
        h[s] = c
    return h


def kraft(lengths) -> float:
    return sum(2.0 ** -int(l) for l in lengths if l)


def test_textbook_example():
    h = hist_of({ord(c): n for c, n in zip("abcdef", (45, 13, 12, 16, 9, 5))})
    L = oracle.huff_lengths(h)
    assert int((h * L).sum()) == 224
    assert sorted(int(L[ord(c)]) for c in "abcdef") == [1, 3, 3, 3, 4, 4]
    assert L[ord("a")] == 1 and kraft(L) == 1.0


def test_optimal_cost_equals_heap_huffman():
    rng = np.random.default_rng(1)
    for trial in range(200):
        n = int(rng.integers(2, 257))
        counts = rng.integers(1, 1000, n) * (rng.random(n) < 0.9)
        counts[:2] = np.maximum(counts[:2], 1)
        h = np.zeros(256, np.uint64)
        h[rng.permutation(256)[:n]] = counts
        L = oracle.huff_lengths(h)
        unl = huffman_cost_heap(h.tolist())
        if int(L.max()) < oracle.HUFF_MAX_LEN:  # the limit cannot bind
            assert int((h * L).sum()) == unl, trial
        else:
            assert int((h * L).sum()) >= unl
        assert abs(kraft(L) - 1.0) < 1e-12
        assert all((L > 0) == (h > 0))


@pytest.mark.parametrize("max_len", [2, 3, 4])
def test_length_limited_optimum_brute_force(max_len):
    """Every length vector with lengths 1..max_len and Kraft sum <= 1: the
    least cost equals package-merge's."""
    rng = np.random.default_rng(max_len)
    for trial in range(60):
        n = int(rng.integers(2, min(7, 2 ** max_len + 1)))
        counts = [int(c) for c in rng.integers(1, 60, n)]
        if trial % 3 == 0:
            counts = [1, 1, 2, 3, 5, 8, 13][:n]
        best = min(sum(c * l for c, l in zip(counts, ls))
                   for ls in itertools.product(range(1, max_len + 1), repeat=n)
                   if sum(2.0 ** -l for l in ls) <= 1.0)
        L = oracle.huff_lengths(hist_of(dict(enumerate(counts))), max_len)
        assert sum(c * int(L[i]) for i, c in enumerate(counts)) == best
        assert int(L[:n].max()) <= max_len and abs(kraft(L) - 1.0) < 1e-12


def test_limit_binds_on_fibonacci_counts():
    fib = [1, 1]
    while len(fib) < 30:
        fib.append(fib[-1] + fib[-2])
    h = hist_of(dict(enumerate(fib)))
    L = oracle.huff_lengths(h)
    assert int(L.max()) == oracle.HUFF_MAX_LEN  # unlimited Huffman would go to 29
    assert abs(kraft(L) - 1.0) < 1e-12
    assert int((h * L).sum()) > huffman_cost_heap(fib)


def test_canonical_codes_rfc1951_example():
    L = np.zeros(256, np.uint8)
    L[ord("A"):ord("H") + 1] = [3, 3, 3, 3, 3, 2, 4, 4]
    C = oracle.huff_codes(L)
    want = ["010", "011", "100", "101", "110", "00", "1110", "1111"]
    got = [format(int(C[ord(c)]), f"0{int(L[ord(c)])}b") for c in "ABCDEFGH"]
    assert got == want


def test_canonical_codes_prefix_free():
    rng = np.random.default_rng(5)
    for _ in range(30):
        h = np.zeros(256, np.uint64)
        h[rng.permutation(256)[: int(rng.integers(2, 257))]] = rng.integers(1, 10**6, 256)[:1]
        h[h > 0] = rng.integers(1, 10**6, int((h > 0).sum()))
        L = oracle.huff_lengths(h)
        C = oracle.huff_codes(L)
        words = sorted(format(int(C[s]), f"0{int(L[s])}b") for s in range(256) if L[s])
        for a, b in zip(words, words[1:]):
            assert not b.startswith(a)


def _layout(stream):
    s = np.asarray(stream, np.uint8)
    assert bytes(s[:4]) == b"GHF1"
    blk, n = struct.unpack_from("<IQ", s.tobytes(), 4)
    nb = (n + blk - 1) // blk
    L = s[16:272]
    ends = s[272:272 + 8 * nb].view(np.uint64).astype(np.int64)
    table = np.diff(np.concatenate([[0], ends]))  # bytes of each block
    subs = s[272 + 8 * nb: 272 + 8 * nb + 128 * nb].view(np.uint32).reshape(nb, 32)
    return n, nb, L, table, subs, 272 + 136 * nb


@pytest.mark.parametrize("kind", ["empty", "one", "two", "all256", "random", "skewed", "lzss"])
def test_stream_round_trip_and_size_identity(kind):
    rng = np.random.default_rng(11)
    x = {
        "empty": np.zeros(0, np.uint8),
        "one": np.full(70_000, 42, np.uint8),
        "two": rng.integers(0, 2, 50_001).astype(np.uint8) * 200,
        "all256": np.arange(256 * 300, dtype=np.uint32).astype(np.uint8),
        "random": rng.integers(0, 256, 100_003).astype(np.uint8),
        "skewed": np.minimum(rng.geometric(0.2, 200_000), 255).astype(np.uint8),
        "lzss": oracle.compress(np.repeat(rng.integers(0, 9, 40_000), 3).astype(np.uint16),
                                oracle.Params(2, 4096, 128, 3, 255)),
    }[kind]
    s = oracle.huff_compress(x)
    assert np.array_equal(oracle.huff_decompress(s), x)
    n, nb, L, table, subs, bits_at = _layout(s)
    assert n == x.size and nb == (x.size + 32767) // 32768
    assert s.size == bits_at + int(table.sum())
    for b in range(nb):
        blk = x[b * 32768:(b + 1) * 32768]
        lens = L[blk].astype(np.int64)
        assert table[b] == (lens.sum() + 31) // 32 * 4
        for j in range(32):
            assert subs[b, j] == lens[: j * 1024].sum()
    if kind == "one":
        assert L[42] == 1 and int((L > 0).sum()) == 1


def test_decoder_rejects_corruption():
    x = np.minimum(np.random.default_rng(3).geometric(0.1, 40_000), 255).astype(np.uint8)
    good = bytearray(oracle.huff_compress(x).tobytes())
    assert oracle.huff_decompress_status(bytes(good))[0] == oracle.OK
    n, nb, L, table, subs, bits_at = _layout(np.frombuffer(bytes(good), np.uint8))
    used = [int(i) for i in np.nonzero(L)[0]]
    cases = []
    b = bytearray(good); b[0] = ord("X"); cases.append(b)                    # magic
    b = bytearray(good); b[5] = 0; cases.append(b)                           # block size
    b = bytearray(good); b[16 + used[-1]] = 13; cases.append(b)              # length > 12
    b = bytearray(good); b[16 + used[-1]] = 0; cases.append(b)               # incomplete code
    b = bytearray(good); b[272] += 4; cases.append(b)                        # block end
    b = bytearray(good); b[272 + 8 * nb + 4] += 1; cases.append(b)           # sub offset
    cases.append(good[:-4])                                                  # truncated
    for i, c in enumerate(cases):
        assert oracle.huff_decompress_status(bytes(c))[0] == oracle.ECORRUPT, i
