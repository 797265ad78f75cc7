"""Pins for the CPU oracle: checks against things other than itself.

* hand-worked golden fixtures (tests/golden/*.txt, each citing its passage);
* brute force over all offsets and lengths on tiny inputs (a different route:
  slice comparison, longest length first);
* closed forms: constant runs, period-q sequences;
* invariants: round trip, size identity, token validity, chunk independence;
* decoder rejects corrupt streams.
"""
from __future__ import annotations

import glob
import itertools
import os

import numpy as np
import pytest

import oracle
from oracle import Params
from tests import glz1_reader

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --- brute force (definition, different route) --------------------------------

def brute_longest(sym: list, p: int, W: int, M: int):
    """All (d, l): for each offset take the longest l <= min(M, d, k-p) whose
    source slice equals the look-ahead slice, trying l from the top down."""
    k = len(sym)
    best, best_d = 0, 0
    for d in range(1, min(W, p) + 1):
        for l in range(min(M, d, k - p), 0, -1):
            if sym[p:p + l] == sym[p - d:p - d + l]:
                break
        else:
            l = 0
        if l > best:
            best, best_d = l, d
    return best, best_d


def brute_parse(sym: list, W: int, m: int, M: int):
    toks, p = [], 0
    while p < len(sym):
        l, d = brute_longest(sym, p, W, M)
        if l >= m:
            toks.append((l, d))
            p += l
        else:
            toks.append((1, 0))
            p += 1
    return toks


def symbols(b: bytes, S: int) -> list:
    return [b[i:i + S] for i in range(0, len(b), S)]


# --- golden fixtures ----------------------------------------------------------

def _load_fixture(path):
    spec = {}
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        key, _, val = line.partition(" ")
        spec[key] = val
    params = dict(kv.split("=") for kv in spec["params"].split())
    P = Params(*(int(params[k]) for k in ("S", "C", "W", "m", "M")))
    if "input_hex" in spec:
        data = bytes.fromhex(spec["input_hex"])
    elif "input_ranges" in spec:
        dt, *ns = spec["input_ranges"].split()
        data = np.concatenate([np.arange(int(n)) for n in ns]).astype(
            {"u8": np.uint8, "u16": np.uint16, "u32": np.uint32}[dt]).tobytes()
    else:
        dt, n, v = spec["input_const"].split()
        data = np.full(int(n), int(v),
                       {"u8": np.uint8, "u16": np.uint16}[dt]).tobytes()
    chunks = []
    for part in spec["tokens"].split("|"):
        toks = []
        for t in part.split():
            if t.startswith("L*"):
                toks += [(1, 0)] * int(t[2:])
            elif t == "L":
                toks.append((1, 0))
            else:
                l, d = t.split("@")
                toks.append((int(l), int(d)))
        chunks.append(toks)
    stream = bytes.fromhex(spec["stream_hex"].replace(" ", "")) if "stream_hex" in spec else None
    mp = bytes.fromhex(spec["match_payload_hex"]) if "match_payload_hex" in spec else None
    return P, data, chunks, stream, mp


FIXTURES = sorted(glob.glob(os.path.join(GOLDEN, "*.txt")))


@pytest.mark.parametrize("path", FIXTURES, ids=[os.path.basename(f) for f in FIXTURES])
def test_golden_fixture(path):
    P, data, chunk_tokens, stream, match_payload = _load_fixture(path)
    out = oracle.compress(np.frombuffer(data, np.uint8), P).tobytes()
    st = glz1_reader.read(out)
    assert st.tokens == chunk_tokens
    if stream is not None:
        assert out == stream
    if match_payload is not None:
        assert match_payload in out
    # the fixture's tokens are also what brute force says
    for c, toks in enumerate(chunk_tokens):
        chunk = data[c * P.C:(c + 1) * P.C]
        assert brute_parse(symbols(chunk, P.S), P.W, P.m, P.M) == toks
    assert oracle.decompress(out).tobytes() == data


def test_fixture_count():
    assert len(FIXTURES) >= 6


# --- brute force --------------------------------------------------------------

@pytest.mark.parametrize("alpha", [1, 2, 3])
def test_longest_match_exhaustive_tiny(alpha):
    """Every sequence of up to 7 one-byte symbols over a small alphabet, every
    position, several windows and caps."""
    for n in range(1, 8):
        for seq in itertools.product(range(alpha), repeat=n):
            b = bytes(seq)
            sym = symbols(b, 1)
            for W, M in ((1, 255), (2, 3), (3, 2), (8, 255)):
                for p in range(n):
                    assert oracle.longest_match(b, p, 1, W, M) == brute_longest(sym, p, W, M)


@pytest.mark.parametrize("S", [1, 2, 4])
def test_parse_random_small(S):
    rng = np.random.default_rng(100 + S)
    for trial in range(60):
        k = int(rng.integers(1, 90))
        alpha = int(rng.integers(1, 5))
        vals = rng.integers(0, alpha, k)
        # multi-byte symbols whose bytes differ, so byte matches != symbol matches
        words = (vals * 0x01010101 + np.arange(k) % 2 * 0x100).astype(np.uint32)
        b = words.astype({1: np.uint8, 2: np.uint16, 4: np.uint32}[S]).tobytes()
        W = int(rng.integers(1, 40))
        M = int(rng.integers(1, 40))
        m = int(rng.integers(1, M + 1))
        got = oracle.parse_chunk(np.frombuffer(b, np.uint8), S, W, m, M)
        assert got == brute_parse(symbols(b, S), W, m, M)


def test_stream_tokens_are_brute_force_tokens():
    rng = np.random.default_rng(7)
    for S in (1, 2, 4):
        P = Params(S, 64, 24, 2 if S == 4 else 3, 40)
        vals = rng.integers(0, 3, 64 * 5 // S)  # five chunks
        b = vals.astype({1: np.uint8, 2: np.uint16, 4: np.uint32}[S]).tobytes()
        b = b[: len(b) - S]  # ragged last chunk
        st = glz1_reader.read(oracle.compress(np.frombuffer(b, np.uint8), P).tobytes())
        for c in range(st.n_chunks):
            chunk = b[c * P.C:(c + 1) * P.C]
            assert st.tokens[c] == brute_parse(symbols(chunk, S), P.W, P.m, P.M)


# --- closed forms -------------------------------------------------------------

def test_constant_run_closed_form():
    """S=2, W=128, m=3, M=255, 2048 equal symbols: 3 literals, pointers 3, 6,
    12, 24, 48, 96 (each bounded by off <= p), fourteen (128,128), then the
    64 symbols left as (64,64)."""
    x = np.full(2048, 0x1234, np.uint16)
    toks = oracle.parse_chunk(x, 2, 128, 3, 255)
    expect = [(1, 0)] * 3 + [(l, l) for l in (3, 6, 12, 24, 48, 96)]
    expect += [(128, 128)] * 14 + [(64, 64)]
    assert toks == expect


def period_closed_form(k, q, W, m, M):
    """x[i] = i mod q: only multiples of q match, each for min(M, d, k-p)
    symbols; the nearest multiple reaching the best length wins."""
    toks, p = [], 0
    while p < k:
        dmax = (min(W, p) // q) * q
        L = min(M, dmax, k - p) if dmax >= q else 0
        if L >= m:
            d = q * -(-L // q)  # smallest multiple of q that is >= L
            toks.append((L, d))
            p += L
        else:
            toks.append((1, 0))
            p += 1
    return toks


@pytest.mark.parametrize("q,W,M,m,k", [(1, 16, 255, 3, 100), (3, 64, 255, 3, 500),
                                       (5, 128, 20, 2, 777), (7, 32, 255, 3, 2048),
                                       (16, 256, 255, 4, 1024), (30, 40, 255, 3, 300)])
def test_period_closed_form(q, W, M, m, k):
    x = (np.arange(k) % q).astype(np.uint16)
    assert oracle.parse_chunk(x, 2, W, m, M) == period_closed_form(k, q, W, m, M)


def test_random_bytes_nearly_all_literals_and_size_identity():
    rng = np.random.default_rng(3)
    x = rng.integers(0, 256, 1 << 16, dtype=np.uint8)
    P = Params(1, 4096, 128, 3, 255)
    out = oracle.compress(x, P)
    st = glz1_reader.read(out.tobytes())
    n_match = sum(1 for toks in st.tokens for t in toks if t[1])
    # expected matches ~ positions * W * 2^-24: far below 1% of positions
    assert n_match < 0.01 * x.size
    size = 32 + 8 * st.n_chunks + 8 * ((st.n_chunks + 63) // 64)
    for ntok, pay in st.table:
        size += (ntok + 7) // 8 + pay
    assert size == len(out) == st.total_bytes
    # literals only -> n + n/8 + table, up to the few pointers
    assert abs(len(out) - (x.size + x.size // 8 + 32 + 8 * 16 + 8)) < 4 * n_match + 1


# --- invariants ---------------------------------------------------------------

@pytest.mark.parametrize("S,C,W,m,M", [(1, 64, 16, 3, 255), (2, 4096, 128, 3, 255),
                                       (4, 8192, 256, 2, 255), (1, 2048, 512, 3, 255),
                                       (2, 16, 1, 1, 1), (4, 32768, 1024, 1, 255)])
def test_round_trip_and_token_validity(S, C, W, m, M):
    rng = np.random.default_rng(S * 1000 + W)
    n_sym = (3 * C + 5 * S) // S  # three full chunks and a ragged tail
    x = rng.integers(0, 4, n_sym).astype({1: np.uint8, 2: np.uint16, 4: np.uint32}[S])
    P = Params(S, C, W, m, M)
    out = oracle.compress(x, P)
    assert len(out) <= oracle.bound(x.nbytes, P)
    assert np.array_equal(oracle.decompress(out), x.view(np.uint8))
    st = glz1_reader.read(out.tobytes())
    for c, toks in enumerate(st.tokens):
        p = 0
        for l, d in toks:
            if d:
                assert m <= l <= min(M, d) and 1 <= d <= min(W, p)
            p += l
        assert p * S == min(C, x.nbytes - c * C)
    # index = running record offset at every 64th chunk
    for j, v in enumerate(st.index):
        assert v == st.record_offsets[64 * j]


def test_index_over_many_chunks():
    x = np.arange(200 * 16, dtype=np.uint8)  # 200 chunks of 16 bytes
    P = Params(1, 16, 8, 3, 255)
    st = glz1_reader.read(oracle.compress(x, P).tobytes())
    assert st.n_chunks == 200 and len(st.index) == 4
    assert [st.index[j] for j in range(4)] == [st.record_offsets[64 * j] for j in range(4)]


def test_chunks_are_independent():
    """Compressing each chunk alone gives the same record as in the full stream."""
    rng = np.random.default_rng(11)
    x = rng.integers(0, 3, 4 * 256 + 64).astype(np.uint8)
    P = Params(1, 256, 64, 3, 255)
    full = glz1_reader.read(oracle.compress(x, P).tobytes())
    for c in range(full.n_chunks):
        one = glz1_reader.read(oracle.compress(x[c * 256:(c + 1) * 256], P).tobytes())
        assert one.tokens[0] == full.tokens[c]


def test_empty_input():
    P = Params(2, 4096, 128, 3, 255)
    out = oracle.compress(np.zeros(0, np.uint8), P)
    assert len(out) == 32 and oracle.bound(0, P) == 32
    assert oracle.decompressed_size(out) == 0
    assert oracle.decompress(out).size == 0


def test_bound_is_attained_by_worst_case():
    # S=1, m=1, offB=1: every symbol a pointer of length 1 costs 2 bytes
    P = Params(1, 16, 8, 1, 255)
    x = np.array([5] + [5] * 15, np.uint8)
    # constant run with M=1 forces 1-symbol pointers everywhere after p=0
    P1 = Params(1, 16, 8, 1, 1)
    out = oracle.compress(x, P1)
    assert len(out) <= oracle.bound(16, P1)
    assert len(out) == 32 + 8 + 8 + 2 + 1 + 15 * 2
    assert oracle.bound(16, P1) == 32 + 8 + 8 + 2 + 16 * 2  # S*k + (1+1-1)*k
    assert oracle.bound(16, P) == oracle.bound(16, P1)


def test_invalid_params_rejected():
    bad = [Params(3, 4096, 128, 3), Params(2, 4095, 128, 3), Params(2, 65536, 128, 3),
           Params(2, 4096, 0, 3), Params(2, 4096, 2048, 3), Params(2, 4096, 128, 0),
           Params(2, 4096, 128, 5, 4), Params(2, 4096, 128, 3, 256)]
    for P in bad:
        assert not oracle.check_params(P)
        assert oracle.bound(100, P) == 0
    with pytest.raises(oracle.OracleError):
        oracle.compress(np.zeros(3, np.uint8), Params(2, 4096, 128, 3))  # n % S


# --- decoder rejects corrupt streams ------------------------------------------

def _good_stream():
    x = np.frombuffer(b"abcabcabcabcXYZa" * 5, np.uint8)
    return bytearray(oracle.compress(x, Params(1, 16, 8, 3, 255)).tobytes())


def test_decoder_rejects_corruption():
    good = _good_stream()
    assert oracle.decompress_status(bytes(good)) == 0
    cases = []
    b = bytearray(good); b[0] = ord("X"); cases.append(b)          # magic
    b = bytearray(good); b[4] = 2; cases.append(b)                 # version
    b = bytearray(good); b[6] = 2; cases.append(b)                 # offB vs W
    b = bytearray(good); b[20] = 9; cases.append(b)                # n_chunks
    cases.append(good[:-1])                                        # truncated
    cases.append(good[:40])                                        # no table
    b = bytearray(good); b[32] += 1; cases.append(b)               # n_tokens
    b = bytearray(good); b[36] += 1; cases.append(b)               # payload size
    st = glz1_reader.read(bytes(good))
    first = st.records_at
    b = bytearray(good); b[first + 2 + 3 + 1] = 200; cases.append(b)  # offset 201 > p
    b = bytearray(good); b[first + 2 + 3] = 0; cases.append(b)        # length 0
    # offset beyond the window: W=8, last pointer (6,6) of chunk 0 -> offset 9
    b = bytearray(good); b[first + 2 + 3 + 2 + 1] = 8; cases.append(b)
    b = bytearray(good); b[st.records_at - 8] = 1; cases.append(b)    # index
    for i, c in enumerate(cases):
        assert oracle.decompress_status(bytes(c)) == oracle.ECORRUPT, i
