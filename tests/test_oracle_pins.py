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


def paper_jump(sym: list, p: int, W: int, M: int):
    """The paper's matcher (section 3.3.2) restated as jumps between run
    starts instead of pointer steps.  E = the window positions holding
    x[p].  The scan meets the smallest w in E and follows the run from w as
    far as it goes (not into p, not past the look-ahead of min(M, k-p)
    symbols).  Unless the run reached p or the look-ahead end, the scan goes
    on at the smallest w in E beyond the symbol that broke the run (that
    symbol itself is never tried as a start).  The first run of the
    greatest length wins."""
    k = len(sym)
    lo, end = max(0, p - W), min(k, p + M)
    E = [w for w in range(lo, p) if sym[w] == sym[p]]
    best, best_d, after = 0, 0, lo
    for w in E:
        if w < after:
            continue
        l = 0
        while w + l < p and p + l < end and sym[w + l] == sym[p + l]:
            l += 1
        if l > best:
            best, best_d = l, p - w
        if w + l == p or p + l == end:
            break
        after = w + l + 1
    return best, best_d


def jump_parse(sym: list, W: int, m: int, M: int):
    toks, p = [], 0
    while p < len(sym):
        l, d = paper_jump(sym, p, W, M)
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
        if part.strip() == "stored":
            chunks.append("stored")
            continue
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
    mode = {"exact": oracle.MATCH_EXACT, "paper": oracle.MATCH_PAPER}[spec.get("mode", "exact")]
    return P, data, chunks, stream, mp, mode, int(spec.get("version", "1"))


FIXTURES = sorted(glob.glob(os.path.join(GOLDEN, "*.txt")))


@pytest.mark.parametrize("path", FIXTURES, ids=[os.path.basename(f) for f in FIXTURES])
def test_golden_fixture(path):
    P, data, chunk_tokens, stream, match_payload, mode, version = _load_fixture(path)
    out = oracle.compress(np.frombuffer(data, np.uint8), P, mode=mode, version=version).tobytes()
    st = glz1_reader.read(out)
    assert st.version == version
    assert st.stored == [t == "stored" for t in chunk_tokens]
    assert st.tokens == [[] if t == "stored" else t for t in chunk_tokens]
    if stream is not None:
        assert out == stream
    if match_payload is not None:
        assert match_payload in out
    # the fixture's tokens are also what brute force says; a stored chunk is
    # one whose brute-force record would not be smaller than the chunk
    parse = brute_parse if mode == oracle.MATCH_EXACT else jump_parse
    offB = 1 if P.W <= 256 else 2
    for c, toks in enumerate(chunk_tokens):
        chunk = data[c * P.C:(c + 1) * P.C]
        bf = parse(symbols(chunk, P.S), P.W, P.m, P.M)
        if toks == "stored":
            rec = (len(bf) + 7) // 8 + sum(1 + offB if d else P.S for _, d in bf)
            assert version == 2 and rec >= len(chunk)
            rec_at = st.records_at + st.record_offsets[c]
            assert out[rec_at:rec_at + len(chunk)] == chunk
        else:
            assert bf == toks
    assert oracle.decompress(out).tobytes() == data


def test_fixture_count():
    assert len(FIXTURES) >= 9


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
    b = bytearray(good); b[4] = 3; cases.append(b)                 # version
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


# --- the paper's matcher (section 3.3.2), mode MATCH_PAPER --------------------

@pytest.mark.parametrize("alpha", [1, 2, 3])
def test_paper_match_exhaustive_tiny(alpha):
    """Every sequence of up to 7 one-byte symbols over a small alphabet, every
    position, several windows and caps: the oracle's pointer walk equals
    the jump formulation."""
    for n in range(1, 8):
        for seq in itertools.product(range(alpha), repeat=n):
            b = bytes(seq)
            sym = symbols(b, 1)
            for W, M in ((1, 255), (2, 3), (3, 2), (8, 255), (4, 1)):
                for p in range(n):
                    assert oracle.paper_match(b, p, 1, W, M) == paper_jump(sym, p, W, M), \
                        (seq, p, W, M)


@pytest.mark.parametrize("S", [1, 2, 4])
def test_paper_parse_random_small(S):
    """Random chunks over small alphabets (many partial runs, which is where
    the scan skips candidates): whole parses equal the jump formulation."""
    rng = np.random.default_rng(40 + S)
    for trial in range(60):
        k = int(rng.integers(1, 90))
        alpha = int(rng.integers(1, 5))
        W = int(rng.integers(1, 40))
        M = int(rng.integers(1, 20))
        m = int(rng.integers(1, M + 1))
        x = rng.integers(0, alpha, k).astype({1: np.uint8, 2: np.uint16, 4: np.uint32}[S])
        b = x.tobytes()
        assert oracle.parse_chunk(b, S, W, m, M, mode=oracle.MATCH_PAPER) == \
            jump_parse(symbols(b, S), W, m, M), (trial, k, alpha, W, M, m)


def test_paper_constant_run_closed_form():
    """All symbols equal: at p the scan starts at lo = max(0, p-W), the first
    run never breaks and ends at p or at the look-ahead end, so the match is
    length min(W, p, k-p, M) at offset min(W, p) (farthest, where the exact
    matcher takes the nearest)."""
    for S, k, W, M in ((2, 2048, 128, 255), (1, 300, 256, 255), (4, 97, 16, 5)):
        b = np.full(k, 9, {1: np.uint8, 2: np.uint16, 4: np.uint32}[S]).tobytes()
        for p in range(k):
            L = min(W, p, k - p, M)
            assert oracle.paper_match(b, p, S, W, M) == (L, min(W, p) if L else 0), (S, p)


@pytest.mark.parametrize("q,W,M,k", [(1, 16, 255, 100), (3, 64, 255, 500), (7, 50, 20, 400),
                                     (5, 5, 255, 60)])
def test_paper_period_closed_form(q, W, M, k):
    """x[i] = i mod q: the first window position holding x[p] is lo + ((p -
    lo) mod q); its run never breaks, so the offset is the largest multiple
    of q that is <= min(W, p) and the length is min(offset, k-p, M)."""
    b = (np.arange(k) % q).astype(np.uint8).tobytes()
    for p in range(k):
        d = (min(W, p) // q) * q
        L = min(d, k - p, M)
        assert oracle.paper_match(b, p, 1, W, M) == ((L, d) if L else (0, 0)), p


def test_paper_match_never_exceeds_exact_and_is_valid():
    """Every run the scan keeps is a true match with length <= offset <=
    min(W, p), <= M and <= k - p, and is never longer than the exact
    longest match; on data with one distinct repeat the two agree."""
    rng = np.random.default_rng(7)
    shorter = 0
    for trial in range(40):
        k = int(rng.integers(20, 300))
        x = rng.integers(0, int(rng.integers(2, 6)), k).astype(np.uint8)
        W, M = int(rng.integers(1, 64)), int(rng.integers(1, 40))
        b = x.tobytes()
        for p in range(k):
            l, d = oracle.paper_match(b, p, 1, W, M)
            le, _ = oracle.longest_match(b, p, 1, W, M)
            assert l <= le
            shorter += l < le
            if l:
                assert 1 <= l <= d <= min(W, p) and l <= M and l <= k - p
                assert b[p:p + l] == b[p - d:p - d + l]
    assert shorter > 0  # the heuristic does miss longer matches
    y = np.arange(200, dtype=np.uint8)
    y[150:160] = y[40:50]
    assert oracle.paper_match(y.tobytes(), 150, 1, 255, 255) == \
        oracle.longest_match(y.tobytes(), 150, 1, 255, 255) == (10, 110)


@pytest.mark.parametrize("S,C,W,m,M", [(1, 64, 16, 3, 255), (2, 4096, 128, 3, 255),
                                       (4, 8192, 256, 2, 255), (1, 1024, 300, 2, 255)])
def test_paper_round_trip(S, C, W, m, M):
    """Streams parsed with the paper's matcher use the same layout and decode
    with the same decoder."""
    rng = np.random.default_rng(S + W)
    x = np.repeat(rng.integers(0, 5, 3000), rng.integers(1, 6, 3000))[: 9000 // S * S]
    x = x.astype({1: np.uint8, 2: np.uint16, 4: np.uint32}[S])
    P = Params(S, C, W, m, M)
    s = oracle.compress(x, P, mode=oracle.MATCH_PAPER)
    assert np.array_equal(oracle.decompress(s), x.view(np.uint8))
    assert s.size >= oracle.compress(x, P).size * 0.9  # comparable, usually larger
    st = glz1_reader.read(s.tobytes())
    assert sum(sum(l for l, _ in t) for t in st.tokens) == x.size


# --- parameter policy (section 3.2.3) -----------------------------------------

def test_policy_min_match_is_shortest_profitable():
    """m is the smallest length whose pointer bytes (1 + offB) are fewer than
    the literal bytes S * m it replaces: checked against that definition by
    enumeration."""
    for S in (1, 2, 4):
        for W in (32, 255, 256, 257, 1020):
            offB = 1 if W <= 256 else 2
            m = next(l for l in range(1, 10) if 1 + offB < S * l)
            assert oracle.min_profitable_match(S, W) == m


def test_policy_ratio_test_is_exact():
    assert not oracle.ratio_below(3, 2)        # exactly 1.5 keeps multi-byte
    assert oracle.ratio_below(299, 200)        # 1.495
    assert not oracle.ratio_below(301, 200)    # 1.505
    assert oracle.ratio_below(10, 11)          # expansion


def test_policy_decisions():
    """One-byte data needs no trial; a constant field keeps 4-byte symbols
    with the window enlarged 4x; noisy words (ratio < 1) fall back to
    single bytes with the level's window; the trial is the oracle's own
    stream size."""
    assert oracle.select_params(np.arange(100, dtype=np.uint8), 1, 2) == Params(1, 4096, 64, 3, 255)
    c = np.full(20_000, 9, np.uint32)
    assert oracle.select_params(c, 4, 1) == Params(4, 4096, 128, 1, 255)
    assert oracle.select_params(c, 4, 4) == Params(4, 4096, 1020, 1, 255)
    r = np.random.default_rng(0).integers(0, 1 << 32, 20_000, dtype=np.uint64).astype(np.uint32)
    assert oracle.select_params(r, 4, 3) == Params(1, 4096, 128, 3, 255)
    x = np.repeat(np.arange(50, dtype=np.uint16), 40)
    multi = Params(2, 4096, 256, 2, 255)
    keep = not oracle.ratio_below(x.nbytes, oracle.compress(x, multi).size)
    assert keep and oracle.select_params(x, 2, 3) == multi


# --- stream version 2: stored chunks -------------------------------------------

@pytest.mark.parametrize("S,C,W,m,M", [(1, 64, 16, 3, 255), (2, 4096, 128, 3, 255),
                                       (4, 8192, 256, 2, 255), (1, 1024, 300, 2, 255),
                                       (2, 16, 1, 1, 1)])
def test_v2_stores_exactly_the_chunks_that_do_not_shrink(S, C, W, m, M):
    """Version 2 keeps every coded record that is smaller than its chunk,
    byte for byte as in version 1, and stores the others as they are; it is
    never larger than version 1 and decodes to the input."""
    rng = np.random.default_rng(S * 7 + C)
    dt = {1: np.uint8, 2: np.uint16, 4: np.uint32}[S]
    n_sym = (7 * C + C // 3) // S
    parts = [rng.integers(0, 3, n_sym // 3), rng.integers(0, 1 << (8 * S), n_sym // 3, dtype=np.uint64),
             np.repeat(rng.integers(0, 50, n_sym), 3)]
    x = np.concatenate(parts)[:n_sym].astype(dt)
    P = Params(S, C, W, m, M)
    v1 = oracle.compress(x, P).tobytes()
    v2 = oracle.compress(x, P, version=2).tobytes()
    a, b = glz1_reader.read(v1), glz1_reader.read(v2)
    assert len(v2) <= len(v1) and any(b.stored)
    xb = x.tobytes()
    for c in range(a.n_chunks):
        ntok, pay = a.table[c]
        raw = xb[c * C:(c + 1) * C]
        if (ntok + 7) // 8 + pay >= len(raw):
            assert b.stored[c] and b.table[c] == (0, len(raw))
            at = b.records_at + b.record_offsets[c]
            assert v2[at:at + len(raw)] == raw
        else:
            assert not b.stored[c] and b.table[c] == a.table[c] and b.tokens[c] == a.tokens[c]
    assert oracle.decompress(v2).tobytes() == xb
    assert oracle.decompress(v1).tobytes() == xb


def test_v2_decoder_rejects_bad_stored_chunks():
    x = np.frombuffer(bytes(range(64)), np.uint8)  # nothing repeats: all stored
    good = bytearray(oracle.compress(x, Params(1, 16, 8, 3, 255), version=2).tobytes())
    assert oracle.decompress_status(bytes(good)) == 0
    b = bytearray(good); b[36] = 15; assert oracle.decompress_status(bytes(b)) == oracle.ECORRUPT
    b = bytearray(good); b[4] = 1; assert oracle.decompress_status(bytes(b)) == oracle.ECORRUPT
    b = bytearray(good); b[4] = 3; assert oracle.decompress_status(bytes(b)) == oracle.ECORRUPT


@pytest.mark.parametrize("S", [2, 4])
def test_v2_tail_bytes(S):
    """Version 2 takes n % S != 0: the last chunk's bytes after its last whole
    symbol follow its payload as they are (version 1 rejects such n)."""
    rng = np.random.default_rng(S)
    for n in (1, S - 1, S + 1, 16 + 1, 16 * 3 + S + 1, 4096 * 2 + 3):
        if n % S == 0:
            continue
        x = np.repeat(rng.integers(0, 4, n), 2)[:n].astype(np.uint8)
        P = Params(S, 16 if n < 1000 else 4096, 8, 2 if S == 2 else 1, 255)
        with pytest.raises(oracle.OracleError):
            oracle.compress(x, P)
        s = oracle.compress(x, P, version=2)
        assert oracle.decompress(s).tobytes() == x.tobytes()
        assert s.size <= oracle.bound(n, P)
        st = glz1_reader.read(s.tobytes())
        last = n - (st.n_chunks - 1) * P.C
        k, tail = last // S, last % S
        at = st.records_at + st.record_offsets[-1]
        if st.stored[-1]:
            assert s.tobytes()[at:at + last] == x.tobytes()[n - last:]
        else:
            ntok, pay = st.table[-1]
            rec = s.tobytes()[at + (ntok + 7) // 8: at + (ntok + 7) // 8 + pay]
            assert rec[-tail:] == x.tobytes()[n - tail:]
            assert sum(l for l, _ in st.tokens[-1]) == k


# --- stream version 2: overlap-allowed mode ---------------------------------------

def brute_longest_overlap(sym: list, p: int, W: int, M: int):
    """Longest match when it may run into the look-ahead: for each offset the
    longest l <= min(M, k - p) with equal slices (slices of the input may
    overlap), longest first; nearest offset on ties."""
    k = len(sym)
    best, best_d = 0, 0
    for d in range(1, min(W, p) + 1):
        for l in range(min(M, k - p), 0, -1):
            if sym[p:p + l] == sym[p - d:p - d + l]:
                break
        else:
            l = 0
        if l > best:
            best, best_d = l, d
    return best, best_d


@pytest.mark.parametrize("alpha", [1, 2, 3])
def test_overlap_match_exhaustive_tiny(alpha):
    for n in range(1, 8):
        for seq in itertools.product(range(alpha), repeat=n):
            b = bytes(seq)
            sym = symbols(b, 1)
            for W, M in ((1, 255), (2, 3), (3, 2), (8, 255)):
                for p in range(n):
                    assert oracle.longest_match_overlap(b, p, 1, W, M) == \
                        brute_longest_overlap(sym, p, W, M)


def test_overlap_closed_forms():
    """A constant run is one literal and then pointers at offset 1 of length
    min(M, symbols left); x[i] = i mod q takes offset q with the longest
    length the chunk and M allow."""
    k, M = 1000, 255
    toks = oracle.parse_chunk(np.full(k, 5, np.uint8).tobytes(), 1, 64, 3, M, mode=oracle.MATCH_OVERLAP)
    want, p = [(1, 0)], 1
    while p < k:
        l = min(M, k - p)
        want.append((l, 1) if l >= 3 else (1, 0))
        p += l if l >= 3 else 1
    assert toks == want
    for q in (2, 5, 17):
        x = (np.arange(600) % q).astype(np.uint8).tobytes()
        for p in range(q, 600, 37):
            assert oracle.longest_match_overlap(x, p, 1, 64, 255) == (min(255, 600 - p), q)


@pytest.mark.parametrize("S", [1, 2, 4])
def test_overlap_round_trip_and_flag(S):
    rng = np.random.default_rng(S + 50)
    x = np.repeat(rng.integers(0, 4, 3000), rng.integers(1, 30, 3000))[: 12000 // S * S]
    x = x.astype({1: np.uint8, 2: np.uint16, 4: np.uint32}[S])
    P = Params(S, 4096, 128, 2, 255)
    with pytest.raises(oracle.OracleError):
        oracle.compress(x, P, mode=oracle.MATCH_OVERLAP)  # version 1 has no overlaps
    s = oracle.compress(x, P, mode=oracle.MATCH_OVERLAP, version=2)
    assert s[9] == 1 and np.array_equal(oracle.decompress(s), x.view(np.uint8))
    st = glz1_reader.read(s.tobytes())
    assert st.overlap and any(l > d for t in st.tokens for l, d in t if d)
    assert s.size < oracle.compress(x, P, version=2).size
    bad = bytearray(s.tobytes()); bad[9] = 0   # pointers longer than their offset, no flag
    assert oracle.decompress_status(bytes(bad)) == oracle.ECORRUPT
    bad = bytearray(s.tobytes()); bad[9] = 2
    assert oracle.decompress_status(bytes(bad)) == oracle.ECORRUPT
