"""CUDA path vs the CPU oracle, through the C ABI: compressed streams must be
byte-identical, decompression bit-exact.  Sizes here let the oracle finish
in seconds while spanning many chunks, superblocks and a ragged tail."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from oracle import Params
from paper_2304_07342_gb300 import synth
from tests import gpu_util as G

pytestmark = pytest.mark.gpu

DT = {1: np.uint8, 2: np.uint16, 4: np.uint32}


@pytest.fixture(scope="module")
def codec():
    c = G.codec()
    yield c
    c.close()


def make_input(kind: str, n_sym: int, S: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    dt = DT[S]
    if kind == "alpha3":
        return rng.integers(0, 3, n_sym).astype(dt)
    if kind == "quant":
        v = synth.quant_codes_laplace(n_sym, seed=seed).astype(np.uint32)
        return (v if S > 1 else v % 256).astype(dt)
    if kind == "markov":
        v = synth.markov_codes(n_sym, seed=seed)
        return (v if S > 1 else v % 256).astype(dt)
    if kind == "periodic":
        return (np.arange(n_sym) % int(rng.integers(1, 40))).astype(dt)
    if kind == "const":
        return np.full(n_sym, 7, dt)
    if kind == "random":
        return synth.uniform_bytes(n_sym * S, seed=seed).view(dt)
    if kind == "mixed":
        parts = [make_input(k, n_sym // 5 + 1, S, seed + i)
                 for i, k in enumerate(("alpha3", "random", "const", "periodic", "quant"))]
        return np.concatenate(parts)[:n_sym]
    raise ValueError(kind)


def check(codec, x: np.ndarray, P: Params, in_offset: int = 0):
    ref = oracle.compress(x, P)
    got = G.gpu_compress(codec, x, P, in_offset=in_offset)
    assert np.array_equal(got, ref), G.first_difference(got, ref)
    back = G.gpu_decompress(codec, got)
    assert np.array_equal(back, x.view(np.uint8).reshape(-1))
    return got


def test_small_workload_byte_identical(codec):
    """1 MiB of uint16 quantization-code-like symbols, S=2, C=4096, W=128,
    m=3, M=255: one launch, byte-identical to the oracle, round trip exact."""
    x = synth.workload_small(seed=0)
    P = Params(2, 4096, 128, 3, 255)
    got = check(codec, x, P)
    assert np.array_equal(oracle.decompress(got), x.view(np.uint8))


GRID = [
    # S, C, W, m, M
    (1, 4096, 128, 3, 255), (2, 4096, 128, 3, 255), (4, 8192, 256, 2, 255),
    (1, 2048, 64, 3, 255), (1, 16384, 512, 3, 255), (2, 8192, 512, 3, 255),
    (4, 16384, 512, 2, 255), (2, 2048, 256, 3, 255), (4, 4096, 257, 2, 255),
    (1, 64, 33, 1, 1), (2, 16, 1, 1, 1), (4, 32, 7, 2, 3), (1, 256, 31, 2, 10),
    (2, 1024, 1024, 3, 255), (1, 512, 100, 4, 40), (4, 2048, 32, 1, 255),
]
KINDS = ["alpha3", "quant", "markov", "periodic", "const", "random", "mixed"]


@pytest.mark.parametrize("S,C,W,m,M", GRID)
@pytest.mark.parametrize("kind", KINDS)
def test_param_grid(codec, S, C, W, m, M, kind):
    P = Params(S, C, W, m, M)
    chunks = 5 if C >= 4096 else 9
    n_sym = (chunks * C + C // 2) // S  # several chunks and a ragged tail
    x = make_input(kind, n_sym, S, seed=S * 100 + W)
    check(codec, x, P)


@pytest.mark.parametrize("S", [1, 2, 4])
def test_maximum_parameters(codec, S):
    """Largest chunk (32 KiB), window (1024) and match (255)."""
    P = Params(S, 32768, 1024, 1 if S == 4 else 3, 255)
    x = make_input("mixed", (3 * 32768 + 4 * S) // S, S, seed=5)
    check(codec, x, P)


@pytest.mark.parametrize("n_sym", [0, 1, 2, 7, 8, 9, 64 * 8, 64 * 8 + 1, 129 * 8 + 3])
def test_edge_sizes(codec, n_sym):
    """Empty input, one symbol, exactly one chunk, one chunk plus one symbol,
    65 and 130 chunks (more than one index superblock)."""
    P = Params(2, 16, 8, 2, 255)
    x = make_input("alpha3", n_sym, 2, seed=n_sym)
    check(codec, x, P)


@pytest.mark.parametrize("offset", [1, 2, 4, 8])
def test_misaligned_input(codec, offset):
    """Input pointers that are not 16-byte aligned take the plain-load path."""
    P = Params(1, 4096, 128, 3, 255)
    x = make_input("quant", 3 * 4096 + 100, 1, seed=offset)
    check(codec, x, P, in_offset=offset)


@pytest.mark.parametrize("offset", [1, 2, 3])
def test_misaligned_output(codec, offset):
    P = Params(4, 4096, 128, 2, 255)
    x = make_input("markov", 3000, 4, seed=offset)
    s = oracle.compress(x, P)
    back = G.gpu_decompress(codec, s, out_offset=offset)
    assert np.array_equal(back, x.view(np.uint8))


def test_repeated_calls_share_context(codec):
    """Back-to-back calls on one context give identical streams (the scratch
    is cleared per call)."""
    P = Params(2, 2048, 128, 3, 255)
    x = make_input("quant", 50_000, 2, seed=3)
    ref = oracle.compress(x, P)
    for _ in range(4):
        assert np.array_equal(G.gpu_compress(codec, x, P), ref)


def test_decode_oracle_streams(codec):
    """The GPU decoder reads streams produced by the oracle."""
    for S, kind in ((1, "random"), (2, "quant"), (4, "periodic")):
        P = Params(S, 2048, 200, 2, 100)
        x = make_input(kind, 20_000 // S * 4, S, seed=S)
        assert np.array_equal(G.gpu_decompress(codec, oracle.compress(x, P)), x.view(np.uint8))
