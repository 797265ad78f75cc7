"""The paper's matcher on the GPU (lz_compress_ex with LZ_MATCH_PAPER):
streams byte-identical to the oracle run with MATCH_PAPER (section 3.3.2's
forward scan) on the parameter grid, the small quantization-code workload
and edge sizes, decoded bit-exactly by the common decoder."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
from oracle import Params
from paper_2304_07342_gb300 import lz, synth
from tests import gpu_util as G
from tests.test_gpu_parity import GRID, KINDS, make_input

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def codec():
    c = G.codec()
    yield c
    c.close()


def gpu_paper(codec, x: np.ndarray, P: Params) -> np.ndarray:
    d = G.to_dev(x)
    return codec.compress_sync(d, lz.Params(*P.tuple()), match=lz.LZ_MATCH_PAPER).cpu().numpy()


def check(codec, x: np.ndarray, P: Params):
    ref = oracle.compress(x, P, mode=oracle.MATCH_PAPER)
    got = gpu_paper(codec, x, P)
    assert np.array_equal(got, ref), G.first_difference(got, ref)
    assert np.array_equal(G.gpu_decompress(codec, got), x.view(np.uint8).reshape(-1))
    return got


def test_small_workload_paper_matcher(codec):
    """1 MiB of uint16 quantization codes (S=2, C=4096, W=128, m=3, M=255):
    byte-identical to the oracle, and no smaller than the exact parse's
    stream by more than a few percent (the scan can miss longer matches)."""
    x = synth.workload_small(seed=0)
    P = Params(2, 4096, 128, 3, 255)
    got = check(codec, x, P)
    exact = oracle.compress(x, P)
    assert got.size >= exact.size
    assert got.size <= exact.size * 1.5


@pytest.mark.parametrize("S,C,W,m,M", GRID)
@pytest.mark.parametrize("kind", KINDS)
def test_paper_param_grid(codec, S, C, W, m, M, kind):
    P = Params(S, C, W, m, M)
    chunks = 4 if C >= 4096 else 7
    n_sym = (chunks * C + C // 2) // S
    x = make_input(kind, n_sym, S, seed=S * 100 + W + 7)
    check(codec, x, P)


@pytest.mark.parametrize("n_sym", [0, 1, 2, 9, 64 * 8 + 1])
def test_paper_edge_sizes(codec, n_sym):
    P = Params(2, 16, 8, 2, 255)
    check(codec, make_input("alpha3", n_sym, 2, seed=n_sym), P)


def test_paper_and_exact_differ_where_the_scan_skips(codec):
    """A chunk built so that the scan's first run breaks inside the longest
    match: the two matchers give different streams, each identical to its
    oracle."""
    unit = np.frombuffer(b"ABABCx", np.uint8)
    x = np.concatenate([unit, np.frombuffer(b"ABC", np.uint8)] * 50)
    P = Params(1, 64, 32, 2, 255)
    paper = check(codec, x, P)
    exact = G.gpu_compress(codec, x, P)
    assert np.array_equal(exact, oracle.compress(x, P))
    assert not np.array_equal(paper, exact)


def test_unknown_matcher_rejected(codec):
    d = torch.zeros(64, dtype=torch.uint8, device="cuda")
    out = torch.empty(4096, dtype=torch.uint8, device="cuda")
    nb = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(lz.LzError):
        lz.lz_compress_ex(codec.ctx, d.data_ptr(), 64, lz.Params(1, 64, 8, 2, 255),
                          out.data_ptr(), out.numel(), nb.data_ptr(),
                          torch.cuda.current_stream().cuda_stream, match=2)
