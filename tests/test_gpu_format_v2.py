"""Stream version 2 (stored chunks) on the GPU: lz_compress_ex with version 2
writes streams byte-identical to the oracle's version-2 streams (a chunk
whose coded record would not be smaller than the chunk is stored as it is),
with both matchers; the GPU decoder (single and batched) reads them, and
reads the oracle's version-2 streams too."""
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


def gpu_v2(codec, x: np.ndarray, P: Params, match: int = 0, in_offset: int = 0) -> np.ndarray:
    d = G.to_dev(x, in_offset)
    return codec.compress_sync(d, lz.Params(*P.tuple()), match=match, version=2).cpu().numpy()


def check(codec, x, P, match=0, in_offset=0):
    ref = oracle.compress(x, P, mode=match, version=2)
    got = gpu_v2(codec, x, P, match, in_offset)
    assert np.array_equal(got, ref), G.first_difference(got, ref)
    assert np.array_equal(G.gpu_decompress(codec, got), x.view(np.uint8).reshape(-1))
    return got


@pytest.mark.parametrize("S,C,W,m,M", GRID)
@pytest.mark.parametrize("kind", KINDS)
def test_v2_param_grid(codec, S, C, W, m, M, kind):
    P = Params(S, C, W, m, M)
    n_sym = (4 * C + C // 2) // S
    check(codec, make_input(kind, n_sym, S, seed=S * 31 + W), P)


@pytest.mark.parametrize("S", [1, 2, 4])
def test_v2_paper_matcher(codec, S):
    P = Params(S, 4096, 128, 2 if S == 4 else 3, 255)
    check(codec, make_input("mixed", 6 * 4096 // S + 3, S, seed=S), P, match=lz.LZ_MATCH_PAPER)


def test_v2_field_is_stored_and_smaller(codec):
    """The noisy float field at S=4: every chunk stored, so the stream is the
    input plus header, table and index."""
    x = synth.gaussian_field((16, 128, 256), seed=3)
    P = Params(4, 8192, 256, 2, 255)
    got = check(codec, x, P)
    nc = x.nbytes // 8192
    assert got.size == 32 + 8 * nc + 8 * ((nc + 63) // 64) + x.nbytes


@pytest.mark.parametrize("offset", [1, 4, 8])
def test_v2_misaligned_input(codec, offset):
    P = Params(2, 4096, 128, 3, 255)
    check(codec, make_input("mixed", 5 * 2048 + 77, 2, seed=offset), P, in_offset=offset)


@pytest.mark.parametrize("out_offset", [0, 3])
def test_v2_decode_oracle_streams(codec, out_offset):
    for S, kind in ((1, "random"), (2, "mixed"), (4, "quant")):
        P = Params(S, 2048, 200, 2, 100)
        x = make_input(kind, 30_000 // S * 2, S, seed=S + 9)
        s = oracle.compress(x, P, version=2)
        back = G.gpu_decompress(codec, s, out_offset=out_offset)
        assert np.array_equal(back, x.view(np.uint8))


def test_v2_batched_decompress(codec):
    """Version-2 streams decode through the batched launch too."""
    xs = [make_input(k, 3000 + 517 * i, 2, seed=i) for i, k in enumerate(KINDS)]
    P = Params(2, 2048, 128, 3, 255)
    streams = [G.to_dev(oracle.compress(x, P, version=2)) for x in xs]
    outs = [torch.empty(x.nbytes, dtype=torch.uint8, device="cuda") for x in xs]
    nbs = [torch.zeros(1, dtype=torch.int64, device="cuda") for _ in xs]
    items = [(s.data_ptr(), s.numel(), o.data_ptr(), o.numel(), nb.data_ptr(), None)
             for s, o, nb in zip(streams, outs, nbs)]
    st = torch.cuda.current_stream().cuda_stream
    b = lz.lz_batch_create(codec.ctx, items, decompress=True, stream=st)
    lz.lz_batch_run(codec.ctx, b, st)
    lz.lz_batch_destroy(b, st)
    assert codec.sync() == lz.LZ_OK
    for x, o in zip(xs, outs):
        assert np.array_equal(o.cpu().numpy(), x.view(np.uint8))


def test_v2_unknown_version_rejected(codec):
    d = torch.zeros(64, dtype=torch.uint8, device="cuda")
    out = torch.empty(4096, dtype=torch.uint8, device="cuda")
    nb = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(lz.LzError):
        lz.lz_compress_ex(codec.ctx, d.data_ptr(), 64, lz.Params(1, 64, 8, 2, 255),
                          out.data_ptr(), out.numel(), nb.data_ptr(),
                          torch.cuda.current_stream().cuda_stream, version=3)


@pytest.mark.parametrize("S", [2, 4])
@pytest.mark.parametrize("kind", ["alpha3", "quant", "random", "const"])
def test_v2_tail_bytes(codec, S, kind):
    """n % S != 0 (version 2): the bytes after the last whole symbol follow the
    last chunk's payload; byte-identical to the oracle, round trip exact,
    and version 1 still rejects such n."""
    P = Params(S, 4096, 128, 2 if S == 4 else 3, 255)
    base = make_input(kind, 3 * 4096 // S + 100, S, seed=S + 17).view(np.uint8)
    for cut in (1, S - 1, 4096 + 1, 3 * 4096 + 3):
        if cut % S == 0:
            continue
        x = np.ascontiguousarray(base[:cut])
        ref = oracle.compress(x, P, version=2)
        d = G.to_dev(x)
        got = codec.compress_sync(d, lz.Params(*P.tuple()), version=2).cpu().numpy()
        assert np.array_equal(got, ref), (cut, G.first_difference(got, ref))
        assert np.array_equal(G.gpu_decompress(codec, got), x)
        with pytest.raises(lz.LzError):
            codec.compress(d, lz.Params(*P.tuple()))


OVERLAP_GRID = [(1, 4096, 128, 3, 255), (2, 4096, 128, 3, 255), (4, 8192, 256, 2, 255),
                (1, 64, 33, 1, 1), (2, 16, 1, 1, 1), (4, 32, 7, 2, 3), (1, 512, 100, 4, 40),
                (2, 1024, 1024, 3, 255), (4, 2048, 32, 1, 255), (1, 16384, 512, 3, 255)]


@pytest.mark.parametrize("S,C,W,m,M", OVERLAP_GRID)
@pytest.mark.parametrize("kind", KINDS)
def test_v2_overlap_mode(codec, S, C, W, m, M, kind):
    """LZ_MATCH_OVERLAP (pointers may be longer than their offset): streams
    byte-identical to the oracle's MATCH_OVERLAP streams, decoded exactly."""
    P = Params(S, C, W, m, M)
    n_sym = (4 * C + C // 2) // S
    check(codec, make_input(kind, n_sym, S, seed=S * 13 + W), P, match=lz.LZ_MATCH_OVERLAP)


def test_v2_overlap_needs_version2_and_flag(codec):
    d = torch.zeros(64, dtype=torch.uint8, device="cuda")
    out = torch.empty(4096, dtype=torch.uint8, device="cuda")
    nb = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(lz.LzError):
        lz.lz_compress_ex(codec.ctx, d.data_ptr(), 64, lz.Params(1, 64, 8, 2, 255),
                          out.data_ptr(), out.numel(), nb.data_ptr(),
                          torch.cuda.current_stream().cuda_stream, match=lz.LZ_MATCH_OVERLAP,
                          version=1)
    x = np.full(5000, 9, np.uint8)
    s = oracle.compress(x, Params(1, 4096, 64, 3, 255), mode=oracle.MATCH_OVERLAP, version=2)
    assert np.array_equal(G.gpu_decompress(codec, s), x)
    bad = s.copy()
    bad[9] = 0  # pointers longer than their offset without the flag: corrupt
    with pytest.raises(lz.LzError):
        G.gpu_decompress(codec, bad)
