"""The Huffman stage on the GPU (lz_huff_compress / lz_huff_decompress):
streams byte-identical to the oracle's (huffref.c: package-merge lengths,
canonical codes, GHF1 layout), bit-exact decoding of GPU and oracle
streams, rejection of corrupt streams, the capacity check, and the paper's
pipeline (LZSS, then Huffman) on quantization codes."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
from paper_2304_07342_gb300 import lz, synth
from tests import gpu_util as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def codec():
    c = G.codec()
    yield c
    c.close()


def stream_of(t: torch.Tensor) -> int:
    return torch.cuda.current_stream().cuda_stream


def gpu_huff(codec, x: np.ndarray, in_offset: int = 0, cap: int | None = None):
    d = G.to_dev(x, in_offset)
    n = d.numel() if x.size else 0
    cap = lz.lz_huff_bound(n) if cap is None else cap
    out = torch.empty(max(cap, 8), dtype=torch.uint8, device="cuda")
    nb = torch.zeros(1, dtype=torch.int64, device="cuda")
    lz.lz_huff_compress(codec.ctx, d.data_ptr(), n, out.data_ptr(), cap, nb.data_ptr(),
                        stream_of(d))
    st = codec.sync()
    return st, out[: int(nb.item())].cpu().numpy() if st == lz.LZ_OK else None, int(nb.item())


def gpu_unhuff(codec, s: np.ndarray, out_offset: int = 0):
    d = G.to_dev(s)
    n = lz.lz_huff_decompressed_size(d.data_ptr(), d.numel())
    buf = torch.empty(n + out_offset + 16, dtype=torch.uint8, device="cuda")
    out = buf[out_offset:]
    nb = torch.zeros(1, dtype=torch.int64, device="cuda")
    lz.lz_huff_decompress(codec.ctx, d.data_ptr(), d.numel(), out.data_ptr(), n, nb.data_ptr(),
                          stream_of(d))
    st = codec.sync()
    return st, (out[:n].cpu().numpy() if st == lz.LZ_OK else None)


def inputs():
    rng = np.random.default_rng(21)
    yield "empty", np.zeros(0, np.uint8)
    yield "one byte", np.array([7], np.uint8)
    yield "single symbol", np.full(70_000, 42, np.uint8)
    yield "two symbols", (rng.integers(0, 2, 50_001) * 200).astype(np.uint8)
    yield "all 256", np.arange(256 * 300, dtype=np.uint32).astype(np.uint8)
    yield "random", rng.integers(0, 256, 100_003).astype(np.uint8)
    yield "skewed", np.minimum(rng.geometric(0.2, 300_000), 255).astype(np.uint8)
    yield "fibonacci-like", np.repeat(np.arange(24, dtype=np.uint8),
                                      [int(1.6 ** i) + 1 for i in range(24)])
    yield "lzss stream", oracle.compress(synth.quant_codes_laplace(150_000, seed=2),
                                         oracle.Params(2, 4096, 128, 3, 255))
    for n in (1023, 1024, 1025, 32767, 32768, 32769, 65536 + 1000):
        yield f"size {n}", np.minimum(rng.geometric(0.05, n), 255).astype(np.uint8)


@pytest.mark.parametrize("name,x", list(inputs()), ids=[n for n, _ in inputs()])
def test_huff_byte_identical_and_round_trip(codec, name, x):
    st, got, _ = gpu_huff(codec, x)
    assert st == lz.LZ_OK
    ref = oracle.huff_compress(x)
    assert got.size == ref.size and np.array_equal(got, ref), name
    st, back = gpu_unhuff(codec, got)
    assert st == lz.LZ_OK and np.array_equal(back, x)


@pytest.mark.parametrize("offset", [1, 2, 3])
def test_huff_misaligned_input_and_output(codec, offset):
    x = np.minimum(np.random.default_rng(offset).geometric(0.1, 77_777), 255).astype(np.uint8)
    st, got, _ = gpu_huff(codec, x, in_offset=offset)
    assert st == lz.LZ_OK and np.array_equal(got, oracle.huff_compress(x))
    st, back = gpu_unhuff(codec, got, out_offset=offset)
    assert st == lz.LZ_OK and np.array_equal(back, x)


def test_huff_decodes_oracle_streams(codec):
    for seed in range(3):
        x = np.minimum(np.random.default_rng(seed).geometric(0.03, 40_000 + seed), 255)
        s = oracle.huff_compress(x.astype(np.uint8))
        st, back = gpu_unhuff(codec, s)
        assert st == lz.LZ_OK and np.array_equal(back, x.astype(np.uint8))


def test_huff_capacity_too_small(codec):
    x = np.random.default_rng(4).integers(0, 256, 100_000).astype(np.uint8)
    need = oracle.huff_compress(x).size
    st, _, reported = gpu_huff(codec, x, cap=need - 4)
    assert st == lz.LZ_ERR_BUFFER_TOO_SMALL and reported == need
    # the context recovers
    st, got, _ = gpu_huff(codec, x)
    assert st == lz.LZ_OK and got.size == need


def test_huff_rejects_corruption_like_the_oracle(codec):
    x = np.minimum(np.random.default_rng(3).geometric(0.1, 40_000), 255).astype(np.uint8)
    good = oracle.huff_compress(x).tobytes()
    nb = (x.size + 32767) // 32768
    L = np.frombuffer(good[16:272], np.uint8)
    used = [int(i) for i in np.nonzero(L)[0]]
    cases = []
    b = bytearray(good); b[0] = ord("X"); cases.append(b)
    b = bytearray(good); b[16 + used[-1]] = 13; cases.append(b)
    b = bytearray(good); b[16 + used[-1]] = 0; cases.append(b)
    b = bytearray(good); b[272] += 4; cases.append(b)
    b = bytearray(good); b[272 + 8 * nb + 4] += 1; cases.append(b)
    b = bytearray(good); b[len(good) - 40] ^= 0xFF; cases.append(b)
    for i, c in enumerate(cases):
        rc, _ = oracle.huff_decompress_status(bytes(c))
        if rc != oracle.ECORRUPT:  # a flipped payload can still decode to other bytes
            assert i == len(cases) - 1
            continue
        st, _ = gpu_unhuff(codec, np.frombuffer(bytes(c), np.uint8)) if i != 0 else (None, None)
        if i == 0:
            d = G.to_dev(np.frombuffer(bytes(c), np.uint8))
            with pytest.raises(lz.LzError):
                lz.lz_huff_decompressed_size(d.data_ptr(), d.numel())
            continue
        assert st == lz.LZ_ERR_CORRUPT, i
        st, back = gpu_unhuff(codec, np.frombuffer(good, np.uint8))
        assert st == lz.LZ_OK and np.array_equal(back, x)


def test_lzss_then_huffman_pipeline(codec):
    """The paper's use case: quantization codes compressed by LZSS, then the
    stream Huffman-coded; both stages identical to the oracle's, the
    pipeline round-trips, and Huffman shrinks the LZSS stream further."""
    x = synth.quant_codes_laplace(1 << 20, seed=9)  # 2 MiB of uint16 codes
    P = lz.Params(2, 4096, 128, 3, 255)
    s1 = G.gpu_compress(codec, x, P)
    assert np.array_equal(s1, oracle.compress(x, oracle.Params(2, 4096, 128, 3, 255)))
    st, s2, _ = gpu_huff(codec, s1)
    assert st == lz.LZ_OK and np.array_equal(s2, oracle.huff_compress(s1))
    assert s2.size < s1.size
    st, back1 = gpu_unhuff(codec, s2)
    assert st == lz.LZ_OK and np.array_equal(back1, s1)
    assert np.array_equal(G.gpu_decompress(codec, back1), x.view(np.uint8))
