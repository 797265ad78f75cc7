"""Error behaviour of the CUDA path: argument errors are synchronous, device
errors are sticky until lz_sync, and a context stays usable afterwards."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
from oracle import Params
from paper_2304_07342_gb300 import lz
from tests import glz1_reader
from tests import gpu_util as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def codec():
    c = G.codec()
    yield c
    c.close()


def _stream():
    x = np.frombuffer(b"abcabcabcabcXYZa" * 5, np.uint8)
    return bytearray(oracle.compress(x, Params(1, 16, 8, 3, 255)).tobytes()), x


def _decode_status(codec, s: bytes) -> int:
    d = G.to_dev(np.frombuffer(bytes(s), np.uint8))
    out = torch.empty(4096, dtype=torch.uint8, device="cuda")
    ob = torch.zeros(1, dtype=torch.int64, device="cuda")
    lz.lz_decompress(codec.ctx, d.data_ptr(), d.numel(), out.data_ptr(), out.numel(),
                     ob.data_ptr(), torch.cuda.current_stream().cuda_stream)
    return codec.sync()


def test_corrupt_streams_rejected_like_the_oracle(codec):
    good, x = _stream()
    assert _decode_status(codec, good) == lz.LZ_OK
    st = glz1_reader.read(bytes(good))
    first = st.records_at
    cases = []
    b = bytearray(good); b[0] = ord("X"); cases.append(b)
    b = bytearray(good); b[4] = 3; cases.append(b)
    b = bytearray(good); b[6] = 2; cases.append(b)
    b = bytearray(good); b[20] = 9; cases.append(b)
    cases.append(good[:-1])
    cases.append(good[:40])
    b = bytearray(good); b[32] += 1; cases.append(b)
    b = bytearray(good); b[36] += 1; cases.append(b)
    b = bytearray(good); b[first + 2 + 3 + 1] = 200; cases.append(b)
    b = bytearray(good); b[first + 2 + 3] = 0; cases.append(b)
    b = bytearray(good); b[first + 2 + 3 + 2 + 1] = 8; cases.append(b)
    b = bytearray(good); b[st.records_at - 8] = 1; cases.append(b)
    for i, c in enumerate(cases):
        assert oracle.decompress_status(bytes(c)) == oracle.ECORRUPT, i
        if len(c) < 32:
            continue
        assert _decode_status(codec, c) == lz.LZ_ERR_CORRUPT, i
        # the context recovers: a good stream decodes next
        assert _decode_status(codec, good) == lz.LZ_OK, i


def test_short_input_rejected_synchronously(codec):
    d = torch.zeros(31, dtype=torch.uint8, device="cuda")
    ob = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(lz.LzError) as e:
        lz.lz_decompress(codec.ctx, d.data_ptr(), 31, d.data_ptr(), 31, ob.data_ptr())
    assert e.value.status == lz.LZ_ERR_CORRUPT


def test_random_garbage_never_faults(codec):
    """Random bytes behind a valid header: the decoder reports CORRUPT (or
    decodes) without touching memory outside its buffers."""
    good, _ = _stream()
    rng = np.random.default_rng(1)
    for trial in range(40):
        b = bytearray(good)
        for _ in range(int(rng.integers(1, 6))):
            i = int(rng.integers(32, len(b)))
            b[i] = int(rng.integers(0, 256))
        st = _decode_status(codec, b)
        assert st in (lz.LZ_OK, lz.LZ_ERR_CORRUPT)
        assert st == (lz.LZ_OK if oracle.decompress_status(bytes(b)) == 0 else lz.LZ_ERR_CORRUPT)


def test_compress_output_too_small(codec):
    P = lz.Params(2, 4096, 128, 3, 255)
    x = torch.from_numpy(np.random.default_rng(0).integers(0, 3, 40000).astype(np.uint16)).cuda()
    n = x.numel() * 2
    nc = -(-n // 4096)
    records_at = 32 + 8 * nc + 8 * (-(-nc // 64))
    ob = torch.zeros(1, dtype=torch.int64, device="cuda")
    out = torch.empty(records_at - 1, dtype=torch.uint8, device="cuda")
    with pytest.raises(lz.LzError) as e:
        lz.lz_compress(codec.ctx, x.data_ptr(), n, P, out.data_ptr(), out.numel(), ob.data_ptr())
    assert e.value.status == lz.LZ_ERR_BUFFER_TOO_SMALL
    # room for the table but not the records: device-side error, size reported
    ref = oracle.compress(x.cpu().numpy(), Params(2, 4096, 128, 3, 255))
    out = torch.empty(records_at + 100, dtype=torch.uint8, device="cuda")
    lz.lz_compress(codec.ctx, x.data_ptr(), n, P, out.data_ptr(), out.numel(), ob.data_ptr())
    assert codec.sync() == lz.LZ_ERR_BUFFER_TOO_SMALL
    assert int(ob.item()) == len(ref)
    # exactly enough
    out = torch.empty(len(ref), dtype=torch.uint8, device="cuda")
    lz.lz_compress(codec.ctx, x.data_ptr(), n, P, out.data_ptr(), out.numel(), ob.data_ptr())
    assert codec.sync() == lz.LZ_OK
    assert np.array_equal(out.cpu().numpy(), ref)


def test_decompress_output_too_small(codec):
    good, x = _stream()
    d = G.to_dev(np.frombuffer(bytes(good), np.uint8))
    out = torch.empty(x.size - 1, dtype=torch.uint8, device="cuda")
    ob = torch.zeros(1, dtype=torch.int64, device="cuda")
    lz.lz_decompress(codec.ctx, d.data_ptr(), d.numel(), out.data_ptr(), out.numel(),
                     ob.data_ptr())
    assert codec.sync() == lz.LZ_ERR_BUFFER_TOO_SMALL


def test_invalid_arguments(codec):
    x = torch.zeros(64, dtype=torch.uint8, device="cuda")
    out = torch.empty(4096, dtype=torch.uint8, device="cuda")
    ob = torch.zeros(2, dtype=torch.int64, device="cuda")
    bad_params = [lz.Params(3, 4096, 128, 3), lz.Params(2, 4008, 128, 3), lz.Params(2, 32784, 128, 3),
                  lz.Params(2, 4096, 0, 3), lz.Params(2, 4096, 2000, 3),
                  lz.Params(2, 4096, 128, 0), lz.Params(2, 4096, 128, 9, 8)]
    for P in bad_params:
        with pytest.raises(lz.LzError) as e:
            lz.lz_compress(codec.ctx, x.data_ptr(), 64, P, out.data_ptr(), 4096, ob.data_ptr())
        assert e.value.status == lz.LZ_ERR_INVALID_ARG
    P = lz.Params(2, 4096, 128, 3)
    cases = [
        (x.data_ptr(), 63, out.data_ptr(), ob.data_ptr()),       # n % S
        (x.data_ptr(), 64, 0, ob.data_ptr()),                     # null output
        (x.data_ptr(), 64, out.data_ptr(), 0),                    # null size
        (x.data_ptr(), 64, out.data_ptr(), ob.data_ptr() + 4),    # misaligned size
        (0, 64, out.data_ptr(), ob.data_ptr()),                   # null input
    ]
    for din, n, dout, dob in cases:
        with pytest.raises(lz.LzError) as e:
            lz.lz_compress(codec.ctx, din, n, P, dout, 4096, dob)
        assert e.value.status == lz.LZ_ERR_INVALID_ARG
    assert codec.sync() == lz.LZ_OK


def test_corrupt_version2_streams_rejected_like_the_oracle(codec):
    """Stream version 2: a stored chunk whose size disagrees with the chunk,
    and a token count of 0 in a version-1 stream, are corrupt on both sides."""
    x = np.frombuffer(bytes(range(48)) + b"abcabcabcabcabca", np.uint8)  # 3 stored, 1 coded
    P = oracle.Params(1, 16, 8, 3, 255)
    good = bytearray(oracle.compress(x, P, version=2).tobytes())
    assert _decode_status(codec, good) == lz.LZ_OK
    st = glz1_reader.read(bytes(good))
    assert st.stored == [True, True, True, False]
    cases = []
    b = bytearray(good); b[36] = 15; cases.append(b)   # stored size 15 != 16
    b = bytearray(good); b[4] = 1; cases.append(b)     # token count 0 in version 1
    for i, c in enumerate(cases):
        assert oracle.decompress_status(bytes(c)) == oracle.ECORRUPT, i
        assert _decode_status(codec, c) == lz.LZ_ERR_CORRUPT, i
        assert _decode_status(codec, good) == lz.LZ_OK, i
