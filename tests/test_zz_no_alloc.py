"""lz_compress_noalloc: compression for callers that must not allocate device
memory (code running inside an allocator or an out-of-memory handler, or a
pipeline that forbids allocation after start-up).  Its scratch is a fixed
array inside the library, shared by every call, so two calls in a row must
both produce exactly what the regular entry point produces.

Kept in a file of its own, collected after every other test file.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

from paper_2304_07342_gb300 import lz, synth
from tests import gpu_util as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def codec():
    c = G.codec()
    yield c
    c.close()


CASES = [
    ("quant u16", lambda: synth.quant_codes_laplace(300_000, seed=4), lz.Params(2, 4096, 128, 3, 255)),
    ("field f32", lambda: synth.gaussian_field((8, 64, 256), seed=2), lz.Params(4, 8192, 256, 2, 255)),
    ("markov u8", lambda: (synth.markov_codes(200_003, seed=5) % 256).astype(np.uint8),
     lz.Params(1, 2048, 512, 3, 255)),
]


@pytest.mark.parametrize("name,gen,P", CASES, ids=[c[0] for c in CASES])
def test_noalloc_matches_regular_entry_point_twice(codec, name, gen, P):
    x = gen()
    d_in = torch.from_numpy(np.ascontiguousarray(x).view(np.uint8).reshape(-1)).cuda()
    ref = codec.compress_sync(d_in, P)  # the regular entry point
    cap = lz.lz_compressed_bound(d_in.numel(), P)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        # stale bytes from an earlier call must not leak into the output
        out = torch.full((cap,), 0xA5, dtype=torch.uint8, device="cuda")
        nb = torch.zeros(1, dtype=torch.int64, device="cuda")
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        lz.lz_compress_noalloc(d_in.data_ptr(), d_in.numel(), P, out.data_ptr(), cap,
                               nb.data_ptr(), stream)
        torch.cuda.synchronize()
        if call == 1:
            # the second call of a kernel variant (its code is loaded by the
            # first) takes no device memory at all
            assert torch.cuda.mem_get_info()[0] == free_before
        size = int(nb.item())
        assert 0 < size <= cap, (call, size)
        assert size == ref.numel(), call
        assert torch.equal(out[:size], ref), call


def test_noalloc_limits(codec):
    P = lz.Params(2, 16, 8, 2, 255)
    x = torch.zeros(16 * 65537, dtype=torch.uint8, device="cuda")  # 65537 chunks
    out = torch.empty(lz.lz_compressed_bound(x.numel(), P), dtype=torch.uint8, device="cuda")
    nb = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(lz.LzError) as e:
        lz.lz_compress_noalloc(x.data_ptr(), x.numel(), P, out.data_ptr(), out.numel(),
                               nb.data_ptr())
    assert e.value.status == lz.LZ_ERR_INVALID_ARG
    # exactly the maximum is accepted and matches the regular entry point
    x = x[: 16 * 65536]
    ref = codec.compress_sync(x, P)
    lz.lz_compress_noalloc(x.data_ptr(), x.numel(), P, out.data_ptr(), out.numel(),
                           nb.data_ptr())
    torch.cuda.synchronize()
    assert int(nb.item()) == ref.numel()
    assert torch.equal(out[: ref.numel()], ref)


def test_noalloc_reports_small_output(codec):
    P = lz.Params(2, 4096, 128, 3, 255)
    x = torch.from_numpy(synth.quant_codes_laplace(100_000, seed=9).view(np.uint8)).cuda()
    ref = codec.compress_sync(x, P)
    nc = -(-x.numel() // 4096)
    records_at = 32 + 8 * nc + 8 * (-(-nc // 64))
    out = torch.empty(records_at + 10, dtype=torch.uint8, device="cuda")
    nb = torch.zeros(1, dtype=torch.int64, device="cuda")
    lz.lz_compress_noalloc(x.data_ptr(), x.numel(), P, out.data_ptr(), out.numel(),
                           nb.data_ptr())
    torch.cuda.synchronize()
    assert int(nb.item()) == ref.numel() > out.numel()  # the size that was needed
