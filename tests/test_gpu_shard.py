"""Sharded compression on the GPU: shards compressed by separate calls and
placed by lz_stitch give exactly the whole-input stream (the single call's
and the oracle's); argument and header checks of lz_stitch."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
from paper_2304_07342_gb300 import lz, shard, synth
from tests import gpu_util as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def codec():
    c = G.codec()
    yield c
    c.close()


CASES = [  # (name, bytes, params)
    ("empty", lambda: np.zeros(0, np.uint8), lz.Params(1, 256, 64, 3)),
    ("one partial chunk", lambda: (synth.markov_codes(100, seed=1) % 256).astype(np.uint8),
     lz.Params(1, 256, 64, 3)),
    ("quant u16 ragged", lambda: synth.quant_codes_laplace(5 * 64 * 256 + 333, seed=2),
     lz.Params(2, 512, 128, 3)),
    ("indices i32 W300", lambda: synth.sorted_indices(7 * 64 * 256 + 5, seed=3),
     lz.Params(4, 1024, 300, 2)),
]


def _sharded(codec, d, P, world, fill=0xEE):
    n = d.numel()
    ranges = shard.shard_ranges(n, P.C, world)
    streams = [codec.compress_sync(d[b0:b1], P) for b0, b1 in ranges]
    meta = [(shard.div_up(b1 - b0, P.C), s.numel()) for (b0, b1), s in zip(ranges, streams)]
    layout = shard.plan(meta, n, P.C)
    out = torch.full((layout.stream_bytes,), fill, dtype=torch.uint8, device="cuda")
    shard.stitch(codec, layout, streams, out.data_ptr(), out.numel())
    assert codec.sync() == lz.LZ_OK
    return out


@pytest.mark.parametrize("world", [1, 2, 3, 5])
@pytest.mark.parametrize("name,gen,P", CASES, ids=[c[0] for c in CASES])
def test_stitched_equals_single_call_and_oracle(codec, name, gen, P, world):
    x = np.ascontiguousarray(gen()).view(np.uint8).reshape(-1)
    d = torch.from_numpy(x.copy()).cuda()
    whole = codec.compress_sync(d, P)
    got = _sharded(codec, d, P, world)
    assert torch.equal(got, whole)
    ref = oracle.compress(x, oracle.Params(P.S, P.C, P.W, P.m, P.M))
    assert np.array_equal(got.cpu().numpy(), ref)


def test_stitched_field_four_shards(codec):
    x = synth.gaussian_field((64, 128, 256), seed=5).view(np.uint8).reshape(-1)  # 8 MiB
    P = lz.Params(4, 8192, 256, 2)
    d = torch.from_numpy(x.copy()).cuda()
    got = _sharded(codec, d, P, 4)
    assert torch.equal(got, codec.compress_sync(d, P))
    assert torch.equal(codec.decompress_sync(got), d)


def test_stitch_argument_checks(codec):
    P = lz.Params(2, 512, 128, 3)
    x = torch.from_numpy(synth.quant_codes_laplace(2 * 64 * 256, seed=6).view(np.uint8)).cuda()
    s = codec.compress_sync(x[: 64 * 512], P)          # first superblock
    NC = 128
    out = torch.zeros(1 << 20, dtype=torch.uint8, device="cuda")
    base = out.data_ptr()

    def call(**kw):
        a = dict(d_shard=s.data_ptr(), shard_bytes=s.numel(), shard_chunks=64, chunk_base=0,
                 total_chunks=NC, total_bytes=x.numel(), record_base=0, d_out=base,
                 out_cap=out.numel())
        a.update(kw)
        lz.lz_stitch(codec.ctx, a["d_shard"], a["shard_bytes"], a["shard_chunks"],
                     a["chunk_base"], a["total_chunks"], a["total_bytes"], a["record_base"],
                     a["d_out"], a["out_cap"])

    for kw, status in [
        (dict(d_out=base + 4), lz.LZ_ERR_INVALID_ARG),           # misaligned output
        (dict(chunk_base=32), lz.LZ_ERR_INVALID_ARG),            # not on a superblock
        (dict(chunk_base=96), lz.LZ_ERR_INVALID_ARG),            # runs past the input
        (dict(shard_bytes=100), lz.LZ_ERR_INVALID_ARG),          # shorter than its table
        (dict(out_cap=1000), lz.LZ_ERR_BUFFER_TOO_SMALL),
        (dict(record_base=(1 << 20) - 2000), lz.LZ_ERR_BUFFER_TOO_SMALL),
    ]:
        with pytest.raises(lz.LzError) as e:
            call(**kw)
        assert e.value.status == status, kw
    torch.cuda.synchronize()
    assert int(out.count_nonzero()) == 0                          # nothing was enqueued
    # a header that disagrees with the arguments: corrupt, nothing written
    for kw in (dict(shard_chunks=63, shard_bytes=s.numel()),      # chunk count
               dict(total_bytes=x.numel() - 512 * 64)):           # chunk count of the input
        call(**kw)
        assert codec.sync() == lz.LZ_ERR_CORRUPT
        assert int(out.count_nonzero()) == 0
    # the valid call then works on the same context
    call()
    assert codec.sync() == lz.LZ_OK
    assert int(out.count_nonzero()) > 0
