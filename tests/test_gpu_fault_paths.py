"""Failure detection without a GPU fault: the context's test hooks make a
bounded device wait run out (a look-back whose predecessor chunk is never
compressed, so its prefix never comes) and make an allocation fail, and the
library must report LZ_ERR_TIMEOUT / LZ_ERR_NOMEM, return, and leave the
context usable.  Nothing here traps, faults or hangs the GPU: every device
wait in the compressor gives up after the hook's poll limit."""
from __future__ import annotations

import time

import numpy as np
import pytest
import torch

import oracle
from paper_2304_07342_gb300 import lz, synth
from tests import gpu_util as G

pytestmark = pytest.mark.gpu

P = lz.Params(2, 4096, 128, 3, 255)


def _input(n_sym: int = 64 * 2048):
    x = synth.quant_codes_laplace(n_sym, seed=21)
    return x, torch.from_numpy(x.view(np.uint8)).cuda()


def _compress(codec, d, cap=None):
    cap = cap or lz.lz_compressed_bound(d.numel(), P)
    out = torch.empty(cap, dtype=torch.uint8, device="cuda")
    nb = torch.zeros(1, dtype=torch.int64, device="cuda")
    lz.lz_compress(codec.ctx, d.data_ptr(), d.numel(), P, out.data_ptr(), cap, nb.data_ptr(),
                   torch.cuda.current_stream().cuda_stream)
    return out, nb


@pytest.mark.parametrize("first_chunk", [1, 5])
def test_lookback_wait_runs_out(first_chunk):
    codec = G.codec()
    try:
        x, d = _input()
        lz.lz_set_test_hooks(codec.ctx, spin_limit=2000, first_chunk=first_chunk)
        t = time.perf_counter()
        _compress(codec, d)
        st = codec.sync()
        elapsed = time.perf_counter() - t
        assert st == lz.LZ_ERR_TIMEOUT
        assert elapsed < 5.0, elapsed  # the kernel gave up, it did not hang
        # the context is usable again once the hooks are cleared
        lz.lz_set_test_hooks(codec.ctx)
        out, nb = _compress(codec, d)
        assert codec.sync() == lz.LZ_OK
        ref = oracle.compress(x, oracle.Params(2, 4096, 128, 3, 255))
        assert int(nb.item()) == ref.size
        assert np.array_equal(out[: ref.size].cpu().numpy(), ref)
    finally:
        codec.close()


def test_poll_limit_alone_changes_nothing():
    """A small poll limit with every chunk handed out still compresses
    exactly: the limit only matters for a wait that cannot end."""
    codec = G.codec()
    try:
        x, d = _input(16 * 2048)
        lz.lz_set_test_hooks(codec.ctx, spin_limit=1 << 16)
        out, nb = _compress(codec, d)
        assert codec.sync() == lz.LZ_OK
        ref = oracle.compress(x, oracle.Params(2, 4096, 128, 3, 255))
        assert np.array_equal(out[: int(nb.item())].cpu().numpy(), ref)
    finally:
        codec.close()


def test_injected_allocation_failure():
    codec = G.codec()  # a new context holds 64 KiB of scratch
    try:
        x, d = _input(256 * 2048)  # 256 chunks: more look-back and parking scratch
        lz.lz_set_test_hooks(codec.ctx, fail_alloc=1)
        with pytest.raises(lz.LzError) as e:
            _compress(codec, d)
        assert e.value.status == lz.LZ_ERR_NOMEM
        item = (d.data_ptr(), d.numel(), d.data_ptr(), d.numel(),
                torch.zeros(1, dtype=torch.int64, device="cuda").data_ptr(), P)
        with pytest.raises(lz.LzError) as e:
            lz.lz_batch_create(codec.ctx, [item])
        assert e.value.status == lz.LZ_ERR_NOMEM
        assert codec.sync() == lz.LZ_OK  # nothing was enqueued
        lz.lz_set_test_hooks(codec.ctx)
        out, nb = _compress(codec, d)
        assert codec.sync() == lz.LZ_OK
        ref = oracle.compress(x, oracle.Params(2, 4096, 128, 3, 255))
        assert np.array_equal(out[: int(nb.item())].cpu().numpy(), ref)
    finally:
        codec.close()
