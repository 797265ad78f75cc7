"""Launch shape and autotuning change how chunks are spread over the GPU,
never the stream: every warps-per-block setting gives the oracle's bytes,
and lz_autotune_ex returns parameters from its grid, a launch shape, and
the trials it timed."""
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


@pytest.mark.parametrize("wpb", [0, 1, 2, 4, 8])
@pytest.mark.parametrize("S,C,W,m", [(2, 4096, 128, 3), (1, 2048, 300, 3), (4, 8192, 256, 2)])
def test_launch_shape_keeps_the_stream(codec, wpb, S, C, W, m):
    x = synth.markov_codes(300_000 // S, seed=S + wpb).astype({1: np.uint8, 2: np.uint16, 4: np.uint32}[S])
    P = lz.Params(S, C, W, m, 255)
    d = torch.from_numpy(x.view(np.uint8)).cuda()
    out, nb = codec.compress(d, P)
    cap = out.numel()
    lz.lz_compress_ex(codec.ctx, d.data_ptr(), d.numel(), P, out.data_ptr(), cap, nb.data_ptr(),
                      torch.cuda.current_stream().cuda_stream, warps_per_block=wpb)
    assert codec.sync() == lz.LZ_OK
    ref = oracle.compress(x, oracle.Params(S, C, W, m, 255))
    assert np.array_equal(out[: int(nb.item())].cpu().numpy(), ref)


def test_bad_launch_shape_rejected(codec):
    d = torch.zeros(4096, dtype=torch.uint8, device="cuda")
    out = torch.empty(8192, dtype=torch.uint8, device="cuda")
    nb = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(lz.LzError) as e:
        lz.lz_compress_ex(codec.ctx, d.data_ptr(), 4096, lz.Params(1, 4096, 64, 3), out.data_ptr(),
                          8192, nb.data_ptr(), warps_per_block=3)
    assert e.value.status == lz.LZ_ERR_INVALID_ARG


def test_autotune_ex_reports_trials(codec):
    x = synth.quant_codes_laplace(1 << 20, seed=5)
    d = torch.from_numpy(x.view(np.uint8)).cuda()
    P, wpb, trials = lz.lz_autotune_ex(codec.ctx, d.data_ptr(), d.numel(), 2)
    assert (P.C, P.W) in {(C, W) for C in (2048, 4096, 8192, 16384) for W in (64, 128, 256, 512)}
    assert P.S == 2 and P.m == 3 and P.M == 255
    assert wpb in (0, 1, 2, 4, 8)
    assert len(trials) >= 17
    assert {(t["C"], t["W"]) for t in trials[:16]} == {(C, W) for C in (2048, 4096, 8192, 16384)
                                                      for W in (64, 128, 256, 512)}
    assert all(t["ms"] > 0 and t["ratio"] > 1 for t in trials)
    # the choice compresses exactly as the oracle does
    out, nb = codec.compress(d, P)
    lz.lz_compress_ex(codec.ctx, d.data_ptr(), d.numel(), P, out.data_ptr(), out.numel(),
                      nb.data_ptr(), torch.cuda.current_stream().cuda_stream, warps_per_block=wpb)
    assert codec.sync() == lz.LZ_OK
    ref = oracle.compress(x, oracle.Params(P.S, P.C, P.W, P.m, P.M))
    assert np.array_equal(out[: int(nb.item())].cpu().numpy(), ref)
