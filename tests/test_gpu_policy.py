"""lz_select_params (the paper's parameter selection, section 3.2.3) on the
GPU makes the same choice as the oracle's policy on the same sample: both
compress the sample with multi-byte matching and compare the ratio with 1.5
in integers, and the two compressors' streams are byte-identical, so the
decisions must agree exactly."""
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


def inputs():
    rng = np.random.default_rng(3)
    yield "quant u16", synth.quant_codes_laplace(200_000, seed=1), 2
    yield "markov u16", synth.markov_codes(150_000, seed=2).astype(np.uint16), 2
    yield "markov u32", synth.markov_codes(80_000, seed=3).astype(np.uint32), 4
    yield "field f32", synth.gaussian_field((4, 64, 256), seed=4), 4
    yield "indices i32", synth.sorted_indices(60_000, seed=5), 4
    yield "random u32", synth.uniform_bytes(200_000, seed=6).view(np.uint32), 4
    yield "const u32", np.full(50_000, 5, np.uint32), 4
    yield "codes u8", synth.markov_codes(100_000, seed=7).astype(np.uint8), 1
    # a mix whose multi-byte ratio sits near the threshold
    a = synth.markov_codes(40_000, seed=8).astype(np.uint16)
    b = rng.integers(0, 1 << 16, 40_000).astype(np.uint16)
    yield "mixed u16", np.concatenate([a, b]), 2


@pytest.mark.parametrize("level", [1, 2, 3, 4])
def test_policy_matches_oracle(codec, level):
    for name, x, D in inputs():
        d = G.to_dev(x)
        got = lz.lz_select_params(codec.ctx, d.data_ptr(), d.numel(), D, level, 4096,
                                  torch.cuda.current_stream().cuda_stream)
        ref = oracle.select_params(x, D, level, 4096)
        assert (got.S, got.C, got.W, got.m, got.M) == ref.tuple(), (name, level)


def test_policy_choices(codec):
    """The decisions themselves on clear cases: repetitive codes keep
    multi-byte matching, the noisy field and random words fall back to
    single bytes."""
    st = torch.cuda.current_stream().cuda_stream
    pick = {}
    for name, x, D in inputs():
        d = G.to_dev(x)
        pick[name] = lz.lz_select_params(codec.ctx, d.data_ptr(), d.numel(), D, 3, 4096, st)
    assert pick["const u32"].S == 4 and pick["const u32"].W == 512
    assert pick["quant u16"].S == 2 and pick["quant u16"].W == 256
    assert pick["field f32"].S == 1 and pick["field f32"].W == 128
    assert pick["random u32"].S == 1
    assert pick["codes u8"].S == 1 and pick["codes u8"].m == 3


def test_policy_rejects_bad_arguments(codec):
    d = G.to_dev(np.zeros(64, np.uint8))
    st = torch.cuda.current_stream().cuda_stream
    for D, level, C, n in ((3, 3, 4096, 64), (2, 0, 4096, 64), (2, 5, 4096, 64),
                           (2, 3, 100, 64), (4, 3, 4096, 2)):
        with pytest.raises(lz.LzError):
            lz.lz_select_params(codec.ctx, d.data_ptr(), n, D, level, C, st)
