"""lz_compress_host: host buffers in and out, compressed in overlapping
pieces of whole index superblocks (small at both ends, about 64 MiB in the
middle).  The stream must be byte-identical to the
CPU oracle's (and so to lz_compress of the same bytes): chunks are
independent (section 3.3.1), so the pieces' records, table entries and
rebased index entries are the whole input's."""
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


def _host(codec, x: np.ndarray, P: lz.Params, pinned: bool = True, cap=None):
    xb = np.ascontiguousarray(x).view(np.uint8).reshape(-1)
    hin = torch.from_numpy(xb.copy())
    cap = lz.lz_compressed_bound(xb.size, P) if cap is None else cap
    hout = torch.empty(max(cap, 1), dtype=torch.uint8)
    if pinned:
        hin, hout = hin.pin_memory(), hout.pin_memory()
    n = lz.lz_compress_host(codec.ctx, hin.data_ptr(), xb.size, P, hout.data_ptr(), cap)
    return hout[:n].numpy().copy()


CASES = [
    ("quant u16, 40 superblocks + ragged", lambda: synth.quant_codes_laplace(5_300_001, seed=7),
     lz.Params(2, 4096, 128, 3, 255)),
    ("markov u8, 2 KiB chunks", lambda: (synth.markov_codes(9_000_000, seed=3) % 256).astype(np.uint8),
     lz.Params(1, 2048, 300, 3, 255)),
    ("field f32", lambda: synth.gaussian_field((40, 128, 256), seed=5), lz.Params(4, 8192, 256, 2, 255)),
    # pieces that grow (6, 16, 8 MiB and the rest): the scratch must keep
    # the earlier pieces' look-back words
    ("quant u16, 30 MiB in growing pieces", lambda: synth.quant_codes_laplace(15_728_640 + 999, seed=2),
     lz.Params(2, 4096, 128, 3, 255)),
    ("one chunk", lambda: synth.quant_codes_laplace(1000, seed=1), lz.Params(2, 4096, 128, 3, 255)),
    ("empty", lambda: np.zeros(0, np.uint16), lz.Params(2, 4096, 128, 3, 255)),
]


@pytest.mark.parametrize("name,gen,P", CASES, ids=[c[0] for c in CASES])
def test_host_stream_equals_oracle(codec, name, gen, P):
    x = gen()
    ref = oracle.compress(x, oracle.Params(P.S, P.C, P.W, P.m, P.M))
    got = _host(codec, x, P)
    assert got.size == ref.size
    assert np.array_equal(got, ref)
    assert codec.sync() == lz.LZ_OK


def test_pageable_buffers(codec):
    x = synth.quant_codes_laplace(3_000_000, seed=9)
    P = lz.Params(2, 4096, 128, 3, 255)
    ref = oracle.compress(x, oracle.Params(2, 4096, 128, 3, 255))
    assert np.array_equal(_host(codec, x, P, pinned=False), ref)


def test_output_too_small_reports_needed_size(codec):
    x = synth.quant_codes_laplace(2_500_000, seed=2)
    P = lz.Params(2, 4096, 128, 3, 255)
    ref = oracle.compress(x, oracle.Params(2, 4096, 128, 3, 255))
    xb = torch.from_numpy(x.view(np.uint8).copy()).pin_memory()
    out = torch.empty(ref.size - 1, dtype=torch.uint8).pin_memory()
    nb = lz.ctypes.c_uint64()
    st = lz.load().lz_compress_host(codec.ctx, xb.data_ptr(), xb.numel(), lz.ctypes.byref(P.c()),
                                    out.data_ptr(), out.numel(), lz.ctypes.byref(nb), None)
    assert st == lz.LZ_ERR_BUFFER_TOO_SMALL
    assert nb.value == ref.size
    # the context is still usable
    assert np.array_equal(_host(codec, x, P), ref)
