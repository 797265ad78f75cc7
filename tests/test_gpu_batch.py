"""Batched launches: every item of a batch (mixed sizes and parameters,
empty items included) is byte-identical to compressing it alone, re-runs
and CUDA-graph replays give the same bytes, and batched decompression
restores every input."""
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


def _items(seed=0, n=40):
    rng = np.random.default_rng(seed)
    params = [lz.Params(1, 2048, 64, 3), lz.Params(2, 4096, 128, 3), lz.Params(4, 8192, 256, 2),
              lz.Params(2, 1024, 512, 2, 40), lz.Params(1, 16, 8, 1, 4)]
    out = []
    for i in range(n):
        P = params[i % len(params)]
        kind = i % 4
        nbytes = int(np.exp(rng.uniform(np.log(16), np.log(300_000))))
        nbytes -= nbytes % 16
        if i == 3:
            nbytes = 0
        if i == 7:
            nbytes = P.S
        n_sym = nbytes // P.S
        if kind == 0:
            x = synth.quant_codes_laplace(n_sym, seed=i).astype(np.uint32)
        elif kind == 1:
            x = synth.markov_codes(n_sym, seed=i)
        elif kind == 2:
            x = synth.uniform_bytes(n_sym * 4, seed=i).view(np.uint32)
        else:
            x = synth.sorted_indices(n_sym, seed=i).astype(np.uint32)
        x = x.astype({1: np.uint8, 2: np.uint16, 4: np.uint32}[P.S])
        out.append((x, P))
    return out


def _run_batch(codec, items):
    ins, outs, nbs, desc = [], [], [], []
    for x, P in items:
        d = G.to_dev(x) if x.nbytes else torch.empty(16, dtype=torch.uint8, device="cuda")[:0]
        cap = lz.lz_compressed_bound(x.nbytes, P)
        o = torch.full((cap,), 0x5A, dtype=torch.uint8, device="cuda")
        nb = torch.zeros(1, dtype=torch.int64, device="cuda")
        ins.append(d); outs.append(o); nbs.append(nb)
        desc.append((d.data_ptr() if x.nbytes else 0, x.nbytes, o.data_ptr(), cap, nb.data_ptr(), P))
    b = lz.lz_batch_create(codec.ctx, desc)
    torch.cuda.synchronize()  # plan uploads done before runs on any stream
    return b, ins, outs, nbs


def test_batch_items_equal_single_calls(codec):
    items = _items()
    b, ins, outs, nbs = _run_batch(codec, items)
    try:
        for rep in range(2):
            lz.lz_batch_run(codec.ctx, b, torch.cuda.current_stream().cuda_stream)
            assert codec.sync() == lz.LZ_OK
            for (x, P), d, o, nb in zip(items, ins, outs, nbs):
                size = int(nb.item())
                got = o[:size].cpu().numpy()
                if x.nbytes <= 64 * 1024:
                    ref = oracle.compress(x, oracle.Params(*P.__dict__.values()))
                else:
                    ref = codec.compress_sync(d, P).cpu().numpy()
                assert np.array_equal(got, ref), (rep, P, x.nbytes, G.first_difference(got, ref))
    finally:
        lz.lz_batch_destroy(b)


def test_batch_decompress_restores_inputs(codec):
    items = _items(seed=1, n=33)
    b, ins, outs, nbs = _run_batch(codec, items)
    lz.lz_batch_run(codec.ctx, b)
    assert codec.sync() == lz.LZ_OK
    lz.lz_batch_destroy(b)
    desc, decs, dnbs = [], [], []
    for (x, P), o, nb in zip(items, outs, nbs):
        size = int(nb.item())
        dec = torch.full((max(x.nbytes, 1),), 0x33, dtype=torch.uint8, device="cuda")
        dnb = torch.full((1,), -1, dtype=torch.int64, device="cuda")
        decs.append(dec); dnbs.append(dnb)
        desc.append((o.data_ptr(), size, dec.data_ptr(), x.nbytes, dnb.data_ptr(), None))
    db = lz.lz_batch_create(codec.ctx, desc, decompress=True)
    try:
        for rep in range(2):
            lz.lz_batch_run(codec.ctx, db)
            assert codec.sync() == lz.LZ_OK
            for (x, P), dec, dnb in zip(items, decs, dnbs):
                assert int(dnb.item()) == x.nbytes
                assert np.array_equal(dec[: x.nbytes].cpu().numpy(), x.view(np.uint8).reshape(-1))
    finally:
        lz.lz_batch_destroy(db)


def test_batch_graph_capture_replay(codec):
    items = _items(seed=2, n=24)
    b, ins, outs, nbs = _run_batch(codec, items)
    try:
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            lz.lz_batch_run(codec.ctx, b, s.cuda_stream)  # warm-up outside the graph
        torch.cuda.synchronize()
        ref = [o[: int(nb.item())].clone() for o, nb in zip(outs, nbs)]
        for o in outs:
            o.fill_(0)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            lz.lz_batch_run(codec.ctx, b, s.cuda_stream)
        for rep in range(3):
            g.replay()
            torch.cuda.synchronize()
            assert codec.sync() == lz.LZ_OK
            for r, o, nb in zip(ref, outs, nbs):
                assert int(nb.item()) == r.numel()
                assert torch.equal(o[: r.numel()], r)
    finally:
        torch.cuda.synchronize()
        lz.lz_batch_destroy(b)


def test_autotune_picks_valid_exact_params(codec):
    x = synth.markov_codes(1 << 20, seed=3).astype(np.uint16)
    d = G.to_dev(x)
    P = lz.lz_autotune(codec.ctx, d.data_ptr(), d.numel(), 2)
    assert lz.lz_check_params(P) == lz.LZ_OK and P.S == 2
    assert P.C in (2048, 4096, 8192) and P.W in (64, 128, 256)
    small = x[: 20_000]
    got = G.gpu_compress(codec, small, P)
    assert np.array_equal(got, oracle.compress(small, oracle.Params(P.S, P.C, P.W, P.m, P.M)))


@pytest.mark.parametrize("match,version", [(lz.LZ_MATCH_EXACT, 2), (lz.LZ_MATCH_PAPER, 1),
                                           (lz.LZ_MATCH_PAPER, 2), (lz.LZ_MATCH_OVERLAP, 2)])
def test_batch_options_equal_single_calls(codec, match, version):
    """lz_batch_create_ex: every item equals lz_compress_ex with the same
    matcher and stream version (and the oracle for the small ones); the
    streams decode through a batched decompression."""
    items = _items(seed=5, n=24)
    ins, outs, nbs, desc = [], [], [], []
    for x, P in items:
        d = G.to_dev(x) if x.nbytes else torch.empty(16, dtype=torch.uint8, device="cuda")[:0]
        cap = lz.lz_compressed_bound(x.nbytes, P)
        o = torch.full((cap,), 0x5A, dtype=torch.uint8, device="cuda")
        nb = torch.zeros(1, dtype=torch.int64, device="cuda")
        ins.append(d); outs.append(o); nbs.append(nb)
        desc.append((d.data_ptr() if x.nbytes else 0, x.nbytes, o.data_ptr(), cap, nb.data_ptr(), P))
    st = torch.cuda.current_stream().cuda_stream
    b = lz.lz_batch_create(codec.ctx, desc, stream=st, match=match, version=version)
    lz.lz_batch_run(codec.ctx, b, st)
    lz.lz_batch_destroy(b, st)
    assert codec.sync() == lz.LZ_OK
    for (x, P), d, o, nb in zip(items, ins, outs, nbs):
        got = o[: int(nb.item())].cpu().numpy()
        if x.nbytes <= 64 * 1024:
            ref = oracle.compress(x, oracle.Params(P.S, P.C, P.W, P.m, P.M), mode=match,
                                  version=version)
        else:
            ref = codec.compress_sync(d, P, match=match, version=version).cpu().numpy()
        assert np.array_equal(got, ref), (P, x.nbytes, G.first_difference(got, ref))
        if x.nbytes:
            assert np.array_equal(G.gpu_decompress(codec, got), x.view(np.uint8).reshape(-1))
    with pytest.raises(lz.LzError):
        lz.lz_batch_create(codec.ctx, desc, stream=st, match=lz.LZ_MATCH_OVERLAP, version=1)
