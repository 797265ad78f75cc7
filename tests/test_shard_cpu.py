"""Sharded compression, host side: cut points, the offset plan and the
rank exchange (gloo, CPU processes).  Shard streams come from the oracle;
the test places them with a plain numpy transcription of what the stitch
kernel writes, and the result must be the oracle's whole-input stream."""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from oracle import Params
from paper_2304_07342_gb300 import shard, synth


def np_stitch(layout: shard.Layout, streams) -> np.ndarray:
    out = np.full(layout.stream_bytes, 0xEE, np.uint8)
    NC = layout.total_chunks
    for p, s in zip(layout.shards, streams):
        s = np.asarray(s, np.uint8)
        nc, cb = p.shard_chunks, p.chunk_base
        if cb == 0:
            h = s[:32].copy()
            h[20:24] = np.frombuffer(np.uint32(NC).tobytes(), np.uint8)
            h[24:32] = np.frombuffer(np.uint64(layout.total_bytes).tobytes(), np.uint8)
            out[:32] = h
        out[32 + 8 * cb: 32 + 8 * (cb + nc)] = s[32: 32 + 8 * nc]
        idx = s[32 + 8 * nc: p.src_records].view("<u8") + np.uint64(p.record_base)
        at = 32 + 8 * NC + 8 * (cb // 64)
        out[at: at + idx.size * 8] = idx.view(np.uint8)
        out[p.dst_records: p.dst_records + p.record_bytes] = s[p.src_records:]
    return out


def data_for(kind: int, n: int) -> np.ndarray:
    if kind == 0:
        return (synth.markov_codes(n, seed=11) % 256).astype(np.uint8)
    if kind == 1:
        return synth.quant_codes_laplace(n // 2, seed=12).view(np.uint8)
    return synth.sorted_indices(n // 4, seed=13).view(np.uint8)


CASES = [  # (S, C, W, m, n_bytes)
    (1, 256, 64, 3, 0),
    (1, 256, 64, 3, 100),              # one partial chunk
    (2, 512, 128, 3, 64 * 512),        # exactly one superblock
    (2, 512, 128, 3, 64 * 512 + 2),    # one more symbol
    (1, 256, 200, 3, 3 * 64 * 256 + 5 * 256 + 17),
    (4, 1024, 300, 2, 5 * 64 * 1024 + 1024 * 7 + 12),   # two offset bytes
]


@pytest.mark.parametrize("world", [1, 2, 3, 5])
def test_shard_ranges_cover_in_superblocks(world):
    for n in (0, 1, 4095, 4096, 64 * 4096, 64 * 4096 + 1, 1000 * 4096 + 3):
        r = shard.shard_ranges(n, 4096, world)
        assert len(r) == world and r[0][0] == 0 and r[-1][1] == n
        assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
        sbs = [shard.div_up(b1 - b0, 64 * 4096) for b0, b1 in r]
        assert max(sbs) - min(sbs) <= 1 and sbs == sorted(sbs, reverse=True)
        for b0, b1 in r:
            assert b0 % (64 * 4096) == 0 or b0 == n


@pytest.mark.parametrize("case", CASES, ids=[str(c) for c in CASES])
@pytest.mark.parametrize("world", [1, 2, 3, 5])
def test_stitched_shards_equal_whole_stream(case, world):
    S, C, W, m, n = case
    P = Params(S, C, W, m)
    x = data_for({1: 0, 2: 1, 4: 2}[S], n)[:n]
    whole = oracle.compress(x, P)
    ranges = shard.shard_ranges(n, C, world)
    streams = [oracle.compress(x[b0:b1], P) for b0, b1 in ranges]
    meta = [(shard.div_up(b1 - b0, C), s.size) for (b0, b1), s in zip(ranges, streams)]
    layout = shard.plan(meta, n, C)
    assert layout.stream_bytes == whole.size
    assert np.array_equal(np_stitch(layout, streams), whole)
    assert np.array_equal(oracle.decompress(np_stitch(layout, streams)), x)


def test_plan_rejects_bad_meta():
    with pytest.raises(ValueError):
        shard.plan([(10, 200)], 11 * 256, 256)          # chunk count mismatch
    with pytest.raises(ValueError):
        shard.plan([(10, 200), (5, 200)], 15 * 256, 256)  # second shard mid-superblock
    with pytest.raises(ValueError):
        shard.plan([(10, 40)], 10 * 256, 256)            # stream shorter than its table


# --- two and three ranks over gloo --------------------------------------------

def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, case, outdir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        S, C, W, m, n = case
        P = Params(S, C, W, m)
        x = data_for({1: 0, 2: 1, 4: 2}[S], n)[:n]   # every rank draws the same input
        b0, b1 = shard.shard_ranges(n, C, world)[rank]
        mine = torch.from_numpy(oracle.compress(x[b0:b1], P))
        meta = shard.exchange_meta(torch, dist, shard.div_up(b1 - b0, C), mine.numel())
        layout = shard.plan(meta, n, C)
        got = shard.gather_streams(torch, dist, mine, layout, root=0)
        if rank == 0:
            out = np_stitch(layout, [g.numpy() for g in got])
            np.save(os.path.join(outdir, "stream.npy"), out)
        else:
            assert got is None
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("case", [CASES[1], CASES[4], CASES[5]], ids=["tiny", "s1", "s4"])
def test_gloo_ranks_assemble_whole_stream(tmp_path, world, case):
    mp.spawn(_rank_main, args=(world, _free_port(), case, str(tmp_path)), nprocs=world,
             join=True)
    S, C, W, m, n = case
    x = data_for({1: 0, 2: 1, 4: 2}[S], n)[:n]
    got = np.load(tmp_path / "stream.npy")
    assert np.array_equal(got, oracle.compress(x, Params(S, C, W, m)))
