"""Data-parallel compression of one input split across ranks (one GPU each).

Chunks are compressed independently (section 3.3.1), so an input can be cut
into shards, each compressed on its own rank, and the shard streams placed
side by side to form exactly the stream a single call would write.  The cut
points fall on index superblocks (64 chunks): then a shard's records, table
entries and index entries are those of the whole-input stream, the index
entries shifted by the record bytes of the shards before it.

The only exchange between ranks is the all-gather of each shard's (chunk
count, stream bytes); exclusive scans of it give every shard its place
(``plan``).  The shard streams are then gathered on one rank and placed by
the ``lz_stitch`` kernel.  Every byte of compressed data is produced and
moved by the library's CUDA kernels; this module only computes offsets and
calls ``torch.distributed``.
"""
from __future__ import annotations

from dataclasses import dataclass

from . import lz

SUPERBLOCK = 64     # chunks per index entry of the GLZ1 stream
HEADER = 32
TABLE_ENTRY = 8


def div_up(a: int, b: int) -> int:
    return -(-a // b)


def records_at(n_chunks: int) -> int:
    """Byte offset of the records region of a stream with n_chunks chunks."""
    return HEADER + TABLE_ENTRY * n_chunks + 8 * div_up(n_chunks, SUPERBLOCK)


def shard_ranges(n_bytes: int, chunk_bytes: int, world: int) -> list:
    """Byte ranges [b0, b1) of each rank: contiguous runs of whole
    superblocks, as even as possible, earlier ranks taking the extra ones
    (a rank gets an empty range only when there are fewer superblocks than
    ranks)."""
    if world < 1 or chunk_bytes < 1:
        raise ValueError("world and chunk_bytes must be positive")
    span = SUPERBLOCK * chunk_bytes
    n_sb = div_up(n_bytes, span)
    q, rem = divmod(n_sb, world)
    cuts = [r * q + min(r, rem) for r in range(world + 1)]
    return [(min(n_bytes, cuts[r] * span), min(n_bytes, cuts[r + 1] * span))
            for r in range(world)]


@dataclass
class Placement:
    rank: int
    shard_chunks: int
    shard_bytes: int
    chunk_base: int     # chunks of the shards before it
    record_base: int    # record bytes of the shards before it
    src_records: int    # where its records start in the shard stream
    record_bytes: int
    dst_records: int    # where they go in the whole stream


@dataclass
class Layout:
    total_bytes: int
    total_chunks: int
    records_at: int
    stream_bytes: int
    shards: list


def plan(meta: list, total_bytes: int, chunk_bytes: int) -> Layout:
    """Places of the shards, from every rank's (shard_chunks, shard_bytes)
    in rank order (the exclusive scans of the exchange)."""
    total_chunks = div_up(total_bytes, chunk_bytes)
    if sum(c for c, _ in meta) != total_chunks:
        raise ValueError("shard chunk counts do not add up to the input's")
    at = records_at(total_chunks)
    shards, cbase, rbase = [], 0, 0
    for r, (nc, nb) in enumerate(meta):
        if nc and cbase % SUPERBLOCK:
            raise ValueError(f"shard {r} does not start on a superblock")
        src = records_at(nc)
        if nb < src:
            raise ValueError(f"shard {r}: stream shorter than its table")
        shards.append(Placement(r, nc, nb, cbase, rbase, src, nb - src, at + rbase))
        cbase += nc
        rbase += nb - src
    return Layout(total_bytes, total_chunks, at, at + rbase, shards)


def exchange_meta(torch, dist, shard_chunks: int, shard_bytes: int, group=None,
                  device="cpu") -> list:
    """All-gather of every rank's (shard_chunks, shard_bytes)."""
    world = dist.get_world_size(group)
    mine = torch.tensor([shard_chunks, shard_bytes], dtype=torch.int64, device=device)
    every = [torch.empty_like(mine) for _ in range(world)]
    dist.all_gather(every, mine, group=group)
    return [tuple(int(v) for v in t.cpu()) for t in every]


def gather_streams(torch, dist, stream, layout: Layout, root: int = 0, group=None) -> list:
    """Gather every shard stream (a uint8 tensor on each rank) on `root`,
    padded to the longest; returns the trimmed list on root, None elsewhere."""
    longest = max(1, max(p.shard_bytes for p in layout.shards))
    mine = torch.zeros(longest, dtype=torch.uint8, device=stream.device)
    mine[: stream.numel()] = stream
    rank = dist.get_rank(group)
    bucket = ([torch.empty_like(mine) for _ in layout.shards] if rank == root else None)
    dist.gather(mine, bucket, dst=root, group=group)
    if rank != root:
        return None
    return [t[: p.shard_bytes] for t, p in zip(bucket, layout.shards)]


def stitch(codec, layout: Layout, streams: list, d_out: int, out_cap: int,
           stream: int = 0) -> None:
    """Place every shard stream (device tensors, 8-byte aligned) in d_out."""
    for p, s in zip(layout.shards, streams):
        lz.lz_stitch(codec.ctx, s.data_ptr(), p.shard_bytes, p.shard_chunks, p.chunk_base,
                     layout.total_chunks, layout.total_bytes, p.record_base, d_out, out_cap,
                     stream)


def compress_sharded(torch, dist, codec, d_local, params, total_bytes: int, root: int = 0,
                     group=None):
    """Compress this rank's shard (``d_local``: its byte range of the input,
    from ``shard_ranges``) and assemble the whole-input stream on ``root``.
    Returns the stream (a device uint8 tensor) on root, None elsewhere."""
    nc = div_up(d_local.numel(), params.C)
    mine = codec.compress_sync(d_local, params)
    meta = exchange_meta(torch, dist, nc, mine.numel(), group, device=d_local.device)
    layout = plan(meta, total_bytes, params.C)
    streams = gather_streams(torch, dist, mine, layout, root, group)
    if streams is None:
        return None
    # gathered rows are 8-byte aligned (fresh allocations); so is `out`
    out = torch.empty(layout.stream_bytes, dtype=torch.uint8, device=d_local.device)
    stitch(codec, layout, streams, out.data_ptr(), out.numel(),
           torch.cuda.current_stream().cuda_stream)
    st = codec.sync()
    if st != lz.LZ_OK:
        raise lz.LzError(st, "lz_stitch")
    return out
