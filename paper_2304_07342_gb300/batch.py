"""Batched compression of many uneven buffers (one persistent launch).

Builds the many-buffer workload (sizes log-uniform over [4 KiB, 16 MiB],
element types drawn uniformly from 1-byte codes, 2-byte codes, float32
field slices and int32 indices) as slices of device-resident pools, plans
one batch per direction through the C ABI (``lz_batch_create``), captures
its run in a CUDA graph and times it against one plain launch per buffer.
All work runs in the CUDA kernels of ``liblz.so``.
"""
from __future__ import annotations

import time
from dataclasses import dataclass

import numpy as np

from . import lz, synth

KIND_NAMES = ("uint8 codes", "uint16 codes", "float32 field", "int32 indices")
KIND_S = (1, 2, 4, 4)


@dataclass
class Workload:
    sizes: np.ndarray
    kinds: np.ndarray
    params: list            # per kind
    pools: list             # device uint8 tensors per kind
    ins: list               # device views, one per buffer
    out_arena: object       # device uint8 tensor holding every output
    out_offsets: np.ndarray
    out_caps: np.ndarray
    out_bytes: object       # device int64 [n]

    @property
    def total_bytes(self) -> int:
        return int(self.sizes.sum())


def make_pools(torch, pool_bytes: int = 256 << 20, seed: int = 0, device="cuda"):
    """One device pool per kind, generated by the seeded generators."""
    codes = synth.markov_codes(pool_bytes // 2, seed=seed)
    nf = pool_bytes // 4
    side = max(1, int(round((nf / 256) ** 0.5)))
    field = synth.gaussian_field((side, side, 256), seed=seed).reshape(-1)
    arrs = [(codes % 256).astype(np.uint8)[:pool_bytes],
            codes.astype(np.uint16),
            field,
            synth.sorted_indices(nf, seed=seed)]
    return [torch.from_numpy(np.ascontiguousarray(a).view(np.uint8).reshape(-1)).to(device)
            for a in arrs]


def autotuned_params(codec, pools, sample_bytes: int = 8 << 20, report: list | None = None) -> list:
    """Chunk size and window per kind from ``lz_autotune_ex`` on the head of
    each kind's pool (its launch-shape choice and every trial go to
    `report`).  One launch sizes every warp's shared memory for the largest
    chunk of the batch, so a kind whose sample does not compress (where a
    large chunk only saves per-chunk overhead) is held to the largest chunk
    chosen for a kind that does compress."""
    out, ratios = [], []
    for k, pool in enumerate(pools):
        n = min(pool.numel(), sample_bytes)
        n -= n % KIND_S[k]
        p, wpb, trials = lz.lz_autotune_ex(codec.ctx, pool.data_ptr(), n, KIND_S[k])
        s = codec.compress_sync(pool[:n], p)
        out.append(p)
        ratios.append(n / max(1, s.numel()))
        if report is not None:
            report.append({"kind": KIND_NAMES[k], "chosen": dict(S=p.S, C=p.C, W=p.W, m=p.m, M=p.M),
                           "warps_per_block": wpb, "trials": trials})
    return hold_chunks(out, ratios)


def hold_chunks(params: list, ratios: list, min_ratio: float = 1.05) -> list:
    """Per-kind parameters with the chunk of every kind whose sample ratio is
    below `min_ratio` held to the largest chunk of the kinds at or above it
    (unchanged when no kind compresses, or when its chunk is already no
    larger)."""
    caps = [p.C for p, r in zip(params, ratios) if r >= min_ratio]
    if not caps:
        return list(params)
    cap = max(caps)
    return [p if r >= min_ratio or p.C <= cap else lz.Params(p.S, cap, p.W, p.m, p.M)
            for p, r in zip(params, ratios)]


def build(torch, n_buffers: int = 10_000, seed: int = 0, params=None, pools=None,
          lo_bytes: int = 4096, hi_bytes: int = 16 << 20, device="cuda",
          autotune_codec=None, report: list | None = None) -> Workload:
    """Buffers are 16-byte aligned slices of the pools; outputs live in one
    arena at 256-byte aligned offsets.  Parameters per kind: ``params``, else
    autotuned when a codec is given, else fixed defaults."""
    sizes, kinds = synth.batch_buffers(n_buffers, seed=seed, lo_bytes=lo_bytes,
                                       hi_bytes=hi_bytes)
    pools = pools if pools is not None else make_pools(torch, seed=seed, device=device)
    if params is None and autotune_codec is not None:
        params = autotuned_params(autotune_codec, pools, report=report)
    if params is None:
        params = [lz.Params(KIND_S[k], 4096 if KIND_S[k] < 4 else 8192,
                            128 if KIND_S[k] < 4 else 256, 3 if KIND_S[k] < 4 else 2)
                  for k in range(4)]
    rng = np.random.default_rng(seed + 1)
    ins = []
    for sz, k in zip(sizes, kinds):
        pool = pools[k]
        s = int(sz) - int(sz) % params[k].S
        off = int(rng.integers(0, (pool.numel() - s) // 16 + 1)) * 16
        ins.append(pool[off:off + s])
    sizes = np.array([t.numel() for t in ins], np.int64)
    caps = np.array([lz.lz_compressed_bound(int(s), params[k]) for s, k in zip(sizes, kinds)],
                    np.int64)
    offs = np.zeros(n_buffers, np.int64)
    offs[1:] = np.cumsum((caps + 255) // 256 * 256)[:-1]
    arena = torch.empty(int(offs[-1] + caps[-1] + 256), dtype=torch.uint8, device=device)
    out_bytes = torch.zeros(n_buffers, dtype=torch.int64, device=device)
    return Workload(sizes, kinds, params, pools, ins, arena, offs, caps, out_bytes)


def compress_items(w: Workload):
    base = w.out_arena.data_ptr()
    nb = w.out_bytes.data_ptr()
    return [(t.data_ptr(), t.numel(), base + int(o), int(c), nb + 8 * i, w.params[k])
            for i, (t, o, c, k) in enumerate(zip(w.ins, w.out_offsets, w.out_caps, w.kinds))]


def time_gpu(torch, fn, steps: int, warmup: int = 3) -> float:
    """Average seconds per call of fn() measured with CUDA events."""
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / steps / 1e3


def run(torch, codec, w: Workload, steps: int = 3, check: int = 64) -> dict:
    """Batched (one persistent launch, CUDA graph) vs one plain launch per
    buffer, for compression and decompression of the whole workload."""
    stream = torch.cuda.current_stream()
    items = compress_items(w)
    t0 = time.perf_counter()
    b = lz.lz_batch_create(codec.ctx, items, stream=stream.cuda_stream)
    plan_s = time.perf_counter() - t0
    torch.cuda.synchronize()
    out = {"buffers": len(items), "input_bytes": w.total_bytes, "plan_seconds": round(plan_s, 4)}
    try:
        g_stream = torch.cuda.Stream()
        with torch.cuda.stream(g_stream):
            lz.lz_batch_run(codec.ctx, b, g_stream.cuda_stream)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=g_stream):
            lz.lz_batch_run(codec.ctx, b, g_stream.cuda_stream)
        t_batch = time_gpu(torch, graph.replay, steps)
        st = codec.sync()
        if st != lz.LZ_OK:
            raise lz.LzError(st, "batched compress")
        sizes = w.out_bytes.cpu().numpy().copy()

        def per_buffer():
            for it in items:
                lz.lz_compress(codec.ctx, it[0], it[1], it[5], it[2], it[3], it[4],
                               stream.cuda_stream)
        t_plain = time_gpu(torch, per_buffer, max(1, steps // 2), warmup=1)
        st = codec.sync()
        if st != lz.LZ_OK:
            raise lz.LzError(st, "per-buffer compress")
        same = np.array_equal(sizes, w.out_bytes.cpu().numpy())
    finally:
        torch.cuda.synchronize()
        lz.lz_batch_destroy(b, stream.cuda_stream)
    # spot check: a sample of buffers is identical to compressing it alone
    rng = np.random.default_rng(0)
    for i in rng.choice(len(items), size=min(check, len(items)), replace=False):
        ref = codec.compress_sync(w.ins[i], w.params[w.kinds[i]])
        o = int(w.out_offsets[i])
        got = w.out_arena[o:o + int(sizes[i])]
        if ref.numel() != int(sizes[i]) or not torch.equal(ref, got):
            raise AssertionError(f"batched buffer {i} differs from a single call")
    # decompression of every stream, batched vs per buffer
    dec = torch.empty(int(w.sizes.sum()) + 16 * len(items), dtype=torch.uint8, device="cuda")
    doffs = np.zeros(len(items), np.int64)
    doffs[1:] = np.cumsum((w.sizes + 15) // 16 * 16)[:-1]
    dnb = torch.zeros(len(items), dtype=torch.int64, device="cuda")
    ditems = [(w.out_arena.data_ptr() + int(o), int(s), dec.data_ptr() + int(do), int(n),
               dnb.data_ptr() + 8 * i, None)
              for i, (o, s, do, n) in enumerate(zip(w.out_offsets, sizes, doffs, w.sizes))]
    db = lz.lz_batch_create(codec.ctx, ditems, decompress=True, stream=stream.cuda_stream)
    torch.cuda.synchronize()
    try:
        # one run, then the run captured in a CUDA graph and replayed
        with torch.cuda.stream(g_stream):
            lz.lz_batch_run(codec.ctx, db, g_stream.cuda_stream)
        torch.cuda.synchronize()
        dgraph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(dgraph, stream=g_stream):
            lz.lz_batch_run(codec.ctx, db, g_stream.cuda_stream)
        t_dbatch = time_gpu(torch, dgraph.replay, steps)

        def per_buffer_dec():
            for it in ditems:
                lz.lz_decompress(codec.ctx, it[0], it[1], it[2], it[3], it[4], stream.cuda_stream)
        t_dplain = time_gpu(torch, per_buffer_dec, max(1, steps // 2), warmup=1)
        st = codec.sync()
        if st != lz.LZ_OK:
            raise lz.LzError(st, "decompress")
    finally:
        torch.cuda.synchronize()
        lz.lz_batch_destroy(db, stream.cuda_stream)
    for i in rng.choice(len(items), size=min(check, len(items)), replace=False):
        do, n = int(doffs[i]), int(w.sizes[i])
        if not torch.equal(dec[do:do + n], w.ins[i]):
            raise AssertionError(f"batched decompression of buffer {i} differs")
    n = w.total_bytes
    out.update({
        "compress_batched_gbs": round(n / t_batch / 1e9, 3),
        "compress_per_buffer_gbs": round(n / t_plain / 1e9, 3),
        "decompress_batched_gbs": round(n / t_dbatch / 1e9, 3),
        "decompress_per_buffer_gbs": round(n / t_dplain / 1e9, 3),
        "ratio": round(n / float(sizes.sum()), 4),
        "sizes_equal_per_buffer": bool(same),
        "launches": {"batched": 2, "per_buffer": 2 * len(items)},
        "graphs": "both batched runs replayed from captured CUDA graphs",
        "params": [dict(kind=KIND_NAMES[k], S=p.S, C=p.C, W=p.W, m=p.m, M=p.M)
                   for k, p in enumerate(w.params)],
    })
    return out
