"""Continuous-batching request loop for compress / decompress requests.

Requests (Poisson arrivals; sizes lognormal; 1-, 2- or 4-byte symbols; a
share of them decompress streams produced earlier) reference device-
resident input slices.  The loop:

* admits queued requests in arrival order while their output space fits a
  stated HBM budget (a first-fit allocator over one preallocated buffer);
* runs every admitted group as one batch per direction (one persistent
  launch each) on one of a few streams, so groups admitted while others are
  still on the GPU overlap with them.  Each stream keeps its two batches and
  re-plans them for every group (``lz_batch_update``: descriptors uploaded
  into the batch's own device memory); decompression items state their
  stream's parameters and size, so no plan waits on the GPU;
* takes completion times from CUDA events (GPU clock, same origin as the
  arrival clock), hands each finished request to an optional callback and
  then frees its output space.

``run_plain`` is the comparison: one plain launch per request, in arrival
order, on one stream, with the same budget.  Latency = completion - arrival;
p50/p99 and the sustained GB/s (request bytes over the makespan) are
reported for both.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import lz, synth


@dataclass
class Request:
    rid: int
    arrival: float          # seconds from the start of the trace
    compress: bool
    d_in: int               # device pointer
    n_in: int
    params: object          # lz.Params (compress: to use; decompress: the stream's)
    n_out_max: int          # output capacity needed (decompress: the exact size)
    n_orig: int             # uncompressed size
    out_off: int = -1       # arena offset once admitted
    done: float = -1.0
    source: object = None   # device view of the uncompressed bytes


class Arena:
    """First-fit allocator over one device buffer, 256-byte granules."""

    def __init__(self, nbytes: int):
        self.free = [(0, nbytes)]

    @staticmethod
    def _round(n: int) -> int:
        return max(256, (n + 255) // 256 * 256)

    def alloc(self, n: int) -> int:
        n = self._round(n)
        for i, (o, s) in enumerate(self.free):
            if s >= n:
                if s == n:
                    self.free.pop(i)
                else:
                    self.free[i] = (o + n, s - n)
                return o
        return -1

    def release(self, o: int, n: int):
        self.free.append((o, self._round(n)))
        self.free.sort()
        merged = []
        for fo, fs in self.free:
            if merged and merged[-1][0] + merged[-1][1] == fo:
                merged[-1] = (merged[-1][0], merged[-1][1] + fs)
            else:
                merged.append((fo, fs))
        self.free = merged


@dataclass
class Trace:
    requests: list
    keep: list = field(default_factory=list)   # device pools and produced streams


def build_trace(torch, codec, rate=2000.0, duration=60.0, seed=0, pool_bytes=256 << 20,
                median_bytes=256 << 10, sigma=1.5, cap_bytes=64 << 20,
                device="cuda") -> Trace:
    """Requests over device-resident pools of 1-, 2- and 4-byte Markov codes.
    Decompress requests get streams produced beforehand, so every mode sees
    identical inputs."""
    t, comp, sizes, sym = synth.serving_trace(rate=rate, duration=duration, seed=seed,
                                              median_bytes=median_bytes, sigma=sigma,
                                              cap_bytes=cap_bytes)
    codes = synth.markov_codes(pool_bytes // 4, seed=seed)
    pools = {1: torch.from_numpy((codes % 256).astype(np.uint8)).to(device),
             2: torch.from_numpy(codes.astype(np.uint16).view(np.uint8)).to(device),
             4: torch.from_numpy(codes.view(np.uint8)).to(device)}
    params = {1: lz.Params(1, 4096, 128, 3), 2: lz.Params(2, 4096, 128, 3),
              4: lz.Params(4, 8192, 256, 2)}
    rng = np.random.default_rng(seed + 7)
    reqs, keep = [], list(pools.values())
    for i in range(len(t)):
        S = int(sym[i])
        n = int(min(sizes[i], pools[S].numel() - 16))
        n -= n % S
        off = int(rng.integers(0, (pools[S].numel() - n) // 16 + 1)) * 16
        view = pools[S][off:off + n]
        P = params[S]
        if comp[i]:
            reqs.append(Request(i, float(t[i]), True, view.data_ptr(), n, P,
                                lz.lz_compressed_bound(n, P), n, source=view))
        else:
            s = codec.compress_sync(view, P)
            keep.append(s)
            reqs.append(Request(i, float(t[i]), False, s.data_ptr(), s.numel(), P, n, n,
                                source=view))
    return Trace(reqs, keep)


def check_budget(trace: Trace, budget_bytes: int):
    """A request whose output space exceeds the whole budget could never be
    admitted: refuse the trace up front instead of waiting forever."""
    for r in trace.requests:
        if Arena._round(r.n_out_max) > budget_bytes:
            raise ValueError(f"request {r.rid} needs {r.n_out_max} output bytes, "
                             f"more than the {budget_bytes}-byte budget")


def _stats(trace: Trace, extra: dict) -> dict:
    lat = np.array([r.done - r.arrival for r in trace.requests]) * 1e3
    makespan = max(r.done for r in trace.requests) - min(r.arrival for r in trace.requests)
    nbytes = sum(r.n_orig for r in trace.requests)
    return {"requests": len(lat), "gbs": round(nbytes / makespan / 1e9, 4),
            "p50_ms": round(float(np.percentile(lat, 50)), 4),
            "p99_ms": round(float(np.percentile(lat, 99)), 4),
            "max_ms": round(float(lat.max()), 4), **extra}


def run_batched(torch, codec, trace: Trace, budget_bytes: int = 40 << 30, n_streams: int = 4,
                max_group: int = 1024, on_done=None) -> dict:
    """Continuous batching.  on_done(request, out_tensor_view, size) is called
    for every request once its group has finished, before its space is freed."""
    check_budget(trace, budget_bytes)
    arena_t = torch.empty(budget_bytes, dtype=torch.uint8, device="cuda")
    arena = Arena(budget_bytes)
    sizes_t = torch.zeros(len(trace.requests), dtype=torch.int64, device="cuda")
    base, nb = arena_t.data_ptr(), sizes_t.data_ptr()
    streams = [torch.cuda.Stream() for _ in range(n_streams)]
    busy = [None] * n_streams  # (event, group) per stream
    plans = [[None, None] for _ in range(n_streams)]  # compress, decompress batch per stream
    origin = torch.cuda.Event(enable_timing=True)
    pending = trace.requests
    queue, groups = [], []
    torch.cuda.synchronize()
    origin.record()
    t0 = time.perf_counter()
    nxt = 0
    while nxt < len(pending) or queue or any(b is not None for b in busy):
        now = time.perf_counter() - t0
        while nxt < len(pending) and pending[nxt].arrival <= now:
            queue.append(pending[nxt])
            nxt += 1
        for si, slot in enumerate(busy):
            if slot is not None and slot[0].query():
                ev, group = slot
                done = origin.elapsed_time(ev) / 1e3
                if on_done is not None:
                    sz = sizes_t[[r.rid for r in group]].cpu().numpy()
                for j, r in enumerate(group):
                    r.done = done
                    if on_done is not None:
                        on_done(r, arena_t[r.out_off:r.out_off + int(sz[j])], int(sz[j]))
                    arena.release(r.out_off, r.n_out_max)
                busy[si] = None
        free = [si for si, slot in enumerate(busy) if slot is None]
        if queue and free:
            group = []
            while queue and len(group) < max_group:
                o = arena.alloc(queue[0].n_out_max)
                if o < 0:
                    break  # budget full: wait for a group to finish
                queue[0].out_off = o
                group.append(queue.pop(0))
            if group:
                s = streams[free[0]]
                for d in (False, True):
                    its = [(r.d_in, r.n_in, base + r.out_off, r.n_out_max, nb + 8 * r.rid,
                            r.params) for r in group if r.compress != d]
                    if its:
                        b = plans[free[0]][d]
                        if b is None:
                            b = lz.lz_batch_create(codec.ctx, its, decompress=d,
                                                   stream=s.cuda_stream)
                            plans[free[0]][d] = b
                        else:
                            lz.lz_batch_update(codec.ctx, b, its, s.cuda_stream)
                        lz.lz_batch_run(codec.ctx, b, s.cuda_stream)
                ev = torch.cuda.Event(enable_timing=True)
                ev.record(s)
                busy[free[0]] = (ev, group)
                groups.append(len(group))
                continue
        if not queue and nxt < len(pending) and all(b is None for b in busy):
            wait = pending[nxt].arrival - (time.perf_counter() - t0)
            if wait > 0.0002:
                time.sleep(min(wait, 0.0005))
    torch.cuda.synchronize()
    for pair, s in zip(plans, streams):
        for b in pair:
            if b is not None:
                lz.lz_batch_destroy(b, s.cuda_stream)
    torch.cuda.synchronize()
    st = codec.sync()
    if st != lz.LZ_OK:
        raise lz.LzError(st, "serving (batched)")
    return _stats(trace, {"groups": len(groups),
                          "mean_group": round(float(np.mean(groups)), 2) if groups else 0.0,
                          "budget_bytes": budget_bytes})


def run_plain(torch, codec, trace: Trace, budget_bytes: int = 40 << 30, on_done=None) -> dict:
    """One plain launch per request, in arrival order, on one stream; output
    space from the same kind of budgeted arena."""
    check_budget(trace, budget_bytes)
    arena_t = torch.empty(budget_bytes, dtype=torch.uint8, device="cuda")
    arena = Arena(budget_bytes)
    sizes_t = torch.zeros(len(trace.requests), dtype=torch.int64, device="cuda")
    base, nb = arena_t.data_ptr(), sizes_t.data_ptr()
    stream = torch.cuda.current_stream()
    origin = torch.cuda.Event(enable_timing=True)
    inflight = []  # (event, request) in order
    torch.cuda.synchronize()
    origin.record()
    t0 = time.perf_counter()

    def retire(block: bool):
        while inflight and (block or inflight[0][0].query()):
            ev, r = inflight.pop(0)
            ev.synchronize()
            r.done = origin.elapsed_time(ev) / 1e3
            if on_done is not None:
                sz = int(sizes_t[r.rid].item())
                on_done(r, arena_t[r.out_off:r.out_off + sz], sz)
            arena.release(r.out_off, r.n_out_max)
            block = False

    for r in trace.requests:
        while time.perf_counter() - t0 < r.arrival:
            retire(False)
        o = arena.alloc(r.n_out_max)
        while o < 0:
            retire(True)
            o = arena.alloc(r.n_out_max)
        r.out_off = o
        if r.compress:
            lz.lz_compress(codec.ctx, r.d_in, r.n_in, r.params, base + o, r.n_out_max,
                           nb + 8 * r.rid, stream.cuda_stream)
        else:
            lz.lz_decompress(codec.ctx, r.d_in, r.n_in, base + o, r.n_out_max,
                             nb + 8 * r.rid, stream.cuda_stream)
        ev = torch.cuda.Event(enable_timing=True)
        ev.record(stream)
        inflight.append((ev, r))
        retire(False)
    while inflight:
        retire(True)
    st = codec.sync()
    if st != lz.LZ_OK:
        raise lz.LzError(st, "serving (plain)")
    return _stats(trace, {"budget_bytes": budget_bytes})
