"""Benchmark: chunked multi-byte LZSS compression/decompression on one GB300.

Default workload (one GPU): the large-field configuration -- a 512x512x256
float32 smooth field (sum of 16 Gaussians + N(0, 1e-4) noise, 256 MiB) and a
128 Mi-entry int32 sorted-index array (geometric(0.3) gaps, 512 MiB), both
compressed as 4-byte symbols with chunk 8192 B, window 256, min match 2,
max match 255.  One step = compress both arrays + decompress both streams
(the whole path); `value` is compression throughput in input GB/s, and the
line also carries decompression GB/s and the compression ratio.

Timing: W untimed warm-up steps, then K steps bracketed by a barrier and
torch.cuda.synchronize(), CUDA events on the launching stream; inputs (768
MiB) are larger than L2 (126 MB), so no extra flush is needed.  SM clocks
are sampled with nvidia-smi during the timed region.  Under torchrun each
rank compresses its own shard (independent data, weak scaling); there is no
data-path collective.

After the timed steps (not part of them) the line gets more sections on
the same GPU: `stream_version2` -- the same items as stream version 2
(stored chunks); `compressible` -- inputs with matches: the 1 MiB
quantization codes of the small configuration, 256 MiB of them and one
cell per symbol size of the 1 GiB symbol-size sweep, with compress and
decompress GB/s and HBM fractions; `paper_matcher` -- the paper's own matcher (section 3.3.2)
beside the exact one on 256 MiB of uint16 quantization codes; `huffman` --
the paper's use case (section 4.5), Huffman coding after LZSS, on the same
codes; `batched` --
10,000 uneven buffers (4 KiB-16 MiB, four
kinds, about 20 GB) compressed and decompressed by one persistent launch
under a CUDA graph vs one plain launch per buffer -- and `served` -- a
Poisson request stream (2000 requests/s for 60 s, the full trace; --served
sets the seconds) under continuous batching vs one launch per request, with
p50/p99 latency, then a load sweep to saturation.

`--impl reference` times the CPU oracle (the plain definition) on a bounded
sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("compress/decompress input GB/s + ratio vs HBM roofline; "
          "batched/served GB/s, p50/p99 latency")

# workload name -> list of (label, generator, params (S, C, W, m, M))
def _workloads():
    from paper_2304_07342_gb300 import synth
    return {
        "field+indices": [
            ("float32 field 512x512x256", lambda r: synth.gaussian_field(seed=r),
             (4, 8192, 256, 2, 255)),
            ("int32 sorted indices 128Mi", lambda r: synth.sorted_indices(128 << 20, seed=r),
             (4, 8192, 256, 2, 255)),
        ],
        "quant-small": [
            ("uint16 quant codes 1MiB", lambda r: synth.workload_small(seed=r),
             (2, 4096, 128, 3, 255)),
        ],
        # small cases for profiling: same kernels, a few GB at most
        "field-32MiB": [
            ("float32 field 64x512x256", lambda r: synth.gaussian_field((64, 512, 256), seed=r),
             (4, 8192, 256, 2, 255)),
        ],
        "field-256MiB": [
            ("float32 field 512x512x256", lambda r: synth.gaussian_field(seed=r),
             (4, 8192, 256, 2, 255)),
        ],
        "quant-256MiB": [
            ("uint16 quant codes 128Mi", lambda r: synth.quant_codes_laplace(128 << 20, seed=r),
             (2, 4096, 128, 3, 255)),
        ],
        "markov16-64MiB": [
            ("uint16 markov codes 32Mi", lambda r: synth.markov_codes(32 << 20, seed=r).astype(np.uint16),
             (2, 4096, 128, 3, 255)),
        ],
    }


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.samples = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(
                    ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                     "--format=csv,noheader,nounits"],
                    capture_output=True, text=True, timeout=5).stdout.strip()
                if out:
                    self.samples.append([f.strip() for f in out.split(",")])
            except Exception:
                pass
            self._stop.wait(0.05)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *exc):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for s in self.samples:
            for name, v in zip(names, s[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.samples)}


# The compression kernel's sources: a DRAM traffic figure from an ncu capture
# holds only while these are unchanged.
KERNEL_SOURCES = ("compress_impl.cuh", "compress_launch.cuh", "compress_s4.cu",
                  "glz_common.h", "glz_device.cuh")
PROFILE = os.path.join(ROOT, "profiles", "compress_kernel_field-256MiB.md")


# The decompression kernel's sources (for its ncu figures).
DECODE_SOURCES = ("decompress.cu", "glz_common.h", "glz_device.cuh", "launch_cache.cuh")


def kernel_sources_sha(names=KERNEL_SOURCES) -> str:
    import hashlib
    h = hashlib.sha256()
    for name in names:
        with open(os.path.join(ROOT, "paper_2304_07342_gb300", "csrc", name), "rb") as f:
            h.update(name.encode() + b"\0" + f.read())
    return h.hexdigest()


def _profiled_traffic():
    """DRAM bytes per launch of compress_kernel on the float field, from the
    committed ncu summary, if it was taken on the current kernel sources."""
    try:
        fields = dict(line.strip().strip("- `").split(": ", 1) for line in open(PROFILE)
                      if line.startswith("- `") and ": " in line)
        sha = fields.get("sources_sha256", "").strip("` ")
        if sha != kernel_sources_sha():
            return None, "kernel changed since the ncu capture"
        return int(fields["dram_bytes_per_launch"].strip("` ")), "ncu capture " + os.path.basename(PROFILE)
    except (OSError, KeyError, ValueError):
        return None, "no ncu capture"


def _profile_fields(name: str) -> dict:
    """The `- `key: value`` lines of a committed ncu summary."""
    try:
        return {k.strip(): v.strip("` ") for k, v in
                (line.strip().strip("- `").split(": ", 1) for line in
                 open(os.path.join(ROOT, "profiles", name))
                 if line.startswith("- `") and ": " in line)}
    except OSError:
        return {}


def _issue_roofline(kernel: str, profile: str, sources, ms: float, n_sym: int,
                    sms: int, mhz: float) -> dict:
    """Instruction-issue roofline of a kernel bound by issue, not by memory:
    warp instructions per launch (from the committed ncu summary, if it was
    taken on the current sources) over the live launch time, against one
    warp instruction per cycle per SM sub-partition (4 per SM) at the SM
    clock."""
    f = _profile_fields(profile)
    out = {"kernel": kernel, "bound": "issue", "unit": "G warp-inst/s",
           "peak": round(sms * 4 * mhz * 1e6 / 1e9, 1),
           "peak_source": f"{sms} SMs x 4 sub-partitions x {mhz:.0f} MHz"}
    if f.get("sources_sha256") != kernel_sources_sha(sources) or "warp_inst_per_launch" not in f:
        return {**out, "achieved": None, "frac": None,
                "note": "kernel changed since the ncu capture " + profile}
    inst = int(f["warp_inst_per_launch"])
    ach = inst / (ms * 1e-3) / 1e9
    return {**out, "achieved": round(ach, 1), "frac": round(ach / out["peak"], 4),
            "warp_inst_per_launch": inst, "warp_inst_per_symbol": round(inst / n_sym, 2),
            "issue_active_pct_ncu": float(f.get("issue_active_pct", "nan")),
            "source": "ncu capture " + profile}


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def run_gpu(args):
    import torch
    import torch.distributed as dist

    from paper_2304_07342_gb300 import build, lz
    rank, world, local = _dist()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if rank == 0:
        build.build()  # a no-op when the library is up to date
    if world > 1:
        dist.barrier()  # the other ranks load what rank 0 built
    codec = lz.Codec(local)
    stream = torch.cuda.current_stream()

    items = []
    for label, gen, P in _workloads()[args.workload]:
        x = gen(args.seed + rank)  # each rank: its own shard of independent data
        xb = np.ascontiguousarray(x).view(np.uint8).reshape(-1)
        p = lz.Params(*P)
        d_in = torch.from_numpy(xb).to(f"cuda:{local}")
        cap = lz.lz_compressed_bound(xb.size, p)
        d_out = torch.empty(cap, dtype=torch.uint8, device=d_in.device)
        d_nb = torch.zeros(1, dtype=torch.int64, device=d_in.device)
        d_dec = torch.empty_like(d_in)
        d_db = torch.zeros(1, dtype=torch.int64, device=d_in.device)
        items.append(dict(label=label, host=xb, p=p, d_in=d_in, d_out=d_out, d_nb=d_nb,
                          d_dec=d_dec, d_db=d_db, cap=cap))

    def compress_all():
        for it in items:
            lz.lz_compress(codec.ctx, it["d_in"].data_ptr(), it["d_in"].numel(), it["p"],
                           it["d_out"].data_ptr(), it["cap"], it["d_nb"].data_ptr(),
                           stream.cuda_stream)

    def decompress_all():
        for it in items:
            lz.lz_decompress(codec.ctx, it["d_out"].data_ptr(), it["size"],
                             it["d_dec"].data_ptr(), it["d_dec"].numel(),
                             it["d_db"].data_ptr(), stream.cuda_stream)

    # first pass: sizes and a correctness check of the round trip
    compress_all()
    if codec.sync() != lz.LZ_OK:
        raise RuntimeError("compress failed on the device")
    for it in items:
        it["size"] = int(it["d_nb"].item())
    decompress_all()
    if codec.sync() != lz.LZ_OK:
        raise RuntimeError("decompress failed on the device")
    for it in items:
        if not torch.equal(it["d_dec"], it["d_in"]):
            raise RuntimeError(f"round trip mismatch: {it['label']}")

    n_in = sum(it["d_in"].numel() for it in items)
    n_out = sum(it["size"] for it in items)

    for _ in range(args.warmup):
        compress_all()
        decompress_all()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    # per-kernel events for the roofline: first item's compress launch
    kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for s in range(args.steps):
            a, b, c = ev[s]
            a.record(stream)
            ka, kb = kev[s]
            for i, it in enumerate(items):
                if i == 0:
                    ka.record(stream)
                lz.lz_compress(codec.ctx, it["d_in"].data_ptr(), it["d_in"].numel(), it["p"],
                               it["d_out"].data_ptr(), it["cap"], it["d_nb"].data_ptr(),
                               stream.cuda_stream)
                if i == 0:
                    kb.record(stream)
            b.record(stream)
            decompress_all()
            c.record(stream)
        t1.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    if codec.sync() != lz.LZ_OK:
        raise RuntimeError("device error during the timed steps")

    total_ms = t0.elapsed_time(t1)
    comp_ms = sum(a.elapsed_time(b) for a, b, _ in ev) / args.steps
    dec_ms = sum(b.elapsed_time(c) for _, b, c in ev) / args.steps
    k_ms = sum(a.elapsed_time(b) for a, b in kev) / args.steps
    if world > 1:
        t = torch.tensor([total_ms, comp_ms, dec_ms], device=f"cuda:{local}")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms, comp_ms, dec_ms = t.tolist()

    # end to end through the public API with host buffers: pinned input ->
    # device, compress, compressed stream -> pinned host, every step
    e2e = _e2e(codec, items, stream, args)
    v2 = _version2(codec, items, stream) if args.version2 else None

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return None
    peaks = _peaks() or {}
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    it0 = items[0]
    k_bytes = it0["d_in"].numel() + it0["size"]  # read input + write stream
    achieved = k_bytes / (k_ms * 1e-3) / 1e9
    traffic, traffic_note = _profiled_traffic()
    if args.workload not in ("field+indices", "field-256MiB"):
        traffic, traffic_note = None, "ncu capture is of the float field workload"
    line = {
        "metric": METRIC,
        "value": round(n_in * world / (comp_ms * 1e-3) / 1e9, 3),
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(total_ms / args.steps, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": DTYPE,
        "data": "synthetic (seeded generators shaped like the paper's workloads)",
        "config": {"workload": args.workload,
                   "items": [dict(label=it["label"], bytes=int(it["d_in"].numel()),
                                  params=dict(zip("SCWmM", [it["p"].S, it["p"].C, it["p"].W,
                                                             it["p"].m, it["p"].M])))
                             for it in items],
                   "l2": "inputs larger than L2, no flush", "parallelism": f"replicas{world}"},
        "compress_gbs": round(n_in / (comp_ms * 1e-3) / 1e9, 3),
        "decompress_gbs": round(n_in / (dec_ms * 1e-3) / 1e9, 3),
        "ratio": round(n_in / n_out, 4),
        "compress_ms": round(comp_ms, 4),
        "decompress_ms": round(dec_ms, 4),
        "roofline": {"kernel": "compress_kernel (" + it0["label"] + ")",
                     "bound": "hbm", "achieved": round(achieved, 2),
                     "peak": hbm_peak, "unit": "GB/s", "frac": round(achieved / hbm_peak, 5),
                     "traffic": traffic, "traffic_source": traffic_note,
                     "algorithmic_bytes": k_bytes,
                     "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)"},
        "e2e": e2e,
        "gpu_launches": args.steps * len(items) * 2,
        "stream_version2": v2,
        "clocks": clk.summary(),
    }
    if args.cpu_baseline:
        line["cpu_baseline"] = _cpu_baseline(args, hosts=[it["host"] for it in items])
    if world > 1:
        dist.destroy_process_group()
        return line
    # the two patterns built on the same kernels, each against plain launches
    for it in items:
        for k in ("d_in", "d_out", "d_dec"):
            it[k] = None
    torch.cuda.empty_cache()
    if args.compressible:
        line["compressible"] = _compressible(torch, codec, args, hbm_peak,
                                             line["clocks"].get("sm_max_mhz"))
    if args.paper_matcher:
        line["paper_matcher"] = _paper_matcher(torch, codec, args)
    if args.huffman:
        line["huffman"] = _huffman(torch, codec, args)
    if args.sweep:
        line["sweep"] = _sweep(torch, codec, args)
    if args.batched:
        line["batched"] = _batched(torch, codec, args)
    if args.served > 0:
        line["served"] = _served(torch, codec, args, args.served)
    return line


def _time_codec(torch, codec, d, P, reps: int):
    """Compress and decompress device tensor d with P: (ratio, compress ms,
    decompress ms, stream bytes), CUDA events over `reps` calls each after a
    checked round trip."""
    from paper_2304_07342_gb300 import lz
    st = torch.cuda.current_stream()
    n = d.numel()
    out, nb = codec.compress(d, P)
    back, bb = codec.decompress(out, n_bytes=n)
    if codec.sync() != lz.LZ_OK:
        raise RuntimeError("compress/decompress failed on the device")
    size = int(nb.item())
    if not torch.equal(back, d):
        raise RuntimeError("round trip differs")
    for _ in range(2):
        codec.compress(d, P, out=out, out_bytes=nb)
        codec.decompress(out, n_bytes=n, out=back, out_bytes=bb, in_bytes=size)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    ev[0].record(st)
    for _ in range(reps):
        codec.compress(d, P, out=out, out_bytes=nb)
    ev[1].record(st)
    for _ in range(reps):
        codec.decompress(out, n_bytes=n, out=back, out_bytes=bb, in_bytes=size)
    ev[2].record(st)
    torch.cuda.synchronize()
    if codec.sync() != lz.LZ_OK:
        raise RuntimeError("timed compress/decompress failed on the device")
    return n / size, ev[0].elapsed_time(ev[1]) / reps, ev[1].elapsed_time(ev[2]) / reps, size


def _compressible(torch, codec, args, hbm_peak: float, sm_mhz=None):
    """Workloads with matches, where the parse and the decoder's pointer
    resolution do the work: the 1 MiB quantization codes of the small
    configuration (a single launch, bound by launch latency), 256 MiB of
    the same codes, and one chunk/window cell per symbol size of the
    symbol-size sweep (1 GiB of first-order Markov codes stored as uint8,
    uint16 and uint32, C = 4096, W = 128).  Per input: compress and
    decompress GB/s (input bytes), the ratio, and each kernel's HBM fraction
    counting the bytes it must move (input + stream).  For the 256 MiB of
    quantization codes, where both kernels are bound by instruction issue,
    also the issue roofline of each."""
    from paper_2304_07342_gb300 import lz, synth
    rows = []
    issue = {}

    def run(name, x, P, reps):
        d = torch.from_numpy(np.ascontiguousarray(x).view(np.uint8).reshape(-1)).cuda()
        ratio, c_ms, d_ms, size = _time_codec(torch, codec, d, P, reps)
        n = d.numel()
        if name == "uint16 quant codes 256 MiB":
            sms = torch.cuda.get_device_properties(d.device).multi_processor_count
            mhz = float(sm_mhz or 2070.0)
            issue["compress"] = _issue_roofline("compress_kernel", "compress_kernel_quant-256MiB.md",
                                                KERNEL_SOURCES, c_ms, n // P.S, sms, mhz)
            issue["decompress"] = _issue_roofline("decompress_kernel",
                                                  "decompress_kernel_quant-256MiB.md",
                                                  DECODE_SOURCES, d_ms, n // P.S, sms, mhz)
        moved = n + size
        rows.append({"input": name, "bytes": n, "params": dict(zip("SCWmM", (P.S, P.C, P.W, P.m, P.M))),
                     "ratio": round(ratio, 4),
                     "compress_gbs": round(n / (c_ms * 1e-3) / 1e9, 2),
                     "decompress_gbs": round(n / (d_ms * 1e-3) / 1e9, 2),
                     "compress_hbm_frac": round(moved / (c_ms * 1e-3) / 1e9 / hbm_peak, 4),
                     "decompress_hbm_frac": round(moved / (d_ms * 1e-3) / 1e9 / hbm_peak, 4)})
        del d
        torch.cuda.empty_cache()

    run("uint16 quant codes 1 MiB (small configuration)", synth.workload_small(seed=args.seed),
        lz.Params(2, 4096, 128, 3, 255), 50)
    run("uint16 quant codes 256 MiB", synth.quant_codes_laplace(128 << 20, seed=args.seed),
        lz.Params(2, 4096, 128, 3, 255), 5)
    chain = synth.markov_codes(1 << 30, seed=args.seed)
    for S in (1, 2, 4):
        x = ((chain % 256).astype(np.uint8) if S == 1 else
             chain[: (1 << 30) // S].astype({2: np.uint16, 4: np.uint32}[S]))
        run(f"markov u{8 * S} 1 GiB", x, lz.Params(S, 4096, 128, 2 if S == 4 else 3, 255), 3)
        del x
    del chain
    return {"workload": "quant codes (1 MiB, 256 MiB) and 1 GiB Markov codes at S = 1, 2, 4",
            "peak_gbs": hbm_peak, "points": rows, "issue_roofline_quant_256MiB": issue}


def _paper_matcher(torch, codec, args, n_sym: int = 128 << 20):
    """The paper's own matcher (section 3.3.2) beside the exact one, on 256
    MiB of uint16 quantization codes with the small workload's parameters
    (S=2, C=4096, W=128, m=3, M=255): compression GB/s and ratio of each."""
    from paper_2304_07342_gb300 import lz, synth
    x = synth.quant_codes_laplace(n_sym, seed=args.seed)
    d = torch.from_numpy(x.view(np.uint8)).cuda()
    P = lz.Params(2, 4096, 128, 3, 255)
    stream = torch.cuda.current_stream()
    out = {"workload": f"uint16 quant codes, {d.numel() >> 20} MiB", "params": "S=2 C=4096 W=128 m=3 M=255"}
    for name, mode in (("exact", lz.LZ_MATCH_EXACT), ("paper", lz.LZ_MATCH_PAPER)):
        buf, nb = codec.compress(d, P, match=mode)
        for _ in range(3):
            codec.compress(d, P, out=buf, out_bytes=nb, match=mode)
        if codec.sync() != lz.LZ_OK:
            raise RuntimeError("compress failed on the device")
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(5):
            codec.compress(d, P, out=buf, out_bytes=nb, match=mode)
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / 5
        out[name] = {"compress_gbs": round(d.numel() / (ms * 1e-3) / 1e9, 3),
                     "ratio": round(d.numel() / int(nb.item()), 4)}
        del buf
    del d
    torch.cuda.empty_cache()
    return out


def _huffman(torch, codec, args, n_sym: int = 128 << 20, reps: int = 5):
    """The paper's use case (section 4.5): Huffman coding after LZSS, on 256
    MiB of uint16 quantization codes.  Ratios of Huffman alone, LZSS alone
    and LZSS then Huffman; GB/s of the Huffman encoder (input bytes) and
    decoder (output bytes), CUDA events over `reps` calls."""
    from paper_2304_07342_gb300 import lz, synth
    x = synth.quant_codes_laplace(n_sym, seed=args.seed)
    d = torch.from_numpy(x.view(np.uint8)).cuda()
    st = torch.cuda.current_stream()
    n = d.numel()

    def huff(src, nbytes):
        cap = lz.lz_huff_bound(nbytes)
        out = torch.empty(cap, dtype=torch.uint8, device="cuda")
        nb = torch.zeros(1, dtype=torch.int64, device="cuda")
        lz.lz_huff_compress(codec.ctx, src.data_ptr(), nbytes, out.data_ptr(), cap, nb.data_ptr(),
                            st.cuda_stream)
        if codec.sync() != lz.LZ_OK:
            raise RuntimeError("huffman compress failed on the device")
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        for _ in range(reps):
            lz.lz_huff_compress(codec.ctx, src.data_ptr(), nbytes, out.data_ptr(), cap,
                                nb.data_ptr(), st.cuda_stream)
        b.record(st)
        torch.cuda.synchronize()
        return out, int(nb.item()), a.elapsed_time(b) / reps

    h1, h1_bytes, h1_ms = huff(d, n)
    back = torch.empty_like(d)
    nb = torch.zeros(1, dtype=torch.int64, device="cuda")
    lz.lz_huff_decompress(codec.ctx, h1.data_ptr(), h1_bytes, back.data_ptr(), n, nb.data_ptr(),
                          st.cuda_stream)
    if codec.sync() != lz.LZ_OK or not torch.equal(back, d):
        raise RuntimeError("huffman round trip failed")
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(st)
    for _ in range(reps):
        lz.lz_huff_decompress(codec.ctx, h1.data_ptr(), h1_bytes, back.data_ptr(), n,
                              nb.data_ptr(), st.cuda_stream)
    b.record(st)
    torch.cuda.synchronize()
    dec_ms = a.elapsed_time(b) / reps
    del h1, back
    s1 = codec.compress_sync(d, lz.Params(2, 4096, 128, 3, 255))
    h2, h2_bytes, h2_ms = huff(s1, s1.numel())
    out = {"workload": f"uint16 quant codes, {n >> 20} MiB; LZSS S=2 C=4096 W=128 m=3 M=255",
           "huffman_only": {"ratio": round(n / h1_bytes, 4),
                            "compress_gbs": round(n / (h1_ms * 1e-3) / 1e9, 2),
                            "decompress_gbs": round(n / (dec_ms * 1e-3) / 1e9, 2)},
           "lzss_only": {"ratio": round(n / s1.numel(), 4)},
           "lzss_then_huffman": {"ratio": round(n / h2_bytes, 4),
                                 "huffman_gbs_on_stream": round(s1.numel() / (h2_ms * 1e-3) / 1e9, 2)}}
    del d, s1, h2
    torch.cuda.empty_cache()
    return out


def _sweep(torch, codec, args, reps: int = 3):
    """The symbol-size sweep workload: 1 GiB of first-order Markov codes
    stored as uint8, uint16 and uint32 (S = 1, 2, 4), compressed with chunk
    2-16 KiB x window 64-512 symbols (m = 3 for S = 1, 2 and 2 for S = 4),
    and 1 GiB of uniform random bytes as the control.  Per point: compress
    and decompress GB/s (CUDA events, `reps` calls after a checked one) and
    the ratio."""
    from paper_2304_07342_gb300 import lz, synth
    st = torch.cuda.current_stream()
    chain = synth.markov_codes(1 << 30, seed=args.seed)
    rows = []
    inputs = [(f"markov u{8 * S}", S, ((chain % 256).astype(np.uint8) if S == 1 else
                                       chain[: (1 << 30) // S].astype({2: np.uint16, 4: np.uint32}[S])))
              for S in (1, 2, 4)]
    del chain
    inputs.append(("uniform bytes", 1, synth.uniform_bytes(1 << 30, seed=args.seed + 7)))
    for name, S, x in inputs:
        d = torch.from_numpy(np.ascontiguousarray(x).view(np.uint8)).cuda()
        n = d.numel()
        grid = [(C, W) for C in (2048, 4096, 8192, 16384) for W in (64, 128, 256, 512)]
        if name == "uniform bytes":
            grid = [(8192, 256)]
        for C, W in grid:
            P = lz.Params(S, C, W, 2 if S == 4 else 3, 255)
            out, nb = codec.compress(d, P)
            back, bb = codec.decompress(out, n_bytes=n)
            if codec.sync() != lz.LZ_OK:
                raise RuntimeError("sweep point failed on the device")
            size = int(nb.item())
            if not torch.equal(back, d):
                raise RuntimeError(f"sweep round trip differs: {name} C={C} W={W}")
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            ev[0].record(st)
            for _ in range(reps):
                codec.compress(d, P, out=out, out_bytes=nb)
            ev[1].record(st)
            for _ in range(reps):
                codec.decompress(out, n_bytes=n, out=back, out_bytes=bb, in_bytes=size)
            ev[2].record(st)
            torch.cuda.synchronize()
            c_ms = ev[0].elapsed_time(ev[1]) / reps
            d_ms = ev[1].elapsed_time(ev[2]) / reps
            rows.append({"input": name, "S": S, "C": C, "W": W, "ratio": round(n / size, 4),
                         "compress_gbs": round(n / (c_ms * 1e-3) / 1e9, 2),
                         "decompress_gbs": round(n / (d_ms * 1e-3) / 1e9, 2)})
            del out, back
        del d
        torch.cuda.empty_cache()
    return {"workload": "1 GiB Markov codes as uint8/uint16/uint32 + 1 GiB uniform bytes",
            "points": rows}


def _batched(torch, codec, args, n_buffers: int = 10_000):
    """Many uneven buffers: one persistent launch under a CUDA graph vs one
    plain launch per buffer (compress and decompress of every buffer)."""
    from paper_2304_07342_gb300 import batch
    t = time.perf_counter()
    tuning = []
    w = batch.build(torch, n_buffers=n_buffers, seed=args.seed, autotune_codec=codec,
                    report=tuning)
    build_s = time.perf_counter() - t
    r = batch.run(torch, codec, w, steps=3)
    r.update({"workload": f"{n_buffers} buffers, log-uniform 4 KiB-16 MiB, 4 kinds",
              "setup_seconds": round(build_s, 2), "autotune": tuning,
              "speedup_vs_per_buffer": round(r["compress_batched_gbs"] /
                                             r["compress_per_buffer_gbs"], 3)})
    del w
    torch.cuda.empty_cache()
    return r


def _served(torch, codec, args, seconds: float, budget: int = 40 * 10 ** 9):
    """Poisson request stream: continuous batching vs one plain launch per
    request, same trace, same HBM budget.  Then a load sweep: traces of
    about 6,000 requests at rising arrival rates, each run both ways, to
    show where one launch per request saturates."""
    from paper_2304_07342_gb300 import serve
    tr = serve.build_trace(torch, codec, rate=2000.0, duration=seconds, seed=args.seed)
    b = serve.run_batched(torch, codec, tr, budget_bytes=budget)
    torch.cuda.empty_cache()
    p = serve.run_plain(torch, codec, tr, budget_bytes=budget)
    tr = None
    torch.cuda.empty_cache()
    out = {"workload": f"2000 req/s Poisson for {seconds:g} s, 70% compress, "
                       "lognormal(256 KiB, 1.5) sizes capped at 64 MiB, S in {1,2,4}",
           "budget_bytes": budget, "batched": b, "plain": p}
    if args.served_sweep:
        sweep = []
        for rate in (8000.0, 32000.0, 128000.0, 512000.0):
            trs = serve.build_trace(torch, codec, rate=rate, duration=6000.0 / rate,
                                    seed=args.seed + 1)
            sb = serve.run_batched(torch, codec, trs, budget_bytes=budget)
            sp = serve.run_plain(torch, codec, trs, budget_bytes=budget)
            sweep.append({"rate": rate, "requests": sb["requests"], "batched": sb, "plain": sp})
            trs = None
            torch.cuda.empty_cache()
        out["load_sweep"] = sweep
    return out


def _version2(codec, items, stream, reps: int = 5):
    """The same items compressed as stream version 2 (a chunk that would not
    shrink is stored as it is) and decompressed again: GB/s and ratio,
    CUDA events over `reps` passes (after one checked pass)."""
    import torch

    from paper_2304_07342_gb300 import lz
    for it in items:
        lz.lz_compress_ex(codec.ctx, it["d_in"].data_ptr(), it["d_in"].numel(), it["p"],
                          it["d_out"].data_ptr(), it["cap"], it["d_nb"].data_ptr(),
                          stream.cuda_stream, version=2)
    if codec.sync() != lz.LZ_OK:
        raise RuntimeError("version-2 compress failed on the device")
    sizes = [int(it["d_nb"].item()) for it in items]
    for it, sz in zip(items, sizes):
        lz.lz_decompress(codec.ctx, it["d_out"].data_ptr(), sz, it["d_dec"].data_ptr(),
                         it["d_dec"].numel(), it["d_db"].data_ptr(), stream.cuda_stream)
    if codec.sync() != lz.LZ_OK:
        raise RuntimeError("version-2 decompress failed on the device")
    for it in items:
        if not torch.equal(it["d_dec"], it["d_in"]):
            raise RuntimeError(f"version-2 round trip mismatch: {it['label']}")
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    ev[0].record(stream)
    for _ in range(reps):
        for it in items:
            lz.lz_compress_ex(codec.ctx, it["d_in"].data_ptr(), it["d_in"].numel(), it["p"],
                              it["d_out"].data_ptr(), it["cap"], it["d_nb"].data_ptr(),
                              stream.cuda_stream, version=2)
    ev[1].record(stream)
    for _ in range(reps):
        for it, sz in zip(items, sizes):
            lz.lz_decompress(codec.ctx, it["d_out"].data_ptr(), sz, it["d_dec"].data_ptr(),
                             it["d_dec"].numel(), it["d_db"].data_ptr(), stream.cuda_stream)
    ev[2].record(stream)
    torch.cuda.synchronize()
    n_in = sum(it["d_in"].numel() for it in items)
    c_ms = ev[0].elapsed_time(ev[1]) / reps
    d_ms = ev[1].elapsed_time(ev[2]) / reps
    # restore the version-1 streams the rest of the run expects
    for it in items:
        lz.lz_compress(codec.ctx, it["d_in"].data_ptr(), it["d_in"].numel(), it["p"],
                       it["d_out"].data_ptr(), it["cap"], it["d_nb"].data_ptr(), stream.cuda_stream)
    torch.cuda.synchronize()
    return {"compress_gbs": round(n_in / (c_ms * 1e-3) / 1e9, 3),
            "decompress_gbs": round(n_in / (d_ms * 1e-3) / 1e9, 3),
            "ratio": round(n_in / sum(sizes), 5),
            "note": "same items, lz_compress_ex version 2 (stored chunks); not the headline"}


def _e2e(codec, items, stream, args):
    """End to end through the public API with host buffers: every step calls
    lz_compress_host once per item -- pinned host input in, pinned host
    stream out, copies inside the call (it overlaps the copy-in,
    compression and copy-out of successive pieces of the item).  The call is
    synchronous, so the step is timed on the host clock, after the bench's
    warm-up count of untimed steps (at least 3)."""
    import torch

    from paper_2304_07342_gb300 import lz
    pinned_in = [torch.from_numpy(it["host"]).pin_memory() for it in items]
    pinned_out = [torch.empty(it["cap"], dtype=torch.uint8).pin_memory() for it in items]
    steps = max(5, min(args.steps, 20))

    def one():
        sizes = []
        for it, hi, ho in zip(items, pinned_in, pinned_out):
            sizes.append(lz.lz_compress_host(codec.ctx, hi.data_ptr(), hi.numel(), it["p"],
                                             ho.data_ptr(), ho.numel(), stream.cuda_stream))
        return sizes

    rank, world, local = _dist()
    sizes = one()
    for _ in range(max(args.warmup, 3) - 1):
        one()
    for it, ho, sz in zip(items, pinned_out, sizes):
        if sz != it["size"] or not torch.equal(ho[:sz], it["d_out"][:sz].cpu()):
            raise RuntimeError("end-to-end stream differs from the device call's")
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    per_step = []
    for _ in range(steps):
        t = time.perf_counter()
        one()
        per_step.append((time.perf_counter() - t) * 1e3)
    # the median step: an occasional step stalls on the host (about 2x, one
    # in ten); the mean is reported beside it
    ms = statistics.median(per_step)
    mean_ms = sum(per_step) / len(per_step)
    if world > 1:  # every rank's bytes over the slowest rank's time
        import torch.distributed as dist
        tt = torch.tensor([ms], device=f"cuda:{local}")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms = tt.item()
    n_in = sum(it["d_in"].numel() for it in items)
    n_out = sum(it["size"] for it in items)
    streams = [stream, torch.cuda.Stream()]
    link = _link_bandwidth(items, pinned_in, pinned_out, streams)
    if world > 1:  # the whole job's bytes
        tt = torch.tensor([n_in, n_out], dtype=torch.float64, device=f"cuda:{local}")
        dist.all_reduce(tt, op=dist.ReduceOp.SUM)
        n_in, n_out = (int(v) for v in tt.tolist())
    return {"value": round(n_in / (ms * 1e-3) / 1e9, 3), "unit": UNIT,
            "h2d_bytes_per_step": int(n_in),
            "d2h_bytes_per_step": int(n_out),
            "steps": steps, "median_ms": round(ms, 3), "mean_ms": round(mean_ms, 3),
            "min_ms": round(min(per_step), 3), "max_ms": round(max(per_step), 3),
            "mean_value": round(n_in / (mean_ms * 1e-3) / 1e9, 3),
            "link": link,
            "note": "lz_compress_host (C ABI, pinned host buffers in and out): the input "
                    "copied in in pieces of whole index superblocks, each piece compressed "
                    "as it arrives and its records copied out as soon as it is done, both "
                    "directions of the host link busy at once; host clock around each "
                    "synchronous step, median of the steps"}


def _link_bandwidth(items, pinned_in, pinned_out, streams):
    """Host-link bandwidth on the end-to-end pass's own pinned buffers:
    all inputs host to device, all streams device to host, and both at once
    on two streams (CUDA events, best of 3 after one warm-up)."""
    import torch

    n_in = sum(it["d_in"].numel() for it in items)
    n_out = sum(it["size"] for it in items)
    s_in, s_out = streams[0], (streams[1] if len(streams) > 1 else torch.cuda.Stream())

    def h2d():
        for it, hi in zip(items, pinned_in):
            with torch.cuda.stream(s_in):
                it["d_in"].copy_(hi, non_blocking=True)

    def d2h():
        for it, ho in zip(items, pinned_out):
            with torch.cuda.stream(s_out):
                ho[: it["size"]].copy_(it["d_out"][: it["size"]], non_blocking=True)

    def timed(fn):
        best = float("inf")
        for rep in range(4):
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(s_in)
            s_out.wait_stream(s_in)
            fn()
            s_in.wait_stream(s_out)
            b.record(s_in)
            torch.cuda.synchronize()
            if rep:
                best = min(best, a.elapsed_time(b))
        return best

    t_in, t_out = timed(h2d), timed(d2h)
    t_both = timed(lambda: (h2d(), d2h()))
    return {"h2d_gbs": round(n_in / (t_in * 1e-3) / 1e9, 1),
            "d2h_gbs": round(n_out / (t_out * 1e-3) / 1e9, 1),
            "both_gbs": round((n_in + n_out) / (t_both * 1e-3) / 1e9, 1),
            "note": "pinned copies of the same buffers, no compression"}


UNIT = "GB/s (input bytes compressed per second)"
DTYPE = "u8/u32 symbols (integer/byte path, lossless)"


def _cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def _oracle_pool_rate(items, threads: int) -> float:
    """Bytes per second of the oracle compressing `items` -- (bytes, Params,
    chunk) -- on `threads` host threads.  Each item is cut into pieces of
    whole index superblocks (64 chunks); chunks are independent (section
    3.3.1), so the pieces are the same work as the whole.  The oracle's
    ctypes calls release the interpreter lock, so the threads run on
    separate cores."""
    from concurrent.futures import ThreadPoolExecutor

    import oracle
    pieces = []
    for x, p, C in items:
        step = max(64 * C, (x.size // max(1, 4 * threads)) // (64 * C) * (64 * C))
        pieces += [(x[o:o + step], p) for o in range(0, x.size, step)]
    t = time.perf_counter()
    with ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(lambda a: oracle.compress(*a), pieces))
    return sum(x.size for x, _, _ in items) / (time.perf_counter() - t)


def _cpu_sample(args, hosts, budget_s: float, threads: int):
    """Leading whole chunks of each item of the workload, sized so that the
    oracle on `threads` threads takes about budget_s seconds in all."""
    import oracle
    oracle.build()
    wl = _workloads()[args.workload]
    probe = []
    for i, (label, gen, P) in enumerate(wl):
        x = hosts[i] if hosts is not None else gen(args.seed)
        x = np.ascontiguousarray(x).view(np.uint8).reshape(-1)
        probe.append((label, x, oracle.Params(*P), P[1]))
    # rate from a small sample (64 chunks per thread of every item)
    small = [(x[: min(x.size, 64 * C * threads)], p, C) for _, x, p, C in probe]
    rate = _oracle_pool_rate(small, threads)
    per_item = max(64 * max(C for *_, C in probe), int(rate * budget_s / len(probe)))
    sample = []
    for label, x, p, C in probe:
        n = min(x.size, max(C, per_item - per_item % (64 * C)))
        sample.append((label, x[:n], p, C))
    return sample


def _cpu_baseline(args, budget_s: float = 15.0, hosts=None):
    """The oracle as it stands on the host cores, on a bounded sample (leading
    whole chunks of each item) of the same workload: all cores (the value)
    and one core."""
    threads = os.cpu_count() or 1
    sample = _cpu_sample(args, hosts, budget_s, threads)
    items = [(x, p, C) for _, x, p, C in sample]
    value = _oracle_pool_rate(items, threads)
    one = [(x[: max(C, x.size // threads // C * C)], p, C) for x, p, C in items]
    single = _oracle_pool_rate(one, 1)
    return {"value": round(value / 1e9, 6), "unit": UNIT, "cores": threads, "kind": "oracle",
            "single_core_value": round(single / 1e9, 6), "cpu_model": _cpu_model(),
            "sample": "; ".join(f"{label}: first {x.size} bytes" for label, x, _, _ in sample) +
                      f" (one core: the first 1/{threads} of each)"}


def run_reference(args):
    """The reference arm: the oracle as it stands on all host cores (one
    thread per core over superblock-aligned pieces), W warm-up and K timed
    steps, each step compressing the same bounded sample (the leading whole
    chunks of every item of the workload), sized so that the whole run takes
    about a minute."""
    rank, world, local = _dist()
    if rank != 0:
        return None
    threads = os.cpu_count() or 1
    step_s = min(5.0, max(0.2, 60.0 / max(1, args.steps + args.warmup)))
    sample = _cpu_sample(args, None, step_s, threads)
    items = [(x, p, C) for _, x, p, C in sample]
    for _ in range(max(1, args.warmup)):
        _oracle_pool_rate(items, threads)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        _oracle_pool_rate(items, threads)
    dt = time.perf_counter() - t0
    step_bytes = sum(x.size for x, _, _ in items)
    value = round(args.steps * step_bytes / dt / 1e9, 6)
    cb = {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
          "cpu_model": _cpu_model(),
          "sample": "; ".join(f"{label}: first {x.size} bytes" for label, x, _, _ in sample) +
                    f" (every step; {args.steps} timed steps of {dt / max(1, args.steps):.3f} s)"}
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(dt / max(1, args.steps) * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPE, "data": "synthetic (seeded generators shaped like the paper's workloads)",
        "config": {"workload": args.workload},
        "cpu_baseline": cb,
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="field+indices")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--no-version2", dest="version2", action="store_false",
                    help="skip the stream-version-2 (stored chunks) pass")
    ap.add_argument("--sweep", action="store_true",
                    help="also run the 1 GiB symbol-size sweep (S x chunk x window)")
    ap.add_argument("--no-huffman", dest="huffman", action="store_false",
                    help="skip the LZSS-then-Huffman use case")
    ap.add_argument("--no-compressible", dest="compressible", action="store_false",
                    help="skip the compressible workloads (small configuration, quant codes, "
                         "one sweep cell per symbol size)")
    ap.add_argument("--no-paper-matcher", dest="paper_matcher", action="store_false",
                    help="skip the exact-vs-paper matcher comparison")
    ap.add_argument("--no-batched", dest="batched", action="store_false",
                    help="skip the 10,000-buffer batched comparison")
    ap.add_argument("--served", type=float, default=60.0,
                    help="seconds of the serving trace (the full trace is 60; 0 skips it)")
    ap.add_argument("--no-served-sweep", dest="served_sweep", action="store_false",
                    help="skip the serving load sweep")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl != "reference":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    line = run_reference(args) if args.impl == "reference" else run_gpu(args)
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
