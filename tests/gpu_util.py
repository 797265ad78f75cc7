"""Helpers shared by the GPU tests: run the CUDA path through the C ABI on
numpy inputs, and compare streams chunk by chunk with numpy (fast enough
for streams of hundreds of MiB)."""
from __future__ import annotations

import numpy as np


def codec():
    import torch

    from paper_2304_07342_gb300 import build, lz
    build.build()
    assert torch.cuda.is_available()
    return lz.Codec(0)


def to_dev(x: np.ndarray, offset: int = 0):
    """Device copy of x's bytes starting `offset` bytes into a fresh buffer
    (offset != 0 gives a misaligned device pointer)."""
    import torch
    b = np.array(x, copy=True).view(np.uint8).reshape(-1)
    buf = torch.empty(b.size + offset + 16, dtype=torch.uint8, device="cuda")
    view = buf[offset:offset + b.size]
    view.copy_(torch.from_numpy(b))
    return view


def gpu_compress(c, x: np.ndarray, P, in_offset: int = 0) -> np.ndarray:
    from paper_2304_07342_gb300 import lz
    d = to_dev(x, in_offset)
    out = c.compress_sync(d, lz.Params(*P.tuple()) if not isinstance(P, lz.Params) else P)
    return out.cpu().numpy()


def gpu_decompress(c, stream: np.ndarray, out_offset: int = 0) -> np.ndarray:
    import torch

    from paper_2304_07342_gb300 import lz
    d = to_dev(stream)
    n = lz.lz_decompressed_size(d.data_ptr(), d.numel())
    buf = torch.empty(n + out_offset + 16, dtype=torch.uint8, device="cuda")
    out = buf[out_offset:out_offset + n] if n else buf[out_offset:out_offset + 1]
    ob = torch.zeros(1, dtype=torch.int64, device="cuda")
    lz.lz_decompress(c.ctx, d.data_ptr(), d.numel(), out.data_ptr(), n, ob.data_ptr(),
                     torch.cuda.current_stream().cuda_stream)
    st = c.sync()
    if st != lz.LZ_OK:
        raise lz.LzError(st, "decompress")
    assert int(ob.item()) == n
    return out[:n].cpu().numpy()


def layout(stream: np.ndarray):
    """(n_chunks, table[nc,2], index, records_at, record_offsets[nc+1])."""
    s = np.asarray(stream, np.uint8)
    nc = int(s[20:24].view(np.uint32)[0])
    table = s[32:32 + 8 * nc].view(np.uint32).reshape(nc, 2).astype(np.int64)
    nidx = (nc + 63) // 64
    index = s[32 + 8 * nc:32 + 8 * nc + 8 * nidx].view(np.uint64).astype(np.int64)
    records_at = 32 + 8 * nc + 8 * nidx
    rec = (table[:, 0] + 7) // 8 + table[:, 1]
    offs = np.concatenate([[0], np.cumsum(rec)])
    return nc, table, index, records_at, offs


def record(stream: np.ndarray, c: int) -> bytes:
    nc, table, index, at, offs = layout(stream)
    return bytes(stream[at + offs[c]: at + offs[c + 1]])


def first_difference(a: np.ndarray, b: np.ndarray) -> str:
    """Human-readable location of the first difference of two streams."""
    if len(a) == len(b) and np.array_equal(a, b):
        return "identical"
    n = min(len(a), len(b))
    i = int(np.argmax(a[:n] != b[:n])) if np.any(a[:n] != b[:n]) else n
    msg = f"len {len(a)} vs {len(b)}; first differing byte {i}"
    try:
        nc, ta, _, at, oa = layout(a)
        _, tb, _, _, ob = layout(b)
        bad = np.nonzero(np.any(ta != tb, axis=1))[0]
        if bad.size:
            c = int(bad[0])
            msg += f"; chunk {c} table {ta[c].tolist()} vs {tb[c].tolist()}"
    except Exception as e:  # pragma: no cover - diagnostics only
        msg += f" ({e})"
    return msg
