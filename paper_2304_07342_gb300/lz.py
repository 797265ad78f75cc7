"""Thin Python binding of the C ABI in ``include/lz.h`` (ctypes).

The functions named ``lz_*`` mirror the C entry points one to one and take
raw device pointers (ints) and a ``cudaStream_t`` handle (int, 0 = legacy
default stream).  :class:`Codec` adds torch-tensor marshalling on top.  All
compression work happens in the CUDA kernels of ``liblz.so``; there is no
CPU path, and every call raises :class:`LzError` if the library is missing.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblz.so")

LZ_OK = 0
LZ_ERR_INVALID_ARG = 1
LZ_ERR_BUFFER_TOO_SMALL = 2
LZ_ERR_CORRUPT = 3
LZ_ERR_NOMEM = 4
LZ_ERR_CUDA = 5
LZ_ERR_TIMEOUT = 6
LZ_ERR_INTERNAL = 7

LZ_MATCH_EXACT = 0  # longest match, nearest offset on ties (the definition)
LZ_MATCH_PAPER = 1  # the paper's forward scan (section 3.3.2)
LZ_MATCH_OVERLAP = 2  # exact, matches may overlap their output (stream version 2)

_NAMES = {0: "LZ_OK", 1: "LZ_ERR_INVALID_ARG", 2: "LZ_ERR_BUFFER_TOO_SMALL",
          3: "LZ_ERR_CORRUPT", 4: "LZ_ERR_NOMEM", 5: "LZ_ERR_CUDA",
          6: "LZ_ERR_TIMEOUT", 7: "LZ_ERR_INTERNAL"}

# every symbol include/lz.h declares
EXPORTS = ("lz_create", "lz_destroy", "lz_status_string", "lz_check_params",
           "lz_compressed_bound", "lz_compress", "lz_compress_ex", "lz_compress_host", "lz_decompressed_size",
           "lz_decompress", "lz_sync", "lz_compress_noalloc", "lz_batch_create",
           "lz_batch_run", "lz_batch_update", "lz_batch_destroy", "lz_autotune", "lz_autotune_ex", "lz_stitch", "lz_batch_create_ex",
           "lz_select_params", "lz_huff_bound", "lz_huff_compress",
           "lz_huff_decompressed_size", "lz_huff_decompress", "lz_set_test_hooks")


class LzError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        super().__init__(f"{what}: {_NAMES.get(status, status)}")
        self.status = status


class lz_params(ctypes.Structure):
    _fields_ = [("symbol_bytes", ctypes.c_uint32), ("chunk_bytes", ctypes.c_uint32),
                ("window", ctypes.c_uint32), ("min_match", ctypes.c_uint32),
                ("max_match", ctypes.c_uint32)]


class lz_options(ctypes.Structure):
    _fields_ = [("match", ctypes.c_uint32), ("version", ctypes.c_uint32),
                ("warps_per_block", ctypes.c_uint32)]


class lz_test_hooks(ctypes.Structure):
    _fields_ = [("spin_limit", ctypes.c_uint32), ("first_chunk", ctypes.c_uint32),
                ("fail_alloc", ctypes.c_uint32)]


class lz_tune_trial(ctypes.Structure):
    _fields_ = [("params", lz_params), ("warps_per_block", ctypes.c_uint32),
                ("seconds", ctypes.c_double), ("ratio", ctypes.c_double)]


class lz_batch_item(ctypes.Structure):
    _fields_ = [("d_in", ctypes.c_void_p), ("in_bytes", ctypes.c_uint64),
                ("d_out", ctypes.c_void_p), ("out_cap", ctypes.c_uint64),
                ("d_out_bytes", ctypes.c_void_p), ("params", lz_params)]


@dataclass(frozen=True)
class Params:
    """S symbol bytes, C chunk bytes, W window (symbols), m min match, M max match."""
    S: int
    C: int
    W: int
    m: int
    M: int = 255

    def c(self) -> lz_params:
        return lz_params(self.S, self.C, self.W, self.m, self.M)


_lib = None


def load(path: str = LIB_PATH):
    """Load ``liblz.so`` (raises LzError if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise LzError(LZ_ERR_CUDA, f"CUDA library not built ({path}); run "
                      "paper_2304_07342_gb300.build.build()")
    lib = ctypes.CDLL(path)
    vp, u64, i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int
    pp = ctypes.POINTER(lz_params)
    lib.lz_create.argtypes = [ctypes.POINTER(vp), i32]
    lib.lz_create.restype = i32
    lib.lz_destroy.argtypes = [vp]
    lib.lz_destroy.restype = None
    lib.lz_status_string.argtypes = [i32]
    lib.lz_status_string.restype = ctypes.c_char_p
    lib.lz_check_params.argtypes = [pp]
    lib.lz_check_params.restype = i32
    lib.lz_compressed_bound.argtypes = [u64, pp]
    lib.lz_compressed_bound.restype = u64
    lib.lz_compress.argtypes = [vp, vp, u64, pp, vp, u64, vp, vp]
    lib.lz_compress.restype = i32
    lib.lz_compress_ex.argtypes = [vp, vp, u64, pp, ctypes.POINTER(lz_options), vp, u64, vp, vp]
    lib.lz_compress_ex.restype = i32
    lib.lz_compress_host.argtypes = [vp, vp, u64, pp, vp, u64, ctypes.POINTER(u64), vp]
    lib.lz_compress_host.restype = i32
    lib.lz_decompressed_size.argtypes = [vp, u64, ctypes.POINTER(u64), vp]
    lib.lz_decompressed_size.restype = i32
    lib.lz_decompress.argtypes = [vp, vp, u64, vp, u64, vp, vp]
    lib.lz_decompress.restype = i32
    lib.lz_sync.argtypes = [vp, vp]
    lib.lz_sync.restype = i32
    lib.lz_compress_noalloc.argtypes = [vp, u64, pp, vp, u64, vp, vp]
    lib.lz_compress_noalloc.restype = i32
    lib.lz_batch_create.argtypes = [vp, ctypes.POINTER(lz_batch_item), ctypes.c_uint32, i32,
                                    vp, ctypes.POINTER(vp)]
    lib.lz_batch_create.restype = i32
    lib.lz_batch_create_ex.argtypes = [vp, ctypes.POINTER(lz_batch_item), ctypes.c_uint32, i32,
                                       ctypes.POINTER(lz_options), vp, ctypes.POINTER(vp)]
    lib.lz_batch_create_ex.restype = i32
    lib.lz_batch_update.argtypes = [vp, vp, ctypes.POINTER(lz_batch_item), ctypes.c_uint32, vp]
    lib.lz_batch_update.restype = i32
    lib.lz_batch_run.argtypes = [vp, vp, vp]
    lib.lz_batch_run.restype = i32
    lib.lz_batch_destroy.argtypes = [vp, vp]
    lib.lz_batch_destroy.restype = None
    lib.lz_autotune.argtypes = [vp, vp, u64, ctypes.c_uint32, pp]
    lib.lz_autotune.restype = i32
    lib.lz_autotune_ex.argtypes = [vp, vp, u64, ctypes.c_uint32, pp, ctypes.POINTER(ctypes.c_uint32),
                                   ctypes.POINTER(lz_tune_trial), ctypes.c_uint32,
                                   ctypes.POINTER(ctypes.c_uint32)]
    lib.lz_autotune_ex.restype = i32
    u32 = ctypes.c_uint32
    lib.lz_select_params.argtypes = [vp, vp, u64, u32, u32, u32, pp, vp]
    lib.lz_select_params.restype = i32
    lib.lz_huff_bound.argtypes = [u64]
    lib.lz_huff_bound.restype = u64
    lib.lz_huff_compress.argtypes = [vp, vp, u64, vp, u64, vp, vp]
    lib.lz_huff_compress.restype = i32
    lib.lz_huff_decompressed_size.argtypes = [vp, u64, ctypes.POINTER(u64), vp]
    lib.lz_huff_decompressed_size.restype = i32
    lib.lz_huff_decompress.argtypes = [vp, vp, u64, vp, u64, vp, vp]
    lib.lz_huff_decompress.restype = i32
    lib.lz_set_test_hooks.argtypes = [vp, ctypes.POINTER(lz_test_hooks)]
    lib.lz_set_test_hooks.restype = i32
    lib.lz_stitch.argtypes = [vp, vp, u64, u64, u64, u64, u64, u64, vp, u64, vp]
    lib.lz_stitch.restype = i32
    _lib = lib
    return lib


def _check(status: int, what: str):
    if status != LZ_OK:
        raise LzError(status, what)


# --- the C entry points, same names -------------------------------------------

def lz_create(device: int = 0) -> int:
    h = ctypes.c_void_p()
    _check(load().lz_create(ctypes.byref(h), device), "lz_create")
    return h.value


def lz_destroy(ctx: int) -> None:
    load().lz_destroy(ctx)


def lz_status_string(status: int) -> str:
    return load().lz_status_string(status).decode()


def lz_check_params(p: Params) -> int:
    return load().lz_check_params(ctypes.byref(p.c()))


def lz_compressed_bound(n_bytes: int, p: Params) -> int:
    return int(load().lz_compressed_bound(n_bytes, ctypes.byref(p.c())))


def lz_compress(ctx: int, d_in: int, n_bytes: int, p: Params, d_out: int,
                out_cap: int, d_out_bytes: int, stream: int = 0) -> None:
    _check(load().lz_compress(ctx, d_in, n_bytes, ctypes.byref(p.c()), d_out,
                              out_cap, d_out_bytes, stream), "lz_compress")


def lz_compress_ex(ctx: int, d_in: int, n_bytes: int, p: Params, d_out: int, out_cap: int,
                   d_out_bytes: int, stream: int = 0, match: int = 0, version: int = 1,
                   warps_per_block: int = 0) -> None:
    opt = lz_options(match, version, warps_per_block)
    _check(load().lz_compress_ex(ctx, d_in, n_bytes, ctypes.byref(p.c()), ctypes.byref(opt),
                                 d_out, out_cap, d_out_bytes, stream), "lz_compress_ex")


def lz_compress_host(ctx: int, h_in: int, n_bytes: int, p: Params, h_out: int, out_cap: int,
                     stream: int = 0) -> int:
    """Host buffer in, host buffer out (synchronous); returns the stream size."""
    nb = ctypes.c_uint64()
    _check(load().lz_compress_host(ctx, h_in, n_bytes, ctypes.byref(p.c()), h_out, out_cap,
                                   ctypes.byref(nb), stream), "lz_compress_host")
    return nb.value


def lz_decompressed_size(d_in: int, in_bytes: int, stream: int = 0) -> int:
    n = ctypes.c_uint64()
    _check(load().lz_decompressed_size(d_in, in_bytes, ctypes.byref(n), stream),
           "lz_decompressed_size")
    return n.value


def lz_decompress(ctx: int, d_in: int, in_bytes: int, d_out: int, out_cap: int,
                  d_out_bytes: int, stream: int = 0) -> None:
    _check(load().lz_decompress(ctx, d_in, in_bytes, d_out, out_cap,
                                d_out_bytes, stream), "lz_decompress")


def lz_stitch(ctx: int, d_shard: int, shard_bytes: int, shard_chunks: int, chunk_base: int,
              total_chunks: int, total_bytes: int, record_base: int, d_out: int, out_cap: int,
              stream: int = 0) -> None:
    """Place one shard stream inside the whole-input stream at d_out."""
    _check(load().lz_stitch(ctx, d_shard, shard_bytes, shard_chunks, chunk_base, total_chunks,
                            total_bytes, record_base, d_out, out_cap, stream), "lz_stitch")


def lz_compress_noalloc(d_in: int, n_bytes: int, p: Params, d_out: int, out_cap: int,
                        d_out_bytes: int, stream: int = 0) -> None:
    """Compression without any device allocation (fixed in-library scratch,
    at most 65536 chunks per call); the outcome is in *d_out_bytes."""
    _check(load().lz_compress_noalloc(d_in, n_bytes, ctypes.byref(p.c()), d_out, out_cap,
                                      d_out_bytes, stream), "lz_compress_noalloc")


def lz_batch_create(ctx: int, items, decompress: bool = False, stream: int = 0,
                    match: int = 0, version: int = 1) -> int:
    """Plan a batch; `items` is a list of (d_in, in_bytes, d_out, out_cap,
    d_out_bytes, Params-or-None) tuples of raw device pointers (for a
    decompression item, Params states the stream's parameters and out_cap
    its exact size, so that its header need not be read).  `match` and
    `version` apply to every item of a compression batch (lz_batch_create_ex)."""
    arr = _items(items)
    h = ctypes.c_void_p()
    if match == 0 and version == 1:
        _check(load().lz_batch_create(ctx, arr, len(items), 1 if decompress else 0, stream,
                                      ctypes.byref(h)), "lz_batch_create")
    else:
        opt = lz_options(match, version, 0)
        _check(load().lz_batch_create_ex(ctx, arr, len(items), 1 if decompress else 0,
                                         ctypes.byref(opt), stream, ctypes.byref(h)),
               "lz_batch_create_ex")
    return h.value


def _items(items):
    arr = (lz_batch_item * max(1, len(items)))()
    for i, (din, nin, dout, cap, dnb, p) in enumerate(items):
        arr[i] = lz_batch_item(din, nin, dout, cap, dnb,
                               p.c() if p is not None else lz_params(0, 0, 0, 0, 0))
    return arr


def lz_batch_update(ctx: int, batch: int, items, stream: int = 0) -> None:
    """Re-plan `batch` for new items (same direction and options), reusing
    its device memory where it is large enough."""
    _check(load().lz_batch_update(ctx, batch, _items(items), len(items), stream),
           "lz_batch_update")


def lz_batch_run(ctx: int, batch: int, stream: int = 0) -> None:
    _check(load().lz_batch_run(ctx, batch, stream), "lz_batch_run")


def lz_batch_destroy(batch: int, stream: int = 0) -> None:
    load().lz_batch_destroy(batch, stream)


def lz_autotune(ctx: int, d_sample: int, sample_bytes: int, symbol_bytes: int) -> Params:
    out = lz_params()
    _check(load().lz_autotune(ctx, d_sample, sample_bytes, symbol_bytes, ctypes.byref(out)),
           "lz_autotune")
    return Params(out.symbol_bytes, out.chunk_bytes, out.window, out.min_match, out.max_match)


def lz_autotune_ex(ctx: int, d_sample: int, sample_bytes: int, symbol_bytes: int):
    """(Params, warps_per_block, trials): the choice of lz_autotune, the
    launch shape for it, and every trial as a dict."""
    out = lz_params()
    wpb = ctypes.c_uint32()
    arr = (lz_tune_trial * 64)()
    n = ctypes.c_uint32()
    _check(load().lz_autotune_ex(ctx, d_sample, sample_bytes, symbol_bytes, ctypes.byref(out),
                                 ctypes.byref(wpb), arr, 64, ctypes.byref(n)), "lz_autotune_ex")
    trials = [dict(S=t.params.symbol_bytes, C=t.params.chunk_bytes, W=t.params.window,
                   m=t.params.min_match, M=t.params.max_match, warps_per_block=t.warps_per_block,
                   ms=round(t.seconds * 1e3, 4), ratio=round(t.ratio, 4))
              for t in arr[: min(64, n.value)]]
    return (Params(out.symbol_bytes, out.chunk_bytes, out.window, out.min_match, out.max_match),
            wpb.value, trials)


def lz_select_params(ctx: int, d_sample: int, sample_bytes: int, dtype_bytes: int,
                     level: int = 3, chunk_bytes: int = 4096, stream: int = 0) -> Params:
    """Section 3.2.3 policy: multi-byte matching unless the sample's ratio
    with it is below 1.5 (then single-byte); windows by level 1-4."""
    out = lz_params()
    _check(load().lz_select_params(ctx, d_sample, sample_bytes, dtype_bytes, level, chunk_bytes,
                                   ctypes.byref(out), stream), "lz_select_params")
    return Params(out.symbol_bytes, out.chunk_bytes, out.window, out.min_match, out.max_match)


def lz_huff_bound(n_bytes: int) -> int:
    return int(load().lz_huff_bound(n_bytes))


def lz_huff_compress(ctx: int, d_in: int, n_bytes: int, d_out: int, out_cap: int,
                     d_out_bytes: int, stream: int = 0) -> None:
    _check(load().lz_huff_compress(ctx, d_in, n_bytes, d_out, out_cap, d_out_bytes, stream),
           "lz_huff_compress")


def lz_huff_decompressed_size(d_in: int, in_bytes: int, stream: int = 0) -> int:
    n = ctypes.c_uint64()
    _check(load().lz_huff_decompressed_size(d_in, in_bytes, ctypes.byref(n), stream),
           "lz_huff_decompressed_size")
    return n.value


def lz_huff_decompress(ctx: int, d_in: int, in_bytes: int, d_out: int, out_cap: int,
                       d_out_bytes: int, stream: int = 0) -> None:
    _check(load().lz_huff_decompress(ctx, d_in, in_bytes, d_out, out_cap, d_out_bytes, stream),
           "lz_huff_decompress")


def lz_set_test_hooks(ctx: int, spin_limit: int = 0, first_chunk: int = 0,
                      fail_alloc: int = 0) -> None:
    """Test hooks of a context (all zero: normal operation); see lz.h."""
    h = lz_test_hooks(spin_limit, first_chunk, fail_alloc)
    _check(load().lz_set_test_hooks(ctx, ctypes.byref(h)), "lz_set_test_hooks")


def lz_sync(ctx: int, stream: int = 0) -> int:
    """Return (and clear) the sticky device status; does not raise."""
    return load().lz_sync(ctx, stream)


# --- torch marshalling -----------------------------------------------------------

class Codec:
    """One context on one device; tensors in, tensors out.

    ``compress``/``decompress`` enqueue on the current torch stream and return
    the output buffer plus a device int64 holding the produced size;
    ``*_sync`` variants synchronise, check the sticky status and trim.
    """

    def __init__(self, device: int = 0):
        import torch
        self.torch = torch
        self.device = device
        torch.cuda.set_device(device)
        self.ctx = lz_create(device)

    def close(self):
        if self.ctx:
            lz_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _stream(self, stream):
        s = stream if stream is not None else self.torch.cuda.current_stream(self.device)
        return s.cuda_stream

    def _bytes_of(self, x, stream):
        """x as a flat contiguous uint8 tensor.  A contiguous copy made here
        is marked as used by `stream`, so that its memory is not handed out
        again before the work queued there has read it."""
        xb = x.contiguous().view(-1).view(self.torch.uint8)
        if stream is not None and x.numel() and xb.data_ptr() != x.data_ptr():
            xb.record_stream(stream)
        return xb

    def compress(self, x, p: Params, out=None, out_bytes=None, stream=None,
                 match: int = LZ_MATCH_EXACT, version: int = 1):
        torch = self.torch
        xb = self._bytes_of(x, stream)
        cap = lz_compressed_bound(xb.numel(), p)
        if cap == 0:
            raise LzError(LZ_ERR_INVALID_ARG, "lz_compressed_bound")
        if out is None:
            out = torch.empty(cap, dtype=torch.uint8, device=xb.device)
        if out_bytes is None:
            out_bytes = torch.zeros(1, dtype=torch.int64, device=xb.device)
        lz_compress_ex(self.ctx, xb.data_ptr(), xb.numel(), p, out.data_ptr(), out.numel(),
                       out_bytes.data_ptr(), self._stream(stream), match=match,
                       version=version)
        return out, out_bytes

    def decompress(self, stream_bytes, n_bytes: int | None = None, out=None,
                   out_bytes=None, in_bytes: int | None = None, stream=None):
        torch = self.torch
        sb = self._bytes_of(stream_bytes, stream)
        nin = sb.numel() if in_bytes is None else in_bytes
        if out is None:
            if n_bytes is None:
                n_bytes = lz_decompressed_size(sb.data_ptr(), nin, self._stream(stream))
            out = torch.empty(max(n_bytes, 1), dtype=torch.uint8, device=sb.device)
        if out_bytes is None:
            out_bytes = torch.zeros(1, dtype=torch.int64, device=sb.device)
        lz_decompress(self.ctx, sb.data_ptr(), nin, out.data_ptr(),
                      out.numel() if n_bytes is None else n_bytes,
                      out_bytes.data_ptr(), self._stream(stream))
        return out, out_bytes

    def sync(self, stream=None) -> int:
        return lz_sync(self.ctx, self._stream(stream))

    def compress_sync(self, x, p: Params, stream=None, match: int = LZ_MATCH_EXACT,
                      version: int = 1):
        out, nb = self.compress(x, p, stream=stream, match=match, version=version)
        st = self.sync(stream)
        if st != LZ_OK:
            raise LzError(st, "compress (device)")
        return out[: int(nb.item())]

    def decompress_sync(self, stream_bytes, stream=None):
        out, nb = self.decompress(stream_bytes, stream=stream)
        st = self.sync(stream)
        if st != LZ_OK:
            raise LzError(st, "decompress (device)")
        return out[: int(nb.item())]
