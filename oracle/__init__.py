"""CPU oracle for chunked multi-byte LZSS -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product (the CUDA library and its
Python binding) never imports, links or executes anything here, and this
package imports nothing from the product.

The arithmetic lives in ``lzref.c`` (plain C, compiled by :func:`build`);
this module only marshals numpy buffers through ctypes.  What each function
computes, and which passage of the paper it follows, is documented in
``lzref.h``:

* :func:`longest_match` -- section 2.2 step 2 over S-byte symbols (3.2.3),
  nearest offset on ties, length <= offset (3.3.2);
* :func:`paper_match` -- the paper's own matcher (section 3.3.2, its four
  matching steps), a heuristic that never exceeds :func:`longest_match`;
* :func:`parse_chunk` -- section 2.2 steps 1-6 inside one chunk (3.3.1),
  with either matcher;
* :func:`compress` / :func:`decompress` -- the whole chunked stream;
* :func:`huff_compress` / :func:`huff_decompress` -- the Huffman stage that
  follows LZSS in section 4.5's use case (``huffref.h``).

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
(brute force, closed forms, hand-worked fixtures, round trip).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "lzref.c"), os.path.join(_HERE, "huffref.c")]
_LIB_PATH = os.path.join(_HERE, "liblzref.so")

OK, EINVAL, ESMALL, ECORRUPT = 0, 1, 2, 3


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: oracle returned {code}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile ``lzref.c`` and ``huffref.c`` into ``liblzref.so`` next to
    them (gcc, -O2)."""
    deps = _SRCS + [s[:-2] + ".h" for s in _SRCS]
    if (not force and os.path.exists(_LIB_PATH)
            and all(os.path.getmtime(_LIB_PATH) >= os.path.getmtime(d) for d in deps)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-Wextra",
                           "-shared", "-fPIC", "-o", tmp, *_SRCS])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        u32, u64 = ctypes.c_uint32, ctypes.c_uint64
        u32p, u64p = ctypes.POINTER(u32), ctypes.POINTER(u64)
        lib.lzref_check_params.argtypes = [u32] * 5
        lib.lzref_check_params.restype = ctypes.c_int
        lib.lzref_bound.argtypes = [u64] + [u32] * 5
        lib.lzref_bound.restype = u64
        lib.lzref_longest_match.argtypes = [u8p, u32, u32, u32, u32, u32,
                                            u32p, u32p]
        lib.lzref_longest_match.restype = None
        lib.lzref_parse_chunk.argtypes = [u8p, u32, u32, u32, u32, u32,
                                          u32p, u32p]
        lib.lzref_parse_chunk.restype = u32
        lib.lzref_paper_match.argtypes = [u8p, u32, u32, u32, u32, u32,
                                          u32p, u32p]
        lib.lzref_paper_match.restype = None
        lib.lzref_parse_chunk_mode.argtypes = [u8p, u32, u32, u32, u32, u32,
                                               u32, u32p, u32p]
        lib.lzref_parse_chunk_mode.restype = u32
        lib.lzref_compress_mode.argtypes = [u8p, u64] + [u32] * 6 + [
            u8p, u64, u64p]
        lib.lzref_compress_mode.restype = ctypes.c_int
        lib.lzref_compress_v.argtypes = [u8p, u64] + [u32] * 7 + [
            u8p, u64, u64p]
        lib.lzref_compress_v.restype = ctypes.c_int
        lib.lzref_longest_match_overlap.argtypes = [u8p, u32, u32, u32, u32, u32,
                                                    u32p, u32p]
        lib.lzref_longest_match_overlap.restype = None
        lib.huffref_lengths.argtypes = [u64p, u32, u8p]
        lib.huffref_lengths.restype = None
        lib.huffref_codes.argtypes = [u8p, u32p]
        lib.huffref_codes.restype = None
        lib.huffref_bound.argtypes = [u64]
        lib.huffref_bound.restype = u64
        lib.huffref_compress.argtypes = [u8p, u64, u8p, u64, u64p]
        lib.huffref_compress.restype = ctypes.c_int
        lib.huffref_decompressed_size.argtypes = [u8p, u64, u64p]
        lib.huffref_decompressed_size.restype = ctypes.c_int
        lib.huffref_decompress.argtypes = [u8p, u64, u8p, u64, u64p]
        lib.huffref_decompress.restype = ctypes.c_int
        lib.lzref_compress.argtypes = [u8p, u64] + [u32] * 5 + [u8p, u64,
                                                                u64p]
        lib.lzref_compress.restype = ctypes.c_int
        lib.lzref_decompressed_size.argtypes = [u8p, u64, u64p]
        lib.lzref_decompressed_size.restype = ctypes.c_int
        lib.lzref_decompress.argtypes = [u8p, u64, u8p, u64, u64p]
        lib.lzref_decompress.restype = ctypes.c_int
        _lib = lib
    return _lib


@dataclass(frozen=True)
class Params:
    """S symbol bytes, C chunk bytes, W window (symbols), m min match, M max match."""
    S: int
    C: int
    W: int
    m: int
    M: int = 255

    def tuple(self):
        return (self.S, self.C, self.W, self.m, self.M)


def _bytes(buf) -> np.ndarray:
    a = np.ascontiguousarray(buf)
    return a.view(np.uint8).reshape(-1)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def check_params(p: Params) -> bool:
    return _load().lzref_check_params(*p.tuple()) == OK


def bound(n: int, p: Params) -> int:
    return int(_load().lzref_bound(n, *p.tuple()))


def longest_match(chunk, p_sym: int, S: int, W: int, M: int = 255):
    """(len, off) of the longest, nearest match at symbol ``p_sym``."""
    b = _bytes(chunk)
    k = b.size // S
    ln, off = ctypes.c_uint32(), ctypes.c_uint32()
    _load().lzref_longest_match(_ptr(b), k, p_sym, S, W, M,
                                ctypes.byref(ln), ctypes.byref(off))
    return ln.value, off.value


def longest_match_overlap(chunk, p_sym: int, S: int, W: int, M: int = 255):
    """(len, off) of the longest, nearest match at ``p_sym`` when matches may
    overlap the look-ahead (length bounded by M and the chunk end only)."""
    b = _bytes(chunk)
    k = b.size // S
    ln, off = ctypes.c_uint32(), ctypes.c_uint32()
    _load().lzref_longest_match_overlap(_ptr(b), k, p_sym, S, W, M,
                                        ctypes.byref(ln), ctypes.byref(off))
    return ln.value, off.value


def paper_match(chunk, p_sym: int, S: int, W: int, M: int = 255):
    """(len, off) found at symbol ``p_sym`` by the paper's matcher (section
    3.3.2: forward scan, search pointer never moved back, first run of the
    greatest length)."""
    b = _bytes(chunk)
    k = b.size // S
    ln, off = ctypes.c_uint32(), ctypes.c_uint32()
    _load().lzref_paper_match(_ptr(b), k, p_sym, S, W, M,
                              ctypes.byref(ln), ctypes.byref(off))
    return ln.value, off.value


MATCH_EXACT, MATCH_PAPER, MATCH_OVERLAP = 0, 1, 2


def parse_chunk(chunk, S: int, W: int, m: int, M: int = 255,
                mode: int = MATCH_EXACT):
    """Greedy tokens of one chunk as a list of (len, off); off 0 = literal.
    ``mode`` picks the matcher: MATCH_EXACT (longest, nearest) or
    MATCH_PAPER (the paper's scan)."""
    b = _bytes(chunk)
    k = b.size // S
    tl = np.zeros(max(k, 1), np.uint32)
    to = np.zeros(max(k, 1), np.uint32)
    nt = _load().lzref_parse_chunk_mode(
        _ptr(b), k, S, W, m, M, mode,
        tl.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
        to.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))
    return [(int(tl[i]), int(to[i])) for i in range(nt)]


def compress(data, p: Params, mode: int = MATCH_EXACT, version: int = 1) -> np.ndarray:
    """Compressed GLZ1 stream of ``data`` (any numpy array, taken as bytes),
    parsed with the matcher ``mode``, in stream version ``version`` (2 adds
    stored chunks, see lzref.h)."""
    b = _bytes(data)
    cap = bound(b.size, p)
    if cap == 0:
        raise OracleError(EINVAL, "bound")
    out = np.empty(cap, np.uint8)
    nb = ctypes.c_uint64()
    rc = _load().lzref_compress_v(_ptr(b), b.size, *p.tuple(), mode, version,
                                  _ptr(out), cap, ctypes.byref(nb))
    if rc != OK:
        raise OracleError(rc, "compress")
    return out[: nb.value].copy()


def decompressed_size(stream) -> int:
    b = _bytes(stream)
    n = ctypes.c_uint64()
    rc = _load().lzref_decompressed_size(_ptr(b), b.size, ctypes.byref(n))
    if rc != OK:
        raise OracleError(rc, "decompressed_size")
    return n.value


def decompress(stream) -> np.ndarray:
    b = _bytes(stream)
    n = decompressed_size(b)
    out = np.empty(max(n, 1), np.uint8)
    nb = ctypes.c_uint64()
    rc = _load().lzref_decompress(_ptr(b), b.size, _ptr(out), n,
                                  ctypes.byref(nb))
    if rc != OK:
        raise OracleError(rc, "decompress")
    return out[:n].copy()


def decompress_status(stream) -> int:
    """Return code of decompressing ``stream`` (0 ok, 3 corrupt, ...)."""
    b = _bytes(stream)
    n = ctypes.c_uint64()
    rc = _load().lzref_decompressed_size(_ptr(b), b.size, ctypes.byref(n))
    if rc != OK:
        return rc
    out = np.empty(max(n.value, 1), np.uint8)
    nb = ctypes.c_uint64()
    return _load().lzref_decompress(_ptr(b), b.size, _ptr(out), n.value,
                                    ctypes.byref(nb))


# --- parameter policy (section 3.2.3) -----------------------------------------

LEVEL_WINDOWS = (32, 64, 128, 255)  # levels 1-4: window in symbols


def min_profitable_match(S: int, W: int) -> int:
    """Smallest match length whose pointer (one length byte plus a one- or
    two-byte offset) is shorter than the S-byte literals it replaces."""
    offB = 1 if W <= 256 else 2
    return (1 + offB) // S + 1


def ratio_below(n_bytes: int, stream_bytes: int, num: int = 3, den: int = 2) -> bool:
    """n / stream < num / den, in integers (the ratio test of the policy)."""
    return n_bytes * den < num * stream_bytes


def select_params(sample, dtype_bytes: int, level: int = 3,
                  chunk_bytes: int = 4096) -> Params:
    """The paper's parameter selection (section 3.2.3).  The symbol length
    starts at the data type's size (multi-byte matching, the default) with
    the level's window enlarged S times; the sample is compressed with it,
    and when its compression ratio is below 1.5 the policy falls back to
    single-byte matching with the level's window.  The minimum match is the
    shortest profitable one, the maximum 255."""
    if dtype_bytes not in (1, 2, 4) or level not in (1, 2, 3, 4):
        raise OracleError(EINVAL, "select_params")
    Wl = LEVEL_WINDOWS[level - 1]
    single = Params(1, chunk_bytes, Wl, min_profitable_match(1, Wl), 255)
    if dtype_bytes == 1:
        return single
    Wm = min(1024, dtype_bytes * Wl)
    multi = Params(dtype_bytes, chunk_bytes, Wm, min_profitable_match(dtype_bytes, Wm), 255)
    b = _bytes(sample)
    b = b[: b.size - b.size % dtype_bytes]
    if b.size == 0:
        raise OracleError(EINVAL, "select_params")
    size = compress(b, multi).size
    return single if ratio_below(b.size, size) else multi


# --- Huffman stage after LZSS (section 4.5's use case), huffref.c ----------------

HUFF_MAX_LEN, HUFF_BLOCK, HUFF_SUB = 12, 32768, 1024


def huff_lengths(hist, max_len: int = HUFF_MAX_LEN) -> np.ndarray:
    """Code lengths (0 = absent) of the optimal prefix code with lengths <=
    max_len for 256 counts (package-merge, tie rules in huffref.c)."""
    h = np.ascontiguousarray(hist, dtype=np.uint64)
    assert h.size == 256
    out = np.zeros(256, np.uint8)
    _load().huffref_lengths(h.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                            max_len, _ptr(out))
    return out


def huff_codes(lengths) -> np.ndarray:
    """Canonical code of each byte value for the given lengths."""
    ln = np.ascontiguousarray(lengths, dtype=np.uint8)
    out = np.zeros(256, np.uint32)
    _load().huffref_codes(_ptr(ln), out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))
    return out


def huff_bound(n: int) -> int:
    return int(_load().huffref_bound(n))


def huff_compress(data) -> np.ndarray:
    b = _bytes(data)
    cap = int(_load().huffref_bound(b.size))
    out = np.empty(cap, np.uint8)
    nb = ctypes.c_uint64()
    rc = _load().huffref_compress(_ptr(b), b.size, _ptr(out), cap, ctypes.byref(nb))
    if rc != OK:
        raise OracleError(rc, "huff_compress")
    return out[: nb.value].copy()


def huff_decompress_status(stream):
    """(return code, bytes) of decoding a GHF1 stream."""
    b = _bytes(stream)
    n = ctypes.c_uint64()
    rc = _load().huffref_decompressed_size(_ptr(b), b.size, ctypes.byref(n))
    if rc != OK:
        return rc, None
    out = np.empty(max(n.value, 1), np.uint8)
    nb = ctypes.c_uint64()
    rc = _load().huffref_decompress(_ptr(b), b.size, _ptr(out), n.value, ctypes.byref(nb))
    return rc, (out[: n.value].copy() if rc == OK else None)


def huff_decompress(stream) -> np.ndarray:
    rc, out = huff_decompress_status(stream)
    if rc != OK:
        raise OracleError(rc, "huff_decompress")
    return out
