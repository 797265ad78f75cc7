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
* :func:`parse_chunk` -- section 2.2 steps 1-6 inside one chunk (3.3.1);
* :func:`compress` / :func:`decompress` -- the whole chunked stream.

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
_SRC = os.path.join(_HERE, "lzref.c")
_LIB_PATH = os.path.join(_HERE, "liblzref.so")

OK, EINVAL, ESMALL, ECORRUPT = 0, 1, 2, 3


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: oracle returned {code}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile ``lzref.c`` into ``liblzref.so`` next to it (gcc, -O2)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-Wextra",
                           "-shared", "-fPIC", "-o", tmp, _SRC])
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


def parse_chunk(chunk, S: int, W: int, m: int, M: int = 255):
    """Greedy tokens of one chunk as a list of (len, off); off 0 = literal."""
    b = _bytes(chunk)
    k = b.size // S
    tl = np.zeros(max(k, 1), np.uint32)
    to = np.zeros(max(k, 1), np.uint32)
    nt = _load().lzref_parse_chunk(
        _ptr(b), k, S, W, m, M,
        tl.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
        to.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))
    return [(int(tl[i]), int(to[i])) for i in range(nt)]


def compress(data, p: Params) -> np.ndarray:
    """Compressed GLZ1 stream of ``data`` (any numpy array, taken as bytes)."""
    b = _bytes(data)
    cap = bound(b.size, p)
    if cap == 0:
        raise OracleError(EINVAL, "bound")
    out = np.empty(cap, np.uint8)
    nb = ctypes.c_uint64()
    rc = _load().lzref_compress(_ptr(b), b.size, *p.tuple(), _ptr(out), cap,
                                ctypes.byref(nb))
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
