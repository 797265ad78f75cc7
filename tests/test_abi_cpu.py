"""C ABI checks that need no GPU: the library builds and loads, exports every
entry point include/lz.h declares, and its pure host functions agree with
the oracle (bound, parameter validation)."""
from __future__ import annotations

import ctypes
import itertools
import os
import re

import pytest

import oracle
from paper_2304_07342_gb300 import build, lz

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions(header: str):
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lz_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return lz.load()


def test_every_declared_symbol_is_exported(lib):
    names = [n for n in declared_functions(os.path.join(ROOT, "include", "lz.h"))]
    assert names, "no declarations found"
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(lz.EXPORTS) == sorted(names)


def test_bound_matches_oracle(lib):
    for S, C, W, m, M in itertools.product((1, 2, 4), (16, 4096, 32768), (1, 255, 256, 257, 1024),
                                           (1, 2, 3), (3, 255)):
        if m > M:
            continue
        for n in (0, S, C, C + S, 10 * C - S, 1 << 20):
            n -= n % S
            assert lz.lz_compressed_bound(n, lz.Params(S, C, W, m, M)) == \
                oracle.bound(n, oracle.Params(S, C, W, m, M))


def test_check_params_matches_oracle(lib):
    for S, C, W, m, M in itertools.product((0, 1, 2, 3, 4, 8), (0, 15, 16, 4000, 4096, 32768, 32784),
                                           (0, 1, 1024, 1025), (0, 1, 200), (1, 199, 255, 256)):
        ok_c = lz.lz_check_params(lz.Params(S, C, W, m, M)) == lz.LZ_OK
        assert ok_c == oracle.check_params(oracle.Params(S, C, W, m, M))


def test_status_strings(lib):
    for code, name in [(0, "LZ_OK"), (1, "LZ_ERR_INVALID_ARG"), (2, "LZ_ERR_BUFFER_TOO_SMALL"),
                       (3, "LZ_ERR_CORRUPT"), (4, "LZ_ERR_NOMEM"), (5, "LZ_ERR_CUDA"),
                       (6, "LZ_ERR_TIMEOUT"), (7, "LZ_ERR_INTERNAL")]:
        assert lz.lz_status_string(code) == name


def test_null_arguments_rejected_without_gpu(lib):
    p = lz.Params(2, 4096, 128, 3).c()
    assert lib.lz_compress(None, None, 0, ctypes.byref(p), None, 0, None, None) == lz.LZ_ERR_INVALID_ARG
    assert lib.lz_decompress(None, None, 0, None, 0, None, None) == lz.LZ_ERR_INVALID_ARG
    assert lib.lz_sync(None, None) == lz.LZ_ERR_INVALID_ARG
    assert lib.lz_create(None, 0) == lz.LZ_ERR_INVALID_ARG
    assert lib.lz_compressed_bound(100, None) == 0
    assert lib.lz_set_test_hooks(None, None) == lz.LZ_ERR_INVALID_ARG
    assert lib.lz_batch_update(None, None, None, 0, None) == lz.LZ_ERR_INVALID_ARG


def test_product_does_not_import_oracle():
    """The library and its binding never reference the oracle."""
    pkg = os.path.join(ROOT, "paper_2304_07342_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "lzref" not in text, f


def test_huff_bound_matches_oracle(lib):
    for n in (0, 1, 1023, 32768, 32769, 10**6, 1 << 30):
        assert lz.lz_huff_bound(n) == oracle.huff_bound(n)
