"""The bounds-checked build (-DLZ_CHECKED): every index the kernels compute
into shared or global memory at the guarded sites is checked, a violation
is counted and the access skipped (no trap) and reported as
LZ_ERR_INTERNAL.  A parity grid of small cases runs on that build in a
separate process (the binding loads one library per process): every stream
must equal the oracle's, every round trip must be exact, and no check may
fire."""
from __future__ import annotations

import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import sys
sys.path.insert(0, ROOT)
import numpy as np
import torch
import oracle
from paper_2304_07342_gb300 import build, lz, synth
lz.load(build.build(checked=True))
codec = lz.Codec(0)
rng = np.random.default_rng(0)
kinds = {
    "quant": lambda n: synth.quant_codes_laplace(n, seed=1),
    "markov": lambda n: synth.markov_codes(n, seed=2),
    "const": lambda n: np.full(n, 7, np.uint32),
    "period": lambda n: (np.arange(n) % 5).astype(np.uint32),
    "random": lambda n: rng.integers(0, 1 << 32, n, dtype=np.uint64).astype(np.uint32),
}
grid = [(1, 2048, 128, 3), (1, 1024, 300, 2), (2, 4096, 128, 3), (2, 2048, 512, 2),
        (4, 8192, 256, 2), (4, 1024, 64, 1)]
checked = 0
for S, C, W, m in grid:
    dt = {1: np.uint8, 2: np.uint16, 4: np.uint32}[S]
    for name, gen in kinds.items():
        x = np.asarray(gen(40_000 // S + 7)).astype(np.uint64)
        x = (x % (1 << (8 * S))).astype(dt)
        P = lz.Params(S, C, W, m, 255)
        d = torch.from_numpy(x.view(np.uint8)).cuda()
        got = codec.compress_sync(d, P).cpu().numpy()
        ref = oracle.compress(x, oracle.Params(S, C, W, m, 255))
        assert np.array_equal(got, ref), (S, C, W, m, name)
        back = codec.decompress_sync(torch.from_numpy(got).cuda())
        assert torch.equal(back, d), (S, C, W, m, name)
        for version, match in ((2, lz.LZ_MATCH_EXACT), (2, lz.LZ_MATCH_OVERLAP), (1, lz.LZ_MATCH_PAPER)):
            s2 = codec.compress_sync(d, P, match=match, version=version).cpu().numpy()
            mode = {lz.LZ_MATCH_EXACT: oracle.MATCH_EXACT, lz.LZ_MATCH_OVERLAP: oracle.MATCH_OVERLAP,
                    lz.LZ_MATCH_PAPER: oracle.MATCH_PAPER}[match]
            r2 = oracle.compress(x, oracle.Params(S, C, W, m, 255), mode=mode, version=version)
            assert np.array_equal(s2, r2), (S, C, W, m, name, version, match)
            back = codec.decompress_sync(torch.from_numpy(s2).cuda())
            assert torch.equal(back, d)
        checked += 1
assert codec.sync() == lz.LZ_OK
print("checked", checked)
'''


def test_checked_build_parity_grid():
    out = subprocess.run([sys.executable, "-c", SCRIPT.replace("ROOT", repr(ROOT))],
                         capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert out.returncode == 0, out.stdout[-2000:] + out.stderr[-4000:]
    assert "checked 30" in out.stdout
