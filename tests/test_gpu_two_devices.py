"""One process driving two GPUs: the launch caches (shared-memory opt-in and
occupancy) are kept per device, so compressing and decompressing on device
1 after device 0 must give the oracle's streams there too.  Skipped when
fewer than two GPUs are visible."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from oracle import Params
from paper_2304_07342_gb300 import synth

pytestmark = pytest.mark.gpu


def test_compress_decompress_on_two_devices():
    import torch
    if torch.cuda.device_count() < 2:
        pytest.skip("needs two GPUs")
    from paper_2304_07342_gb300 import build, lz
    build.build()
    x = synth.quant_codes_laplace(300_000, seed=4)
    P = Params(2, 4096, 128, 3, 255)
    ref = oracle.compress(x, P)
    for dev in (0, 1, 0):
        c = lz.Codec(dev)
        d = torch.from_numpy(x.view(np.uint8).copy()).to(f"cuda:{dev}")
        s = c.compress_sync(d, lz.Params(*P.tuple()))
        assert np.array_equal(s.cpu().numpy(), ref), dev
        back, nb = c.decompress(s, n_bytes=d.numel(), in_bytes=s.numel())
        assert c.sync() == lz.LZ_OK
        assert torch.equal(back[:d.numel()], d), dev
        c.close()
    torch.cuda.set_device(0)
