"""Host logic of the batch driver: the chunk hold applied to autotuned
per-kind parameters (no GPU)."""
from __future__ import annotations

from paper_2304_07342_gb300 import batch, lz


def P(S, C, W=128, m=3):
    return lz.Params(S, C, W, m)


def test_incompressible_kind_held_to_largest_compressible_chunk():
    params = [P(1, 2048), P(2, 4096), P(4, 8192, 256, 2), P(4, 8192, 256, 2)]
    ratios = [1.3, 1.8, 0.97, 1.0]
    out = batch.hold_chunks(params, ratios)
    assert out[:2] == params[:2]
    assert [p.C for p in out[2:]] == [4096, 4096]
    # everything but the chunk is kept
    assert all((p.S, p.W, p.m, p.M) == (q.S, q.W, q.m, q.M) for p, q in zip(out, params))


def test_smaller_chunks_and_threshold():
    params = [P(2, 8192), P(4, 2048, 64, 2)]
    # an incompressible kind with a chunk already below the cap is unchanged
    assert batch.hold_chunks(params, [2.0, 0.9]) == params
    # the threshold is inclusive
    assert batch.hold_chunks([P(2, 2048), P(4, 8192)], [1.05, 1.0])[1].C == 2048


def test_no_compressible_kind_leaves_params():
    params = [P(4, 8192), P(4, 16384)]
    assert batch.hold_chunks(params, [0.97, 1.01]) == params
    assert batch.hold_chunks([], []) == []
