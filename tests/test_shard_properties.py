"""Randomised properties of the sharding helpers (CPU, hypothesis): the row
bands of one image partition its rows in order, start on tile rows and differ
by at most one tile row; the longest-first image partition assigns every image
exactly once and keeps the largest rank load within the list-scheduling bound
(mean load plus the largest image)."""
import pytest

from paper_2501_06838_gb300 import shard

hyp = pytest.importorskip("hypothesis")
st = pytest.importorskip("hypothesis.strategies")
given, settings = hyp.given, hyp.settings


@settings(max_examples=200, deadline=None)
@given(st.integers(0, 5000), st.integers(1, 64), st.sampled_from([8, 16, 32]))
def test_band_rows_partition(out_h, parts, tile):
    bands = shard.band_rows(out_h, parts, tile)
    assert len(bands) == parts
    pos = 0
    for r0, rows in bands:
        assert r0 == pos and rows >= 0
        assert r0 % tile == 0 or r0 == out_h
        pos += rows
    assert pos == out_h
    # tile rows per band (the ragged last tile row counts as one): as even as can be
    cdiv = lambda a: -(-a // tile)
    trows = [cdiv(r0 + rows) - cdiv(r0) for r0, rows in bands]
    assert sum(trows) == cdiv(out_h)
    assert max(trows) - min(trows) <= 1


@settings(max_examples=200, deadline=None)
@given(st.lists(st.floats(0.0, 1e6, allow_nan=False), min_size=0, max_size=60),
       st.integers(1, 9))
def test_shard_images_lpt_bound(costs, world):
    parts = shard.shard_images(costs, world)
    assert len(parts) == world
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(len(costs)))
    assert all(p == sorted(p) for p in parts)
    if costs:
        loads = [sum(costs[i] for i in p) for p in parts]
        assert max(loads) <= sum(costs) / world + max(costs) + 1e-6 * (1 + sum(costs))
