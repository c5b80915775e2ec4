"""The force planner's rules, through scgr_plan_preview (host arithmetic, no
GPU): the split lengths cover the reference range without empty splits,
shared-memory-sum shapes take whole two-tile stages, split counts stay
within their caps, small problems go down to one tile and then half a tile
per split, and the 1M x 1M workload gets the plan the benchmark runs."""
import itertools

import pytest

from paper_1902_01061_gb300 import scgr

SMS = 152
TJ = 256


def plan(n, m, p=2.0, bps=4, sms=SMS):
    return scgr.scgr_plan_preview(n, m, p, sms, bps)


SIZES = [1, 255, 256, 257, 1000, 4095, 20000, 35000, 50000, 100_001, 320_000, 1_000_000]


@pytest.mark.parametrize("n,m", list(itertools.product(SIZES, [1, 1000, 30800, 320_000, 1_000_000])))
def test_splits_cover_the_reference_range(scgr_lib, n, m):
    pl = plan(n, m)
    ntiles = -(-n // TJ)
    assert pl["iblocks"] == -(-m // (pl["P"] * pl["tpb"]))
    if pl["half"]:
        assert pl["splits"] == 2 * ntiles and pl["tiles_per_split"] == 1
    else:
        # every split starts inside the range, and together they cover it
        assert (pl["splits"] - 1) * pl["tiles_per_split"] < ntiles <= pl["splits"] * pl["tiles_per_split"]
        assert 1 <= pl["splits"] <= 128


@pytest.mark.parametrize("n", [1000, 35000, 49_999, 100_001, 320_000, 777_777, 1_000_000])
def test_shared_memory_sum_shape_takes_whole_stages(scgr_lib, n):
    """Templates of >= 311,296 points (152 SMs) get 4 points x 128 threads
    with shared-memory sums, which stage two tiles at a time: every split
    length is even, so no block computes a padded tile except at the end of
    the range."""
    pl = plan(n, 320_000, bps=3)
    assert (pl["P"], pl["tpb"], pl["occ"]) == (4, 128, 2)
    assert pl["tiles_per_split"] % 2 == 0
    assert not pl["half"]


@pytest.mark.parametrize("m", [1000, 30800, 320_000, 1_000_000])
def test_split_count_caps(scgr_lib, m):
    for n in (20000, 100_000, 1_000_000):
        for bps in (2, 3, 4):
            pl = plan(n, m, bps=bps)
            if pl["half"]:
                continue
            slots = SMS * bps
            cap = min(128, max(16, -(-12 * slots // pl["iblocks"])))
            assert pl["splits"] <= cap


def test_small_problems_shorten_each_block(scgr_lib):
    """At least two tiles per split while two-tile splits fill a wave; the
    1,000-point case (8 template blocks, 4 tiles) cannot, so it goes down to
    half a tile per split: 8 x 8 blocks of 128 reference points."""
    pl = plan(1000, 1000)
    assert (pl["P"], pl["tpb"], pl["iblocks"]) == (1, 128, 8)
    assert pl["half"] == 1 and pl["splits"] == 8
    # 20,000 reference points: 79 tiles, 79 template blocks of 256 fill the
    # GPU with two-tile splits
    pl = plan(20000, 20000)
    assert not pl["half"] and pl["tiles_per_split"] >= 2
    # half tiles only for the 1 point x 128 threads shape
    for n, m in itertools.product([256, 1000, 5000], [1000, 4000, 5000, 30000]):
        pl = plan(n, m)
        if pl["half"]:
            assert (pl["P"], pl["tpb"], pl["occ"]) == (1, 128, 0)
            assert 2 * pl["iblocks"] * (-(-n // TJ)) <= SMS * 4


def test_benchmark_plan_at_full_size(scgr_lib):
    """1M x 1M on 152 SMs with 4 resident blocks: 4 points x 128 threads,
    shared-memory sums, 14 splits of 280 tiles (1,954 template blocks)."""
    pl = plan(1_000_000, 1_000_000)
    assert pl == {"P": 4, "tpb": 128, "occ": 2, "splits": 14, "tiles_per_split": 280, "iblocks": 1954, "half": 0}


def test_preview_rejects_bad_arguments(scgr_lib):
    for args in ((0, 10, 2.0, SMS, 4), (10, 0, 2.0, SMS, 4), (10, 10, 0.5, SMS, 4), (10, 10, 2.0, 0, 4),
                 (10, 10, 2.0, SMS, 0), (10, 10, float("nan"), SMS, 4)):
        with pytest.raises(scgr.ScgrError) as e:
            scgr.scgr_plan_preview(*args)
        assert e.value.status == 1
