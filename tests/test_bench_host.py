"""Host-side helpers of bench.py, without a GPU: the staged ensemble
grouping, the counted flops of the variants, and the replica-path rate."""
import pytest

import bench


def test_stage_groups_partition_by_size():
    import numpy as np
    from paper_1809_08013_gb300 import ics
    counts = [s ** 3 for s, _ in ics.ensemble_sizes(256, seed=1000)]
    groups = bench.stage_groups(counts, 4)
    flat = [k for g in groups for k in g]
    assert sorted(flat) == list(range(len(counts)))          # a partition
    sizes = [counts[k] for k in flat]
    assert sizes == sorted(sizes)                             # smallest first
    tot = sum(counts)
    parts = [sum(counts[k] for k in g) for g in groups]
    assert len(groups) == 4 and max(parts) <= tot / 4 + max(counts)
    assert bench.stage_groups([5], 4) == [[0]]
    assert bench.stage_groups([3, 1, 2], 1) == [[1, 2, 0]]


def test_variant_flop_counts():
    # kernel derivatives: the spline's 51 + 17; Wendland's derivative shape
    # costs as much; the sinc shape n + 6 operations; IAD per pair and matrix pair
    assert bench.variant_flops(0, 0, 5) == (bench.FLOPS_PAIR_BASE, bench.FLOPS_PAIR_AV, 0)
    assert bench.variant_flops(1, 0, 5) == (51, 17, 0)
    assert bench.variant_flops(2, 0, 5) == (51 - 10 + 2 * 11, 17, 0)
    assert bench.variant_flops(0, 1, 5) == (83 + 12, 17, 27 + 6)


def test_whole_job_rate():
    assert bench.whole_job_rate(4, 1_000_000, 20, 100.0) == pytest.approx(8e8)
