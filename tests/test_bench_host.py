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


def test_summary_line_is_compact():
    # the summary line must stay short enough to survive in a log's tail next
    # to the headline: a few numbers per record
    import json
    main = {"steady_state": {"ms_per_step": 5.05, "step0_ms": 8.6},
            "phases_ms_per_step": {k: 1.23456 for k in
                                   ("cells", "hsearch", "csr", "density", "forces", "update")}}
    rec = {"value": 2.3e8, "ms_per_step": 4.33, "e2e": {"value": 1.8e8},
           "roofline": {"frac": 0.0812}, "phases_ms_per_step": {"forces": 0.91}}
    ens = {"batched": {"updates_per_s": 1.77e8},
           "staged": {"latency_ms_p50": 1430.0, "latency_ms_p99": 4280.0},
           "single_instance_path": {"updates_per_s": 7.9e7, "latency_ms_p50": 4710.0,
                                    "latency_ms_p99": 9410.0},
           "batched_equals_single_bitwise": True}
    srv = {"latency_p50": 2.6, "latency_p99": 6.7, "served_updates_per_s": 1.71e8,
           "offered_updates_per_s": 2.4e8, "requests": 2000,
           "split": {q: {"p50": 0.1, "p99": 1.2} for q in ("tick_wait", "queueing", "run")}}
    serving = {"batched_fp64": srv, "batched_mixed": srv, "single_instance_fp64": srv}
    variants = {"runs": [{"kernel": k, "gradients": g, "precision": p, "ms_per_step": 21.47,
                          "roofline": {"frac": 0.348}}
                         for k, g, p in [(0, 0, 2)] * 9]}
    sm = bench.summary_of(main, {"evrard_mixed": rec, "fp64_pipe": rec}, {"ms_per_step": 0.64},
                          {"fp64": ens, "mixed": ens}, serving, variants)
    txt = json.dumps({"summary": sm})
    assert len(txt) < 1500, len(txt)
    assert sm["serving"]["requests"] == 2000
    assert sm["evrard_mixed"]["roofline_frac"] == 0.0812


def test_ncu_evidence_only_for_the_captured_sources(monkeypatch):
    # the counters of a capture are reported only while the kernel's sources
    # hash to the captured version
    for kind in bench.NCU_EVIDENCE:
        ref = bench.ncu_evidence(kind)
        assert ref is None or ref["dram_bytes"] > 0
    stale = {k: dict(v, sha1="0" * 40) for k, v in bench.NCU_EVIDENCE.items()}
    monkeypatch.setattr(bench, "NCU_EVIDENCE", stale)
    assert all(bench.ncu_evidence(k) is None for k in stale)
    assert bench.ncu_evidence("no such kernel") is None
