"""Serving loop (continuous batching over sph_batch_step): host-side pieces on
the CPU, and on the GPU that every request's result equals stepping it alone
while requests join and leave the batch."""
import math

import numpy as np
import pytest

from paper_1809_08013_gb300 import serve


def test_arena_first_fit_and_coalescing():
    a = serve.Arena(100)
    assert a.take(30) == 0 and a.take(50) == 30 and a.take(30) is None
    assert a.fits(20) and not a.fits(21)
    a.give(0, 30)
    assert a.take(25) == 0
    a.give(30, 50)
    a.give(0, 25)
    assert a.free == [(0, 100)]
    assert a.take(100) == 0


def test_stream_recipe():
    reqs = serve.make_stream(400, rate=20.0, seed=7)
    t = np.array([r.arrival for r in reqs])
    assert np.all(np.diff(t) > 0)
    # Poisson: mean gap 1 / rate within a few standard errors
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() - 0.05) < 4 * 0.05 / math.sqrt(len(gaps))
    for r in reqs:
        assert 10 <= r.steps <= 100 and 2.0 <= r.omega <= 8.0
        if r.kind == "patch":
            side = round(r.n ** (1 / 3))
            assert side ** 3 == r.n
        assert 7000 <= r.n <= 1_010_000
    kinds = [r.kind for r in reqs]
    assert 0.4 < kinds.count("evrard") / len(kinds) < 0.6


def test_fifo_single_timeline():
    reqs = [serve.Request(k, arrival=a, kind="patch", n=8, steps=1, seed=k)
            for k, a in enumerate([0.0, 1.0, 1.5, 10.0])]
    s = serve.fifo_single(reqs, {0: 2.0, 1: 2.0, 2: 1.0, 3: 1.0})
    assert [r.done for r in reqs] == [2.0, 4.0, 5.0, 11.0]
    assert s["latency_p50"] == pytest.approx(np.percentile([2.0, 3.0, 3.5, 1.0], 50))


def test_latency_split_adds_up():
    # latency = tick wait + queueing + run for every request
    reqs = [serve.Request(k, arrival=a, kind="patch", n=8, steps=1, seed=k)
            for k, a in enumerate([0.0, 0.3, 0.6])]
    for r, (ch, ad, dn) in zip(reqs, [(0.0, 0.0, 1.0), (1.0, 1.0, 2.5), (1.0, 2.5, 4.0)]):
        r.chance, r.admitted, r.done = ch, ad, dn
    s = serve.summarize(reqs)
    sp = s["split"]
    assert sp["tick_wait"]["p50"] == pytest.approx(0.4)
    assert sp["queueing"]["p50"] == pytest.approx(0.0) and sp["queueing"]["p99"] > 1.4
    assert sp["run"]["p50"] == pytest.approx(1.5)
    for r in reqs:
        assert (r.chance - r.arrival) + (r.admitted - r.chance) + (r.done - r.admitted) == \
            pytest.approx(r.done - r.arrival)
    # one at a time: no tick wait, the wait is all queueing
    f = serve.fifo_single(reqs, {0: 2.0, 1: 2.0, 2: 1.0})
    assert f["split"]["tick_wait"]["p99"] == 0.0
    assert f["split"]["queueing"]["p50"] == pytest.approx(1.7)


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [0, 1])
def test_served_results_equal_alone(precision):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_08013_gb300 import binding as B
    B.load()
    reqs = serve.make_stream(10, rate=1.0, seed=3, n_min=1000, n_max=20000, steps=(2, 9))
    for k, r in enumerate(reqs):
        r.arrival = float(k // 2)  # two arrivals per tick of the virtual clock
    states = {r.rid: serve.initial_state(r, precision) for r in reqs}
    cap = 45000  # forces waiting for memory as well as for slots
    srv = serve.Server(cap, max_instances=4, quantum=3)
    peak = {"n": 0, "inst": 0}
    orig = srv.tick

    def tick():
        peak["n"] = max(peak["n"], sum(r.req.n for r in srv.active))
        peak["inst"] = max(peak["inst"], len(srv.active))
        return orig()

    srv.tick = tick
    summ = serve.serve(srv, reqs, states, clock="virtual")
    assert summ["requests"] == len(reqs)
    assert srv.status in (B.SPH_OK, B.SPH_E_HNOCONV)
    assert peak["inst"] <= 4 and peak["n"] <= cap
    assert srv.ticks > max(r.steps for r in reqs) // 3  # requests really were split over ticks
    for r in reqs:
        s, p = states[r.rid]
        ctx = B.Context(r.n)
        arr = B.alloc_arrays(s)
        ctx.step(p, arr, nsteps=r.steps)
        ctx.sync()
        for f in serve.OUT_FIELDS:
            got = r.result[f]
            ref = arr[f].cpu().numpy()
            assert np.array_equal(got.view(np.uint8), ref.view(np.uint8)), (r.rid, f)
        assert np.array_equal(r.result["nnb"], arr["nnb"].cpu().numpy()), r.rid
        assert r.result["time"] == float(arr["time"].item()), r.rid
