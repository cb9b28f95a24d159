"""sph_step and sph_batch_step replay one captured CUDA graph per step (per
parity of the double-buffered state) instead of launching its ~35 kernels one
by one. The graph holds the same kernels in the same order, so the results
must be the same bits as the direct launches (taken here with per-phase
timing on, which launches directly), also when sizes, parameters or the
caller's dt/time arrays change between calls (the graph is captured again),
and when the caller records sph_step into a CUDA graph of its own."""
import numpy as np
import pytest

from paper_1809_08013_gb300 import ics

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_08013_gb300 import binding
    binding.load()
    return binding


def host(arr):
    return {k: v.detach().cpu().numpy().copy() for k, v in arr.items()}


def same(a, b):
    for k in a:
        assert np.array_equal(a[k].view(np.uint8), b[k].view(np.uint8)), k


def _case(side, seed, precision=0):
    s, p = ics.square_patch(side, seed=seed)
    p.precision = precision
    return ics.random_velocities(s, seed=seed + 1, scale=1.5), p


def _run(B, ctx, s, prm, nsteps, timing, calls=1):
    arr = B.alloc_arrays(s)
    ctx.timing_enable(timing)
    for _ in range(calls):
        ctx.step(prm, arr, nsteps=nsteps)
    if timing:
        ctx.timing_read()
        ctx.timing_enable(False)
    assert ctx.sync() == B.SPH_OK
    return host(arr)


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_graph_replay_equals_direct_launches(B, precision):
    s, prm = _case(16, 3, precision)
    ctx = B.Context(len(s["x"]))
    direct = _run(B, ctx, s, prm, 3, timing=True)
    graph = _run(B, ctx, s, prm, 3, timing=False)
    same(direct, graph)
    again = _run(B, ctx, s, prm, 1, timing=False, calls=3)  # both parities, cached graphs
    same(direct, again)


def test_graphs_follow_size_and_array_changes(B):
    # one context, two problem sizes and fresh caller arrays (new dt / time
    # pointers) in turn: every call equals a fresh context's direct launches
    a, pa = _case(13, 5)
    b, pb = _case(17, 7)
    ctx = B.Context(len(b["x"]))
    for s, p in ((a, pa), (b, pb), (a, pa), (b, pb)):
        ref = _run(B, B.Context(len(s["x"])), s, p, 2, timing=True)
        got = _run(B, ctx, s, p, 2, timing=False)
        same(ref, got)


def test_batch_step_graphs_equal_direct(B):
    insts = [_case(10, 11), _case(13, 12, 0), _case(9, 13)]
    counts = [len(s["x"]) for s, _ in insts]
    state = {k: np.concatenate([s[k] for s, _ in insts]) for k in B.STATE_FIELDS}
    outs = []
    for timing in (True, False):
        ctx = B.Context(sum(counts), max_instances=4)
        ctx.batch_set(counts, [p for _, p in insts])
        arr = B.alloc_arrays(state, ninst=len(insts))
        ctx.timing_enable(timing)
        ctx.batch_step(arr, nsteps=3)
        if timing:
            ctx.timing_read()
            ctx.timing_enable(False)
        assert ctx.sync() == B.SPH_OK
        outs.append(host(arr))
    same(outs[0], outs[1])


def test_step_inside_a_callers_capture(B):
    # while the caller's stream is being captured the library launches the
    # kernels directly into the caller's graph; replaying that graph gives the
    # same bits as an uncaptured call
    s, prm = _case(14, 21)
    ref = _run(B, B.Context(len(s["x"])), s, prm, 2, timing=False)
    ctx = B.Context(len(s["x"]))
    arr = B.alloc_arrays(s)
    ic = {k: arr[k].clone() for k in B.STATE_FIELDS}
    stream = torch.cuda.Stream()
    ctx.step(prm, arr, nsteps=1, stream=stream)  # first use outside the capture
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        for k in B.STATE_FIELDS:
            arr[k].copy_(ic[k])
        arr["time"].zero_()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        ctx.step(prm, arr, nsteps=2, stream=stream)
    g.replay()
    torch.cuda.synchronize()
    assert ctx.sync() == B.SPH_OK
    same(ref, host(arr))
