"""Batches of independent problems (sph_batch_set / sph_batch_step): every
instance of a batch must give bit for bit the result of stepping it alone,
its neighbour list must stay inside the instance, and the batched step must
replay unchanged from a CUDA graph. Instances mix sizes, equations of state,
periodicity and velocity fields.
"""
import numpy as np
import pytest

from paper_1809_08013_gb300 import ics
from parity_util import TOL_FP64, canon_oracle, check, force_err, normwise, same_sets

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

FIELDS_OUT = ("x", "y", "z", "vx", "vy", "vz", "h", "u", "rho", "p", "c", "ax", "ay", "az",
              "du", "mumax", "nnb")


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_08013_gb300 import binding
    binding.load()
    return binding


def host(t):
    return t.detach().cpu().numpy()


def instances(precision):
    out = []
    s, p = ics.square_patch(12, seed=21, omega=3.0)
    out.append((s, p))
    s, p = ics.square_patch(17, seed=22, omega=7.0)
    out.append((ics.random_velocities(s, seed=23, scale=1.5), p))
    out.append(ics.evrard(3000, seed=24))
    s, p = ics.square_patch(10, seed=25)
    out.append((s, p))
    s, p = ics.evrard(5000, seed=26)
    out.append((ics.random_velocities(s, seed=27, scale=0.2), p))
    for _, p in out:
        p.precision = precision
    return out


def concat(states):
    return {k: np.concatenate([s[k] for s in states]) for k in ics.FIELDS}


def run_batch(B, insts, nsteps, max_instances=None):
    counts = [len(s["x"]) for s, _ in insts]
    ctx = B.Context(sum(counts), max_instances=max_instances or len(insts))
    ctx.batch_set(counts, [p for _, p in insts])
    arr = B.alloc_arrays(concat([s for s, _ in insts]), ninst=len(insts))
    ctx.batch_step(arr, nsteps=nsteps)
    st = ctx.sync()
    return ctx, arr, counts, st


def run_alone(B, s, p, nsteps):
    ctx = B.Context(len(s["x"]))
    arr = B.alloc_arrays(s)
    ctx.step(p, arr, nsteps=nsteps)
    ctx.sync()
    return arr


@pytest.mark.parametrize("precision,tpp", [(0, 0), (1, 0), (0, 1), (0, 4), (1, 4)])
def test_batch_instances_bit_identical_to_alone(B, precision, tpp):
    insts = instances(precision)
    for _, p in insts:
        p.pair_threads = tpp
    _, arr, counts, st = run_batch(B, insts, nsteps=3)
    assert st in (B.SPH_OK, B.SPH_E_HNOCONV)
    off = np.concatenate([[0], np.cumsum(counts)])
    dt, tm = host(arr["dt"]), host(arr["time"])
    for k, (s, p) in enumerate(insts):
        alone = run_alone(B, s, p, nsteps=3)
        for f in FIELDS_OUT:
            a = host(arr[f])[off[k]:off[k + 1]]
            b = host(alone[f])
            assert np.array_equal(a.view(np.uint8), b.view(np.uint8)), (k, f)
        assert dt[k] == host(alone["dt"])[0] and tm[k] == host(alone["time"])[0], k


def test_batch_neighbour_lists_stay_in_their_instance(B, orc):
    insts = instances(0)
    ctx, arr, counts, _ = run_batch(B, insts, nsteps=1)
    offs, idx, ng, order = ctx.neighbors_to_host()
    coff = np.concatenate([[0], np.cumsum(counts)])
    inst_of_caller = np.repeat(np.arange(len(counts)), counts)
    lens = np.diff(offs)
    # empty slots have no caller particle and no row
    assert np.all(lens[order < 0] == 0)
    assert np.count_nonzero(order >= 0) == sum(counts)
    assert np.array_equal(np.sort(order[order >= 0]), np.arange(sum(counts)))
    rows = np.repeat(np.arange(len(order)), lens)
    pos = np.arange(len(idx)) - np.repeat(offs[:-1], lens)
    flag = (pos < np.repeat(ng, lens)).astype(np.int8)
    rc, cc = order[rows].astype(np.int64), order[idx].astype(np.int64)
    assert np.all(rc >= 0) and np.all(cc >= 0)
    # every entry joins two particles of the same instance
    ik = inst_of_caller[rc]
    assert np.array_equal(ik, inst_of_caller[cc])
    # and each instance's sets equal the oracle's for the state the step started from
    for k, (s, p) in enumerate(insts):
        o = orc.pipeline(p, s)
        m = ik == k
        r, c, f = rc[m] - coff[k], cc[m] - coff[k], flag[m]
        key = np.lexsort((f, c, r))
        assert same_sets((r[key], c[key], f[key]), canon_oracle(o["off"], o["idx"], o["ng"])), k


def test_batch_caller_order_export(B, orc):
    # caller rows of a batch: instance k's rows are its caller range, and
    # each equals the oracle's row of that particle
    insts = instances(0)
    ctx, arr, counts, _ = run_batch(B, insts, nsteps=1)
    off, idx, ng = ctx.neighbors_caller(sum(counts))
    coff = np.concatenate([[0], np.cumsum(counts)])
    for k, (s, p) in enumerate(insts):
        o = orc.pipeline(p, s)
        a, b = coff[k], coff[k + 1]
        assert np.array_equal(off[a:b + 1] - off[a], o["off"]), k
        assert np.array_equal(ng[a:b], o["ng"]), k
        for r in range(b - a):
            lo, g, hi = off[a + r], ng[a + r], off[a + r + 1]
            oo, og = o["off"][r], o["ng"][r]
            assert np.array_equal(idx[lo:lo + g] - a, np.sort(o["idx"][oo:oo + og])), (k, r)
            assert np.array_equal(idx[lo + g:hi] - a,
                                  np.sort(o["idx"][oo + og:o["off"][r + 1]])), (k, r)


def test_batch_one_step_matches_oracle(B, orc):
    insts = instances(0)
    _, arr, counts, _ = run_batch(B, insts, nsteps=1)
    off = np.concatenate([[0], np.cumsum(counts)])
    for k, (s, p) in enumerate(insts):
        o = orc.pipeline(p, s)
        sl = slice(off[k], off[k + 1])
        assert np.array_equal(host(arr["h"])[sl].view(np.int64), o["h"].view(np.int64)), k
        assert normwise(host(arr["rho"])[sl], o["rho"]) <= TOL_FP64, k
        check({f: force_err(f, host(arr[f])[sl], o[f], o, p.periodic_z)
               for f in ("ax", "ay", "az", "du")}, TOL_FP64)
        assert abs(host(arr["dt"])[k] - o["dt"]) <= TOL_FP64 * o["dt"], k


def test_batch_instances_anywhere_in_the_arrays(B):
    # instances at scattered, out-of-order offsets of longer arrays (a memory
    # arena): same bits as alone, and entries outside the instances untouched
    insts = instances(0)
    counts = [len(s["x"]) for s, _ in insts]
    first = [30000, 100, 9000, 52000, 18000]
    n = 60000
    rng = np.random.Generator(np.random.PCG64(5))
    state = {k: rng.uniform(-1, 1, n) for k in ics.FIELDS}
    for (s, _), f0 in zip(insts, first):
        for k in ics.FIELDS:
            state[k][f0:f0 + len(s["x"])] = s[k]
    ctx = B.Context(n, max_instances=8)
    ctx.batch_set(counts, [p for _, p in insts], first=first)
    arr = B.alloc_arrays(state, ninst=len(insts))
    before = {k: host(arr[k]).copy() for k in FIELDS_OUT}
    ctx.batch_step(arr, nsteps=2)
    assert ctx.sync() in (B.SPH_OK, B.SPH_E_HNOCONV)
    inside = np.zeros(n, bool)
    for k, ((s, p), f0) in enumerate(zip(insts, first)):
        alone = run_alone(B, s, p, nsteps=2)
        sl = slice(f0, f0 + len(s["x"]))
        inside[sl] = True
        for f in FIELDS_OUT:
            assert np.array_equal(host(arr[f])[sl].view(np.uint8), host(alone[f]).view(np.uint8)), (k, f)
    for f in FIELDS_OUT:
        assert np.array_equal(host(arr[f])[~inside], before[f][~inside]), f
    with pytest.raises(B.SphError):  # overlapping instances
        ctx.batch_set(counts, [p for _, p in insts], first=[0, 100, 200, 300, 400])


def test_batch_step_replays_from_a_cuda_graph(B):
    insts = instances(0)
    counts = [len(s["x"]) for s, _ in insts]
    ctx = B.Context(sum(counts), max_instances=8)
    ctx.batch_set(counts, [p for _, p in insts])
    state = concat([s for s, _ in insts])
    eager = B.alloc_arrays(state, ninst=len(insts))
    ctx.batch_step(eager, nsteps=2)
    ctx.sync()
    arr = B.alloc_arrays(state, ninst=len(insts))
    ic = {k: arr[k].clone() for k in B.STATE_FIELDS}
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        ctx.batch_step(arr, nsteps=2, stream=s)
    for rep in range(2):  # replay twice from the initial conditions
        for k in B.STATE_FIELDS:
            arr[k].copy_(ic[k])
        arr["time"].zero_()
        g.replay()
        torch.cuda.synchronize()
        assert ctx.sync() in (B.SPH_OK, B.SPH_E_HNOCONV)
        for f in FIELDS_OUT + ("dt", "time"):
            assert np.array_equal(host(arr[f]).view(np.uint8), host(eager[f]).view(np.uint8)), (rep, f)


def test_batch_invalid_arguments(B):
    insts = instances(0)
    counts = [len(s["x"]) for s, _ in insts]
    ctx = B.Context(sum(counts), max_instances=4)
    with pytest.raises(B.SphError) as e:  # more instances than the context holds
        ctx.batch_set(counts, [p for _, p in insts])
    assert e.value.status == B.SPH_E_INVAL
    ctx = B.Context(sum(counts) - 1, max_instances=8)
    with pytest.raises(B.SphError):  # more particles than the capacity
        ctx.batch_set(counts, [p for _, p in insts])
    ctx = B.Context(sum(counts), max_instances=8)
    prms = [p for _, p in insts]
    prms[2] = ics.SphParams(**{**prms[2].as_dict(), "precision": 1})
    with pytest.raises(B.SphError):  # mixed precisions in one batch
        ctx.batch_set(counts, prms)
    ok = [p for _, p in insts]
    for far in (2 ** 31 - 1, 2 ** 62, 2 ** 63 - 2):  # past caller index 2^31 - 1 (and
        first = [0] * len(counts)                  # first + count overflowing int64)
        first[1:] = [sum(counts[:k]) for k in range(1, len(counts))]
        first[-1] = far
        with pytest.raises(B.SphError) as e:
            ctx.batch_set(counts, ok, first=first)
        assert e.value.status == B.SPH_E_INVAL
    ctx.batch_set(counts, [p for _, p in insts])
    arr = B.alloc_arrays(concat([s for s, _ in insts[:-1]]), ninst=len(insts))
    with pytest.raises(B.SphError):  # arrays do not match the batch
        ctx.batch_step(arr, nsteps=1)


def test_batch_of_one_equals_single_problem(B):
    s, p = ics.square_patch(13, seed=31)
    _, arr, _, _ = run_batch(B, [(s, p)], nsteps=2, max_instances=3)
    alone = run_alone(B, s, p, nsteps=2)
    for f in FIELDS_OUT:
        assert np.array_equal(host(arr[f]).view(np.uint8), host(alone[f]).view(np.uint8)), f


def test_autotune_picks_a_candidate_and_keeps_results_exact(B):
    insts = instances(0)
    counts = [len(s["x"]) for s, _ in insts]
    ctx = B.Context(sum(counts), max_instances=len(insts))
    ctx.batch_set(counts, [p for _, p in insts])
    state = concat([s for s, _ in insts])
    arr = B.alloc_arrays(state, ninst=len(insts))
    before = {k: host(arr[k]).copy() for k in B.STATE_FIELDS}
    res = ctx.autotune(arr, nsteps=1, cell_scales=[1.0, 1.5], pair_threads=[1, 2],
                       defer_lanes=[8, 16])
    # the caller's state is untouched by the trial runs
    for k in B.STATE_FIELDS:
        assert np.array_equal(host(arr[k]), before[k]), k
    assert res["cell_scale"] in (1.0, 1.25, 1.5)
    assert res["pair_threads"] in (1, 2) and res["defer_lanes"] in (8, 16)
    assert 1 <= len(res["trials"]) <= 6
    assert res["ms_per_step"] == min(t["ms_per_step"] for t in res["trials"])
    ctx.sync()
    # the batch now runs with the chosen knobs: still bit-identical to a single
    # problem given the same knobs, and h / neighbour counts do not depend on them
    ctx.batch_step(arr, nsteps=2)
    assert ctx.sync() in (B.SPH_OK, B.SPH_E_HNOCONV)
    off = np.concatenate([[0], np.cumsum(counts)])
    for k, (s, p) in enumerate(insts):
        q = ics.SphParams(**{**p.as_dict(), "cell_scale": res["cell_scale"],
                             "pair_threads": res["pair_threads"],
                             "defer_lanes": res["defer_lanes"]})
        alone = run_alone(B, s, q, nsteps=2)
        for f in FIELDS_OUT:
            a = host(arr[f])[off[k]:off[k + 1]]
            assert np.array_equal(a.view(np.uint8), host(alone[f]).view(np.uint8)), (k, f)
        plain = run_alone(B, s, p, nsteps=1)
        tuned1 = run_alone(B, s, q, nsteps=1)
        assert np.array_equal(host(plain["h"]), host(tuned1["h"])), k
        assert np.array_equal(host(plain["nnb"]), host(tuned1["nnb"])), k
