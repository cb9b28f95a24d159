"""Candidate lists of the h search (sph_params.list_skin): each particle's
list of the particles within 2 h (1 + skin) is kept across steps and calls
while it still holds every neighbour, and rebuilt otherwise. h and the
neighbour sets are bit-identical with and without the lists; the fields,
summed in another order, agree to rounding; steps served by the lists match
the oracle like any other."""
import numpy as np
import pytest

from paper_1809_08013_gb300 import ics
from parity_util import (TOL_FP64, canon_gpu, canon_oracle, check, force_err, normwise,
                         same_sets)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

STATE = ("x", "y", "z", "vx", "vy", "vz", "m", "h", "u")
OUTS = ("rho", "p", "c", "ax", "ay", "az", "du", "mumax")


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_08013_gb300 import binding
    binding.load()
    return binding


def _case(name, skin=0.15, precision=0):
    if name == "patch":  # periodic z, viscosity active; large enough that a warp's
        # search boxes at the list radius span less than a quarter of the period
        s, p = ics.square_patch(48, seed=51)
        s = ics.random_velocities(s, seed=52, scale=1.0)
    else:
        s, p = ics.evrard(8000, seed=53)
    p.list_skin = skin
    p.precision = precision
    return s, p


def host(t):
    return t.detach().cpu().numpy()


def _state(arr):
    return {k: host(arr[k]).copy() for k in STATE}


def _load(arr, s):
    for k in STATE:
        arr[k].copy_(torch.as_tensor(s[k]))


def _rows(ctx):
    off, idx, ng, order = ctx.neighbors_to_host()
    return off, idx, ng, order


@pytest.mark.parametrize("case", ["patch", "evrard"])
def test_lists_keep_h_and_sets_step_by_step(B, case):
    # two contexts advance from identical inputs at every step, one with the
    # lists (default skin), one without: h and the neighbour sets agree bit
    # for bit, the sums to rounding, and the lists served some of the steps
    s, p_on = _case(case)
    _, p_off = _case(case, skin=-1.0)
    n = len(s["x"])
    on, off = B.Context(n), B.Context(n)
    a_on, a_off = B.alloc_arrays(s), B.alloc_arrays(s)
    for k in range(6):
        _load(a_on, _state(a_off))
        on.step(p_on, a_on, nsteps=1)
        off.step(p_off, a_off, nsteps=1)
        assert on.sync() in (B.SPH_OK, B.SPH_E_HNOCONV)
        assert off.sync() in (B.SPH_OK, B.SPH_E_HNOCONV)
        assert np.array_equal(host(a_on["h"]).view(np.int64), host(a_off["h"]).view(np.int64)), k
        assert np.array_equal(host(a_on["nnb"]), host(a_off["nnb"])), k
        r_on, r_off = _rows(on), _rows(off)
        assert same_sets(canon_gpu(*r_on), canon_gpu(*r_off)), k
        check({f: normwise(host(a_on[f]), host(a_off[f])) for f in ("rho", "p", "c", "ax", "ay")},
              TOL_FP64)
    assert 1 <= on.list_builds() < 6 and off.list_builds() == 0
    if case == "patch":  # a slow rotation: at most one rebuild in six steps
        assert on.list_builds() <= 2


@pytest.mark.parametrize("case", ["patch", "evrard"])
def test_steps_served_by_lists_match_the_oracle(B, orc, case):
    # every step from the state the previous one left, against the oracle's
    # pipeline on that same state: h and the sets bit-exact, fields at 1e-12
    s, p = _case(case)
    ctx = B.Context(len(s["x"]))
    arr = B.alloc_arrays(s)
    for k in range(5):
        before = _state(arr)
        ctx.step(p, arr, nsteps=1)
        assert ctx.sync() in (B.SPH_OK, B.SPH_E_HNOCONV)
        o = orc.pipeline(p, before)
        assert np.array_equal(host(arr["h"]).view(np.int64), o["h"].view(np.int64)), k
        assert np.array_equal(host(arr["nnb"]), o["nnb"]), k
        assert same_sets(canon_gpu(*_rows(ctx)), canon_oracle(o["off"], o["idx"], o["ng"])), k
        errs = {f: normwise(host(arr[f]), o[f]) for f in ("rho", "p", "c")}
        errs.update({f: force_err(f, host(arr[f]), o[f], o, p.periodic_z)
                     for f in ("ax", "ay", "az", "du", "mumax")})
        check(errs, TOL_FP64)


@pytest.mark.parametrize("case", ["patch", "evrard"])
def test_stale_lists_are_rebuilt(B, case):
    # after a few steps every particle moves by half its h: the kept lists no
    # longer cover the neighbourhoods, the step rebuilds them, and its results
    # are the bits of a fresh context on the same state
    s, p = _case(case)
    n = len(s["x"])
    ctx = B.Context(n)
    arr = B.alloc_arrays(s)
    ctx.step(p, arr, nsteps=3)
    ctx.sync()
    st = _state(arr)
    rng = np.random.Generator(np.random.PCG64(7))
    for f in ("x", "y"):
        st[f] = st[f] + 0.5 * st["h"] * rng.choice([-1.0, 1.0], size=n)
    _load(arr, st)
    b0 = ctx.list_builds()
    ctx.step(p, arr, nsteps=1)
    assert ctx.list_builds() == b0 + 1  # this step rebuilt
    fresh = B.Context(n)
    ref = B.alloc_arrays(st)
    fresh.step(p, ref, nsteps=1)
    assert ctx.sync() == fresh.sync()
    for f in STATE + OUTS + ("nnb",):
        assert np.array_equal(host(arr[f]).view(np.uint8), host(ref[f]).view(np.uint8)), f


def test_list_hands_over_to_the_cell_walk(B):
    # h cut to 40 % for every third particle: its bisection grows h past the
    # radius its kept list covers, and the particle finishes with a cell walk
    s, p_on = _case("patch")
    _, p_off = _case("patch", skin=-1.0)
    n = len(s["x"])
    on, off = B.Context(n), B.Context(n)
    a_on, a_off = B.alloc_arrays(s), B.alloc_arrays(s)
    on.step(p_on, a_on, nsteps=2)
    on.sync()
    st = _state(a_on)
    st["h"][::3] *= 0.4
    _load(a_on, st)
    _load(a_off, st)
    on.step(p_on, a_on, nsteps=1)
    off.step(p_off, a_off, nsteps=1)
    assert on.sync() == off.sync()
    assert np.array_equal(host(a_on["h"]).view(np.int64), host(a_off["h"]).view(np.int64))
    assert np.array_equal(host(a_on["nnb"]), host(a_off["nnb"]))
    assert same_sets(canon_gpu(*_rows(on)), canon_gpu(*_rows(off)))


def test_lists_clear_gives_fresh_context_bits(B):
    s, p = _case("evrard")
    n = len(s["x"])
    ctx = B.Context(n)
    arr = B.alloc_arrays(s)
    ctx.step(p, arr, nsteps=3)
    ctx.sync()
    # the same initial state again: cleared lists reproduce a fresh context
    again = B.alloc_arrays(s)
    ctx.lists_clear()
    ctx.step(p, again, nsteps=3)
    fresh = B.Context(n)
    ref = B.alloc_arrays(s)
    fresh.step(p, ref, nsteps=3)
    ctx.sync()
    fresh.sync()
    for f in STATE + OUTS + ("nnb", "dt", "time"):
        assert np.array_equal(host(again[f]).view(np.uint8), host(ref[f]).view(np.uint8)), f
    for first, count in ((n - 1, 2 + ctx.n_capacity), (1, 2 ** 63 - 1), (-1, 1), (2 ** 62, 1)):
        with pytest.raises(B.SphError) as e:  # (first + count overflowing int64 too)
            ctx.lists_clear(first, count)
        assert e.value.status == B.SPH_E_INVAL


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_split_calls_and_batches_keep_the_bits(B, precision):
    # the lists travel with the context: 2 + 4 steps in two calls give the
    # bits of 6 in one, and an instance in a batch those of the same instance
    # alone (its lists and its rebuilds are its own)
    a, pa = _case("patch", precision=precision)
    b, pb = _case("evrard", precision=precision)
    one = B.Context(len(a["x"]))
    x1 = B.alloc_arrays(a)
    one.step(pa, x1, nsteps=6)
    two = B.Context(len(a["x"]))
    x2 = B.alloc_arrays(a)
    two.step(pa, x2, nsteps=2)
    two.step(pa, x2, nsteps=4)
    one.sync()
    two.sync()
    for f in x1:
        assert np.array_equal(host(x1[f]).view(np.uint8), host(x2[f]).view(np.uint8)), f
    counts = [len(b["x"]), len(a["x"])]
    ctx = B.Context(sum(counts), max_instances=2)
    ctx.batch_set(counts, [pb, pa])
    st = {k: np.concatenate([b[k], a[k]]) for k in B.STATE_FIELDS}
    arr = B.alloc_arrays(st, ninst=2)
    ctx.batch_step(arr, nsteps=3)
    ctx.batch_step(arr, nsteps=3)
    ctx.sync()
    sl = slice(counts[0], None)
    for f in STATE + OUTS:
        assert np.array_equal(host(arr[f])[sl].view(np.uint8), host(x1[f]).view(np.uint8)), f
