"""Particles outside the geometry range of the neighbour search (a NaN or an
infinity anywhere in the state, a coordinate beyond the FP32 range, h outside
[0, 2^100]) are reported as SPH_E_NONFINITE and stay contained: the step runs
to its end with every access in bounds, the other particles keep their h and
neighbour counts bit for bit, and the context stays usable."""
import numpy as np
import pytest

from paper_1809_08013_gb300 import ics

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

NAN, INF = float("nan"), float("inf")
# (field, value): the first group leaves a particle's position or h outside
# the geometry range, the second only its dynamics
GEOMETRY_BAD = [("x", NAN), ("z", 1e39), ("y", -INF), ("h", INF), ("h", -1.0), ("h", NAN)]
STATE_BAD = [("vz", NAN), ("u", -INF), ("m", NAN), ("vx", INF)]


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_08013_gb300 import binding
    binding.load()
    return binding


def _case(name, precision):
    if name == "patch":  # periodic z
        s, prm = ics.square_patch(13, seed=61)
        s = ics.random_velocities(s, seed=62, scale=1.0)
    else:
        s, prm = ics.evrard(3000, seed=63)
    prm.precision = precision
    return s, prm


def _spoil(s, seed):
    n = len(s["x"])
    rng = np.random.Generator(np.random.PCG64(seed))
    idx = rng.choice(n, size=len(GEOMETRY_BAD) + len(STATE_BAD), replace=False)
    bad = {k: np.array(v, copy=True) for k, v in s.items()}
    for k, (f, v) in zip(idx, GEOMETRY_BAD + STATE_BAD):
        bad[f][k] = v
    return bad, idx[:len(GEOMETRY_BAD)], idx[len(GEOMETRY_BAD):]


@pytest.mark.parametrize("precision", [0, 1, 2])
@pytest.mark.parametrize("case", ["patch", "evrard"])
def test_others_keep_their_h_and_counts(B, case, precision):
    s, prm = _case(case, precision)
    bad, gidx, _ = _spoil(s, seed=7 + precision)
    ctx = B.Context(len(s["x"]))
    arr = B.alloc_arrays(bad)
    ctx.build_neighbors(prm, arr)
    assert ctx.sync() == B.SPH_E_NONFINITE
    h, nnb = arr["h"].cpu().numpy(), arr["nnb"].cpu().numpy()
    # reference: the particles whose position is out of range removed (never
    # anyone's neighbour), the h-spoiled ones given back their h (a finite
    # position is a candidate for the others whatever its own h)
    pos_bad = [k for k, (f, _) in zip(gidx, GEOMETRY_BAD) if f != "h"]
    ref = {k: np.delete(np.array(v, copy=True), pos_bad) for k, v in s.items()}
    keep = np.setdiff1d(np.arange(len(s["x"])), pos_bad)
    rctx = B.Context(len(keep))
    rarr = B.alloc_arrays(ref)
    rctx.build_neighbors(prm, rarr)
    assert rctx.sync() in (B.SPH_OK, B.SPH_E_HNOCONV)
    rh, rn = rarr["h"].cpu().numpy(), rarr["nnb"].cpu().numpy()
    mine = np.isin(keep, gidx, invert=True)  # drop the h-spoiled ones themselves
    assert np.array_equal(h[keep][mine].view(np.uint64), rh[mine].view(np.uint64))
    assert np.array_equal(nnb[keep][mine], rn[mine])
    assert (nnb[gidx] == 0).all()  # out of range: no search, no neighbours


@pytest.mark.parametrize("precision", [0, 1, 2])
@pytest.mark.parametrize("case", ["patch", "evrard"])
def test_step_reports_and_context_stays_usable(B, case, precision):
    s, prm = _case(case, precision)
    bad, _, _ = _spoil(s, seed=11 + precision)
    if case == "patch":  # far outside the periodic box, but a finite float
        bad["z"][0] = 1e30
    ctx = B.Context(len(s["x"]))
    arr = B.alloc_arrays(bad)
    ctx.step(prm, arr, nsteps=3)
    assert ctx.sync() == B.SPH_E_NONFINITE
    # the same context on clean input gives the bits of a fresh one
    a1 = B.alloc_arrays(s)
    ctx.step(prm, a1, nsteps=2)
    st1 = ctx.sync()
    fresh = B.Context(len(s["x"]))
    a2 = B.alloc_arrays(s)
    fresh.step(prm, a2, nsteps=2)
    assert fresh.sync() == st1 and st1 in (B.SPH_OK, B.SPH_E_HNOCONV)
    for k in ("x", "y", "z", "vx", "vy", "vz", "h", "u", "rho", "ax", "az", "du", "nnb", "dt"):
        assert np.array_equal(a1[k].cpu().numpy(), a2[k].cpu().numpy()), k


@pytest.mark.parametrize("precision", [0, 2])
def test_every_particle_out_of_range(B, precision):
    s, prm = _case("evrard", precision)
    n = len(s["x"])
    for f in ("x", "y", "z"):
        s[f] = np.full(n, NAN)
    ctx = B.Context(n)
    arr = B.alloc_arrays(s)
    ctx.step(prm, arr, nsteps=2)
    assert ctx.sync() == B.SPH_E_NONFINITE
    assert (arr["nnb"].cpu().numpy() == 0).all()
