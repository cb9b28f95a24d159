"""Parity of the CUDA path (through the C ABI) with the CPU oracle on the same
seeded inputs: bit-exact h and neighbour sets, FP64 fields within 1e-12
normwise, per call and per step from identical inputs; plus edge cases.

Workloads (Section 5.1): the rotating square patch at 30^3 (27,000 particles,
one step) and 100^3 (1,000,000, the benchmark size), a ragged 17^3 patch with
random velocities (viscosity active), a variable-h patch, and an Evrard
sphere of 20,000 particles.
"""
import numpy as np
import pytest

from paper_1809_08013_gb300 import ics
from parity_util import (TOL_FP64, canon_gpu, canon_oracle, check, force_err, normwise,
                         same_sets, state_err)

FORCES = ("ax", "ay", "az", "du", "mumax")

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_08013_gb300 import binding
    binding.load()
    return binding


def _case(name):
    if name == "patch27k":
        return ics.square_patch(30, seed=1)
    if name == "patch_ragged_av":
        s, p = ics.square_patch(17, seed=5)
        return ics.random_velocities(s, seed=6, scale=2.0), p
    if name == "patch_varh":
        s, p = ics.square_patch(20, seed=7)
        s = ics.perturb_h(s, seed=8, rel=0.3)
        return ics.random_velocities(s, seed=9, scale=1.0), p
    if name == "evrard20k":
        return ics.evrard(20000, seed=3)
    raise KeyError(name)


CASES = ["patch27k", "patch_ragged_av", "patch_varh", "evrard20k"]
_ORC = {}


def oracle_of(orc, name):
    if name not in _ORC:
        s, prm = _case(name)
        _ORC[name] = (s, prm, orc.pipeline(prm, s), orc.h_iterate(prm, s["x"], s["y"], s["z"], s["h"])[3])
    return _ORC[name]


def host(t):
    return t.detach().cpu().numpy()


def gpu_build(B, prm, s, ctx=None):
    ctx = ctx or B.Context(len(s["x"]))
    arr = B.alloc_arrays(s)
    ctx.build_neighbors(prm, arr)
    st = ctx.sync()
    return ctx, arr, st


@pytest.mark.parametrize("name", CASES)
def test_neighbors_bit_exact(B, orc, name):
    s, prm, o, bad = oracle_of(orc, name)
    ctx, arr, st = gpu_build(B, prm, s)
    assert st == (B.SPH_E_HNOCONV if bad else B.SPH_OK)
    assert np.array_equal(host(arr["h"]).view(np.int64), o["h"].view(np.int64))
    assert np.array_equal(host(arr["nnb"]), o["nnb"])
    off, idx, ng, order = ctx.neighbors_to_host()
    assert np.array_equal(np.sort(order), np.arange(len(order)))
    assert off[-1] == o["off"][-1]
    assert same_sets(canon_gpu(off, idx, ng, order), canon_oracle(o["off"], o["idx"], o["ng"]))


def _parts_sorted(off, idx, ng):
    return all(np.all(np.diff(idx[off[r]:off[r] + ng[r]]) > 0) and
               np.all(np.diff(idx[off[r] + ng[r]:off[r + 1]]) > 0) for r in range(len(off) - 1))


@pytest.mark.parametrize("name", CASES[:2])
def test_caller_order_export_equals_oracle(B, orc, name):
    # rows of sph_neighbors_to_host_caller are the caller's particles: the row
    # lengths and gather counts equal the oracle's entry by entry
    s, prm, o, _ = oracle_of(orc, name)
    ctx, arr, st = gpu_build(B, prm, s)
    n = len(s["x"])
    off, idx, ng = ctx.neighbors_caller(n)
    assert np.array_equal(off, o["off"]) and np.array_equal(ng, o["ng"])
    assert _parts_sorted(off, idx, ng)
    ident = np.arange(n, dtype=np.int32)
    assert same_sets(canon_gpu(off, idx, ng, ident), canon_oracle(o["off"], o["idx"], o["ng"]))
    # and it is the internal export permuted
    off2, idx2, ng2, order = ctx.neighbors_to_host()
    assert same_sets(canon_gpu(off, idx, ng, ident), canon_gpu(off2, idx2, ng2, order))


@pytest.mark.parametrize("name", CASES)
def test_density_eos_forces_from_identical_inputs(B, orc, name):
    s, prm, o, _ = oracle_of(orc, name)
    ctx, arr, st = gpu_build(B, prm, s)
    ctx.density(prm, arr)
    assert normwise(host(arr["rho"]), o["rho"]) <= TOL_FP64
    # EOS and forces from the oracle's density, pressure and sound speed
    arr["rho"].copy_(torch.from_numpy(o["rho"]))
    ctx.eos(prm, arr)
    assert normwise(host(arr["p"]), o["p"]) <= TOL_FP64
    assert normwise(host(arr["c"]), o["c"]) <= TOL_FP64
    arr["p"].copy_(torch.from_numpy(o["p"]))
    arr["c"].copy_(torch.from_numpy(o["c"]))
    ctx.forces(prm, arr)
    assert ctx.sync() in (B.SPH_OK, B.SPH_E_HNOCONV)
    check({k: force_err(k, host(arr[k]), o[k], o, prm.periodic_z) for k in FORCES}, TOL_FP64)
    assert abs(host(arr["dt"])[0] - o["dt"]) <= TOL_FP64 * o["dt"]


@pytest.mark.parametrize("name", CASES)
def test_one_step_matches_oracle(B, orc, name):
    s, prm, o, _ = oracle_of(orc, name)
    st_o, ex = orc.step(prm, s, nsteps=1)
    ctx = B.Context(len(s["x"]))
    arr = B.alloc_arrays(s)
    ctx.step(prm, arr, nsteps=1)
    ctx.sync()
    per = prm.periodic_z
    err = {k: state_err(k, host(arr[k]), st_o[k], o, per, ex["dt"])
           for k in ("x", "y", "z", "vx", "vy", "vz", "u")}
    err.update({k: normwise(host(arr[k]), ex[k]) for k in ("rho", "p", "c")})
    err.update({k: force_err(k, host(arr[k]), ex[k], o, per) for k in FORCES})
    check(err, TOL_FP64)
    assert np.array_equal(host(arr["h"]).view(np.int64), st_o["h"].view(np.int64))
    assert abs(host(arr["dt"])[0] - ex["dt"]) <= TOL_FP64 * ex["dt"]
    assert abs(host(arr["time"])[0] - ex["time"]) <= TOL_FP64 * ex["time"]


@pytest.mark.parametrize("tpp", [1, 4, 8])
def test_one_step_with_several_lanes_per_particle(B, orc, tpp):
    # the pair sums split over tpp lanes per particle round differently but
    # stay within the FP64 bar
    s, prm, o, _ = oracle_of(orc, "patch_ragged_av")
    prm = ics.SphParams(**{**prm.as_dict(), "pair_threads": tpp})
    ctx = B.Context(len(s["x"]))
    arr = B.alloc_arrays(s)
    ctx.step(prm, arr, nsteps=1)
    ctx.sync()
    err = {k: normwise(host(arr[k]), o[k]) for k in ("rho", "p", "c")}
    err.update({k: force_err(k, host(arr[k]), o[k], o, prm.periodic_z) for k in FORCES})
    check(err, TOL_FP64)
    assert abs(host(arr["dt"])[0] - o["dt"]) <= TOL_FP64 * o["dt"]


def test_three_steps_drift_is_small(B, orc):
    # trajectories are reported as drift: an ulp-level position difference can
    # flip a count at a bisection boundary, so only a loose bound is held
    s, prm = _case("patch_ragged_av")
    st_o, ex = orc.step(prm, s, nsteps=3)
    ctx = B.Context(len(s["x"]))
    arr = B.alloc_arrays(s)
    ctx.step(prm, arr, nsteps=3)
    ctx.sync()
    for k in ("x", "y", "z", "vx", "vy", "vz"):
        assert normwise(host(arr[k]), st_o[k]) <= 1e-9, k
    flips = int(np.count_nonzero(host(arr["h"]) != st_o["h"]))
    assert flips <= len(s["x"]) // 100


def test_twenty_steps_drift_27k(B, orc, capsys):
    # 20 steps of the 30^3 patch, each side from its own previous state:
    # reported as drift, as trajectories may part at a bisection boundary (an
    # ulp-level position difference can flip a count). Positions against the
    # box size, velocities against the largest speed; the number of particles
    # whose h bits differ after the 20 steps is reported beside them.
    s, prm = _case("patch27k")
    st_o, ex = orc.step(prm, s, nsteps=20)
    ctx = B.Context(len(s["x"]))
    arr = B.alloc_arrays(s)
    ctx.step(prm, arr, nsteps=20)
    assert ctx.sync() == B.SPH_OK
    got = {k: host(arr[k]) for k in ("x", "y", "z", "vx", "vy", "vz", "h")}
    vmax = float(np.max(np.sqrt(st_o["vx"] ** 2 + st_o["vy"] ** 2 + st_o["vz"] ** 2)))
    drift = {k: float(np.max(np.abs(got[k] - st_o[k]))) for k in ("x", "y", "z")}
    drift.update({k: float(np.max(np.abs(got[k] - st_o[k]))) / vmax for k in ("vx", "vy", "vz")})
    flips = int(np.count_nonzero(got["h"] != st_o["h"]))
    with capsys.disabled():
        print(f"\n20-step drift, 30^3 patch: {drift}, h flips {flips} of {len(s['x'])}")
    assert all(v <= 1e-9 for v in drift.values()), drift
    assert flips <= len(s["x"]) // 100
    assert abs(host(arr["time"])[0] - ex["time"]) <= 1e-9 * ex["time"]


@pytest.mark.parametrize("precision", [0, 1])
def test_split_run_equals_one_run(B, precision):
    # the internal order is a function of the positions only (keys are sorted
    # in caller order), so 2 + 3 steps in two calls give the bits of 5 steps
    s, prm = _case("patch_ragged_av")
    prm = ics.SphParams(**{**prm.as_dict(), "precision": precision})
    ctx = B.Context(len(s["x"]))
    one = B.alloc_arrays(s)
    ctx.step(prm, one, nsteps=5)
    two = B.alloc_arrays(s)
    ctx.step(prm, two, nsteps=2)
    ctx.step(prm, two, nsteps=3)
    ctx.sync()
    for k in one:
        assert np.array_equal(host(one[k]).view(np.uint8), host(two[k]).view(np.uint8)), k


def test_deterministic(B):
    s, prm = _case("patch_ragged_av")
    outs = []
    for _ in range(2):
        ctx = B.Context(len(s["x"]))
        arr = B.alloc_arrays(s)
        ctx.step(prm, arr, nsteps=2)
        ctx.sync()
        outs.append({k: host(v).copy() for k, v in arr.items()})
    for k in outs[0]:
        assert np.array_equal(outs[0][k].view(np.uint8), outs[1][k].view(np.uint8)), k


def test_full_size_one_step_1m(B, orc):
    # the benchmark workload: 100^3 rotating patch, one full step through
    # sph_step, element by element against the oracle
    s, prm = ics.square_patch(100, seed=2)
    o = orc.pipeline(prm, s)
    s1 = dict(s)
    s1["h"] = o["h"]
    st_o = orc.leapfrog(prm, s1, o["dt"], o["ax"], o["ay"], o["az"], o["du"])
    ctx = B.Context(len(s["x"]))
    arr = B.alloc_arrays(s)
    ctx.step(prm, arr, nsteps=1)
    assert ctx.sync() == B.SPH_OK
    assert np.array_equal(host(arr["h"]).view(np.int64), o["h"].view(np.int64))
    assert np.array_equal(host(arr["nnb"]), o["nnb"])
    off, idx, ng, order = ctx.neighbors_to_host()
    assert same_sets(canon_gpu(off, idx, ng, order), canon_oracle(o["off"], o["idx"], o["ng"]))
    per = prm.periodic_z
    err = {k: normwise(host(arr[k]), o[k]) for k in ("rho", "p", "c")}
    err.update({k: force_err(k, host(arr[k]), o[k], o, per) for k in FORCES})
    err.update({k: state_err(k, host(arr[k]), st_o[k], o, per, o["dt"])
                for k in ("x", "y", "z", "vx", "vy", "vz", "u")})
    check(err, TOL_FP64)
    assert abs(host(arr["dt"])[0] - o["dt"]) <= TOL_FP64 * o["dt"]


def test_full_size_twenty_steps_1m(B, orc):
    # the benchmark's launch configuration: one sph_step(20) call on the 1M
    # patch (the step graph replayed 20 times). Its last step is checked
    # element by element against the oracle's step from the GPU's state after
    # 19 steps (a split run gives the bits of one call), and the 20 steps
    # against two conservation laws: central pair forces that are antisymmetric
    # in i and j, with a kick-drift update, keep the linear momentum and the
    # angular momentum about z exactly (the z image shift does not enter L_z).
    s, prm = ics.square_patch(100, seed=2)
    ctx = B.Context(len(s["x"]))
    a20 = B.alloc_arrays(s)
    ctx.step(prm, a20, nsteps=20)
    a19 = B.alloc_arrays(s)
    ctx.step(prm, a19, nsteps=19)
    assert ctx.sync() == B.SPH_OK
    s19 = {k: host(a19[k]).copy() for k in B.STATE_FIELDS}
    o = orc.pipeline(prm, s19)
    s1 = dict(s19)
    s1["h"] = o["h"]
    st_o = orc.leapfrog(prm, s1, o["dt"], o["ax"], o["ay"], o["az"], o["du"])
    assert np.array_equal(host(a20["h"]).view(np.int64), o["h"].view(np.int64))
    assert np.array_equal(host(a20["nnb"]), o["nnb"])
    per = prm.periodic_z
    err = {k: normwise(host(a20[k]), o[k]) for k in ("rho", "p", "c")}
    err.update({k: force_err(k, host(a20[k]), o[k], o, per) for k in FORCES})
    err.update({k: state_err(k, host(a20[k]), st_o[k], o, per, o["dt"])
                for k in ("x", "y", "z", "vx", "vy", "vz", "u")})
    check(err, TOL_FP64)
    assert abs(host(a20["dt"])[0] - o["dt"]) <= TOL_FP64 * o["dt"]
    # conservation over the 20 steps, against the magnitude of the summands
    m = s["m"]
    x, y, vx, vy, vz = (host(a20[k]) for k in ("x", "y", "vx", "vy", "vz"))
    for v0, v in ((s["vx"], vx), (s["vy"], vy), (s["vz"], vz)):
        assert abs(np.sum(m * v) - np.sum(m * v0)) <= 1e-12 * np.sum(m * np.abs(v))
    lz0 = np.sum(m * (s["x"] * s["vy"] - s["y"] * s["vx"]))
    lz = m * (x * vy - y * vx)
    assert abs(np.sum(lz) - lz0) <= 1e-12 * np.sum(np.abs(lz))
    # the time is the sum of the 20 steps' dt
    assert host(a20["time"])[0] > host(a19["time"])[0] > 0.0


# ---------------------------------------------------------------- edge cases
def test_empty_input(B):
    s = {k: np.zeros(0) for k in ics.FIELDS}
    prm = ics.SphParams()
    ctx = B.Context(16)
    arr = B.alloc_arrays(s)
    ctx.build_neighbors(prm, arr)
    ctx.step(prm, arr, nsteps=1)
    assert ctx.sync() == B.SPH_OK
    assert np.isinf(host(arr["dt"])[0])
    off, idx, ng, order = ctx.neighbors_to_host()
    assert off.tolist() == [0] and len(idx) == 0


def test_single_particle(B, orc):
    s = {k: np.zeros(1) for k in ics.FIELDS}
    s["m"][:] = 2.0
    s["h"][:] = 0.1
    prm = ics.SphParams(periodic_z=0, max_h_iter=6)
    ctx = B.Context(1)
    arr = B.alloc_arrays(s)
    ctx.step(prm, arr, nsteps=1)
    assert ctx.sync() == B.SPH_E_HNOCONV and ctx.last_hnoconv() == 1
    st_o, ex = orc.step(prm, s, nsteps=1)
    assert host(arr["h"])[0] == st_o["h"][0]
    assert host(arr["rho"])[0] == pytest.approx(ex["rho"][0], rel=1e-14)
    assert host(arr["ax"])[0] == 0.0 and host(arr["du"])[0] == 0.0
    assert host(arr["dt"])[0] == pytest.approx(ex["dt"], rel=1e-14)


def test_small_target_nonperiodic(B, orc):
    s, prm = ics.square_patch(4, seed=12)
    prm.periodic_z = 0
    prm.n_target, prm.n_tol = 10, 2
    o = orc.pipeline(prm, s)
    ctx, arr, st = gpu_build(B, prm, s)
    assert np.array_equal(host(arr["h"]).view(np.int64), o["h"].view(np.int64))
    off, idx, ng, order = ctx.neighbors_to_host()
    assert same_sets(canon_gpu(off, idx, ng, order), canon_oracle(o["off"], o["idx"], o["ng"]))


def test_perfect_lattice_reports_non_convergence(B, orc):
    s, prm = ics.square_patch(12, seed=0, jitter=0.0)
    prm.max_h_iter = 12
    h, nnb, conv, bad = orc.h_iterate(prm, s["x"], s["y"], s["z"], s["h"])
    ctx, arr, st = gpu_build(B, prm, s)
    assert st == B.SPH_E_HNOCONV
    assert ctx.last_hnoconv() == bad
    assert np.array_equal(host(arr["h"]).view(np.int64), h.view(np.int64))
    assert np.array_equal(host(arr["nnb"]), nnb)
    assert ctx.sync() == B.SPH_OK  # status cleared by the previous sync


def test_capacity_overflow_is_reported_not_fatal(B):
    # the step keeps its rows in per-particle slabs; the CSR of the neighbour
    # list (nnz_capacity entries) is only needed when a caller asks for it
    s, prm = _case("patch27k")
    ctx = B.Context(len(s["x"]), nnz_capacity=1000)
    arr = B.alloc_arrays(s)
    ctx.step(prm, arr, nsteps=1)
    assert ctx.sync() == B.SPH_OK
    ctx.build_neighbors(prm, arr)
    assert ctx.sync() == B.SPH_E_CAPACITY
    # a context with room works afterwards on the same device
    ctx2 = B.Context(len(s["x"]))
    arr2 = B.alloc_arrays(s)
    ctx2.step(prm, arr2, nsteps=1)
    assert ctx2.sync() == B.SPH_OK


def test_invalid_arguments_rejected(B):
    s, prm = ics.square_patch(5, seed=1)
    ctx = B.Context(10)
    arr = B.alloc_arrays(s)  # 125 > capacity 10
    with pytest.raises(B.SphError) as e:
        ctx.build_neighbors(prm, arr)
    assert e.value.status == B.SPH_E_INVAL
    ctx = B.Context(200)
    bad = ics.SphParams(eos=7)
    with pytest.raises(B.SphError):
        ctx.build_neighbors(bad, arr)
    # density before any build of this size
    with pytest.raises(B.SphError):
        ctx.density(prm, arr)


def test_slab_overflow_uses_full_build(B, orc):
    # 150 neighbours per particle exceed the 128-entry gather slab, so the
    # library takes its two-pass CSR build; results must not change
    s, prm = ics.square_patch(17, seed=21)
    prm.n_target = 150
    o = orc.pipeline(prm, s)
    ctx, arr, st = gpu_build(B, prm, s, ctx=B.Context(len(s["x"]), nnz_capacity=260 * len(s["x"])))
    assert st == B.SPH_OK
    assert np.array_equal(host(arr["h"]).view(np.int64), o["h"].view(np.int64))
    off, idx, ng, order = ctx.neighbors_to_host()
    assert same_sets(canon_gpu(off, idx, ng, order), canon_oracle(o["off"], o["idx"], o["ng"]))
    ctx.density(prm, arr)
    assert normwise(host(arr["rho"]), o["rho"]) <= TOL_FP64
    for k in ("rho", "p", "c"):
        arr[k].copy_(torch.from_numpy(o[k]))
    ctx.forces(prm, arr)  # the pair kernels read the fallback CSR
    check({k: force_err(k, host(arr[k]), o[k], o, prm.periodic_z) for k in FORCES}, TOL_FP64)
    # and a whole step through the fallback
    arr2 = B.alloc_arrays(s)
    ctx.step(prm, arr2, nsteps=1)
    assert ctx.sync() == B.SPH_OK
    err = {k: normwise(host(arr2[k]), o[k]) for k in ("rho", "p")}
    err.update({k: force_err(k, host(arr2[k]), o[k], o, prm.periodic_z) for k in FORCES})
    check(err, TOL_FP64)


@pytest.mark.parametrize("cell_scale", [0.5, 0.75, 1.5])
def test_neighbours_do_not_depend_on_cell_width(B, orc, cell_scale):
    s, prm, o, _ = oracle_of(orc, "patch_varh")
    prm2 = ics.SphParams(**prm.as_dict())
    prm2.cell_scale = cell_scale
    ctx, arr, st = gpu_build(B, prm2, s)
    assert np.array_equal(host(arr["h"]).view(np.int64), o["h"].view(np.int64))
    off, idx, ng, order = ctx.neighbors_to_host()
    assert same_sets(canon_gpu(off, idx, ng, order), canon_oracle(o["off"], o["idx"], o["ng"]))


def _moved(name):
    """Inputs far from the unit box: the chunk exponent, the FP32 border band
    of the h search and the periodic wrap all follow the coordinates' range."""
    if name == "evrard_translated":
        s, prm = ics.evrard(4000, seed=61)
        s = ics.random_velocities(s, seed=62, scale=0.5)
        s["x"] = s["x"] + 1000.0
        s["y"] = s["y"] - 500.0
        s["z"] = s["z"] + 250.0
        return s, prm
    s, prm = ics.square_patch(14, seed=63)
    s = ics.random_velocities(s, seed=64, scale=1.0)
    sc = 1e-6
    for k in ("x", "y", "z", "h"):
        s[k] = s[k] * sc
    s["m"] = s["m"] * sc ** 3   # the same density
    prm.lz = prm.lz * sc
    return s, prm


@pytest.mark.parametrize("name", ["evrard_translated", "patch_micro"])
@pytest.mark.parametrize("precision", [0, 2])
def test_far_from_unit_box(B, orc, name, precision):
    s, prm = _moved(name)
    prm.precision = precision
    o = orc.pipeline(prm, s)
    ctx, arr, st = gpu_build(B, prm, s)
    assert np.array_equal(host(arr["h"]).view(np.int64), o["h"].view(np.int64))
    off, idx, ng, order = ctx.neighbors_to_host()
    assert same_sets(canon_gpu(off, idx, ng, order), canon_oracle(o["off"], o["idx"], o["ng"]))
    ctx.density(prm, arr)
    assert normwise(host(arr["rho"]), o["rho"]) <= TOL_FP64
    for k in ("rho", "p", "c"):
        arr[k].copy_(torch.from_numpy(o[k]))
    ctx.forces(prm, arr)
    ctx.sync()
    check({k: force_err(k, host(arr[k]), o[k], o, prm.periodic_z) for k in FORCES}, TOL_FP64)
    assert abs(host(arr["dt"])[0] - o["dt"]) <= TOL_FP64 * o["dt"]


@pytest.mark.parametrize("precision", [0, 2])
@pytest.mark.parametrize("var", [(0, 0), (2, 1)])
def test_coincident_particles(B, orc, precision, var):
    # a particle and its copy at the same place (r = 0): the density counts
    # the copy at W(0), the forces and the IAD matrix skip the pair
    s, prm = ics.square_patch(12, seed=71)
    s = ics.random_velocities(s, seed=72, scale=1.0)
    s = {k: np.concatenate([v, v[[400, 900]]]) for k, v in s.items()}
    prm.precision = precision
    prm.kernel, prm.gradients = var
    o = orc.pipeline(prm, s)
    ctx, arr, st = gpu_build(B, prm, s)
    assert np.array_equal(host(arr["h"]).view(np.int64), o["h"].view(np.int64))
    ctx.density(prm, arr)
    assert normwise(host(arr["rho"]), o["rho"]) <= TOL_FP64
    for k in ("rho", "p", "c"):
        arr[k].copy_(torch.from_numpy(o[k]))
    ctx.forces(prm, arr)
    ctx.sync()
    check({k: force_err(k, host(arr[k]), o[k], o, prm.periodic_z) for k in FORCES}, TOL_FP64)
    assert np.all(np.isfinite(host(arr["ax"])))


def _dense_core():
    """A 16^3 lattice with a dense core of 300 particles at its centre: the
    lattice particles around the core count many core particles among their
    neighbours, while the core particles (small h) count few of them, so some
    rows of S_i are longer than the 224-entry row slab (225 here)."""
    a, p = ics.square_patch(16, seed=3)
    p.periodic_z = 0
    rng = np.random.Generator(np.random.PCG64(1))
    core = {k: np.zeros(300) for k in ics.FIELDS}
    core["x"], core["y"], core["z"] = (rng.uniform(-0.01, 0.01, 300) for _ in range(3))
    core["m"][:] = a["m"][0]
    core["h"][:] = 0.002
    s = {k: np.concatenate([a[k], core[k]]) for k in ics.FIELDS}
    return ics.random_velocities(s, seed=4, scale=1.0), p


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_long_rows_from_the_step(B, orc, precision):
    # at precisions 0 and 1 the step's density kernel decides the outer parts
    # itself; a row that overflows its slab must send the forces to the CSR
    # built after it
    s, prm = _dense_core()
    prm.precision = precision
    o = orc.pipeline(prm, s)
    assert int(np.max(np.diff(o["off"]))) > 224  # the input does overflow a slab
    st_o, ex = orc.step(prm, s, nsteps=1)
    ctx = B.Context(len(s["x"]))
    arr = B.alloc_arrays(s)
    ctx.step(prm, arr, nsteps=1)
    assert ctx.sync() == B.SPH_OK
    assert np.array_equal(host(arr["h"]).view(np.int64), o["h"].view(np.int64))
    off, idx, ng, order = ctx.neighbors_to_host()
    assert same_sets(canon_gpu(off, idx, ng, order), canon_oracle(o["off"], o["idx"], o["ng"]))
    per = prm.periodic_z
    err = {k: normwise(host(arr[k]), ex[k]) for k in ("rho", "p", "c")}
    err.update({k: force_err(k, host(arr[k]), ex[k], o, per) for k in FORCES})
    err.update({k: state_err(k, host(arr[k]), st_o[k], o, per, ex["dt"])
                for k in ("x", "y", "z", "vx", "vy", "vz", "u")})
    check(err, 1e-5 if precision == 1 else TOL_FP64)
