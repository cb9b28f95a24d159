"""Parity of the Table 1 variants on the GPU (Wendland C2 and sinc kernels, IAD
gradients) and of the Section 5.1.1 pressure initial conditions with the CPU
oracle: FP64 fields within 1e-12 normwise per call and per step from
identical inputs, bit-exact h; the variants run alone and batched with the
same bits; invalid combinations are rejected before any launch."""
import dataclasses

import numpy as np
import pytest

from paper_1809_08013_gb300 import ics
from parity_util import TOL_FP64, check, force_err, normwise, state_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

FORCES = ("ax", "ay", "az", "du", "mumax")

# (kernel, gradients, sinc_n) and the precision: 2 runs every variant in the
# FP64-pipe kernels, 0 in the double-float kernels
VARIANTS = [((1, 0, 5), 2), ((2, 0, 5), 2), ((0, 1, 5), 2), ((1, 1, 5), 2), ((2, 1, 6), 2),
            ((2, 0, 5), 0), ((0, 1, 5), 0), ((1, 1, 5), 0), ((2, 1, 6), 0)]
INPUTS = ["patch_ragged_av", "evrard12k"]


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_08013_gb300 import binding
    binding.load()
    return binding


def _input(name):
    if name == "patch_ragged_av":
        s, p = ics.square_patch(17, seed=15)
        return ics.random_velocities(s, seed=16, scale=2.0), p
    if name == "evrard12k":
        s, p = ics.evrard(12000, seed=17)
        return ics.random_velocities(s, seed=18, scale=0.3), p
    raise KeyError(name)


_ORC = {}


def oracle_of(orc, name, var, precision=2):
    key = (name, var, precision)
    if key not in _ORC:
        s, p = _input(name)
        p.kernel, p.gradients, p.sinc_n = var
        p.precision = precision
        _ORC[key] = (s, p, orc.pipeline(p, s))
    return _ORC[key]


def host(t):
    return t.detach().cpu().numpy()


def _check_forces(arr, o, prm):
    check({k: force_err(k, host(arr[k]), o[k], o, prm.periodic_z) for k in FORCES}, TOL_FP64)


@pytest.mark.parametrize("name", INPUTS)
@pytest.mark.parametrize("var,prec", VARIANTS)
def test_variant_density_forces_from_identical_inputs(B, orc, name, var, prec):
    s, prm, o = oracle_of(orc, name, var, precision=prec)
    ctx = B.Context(len(s["x"]))
    arr = B.alloc_arrays(s)
    ctx.build_neighbors(prm, arr)
    assert np.array_equal(host(arr["h"]).view(np.int64), o["h"].view(np.int64))
    ctx.density(prm, arr)
    assert normwise(host(arr["rho"]), o["rho"]) <= TOL_FP64
    for k in ("rho", "p", "c"):
        arr[k].copy_(torch.from_numpy(o[k]))
    ctx.forces(prm, arr)
    assert ctx.sync() in (B.SPH_OK, B.SPH_E_HNOCONV)
    _check_forces(arr, o, prm)
    assert abs(host(arr["dt"])[0] - o["dt"]) <= TOL_FP64 * o["dt"]


@pytest.mark.parametrize("name", INPUTS)
@pytest.mark.parametrize("var,prec", VARIANTS)
def test_variant_one_step_matches_oracle(B, orc, name, var, prec):
    s, prm, o = oracle_of(orc, name, var, precision=prec)
    st_o, ex = orc.step(prm, s, nsteps=1)
    ctx = B.Context(len(s["x"]))
    arr = B.alloc_arrays(s)
    ctx.step(prm, arr, nsteps=1)
    assert ctx.sync() in (B.SPH_OK, B.SPH_E_HNOCONV)
    per = prm.periodic_z
    err = {k: state_err(k, host(arr[k]), st_o[k], o, per, ex["dt"])
           for k in ("x", "y", "z", "vx", "vy", "vz", "u")}
    err.update({k: normwise(host(arr[k]), ex[k]) for k in ("rho", "p", "c")})
    err.update({k: force_err(k, host(arr[k]), ex[k], o, per) for k in FORCES})
    check(err, TOL_FP64)
    assert np.array_equal(host(arr["h"]).view(np.int64), st_o["h"].view(np.int64))
    assert abs(host(arr["dt"])[0] - ex["dt"]) <= TOL_FP64 * ex["dt"]


@pytest.mark.parametrize("var", [(1, 0, 5), (2, 0, 3), (0, 1, 5), (1, 1, 5), (2, 1, 8)])
@pytest.mark.parametrize("lanes", [1, 4])
@pytest.mark.parametrize("name", INPUTS)
def test_double_float_variants_with_lanes(B, orc, name, lanes, var):
    # the variants at precision 0 run in the double-float kernels: per call
    # and one step against the oracle with 1 and 4 lanes per particle
    s, prm0, o = oracle_of(orc, name, var, precision=0)
    prm = dataclasses.replace(prm0, pair_threads=lanes)  # the cached parameters stay as they are
    ctx = B.Context(len(s["x"]))
    arr = B.alloc_arrays(s)
    ctx.build_neighbors(prm, arr)
    ctx.density(prm, arr)
    assert normwise(host(arr["rho"]), o["rho"]) <= TOL_FP64
    for k in ("rho", "p", "c"):
        arr[k].copy_(torch.from_numpy(o[k]))
    ctx.forces(prm, arr)
    assert ctx.sync() in (B.SPH_OK, B.SPH_E_HNOCONV)
    _check_forces(arr, o, prm)
    st_o, ex = orc.step(prm, s, nsteps=1)
    arr = B.alloc_arrays(s)
    ctx.step(prm, arr, nsteps=1)
    assert ctx.sync() in (B.SPH_OK, B.SPH_E_HNOCONV)
    err = {k: normwise(host(arr[k]), ex[k]) for k in ("rho", "p", "c")}
    err.update({k: force_err(k, host(arr[k]), ex[k], o, prm.periodic_z) for k in FORCES})
    check(err, TOL_FP64)
    # and it is not the native FP64 kernel (different rounding, same values)
    prm.precision = 2
    arr2 = B.alloc_arrays(s)
    ctx.step(prm, arr2, nsteps=1)
    ctx.sync()
    assert not np.array_equal(host(arr2["ax"]), host(arr["ax"]))


@pytest.mark.parametrize("var", [(1, 0, 5), (2, 0, 5), (0, 1, 5), (2, 1, 5)])
def test_precision_0_and_2_take_different_kernels(B, var):
    # precision 0 (double-float) and 2 (FP64 pipe) round differently: the
    # variant really runs in the kernels its precision names
    s, prm = _input("patch_ragged_av")
    prm.kernel, prm.gradients, prm.sinc_n = var
    out = []
    for prec in (0, 2):
        prm.precision = prec
        ctx = B.Context(len(s["x"]))
        arr = B.alloc_arrays(s)
        ctx.step(prm, arr, nsteps=1)
        assert ctx.sync() in (B.SPH_OK, B.SPH_E_HNOCONV)
        out.append(host(arr["ax"]))
    assert not np.array_equal(out[0], out[1])


@pytest.mark.parametrize("field,value", [("kernel", 3), ("kernel", -1), ("gradients", 2),
                                         ("sinc_n", 1), ("sinc_n", 13)])
def test_invalid_variant_is_rejected(B, field, value):
    s, prm = _input("patch_ragged_av")
    prm.kernel = 2  # so that sinc_n is read
    setattr(prm, field, value)
    ctx = B.Context(len(s["x"]))
    arr = B.alloc_arrays(s)
    l0 = ctx.launch_count()
    with pytest.raises(B.SphError) as e:
        ctx.step(prm, arr, nsteps=1)
    assert e.value.status == B.SPH_E_INVAL
    assert ctx.launch_count() == l0


@pytest.mark.parametrize("var", [(1, 0, 5), (0, 1, 5)])
def test_mixed_precision_rejects_variants(B, var):
    s, prm = _input("patch_ragged_av")
    prm.kernel, prm.gradients, prm.sinc_n = var
    prm.precision = 1
    ctx = B.Context(len(s["x"]))
    arr = B.alloc_arrays(s)
    with pytest.raises(B.SphError) as e:
        ctx.step(prm, arr, nsteps=1)
    assert e.value.status == B.SPH_E_INVAL


@pytest.mark.parametrize("var", [(2, 1, 4), (1, 1, 5)])
def test_variants_batched_equal_alone(B, var):
    # two IAD instances of different sizes in one batch (sinc on the FP64 pipe,
    # Wendland in double-float): each equals its run alone
    insts = []
    for k, side in enumerate((9, 14)):
        s, p = ics.square_patch(side, seed=200 + k, omega=3.0 + k)
        s = ics.random_velocities(s, seed=210 + k, scale=1.0)
        p.kernel, p.gradients, p.sinc_n = var
        insts.append((s, p))
    alone = []
    for s, p in insts:
        ctx = B.Context(len(s["x"]))
        arr = B.alloc_arrays(s)
        ctx.step(p, arr, nsteps=3)
        ctx.sync()
        alone.append({k: host(arr[k]) for k in ("x", "vy", "u", "h", "rho", "ax", "du")})
    cat = {k: np.concatenate([s[k] for s, _ in insts]) for k in insts[0][0]}
    counts = [len(s["x"]) for s, _ in insts]
    ctx = B.Context(sum(counts), max_instances=4)
    arr = B.alloc_arrays(cat, ninst=2)
    ctx.batch_set(counts, [p for _, p in insts])
    ctx.batch_step(arr, nsteps=3)
    assert ctx.sync() in (B.SPH_OK, B.SPH_E_HNOCONV)
    a = 0
    for k, c in enumerate(counts):
        for f, ref in alone[k].items():
            got = host(arr[f])[a:a + c]
            assert np.array_equal(got.view(np.uint8), ref.view(np.uint8)), (k, f)
        a += c


def test_batch_rejects_mixed_variants(B):
    s, p = ics.square_patch(8, seed=1)
    q = ics.SphParams(**p.as_dict())
    q.gradients = 1
    ctx = B.Context(2 * len(s["x"]), max_instances=4)
    with pytest.raises(B.SphError) as e:
        ctx.batch_set([len(s["x"])] * 2, [p, q])
    assert e.value.status == B.SPH_E_INVAL


@pytest.mark.parametrize("var", [(0, 0, 5), (1, 1, 5)])
def test_pressure_initial_conditions_one_step(B, orc, var):
    # variable masses from the series pressure (Section 5.1.1)
    s, prm = ics.square_patch(16, seed=220, pressure_ic=True)
    prm.kernel, prm.gradients, prm.sinc_n = var
    o = orc.pipeline(prm, s)
    st_o, ex = orc.step(prm, s, nsteps=1)
    ctx = B.Context(len(s["x"]))
    arr = B.alloc_arrays(s)
    ctx.step(prm, arr, nsteps=1)
    assert ctx.sync() in (B.SPH_OK, B.SPH_E_HNOCONV)
    assert np.array_equal(host(arr["h"]).view(np.int64), st_o["h"].view(np.int64))
    err = {k: normwise(host(arr[k]), ex[k]) for k in ("rho", "p")}
    err.update({k: force_err(k, host(arr[k]), ex[k], o, prm.periodic_z) for k in FORCES})
    check(err, TOL_FP64)
