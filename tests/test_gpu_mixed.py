"""Parity of the mixed-precision pair kernels (precision = 1: FP32 relative
coordinates, FP32 kernel, gradient and viscosity terms, double-float sums;
positions, h, neighbour sets, dt and integration in FP64) with the FP64
oracle on the Evrard collapse (Section 5.1.2, hydrodynamics only) and the
rotating square patch.

Bar: density and acceleration within 1e-5 (normwise; only the cancelling sums
-- du, mu and the periodic patch's a_z -- against the magnitude of their
terms, as for the FP64 path). Every other field is
checked at the same bar and its error printed. The neighbour search does not
depend on the precision, so h and the neighbour sets stay bit-exact.
"""
import numpy as np
import pytest

from paper_1809_08013_gb300 import ics
from parity_util import (TOL_FP64, canon_gpu, canon_oracle, force_err, normwise, same_sets,
                         state_err)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL_MIXED = 1e-5
MIXED = 1
FORCES = ("ax", "ay", "az", "du", "mumax")


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_08013_gb300 import binding
    binding.load()
    return binding


def host(t):
    return t.detach().cpu().numpy()


def _case(name):
    if name == "evrard20k":
        s, p = ics.evrard(20000, seed=3)
    elif name == "evrard_moving":
        s, p = ics.evrard(12000, seed=11)
        s = ics.random_velocities(s, seed=12, scale=0.3)
    elif name == "patch27k":
        s, p = ics.square_patch(30, seed=1)
    elif name == "patch_ragged_av":
        s, p = ics.square_patch(17, seed=5)
        s = ics.random_velocities(s, seed=6, scale=2.0)
    else:
        raise KeyError(name)
    p.precision = MIXED
    return s, p


CASES = ["evrard20k", "evrard_moving", "patch27k", "patch_ragged_av"]
_ORC = {}


def oracle_of(orc, name):
    if name not in _ORC:
        s, prm = _case(name)
        _ORC[name] = (s, prm, orc.pipeline(prm, s))
    return _ORC[name]


def field_errors(arr, o, periodic_z, sc=None):
    """Per-field errors against the oracle values o; the summed-term scales
    of the cancelling fields come from sc (default o: a pipeline run on the
    same inputs)."""
    sc = o if sc is None else sc
    err = {k: normwise(host(arr[k]), o[k]) for k in ("rho", "p", "c")}
    err.update({k: force_err(k, host(arr[k]), o[k], sc, periodic_z) for k in FORCES})
    return err


@pytest.mark.parametrize("name", CASES)
def test_mixed_per_call_from_identical_inputs(B, orc, name):
    s, prm, o = oracle_of(orc, name)
    ctx = B.Context(len(s["x"]))
    arr = B.alloc_arrays(s)
    ctx.build_neighbors(prm, arr)
    ctx.sync()
    assert np.array_equal(host(arr["h"]).view(np.int64), o["h"].view(np.int64))
    ctx.density(prm, arr)
    e_rho = normwise(host(arr["rho"]), o["rho"])
    arr["rho"].copy_(torch.from_numpy(o["rho"]))
    arr["p"].copy_(torch.from_numpy(o["p"]))
    arr["c"].copy_(torch.from_numpy(o["c"]))
    ctx.forces(prm, arr)
    assert ctx.sync() in (B.SPH_OK, B.SPH_E_HNOCONV)
    err = field_errors(arr, o, prm.periodic_z)
    err["rho"] = e_rho
    err["dt"] = abs(host(arr["dt"])[0] - o["dt"]) / o["dt"]
    print(name, {k: f"{v:.2e}" for k, v in err.items()})
    for k in ("rho", "ax", "ay", "az", "du", "mumax", "dt"):
        assert err[k] <= TOL_MIXED, (k, err[k])


@pytest.mark.parametrize("name", CASES)
def test_mixed_one_step(B, orc, name):
    s, prm, o = oracle_of(orc, name)
    st_o, ex = orc.step(prm, s, nsteps=1)
    ctx = B.Context(len(s["x"]))
    arr = B.alloc_arrays(s)
    ctx.step(prm, arr, nsteps=1)
    assert ctx.sync() in (B.SPH_OK, B.SPH_E_HNOCONV)
    assert np.array_equal(host(arr["h"]).view(np.int64), st_o["h"].view(np.int64))
    err = field_errors(arr, ex, prm.periodic_z, o)
    err.update({k: state_err(k, host(arr[k]), st_o[k], o, prm.periodic_z, ex["dt"])
                for k in ("x", "y", "z", "vx", "vy", "vz", "u")})
    err["dt"] = abs(host(arr["dt"])[0] - ex["dt"]) / ex["dt"]
    print(name, {k: f"{v:.2e}" for k, v in err.items()})
    for k, v in err.items():
        assert v <= TOL_MIXED, (k, v)


@pytest.mark.parametrize("tpp", [1, 4])
def test_mixed_with_several_lanes_per_particle(B, orc, tpp):
    s, prm, o = oracle_of(orc, "evrard_moving")
    prm = ics.SphParams(**{**prm.as_dict(), "pair_threads": tpp})
    ctx = B.Context(len(s["x"]))
    arr = B.alloc_arrays(s)
    ctx.step(prm, arr, nsteps=1)
    ctx.sync()
    err = field_errors(arr, o, prm.periodic_z)
    for k in ("rho", "ax", "ay", "az", "du", "mumax"):
        assert err[k] <= TOL_MIXED, (k, err[k])


def test_mixed_is_a_distinct_path(B, orc):
    # the FP32 pair terms leave a trace well above the FP64 path's round-off:
    # a dispatch that silently ran the FP64 kernels would fail here
    s, prm, o = oracle_of(orc, "evrard20k")
    ctx = B.Context(len(s["x"]))
    arr = B.alloc_arrays(s)
    ctx.step(prm, arr, nsteps=1)
    ctx.sync()
    assert normwise(host(arr["rho"]), o["rho"]) > 100 * TOL_FP64


def test_mixed_evrard_at_rest_has_no_viscosity(B, orc):
    # v = 0: every v_ij . r_ij is exactly zero, so mu, Pi and du vanish bitwise
    s, prm, o = oracle_of(orc, "evrard20k")
    ctx = B.Context(len(s["x"]))
    arr = B.alloc_arrays(s)
    ctx.step(prm, arr, nsteps=1)
    ctx.sync()
    assert np.max(np.abs(o["du"])) == 0.0 and np.max(np.abs(o["mumax"])) == 0.0
    assert np.max(np.abs(host(arr["du"]))) == 0.0
    assert np.max(np.abs(host(arr["mumax"]))) == 0.0


def test_mixed_full_size_evrard_1m(B, orc):
    # the mixed-precision workload: Evrard sphere, 10^6 particles, one step
    # through sph_step, every field against the FP64 oracle
    s, prm = ics.evrard(1_000_000, seed=3)
    prm.precision = MIXED
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
    err = field_errors(arr, o, prm.periodic_z)
    err.update({k: state_err(k, host(arr[k]), st_o[k], o, prm.periodic_z, o["dt"])
                for k in ("x", "y", "z", "vx", "vy", "vz", "u")})
    err["dt"] = abs(host(arr["dt"])[0] - o["dt"]) / o["dt"]
    print("evrard1m", {k: f"{v:.2e}" for k, v in err.items()})
    for k, v in err.items():
        assert v <= TOL_MIXED, (k, v)


def test_invalid_precision_rejected(B):
    s, prm = _case("evrard20k")
    prm.precision = 3
    ctx = B.Context(len(s["x"]))
    arr = B.alloc_arrays(s)
    with pytest.raises(B.SphError) as e:
        ctx.step(prm, arr, nsteps=1)
    assert e.value.status == B.SPH_E_INVAL
