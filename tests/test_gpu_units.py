"""The pair kernels' own units (precision 0: float pairs; precision 1: FP32).

Both work in per-instance power-of-two units of length, mass and velocity
near the instance's mean h, largest mass and velocity scale, so the caller's
choice of units cannot push 1/h^4, masses or pair terms out of the float
range. Checked here: (1) rescaling the input by exact powers of two gives
exactly rescaled outputs, bit for bit, in all three precisions (for the
float-pair kernels at scales where the unscaled values would overflow FP32);
(2) the Evrard collapse in SI units (M = 2e30 kg, R = 7e8 m, G = 6.674e-11)
and the rotating patch shrunk by 1e-9 match the FP64 oracle at the FP64 bar
(precision 0) and the mixed bar (precision 1); (3) input beyond the range
those kernels hold is reported as SPH_E_RANGE.
"""
import numpy as np
import pytest

from paper_1809_08013_gb300 import ics
from parity_util import TOL_FP64, check, force_err, normwise, state_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL_MIXED = 1e-5
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


def _patch():
    s, p = ics.square_patch(17, seed=31)
    return ics.random_velocities(s, seed=32, scale=2.0), p


def _rescaled(s, prm, kl, km):
    """Lengths times 2^kl and masses times 2^km (3 kl = km keeps rho, p and c;
    velocities and u unchanged): a ~ V^2/L and du ~ V^3/L scale by 2^-kl, dt
    by 2^kl, everything else is unchanged or scales like a length."""
    s2 = dict(s)
    for k in ("x", "y", "z", "h"):
        s2[k] = np.ldexp(s[k], kl)
    s2["m"] = np.ldexp(s["m"], km)
    p2 = ics.SphParams(**prm.as_dict())
    p2.lz = float(np.ldexp(prm.lz, kl))
    return s2, p2


# exponent of each output's factor, in units of kl
SCALE_OUT = {"x": 1, "y": 1, "z": 1, "h": 1, "m": 3, "ax": -1, "ay": -1, "az": -1, "du": -1,
             "dt": 1, "time": 1}


@pytest.mark.parametrize("precision", [0, 1, 2])
@pytest.mark.parametrize("kl", [-30, 40])
def test_power_of_two_rescaling_gives_the_same_bits(B, precision, kl):
    s, prm = _patch()
    prm.precision = precision
    km = 3 * kl
    s2, prm2 = _rescaled(s, prm, kl, km)
    outs = []
    for st, p in ((s, prm), (s2, prm2)):
        ctx = B.Context(len(st["x"]))
        arr = B.alloc_arrays(st)
        ctx.step(p, arr, nsteps=2)
        assert ctx.sync() == B.SPH_OK
        outs.append({k: host(v).copy() for k, v in arr.items()})
    a, b = outs
    for k in a:
        e = SCALE_OUT.get(k, 0) * kl
        want = np.ldexp(a[k], e) if a[k].dtype == np.float64 else a[k]
        assert np.array_equal(want.view(np.uint8), b[k].view(np.uint8)), k


def _si_evrard():
    """Evrard sphere in SI units: M = 2e30 kg, R = 7e8 m, with G = 6.674e-11
    the code-unit velocity is sqrt(G M / R) and u scales by its square."""
    s, p = ics.evrard(6000, seed=41)
    s = ics.random_velocities(s, seed=42, scale=0.3)
    M, R = 2.0e30, 7.0e8
    V = np.sqrt(6.674e-11 * M / R)
    out = dict(s)
    for k in ("x", "y", "z", "h"):
        out[k] = s[k] * R
    out["m"] = s["m"] * M
    for k in ("vx", "vy", "vz"):
        out[k] = s[k] * V
    out["u"] = s["u"] * V * V
    return out, p


def _nano_patch():
    s, p = _patch()
    sc = 1e-9
    s = dict(s)
    for k in ("x", "y", "z", "h"):
        s[k] = s[k] * sc
    s["m"] = s["m"] * sc ** 3  # the same density
    p.lz = p.lz * sc
    return s, p


CASES = {"evrard_si": _si_evrard, "patch_1e-9": _nano_patch}


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name", list(CASES))
def test_far_units_match_the_oracle(B, orc, name, precision):
    s, prm = CASES[name]()
    prm.precision = precision
    tol = TOL_FP64 if precision == 0 else TOL_MIXED
    per = prm.periodic_z
    o = orc.pipeline(prm, s)
    ctx = B.Context(len(s["x"]))
    arr = B.alloc_arrays(s)
    ctx.build_neighbors(prm, arr)
    assert ctx.sync() == B.SPH_OK
    assert np.array_equal(host(arr["h"]).view(np.int64), o["h"].view(np.int64))
    ctx.density(prm, arr)
    err = {"rho": normwise(host(arr["rho"]), o["rho"])}
    for k in ("rho", "p", "c"):
        arr[k].copy_(torch.from_numpy(o[k]))
    ctx.forces(prm, arr)
    assert ctx.sync() == B.SPH_OK
    err.update({k: force_err(k, host(arr[k]), o[k], o, per) for k in FORCES})
    err["dt"] = abs(host(arr["dt"])[0] - o["dt"]) / o["dt"]
    check(err, tol)
    # and one whole step
    st_o, ex = orc.step(prm, s, nsteps=1)
    arr = B.alloc_arrays(s)
    ctx.step(prm, arr, nsteps=1)
    assert ctx.sync() == B.SPH_OK
    err = {k: state_err(k, host(arr[k]), st_o[k], o, per, ex["dt"])
           for k in ("x", "y", "z", "vx", "vy", "vz", "u")}
    err.update({k: normwise(host(arr[k]), ex[k]) for k in ("rho", "p", "c")})
    err.update({k: force_err(k, host(arr[k]), ex[k], o, per) for k in FORCES})
    check(err, tol)


def _two_scales():
    """Two lattices 50 apart, one with spacing 1, the other with spacing 1e-6:
    one instance whose smoothing lengths differ by ~2^20."""
    a, p = ics.square_patch(10, seed=51)
    b, _ = ics.square_patch(10, seed=52)
    p.periodic_z = 0
    s = {}
    for k in ics.FIELDS:
        lo, hi = a[k].copy(), b[k].copy()
        if k in ("x", "y", "z", "h"):
            hi = hi * 1e-6
        if k == "x":
            hi = hi + 50.0
        if k == "m":
            hi = hi * 1e-18
        s[k] = np.concatenate([lo, hi])
    return s, p


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_out_of_range_input_is_reported(B, precision):
    s, prm = _two_scales()
    prm.precision = precision
    ctx = B.Context(len(s["x"]))
    arr = B.alloc_arrays(s)
    ctx.build_neighbors(prm, arr)
    assert ctx.sync() == B.SPH_OK
    ctx.density(prm, arr)
    ctx.eos(prm, arr)
    ctx.forces(prm, arr)
    st = ctx.sync()
    if precision == 2:
        assert st == B.SPH_OK  # native FP64 holds it
    else:
        assert st == B.SPH_E_RANGE, B.STATUS_NAMES.get(st)
    assert ctx.sync() == B.SPH_OK  # cleared
