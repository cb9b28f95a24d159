"""sph_step_host: the step on HOST arrays through the C ABI (pinned arrays
read in place and written by a copy kernel, others copied through staging
buffers, all inside the call) gives the bits of sph_step on device arrays."""
import numpy as np
import pytest

from paper_1809_08013_gb300 import ics

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

FIELDS = ("x", "y", "z", "vx", "vy", "vz", "m", "h", "u")
OUTS = ("rho", "p", "c", "ax", "ay", "az", "du", "mumax")


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_08013_gb300 import binding
    binding.load()
    return binding


def _device_run(B, s, prm, nsteps):
    ctx = B.Context(len(s["x"]))
    arr = B.alloc_arrays(s)
    ctx.step(prm, arr, nsteps=nsteps)
    ctx.sync()
    return {k: arr[k].cpu().numpy() for k in FIELDS + OUTS + ("nnb", "time", "dt")}


def _host_arrays(s, pinned, outputs=True):
    n = len(s["x"])
    if pinned:
        h = {k: torch.from_numpy(np.ascontiguousarray(s[k])).clone().pin_memory() for k in FIELDS}
        mk = lambda dt, m: torch.zeros(m, dtype=dt).pin_memory()  # noqa: E731
        f64, i32 = torch.float64, torch.int32
    else:
        h = {k: np.ascontiguousarray(s[k]).copy() for k in FIELDS}
        mk = lambda dt, m: np.zeros(m, dtype=dt)  # noqa: E731
        f64, i32 = np.float64, np.int32
    h["time"] = mk(f64, 1)
    h["dt"] = mk(f64, 1)
    if outputs:
        for k in OUTS:
            h[k] = mk(f64, n)
        h["nnb"] = mk(i32, n)
    return h


def _np(a):
    return a.numpy() if hasattr(a, "numpy") else a


def _case(name):
    if name == "patch":
        s, prm = ics.square_patch(13, seed=31)
        return ics.random_velocities(s, seed=32, scale=1.0), prm
    return ics.evrard(6000, seed=33)


@pytest.mark.parametrize("pinned", [False, True])
@pytest.mark.parametrize("case", ["patch", "evrard"])
def test_step_host_equals_device_step(B, pinned, case):
    s, prm = _case(case)
    ref = _device_run(B, s, prm, 3)
    ctx = B.Context(len(s["x"]))
    h = _host_arrays(s, pinned)
    ctx.step_host(prm, h, nsteps=3)
    assert ctx.sync() in (B.SPH_OK, B.SPH_E_HNOCONV)
    for k in FIELDS + OUTS + ("nnb", "time", "dt"):
        got = _np(h[k])
        assert np.array_equal(got.view(np.uint8), ref[k].view(np.uint8)), k


def test_step_host_state_only_and_repeated_calls(B):
    # outputs may be NULL; two calls of 2 steps give the bits of one call of 4
    s, prm = ics.square_patch(11, seed=41)
    ref = _device_run(B, s, prm, 4)
    ctx = B.Context(len(s["x"]))
    h = _host_arrays(s, pinned=False, outputs=False)
    ctx.step_host(prm, h, nsteps=2)
    ctx.step_host(prm, h, nsteps=2)
    ctx.sync()
    for k in FIELDS + ("time", "dt"):
        assert np.array_equal(h[k].view(np.uint8), ref[k].view(np.uint8)), k


def test_step_host_zero_steps_and_invalid(B):
    s, prm = ics.square_patch(8, seed=43)
    ctx = B.Context(len(s["x"]))
    h = _host_arrays(s, pinned=False)
    before = {k: h[k].copy() for k in FIELDS}
    ctx.step_host(prm, h, nsteps=0)
    ctx.sync()
    for k in FIELDS:
        assert np.array_equal(h[k], before[k])
    bad = dict(h)
    del bad["vx"]
    l0 = ctx.launch_count()
    with pytest.raises(B.SphError) as e:
        ctx.step_host(prm, bad, nsteps=1)
    assert e.value.status == B.SPH_E_INVAL and ctx.launch_count() == l0
    big = {k: np.zeros(len(s["x"]) + 1) for k in FIELDS}
    big.update(time=np.zeros(1), dt=np.zeros(1))
    with pytest.raises(B.SphError) as e:
        ctx.step_host(prm, big, nsteps=1)
    assert e.value.status == B.SPH_E_INVAL


def test_step_host_mixed_pinned_and_pageable(B):
    # pinned arrays are read and written in place by the kernels, pageable ones
    # go through the staging copies: any mix gives the bits of the device step
    s, prm = _case("patch")
    ref = _device_run(B, s, prm, 2)
    ctx = B.Context(len(s["x"]))
    h = _host_arrays(s, pinned=False)
    for k in ("x", "vy", "h", "rho", "az", "nnb", "time"):
        h[k] = torch.from_numpy(h[k].copy()).pin_memory()
    for k in ("u", "du"):  # views 8 bytes into pinned buffers: not 16-byte aligned
        buf = torch.zeros(len(h[k]) + 1, dtype=torch.float64).pin_memory()
        buf[1:] = torch.from_numpy(h[k])
        h[k] = buf[1:]
        assert h[k].data_ptr() % 16 == 8
    ctx.step_host(prm, h, nsteps=2)
    assert ctx.sync() in (B.SPH_OK, B.SPH_E_HNOCONV)
    for k in FIELDS + OUTS + ("nnb", "time", "dt"):
        assert np.array_equal(_np(h[k]).view(np.uint8), ref[k].view(np.uint8)), k
