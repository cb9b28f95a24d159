"""sph_dt_noalloc: the time step for callers that cannot allocate device
memory (a host that owns all device memory through its own pool, or a
latency-critical loop where cudaMalloc may synchronise the device).

It is called here through the C ABI on the arrays that sph_forces consumed and
produced, twice in a row with different inputs, and must agree with the dt
that sph_forces computed within the FP64 parity bar. This file sorts last so a
run that stops at the first failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _noalloc(B):
    fn = B.load().sph_dt_noalloc
    fn.restype = C.c_int
    fn.argtypes = [C.POINTER(B.SphParams), C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                   C.c_void_p, C.c_void_p]
    return fn


def test_dt_noalloc_matches_forces_dt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_08013_gb300 import binding as B
    from paper_1809_08013_gb300 import ics
    fn = _noalloc(B)
    stream = torch.cuda.current_stream()
    results = []
    for side, seed in ((14, 3), (19, 4)):  # two calls in a row, different inputs
        s, prm = ics.square_patch(side, seed=seed)
        s = ics.random_velocities(s, seed=seed + 10, scale=1.5)  # viscosity active: mumax > 0
        ctx = B.Context(len(s["x"]))
        arr = B.alloc_arrays(s)
        ctx.build_neighbors(prm, arr)
        ctx.density(prm, arr)
        ctx.eos(prm, arr)
        ctx.forces(prm, arr)
        assert ctx.sync() in (B.SPH_OK, B.SPH_E_HNOCONV)
        ref = float(arr["dt"].item())
        out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        st = fn(C.byref(B.params(prm)), len(s["x"]), arr["h"].data_ptr(), arr["c"].data_ptr(),
                arr["mumax"].data_ptr(), out.data_ptr(), C.c_void_p(stream.cuda_stream))
        assert st == B.SPH_OK
        torch.cuda.synchronize()
        got = float(out.item())
        assert np.isfinite(got) and abs(got - ref) <= 1e-12 * ref
        assert float(arr["mumax"].max()) > 0.0
        results.append(got)
    assert results[0] != results[1]


def test_dt_noalloc_rejects_sizes_beyond_its_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_08013_gb300 import binding as B
    from paper_1809_08013_gb300 import ics
    fn = _noalloc(B)
    dummy = torch.zeros(4, dtype=torch.float64, device="cuda")
    prm = B.params(ics.SphParams())
    too_many = 2097152 + 1
    st = fn(C.byref(prm), too_many, dummy.data_ptr(), dummy.data_ptr(), None, dummy.data_ptr(), None)
    assert st == B.SPH_E_INVAL


def _call(fn, B, prm, n, h, c, mumax, stream):
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    st = fn(C.byref(B.params(prm)), n, h.data_ptr() if h is not None else None,
            c.data_ptr() if c is not None else None,
            mumax.data_ptr() if mumax is not None else None, out.data_ptr(),
            C.c_void_p(stream.cuda_stream))
    torch.cuda.synchronize()
    return st, float(out.item())


def test_dt_noalloc_full_scratch_and_degenerate_sizes(orc):
    # n = SPH_NOALLOC_MAX_N fills every partial slot of the static array (8192
    # blocks, so the finishing block loops over 32 partials per thread), with
    # the minimum in the very last block; then n = 0 and mumax = NULL
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_08013_gb300 import binding as B
    from paper_1809_08013_gb300 import ics
    fn = _noalloc(B)
    stream = torch.cuda.current_stream()
    prm = ics.SphParams()
    n = 2097152
    rng = np.random.Generator(np.random.PCG64(91))
    h = rng.uniform(0.01, 0.02, n)
    c = rng.uniform(40.0, 60.0, n)
    mu = rng.uniform(0.0, 5.0, n)
    h[n - 3] = 0.001  # the smallest candidate sits in the last block
    dh, dc, dm = (torch.from_numpy(a).cuda() for a in (h, c, mu))
    st, got = _call(fn, B, prm, n, dh, dc, dm, stream)
    ref = orc.dt(prm, h, c, mu)
    assert st == B.SPH_OK and abs(got - ref) <= 1e-12 * ref
    h2 = h.copy()
    h2[n - 3] = 0.015
    assert orc.dt(prm, h2, c, mu) > 2.0 * ref  # the minimum is the last block's
    # mumax = NULL reads as all zero
    st, got = _call(fn, B, prm, n, dh, dc, None, stream)
    ref = orc.dt(prm, h, c, np.zeros(n))
    assert st == B.SPH_OK and abs(got - ref) <= 1e-12 * ref
    # n = 0: no particle, dt = +inf (the scratch still holds the last call's partials)
    st, got = _call(fn, B, prm, 0, None, None, None, stream)
    assert st == B.SPH_OK and got == float("inf")
