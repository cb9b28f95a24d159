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
