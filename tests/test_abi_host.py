"""Host-side checks of the C ABI (no GPU needed): the library builds for
sm_103a, loads, exports every function include/sph.h declares, and rejects
bad arguments on the host without launching anything."""
import ctypes as C

import pytest

from paper_1809_08013_gb300 import binding, ics


@pytest.fixture(scope="module")
def lib():
    return binding.load()


def test_header_declares_the_boundary():
    names = set(binding.header_functions())
    for required in ("sph_ctx_create", "sph_ctx_destroy", "sph_build_neighbors", "sph_density",
                     "sph_eos", "sph_forces", "sph_step", "sph_sync", "sph_last_error"):
        assert required in names


def test_library_exports_every_header_symbol(lib):
    for name in binding.header_functions():
        assert hasattr(lib, name), name


def test_version_string(lib):
    assert b"sm_103a" in lib.sph_version()


def test_null_context_is_rejected_without_launch(lib):
    prm = binding.params(ics.SphParams())
    P = binding.SphParticles()
    assert lib.sph_build_neighbors(None, C.byref(prm), C.byref(P), None, None) == binding.SPH_E_INVAL
    assert lib.sph_density(None, C.byref(prm), C.byref(P), None) == binding.SPH_E_INVAL
    assert lib.sph_eos(None, C.byref(prm), C.byref(P), None) == binding.SPH_E_INVAL
    assert lib.sph_forces(None, C.byref(prm), C.byref(P), None) == binding.SPH_E_INVAL
    assert lib.sph_step(None, C.byref(prm), C.byref(P), 1, None) == binding.SPH_E_INVAL
    assert lib.sph_sync(None, None) == binding.SPH_E_INVAL
    assert lib.sph_last_error(None) == b"context is NULL"
    lib.sph_ctx_destroy(None)  # no-op


def test_ctx_create_rejects_bad_sizes(lib):
    h = C.c_void_p()
    assert lib.sph_ctx_create(C.byref(h), -1, 10, 0) == binding.SPH_E_INVAL
    assert lib.sph_ctx_create(C.byref(h), 10, -5, 0) == binding.SPH_E_INVAL
    assert lib.sph_ctx_create(None, 10, 10, 0) == binding.SPH_E_INVAL
    assert not h.value


def test_param_struct_layout_matches_header():
    # offsets of the C struct (int32 x 6, then 9 doubles)
    assert C.sizeof(binding.SphParams) == 6 * 4 + 9 * 8
    assert binding.SphParams.rho0.offset == 24
    assert C.sizeof(binding.SphParticles) == 8 + 20 * 8
    assert C.sizeof(binding.SphNeighbors) == 8 + 5 * 8
