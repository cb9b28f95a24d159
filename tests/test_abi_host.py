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


def test_status_codes_match_header():
    # the binding's status constants and names are the header's enum
    import re
    from pathlib import Path
    hdr = (Path(__file__).resolve().parents[1] / "include" / "sph.h").read_text()
    body = hdr[hdr.index("typedef enum {"):hdr.index("} sph_status;")]
    enum = {int(v): k for k, v in re.findall(r"\b(SPH_[A-Z_]+)\s*=\s*(\d+)", body)}
    assert enum == binding.STATUS_NAMES
    for v, k in enum.items():
        assert getattr(binding, k) == v


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
    assert lib.sph_step_host(None, C.byref(prm), C.byref(P), 1, None) == binding.SPH_E_INVAL
    assert lib.sph_sync(None, None) == binding.SPH_E_INVAL
    assert lib.sph_lists_clear(None, 0, 1, None) == binding.SPH_E_INVAL
    off = (C.c_int64 * 2)()
    assert lib.sph_neighbors_to_host_caller(None, 1, off, None, 0, None, None) == binding.SPH_E_INVAL
    v = C.c_int64(7)
    assert lib.sph_list_builds(None, C.byref(v), None) == binding.SPH_E_INVAL
    assert lib.sph_last_error(None) == b"context is NULL"
    lib.sph_ctx_destroy(None)  # no-op


def test_ctx_create_rejects_bad_sizes(lib):
    h = C.c_void_p()
    assert lib.sph_ctx_create(C.byref(h), -1, 10, 0) == binding.SPH_E_INVAL
    assert lib.sph_ctx_create(C.byref(h), 10, -5, 0) == binding.SPH_E_INVAL
    assert lib.sph_ctx_create(None, 10, 10, 0) == binding.SPH_E_INVAL
    for ncap in (2 ** 31, 2 ** 63 - 1):  # slots are int32 (and ncap + gaps must not wrap)
        assert lib.sph_ctx_create(C.byref(h), ncap, 10, 0) == binding.SPH_E_INVAL
        assert lib.sph_ctx_bytes(ncap, 10, 1) == -1
    assert not h.value


def _c_layout(struct, fields):
    """sizeof and offsetof of a struct of include/sph.h, as the C compiler lays it out."""
    import os
    import subprocess
    import tempfile
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    body = "".join(f'printf("%zu\\n", offsetof({struct}, {f}));' for f in fields)
    src = ("#include <stddef.h>\n#include <stdio.h>\n#include \"sph.h\"\n"
           f'int main(void) {{ printf("%zu\\n", sizeof({struct})); {body} return 0; }}\n')
    with tempfile.TemporaryDirectory() as d:
        c, exe = os.path.join(d, "l.c"), os.path.join(d, "l")
        with open(c, "w") as f:
            f.write(src)
        subprocess.check_call(["gcc", "-I", inc, c, "-o", exe])
        out = [int(v) for v in subprocess.check_output([exe]).split()]
    return out[0], out[1:]


def test_param_struct_layout_matches_header():
    # the ctypes mirrors must lay out exactly like the C structs of the header
    for cls, name in ((binding.SphParams, "sph_params"), (binding.SphParticles, "sph_particles"),
                      (binding.SphNeighbors, "sph_neighbors"), (binding.SphTuneSpace, "sph_tune_space"),
                      (binding.SphTuneTrial, "sph_tune_trial"), (binding.SphTuneResult, "sph_tune_result")):
        fields = [f for f, _ in cls._fields_]
        size, offs = _c_layout(name, fields)
        assert C.sizeof(cls) == size, name
        assert [getattr(cls, f).offset for f in fields] == offs, name

def test_plain_c_caller_compiles_and_links(lib):
    # the header is plain C99 and every symbol the example calls resolves
    # against the library at link time (the program is not run here)
    import os
    import subprocess
    import tempfile
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    so = binding.lib_path()
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "example")
        subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(root, "include"),
                               os.path.join(root, "tests", "c_abi_example.c"),
                               "-L", os.path.dirname(so), "-l:" + os.path.basename(so),
                               "-Wl,-rpath," + os.path.dirname(so), "-lm", "-o", exe])
        assert os.path.getsize(exe) > 0


@pytest.mark.gpu
def test_plain_c_caller_runs():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import os
    import subprocess
    import tempfile
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    so = binding.lib_path()
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "example")
        subprocess.check_call(["gcc", "-std=c99", "-I", os.path.join(root, "include"),
                               os.path.join(root, "tests", "c_abi_example.c"),
                               "-L", os.path.dirname(so), "-l:" + os.path.basename(so),
                               "-Wl,-rpath," + os.path.dirname(so), "-lm", "-o", exe])
        out = subprocess.check_output([exe], text=True)
    assert "sm_103a" in out and "dt=" in out
