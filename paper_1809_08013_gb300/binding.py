"""Thin ctypes binding of libsph (include/sph.h): argument marshalling only.

Every step of the SPH path runs in the CUDA library. PyTorch supplies the
device arrays (float64 CUDA tensors) and the stream. If the library cannot be
built or loaded this module raises; there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os
import re

from . import build as _build

(SPH_OK, SPH_E_INVAL, SPH_E_NOMEM, SPH_E_CUDA, SPH_E_CAPACITY, SPH_E_HNOCONV, SPH_E_TIMEOUT,
 SPH_E_RANGE, SPH_E_NONFINITE) = range(9)
STATUS_NAMES = {0: "SPH_OK", 1: "SPH_E_INVAL", 2: "SPH_E_NOMEM", 3: "SPH_E_CUDA",
                4: "SPH_E_CAPACITY", 5: "SPH_E_HNOCONV", 6: "SPH_E_TIMEOUT", 7: "SPH_E_RANGE",
                8: "SPH_E_NONFINITE"}

PHASES = ("cells", "hsearch", "csr", "density", "forces", "update")
STATE_FIELDS = ("x", "y", "z", "vx", "vy", "vz", "m", "h", "u")
OUT_FIELDS = ("rho", "p", "c", "ax", "ay", "az", "du", "mumax")


class SphParams(C.Structure):
    _fields_ = [
        ("eos", C.c_int32), ("n_target", C.c_int32), ("n_tol", C.c_int32),
        ("max_h_iter", C.c_int32), ("periodic_z", C.c_int32), ("precision", C.c_int32),
        ("pair_threads", C.c_int32), ("defer_lanes", C.c_int32),
        ("rho0", C.c_double), ("c0", C.c_double), ("gamma", C.c_double),
        ("alpha", C.c_double), ("beta", C.c_double), ("eta2", C.c_double),
        ("cfl", C.c_double), ("lz", C.c_double), ("cell_scale", C.c_double),
        ("kernel", C.c_int32), ("gradients", C.c_int32), ("sinc_n", C.c_int32),
        ("list_skin", C.c_double),
    ]


_DP = C.c_void_p


class SphParticles(C.Structure):
    _fields_ = [("n", C.c_int64)] + [(f, _DP) for f in (
        "x", "y", "z", "vx", "vy", "vz", "m", "h", "u", "rho", "p", "c", "ax", "ay", "az", "du",
        "mumax", "nnb", "time", "dt")]


class SphNeighbors(C.Structure):
    _fields_ = [("n", C.c_int64), ("offsets", _DP), ("idx", _DP), ("ngather", _DP),
                ("order", _DP), ("nnz_dev", _DP)]


class SphTuneSpace(C.Structure):
    _fields_ = [("cell_scales", _DP), ("n_cell_scales", C.c_int32),
                ("pair_threads", _DP), ("n_pair_threads", C.c_int32),
                ("defer_lanes", _DP), ("n_defer_lanes", C.c_int32)]


class SphTuneTrial(C.Structure):
    _fields_ = [("cell_scale", C.c_double), ("pair_threads", C.c_int32),
                ("defer_lanes", C.c_int32), ("ms_per_step", C.c_double)]


SPH_TUNE_MAX_TRIALS = 16


class SphTuneResult(C.Structure):
    _fields_ = [("cell_scale", C.c_double), ("pair_threads", C.c_int32),
                ("defer_lanes", C.c_int32), ("ms_per_step", C.c_double),
                ("n_trials", C.c_int32), ("trials", SphTuneTrial * SPH_TUNE_MAX_TRIALS)]


class SphError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None


def header_functions() -> list:
    """Names of the functions declared in include/sph.h."""
    with open(os.path.join(_build.INC, "sph.h")) as f:
        text = f.read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[\w\s\*]*?\b(sph_\w+)\s*\(", text, re.M)))


def lib_path() -> str:
    """Path of the in-tree libsph.so (built if missing or stale)."""
    return _build.build()


def load(rebuild: bool = True):
    """Load libsph.so (building it first if sources changed). Raises if it cannot."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if rebuild else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libsph not found at {path}; run paper_1809_08013_gb300.build.build()")
    L = C.CDLL(path)
    P = C.POINTER
    L.sph_version.restype = C.c_char_p
    L.sph_last_error.restype = C.c_char_p
    L.sph_last_error.argtypes = [_DP]
    L.sph_last_hnoconv.restype = C.c_int64
    L.sph_last_hnoconv.argtypes = [_DP]
    L.sph_ctx_create.restype = C.c_int
    L.sph_ctx_create.argtypes = [P(_DP), C.c_int64, C.c_int64, C.c_int]
    L.sph_ctx_bytes.restype = C.c_int64
    L.sph_ctx_bytes.argtypes = [C.c_int64, C.c_int64, C.c_int32]
    L.sph_ctx_create_batch.restype = C.c_int
    L.sph_ctx_create_batch.argtypes = [P(_DP), C.c_int64, C.c_int64, C.c_int32, C.c_int]
    L.sph_batch_set.restype = C.c_int
    L.sph_batch_set.argtypes = [_DP, C.c_int32, P(C.c_int64), P(C.c_int64), P(SphParams), _DP]
    L.sph_autotune.restype = C.c_int
    L.sph_autotune.argtypes = [_DP, P(SphParticles), C.c_int, P(SphTuneSpace), P(SphTuneResult),
                               _DP]
    L.sph_batch_step.restype = C.c_int
    L.sph_batch_step.argtypes = [_DP, P(SphParticles), C.c_int, _DP]
    L.sph_ctx_destroy.restype = None
    L.sph_ctx_destroy.argtypes = [_DP]
    L.sph_build_neighbors.restype = C.c_int
    L.sph_build_neighbors.argtypes = [_DP, P(SphParams), P(SphParticles), P(SphNeighbors), _DP]
    for name in ("sph_density", "sph_eos", "sph_forces"):
        fn = getattr(L, name)
        fn.restype = C.c_int
        fn.argtypes = [_DP, P(SphParams), P(SphParticles), _DP]
    L.sph_step.restype = C.c_int
    L.sph_step.argtypes = [_DP, P(SphParams), P(SphParticles), C.c_int, _DP]
    L.sph_step_host.restype = C.c_int
    L.sph_step_host.argtypes = [_DP, P(SphParams), P(SphParticles), C.c_int, _DP]
    L.sph_neighbors_to_host.restype = C.c_int
    L.sph_neighbors_to_host.argtypes = [_DP, _DP, _DP, C.c_int64, _DP, _DP, _DP]
    L.sph_neighbors_to_host_caller.restype = C.c_int
    L.sph_neighbors_to_host_caller.argtypes = [_DP, C.c_int64, _DP, _DP, C.c_int64, _DP, _DP]
    L.sph_sync.restype = C.c_int
    L.sph_sync.argtypes = [_DP, _DP]
    L.sph_timing_enable.restype = C.c_int
    L.sph_timing_enable.argtypes = [_DP, C.c_int]
    L.sph_timing_read.restype = C.c_int
    L.sph_timing_read.argtypes = [_DP, _DP, _DP, _DP]
    L.sph_lists_clear.restype = C.c_int
    L.sph_lists_clear.argtypes = [_DP, C.c_int64, C.c_int64, _DP]
    L.sph_list_builds.restype = C.c_int
    L.sph_list_builds.argtypes = [_DP, C.POINTER(C.c_int64), _DP]
    L.sph_launch_count.restype = C.c_int64
    L.sph_launch_count.argtypes = [_DP]
    L.sph_neighbor_rows.restype = C.c_int64
    L.sph_neighbor_rows.argtypes = [_DP]
    L.sph_probe_fma_peak.restype = C.c_int
    L.sph_probe_fma_peak.argtypes = [C.c_int, C.c_int, _DP, C.POINTER(C.c_double)]
    _lib = L
    return L


def ctx_bytes(n_capacity: int, nnz_capacity: int | None = None, max_instances: int = 1) -> int:
    """Device bytes of a context with these capacities (see sph_ctx_bytes)."""
    if nnz_capacity is None:
        nnz_capacity = max(1024, 160 * int(n_capacity))
    return int(load().sph_ctx_bytes(int(n_capacity), int(nnz_capacity), int(max_instances)))


def probe_fma_peak(device: int = 0, fp64: bool = True, stream=None) -> float:
    """Measured FMA throughput in flop/s (2 per FMA) of the device."""
    L = load()
    out = C.c_double()
    st = L.sph_probe_fma_peak(int(device), int(bool(fp64)), _stream(stream), C.byref(out))
    if st != SPH_OK:
        raise SphError(st, "sph_probe_fma_peak failed")
    return float(out.value)


def params(p) -> SphParams:
    """Marshal an object with the SphParams attributes (see ics.SphParams)."""
    return SphParams(int(p.eos), int(p.n_target), int(p.n_tol), int(p.max_h_iter),
                     int(p.periodic_z), int(getattr(p, "precision", 0)),
                     int(getattr(p, "pair_threads", 0)), int(getattr(p, "defer_lanes", 0)),
                     float(p.rho0), float(p.c0), float(p.gamma),
                     float(p.alpha), float(p.beta), float(p.eta2), float(p.cfl), float(p.lz),
                     float(getattr(p, "cell_scale", 0.0)), int(getattr(p, "kernel", 0)),
                     int(getattr(p, "gradients", 0)), int(getattr(p, "sinc_n", 5)),
                     float(getattr(p, "list_skin", 0.0)))


def _ptr(t):
    if t is None:
        return None
    return C.c_void_p(t.data_ptr())


def particles(arrays: dict) -> SphParticles:
    """Build the C struct from a dict of CUDA tensors (float64, contiguous;
    'nnb' int32). Missing names become NULL."""
    n = int(arrays["x"].numel())
    s = SphParticles()
    s.n = n
    for f in STATE_FIELDS + OUT_FIELDS + ("nnb", "time", "dt"):
        t = arrays.get(f)
        if t is not None:
            if not t.is_cuda or not t.is_contiguous():
                raise ValueError(f"{f} must be a contiguous CUDA tensor")
            setattr(s, f, t.data_ptr())
    return s


def host_particles(arrays: dict) -> SphParticles:
    """The C struct over HOST arrays: numpy arrays or CPU torch tensors
    (float64, contiguous; 'nnb' int32; 'time' and 'dt' of one element).
    Missing names become NULL."""
    import numpy as np
    n = int(len(arrays["x"]))
    s = SphParticles()
    s.n = n
    for f in STATE_FIELDS + OUT_FIELDS + ("nnb", "time", "dt"):
        a = arrays.get(f)
        if a is None:
            continue
        if isinstance(a, np.ndarray):
            want = np.int32 if f == "nnb" else np.float64
            if a.dtype != want or not a.flags.c_contiguous:
                raise ValueError(f"{f} must be a contiguous {np.dtype(want).name} array")
            setattr(s, f, a.ctypes.data)
        else:
            if a.is_cuda or not a.is_contiguous():
                raise ValueError(f"{f} must be a contiguous host tensor")
            setattr(s, f, a.data_ptr())
    return s


def alloc_arrays(state: dict, device="cuda", ninst: int = 1):
    """Device arrays for a host state dict (numpy arrays x..u): the state
    itself plus outputs, nnb, and the time / dt scalars (one per instance)."""
    import torch
    out = {}
    n = len(state["x"])
    for f in STATE_FIELDS:
        out[f] = torch.as_tensor(state[f], dtype=torch.float64).to(device).contiguous()
    for f in OUT_FIELDS:
        out[f] = torch.zeros(n, dtype=torch.float64, device=device)
    out["nnb"] = torch.zeros(n, dtype=torch.int32, device=device)
    out["time"] = torch.zeros(ninst, dtype=torch.float64, device=device)
    out["dt"] = torch.zeros(ninst, dtype=torch.float64, device=device)
    return out


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


class Context:
    """Owns an sph_ctx: scratch, cell table and neighbour list on one device."""

    def __init__(self, n_capacity: int, nnz_capacity: int | None = None, device: int = 0,
                 max_instances: int = 1):
        self.lib = load()
        if nnz_capacity is None:
            nnz_capacity = max(1024, 160 * int(n_capacity))
        h = C.c_void_p()
        st = self.lib.sph_ctx_create_batch(C.byref(h), int(n_capacity), int(nnz_capacity),
                                           int(max_instances), int(device))
        if st != SPH_OK:
            raise SphError(st, "sph_ctx_create_batch failed")
        self.h = h
        self.n_capacity = int(n_capacity)
        self.nnz_capacity = int(nnz_capacity)
        self.device = device

    def close(self):
        if getattr(self, "h", None):
            self.lib.sph_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != SPH_OK:
            raise SphError(st, self.lib.sph_last_error(self.h).decode())

    def error(self) -> str:
        return self.lib.sph_last_error(self.h).decode()

    def build_neighbors(self, prm, arrays: dict, stream=None) -> SphNeighbors:
        P = particles(arrays)
        nb = SphNeighbors()
        self._check(self.lib.sph_build_neighbors(self.h, C.byref(params(prm)), C.byref(P),
                                                 C.byref(nb), _stream(stream)))
        return nb

    def density(self, prm, arrays: dict, stream=None):
        P = particles(arrays)
        self._check(self.lib.sph_density(self.h, C.byref(params(prm)), C.byref(P), _stream(stream)))

    def eos(self, prm, arrays: dict, stream=None):
        P = particles(arrays)
        self._check(self.lib.sph_eos(self.h, C.byref(params(prm)), C.byref(P), _stream(stream)))

    def forces(self, prm, arrays: dict, stream=None):
        P = particles(arrays)
        self._check(self.lib.sph_forces(self.h, C.byref(params(prm)), C.byref(P), _stream(stream)))

    def step(self, prm, arrays: dict, nsteps: int = 1, stream=None):
        P = particles(arrays)
        self._check(self.lib.sph_step(self.h, C.byref(params(prm)), C.byref(P), int(nsteps),
                                      _stream(stream)))

    def step_host(self, prm, arrays: dict, nsteps: int = 1, stream=None):
        """sph_step_host: `arrays` are host arrays (see host_particles). Pinned
        arrays are read and written in place by the library's kernels; others
        are copied through device staging buffers on the stream."""
        P = host_particles(arrays)
        self._check(self.lib.sph_step_host(self.h, C.byref(params(prm)), C.byref(P), int(nsteps),
                                           _stream(stream)))

    def batch_set(self, counts, prms, first=None, stream=None):
        """Describe a batch: counts[k] particles of instance k, at
        [first[k], first[k] + counts[k]) of the arrays (None: back to back),
        prms[k] its parameters."""
        k = len(counts)
        cnt = (C.c_int64 * k)(*[int(v) for v in counts])
        fst = None if first is None else (C.c_int64 * k)(*[int(v) for v in first])
        pa = (SphParams * k)(*[params(p) for p in prms])
        self._check(self.lib.sph_batch_set(self.h, k, cnt, fst, pa, _stream(stream)))

    def batch_step(self, arrays: dict, nsteps: int = 1, stream=None):
        P = particles(arrays)
        self._check(self.lib.sph_batch_step(self.h, C.byref(P), int(nsteps), _stream(stream)))

    def autotune(self, arrays: dict, nsteps: int = 2, cell_scales=None, pair_threads=None,
                 defer_lanes=None, stream=None) -> dict:
        """Time the knob candidates on the current batch (see sph_autotune);
        None for all three lists uses the library's default search space."""
        P = particles(arrays)
        res = SphTuneResult()
        sp = None
        keep = []
        if cell_scales is not None or pair_threads is not None or defer_lanes is not None:
            cs = (C.c_double * max(1, len(cell_scales or [])))(*(cell_scales or []))
            tp = (C.c_int32 * max(1, len(pair_threads or [])))(*(pair_threads or []))
            dl = (C.c_int32 * max(1, len(defer_lanes or [])))(*(defer_lanes or []))
            keep = [cs, tp, dl]
            sp = SphTuneSpace(C.cast(cs, _DP), len(cell_scales or []), C.cast(tp, _DP),
                              len(pair_threads or []), C.cast(dl, _DP), len(defer_lanes or []))
        self._check(self.lib.sph_autotune(self.h, C.byref(P), int(nsteps),
                                          C.byref(sp) if sp is not None else None,
                                          C.byref(res), _stream(stream)))
        del keep
        trials = [{"cell_scale": t.cell_scale, "pair_threads": t.pair_threads,
                   "defer_lanes": t.defer_lanes, "ms_per_step": t.ms_per_step}
                  for t in res.trials[:res.n_trials]]
        return {"cell_scale": res.cell_scale, "pair_threads": res.pair_threads,
                "defer_lanes": res.defer_lanes, "ms_per_step": res.ms_per_step,
                "trials": trials}

    def sync(self, stream=None) -> int:
        """Wait for the stream; return the device status (SPH_OK, SPH_E_NONFINITE,
        SPH_E_CAPACITY, SPH_E_RANGE, SPH_E_HNOCONV) without raising."""
        return int(self.lib.sph_sync(self.h, _stream(stream)))

    def timing_enable(self, on: bool = True):
        self._check(self.lib.sph_timing_enable(self.h, int(bool(on))))

    def timing_read(self):
        """Per-phase device ms and launches since the last read, and the
        number of timed steps: (dict ms, dict launches, steps)."""
        ms = (C.c_double * len(PHASES))()
        ln = (C.c_int64 * len(PHASES))()
        st = C.c_int64()
        self._check(self.lib.sph_timing_read(self.h, C.cast(ms, C.c_void_p), C.cast(ln, C.c_void_p),
                                             C.cast(C.pointer(st), C.c_void_p)))
        return dict(zip(PHASES, list(ms))), dict(zip(PHASES, list(ln))), int(st.value)

    def lists_clear(self, first: int = 0, count: int | None = None, stream=None):
        """sph_lists_clear: forget the candidate lists of [first, first + count)."""
        if count is None:
            count = self.n_capacity - first
        self._check(self.lib.sph_lists_clear(self.h, int(first), int(count), _stream(stream)))

    def list_builds(self, stream=None) -> int:
        """sph_list_builds: candidate-list builds so far (synchronises)."""
        v = C.c_int64()
        self._check(self.lib.sph_list_builds(self.h, C.byref(v), _stream(stream)))
        return int(v.value)

    def launch_count(self) -> int:
        return int(self.lib.sph_launch_count(self.h))

    def last_hnoconv(self) -> int:
        return int(self.lib.sph_last_hnoconv(self.h))

    def neighbors_caller(self, ncaller: int, stream=None):
        """sph_neighbors_to_host_caller: the neighbour list in caller order
        (offsets, idx, ngather) as host numpy arrays."""
        import numpy as np
        off = np.zeros(int(ncaller) + 1, dtype=np.int64)
        I64, I32 = C.POINTER(C.c_int64), C.POINTER(C.c_int32)
        self._check(self.lib.sph_neighbors_to_host_caller(
            self.h, int(ncaller), off.ctypes.data_as(I64), None, 0, None, _stream(stream)))
        nnz = int(off[-1])
        idx = np.zeros(max(nnz, 1), dtype=np.int32)
        ng = np.zeros(max(int(ncaller), 1), dtype=np.int32)
        self._check(self.lib.sph_neighbors_to_host_caller(
            self.h, int(ncaller), off.ctypes.data_as(I64), idx.ctypes.data_as(I32), len(idx),
            ng.ctypes.data_as(I32), _stream(stream)))
        return off, idx[:nnz], ng[:int(ncaller)]

    def neighbors_to_host(self, stream=None):
        """Neighbour list of the last build as host numpy arrays (offsets,
        idx, ngather, order); rows in internal order, see sph_neighbors."""
        import numpy as np
        n = int(self.lib.sph_neighbor_rows(self.h))
        off = np.zeros(n + 1, dtype=np.int64)
        ng = np.zeros(max(n, 1), dtype=np.int32)
        order = np.zeros(max(n, 1), dtype=np.int32)
        I64, I32 = C.POINTER(C.c_int64), C.POINTER(C.c_int32)
        self._check(self.lib.sph_neighbors_to_host(
            self.h, off.ctypes.data_as(I64), None, 0, ng.ctypes.data_as(I32),
            order.ctypes.data_as(I32), _stream(stream)))
        nnz = int(off[-1])
        idx = np.zeros(max(nnz, 1), dtype=np.int32)
        self._check(self.lib.sph_neighbors_to_host(
            self.h, None, idx.ctypes.data_as(I32), len(idx), None, None, _stream(stream)))
        return off, idx[:nnz], ng[:n], order[:n]
