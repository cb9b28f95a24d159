"""CPU oracle of the SPH time step: a ctypes wrapper over ``sph_oracle.c``.

TEST INFRASTRUCTURE. Only the tests, the smoke check and the CPU-baseline leg
of the benchmark import this package; the product path (the CUDA library and
its binding) never does, and nothing here imports the product path. The two
sides share only the seeded input generators.

Every function takes and returns float64 / int numpy arrays in the caller's
particle order. See ``sph_oracle.c`` for the definitions each routine follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sph_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-Wall"]


class OrcParams(C.Structure):
    _fields_ = [
        ("eos", C.c_int32), ("n_target", C.c_int32), ("n_tol", C.c_int32),
        ("max_h_iter", C.c_int32), ("periodic_z", C.c_int32), ("kernel", C.c_int32),
        ("gradients", C.c_int32), ("sinc_n", C.c_int32),
        ("rho0", C.c_double), ("c0", C.c_double), ("gamma", C.c_double),
        ("alpha", C.c_double), ("beta", C.c_double), ("eta2", C.c_double),
        ("cfl", C.c_double), ("lz", C.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (in-tree, under oracle/_build)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *_CFLAGS, _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None
_D = C.POINTER(C.c_double)
_I64 = C.POINTER(C.c_int64)
_I32 = C.POINTER(C.c_int32)
_U8 = C.POINTER(C.c_uint8)
_P = C.POINTER(OrcParams)


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        L.orc_W.restype = C.c_double
        L.orc_W.argtypes = [C.c_double, C.c_double]
        L.orc_dWdr.restype = C.c_double
        L.orc_dWdr.argtypes = [C.c_double, C.c_double]
        L.orc_sinc_norm.restype = C.c_double
        L.orc_sinc_norm.argtypes = [C.c_int]
        L.orc_kernel_W.restype = C.c_double
        L.orc_kernel_W.argtypes = [_P, C.c_double, C.c_double]
        L.orc_kernel_dWdr.restype = C.c_double
        L.orc_kernel_dWdr.argtypes = [_P, C.c_double, C.c_double]
        L.orc_iad.argtypes = [_P, C.c_int64] + [_D] * 6 + [_I64, _I32, _I32, _D]
        L.orc_iad_gradient.argtypes = ([_P, C.c_int64] + [_D] * 6 + [_I64, _I32, _I32] +
                                       [_D] * 5)
        L.orc_set_threads.argtypes = [C.c_int]
        L.orc_get_threads.restype = C.c_int
        L.orc_count_brute.restype = C.c_int64
        L.orc_count_brute.argtypes = [_P, C.c_int64, _D, _D, _D, C.c_int64, C.c_double]
        L.orc_h_iterate.restype = C.c_int64
        L.orc_h_iterate.argtypes = [_P, C.c_int64, _D, _D, _D, _D, _D, _I32, _U8, C.c_int]
        L.orc_csr_count.restype = C.c_int
        L.orc_csr_count.argtypes = [_P, C.c_int64, _D, _D, _D, _D, _I64, C.c_int]
        L.orc_csr_fill.restype = C.c_int
        L.orc_csr_fill.argtypes = [_P, C.c_int64, _D, _D, _D, _D, _I64, _I32, _I32, C.c_int]
        L.orc_density.argtypes = [_P, C.c_int64, _D, _D, _D, _D, _D, _I64, _I32, _I32, _D]
        L.orc_eos.argtypes = [_P, C.c_int64, _D, _D, _D, _D]
        L.orc_forces.argtypes = [_P, C.c_int64] + [_D] * 11 + [_I64, _I32] + [_D] * 6
        L.orc_forces_scale.argtypes = [_P, C.c_int64] + [_D] * 11 + [_I64, _I32] + [_D] * 4
        L.orc_dt.restype = C.c_double
        L.orc_dt.argtypes = [_P, C.c_int64, _D, _D, _D]
        L.orc_leapfrog.argtypes = [_P, C.c_int64, C.c_double] + [_D] * 11
        L.orc_step.restype = C.c_int
        L.orc_step.argtypes = ([_P, C.c_int64, C.c_int] + [_D] * 9 + [_D] * 8 + [_D, _D, _I64])
        _lib = L
    return _lib


def params(p) -> OrcParams:
    """Marshal an object with the SphParams attributes into the oracle's struct."""
    return OrcParams(int(p.eos), int(p.n_target), int(p.n_tol), int(p.max_h_iter),
                     int(p.periodic_z), int(getattr(p, "kernel", 0)),
                     int(getattr(p, "gradients", 0)), int(getattr(p, "sinc_n", 5)),
                     float(p.rho0), float(p.c0), float(p.gamma),
                     float(p.alpha), float(p.beta), float(p.eta2), float(p.cfl), float(p.lz))


def _d(a):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def _c64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def set_threads(k: int) -> None:
    lib().orc_set_threads(int(k))


def get_threads() -> int:
    return int(lib().orc_get_threads())


def W(r: float, h: float) -> float:
    return lib().orc_W(float(r), float(h))


def dWdr(r: float, h: float) -> float:
    return lib().orc_dWdr(float(r), float(h))


def sinc_norm(n: int) -> float:
    """Normalisation B_n of the sinc kernel S(pi q / 2)^n."""
    return float(lib().orc_sinc_norm(int(n)))


def kernel_W(prm, r: float, h: float) -> float:
    """W(r, h) of the kernel prm.kernel selects (0 M4, 1 Wendland C2, 2 sinc)."""
    P = params(prm)
    return float(lib().orc_kernel_W(C.byref(P), float(r), float(h)))


def kernel_dWdr(prm, r: float, h: float) -> float:
    P = params(prm)
    return float(lib().orc_kernel_dWdr(C.byref(P), float(r), float(h)))


def _csr_args(off, idx, ng=None):
    off = np.ascontiguousarray(off, dtype=np.int64)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    if len(idx) == 0:
        idx = np.zeros(1, dtype=np.int32)
    out = [off.ctypes.data_as(_I64), idx.ctypes.data_as(_I32)]
    keep = [off, idx]
    if ng is not None:
        ng = np.ascontiguousarray(ng, dtype=np.int32)
        out.append(ng.ctypes.data_as(_I32))
        keep.append(ng)
    return out, keep


def iad(prm, s: dict, rho, off, idx, ng):
    """IAD matrices C_i = tau_i^-1, shape (n, 6): xx, xy, xz, yy, yz, zz."""
    arrs = [_c64(s[k]) for k in ("x", "y", "z", "m", "h")]
    rho = _c64(rho)
    n = len(arrs[0])
    cm = np.zeros((max(n, 1), 6))
    a, keep = _csr_args(off, idx, ng)
    P = params(prm)
    lib().orc_iad(C.byref(P), n, *[_d(v) for v in arrs], _d(rho), *a, _d(cm))
    return cm[:n]


def iad_gradient(prm, s: dict, rho, off, idx, ng, cm, f):
    """IAD gradient of the per-particle field f; returns (gx, gy, gz)."""
    arrs = [_c64(s[k]) for k in ("x", "y", "z", "m", "h")]
    rho, f = _c64(rho), _c64(f)
    cm = np.ascontiguousarray(cm, dtype=np.float64)
    n = len(arrs[0])
    out = [np.empty(n) for _ in range(3)]
    a, keep = _csr_args(off, idx, ng)
    P = params(prm)
    lib().orc_iad_gradient(C.byref(P), n, *[_d(v) for v in arrs], _d(rho), *a, _d(cm), _d(f),
                           *[_d(v) for v in out])
    return tuple(out)


def count_brute(prm, x, y, z, i: int, h: float) -> int:
    x, y, z = _c64(x), _c64(y), _c64(z)
    P = params(prm)
    return int(lib().orc_count_brute(C.byref(P), len(x), _d(x), _d(y), _d(z), int(i), float(h)))


def h_iterate(prm, x, y, z, h_in, brute: bool = False):
    """Smoothing-length iteration. Returns (h, nnb, conv, n_not_converged)."""
    x, y, z, h_in = _c64(x), _c64(y), _c64(z), _c64(h_in)
    n = len(x)
    h = np.empty(n)
    nnb = np.zeros(n, dtype=np.int32)
    conv = np.zeros(n, dtype=np.uint8)
    P = params(prm)
    bad = lib().orc_h_iterate(C.byref(P), n, _d(x), _d(y), _d(z), _d(h_in), _d(h),
                              nnb.ctypes.data_as(_I32), conv.ctypes.data_as(_U8), int(brute))
    if bad < 0:
        raise MemoryError("oracle h iteration: allocation failed")
    return h, nnb, conv, int(bad)


def csr(prm, x, y, z, h, brute: bool = False):
    """Symmetric interaction set S_i as CSR. Returns (offsets int64[n+1],
    idx int32[nnz], ngather int32[n]); row i lists N_i first, each part in
    ascending j."""
    x, y, z, h = _c64(x), _c64(y), _c64(z), _c64(h)
    n = len(x)
    P = params(prm)
    off = np.zeros(n + 1, dtype=np.int64)
    if lib().orc_csr_count(C.byref(P), n, _d(x), _d(y), _d(z), _d(h),
                           off[1:].ctypes.data_as(_I64), int(brute)) != 0:
        raise MemoryError("oracle csr count failed")
    np.cumsum(off, out=off)
    idx = np.zeros(max(int(off[-1]), 1), dtype=np.int32)
    ng = np.zeros(n, dtype=np.int32)
    if lib().orc_csr_fill(C.byref(P), n, _d(x), _d(y), _d(z), _d(h), off.ctypes.data_as(_I64),
                          idx.ctypes.data_as(_I32), ng.ctypes.data_as(_I32), int(brute)) != 0:
        raise RuntimeError("oracle csr fill failed")
    return off, idx[: int(off[-1])], ng


def density(prm, x, y, z, m, h, off, idx, ng):
    x, y, z, m, h = map(_c64, (x, y, z, m, h))
    off = np.ascontiguousarray(off, dtype=np.int64)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    if len(idx) == 0:
        idx = np.zeros(1, dtype=np.int32)
    ng = np.ascontiguousarray(ng, dtype=np.int32)
    rho = np.empty(len(x))
    P = params(prm)
    lib().orc_density(C.byref(P), len(x), _d(x), _d(y), _d(z), _d(m), _d(h),
                      off.ctypes.data_as(_I64), idx.ctypes.data_as(_I32),
                      ng.ctypes.data_as(_I32), _d(rho))
    return rho


def eos(prm, rho, u):
    rho, u = _c64(rho), _c64(u)
    p = np.empty(len(rho))
    c = np.empty(len(rho))
    P = params(prm)
    lib().orc_eos(C.byref(P), len(rho), _d(rho), _d(u), _d(p), _d(c))
    return p, c


def _cmat(prm, cm, n):
    if int(getattr(prm, "gradients", 0)) == 1:
        if cm is None:
            raise ValueError("IAD gradients need the matrices of iad()")
        return np.ascontiguousarray(cm, dtype=np.float64).reshape(-1)
    return np.zeros(1)


def forces(prm, s: dict, rho, p, c, off, idx, cm=None):
    """Returns (ax, ay, az, du, mumax) for the state dict s (x..u); cm are the
    IAD matrices when prm.gradients == 1."""
    arrs = [_c64(s[k]) for k in ("x", "y", "z", "vx", "vy", "vz", "m", "h")]
    rho, p, c = _c64(rho), _c64(p), _c64(c)
    off = np.ascontiguousarray(off, dtype=np.int64)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    if len(idx) == 0:
        idx = np.zeros(1, dtype=np.int32)
    n = len(arrs[0])
    out = [np.empty(n) for _ in range(5)]
    cmf = _cmat(prm, cm, n)
    P = params(prm)
    lib().orc_forces(C.byref(P), n, *[_d(a) for a in arrs], _d(rho), _d(p), _d(c),
                     off.ctypes.data_as(_I64), idx.ctypes.data_as(_I32), _d(cmf),
                     *[_d(a) for a in out])
    return tuple(out)


def forces_scale(prm, s: dict, rho, p, c, off, idx, cm=None):
    """Per-particle magnitudes of the summed force terms (sa, sdu, smu); see
    orc_forces_scale."""
    arrs = [_c64(s[k]) for k in ("x", "y", "z", "vx", "vy", "vz", "m", "h")]
    rho, p, c = _c64(rho), _c64(p), _c64(c)
    off = np.ascontiguousarray(off, dtype=np.int64)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    if len(idx) == 0:
        idx = np.zeros(1, dtype=np.int32)
    n = len(arrs[0])
    out = [np.empty(n) for _ in range(3)]
    cmf = _cmat(prm, cm, n)
    P = params(prm)
    lib().orc_forces_scale(C.byref(P), n, *[_d(a) for a in arrs], _d(rho), _d(p), _d(c),
                           off.ctypes.data_as(_I64), idx.ctypes.data_as(_I32), _d(cmf),
                           *[_d(a) for a in out])
    return tuple(out)


def dt(prm, h, c, mumax) -> float:
    h, c, mumax = _c64(h), _c64(c), _c64(mumax)
    P = params(prm)
    return float(lib().orc_dt(C.byref(P), len(h), _d(h), _d(c), _d(mumax)))


def leapfrog(prm, s: dict, dt_: float, ax, ay, az, du) -> dict:
    out = {k: _c64(v).copy() for k, v in s.items()}
    ax, ay, az, du = map(_c64, (ax, ay, az, du))
    P = params(prm)
    lib().orc_leapfrog(C.byref(P), len(out["x"]), float(dt_),
                       *[_d(out[k]) for k in ("x", "y", "z", "vx", "vy", "vz", "u")],
                       _d(ax), _d(ay), _d(az), _d(du))
    return out


def step(prm, s: dict, nsteps: int = 1, time: float = 0.0):
    """Run nsteps full steps. Returns (state', extras) where extras holds rho,
    p, c, ax, ay, az, du, mumax of the last force evaluation, time, dt, nnz,
    and the number of non-converged h searches summed over the steps."""
    st = {k: _c64(v).copy() for k, v in s.items()}
    n = len(st["x"])
    ex = {k: np.zeros(n) for k in ("rho", "p", "c", "ax", "ay", "az", "du", "mumax")}
    t = np.array([time])
    d = np.array([0.0])
    stats = np.zeros(2, dtype=np.int64)
    P = params(prm)
    rc = lib().orc_step(C.byref(P), n, int(nsteps),
                        *[_d(st[k]) for k in ("x", "y", "z", "vx", "vy", "vz", "m", "h", "u")],
                        *[_d(ex[k]) for k in ("rho", "p", "c", "ax", "ay", "az", "du", "mumax")],
                        _d(t), _d(d), stats.ctypes.data_as(_I64))
    if rc != 0:
        raise MemoryError("oracle step: allocation failed")
    ex.update(time=float(t[0]), dt=float(d[0]), nnz=int(stats[0]), not_converged=int(stats[1]))
    return st, ex


def pipeline(prm, s: dict):
    """One step's quantities from state s, computed call by call (no update):
    returns a dict with h, nnb, conv, off, idx, ng, rho, p, c, ax, ay, az, du,
    mumax, dt."""
    h, nnb, conv, _ = h_iterate(prm, s["x"], s["y"], s["z"], s["h"])
    off, idx, ng = csr(prm, s["x"], s["y"], s["z"], h)
    s2 = dict(s)
    s2["h"] = h
    rho = density(prm, s["x"], s["y"], s["z"], s["m"], h, off, idx, ng)
    p, c = eos(prm, rho, s["u"])
    cm = iad(prm, s2, rho, off, idx, ng) if int(getattr(prm, "gradients", 0)) == 1 else None
    ax, ay, az, du, mumax = forces(prm, s2, rho, p, c, off, idx, cm)
    sa, sdu, smu = forces_scale(prm, s2, rho, p, c, off, idx, cm)
    return dict(h=h, nnb=nnb, conv=conv, off=off, idx=idx, ng=ng, rho=rho, p=p, c=c, ax=ax,
                ay=ay, az=az, du=du, mumax=mumax, dt=dt(prm, h, c, mumax),
                scale_a=sa, scale_du=sdu, scale_mu=smu, iad=cm)
