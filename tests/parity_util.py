"""Helpers shared by the GPU parity tests: canonical neighbour sets and the
normwise error metric. Expected values always come from the oracle."""
import numpy as np

# FP64 parity bar: max_i |f_i - f_i^ref| / max_i |f_i^ref| per field, for one
# call or one step from identical inputs. The pair sums round differently
# (FMA contraction, summation order, rsqrt) but every term is O(1e-16)
# relative, so 1e-12 leaves a wide margin.
TOL_FP64 = 1e-12


def normwise(a, ref) -> float:
    a = np.asarray(a, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    scale = np.max(np.abs(ref)) if ref.size else 0.0
    err = np.max(np.abs(a - ref)) if ref.size else 0.0
    if scale == 0.0:
        return float(err)
    return float(err / scale)


def scaled(a, ref, scale) -> float:
    """Normwise error against the larger of the result's magnitude and the
    magnitude of the terms it sums (scale from the oracle's orc_forces_scale).
    For a field whose exact value cancels to zero (du and mu under rigid
    rotation, where v_ij . r_ij = 0 for every pair) both sides hold rounding
    noise, and only the summed-term magnitude is a meaningful yardstick."""
    a = np.asarray(a, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = max(float(np.max(np.abs(ref))) if ref.size else 0.0,
              float(np.max(np.abs(scale))) if np.size(scale) else 0.0)
    err = float(np.max(np.abs(a - ref))) if ref.size else 0.0
    return err / den if den > 0.0 else err


# Summed-term scale of each force field (orc_forces_scale).
SCALE_OF = {"ax": "scale_a", "ay": "scale_a", "az": "scale_a", "du": "scale_du",
            "mumax": "scale_mu"}


def cancels(k, periodic_z) -> bool:
    """Fields whose exact value is a cancelling sum in these workloads: du and
    mu (v_ij . r_ij = 0 for every pair of a rigidly rotating patch, so both
    sides hold rounding noise) and a_z of the z-periodic patch (no net force
    along the periodic axis). Only these are measured against the summed-term
    scale; ax, ay and a non-periodic az are held to the plain normwise bar."""
    return k in ("du", "mumax") or (k == "az" and bool(periodic_z))


def force_err(k, got, ref, o, periodic_z) -> float:
    """Error of force field k (ax, ay, az, du, mumax) from one call: normwise,
    or against the summed-term scale for a cancelling field; a field that is
    exactly zero in the oracle with a zero term scale must be exactly zero."""
    if not cancels(k, periodic_z):
        return normwise(got, ref)
    sc = o[SCALE_OF[k]]
    if np.max(np.abs(ref)) == 0.0 and np.max(np.abs(sc)) == 0.0:
        return 0.0 if np.max(np.abs(got)) == 0.0 else float("inf")
    return scaled(got, ref, sc)


def state_err(k, got, ref, o, periodic_z, dt) -> float:
    """Error of state field k after one step. v = v0 + dt a and u = u0 + dt du
    inherit the bar of the field they integrate: u and the periodic patch's v_z
    against dt times the summed-term scale, everything else normwise."""
    if k == "u":
        return scaled(got, ref, dt * o["scale_du"])
    if k == "vz" and periodic_z:
        return scaled(got, ref, dt * o["scale_a"])
    return normwise(got, ref)


def check(errs, tol):
    """Assert every error in the dict is within tol (all failures listed)."""
    bad = {k: e for k, e in errs.items() if not e <= tol}
    assert not bad, f"over {tol:g}: " + ", ".join(f"{k}={e:.3e}" for k, e in bad.items())


def canon_oracle(off, idx, ng):
    """Sorted (row, col, gather-flag) triples of the oracle CSR (caller ids)."""
    n = len(off) - 1
    lens = np.diff(off)
    rows = np.repeat(np.arange(n, dtype=np.int64), lens)
    pos = np.arange(len(idx), dtype=np.int64) - np.repeat(off[:-1], lens)
    flag = (pos < np.repeat(ng, lens)).astype(np.int8)
    key = np.lexsort((flag, idx.astype(np.int64), rows))
    return rows[key], idx.astype(np.int64)[key], flag[key]


def canon_gpu(off, idx, ng, order):
    """Same triples for the library's CSR (internal rows mapped to caller ids)."""
    n = len(off) - 1
    lens = np.diff(off)
    rows_int = np.repeat(np.arange(n, dtype=np.int64), lens)
    pos = np.arange(len(idx), dtype=np.int64) - np.repeat(off[:-1], lens)
    flag = (pos < np.repeat(ng, lens)).astype(np.int8)
    rows = order.astype(np.int64)[rows_int]
    cols = order.astype(np.int64)[idx.astype(np.int64)]
    key = np.lexsort((flag, cols, rows))
    return rows[key], cols[key], flag[key]


def same_sets(a, b) -> bool:
    return all(np.array_equal(u, v) for u, v in zip(a, b))
