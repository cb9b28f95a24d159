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
