"""Seeded synthetic initial conditions for the two test problems of the paper.

This module only draws and lays out inputs (positions, velocities, masses,
internal energies, a first smoothing-length guess) and the physical
parameters of each workload. It holds none of the SPH arithmetic (kernel,
density, equation of state, forces, integration); the CUDA path and the CPU
oracle both receive its arrays unchanged.

Workloads (Section 4.1, Table 5):

* Rotating square patch (Section 4.1.1): a 3D cube of particles on a cubic
  lattice filling [-0.5, 0.5]^3, periodic along z, rotating rigidly with
  v_x = omega*y, v_y = -omega*x (the rigid-rotation velocity equation),
  omega = 5. Tait equation of state with rho0 = 1000, c0 = 50, u = 0.
* Evrard collapse (Section 4.1.2): a sphere of radius R = 1 and mass M = 1
  with rho(r) = M / (2 pi R^2 r) (the Evrard density profile), u0 = 0.05,
  ideal gas gamma = 5/3, v = 0. Self-gravity is not part of this build.

Readings where the paper is silent or garbled:

* Lattice jitter: each coordinate gets an independent U[-0.01 dx, 0.01 dx]
  offset; the rigid-rotation velocity is evaluated at the jittered position.
* Evrard radii: rho ~ 1/r gives an enclosed mass M(<r) = M r^2 / R^2, so the
  inverse-CDF radius is r = R * sqrt(U) (the "R*U^(3/2)" form would give
  rho ~ r^(-7/3) and contradicts the profile). Directions are isotropic:
  cos(theta) ~ U[-1, 1], phi ~ U[0, 2 pi).
* First smoothing-length guess: h0 = 1.4395 dx on the lattice, which puts
  about 100 lattice points inside 2 h0; h0 = 1.44 (m / rho(r))^(1/3) for the
  Evrard sphere. The neighbour-count iteration then fixes h.

Random numbers come from numpy's PCG64 generator with a fixed seed, so a
given (workload, size, seed) always yields the same arrays.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

FIELDS = ("x", "y", "z", "vx", "vy", "vz", "m", "h", "u")

EOS_TAIT = 0
EOS_IDEAL = 1


@dataclasses.dataclass
class SphParams:
    """Physical and numerical parameters of one SPH problem instance.

    Both the CUDA binding and the oracle marshal this into their own C struct.
    """

    eos: int = EOS_TAIT          # 0 = Tait (square patch), 1 = ideal gas (Evrard)
    rho0: float = 1000.0         # Tait reference density
    c0: float = 50.0             # Tait reference sound speed
    gamma: float = 5.0 / 3.0     # ideal-gas adiabatic index
    alpha: float = 1.0           # Monaghan artificial viscosity, linear term
    beta: float = 2.0            # Monaghan artificial viscosity, quadratic term
    eta2: float = 0.01           # singularity guard eta^2 in mu_ij
    cfl: float = 0.3             # Courant factor of the time-step criterion
    n_target: int = 100          # target neighbour count
    n_tol: int = 5               # accepted |n - n_target|
    max_h_iter: int = 64         # smoothing-length iterations before giving up
    periodic_z: int = 1          # 1: minimum-image periodicity along z
    lz: float = 1.0              # period along z
    cell_scale: float = 0.0      # neighbour-search cell width / (2 <h>); 0 = library default
    precision: int = 0           # pair arithmetic: 0 FP64-accurate, 1 mixed FP32/double-float,
                                 # 2 native FP64 (the oracle is FP64 throughout)
    pair_threads: int = 0        # lanes per particle in the pair sums (0 = library default)
    defer_lanes: int = 0         # h-search hand-over threshold (0 = library default)

    def as_dict(self) -> dict:
        return dataclasses.asdict(self)


def _empty_state(n: int) -> dict:
    return {f: np.zeros(n, dtype=np.float64) for f in FIELDS}


def square_patch(n_side: int, seed: int, omega: float = 5.0, rho0: float = 1000.0,
                 c0: float = 50.0, jitter: float = 0.01):
    """Rotating square patch on an n_side^3 lattice in [-0.5, 0.5]^3.

    Returns (state, params). state maps each name in FIELDS to a float64
    array of length n_side**3 in lattice order (x fastest).
    """
    if n_side < 1:
        raise ValueError("n_side must be >= 1")
    n = n_side ** 3
    dx = 1.0 / n_side
    k = np.arange(n_side, dtype=np.float64)
    centres = -0.5 + (k + 0.5) * dx
    zz, yy, xx = np.meshgrid(centres, centres, centres, indexing="ij")
    rng = np.random.Generator(np.random.PCG64(seed))
    off = rng.uniform(-jitter * dx, jitter * dx, size=(3, n))
    s = _empty_state(n)
    s["x"][:] = xx.reshape(-1) + off[0]
    s["y"][:] = yy.reshape(-1) + off[1]
    s["z"][:] = zz.reshape(-1) + off[2]
    s["vx"][:] = omega * s["y"]
    s["vy"][:] = -omega * s["x"]
    s["m"][:] = rho0 * dx ** 3
    s["h"][:] = 1.4395 * dx
    s["u"][:] = 0.0
    prm = SphParams(eos=EOS_TAIT, rho0=rho0, c0=c0, periodic_z=1, lz=1.0)
    return s, prm


def evrard(n: int, seed: int, radius: float = 1.0, mass: float = 1.0, u0: float = 0.05,
           gamma: float = 5.0 / 3.0):
    """Evrard sphere: n equal-mass particles with rho(r) = M / (2 pi R^2 r)."""
    if n < 1:
        raise ValueError("n must be >= 1")
    rng = np.random.Generator(np.random.PCG64(seed))
    u_r, u_c, u_p = rng.random((3, n))
    r = radius * np.sqrt(u_r)
    cos_t = 2.0 * u_c - 1.0
    sin_t = np.sqrt(np.maximum(0.0, 1.0 - cos_t * cos_t))
    phi = 2.0 * math.pi * u_p
    s = _empty_state(n)
    s["x"][:] = r * sin_t * np.cos(phi)
    s["y"][:] = r * sin_t * np.sin(phi)
    s["z"][:] = r * cos_t
    m = mass / n
    s["m"][:] = m
    rho_r = mass / (2.0 * math.pi * radius * radius * np.maximum(r, 1e-6 * radius))
    s["h"][:] = 1.44 * np.cbrt(m / rho_r)
    s["u"][:] = u0
    prm = SphParams(eos=EOS_IDEAL, gamma=gamma, periodic_z=0, lz=0.0)
    return s, prm


def random_velocities(state: dict, seed: int, scale: float) -> dict:
    """Replace the velocities by seeded U[-scale, scale] draws (test inputs that
    switch the artificial viscosity on for a good share of the pairs)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = {k: v.copy() for k, v in state.items()}
    v = rng.uniform(-scale, scale, size=(3, len(out["x"])))
    out["vx"][:], out["vy"][:], out["vz"][:] = v
    return out


def perturb_h(state: dict, seed: int, rel: float) -> dict:
    """Multiply each h by a seeded factor in [1 - rel, 1 + rel] (variable-h inputs)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = {k: v.copy() for k, v in state.items()}
    out["h"][:] = out["h"] * rng.uniform(1.0 - rel, 1.0 + rel, size=len(out["h"]))
    return out


def ensemble_sizes(count: int, seed: int, n_min: int = 4096, n_max: int = 262144):
    """Per-instance lattice sides for a batched ensemble: N log-uniform in
    [n_min, n_max], rounded to the nearest cube; omega ~ U[2, 8]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    logn = rng.uniform(math.log(n_min), math.log(n_max), size=count)
    sides = np.maximum(2, np.rint(np.cbrt(np.exp(logn)))).astype(int)
    omegas = rng.uniform(2.0, 8.0, size=count)
    return [(int(s), float(w)) for s, w in zip(sides, omegas)]
