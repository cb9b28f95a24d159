"""Seeded synthetic initial conditions for the two test problems of the paper.

This module only draws and lays out inputs (positions, velocities, masses,
internal energies, a first smoothing-length guess) and the physical
parameters of each workload. It holds none of the SPH arithmetic (kernel,
density, equation of state, forces, integration); the CUDA path and the CPU
oracle both receive its arrays unchanged.

Workloads (Section 5.1, Table 5):

* Rotating square patch (Section 5.1.1): a 3D cube of particles on a cubic
  lattice filling [-0.5, 0.5]^3, periodic along z, rotating rigidly with
  v_x = omega*y, v_y = -omega*x (the rigid-rotation velocity equation),
  omega = 5. Tait equation of state with rho0 = 1000, c0 = 50, u = 0.
* Evrard collapse (Section 5.1.2): a sphere of radius R = 1 and mass M = 1
  with rho(r) = M / (2 pi R^2 r) (the Evrard density profile), u0 = 0.05,
  ideal gas gamma = 5/3, v = 0. Self-gravity (Algorithm 1 step 4) is not computed.

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

KERNEL_M4 = 0        # M4 cubic spline (Table 1)
KERNEL_WENDLAND = 1  # Wendland C2 (Table 1)
KERNEL_SINC = 2      # sinc kernel S(pi q / 2)^n (Table 1)

GRAD_KERNEL = 0      # kernel-derivative gradients (Table 1)
GRAD_IAD = 1         # integral approach to derivatives (Table 1)


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
    kernel: int = KERNEL_M4      # 0 M4 cubic spline, 1 Wendland C2, 2 sinc
    gradients: int = GRAD_KERNEL # 0 kernel derivatives, 1 IAD
    sinc_n: int = 5              # exponent of the sinc kernel (2..12)
    list_skin: float = 0.0       # h-search candidate lists' skin (> 0 turns them on;
                                 # the oracle has none)

    def as_dict(self) -> dict:
        return dataclasses.asdict(self)


def _empty_state(n: int) -> dict:
    return {f: np.zeros(n, dtype=np.float64) for f in FIELDS}


def patch_pressure(x, y, omega: float, rho: float, side: float = 1.0, terms: int = 64,
                   chunk: int = 1 << 15):
    """Initial pressure of the rotating square patch (Section 5.1.1): the
    solution of the incompressible pressure Poisson equation lap p = 2 rho
    omega^2 on the square of side L with p = 0 on its edges, as the double
    sine series over odd m and n (the printed series is garbled: it writes x
    where y is meant, and its m = 0 or n = 0 terms are singular),

      p = rho sum_{m, n odd} -32 omega^2 / (m n pi^2 ((m pi/L)^2 + (n pi/L)^2))
                             sin(m pi x'/L) sin(n pi y'/L),

    with x' = x + L/2, y' = y + L/2 measured from the patch corner. `terms`
    odd values of each index are summed."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    k = 2.0 * np.arange(terms, dtype=np.float64) + 1.0   # odd m, n
    kk = (k * math.pi / side) ** 2
    coef = -32.0 * omega * omega / (np.outer(k, k) * math.pi ** 2 * (kk[:, None] + kk[None, :]))
    out = np.empty(x.shape)
    for a in range(0, x.size, chunk):
        xs = x.reshape(-1)[a:a + chunk] + 0.5 * side
        ys = y.reshape(-1)[a:a + chunk] + 0.5 * side
        sx = np.sin(np.outer(k, xs) * (math.pi / side))
        sy = np.sin(np.outer(k, ys) * (math.pi / side))
        out.reshape(-1)[a:a + chunk] = rho * np.einsum("mi,mn,ni->i", sx, coef, sy)
    return out


def square_patch(n_side: int, seed: int, omega: float = 5.0, rho0: float = 1000.0,
                 c0: float = 50.0, jitter: float = 0.01, pressure_ic: bool = False,
                 pressure_terms: int = 64):
    """Rotating square patch on an n_side^3 lattice in [-0.5, 0.5]^3.

    Returns (state, params). state maps each name in FIELDS to a float64
    array of length n_side**3 in lattice order (x fastest).

    pressure_ic: start from the series pressure of patch_pressure instead of
    p = 0. Reading: with the Tait equation the pressure fixes the density,
    rho = rho0 (1 + 7 p / (c0^2 rho0))^(1/7), and each particle carries the
    mass rho dx^3 of its lattice cell, so the summed density starts near it.
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
    if pressure_ic:
        p0 = patch_pressure(s["x"], s["y"], omega, rho0, 1.0, pressure_terms)
        s["m"][:] = rho0 * (1.0 + 7.0 * p0 / (c0 * c0 * rho0)) ** (1.0 / 7.0) * dx ** 3
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
