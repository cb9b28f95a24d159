"""Pins of the oracle's variants of Table 1 (Wendland C2 and sinc kernels, IAD
gradients) and of the initial-pressure series of Section 5.1.1, against facts
fixed by the mathematics: kernel normalisation by independent quadrature, a
closed-form normalisation, finite differences, lattice sums by integer
enumeration, exactness of IAD on linear fields, conservation laws, and a
finite-difference Poisson solve."""
import math

import numpy as np
import pytest

from paper_1809_08013_gb300 import ics

KERNELS = [(1, 0), (2, 2), (2, 3), (2, 5), (2, 8), (2, 12)]  # (kernel, sinc_n)


def _prm(kernel=0, sinc_n=5, gradients=0, base=None):
    p = base if base is not None else ics.SphParams()
    p.kernel, p.sinc_n, p.gradients = kernel, sinc_n, gradients
    return p


# --------------------------------------------------------------------------
# Kernels
# --------------------------------------------------------------------------
@pytest.mark.parametrize("kernel,sn", KERNELS)
@pytest.mark.parametrize("h", [1.0, 0.0137])
def test_variant_kernel_normalisation(orc, kernel, sn, h):
    # 4 pi int_0^{2h} r^2 W(r, h) dr = 1, by adaptive quadrature (scipy),
    # independent of the oracle's own Simpson rule for B_n
    quad = pytest.importorskip("scipy.integrate").quad
    prm = _prm(kernel, sn)
    val, err = quad(lambda r: 4.0 * math.pi * r * r * orc.kernel_W(prm, r, h), 0.0, 2.0 * h,
                    epsabs=1e-15, epsrel=1e-13, limit=200)
    assert abs(val - 1.0) < 1e-12


def test_sinc_square_normalisation_closed_form(orc):
    # n = 2: int_0^2 q^2 sinc^2(pi q / 2) dq = (8 / pi^3) int_0^pi sin^2 x dx = 4 / pi^2,
    # so B_2 = 1 / (4 pi * 4 / pi^2) = pi / 16
    assert orc.sinc_norm(2) == pytest.approx(math.pi / 16.0, rel=1e-14)


@pytest.mark.parametrize("kernel,sn", KERNELS)
def test_variant_kernel_support_and_shape(orc, kernel, sn):
    prm = _prm(kernel, sn)
    h = 0.7
    w0 = orc.kernel_W(prm, 0.0, h)
    qs = np.linspace(0.0, 2.0, 401)
    w = np.array([orc.kernel_W(prm, q * h, h) for q in qs])
    assert np.all(np.diff(w) <= 0.0) and w0 > 0.0      # monotone, positive at 0
    assert w[-1] == 0.0 and orc.kernel_W(prm, 2.5 * h, h) == 0.0
    # continuous at the edge of the support: the kernel and its slope vanish at q = 2
    assert orc.kernel_W(prm, (2.0 - 1e-6) * h, h) < 1e-9 * w0
    assert abs(orc.kernel_dWdr(prm, (2.0 - 1e-6) * h, h)) < 1e-5 * w0 / h
    assert orc.kernel_dWdr(prm, 0.0, h) == 0.0         # smooth at the origin
    # the same scaling with h as the spline: h^3 W(q h, h) depends on q only
    for q in (0.3, 1.1, 1.7):
        assert 0.29 ** 3 * orc.kernel_W(prm, q * 0.29, 0.29) == pytest.approx(
            h ** 3 * orc.kernel_W(prm, q * h, h), rel=1e-13)


@pytest.mark.parametrize("kernel,sn", KERNELS)
@pytest.mark.parametrize("q", [0.05, 0.4, 0.93, 1.3, 1.81])
def test_variant_kernel_derivative_matches_central_difference(orc, kernel, sn, q):
    prm = _prm(kernel, sn)
    h = 0.8
    r = q * h
    eps = 1e-6 * h
    fd = (orc.kernel_W(prm, r + eps, h) - orc.kernel_W(prm, r - eps, h)) / (2 * eps)
    scale = orc.kernel_W(prm, 0.0, h) / h
    assert abs(orc.kernel_dWdr(prm, r, h) - fd) <= 1e-8 * scale


@pytest.mark.parametrize("kernel,sn", [(1, 5), (2, 5)])
def test_variant_lattice_density_equals_integer_enumeration(orc, kernel, sn):
    n = 12
    s, prm = ics.square_patch(n, seed=0, jitter=0.0)
    _prm(kernel, sn, base=prm)
    dx = 1.0 / n
    hh = 1.45 * dx
    h = np.full(n ** 3, hh)
    off, idx, ng = orc.csr(prm, s["x"], s["y"], s["z"], h)
    rho = orc.density(prm, s["x"], s["y"], s["z"], s["m"], h, off, idx, ng)
    m = s["m"][0]
    expect = 0.0
    a = np.arange(-3, 4)
    for i in a:
        for j in a:
            for k in a:
                d2 = float(i * i + j * j + k * k)
                if d2 * dx * dx < (2 * hh) ** 2:
                    expect += m * orc.kernel_W(prm, dx * math.sqrt(d2), hh)
    inner = (np.abs(s["x"]) < 0.5 - 3 * dx) & (np.abs(s["y"]) < 0.5 - 3 * dx)
    assert np.max(np.abs(rho[inner] - expect)) <= 1e-13 * expect


@pytest.mark.parametrize("kernel,sn", [(1, 5), (2, 3), (2, 6)])
def test_variant_force_is_gradient_of_total_density(orc, kernel, sn):
    # A = 1, no viscosity, equal masses: a_i = -d(sum_k rho_k)/dr_i at fixed
    # per-particle h (pins the variant dW/dr, both h terms and the sign)
    s, prm = ics.square_patch(8, seed=131)
    s = ics.perturb_h(s, seed=132, rel=0.25)
    _prm(kernel, sn, base=prm)
    prm.alpha = prm.beta = 0.0
    prm.periodic_z = 0
    h = s["h"]
    off, idx, ng = orc.csr(prm, s["x"], s["y"], s["z"], h)
    rho = orc.density(prm, s["x"], s["y"], s["z"], s["m"], h, off, idx, ng)
    ax, ay, az, _, _ = orc.forces(prm, s, rho, rho * rho, np.ones_like(rho), off, idx)

    def total_rho(xx, yy, zz):
        o, ii, g = orc.csr(prm, xx, yy, zz, h)
        return orc.density(prm, xx, yy, zz, s["m"], h, o, ii, g).sum()

    eps = 1e-6 / 8
    for i in (0, 100, 255, 300, 511):
        grad = []
        for comp in ("x", "y", "z"):
            pp = {k: s[k].copy() for k in ("x", "y", "z")}
            mm = {k: s[k].copy() for k in ("x", "y", "z")}
            pp[comp][i] += eps
            mm[comp][i] -= eps
            grad.append((total_rho(pp["x"], pp["y"], pp["z"])
                         - total_rho(mm["x"], mm["y"], mm["z"])) / (2 * eps))
        a = np.array([ax[i], ay[i], az[i]])
        scale = max(np.abs(grad).max(), 1e-3 * np.abs(ax).max())
        assert np.allclose(a, -np.array(grad), rtol=0, atol=1e-5 * scale), i


# --------------------------------------------------------------------------
# IAD gradients
# --------------------------------------------------------------------------
def _iad_inputs(orc, s, prm):
    h, _, _, _ = orc.h_iterate(prm, s["x"], s["y"], s["z"], s["h"])
    s = dict(s)
    s["h"] = h
    off, idx, ng = orc.csr(prm, s["x"], s["y"], s["z"], h)
    rho = orc.density(prm, s["x"], s["y"], s["z"], s["m"], h, off, idx, ng)
    return s, off, idx, ng, rho


@pytest.mark.parametrize("kernel", [0, 1, 2])
def test_iad_gradient_exact_for_linear_fields(orc, kernel):
    # C_i sum_j V_j (f_j - f_i) W_ij (r_j - r_i) = C_i tau_i b = b for f = a + b.r,
    # at every particle (the surface ones included)
    s, prm = ics.evrard(2500, seed=141)
    _prm(kernel, 4, 1, base=prm)
    s, off, idx, ng, rho = _iad_inputs(orc, s, prm)
    cm = orc.iad(prm, s, rho, off, idx, ng)
    b = np.array([2.0, -5.0, 0.5])
    f = 3.0 + b[0] * s["x"] + b[1] * s["y"] + b[2] * s["z"]
    g = np.stack(orc.iad_gradient(prm, s, rho, off, idx, ng, cm, f))
    assert np.max(np.abs(g - b[:, None])) <= 1e-9 * np.abs(b).max()
    # on the periodic patch, for a field linear in x and y
    s2, prm2 = ics.square_patch(9, seed=142)
    _prm(kernel, 4, 1, base=prm2)
    s2, off, idx, ng, rho = _iad_inputs(orc, s2, prm2)
    cm = orc.iad(prm2, s2, rho, off, idx, ng)
    f = 1.0 - 4.0 * s2["x"] + 7.0 * s2["y"]
    g = np.stack(orc.iad_gradient(prm2, s2, rho, off, idx, ng, cm, f))
    assert np.max(np.abs(g - np.array([-4.0, 7.0, 0.0])[:, None])) <= 1e-9 * 7.0


def test_iad_matrix_on_perfect_lattice_is_enumerated_sum(orc):
    # interior of a perfect lattice, uniform h and rho: by the cubic symmetry
    # tau = (m / rho) (sum_lattice |d|^2 W(|d|, h) / 3) I
    n = 14
    s, prm = ics.square_patch(n, seed=0, jitter=0.0)
    prm.gradients = 1
    dx = 1.0 / n
    hh = 1.45 * dx
    s["h"][:] = hh
    off, idx, ng = orc.csr(prm, s["x"], s["y"], s["z"], s["h"])
    rho = np.full(n ** 3, 997.0)
    cm = orc.iad(prm, s, rho, off, idx, ng)
    tot = 0.0
    a = np.arange(-3, 4)
    for i in a:
        for j in a:
            for k in a:
                d2 = float(i * i + j * j + k * k) * dx * dx
                if 0.0 < d2 < (2 * hh) ** 2:
                    tot += d2 * orc.W(math.sqrt(d2), hh)
    diag = 1.0 / (s["m"][0] / 997.0 * tot / 3.0)
    inner = (np.abs(s["x"]) < 0.5 - 3 * dx) & (np.abs(s["y"]) < 0.5 - 3 * dx)
    assert inner.sum() > 100
    for comp in (0, 3, 5):
        assert np.max(np.abs(cm[inner, comp] - diag)) <= 1e-12 * diag
    for comp in (1, 2, 4):
        assert np.max(np.abs(cm[inner, comp])) <= 1e-12 * diag


@pytest.mark.parametrize("kernel", [0, 1, 2])
def test_iad_forces_conserve_momentum_and_energy(orc, kernel):
    s, prm = ics.square_patch(10, seed=151)
    s = ics.random_velocities(s, seed=152, scale=3.0)
    s = ics.perturb_h(s, seed=153, rel=0.2)
    _prm(kernel, 5, 1, base=prm)
    o = orc.pipeline(prm, s)
    m = s["m"]
    a = np.stack([o["ax"], o["ay"], o["az"]])
    for k in range(3):
        assert abs(np.sum(m * a[k])) <= 1e-13 * np.sum(m * np.abs(a[k]))
    pw = m * (s["vx"] * o["ax"] + s["vy"] * o["ay"] + s["vz"] * o["az"])
    assert abs(pw.sum() + np.sum(m * o["du"])) <= 1e-13 * (np.abs(pw).sum() +
                                                          np.sum(m * np.abs(o["du"])))
    assert np.count_nonzero(o["mumax"]) > 0.5 * len(m)
    # IAD changes the forces (the variant is really selected)
    prm.gradients = 0
    o0 = orc.pipeline(prm, s)
    assert np.max(np.abs(o0["ax"] - o["ax"])) > 1e-3 * np.max(np.abs(o0["ax"]))


def test_iad_static_evrard_has_exact_zero_viscosity(orc):
    s, prm = ics.evrard(3000, seed=161)
    prm.gradients = 1
    o = orc.pipeline(prm, s)
    assert np.all(o["du"] == 0.0) and np.all(o["mumax"] == 0.0)
    assert np.all(np.isfinite(o["ax"]))


def test_iad_uniform_pressure_lattice_interior_is_force_free(orc):
    # uniform p, rho and h on a perfect lattice: where a particle and all its
    # neighbours have full neighbourhoods (6 dx from the free surface) every
    # pair term has its mirror image, so the accelerations cancel
    n = 16
    s, prm = ics.square_patch(n, seed=0, jitter=0.0, omega=0.0)
    prm.gradients = 1
    dx = 1.0 / n
    s["h"][:] = 1.45 * dx
    off, idx, ng = orc.csr(prm, s["x"], s["y"], s["z"], s["h"])
    rho = np.full(n ** 3, 1000.0)
    cm = orc.iad(prm, s, rho, off, idx, ng)
    p = np.full(n ** 3, 250.0)
    ax, ay, az, du, _ = orc.forces(prm, s, rho, p, np.ones_like(rho), off, idx, cm)
    sa, _, _ = orc.forces_scale(prm, s, rho, p, np.ones_like(rho), off, idx, cm)
    inner = (np.abs(s["x"]) < 0.5 - 6 * dx) & (np.abs(s["y"]) < 0.5 - 6 * dx)
    assert inner.sum() >= 256
    for a in (ax, ay, az):
        assert np.max(np.abs(a[inner])) <= 1e-13 * np.max(sa)
    # near the free surface the pressure pushes outwards
    edge = s["x"] > 0.5 - dx
    assert np.all(ax[edge] > 0.0)


# --------------------------------------------------------------------------
# Initial pressure of the rotating square patch (Section 5.1.1)
# --------------------------------------------------------------------------
def test_patch_pressure_vanishes_on_the_edges_and_is_symmetric():
    t = np.linspace(-0.5, 0.5, 23)
    for edge in (-0.5, 0.5):
        pe = ics.patch_pressure(np.full_like(t, edge), t, 5.0, 1000.0)
        pf = ics.patch_pressure(t, np.full_like(t, edge), 5.0, 1000.0)
        assert np.max(np.abs(pe)) < 1e-9 and np.max(np.abs(pf)) < 1e-9
    x, y = np.meshgrid(t, t)
    p = ics.patch_pressure(x, y, 5.0, 1000.0)
    assert np.allclose(p, p.T, rtol=0, atol=1e-9) and np.allclose(p, p[:, ::-1], rtol=0, atol=1e-9)
    assert np.all(p[1:-1, 1:-1] < 0.0)
    # p scales as rho omega^2 L^2
    assert ics.patch_pressure(0.1, 0.2, 3.0, 10.0) == pytest.approx(
        ics.patch_pressure(0.1, 0.2, 5.0, 1000.0) * (10.0 * 9.0) / (1000.0 * 25.0), rel=1e-13)


def test_patch_pressure_solves_the_poisson_problem():
    # lap p = 2 rho omega^2 in the square, p = 0 on its edges: a second-order
    # finite-difference solve on two grids, Richardson-extrapolated, gives the
    # solution at a few points to ~1e-6; the series must agree
    sp = pytest.importorskip("scipy.sparse")
    spl = pytest.importorskip("scipy.sparse.linalg")
    rho, omega = 1000.0, 5.0
    pts = [(0.0, 0.0), (0.25, 0.0), (-0.25, 0.125), (0.375, 0.375)]

    def fd(N):
        hgrid = 1.0 / N
        m = N - 1
        one = np.ones(m)
        T = sp.diags([one[:-1], -2 * one, one[:-1]], [-1, 0, 1]) / hgrid ** 2
        I = sp.identity(m)
        A = (sp.kron(I, T) + sp.kron(T, I)).tocsc()
        u = spl.spsolve(A, np.full(m * m, 2.0 * rho * omega ** 2)).reshape(m, m)
        out = []
        for (x, y) in pts:
            i = int(round((y + 0.5) * N)) - 1
            j = int(round((x + 0.5) * N)) - 1
            out.append(u[i, j])
        return np.array(out)

    a, b = fd(128), fd(256)
    ref = b + (b - a) / 3.0
    got = ics.patch_pressure(np.array([p[0] for p in pts]), np.array([p[1] for p in pts]),
                             omega, rho, terms=256)
    assert np.max(np.abs(got - ref)) <= 2e-5 * np.max(np.abs(ref))


def test_pressure_ic_masses_follow_the_tait_inverse():
    s, prm = ics.square_patch(10, seed=5, pressure_ic=True)
    s0, _ = ics.square_patch(10, seed=5)
    for k in ("x", "y", "z", "vx", "vy", "h"):
        assert np.array_equal(s[k], s0[k])
    rho = s["m"] / 0.1 ** 3
    p = (prm.c0 ** 2 * prm.rho0 / 7.0) * ((rho / prm.rho0) ** 7 - 1.0)
    p0 = ics.patch_pressure(s["x"], s["y"], 5.0, prm.rho0)
    assert np.max(np.abs(p - p0)) <= 1e-9 * np.max(np.abs(p0))
