"""Physics pins of the full oracle step against textbook closed forms and the
paper's own checks: Poiseuille flow, shear-wave decay (nu <-> omega,
Eq. nuomega), Laplace's law (Eqs. pstar, Fcap), the equilibrium tanh profile
of the CAC equation (Eq. kappa_delta), the static contact angle (Sect. 3.1),
and the D3Q27 / D2Q9 equivalence on a one-node-thick periodic slab."""
import math

import numpy as np
import pytest

from oracle import diagnostics as Dg
from oracle import oracle as O
from paper_2607_25444_b300 import inputs as I

CS2 = 1.0 / 3.0


def test_poiseuille_body_force():
    """Single phase (phi = 1) between halfway bounce-back walls driven by
    F_ext = (rho - rho_g) g: u(y) = a/(2 nu) (y - y0)(H - (y - y0)) with
    a = F/rho, walls at y0 = 0.5 and y0 + H."""
    H = 32
    ny = H + 2
    nu = 0.1
    p = I.base_params(1, ny, 1, dim=2, periodic=(1, 0, 1), rho_l=1.0,
                      rho_g=0.5, nu_l=nu, nu_g=nu, gravity=(1e-6, 0, 0))
    o = O.Oracle(p)
    o.set_geometry(I.walls_y(1, ny, 1))
    o.set_fields(np.ones((1, ny, 1)))
    o.step(20000)
    ux = o.fields()[1][0, 0, :, 0]
    a = 0.5e-6
    y = np.arange(ny) - 0.5
    exact = a / (2 * nu) * y * (H - y)
    assert np.abs(ux[1:-1] - exact[1:-1]).max() < 1e-3 * exact.max()


def _layered_channel(rho_g, nu_l, nu_g, H=48, g=1e-6, W=4.0, steps=20000):
    """Two-phase channel flow along x between halfway bounce-back walls at
    y = 1/2 and y = H + 1/2 (2D, one node in x): liquid (phi = 1) in the
    lower half, gas above, a flat tanh interface of width W at mid-height, a
    body force F_ext = (rho(phi) - rho_g) g along x that acts on the liquid
    only. Returns the oracle's u_x(y), the continuum profile and the node
    heights."""
    from scipy.integrate import cumulative_trapezoid
    ny = H + 2
    p = I.base_params(1, ny, 1, dim=2, periodic=(1, 0, 1), rho_l=1.0,
                      rho_g=rho_g, nu_l=nu_l, nu_g=nu_g, gravity=(g, 0, 0),
                      sigma=0.01, width=W)
    o = O.Oracle(p)
    o.set_geometry(I.walls_y(1, ny, 1))
    y = np.arange(ny, dtype=float)
    h = 0.5 + H / 2
    o.set_fields((0.5 * (1 + np.tanh(2 * (h - y) / W))).reshape(1, ny, 1))
    o.step(steps)
    ux = o.fields()[1][0, 0, :, 0]
    # steady shear flow of the continuum with the same diffuse layers:
    # d/dy (mu du/dy) = -(rho - rho_g) g, u = 0 on both walls, with
    # mu = rho_g nu_g + (rho_l nu_l - rho_g nu_g) phi and the same tanh phi
    yy = np.linspace(0.5, ny - 1.5, 200001)
    ph = 0.5 * (1 + np.tanh(2 * (h - yy) / W))
    mu = rho_g * nu_g + (nu_l - rho_g * nu_g) * ph
    F = cumulative_trapezoid((1.0 - rho_g) * ph * g, yy, initial=0.0)
    inv_mu = cumulative_trapezoid(1.0 / mu, yy, initial=0.0)
    f_mu = cumulative_trapezoid(F / mu, yy, initial=0.0)
    exact = (f_mu[-1] / inv_mu[-1]) * inv_mu - f_mu
    return ux, np.interp(y, yy, exact), y, h


@pytest.mark.parametrize("rho_g,nu_l,nu_g", [(0.1, 0.1, 0.1), (0.05, 0.05, 0.1)])
def test_layered_two_phase_channel_flow(rho_g, nu_l, nu_g):
    """Pins the viscous correction F_nu (Eqs. Fsplit, Fnu, mu_mix_linear):
    with a density jump across the layers (ratio 10 or 20) and a dynamic
    viscosity ratio of 10, the shear stress mu du/dy is continuous across
    the interface only if F_nu = -(nu omega / c_s^2) Pi . grad rho restores
    the variable-density viscous term; without it the lattice carries
    nu du/dy instead. Away from the interface band the oracle's steady
    profile must match the continuum one within 2.5 % of its maximum
    (it does to 0.8 %; with F_nu dropped the error is 29-43 %, with its
    sign flipped 60 %)."""
    ux, exact, y, h = _layered_channel(rho_g, nu_l, nu_g)
    far = (np.abs(y - h) > 8.0) & (y >= 1) & (y <= len(y) - 2)
    err = np.abs(ux - exact)[far].max() / np.abs(exact).max()
    assert err < 0.025, err


def test_shear_wave_decay_rate():
    """u_x = U sin(k y) decays as exp(-nu k^2 t) (Eq. nuomega)."""
    ny = 32
    nu = 0.1
    p = I.base_params(1, ny, 1, dim=2, periodic=(1, 1, 1), nu_l=nu, nu_g=nu)
    o = O.Oracle(p)
    o.set_geometry(np.zeros((1, ny, 1), np.uint8))
    k = 2 * math.pi / ny
    u = np.zeros((3, 1, ny, 1))
    u[0, 0, :, 0] = 1e-3 * np.sin(k * np.arange(ny))
    o.set_fields(np.ones((1, ny, 1)), u)
    o.step(100)
    a1 = np.abs(o.fields()[1][0]).max()
    o.step(400)
    a2 = np.abs(o.fields()[1][0]).max()
    rate = -math.log(a2 / a1) / 400
    assert abs(rate - nu * k * k) < 1e-2 * nu * k * k


def _laplace(dim, n, R, rho_g, steps, avg):
    """Pressure jump p_in - p_out (p = rho c_s^2 p*, Eq. pstar), averaged over
    the last ``avg`` steps to filter the acoustic modes, and sigma/R (2D) or
    2 sigma/R (3D) with R from the liquid area or volume."""
    sigma = 0.01
    nz = n if dim == 3 else 1
    p = I.base_params(n, n, nz, dim=dim, periodic=(1, 1, 1), sigma=sigma,
                      rho_l=1.0, rho_g=rho_g, nu_l=0.3, nu_g=0.3)
    o = O.Oracle(p)
    o.set_geometry(np.zeros((nz, n, n), np.uint8))
    c = (n / 2, n / 2, nz / 2 if dim == 3 else 0.0)
    o.set_fields(I.droplet(n, n, nz, c, R, 4.0, dtype=np.float64))
    o.step(steps - avg)
    acc = []
    for _ in range(avg // 20):
        o.step(20)
        phi, u, ps = o.fields()
        rho = rho_g + (1.0 - rho_g) * phi
        pres = rho * CS2 * ps
        acc.append(pres[phi > 0.99].mean() - pres[phi < 0.01].mean())
    vol = phi.sum()
    Rm = math.sqrt(vol / math.pi) if dim == 2 else (3 * vol / (4 * math.pi)) ** (1 / 3)
    exp = sigma / Rm if dim == 2 else 2 * sigma / Rm
    return float(np.mean(acc)), exp


def test_laplace_2d_scaling():
    """Delta p = sigma/R: the jump scales as 1/R (within 3% between R = 12 and
    R = 20) and matches sigma/R within 8% (the W = 4 diffuse profile carries
    a few per cent less tension than nominal in 2D)."""
    r = {}
    for R in (12.0, 20.0):
        dp, exp = _laplace(2, 64, R, 1.0, 3000, 1000)
        r[R] = dp / exp
        assert abs(r[R] - 1.0) < 0.08, r
    assert abs(r[12.0] / r[20.0] - 1.0) < 0.03, r


def test_laplace_2d_density_ratio():
    """Density ratio 10: the pressure p = rho c_s^2 p* (Eq. pstar) with the
    correction force F_p (Eq. Fp) still gives Delta p = sigma/R."""
    dp, exp = _laplace(2, 64, 16.0, 0.1, 3000, 1000)
    assert abs(dp / exp - 1.0) < 0.08, (dp, exp)


def test_laplace_3d():
    dp, exp = _laplace(3, 24, 7.0, 1.0, 600, 200)
    assert abs(dp / exp - 1.0) < 0.05, (dp, exp)


def test_flat_interface_relaxes_to_set_width():
    """The fixed point of the CAC equation is phi = 1/2 [1 + tanh(2x/delta)]
    when kappa = 4D/delta (Eq. kappa_delta). A start of width 2 relaxes to
    width delta = 4, measured through int phi (1 - phi) dx = delta/4 per
    interface (two interfaces here)."""
    n = 64
    p = I.base_params(n, 1, 1, dim=2, periodic=(1, 1, 1), sigma=0.01,
                      mobility=0.05)
    o = O.Oracle(p)
    o.set_geometry(np.zeros((1, 1, n), np.uint8))
    x = np.arange(n, dtype=float)
    phi = 0.5 * (1 + np.tanh(2 * (np.minimum(x - 16, 48 - x)) / 2.0))
    assert abs(2 * np.sum(phi * (1 - phi)) - 2.0) < 0.02
    o.set_fields(phi.reshape(1, 1, n))
    o.step(3000)
    cur = o.fields()[0].reshape(-1)
    width = 2 * np.sum(cur * (1 - cur))
    assert abs(width - 4.0) < 0.02 * 4.0, width


def test_d3q27_slab_matches_d2q9_on_flat_walls():
    """A D3Q27 run on a periodic slab one node thick reproduces the D2Q9 run
    (weights lump exactly, flat-wall normals and donors coincide)."""
    p2, solid, phi = I.static_droplet_2d(60.0)
    o2 = O.Oracle(p2)
    o2.set_geometry(solid)
    o2.set_fields(phi.astype(np.float64))
    p3 = dict(p2, dim=3)
    o3 = O.Oracle(p3)
    o3.set_geometry(solid)
    o3.set_fields(phi.astype(np.float64))
    o2.step(50)
    o3.step(50)
    f2, u2, p2_ = o2.fields()
    f3, u3, p3_ = o3.fields()
    assert np.abs(f2 - f3).max() < 1e-12
    assert np.abs(u2 - u3).max() < 1e-13
    assert np.abs(p2_ - p3_).max() < 1e-12


@pytest.mark.slow
def test_static_contact_angle_2d():
    """2D static droplet (128 x 64, R = 20, W = 4): the measured angle
    follows the imposed one within 8 deg and lies on the correct side of
    90 deg. Sect. 3.1 reports deviations of a few degrees at R0 = 40 in 3D;
    at R = 20 in 2D the oracle settles (10000 to 40000 steps agree within
    0.01 deg) at 55.7 deg for 60 and 127.4 deg for 120: the first-order
    extrapolation of the wetting condition under-shoots a hydrophilic angle
    and over-shoots a hydrophobic one."""
    got = {}
    for th in (60.0, 120.0):
        p, solid, phi = I.static_droplet_2d(th)
        o = O.Oracle(p)
        o.set_geometry(solid)
        o.set_fields(phi.astype(np.float64))
        o.step(10000)
        got[th], _ = Dg.contact_angle(o.fields()[0][0], 0.5)
    assert 52.0 < got[60.0] < 60.0, got
    assert 120.0 < got[120.0] < 128.0, got


def test_contact_angle_fit_on_exact_circle():
    """The circle-fit diagnostic returns the angle of an exact circular cap
    (Eq. measured_contact_angle)."""
    nx, nz = 160, 80
    for th in (45.0, 90.0, 135.0):
        R = 30.0
        z0 = 0.5 - R * math.cos(math.radians(th))
        z, x = np.meshgrid(np.arange(nz, dtype=float), np.arange(nx, dtype=float),
                           indexing="ij")
        r = np.sqrt((x - 80) ** 2 + (z - z0) ** 2)
        phi = 0.5 * (1 + np.tanh(2 * (R - r) / 4))
        phi[z < 0.5] = 0.0
        got, _ = Dg.contact_angle(phi, 0.5, z_min=1.0)
        assert abs(got - th) < 0.5
