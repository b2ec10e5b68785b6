"""Pins of the oracle's phase-field update and volume correction (Sect. 2.1.1,
Eq. phi_update_muscl and the MUSCL-minmod scheme; Sect. 2.3)."""
import os

import numpy as np

from oracle import oracle as O
from paper_2607_25444_b300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _oracle(nx, ny, nz, dim=3, solid=None, **kw):
    kw.setdefault("periodic", (1, 1, 1))
    o = O.Oracle(I.base_params(nx, ny, nz, dim=dim, **kw))
    o.set_geometry(np.zeros((nz, ny, nx), np.uint8) if solid is None else solid)
    return o


def test_muscl_hand_worked_six_cells():
    tab = np.loadtxt(os.path.join(GOLDEN, "muscl_6cell.txt"))
    phi, ux, exp = tab[:, 0], tab[:, 1], tab[:, 2]
    o = _oracle(6, 1, 1, dim=2, mobility=0.0)
    o.set_fields(phi.reshape(1, 1, 6))
    u = np.zeros((3, 1, 1, 6))
    u[0, 0, 0] = ux
    o.set_velocity(u)
    o.phase_update()
    np.testing.assert_allclose(o.fields()[0].reshape(-1), exp, atol=1e-15)


def test_linear_profile_advected_exactly():
    """Second-order MUSCL reproduces a linear profile's update exactly:
    phi* = phi - u b at interior cells (D = kappa = 0)."""
    n = 16
    x = np.arange(n, dtype=float)
    phi = (0.2 + 0.03 * x).reshape(1, 1, n)
    for ux in (0.3, -0.25):
        o = _oracle(n, 1, 1, dim=2, mobility=0.0)
        o.set_fields(phi)
        u = np.zeros((3, 1, 1, n))
        u[0] = ux
        o.set_velocity(u)
        o.phase_update()
        out = o.fields()[0].reshape(-1)
        np.testing.assert_allclose(out[3:-3], phi.reshape(-1)[3:-3] - ux * 0.03,
                                   atol=1e-15)


def test_tvd_step_profile():
    """Constant-velocity advection of a step: no new extrema and the total
    variation does not grow (TVD, Eq. minmod)."""
    n = 40
    phi = np.where((np.arange(n) >= 10) & (np.arange(n) < 20), 1.0, 0.0)
    o = _oracle(n, 1, 1, dim=2, mobility=0.0)
    o.set_fields(phi.reshape(1, 1, n))
    tv0 = np.abs(np.diff(np.r_[phi, phi[0]])).sum()
    for _ in range(30):
        u = np.zeros((3, 1, 1, n))
        u[0] = 0.4
        o.set_velocity(u)
        o.phase_update()
        cur = o.fields()[0].reshape(-1)
        assert cur.min() >= -1e-15 and cur.max() <= 1 + 1e-15
        tv = np.abs(np.diff(np.r_[cur, cur[0]])).sum()
        assert tv <= tv0 + 1e-13
        tv0 = tv
        o.set_phi(cur.reshape(1, 1, n))


def test_diffusion_term_on_quadratic():
    """With kappa -> 0 (huge width) and u = 0, phi* = phi + D lap_iso phi,
    exact on a quadratic at interior nodes."""
    n = 9
    z, y, x = np.meshgrid(*(np.arange(n, dtype=float),) * 3, indexing="ij")
    phi = 0.3 + 0.01 * x * x - 0.02 * y * z + 0.005 * z * z
    o = _oracle(n, n, n, mobility=0.1, width=1e30)
    o.set_fields(phi)
    o.set_velocity(np.zeros((3, n, n, n)))
    o.phase_update()
    out = o.fields()[0]
    lap = 0.02 + 0.01
    np.testing.assert_allclose(out[1:-1, 1:-1, 1:-1],
                               (phi + 0.1 * lap)[1:-1, 1:-1, 1:-1], atol=1e-14)


def test_periodic_update_conserves_mass_by_telescoping():
    """Without walls every term of Eq. phi_update_muscl is a divergence, so
    sum phi* = sum phi to round-off for random phi and u."""
    n = 8
    phi = I.fast_uniform((n, n, n), seed=3)
    u = I.fast_uniform((3, n, n, n), seed=4, lo=-0.1, hi=0.1)
    o = _oracle(n, n, n, mobility=0.05)
    o.set_fields(phi)
    o.set_velocity(u)
    o.phase_update()
    out = o.fields()[0]
    assert abs(out.sum() - phi.sum()) < 1e-12 * phi.sum()


def test_volume_correction_restores_mass_in_band_only():
    """Sect. 2.3: after the correction the fluid mass equals M_ref; nodes
    outside (eps, 1 - eps) are untouched; solid nodes are untouched."""
    n = 12
    solid = I.walls_z(n, n, n)
    phi = I.droplet(n, n, n, (6, 6, 0.5), 5.0, 4.0).astype(np.float64)
    o = _oracle(n, n, n, solid=solid, periodic=(1, 1, 0), theta_deg=45.0)
    o.set_fields(phi)
    m_ref = o.mass()["m_ref"]
    o.ghost_update()
    o.lb_collide()
    o.phase_update()
    before = o.fields()[0].copy()
    o.volume_correct()
    after = o.fields()[0]
    m = o.mass()
    assert abs(m["m_star"] - m_ref) > 1e-9  # something to correct
    assert abs(o.fluid_mass() - m_ref) < 1e-13 * m_ref
    outside = (before <= 1e-3) | (before >= 1 - 1e-3) | (solid == 1)
    assert np.array_equal(after[outside], before[outside])
    chi = np.where(~outside, before * (1 - before), 0.0)
    assert abs(m["w_sum"] - chi[solid == 0].sum()) < 1e-12 * m["w_sum"]


def test_no_interface_means_no_correction():
    n = 6
    o = _oracle(n, n, n, solid=I.walls_z(n, n, n), periodic=(1, 1, 0),
                mobility=0.0)
    phi = np.zeros((n, n, n))
    phi[:, :, :3] = 1.0
    phi[:, :, 3:] = 0.0
    o.set_fields(phi)
    o.set_mass_ref(o.mass()["m_ref"] + 1.0)
    o.phase_update()
    before = o.fields()[0].copy()
    o.volume_correct()
    m = o.mass()
    assert m["lam"] == 0.0
    assert np.array_equal(o.fields()[0], before)


def test_full_step_mass_held_with_wetting():
    n = 16
    solid = I.walls_z(n, n, n)
    phi = I.droplet(n, n, n, (8, 8, 0.5), 6.0, 4.0).astype(np.float64)
    o = _oracle(n, n, n, solid=solid, periodic=(1, 1, 0), theta_deg=40.0,
                sigma=0.01)
    o.set_fields(phi)
    m0 = o.fluid_mass()
    o.step(30)
    assert abs(o.fluid_mass() - m0) < 1e-13 * m0
