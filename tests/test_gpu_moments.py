"""Moment-form storage (CACL_F32_MOMENTS, the paper's thread-safe form of
Sect. 2.1): each node keeps the 17 coefficients of its post-collision
polynomial and the collide-stream rebuilds the populations it pulls from
its neighbours' coefficients. From a state at rest it is bit-identical to
FP32 population storage; from a moving start it matches the FP64 oracle."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2607_25444_b300 import inputs as I

pytestmark = pytest.mark.gpu


def _run(p, solid, phi, steps, theta=None, u=None):
    from paper_2607_25444_b300 import cacl
    s = cacl.Solver(p)
    s.set_geometry(solid)
    if theta is not None:
        s.set_contact_angle(theta)
    s.set_fields(phi, u)
    s.step(steps)
    s.check_finite()
    out = s.fields() + (s.populations(),)
    s.close()
    return out


def _cases():
    nx, ny, nz = 40, 36, 30
    p = I.base_params(nx, ny, nz, sigma=0.01, rho_g=0.2, nu_g=0.1,
                      theta_deg=60.0, gravity=(0.0, 0.0, -1e-5))
    theta = (50.0 + 60.0 * I.fast_uniform((nz, ny, nx), seed=3)).astype(np.float32)
    yield "walls", p, I.walls_z(nx, ny, nz), I.droplet(nx, ny, nz, (20, 18, 0.5), 9.0, 4.0), theta
    nx, ny, nz = 24, 24, 40
    p = I.base_params(nx, ny, nz, sigma=0.01, rho_g=0.02, theta_deg=60.0,
                      gravity=(0.0, 0.0, -2e-5))
    solid = I.orifice_plate(nx, ny, nz, 16, 4, 8)
    phi = I.droplet(nx, ny, nz, (12, 12, 28), 6.0, 4.0)
    yield "orifice", p, solid, phi, None
    nx, ny, nz = 33, 20, 18  # ragged tiles in x, y and z, fully periodic
    p = I.base_params(nx, ny, nz, sigma=0.01, rho_g=0.5, periodic=(1, 1, 1))
    yield "periodic", p, np.zeros((nz, ny, nx), np.uint8), \
        I.droplet(nx, ny, nz, (16, 10, 9), 6.0, 4.0), None


@pytest.mark.parametrize("name,p,solid,phi,theta", list(_cases()),
                         ids=lambda v: v if isinstance(v, str) else "")
def test_moments_bit_identical_to_f32_populations(name, p, solid, phi, theta):
    a = _run(dict(p, storage="f32"), solid, phi, 25, theta)
    b = _run(dict(p, storage="moments"), solid, phi, 25, theta)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_moments_match_oracle_from_a_moving_start():
    """Initial velocity field (random, 0.02) at rest elsewhere: the moment
    form's equilibrium coefficients and its first step and tenth step
    against the FP64 oracle."""
    nx, ny, nz = 26, 22, 18
    p = I.base_params(nx, ny, nz, sigma=0.01, rho_g=0.1, nu_g=0.1, theta_deg=70.0,
                      storage="moments")
    solid = I.walls_z(nx, ny, nz)
    phi = I.droplet(nx, ny, nz, (13, 11, 0.5), 7.0, 4.0)
    u = I.fast_uniform((3, nz, ny, nx), seed=9, lo=-0.02, hi=0.02).astype(np.float32)
    u[:, solid == 1] = 0.0
    for steps, tol in ((0, 1e-6), (1, 1e-5), (10, 1e-5)):
        g_phi, g_u, g_p, g_f = _run(p, solid, phi, steps, u=u)
        o = O.Oracle(p)
        o.set_geometry(solid)
        o.set_fields(phi.astype(np.float64), u.astype(np.float64))
        o.step(steps)
        r_phi, r_u, r_p = o.fields()
        fluid = solid == 0
        rf = o.populations()[:, fluid]
        assert np.abs(g_f[:, fluid] - rf).max() / np.abs(rf).max() < tol, steps
        if steps:
            assert np.abs(g_phi - r_phi).max() / np.abs(r_phi).max() < tol
            assert np.abs(g_u - r_u).max() / np.abs(r_u).max() < tol


def test_moments_reject_population_setters_and_batches():
    from paper_2607_25444_b300 import cacl
    p = I.base_params(16, 16, 12, storage="moments")
    s = cacl.Solver(p)
    s.set_geometry(I.walls_z(16, 16, 12))
    s.set_fields(I.droplet(16, 16, 12, (8, 8, 0.5), 5.0, 4.0))
    with pytest.raises(cacl.CaclError):
        s.set_populations(np.zeros((27, 12, 16, 16), np.float32))
    with pytest.raises(cacl.CaclError):
        s.set_option(cacl.OPT_LB_PIPE, 1)
    s.close()
    with pytest.raises(cacl.CaclError):
        cacl.Batch([p, p])
