"""Degenerate cases of the step, through the C ABI, against the FP64 oracle:
a box filled with one phase (no interface band, so the correction weight
W of Sect. 2.3 is zero and lambda is 0 by Eq. mass_correction_normalization's
rule), a box filled with gas (no density difference, so gravity exerts no
force and nothing moves), and a grid that is solid everywhere (no fluid
node, no wall node, zero mass)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2607_25444_b300 import inputs as I

pytestmark = pytest.mark.gpu


def _pair(p, solid, phi, steps):
    from paper_2607_25444_b300 import cacl
    g = cacl.Solver(p)
    g.set_geometry(solid)
    g.set_fields(phi)
    g.step(steps)
    g.check_finite()
    o = O.Oracle(p)
    o.set_geometry(solid)
    o.set_fields(phi.astype(np.float64))
    o.step(steps)
    return g, o


def test_liquid_filled_channel():
    """phi = 1 at every fluid node between two walls with gravity along x:
    the body force (rho_l - rho_g) g drives a channel flow; phi stays in
    [1 - eps, 1] (no band, W = 0, lambda = 0) and the velocity matches the
    oracle's."""
    nx, ny, nz = 16, 12, 14
    p = I.base_params(nx, ny, nz, sigma=0.01, rho_l=1.0, rho_g=0.1, nu_l=0.05,
                      nu_g=0.1, theta_deg=70.0, gravity=(2e-5, 0.0, 0.0))
    solid = I.walls_z(nx, ny, nz)
    phi = np.ones((nz, ny, nx), np.float32)
    g, o = _pair(p, solid, phi, 30)
    fluid = solid == 0
    gp, gu, _ = g.fields()
    op, ou, _ = o.fields()
    m = g.mass()
    assert m["w_sum"] == 0.0 and m["lam"] == 0.0
    assert np.all(gp[fluid] <= 1.0) and np.all(gp[fluid] >= 1.0 - 1e-3)
    assert np.abs(gp[fluid] - op[fluid]).max() < 1e-6
    umax = np.abs(ou[:, fluid]).max()
    assert umax > 1e-5  # the force acts
    assert np.abs(gu[:, fluid] - ou[:, fluid]).max() < 1e-5 * umax
    g.close()


def test_gas_filled_box_stays_at_rest():
    """phi = 0 everywhere: rho = rho_g, so F_ext = (rho - rho_g) g = 0, the
    chemical potential vanishes and the field stays exactly as it was."""
    nx, ny, nz = 12, 10, 12
    p = I.base_params(nx, ny, nz, sigma=0.01, rho_l=1.0, rho_g=0.1, nu_l=0.05,
                      nu_g=0.1, theta_deg=70.0, gravity=(0.0, 0.0, -2e-5))
    solid = I.walls_z(nx, ny, nz)
    phi = np.zeros((nz, ny, nx), np.float32)
    g, o = _pair(p, solid, phi, 20)
    gp, gu, gs = g.fields()
    fluid = solid == 0
    assert np.all(gp[fluid] == 0.0)
    assert np.all(gu[:, fluid] == 0.0)
    assert np.all(o.fields()[0][fluid] == 0.0)
    assert g.mass()["lam"] == 0.0
    g.close()


def test_all_solid_grid():
    """A grid without fluid nodes: no wall node (none has a fluid
    neighbour), M_ref = 0, and steps run and leave phi at the solid nodes as
    it was set."""
    nx, ny, nz = 8, 8, 8
    p = I.base_params(nx, ny, nz, sigma=0.01, theta_deg=70.0)
    solid = np.ones((nz, ny, nx), np.uint8)
    phi = I.fast_uniform((nz, ny, nx), seed=3).astype(np.float32)
    from paper_2607_25444_b300 import cacl
    g = cacl.Solver(p)
    g.set_geometry(solid)
    assert g.wall_list()["idx"].size == 0
    g.set_fields(phi)
    g.step(5)
    g.check_finite()
    m = g.mass()
    assert m["m_ref"] == 0.0 and m["lam"] == 0.0
    assert np.array_equal(g.fields()[0], phi)
    g.close()


@pytest.mark.parametrize("bad", [dict(nx=0), dict(ny=-3), dict(width=0.0), dict(rho_g=0.0),
                                 dict(nu_l=-0.1), dict(eps_phi=0.5), dict(sigma=-1.0),
                                 dict(storage=7)])
def test_invalid_parameters_are_rejected(bad):
    """An empty or negative grid, a non-positive width, density or viscosity,
    a band threshold outside (0, 1/2), a negative surface tension and an
    unknown storage are refused at creation, before any device memory is
    taken."""
    from paper_2607_25444_b300 import cacl
    p = I.base_params(8, 8, 8)
    p.update(bad)
    with pytest.raises(cacl.CaclError):
        cacl.Solver(p)


def test_zero_steps_and_single_node_rows():
    """step(0) changes nothing; a grid one node wide in x and y (every
    neighbour wraps onto the node itself) steps like the oracle."""
    nx, ny, nz = 1, 1, 12
    p = I.base_params(nx, ny, nz, sigma=0.01, rho_l=1.0, rho_g=0.2, nu_l=0.05,
                      nu_g=0.1, theta_deg=70.0, gravity=(0.0, 0.0, -1e-5))
    solid = I.walls_z(nx, ny, nz)
    phi = np.zeros((nz, ny, nx), np.float32)
    phi[1:6] = 1.0
    phi[6] = 0.5
    from paper_2607_25444_b300 import cacl
    g = cacl.Solver(p)
    g.set_geometry(solid)
    g.set_fields(phi)
    before = [x.copy() for x in g.fields()]
    g.step(0)
    for a, b in zip(before, g.fields()):
        assert np.array_equal(a, b)
    g.close()
    g, o = _pair(p, solid, phi, 10)
    fluid = solid == 0
    gp, gu, _ = g.fields()
    op, ou, _ = o.fields()
    assert np.abs(gp[fluid] - op[fluid]).max() < 1e-5
    assert np.abs(gu[:, fluid] - ou[:, fluid]).max() < 1e-5 * max(np.abs(ou).max(), 1e-12) + 1e-9
    g.close()
