"""z-slab decomposition on one GPU: the problem split into slabs (one
library context each, two halo planes per side), stepped with halo
exchanges and the gathered partial sums of the volume correction, gives
bit for bit the fields of the undivided step when the slabs' interiors
start on multiples of the phi update's tile depth; otherwise it agrees to
rounding."""
import numpy as np
import pytest

from paper_2607_25444_b300 import inputs as I
from paper_2607_25444_b300 import slab as S

pytestmark = pytest.mark.gpu


def _run(p, solid, phi, theta, parts, steps, aligned=True):
    from paper_2607_25444_b300 import cacl
    whole = cacl.Solver(p)
    whole.set_geometry(solid)
    if theta is not None:
        whole.set_contact_angle(theta)
    whole.set_fields(phi)
    m_ref = whole.mass()["m_ref"]
    whole.step(steps)
    whole.check_finite()
    ref_phi, ref_u, ref_p = whole.fields()
    ref_f = whole.populations()
    whole.close()
    ranges = S.partition(p["nz"], parts, align=32 if aligned else 1)
    slabs = []
    for z0, n in ranges:
        s = S.SlabSolver(p, z0, n)
        s.set_geometry(solid)
        if theta is not None:
            s.set_contact_angle(theta)
        s.set_fields(phi, m_ref=m_ref)
        slabs.append(s)
    S.step_local(slabs, steps)
    got_phi = np.concatenate([s.fields()[0] for s in slabs])
    got_u = np.concatenate([s.fields()[1] for s in slabs], axis=1)
    got_p = np.concatenate([s.fields()[2] for s in slabs])
    got_f = np.concatenate([s.populations() for s in slabs], axis=1)
    for s in slabs:
        s.close()
    return (ref_phi, ref_u, ref_p, ref_f), (got_phi, got_u, got_p, got_f)


@pytest.mark.parametrize("parts", [2, 4])
def test_slabs_bit_identical_on_walls_and_drop(parts):
    """Walls at z = 0 and z = 127, a drop on the bottom wall reaching into
    the second slab, patterned contact angles, density ratio 5, gravity:
    2 and 4 slabs of 64 / 32 planes, 30 steps."""
    nx, ny, nz = 24, 20, 128
    p = I.base_params(nx, ny, nz, sigma=0.01, rho_g=0.2, nu_g=0.1,
                      theta_deg=60.0, gravity=(0.0, 0.0, -1e-5))
    solid = I.walls_z(nx, ny, nz)
    phi = I.droplet(nx, ny, nz, (12, 10, 0.5), 40.0, p["width"])
    theta = (50.0 + 60.0 * I.fast_uniform((nz, ny, nx), seed=3)).astype(np.float32)
    ref, got = _run(p, solid, phi, theta, parts, 30)
    for a, b in zip(ref, got):
        assert np.array_equal(a, b)


def test_slabs_bit_identical_interface_and_plate_across_the_cut():
    """A free drop centred on the cut between two slabs of a fully periodic
    box, and an orifice plate straddling it (wall nodes and ghosts on both
    sides of the cut): 40 steps, bit-identical."""
    nx, ny, nz = 32, 24, 64
    p = I.base_params(nx, ny, nz, sigma=0.01, rho_g=0.3, nu_g=0.08,
                      theta_deg=70.0, periodic=(1, 1, 1))
    solid = np.zeros((nz, ny, nx), np.uint8)
    solid[30:34] = 1
    solid[30:34, 8:16, 12:20] = 0   # square hole through the plate
    phi = I.droplet(nx, ny, nz, (16, 12, 32.0), 9.0, p["width"])
    phi[solid == 1] = 0.0
    ref, got = _run(p, solid, phi, None, 2, 40)
    for a, b in zip(ref, got):
        assert np.array_equal(a, b)


def test_unaligned_slabs_agree_to_rounding():
    """Slabs of 21, 21 and 22 planes (interiors not on tile boundaries):
    the correction's partial sums are grouped differently, so lambda and
    the fields agree to rounding instead of bit for bit."""
    nx, ny, nz = 24, 16, 64
    p = I.base_params(nx, ny, nz, sigma=0.01, rho_g=0.5, theta_deg=80.0)
    solid = I.walls_z(nx, ny, nz)
    phi = I.droplet(nx, ny, nz, (12, 8, 0.5), 14.0, p["width"])
    ref, got = _run(p, solid, phi, None, 3, 20, aligned=False)
    assert np.abs(ref[0] - got[0]).max() < 1e-5
    assert np.abs(ref[1] - got[1]).max() < 1e-6


def test_slabs_bit_identical_odd_nx():
    """nx = 23 (the phi update staged element by element, one node per
    thread in the collide-stream) and ny = 18: 2 slabs of 32 planes, walls,
    a drop on the bottom wall reaching the cut, 25 steps, bit-identical."""
    nx, ny, nz = 23, 18, 64
    p = I.base_params(nx, ny, nz, sigma=0.01, rho_g=0.25, nu_g=0.1,
                      theta_deg=75.0, gravity=(0.0, 0.0, -1e-5))
    solid = I.walls_z(nx, ny, nz)
    phi = I.droplet(nx, ny, nz, (11.5, 9.0, 0.5), 30.0, p["width"])
    ref, got = _run(p, solid, phi, None, 2, 25)
    for a, b in zip(ref, got):
        assert np.array_equal(a, b)
