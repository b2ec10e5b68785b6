"""Parity of the sm_103a CUDA path (through the C ABI) with the FP64 CPU
oracle on identical seeded inputs.

Bars: bit-exact flags-derived wall lists (node, donor, integer normal, FP32
unit normal); FP32 fields within max relative error 1e-5 of the oracle after
one step (norm-wise per field: max |gpu - ref| / max |ref|) and within 1e-3
in phi after 1000 steps.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2607_25444_b300 import inputs as I

pytestmark = pytest.mark.gpu

TOL_1STEP = 1e-5


def _solver(params):
    from paper_2607_25444_b300 import cacl
    return cacl.Solver(params)


def _pair(params, solid, phi, u=None, theta=None):
    g = _solver(params)
    g.set_geometry(solid)
    if theta is not None:
        g.set_contact_angle(theta)
    g.set_fields(phi, u)
    o = O.Oracle(params)
    o.set_geometry(solid)
    if theta is not None:
        o.set_contact_angle(theta.astype(np.float64))
    o.set_fields(phi.astype(np.float64),
                 None if u is None else u.astype(np.float64))
    return g, o


def _rel(a, b):
    den = np.abs(b).max()
    return float(np.abs(a - b).max() / (den if den > 0 else 1.0))


def _geometries():
    yield "walls", I.walls_z(20, 18, 16), (1, 1, 0)
    yield "orifice", I.orifice_plate(24, 24, 40, 16, 4, 8), (1, 1, 0)
    n = 14
    rnd = (I.fast_uniform((n, n, n), seed=21) < 0.4).astype(np.uint8)
    yield "random", rnd, (1, 1, 1)
    yield "sphere", I.sphere_solid(21, 21, 21, (10, 10, 10), 6.0), (1, 1, 1)
    yield "cylinder", I.cylinder_solid(29, 29, 6, (14.0, 14.0), 9.5), (1, 1, 1)
    yield "rough", I.rough_wall_z(24, 20, 14, 3, seed=5), (1, 1, 0)
    lone = np.ones((5, 5, 5), np.uint8)
    lone[2, 2, 2] = 0
    yield "lone", lone, (1, 1, 1)


@pytest.mark.parametrize("name,solid,periodic",
                         list(_geometries()), ids=lambda v: v if isinstance(v, str) else "")
def test_wall_list_bit_exact(name, solid, periodic):
    nz, ny, nx = solid.shape
    p = I.base_params(nx, ny, nz, periodic=periodic)
    g = _solver(p)
    g.set_geometry(solid)
    o = O.Oracle(p)
    o.set_geometry(solid)
    gw, ow = g.wall_list(), o.wall_list()
    assert np.array_equal(gw["idx"], ow["idx"])
    assert np.array_equal(gw["qstar"], ow["qstar"])
    assert np.array_equal(gw["ntilde6"], ow["ntilde6"])
    assert np.array_equal(gw["nw_f32"].view(np.uint32), ow["nw_f32"].view(np.uint32))


def test_geometry_rejects_open_axis():
    from paper_2607_25444_b300 import cacl
    p = I.base_params(8, 8, 8, periodic=(1, 1, 0))
    g = _solver(p)
    with pytest.raises(cacl.CaclError):
        g.set_geometry(np.zeros((8, 8, 8), np.uint8))


def _droplet_case(nx=26, ny=22, nz=18, theta=60.0, **kw):
    p = I.base_params(nx, ny, nz, sigma=0.01, rho_l=1.0, rho_g=0.1, nu_l=0.05,
                      nu_g=0.1, theta_deg=theta, gravity=(0.0, 0.0, -2e-6), **kw)
    solid = I.walls_z(nx, ny, nz)
    phi = I.droplet(nx, ny, nz, (nx / 2, ny / 2, 0.5), 7.0, p["width"])
    return p, solid, phi


@pytest.mark.parametrize("variant,pipe,shape", [(2, 3, (64, 40, 70)), (0, 1, (37, 35, 20)),
                                                (3, 2, (96, 24, 40)), (1, 3, (48, 17, 33))])
def test_tile_skipping_correction(variant, pipe, shape):
    """The step's correction (Sect. 2.3, Eq. mass_corrected_phi) visits only
    the phi-update tiles whose chi sum is positive: a small drop in a larger
    box leaves most tiles without interface-band nodes. Stepping through the
    graph gives bit for bit the fields of the same steps composed of the
    parts, whose correction visits every node, for every tile shape, both
    staging pipelines, nx a multiple of 4 or odd, and ragged tiles in y and
    z."""
    from paper_2607_25444_b300 import cacl
    nx, ny, nz = shape
    p = I.base_params(nx, ny, nz, sigma=0.01, rho_l=1.0, rho_g=0.1, nu_l=0.05,
                      nu_g=0.1, theta_deg=65.0, gravity=(0.0, 0.0, -2e-6))
    solid = I.walls_z(nx, ny, nz)
    phi = I.droplet(nx, ny, nz, (nx / 3, ny / 2, 0.5), 6.0, p["width"])
    runs = []
    for parts in (False, True):
        g = _solver(p)
        g.set_option(cacl.OPT_PHASE_TILE, variant)
        if nx % 4 == 0:
            g.set_option(cacl.OPT_PHASE_PIPE, pipe)
        g.set_geometry(solid)
        g.set_fields(phi)
        for _ in range(6):
            if parts:
                g.ghost_update()
                g.lb_collide()
                g.phase_update()
                g.volume_correct()
            else:
                g.step(1)
        runs.append((g.fields(), g.mass()))
    (fa, ma), (fb, mb) = runs
    for a, b in zip(fa, fb):
        assert np.array_equal(a, b)
    assert ma["lam"] == mb["lam"] and ma["lam"] != 0.0


def test_ghost_update_part():
    p, solid, phi = _droplet_case(theta=50.0)
    g, o = _pair(p, solid, phi)
    g.ghost_update()
    o.ghost_update()
    assert _rel(g.fields()[0], o.fields()[0]) < TOL_1STEP


def test_lb_collide_part_random_populations():
    p, solid, phi = _droplet_case()
    g, o = _pair(p, solid, phi)
    f = (I.random_state((p["nz"], p["ny"], p["nx"]), 27, seed=5, amp=2e-3))
    g.set_populations(f)
    o.set_populations(f.astype(np.float64))
    g.lb_collide()
    o.lb_collide()
    gf, of = g.populations(), o.populations()
    fluid = solid == 0
    assert _rel(gf[:, fluid], of[:, fluid]) < TOL_1STEP
    assert _rel(g.fields()[1], o.fields()[1]) < TOL_1STEP
    assert _rel(g.fields()[2], o.fields()[2]) < TOL_1STEP


def test_phase_update_part_random_velocity():
    p, solid, phi = _droplet_case()
    g, o = _pair(p, solid, phi)
    u = I.fast_uniform((3, p["nz"], p["ny"], p["nx"]), seed=8, lo=-0.05,
                       hi=0.05).astype(np.float32)
    u[:, solid == 1] = 0.0
    g.set_velocity(u)
    o.set_velocity(u.astype(np.float64))
    g.phase_update()
    o.phase_update()
    assert _rel(g.fields()[0], o.fields()[0]) < TOL_1STEP
    g.volume_correct()
    o.volume_correct()
    gm, om = g.mass(), o.mass()
    assert abs(gm["m_star"] - om["m_star"]) < 1e-5 * om["m_star"]
    assert abs(gm["w_sum"] - om["w_sum"]) < 1e-5 * om["w_sum"]
    assert _rel(g.fields()[0], o.fields()[0]) < TOL_1STEP


@pytest.mark.parametrize("theta", [30.0, 90.0, 150.0])
def test_one_step_full(theta):
    p, solid, phi = _droplet_case(theta=theta)
    u = np.zeros((3,) + phi.shape, np.float32)
    u[0] = 0.01 * (phi > 0.5)
    g, o = _pair(p, solid, phi, u)
    g.step(1)
    o.step(1)
    gphi, gu, gp = g.fields()
    ophi, ou, op = o.fields()
    assert _rel(gphi, ophi) < TOL_1STEP
    assert _rel(gu, ou) < TOL_1STEP
    assert _rel(gp, op) < TOL_1STEP
    fluid = solid == 0
    assert _rel(g.populations()[:, fluid], o.populations()[:, fluid]) < TOL_1STEP


def test_ragged_sizes_and_patterned_angles():
    """Sizes that are not multiples of any tile, all three axes wrapping in
    x and y, per-node contact angles."""
    nx, ny, nz = 37, 13, 11
    p = I.base_params(nx, ny, nz, sigma=0.02, theta_deg=70.0, rho_g=0.5)
    solid = I.walls_z(nx, ny, nz)
    solid[1:4, 5:8, 10:20] = 1  # a block on the floor
    phi = I.droplet(nx, ny, nz, (18, 6, 3), 5.0, 4.0)
    theta = (45.0 + 90.0 * I.fast_uniform((nz, ny, nx), seed=4)).astype(np.float32)
    g, o = _pair(p, solid, phi, theta=theta)
    g.step(3)
    o.step(3)
    gphi, gu, gp = g.fields()
    ophi, ou, op = o.fields()
    assert _rel(gphi, ophi) < 3 * TOL_1STEP
    assert _rel(gu, ou) < 3 * TOL_1STEP


@pytest.mark.parametrize("kind", ["cylinder", "rough", "sphere"])
def test_curved_and_rough_walls_steps(kind):
    """A drop in contact with a cylinder (periodic box), a rough floor
    (seeded column heights 0..3) or a ball, with patterned contact angles:
    ghosts on staircase walls with quantised normals, bounce-back on
    irregular links; three full steps against the oracle."""
    if kind == "cylinder":
        nx, ny, nz = 32, 30, 12
        solid = I.cylinder_solid(nx, ny, nz, (15.5, 14.5), 7.0)
        phi = I.droplet(nx, ny, nz, (24.0, 14.5, 6.0), 6.0, 4.0)
        periodic = (1, 1, 1)
    elif kind == "rough":
        nx, ny, nz = 30, 26, 16
        solid = I.rough_wall_z(nx, ny, nz, 3, seed=9)
        phi = I.droplet(nx, ny, nz, (15.0, 13.0, 3.0), 7.0, 4.0)
        periodic = (1, 1, 0)
    else:
        nx, ny, nz = 28, 28, 28
        solid = I.sphere_solid(nx, ny, nz, (13.5, 13.5, 10.0), 6.5)
        phi = I.droplet(nx, ny, nz, (13.5, 13.5, 19.0), 6.0, 4.0)
        periodic = (1, 1, 1)
    p = I.base_params(nx, ny, nz, sigma=0.01, rho_g=0.2, periodic=periodic)
    theta = (40.0 + 100.0 * I.fast_uniform((nz, ny, nx), seed=13)).astype(np.float32)
    g, o = _pair(p, solid, phi, theta=theta)
    g.step(3)
    o.step(3)
    gphi, gu, gp = g.fields()
    ophi, ou, op = o.fields()
    assert _rel(gphi, ophi) < 3 * TOL_1STEP
    assert _rel(gu, ou) < 3 * TOL_1STEP
    assert _rel(gp, op) < 3 * TOL_1STEP


def test_no_walls_fully_periodic():
    """No solid node at all. Where grad phi vanishes inside the diffuse
    region (the droplet centre, the saddles between the droplet and its
    periodic images) the unit normal of the compressive term is rounding
    noise, so parity is only defined where phi (1 - phi) is negligible at
    those points: R = 12 (phi(1 - phi) ~ 6e-6 at the centre) in a box of 48
    (the same at the saddles)."""
    n = 48
    p = I.base_params(n, n, n, periodic=(1, 1, 1), sigma=0.01)
    solid = np.zeros((n, n, n), np.uint8)
    phi = I.droplet(n, n, n, (24, 24, 24), 12.0, 4.0)
    g, o = _pair(p, solid, phi)
    assert g.wall_list()["idx"].size == 0
    g.step(1)
    o.step(1)
    assert _rel(g.fields()[0], o.fields()[0]) < TOL_1STEP
    g.step(4)
    o.step(4)
    assert _rel(g.fields()[0], o.fields()[0]) < 2e-5
    assert _rel(g.fields()[1], o.fields()[1]) < 1e-4


def test_two_dimensional_slab_config():
    """The 2D static droplet (128 x 64, periodic in x, walls at y = 0 and
    y = 63) as a D3Q27 slab one node thick, against the oracle's D3Q27 slab
    and its D2Q9 run."""
    p2, solid, phi = I.static_droplet_2d(60.0)
    p3 = dict(p2, dim=3)
    g, o3 = _pair(p3, solid, phi)
    o2 = O.Oracle(p2)
    o2.set_geometry(solid)
    o2.set_fields(phi.astype(np.float64))
    g.step(200)
    o3.step(200)
    o2.step(200)
    assert _rel(g.fields()[0], o3.fields()[0]) < 1e-4
    assert _rel(g.fields()[0], o2.fields()[0]) < 1e-4


def test_thousand_steps_phi():
    nx, ny, nz = 24, 24, 20
    p = I.base_params(nx, ny, nz, sigma=0.01, rho_l=1.0, rho_g=0.1, nu_l=0.05,
                      nu_g=0.1, theta_deg=60.0)
    solid = I.walls_z(nx, ny, nz)
    phi = I.droplet(nx, ny, nz, (12, 12, 0.5), 7.0, 4.0)
    g, o = _pair(p, solid, phi)
    g.step(1000)
    o.step(1000)
    gphi, ophi = g.fields()[0], o.fields()[0]
    assert _rel(gphi, ophi) < 1e-3
    m0 = o.mass()["m_ref"]
    assert abs(g.mass()["m_ref"] - m0) < 1e-9 * m0


def test_mass_held_and_deterministic():
    p, solid, phi = _droplet_case(nx=40, ny=36, nz=30, theta=40.0)
    runs = []
    for _ in range(2):
        g = _solver(p)
        g.set_geometry(solid)
        g.set_fields(phi)
        g.step(50)
        runs.append((g.fields()[0], g.mass()))
    assert np.array_equal(runs[0][0], runs[1][0])
    fphi = runs[0][0].astype(np.float64)
    m = fphi[solid == 0].sum()
    m_ref = runs[0][1]["m_ref"]
    assert abs(m - m_ref) < 1e-8 * m_ref


def test_state_errors():
    from paper_2607_25444_b300 import cacl
    p, solid, phi = _droplet_case()
    g = _solver(p)
    with pytest.raises(cacl.CaclError):
        g.step(1)
    with pytest.raises(cacl.CaclError):
        g.set_fields(phi)
    g.set_geometry(solid)
    g.set_fields(phi)
    with pytest.raises(cacl.CaclError):
        g.step(-1)
    bad = phi.copy()
    bad[5, 5, 5] = np.nan
    g.set_phi(bad)
    with pytest.raises(cacl.CaclError):
        g.check_finite()


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
def test_phase_tile_variants(variant):
    """Every tile shape of the phase update gives the oracle's phi* on a
    case that spans several tiles in x, y and z with ragged edges."""
    from paper_2607_25444_b300 import cacl
    p, solid, phi = _droplet_case(nx=70, ny=37, nz=45, theta=50.0)
    g, o = _pair(p, solid, phi)
    g.set_option(cacl.OPT_PHASE_TILE, variant)
    u = I.fast_uniform((3, p["nz"], p["ny"], p["nx"]), seed=9, lo=-0.05,
                       hi=0.05).astype(np.float32)
    u[:, solid == 1] = 0.0
    g.set_velocity(u)
    o.set_velocity(u.astype(np.float64))
    for _ in range(2):
        g.ghost_update()
        o.ghost_update()
        g.phase_update()
        o.phase_update()
        g.volume_correct()
        o.volume_correct()
    assert _rel(g.fields()[0], o.fields()[0]) < TOL_1STEP
    assert abs(g.mass()["m_star"] - o.mass()["m_star"]) < 1e-6 * o.mass()["m_star"]


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
@pytest.mark.parametrize("shape", [(68, 37, 45), (12, 20, 9), (37, 21, 19), (70, 9, 34),
                                   (5, 12, 6)])
def test_phase_copy_pipeline(variant, shape):
    """The phase update staged by asynchronous copies (16-byte copies when nx
    is a multiple of 4; 4-byte copies element by element with the flag bytes
    staged through registers when nx is odd or 2 mod 4) gives bit for bit
    the phi* and partial sums of the register-staged update, and the
    oracle's phi*, on ragged tiles and on grids narrower than the staged
    window (x wraps several times inside it)."""
    from paper_2607_25444_b300 import cacl
    nx, ny, nz = shape
    p, solid, phi = _droplet_case(nx=nx, ny=ny, nz=nz, theta=50.0)
    u = I.fast_uniform((3, nz, ny, nx), seed=9, lo=-0.05, hi=0.05).astype(np.float32)
    u[:, solid == 1] = 0.0
    runs = []
    for pipe in (1, 2):
        g = _solver(p)
        g.set_geometry(solid)
        g.set_fields(phi)
        g.set_option(cacl.OPT_PHASE_TILE, variant)
        g.set_option(cacl.OPT_PHASE_PIPE, pipe)
        g.set_velocity(u)
        for _ in range(2):
            g.ghost_update()
            g.phase_update()
            g.volume_correct()
        runs.append((g.fields()[0], g.mass()))
    assert np.array_equal(runs[0][0], runs[1][0])
    assert runs[0][1]["m_star"] == runs[1][1]["m_star"]
    assert runs[0][1]["w_sum"] == runs[1][1]["w_sum"]
    o = O.Oracle(p)
    o.set_geometry(solid)
    o.set_fields(phi.astype(np.float64))
    o.set_velocity(u.astype(np.float64))
    for _ in range(2):
        o.ghost_update()
        o.phase_update()
        o.volume_correct()
    assert _rel(runs[1][0], o.fields()[0]) < TOL_1STEP


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
@pytest.mark.parametrize("shape", [(68, 37, 45), (12, 20, 9), (36, 5, 33)])
def test_phase_quad_pipeline(variant, shape):
    """The 2 x 2 phase update (copy-staged, an x pair on two rows per
    thread, packed pair arithmetic) gives bit for bit the phi* of the
    two-node copy-staged update at every node, including solid, wall and
    ragged-edge nodes and a grid narrower than the staged window; its
    partial sums agree to the rounding of their summation order; and two
    steps with the correction match the oracle."""
    from paper_2607_25444_b300 import cacl
    nx, ny, nz = shape
    p, solid, phi = _droplet_case(nx=nx, ny=ny, nz=nz, theta=50.0)
    u = I.fast_uniform((3, nz, ny, nx), seed=11, lo=-0.05, hi=0.05).astype(np.float32)
    u[:, solid == 1] = 0.0
    runs = []
    for pipe in (2, 3):
        g = _solver(p)
        g.set_geometry(solid)
        g.set_fields(phi)
        g.set_option(cacl.OPT_PHASE_TILE, variant)
        g.set_option(cacl.OPT_PHASE_PIPE, pipe)
        g.set_velocity(u)
        g.ghost_update()
        g.phase_update()
        star = g.fields()[0]
        m = g.mass()
        g.volume_correct()
        for _ in range(1):
            g.ghost_update()
            g.phase_update()
            g.volume_correct()
        runs.append((star, m, g.fields()[0]))
        g.close()
    assert np.array_equal(runs[0][0].view(np.uint32), runs[1][0].view(np.uint32))
    for key in ("m_star", "w_sum"):
        assert abs(runs[0][1][key] - runs[1][1][key]) <= 1e-12 * abs(runs[0][1][key])
    o = O.Oracle(p)
    o.set_geometry(solid)
    o.set_fields(phi.astype(np.float64))
    o.set_velocity(u.astype(np.float64))
    for _ in range(2):
        o.ghost_update()
        o.phase_update()
        o.volume_correct()
    assert _rel(runs[1][2], o.fields()[0]) < TOL_1STEP


def test_phase_copy_pipeline_rejects_unaligned_nx():
    """The 2 x 2 update needs nx % 4 == 0; the two-node copy-staged update
    takes any nx but needs nz >= 2 (planes are wrapped once)."""
    from paper_2607_25444_b300 import cacl
    p, solid, phi = _droplet_case(nx=70, ny=37, nz=45, theta=50.0)
    g = _solver(p)
    with pytest.raises(cacl.CaclError):
        g.set_option(cacl.OPT_PHASE_PIPE, 3)
    g.set_option(cacl.OPT_PHASE_PIPE, 2)
    g.set_option(cacl.OPT_PHASE_PIPE, 0)
    q = I.base_params(12, 10, 1, periodic=(1, 1, 1))
    h = _solver(q)
    for pipe in (2, 3):
        with pytest.raises(cacl.CaclError):
            h.set_option(cacl.OPT_PHASE_PIPE, pipe)
    h.set_option(cacl.OPT_PHASE_PIPE, 1)


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("shape", [(144, 10, 9), (16, 12, 10)])
def test_lb_staged_pipeline(storage, shape):
    """The collide-stream reading its pulled rows from bulk asynchronous
    copies gives bit for bit the populations, u and phi of direct loads over
    20 full steps: a partial last row segment (nx = 144 = 128 + 16) and a
    row narrower than the 16-byte pads' reach (both pads wrap)."""
    from paper_2607_25444_b300 import cacl
    nx, ny, nz = shape
    p, solid, phi = _droplet_case(nx=nx, ny=ny, nz=nz, theta=70.0)
    p = dict(p, storage=storage)
    u = I.fast_uniform((3, nz, ny, nx), seed=5, lo=-0.02, hi=0.02).astype(np.float32)
    u[:, solid == 1] = 0.0
    runs = []
    for pipe in (0, 1):
        g = _solver(p)
        g.set_option(cacl.OPT_LB_PIPE, pipe)
        g.set_geometry(solid)
        g.set_fields(phi, u)
        g.step(20)
        g.check_finite()
        ph, uu, _ = g.fields()
        runs.append((ph, uu, g.populations()))
    for a, b in zip(runs[0], runs[1]):
        assert np.array_equal(a, b)


def _lb_pipes_agree(p, solid, phi, u, pipes, steps=20):
    from paper_2607_25444_b300 import cacl
    runs = []
    for pipe in pipes:
        g = _solver(p)
        g.set_option(cacl.OPT_LB_PIPE, pipe)
        g.set_geometry(solid)
        g.set_fields(phi, u)
        g.step(steps)
        g.check_finite()
        ph, uu, ps = g.fields()
        runs.append((ph, uu, ps, g.populations()))
    for other in runs[1:]:
        for a, b in zip(runs[0], other):
            assert np.array_equal(a, b)


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("shape", [(64, 10, 9), (130, 6, 8), (2, 5, 6), (36, 12, 10),
                                   (136, 6, 8), (16, 12, 10), (256, 4, 5), (68, 7, 5)])
def test_lb_kernels_bit_identical(storage, shape):
    """Two nodes per thread with packed pair arithmetic (the default), one
    node per thread, and the TMA-tiled form (where nx is a multiple of 8)
    give bit for bit the same populations, u, p* and phi over 20 full steps: one tile row narrower than a tile (nx = 64, 16), two tiles with
    both x edges (256), a partial last tile (136), a partial last block with
    the x wrap inside it for the pair kernel (nx = 130), a row that is a
    single pair (both neighbours wrap onto the row itself), a small box and
    an odd number of rows (a partial last block in y for the four-node
    kernel)."""
    nx, ny, nz = shape
    p, solid, phi = _droplet_case(nx=nx, ny=ny, nz=nz, theta=70.0)
    p = dict(p, storage=storage, rho_g=0.3, nu_g=0.08)
    u = I.fast_uniform((3, nz, ny, nx), seed=5, lo=-0.02, hi=0.02).astype(np.float32)
    u[:, solid == 1] = 0.0
    _lb_pipes_agree(p, solid, phi, u, (0, 2, 3))


@pytest.mark.parametrize("storage", ["f32", "f16"])
@pytest.mark.parametrize("kind", ["orifice", "rough", "periodic"])
def test_lb_kernels_mixed_pairs(storage, kind):
    """Pairs next to walls (bounce-back links) take the one-node path inside
    the same tiles and warps as interior pairs: orifice plate and rough
    floor; and a fully periodic box (every row wraps in y and z), all bit
    for bit equal to one node per thread."""
    if kind == "orifice":
        nx, ny, nz = 24, 24, 40
        solid = I.orifice_plate(nx, ny, nz, 16, 4, 8)
        c = (12.0, 12.0, 30.0)
        per = (1, 1, 0)
    elif kind == "rough":
        nx, ny, nz = 24, 20, 14
        solid = I.rough_wall_z(nx, ny, nz, 3, seed=5)
        c = (12.0, 10.0, 4.0)
        per = (1, 1, 0)
    else:
        nx, ny, nz = 32, 12, 10
        solid = np.zeros((nz, ny, nx), np.uint8)
        c = (16.0, 6.0, 5.0)
        per = (1, 1, 1)
    p = I.base_params(nx, ny, nz, sigma=0.01, rho_g=0.2, nu_g=0.1,
                      theta_deg=60.0, gravity=(0.0, 0.0, -2e-5), periodic=per,
                      storage=storage)
    phi = I.droplet(nx, ny, nz, c, 6.0, p["width"])
    phi[solid == 1] = 0.0
    _lb_pipes_agree(p, solid, phi, None, (0, 2, 3))


def _quantize(f, storage):
    """Round f_i / w_i to the 16-bit storage (nearest even) and scale back."""
    import torch
    c, w = O.lattice(3)
    wv = w.reshape((27,) + (1,) * (f.ndim - 1)).astype(np.float32)
    h = (f / wv).astype(np.float32)
    if storage == "f16":
        hq = h.astype(np.float16).astype(np.float32)
    else:
        hq = torch.from_numpy(h).to(torch.bfloat16).to(torch.float32).numpy()
    return (hq * wv).astype(np.float32)


@pytest.mark.parametrize("storage,tol", [("f16", 6e-4), ("bf16", 4.5e-3)])
def test_reduced_storage_collide_parity(storage, tol):
    """16-bit population storage with FP32 arithmetic: from populations that
    the storage represents exactly, the moments and forces of one collide
    match the oracle to FP32 round-off; the stored f* match to half an ulp
    of the storage format (relative to the largest population)."""
    p, solid, phi = _droplet_case()
    p = dict(p, storage=storage)
    g, o = _pair(p, solid, phi)
    f = _quantize(I.random_state((p["nz"], p["ny"], p["nx"]), 27, seed=5,
                                 amp=2e-3), storage)
    g.set_populations(f)
    o.set_populations(f.astype(np.float64))
    assert np.array_equal(g.populations(), f)
    g.lb_collide()
    o.lb_collide()
    fluid = solid == 0
    assert _rel(g.fields()[1], o.fields()[1]) < TOL_1STEP
    assert _rel(g.populations()[:, fluid], o.populations()[:, fluid]) < tol


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_reduced_storage_full_steps(storage):
    """100 full steps with 16-bit storage stay close to the FP32 GPU run
    and to the oracle in phi, hold mass, and are deterministic."""
    p, solid, phi = _droplet_case(nx=32, ny=32, nz=24, theta=60.0)
    runs = {}
    for st in ("f32", storage, storage):
        g = _solver(dict(p, storage=st))
        g.set_geometry(solid)
        g.set_fields(phi)
        g.step(100)
        runs.setdefault(st, []).append((g.fields()[0], g.mass()))
    o = O.Oracle(p)
    o.set_geometry(solid)
    o.set_fields(phi.astype(np.float64))
    o.step(100)
    ref = o.fields()[0]
    lo, hi = runs[storage]
    assert np.array_equal(lo[0], hi[0])
    bound = 2e-3 if storage == "f16" else 1e-2
    assert _rel(lo[0], ref) < bound
    assert _rel(runs["f32"][0][0], ref) < 1e-4
    m = lo[0].astype(np.float64)[solid == 0].sum()
    assert abs(m - lo[1]["m_ref"]) < 1e-8 * lo[1]["m_ref"]
