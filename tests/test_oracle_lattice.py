"""Pins of the oracle's lattice, equilibrium, collision and stencils against
what the mathematics fixes (Sect. 2.1): lattice isotropy, Hermite moment
closed forms, exactness of the isotropic stencils on polynomials."""
import itertools

import numpy as np
import pytest

from oracle import oracle as O
from paper_2607_25444_b300 import inputs as I

CS2 = 1.0 / 3.0


@pytest.mark.parametrize("dim", [2, 3])
def test_lattice_isotropy(dim):
    c, w = O.lattice(dim)
    Q = 27 if dim == 3 else 9
    assert c.shape == (Q, 3)
    D = dim
    cc = c[:, :D].astype(float)
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.abs(w @ cc).max() < 1e-15
    np.testing.assert_allclose(np.einsum("q,qa,qb->ab", w, cc, cc),
                               CS2 * np.eye(D), atol=1e-15)
    assert np.abs(np.einsum("q,qa,qb,qc->abc", w, cc, cc, cc)).max() < 1e-15
    m4 = np.einsum("q,qa,qb,qc,qd->abcd", w, cc, cc, cc, cc)
    I2 = np.eye(D)
    iso = CS2 ** 2 * (np.einsum("ab,cd->abcd", I2, I2) +
                      np.einsum("ac,bd->abcd", I2, I2) +
                      np.einsum("ad,bc->abcd", I2, I2))
    np.testing.assert_allclose(m4, iso, atol=1e-15)
    # opposite directions exist and the enumeration is (cz, cy, cx) lexicographic
    for q in range(Q):
        assert any((c[p] == -c[q]).all() for p in range(Q))
    order = [tuple(x) for x in c[:, ::-1]]
    assert order == sorted(order)


def test_d3q27_lumps_to_d2q9():
    """Summing D3Q27 weights over c_z gives D2Q9's 4/9, 1/9, 1/36."""
    c3, w3 = O.lattice(3)
    c2, w2 = O.lattice(2)
    for q in range(9):
        m = (c3[:, 0] == c2[q, 0]) & (c3[:, 1] == c2[q, 1])
        assert abs(w3[m].sum() - w2[q]) < 1e-16


def _moments(f, c):
    c = c.astype(float)
    return (f.sum(), f @ c, np.einsum("q,qa,qb->ab", f, c, c),
            np.einsum("q,qa,qb,qc->abc", f, c, c, c))


@pytest.mark.parametrize("dim", [2, 3])
def test_equilibrium_moments(dim):
    """Third-order Hermite equilibrium (Eq. feq3): moments up to second order
    are p*, u, p* c_s^2 I + uu; the lattice-supported third moments are
    c_s^2 (u d + perms) + uuu (xyz, xxy, ...)."""
    g = I.SplitMix64(7)
    c, _ = O.lattice(dim)
    for _ in range(5):
        p = g.uniform(-0.5, 0.5)
        u = np.array([g.uniform(-0.1, 0.1) for _ in range(3)])
        if dim == 2:
            u[2] = 0.0
        f = O.feq(p, u, dim)
        m0, m1, m2, m3 = _moments(f, c)
        assert abs(m0 - p) < 1e-15
        np.testing.assert_allclose(m1, u, atol=1e-15)
        np.testing.assert_allclose(m2, p * CS2 * np.eye(3) * (np.arange(3) < dim)
                                   + np.outer(u, u), atol=1e-15)
        D = dim
        for a, b, cc in itertools.product(range(D), repeat=3):
            if a == b == cc:
                continue  # c_a^3 = c_a on the lattice: not a free moment
            d = np.eye(3)
            exp = CS2 * (u[a] * d[b, cc] + u[b] * d[a, cc] + u[cc] * d[a, b]) \
                + u[a] * u[b] * u[cc]
            assert abs(m3[a, b, cc] - exp) < 1e-15, (a, b, cc)


def _collide_case(seed, dim=3, **kw):
    g = I.SplitMix64(seed)
    params = I.base_params(4, 4, 4 if dim == 3 else 1, dim=dim,
                           periodic=(1, 1, 1), sigma=0.02, rho_l=1.0,
                           rho_g=0.1, nu_l=0.05, nu_g=0.2,
                           gravity=(1e-5, -2e-5, 3e-5), **kw)
    o = O.Oracle(params)
    Q = o.Q
    c, w = O.lattice(dim)
    f_in = O.feq(g.uniform(-0.1, 0.1),
                 [g.uniform(-0.05, 0.05) for _ in range(3)], dim)
    f_in = f_in + w * np.array([g.uniform(-0.02, 0.02) for _ in range(Q)])
    phi = g.uniform(0.1, 0.9)
    grad = np.array([g.uniform(-0.2, 0.2) for _ in range(3)])
    if dim == 2:
        grad[2] = 0.0
    lap = g.uniform(-0.05, 0.05)
    return o, c, f_in, phi, grad, lap


@pytest.mark.parametrize("seed", [1, 2, 3])
@pytest.mark.parametrize("dim", [2, 3])
def test_collision_moment_closed_forms(seed, dim):
    """Regularised collision with Guo forcing (Eqs. feq3, guo, fneq3, A3rec):
    sum f* = p*, sum f* c = u + a/2, sum f* cc = p* cs2 I + uu + (1-omega) A2
    + (u a + a u)/2 with A2 the second moment of f - (f^eq - S/2), and the
    third-order moments carry (1-omega) A3 with A3 = S(u A2)."""
    o, c, f_in, phi, grad, lap = _collide_case(seed, dim)
    f_out, u, a, omega = o.collide_node(f_in, phi, grad, lap)
    cf = c.astype(float)
    p = f_in.sum()
    j = f_in @ cf
    np.testing.assert_allclose(u, j + 0.5 * a, atol=1e-15)
    m0, m1, m2, m3 = _moments(f_out, c)
    assert abs(m0 - p) < 1e-14
    np.testing.assert_allclose(m1, u + 0.5 * a, atol=1e-15)
    D = dim
    mask = np.zeros((3, 3))
    mask[:D, :D] = 1
    Pi_in = np.einsum("q,qa,qb->ab", f_in, cf, cf)
    ua = np.outer(u, a) + np.outer(a, u)
    A2 = (Pi_in - p * CS2 * np.eye(3) * mask - np.outer(u, u) + 0.5 * ua) * mask
    exp2 = p * CS2 * np.eye(3) * mask + np.outer(u, u) + (1 - omega) * A2 + 0.5 * ua
    np.testing.assert_allclose(m2, exp2 * mask, atol=1e-14)
    A3 = (np.einsum("a,bc->abc", u, A2) + np.einsum("b,ac->abc", u, A2)
          + np.einsum("c,ab->abc", u, A2))
    if dim == 3:
        exp_xyz = u[0] * u[1] * u[2] + (1 - omega) * A3[0, 1, 2]
        assert abs(m3[0, 1, 2] - exp_xyz) < 1e-14
    # H3_xxy projection: sum f* (c_x^2 c_y - cs2 c_y) = u_x^2 u_y + (1-omega) A3_xxy
    for (a_, b_) in [(0, 1), (1, 0)] + ([(0, 2), (2, 1)] if dim == 3 else []):
        h3 = cf[:, a_] ** 2 * cf[:, b_] - CS2 * cf[:, b_]
        exp = u[a_] ** 2 * u[b_] + (1 - omega) * A3[a_, a_, b_]
        assert abs(f_out @ h3 - exp) < 1e-14


def test_relaxation_frequency_and_mixture():
    """omega = (1/2 + nu/cs2)^-1 with nu = mu/rho, rho and mu linear in phi
    (Eqs. rho_mix_linear, mu_mix_linear, omega_phi): check at phi = 0, 1."""
    o, c, f_in, _, grad, lap = _collide_case(4)
    for phi, nu in [(0.0, 0.2), (1.0, 0.05)]:
        _, _, _, omega = o.collide_node(f_in, phi, grad * 0, 0.0)
        assert abs(omega - 1.0 / (0.5 + nu / CS2)) < 1e-14
    # half way: mu = (0.1*0.2 + 1*0.05)/2, rho = 0.55
    _, _, _, omega = o.collide_node(f_in, 0.5, grad * 0, 0.0)
    nu = 0.5 * (0.1 * 0.2 + 1.0 * 0.05) / 0.55
    assert abs(omega - 1.0 / (0.5 + nu / CS2)) < 1e-14


def test_force_free_state_is_invariant():
    """phi in a bulk phase with no gradient and no gravity: an equilibrium
    f^eq(p*, u) is a fixed point of the collision (S = 0, f^neq = 0)."""
    params = I.base_params(4, 4, 4, periodic=(1, 1, 1), rho_l=2.0, rho_g=1.0)
    o = O.Oracle(params)
    f = O.feq(0.03, [0.02, -0.01, 0.015])
    f_out, u, a, _ = o.collide_node(f, 1.0, np.zeros(3), 0.0)
    np.testing.assert_allclose(f_out, f, atol=1e-16)
    assert np.abs(a).max() == 0.0


@pytest.mark.parametrize("dim", [2, 3])
def test_isotropic_stencils_exact_on_polynomials(dim):
    """Eq. grad_iso is exact on quadratics, Eq. lap_iso on cubics (interior
    nodes, away from the periodic seam)."""
    n = 9
    nz = n if dim == 3 else 1
    o = O.Oracle(I.base_params(n, n, nz, dim=dim, periodic=(1, 1, 1)))
    z, y, x = np.meshgrid(np.arange(nz, dtype=float), np.arange(n, dtype=float),
                          np.arange(n, dtype=float), indexing="ij")
    g = I.SplitMix64(11)
    k = [g.uniform(-1, 1) for _ in range(20)]
    quad = (k[0] + k[1] * x + k[2] * y + k[3] * x * x + k[4] * x * y +
            k[5] * y * y)
    gq_x = k[1] + 2 * k[3] * x + k[4] * y
    gq_y = k[2] + k[4] * x + 2 * k[5] * y
    cub = quad + k[6] * x ** 3 + k[7] * x * x * y + k[8] * y ** 3
    lc = 2 * k[3] + 2 * k[5] + 6 * k[6] * x + 2 * k[7] * y + 6 * k[8] * y
    if dim == 3:
        quad = quad + k[9] * z + k[10] * z * z + k[11] * x * z
        gq_x = gq_x + k[11] * z
        gq_z = k[9] + 2 * k[10] * z + k[11] * x
        cub = cub + k[9] * z + k[10] * z * z + k[11] * x * z + k[12] * z ** 3 \
            + k[13] * x * y * z
        lc = lc + 2 * k[10] + 6 * k[12] * z
    grad, _ = o.grad_lap(quad)
    _, lap = o.grad_lap(cub)
    sl = (slice(1, -1) if dim == 3 else slice(None), slice(1, -1), slice(1, -1))
    np.testing.assert_allclose(grad[0][sl], gq_x[sl], atol=1e-12)
    np.testing.assert_allclose(grad[1][sl], gq_y[sl], atol=1e-12)
    if dim == 3:
        np.testing.assert_allclose(grad[2][sl], gq_z[sl], atol=1e-12)
    np.testing.assert_allclose(lap[sl], lc[sl], atol=1e-11)
