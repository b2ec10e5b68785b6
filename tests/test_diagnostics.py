"""The package's diagnostics on exact shapes (circle cap, disc, rod)."""
import math

import numpy as np
import pytest

from paper_2607_25444_b300 import diagnostics as D


def _cap(theta, R=30.0, nx=160, ny=8, nz=80):
    z0 = 0.5 - R * math.cos(math.radians(theta))
    z, y, x = np.meshgrid(np.arange(nz, dtype=float), np.arange(ny, dtype=float),
                          np.arange(nx, dtype=float), indexing="ij")
    r = np.sqrt((x - 80) ** 2 + (z - z0) ** 2)
    phi = 0.5 * (1 + np.tanh(2 * (R - r) / 4))
    phi[z < 0.5] = 0.0
    return phi


def test_contact_angle_of_exact_caps():
    for th in (40.0, 90.0, 140.0):
        assert abs(D.contact_angle(_cap(th), 0.5, z_min=1.0) - th) < 0.5


def test_band_fit_of_exact_caps():
    """The band fit (node centres with |phi - 1/2| < eps) recovers the cap's
    angle; it reads a band of nodes around the crossing, so it is checked
    to 1.5 deg."""
    for th in (40.0, 90.0, 140.0):
        for eps in (0.1, 0.2):
            assert abs(D.contact_angle_band(_cap(th), eps, 0.5, z_min=1.0) - th) < 1.5


def test_footprint_of_a_disc():
    n = 101
    y, x = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    disc = ((x - 50) ** 2 + (y - 50) ** 2 <= 30 ** 2).astype(float)
    phi = np.zeros((3, n, n))
    phi[1] = disc
    assert abs(D.footprint_radius(phi) - 30.0) < 0.1


def test_extent_of_a_rod():
    phi = np.zeros((4, 5, 64))
    x = np.arange(64, dtype=float)
    phi[2, 3] = 0.5 * (np.tanh(2 * (x - 10.25) / 4) - np.tanh(2 * (x - 40.75) / 4))
    assert abs(D.max_extent(phi) - 30.5) < 0.05


@pytest.mark.parametrize("theta", [45.0, 90.0, 135.0])
def test_contact_angle_on_disc_synthetic(theta):
    """A tanh drop of radius 30 whose circle meets a wall circle of radius
    40 at a known angle (centres d apart with d^2 = r^2 + R^2 - 2 r R cos
    theta): the disc diagnostic returns that angle."""
    r, R = 30.0, 40.0
    d = math.sqrt(r * r + R * R - 2 * r * R * math.cos(math.radians(theta)))
    n = 200
    yy, xx = np.mgrid[0:n, 0:n].astype(np.float64)
    cw = (100.0, 60.0)
    cd = (100.0, 60.0 + d)
    phi = 0.5 * (1.0 - np.tanh((np.hypot(xx - cd[0], yy - cd[1]) - r) / 2.0))
    got = D.contact_angle_on_disc(phi, cw, R, min_gap=3.5)
    assert abs(got - theta) < 0.05, got
