"""The package's diagnostics on exact shapes (circle cap, disc, rod)."""
import math

import numpy as np

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
