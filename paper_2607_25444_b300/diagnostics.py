"""Diagnostics of phase fields from the CUDA path (numpy, host side).

Contact angle by an algebraic circle fit of the phi = 1/2 crossings on a
vertical slice (Sect. 3.1, Eqs. circle_fit_error, measured_contact_angle),
footprint radius on the first fluid layer, largest horizontal extent of the
liquid (for the maximum spreading factor of impacts), and the liquid centre
of mass. Arrays have shape (nz, ny, nx).
"""
import math

import numpy as np


def _crossings(slice2d, level=0.5):
    """phi = level crossings of slice2d[z, x] along both grid directions,
    linearly interpolated; returns (x, z) arrays."""
    v = np.asarray(slice2d, dtype=np.float64) - level
    xs, zs = [], []
    a, b = v[:, :-1], v[:, 1:]
    iz, ix = np.nonzero(a * b < 0)
    t = a[iz, ix] / (a[iz, ix] - b[iz, ix])
    xs.append(ix + t)
    zs.append(iz.astype(np.float64))
    a, b = v[:-1, :], v[1:, :]
    iz, ix = np.nonzero(a * b < 0)
    t = a[iz, ix] / (a[iz, ix] - b[iz, ix])
    xs.append(ix.astype(np.float64))
    zs.append(iz + t)
    return np.concatenate(xs), np.concatenate(zs)


def fit_circle(x, z):
    """Algebraic least-squares circle through the points (Eq.
    circle_fit_error): returns (x0, z0, R)."""
    x = np.asarray(x, np.float64)
    z = np.asarray(z, np.float64)
    A = np.stack([2 * x, 2 * z, np.ones_like(x)], axis=1)
    x0, z0, c = np.linalg.lstsq(A, x * x + z * z, rcond=None)[0]
    return x0, z0, math.sqrt(c + x0 * x0 + z0 * z0)


def contact_angle_on_disc(phi2d, centre, radius, min_gap=3.5):
    """Angle (degrees, through the liquid) between a drop and a circular
    wall in a 2D field phi2d[y, x]: the circle fitted to the phi = 1/2
    crossings farther than radius + min_gap from the wall's centre has
    centre C and radius r; with d = |C - centre| and R = radius, the angle
    between the outward normals of the drop and of the wall at their
    intersection gives cos(theta) = (r^2 + R^2 - d^2) / (2 r R)."""
    x, y = _crossings(phi2d)
    keep = np.hypot(x - centre[0], y - centre[1]) > radius + min_gap
    x0, y0, r = fit_circle(x[keep], y[keep])
    d2 = (x0 - centre[0]) ** 2 + (y0 - centre[1]) ** 2
    c = (r * r + radius * radius - d2) / (2.0 * r * radius)
    return math.degrees(math.acos(min(1.0, max(-1.0, c))))


def contact_angle(phi, z_wall=0.5, y=None, z_min=None):
    """Angle (degrees) through the liquid of the circle fitted to the
    phi = 1/2 crossings of the slice y (default ny/2)."""
    nz, ny, nx = phi.shape
    sl = phi[:, ny // 2 if y is None else y, :]
    x, z = _crossings(sl)
    if z_min is not None:
        keep = z >= z_min
        x, z = x[keep], z[keep]
    A = np.stack([2 * x, 2 * z, np.ones_like(x)], axis=1)
    sol = np.linalg.lstsq(A, x * x + z * z, rcond=None)[0]
    x0, z0, c = sol
    R = math.sqrt(c + x0 * x0 + z0 * z0)
    arg = min(1.0, max(-1.0, (z0 - z_wall) / R))
    return math.degrees(math.pi - math.acos(arg))


def contact_angle_band(phi, eps_fit=0.1, z_wall=0.5, y=None, z_min=None):
    """The same angle from the circle fitted to the node centres of the
    slice y with |phi - 1/2| < eps_fit (the band fit of Eq.
    measured_contact_angle) instead of the interpolated crossings."""
    nz, ny, nx = phi.shape
    sl = np.asarray(phi[:, ny // 2 if y is None else y, :], dtype=np.float64)
    iz, ix = np.nonzero(np.abs(sl - 0.5) < eps_fit)
    x, z = ix.astype(np.float64), iz.astype(np.float64)
    if z_min is not None:
        keep = z >= z_min
        x, z = x[keep], z[keep]
    x0, z0, R = fit_circle(x, z)
    arg = min(1.0, max(-1.0, (z0 - z_wall) / R))
    return math.degrees(math.pi - math.acos(arg))


def footprint_radius(phi, layer=1):
    """r = sqrt(A / pi), A the area of phi > 1/2 on a fluid layer."""
    return math.sqrt(float((phi[layer] > 0.5).sum()) / math.pi)


def max_extent(phi, axis=2):
    """Largest extent of phi > 1/2 along x over all rows (interpolated
    crossings), the spreading diameter D(t)."""
    v = np.moveaxis(np.asarray(phi, np.float64), axis, -1) - 0.5
    v = v.reshape(-1, v.shape[-1])
    best = 0.0
    rows = np.nonzero((v > 0).any(axis=1))[0]
    for r in rows:
        row = v[r]
        idx = np.nonzero(row[:-1] * row[1:] < 0)[0]
        if idx.size < 2:
            continue
        t = row[idx] / (row[idx] - row[idx + 1])
        pos = idx + t
        best = max(best, float(pos.max() - pos.min()))
    return best


def centre_of_mass_z(phi, solid):
    z = np.arange(phi.shape[0])[:, None, None]
    m = np.where(solid == 0, phi, 0.0)
    return float((z * m).sum() / m.sum())
