"""Post-processing of oracle fields -- TEST INFRASTRUCTURE.

Contact angle by an algebraic circle fit (Sect. 3.1, Eqs. circle_fit_error and
measured_contact_angle), footprint radius, centre of mass. Only tests and the
bench's CPU-baseline leg use this module; the CUDA package has its own.
"""
import numpy as np


def crossings_2d(phi2d, level=0.5):
    """Points where phi crosses ``level`` along grid lines of a 2D slice
    phi2d[z, x], by linear interpolation. Returns arrays (x, z)."""
    pts = []
    nz, nx = phi2d.shape
    for z in range(nz):
        row = phi2d[z]
        for x in range(nx - 1):
            a, b = row[x] - level, row[x + 1] - level
            if a == 0.0:
                pts.append((float(x), float(z)))
            elif a * b < 0.0:
                pts.append((x + a / (a - b), float(z)))
    for x in range(nx):
        col = phi2d[:, x]
        for z in range(nz - 1):
            a, b = col[z] - level, col[z + 1] - level
            if a * b < 0.0:
                pts.append((float(x), z + a / (a - b)))
    if not pts:
        return np.zeros(0), np.zeros(0)
    p = np.array(pts)
    return p[:, 0], p[:, 1]


def circle_fit(x, z):
    """Minimise sum [(x-x0)^2 + (z-z0)^2 - R^2]^2 (Kasa): linear least
    squares in (x0, z0, R^2 - x0^2 - z0^2)."""
    A = np.stack([2 * x, 2 * z, np.ones_like(x)], axis=1)
    b = x * x + z * z
    sol, *_ = np.linalg.lstsq(A, b, rcond=None)
    x0, z0, c = sol
    R = np.sqrt(c + x0 * x0 + z0 * z0)
    return x0, z0, R


def contact_angle(phi2d, z_wall, z_min=None):
    """theta_num = pi - arccos((z0 - z_w)/R), argument clipped to [-1, 1],
    from the phi = 1/2 crossings of a vertical slice phi2d[z, x] (liquid
    phi > 1/2). Points below ``z_min`` are dropped. Degrees."""
    x, z = crossings_2d(phi2d)
    if z_min is not None:
        keep = z >= z_min
        x, z = x[keep], z[keep]
    x0, z0, R = circle_fit(x, z)
    arg = np.clip((z0 - z_wall) / R, -1.0, 1.0)
    return float(np.degrees(np.pi - np.arccos(arg))), (x0, z0, R)


def centre_of_mass_z(phi, solid):
    z = np.arange(phi.shape[0])[:, None, None]
    m = np.where(solid == 0, phi, 0.0)
    return float((z * m).sum() / m.sum())


def footprint_radius(phi, layer=1):
    """r = sqrt(A / pi) with A the count of nodes with phi > 1/2 on a layer."""
    area = 0
    for row in phi[layer]:
        for v in row:
            if v > 0.5:
                area += 1
    return float(np.sqrt(area / np.pi))


def max_extent(phi):
    """Largest x-extent of phi > 1/2 over all (z, y) rows, from linearly
    interpolated crossings."""
    best = 0.0
    nz, ny, nx = phi.shape
    for z in range(nz):
        for y in range(ny):
            row = phi[z, y]
            pos = []
            for x in range(nx - 1):
                a, b = row[x] - 0.5, row[x + 1] - 0.5
                if a * b < 0.0:
                    pos.append(x + a / (a - b))
            if len(pos) >= 2:
                best = max(best, max(pos) - min(pos))
    return best
