"""Seeded synthetic inputs for the CAC-LB wetting step.

This module builds geometries, initial phase fields and parameter sets shaped
like the paper's workloads (static droplet, spreading, impact, orifice
passage). It holds none of the method's arithmetic: it only draws numbers and
lays out arrays, so that the CUDA library and the CPU oracle can be fed
identical inputs. It imports nothing else from this package.

Random numbers come from splitmix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), written out here so that any
language can reproduce the same stream.

Array layout: node n = x + nx*(y + ny*z); arrays have shape (nz, ny, nx).
"""
import math

import numpy as np

SEED = 25444
MASK64 = (1 << 64) - 1


class SplitMix64:
    """splitmix64: state += golden gamma; output = mix(state)."""

    def __init__(self, seed=SEED):
        self.state = seed & MASK64

    def next_u64(self):
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self, lo=0.0, hi=1.0):
        """Uniform double in [lo, hi) from the top 53 bits."""
        return lo + (hi - lo) * ((self.next_u64() >> 11) * (1.0 / (1 << 53)))

    def array(self, n, lo=0.0, hi=1.0):
        return np.array([self.uniform(lo, hi) for _ in range(n)])


def fast_uniform(shape, seed=SEED, lo=0.0, hi=1.0):
    """Vectorised splitmix64 stream (same outputs as SplitMix64.uniform in
    order), for the large random fields of parity tests."""
    n = int(np.prod(shape))
    with np.errstate(over="ignore"):
        k = np.arange(1, n + 1, dtype=np.uint64)
        z = np.uint64(seed) + k * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    v = (z >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))
    return (lo + (hi - lo) * v).reshape(shape)


# ---------------------------------------------------------------- geometry

def walls_z(nx, ny, nz):
    """Solid layers at z=0 and z=nz-1; periodic in x and y."""
    s = np.zeros((nz, ny, nx), dtype=np.uint8)
    s[0] = 1
    s[-1] = 1
    return s


def walls_y(nx, ny, nz=1):
    """Solid layers at y=0 and y=ny-1 (the 2D channel of the 2D droplet)."""
    s = np.zeros((nz, ny, nx), dtype=np.uint8)
    s[:, 0, :] = 1
    s[:, -1, :] = 1
    return s


def orifice_plate(nx, ny, nz, z0, thickness, side):
    """Walls at z=0 and z=nz-1 plus a plate on [z0, z0+thickness) with a
    centred square hole of the given side."""
    s = walls_z(nx, ny, nz)
    s[z0:z0 + thickness] = 1
    x0 = (nx - side) // 2
    y0 = (ny - side) // 2
    s[z0:z0 + thickness, y0:y0 + side, x0:x0 + side] = 0
    return s


def sphere_solid(nx, ny, nz, centre, radius):
    """Solid ball (for curved-wall geometry checks), fully periodic box."""
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx),
                          indexing="ij")
    r2 = (x - centre[0]) ** 2 + (y - centre[1]) ** 2 + (z - centre[2]) ** 2
    return (r2 <= radius * radius).astype(np.uint8)


def cylinder_solid(nx, ny, nz, centre_xy, radius):
    """Solid cylinder along z (curved-wall geometry checks), periodic box."""
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx),
                          indexing="ij")
    r2 = (x - centre_xy[0]) ** 2 + (y - centre_xy[1]) ** 2
    return (r2 <= radius * radius).astype(np.uint8)


def rough_wall_z(nx, ny, nz, amplitude, seed=SEED):
    """Walls at z = 0 and nz - 1, the bottom one rough: column (x, y) is
    solid up to a seeded height drawn uniformly from 0 .. amplitude."""
    h = np.floor(fast_uniform((ny, nx), seed=seed, lo=0.0,
                              hi=amplitude + 1.0)).astype(np.int64)
    z = np.arange(nz)[:, None, None]
    solid = (z <= h[None]).astype(np.uint8)
    solid[-1] = 1
    return solid


# ------------------------------------------------------------ phase fields

def droplet(nx, ny, nz, centre, radius, width, dtype=np.float32):
    """Diffuse droplet phi = 1/2 [1 + tanh(2 (R - |x - x_c|) / width)],
    liquid (phi = 1) inside."""
    z, y, x = np.meshgrid(np.arange(nz, dtype=np.float64),
                          np.arange(ny, dtype=np.float64),
                          np.arange(nx, dtype=np.float64), indexing="ij")
    r = np.sqrt((x - centre[0]) ** 2 + (y - centre[1]) ** 2 +
                (z - centre[2]) ** 2)
    return (0.5 * (1.0 + np.tanh(2.0 * (radius - r) / width))).astype(dtype)


def flat_interface(nx, ny, nz, x0, width, axis=0, dtype=np.float32):
    """Planar diffuse interface normal to ``axis``, liquid for coordinate
    below x0."""
    coords = np.meshgrid(np.arange(nz, dtype=np.float64),
                         np.arange(ny, dtype=np.float64),
                         np.arange(nx, dtype=np.float64), indexing="ij")
    c = coords[2 - axis]
    return (0.5 * (1.0 + np.tanh(2.0 * (x0 - c) / width))).astype(dtype)


# -------------------------------------------------------------- parameters

def base_params(nx, ny, nz, **kw):
    """Parameter dict with the conventions of the paper's benchmarks:
    width 4, mobility 0.02, periodic in x and y, walls along z."""
    p = dict(dim=3, nx=nx, ny=ny, nz=nz, periodic=(1, 1, 0), width=4.0,
             mobility=0.02, sigma=0.01, rho_l=1.0, rho_g=1.0, nu_l=0.04,
             nu_g=0.04, gravity=(0.0, 0.0, 0.0), theta_deg=90.0, eps_phi=1e-3)
    p.update(kw)
    return p


def static_droplet_256(theta_deg=60.0):
    """Static contact angle test shaped like Sect. 3.1: 256^3, cap R0 = 40
    centred on the bottom wall, equal densities and viscosities nu = 0.04,
    sigma = 0.02."""
    n = 256
    p = base_params(n, n, n, sigma=0.02, theta_deg=theta_deg)
    solid = walls_z(n, n, n)
    phi = droplet(n, n, n, (n / 2, n / 2, 0.5), 40.0, p["width"])
    return p, solid, phi


def spreading_128(theta_deg=60.0):
    """3D spreading on a flat wall: 128^3, hemispherical cap R = 24 at rest,
    density ratio 10, viscosity ratio 10, sigma = 0.005."""
    n = 128
    p = base_params(n, n, n, sigma=0.005, rho_l=1.0, rho_g=0.1, nu_l=0.05,
                    nu_g=0.05, theta_deg=theta_deg)
    solid = walls_z(n, n, n)
    phi = droplet(n, n, n, (n / 2, n / 2, 0.5), 24.0, p["width"])
    return p, solid, phi


def orifice_128x128x256(side=24, theta_deg=60.0, bond=1.0):
    """Gravity-driven droplet above a plate 8 nodes thick at z = 128 with a
    centred square hole; density ratio 50, Bond number sets g_z."""
    nx, ny, nz = 128, 128, 256
    sigma, rho_l, rho_g, R = 0.01, 1.0, 0.02, 20.0
    D = 2 * R
    gz = -bond * sigma / ((rho_l - rho_g) * D * D)
    p = base_params(nx, ny, nz, sigma=sigma, rho_l=rho_l, rho_g=rho_g,
                    nu_l=0.05, nu_g=0.05, gravity=(0.0, 0.0, gz),
                    theta_deg=theta_deg)
    solid = orifice_plate(nx, ny, nz, 128, 8, side)
    phi = droplet(nx, ny, nz, (nx / 2, ny / 2, 128 + 8 + 2 * R), R, p["width"])
    return p, solid, phi


def static_droplet_2d(theta_deg=60.0):
    """2D static droplet: 128 x 64, periodic in x, walls at y = 0 and
    y = 63, semicircle of radius 20 on the bottom wall, W = 4, sigma = 0.01,
    mobility 0.02, equal densities and viscosities (nu = 0.04)."""
    nx, ny = 128, 64
    p = base_params(nx, ny, 1, dim=2, periodic=(1, 0, 1), sigma=0.01,
                    theta_deg=theta_deg)
    solid = walls_y(nx, ny, 1)
    phi = droplet(nx, ny, 1, (nx / 2, 0.5, 0.0), 20.0, p["width"])
    return p, solid, phi


def random_state(shape, Q, seed=SEED, amp=1e-2):
    """Random post-collision populations and velocities for one-step parity:
    f_q = w-free small perturbations in [-amp, amp)."""
    f = fast_uniform((Q,) + tuple(shape), seed=seed, lo=-amp, hi=amp)
    return f.astype(np.float32)


def impact_sweep(ncases=48, seed=SEED):
    """Batched impact cases: edge n in [64, 160], R = 0.2 n, theta in
    [120, 160] deg, We in [1, 80], density ratio 100."""
    g = SplitMix64(seed)
    cases = []
    for _ in range(ncases):
        n = 64 + int(g.uniform(0.0, 97.0))
        theta = g.uniform(120.0, 160.0)
        we = g.uniform(1.0, 80.0)
        R = 0.2 * n
        sigma, rho_l = 0.003, 1.0
        U0 = math.sqrt(we * sigma / (rho_l * 2.0 * R))
        cases.append(dict(n=n, theta_deg=theta, we=we, radius=R, u0=U0))
    return cases
