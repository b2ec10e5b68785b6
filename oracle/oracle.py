"""ctypes wrapper of the FP64 CPU oracle -- TEST INFRASTRUCTURE.

Only tests, ``__graft_entry__.smoke()`` and the bench's CPU-baseline leg may
import this module. It loads ``oracle/libcacl_oracle.so`` (built by
``oracle/build.py``) and exposes the oracle's step and its parts on numpy
arrays. Field layout: node n = x + nx*(y + ny*z); arrays returned here have
shape (nz, ny, nx), populations (Q, nz, ny, nx), velocity (3, nz, ny, nx).
It imports nothing from the CUDA package.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None


class OrcParams(C.Structure):
    _fields_ = [
        ("dim", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("periodic", C.c_int * 3),
        ("width", C.c_double), ("mobility", C.c_double), ("sigma", C.c_double),
        ("rho_l", C.c_double), ("rho_g", C.c_double),
        ("nu_l", C.c_double), ("nu_g", C.c_double),
        ("gravity", C.c_double * 3),
        ("theta_deg", C.c_double), ("eps_phi", C.c_double),
    ]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        P = C.c_void_p
        dp = C.POINTER(C.c_double)
        L.orc_create.restype = P
        L.orc_create.argtypes = [C.POINTER(OrcParams)]
        L.orc_destroy.argtypes = [P]
        L.orc_error.restype = C.c_char_p
        L.orc_error.argtypes = [P]
        for name in ("orc_set_geometry", "orc_set_contact_angle",
                     "orc_set_fields", "orc_set_populations", "orc_set_phi",
                     "orc_set_velocity", "orc_get_fields",
                     "orc_get_populations", "orc_get_wall_list", "orc_get_mass",
                     "orc_grad_lap", "orc_collide_node"):
            getattr(L, name).restype = C.c_int
        L.orc_set_geometry.argtypes = [P, C.c_void_p]
        L.orc_set_contact_angle.argtypes = [P, C.c_void_p]
        L.orc_set_fields.argtypes = [P, C.c_void_p, C.c_void_p]
        L.orc_set_populations.argtypes = [P, C.c_void_p]
        L.orc_set_phi.argtypes = [P, C.c_void_p]
        L.orc_set_velocity.argtypes = [P, C.c_void_p]
        L.orc_set_mass_ref.argtypes = [P, C.c_double]
        L.orc_set_mass_ref.restype = C.c_int
        for name in ("orc_step",):
            getattr(L, name).argtypes = [P, C.c_int]
            getattr(L, name).restype = C.c_int
        for name in ("orc_ghost_update", "orc_lb_collide", "orc_phase_update",
                     "orc_volume_correct", "orc_get_wall_count"):
            getattr(L, name).argtypes = [P]
            getattr(L, name).restype = C.c_int
        L.orc_fluid_mass.argtypes = [P]
        L.orc_fluid_mass.restype = C.c_double
        L.orc_get_fields.argtypes = [P, C.c_void_p, C.c_void_p, C.c_void_p]
        L.orc_get_populations.argtypes = [P, C.c_void_p]
        L.orc_get_wall_list.argtypes = [P] + [C.c_void_p] * 5
        L.orc_get_mass.argtypes = [P, dp, dp, dp, dp]
        L.orc_lattice.argtypes = [C.c_int, C.c_void_p, C.c_void_p]
        L.orc_lattice.restype = C.c_int
        L.orc_feq.argtypes = [C.c_int, C.c_double, C.c_void_p, C.c_void_p]
        L.orc_feq.restype = C.c_int
        L.orc_collide_node.argtypes = [P, C.c_void_p, C.c_double, C.c_void_p,
                                       C.c_double, C.c_void_p, C.c_void_p,
                                       C.c_void_p, C.c_void_p]
        L.orc_grad_lap.argtypes = [P, C.c_void_p, C.c_void_p, C.c_void_p]
        L.orc_ghost_value.argtypes = [C.c_double, C.c_void_p, C.c_void_p,
                                      C.c_void_p, C.c_double]
        L.orc_ghost_value.restype = C.c_double
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def lattice(dim=3):
    """(c[Q,3] int, w[Q] float64) in the oracle's direction order."""
    c = np.zeros((27, 3), dtype=np.int32)
    w = np.zeros(27, dtype=np.float64)
    Q = lib().orc_lattice(dim, _ptr(c), _ptr(w))
    return c[:Q].copy(), w[:Q].copy()


def feq(pstar, u, dim=3):
    out = np.zeros(27, dtype=np.float64)
    uu = _f64(list(u) + [0.0] * (3 - len(u)))
    Q = lib().orc_feq(dim, float(pstar), _ptr(uu), _ptr(out))
    return out[:Q].copy()


def ghost_value(phi_f, grad_f, nw, r_fs, theta_deg):
    return lib().orc_ghost_value(float(phi_f), _ptr(_f64(grad_f)),
                                 _ptr(_f64(nw)), _ptr(_f64(r_fs)),
                                 float(theta_deg))


class Oracle:
    """One oracle state. ``params`` is a dict with the keys of OrcParams."""

    def __init__(self, params):
        p = OrcParams()
        p.dim = int(params.get("dim", 3))
        p.nx, p.ny, p.nz = (int(params["nx"]), int(params["ny"]),
                            int(params["nz"]))
        for a, v in enumerate(params.get("periodic", (1, 1, 0))):
            p.periodic[a] = int(v)
        p.width = float(params.get("width", 4.0))
        p.mobility = float(params.get("mobility", 0.02))
        p.sigma = float(params.get("sigma", 0.01))
        p.rho_l = float(params.get("rho_l", 1.0))
        p.rho_g = float(params.get("rho_g", 1.0))
        p.nu_l = float(params.get("nu_l", 0.04))
        p.nu_g = float(params.get("nu_g", 0.04))
        for a, v in enumerate(params.get("gravity", (0.0, 0.0, 0.0))):
            p.gravity[a] = float(v)
        p.theta_deg = float(params.get("theta_deg", 90.0))
        p.eps_phi = float(params.get("eps_phi", 1e-3))
        self.p = p
        self.shape = (p.nz, p.ny, p.nx)
        self.N = p.nx * p.ny * p.nz
        self.Q = 27 if p.dim == 3 else 9
        self.h = lib().orc_create(C.byref(p))
        if not self.h:
            raise ValueError("oracle rejected the parameters")

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            lib().orc_destroy(h)
            self.h = None

    def _check(self, rc):
        if rc != 0:
            raise RuntimeError(lib().orc_error(self.h).decode() or f"rc={rc}")

    def set_geometry(self, solid):
        s = np.ascontiguousarray(solid, dtype=np.uint8).reshape(-1)
        assert s.size == self.N
        self._check(lib().orc_set_geometry(self.h, _ptr(s)))

    def set_contact_angle(self, theta_deg=None):
        t = None if theta_deg is None else _f64(theta_deg).reshape(-1)
        self._check(lib().orc_set_contact_angle(self.h, _ptr(t)))

    def set_fields(self, phi, u=None):
        ph = _f64(phi).reshape(-1)
        uu = None if u is None else _f64(u).reshape(-1)
        self._check(lib().orc_set_fields(self.h, _ptr(ph), _ptr(uu)))

    def set_populations(self, f):
        ff = _f64(f).reshape(-1)
        assert ff.size == self.Q * self.N
        self._check(lib().orc_set_populations(self.h, _ptr(ff)))

    def set_phi(self, phi):
        self._check(lib().orc_set_phi(self.h, _ptr(_f64(phi).reshape(-1))))

    def set_velocity(self, u):
        self._check(lib().orc_set_velocity(self.h, _ptr(_f64(u).reshape(-1))))

    def set_mass_ref(self, m):
        self._check(lib().orc_set_mass_ref(self.h, float(m)))

    def step(self, n=1):
        self._check(lib().orc_step(self.h, int(n)))

    def ghost_update(self):
        self._check(lib().orc_ghost_update(self.h))

    def lb_collide(self):
        self._check(lib().orc_lb_collide(self.h))

    def phase_update(self):
        self._check(lib().orc_phase_update(self.h))

    def volume_correct(self):
        self._check(lib().orc_volume_correct(self.h))

    def fields(self):
        phi = np.zeros(self.N)
        u = np.zeros(3 * self.N)
        ps = np.zeros(self.N)
        self._check(lib().orc_get_fields(self.h, _ptr(phi), _ptr(u), _ptr(ps)))
        return (phi.reshape(self.shape), u.reshape((3,) + self.shape),
                ps.reshape(self.shape))

    def populations(self):
        f = np.zeros(self.Q * self.N)
        self._check(lib().orc_get_populations(self.h, _ptr(f)))
        return f.reshape((self.Q,) + self.shape)

    def wall_list(self):
        W = lib().orc_get_wall_count(self.h)
        idx = np.zeros(W, dtype=np.int32)
        q = np.zeros(W, dtype=np.int8)
        n6 = np.zeros(3 * W, dtype=np.int16)
        nwf = np.zeros(3 * W, dtype=np.float32)
        nwd = np.zeros(3 * W, dtype=np.float64)
        self._check(lib().orc_get_wall_list(self.h, _ptr(idx), _ptr(q),
                                            _ptr(n6), _ptr(nwf), _ptr(nwd)))
        return dict(idx=idx, qstar=q, ntilde6=n6.reshape(W, 3),
                    nw_f32=nwf.reshape(W, 3), nw=nwd.reshape(W, 3))

    def mass(self):
        vals = [C.c_double() for _ in range(4)]
        self._check(lib().orc_get_mass(self.h, *[C.byref(v) for v in vals]))
        return dict(m_ref=vals[0].value, m_star=vals[1].value,
                    w_sum=vals[2].value, lam=vals[3].value)

    def fluid_mass(self):
        return lib().orc_fluid_mass(self.h)

    def grad_lap(self, field):
        fld = _f64(field).reshape(-1)
        g = np.zeros(3 * self.N)
        lap = np.zeros(self.N)
        self._check(lib().orc_grad_lap(self.h, _ptr(fld), _ptr(g), _ptr(lap)))
        return g.reshape((3,) + self.shape), lap.reshape(self.shape)

    def collide_node(self, f_in, phi, grad_phi, lap_phi):
        fin = _f64(f_in)
        fo = np.zeros(self.Q)
        u = np.zeros(3)
        a = np.zeros(3)
        om = C.c_double()
        self._check(lib().orc_collide_node(self.h, _ptr(fin), float(phi),
                                           _ptr(_f64(grad_phi)), float(lap_phi),
                                           _ptr(fo), _ptr(u), _ptr(a),
                                           C.byref(om)))
        return fo, u, a, om.value
