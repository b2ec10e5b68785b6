"""Python binding of libcacl.so (include/cacl.h): argument marshalling only.

Every step of the method runs in the library's sm_103a kernels. PyTorch
supplies the CUDA stream (``torch.cuda.current_stream()``) and, for the
device-pointer getters, device memory. There is no CPU fallback: if the
library is missing or no GPU is present the calls raise.
"""
import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcacl.so")

CACL_OK = 0
STATUS = {0: "CACL_OK", -1: "CACL_ERR_ARG", -2: "CACL_ERR_CUDA",
          -3: "CACL_ERR_STATE", -4: "CACL_ERR_GEOMETRY",
          -5: "CACL_ERR_DIVERGED", -6: "CACL_ERR_TIMEOUT",
          -7: "CACL_ERR_TOO_LARGE"}
STORAGE = {"f32": 0, "f16": 1, "bf16": 2, "moments": 3}

EXPORTS = (
    "cacl_create", "cacl_destroy", "cacl_last_error", "cacl_set_geometry",
    "cacl_set_contact_angle", "cacl_set_fields", "cacl_set_populations",
    "cacl_set_phi", "cacl_set_velocity", "cacl_set_mass_ref", "cacl_step",
    "cacl_ghost_update", "cacl_lb_collide", "cacl_phase_update",
    "cacl_volume_correct", "cacl_get_fields", "cacl_get_populations",
    "cacl_get_wall_list", "cacl_get_mass", "cacl_check_finite",
    "cacl_set_option", "cacl_get_info", "cacl_volume_correct_noalloc",
    "cacl_batch_create", "cacl_batch_destroy", "cacl_batch_last_error",
    "cacl_batch_case", "cacl_batch_step", "cacl_batch_set_option",
    "cacl_batch_autotune", "cacl_set_wall_angles", "cacl_set_sigma",
    "cacl_adjoint_forward", "cacl_adjoint_forward_levels", "cacl_adjoint_backward",
    "cacl_adjoint_timing", "cacl_adjoint_stage", "cacl_state_bytes", "cacl_save_state",
    "cacl_load_state", "cacl_inject_wait_timeout", "cacl_inject_copy_stall", "cacl_slab_create", "cacl_slab_stage", "cacl_slab_partials", "cacl_slab_correct",
    "cacl_slab_halo", "cacl_slab_halo_bytes",
)
OPT_PHASE_TILE = 1
OPT_PHASE_PIPE = 2  # 0 auto, 1 registers, 2 copies (2 nodes/thread), 3 copies (2 x 2)
OPT_LB_PIPE = 3  # 0 direct loads, 1 bulk-copy staged rows
OPT_INDEX64 = 4  # 1: the 64-bit offset forms of the kernels, at any size
ADJ_CORRECT, ADJ_PHASE, ADJ_COLLIDE, ADJ_GHOST = 0, 1, 2, 3  # cacl_adjoint_stage


class CaclError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class CaclParams(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("periodic", C.c_int * 3),
        ("width", C.c_double), ("mobility", C.c_double), ("sigma", C.c_double),
        ("rho_l", C.c_double), ("rho_g", C.c_double),
        ("nu_l", C.c_double), ("nu_g", C.c_double),
        ("gravity", C.c_double * 3),
        ("theta_deg", C.c_double), ("eps_phi", C.c_double),
        ("storage", C.c_int),
    ]


_lib = None


def load():
    """Load libcacl.so; raise if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(
            f"CUDA library not built: {LIB_PATH} is missing "
            "(run __graft_entry__.build() or paper_2607_25444_b300/build.py)")
    L = C.CDLL(LIB_PATH)
    vp = C.c_void_p
    L.cacl_create.argtypes = [C.POINTER(CaclParams), vp, C.POINTER(vp)]
    L.cacl_destroy.argtypes = [vp]
    L.cacl_destroy.restype = None
    L.cacl_last_error.argtypes = [vp]
    L.cacl_last_error.restype = C.c_char_p
    L.cacl_set_geometry.argtypes = [vp, vp]
    L.cacl_set_contact_angle.argtypes = [vp, vp]
    L.cacl_set_fields.argtypes = [vp, vp, vp]
    L.cacl_set_populations.argtypes = [vp, vp]
    L.cacl_set_phi.argtypes = [vp, vp]
    L.cacl_set_velocity.argtypes = [vp, vp]
    L.cacl_set_mass_ref.argtypes = [vp, C.c_double]
    L.cacl_step.argtypes = [vp, C.c_int]
    for name in ("cacl_ghost_update", "cacl_lb_collide", "cacl_phase_update",
                 "cacl_volume_correct", "cacl_check_finite"):
        getattr(L, name).argtypes = [vp]
    L.cacl_get_fields.argtypes = [vp, vp, vp, vp, C.c_int]
    L.cacl_get_populations.argtypes = [vp, vp, C.c_int]
    L.cacl_get_wall_list.argtypes = [vp, vp, vp, vp, vp, C.POINTER(C.c_int32)]
    dp = C.POINTER(C.c_double)
    L.cacl_get_mass.argtypes = [vp, dp, dp, dp, dp]
    L.cacl_set_option.argtypes = [vp, C.c_int, C.c_int]
    L.cacl_get_info.argtypes = [vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                C.POINTER(C.c_int32)]
    L.cacl_volume_correct_noalloc.argtypes = [vp, vp, C.c_int64, C.c_double,
                                              C.c_double, vp, vp]
    L.cacl_batch_create.argtypes = [C.POINTER(CaclParams), C.c_int, vp,
                                    C.POINTER(vp)]
    L.cacl_batch_destroy.argtypes = [vp]
    L.cacl_batch_destroy.restype = None
    L.cacl_batch_last_error.argtypes = [vp]
    L.cacl_batch_last_error.restype = C.c_char_p
    L.cacl_batch_case.argtypes = [vp, C.c_int, C.POINTER(vp)]
    L.cacl_batch_step.argtypes = [vp, C.c_int]
    L.cacl_batch_set_option.argtypes = [vp, C.c_int, C.c_int]
    L.cacl_batch_autotune.argtypes = [vp, C.c_int, C.POINTER(C.c_int),
                                      C.POINTER(C.c_int), C.POINTER(C.c_float)]
    L.cacl_set_wall_angles.argtypes = [vp, vp]
    L.cacl_set_sigma.argtypes = [vp, C.c_double]
    L.cacl_adjoint_forward.argtypes = [vp, C.c_int, C.c_int]
    L.cacl_adjoint_forward_levels.argtypes = [vp, C.c_int, C.c_int, C.c_int]
    L.cacl_adjoint_backward.argtypes = [vp, vp, vp, vp]
    L.cacl_adjoint_timing.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_double)]
    L.cacl_adjoint_stage.argtypes = [vp, C.c_int, vp, vp, vp, vp]
    L.cacl_state_bytes.argtypes = [vp]
    L.cacl_state_bytes.restype = C.c_int64
    L.cacl_save_state.argtypes = [vp, vp, C.c_int64]
    L.cacl_load_state.argtypes = [vp, vp, C.c_int64]
    L.cacl_inject_wait_timeout.argtypes = [vp]
    L.cacl_inject_copy_stall.argtypes = [vp, C.c_int]
    L.cacl_slab_create.argtypes = [C.POINTER(CaclParams), C.c_int, C.c_int, vp,
                                   C.POINTER(vp)]
    L.cacl_slab_stage.argtypes = [vp, C.c_int]
    L.cacl_slab_partials.argtypes = [vp, vp, C.POINTER(C.c_int)]
    L.cacl_slab_correct.argtypes = [vp, vp, C.c_int]
    L.cacl_slab_halo.argtypes = [vp, C.c_int, C.c_int, C.c_int, vp]
    L.cacl_slab_halo_bytes.argtypes = [vp, C.c_int]
    for name in EXPORTS:
        f = getattr(L, name)
        if name not in ("cacl_destroy", "cacl_last_error", "cacl_batch_destroy",
                        "cacl_batch_last_error", "cacl_slab_halo_bytes"):
            f.restype = C.c_int
    L.cacl_slab_halo_bytes.restype = C.c_int64
    _lib = L
    return L


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f32(a, n=None):
    a = np.ascontiguousarray(a, dtype=np.float32).reshape(-1)
    if n is not None and a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


def make_params(d):
    p = CaclParams()
    p.nx, p.ny, p.nz = int(d["nx"]), int(d["ny"]), int(d["nz"])
    for a, v in enumerate(d.get("periodic", (1, 1, 0))):
        p.periodic[a] = int(v)
    p.width = float(d.get("width", 4.0))
    p.mobility = float(d.get("mobility", 0.02))
    p.sigma = float(d.get("sigma", 0.01))
    p.rho_l = float(d.get("rho_l", 1.0))
    p.rho_g = float(d.get("rho_g", 1.0))
    p.nu_l = float(d.get("nu_l", 0.04))
    p.nu_g = float(d.get("nu_g", 0.04))
    for a, v in enumerate(d.get("gravity", (0.0, 0.0, 0.0))):
        p.gravity[a] = float(v)
    p.theta_deg = float(d.get("theta_deg", 90.0))
    p.eps_phi = float(d.get("eps_phi", 1e-3))
    st = d.get("storage", "f32")
    p.storage = STORAGE[st] if isinstance(st, str) else int(st)
    return p


def volume_correct_noalloc(phi, solid, m_ref, eps_phi=1e-3, out=None,
                           stream=None):
    """Allocation-free volume correction of a phase field held in torch
    CUDA tensors: ``phi`` (float32, corrected in place), ``solid`` (uint8,
    nonzero = solid), ``out`` (float64, at least 3 values: M*, W, lambda) or
    None. All tensors must be contiguous and on one CUDA device; the call
    runs with that device current, enqueued on ``stream`` (default: that
    device's current torch stream)."""
    import torch
    L = load()
    tens = [("phi", phi, torch.float32), ("solid", solid, torch.uint8)]
    if out is not None:
        tens.append(("out", out, torch.float64))
    for name, t, dt in tens:
        if not (t.is_cuda and t.is_contiguous()):
            raise ValueError(f"{name} must be a contiguous CUDA tensor")
        if t.dtype != dt:
            raise ValueError(f"{name} must be {dt}, got {t.dtype}")
        if t.device != phi.device:
            raise ValueError(f"{name} is on {t.device}, phi on {phi.device}")
    if phi.numel() != solid.numel():
        raise ValueError("phi and solid differ in size")
    if out is not None and out.numel() < 3:
        raise ValueError("out must hold at least 3 doubles")
    with torch.cuda.device(phi.device):
        s = torch.cuda.current_stream().cuda_stream if stream is None else stream
        rc = L.cacl_volume_correct_noalloc(
            C.c_void_p(phi.data_ptr()), C.c_void_p(solid.data_ptr()),
            int(phi.numel()), float(m_ref), float(eps_phi),
            None if out is None else C.c_void_p(out.data_ptr()), C.c_void_p(s))
    if rc != CACL_OK:
        raise CaclError(rc, "cacl_volume_correct_noalloc")


def current_stream():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("no CUDA device: the CAC-LB library runs on the GPU only")
    return torch.cuda.current_stream().cuda_stream


class Solver:
    """One CAC-LB state on the current CUDA device and stream.

    ``params`` is a dict with the fields of cacl_params (D3Q27 only: a
    two-dimensional problem is a periodic slab one node thick).
    """

    def __init__(self, params, stream=None, handle=None, local_shape=None):
        self.L = load()
        if handle is not None and local_shape is not None:
            # a slab context (slab.SlabSolver): owned, local grid given
            self.params = None
            self.shape = tuple(int(v) for v in local_shape)
            self.N = int(np.prod(self.shape))
            self.h = C.c_void_p(handle)
            self._owned = True
            return
        if handle is not None:  # a case owned by a Batch
            self.params = dict(params)
            self.p = make_params(params)
            self.shape = (self.p.nz, self.p.ny, self.p.nx)
            self.N = self.p.nx * self.p.ny * self.p.nz
            self.h = handle
            self._owned = False
            return
        self._owned = True
        if params.get("dim", 3) != 3 and params.get("nz", 1) != 1:
            raise ValueError("dim 2 runs as a D3Q27 slab with nz = 1")
        self.params = dict(params)
        self.p = make_params(params)
        self.shape = (self.p.nz, self.p.ny, self.p.nx)
        self.N = self.p.nx * self.p.ny * self.p.nz
        s = current_stream() if stream is None else stream
        h = C.c_void_p()
        rc = self.L.cacl_create(C.byref(self.p), C.c_void_p(s), C.byref(h))
        if rc != CACL_OK:
            raise CaclError(rc, "cacl_create rejected the parameters or failed")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            if getattr(self, "_owned", True):
                self.L.cacl_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != CACL_OK:
            msg = self.L.cacl_last_error(self.h)
            raise CaclError(rc, msg.decode() if msg else "")

    # -- set-up
    def set_geometry(self, solid):
        s = np.ascontiguousarray(solid, dtype=np.uint8).reshape(-1)
        if s.size != self.N:
            raise ValueError("occupancy has the wrong size")
        self._check(self.L.cacl_set_geometry(self.h, _ptr(s)))

    def set_contact_angle(self, theta_deg=None):
        t = None if theta_deg is None else _f32(theta_deg, self.N)
        self._check(self.L.cacl_set_contact_angle(self.h, _ptr(t)))

    def set_fields(self, phi, u=None):
        ph = _f32(phi, self.N)
        uu = None if u is None else _f32(u, 3 * self.N)
        self._check(self.L.cacl_set_fields(self.h, _ptr(ph), _ptr(uu)))

    def set_populations(self, f):
        self._check(self.L.cacl_set_populations(self.h, _ptr(_f32(f, 27 * self.N))))

    def set_phi(self, phi):
        self._check(self.L.cacl_set_phi(self.h, _ptr(_f32(phi, self.N))))

    def set_velocity(self, u):
        self._check(self.L.cacl_set_velocity(self.h, _ptr(_f32(u, 3 * self.N))))

    def set_mass_ref(self, m):
        self._check(self.L.cacl_set_mass_ref(self.h, float(m)))

    # -- the step and its parts
    def step(self, n=1):
        self._check(self.L.cacl_step(self.h, int(n)))

    def ghost_update(self):
        self._check(self.L.cacl_ghost_update(self.h))

    def lb_collide(self):
        self._check(self.L.cacl_lb_collide(self.h))

    def phase_update(self):
        self._check(self.L.cacl_phase_update(self.h))

    def volume_correct(self):
        self._check(self.L.cacl_volume_correct(self.h))

    # -- queries
    def fields(self):
        phi = np.empty(self.N, np.float32)
        u = np.empty(3 * self.N, np.float32)
        ps = np.empty(self.N, np.float32)
        self._check(self.L.cacl_get_fields(self.h, _ptr(phi), _ptr(u), _ptr(ps), 0))
        return (phi.reshape(self.shape), u.reshape((3,) + self.shape),
                ps.reshape(self.shape))

    def fields_device(self, phi=None, u=None, pstar=None):
        """Copy into torch CUDA tensors (float32, contiguous) on the stream."""
        def dp(t):
            return None if t is None else C.c_void_p(t.data_ptr())
        self._check(self.L.cacl_get_fields(self.h, dp(phi), dp(u), dp(pstar), 1))

    def populations(self):
        f = np.empty(27 * self.N, np.float32)
        self._check(self.L.cacl_get_populations(self.h, _ptr(f), 0))
        return f.reshape((27,) + self.shape)

    def wall_list(self):
        cnt = C.c_int32()
        self._check(self.L.cacl_get_wall_list(self.h, None, None, None, None,
                                              C.byref(cnt)))
        W = cnt.value
        idx = np.empty(W, np.int32)
        q = np.empty(W, np.int8)
        n6 = np.empty(3 * W, np.int16)
        nw = np.empty(3 * W, np.float32)
        self._check(self.L.cacl_get_wall_list(self.h, _ptr(idx), _ptr(q),
                                              _ptr(n6), _ptr(nw), C.byref(cnt)))
        return dict(idx=idx, qstar=q, ntilde6=n6.reshape(W, 3),
                    nw_f32=nw.reshape(W, 3))

    def mass(self):
        v = [C.c_double() for _ in range(4)]
        self._check(self.L.cacl_get_mass(self.h, *[C.byref(x) for x in v]))
        return dict(m_ref=v[0].value, m_star=v[1].value, w_sum=v[2].value,
                    lam=v[3].value)

    def check_finite(self):
        self._check(self.L.cacl_check_finite(self.h))

    def set_wall_angles(self, theta_deg_wall):
        t = _f32(theta_deg_wall)
        self._check(self.L.cacl_set_wall_angles(self.h, _ptr(t)))

    def set_sigma(self, sigma):
        self._check(self.L.cacl_set_sigma(self.h, float(sigma)))

    def adjoint_forward(self, nsteps, ckpt_every, outer_every=0):
        """Forward rollout keeping checkpoints for the adjoint; outer_every > 0
        (a multiple of ckpt_every) selects two-level checkpointing."""
        if outer_every:
            self._check(self.L.cacl_adjoint_forward_levels(
                self.h, int(nsteps), int(ckpt_every), int(outer_every)))
        else:
            self._check(self.L.cacl_adjoint_forward(self.h, int(nsteps),
                                                    int(ckpt_every)))

    def adjoint_backward(self, dl_dphi, dl_dtheta, dl_dsigma):
        """Device torch tensors: dl_dphi (float32, N), dl_dtheta (float64,
        W), dl_dsigma (float64, 1)."""
        self._check(self.L.cacl_adjoint_backward(
            self.h, C.c_void_p(dl_dphi.data_ptr()), C.c_void_p(dl_dtheta.data_ptr()),
            C.c_void_p(dl_dsigma.data_ptr())))

    def adjoint_stage(self, stage, cot_in, out, dparam=None, state=None):
        """One stage's transpose at step 0 of the last forward (test hook,
        cacl_adjoint_stage): device torch tensors, float32 cot_in / out /
        state, float64 dparam."""
        import torch
        for t, dt in ((cot_in, torch.float32), (out, torch.float32), (dparam, torch.float64),
                      (state, torch.float32)):
            if t is not None and (not t.is_cuda or t.dtype != dt or not t.is_contiguous()):
                raise ValueError("adjoint_stage: contiguous CUDA tensors of the stated dtypes")
        ptr = lambda t: None if t is None else C.c_void_p(t.data_ptr())
        self._check(self.L.cacl_adjoint_stage(self.h, int(stage), ptr(cot_in), ptr(out),
                                              ptr(dparam), ptr(state)))

    def save_state(self):
        """The complete dynamic state (cacl_save_state) as a bytes object."""
        n = self.L.cacl_state_bytes(self.h)
        if n < 0:
            raise CaclError(-3, "cacl_state_bytes: set_geometry first")
        buf = C.create_string_buffer(int(n))
        self._check(self.L.cacl_save_state(self.h, buf, C.c_int64(n)))
        return buf.raw

    def load_state(self, state):
        """Restore a state from save_state (same grid, storage, geometry)."""
        buf = C.create_string_buffer(bytes(state), len(state))
        self._check(self.L.cacl_load_state(self.h, buf, C.c_int64(len(state))))

    def inject_wait_timeout(self):
        """Test hook: mark the context as if a copy wait had given up."""
        self._check(self.L.cacl_inject_wait_timeout(self.h))

    def inject_copy_stall(self, on=True):
        """Test hook: make the copy-staged and TMA-tiled collide-stream's
        first waits run out (CACL_OPT_LB_PIPE = 1 or 3; each after 0.5 s)."""
        self._check(self.L.cacl_inject_copy_stall(self.h, 1 if on else 0))

    def adjoint_timing(self):
        """GPU milliseconds of the last backward: (recompute, total)."""
        r, t = C.c_double(), C.c_double()
        self._check(self.L.cacl_adjoint_timing(self.h, C.byref(r), C.byref(t)))
        return r.value, t.value

    def set_option(self, option, value):
        self._check(self.L.cacl_set_option(self.h, int(option), int(value)))

    def info(self):
        n, b, w = C.c_int64(), C.c_int64(), C.c_int32()
        self._check(self.L.cacl_get_info(self.h, C.byref(n), C.byref(b), C.byref(w)))
        return dict(nodes=n.value, device_bytes=b.value, wall_count=w.value)


class Batch:
    """Many cases advanced together: each stage of the step is one launch
    over all cases. ``cases[i]`` is a Solver view of case i for set-up and
    queries (owned by the batch)."""

    def __init__(self, params_list, stream=None):
        self.L = load()
        arr = (CaclParams * len(params_list))(*[make_params(p) for p in params_list])
        s = current_stream() if stream is None else stream
        h = C.c_void_p()
        rc = self.L.cacl_batch_create(arr, len(params_list), C.c_void_p(s),
                                      C.byref(h))
        if rc != CACL_OK:
            raise CaclError(rc, "cacl_batch_create failed")
        self.h = h
        self.cases = []
        for i, p in enumerate(params_list):
            ch = C.c_void_p()
            self._check(self.L.cacl_batch_case(self.h, i, C.byref(ch)))
            self.cases.append(Solver(p, handle=ch))

    def _check(self, rc):
        if rc != CACL_OK:
            msg = self.L.cacl_batch_last_error(self.h)
            raise CaclError(rc, msg.decode() if msg else "")

    def step(self, n=1):
        self._check(self.L.cacl_batch_step(self.h, int(n)))

    def set_option(self, lb_variant, phase_variant):
        self._check(self.L.cacl_batch_set_option(self.h, int(lb_variant),
                                                 int(phase_variant)))

    def autotune(self, steps=3):
        lv, pv, ms = C.c_int(), C.c_int(), C.c_float()
        self._check(self.L.cacl_batch_autotune(self.h, int(steps), C.byref(lv),
                                               C.byref(pv), C.byref(ms)))
        return dict(lb_variant=lv.value, phase_variant=pv.value,
                    ms_per_step=ms.value)

    def close(self):
        if getattr(self, "h", None):
            for c in self.cases:
                c.h = None
            self.L.cacl_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
