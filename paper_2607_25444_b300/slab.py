"""z-slab decomposition of one CAC-LB problem: the plane layout, the halo
exchange schedule of a step, and the gather of the volume correction's
partial sums. Argument marshalling and data movement only: every stage of
the step runs in the library's kernels (cacl_slab_* in include/cacl.h).

A slab owns the global planes [z0, z0 + n) and holds them in a context of
n + 4 planes, local plane l being global plane (z0 - 2 + l) mod nz. One
step, on every slab (exchanges between the stages):

    ghost update          -> exchange phi (2 planes per side, with ghosts)
    collide-stream        -> exchange f* (1 plane) and u, a (1 plane)
    phi update (interior) -> gather the block partial sums of all slabs
    correction (lambda from the gathered sums) -> exchange phi (2 planes)

The exchange is a ring: a slab's lowest interior planes go to the halo of
the slab below (its high side), its highest ones to the slab above (its
low side), and the ends wrap as the grid's z axis does. ``DistExchange``
runs it between ranks of a torch.distributed process group (NCCL tensors
on the GPU, gloo tensors on the CPU); ``LocalExchange`` between slabs of
one process (a decomposition checked on one GPU).
"""
import ctypes as C

import numpy as np

HALO = 2
PHI, F, UA = 0, 1, 2          # exchanged fields (CACL_SLAB_*)
GHOST, COLLIDE, PHASE = 0, 1, 2  # slab stages
PHI_TILE_DEPTH = 32           # z depth of the phi update's default tile


def partition(nz, parts, align=PHI_TILE_DEPTH):
    """Interior plane ranges (z0, n) of `parts` slabs covering nz planes:
    equal shares in units of `align` planes (so that every interior starts
    on a multiple of it), the remainder to the last slab."""
    if parts < 1 or nz < parts:
        raise ValueError("need at least one plane per slab")
    units = nz // align if nz >= align * parts else 0
    if units >= parts:
        per = (units // parts) * align
        out = [(r * per, per) for r in range(parts)]
    else:
        per = nz // parts
        out = [(r * per, per) for r in range(parts)]
    z0, n = out[-1]
    out[-1] = (z0, nz - z0)
    return out


def local_planes(z0, n, nz):
    """Global plane index of each of the n + 4 local planes."""
    return [(z0 - HALO + l) % nz for l in range(n + 2 * HALO)]


def halo_planes(field):
    return 2 if field == PHI else 1


class LocalExchange:
    """Ring exchange between the slabs of one process, in slab order."""

    def __init__(self, nslabs):
        self.n = nslabs

    def run(self, packs):
        """packs[r] = (low, high) packed by slab r -> received[r] = (the
        high pack of slab r - 1, the low pack of slab r + 1)."""
        n = self.n
        return [(packs[(r - 1) % n][1], packs[(r + 1) % n][0]) for r in range(n)]


class DistExchange:
    """Ring exchange and partial-sum gather between the ranks of a
    torch.distributed process group (one slab per rank)."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)

    def sendrecv(self, low, high):
        """Send `low` to the rank below and `high` to the rank above;
        return (what the rank below sent up, what the rank above sent
        down)."""
        import torch
        if self.world == 1:
            return high.clone(), low.clone()
        d = self.dist
        down, up = (self.rank - 1) % self.world, (self.rank + 1) % self.world
        recv_lo = torch.empty_like(high)
        recv_hi = torch.empty_like(low)
        ops = [d.P2POp(d.isend, low, down, self.group),
               d.P2POp(d.irecv, recv_hi, up, self.group),
               d.P2POp(d.isend, high, up, self.group),
               d.P2POp(d.irecv, recv_lo, down, self.group)]
        for req in d.batch_isend_irecv(ops):
            req.wait()
        return recv_lo, recv_hi

    def gather_partials(self, local):
        """local = this rank's 2 nb sums (phi* parts, then chi parts; nb
        may differ between ranks) -> every rank's phi* parts in rank order,
        then every rank's chi parts."""
        import torch
        nb = local.numel() // 2
        counts = [torch.zeros(1, dtype=torch.int64, device=local.device)
                  for _ in range(self.world)]
        self.dist.all_gather(counts, torch.tensor([nb], dtype=torch.int64,
                                                  device=local.device),
                             group=self.group)
        nbs = [int(c.item()) for c in counts]
        top = max(nbs)
        padded = torch.zeros(2 * top, dtype=local.dtype, device=local.device)
        padded[:nb] = local[:nb]
        padded[top:top + nb] = local[nb:]
        parts = [torch.empty_like(padded) for _ in range(self.world)]
        self.dist.all_gather(parts, padded, group=self.group)
        return torch.cat([p[:k] for p, k in zip(parts, nbs)] +
                         [p[top:top + k] for p, k in zip(parts, nbs)])


def gather_local(partials):
    """The same gather for the slabs of one process (tensors in slab
    order)."""
    import torch
    nbs = [p.numel() // 2 for p in partials]
    return torch.cat([p[:nb] for p, nb in zip(partials, nbs)] +
                     [p[nb:] for p, nb in zip(partials, nbs)])


class SlabSolver:
    """One slab on the current CUDA device and stream (the library's
    context of n + 4 planes)."""

    def __init__(self, params, z0, n, stream=None):
        import torch

        from . import cacl
        self.cacl = cacl
        self.L = cacl.load()
        self.global_shape = (int(params["nz"]), int(params["ny"]), int(params["nx"]))
        self.z0, self.n = int(z0), int(n)
        self.planes = local_planes(self.z0, self.n, self.global_shape[0])
        self.p = cacl.make_params(params)
        s = cacl.current_stream() if stream is None else stream
        h = C.c_void_p()
        rc = self.L.cacl_slab_create(C.byref(self.p), self.z0, self.n, C.c_void_p(s),
                                     C.byref(h))
        if rc != cacl.CACL_OK:
            raise cacl.CaclError(rc, "cacl_slab_create")
        self.solver = cacl.Solver(None, handle=h.value,
                                  local_shape=(self.n + 2 * HALO,) + self.global_shape[1:])
        self.torch = torch
        self._buf = {}

    # ---- set-up from global arrays
    def _local(self, a, lead=0):
        a = np.asarray(a)
        return np.ascontiguousarray(a[(slice(None),) * lead + (self.planes,)])

    def set_geometry(self, solid):
        self.solver.set_geometry(self._local(solid))

    def set_contact_angle(self, theta_deg=None):
        self.solver.set_contact_angle(None if theta_deg is None else self._local(theta_deg))

    def set_fields(self, phi, u=None, m_ref=None):
        """Global phi (and u); m_ref: the global fluid mass (FP64) the
        correction restores."""
        self.solver.set_fields(self._local(phi), None if u is None else self._local(u, 1))
        if m_ref is not None:
            self.solver.set_mass_ref(float(m_ref))

    def fields(self):
        """phi, u, p* of the interior planes."""
        ph, u, ps = self.solver.fields()
        sl = slice(HALO, HALO + self.n)
        return ph[sl], u[:, sl], ps[sl]

    def populations(self):
        return self.solver.populations()[:, HALO:HALO + self.n]

    # ---- stages, exchange, correction
    def stage(self, which):
        self.solver._check(self.L.cacl_slab_stage(self.solver.h, which))

    def pack(self, field, side):
        torch = self.torch
        nbytes = self.L.cacl_slab_halo_bytes(self.solver.h, field)
        buf = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        self.solver._check(self.L.cacl_slab_halo(self.solver.h, field, side, 0,
                                                 C.c_void_p(buf.data_ptr())))
        return buf

    def unpack(self, field, side, buf):
        self.solver._check(self.L.cacl_slab_halo(self.solver.h, field, side, 1,
                                                 C.c_void_p(buf.data_ptr())))

    def partials(self):
        torch = self.torch
        nb = C.c_int()
        self.solver._check(self.L.cacl_slab_partials(self.solver.h, None, C.byref(nb)))
        out = torch.empty(2 * nb.value, dtype=torch.float64, device="cuda")
        self.solver._check(self.L.cacl_slab_partials(self.solver.h,
                                                     C.c_void_p(out.data_ptr()),
                                                     C.byref(nb)))
        return out

    def correct(self, gathered):
        self.solver._check(self.L.cacl_slab_correct(
            self.solver.h, C.c_void_p(gathered.data_ptr()), gathered.numel() // 2))

    def close(self):
        self.solver.close()


def exchange_local(slabs, field):
    packs = [(s.pack(field, 0), s.pack(field, 1)) for s in slabs]
    for s, (lo, hi) in zip(slabs, LocalExchange(len(slabs)).run(packs)):
        s.unpack(field, 0, lo)
        s.unpack(field, 1, hi)


def step_local(slabs, nsteps=1):
    """nsteps steps of a decomposition whose slabs live in this process."""
    for _ in range(nsteps):
        for s in slabs:
            s.stage(GHOST)
        exchange_local(slabs, PHI)
        for s in slabs:
            s.stage(COLLIDE)
        exchange_local(slabs, F)
        exchange_local(slabs, UA)
        for s in slabs:
            s.stage(PHASE)
        gathered = gather_local([s.partials() for s in slabs])
        for s in slabs:
            s.correct(gathered)
        exchange_local(slabs, PHI)


def exchange_dist(slab, ex, field):
    lo, hi = ex.sendrecv(slab.pack(field, 0), slab.pack(field, 1))
    slab.unpack(field, 0, lo)
    slab.unpack(field, 1, hi)


def step_dist(slab, ex, nsteps=1):
    """nsteps steps of a decomposition with one slab per rank."""
    for _ in range(nsteps):
        slab.stage(GHOST)
        exchange_dist(slab, ex, PHI)
        slab.stage(COLLIDE)
        exchange_dist(slab, ex, F)
        exchange_dist(slab, ex, UA)
        slab.stage(PHASE)
        slab.correct(ex.gather_partials(slab.partials()))
        exchange_dist(slab, ex, PHI)
