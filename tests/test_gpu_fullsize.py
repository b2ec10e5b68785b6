"""Parity at the benchmark's full size (256^3 static droplet, the launch
configuration bench.py times; FP32, FP16 and BF16 population storage) and at
432^3, where 27 N exceeds 2^31 and the collide-stream runs its 64-bit-offset
kernel: one step of the GPU state after 100 steps is
compared, node by node, with the oracle stepping 14^3 windows cut from that
state around sampled nodes (bulk, interface, contact line); the interior of
each window beyond the reach of one step (5 nodes) is checked. The global
volume correction is checked against FP64 sums over the whole field."""
import numpy as np
import pytest

from oracle import oracle as O

pytestmark = pytest.mark.gpu

WIN = 14
REACH = 5  # ghosts (2) + collide-stream (1) + phi update (2)


def _window_idx(lo, n, size=WIN):
    return (np.arange(lo, lo + size) % n).astype(np.int64)


# stored f* of 16-bit storage: half an ulp of the format, relative to the
# largest population (as in the small-grid collide parity)
F_TOL = {"f32": 1e-5, "f16": 6e-4, "bf16": 4.5e-3}


@pytest.mark.parametrize("n,storage", [(256, "f32"), (432, "f32"), (256, "f16"),
                                       (256, "bf16")])
def test_fullsize_one_step_windows(n, storage):
    import sys

    import torch

    sys.path.insert(0, __file__.rsplit("/tests/", 1)[0])
    import bench
    from paper_2607_25444_b300 import cacl
    p, solid, phi = bench.workload(n)
    p["storage"] = storage
    s = cacl.Solver(p)
    s.set_geometry(solid)
    s.set_fields(phi)
    s.step(100)
    N = n ** 3
    f0 = torch.empty(27 * N, dtype=torch.float32, device="cuda")
    s.L.cacl_get_populations(s.h, cacl.C.c_void_p(f0.data_ptr()), 1)
    ph0 = torch.empty(N, dtype=torch.float32, device="cuda")
    s.fields_device(phi=ph0)
    s.ghost_update()
    s.lb_collide()
    s.phase_update()
    phs = torch.empty(N, dtype=torch.float32, device="cuda")
    u1 = torch.empty(3 * N, dtype=torch.float32, device="cuda")
    s.fields_device(phi=phs, u=u1)
    f1 = torch.empty(27 * N, dtype=torch.float32, device="cuda")
    s.L.cacl_get_populations(s.h, cacl.C.c_void_p(f1.data_ptr()), 1)
    s.volume_correct()
    ph1 = torch.empty(N, dtype=torch.float32, device="cuda")
    s.fields_device(phi=ph1)
    torch.cuda.synchronize()
    mass = s.mass()

    f0 = f0.view(27, n, n, n)
    f1 = f1.view(27, n, n, n)
    ph0v, phsv, u1v = ph0.view(n, n, n), phs.view(n, n, n), u1.view(3, n, n, n)

    # sampled window origins (z0, y0, x0): contact line, interface, bulk
    sc = lambda v: int(round(v * n / 256))
    c, R = n // 2, sc(40)
    origins = [(0, c - 7, c + R - 7), (0, c - 7, c - R - 7),
               (0, c + sc(28) - 7, c + sc(28) - 7), (sc(20), c + sc(22) - 7, c - 7),
               (sc(30), sc(100), sc(100)), (sc(120), sc(10), sc(200)),
               (n - 16, sc(50), sc(60)), (0, 0, 0)]
    worst = dict(phi=0.0, u=0.0, f=0.0)
    for (z0, y0, x0) in origins:
        zi, yi, xi = _window_idx(z0, n), _window_idx(y0, n), _window_idx(x0, n)
        ix = np.ix_(zi, yi, xi)
        wsolid = solid[ix].copy()
        at_wall = z0 == 0
        if at_wall:
            wsolid[-1] = 1  # close the window on top; the bottom is the wall
        params = dict(p, nx=WIN, ny=WIN, nz=WIN,
                      periodic=(1, 1, 0) if at_wall else (1, 1, 1))
        o = O.Oracle(params)
        o.set_geometry(wsolid)
        tz, ty, tx = (torch.from_numpy(a).cuda() for a in (zi, yi, xi))
        sel = lambda t: t[..., tz[:, None, None], ty[None, :, None], tx[None, None, :]]
        o.set_fields(sel(ph0v).double().cpu().numpy())
        o.set_populations(sel(f0).double().cpu().numpy())
        o.ghost_update()
        o.lb_collide()
        o.phase_update()
        rp, ru, _ = o.fields()
        rf = o.populations()
        gp = sel(phsv).double().cpu().numpy()
        gu = sel(u1v).double().cpu().numpy()
        gf = sel(f1).double().cpu().numpy()
        lo, hi = REACH, WIN - REACH
        zl, zh = (0, WIN - 1 - REACH) if at_wall else (lo, hi)
        core = (slice(zl, zh), slice(lo, hi), slice(lo, hi))
        fl = wsolid[core] == 0
        e_phi = np.abs(gp[core] - rp[core])[fl].max() / max(np.abs(rp[core]).max(), 1e-3)
        e_u = np.abs(gu[(slice(None),) + core] - ru[(slice(None),) + core]).max() / \
            max(np.abs(ru[(slice(None),) + core]).max(), 1e-6)
        e_f = np.abs((gf - rf)[(slice(None),) + core][:, fl]).max() / \
            max(np.abs(rf[(slice(None),) + core][:, fl]).max(), 1e-9)
        worst = {k: max(worst[k], v) for k, v in
                 dict(phi=e_phi, u=e_u, f=e_f).items()}
    print(f"full-size window parity at {n}^3, {storage}", worst)
    assert worst["phi"] < 1e-5 and worst["u"] < 1e-4 and worst["f"] < F_TOL[storage], worst

    # the volume correction: lambda from FP64 sums of the whole phi*
    fluid = torch.from_numpy((solid == 0).reshape(-1)).cuda()
    v = phs.double()
    eps = p["eps_phi"]
    chi = torch.where((v > eps) & (v < 1 - eps), v * (1 - v), torch.zeros_like(v))
    m_star = v[fluid].sum().item()
    w_sum = chi[fluid].sum().item()
    lam = (mass["m_ref"] - m_star) / w_sum
    assert abs(m_star - mass["m_star"]) < 1e-9 * m_star
    assert abs(w_sum - mass["w_sum"]) < 1e-9 * w_sum
    assert abs(lam - mass["lam"]) < 1e-6 * abs(lam) + 1e-15
    expect = torch.where(fluid, (v + lam * chi).float(), phs)
    assert (ph1 - expect).abs().max().item() < 1e-6
    s.close()
