"""Each stage of the GPU adjoint on its own (cacl_adjoint_stage) against the
FP64 restatement of the step (oracle/torch_step.py) at the same
linearisation point: element by element against its reverse mode
(vector-Jacobian products; measured 1e-7 to 3e-7 of the largest entry, the
FP32 rounding of the kernels), and the dot-product identity
<J v, w> = <v, J^T w> with J v from its forward mode. The stages are the
volume correction (Sect. 2.3, Eqs. mass_corrected_phi and
mass_correction_normalization), the phi update with the compressive vector
as an input (Sect. 2.1.1, Eq. phi_update_muscl), the collide-stream with the
compressive vector and the next step's pull (Sect. 2.1, Eqs. lbe .. lap_iso)
and the ghost map (Sect. 2.2)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2607_25444_b300 import inputs as I

pytestmark = pytest.mark.gpu

NX, NY, NZ = 16, 16, 12
N = NX * NY * NZ
SH = (NZ, NY, NX)


def _case():
    p = I.base_params(NX, NY, NZ, sigma=0.01, rho_l=1.0, rho_g=0.5,
                      nu_l=0.05, nu_g=0.1, theta_deg=80.0,
                      gravity=(0.0, 0.0, -1e-5))
    solid = I.walls_z(NX, NY, NZ)
    phi = I.droplet(NX, NY, NZ, (8.0, 8.0, 0.5), 5.0, p["width"])
    z, y, x = np.meshgrid(np.arange(NZ), np.arange(NY), np.arange(NX), indexing="ij")
    patch = (x >= NX // 2).astype(int) + 2 * (y >= NY // 2).astype(int)
    theta = np.array([55.0, 75.0, 105.0, 125.0])[patch].astype(np.float32)
    return p, solid, phi, theta


@pytest.fixture(scope="module")
def lin():
    """A GPU context six steps into the case (moving interface, developed
    velocity), a one-step one-level forward from there, and the
    restatement on the same geometry with the GPU's linearisation point."""
    import torch

    from oracle import torch_step as TS
    from paper_2607_25444_b300 import cacl
    p, solid, phi, theta = _case()
    s = cacl.Solver(p)
    s.set_geometry(solid)
    wl = s.wall_list()
    th_w = theta.reshape(-1)[wl["idx"]]
    s.set_fields(phi)
    s.set_wall_angles(th_w)
    s.step(6)
    s.adjoint_forward(1, 1)
    state = torch.zeros(36 * N, dtype=torch.float32, device="cuda")
    dummy_in = torch.zeros(N, dtype=torch.float32, device="cuda")
    dummy_out = torch.zeros(N, dtype=torch.float32, device="cuda")
    s.adjoint_stage(cacl.ADJ_CORRECT, dummy_in, dummy_out, state=state)
    st = state.cpu().numpy().astype(np.float64)
    o = O.Oracle(p)
    o.set_geometry(solid)
    ts = TS.TorchStep(p, solid, o.wall_list(), frozen_bulk_normal=True)
    assert np.array_equal(o.wall_list()["idx"], wl["idx"])
    off = np.cumsum([0, N, 27 * N, N, 3 * N, 3 * N, N])
    parts = [st[off[i]:off[i + 1]] for i in range(6)]
    T = lambda a, shape: torch.tensor(a.reshape(shape), dtype=torch.float64)
    return dict(s=s, ts=ts, solid=solid.astype(bool), W=wl["idx"].size,
                phi=T(parts[0], SH), f=T(parts[1], (27,) + SH), phig=T(parts[2], SH),
                u=T(parts[3], (3,) + SH), a=T(parts[4], (3,) + SH),
                phis=T(parts[5], SH), m_ref=float(s.mass()["m_ref"]),
                theta=torch.tensor(th_w.astype(np.float64)),
                sigma=torch.tensor(p["sigma"], dtype=torch.float64))


def _rand(shape, seed):
    return I.fast_uniform(shape, seed=seed, lo=-1.0, hi=1.0).astype(np.float64)


def _gpu_stage(lin, stage, cot, nout, nparam=0):
    import torch
    cin = torch.from_numpy(np.ascontiguousarray(cot).reshape(-1).astype(np.float32)).cuda()
    out = torch.zeros(nout, dtype=torch.float32, device="cuda")
    dp = torch.zeros(max(nparam, 1), dtype=torch.float64, device="cuda")
    lin["s"].adjoint_stage(stage, cin, out, dparam=dp if nparam else None)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64), dp.cpu().numpy()[:nparam]


def _vjp(fn, xs, w):
    """Reverse mode of the restatement: J^T w for inputs xs (tensors)."""
    import torch
    xs = [x.clone().requires_grad_(True) for x in xs]
    ys = fn(*xs)
    ys = ys if isinstance(ys, tuple) else (ys,)
    dot = sum((y * torch.as_tensor(wi, dtype=torch.float64)).sum() for y, wi in zip(ys, w))
    grads = torch.autograd.grad(dot, xs, allow_unused=True)
    return [np.zeros(tuple(x.shape)) if g is None else g.numpy() for x, g in zip(xs, grads)]


def _jvp(fn, xs, vs):
    """Forward mode of the restatement: J v."""
    import torch
    _, jv = torch.func.jvp(fn, tuple(xs), tuple(torch.as_tensor(v, dtype=torch.float64)
                                                 for v in vs))
    jv = jv if isinstance(jv, tuple) else (jv,)
    return [j.detach().numpy() for j in jv]


def _close(got, ref, tol):
    scale = np.abs(ref).max()
    err = np.abs(got - ref).max() / scale
    assert err < tol, err
    return err


def _dot_identity(jv, w, v, gpu, tol):
    lhs = sum(float((a * b).sum()) for a, b in zip(jv, w))
    rhs = sum(float((a * b).sum()) for a, b in zip(v, gpu))
    assert abs(lhs - rhs) <= tol * max(abs(lhs), 1e-30), (lhs, rhs)


def test_correction_stage(lin):
    from paper_2607_25444_b300 import cacl
    ts, m_ref = lin["ts"], lin["m_ref"]
    w = _rand(SH, 101)
    got, _ = _gpu_stage(lin, cacl.ADJ_CORRECT, w, N)
    fn = lambda ps: ts.correct(ps, m_ref)
    (ref,) = _vjp(fn, [lin["phis"]], [w])
    err = _close(got.reshape(SH), ref, 3e-6)
    v = _rand(SH, 102)
    _dot_identity(_jvp(fn, [lin["phis"]], [v]), [w], [v], [got.reshape(SH)], 1e-5)
    print(f"correction: max rel err {err:.2e}")


def test_phase_stage(lin):
    from paper_2607_25444_b300 import cacl
    ts = lin["ts"]
    w = _rand(SH, 111)
    got, _ = _gpu_stage(lin, cacl.ADJ_PHASE, w, 7 * N)
    g_phi, g_u, g_a = got[:N].reshape(SH), got[N:4 * N].reshape((3,) + SH), \
        got[4 * N:].reshape((3,) + SH)
    fn = lambda ph, u, a: ts.phase(ph, u, a)
    xs = [lin["phig"], lin["u"], lin["a"]]
    r_phi, r_u, r_a = _vjp(fn, xs, [w])
    errs = [_close(g_phi, r_phi, 3e-6), _close(g_u, r_u, 3e-6), _close(g_a, r_a, 3e-6)]
    vs = [_rand(SH, 112), _rand((3,) + SH, 113) * 0.01, _rand((3,) + SH, 114) * 0.01]
    _dot_identity(_jvp(fn, xs, vs), [w], vs, [g_phi, g_u, g_a], 1e-5)
    print("phase: max rel err phi_g %.2e u %.2e a %.2e" % tuple(errs))


def test_collide_stage(lin):
    import torch

    from paper_2607_25444_b300 import cacl
    ts, solid = lin["ts"], lin["solid"]
    fluid = ~solid
    w_f = _rand((27,) + SH, 121) * fluid
    w_u = _rand((3,) + SH, 122) * fluid
    w_a = _rand((3,) + SH, 123) * fluid
    cot = np.concatenate([w_f.reshape(-1), w_u.reshape(-1), w_a.reshape(-1)])
    got, dsig = _gpu_stage(lin, cacl.ADJ_COLLIDE, cot, 28 * N, 1)
    g_fin = got[:27 * N].reshape((27,) + SH)
    g_phi = got[27 * N:].reshape(SH)
    sol = torch.tensor(solid)

    def fn(fin, ph, sg):
        fout, u = ts.collide_pulled(fin, ph, sg)
        fout = torch.where(sol, torch.zeros_like(fout), fout)
        return ts.pull(fout), u, ts.compressive(ph)

    fin0 = ts.pull(lin["f"]).detach()
    xs = [fin0, lin["phig"], lin["sigma"]]
    r_fin, r_phi, r_sig = _vjp(fn, xs, [w_f, w_u, w_a])
    e_f = _close(g_fin * fluid, r_fin * fluid, 5e-6)
    e_p = _close(g_phi, r_phi, 5e-6)
    e_s = abs(dsig[0] - float(r_sig)) / abs(float(r_sig))
    assert e_s < 1e-6, (dsig[0], float(r_sig))
    vs = [_rand((27,) + SH, 124) * fluid * 1e-3, _rand(SH, 125) * 1e-3, np.array(1e-3)]
    jv = _jvp(fn, xs, vs)
    _dot_identity(jv, [w_f, w_u, w_a], vs, [g_fin * fluid, g_phi, dsig[0]], 1e-4)
    print(f"collide: max rel err f_in {e_f:.2e} phi_g {e_p:.2e} sigma {e_s:.2e}")


def test_ghost_stage(lin):
    from paper_2607_25444_b300 import cacl
    ts = lin["ts"]
    w = _rand(SH, 131)
    got, dth = _gpu_stage(lin, cacl.ADJ_GHOST, w, N, lin["W"])
    fn = lambda ph, th: ts.ghost(ph, th)
    xs = [lin["phi"], lin["theta"]]
    r_phi, r_th = _vjp(fn, xs, [w])
    e_p = _close(got.reshape(SH), r_phi, 3e-6)
    e_t = _close(dth, r_th, 3e-6)
    vs = [_rand(SH, 132), _rand((lin["W"],), 133)]
    _dot_identity(_jvp(fn, xs, vs), [w], vs, [got.reshape(SH), dth], 1e-5)
    print(f"ghost: max rel err phi {e_p:.2e} theta {e_t:.2e}")
