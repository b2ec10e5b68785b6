"""The allocation-free volume correction (cacl_volume_correct_noalloc)
gives the context's correction, on two calls in a row.

Callers that cannot allocate device memory (their memory belongs to another
allocator's pool, or allocation is forbidden once they serve) use this entry
point; its scratch is a fixed array inside the library. This file is
collected last so that a run stopping at the first failure has already run
every other test."""
import ctypes

import numpy as np
import pytest

from paper_2607_25444_b300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-5  # the one-step field tolerance of the parity tests


def test_noalloc_correction_matches_context_path():
    import torch

    from paper_2607_25444_b300 import cacl
    nx, ny, nz = 40, 36, 30
    p = I.base_params(nx, ny, nz, sigma=0.01, rho_g=0.2, nu_g=0.1,
                      theta_deg=45.0)
    solid = I.walls_z(nx, ny, nz)
    phi = I.droplet(nx, ny, nz, (20, 18, 0.5), 9.0, p["width"])
    s = cacl.Solver(p)
    s.set_geometry(solid)
    s.set_fields(phi)
    m_ref = s.mass()["m_ref"]
    dphi = torch.empty(phi.size, dtype=torch.float32, device="cuda")
    dsolid = torch.from_numpy(solid.reshape(-1).copy()).cuda()
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    for _ in range(2):
        s.ghost_update()
        s.lb_collide()
        s.phase_update()
        s.fields_device(phi=dphi)  # phi* before the context's correction
        s.volume_correct()
        ref = s.fields()[0]
        ref_mass = s.mass()
        cacl.volume_correct_noalloc(dphi, dsolid, m_ref, p["eps_phi"], out)
        torch.cuda.synchronize()
        got = dphi.cpu().numpy().reshape(ref.shape)
        assert np.abs(got - ref).max() / np.abs(ref).max() < TOL
        m_star, w_sum, lam = out.cpu().numpy()
        assert abs(m_star - ref_mass["m_star"]) < 1e-9 * ref_mass["m_star"]
        assert abs(w_sum - ref_mass["w_sum"]) < 1e-9 * ref_mass["w_sum"]
        assert abs(lam - ref_mass["lam"]) < 1e-5 * abs(ref_mass["lam"]) + 1e-15
    s.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch

    from paper_2607_25444_b300 import cacl
    L = cacl.load()
    buf = torch.zeros(16, dtype=torch.float32, device="cuda")
    sol = torch.zeros(16, dtype=torch.uint8, device="cuda")
    too_many = 4096 * 16384 + 1  # rejected before anything is enqueued
    rc = L.cacl_volume_correct_noalloc(ctypes.c_void_p(buf.data_ptr()),
                                       ctypes.c_void_p(sol.data_ptr()),
                                       too_many, 1.0, 1e-3, None, None)
    assert cacl.STATUS[rc] == "CACL_ERR_TOO_LARGE"


def test_noalloc_holds_mass_over_repeated_calls():
    """A mass target a few parts in 1e9 away from the field's mass needs
    corrections below the FP32 resolution of phi in the bulk of the band;
    the unbiased rounding applies them on average, so over hundreds of
    calls the post-correction mass stays at the target (Sect. 2.3) instead
    of keeping the defect."""
    import torch

    from paper_2607_25444_b300 import cacl
    n = 48
    solid = I.walls_z(n, n, n)
    phi = I.droplet(n, n, n, (24, 24, 0.5), 12.0, 4.0)
    fluid = solid.reshape(-1) == 0
    m0 = float(phi.reshape(-1)[fluid].astype(np.float64).sum())
    m_ref = m0 * (1.0 + 3e-9)
    dphi = torch.from_numpy(phi.reshape(-1).copy()).cuda()
    dsolid = torch.from_numpy(solid.reshape(-1).copy()).cuda()
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    pre = []
    for _ in range(300):
        cacl.volume_correct_noalloc(dphi, dsolid, m_ref, 1e-3, out)
        pre.append(float(out[0].item()))  # mass before this call's update
    rel = (np.array(pre[100:]) - m_ref) / m_ref
    assert abs(rel.mean()) < 3e-10, rel.mean()
    assert np.abs(rel).max() < 2e-9, np.abs(rel).max()
    final = float(dphi.cpu().numpy()[fluid].astype(np.float64).sum())
    assert abs(final - m_ref) / m_ref < 2e-9


def test_noalloc_sums_at_192_cube():
    """More partial blocks than the finalize kernel has threads (1729 at
    192^3): M*, W and lambda against FP64 sums of the same field on the
    host."""
    import torch

    from paper_2607_25444_b300 import cacl
    n = 192
    solid = I.walls_z(n, n, n)
    phi = I.droplet(n, n, n, (96, 96, 0.5), 40.0, 4.0)
    flat = phi.reshape(-1)
    fluid = solid.reshape(-1) == 0
    v = flat[fluid]
    eps = np.float32(1e-3)
    chi = np.where((v > eps) & (v < np.float32(1.0) - eps),
                   v * (np.float32(1.0) - v), np.float32(0.0))
    m_star = float(v.astype(np.float64).sum())
    w_sum = float(chi.astype(np.float64).sum())
    m_ref = m_star * (1.0 + 1e-6)
    lam = (m_ref - m_star) / w_sum
    dphi = torch.from_numpy(flat.copy()).cuda()
    dsolid = torch.from_numpy(solid.reshape(-1).copy()).cuda()
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    cacl.volume_correct_noalloc(dphi, dsolid, m_ref, 1e-3, out)
    got = out.cpu().numpy()
    assert abs(got[0] - m_star) <= 1e-12 * m_star
    assert abs(got[1] - w_sum) <= 1e-12 * w_sum
    assert abs(got[2] - lam) <= 1e-6 * abs(lam)
    after = float(dphi.cpu().numpy()[fluid].astype(np.float64).sum())
    assert abs(after - m_ref) / m_ref < 1e-9


def test_noalloc_binding_rejects_wrong_dtypes():
    import torch

    from paper_2607_25444_b300 import cacl
    phi = torch.zeros(64, dtype=torch.float32, device="cuda")
    sol = torch.zeros(64, dtype=torch.uint8, device="cuda")
    with pytest.raises(ValueError):
        cacl.volume_correct_noalloc(phi, sol, 1.0, 1e-3,
                                    torch.zeros(3, dtype=torch.float32, device="cuda"))
    with pytest.raises(ValueError):
        cacl.volume_correct_noalloc(phi, sol, 1.0, 1e-3,
                                    torch.zeros(2, dtype=torch.float64, device="cuda"))
    with pytest.raises(ValueError):
        cacl.volume_correct_noalloc(phi.double(), sol, 1.0)
    with pytest.raises(ValueError):
        cacl.volume_correct_noalloc(phi, sol.to(torch.int32), 1.0)
