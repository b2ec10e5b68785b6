"""The 64-bit offset forms of the collide-stream and adjoint kernels, which
only grids with 27 N >= 2^31 nodes take by themselves, checked on small
grids by forcing them (CACL_OPT_INDEX64): the populations, phi, u and the
gradients they produce are bit-identical to the 32-bit forms. The step is
the pull collide-stream of Sect. 2.1 (Eqs. lbe .. lap_iso) and the adjoint
the reverse of one full step (Sect. 2.1 to 2.3); widening the offsets must
change no arithmetic."""
import numpy as np
import pytest

from paper_2607_25444_b300 import inputs as I

pytestmark = pytest.mark.gpu


def _case(storage, n):
    nx, ny, nz = n
    p = I.base_params(nx, ny, nz, sigma=0.01, rho_l=1.0, rho_g=0.2, nu_l=0.05,
                      nu_g=0.1, theta_deg=70.0, gravity=(0.0, 0.0, -1e-5),
                      storage=storage)
    solid = I.walls_z(nx, ny, nz)
    phi = I.droplet(nx, ny, nz, (nx / 2, ny / 2, 0.5), 6.5, p["width"])
    return p, solid, phi


def _run(p, solid, phi, lb_pipe, index64, steps):
    from paper_2607_25444_b300 import cacl
    s = cacl.Solver(p)
    s.set_geometry(solid)
    s.set_option(cacl.OPT_LB_PIPE, lb_pipe)
    s.set_option(cacl.OPT_INDEX64, index64)
    s.set_fields(phi)
    s.step(steps)
    out = [x.copy() for x in s.fields()] + [s.populations().copy()]
    s.close()
    return out


def _same(a, b):
    for x, y in zip(a, b):
        assert x.dtype == y.dtype and x.shape == y.shape
        assert np.array_equal(x.view(np.uint8), y.view(np.uint8))


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("n", [(32, 18, 14), (27, 13, 11)])
def test_one_node_kernel_index_widths_agree(storage, n):
    p, solid, phi = _case(storage, n)
    ref = _run(p, solid, phi, 2, 0, 17)      # one node per thread, 32-bit
    got = _run(p, solid, phi, 0, 1, 17)      # default pipeline forced to 64-bit
    _same(ref, got)


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_staged_kernel_index_widths_agree(storage):
    p, solid, phi = _case(storage, (32, 20, 12))
    ref = _run(p, solid, phi, 1, 0, 13)
    got = _run(p, solid, phi, 1, 1, 13)
    _same(ref, got)
    _same(ref, _run(p, solid, phi, 2, 0, 13))  # and the staged rows equal one node


def test_option_values_are_checked():
    from paper_2607_25444_b300 import cacl
    p, solid, _ = _case("f32", (16, 12, 10))
    s = cacl.Solver(p)
    s.set_geometry(solid)
    with pytest.raises(cacl.CaclError):
        s.set_option(cacl.OPT_INDEX64, 2)
    s.set_option(cacl.OPT_INDEX64, 1)
    s.set_option(cacl.OPT_INDEX64, 0)
    s.close()


def _grad(index64, outer):
    import torch

    from paper_2607_25444_b300 import cacl
    nx, ny, nz = 16, 16, 12
    p, solid, phi = _case("f32", (nx, ny, nz))
    s = cacl.Solver(p)
    s.set_geometry(solid)
    s.set_option(cacl.OPT_INDEX64, index64)
    wl = s.wall_list()
    idx = wl["idx"]
    theta = (55.0 + 50.0 * ((idx % nx) >= nx // 2)).astype(np.float32)
    s.set_fields(phi)
    s.set_wall_angles(theta)
    s.adjoint_forward(12, 2, outer)
    r = I.fast_uniform((nz, ny, nx), seed=77, lo=-1.0, hi=1.0)
    r[solid == 1] = 0.0
    g = torch.from_numpy(r.reshape(-1).astype(np.float32)).cuda()
    dth = torch.zeros(idx.size, dtype=torch.float64, device="cuda")
    dsg = torch.zeros(1, dtype=torch.float64, device="cuda")
    s.adjoint_backward(g, dth, dsg)
    torch.cuda.synchronize()
    out = (s.fields()[0].copy(), dth.cpu().numpy(), dsg.cpu().numpy())
    s.close()
    return out


@pytest.mark.parametrize("outer", [0, 6])
def test_adjoint_index_widths_agree(outer):
    ref = _grad(0, outer)
    got = _grad(1, outer)
    assert np.abs(ref[1]).max() > 0 and ref[2][0] != 0
    _same(ref, got)
