"""Checkpoint and resume (cacl_save_state / cacl_load_state): a context
restored from a saved state steps on bit for bit like the one it was saved
from, including the unbiased rounding of the volume correction (Sect. 2.3),
whose key is part of the state; and the failure-detection path of a copy
wait that gave up, exercised by setting its error word from the host and by
making the bounded wait itself run out on the GPU (no fault is made)."""
import numpy as np
import pytest

from paper_2607_25444_b300 import inputs as I

pytestmark = pytest.mark.gpu


def _case(storage, n=(28, 24, 20)):
    nx, ny, nz = n
    p = I.base_params(nx, ny, nz, sigma=0.01, rho_l=1.0, rho_g=0.2, nu_l=0.05,
                      nu_g=0.1, theta_deg=70.0, gravity=(0.0, 0.0, -1e-5),
                      storage=storage)
    solid = I.walls_z(nx, ny, nz)
    phi = I.droplet(nx, ny, nz, (nx / 2, ny / 2, 0.5), 7.0, p["width"])
    return p, solid, phi


def _solver(p, solid):
    from paper_2607_25444_b300 import cacl
    s = cacl.Solver(p)
    s.set_geometry(solid)
    return s


@pytest.mark.parametrize("storage", ["f32", "f16", "moments"])
def test_resume_is_bit_identical(storage):
    p, solid, phi = _case(storage)
    a = _solver(p, solid)
    idx = a.wall_list()["idx"]
    theta = (60.0 + 40.0 * ((idx % p["nx"]) >= p["nx"] // 2)).astype(np.float32)
    a.set_fields(phi)
    a.set_wall_angles(theta)
    a.step(30)
    state = a.save_state()
    a.step(25)
    b = _solver(p, solid)
    b.load_state(state)
    b.step(25)
    for x, y in zip(a.fields(), b.fields()):
        assert np.array_equal(x.view(np.uint32), y.view(np.uint32))
    assert np.array_equal(a.populations(), b.populations())
    ma, mb = a.mass(), b.mass()
    assert ma == mb, (ma, mb)
    a.close()
    b.close()


def test_load_rejects_foreign_states():
    from paper_2607_25444_b300 import cacl
    p, solid, phi = _case("f32")
    a = _solver(p, solid)
    a.set_fields(phi)
    a.step(3)
    state = a.save_state()
    q, solid2, _ = _case("f32", (28, 24, 24))
    b = _solver(q, solid2)
    with pytest.raises(cacl.CaclError):
        b.load_state(state)  # another grid
    c = _solver(dict(p, storage="f16"), solid)
    with pytest.raises(cacl.CaclError):
        c.load_state(state)  # another storage
    d = _solver(p, solid)
    with pytest.raises(cacl.CaclError):
        d.load_state(b"\0" * len(state))  # not a saved state
    with pytest.raises(cacl.CaclError):
        d.load_state(state[:100])  # truncated
    d.load_state(state)
    for s in (a, b, c, d):
        s.close()


def test_injected_wait_timeout_is_reported():
    from paper_2607_25444_b300 import cacl
    p, solid, phi = _case("f32")
    s = _solver(p, solid)
    s.set_fields(phi)
    s.step(2)
    s.check_finite()
    s.inject_wait_timeout()
    with pytest.raises(cacl.CaclError) as e:
        s.check_finite()
    assert e.value.status == -6  # CACL_ERR_TIMEOUT
    s.close()


@pytest.mark.parametrize("pipe", [1, 3])
def test_copy_wait_runs_out_and_is_reported(pipe):
    """The bounded wait of the copy-staged (pipeline 1) and TMA-tiled
    (pipeline 3) collide-stream made to run out (each block registers 16
    bytes more than its first copies deliver): the step ends after the
    wait's 0.5-s limit, cacl_check_finite reports CACL_ERR_TIMEOUT, and the
    device stays usable: a new context with the same pipeline steps bit for
    bit like the default pipeline."""
    import time
    from paper_2607_25444_b300 import cacl
    p, solid, phi = _case("f32", n=(32, 16, 12))
    s = _solver(p, solid)
    s.set_option(cacl.OPT_LB_PIPE, pipe)
    s.set_fields(phi)
    s.step(2)
    s.check_finite()
    s.fields()
    s.inject_copy_stall(True)
    t0 = time.perf_counter()
    s.step(1)
    s.fields()  # waits for the step
    dt = time.perf_counter() - t0
    with pytest.raises(cacl.CaclError) as e:
        s.check_finite()
    assert e.value.status == -6  # CACL_ERR_TIMEOUT
    assert 0.45 < dt < 30.0, dt
    s.inject_copy_stall(False)
    s.close()

    a = _solver(p, solid)
    a.set_option(cacl.OPT_LB_PIPE, pipe)
    a.set_fields(phi)
    a.step(3)
    a.check_finite()
    b = _solver(p, solid)
    b.set_fields(phi)
    b.step(3)
    fluid = solid == 0
    (pa, ua, _), (pb, ub, _) = a.fields(), b.fields()
    assert np.array_equal(pa[fluid], pb[fluid])
    assert np.array_equal(ua[:, fluid], ub[:, fluid])
    a.close()
    b.close()
