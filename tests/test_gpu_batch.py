"""Batched stepping: cases of uneven size, parameters and geometry advanced
together give, bit for bit, what each case gives on its own, and one case
matches the oracle."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2607_25444_b300 import inputs as I

pytestmark = pytest.mark.gpu


def _cases(storage="f32"):
    out = []
    # spreading-like, density ratio 10
    n = (26, 22, 18)
    p = I.base_params(*n, sigma=0.01, rho_g=0.1, nu_g=0.1, theta_deg=50.0,
                      storage=storage)
    out.append((p, I.walls_z(*n), I.droplet(*n, (13, 11, 0.5), 7.0, 4.0), None))
    # ragged sizes, hydrophobic, gravity
    n = (37, 13, 11)
    p = I.base_params(*n, sigma=0.02, rho_g=0.5, theta_deg=140.0,
                      gravity=(0.0, 0.0, -1e-5), storage=storage)
    out.append((p, I.walls_z(*n), I.droplet(*n, (18, 6, 3.5), 4.0, 4.0), None))
    # impact: initial downward velocity inside the drop
    n = (40, 40, 32)
    p = I.base_params(*n, sigma=0.003, rho_g=0.01, nu_l=0.03, nu_g=0.03,
                      theta_deg=150.0, storage=storage)
    phi = I.droplet(*n, (20, 20, 9.5), 8.0, 4.0)
    u = np.zeros((3,) + phi.shape, np.float32)
    u[2] = np.where(phi > 0.5, -0.04, 0.0)
    out.append((p, I.walls_z(*n), phi, u))
    # orifice plate
    n = (24, 24, 40)
    p = I.base_params(*n, sigma=0.01, rho_g=0.02, theta_deg=60.0,
                      gravity=(0.0, 0.0, -2e-5), storage=storage)
    out.append((p, I.orifice_plate(*n, 16, 4, 8), I.droplet(*n, (12, 12, 28), 6.0, 4.0), None))
    return out


@pytest.mark.parametrize("storage", ["f32", "f16"])
@pytest.mark.parametrize("lb_variant,phase_variant", [(1, 0), (0, 2), (2, 3), (4, 1)])
def test_batch_equals_cases_alone(storage, lb_variant, phase_variant):
    from paper_2607_25444_b300 import cacl
    cases = _cases(storage)
    b = cacl.Batch([c[0] for c in cases])
    b.set_option(lb_variant, phase_variant)
    for view, (p, solid, phi, u) in zip(b.cases, cases):
        view.set_geometry(solid)
        view.set_fields(phi, u)
    b.step(15)
    for view, (p, solid, phi, u) in zip(b.cases, cases):
        s = cacl.Solver(p)
        s.set_option(cacl.OPT_PHASE_TILE, phase_variant)
        s.set_geometry(solid)
        s.set_fields(phi, u)
        s.step(15)
        a, bb = view.fields(), s.fields()
        for x, y in zip(a, bb):
            assert np.array_equal(x, y)
        assert view.mass()["lam"] == s.mass()["lam"]
        s.close()
    b.close()


def test_batch_case_matches_oracle():
    from paper_2607_25444_b300 import cacl
    cases = _cases()
    b = cacl.Batch([c[0] for c in cases])
    for view, (p, solid, phi, u) in zip(b.cases, cases):
        view.set_geometry(solid)
        view.set_fields(phi, u)
    b.step(1)
    p, solid, phi, u = cases[2]
    o = O.Oracle(p)
    o.set_geometry(solid)
    o.set_fields(phi.astype(np.float64), u.astype(np.float64))
    o.step(1)
    g, r = b.cases[2].fields(), o.fields()
    for x, y in zip(g, r):
        assert np.abs(x - y).max() / np.abs(y).max() < 1e-5
    b.close()


def test_autotune_and_lockstep():
    from paper_2607_25444_b300 import cacl
    cases = _cases()
    b = cacl.Batch([c[0] for c in cases])
    for view, (p, solid, phi, u) in zip(b.cases, cases):
        view.set_geometry(solid)
        view.set_fields(phi, u)
    best = b.autotune(steps=2)
    assert 0 <= best["lb_variant"] < 6 and 0 <= best["phase_variant"] < 4
    assert best["ms_per_step"] > 0
    b.step(2)
    for view in b.cases:
        view.check_finite()
    b.cases[1].step(1)  # one case alone breaks the lockstep
    with pytest.raises(cacl.CaclError):
        b.step(1)
    b.close()


def test_sweep_cases_batch_equals_alone():
    """Six cases of the batched impact sweep (edges 69, 70, 78, 80, 87 and
    96: every collide-stream width and phi-update pipeline, FP16 storage,
    the drop moving toward the wall) after 10 steps: the batch, with its
    width classes as concurrent branches, gives bit for bit what each case
    gives alone."""
    import sys

    sys.path.insert(0, __file__.rsplit("/tests/", 1)[0])
    import bench
    from paper_2607_25444_b300 import cacl
    cases = bench.impact_sweep_cases(pick=[8, 47, 11, 5, 23, 28])
    assert sorted(c[0]["nx"] % 4 for c in cases) == [0, 0, 1, 2, 2, 3]
    b = cacl.Batch([c[0] for c in cases])
    b.set_option(1, 2)
    for view, (p, solid, phi, u) in zip(b.cases, cases):
        view.set_geometry(solid)
        view.set_fields(phi, u)
    b.step(10)
    for view, (p, solid, phi, u) in zip(b.cases, cases):
        s = cacl.Solver(p)
        s.set_option(cacl.OPT_PHASE_TILE, 2)
        s.set_geometry(solid)
        s.set_fields(phi, u)
        s.step(10)
        for x, y in zip(view.fields(), s.fields()):
            assert np.array_equal(x, y)
        assert np.array_equal(view.populations(), s.populations())
        assert view.mass()["lam"] == s.mass()["lam"]
        s.close()
    b.close()
