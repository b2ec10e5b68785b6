"""Pins of the FP64 CPU adjoint (oracle/torch_step.py), the reference of
the GPU adjoint: its forward equals the C++ oracle's step, and its reverse
mode (autograd) equals central differences of the C++ oracle for dL/dtheta
and dL/dsigma (Sect. 2.2, Eqs. tangential_gradient_contact_angle ..
ghost_contact_angle_extrapolation; Sect. 2.1, Eq. Fcap)."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from oracle import torch_step as TS
from paper_2607_25444_b300 import inputs as I

NX, NY, NZ = 12, 12, 10


def _case():
    p = I.base_params(NX, NY, NZ, sigma=0.01, rho_l=1.0, rho_g=0.5,
                      nu_l=0.05, nu_g=0.1, theta_deg=80.0,
                      gravity=(0.0, 0.0, -1e-5))
    solid = I.walls_z(NX, NY, NZ)
    phi = I.droplet(NX, NY, NZ, (6.0, 6.0, 0.5), 4.0, p["width"]).astype(np.float64)
    z, y, x = np.meshgrid(np.arange(NZ), np.arange(NY), np.arange(NX), indexing="ij")
    patch = (x >= NX // 2).astype(int) + 2 * (y >= NY // 2).astype(int)
    theta = np.array([55.0, 75.0, 105.0, 125.0])[patch]
    r = I.fast_uniform((NZ, NY, NX), seed=31, lo=-1.0, hi=1.0).astype(np.float64)
    r[solid == 1] = 0.0
    return p, solid, phi, theta, patch, r


def _oracle(p, solid, phi, theta, steps):
    o = O.Oracle(p)
    o.set_geometry(solid)
    o.set_contact_angle(theta)
    o.set_fields(phi)
    o.step(steps)
    return o


def test_torch_step_matches_cpp_oracle():
    """Five steps of the whole-field FP64 restatement reproduce the C++
    oracle's phi, u and populations to round-off (density ratio 2, gravity,
    four contact angles on the walls)."""
    p, solid, phi, theta, patch, r = _case()
    o0 = O.Oracle(p)
    o0.set_geometry(solid)
    wall = o0.wall_list()
    ts = TS.TorchStep(p, solid, wall)
    th = torch.tensor(theta.reshape(-1)[wall["idx"]])
    f, ph, u = ts.rollout(phi, th, torch.tensor(p["sigma"], dtype=torch.float64), 5)
    o = _oracle(p, solid, phi, theta, 5)
    rphi, ru, _ = o.fields()
    rf = o.populations()
    fluid = solid == 0
    assert np.abs(ph.numpy() - rphi).max() < 1e-12
    assert np.abs(u.numpy()[:, fluid] - ru[:, fluid]).max() < 1e-14
    assert np.abs(f.numpy()[:, fluid] - rf[:, fluid]).max() < 1e-14


def test_torch_adjoint_matches_oracle_central_differences():
    """Reverse mode of the FP64 restatement (exact derivative, no frozen
    normal) against central differences of the C++ oracle over 12 steps:
    dL/dtheta summed over each of the four wall patches and dL/dsigma,
    L = sum r phi. h = 1e-3 deg and 1e-5 sigma; agreement to 1e-6
    relative."""
    steps = 12
    p, solid, phi, theta, patch, r = _case()
    o0 = O.Oracle(p)
    o0.set_geometry(solid)
    wall = o0.wall_list()
    ts = TS.TorchStep(p, solid, wall)
    th = torch.tensor(theta.reshape(-1)[wall["idx"]], requires_grad=True)
    sg = torch.tensor(p["sigma"], dtype=torch.float64, requires_grad=True)
    _, ph, _ = ts.rollout(phi, th, sg, steps)
    L = (ph * torch.tensor(r)).sum()
    L.backward()
    dth = th.grad.numpy()
    wpatch = patch.reshape(-1)[wall["idx"]]

    def loss(theta_field, sigma):
        o = _oracle(dict(p, sigma=sigma), solid, phi, theta_field, steps)
        return float((o.fields()[0] * r).sum())

    h = 1e-3
    for k in range(4):
        tp, tm = theta.copy(), theta.copy()
        tp[patch == k] += h
        tm[patch == k] -= h
        fd = (loss(tp, p["sigma"]) - loss(tm, p["sigma"])) / (2 * h)
        ad = dth[wpatch == k].sum()
        assert abs(ad - fd) <= 1e-6 * abs(fd) + 1e-12, (k, ad, fd)
    hs = 1e-5 * p["sigma"]
    fd = (loss(theta, p["sigma"] + hs) - loss(theta, p["sigma"] - hs)) / (2 * hs)
    assert abs(sg.grad.item() - fd) <= 1e-6 * abs(fd), (sg.grad.item(), fd)


def test_frozen_bulk_normal_is_a_small_departure():
    """The rule the GPU adjoint applies (normal of the compressive vector
    held fixed outside the interface band) changes the short-horizon
    gradient by well under 1 % here."""
    p, solid, phi, theta, patch, r = _case()
    o0 = O.Oracle(p)
    o0.set_geometry(solid)
    wall = o0.wall_list()
    grads = []
    for frozen in (False, True):
        ts = TS.TorchStep(p, solid, wall, frozen_bulk_normal=frozen)
        th = torch.tensor(theta.reshape(-1)[wall["idx"]], requires_grad=True)
        sg = torch.tensor(p["sigma"], dtype=torch.float64, requires_grad=True)
        _, ph, _ = ts.rollout(phi, th, sg, 12)
        (ph * torch.tensor(r)).sum().backward()
        grads.append((th.grad.numpy().copy(), sg.grad.item()))
    d = np.abs(grads[0][0] - grads[1][0]).max() / np.abs(grads[0][0]).max()
    assert d < 1e-2, d
    assert abs(grads[0][1] - grads[1][1]) < 1e-2 * abs(grads[0][1])
