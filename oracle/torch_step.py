"""Differentiable FP64 restatement of the CAC-LB wetting step on the CPU --
TEST INFRASTRUCTURE, not part of the product.

The same step as ``cacl_oracle.cpp`` (arXiv 2607.25444, Sects. 2.1-2.3),
written again with whole-field PyTorch CPU operations in float64 so that
reverse-mode automatic differentiation gives the exact adjoint of the FP64
step: the reference for the hand-written GPU adjoint (dL/dtheta per wall
node, dL/dsigma). Every field is an array over (z, y, x); a shift by a
lattice vector is a periodic roll (non-periodic axes are closed by solid
layers, as in the C++ oracle). It shares no code with the CUDA library; it
reads the wall list (normals, donor links) from the C++ oracle, whose
geometry is pinned separately.

Order of one step (the C++ oracle's): ghost update (Jacobi, Algorithm 1) ->
pull collide-stream with halfway bounce-back and the regularised Guo
collision -> MUSCL-minmod phase update with isotropic diffusion and the
isotropic compressive divergence -> global volume correction.

One switch, ``frozen_bulk_normal``: when set, the unit normal of the
compressive vector a = phi (1 - phi) grad phi / |grad phi| is held constant
(no derivative) at nodes outside the interface band eps_phi < phi <
1 - eps_phi of the volume correction. The GPU adjoint applies that rule (its
exact linearisation is unbounded on the bulk plateaus over long rollouts);
with the switch off the derivative is the exact one.

Parity unpinned: none; the forward is pinned to the C++ oracle and the
gradient to central differences of the C++ oracle (tests/test_oracle_adjoint.py).
"""
import math

import numpy as np
import torch

CS2 = 1.0 / 3.0
TD = torch.float64


def lattice():
    """D3Q27: q = 9 (cz + 1) + 3 (cy + 1) + (cx + 1); weights 8/27, 2/27,
    1/54, 1/216 by |c|^2 (Sect. 2.1)."""
    c = np.array([(cx, cy, cz) for cz in (-1, 0, 1) for cy in (-1, 0, 1)
                  for cx in (-1, 0, 1)], dtype=np.int64)
    m = (c * c).sum(1)
    w = np.array([8 / 27, 2 / 27, 1 / 54, 1 / 216])[m]
    opp = np.array([np.where((c == -ci).all(1))[0][0] for ci in c])
    return c, w, opp


C_, W_, OPP = lattice()
CT = torch.tensor(C_, dtype=TD)          # (27, 3)
WT = torch.tensor(W_, dtype=TD)          # (27,)
EYE = torch.eye(3, dtype=TD)
# Hermite tensors, Eqs. H2 and H3
H2 = torch.einsum("ia,ib->iab", CT, CT) - CS2 * EYE
H3 = (torch.einsum("ia,ib,ig->iabg", CT, CT, CT)
      - CS2 * (torch.einsum("ia,bg->iabg", CT, EYE)
               + torch.einsum("ib,ag->iabg", CT, EYE)
               + torch.einsum("ig,ab->iabg", CT, EYE)))


def at(field, c):
    """field(x + c) on the periodic grid, c = (cx, cy, cz)."""
    return torch.roll(field, shifts=(-int(c[2]), -int(c[1]), -int(c[0])),
                      dims=(-3, -2, -1))


def bcast(v, x):
    """Per-direction weights v (27,) shaped to broadcast against x (27, ...)."""
    return v.reshape((-1,) + (1,) * (x.dim() - 1))


def grad_iso(psi):
    """Eq. grad_iso: c_s^-2 sum_i w_i psi(x + c_i) c_i."""
    g = torch.zeros((3,) + psi.shape, dtype=TD)
    for i in range(27):
        v = at(psi, C_[i]) * W_[i]
        for a in range(3):
            if C_[i][a] != 0:
                g[a] = g[a] + C_[i][a] * v
    return g / CS2


def lap_iso(psi):
    """Eq. lap_iso: 2 c_s^-2 (sum_{i != 0} w_i psi(x + c_i) - (1 - w_0) psi)."""
    acc = torch.zeros_like(psi)
    for i in range(27):
        if i == 13:
            continue
        acc = acc + W_[i] * at(psi, C_[i])
    return 2.0 / CS2 * (acc - (1.0 - W_[13]) * psi)


def safe_sqrt(x):
    """sqrt(x) for x >= 0 with derivative 0 where x == 0 (the branch the
    value takes there) instead of an infinite one."""
    pos = x > 0
    return torch.where(pos, torch.sqrt(torch.where(pos, x, torch.ones_like(x))),
                       torch.zeros_like(x))


def minmod(a, b):
    """Eq. minmod: 0 if a b <= 0, else sign(a) min(|a|, |b|)."""
    m = torch.where(a.abs() < b.abs(), a, b)
    return torch.where(a * b <= 0, torch.zeros_like(a), m)


def equilibrium(pstar, u):
    """Eq. feq3 with p*: w_i (p* + c.u / c_s^2 + H2:uu / (2 c_s^4) +
    H3:uuu / (6 c_s^6)); pstar (...), u (3, ...) -> (27, ...)."""
    cu = torch.einsum("ia,a...->i...", CT, u)
    h2 = torch.einsum("iab,a...,b...->i...", H2, u, u)
    h3 = torch.einsum("iabg,a...,b...,g...->i...", H3, u, u, u)
    return bcast(WT, cu) * (pstar + cu / CS2 + h2 / (2 * CS2 ** 2)
                            + h3 / (6 * CS2 ** 3))


def guo(u, acc):
    """Eq. guo: w_i [(c_i - u)/c_s^2 + (c_i.u) c_i / c_s^4] . a."""
    cu = torch.einsum("ia,a...->i...", CT, u)
    ca = torch.einsum("ia,a...->i...", CT, acc)
    ua = (u * acc).sum(0)
    return bcast(WT, cu) * ((ca - ua) / CS2 + cu * ca / CS2 ** 2)


class TorchStep:
    """The step on one geometry. ``wall`` is the C++ oracle's wall list
    (dict with idx, qstar, nw); params as for the oracle (3D only)."""

    def __init__(self, params, solid, wall, frozen_bulk_normal=False):
        self.p = dict(params)
        self.shape = tuple(int(s) for s in solid.shape)  # (nz, ny, nx)
        self.solid = torch.tensor(np.asarray(solid) != 0)
        self.fluid = ~self.solid
        self.frozen = frozen_bulk_normal
        nz, ny, nx = self.shape
        idx = np.asarray(wall["idx"], dtype=np.int64)
        q = np.asarray(wall["qstar"], dtype=np.int64)
        x, y, z = idx % nx, (idx // nx) % ny, idx // (nx * ny)
        c = C_[q]
        xd, yd, zd = (x + c[:, 0]) % nx, (y + c[:, 1]) % ny, (z + c[:, 2]) % nz
        self.w_idx = torch.tensor(idx)
        self.w_donor = torch.tensor(xd + nx * (yd + ny * zd))
        self.w_nw = torch.tensor(np.asarray(wall["nw"], dtype=np.float64))
        self.w_rfs = torch.tensor(-c.astype(np.float64))  # Eq. donor_to_solid
        # pulled from a solid node: halfway bounce-back mask per direction
        self.bb = torch.stack([at(self.solid, -C_[i]) for i in range(27)])

    # ------------------------------------------------------------- parts
    def ghost(self, phi, theta_w):
        """Sect. 2.2, Algorithm 1 (Jacobi): every ghost value from the
        current field, then all assigned."""
        if self.w_idx.numel() == 0:
            return phi
        flat = phi.reshape(-1)
        g = grad_iso(phi).reshape(3, -1)[:, self.w_donor].T       # (W, 3)
        phi_f = flat[self.w_donor]
        n = self.w_nw
        gn = (g * n).sum(1, keepdim=True)
        gpar = g - gn * n                                         # Eq. tangential
        t = safe_sqrt((gpar * gpar).sum(1))
        thc = math.pi - theta_w * (math.pi / 180.0)               # internal angle
        sn, cs = torch.sin(thc), torch.cos(thc)
        reg = sn.abs() < 1e-6
        cot = torch.where(reg, torch.sign(cs).detach() * 1e6,
                          cs / torch.where(reg, torch.ones_like(sn), sn))
        dn = -t * cot
        gc = gpar + dn[:, None] * n
        lam = safe_sqrt(torch.clamp(4.0 * phi_f * (1.0 - phi_f), min=0.0))
        gval = phi_f + lam * (gc * self.w_rfs).sum(1)
        return flat.index_put((self.w_idx,), gval).reshape(self.shape)

    def pull(self, f):
        """Sect. 2.1: the populations a node pulls, f_q(x - c_q), with
        halfway bounce-back f_q(x) = f_opp(q)(x) where x - c_q is solid."""
        pulled = torch.stack([at(f[i], -C_[i]) for i in range(27)])
        return torch.where(self.bb, f[OPP], pulled)

    def collide(self, f, phi, sigma):
        """Sect. 2.1: pull with halfway bounce-back, then the regularised
        collision; solid nodes keep their populations."""
        fout, u = self.collide_pulled(self.pull(f), phi, sigma)
        return torch.where(self.solid, f, fout), u

    def collide_pulled(self, fin, phi, sigma):
        """Sect. 2.1: the regularised collision of the pulled populations
        with the Guo source of F = F_sigma + F_p + F_ext + F_nu; returns the
        post-collision populations (meaningful at fluid nodes) and u (0 at
        solid nodes)."""
        p = self.p
        g = grad_iso(phi)
        lap = lap_iso(phi)
        drho = p["rho_l"] - p["rho_g"]
        rho = p["rho_g"] + drho * phi
        mu = p["rho_g"] * p["nu_g"] + (p["rho_l"] * p["nu_l"] - p["rho_g"] * p["nu_g"]) * phi
        nu = mu / rho
        omega = 1.0 / (0.5 + nu / CS2)
        beta = 12.0 * sigma / p["width"]
        kphi = 1.5 * sigma * p["width"]
        pstar = fin.sum(0)
        j = torch.einsum("ia,i...->a...", CT, fin)
        grad_rho = drho * g
        mu_phi = 4.0 * beta * phi * (phi - 1.0) * (phi - 0.5) - kphi * lap
        grav = torch.tensor(p["gravity"], dtype=TD).reshape(3, 1, 1, 1)
        F0 = mu_phi * g - pstar * CS2 * grad_rho + (rho - p["rho_g"]) * grav
        a0 = F0 / rho
        u0 = j + 0.5 * a0
        feq0 = equilibrium(pstar, u0)
        Pi0 = (torch.einsum("ia,ib,i...->ab...", CT, CT, fin - feq0)
               + 0.5 * (torch.einsum("a...,b...->ab...", u0, a0)
                        + torch.einsum("a...,b...->ab...", a0, u0)))
        Fnu = -(nu * omega / CS2) * torch.einsum("ab...,b...->a...", Pi0, grad_rho)
        acc = (F0 + Fnu) / rho
        u = j + 0.5 * acc
        feq = equilibrium(pstar, u)
        S = guo(u, acc)
        A2 = torch.einsum("ia,ib,i...->ab...", CT, CT, fin - feq + 0.5 * S)
        A3 = (torch.einsum("a...,bg...->abg...", u, A2)
              + torch.einsum("b...,ag...->abg...", u, A2)
              + torch.einsum("g...,ab...->abg...", u, A2))
        fneq = bcast(WT, fin) * (torch.einsum("iab,ab...->i...", H2, A2) / (2 * CS2 ** 2)
                                 + torch.einsum("iabg,abg...->i...", H3, A3) / (6 * CS2 ** 3))
        fout = feq + (1.0 - omega) * fneq + 0.5 * S
        u = torch.where(self.solid, torch.zeros_like(u), u)
        return fout, u

    def compressive(self, phi):
        """a = phi (1 - phi) grad phi / |grad phi| at fluid nodes; 0 at solid
        nodes and where |grad phi| < 1e-12 (Sect. 2.1.1)."""
        g = grad_iso(phi)
        gm = safe_sqrt((g * g).sum(0))
        ok = (gm >= 1e-12) & self.fluid
        h = g / torch.where(ok, gm, torch.ones_like(gm))
        if self.frozen:
            eps = self.p["eps_phi"]
            band = (phi > eps) & (phi < 1.0 - eps)
            h = torch.where(band, h, h.detach())
        return torch.where(ok, phi * (1.0 - phi) * h, torch.zeros_like(h))

    def phase(self, phi, u, a=None):
        """Sect. 2.1.1, Eq. phi_update_muscl at fluid nodes; a: the
        compressive vector (formed from phi when not given)."""
        p = self.p
        kappa = 4.0 * p["mobility"] / p["width"]
        div = torch.zeros_like(phi)
        for d in range(3):
            e = [0, 0, 0]
            e[d] = 1
            em = [-v for v in e]
            slope = minmod(phi - at(phi, em), at(phi, e) - phi)
            r_sol = at(self.solid, e)
            uf = 0.5 * (u[d] + at(u[d], e))
            phiL = phi + 0.5 * slope
            phiR = at(phi, e) - 0.5 * at(slope, e)
            flux = uf * torch.where(uf >= 0, phiL, phiR)
            flux = torch.where(self.solid | r_sol, torch.zeros_like(flux), flux)
            div = div + flux - at(flux, em)
        if a is None:
            a = self.compressive(phi)
        diva = torch.zeros_like(phi)
        for i in range(27):
            ca = sum(C_[i][k] * at(a[k], C_[i]) for k in range(3) if C_[i][k] != 0)
            if isinstance(ca, int):
                continue
            diva = diva + (W_[i] / CS2) * ca
        out = phi - div + p["mobility"] * lap_iso(phi) - kappa * diva
        return torch.where(self.solid, phi, out)

    def correct(self, phi, m_ref):
        """Sect. 2.3: phi = phi* + lambda chi(phi*) at fluid nodes."""
        eps = self.p["eps_phi"]
        chi = torch.where((phi > eps) & (phi < 1.0 - eps), phi * (1.0 - phi),
                          torch.zeros_like(phi))
        chi = torch.where(self.fluid, chi, torch.zeros_like(chi))
        M = torch.where(self.fluid, phi, torch.zeros_like(phi)).sum()
        Wsum = chi.sum()
        lam = (m_ref - M) / Wsum if float(Wsum.detach()) > 0 else torch.zeros((), dtype=TD)
        return phi + lam * chi

    # ------------------------------------------------------------- step
    def init_state(self, phi0, u0=None):
        """f = f^eq(p* = 0, u) and M_ref = sum over fluid of phi (the C++
        oracle's set_fields)."""
        phi = torch.tensor(np.asarray(phi0, dtype=np.float64))
        u = (torch.zeros((3,) + self.shape, dtype=TD) if u0 is None
             else torch.tensor(np.asarray(u0, dtype=np.float64)))
        u = torch.where(self.solid, torch.zeros_like(u), u)
        f = equilibrium(torch.zeros(self.shape, dtype=TD), u)
        m_ref = float(phi[self.fluid].sum())
        return f, phi, u, m_ref

    def step(self, f, phi, m_ref, theta_w, sigma):
        phi_g = self.ghost(phi, theta_w)
        f, u = self.collide(f, phi_g, sigma)
        phis = self.phase(phi_g, u)
        return f, self.correct(phis, m_ref), u

    def rollout(self, phi0, theta_w, sigma, nsteps, u0=None):
        f, phi, u, m_ref = self.init_state(phi0, u0)
        for _ in range(nsteps):
            f, phi, u = self.step(f, phi, m_ref, theta_w, sigma)
        return f, phi, u
