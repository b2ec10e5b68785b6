/*
 * cacl_oracle.cpp -- TEST INFRASTRUCTURE, not part of the product.
 *
 * Plain FP64 CPU restatement of the CAC-LB wetting step of arXiv 2607.25444,
 * written from the paper's equations in the paper's notation.  It is slow on
 * purpose: tensors are contracted with explicit index loops, each stencil is
 * evaluated on the field the equation names, nothing is fused or reordered
 * beyond what the equations state.  Only tests, the smoke check and the bench's CPU baseline
 * may load it.  It shares nothing with the CUDA library.
 *
 * Order of one step n (state f*^{n-1}, phi^n incl. ghosts -> f*^n, u^n,
 * phi^{n+1}):
 *   1. ghost update over the wall list, Jacobi (Sect. 2.2, Algorithm 1)
 *   2. LB pull collide-stream with forces (Sect. 2.1)
 *   3. CAC update with MUSCL-minmod advection, isotropic diffusion and the
 *      isotropic compressive divergence (Sect. 2.1.1, Eq. phi_update_muscl)
 *   4. global volume correction (Sect. 2.3, Eqs. mass_defect..mass_corrected_phi)
 *
 * Readings of points where the paper is silent (each is listed in the design
 * notes of the repository):
 *   - hydrodynamic wall: halfway bounce-back, f_i(x) = f*_{opp i}(x) when
 *     x - c_i is solid;
 *   - F in Guo's term and in the half-force shift is the acceleration F/rho,
 *     because f^eq carries u (Eq. feq3), not rho u;
 *   - F_nu is evaluated explicitly from the predictor u0 = j + F0/(2 rho)
 *     with the non-equilibrium taken against the shifted equilibrium
 *     f^eq - S/2 (Eq. Fnu with Eq. guo's shift);
 *   - regularised collision f* = f^eq + (1-omega) f^neq + S/2, f^neq the
 *     Hermite projection (Eq. fneq3) of f - (f^eq - S/2); this is Eq. lbe with
 *     the shift of Sect. 2.1 applied to the regularised non-equilibrium;
 *   - F_ext = (rho(phi) - rho_g) g;
 *   - face velocity is 0 on fluid-solid faces; the compressive vector a is 0
 *     at solid nodes and where |grad phi| < 1e-12; the compressive weights
 *     (p1,p2,p3) are w_i / c_s^2, i.e. the divergence form of Eq. grad_iso;
 *   - wall node skipped when the integer normal is exactly zero; donor ties go
 *     to the lowest q; cot(theta_c) = sign(cos theta_c) 1e6 if |sin| < 1e-6;
 *     lambda_s = sqrt(max(0, 4 phi_f (1 - phi_f)));
 *   - ghosts are computed from the current field, then all assigned (Jacobi);
 *   - M_ref is the mass at set_fields (the paper's M^n, which every step
 *     restores), eps_phi is a parameter.
 */
#include "cacl_oracle.h"

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

namespace {

const double kPi = 3.14159265358979323846;

/* Sect. 2.1: lattice velocities c_i and quadrature weights w_i, c_s^2 = 1/3. */
struct Lattice {
  int dim = 3;
  int Q = 0;
  int rest = 0;
  int c[27][3];
  double w[27];
  int opp[27];
};

Lattice make_lattice(int dim) {
  Lattice L;
  L.dim = dim;
  int q = 0;
  const int zlo = (dim == 3) ? -1 : 0, zhi = (dim == 3) ? 1 : 0;
  for (int cz = zlo; cz <= zhi; ++cz)
    for (int cy = -1; cy <= 1; ++cy)
      for (int cx = -1; cx <= 1; ++cx) {
        L.c[q][0] = cx;
        L.c[q][1] = cy;
        L.c[q][2] = cz;
        const int m = cx * cx + cy * cy + cz * cz;
        if (dim == 3) {
          const double wt[4] = {8.0 / 27.0, 2.0 / 27.0, 1.0 / 54.0, 1.0 / 216.0};
          L.w[q] = wt[m];
        } else {
          const double wt[3] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 36.0};
          L.w[q] = wt[m];
        }
        if (m == 0) L.rest = q;
        ++q;
      }
  L.Q = q;
  for (int i = 0; i < L.Q; ++i)
    for (int j = 0; j < L.Q; ++j)
      if (L.c[j][0] == -L.c[i][0] && L.c[j][1] == -L.c[i][1] &&
          L.c[j][2] == -L.c[i][2])
        L.opp[i] = j;
  return L;
}

const double cs2 = 1.0 / 3.0;

double kron(int a, int b) { return a == b ? 1.0 : 0.0; }

/* Eq. H2: H^(2)_i,ab = c_a c_b - c_s^2 delta_ab. */
double H2(const Lattice& L, int i, int a, int b) {
  return L.c[i][a] * L.c[i][b] - cs2 * kron(a, b);
}

/* Eq. H3: H^(3)_i,abg = c_a c_b c_g - c_s^2 (c_a d_bg + c_b d_ag + c_g d_ab). */
double H3(const Lattice& L, int i, int a, int b, int g) {
  return L.c[i][a] * L.c[i][b] * L.c[i][g] -
         cs2 * (L.c[i][a] * kron(b, g) + L.c[i][b] * kron(a, g) +
                L.c[i][g] * kron(a, b));
}

/* Eq. feq3: third-order Hermite equilibrium with pressure-like p*. */
void equilibrium(const Lattice& L, double pstar, const double u[3],
                 double* feq) {
  const int D = L.dim;
  for (int i = 0; i < L.Q; ++i) {
    double cu = 0.0;
    for (int a = 0; a < D; ++a) cu += L.c[i][a] * u[a];
    double h2uu = 0.0;
    for (int a = 0; a < D; ++a)
      for (int b = 0; b < D; ++b) h2uu += H2(L, i, a, b) * u[a] * u[b];
    double h3uuu = 0.0;
    for (int a = 0; a < D; ++a)
      for (int b = 0; b < D; ++b)
        for (int g = 0; g < D; ++g)
          h3uuu += H3(L, i, a, b, g) * u[a] * u[b] * u[g];
    feq[i] = L.w[i] * (pstar + cu / cs2 + h2uu / (2.0 * cs2 * cs2) +
                       h3uuu / (6.0 * cs2 * cs2 * cs2));
  }
}

/* Eq. guo: S_i = w_i [ (c_i - u)/c_s^2 + (c_i.u) c_i / c_s^4 ] . a */
void guo_source(const Lattice& L, const double u[3], const double acc[3],
                double* S) {
  const int D = L.dim;
  for (int i = 0; i < L.Q; ++i) {
    double cu = 0.0;
    for (int a = 0; a < D; ++a) cu += L.c[i][a] * u[a];
    double s = 0.0;
    for (int a = 0; a < D; ++a)
      s += ((L.c[i][a] - u[a]) / cs2 + cu * L.c[i][a] / (cs2 * cs2)) * acc[a];
    S[i] = L.w[i] * s;
  }
}

}  // namespace

struct orc_state {
  orc_params p;
  Lattice L;
  long N = 0;
  std::vector<uint8_t> solid;
  std::vector<double> f;      // post-collision populations f*, [q][n]
  std::vector<double> phi;    // phase field incl. ghost values at wall nodes
  std::vector<double> u;      // [3][n]
  std::vector<double> theta;  // per-node contact angle (degrees)
  // wall list, sorted by node index
  std::vector<int32_t> w_idx;
  std::vector<int8_t> w_q;
  std::vector<int16_t> w_n6;  // [3*W]
  std::vector<float> w_nwf;   // [3*W] FP32 comparison form of n_w
  std::vector<double> w_nw;   // [3*W]
  double M_ref = 0.0, M_star = 0.0, W_sum = 0.0, lambda = 0.0;
  bool has_geom = false, has_fields = false;
  std::string err;
  // derived constants (Sect. 2.1, Eq. Fcap; Sect. 2.1.1, Eq. kappa_delta)
  double beta = 0.0, kappa_phi = 0.0, kappa = 0.0;

  long node(int x, int y, int z) const {
    return x + (long)p.nx * (y + (long)p.ny * z);
  }
  void coords(long n, int& x, int& y, int& z) const {
    x = (int)(n % p.nx);
    y = (int)((n / p.nx) % p.ny);
    z = (int)(n / ((long)p.nx * p.ny));
  }
  // Neighbour with wrap-around on every axis; non-periodic axes are closed by
  // solid layers, so a wrapped neighbour of a boundary node is solid.
  long nb(long n, int dx, int dy, int dz) const {
    int x, y, z;
    coords(n, x, y, z);
    x = (x + dx + p.nx) % p.nx;
    y = (y + dy + p.ny) % p.ny;
    z = (z + dz + p.nz) % p.nz;
    return node(x, y, z);
  }
  long nbq(long n, int q, int sign) const {
    return nb(n, sign * L.c[q][0], sign * L.c[q][1], sign * L.c[q][2]);
  }
  bool is_solid(long n) const { return solid[n] != 0; }
};

namespace {

int fail(orc_state* s, const char* msg) {
  s->err = msg;
  return -1;
}

/* Eq. grad_iso: grad Psi(x) = c_s^-2 sum_i w_i Psi(x + c_i) c_i. */
void grad_iso(const orc_state* s, const double* psi, long n, double g[3]) {
  g[0] = g[1] = g[2] = 0.0;
  for (int i = 0; i < s->L.Q; ++i) {
    const double v = psi[s->nbq(n, i, +1)];
    for (int a = 0; a < 3; ++a) g[a] += s->L.w[i] * v * s->L.c[i][a];
  }
  for (int a = 0; a < 3; ++a) g[a] /= cs2;
}

/* Eq. lap_iso: lap Psi = 2 c_s^-2 ( sum_{i!=0} w_i Psi(x+c_i) - (1-w_0) Psi(x) ). */
double lap_iso(const orc_state* s, const double* psi, long n) {
  double acc = 0.0;
  for (int i = 0; i < s->L.Q; ++i) {
    if (i == s->L.rest) continue;
    acc += s->L.w[i] * psi[s->nbq(n, i, +1)];
  }
  return 2.0 / cs2 * (acc - (1.0 - s->L.w[s->L.rest]) * psi[n]);
}

/* Mixture laws, Eqs. rho_mix_linear, mu_mix_linear, omega_phi. */
void mixture(const orc_params& p, double phi, double& rho, double& nu,
             double& omega) {
  rho = p.rho_g + (p.rho_l - p.rho_g) * phi;
  const double mu_g = p.rho_g * p.nu_g, mu_l = p.rho_l * p.nu_l;
  const double mu = mu_g + (mu_l - mu_g) * phi;
  nu = mu / rho;
  omega = 1.0 / (0.5 + nu / cs2);
}

/*
 * One node of the LB collision (Sect. 2.1), from the pulled populations f_in.
 * Moments Eqs. pstar_moment/u_moment, forces Eqs. Fsplit..Fnu, equilibrium
 * Eq. feq3, Guo source Eq. guo, recursive regularisation Eqs. fneq3/A3rec.
 */
void collide_node(const orc_state* s, const double* fin, double phi,
                  const double grad_phi[3], double lap_phi, double* fout,
                  double u_out[3], double a_out[3], double* omega_out) {
  const Lattice& L = s->L;
  const orc_params& p = s->p;
  const int D = L.dim;
  double rho, nu, omega;
  mixture(p, phi, rho, nu, omega);

  double pstar = 0.0, j[3] = {0, 0, 0};
  for (int i = 0; i < L.Q; ++i) {
    pstar += fin[i];
    for (int a = 0; a < 3; ++a) j[a] += fin[i] * L.c[i][a];
  }
  double grad_rho[3];
  for (int a = 0; a < 3; ++a) grad_rho[a] = (p.rho_l - p.rho_g) * grad_phi[a];

  // Eq. Fcap: mu_phi = 4 beta (phi - phi_l)(phi - phi_g)(phi - phi_0) - kappa_phi lap phi
  const double mu_phi = 4.0 * s->beta * (phi - 1.0) * (phi - 0.0) * (phi - 0.5) -
                        s->kappa_phi * lap_phi;
  double F0[3];
  for (int a = 0; a < 3; ++a) {
    const double F_sigma = mu_phi * grad_phi[a];
    const double F_p = -pstar * cs2 * grad_rho[a];  // Eq. Fp
    const double F_ext = (rho - p.rho_g) * p.gravity[a];
    F0[a] = F_sigma + F_p + F_ext;
  }
  if (D == 2) F0[2] = 0.0;

  // Predictor for F_nu (Eq. Fnu): u0 = j + a0/2, Pi0 against f^eq - S/2.
  double a0[3], u0[3];
  for (int a = 0; a < 3; ++a) {
    a0[a] = F0[a] / rho;
    u0[a] = j[a] + 0.5 * a0[a];
  }
  std::vector<double> feq(L.Q), S(L.Q);
  equilibrium(L, pstar, u0, feq.data());
  double Pi0[3][3] = {{0}};
  for (int a = 0; a < D; ++a)
    for (int b = 0; b < D; ++b) {
      double acc = 0.0;
      for (int i = 0; i < L.Q; ++i)
        acc += (fin[i] - feq[i]) * L.c[i][a] * L.c[i][b];
      Pi0[a][b] = acc + 0.5 * (u0[a] * a0[b] + a0[a] * u0[b]);
    }
  double F[3];
  for (int a = 0; a < 3; ++a) {
    double pg = 0.0;
    for (int b = 0; b < D; ++b) pg += Pi0[a][b] * grad_rho[b];
    const double F_nu = (a < D) ? -(nu * omega / cs2) * pg : 0.0;
    F[a] = F0[a] + F_nu;  // Eq. Fsplit
  }

  double acc_[3], u[3];
  for (int a = 0; a < 3; ++a) {
    acc_[a] = F[a] / rho;
    u[a] = j[a] + 0.5 * acc_[a];  // Eq. u_moment with sum_i S_i c_i = a
  }
  equilibrium(L, pstar, u, feq.data());
  guo_source(L, u, acc_, S.data());

  // A2: second moment of f - (f^eq - S/2); A3 by recursion, Eq. A3rec.
  double A2[3][3] = {{0}};
  for (int a = 0; a < D; ++a)
    for (int b = 0; b < D; ++b) {
      double m = 0.0;
      for (int i = 0; i < L.Q; ++i)
        m += (fin[i] - feq[i] + 0.5 * S[i]) * L.c[i][a] * L.c[i][b];
      A2[a][b] = m;
    }
  double A3[3][3][3] = {{{0}}};
  for (int a = 0; a < D; ++a)
    for (int b = 0; b < D; ++b)
      for (int g = 0; g < D; ++g)
        A3[a][b][g] = u[a] * A2[b][g] + u[b] * A2[a][g] + u[g] * A2[a][b];

  for (int i = 0; i < L.Q; ++i) {
    double h2 = 0.0, h3 = 0.0;
    for (int a = 0; a < D; ++a)
      for (int b = 0; b < D; ++b) {
        h2 += H2(L, i, a, b) * A2[a][b];
        for (int g = 0; g < D; ++g) h3 += H3(L, i, a, b, g) * A3[a][b][g];
      }
    const double fneq =
        L.w[i] * (h2 / (2.0 * cs2 * cs2) + h3 / (6.0 * cs2 * cs2 * cs2));
    fout[i] = feq[i] + (1.0 - omega) * fneq + 0.5 * S[i];
  }
  for (int a = 0; a < 3; ++a) {
    u_out[a] = u[a];
    a_out[a] = acc_[a];
  }
  if (omega_out) *omega_out = omega;
}

/* cot(theta_c), theta_c = pi - theta (Eq. internal_contact_angle), with the
 * regularisation of Sect. 2.2 near |sin theta_c| -> 0. */
double cot_theta_c(double theta_deg) {
  const double thc = kPi - theta_deg * kPi / 180.0;
  const double sn = std::sin(thc), cs = std::cos(thc);
  if (std::fabs(sn) < 1e-6) return (cs >= 0.0 ? 1.0 : -1.0) * 1e6;
  return cs / sn;
}

/* Eqs. tangential_gradient_contact_angle .. ghost_contact_angle_extrapolation. */
double ghost_value(double phi_f, const double g[3], const double nw[3],
                   const double rfs[3], double theta_deg) {
  const double gn = g[0] * nw[0] + g[1] * nw[1] + g[2] * nw[2];
  double gpar[3];
  for (int a = 0; a < 3; ++a) gpar[a] = g[a] - gn * nw[a];
  const double t =
      std::sqrt(gpar[0] * gpar[0] + gpar[1] * gpar[1] + gpar[2] * gpar[2]);
  const double dn = -t * cot_theta_c(theta_deg);
  double gc[3];
  for (int a = 0; a < 3; ++a) gc[a] = gpar[a] + dn * nw[a];
  const double lam = std::sqrt(std::max(0.0, 4.0 * phi_f * (1.0 - phi_f)));
  return phi_f + lam * (gc[0] * rfs[0] + gc[1] * rfs[1] + gc[2] * rfs[2]);
}

/* Eq. minmod. */
double minmod(double a, double b) {
  if (a * b <= 0.0) return 0.0;
  return (a > 0.0 ? 1.0 : -1.0) * std::min(std::fabs(a), std::fabs(b));
}

/* Eq. interface_weight_mass_correction. */
double chi(double v, double eps) {
  return (v > eps && v < 1.0 - eps) ? v * (1.0 - v) : 0.0;
}

/* Discrete compressive vector a(y) = phi(1-phi) n at fluid y (Sect. 2.1.1). */
void compressive_vector(const orc_state* s, const double* phi, long y,
                        double a[3]) {
  a[0] = a[1] = a[2] = 0.0;
  if (s->is_solid(y)) return;
  double g[3];
  grad_iso(s, phi, y, g);
  const double gm = std::sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
  if (gm < 1e-12) return;
  const double v = phi[y];
  for (int d = 0; d < 3; ++d) a[d] = v * (1.0 - v) * g[d] / gm;
}

}  // namespace

extern "C" {

orc_state* orc_create(const orc_params* p) {
  if (!p) return nullptr;
  if (p->dim != 2 && p->dim != 3) return nullptr;
  if (p->nx < 1 || p->ny < 1 || p->nz < 1) return nullptr;
  if (p->dim == 2 && p->nz != 1) return nullptr;
  if (!(p->width > 0) || p->mobility < 0 || p->rho_l <= 0 || p->rho_g <= 0 ||
      p->nu_l <= 0 || p->nu_g <= 0)
    return nullptr;
  orc_state* s = new orc_state();
  s->p = *p;
  s->L = make_lattice(p->dim);
  s->N = (long)p->nx * p->ny * p->nz;
  s->solid.assign(s->N, 0);
  s->f.assign((size_t)s->L.Q * s->N, 0.0);
  s->phi.assign(s->N, 0.0);
  s->u.assign(3 * (size_t)s->N, 0.0);
  s->theta.assign(s->N, p->theta_deg);
  s->beta = 12.0 * p->sigma / p->width;         // Sect. 2.1, below Eq. Fcap
  s->kappa_phi = 3.0 * p->sigma * p->width / 2.0;
  s->kappa = 4.0 * p->mobility / p->width;      // Eq. kappa_delta
  return s;
}

void orc_destroy(orc_state* s) { delete s; }

const char* orc_error(const orc_state* s) { return s ? s->err.c_str() : ""; }

/* Wall-normal reconstruction and donor selection, Sect. 2.2
 * (Eqs. local_wall_normal .. donor_to_solid). Integer form: m_q = 6 w_q. */
int orc_set_geometry(orc_state* s, const uint8_t* solid) {
  if (!s || !solid) return -1;
  const orc_params& p = s->p;
  for (long n = 0; n < s->N; ++n) s->solid[n] = solid[n] ? 1 : 0;
  // Non-periodic axes must be closed by solid boundary layers.
  for (int ax = 0; ax < 3; ++ax) {
    if (p.periodic[ax]) continue;
    const int ext[3] = {p.nx, p.ny, p.nz};
    if (ext[ax] < 2) return fail(s, "non-periodic axis shorter than 2");
    for (long n = 0; n < s->N; ++n) {
      int c[3];
      s->coords(n, c[0], c[1], c[2]);
      if ((c[ax] == 0 || c[ax] == ext[ax] - 1) && !s->solid[n])
        return fail(s, "non-periodic axis not closed by solid layers");
    }
  }
  s->w_idx.clear();
  s->w_q.clear();
  s->w_n6.clear();
  s->w_nwf.clear();
  s->w_nw.clear();
  const Lattice& L = s->L;
  for (long n = 0; n < s->N; ++n) {
    if (!s->solid[n]) continue;
    int n6[3] = {0, 0, 0};
    bool any_fluid = false;
    for (int q = 0; q < L.Q; ++q) {
      if (q == L.rest) continue;
      if (s->is_solid(s->nbq(n, q, +1))) continue;
      any_fluid = true;
      const int m2 = L.c[q][0] * L.c[q][0] + L.c[q][1] * L.c[q][1] +
                     L.c[q][2] * L.c[q][2];
      const int mq = 6 / m2;  // 6 w_q with w_q = 1, 1/2, 1/3
      for (int a = 0; a < 3; ++a) n6[a] -= mq * L.c[q][a];
    }
    if (!any_fluid) continue;  // not adjacent to the fluid
    const long nn = (long)n6[0] * n6[0] + (long)n6[1] * n6[1] + (long)n6[2] * n6[2];
    if (nn == 0) continue;     // |n~| below tolerance: skipped
    // Donor: argmax of S_q = (-c_q . n_w)/|c_q| over the fluid links, compared
    // exactly as a_q/sqrt(m_q) with a_q = -c_q . n~6, m_q = |c_q|^2.
    int best = -1;
    long ba = 0, bm = 1;
    for (int q = 0; q < L.Q; ++q) {
      if (q == L.rest) continue;
      if (s->is_solid(s->nbq(n, q, +1))) continue;
      const long a = -(long)(L.c[q][0] * n6[0] + L.c[q][1] * n6[1] + L.c[q][2] * n6[2]);
      const long m = L.c[q][0] * L.c[q][0] + L.c[q][1] * L.c[q][1] + L.c[q][2] * L.c[q][2];
      bool better;
      if (best < 0) {
        better = true;
      } else if (a > 0 && ba <= 0) {
        better = true;
      } else if (a <= 0 && ba > 0) {
        better = false;
      } else if (a > 0) {
        better = a * a * bm > ba * ba * m;
      } else {
        better = a * a * bm < ba * ba * m;
      }
      if (better) {
        best = q;
        ba = a;
        bm = m;
      }
    }
    s->w_idx.push_back((int32_t)n);
    s->w_q.push_back((int8_t)best);
    const double nrm = std::sqrt((double)nn);
    const float nrmf = std::sqrt((float)nn);
    for (int a = 0; a < 3; ++a) {
      s->w_n6.push_back((int16_t)n6[a]);
      s->w_nw.push_back(n6[a] / nrm);
      s->w_nwf.push_back((float)n6[a] / nrmf);
    }
  }
  s->has_geom = true;
  s->has_fields = false;
  return 0;
}

int orc_set_contact_angle(orc_state* s, const double* theta) {
  if (!s) return -1;
  for (long n = 0; n < s->N; ++n) s->theta[n] = theta ? theta[n] : s->p.theta_deg;
  return 0;
}

double orc_fluid_mass(const orc_state* s) {
  double m = 0.0;  // Eq. phase_field_mass, Delta V = 1
  for (long n = 0; n < s->N; ++n)
    if (!s->solid[n]) m += s->phi[n];
  return m;
}

/* Initial state: f* = f^eq(p* = 0, u) with f^neq = 0; M_ref = sum over fluid. */
int orc_set_fields(orc_state* s, const double* phi, const double* u) {
  if (!s || !phi) return -1;
  if (!s->has_geom) return fail(s, "set_geometry first");
  for (long n = 0; n < s->N; ++n) s->phi[n] = phi[n];
  std::vector<double> feq(s->L.Q);
  for (long n = 0; n < s->N; ++n) {
    double un[3] = {0, 0, 0};
    if (u && !s->solid[n])
      for (int a = 0; a < 3; ++a) un[a] = u[a * s->N + n];
    if (s->L.dim == 2) un[2] = 0.0;
    for (int a = 0; a < 3; ++a) s->u[a * s->N + n] = un[a];
    equilibrium(s->L, 0.0, un, feq.data());
    for (int q = 0; q < s->L.Q; ++q) s->f[q * s->N + n] = feq[q];
  }
  s->M_ref = orc_fluid_mass(s);
  s->lambda = s->M_star = s->W_sum = 0.0;
  s->has_fields = true;
  return 0;
}

int orc_set_populations(orc_state* s, const double* f) {
  if (!s || !f) return -1;
  std::memcpy(s->f.data(), f, sizeof(double) * s->L.Q * s->N);
  return 0;
}

int orc_set_phi(orc_state* s, const double* phi) {
  if (!s || !phi) return -1;
  std::memcpy(s->phi.data(), phi, sizeof(double) * s->N);
  return 0;
}

int orc_set_velocity(orc_state* s, const double* u) {
  if (!s || !u) return -1;
  std::memcpy(s->u.data(), u, sizeof(double) * 3 * s->N);
  return 0;
}

int orc_set_mass_ref(orc_state* s, double m) {
  if (!s) return -1;
  s->M_ref = m;
  return 0;
}

/* Sect. 2.2, Algorithm 1: every ghost from the current field, then assign. */
int orc_ghost_update(orc_state* s) {
  if (!s || !s->has_fields) return -1;
  const long W = (long)s->w_idx.size();
  std::vector<double> g(W);
#pragma omp parallel for schedule(static)
  for (long w = 0; w < W; ++w) {
    const long xs = s->w_idx[w];
    const int q = s->w_q[w];
    const long xf = s->nbq(xs, q, +1);  // x_f = x_s + c_{q*}
    const double phi_f = s->phi[xf];
    double grad_f[3];
    grad_iso(s, s->phi.data(), xf, grad_f);
    const double rfs[3] = {-(double)s->L.c[q][0], -(double)s->L.c[q][1],
                           -(double)s->L.c[q][2]};  // Eq. donor_to_solid
    g[w] = ghost_value(phi_f, grad_f, &s->w_nw[3 * w], rfs, s->theta[xs]);
  }
  for (long w = 0; w < W; ++w) s->phi[s->w_idx[w]] = g[w];
  return 0;
}

/* Sect. 2.1: pull streaming with halfway bounce-back, then collision. */
int orc_lb_collide(orc_state* s) {
  if (!s || !s->has_fields) return -1;
  const Lattice& L = s->L;
  const long N = s->N;
  std::vector<double> fnew(s->f.size());
#pragma omp parallel for schedule(static)
  for (long n = 0; n < N; ++n) {
    if (s->solid[n]) {
      for (int q = 0; q < L.Q; ++q) fnew[q * N + n] = s->f[q * N + n];
      continue;
    }
    double fin[27], fout[27];
    for (int q = 0; q < L.Q; ++q) {
      const long src = s->nbq(n, q, -1);  // x - c_q
      fin[q] = s->is_solid(src) ? s->f[L.opp[q] * N + n] : s->f[q * N + src];
    }
    double g[3];
    grad_iso(s, s->phi.data(), n, g);
    const double lap = lap_iso(s, s->phi.data(), n);
    double u[3], a[3];
    collide_node(s, fin, s->phi[n], g, lap, fout, u, a, nullptr);
    for (int q = 0; q < L.Q; ++q) fnew[q * N + n] = fout[q];
    for (int d = 0; d < 3; ++d) s->u[d * N + n] = u[d];
  }
  s->f.swap(fnew);
  return 0;
}

/* Sect. 2.1.1, Eq. phi_update_muscl at fluid nodes; phi* replaces phi. The
 * limited slopes s^d (Eq. slope_minmod_x) and the compressive vector field a
 * are node fields; they are formed first, then differenced. */
int orc_phase_update(orc_state* s) {
  if (!s || !s->has_fields) return -1;
  const long N = s->N;
  const int D = s->L.dim;
  const double* phi = s->phi.data();
  std::vector<double> out(N), slope(3 * (size_t)N, 0.0), a(3 * (size_t)N, 0.0);
#pragma omp parallel for schedule(static)
  for (long y = 0; y < N; ++y) {
    for (int d = 0; d < D; ++d) {
      int e[3] = {0, 0, 0};
      e[d] = 1;
      const long yp = s->nb(y, e[0], e[1], e[2]);
      const long ym = s->nb(y, -e[0], -e[1], -e[2]);
      slope[d * N + y] = minmod(phi[y] - phi[ym], phi[yp] - phi[y]);
    }
    double av[3];
    compressive_vector(s, phi, y, av);
    for (int d = 0; d < 3; ++d) a[d * N + y] = av[d];
  }
  // face flux between cell l and its +d neighbour r, Eqs. face_flux_def,
  // recon_lr_x, upwind_select_x; zero across a fluid-solid face.
  auto face_flux = [&](long l, int d) {
    int e[3] = {0, 0, 0};
    e[d] = 1;
    const long r = s->nb(l, e[0], e[1], e[2]);
    if (s->is_solid(l) || s->is_solid(r)) return 0.0;
    const double uf = 0.5 * (s->u[d * N + l] + s->u[d * N + r]);
    const double phiL = phi[l] + 0.5 * slope[d * N + l];
    const double phiR = phi[r] - 0.5 * slope[d * N + r];
    const double up = (uf >= 0.0) ? phiL : phiR;
    return uf * up;
  };
#pragma omp parallel for schedule(static)
  for (long n = 0; n < N; ++n) {
    if (s->solid[n]) {
      out[n] = phi[n];
      continue;
    }
    // Eq. divF
    double div = 0.0;
    for (int d = 0; d < D; ++d) {
      int e[3] = {0, 0, 0};
      e[d] = 1;
      const long m = s->nb(n, -e[0], -e[1], -e[2]);
      div += face_flux(n, d) - face_flux(m, d);
    }
    const double lap = lap_iso(s, phi, n);
    // Eq. source_sharp: S = -kappa div_h(a), isotropic divergence with
    // weights (p1, p2, p3) = w_i / c_s^2
    double diva = 0.0;
    for (int i = 0; i < s->L.Q; ++i) {
      const long y = s->nbq(n, i, +1);
      diva += s->L.w[i] / cs2 *
              (a[0 * N + y] * s->L.c[i][0] + a[1 * N + y] * s->L.c[i][1] +
               a[2 * N + y] * s->L.c[i][2]);
    }
    out[n] = phi[n] - div + s->p.mobility * lap - s->kappa * diva;
  }
  s->phi.swap(out);
  return 0;
}

/* Sect. 2.3, Eqs. tentative_phase_field_mass .. mass_corrected_phi. */
int orc_volume_correct(orc_state* s) {
  if (!s || !s->has_fields) return -1;
  const long N = s->N;
  const double eps = s->p.eps_phi;
  double M = 0.0, W = 0.0;
  for (long n = 0; n < N; ++n) {
    if (s->solid[n]) continue;
    M += s->phi[n];
    W += chi(s->phi[n], eps);
  }
  s->M_star = M;
  s->W_sum = W;
  s->lambda = (W > 0.0) ? (s->M_ref - M) / W : 0.0;
  for (long n = 0; n < N; ++n) {
    if (s->solid[n]) continue;
    s->phi[n] = s->phi[n] + s->lambda * chi(s->phi[n], eps);
  }
  return 0;
}

int orc_step(orc_state* s, int nsteps) {
  if (!s || !s->has_fields) return -1;
  for (int k = 0; k < nsteps; ++k) {
    if (orc_ghost_update(s) || orc_lb_collide(s) || orc_phase_update(s) ||
        orc_volume_correct(s))
      return -1;
  }
  return 0;
}

int orc_get_fields(const orc_state* s, double* phi, double* u, double* pstar) {
  if (!s) return -1;
  const long N = s->N;
  if (phi) std::memcpy(phi, s->phi.data(), sizeof(double) * N);
  if (u) std::memcpy(u, s->u.data(), sizeof(double) * 3 * N);
  if (pstar) {
    // Eq. pstar_moment: the collision keeps sum_i f_i, so sum f* is p*.
    for (long n = 0; n < N; ++n) {
      double acc = 0.0;
      for (int q = 0; q < s->L.Q; ++q) acc += s->f[q * N + n];
      pstar[n] = s->solid[n] ? 0.0 : acc;
    }
  }
  return 0;
}

int orc_get_populations(const orc_state* s, double* f) {
  if (!s || !f) return -1;
  std::memcpy(f, s->f.data(), sizeof(double) * s->L.Q * s->N);
  return 0;
}

int orc_get_wall_count(const orc_state* s) {
  return s ? (int)s->w_idx.size() : -1;
}

int orc_get_wall_list(const orc_state* s, int32_t* idx, int8_t* qstar,
                      int16_t* ntilde6, float* nw_f32, double* nw_f64) {
  if (!s) return -1;
  const size_t W = s->w_idx.size();
  if (idx) std::memcpy(idx, s->w_idx.data(), W * sizeof(int32_t));
  if (qstar) std::memcpy(qstar, s->w_q.data(), W * sizeof(int8_t));
  if (ntilde6) std::memcpy(ntilde6, s->w_n6.data(), 3 * W * sizeof(int16_t));
  if (nw_f32) std::memcpy(nw_f32, s->w_nwf.data(), 3 * W * sizeof(float));
  if (nw_f64) std::memcpy(nw_f64, s->w_nw.data(), 3 * W * sizeof(double));
  return 0;
}

int orc_get_mass(const orc_state* s, double* m_ref, double* m_star,
                 double* w_sum, double* lambda) {
  if (!s) return -1;
  if (m_ref) *m_ref = s->M_ref;
  if (m_star) *m_star = s->M_star;
  if (w_sum) *w_sum = s->W_sum;
  if (lambda) *lambda = s->lambda;
  return 0;
}

int orc_lattice(int dim, int* c, double* w) {
  if (dim != 2 && dim != 3) return -1;
  const Lattice L = make_lattice(dim);
  for (int q = 0; q < L.Q; ++q) {
    for (int a = 0; a < 3; ++a) c[3 * q + a] = L.c[q][a];
    w[q] = L.w[q];
  }
  return L.Q;
}

int orc_feq(int dim, double pstar, const double* u, double* feq) {
  if (dim != 2 && dim != 3) return -1;
  const Lattice L = make_lattice(dim);
  double uu[3] = {u[0], u[1], dim == 3 ? u[2] : 0.0};
  equilibrium(L, pstar, uu, feq);
  return L.Q;
}

int orc_collide_node(const orc_state* s, const double* f_in, double phi,
                     const double* grad_phi, double lap_phi, double* f_out,
                     double* u_out, double* a_out, double* omega_out) {
  if (!s) return -1;
  collide_node(s, f_in, phi, grad_phi, lap_phi, f_out, u_out, a_out, omega_out);
  return 0;
}

int orc_grad_lap(const orc_state* s, const double* field, double* grad,
                 double* lap) {
  if (!s) return -1;
  for (long n = 0; n < s->N; ++n) {
    double g[3];
    grad_iso(s, field, n, g);
    for (int a = 0; a < 3; ++a) grad[a * s->N + n] = g[a];
    lap[n] = lap_iso(s, field, n);
  }
  return 0;
}

double orc_ghost_value(double phi_f, const double* grad_f, const double* nw,
                       const double* r_fs, double theta_deg) {
  return ghost_value(phi_f, grad_f, nw, r_fs, theta_deg);
}

}  // extern "C"
