// lb.cu -- fused D3Q27 pull collide-stream with the multiphase forces
// (Sect. 2.1: Eqs. pstar_moment, u_moment, rho_mix_linear, mu_mix_linear,
// omega_phi, feq3, H2, H3, fneq3, A3rec, guo, Fsplit, Fcap, Fp, Fnu,
// grad_iso, lap_iso).
//
// One thread per node, x fastest. Populations are structure-of-arrays
// f[q][n]; the pull reads f*_q(x - c_q) (halfway bounce-back f*_{opp q}(x)
// when x - c_q is solid), the phi stencil is read through the read-only
// cache, and the node writes its 27 post-collision populations, u, and the
// compressive vector a = phi (1 - phi) grad phi / |grad phi| of the same
// phi^n, which the phi update of this step needs at every node (Sect. 2.1.1):
// the gradient is already in registers here.
//
// Collision algebra. With A2 = Pi - p* c_s^2 I - u u + (u a + a u)/2 (the
// second moment of f - (f^eq - S/2), using sum f^eq c c = p* c_s^2 I + u u),
// tr = trace A2, v = A2 u, and for each direction cu = c.u, ca = c.a,
// cAc = c.A2.c, cAu = c.v, the post-collision population
//   f*_i = f^eq_i + (1 - omega) f^neq_i + S_i / 2
// is w_i P(c_i) with P = E + O,
//   E = k1 + 4.5 cu^2 + om45 cAc + 4.5 cu ca
//   O = cu (k2 + 4.5 cu^2 + 3 om45 cAc) - 2 om45 cAu + 1.5 ca
// where om45 = 4.5 (1 - omega), k1 = p* - 1.5 (u.u + u.a) - om45 tr / 3,
// k2 = 3 - 4.5 u.u - om45 tr.
//
// Evaluation. On the D3Q27 velocities every c_a is -1, 0 or 1, so c_a^3 =
// c_a and c_a^2 = |c_a| =: e_a, and P is a combination of the separable
// monomials b_i(cx) b_j(cy) b_k(cz), b in {1, c, e}. Expanding E and O gives
// 17 nonzero coefficients:
//   1: k1          c_a: L_a = u_a (k2 + 4.5 u_a^2 + 3 om45 A_aa)
//                                 - 2 om45 v_a + 1.5 a_a
//   e_a: D_a = 4.5 u_a (u_a + a_a) + om45 A_aa
//   c_a c_b (a < b): F_ab = 9 u_a u_b + 2 om45 A_ab + 4.5 (u_a a_b + u_b a_a)
//   e_a c_b (a != b): M_ab = u_b (13.5 u_a^2 + 3 om45 A_aa) + 6 om45 u_a A_ab
//   cx cy cz: X = 27 ux uy uz + 6 om45 (ux A_yz + uy A_xz + uz A_xy)
// and P is evaluated at all 27 velocities by three one-axis transforms
// (z, then y, then x: g(0) = g_1, g(+-1) = g_1 + g_e +- g_c), about 70
// operations instead of a separate polynomial per direction pair. The
// moments are formed the same way in reverse (sums and differences along x,
// then y, then z).
#include <cudaTypedefs.h>

#include <algorithm>

#include "cacl_internal.cuh"

namespace cacl {
namespace {

constexpr int LB_BX = 128;
constexpr int LB_BY = 1;
// two-node (x pair) kernel: PX pairs along x times PY rows per block
constexpr int LB2_PX = 32;
constexpr int LB2_PY = 4;

// Post-collision state of one node (V = float) or of an x pair of nodes
// (V = float2, both lanes rounded exactly as the one-node form).
template <typename V>
struct NodeOut {
  V P[Q];  // f*_q / w_q
  V ux, uy, uz;
};

// The 17 coefficients of the post-collision polynomial P in the separable
// monomials (the node's post-collision state in moment form), in storage
// order: 1; c_x, c_y, c_z; e_x, e_y, e_z; c_x c_y, c_x c_z, c_y c_z;
// e_x c_y, e_x c_z, e_y c_x, e_y c_z, e_z c_x, e_z c_y; c_x c_y c_z.
template <typename V>
struct Coefs {
  V k1, Lx, Ly, Lz, Dx, Dy, Dz, Fxy, Fxz, Fyz, Mxy, Mxz, Myx, Myz, Mzx, Mzy, X;
};

// P at all 27 velocities from the coefficients: three one-axis transforms
// (z, then y, then x: g(0) = g_1, g(+-1) = g_1 + g_e +- g_c).
template <typename V>
__device__ __forceinline__ void coefs_to_P(const Coefs<V>& c, V (&P)[Q]) {
  // z transform: Z_ij(cz) for x basis i, y basis j (1, c, e); index cz+1
  V Z00[3], Z10[3], Z20[3], Z01[3], Z11[3], Z02[3];
  {
    const V t00 = vadd(c.k1, c.Dz), t10 = vadd(c.Lx, c.Mzx), t01 = vadd(c.Ly, c.Mzy);
    Z00[0] = vsub(t00, c.Lz); Z00[1] = c.k1; Z00[2] = vadd(t00, c.Lz);
    Z10[0] = vsub(t10, c.Fxz); Z10[1] = c.Lx; Z10[2] = vadd(t10, c.Fxz);
    Z20[0] = vsub(c.Dx, c.Mxz); Z20[1] = c.Dx; Z20[2] = vadd(c.Dx, c.Mxz);
    Z01[0] = vsub(t01, c.Fyz); Z01[1] = c.Ly; Z01[2] = vadd(t01, c.Fyz);
    Z11[0] = vsub(c.Fxy, c.X); Z11[1] = c.Fxy; Z11[2] = vadd(c.Fxy, c.X);
    Z02[0] = vsub(c.Dy, c.Myz); Z02[1] = c.Dy; Z02[2] = vadd(c.Dy, c.Myz);
  }
  // y transform then x transform, line by line (cy, cz)
#pragma unroll
  for (int kz = 0; kz < 3; ++kz) {
    const V t0 = vadd(Z00[kz], Z02[kz]), t1 = vadd(Z10[kz], c.Myx);
    const V Y0[3] = {vsub(t0, Z01[kz]), Z00[kz], vadd(t0, Z01[kz])};
    const V Y1[3] = {vsub(t1, Z11[kz]), Z10[kz], vadd(t1, Z11[kz])};
    const V Y2[3] = {vsub(Z20[kz], c.Mxy), Z20[kz], vadd(Z20[kz], c.Mxy)};
#pragma unroll
    for (int jy = 0; jy < 3; ++jy) {
      const int q = 9 * kz + 3 * jy;
      const V t = vadd(Y0[jy], Y2[jy]);
      P[q] = vsub(t, Y1[jy]);
      P[q + 1] = Y0[jy];
      P[q + 2] = vadd(t, Y1[jy]);
    }
  }
}

// The collision up to the coefficients of P (and u).
template <typename V>
__device__ __forceinline__ void collide_coefs(const V (&f)[Q], V phi0, V gx, V gy,
                                              V gz, V lap, const Consts& k,
                                              Coefs<V>& cf, V& uxo, V& uyo, V& uzo) {
  // moments by sum factorisation: along x for each (cy, cz) line l, then
  // along y for each cz, then along z (q = 9 (cz+1) + 3 (cy+1) + (cx+1))
  V m0[9], m1[9], m2[9];  // sum f, sum cx f, sum cx^2 f over the line
#pragma unroll
  for (int l = 0; l < 9; ++l) {
    m2[l] = vadd(f[3 * l + 2], f[3 * l]);
    m1[l] = vsub(f[3 * l + 2], f[3 * l]);
    m0[l] = vadd(m2[l], f[3 * l + 1]);
  }
  V n00[3], n01[3], n02[3], n10[3], n11[3], n20[3];
#pragma unroll
  for (int kz = 0; kz < 3; ++kz) {
    const int l = 3 * kz;  // lines cy = -1, 0, 1 at l, l+1, l+2
    n02[kz] = vadd(m0[l + 2], m0[l]);      // sum cy^2 f
    n01[kz] = vsub(m0[l + 2], m0[l]);      // sum cy f
    n00[kz] = vadd(n02[kz], m0[l + 1]);    // sum f
    n11[kz] = vsub(m1[l + 2], m1[l]);      // sum cx cy f
    n10[kz] = vadd(vadd(m1[l + 2], m1[l]), m1[l + 1]);  // sum cx f
    n20[kz] = vadd(vadd(m2[l + 2], m2[l]), m2[l + 1]);  // sum cx^2 f
  }
  const V Pzz = vadd(n00[2], n00[0]);
  const V p = vadd(Pzz, n00[1]);
  const V jz = vsub(n00[2], n00[0]);
  const V jy = vadd(vadd(n01[2], n01[0]), n01[1]);
  const V Pyz = vsub(n01[2], n01[0]);
  const V Pyy = vadd(vadd(n02[2], n02[0]), n02[1]);
  const V jx = vadd(vadd(n10[2], n10[0]), n10[1]);
  const V Pxz = vsub(n10[2], n10[0]);
  const V Pxy = vadd(vadd(n11[2], n11[0]), n11[1]);
  const V Pxx = vadd(vadd(n20[2], n20[0]), n20[1]);

  // Every product and sum below is an explicit round-to-nearest operation
  // (vfma / vmul / vadd, never contracted), so that each kernel that
  // inlines the collision rounds it the same way.
  auto C = [](float c) { return splat<V>(c); };
  const V rho = vfma(C(k.drho), phi0, C(k.rho_g));
  const V mu = vfma(C(k.dmu), phi0, C(k.mu_g));
  const V inv_rho = vrcp(rho);
  const V nu = vmul(mu, inv_rho);
  const V omega = vrcp(vfma(C(3.0f), nu, C(0.5f)));
  const V grx = vmul(C(k.drho), gx), gry = vmul(C(k.drho), gy),
          grz = vmul(C(k.drho), gz);
  const V muphi = vfma(C(-k.kappa_phi), lap,
                       vmul(vmul(vmul(C(k.beta4), phi0), vadd(phi0, C(-1.0f))),
                            vadd(phi0, C(-0.5f))));
  const V p3 = vmul(p, C(1.0f / 3.0f));
  const V rb = vadd(rho, C(-k.rho_g));
  const V F0x = vfma(rb, C(k.gx), vfma(vneg(p3), grx, vmul(muphi, gx)));
  const V F0y = vfma(rb, C(k.gy), vfma(vneg(p3), gry, vmul(muphi, gy)));
  const V F0z = vfma(rb, C(k.gz), vfma(vneg(p3), grz, vmul(muphi, gz)));
  // predictor for the viscous correction (Eq. Fnu)
  const V a0x = vmul(F0x, inv_rho), a0y = vmul(F0y, inv_rho),
          a0z = vmul(F0z, inv_rho);
  const V u0x = vfma(C(0.5f), a0x, jx), u0y = vfma(C(0.5f), a0y, jy),
          u0z = vfma(C(0.5f), a0z, jz);
  // Q0 = Pi - p* c_s^2 I - u0 u0 + (u0 a0 + a0 u0) / 2
  auto qd = [](V P, V p3_, V uu_, V aa_) {
    return vfma(uu_, vadd(aa_, vneg(uu_)), vadd(P, vneg(p3_)));
  };
  auto qo = [](V P, V ua, V ub, V aa, V ab) {
    return vfma(splat<V>(0.5f), vfma(ua, ab, vmul(aa, ub)), vfma(vneg(ua), ub, P));
  };
  const V Q0xx = qd(Pxx, p3, u0x, a0x);
  const V Q0yy = qd(Pyy, p3, u0y, a0y);
  const V Q0zz = qd(Pzz, p3, u0z, a0z);
  const V Q0xy = qo(Pxy, u0x, u0y, a0x, a0y);
  const V Q0xz = qo(Pxz, u0x, u0z, a0x, a0z);
  const V Q0yz = qo(Pyz, u0y, u0z, a0y, a0z);
  const V cnu = vmul(vmul(C(-3.0f), nu), omega);
  auto dot3 = [](V a1, V b1, V a2, V b2, V a3, V b3) {
    return vfma(a3, b3, vfma(a2, b2, vmul(a1, b1)));
  };
  const V Fx = vfma(cnu, dot3(Q0xx, grx, Q0xy, gry, Q0xz, grz), F0x);
  const V Fy = vfma(cnu, dot3(Q0xy, grx, Q0yy, gry, Q0yz, grz), F0y);
  const V Fz = vfma(cnu, dot3(Q0xz, grx, Q0yz, gry, Q0zz, grz), F0z);
  const V ax = vmul(Fx, inv_rho), ay = vmul(Fy, inv_rho), az = vmul(Fz, inv_rho);
  const V ux = vfma(C(0.5f), ax, jx), uy = vfma(C(0.5f), ay, jy),
          uz = vfma(C(0.5f), az, jz);
  const V Axx = qd(Pxx, p3, ux, ax);
  const V Ayy = qd(Pyy, p3, uy, ay);
  const V Azz = qd(Pzz, p3, uz, az);
  const V Axy = qo(Pxy, ux, uy, ax, ay);
  const V Axz = qo(Pxz, ux, uz, ax, az);
  const V Ayz = qo(Pyz, uy, uz, ay, az);
  const V tr = vadd(vadd(Axx, Ayy), Azz);
  const V vx = dot3(Axx, ux, Axy, uy, Axz, uz);
  const V vy = dot3(Axy, ux, Ayy, uy, Ayz, uz);
  const V vz = dot3(Axz, ux, Ayz, uy, Azz, uz);
  const V uu = dot3(ux, ux, uy, uy, uz, uz);
  const V ua = dot3(ux, ax, uy, ay, uz, az);
  const V om45 = vmul(C(4.5f), vadd(C(1.0f), vneg(omega)));
  const V k1 = vfma(vneg(vmul(om45, tr)), C(1.0f / 3.0f),
                    vfma(C(-1.5f), vadd(uu, ua), p));
  const V k2 = vfma(vneg(om45), tr, vfma(C(-4.5f), uu, C(3.0f)));

  // coefficients of P in the separable monomials
  const V om3 = vmul(C(3.0f), om45), om6 = vmul(C(6.0f), om45),
          om2 = vmul(C(2.0f), om45);
  auto coefD = [&](V u_, V a_, V A_) {
    return vfma(om45, A_, vmul(vmul(C(4.5f), u_), vadd(u_, a_)));
  };
  auto coefG = [&](V u_, V A_) {
    return vfma(om3, A_, vmul(vmul(C(13.5f), u_), u_));
  };
  auto coefL = [&](V u_, V a_, V A_, V v_) {
    const V in = vfma(om3, A_, vfma(vmul(C(4.5f), u_), u_, k2));
    return vfma(C(1.5f), a_, vfma(vneg(om2), v_, vmul(u_, in)));
  };
  auto coefF = [&](V ua_, V ub_, V aa_, V ab_, V A_) {
    return vfma(C(4.5f), vfma(ua_, ab_, vmul(ub_, aa_)),
                vfma(om2, A_, vmul(vmul(C(9.0f), ua_), ub_)));
  };
  const V Dx = coefD(ux, ax, Axx), Dy = coefD(uy, ay, Ayy), Dz = coefD(uz, az, Azz);
  const V Gx = coefG(ux, Axx), Gy = coefG(uy, Ayy), Gz = coefG(uz, Azz);
  const V Lx = coefL(ux, ax, Axx, vx);
  const V Ly = coefL(uy, ay, Ayy, vy);
  const V Lz = coefL(uz, az, Azz, vz);
  const V Fxy = coefF(ux, uy, ax, ay, Axy);
  const V Fxz = coefF(ux, uz, ax, az, Axz);
  const V Fyz = coefF(uy, uz, ay, az, Ayz);
  const V Hxy = vmul(om6, Axy), Hxz = vmul(om6, Axz), Hyz = vmul(om6, Ayz);
  const V Mxy = vfma(ux, Hxy, vmul(uy, Gx));  // e_x c_y
  const V Mxz = vfma(ux, Hxz, vmul(uz, Gx));  // e_x c_z
  const V Myx = vfma(uy, Hxy, vmul(ux, Gy));  // e_y c_x
  const V Myz = vfma(uy, Hyz, vmul(uz, Gy));  // e_y c_z
  const V Mzx = vfma(uz, Hxz, vmul(ux, Gz));  // e_z c_x
  const V Mzy = vfma(uz, Hyz, vmul(uy, Gz));  // e_z c_y
  const V X = vfma(om6, dot3(ux, Ayz, uy, Axz, uz, Axy),
                   vmul(vmul(vmul(C(27.0f), ux), uy), uz));

  cf.k1 = k1; cf.Lx = Lx; cf.Ly = Ly; cf.Lz = Lz;
  cf.Dx = Dx; cf.Dy = Dy; cf.Dz = Dz;
  cf.Fxy = Fxy; cf.Fxz = Fxz; cf.Fyz = Fyz;
  cf.Mxy = Mxy; cf.Mxz = Mxz; cf.Myx = Myx; cf.Myz = Myz; cf.Mzx = Mzx; cf.Mzy = Mzy;
  cf.X = X;
  uxo = ux;
  uyo = uy;
  uzo = uz;
}

template <typename V>
__device__ __forceinline__ void collide(const V (&f)[Q], V phi0, V gx, V gy,
                                        V gz, V lap, const Consts& k,
                                        NodeOut<V>& o) {
  Coefs<V> cf;
  collide_coefs(f, phi0, gx, gy, gz, lap, k, cf, o.ux, o.uy, o.uz);
  coefs_to_P(cf, o.P);
}

// Laplacian of Eq. lap_iso from the neighbour sum: 6 (ssum - (1 - w_0) phi).
template <typename V>
__device__ __forceinline__ V lap_from_sum(V phi0, V ssum) {
  return vmul(splat<V>(6.0f), vfma(splat<V>(-(1.0f - wq(REST))), phi0, ssum));
}

// Everything after the pull and the phi stencil of one node: the
// Laplacian, the compressive vector a and the collision.
template <typename V>
__device__ __forceinline__ void node_eval(const V (&f)[Q], V phi0, V gx, V gy,
                                          V gz, V ssum, const Consts& k,
                                          NodeOut<V>& o, V& ax, V& ay, V& az) {
  const V lap = lap_from_sum(phi0, ssum);
  compressive(phi0, gx, gy, gz, ax, ay, az);
  collide(f, phi0, gx, gy, gz, lap, k, o);
}

// Stores of one node's f*, u and a.
template <typename Store, typename IDX>
__device__ __forceinline__ void node_store(IDX n, IDX N, const NodeOut<float>& o,
                                           float ax, float ay, float az,
                                           typename Store::T* __restrict__ fout,
                                           float* __restrict__ u,
                                           float* __restrict__ a) {
  a[n] = ax;
  a[N + n] = ay;
  a[2 * N + n] = az;
#pragma unroll
  for (int q = 0; q < Q; ++q) fout[q * N + n] = Store::encode_w(o.P[q], q);
  u[n] = o.ux;
  u[N + n] = o.uy;
  u[2 * N + n] = o.uz;
}

// Everything after the pull and the phi stencil: the compressive vector
// (written to a before the collision, so that it is not held across it),
// the collision, and the stores of f*, u.
template <typename Store, typename IDX>
__device__ __forceinline__ void lb_finish(IDX n, IDX N, const float (&f)[Q],
                                          float phi0, float gx, float gy,
                                          float gz, float ssum,
                                          typename Store::T* __restrict__ fout,
                                          float* __restrict__ u,
                                          float* __restrict__ a,
                                          const Consts& k) {
  const float lap = lap_from_sum(phi0, ssum);
  float ax, ay, az;
  compressive(phi0, gx, gy, gz, ax, ay, az);
  a[n] = ax;
  a[N + n] = ay;
  a[2 * N + n] = az;
  NodeOut<float> o;
  collide(f, phi0, gx, gy, gz, lap, k, o);
#pragma unroll
  for (int q = 0; q < Q; ++q) fout[q * N + n] = Store::encode_w(o.P[q], q);
  u[n] = o.ux;
  u[N + n] = o.uy;
  u[2 * N + n] = o.uz;
}

// Pull and phi stencil of the fluid node (x, y, z) of one grid, read from
// global memory (halfway bounce-back on links from solid nodes), then the
// node's evaluation. Returns false for a solid node (nothing evaluated).
// IDX is int when 27 N fits in 31 bits (every offset then needs one 32-bit
// multiply-add and one widening address computation), int64_t otherwise.
template <typename Store, typename IDX>
__device__ __forceinline__ bool lb_node_eval(int x, int y, int z,
                                             const typename Store::T* __restrict__ fin,
                                             const float* __restrict__ phi,
                                             const uint8_t* __restrict__ flags,
                                             const Grid& g, const Consts& k,
                                             NodeOut<float>& o, float& ax,
                                             float& ay, float& az) {
  const IDX nx = g.nx;
  const IDX nxy = (IDX)g.nx * g.ny;
  const IDX N = (IDX)g.N;
  const IDX n = x + nx * y + nxy * z;
  const uint8_t fl = flags[n];
  if (fl & FLAG_SOLID) return false;
  const IDX xo[3] = {(IDX)wrap(x, -1, g.nx), (IDX)x, (IDX)wrap(x, 1, g.nx)};
  const IDX yo[3] = {wrap(y, -1, g.ny) * nx, y * nx, wrap(y, 1, g.ny) * nx};
  const IDX zo[3] = {wrap(z, -1, g.nz) * nxy, z * nxy, wrap(z, 1, g.nz) * nxy};
  IDX yz[3][3];
#pragma unroll
  for (int b = 0; b < 3; ++b)
#pragma unroll
    for (int c = 0; c < 3; ++c) yz[b][c] = yo[b] + zo[c];

  float f[Q];
  if (fl & FLAG_NEAR) {
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const IDX src = xo[1 - cx(q)] + yz[1 - cy(q)][1 - cz(q)];
      const bool bb = (q != REST) && (__ldg(flags + src) & FLAG_SOLID);
      f[q] = Store::decode(bb ? __ldg(fin + (opp(q) * N + n)) : __ldg(fin + (q * N + src)), q);
    }
  } else {
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const IDX src = xo[1 - cx(q)] + yz[1 - cy(q)][1 - cz(q)];
      f[q] = Store::decode(__ldg(fin + (q * N + src)), q);
    }
  }

  // isotropic gradient and Laplacian of phi (Eqs. grad_iso, lap_iso)
  const float phi0 = __ldg(phi + n);
  float gx = 0.f, gy = 0.f, gz = 0.f, ssum = 0.f;
#pragma unroll
  for (int q = 0; q < REST; ++q) {
    const float vp = __ldg(phi + (xo[1 + cx(q)] + yz[1 + cy(q)][1 + cz(q)]));
    const float vm = __ldg(phi + (xo[1 - cx(q)] + yz[1 - cy(q)][1 - cz(q)]));
    stencil_pair(q, vp, vm, gx, gy, gz, ssum);
  }
  node_eval(f, phi0, gx, gy, gz, ssum, k, o, ax, ay, az);
  return true;
}

// The node (x, y, z) of one grid: pull, stencil, collision, stores.
template <typename Store, typename IDX>
__device__ __forceinline__ void lb_node(int x, int y, int z,
                                        const typename Store::T* __restrict__ fin,
                                        typename Store::T* __restrict__ fout,
                                        const float* __restrict__ phi,
                                        float* __restrict__ u,
                                        float* __restrict__ a,
                                        const uint8_t* __restrict__ flags,
                                        const Grid& g, const Consts& k) {
  const IDX nx = g.nx;
  const IDX nxy = (IDX)g.nx * g.ny;
  const IDX N = (IDX)g.N;
  const IDX n = x + nx * y + nxy * z;
  const uint8_t fl = flags[n];
  if (fl & FLAG_SOLID) return;
  const IDX xo[3] = {(IDX)wrap(x, -1, g.nx), (IDX)x, (IDX)wrap(x, 1, g.nx)};
  const IDX yo[3] = {wrap(y, -1, g.ny) * nx, y * nx, wrap(y, 1, g.ny) * nx};
  const IDX zo[3] = {wrap(z, -1, g.nz) * nxy, z * nxy, wrap(z, 1, g.nz) * nxy};
  IDX yz[3][3];
#pragma unroll
  for (int b = 0; b < 3; ++b)
#pragma unroll
    for (int c = 0; c < 3; ++c) yz[b][c] = yo[b] + zo[c];

  float f[Q];
  if (fl & FLAG_NEAR) {
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const IDX src = xo[1 - cx(q)] + yz[1 - cy(q)][1 - cz(q)];
      const bool bb = (q != REST) && (__ldg(flags + src) & FLAG_SOLID);
      f[q] = Store::decode(bb ? __ldg(fin + (opp(q) * N + n)) : __ldg(fin + (q * N + src)), q);
    }
  } else {
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const IDX src = xo[1 - cx(q)] + yz[1 - cy(q)][1 - cz(q)];
      f[q] = Store::decode(__ldg(fin + (q * N + src)), q);
    }
  }

  // isotropic gradient and Laplacian of phi (Eqs. grad_iso, lap_iso)
  const float phi0 = __ldg(phi + n);
  float gx = 0.f, gy = 0.f, gz = 0.f, ssum = 0.f;
#pragma unroll
  for (int q = 0; q < REST; ++q) {
    const float vp = __ldg(phi + (xo[1 + cx(q)] + yz[1 + cy(q)][1 + cz(q)]));
    const float vm = __ldg(phi + (xo[1 - cx(q)] + yz[1 - cy(q)][1 - cz(q)]));
    stencil_pair(q, vp, vm, gx, gy, gz, ssum);
  }
  lb_finish<Store, IDX>(n, N, f, phi0, gx, gy, gz, ssum, fout, u, a, k);
}

// Isotropic gradient and neighbour sum (Eqs. grad_iso, lap_iso) of an x
// pair of nodes (x0, x0 + 1) from the 9 phi rows of its stencil, each row
// given as (phi(x0 - 1), (phi(x0), phi(x0 + 1)), phi(x0 + 2)), rows indexed
// [dy + 1][dz + 1]; packed pair arithmetic, bit-identical to the one-node
// stencil on each node.
__device__ __forceinline__ void pair_stencil(const float2 (&pc)[3][3],
                                             const float (&pl)[3][3],
                                             const float (&pr)[3][3], float2& phi0,
                                             float2& gx, float2& gy, float2& gz,
                                             float2& ssum) {
  // phi at x + d for both nodes of the pair, d = -1, 0, +1
  auto shifted = [&](int b, int c, int d) {
    return d == 0 ? pc[b][c]
         : d > 0 ? make_float2(pc[b][c].y, pr[b][c])
                 : make_float2(pl[b][c], pc[b][c].x);
  };
  phi0 = pc[1][1];
  gx = make_float2(0.f, 0.f);
  gy = gx;
  gz = gx;
  ssum = gx;
#pragma unroll
  for (int q = 0; q < REST; ++q) {
    const float2 vp = shifted(1 + cy(q), 1 + cz(q), cx(q));
    const float2 vm = shifted(1 - cy(q), 1 - cz(q), -cx(q));
    stencil_pair(q, vp, vm, gx, gy, gz, ssum);
  }
}

// The whole evaluation of such a pair (stencil, compressive vector,
// collision) from its 27 pulled population pairs.
__device__ __forceinline__ void pair_eval(const float2 (&f)[Q],
                                          const float2 (&pc)[3][3],
                                          const float (&pl)[3][3],
                                          const float (&pr)[3][3],
                                          const Consts& k, NodeOut<float2>& o,
                                          float2& ax, float2& ay, float2& az) {
  float2 phi0, gx, gy, gz, ssum;
  pair_stencil(pc, pl, pr, phi0, gx, gy, gz, ssum);
  node_eval(f, phi0, gx, gy, gz, ssum, k, o, ax, ay, az);
}

// An x pair of nodes (x0, x0 + 1), x0 even, both fluid and away from walls:
// pull, stencil, collision and stores with two nodes per thread, the
// arithmetic in packed pair operations. Loads and stores of the pair are
// one aligned access per population, phi row and field; the pulled
// populations of the links with c_x = +1 (-1) take the element left of
// (right of) the pair from a second load, with the periodic wrap in x.
// Bit-identical to lb_node on each node.
template <typename Store>
__device__ __forceinline__ void lb_pair(int x0, int y, int z,
                                        const typename Store::T* __restrict__ fin,
                                        typename Store::T* __restrict__ fout,
                                        const float* __restrict__ phi,
                                        float* __restrict__ u,
                                        float* __restrict__ a, const Grid& g,
                                        const Consts& k) {
  using T = typename Store::T;
  using T2 = typename Store::T2;
  const int nx = g.nx;
  const int nxy = g.nx * g.ny;
  const int N = (int)g.N;
  const int n = x0 + nx * y + nxy * z;
  // the element left of the pair and the one right of it (x wraps)
  const int xl = (x0 == 0) ? nx - 1 : x0 - 1;
  const int xr = (x0 + 2 == nx) ? 0 : x0 + 2;
  const int yo[3] = {wrap(y, -1, g.ny) * nx, y * nx, wrap(y, 1, g.ny) * nx};
  const int zo[3] = {wrap(z, -1, g.nz) * nxy, z * nxy, wrap(z, 1, g.nz) * nxy};

  // phi stencil first: its rows are dead before the populations arrive
  float2 phi0, gx, gy, gz, ssum;
  {
    float2 pc[3][3];
    float pl[3][3], pr[3][3];
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const int row = yo[b] + zo[c];
        pc[b][c] = __ldg(reinterpret_cast<const float2*>(phi + row + x0));
        pl[b][c] = __ldg(phi + row + xl);
        pr[b][c] = __ldg(phi + row + xr);
      }
    pair_stencil(pc, pl, pr, phi0, gx, gy, gz, ssum);
  }

  // pulled populations f*_q(x - c_q) of both nodes
  float2 f[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const T* src = fin + q * N + yo[1 - cy(q)] + zo[1 - cz(q)];
    const T2 own = __ldg(reinterpret_cast<const T2*>(src + x0));
    T2 v;
    if (cx(q) == 0)
      v = own;
    else if (cx(q) > 0)
      v = Store::pack(__ldg(src + xl), Store::lo(own));
    else
      v = Store::pack(Store::hi(own), __ldg(src + xr));
    f[q] = Store::decode2(v, q);
  }

  float2 ax, ay, az;
  compressive(phi0, gx, gy, gz, ax, ay, az);
  *reinterpret_cast<float2*>(a + n) = ax;
  *reinterpret_cast<float2*>(a + N + n) = ay;
  *reinterpret_cast<float2*>(a + 2 * N + n) = az;
  NodeOut<float2> o;
  collide(f, phi0, gx, gy, gz, lap_from_sum(phi0, ssum), k, o);
#pragma unroll
  for (int q = 0; q < Q; ++q)
    *reinterpret_cast<T2*>(fout + q * N + n) = Store::encode_w2(o.P[q], q);
  *reinterpret_cast<float2*>(u + n) = o.ux;
  *reinterpret_cast<float2*>(u + N + n) = o.uy;
  *reinterpret_cast<float2*>(u + 2 * N + n) = o.uz;
}

// mbarrier and bulk-copy primitives (PTX): a CTA-local barrier that counts
// one arrival plus the bytes of the copies registered on it.
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)),
               "r"(count)
               : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile(
      "mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)),
      "r"(bytes)
      : "memory");
}
// One test of phase `parity` of the barrier.
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n"
      " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Nanoseconds of the GPU's global timer.
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait for phase `parity` of the barrier, sleeping between tests
// so that a waiting warp leaves the issue slots to the others: false once
// 0.5 s have passed on the global timer (or after 2^22 tests, whichever
// comes first, whatever time one test takes).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint64_t t0 = global_ns();
  for (int i = 0; i < (1 << 22); ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > 500000000ull) return false;
    __nanosleep(200);
  }
  return false;
}
// bytes (a multiple of 16) from global src to shared dst (both 16-byte
// aligned), completing on bar
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src,
                                         uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes "
      "[%0], [%1], %2, [%3];\n" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Copy-staged collide-stream. A row segment is up to SEG nodes x0 .. x0+L-1
// of row y, plane z. The 27 population rows it pulls from (row y - c_y of
// plane z - c_z, shifted by c_x) and the 9 phi rows of its stencil
// (y + dy, z + dz) arrive in shared memory, each as one bulk asynchronous
// copy of its run x0 .. x0+L-1 (completed on an mbarrier) and its two
// neighbours x0-1 and x0+L (x wraps periodically) loaded by the thread that
// owns the row.
// Persistent blocks walk the segments (block b takes b, b + G, ...) through
// a two-stage ring: the copies of the next segment are in flight while the
// current one is computed. The arithmetic is lb_node's, in the same order.
// Requires nx a multiple of 16 / sizeof(T) and of 4 (16-byte aligned runs).
constexpr int SEG = 128;

template <typename Store>
struct StagedRows {
  using T = typename Store::T;
  static constexpr int PF = 16 / (int)sizeof(T);  // pad of a population row
  static constexpr int FW = SEG + 2 * PF;
  static constexpr int PW = SEG + 8;              // phi rows, pad 4
  T f[Q][FW];
  float p[9][PW];
};

struct Segment {
  int x0, y, z, L;
};

__device__ __forceinline__ Segment segment_of(int s, const Grid& g) {
  const int nsx = (g.nx + SEG - 1) / SEG;
  const int row = s / nsx;
  Segment r;
  r.x0 = (s - row * nsx) * SEG;
  r.y = row % g.ny;
  r.z = row / g.ny;
  r.L = min(SEG, g.nx - r.x0);
  return r;
}

template <typename Store>
__device__ __forceinline__ uint32_t staged_bytes(int L) {
  return (uint32_t)(Q * L * sizeof(typename Store::T) + 9 * L * sizeof(float));
}

// Thread tid < 36 owns one row of segment sg: it issues the bulk copy of
// the run x0 .. x0+L-1 into stage st and loads the row's neighbours x0-1
// and x0+L (returned in fl_ / fr_ or pl / pr; staged_pads stores them).
template <typename Store, typename IDX>
__device__ __forceinline__ void staged_issue(StagedRows<Store>& st, uint64_t* bar,
                                             const Segment& sg, int tid,
                                             const typename Store::T* fin,
                                             const float* phi, const Grid& g,
                                             typename Store::T& fl_, typename Store::T& fr_,
                                             float& pl, float& pr) {
  using R = StagedRows<Store>;
  using T = typename Store::T;
  const IDX nx = g.nx;
  const IDX nxy = (IDX)g.nx * g.ny;
  const int x0 = sg.x0, L = sg.L;
  const int xl = (x0 == 0) ? g.nx - 1 : x0 - 1;
  const int xr = (x0 + L == g.nx) ? 0 : x0 + L;
  if (tid < Q) {  // population row q from (y - c_y, z - c_z)
    const int q = tid;
    const IDX base = (IDX)q * (IDX)g.N + (IDX)wrap(sg.z, -cz(q), g.nz) * nxy +
                     (IDX)wrap(sg.y, -cy(q), g.ny) * nx;
    bulk_g2s(&st.f[q][R::PF], fin + base + x0, (uint32_t)(L * sizeof(T)), bar);
    fl_ = __ldg(fin + base + xl);
    fr_ = __ldg(fin + base + xr);
  } else if (tid < Q + 9) {  // phi row (y + dy, z + dz)
    const int j = tid - Q;
    const IDX base = (IDX)wrap(sg.z, j / 3 - 1, g.nz) * nxy +
                     (IDX)wrap(sg.y, j % 3 - 1, g.ny) * nx;
    bulk_g2s(&st.p[j][4], phi + base + x0, (uint32_t)(L * sizeof(float)), bar);
    pl = __ldg(phi + base + xl);
    pr = __ldg(phi + base + xr);
  }
}

// Store the wrap neighbours loaded by staged_issue next to the run.
template <typename Store>
__device__ __forceinline__ void staged_pads(StagedRows<Store>& st, int L, int tid,
                                            typename Store::T fl_,
                                            typename Store::T fr_, float pl,
                                            float pr) {
  using R = StagedRows<Store>;
  if (tid < Q) {
    st.f[tid][R::PF - 1] = fl_;
    st.f[tid][R::PF + L] = fr_;
  } else if (tid < Q + 9) {
    st.p[tid - Q][3] = pl;
    st.p[tid - Q][4 + L] = pr;
  }
}

template <typename Store, typename IDX>
__global__ void __launch_bounds__(SEG)
lb_collide_staged(const typename Store::T* __restrict__ fin,
                  typename Store::T* __restrict__ fout,
                  const float* __restrict__ phi, float* __restrict__ u,
                  float* __restrict__ a, const uint8_t* __restrict__ flags,
                  Grid g, Consts k, int nseg, unsigned* __restrict__ wait_err) {
  // wait_err[0]: set when a wait gave up; wait_err[1]: test request
  // (cacl_inject_copy_stall) to register 16 bytes more for the first
  // segment than its copies deliver, so that its wait cannot complete
  using R = StagedRows<Store>;
  extern __shared__ __align__(16) unsigned char lb_smem[];
  R* st = reinterpret_cast<R*>(lb_smem);  // [2]
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ int s_fail;

  const int tid = threadIdx.x;
  const int G = gridDim.x;
  const IDX nx = g.nx;
  const IDX nxy = (IDX)g.nx * g.ny;
  const IDX N = (IDX)g.N;
  int s = blockIdx.x;
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    s_fail = 0;
    if (s < nseg)
      mbar_arrive_expect_tx(&bar[0], staged_bytes<Store>(segment_of(s, g).L) +
                                         (wait_err[1] ? 16u : 0u));
    if (s + G < nseg)
      mbar_arrive_expect_tx(&bar[1], staged_bytes<Store>(segment_of(s + G, g).L));
  }
  __syncthreads();
  using T = typename Store::T;
  T fl_ = T(), fr_ = T();
  float pl = 0.f, pr = 0.f;
  if (s < nseg) {
    const Segment s0 = segment_of(s, g);
    staged_issue<Store, IDX>(st[0], &bar[0], s0, tid, fin, phi, g, fl_, fr_, pl, pr);
    staged_pads<Store>(st[0], s0.L, tid, fl_, fr_, pl, pr);
  }
  __syncthreads();

  for (int i = 0; s < nseg; ++i, s += G) {
    const int cur = i & 1;
    // the copies of the next segment (its bytes were registered before the
    // last block barrier, and its stage was last read before it); its wrap
    // neighbours are stored at the end of this step
    const Segment nxt = segment_of(s + G < nseg ? s + G : s, g);
    if (s + G < nseg)
      staged_issue<Store, IDX>(st[cur ^ 1], &bar[cur ^ 1], nxt, tid, fin, phi, g,
                               fl_, fr_, pl, pr);
    const bool arrived = mbar_wait(&bar[cur], (i >> 1) & 1);
    if (!arrived) {
      s_fail = 1;
      atomicOr(wait_err, 1u);
    }
    const Segment sg = segment_of(s, g);
    const R& sr = st[cur];
    if (tid < sg.L) {
      const int x = sg.x0 + tid;
      const IDX n = x + nx * sg.y + nxy * sg.z;
      const uint8_t fl = flags[n];
      if (!(fl & FLAG_SOLID)) {
        float f[Q];
        if (fl & FLAG_NEAR) {
          const int y = sg.y, z = sg.z;
          const IDX xo[3] = {(IDX)wrap(x, -1, g.nx), (IDX)x, (IDX)wrap(x, 1, g.nx)};
          const IDX yo[3] = {wrap(y, -1, g.ny) * nx, y * nx, wrap(y, 1, g.ny) * nx};
          const IDX zo[3] = {wrap(z, -1, g.nz) * nxy, z * nxy, wrap(z, 1, g.nz) * nxy};
#pragma unroll
          for (int q = 0; q < Q; ++q) {
            const IDX src = xo[1 - cx(q)] + yo[1 - cy(q)] + zo[1 - cz(q)];
            const bool bb = (q != REST) && (__ldg(flags + src) & FLAG_SOLID);
            f[q] = Store::decode(
                bb ? __ldg(fin + (opp(q) * N + n)) : sr.f[q][R::PF + tid - cx(q)], q);
          }
        } else {
#pragma unroll
          for (int q = 0; q < Q; ++q)
            f[q] = Store::decode(sr.f[q][R::PF + tid - cx(q)], q);
        }
        // isotropic gradient and Laplacian of phi (Eqs. grad_iso, lap_iso);
        // phi row j holds (y + j % 3 - 1, z + j / 3 - 1)
        const float phi0 = sr.p[4][4 + tid];
        float gx = 0.f, gy = 0.f, gz = 0.f, ssum = 0.f;
#pragma unroll
        for (int q = 0; q < REST; ++q) {
          const float vp = sr.p[(1 + cy(q)) + 3 * (1 + cz(q))][4 + tid + cx(q)];
          const float vm = sr.p[(1 - cy(q)) + 3 * (1 - cz(q))][4 + tid - cx(q)];
          stencil_pair(q, vp, vm, gx, gy, gz, ssum);
        }
        lb_finish<Store, IDX>(n, N, f, phi0, gx, gy, gz, ssum, fout, u, a, k);
      }
    }
    // register the bytes of the segment after next, whose copies go to this
    // stage once every thread is past the barrier below (not after a wait
    // that gave up: the barrier's phase is still open, and a second arrival
    // on it is not allowed)
    if (tid == 0 && arrived && s + 2 * G < nseg)
      mbar_arrive_expect_tx(&bar[cur], staged_bytes<Store>(segment_of(s + 2 * G, g).L));
    if (s + G < nseg) staged_pads<Store>(st[cur ^ 1], nxt.L, tid, fl_, fr_, pl, pr);
    __syncthreads();
    if (s_fail) {
      // stop; the copies still in flight target this block
      if (tid == 0 && s + G < nseg) mbar_wait(&bar[cur ^ 1], ((i + 1) >> 1) & 1);
      return;
    }
  }
}

template <typename Store, typename IDX>
__global__ void __launch_bounds__(LB_BX * LB_BY)
lb_collide(const typename Store::T* __restrict__ fin,
           typename Store::T* __restrict__ fout, const float* __restrict__ phi,
           float* __restrict__ u, float* __restrict__ a,
           const uint8_t* __restrict__ flags, Grid g, Consts k) {
  const int x = blockIdx.x * LB_BX + threadIdx.x;
  const int y = blockIdx.y * LB_BY + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= g.nx || y >= g.ny) return;
  lb_node<Store, IDX>(x, y, z, fin, fout, phi, u, a, flags, g, k);
}

// Four x-adjacent nodes per thread for 16-bit populations (nx a multiple
// of 4): one 8-byte load per population of the quad (its pairs A = (x0,
// x0+1) and B = (x0+2, x0+3)), the element left of and right of the quad
// from 2-byte loads (x wraps), one 16-byte load per phi row, and one
// 8-byte store per population of the quad (both pairs together). Each pair
// is evaluated exactly as in lb_pair, so the result is bit-identical; the
// address arithmetic of a population, phi row or field serves four nodes.
template <typename Store>
__device__ __forceinline__ void lb_quad(int x0, int y, int z,
                                        const typename Store::T* __restrict__ fin,
                                        typename Store::T* __restrict__ fout,
                                        const float* __restrict__ phi,
                                        float* __restrict__ u,
                                        float* __restrict__ a, const Grid& g,
                                        const Consts& k) {
  using T = typename Store::T;
  using T2 = typename Store::T2;
  const int nx = g.nx;
  const int nxy = g.nx * g.ny;
  const int N = (int)g.N;
  const int n = x0 + nx * y + nxy * z;
  const int xl = (x0 == 0) ? nx - 1 : x0 - 1;
  const int xr = (x0 + 4 == nx) ? 0 : x0 + 4;
  const int yo[3] = {wrap(y, -1, g.ny) * nx, y * nx, wrap(y, 1, g.ny) * nx};
  const int zo[3] = {wrap(z, -1, g.nz) * nxy, z * nxy, wrap(z, 1, g.nz) * nxy};

  // phi stencils of both pairs
  float2 phiA, gxA, gyA, gzA, ssA, phiB, gxB, gyB, gzB, ssB;
  {
    float2 pcA[3][3], pcB[3][3];
    float plA[3][3], prA[3][3], plB[3][3], prB[3][3];
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const int row = yo[b] + zo[c];
        const float4 v = __ldg(reinterpret_cast<const float4*>(phi + row + x0));
        pcA[b][c] = make_float2(v.x, v.y);
        pcB[b][c] = make_float2(v.z, v.w);
        plA[b][c] = __ldg(phi + row + xl);
        prA[b][c] = v.z;
        plB[b][c] = v.y;
        prB[b][c] = __ldg(phi + row + xr);
      }
    pair_stencil(pcA, plA, prA, phiA, gxA, gyA, gzA, ssA);
    pair_stencil(pcB, plB, prB, phiB, gxB, gyB, gzB, ssB);
  }

  // pulled populations: pair A decoded, pair B kept packed until A is done
  float2 fA[Q];
  T2 hB[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const T* src = fin + q * N + yo[1 - cy(q)] + zo[1 - cz(q)];
    const uint2 w = __ldg(reinterpret_cast<const uint2*>(src + x0));
    const T2 w0 = *reinterpret_cast<const T2*>(&w.x);
    const T2 w1 = *reinterpret_cast<const T2*>(&w.y);
    T2 vA;
    if (cx(q) == 0) {
      vA = w0;
      hB[q] = w1;
    } else if (cx(q) > 0) {
      vA = Store::pack(__ldg(src + xl), Store::lo(w0));
      hB[q] = Store::pack(Store::hi(w0), Store::lo(w1));
    } else {
      vA = Store::pack(Store::hi(w0), Store::lo(w1));
      hB[q] = Store::pack(Store::hi(w1), __ldg(src + xr));
    }
    fA[q] = Store::decode2(vA, q);
  }

  float2 axA, ayA, azA;
  compressive(phiA, gxA, gyA, gzA, axA, ayA, azA);
  float2 uxA, uyA, uzA;
  T2 eA[Q];  // pair A's encoded f*, stored with pair B's as one 8-byte word
  {
    NodeOut<float2> o;
    collide(fA, phiA, gxA, gyA, gzA, lap_from_sum(phiA, ssA), k, o);
#pragma unroll
    for (int q = 0; q < Q; ++q) eA[q] = Store::encode_w2(o.P[q], q);
    uxA = o.ux;
    uyA = o.uy;
    uzA = o.uz;
  }
  float2 axB, ayB, azB;
  compressive(phiB, gxB, gyB, gzB, axB, ayB, azB);
  *reinterpret_cast<float4*>(a + n) = make_float4(axA.x, axA.y, axB.x, axB.y);
  *reinterpret_cast<float4*>(a + N + n) = make_float4(ayA.x, ayA.y, ayB.x, ayB.y);
  *reinterpret_cast<float4*>(a + 2 * N + n) = make_float4(azA.x, azA.y, azB.x, azB.y);
  {
    float2 fB[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) fB[q] = Store::decode2(hB[q], q);
    NodeOut<float2> o;
    collide(fB, phiB, gxB, gyB, gzB, lap_from_sum(phiB, ssB), k, o);
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const T2 eB = Store::encode_w2(o.P[q], q);
      uint2 w;
      w.x = *reinterpret_cast<const uint32_t*>(&eA[q]);
      w.y = *reinterpret_cast<const uint32_t*>(&eB);
      *reinterpret_cast<uint2*>(fout + q * N + n) = w;
    }
    *reinterpret_cast<float4*>(u + n) = make_float4(uxA.x, uxA.y, o.ux.x, o.ux.y);
    *reinterpret_cast<float4*>(u + N + n) = make_float4(uyA.x, uyA.y, o.uy.x, o.uy.y);
    *reinterpret_cast<float4*>(u + 2 * N + n) = make_float4(uzA.x, uzA.y, o.uz.x, o.uz.y);
  }
}

// Block (LBQ_PX, LBQ_PY): 4 LBQ_PX nodes of LBQ_PY rows. A quad with a solid
// node or a wall neighbour runs the one-node path on each node. Bounded to
// 128 registers (eight blocks of 64 threads per SM; ptxas spills about 70
// bytes). FP16 at 256^3: 0.464 ms per launch (BF16 0.459); before the
// shifted pairs were assembled on the bits, 0.474 here against 0.479 with
// four blocks of 128 threads and 0.474 at 168 registers (BF16 0.513 there,
// 0.480 here), and 0.511 when each pair's populations were stored as soon
// as the pair was done (4-byte stores) rather than together (8-byte stores).
constexpr int LBQ_PX = 32;
constexpr int LBQ_PY = 2;
template <typename Store>
__global__ void __launch_bounds__(LBQ_PX * LBQ_PY, 8)
lb_collide_quad(const typename Store::T* __restrict__ fin,
                typename Store::T* __restrict__ fout, const float* __restrict__ phi,
                float* __restrict__ u, float* __restrict__ a,
                const uint8_t* __restrict__ flags, Grid g, Consts k) {
  const int x0 = 4 * (blockIdx.x * LBQ_PX + threadIdx.x);
  const int y = blockIdx.y * LBQ_PY + threadIdx.y;
  const int z = blockIdx.z;
  if (x0 >= g.nx || y >= g.ny) return;
  const int n = x0 + g.nx * (y + g.ny * z);
  const uchar4 fl = *reinterpret_cast<const uchar4*>(flags + n);
  if (((fl.x | fl.y | fl.z | fl.w) & (FLAG_SOLID | FLAG_NEAR)) == 0) {
    lb_quad<Store>(x0, y, z, fin, fout, phi, u, a, g, k);
    return;
  }
#pragma unroll 1
  for (int j = 0; j < 4; ++j)
    lb_node<Store, int>(x0 + j, y, z, fin, fout, phi, u, a, flags, g, k);
}

// Two nodes per thread: block (LB2_PX, LB2_PY) covers 2 LB2_PX nodes of
// LB2_PY rows of one plane. A pair with a solid node or a wall neighbour
// (bounce-back links) runs the one-node path for each of its nodes.
template <typename Store>
__device__ __forceinline__ void lb_pair_block(const typename Store::T* __restrict__ fin,
                                              typename Store::T* __restrict__ fout,
                                              const float* __restrict__ phi,
                                              float* __restrict__ u,
                                              float* __restrict__ a,
                                              const uint8_t* __restrict__ flags,
                                              const Grid& g, const Consts& k) {
  const int x0 = 2 * (blockIdx.x * LB2_PX + threadIdx.x);
  const int y = blockIdx.y * LB2_PY + threadIdx.y;
  const int z = blockIdx.z;
  if (x0 >= g.nx || y >= g.ny) return;
  const int n = x0 + g.nx * (y + g.ny * z);
  const uchar2 fl = *reinterpret_cast<const uchar2*>(flags + n);
  if (((fl.x | fl.y) & (FLAG_SOLID | FLAG_NEAR)) == 0) {
    lb_pair<Store>(x0, y, z, fin, fout, phi, u, a, g, k);
  } else {
#pragma unroll 1
    for (int j = 0; j < 2; ++j)
      lb_node<Store, int>(x0 + j, y, z, fin, fout, phi, u, a, flags, g, k);
  }
}

// FP32 populations: at most 80 registers (six blocks of 128 per SM; 4 bytes
// of spills): 0.625 ms per 256^3 launch against 0.647 at 96 registers (five
// blocks, no spills), 0.707 at 128 and 0.725 at 72 (seven blocks, 120 bytes
// of spills). 16-bit populations (the two-node form runs when nx is 2 mod
// 4): six blocks as well, FP16 at 250^3 0.494 ms per launch against 0.521
// at the compiler's own 96 registers (BF16 0.488 against 0.494).
template <typename Store>
__global__ void __launch_bounds__(LB2_PX * LB2_PY, 6)
lb_collide_pair32(const typename Store::T* __restrict__ fin,
                  typename Store::T* __restrict__ fout, const float* __restrict__ phi,
                  float* __restrict__ u, float* __restrict__ a,
                  const uint8_t* __restrict__ flags, Grid g, Consts k) {
  lb_pair_block<Store>(fin, fout, phi, u, a, flags, g, k);
}

template <typename Store>
__global__ void __launch_bounds__(LB2_PX * LB2_PY, 6)
lb_collide_pair16(const typename Store::T* __restrict__ fin,
                  typename Store::T* __restrict__ fout, const float* __restrict__ phi,
                  float* __restrict__ u, float* __restrict__ a,
                  const uint8_t* __restrict__ flags, Grid g, Consts k) {
  lb_pair_block<Store>(fin, fout, phi, u, a, flags, g, k);
}

// TMA-tiled collide-stream (CACL_OPT_LB_PIPE = 3). A tile is TX consecutive
// nodes of one row (x0 .. x0 + TX - 1, row y, plane z), two nodes per
// thread, one tile per block. The tensor memory accelerator copies into
// shared memory, completing on an mbarrier: for each of the 9 (c_y, c_z)
// lines the three population rows q = 3 l .. 3 l + 2 of source row
// (y - c_y, z - c_z), columns x0 - PAD .. x0 + TX + PAD - 1 (PAD = 16 bytes
// of elements, so that every copy starts on a 16-byte boundary), and the 9
// phi rows (y + dy, z + dz), columns x0 - 4 .. x0 + TX + 3; the 18 copies
// are issued by 18 lanes of the first warp. y and z wrap through the copy
// coordinates; the elements left of x = 0 and right of x = nx - 1 come back
// as the fill value and the block patches the two it needs from global
// memory. Every thread reads its pair's operands at fixed offsets from one
// shared address (no per-element address arithmetic), evaluates the pair
// (pair_eval) and writes f*, u and a into an output tile, which one thread
// stores with three tensor copies. Pairs with a solid node or a wall
// neighbour read global memory (lb_node_eval); solid nodes get f* = 0,
// u = 0, a = 0. Bit-identical to lb_node at fluid nodes.
template <typename Store, int TX>
struct TmaTile {
  using T = typename Store::T;
  static constexpr int ES = (int)sizeof(T);
  static constexpr int PAD = 16 / ES;
  static constexpr int W = TX + 2 * PAD;                         // row, elements
  static constexpr int LINE_B = (3 * W * ES + 127) / 128 * 128;  // 3 rows of a line
  static constexpr int PADP = 4;
  static constexpr int WP = TX + 2 * PADP;
  static constexpr int ROWP_B = (WP * 4 + 127) / 128 * 128;
  static constexpr int IN_B = 9 * LINE_B + 9 * ROWP_B;
  static constexpr int OUTF_B = Q * TX * ES;                     // f* of the tile
  static constexpr int OUTV_B = 3 * TX * 4;                      // u or a
  static constexpr int SMEM_B = IN_B + OUTF_B + 2 * OUTV_B + 64;
  static constexpr uint32_t TX_BYTES = 27u * W * ES + 9u * WP * 4;
  static_assert(W <= 256 && WP <= 256, "tensor copy boxes hold at most 256 elements");
  static_assert(OUTF_B % 128 == 0 && OUTV_B % 128 == 0, "output boxes 128-byte aligned");
};

struct LbTmaArgs {
  CUtensorMap fin;   // (x, y, z, q), box (W, 1, 1, 3)
  CUtensorMap fout;  // (x, y, z, q), box (TX, 1, 1, 27)
  CUtensorMap phi;   // (x, y, z), box (WP, 1, 1)
  CUtensorMap u;     // (x, y, z, component), box (TX, 1, 1, 3)
  CUtensorMap a;
};

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0,
                                            int c1, int c2, int c3, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];\n" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3),
      "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int c0,
                                            int c1, int c2, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2),
      "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tma_store_4d(const CUtensorMap* map, int c0, int c1,
                                             int c2, int c3, const void* src) {
  asm volatile(
      "cp.async.bulk.tensor.4d.global.shared::cta.tile.bulk_group"
      " [%0, {%1, %2, %3, %4}], [%5];\n" ::"l"(reinterpret_cast<uint64_t>(map)),
      "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(src))
      : "memory");
}
__device__ __forceinline__ void bulk_commit() {
  asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
}
// the stores committed so far have finished reading shared memory
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory");
}
// orders this thread's shared-memory accesses with later tensor copies
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

template <typename Store, int TX>
__global__ void __launch_bounds__(TX / 2)
lb_collide_tma(const __grid_constant__ LbTmaArgs m,
               const typename Store::T* __restrict__ fin,
               const float* __restrict__ phi, const uint8_t* __restrict__ flags,
               Grid g, Consts k, unsigned* __restrict__ wait_err) {
  using L = TmaTile<Store, TX>;
  using T = typename Store::T;
  using T2 = typename Store::T2;
  extern __shared__ __align__(128) unsigned char lbt_smem[];
  unsigned char* const base = lbt_smem;
  T* const sf = reinterpret_cast<T*>(lbt_smem + L::IN_B);
  float* const su = reinterpret_cast<float*>(lbt_smem + L::IN_B + L::OUTF_B);
  float* const sa = su + 3 * TX;
  uint64_t* const bar = reinterpret_cast<uint64_t*>(lbt_smem + L::IN_B + L::OUTF_B +
                                                    2 * L::OUTV_B);
  const int tid = threadIdx.x;
  const int x0 = blockIdx.x * TX, y = blockIdx.y, z = blockIdx.z;

  if (tid < 32) {
    if (tid == 0) {
      mbar_init(bar, 1);
      // wait_err[1]: the test request of cacl_inject_copy_stall (16 bytes
      // more than the copies deliver, so that the wait below runs out)
      mbar_arrive_expect_tx(bar, L::TX_BYTES + (wait_err[1] ? 16u : 0u));
    }
    __syncwarp();
    if (tid < 9) {
      tma_load_4d(base + tid * L::LINE_B, &m.fin, x0 - L::PAD,
                  wrap(y, -(tid % 3 - 1), g.ny), wrap(z, -(tid / 3 - 1), g.nz), 3 * tid,
                  bar);
    } else if (tid < 18) {
      const int j = tid - 9;
      tma_load_3d(base + 9 * L::LINE_B + j * L::ROWP_B, &m.phi, x0 - L::PADP,
                  wrap(y, j % 3 - 1, g.ny), wrap(z, j / 3 - 1, g.nz), bar);
    }
  }
  __syncthreads();  // the barrier is initialised before anyone waits on it
  const bool ok = mbar_wait(bar, 0);
  if (__syncthreads_or(!ok)) {
    // give up: record it, let the copies in flight land (bounded), return
    if (tid == 0) {
      atomicOr(wait_err, 1u);
      mbar_wait(bar, 0);
    }
    return;
  }
  const int nx = g.nx, nxy = g.nx * g.ny, N = (int)g.N;

  // periodic wrap in x: the element left of x = 0 and the one right of
  // x = nx - 1, for the 27 population rows and the 9 phi rows
  const bool left = (x0 == 0), right = (x0 + TX >= nx);
  if (left || right) {
#pragma unroll 1
    for (int e = tid; e < 72; e += TX / 2) {
      const int side = e / 36, r = e - 36 * side;
      if (side == 0 ? !left : !right) continue;
      const int xs = (side == 0) ? nx - 1 : 0;
      if (r < Q) {
        const int col = (side == 0) ? L::PAD - 1 : L::PAD + (nx - x0);
        const int src = wrap(z, -cz(r), g.nz) * nxy + wrap(y, -cy(r), g.ny) * nx + xs;
        T* dst = reinterpret_cast<T*>(base + (r / 3) * L::LINE_B) + (r % 3) * L::W + col;
        *dst = fin[r * N + src];
      } else {
        const int j = r - Q;
        const int col = (side == 0) ? L::PADP - 1 : L::PADP + (nx - x0);
        const int src = wrap(z, j / 3 - 1, g.nz) * nxy + wrap(y, j % 3 - 1, g.ny) * nx + xs;
        float* dst = reinterpret_cast<float*>(base + 9 * L::LINE_B + j * L::ROWP_B) + col;
        *dst = phi[src];
      }
    }
    __syncthreads();
  }

  const int x = x0 + 2 * tid;
  if (x < nx) {
    const int n = x + nx * y + nxy * z;
    const uchar2 fl = *reinterpret_cast<const uchar2*>(flags + n);
    if (((fl.x | fl.y) & (FLAG_SOLID | FLAG_NEAR)) == 0) {
      float2 f[Q];
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const T* ln = reinterpret_cast<const T*>(base + (q / 3) * L::LINE_B) +
                      (q % 3) * L::W + L::PAD + 2 * tid;
        const T2 own = *reinterpret_cast<const T2*>(ln);
        T2 v;
        if (cx(q) == 0)
          v = own;
        else if (cx(q) > 0)
          v = Store::pack(ln[-1], Store::lo(own));
        else
          v = Store::pack(Store::hi(own), ln[2]);
        f[q] = Store::decode2(v, q);
      }
      float2 pc[3][3];
      float pl[3][3], pr[3][3];
#pragma unroll
      for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float* r = reinterpret_cast<const float*>(
                               base + 9 * L::LINE_B + (3 * c + b) * L::ROWP_B) +
                           L::PADP + 2 * tid;
          pc[b][c] = *reinterpret_cast<const float2*>(r);
          pl[b][c] = r[-1];
          pr[b][c] = r[2];
        }
      NodeOut<float2> o;
      float2 ax, ay, az;
      pair_eval(f, pc, pl, pr, k, o, ax, ay, az);
#pragma unroll
      for (int q = 0; q < Q; ++q)
        *reinterpret_cast<T2*>(sf + q * TX + 2 * tid) = Store::encode_w2(o.P[q], q);
      *reinterpret_cast<float2*>(su + 2 * tid) = o.ux;
      *reinterpret_cast<float2*>(su + TX + 2 * tid) = o.uy;
      *reinterpret_cast<float2*>(su + 2 * TX + 2 * tid) = o.uz;
      *reinterpret_cast<float2*>(sa + 2 * tid) = ax;
      *reinterpret_cast<float2*>(sa + TX + 2 * tid) = ay;
      *reinterpret_cast<float2*>(sa + 2 * TX + 2 * tid) = az;
    } else {
#pragma unroll 1
      for (int j = 0; j < 2; ++j) {
        NodeOut<float> on;
        float bx = 0.f, by = 0.f, bz = 0.f;
        const int c = 2 * tid + j;
        if (lb_node_eval<Store, int>(x + j, y, z, fin, phi, flags, g, k, on, bx, by, bz)) {
#pragma unroll
          for (int q = 0; q < Q; ++q) sf[q * TX + c] = Store::encode_w(on.P[q], q);
          su[c] = on.ux;
          su[TX + c] = on.uy;
          su[2 * TX + c] = on.uz;
        } else {
#pragma unroll
          for (int q = 0; q < Q; ++q) sf[q * TX + c] = Store::encode_w(0.0f, q);
          su[c] = su[TX + c] = su[2 * TX + c] = 0.f;
        }
        sa[c] = bx;
        sa[TX + c] = by;
        sa[2 * TX + c] = bz;
      }
    }
  }
  fence_proxy_async();
  __syncthreads();
  if (tid == 0) {
    tma_store_4d(&m.fout, x0, y, z, 0, sf);
    tma_store_4d(&m.u, x0, y, z, 0, su);
    tma_store_4d(&m.a, x0, y, z, 0, sa);
    bulk_commit();
    bulk_wait_read();  // shared memory stays valid until the stores read it
  }
}

// Collide-stream in moment form (storage CACL_F32_MOMENTS): a node stores
// the 17 coefficients of its post-collision polynomial P instead of its 27
// populations, f*_q = w_q P(c_q) (the paper's thread-safe form, in which a
// node keeps macroscopic moments and its neighbours rebuild the pulled
// populations, Sect. 2.1). A block owns a MX x MY column of nodes and
// marches up MZC planes. For each plane z' it rebuilds, for the column and
// a one-node halo in x and y, every node's 27 populations from its
// coefficients with the transforms of the collision and keeps them in
// shared memory by the plane that pulls them: those with c_z = +1 for
// plane z' + 1 (a ring of three planes), c_z = 0 for z' (two) and c_z = -1
// for z' - 1 (one). Plane z then pulls f_q from the node x - c_q of the
// right slot; the values are the very numbers the population form would
// have stored (same transform, same w_q rounding), so the two forms are
// bit-identical at fluid nodes. Near a wall the bounced-back populations
// come from the node's own coefficients. The collision writes the 17
// coefficients, u and a.
constexpr int MX = 32, MY = 8, MZC = 16;
constexpr int MHX = MX + 2, MHY = MY + 2, MNH = MHX * MHY;  // halo tile

struct MomentSmem {
  float sp[3][9][MNH];  // c_z = +1 populations of plane z' (ring by z' mod 3)
  float s0[2][9][MNH];  // c_z = 0 (ring by z' mod 2)
  float sm[9][MNH];     // c_z = -1 of the plane above the one computed
};

__device__ __forceinline__ void load_coefs(const float* __restrict__ C, int64_t n,
                                           int64_t N, Coefs<float>& c) {
  c.k1 = __ldg(C + n);
  c.Lx = __ldg(C + N + n);
  c.Ly = __ldg(C + 2 * N + n);
  c.Lz = __ldg(C + 3 * N + n);
  c.Dx = __ldg(C + 4 * N + n);
  c.Dy = __ldg(C + 5 * N + n);
  c.Dz = __ldg(C + 6 * N + n);
  c.Fxy = __ldg(C + 7 * N + n);
  c.Fxz = __ldg(C + 8 * N + n);
  c.Fyz = __ldg(C + 9 * N + n);
  c.Mxy = __ldg(C + 10 * N + n);
  c.Mxz = __ldg(C + 11 * N + n);
  c.Myx = __ldg(C + 12 * N + n);
  c.Myz = __ldg(C + 13 * N + n);
  c.Mzx = __ldg(C + 14 * N + n);
  c.Mzy = __ldg(C + 15 * N + n);
  c.X = __ldg(C + 16 * N + n);
}

__device__ __forceinline__ void store_coefs(float* __restrict__ C, int64_t n, int64_t N,
                                            const Coefs<float>& c) {
  C[n] = c.k1;
  C[N + n] = c.Lx;
  C[2 * N + n] = c.Ly;
  C[3 * N + n] = c.Lz;
  C[4 * N + n] = c.Dx;
  C[5 * N + n] = c.Dy;
  C[6 * N + n] = c.Dz;
  C[7 * N + n] = c.Fxy;
  C[8 * N + n] = c.Fxz;
  C[9 * N + n] = c.Fyz;
  C[10 * N + n] = c.Mxy;
  C[11 * N + n] = c.Mxz;
  C[12 * N + n] = c.Myx;
  C[13 * N + n] = c.Myz;
  C[14 * N + n] = c.Mzx;
  C[15 * N + n] = c.Mzy;
  C[16 * N + n] = c.X;
}

// f*_q = w_q P(c_q) of one node from its coefficients (the population
// form's stored value)
__device__ __forceinline__ void coefs_to_pops(const Coefs<float>& c, float (&f)[Q]) {
  float P[Q];
  coefs_to_P(c, P);
#pragma unroll
  for (int q = 0; q < Q; ++q) f[q] = StoreF32::encode_w(P[q], q);
}

__global__ void __launch_bounds__(MX * MY)
lb_collide_moments(const float* __restrict__ Cin, float* __restrict__ Cout,
                   const float* __restrict__ phi, float* __restrict__ u,
                   float* __restrict__ a, const uint8_t* __restrict__ flags, Grid g,
                   Consts k) {
  extern __shared__ __align__(16) float msm[];
  MomentSmem& sh = *reinterpret_cast<MomentSmem*>(msm);
  const int tid = threadIdx.x;
  const int tx = tid % MX, ty = tid / MX;
  const int x0 = blockIdx.x * MX, y0 = blockIdx.y * MY, z0 = blockIdx.z * MZC;
  const int z1 = min(z0 + MZC, g.nz);
  const int64_t N = g.N;
  const int64_t nxy = (int64_t)g.nx * g.ny;

  // the halo nodes this thread rebuilds (at most two of MNH)
  int hcol[2];
  bool hact[2];
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int h = tid + r * MX * MY;
    hact[r] = h < MNH;
    const int hx = h % MHX, hy = h / MHX;
    hcol[r] = ((x0 - 1 + hx) % g.nx + g.nx) % g.nx +
              g.nx * (((y0 - 1 + hy) % g.ny + g.ny) % g.ny);
  }
  auto rebuild = [&](int zp) {  // plane zp (any integer, wrapped)
    const int zw = ((zp % g.nz) + g.nz) % g.nz;
    const int sp = ((zp % 3) + 3) % 3, s0 = zp & 1;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      if (!hact[r]) continue;
      const int h = tid + r * MX * MY;
      Coefs<float> c;
      load_coefs(Cin, hcol[r] + zw * nxy, N, c);
      float f[Q];
      coefs_to_pops(c, f);
#pragma unroll
      for (int j = 0; j < 9; ++j) {
        sh.sm[j][h] = f[j];
        sh.s0[s0][j][h] = f[9 + j];
        sh.sp[sp][j][h] = f[18 + j];
      }
    }
  };

  rebuild(z0 - 1);
  __syncthreads();
  rebuild(z0);
  const int x = x0 + tx, y = y0 + ty;
  const bool act = x < g.nx && y < g.ny;
  const int hme = (ty + 1) * MHX + (tx + 1);
  for (int z = z0; z < z1; ++z) {
    __syncthreads();  // every thread is done with the slots rebuilt below
    rebuild(z + 1);
    __syncthreads();
    if (!act) continue;
    const int64_t n = x + (int64_t)g.nx * y + nxy * z;
    const uint8_t fl = flags[n];
    if (fl & FLAG_SOLID) continue;
    const int spm = (((z - 1) % 3) + 3) % 3, s0c = z & 1;
    float f[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int h = hme - cy(q) * MHX - cx(q);
      const int j = q % 9;
      f[q] = cz(q) > 0 ? sh.sp[spm][j][h] : (cz(q) == 0 ? sh.s0[s0c][j][h] : sh.sm[j][h]);
    }
    const int xo[3] = {wrap(x, -1, g.nx), x, wrap(x, 1, g.nx)};
    const int64_t yo[3] = {(int64_t)wrap(y, -1, g.ny) * g.nx, (int64_t)y * g.nx,
                           (int64_t)wrap(y, 1, g.ny) * g.nx};
    const int64_t zo[3] = {wrap(z, -1, g.nz) * nxy, z * nxy, wrap(z, 1, g.nz) * nxy};
    if (fl & FLAG_NEAR) {
      // halfway bounce-back: f_q = f*_{opp q}(x) of the previous step
      Coefs<float> own;
      load_coefs(Cin, n, N, own);
      float fo[Q];
      coefs_to_pops(own, fo);
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        if (q == REST) continue;
        const int64_t src = xo[1 - cx(q)] + yo[1 - cy(q)] + zo[1 - cz(q)];
        if (__ldg(flags + src) & FLAG_SOLID) f[q] = fo[opp(q)];
      }
    }
    // isotropic gradient and Laplacian of phi (Eqs. grad_iso, lap_iso)
    const float phi0 = __ldg(phi + n);
    float gx = 0.f, gy = 0.f, gz = 0.f, ssum = 0.f;
#pragma unroll
    for (int q = 0; q < REST; ++q) {
      const float vp = __ldg(phi + (xo[1 + cx(q)] + yo[1 + cy(q)] + zo[1 + cz(q)]));
      const float vm = __ldg(phi + (xo[1 - cx(q)] + yo[1 - cy(q)] + zo[1 - cz(q)]));
      stencil_pair(q, vp, vm, gx, gy, gz, ssum);
    }
    const float lap = lap_from_sum(phi0, ssum);
    float ax, ay, az;
    compressive(phi0, gx, gy, gz, ax, ay, az);
    a[n] = ax;
    a[N + n] = ay;
    a[2 * N + n] = az;
    Coefs<float> cf;
    float ux, uy, uz;
    collide_coefs(f, phi0, gx, gy, gz, lap, k, cf, ux, uy, uz);
    store_coefs(Cout, n, N, cf);
    u[n] = ux;
    u[N + n] = uy;
    u[2 * N + n] = uz;
  }
}

// Populations (27 N, FP32) of every node from the moment form, and p*.
__global__ void __launch_bounds__(256)
moments_to_pops(const float* __restrict__ C, float* __restrict__ f,
                float* __restrict__ pstar, const uint8_t* __restrict__ flags, int64_t N) {
  const int64_t n = (int64_t)blockIdx.x * 256 + threadIdx.x;
  if (n >= N) return;
  Coefs<float> c;
  load_coefs(C, n, N, c);
  float v[Q];
  coefs_to_pops(c, v);
  if (f) {
#pragma unroll
    for (int q = 0; q < Q; ++q) f[q * N + n] = v[q];
  }
  if (pstar) {
    float s = 0.f;
#pragma unroll
    for (int q = 0; q < Q; ++q) s += v[q];
    pstar[n] = (flags[n] & FLAG_SOLID) ? 0.f : s;
  }
}

// Equilibrium f^eq(p* = 0, u) in moment form (u = 0 at solid nodes): the
// coefficients of Eq. feq3 with no non-equilibrium part and no force.
__global__ void __launch_bounds__(256)
moments_init(float* __restrict__ C0, float* __restrict__ C1, float* __restrict__ u,
             const uint8_t* __restrict__ flags, int64_t N) {
  const int64_t n = (int64_t)blockIdx.x * 256 + threadIdx.x;
  if (n >= N) return;
  float ux = u[n], uy = u[N + n], uz = u[2 * N + n];
  if (flags[n] & FLAG_SOLID) {
    ux = uy = uz = 0.f;
    u[n] = u[N + n] = u[2 * N + n] = 0.f;
  }
  const float uu = ux * ux + uy * uy + uz * uz;
  const float k2 = 3.0f - 4.5f * uu;
  Coefs<float> c;
  c.k1 = -1.5f * uu;
  c.Lx = ux * (k2 + 4.5f * ux * ux);
  c.Ly = uy * (k2 + 4.5f * uy * uy);
  c.Lz = uz * (k2 + 4.5f * uz * uz);
  c.Dx = 4.5f * ux * ux;
  c.Dy = 4.5f * uy * uy;
  c.Dz = 4.5f * uz * uz;
  c.Fxy = 9.0f * ux * uy;
  c.Fxz = 9.0f * ux * uz;
  c.Fyz = 9.0f * uy * uz;
  c.Mxy = 13.5f * ux * ux * uy;
  c.Mxz = 13.5f * ux * ux * uz;
  c.Myx = 13.5f * uy * uy * ux;
  c.Myz = 13.5f * uy * uy * uz;
  c.Mzx = 13.5f * uz * uz * ux;
  c.Mzy = 13.5f * uz * uz * uy;
  c.X = 27.0f * ux * uy * uz;
  store_coefs(C0, n, N, c);
  store_coefs(C1, n, N, c);
}

// Batched collide-stream, W nodes per thread. The cases of the work-list
// are those that run the W-node kernel alone (four-node for 16-bit
// populations with nx a multiple of 4, two-node with nx even, else
// one-node). Their nodes are taken in linear order n = x + nx (y + ny z) in
// units of W nodes, and virtual block b of the work-list is the run of BX
// units (b - start) BX .. of its case, so that only the last block of a
// case has idle threads, whatever nx is. A unit of two or four nodes with a
// solid node or a wall neighbour runs the one-node path on each node, as in
// the single-case kernels: every node gets lb_node's arithmetic, bit for
// bit. Blocks stride through the work-list (b, b + gridDim.x, ...), so that
// the rows in flight at any time are neighbours and their phi stencils
// share cache lines.
// PERSIST: a resident-sized grid strides through the work-list; otherwise
// one block per work item (the block scheduler does the distribution).
// Registers: at most 168 for four nodes (three blocks of 128 threads per
// SM; at 128 the case cursor and the linear indexing push the four-node
// body into 300 bytes of spills), 96 for two (five blocks of 128; six
// blocks made the 48-case sweep 1.7% slower), 85 for one (80 used, six
// blocks of 128; at 64, eight blocks, the persistent forms spill 116 bytes
// and the sweep ran 0.35% slower).
template <int W, int BX>
constexpr int lb_batch_minb() {
  return W == 4 ? (384 + BX - 1) / BX : (W == 2 ? 640 / BX : 768 / BX);
}

template <typename Store, int W, int BX, bool PERSIST>
__global__ void __launch_bounds__(BX, (lb_batch_minb<W, BX>()))
lb_collide_batch(const CaseDesc* __restrict__ cases, WorkList wl, int fc,
                 int pc) {
  using T = typename Store::T;
  __shared__ CaseCursor cur;
  if (threadIdx.x == 0) cur.begin();
  __syncthreads();
  const int stride = PERSIST ? (int)gridDim.x : wl.total;
  for (int b = blockIdx.x; b < wl.total; b += stride) {
    cur.seek(cases, wl, b);
    const CaseDesc& cd = cur.d;
    const int n = ((b - cur.cstart) * BX + (int)threadIdx.x) * W;
    if (n >= (int)cd.g.N) continue;
    const int nxy = cd.g.nx * cd.g.ny;
    const int z = n / nxy;
    const int r = n - z * nxy;
    const int y = r / cd.g.nx;
    const int x0 = r - y * cd.g.nx;
    const T* fin = (const T*)cd.f[fc];
    T* fout = (T*)cd.f[1 - fc];
    const float* phi = cd.phi[pc];
    bool bulk = false;
    if constexpr (W == 4 && sizeof(T) == 2) {
      const uchar4 fl = *reinterpret_cast<const uchar4*>(cd.flags + n);
      bulk = ((fl.x | fl.y | fl.z | fl.w) & (FLAG_SOLID | FLAG_NEAR)) == 0;
      if (bulk) lb_quad<Store>(x0, y, z, fin, fout, phi, cd.u, cd.a, cd.g, cd.k);
    } else if constexpr (W == 2) {
      const uchar2 fl = *reinterpret_cast<const uchar2*>(cd.flags + n);
      bulk = ((fl.x | fl.y) & (FLAG_SOLID | FLAG_NEAR)) == 0;
      if (bulk) lb_pair<Store>(x0, y, z, fin, fout, phi, cd.u, cd.a, cd.g, cd.k);
    }
    if (!bulk) {
#pragma unroll 1
      for (int j = 0; j < W; ++j)
        lb_node<Store, int>(x0 + j, y, z, fin, fout, phi, cd.u, cd.a, cd.flags, cd.g,
                            cd.k);
    }
  }
}

int staged_segments(const Grid& g) { return ((g.nx + SEG - 1) / SEG) * g.ny * g.nz; }

template <typename Store>
void* staged_kernel(const Grid& g, bool index64) {
  return (!index64 && (int64_t)Q * g.N < (int64_t)INT32_MAX)
             ? (void*)lb_collide_staged<Store, int>
             : (void*)lb_collide_staged<Store, int64_t>;
}

template <typename Store>
cudaError_t staged_setup(const Grid& g, bool index64, int* grid) {
  void* fn = staged_kernel<Store>(g, index64);
  const size_t smem = 2 * sizeof(StagedRows<Store>);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  int per_sm = 0, dev = 0, sms = 0;
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, SEG, smem);
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  *grid = std::max(1, std::min(staged_segments(g), std::max(per_sm, 1) * sms));
  return e;
}

constexpr int LBT_TX = 128;  // nodes per tile of the TMA-tiled collide-stream

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                         cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// Row-major tensor map over (x, y, z[, k]) with element size es and the
// given box; false if the driver rejects it.
bool encode_map(CUtensorMap* m, int es, int rank, void* addr, const Grid& g,
                int kdim, const cuuint32_t* box) {
  auto fn = tensor_map_encoder();
  if (!fn) return false;
  const cuuint64_t dims[4] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz,
                              (cuuint64_t)kdim};
  const cuuint64_t strides[3] = {(cuuint64_t)g.nx * es, (cuuint64_t)g.nx * g.ny * es,
                                 (cuuint64_t)g.N * es};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  const CUtensorMapDataType dt =
      es == 2 ? CU_TENSOR_MAP_DATA_TYPE_UINT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  return fn(m, dt, (cuuint32_t)rank, addr, dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <typename Store>
cudaError_t tma_setup(cacl_ctx* c) {
  using L = TmaTile<Store, LBT_TX>;
  const Grid& g = c->g;
  c->lbt_ok = false;
  if (g.nx % 8 != 0 || (int64_t)Q * g.N >= (int64_t)INT32_MAX) return cudaSuccess;
  const cuuint32_t boxf[4] = {(cuuint32_t)L::W, 1, 1, 3};
  const cuuint32_t boxo[4] = {(cuuint32_t)LBT_TX, 1, 1, (cuuint32_t)Q};
  const cuuint32_t boxp[3] = {(cuuint32_t)L::WP, 1, 1};
  const cuuint32_t boxv[4] = {(cuuint32_t)LBT_TX, 1, 1, 3};
  bool ok = true;
  for (int i = 0; i < 2; ++i) {
    ok = ok && encode_map(&c->lbt_fload[i], L::ES, 4, c->f[i], g, Q, boxf);
    ok = ok && encode_map(&c->lbt_fstore[i], L::ES, 4, c->f[i], g, Q, boxo);
    ok = ok && encode_map(&c->lbt_phi[i], 4, 3, c->phi[i], g, 1, boxp);
  }
  ok = ok && encode_map(&c->lbt_u, 4, 4, c->u, g, 3, boxv);
  ok = ok && encode_map(&c->lbt_a, 4, 4, c->a, g, 3, boxv);
  if (!ok) return cudaSuccess;  // the other collide-stream kernels remain
  void* fn = (void*)lb_collide_tma<Store, LBT_TX>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       L::SMEM_B);
  if (e != cudaSuccess) return e;
  c->lbt_ok = true;
  return cudaSuccess;
}

template <typename Store>
void launch_store(cacl_ctx* c, const void* fin, void* fout, const float* phi) {
  using T = typename Store::T;
  const Grid g = c->g;
  if (lb_staged_ok(c, fin, fout, phi)) {
    const int nseg = staged_segments(g);
    void* fn = staged_kernel<Store>(g, c->index64);
    const size_t smem = 2 * sizeof(StagedRows<Store>);
    const int grid = c->lb_grid;
    const T* fi = (const T*)fin;
    T* fo = (T*)fout;
    float* u = c->u;
    float* a = c->a;
    const uint8_t* fl = c->flags;
    Consts k = c->k;
    Grid gg = g;
    int ns = nseg;
    unsigned* err = c->ticket + 1;
    void* args[] = {(void*)&fi, (void*)&fo, (void*)&phi, (void*)&u, (void*)&a,
                    (void*)&fl, (void*)&gg, (void*)&k, (void*)&ns, (void*)&err};
    cudaLaunchKernel(fn, dim3(grid), dim3(SEG), args, smem, c->stream);
    return;
  }
  if (lb_tma_ok(c, fin, fout, phi)) {
    const int fi = (fin == c->f[0]) ? 0 : 1;
    LbTmaArgs m;
    m.fin = c->lbt_fload[fi];
    m.fout = c->lbt_fstore[1 - fi];
    m.phi = c->lbt_phi[(phi == c->phi[0]) ? 0 : 1];
    m.u = c->lbt_u;
    m.a = c->lbt_a;
    const dim3 grid((g.nx + LBT_TX - 1) / LBT_TX, g.ny, g.nz);
    lb_collide_tma<Store, LBT_TX><<<grid, LBT_TX / 2, TmaTile<Store, LBT_TX>::SMEM_B,
                                   c->stream>>>(m, (const T*)fin, phi, c->flags, g,
                                                c->k, c->ticket + 1);
    return;
  }
  if constexpr (sizeof(T) == 2) {
    if (lb_quad_ok(c, fin, fout, phi)) {
      dim3 block(LBQ_PX, LBQ_PY, 1);
      dim3 grid((g.nx / 4 + LBQ_PX - 1) / LBQ_PX, (g.ny + LBQ_PY - 1) / LBQ_PY, g.nz);
      lb_collide_quad<Store><<<grid, block, 0, c->stream>>>(
          (const T*)fin, (T*)fout, phi, c->u, c->a, c->flags, g, c->k);
      return;
    }
  }
  if (lb_pair_ok(c, fin, fout, phi)) {
    dim3 block(LB2_PX, LB2_PY, 1);
    dim3 grid((g.nx / 2 + LB2_PX - 1) / LB2_PX, (g.ny + LB2_PY - 1) / LB2_PY, g.nz);
    if constexpr (sizeof(T) == 4)
      lb_collide_pair32<Store><<<grid, block, 0, c->stream>>>(
          (const T*)fin, (T*)fout, phi, c->u, c->a, c->flags, g, c->k);
    else
      lb_collide_pair16<Store><<<grid, block, 0, c->stream>>>(
          (const T*)fin, (T*)fout, phi, c->u, c->a, c->flags, g, c->k);
    return;
  }
  dim3 block(LB_BX, LB_BY, 1);
  dim3 grid((g.nx + LB_BX - 1) / LB_BX, (g.ny + LB_BY - 1) / LB_BY, g.nz);
  if (!c->index64 && (int64_t)Q * g.N < (int64_t)INT32_MAX)
    lb_collide<Store, int><<<grid, block, 0, c->stream>>>(
        (const T*)fin, (T*)fout, phi, c->u, c->a, c->flags, g, c->k);
  else
    lb_collide<Store, int64_t><<<grid, block, 0, c->stream>>>(
        (const T*)fin, (T*)fout, phi, c->u, c->a, c->flags, g, c->k);
}

}  // namespace

// Resident-sized grid of the persistent copy-staged collide-stream (and its
// shared-memory attribute), set per context (again when the offset width
// changes) outside any graph capture.
cudaError_t lb_init(cacl_ctx* c) {
  if (c->p.storage == CACL_F32_MOMENTS)
    return cudaFuncSetAttribute(lb_collide_moments,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sizeof(MomentSmem));
  switch (c->p.storage) {
    case CACL_F16_SHIFTED: return staged_setup<StoreF16>(c->g, c->index64, &c->lb_grid);
    case CACL_BF16_SHIFTED: return staged_setup<StoreBF16>(c->g, c->index64, &c->lb_grid);
    default: return staged_setup<StoreF32>(c->g, c->index64, &c->lb_grid);
  }
}

// Tensor maps of the TMA-tiled collide-stream over the context's own
// buffers (set once the buffers exist, outside any graph capture).
cudaError_t lb_tma_init(cacl_ctx* c) {
  if (c->p.storage == CACL_F32_MOMENTS) return cudaSuccess;  // not applicable
  switch (c->p.storage) {
    case CACL_F16_SHIFTED: return tma_setup<StoreF16>(c);
    case CACL_BF16_SHIFTED: return tma_setup<StoreBF16>(c);
    default: return tma_setup<StoreF32>(c);
  }
}

// The TMA-tiled collide-stream (CACL_OPT_LB_PIPE = 3) runs on the
// context's own population, phi, u and a buffers when nx is a multiple of 8
// and 27 N < 2^31 (and 64-bit offsets are not forced); otherwise the
// two-node kernel runs.
bool lb_tma_ok(const cacl_ctx* c, const void* fin, const void* fout,
               const void* phi) {
  const bool fpair = (fin == c->f[0] && fout == c->f[1]) ||
                     (fin == c->f[1] && fout == c->f[0]);
  return c->lb_pipe == 3 && c->lbt_ok && !c->index64 && fpair &&
         (phi == c->phi[0] || phi == c->phi[1]);
}

// The copy-staged collide-stream (chosen by CACL_OPT_LB_PIPE = 1) needs
// 16-byte aligned runs: nx a multiple of 16 bytes' worth of populations and
// of 4, aligned fields; otherwise the direct kernel runs.
bool lb_staged_ok(const cacl_ctx* c, const void* fin, const void* fout,
                  const void* phi) {
  const int pf = 16 / storage_bytes(c->p.storage);
  auto al = [](const void* p) { return ((uintptr_t)p & 15u) == 0; };
  return c->lb_pipe == 1 && c->g.nx % pf == 0 && c->g.nx % 4 == 0 &&
         al(fin) && al(fout) && al(phi);
}

// The two-node collide-stream (the default, CACL_OPT_LB_PIPE = 0, and the
// fallback of 3) needs nx even, 27 N below 2^31 (32-bit offsets, not
// forced to 64) and buffers aligned for the pair accesses; otherwise, or
// with CACL_OPT_LB_PIPE = 2, one node per thread.
bool lb_pair_ok(const cacl_ctx* c, const void* fin, const void* fout,
                const void* phi) {
  const uintptr_t fa = 2 * storage_bytes(c->p.storage) - 1;
  auto al = [](const void* p, uintptr_t m) { return ((uintptr_t)p & m) == 0; };
  return (c->lb_pipe == 0 || c->lb_pipe == 3) && c->g.nx % 2 == 0 && !c->index64 &&
         (int64_t)Q * c->g.N < (int64_t)INT32_MAX && al(fin, fa) && al(fout, fa) &&
         al(phi, 7) && al(c->u, 7) && al(c->a, 7);
}

// The four-node collide-stream (16-bit populations, the default there)
// needs nx a multiple of 4, 27 N below 2^31 (offsets not forced to 64 bits)
// and 8-byte aligned population
// and 16-byte aligned phi, u, a buffers; otherwise the two-node kernel.
bool lb_quad_ok(const cacl_ctx* c, const void* fin, const void* fout,
                const void* phi) {
  auto al = [](const void* p, uintptr_t m) { return ((uintptr_t)p & m) == 0; };
  return c->lb_pipe == 0 && storage_bytes(c->p.storage) == 2 && c->g.nx % 4 == 0 &&
         !c->index64 && (int64_t)Q * c->g.N < (int64_t)INT32_MAX && al(fin, 7) && al(fout, 7) &&
         al(phi, 15) && al(c->u, 15) && al(c->a, 15);
}

cudaError_t launch_lb(cacl_ctx* c, const void* fin, void* fout,
                      const float* phi) {
  if (c->p.storage == CACL_F32_MOMENTS) {
    const Grid g = c->g;
    const dim3 grid((g.nx + MX - 1) / MX, (g.ny + MY - 1) / MY, (g.nz + MZC - 1) / MZC);
    lb_collide_moments<<<grid, MX * MY, sizeof(MomentSmem), c->stream>>>(
        (const float*)fin, (float*)fout, phi, c->u, c->a, c->flags, g, c->k);
    return cudaGetLastError();
  }
  switch (c->p.storage) {
    case CACL_F16_SHIFTED: launch_store<StoreF16>(c, fin, fout, phi); break;
    case CACL_BF16_SHIFTED: launch_store<StoreBF16>(c, fin, fout, phi); break;
    default: launch_store<StoreF32>(c, fin, fout, phi); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_moments_init(cacl_ctx* c) {
  const int nb = (int)((c->g.N + 255) / 256);
  moments_init<<<nb, 256, 0, c->stream>>>((float*)c->f[0], (float*)c->f[1], c->u,
                                          c->flags, c->g.N);
  return cudaGetLastError();
}

cudaError_t launch_moments_expand(cacl_ctx* c, const void* C, float* f, float* pstar) {
  const int nb = (int)((c->g.N + 255) / 256);
  moments_to_pops<<<nb, 256, 0, c->stream>>>((const float*)C, f, pstar, c->flags, c->g.N);
  return cudaGetLastError();
}

int lb_batch_row(int variant) {
  const int r = variant % 3;
  return r == 0 ? 64 : r == 2 ? 256 : 128;
}

bool lb_batch_persistent(int variant) { return variant < 3; }

namespace {
template <typename Store, int W>
void* lb_batch_fn(int variant) {
  switch (variant) {
    case 0: return (void*)lb_collide_batch<Store, W, 64, true>;
    case 2: return (void*)lb_collide_batch<Store, W, 256, true>;
    case 3: return (void*)lb_collide_batch<Store, W, 64, false>;
    case 4: return (void*)lb_collide_batch<Store, W, 128, false>;
    case 5: return (void*)lb_collide_batch<Store, W, 256, false>;
    default: return (void*)lb_collide_batch<Store, W, 128, true>;
  }
}

template <typename Store>
void* lb_batch_width(int width, int variant) {
  if constexpr (sizeof(typename Store::T) == 2) {
    if (width == 4) return lb_batch_fn<Store, 4>(variant);
  }
  return width == 2 ? lb_batch_fn<Store, 2>(variant) : lb_batch_fn<Store, 1>(variant);
}

void* lb_batch_kernel(int storage, int width, int variant) {
  switch (storage) {
    case CACL_F16_SHIFTED: return lb_batch_width<StoreF16>(width, variant);
    case CACL_BF16_SHIFTED: return lb_batch_width<StoreBF16>(width, variant);
    default: return lb_batch_width<StoreF32>(width == 4 ? 1 : width, variant);
  }
}
}  // namespace

int lb_batch_occupancy(int storage, int width, int variant) {
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &nb, lb_batch_kernel(storage, width, variant), lb_batch_row(variant), 0);
  return nb;
}

cudaError_t launch_lb_batch(const CaseDesc* cases, WorkList wl, int storage, int width,
                            int variant, int grid, int fc, int pc, cudaStream_t st) {
  void* fn = lb_batch_kernel(storage, width, variant);
  void* args[] = {(void*)&cases, (void*)&wl, (void*)&fc, (void*)&pc};
  return cudaLaunchKernel(fn, dim3(grid), dim3(lb_batch_row(variant)), args, 0, st);
}

}  // namespace cacl
