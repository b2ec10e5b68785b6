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
// phi^n, which the phi update of this step needs at every node (Sect. 2.2):
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
#include <algorithm>

#include "cacl_internal.cuh"

namespace cacl {
namespace {

constexpr int LB_BX = 128;
constexpr int LB_BY = 1;

struct NodeOut {
  float P[Q];  // f*_q / w_q
  float ux, uy, uz;
};

__device__ __forceinline__ void collide(const float (&f)[Q], float phi0,
                                        float gx, float gy, float gz, float lap,
                                        const Consts& k, NodeOut& o) {
  // moments by sum factorisation: along x for each (cy, cz) line l, then
  // along y for each cz, then along z (q = 9 (cz+1) + 3 (cy+1) + (cx+1))
  float m0[9], m1[9], m2[9];  // sum f, sum cx f, sum cx^2 f over the line
#pragma unroll
  for (int l = 0; l < 9; ++l) {
    m2[l] = f[3 * l + 2] + f[3 * l];
    m1[l] = f[3 * l + 2] - f[3 * l];
    m0[l] = m2[l] + f[3 * l + 1];
  }
  float n00[3], n01[3], n02[3], n10[3], n11[3], n20[3];
#pragma unroll
  for (int kz = 0; kz < 3; ++kz) {
    const int l = 3 * kz;  // lines cy = -1, 0, 1 at l, l+1, l+2
    n02[kz] = m0[l + 2] + m0[l];      // sum cy^2 f
    n01[kz] = m0[l + 2] - m0[l];      // sum cy f
    n00[kz] = n02[kz] + m0[l + 1];    // sum f
    n11[kz] = m1[l + 2] - m1[l];      // sum cx cy f
    n10[kz] = (m1[l + 2] + m1[l]) + m1[l + 1];  // sum cx f
    n20[kz] = (m2[l + 2] + m2[l]) + m2[l + 1];  // sum cx^2 f
  }
  const float Pzz = n00[2] + n00[0];
  const float p = Pzz + n00[1];
  const float jz = n00[2] - n00[0];
  const float jy = (n01[2] + n01[0]) + n01[1];
  const float Pyz = n01[2] - n01[0];
  const float Pyy = (n02[2] + n02[0]) + n02[1];
  const float jx = (n10[2] + n10[0]) + n10[1];
  const float Pxz = n10[2] - n10[0];
  const float Pxy = (n11[2] + n11[0]) + n11[1];
  const float Pxx = (n20[2] + n20[0]) + n20[1];

  // Every product and sum below is an explicit round-to-nearest operation
  // (fmaf, or __fmul_rn / __fadd_rn, which are never contracted), so that
  // each kernel that inlines the collision rounds it the same way.
  const float rho = fmaf(k.drho, phi0, k.rho_g);
  const float mu = fmaf(k.dmu, phi0, k.mu_g);
  const float inv_rho = 1.0f / rho;
  const float nu = __fmul_rn(mu, inv_rho);
  const float omega = 1.0f / fmaf(3.0f, nu, 0.5f);
  const float grx = __fmul_rn(k.drho, gx), gry = __fmul_rn(k.drho, gy),
              grz = __fmul_rn(k.drho, gz);
  const float muphi = fmaf(-k.kappa_phi, lap,
                           __fmul_rn(__fmul_rn(__fmul_rn(k.beta4, phi0),
                                               __fadd_rn(phi0, -1.0f)),
                                     __fadd_rn(phi0, -0.5f)));
  const float p3 = __fmul_rn(p, 1.0f / 3.0f);
  const float rb = __fadd_rn(rho, -k.rho_g);
  const float F0x = fmaf(rb, k.gx, fmaf(-p3, grx, __fmul_rn(muphi, gx)));
  const float F0y = fmaf(rb, k.gy, fmaf(-p3, gry, __fmul_rn(muphi, gy)));
  const float F0z = fmaf(rb, k.gz, fmaf(-p3, grz, __fmul_rn(muphi, gz)));
  // predictor for the viscous correction (Eq. Fnu)
  const float a0x = __fmul_rn(F0x, inv_rho), a0y = __fmul_rn(F0y, inv_rho),
              a0z = __fmul_rn(F0z, inv_rho);
  const float u0x = fmaf(0.5f, a0x, jx), u0y = fmaf(0.5f, a0y, jy),
              u0z = fmaf(0.5f, a0z, jz);
  // Q0 = Pi - p* c_s^2 I - u0 u0 + (u0 a0 + a0 u0) / 2
  auto qd = [](float P, float p3_, float uu_, float aa_) {
    return fmaf(uu_, __fadd_rn(aa_, -uu_), __fadd_rn(P, -p3_));
  };
  auto qo = [](float P, float ua, float ub, float aa, float ab) {
    return fmaf(0.5f, fmaf(ua, ab, __fmul_rn(aa, ub)), fmaf(-ua, ub, P));
  };
  const float Q0xx = qd(Pxx, p3, u0x, a0x);
  const float Q0yy = qd(Pyy, p3, u0y, a0y);
  const float Q0zz = qd(Pzz, p3, u0z, a0z);
  const float Q0xy = qo(Pxy, u0x, u0y, a0x, a0y);
  const float Q0xz = qo(Pxz, u0x, u0z, a0x, a0z);
  const float Q0yz = qo(Pyz, u0y, u0z, a0y, a0z);
  const float cnu = __fmul_rn(__fmul_rn(-3.0f, nu), omega);
  auto dot3 = [](float a1, float b1, float a2, float b2, float a3, float b3) {
    return fmaf(a3, b3, fmaf(a2, b2, __fmul_rn(a1, b1)));
  };
  const float Fx = fmaf(cnu, dot3(Q0xx, grx, Q0xy, gry, Q0xz, grz), F0x);
  const float Fy = fmaf(cnu, dot3(Q0xy, grx, Q0yy, gry, Q0yz, grz), F0y);
  const float Fz = fmaf(cnu, dot3(Q0xz, grx, Q0yz, gry, Q0zz, grz), F0z);
  const float ax = __fmul_rn(Fx, inv_rho), ay = __fmul_rn(Fy, inv_rho),
              az = __fmul_rn(Fz, inv_rho);
  const float ux = fmaf(0.5f, ax, jx), uy = fmaf(0.5f, ay, jy), uz = fmaf(0.5f, az, jz);
  const float Axx = qd(Pxx, p3, ux, ax);
  const float Ayy = qd(Pyy, p3, uy, ay);
  const float Azz = qd(Pzz, p3, uz, az);
  const float Axy = qo(Pxy, ux, uy, ax, ay);
  const float Axz = qo(Pxz, ux, uz, ax, az);
  const float Ayz = qo(Pyz, uy, uz, ay, az);
  const float tr = __fadd_rn(__fadd_rn(Axx, Ayy), Azz);
  const float vx = dot3(Axx, ux, Axy, uy, Axz, uz);
  const float vy = dot3(Axy, ux, Ayy, uy, Ayz, uz);
  const float vz = dot3(Axz, ux, Ayz, uy, Azz, uz);
  const float uu = dot3(ux, ux, uy, uy, uz, uz);
  const float ua = dot3(ux, ax, uy, ay, uz, az);
  const float om45 = __fmul_rn(4.5f, __fadd_rn(1.0f, -omega));
  const float k1 = fmaf(-__fmul_rn(om45, tr), 1.0f / 3.0f,
                        fmaf(-1.5f, __fadd_rn(uu, ua), p));
  const float k2 = fmaf(-om45, tr, fmaf(-4.5f, uu, 3.0f));

  // coefficients of P in the separable monomials
  const float om3 = __fmul_rn(3.0f, om45), om6 = __fmul_rn(6.0f, om45),
              om2 = __fmul_rn(2.0f, om45);
  auto coefD = [&](float u_, float a_, float A_) {
    return fmaf(om45, A_, __fmul_rn(__fmul_rn(4.5f, u_), __fadd_rn(u_, a_)));
  };
  auto coefG = [&](float u_, float A_) {
    return fmaf(om3, A_, __fmul_rn(__fmul_rn(13.5f, u_), u_));
  };
  auto coefL = [&](float u_, float a_, float A_, float v_) {
    const float in = fmaf(om3, A_, fmaf(__fmul_rn(4.5f, u_), u_, k2));
    return fmaf(1.5f, a_, fmaf(-om2, v_, __fmul_rn(u_, in)));
  };
  auto coefF = [&](float ua_, float ub_, float aa_, float ab_, float A_) {
    return fmaf(4.5f, fmaf(ua_, ab_, __fmul_rn(ub_, aa_)),
                fmaf(om2, A_, __fmul_rn(__fmul_rn(9.0f, ua_), ub_)));
  };
  const float Dx = coefD(ux, ax, Axx), Dy = coefD(uy, ay, Ayy), Dz = coefD(uz, az, Azz);
  const float Gx = coefG(ux, Axx), Gy = coefG(uy, Ayy), Gz = coefG(uz, Azz);
  const float Lx = coefL(ux, ax, Axx, vx);
  const float Ly = coefL(uy, ay, Ayy, vy);
  const float Lz = coefL(uz, az, Azz, vz);
  const float Fxy = coefF(ux, uy, ax, ay, Axy);
  const float Fxz = coefF(ux, uz, ax, az, Axz);
  const float Fyz = coefF(uy, uz, ay, az, Ayz);
  const float Hxy = __fmul_rn(om6, Axy), Hxz = __fmul_rn(om6, Axz),
              Hyz = __fmul_rn(om6, Ayz);
  const float Mxy = fmaf(ux, Hxy, __fmul_rn(uy, Gx));  // e_x c_y
  const float Mxz = fmaf(ux, Hxz, __fmul_rn(uz, Gx));  // e_x c_z
  const float Myx = fmaf(uy, Hxy, __fmul_rn(ux, Gy));  // e_y c_x
  const float Myz = fmaf(uy, Hyz, __fmul_rn(uz, Gy));  // e_y c_z
  const float Mzx = fmaf(uz, Hxz, __fmul_rn(ux, Gz));  // e_z c_x
  const float Mzy = fmaf(uz, Hyz, __fmul_rn(uy, Gz));  // e_z c_y
  const float X = fmaf(om6, dot3(ux, Ayz, uy, Axz, uz, Axy),
                       __fmul_rn(__fmul_rn(__fmul_rn(27.0f, ux), uy), uz));

  // z transform: Z_ij(cz) for x basis i, y basis j (1, c, e); index cz+1
  float Z00[3], Z10[3], Z20[3], Z01[3], Z11[3], Z02[3];
  {
    const float t00 = k1 + Dz, t10 = Lx + Mzx, t01 = Ly + Mzy;
    Z00[0] = t00 - Lz; Z00[1] = k1; Z00[2] = t00 + Lz;
    Z10[0] = t10 - Fxz; Z10[1] = Lx; Z10[2] = t10 + Fxz;
    Z20[0] = Dx - Mxz; Z20[1] = Dx; Z20[2] = Dx + Mxz;
    Z01[0] = t01 - Fyz; Z01[1] = Ly; Z01[2] = t01 + Fyz;
    Z11[0] = Fxy - X; Z11[1] = Fxy; Z11[2] = Fxy + X;
    Z02[0] = Dy - Myz; Z02[1] = Dy; Z02[2] = Dy + Myz;
  }
  // y transform then x transform, line by line (cy, cz)
#pragma unroll
  for (int kz = 0; kz < 3; ++kz) {
    const float t0 = Z00[kz] + Z02[kz], t1 = Z10[kz] + Myx;
    const float Y0[3] = {t0 - Z01[kz], Z00[kz], t0 + Z01[kz]};
    const float Y1[3] = {t1 - Z11[kz], Z10[kz], t1 + Z11[kz]};
    const float Y2[3] = {Z20[kz] - Mxy, Z20[kz], Z20[kz] + Mxy};
#pragma unroll
    for (int jy = 0; jy < 3; ++jy) {
      const int q = 9 * kz + 3 * jy;
      const float t = Y0[jy] + Y2[jy];
      o.P[q] = t - Y1[jy];
      o.P[q + 1] = Y0[jy];
      o.P[q + 2] = t + Y1[jy];
    }
  }
  o.ux = ux;
  o.uy = uy;
  o.uz = uz;
}

// Everything after the pull and the phi stencil: the compressive vector
// (written to a), the collision, and the stores of f*, u.
template <typename Store, typename IDX>
__device__ __forceinline__ void lb_finish(IDX n, IDX N, const float (&f)[Q],
                                          float phi0, float gx, float gy,
                                          float gz, float ssum,
                                          typename Store::T* __restrict__ fout,
                                          float* __restrict__ u,
                                          float* __restrict__ a,
                                          const Consts& k) {
  const float lap = __fmul_rn(6.0f, fmaf(-(1.0f - wq(REST)), phi0, ssum));
  float ax, ay, az;
  compressive(phi0, gx, gy, gz, ax, ay, az);
  a[n] = ax;
  a[N + n] = ay;
  a[2 * N + n] = az;

  NodeOut o;
  collide(f, phi0, gx, gy, gz, lap, k, o);
#pragma unroll
  for (int q = 0; q < Q; ++q) fout[q * N + n] = Store::encode_w(o.P[q], q);
  u[n] = o.ux;
  u[N + n] = o.uy;
  u[2 * N + n] = o.uz;
}

// IDX is int when 27 N fits in 31 bits (every offset then needs one 32-bit
// multiply-add and one widening address computation), int64_t otherwise.
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
// Bounded wait for phase `parity` of the barrier, sleeping between tests
// so that a waiting warp leaves the issue slots to the others: false after
// the limit (about 0.5 s).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (int i = 0; i < (1 << 20); ++i) {
    if (mbar_try_wait(bar, parity)) return true;
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
    if (s < nseg) mbar_arrive_expect_tx(&bar[0], staged_bytes<Store>(segment_of(s, g).L));
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
    if (!mbar_wait(&bar[cur], (i >> 1) & 1)) {
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
    // stage once every thread is past the barrier below
    if (tid == 0 && s + 2 * G < nseg)
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

// Batched collide-stream: virtual block b of the work-list is row block
// (bx, y, z) of its case; rows of BX threads along x. Blocks stride through
// the work-list (b, b + gridDim.x, ...) so that the rows in flight at any
// time are neighbours, as in a plain launch, and their phi stencils share
// cache lines; the case changes every few thousand rows.
// PERSIST: a resident-sized grid strides through the work-list; otherwise
// one block per work item (the block scheduler does the distribution).
template <typename Store, int BX, bool PERSIST>
__global__ void __launch_bounds__(BX)
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
    const int nbx = (cd.g.nx + BX - 1) / BX;
    const int local = b - cur.cstart;
    const int bx = local % nbx;
    const int row = local / nbx;
    const int y = row % cd.g.ny, z = row / cd.g.ny;
    const int x = bx * BX + threadIdx.x;
    if (x < cd.g.nx)
      lb_node<Store, int>(x, y, z, (const T*)cd.f[fc], (T*)cd.f[1 - fc],
                          cd.phi[pc], cd.u, cd.a, cd.flags, cd.g, cd.k);
  }
}

int staged_segments(const Grid& g) { return ((g.nx + SEG - 1) / SEG) * g.ny * g.nz; }

template <typename Store>
void* staged_kernel(const Grid& g) {
  return ((int64_t)Q * g.N < (int64_t)INT32_MAX)
             ? (void*)lb_collide_staged<Store, int>
             : (void*)lb_collide_staged<Store, int64_t>;
}

template <typename Store>
cudaError_t staged_setup(const Grid& g, int* grid) {
  void* fn = staged_kernel<Store>(g);
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

template <typename Store>
void launch_store(cacl_ctx* c, const void* fin, void* fout, const float* phi) {
  using T = typename Store::T;
  const Grid g = c->g;
  if (lb_staged_ok(c, fin, fout, phi)) {
    const int nseg = staged_segments(g);
    void* fn = staged_kernel<Store>(g);
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
  dim3 block(LB_BX, LB_BY, 1);
  dim3 grid((g.nx + LB_BX - 1) / LB_BX, (g.ny + LB_BY - 1) / LB_BY, g.nz);
  if ((int64_t)Q * g.N < (int64_t)INT32_MAX)
    lb_collide<Store, int><<<grid, block, 0, c->stream>>>(
        (const T*)fin, (T*)fout, phi, c->u, c->a, c->flags, g, c->k);
  else
    lb_collide<Store, int64_t><<<grid, block, 0, c->stream>>>(
        (const T*)fin, (T*)fout, phi, c->u, c->a, c->flags, g, c->k);
}

}  // namespace

// Resident-sized grid of the persistent copy-staged collide-stream (and its
// shared-memory attribute), set once per context outside any graph capture.
cudaError_t lb_init(cacl_ctx* c) {
  switch (c->p.storage) {
    case CACL_F16_SHIFTED: return staged_setup<StoreF16>(c->g, &c->lb_grid);
    case CACL_BF16_SHIFTED: return staged_setup<StoreBF16>(c->g, &c->lb_grid);
    default: return staged_setup<StoreF32>(c->g, &c->lb_grid);
  }
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

cudaError_t launch_lb(cacl_ctx* c, const void* fin, void* fout,
                      const float* phi) {
  switch (c->p.storage) {
    case CACL_F16_SHIFTED: launch_store<StoreF16>(c, fin, fout, phi); break;
    case CACL_BF16_SHIFTED: launch_store<StoreBF16>(c, fin, fout, phi); break;
    default: launch_store<StoreF32>(c, fin, fout, phi); break;
  }
  return cudaGetLastError();
}

int lb_batch_row(int variant) {
  const int r = variant % 3;
  return r == 0 ? 64 : r == 2 ? 256 : 128;
}

bool lb_batch_persistent(int variant) { return variant < 3; }

namespace {
template <typename Store>
void* lb_batch_fn(int variant) {
  switch (variant) {
    case 0: return (void*)lb_collide_batch<Store, 64, true>;
    case 2: return (void*)lb_collide_batch<Store, 256, true>;
    case 3: return (void*)lb_collide_batch<Store, 64, false>;
    case 4: return (void*)lb_collide_batch<Store, 128, false>;
    case 5: return (void*)lb_collide_batch<Store, 256, false>;
    default: return (void*)lb_collide_batch<Store, 128, true>;
  }
}

void* lb_batch_kernel(int storage, int variant) {
  switch (storage) {
    case CACL_F16_SHIFTED: return lb_batch_fn<StoreF16>(variant);
    case CACL_BF16_SHIFTED: return lb_batch_fn<StoreBF16>(variant);
    default: return lb_batch_fn<StoreF32>(variant);
  }
}
}  // namespace

int lb_batch_occupancy(int storage, int variant) {
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, lb_batch_kernel(storage, variant),
                                                lb_batch_row(variant), 0);
  return nb;
}

cudaError_t launch_lb_batch(const CaseDesc* cases, WorkList wl, int storage,
                            int variant, int grid, int fc, int pc, cudaStream_t st) {
  void* fn = lb_batch_kernel(storage, variant);
  void* args[] = {(void*)&cases, (void*)&wl, (void*)&fc, (void*)&pc};
  return cudaLaunchKernel(fn, dim3(grid), dim3(lb_batch_row(variant)), args, 0, st);
}

}  // namespace cacl
