// adjoint.cu -- reverse-mode derivative of the CAC-LB step (hand-written):
// gradients of a loss on the final phi with respect to the contact angle of
// every wall node and to the surface tension.
//
// The forward map of one step n is
//   phi^n  --ghost(theta)-->  phi_g  --collide(f*^{n-1}, sigma)-->  f*^n, u, a
//   (phi_g, u, a) --phi update--> phi*  --correction--> phi^{n+1}.
// Its transpose is applied stage by stage in reverse, every stencil as a
// gather (no atomics, fixed summation order):
//   A1 correction: phi*_bar = (1 + lambda chi'(phi*)) (phi_bar - S/W),
//      S = sum over fluid of phi_bar chi(phi*) (lambda depends on every phi*);
//   A2 phi update: identity, D lap_iso of the fluid-masked phi*_bar, the
//      face fluxes of the MUSCL scheme (per-face adjoints, then a gather),
//      a_bar = kappa grad_iso(phi*_bar on fluid);
//   A3 collide-stream: per node, the collision is recomputed and reversed
//      (moments, forces, regularisation, Guo source); populations go back
//      through the transpose of the pull (a gather with the same bounce-back
//      rule), the phi stencil through the transposes of grad_iso / lap_iso;
//      sigma enters through beta and kappa_phi;
//   A4 ghost map: per wall node, the derivative of the ghost value with
//      respect to its donor stencil and to theta; the stencil part is
//      gathered through a transpose (CSR) of the donor stencils built once.
// Non-smooth points (minmod, upwind choice, chi band edges, |grad| -> 0, the
// cot regularisation) take the derivative of the branch the forward took.
// dL/dtheta and dL/dsigma are accumulated in FP64.
#include <algorithm>
#include <vector>

#include "cacl_internal.cuh"

using namespace cacl;

namespace {

constexpr int AT = 256;  // threads of the element-wise adjoint kernels

// ---------------------------------------------------------------- A1

__global__ void __launch_bounds__(AT)
adj_correct_sum(const float* __restrict__ phib, const float* __restrict__ phis,
                const uint8_t* __restrict__ flags, int64_t N, float eps,
                double* __restrict__ partial) {
  __shared__ double sh[AT];
  double s = 0.0;
  for (int64_t n = (int64_t)blockIdx.x * AT + threadIdx.x; n < N;
       n += (int64_t)gridDim.x * AT) {
    if (flags[n] & FLAG_SOLID) continue;
    const float v = phis[n];
    const float chi = (v > eps && v < 1.f - eps) ? v * (1.f - v) : 0.f;
    s += (double)phib[n] * (double)chi;
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = AT / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

// S / W and lambda for the apply pass, once per step: one block sums the
// block partials of S in a fixed order (thread i adds partials i, i + AT,
// ..., then a fixed tree over the threads).
__global__ void __launch_bounds__(AT)
adj_correct_scalars(const double* __restrict__ partial, int nparts,
                    const MassScalars* __restrict__ ms, float* __restrict__ out) {
  __shared__ double sh[AT];
  double v = 0.0;
  for (int i = threadIdx.x; i < nparts; i += AT) v += __ldcg(partial + i);
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int w = AT / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  const double S = sh[0];
  if (threadIdx.x == 0) {
    const double W = ms->w_sum;
    out[0] = (W > 0.0) ? (float)(S / W) : 0.f;
    out[1] = (W > 0.0) ? ms->lambda_f : 0.f;
  }
}

__global__ void __launch_bounds__(AT)
adj_correct_apply(const float* __restrict__ phib, const float* __restrict__ phis,
                  const uint8_t* __restrict__ flags, int64_t N, float eps,
                  const float* __restrict__ scal, float* __restrict__ phisb) {
  const float s_over_w = scal[0], lam = scal[1];
  const int64_t n = (int64_t)blockIdx.x * AT + threadIdx.x;
  if (n >= N) return;
  if (flags[n] & FLAG_SOLID) {
    phisb[n] = phib[n];
    return;
  }
  const float v = phis[n];
  const float dchi = (v > eps && v < 1.f - eps) ? 1.f - 2.f * v : 0.f;
  phisb[n] = (1.f + lam * dchi) * (phib[n] - s_over_w);
}

// ---------------------------------------------------------------- A2

__device__ __forceinline__ void minmod_d(float a, float b, float& da, float& db) {
  // derivative of minmod(a, b) on the branch taken
  if (a * b <= 0.f) {
    da = db = 0.f;
  } else if (fabsf(a) <= fabsf(b)) {
    da = 1.f;
    db = 0.f;
  } else {
    da = 0.f;
    db = 1.f;
  }
}

__device__ __forceinline__ float minmod_v(float a, float b) {
  const float m = fminf(fabsf(a), fabsf(b));
  return (a * b > 0.f) ? copysignf(m, a) : 0.f;
}

// Per node l and axis d: adjoints of the face flux between l and l + e_d,
// written as contributions to phi at l-1, l, l+1, l+2 and to u_d at l and
// l + 1 (equal halves).
// Node (x, y, z) of a row-shaped launch (128 threads along x, blockIdx.y =
// y, blockIdx.z = z) and the offsets of its neighbours at -2 .. +2 along
// each axis (periodic wrap, any extent >= 1).
template <typename IDX>
struct RowNode {
  int x, y, z;
  IDX n;
  IDX d[3][5];  // d[axis][s + 2]: offset of the node s cells along the axis
  __device__ __forceinline__ bool init(const Grid& g) {
    x = blockIdx.x * 128 + threadIdx.x;
    y = blockIdx.y;
    z = blockIdx.z;
    if (x >= g.nx) return false;
    const IDX nx = g.nx, nxy = (IDX)g.nx * g.ny;
    n = (IDX)x + nx * y + nxy * z;
    const int c[3] = {x, y, z}, e[3] = {g.nx, g.ny, g.nz};
    const IDX st[3] = {1, nx, nxy};
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int s = -2; s <= 2; ++s) {
        int j = c[a] + s;
        if (j < 0) j += e[a];
        if (j < 0) j += e[a];
        if (j >= e[a]) j -= e[a];
        if (j >= e[a]) j -= e[a];
        d[a][s + 2] = (IDX)(j - c[a]) * st[a];
      }
    return true;
  }
};

template <typename IDX>
__global__ void __launch_bounds__(128)
adj_phase_faces(const float* __restrict__ phi, const float* __restrict__ u,
                const uint8_t* __restrict__ flags,
                const float* __restrict__ phisb, float* __restrict__ face,
                Grid g) {
  RowNode<IDX> rn;
  if (!rn.init(g)) return;
  const IDX n = rn.n;
  const IDX N = (IDX)g.N;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    auto at = [&](int s) -> IDX { return n + rn.d[d][s + 2]; };
    float* fc = face + (IDX)d * 5 * N;
    float c0 = 0.f, c1 = 0.f, c2 = 0.f, c3 = 0.f, cu = 0.f;
    const IDX l = n, r = at(1);
    if (!(flags[l] & FLAG_SOLID) && !(flags[r] & FLAG_SOLID)) {
      const IDX lm = at(-1), rp = at(2);
      const float pm = phi[lm], pl = phi[l], pr = phi[r], pp = phi[rp];
      const float fb = phisb[r] - phisb[l];  // d L / d F(l, r)
      const float uf = 0.5f * (u[d * N + l] + u[d * N + r]);
      float up;
      if (uf >= 0.f) {
        float da, db;
        minmod_d(pl - pm, pr - pl, da, db);
        up = pl + 0.5f * minmod_v(pl - pm, pr - pl);
        const float upb = fb * uf;
        // up = pl + s_l / 2, s_l = minmod(pl - pm, pr - pl)
        c1 += upb * (1.f + 0.5f * (da - db));
        c0 += upb * (-0.5f * da);
        c2 += upb * (0.5f * db);
      } else {
        float da, db;
        minmod_d(pr - pl, pp - pr, da, db);
        up = pr - 0.5f * minmod_v(pr - pl, pp - pr);
        const float upb = fb * uf;
        // up = pr - s_r / 2, s_r = minmod(pr - pl, pp - pr)
        c2 += upb * (1.f - 0.5f * (da - db));
        c1 += upb * (0.5f * da);
        c3 += upb * (-0.5f * db);
      }
      cu = 0.5f * fb * up;
    }
    fc[n] = c0;
    fc[N + n] = c1;
    fc[2 * N + n] = c2;
    fc[3 * N + n] = c3;
    fc[4 * N + n] = cu;
  }
}

template <typename IDX>
__global__ void __launch_bounds__(128)
adj_phase_gather(const uint8_t* __restrict__ flags,
                 const float* __restrict__ phisb, const float* __restrict__ face,
                 float* __restrict__ phigb, float* __restrict__ ub,
                 float* __restrict__ ab, Grid g, Consts k) {
  RowNode<IDX> rn;
  if (!rn.init(g)) return;
  const IDX n = rn.n;
  const IDX N = (IDX)g.N;
  // fluid-masked phi*_bar at the 27 neighbours: lap_iso and grad_iso of it
  float lsum = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    if (q == REST) continue;
    const IDX m = n + rn.d[0][2 + cx(q)] + rn.d[1][2 + cy(q)] + rn.d[2][2 + cz(q)];
    const float v = (flags[m] & FLAG_SOLID) ? 0.f : phisb[m];
    lsum += wq(q) * v;
    gx += 3.f * wq(q) * cx(q) * v;
    gy += 3.f * wq(q) * cy(q) * v;
    gz += 3.f * wq(q) * cz(q) * v;
  }
  const float own = (flags[n] & FLAG_SOLID) ? 0.f : phisb[n];
  const float lapb = 6.f * (lsum - (1.f - wq(REST)) * own);
  float acc = phisb[n] + k.mobility * lapb;
  // face flux contributions along each axis
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    auto at = [&](int s) -> IDX { return n + rn.d[d][s + 2]; };
    const float* fc = face + (IDX)d * 5 * N;
    // node n is position l-1 of face (n+1), l of face n, l+1 of face (n-1),
    // l+2 of face (n-2)
    acc += fc[at(1)] + fc[N + n] + fc[2 * N + at(-1)] + fc[3 * N + at(-2)];
    ub[d * N + n] = fc[4 * N + n] + fc[4 * N + at(-1)];
  }
  phigb[n] = acc;
  ab[n] = k.kappa * gx;
  ab[N + n] = k.kappa * gy;
  ab[2 * N + n] = k.kappa * gz;
}

// ---------------------------------------------------------------- A3

struct LbAdjOut {
  float fb[Q];
  float gbx, gby, gbz, lapb, phi0b;
  float beta4b, kphib;
};

// Recompute the collision of one node (same arithmetic as the forward) and
// apply its transpose to the adjoints of f*, u and the compressive vector.
__device__ __forceinline__ void collide_adj(const float (&f)[Q], float phi0,
                                            float gx, float gy, float gz,
                                            float lap, const Consts& k,
                                            const float (&fob)[Q], float ubx,
                                            float uby, float ubz, float acbx,
                                            float acby, float acbz, LbAdjOut& o) {
  // ---- forward
  float p = f[REST], jx = 0.f, jy = 0.f, jz = 0.f;
  float Pxx = 0.f, Pyy = 0.f, Pzz = 0.f, Pxy = 0.f, Pxz = 0.f, Pyz = 0.f;
#pragma unroll
  for (int q = 0; q < REST; ++q) {
    const float s = f[q] + f[opp(q)];
    const float d = f[q] - f[opp(q)];
    p += s;
    jx += cx(q) * d;
    jy += cy(q) * d;
    jz += cz(q) * d;
    Pxx += (cx(q) * cx(q)) * s;
    Pyy += (cy(q) * cy(q)) * s;
    Pzz += (cz(q) * cz(q)) * s;
    Pxy += (cx(q) * cy(q)) * s;
    Pxz += (cx(q) * cz(q)) * s;
    Pyz += (cy(q) * cz(q)) * s;
  }
  const float rho = k.rho_g + k.drho * phi0;
  const float mu = k.mu_g + k.dmu * phi0;
  const float inv_rho = 1.0f / rho;
  const float nu = mu * inv_rho;
  const float omega = 1.0f / (0.5f + 3.0f * nu);
  const float grx = k.drho * gx, gry = k.drho * gy, grz = k.drho * gz;
  const float cub_ = phi0 * (phi0 - 1.0f) * (phi0 - 0.5f);
  const float muphi = k.beta4 * cub_ - k.kappa_phi * lap;
  const float p3 = p * (1.0f / 3.0f);
  const float rb = rho - k.rho_g;
  const float F0x = muphi * gx - p3 * grx + rb * k.gx;
  const float F0y = muphi * gy - p3 * gry + rb * k.gy;
  const float F0z = muphi * gz - p3 * grz + rb * k.gz;
  const float a0x = F0x * inv_rho, a0y = F0y * inv_rho, a0z = F0z * inv_rho;
  const float u0x = jx + 0.5f * a0x, u0y = jy + 0.5f * a0y, u0z = jz + 0.5f * a0z;
  const float Q0xx = Pxx - p3 - u0x * u0x + u0x * a0x;
  const float Q0yy = Pyy - p3 - u0y * u0y + u0y * a0y;
  const float Q0zz = Pzz - p3 - u0z * u0z + u0z * a0z;
  const float Q0xy = Pxy - u0x * u0y + 0.5f * (u0x * a0y + a0x * u0y);
  const float Q0xz = Pxz - u0x * u0z + 0.5f * (u0x * a0z + a0x * u0z);
  const float Q0yz = Pyz - u0y * u0z + 0.5f * (u0y * a0z + a0y * u0z);
  const float cnu = -3.0f * nu * omega;
  const float Qgx = Q0xx * grx + Q0xy * gry + Q0xz * grz;
  const float Qgy = Q0xy * grx + Q0yy * gry + Q0yz * grz;
  const float Qgz = Q0xz * grx + Q0yz * gry + Q0zz * grz;
  const float Fx = F0x + cnu * Qgx, Fy = F0y + cnu * Qgy, Fz = F0z + cnu * Qgz;
  const float ax = Fx * inv_rho, ay = Fy * inv_rho, az = Fz * inv_rho;
  const float ux = jx + 0.5f * ax, uy = jy + 0.5f * ay, uz = jz + 0.5f * az;
  const float Axx = Pxx - p3 - ux * ux + ux * ax;
  const float Ayy = Pyy - p3 - uy * uy + uy * ay;
  const float Azz = Pzz - p3 - uz * uz + uz * az;
  const float Axy = Pxy - ux * uy + 0.5f * (ux * ay + ax * uy);
  const float Axz = Pxz - ux * uz + 0.5f * (ux * az + ax * uz);
  const float Ayz = Pyz - uy * uz + 0.5f * (uy * az + ay * uz);
  const float tr = Axx + Ayy + Azz;
  const float vx = Axx * ux + Axy * uy + Axz * uz;
  const float vy = Axy * ux + Ayy * uy + Ayz * uz;
  const float vz = Axz * ux + Ayz * uy + Azz * uz;
  const float om45 = 4.5f * (1.0f - omega);
  const float uu = ux * ux + uy * uy + uz * uz;
  const float k2 = 3.0f - 4.5f * uu - om45 * tr;

  // ---- reverse
  float k1b = wq(REST) * fob[REST], k2b = 0.f, om45b = 0.f;
  float ubx_ = ubx, uby_ = uby, ubz_ = ubz;  // adjoint of u
  float abx = 0.f, aby = 0.f, abz = 0.f;     // adjoint of a
  float vbx = 0.f, vby = 0.f, vbz = 0.f;
  float Abxx = 0.f, Abyy = 0.f, Abzz = 0.f, Abxy = 0.f, Abxz = 0.f, Abyz = 0.f;
#pragma unroll
  for (int q = 0; q < REST; ++q) {
    const int X = cx(q), Y = cy(q), Z = cz(q);
    const float cu = X * ux + Y * uy + Z * uz;
    const float ca = X * ax + Y * ay + Z * az;
    const float cAu = X * vx + Y * vy + Z * vz;
    const float cAc = (X * X) * Axx + (Y * Y) * Ayy + (Z * Z) * Azz +
                      2.0f * ((X * Y) * Axy + (X * Z) * Axz + (Y * Z) * Ayz);
    const float cu2 = cu * cu;
    const float Eb = wq(q) * (fob[q] + fob[opp(q)]);
    const float Ob = wq(q) * (fob[q] - fob[opp(q)]);
    k1b += Eb;
    const float cuB = Eb * (9.f * cu + 4.5f * ca) +
                      Ob * (k2 + 13.5f * cu2 + 3.f * om45 * cAc);
    const float caB = 4.5f * cu * Eb + 1.5f * Ob;
    const float cAcB = om45 * Eb + 3.f * om45 * cu * Ob;
    const float cAuB = -2.f * om45 * Ob;
    k2b += cu * Ob;
    om45b += cAc * Eb + (3.f * cu * cAc - 2.f * cAu) * Ob;
    ubx_ += X * cuB;
    uby_ += Y * cuB;
    ubz_ += Z * cuB;
    abx += X * caB;
    aby += Y * caB;
    abz += Z * caB;
    vbx += X * cAuB;
    vby += Y * cAuB;
    vbz += Z * cAuB;
    Abxx += (X * X) * cAcB;
    Abyy += (Y * Y) * cAcB;
    Abzz += (Z * Z) * cAcB;
    Abxy += 2.f * (X * Y) * cAcB;
    Abxz += 2.f * (X * Z) * cAcB;
    Abyz += 2.f * (Y * Z) * cAcB;
  }
  // k1 = p - 1.5 (uu + ua) - om45 tr / 3 ; k2 = 3 - 4.5 uu - om45 tr
  float pb = k1b;
  float uub = -1.5f * k1b - 4.5f * k2b;
  const float uab = -1.5f * k1b;
  om45b += -(tr * (1.f / 3.f)) * k1b - tr * k2b;
  const float trb = -(om45 * (1.f / 3.f)) * k1b - om45 * k2b;
  float omegab = -4.5f * om45b;
  // ua = u.a, uu = u.u
  ubx_ += ax * uab + 2.f * ux * uub;
  uby_ += ay * uab + 2.f * uy * uub;
  ubz_ += az * uab + 2.f * uz * uub;
  abx += ux * uab;
  aby += uy * uab;
  abz += uz * uab;
  // v = A u
  Abxx += vbx * ux + trb;
  Abyy += vby * uy + trb;
  Abzz += vbz * uz + trb;
  Abxy += vbx * uy + vby * ux;
  Abxz += vbx * uz + vbz * ux;
  Abyz += vby * uz + vbz * uy;
  ubx_ += Axx * vbx + Axy * vby + Axz * vbz;
  uby_ += Axy * vbx + Ayy * vby + Ayz * vbz;
  ubz_ += Axz * vbx + Ayz * vby + Azz * vbz;
  // A = P - p3 I - u u + (u a + a u)/2
  float Pbxx = Abxx, Pbyy = Abyy, Pbzz = Abzz, Pbxy = Abxy, Pbxz = Abxz, Pbyz = Abyz;
  float p3b = -(Abxx + Abyy + Abzz);
  ubx_ += (-2.f * ux + ax) * Abxx + (-uy + 0.5f * ay) * Abxy + (-uz + 0.5f * az) * Abxz;
  uby_ += (-2.f * uy + ay) * Abyy + (-ux + 0.5f * ax) * Abxy + (-uz + 0.5f * az) * Abyz;
  ubz_ += (-2.f * uz + az) * Abzz + (-ux + 0.5f * ax) * Abxz + (-uy + 0.5f * ay) * Abyz;
  abx += ux * Abxx + 0.5f * uy * Abxy + 0.5f * uz * Abxz;
  aby += uy * Abyy + 0.5f * ux * Abxy + 0.5f * uz * Abyz;
  abz += uz * Abzz + 0.5f * ux * Abxz + 0.5f * uy * Abyz;
  // u = j + a/2
  float jbx = ubx_, jby = uby_, jbz = ubz_;
  abx += 0.5f * ubx_;
  aby += 0.5f * uby_;
  abz += 0.5f * ubz_;
  // a = F / rho
  const float Fbx = inv_rho * abx, Fby = inv_rho * aby, Fbz = inv_rho * abz;
  float inv_rhob = Fx * abx + Fy * aby + Fz * abz;
  // F = F0 + cnu (Q0 gr)
  float F0bx = Fbx, F0by = Fby, F0bz = Fbz;
  const float cnub = Fbx * Qgx + Fby * Qgy + Fbz * Qgz;
  const float Qbxx = cnu * Fbx * grx, Qbyy = cnu * Fby * gry, Qbzz = cnu * Fbz * grz;
  const float Qbxy = cnu * (Fbx * gry + Fby * grx);
  const float Qbxz = cnu * (Fbx * grz + Fbz * grx);
  const float Qbyz = cnu * (Fby * grz + Fbz * gry);
  float grbx = cnu * (Q0xx * Fbx + Q0xy * Fby + Q0xz * Fbz);
  float grby = cnu * (Q0xy * Fbx + Q0yy * Fby + Q0yz * Fbz);
  float grbz = cnu * (Q0xz * Fbx + Q0yz * Fby + Q0zz * Fbz);
  // Q0 = P - p3 I - u0 u0 + (u0 a0 + a0 u0)/2
  Pbxx += Qbxx;
  Pbyy += Qbyy;
  Pbzz += Qbzz;
  Pbxy += Qbxy;
  Pbxz += Qbxz;
  Pbyz += Qbyz;
  p3b -= Qbxx + Qbyy + Qbzz;
  float u0bx = (-2.f * u0x + a0x) * Qbxx + (-u0y + 0.5f * a0y) * Qbxy + (-u0z + 0.5f * a0z) * Qbxz;
  float u0by = (-2.f * u0y + a0y) * Qbyy + (-u0x + 0.5f * a0x) * Qbxy + (-u0z + 0.5f * a0z) * Qbyz;
  float u0bz = (-2.f * u0z + a0z) * Qbzz + (-u0x + 0.5f * a0x) * Qbxz + (-u0y + 0.5f * a0y) * Qbyz;
  float a0bx = u0x * Qbxx + 0.5f * u0y * Qbxy + 0.5f * u0z * Qbxz;
  float a0by = u0y * Qbyy + 0.5f * u0x * Qbxy + 0.5f * u0z * Qbyz;
  float a0bz = u0z * Qbzz + 0.5f * u0x * Qbxz + 0.5f * u0y * Qbyz;
  // u0 = j + a0/2
  jbx += u0bx;
  jby += u0by;
  jbz += u0bz;
  a0bx += 0.5f * u0bx;
  a0by += 0.5f * u0by;
  a0bz += 0.5f * u0bz;
  // a0 = F0 / rho
  F0bx += inv_rho * a0bx;
  F0by += inv_rho * a0by;
  F0bz += inv_rho * a0bz;
  inv_rhob += F0x * a0bx + F0y * a0by + F0z * a0bz;
  // cnu = -3 nu omega
  float nub = -3.f * omega * cnub;
  omegab += -3.f * nu * cnub;
  // F0 = muphi g - p3 gr + rb g_ext
  const float muphib = F0bx * gx + F0by * gy + F0bz * gz;
  float gbx = muphi * F0bx, gby = muphi * F0by, gbz = muphi * F0bz;
  p3b -= F0bx * grx + F0by * gry + F0bz * grz;
  grbx -= p3 * F0bx;
  grby -= p3 * F0by;
  grbz -= p3 * F0bz;
  const float rbb = F0bx * k.gx + F0by * k.gy + F0bz * k.gz;
  pb += p3b * (1.f / 3.f);
  // muphi = beta4 phi(phi-1)(phi-1/2) - kappa_phi lap
  float phi0b = k.beta4 * (3.f * phi0 * phi0 - 3.f * phi0 + 0.5f) * muphib;
  const float lapb = -k.kappa_phi * muphib;
  o.beta4b = cub_ * muphib;
  o.kphib = -lap * muphib;
  // gr = drho g
  gbx += k.drho * grbx;
  gby += k.drho * grby;
  gbz += k.drho * grbz;
  // omega = 1/(1/2 + 3 nu), nu = mu / rho, rho, mu linear in phi
  nub += -3.f * omega * omega * omegab;
  const float mub = inv_rho * nub;
  inv_rhob += mu * nub;
  float rhob = rbb - inv_rho * inv_rho * inv_rhob;
  phi0b += k.dmu * mub + k.drho * rhob;
  // compressive vector a_c = phi (1 - phi) g / |g|. The rotation of the
  // unit normal h = g / |g| has derivative phi (1 - phi) (I - h h) / |g|,
  // whose gain phi (1 - phi) / |g| is width / 4 on an equilibrium interface
  // but unbounded on the plateaus of the bulk phases (|g| << |phi (1 - phi)|,
  // e.g. where phi overshoots 1 inside a drop): there the exact
  // linearisation of the discrete map grows without bound over long
  // rollouts although the map's response stays below |phi (1 - phi)|. The
  // rotation term is therefore kept only inside the interface band of the
  // volume correction, eps_phi < phi < 1 - eps_phi (Eq.
  // interface_weight_mass_correction), and the normal is held fixed in the
  // bulk phases.
  const float g2 = gx * gx + gy * gy + gz * gz;
  if (g2 >= 1e-24f) {
    const float ig = rsqrtf(g2);
    const float hx = gx * ig, hy = gy * ig, hz = gz * ig;
    const float hb = hx * acbx + hy * acby + hz * acbz;
    const float pp = phi0 * (1.f - phi0);
    phi0b += (1.f - 2.f * phi0) * hb;
    if (phi0 > k.eps_phi && phi0 < 1.f - k.eps_phi) {
      gbx += pp * ig * (acbx - hb * hx);
      gby += pp * ig * (acby - hb * hy);
      gbz += pp * ig * (acbz - hb * hz);
    }
  }
  // moments
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int X = cx(q), Y = cy(q), Z = cz(q);
    o.fb[q] = pb + X * jbx + Y * jby + Z * jbz + (X * X) * Pbxx + (Y * Y) * Pbyy +
              (Z * Z) * Pbzz + (X * Y) * Pbxy + (X * Z) * Pbxz + (Y * Z) * Pbyz;
  }
  o.gbx = gbx;
  o.gby = gby;
  o.gbz = gbz;
  o.lapb = lapb;
  o.phi0b = phi0b;
}

// Per fluid node: the collision recomputed from the taped pull and reversed.
// Block = 128 nodes of one x row (blockIdx.y = y, blockIdx.z = z); each
// warp's dL/dsigma share is added to its own slot sig_acc[4 block + warp]
// (no block barrier: a warp that finishes early, or holds only nodes past
// the row's end, leaves at once).
// The adjoint of the node's post-collision populations f*_q(n) is gathered
// from the pulled-population adjoints of the later step (finb_later, or
// zero when null) through the transpose of the pull: f*_q(n) fed
// f_in[q](n + c_q), or f_in[opp q](n) when n + c_q is solid (halfway
// bounce-back; only nodes flagged near have a solid neighbour).
template <typename IDX>
__global__ void __launch_bounds__(128)
adj_lb_node(const float* __restrict__ fprev, const float* __restrict__ phig,
            const uint8_t* __restrict__ flags, const float* __restrict__ finb_later,
            const float* __restrict__ ub, const float* __restrict__ acb,
            float* __restrict__ finb, float* __restrict__ nodeb,
            double* __restrict__ sig_acc, Grid g, Consts k, float dbeta4_dsigma,
            float dkphi_dsigma) {
  const int x = blockIdx.x * 128 + threadIdx.x;
  const int y = blockIdx.y, z = blockIdx.z;
  const IDX N = (IDX)g.N;
  const IDX nx = g.nx;
  const IDX nxy = (IDX)g.nx * g.ny;
  const IDX n = (IDX)x + nx * y + nxy * z;
  double sig = 0.0;
  if (x < g.nx && !(flags[n] & FLAG_SOLID)) {
    const IDX xo[3] = {(IDX)wrap(x, -1, g.nx), (IDX)x, (IDX)wrap(x, 1, g.nx)};
    const IDX yo[3] = {wrap(y, -1, g.ny) * nx, y * nx, wrap(y, 1, g.ny) * nx};
    const IDX zo[3] = {wrap(z, -1, g.nz) * nxy, z * nxy, wrap(z, 1, g.nz) * nxy};
    const bool near = flags[n] & FLAG_NEAR;
    float f[Q], fob[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const IDX src = xo[1 - cx(q)] + yo[1 - cy(q)] + zo[1 - cz(q)];
      const bool bb = near && (q != REST) && (flags[src] & FLAG_SOLID);
      f[q] = bb ? fprev[opp(q) * N + n] : fprev[q * N + src];
      if (finb_later) {
        const IDX dst = xo[1 + cx(q)] + yo[1 + cy(q)] + zo[1 + cz(q)];
        const bool bt = near && (q != REST) && (flags[dst] & FLAG_SOLID);
        fob[q] = bt ? finb_later[opp(q) * N + n] : finb_later[q * N + dst];
      } else {
        fob[q] = 0.f;
      }
    }
    float gx = 0.f, gy = 0.f, gz = 0.f, ssum = 0.f;
#pragma unroll
    for (int q = 0; q < REST; ++q) {
      const float vp = __ldg(phig + (xo[1 + cx(q)] + yo[1 + cy(q)] + zo[1 + cz(q)]));
      const float vm = __ldg(phig + (xo[1 - cx(q)] + yo[1 - cy(q)] + zo[1 - cz(q)]));
      stencil_pair(q, vp, vm, gx, gy, gz, ssum);
    }
    const float phi0 = phig[n];
    const float lap = 6.0f * (ssum - (1.0f - wq(REST)) * phi0);
    LbAdjOut o;
    collide_adj(f, phi0, gx, gy, gz, lap, k, fob, ub[n], ub[N + n], ub[2 * N + n],
                acb[n], acb[N + n], acb[2 * N + n], o);
#pragma unroll
    for (int q = 0; q < Q; ++q) finb[q * N + n] = o.fb[q];
    nodeb[n] = o.gbx;
    nodeb[N + n] = o.gby;
    nodeb[2 * N + n] = o.gbz;
    nodeb[3 * N + n] = o.lapb;
    nodeb[4 * N + n] = o.phi0b;
    sig = (double)o.beta4b * dbeta4_dsigma + (double)o.kphib * dkphi_dsigma;
  } else if (x < g.nx) {
#pragma unroll
    for (int q = 0; q < Q; ++q) finb[q * N + n] = 0.f;
#pragma unroll
    for (int c = 0; c < 5; ++c) nodeb[c * N + n] = 0.f;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) sig += __shfl_down_sync(0xffffffffu, sig, off);
  // each warp owns one accumulator slot: the steps add to it in turn and
  // the slots are summed once after the last step
  if ((threadIdx.x & 31) == 0)
    sig_acc[4 * (blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z)) +
            (threadIdx.x >> 5)] += sig;
}

// Transpose of the phi stencil (gradient, Laplacian, own value) of the
// collide-stream, gathered per node; same launch shape as adj_lb_node.
template <typename IDX>
__global__ void __launch_bounds__(128)
adj_lb_gather(const float* __restrict__ nodeb, float* __restrict__ phigb, Grid g) {
  const int x = blockIdx.x * 128 + threadIdx.x;
  if (x >= g.nx) return;
  const int y = blockIdx.y, z = blockIdx.z;
  const IDX N = (IDX)g.N;
  const IDX nx = g.nx;
  const IDX nxy = (IDX)g.nx * g.ny;
  const IDX n = (IDX)x + nx * y + nxy * z;
  const IDX xo[3] = {(IDX)wrap(x, -1, g.nx), (IDX)x, (IDX)wrap(x, 1, g.nx)};
  const IDX yo[3] = {wrap(y, -1, g.ny) * nx, y * nx, wrap(y, 1, g.ny) * nx};
  const IDX zo[3] = {wrap(z, -1, g.nz) * nxy, z * nxy, wrap(z, 1, g.nz) * nxy};
  // phi at y entered grad_iso and lap_iso of every fluid x = y - c_i, and
  // phi0 of x = y
  float acc = nodeb[4 * N + n];
  float lsum = 0.f;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    if (q == REST) continue;
    const IDX m = xo[1 - cx(q)] + yo[1 - cy(q)] + zo[1 - cz(q)];  // y - c_q
    acc += 3.f * wq(q) *
           (cx(q) * nodeb[m] + cy(q) * nodeb[N + m] + cz(q) * nodeb[2 * N + m]);
    lsum += wq(q) * nodeb[3 * N + m];
  }
  acc += 6.f * (lsum - (1.f - wq(REST)) * nodeb[3 * N + n]);
  phigb[n] += acc;
}

// ---------------------------------------------------------------- A4

// Per wall node: d ghost / d phi at the 27 points of the donor stencil
// (written to wd[w][q]) and dL/dtheta accumulated in FP64.
__global__ void __launch_bounds__(128)
adj_ghost_node(const float* __restrict__ phi, const int32_t* __restrict__ idx,
               const int32_t* __restrict__ donor, const int8_t* __restrict__ qstar,
               const float* __restrict__ nw, const float* __restrict__ cot_c,
               const float* __restrict__ theta_deg, const float* __restrict__ phigb,
               float* __restrict__ wd, double* __restrict__ thetab, int W, Grid g) {
  const int w = blockIdx.x * 128 + threadIdx.x;
  if (w >= W) return;
  const int d = donor[w];
  const int x = d % g.nx;
  const int r = d / g.nx;
  const int y = r % g.ny;
  const int z = r / g.ny;
  const int xo[3] = {wrap(x, -1, g.nx), x, wrap(x, 1, g.nx)};
  const int yo[3] = {wrap(y, -1, g.ny) * g.nx, y * g.nx, wrap(y, 1, g.ny) * g.nx};
  const int64_t nxy = (int64_t)g.nx * g.ny;
  const int64_t zo[3] = {wrap(z, -1, g.nz) * nxy, z * nxy, wrap(z, 1, g.nz) * nxy};
  float Gx, Gy, Gz, ssum;
  phi_stencil(phi, xo, yo, zo, Gx, Gy, Gz, ssum);
  const float phi_f = phi[d];
  const float nx_ = nw[w], ny_ = nw[W + w], nz_ = nw[2 * W + w];
  const int q = qstar[w];
  const float rx = -(float)(q % 3 - 1), ry = -(float)((q / 3) % 3 - 1),
              rz = -(float)(q / 9 - 1);
  const float gn = Gx * nx_ + Gy * ny_ + Gz * nz_;
  const float px = Gx - gn * nx_, py = Gy - gn * ny_, pz = Gz - gn * nz_;
  const float t = sqrtf(px * px + py * py + pz * pz);
  const float cot = cot_c[w];
  const float nr = nx_ * rx + ny_ * ry + nz_ * rz;
  // D = gc . r_fs = gpar . r - t cot (n . r); g = phi_f + lambda_s D
  const float D = px * rx + py * ry + pz * rz - t * cot * nr;
  const float l4 = 4.f * phi_f * (1.f - phi_f);
  const float lam = sqrtf(fmaxf(0.f, l4));
  const float dlam = (l4 > 0.f) ? (2.f - 4.f * phi_f) / lam : 0.f;
  // dD/dG = r - (n.r) n - cot (n.r) gpar / t
  const float it = (t > 0.f) ? 1.f / t : 0.f;
  const float vx = rx - nr * nx_ - cot * nr * px * it;
  const float vy = ry - nr * ny_ - cot * nr * py * it;
  const float vz = rz - nr * nz_ - cot * nr * pz * it;
  const float gb = phigb[idx[w]];
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    float dg = lam * 3.f * wq(i) * (cx(i) * vx + cy(i) * vy + cz(i) * vz);
    if (i == REST) dg += 1.f + dlam * D;
    wd[(int64_t)w * Q + i] = gb * dg;
  }
  // theta: cot(theta_c) = -cot(theta); d/dtheta_deg of -t cot(theta_c) (n.r)
  // = -t (n.r) d cot(theta_c)/dtheta_deg, with d cot(theta_c)/dtheta =
  // 1 / sin^2(theta) per radian (0 where the cot was regularised)
  const float th = theta_deg[w] * (3.14159265358979f / 180.f);
  const float s = sinf(th);
  const bool reg = fabsf(s) < 1e-6f;
  const float dcot = reg ? 0.f : (3.14159265358979f / 180.f) / (s * s);
  thetab[w] += (double)(gb * lam * (-t * nr * dcot));
}

// phi^n_bar from phi_g_bar: identity except at wall nodes (their previous
// value is overwritten), plus the donor-stencil contributions gathered
// through the transpose rows (node -> list of (w, i) entries of wd).
__global__ void __launch_bounds__(AT)
adj_ghost_gather(const uint8_t* __restrict__ flags, const float* __restrict__ phigb,
                 const int32_t* __restrict__ row_start,
                 const int32_t* __restrict__ row_entry,
                 const float* __restrict__ wd, float* __restrict__ phib, int64_t N,
                 const float* __restrict__ phis_next, float eps,
                 double* __restrict__ partial) {
  __shared__ double sh[AT / 32];
  const int64_t n = (int64_t)blockIdx.x * AT + threadIdx.x;
  double s = 0.0;
  if (n < N) {
    const uint8_t fl = flags[n];
    float v = (fl & FLAG_WALL) ? 0.f : phigb[n];
    for (int e = row_start[n]; e < row_start[n + 1]; ++e) v += wd[row_entry[e]];
    phib[n] = v;
    // the next (earlier) step's correction adjoint needs S = sum over fluid
    // of phi_bar chi(phi*): its block partial, formed here (adj_correct_sum
    // on its own otherwise)
    if (phis_next && !(fl & FLAG_SOLID)) {
      const float w = phis_next[n];
      const float chi = (w > eps && w < 1.f - eps) ? w * (1.f - w) : 0.f;
      s = (double)v * (double)chi;
    }
  }
  if (!phis_next) return;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
#pragma unroll
    for (int i = 0; i < AT / 32; ++i) t += sh[i];
    partial[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(128)
sum_partials(const double* __restrict__ partial, int n, double* __restrict__ out) {
  __shared__ double sh[128];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += 128) s += partial[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = 64; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out += sh[0];
}

int nblk(int64_t n, int t) { return (int)((n + t - 1) / t); }

}  // namespace

// ------------------------------------------------------------ host side

struct AdjointState {
  int nsteps = 0, every = 0;
  // two-level checkpointing: outer checkpoints every `outer` steps (0: one
  // level); the inner checkpoints (every `every` steps) then cover one outer
  // segment at a time and are rebuilt by a recompute in the backward pass
  int outer = 0;
  std::vector<float*> ck1_f, ck1_phi;
  MassScalars* ck1_mass = nullptr;
  int64_t N = 0;
  int W = 0;
  // checkpoints: f* (27N floats) and phi (N) at steps 0, every, 2 every, ...
  std::vector<float*> ck_f, ck_phi;
  MassScalars* ck_mass = nullptr;  // mass record (incl. rounding key) per checkpoint
  // per-step tape of one segment
  std::vector<float*> t_fprev, t_phipre, t_phig, t_u, t_a, t_phis;
  MassScalars* t_mass = nullptr;  // [every]
  // adjoint fields
  // fb / fb2: adjoints of the pulled populations f_in of a step and of the
  // step before (ping-pong)
  float *fb = nullptr, *fb2 = nullptr, *phib = nullptr, *phisb = nullptr,
        *phigb = nullptr, *ub = nullptr, *ab = nullptr, *face = nullptr,
        *nodeb = nullptr, *wd = nullptr;
  double *thetab = nullptr, *sigmab = nullptr, *partial = nullptr;
  double* sig_acc = nullptr;  // per-block dL/dsigma, summed after the last step
  // GPU time of the last backward: the taped recomputes of the segments
  // (and of the outer segments with two levels) and the whole call
  double t_recompute_ms = 0.0, t_total_ms = 0.0;
  float* scal = nullptr;  // S / W and lambda of the correction adjoint
  int npart = 0;
  int32_t *row_start = nullptr, *row_entry = nullptr;
  bool forward_done = false;
  // CUDA graphs of the backward steps of one full-length segment (every
  // segment but the first one processed), by which of fb / fb2 holds the
  // later step's adjoints when it starts (slot 0: the lower address); valid
  // while graph_key (the constants, sizes and context buffers the launches
  // bake in) matches
  cudaGraphExec_t seg_graph[2] = {nullptr, nullptr};
  std::vector<unsigned char> graph_key;
};

namespace cacl {
void adjoint_free(AdjointState* s) {
  if (!s) return;
  for (auto& gx : s->seg_graph)
    if (gx) cudaGraphExecDestroy(gx);
  for (auto* v : {&s->ck_f, &s->ck_phi, &s->ck1_f, &s->ck1_phi, &s->t_fprev,
                  &s->t_phipre, &s->t_phig, &s->t_u, &s->t_a, &s->t_phis})
    for (float* p : *v) cudaFree(p);
  void* bufs[] = {s->ck_mass, s->ck1_mass, s->t_mass, s->fb, s->fb2, s->phib, s->phisb, s->phigb, s->ub,
                  s->ab, s->face, s->nodeb, s->wd, s->thetab, s->sigmab,
                  s->partial, s->sig_acc, s->scal, s->row_start, s->row_entry};
  for (void* b : bufs)
    if (b) cudaFree(b);
  delete s;
}
}  // namespace cacl

namespace {

cacl_status afail(cacl_ctx* c, cacl_status st, const std::string& m) {
  c->err = m;
  return st;
}

#define ACK(expr, where)                                                      \
  do {                                                                        \
    cudaError_t e_ = (expr);                                                  \
    if (e_ != cudaSuccess)                                                    \
      return afail(c, CACL_ERR_CUDA, std::string(where) + ": " +             \
                                         cudaGetErrorString(e_));             \
  } while (0)

template <typename T>
cudaError_t alloc(T** p, size_t count) {
  return cudaMalloc((void**)p, sizeof(T) * (count > 0 ? count : 1));
}

// CSR transpose of the donor stencils: for node n, the entries w * 27 + i
// of wd whose stencil point is n, in increasing (w, i) order.
cacl_status build_transpose(cacl_ctx* c, AdjointState* s) {
  const int W = c->wall_count;
  const Grid& g = c->g;
  std::vector<int32_t> donor(W);
  if (W > 0)
    ACK(cudaMemcpy(donor.data(), c->w_donor, 4 * W, cudaMemcpyDeviceToHost),
        "copy donors");
  std::vector<int32_t> count(g.N + 1, 0);
  std::vector<int64_t> node((size_t)W * Q);
  for (int w = 0; w < W; ++w) {
    const int d = donor[w];
    const int x = d % g.nx, y = (d / g.nx) % g.ny, z = d / (g.nx * g.ny);
    for (int i = 0; i < Q; ++i) {
      const int xx = (x + cx(i) + g.nx) % g.nx, yy = (y + cy(i) + g.ny) % g.ny,
                zz = (z + cz(i) + g.nz) % g.nz;
      const int64_t m = xx + (int64_t)g.nx * (yy + (int64_t)g.ny * zz);
      node[(size_t)w * Q + i] = m;
      count[m + 1]++;
    }
  }
  for (int64_t n = 0; n < g.N; ++n) count[n + 1] += count[n];
  std::vector<int32_t> entry((size_t)W * Q), fill(count.begin(), count.end() - 1);
  for (int64_t e = 0; e < (int64_t)W * Q; ++e) entry[fill[node[e]]++] = (int32_t)e;
  ACK(alloc(&s->row_start, g.N + 1), "alloc transpose");
  ACK(alloc(&s->row_entry, (size_t)W * Q), "alloc transpose");
  ACK(cudaMemcpy(s->row_start, count.data(), 4 * (g.N + 1), cudaMemcpyHostToDevice),
      "upload transpose");
  if (W > 0)
    ACK(cudaMemcpy(s->row_entry, entry.data(), 4 * (size_t)W * Q,
                   cudaMemcpyHostToDevice), "upload transpose");
  return CACL_OK;
}

// Copy the current state (populations, phi, mass record incl. the rounding
// key) into a checkpoint.
cacl_status store_checkpoint(cacl_ctx* c, float* f, float* phi, MassScalars* m) {
  const int64_t N = c->g.N;
  ACK(cudaMemcpyAsync(f, c->f[c->fcur], sizeof(float) * Q * N,
                      cudaMemcpyDeviceToDevice, c->stream), "checkpoint");
  ACK(cudaMemcpyAsync(phi, c->phi[c->pcur], sizeof(float) * N,
                      cudaMemcpyDeviceToDevice, c->stream), "checkpoint");
  ACK(cudaMemcpyAsync(m, c->mass, sizeof(MassScalars), cudaMemcpyDeviceToDevice,
                      c->stream), "checkpoint");
  return CACL_OK;
}

// Step t of a segment's recompute, recording tape slot t. The populations
// need no copy: the step reads f*^{n-1} from slot t (the checkpoint was
// restored into slot 0) and the collide-stream writes f*^n straight into
// slot t + 1 (the context's spare buffer after the last step).
cacl_status taped_step(cacl_ctx* c, AdjointState* s, int t, int len) {
  const int64_t N = c->g.N;
  const size_t pb = sizeof(float) * N;
  ACK(cudaMemcpyAsync(s->t_phipre[t], c->phi[c->pcur], pb, cudaMemcpyDeviceToDevice,
                      c->stream), "tape");
  cacl_status st = cacl_ghost_update(c);
  if (st != CACL_OK) return st;
  ACK(cudaMemcpyAsync(s->t_phig[t], c->phi[c->pcur], pb, cudaMemcpyDeviceToDevice,
                      c->stream), "tape");
  float* fout = (t + 1 < len) ? s->t_fprev[t + 1] : (float*)c->f[1 - c->fcur];
  ACK(launch_lb(c, s->t_fprev[t], fout, c->phi[c->pcur]), "collide-stream");
  ACK(cudaMemcpyAsync(s->t_u[t], c->u, 3 * pb, cudaMemcpyDeviceToDevice, c->stream),
      "tape");
  ACK(cudaMemcpyAsync(s->t_a[t], c->a, 3 * pb, cudaMemcpyDeviceToDevice, c->stream),
      "tape");
  // the phi update of a full step reads the compressive vector the
  // collide-stream just wrote (launch_phase, not the part entry point)
  ACK(launch_phase(c, c->phi[c->pcur], c->phi[1 - c->pcur]), "phase");
  c->pcur ^= 1;
  ACK(cudaMemcpyAsync(s->t_phis[t], c->phi[c->pcur], pb, cudaMemcpyDeviceToDevice,
                      c->stream), "tape");
  if ((st = cacl_volume_correct(c)) != CACL_OK) return st;
  ACK(cudaMemcpyAsync(s->t_mass + t, c->mass, sizeof(MassScalars),
                      cudaMemcpyDeviceToDevice, c->stream), "tape");
  return CACL_OK;
}

}  // namespace

extern "C" {

cacl_status cacl_adjoint_forward(cacl_ctx* c, int nsteps, int every) {
  return cacl_adjoint_forward_levels(c, nsteps, every, 0);
}

cacl_status cacl_adjoint_forward_levels(cacl_ctx* c, int nsteps, int every,
                                        int outer) {
  if (!c || nsteps < 1 || every < 1 || outer < 0) return CACL_ERR_ARG;
  if (outer > 0 && outer % every != 0)
    return afail(c, CACL_ERR_ARG, "outer_every must be a multiple of ckpt_every");
  if (!c->has_fields) return afail(c, CACL_ERR_STATE, "set_fields first");
  if (c->p.storage != CACL_F32)
    return afail(c, CACL_ERR_ARG, "the adjoint needs FP32 population storage");
  NvtxRange range("cacl_adjoint_forward");
  if (c->fcur != c->pcur) return afail(c, CACL_ERR_STATE, "step parts out of phase");
  const int64_t N = c->g.N;
  AdjointState* s = c->adj;
  if (!s || s->nsteps != nsteps || s->every != every || s->outer != outer ||
      s->N != N || s->W != c->wall_count) {
    adjoint_free(s);
    c->adj = s = new AdjointState();
    s->nsteps = nsteps;
    s->every = every;
    s->outer = outer;
    s->N = N;
    s->W = c->wall_count;
    // inner checkpoints: the whole rollout (one level) or one outer segment
    const int span = outer > 0 ? std::min(outer, nsteps) : nsteps;
    const int nck = (span + every - 1) / every;
    if (outer > 0) {
      const int nck1 = (nsteps + outer - 1) / outer;
      for (int i = 0; i < nck1; ++i) {
        float *pf, *pp;
        ACK(alloc(&pf, (size_t)Q * N), "alloc checkpoint");
        s->ck1_f.push_back(pf);
        ACK(alloc(&pp, (size_t)N), "alloc checkpoint");
        s->ck1_phi.push_back(pp);
      }
      ACK(alloc(&s->ck1_mass, nck1), "alloc checkpoint");
    }
    for (int i = 0; i < nck; ++i) {
      float *pf, *pp;
      ACK(alloc(&pf, (size_t)Q * N), "alloc checkpoint");
      s->ck_f.push_back(pf);
      ACK(alloc(&pp, (size_t)N), "alloc checkpoint");
      s->ck_phi.push_back(pp);
    }
    for (int t = 0; t < every; ++t) {
      float* p;
      ACK(alloc(&p, (size_t)Q * N), "alloc tape");
      s->t_fprev.push_back(p);
      for (auto* v : {&s->t_phipre, &s->t_phig, &s->t_phis}) {
        ACK(alloc(&p, (size_t)N), "alloc tape");
        v->push_back(p);
      }
      for (auto* v : {&s->t_u, &s->t_a}) {
        ACK(alloc(&p, (size_t)3 * N), "alloc tape");
        v->push_back(p);
      }
    }
    ACK(alloc(&s->t_mass, every), "alloc tape");
    ACK(alloc(&s->ck_mass, nck), "alloc checkpoint");
    ACK(alloc(&s->fb, (size_t)Q * N), "alloc adjoint");
    ACK(alloc(&s->fb2, (size_t)Q * N), "alloc adjoint");
    ACK(alloc(&s->phib, N), "alloc adjoint");
    ACK(alloc(&s->phisb, N), "alloc adjoint");
    ACK(alloc(&s->phigb, N), "alloc adjoint");
    ACK(alloc(&s->ub, 3 * N), "alloc adjoint");
    ACK(alloc(&s->ab, 3 * N), "alloc adjoint");
    ACK(alloc(&s->face, 15 * N), "alloc adjoint");
    ACK(alloc(&s->nodeb, 5 * N), "alloc adjoint");
    ACK(alloc(&s->wd, (size_t)Q * (s->W > 0 ? s->W : 1)), "alloc adjoint");
    ACK(alloc(&s->thetab, s->W > 0 ? s->W : 1), "alloc adjoint");
    ACK(alloc(&s->sigmab, 1), "alloc adjoint");
    s->npart = std::max((int)(((c->g.nx + 127) / 128) * (int64_t)c->g.ny * c->g.nz), 1024);
    ACK(alloc(&s->partial, s->npart), "alloc adjoint");
    ACK(alloc(&s->sig_acc, 4 * (size_t)s->npart), "alloc adjoint");  // per warp
    ACK(alloc(&s->scal, 2), "alloc adjoint");
    const cacl_status st = build_transpose(c, s);
    if (st != CACL_OK) return st;
  }
  // forward, keeping a checkpoint at the start of every segment (outer
  // segments with two levels)
  const int stride = outer > 0 ? outer : every;
  for (int n = 0; n < nsteps; ++n) {
    if (n % stride == 0) {
      const cacl_status st = store_checkpoint(
          c, outer > 0 ? s->ck1_f[n / stride] : s->ck_f[n / stride],
          outer > 0 ? s->ck1_phi[n / stride] : s->ck_phi[n / stride],
          (outer > 0 ? s->ck1_mass : s->ck_mass) + n / stride);
      if (st != CACL_OK) return st;
    }
    const cacl_status st = cacl_step(c, 1);
    if (st != CACL_OK) return st;
  }
  s->forward_done = true;
  return CACL_OK;
}

cacl_status cacl_adjoint_backward(cacl_ctx* c, const float* dL_dphi,
                                  double* dL_dtheta, double* dL_dsigma) {
  if (!c || !dL_dphi) return CACL_ERR_ARG;
  AdjointState* s = c->adj;
  if (!s || !s->forward_done)
    return afail(c, CACL_ERR_STATE, "call cacl_adjoint_forward first");
  NvtxRange range("cacl_adjoint_backward");
  const Grid g = c->g;
  const int64_t N = g.N;
  const int W = s->W;
  const float eps = c->k.eps_phi;
  const double width = c->p.width;
  const float db4 = (float)(48.0 / width), dkp = (float)(1.5 * width);
  cudaStream_t st = c->stream;
  // the forward state is restored at the end
  float* save_f = nullptr;
  float* save_phi = nullptr;
  ACK(alloc(&save_f, (size_t)Q * N), "alloc");
  ACK(alloc(&save_phi, N), "alloc");
  ACK(cudaMemcpyAsync(save_f, c->f[c->fcur], sizeof(float) * Q * N,
                      cudaMemcpyDeviceToDevice, st), "save");
  ACK(cudaMemcpyAsync(save_phi, c->phi[c->pcur], sizeof(float) * N,
                      cudaMemcpyDeviceToDevice, st), "save");
  const int save_fc = c->fcur, save_pc = c->pcur;
  MassScalars save_mass;
  ACK(cudaMemcpyAsync(&save_mass, c->mass, sizeof(MassScalars), cudaMemcpyDeviceToHost,
                      st), "save");
  ACK(cudaStreamSynchronize(st), "sync");

  // events bracketing the recomputes and the whole call (timing only; the
  // synchronisation after each recompute keeps the host in step)
  cudaEvent_t ev_a = nullptr, ev_b = nullptr, ev_0 = nullptr;
  ACK(cudaEventCreate(&ev_a), "event");
  ACK(cudaEventCreate(&ev_b), "event");
  ACK(cudaEventCreate(&ev_0), "event");
  s->t_recompute_ms = 0.0;
  ACK(cudaEventRecord(ev_0, st), "event");
  ACK(cudaMemcpyAsync(s->phib, dL_dphi, sizeof(float) * N, cudaMemcpyDeviceToDevice, st),
      "seed");
  ACK(cudaMemsetAsync(s->thetab, 0, sizeof(double) * (W > 0 ? W : 1), st), "seed");
  ACK(cudaMemsetAsync(s->sigmab, 0, sizeof(double), st), "seed");
  const int nbl_all = 4 * (int)(((g.nx + 127) / 128) * (int64_t)g.ny * g.nz);  // warps
  ACK(cudaMemsetAsync(s->sig_acc, 0, sizeof(double) * nbl_all, st), "seed");

  const bool small = !c->index64 && (int64_t)Q * N < (int64_t)INT32_MAX;  // 32-bit offsets
  const bool small15 = !c->index64 && (int64_t)15 * N < (int64_t)INT32_MAX;  // face buffer
  bool first = true;  // no later step: dL/df* of the final populations is 0
  // the launches of backward step t of a segment of len steps
  auto back_step = [&](int t, int len) -> cudaError_t {
    // A1 correction; S was summed by the ghost gather of the step after this
    // one within the segment, else here
    int nparts = nblk(N, AT);
    if (t == len - 1) {
      nparts = std::min(nblk(N, AT), 1024);
      adj_correct_sum<<<nparts, AT, 0, st>>>(s->phib, s->t_phis[t], c->flags, N, eps,
                                             s->partial);
    }
    adj_correct_scalars<<<1, AT, 0, st>>>(s->partial, nparts, s->t_mass + t, s->scal);
    adj_correct_apply<<<nblk(N, AT), AT, 0, st>>>(s->phib, s->t_phis[t], c->flags, N,
                                                  eps, s->scal, s->phisb);
    // A2 phi update
    const dim3 rows((g.nx + 127) / 128, g.ny, g.nz);
    // threads of a row block: 128, or the row rounded up to whole warps
    const int rt = std::min(128, (g.nx + 31) / 32 * 32);
    if (small15) {
      adj_phase_faces<int><<<rows, rt, 0, st>>>(s->t_phig[t], s->t_u[t], c->flags,
                                                 s->phisb, s->face, g);
      adj_phase_gather<int><<<rows, rt, 0, st>>>(c->flags, s->phisb, s->face, s->phigb,
                                                  s->ub, s->ab, g, c->k);
    } else {
      adj_phase_faces<int64_t><<<rows, rt, 0, st>>>(s->t_phig[t], s->t_u[t], c->flags,
                                                     s->phisb, s->face, g);
      adj_phase_gather<int64_t><<<rows, rt, 0, st>>>(c->flags, s->phisb, s->face,
                                                      s->phigb, s->ub, s->ab, g, c->k);
    }
    // A3 collide-stream; the later step's pulled-population adjoints (none
    // after the last step)
    const float* later = first ? nullptr : s->fb;
    if (small) {
      adj_lb_node<int><<<rows, rt, 0, st>>>(s->t_fprev[t], s->t_phig[t], c->flags, later,
                                             s->ub, s->ab, s->fb2, s->nodeb, s->sig_acc, g,
                                             c->k, db4, dkp);
    } else {
      adj_lb_node<int64_t><<<rows, rt, 0, st>>>(s->t_fprev[t], s->t_phig[t], c->flags,
                                                 later, s->ub, s->ab, s->fb2, s->nodeb,
                                                 s->sig_acc, g, c->k, db4, dkp);
    }
    std::swap(s->fb, s->fb2);  // fb: this step's pulled-population adjoints
    first = false;
    if (small)
      adj_lb_gather<int><<<rows, rt, 0, st>>>(s->nodeb, s->phigb, g);
    else
      adj_lb_gather<int64_t><<<rows, rt, 0, st>>>(s->nodeb, s->phigb, g);
    // A4 ghost map
    if (W > 0)
      adj_ghost_node<<<nblk(W, 128), 128, 0, st>>>(s->t_phipre[t], c->w_idx, c->w_donor,
                                                   c->w_q, c->w_nw, c->w_cot, c->w_theta,
                                                   s->phigb, s->wd, s->thetab, W, g);
    adj_ghost_gather<<<nblk(N, AT), AT, 0, st>>>(c->flags, s->phigb, s->row_start,
                                                 s->row_entry, s->wd, s->phib, N,
                                                 t > 0 ? s->t_phis[t - 1] : nullptr, eps,
                                                 s->partial);
    return cudaGetLastError();
  };

  // everything the captured segment graphs bake in
  {
    std::vector<unsigned char> key;
    auto put = [&](const void* p, size_t n) {
      const unsigned char* b = static_cast<const unsigned char*>(p);
      key.insert(key.end(), b, b + n);
    };
    put(&c->k, sizeof(Consts));
    put(&eps, sizeof eps);
    put(&db4, sizeof db4);
    put(&dkp, sizeof dkp);
    const int64_t dims[] = {g.nx, g.ny, g.nz, g.N, W, s->every, c->index64 ? 1 : 0};
    put(dims, sizeof dims);
    const void* bufs[] = {c->flags, c->w_idx, c->w_donor, c->w_q, c->w_nw, c->w_cot,
                          c->w_theta};
    put(bufs, sizeof bufs);
    if (key != s->graph_key) {
      for (auto& gx : s->seg_graph) {
        if (gx) cudaGraphExecDestroy(gx);
        gx = nullptr;
      }
      s->graph_key = key;
    }
  }
  // outer segments, last first (one segment spanning the rollout with one
  // level); with two levels each is recomputed once from its outer
  // checkpoint to rebuild its inner checkpoints
  const int span = s->outer > 0 ? s->outer : s->nsteps;
  const int nouter = (s->nsteps + span - 1) / span;
  for (int J = nouter - 1; J >= 0; --J) {
    const int m0 = J * span;                          // first step of the segment
    const int mlen = std::min(span, s->nsteps - m0);  // its steps
    if (s->outer > 0) {
      ACK(cudaEventRecord(ev_a, st), "event");
      ACK(cudaMemcpyAsync(c->f[c->fcur], s->ck1_f[J], sizeof(float) * Q * N,
                          cudaMemcpyDeviceToDevice, st), "restore");
      ACK(cudaMemcpyAsync(c->phi[c->pcur], s->ck1_phi[J], sizeof(float) * N,
                          cudaMemcpyDeviceToDevice, st), "restore");
      ACK(cudaMemcpyAsync(c->mass, s->ck1_mass + J, sizeof(MassScalars),
                          cudaMemcpyDeviceToDevice, st), "restore");
      for (int n = 0; n < mlen; ++n) {
        if (n % s->every == 0) {
          const int ck = n / s->every;
          const cacl_status r =
              store_checkpoint(c, s->ck_f[ck], s->ck_phi[ck], s->ck_mass + ck);
          if (r != CACL_OK) return r;
        }
        const cacl_status r = cacl_step(c, 1);
        if (r != CACL_OK) return r;
      }
      ACK(cudaEventRecord(ev_b, st), "event");
      ACK(cudaEventSynchronize(ev_b), "event");
      float ms = 0.f;
      ACK(cudaEventElapsedTime(&ms, ev_a, ev_b), "event");
      s->t_recompute_ms += ms;
    }
    const int nseg = (mlen + s->every - 1) / s->every;
    for (int seg = nseg - 1; seg >= 0; --seg) {
      const int n0 = seg * s->every;
      const int len = std::min(s->every, mlen - n0);
      // recompute the segment with its tape
      ACK(cudaMemcpyAsync(s->t_fprev[0], s->ck_f[seg], sizeof(float) * Q * N,
                          cudaMemcpyDeviceToDevice, st), "restore");
      ACK(cudaMemcpyAsync(c->phi[c->pcur], s->ck_phi[seg], sizeof(float) * N,
                          cudaMemcpyDeviceToDevice, st), "restore");
      ACK(cudaMemcpyAsync(c->mass, s->ck_mass + seg, sizeof(MassScalars),
                          cudaMemcpyDeviceToDevice, st), "restore");
      ACK(cudaEventRecord(ev_a, st), "event");
      for (int t = 0; t < len; ++t) {
        const cacl_status r = taped_step(c, s, t, len);
        if (r != CACL_OK) return r;
      }
      ACK(cudaEventRecord(ev_b, st), "event");
      ACK(cudaEventSynchronize(ev_b), "event");
      float ms = 0.f;
      ACK(cudaEventElapsedTime(&ms, ev_a, ev_b), "event");
      s->t_recompute_ms += ms;
      const bool use_graph = !first && len == s->every;
      if (!use_graph) {
        for (int t = len - 1; t >= 0; --t) ACK(back_step(t, len), "adjoint step");
        continue;
      }
      const int slot = s->fb < s->fb2 ? 0 : 1;
      if (!s->seg_graph[slot]) {
        // capture the segment's backward steps once; the host-side state
        // they change (fb / fb2) is put back and replayed below
        float* const fb0 = s->fb;
        float* const fb20 = s->fb2;
        ACK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal), "capture");
        cudaError_t ce = cudaSuccess;
        for (int t = len - 1; t >= 0 && ce == cudaSuccess; --t) ce = back_step(t, len);
        cudaGraph_t gr = nullptr;
        const cudaError_t ee = cudaStreamEndCapture(st, &gr);
        s->fb = fb0;
        s->fb2 = fb20;
        if (ce != cudaSuccess || ee != cudaSuccess) {
          if (gr) cudaGraphDestroy(gr);
          ACK(ce != cudaSuccess ? ce : ee, "capture adjoint segment");
        }
        const cudaError_t ie = cudaGraphInstantiate(&s->seg_graph[slot], gr, 0);
        cudaGraphDestroy(gr);
        ACK(ie, "instantiate adjoint segment");
      }
      ACK(cudaGraphLaunch(s->seg_graph[slot], st), "adjoint segment");
      if (len % 2) std::swap(s->fb, s->fb2);  // one swap per replayed step
    }
  }
  sum_partials<<<1, 128, 0, st>>>(s->sig_acc, nbl_all, s->sigmab);
  ACK(cudaGetLastError(), "dsigma sum");
  if (dL_dtheta && W > 0)
    ACK(cudaMemcpyAsync(dL_dtheta, s->thetab, sizeof(double) * W,
                        cudaMemcpyDeviceToDevice, st), "copy dtheta");
  if (dL_dsigma)
    ACK(cudaMemcpyAsync(dL_dsigma, s->sigmab, sizeof(double), cudaMemcpyDeviceToDevice,
                        st), "copy dsigma");
  // restore the state reached by the forward run
  c->fcur = save_fc;
  c->pcur = save_pc;
  ACK(cudaMemcpyAsync(c->f[c->fcur], save_f, sizeof(float) * Q * N,
                      cudaMemcpyDeviceToDevice, st), "restore");
  ACK(cudaMemcpyAsync(c->phi[c->pcur], save_phi, sizeof(float) * N,
                      cudaMemcpyDeviceToDevice, st), "restore");
  ACK(cudaMemcpyAsync(c->mass, &save_mass, sizeof(MassScalars), cudaMemcpyHostToDevice,
                      st), "restore");
  ACK(cudaEventRecord(ev_b, st), "event");
  ACK(cudaStreamSynchronize(st), "sync");
  float tot = 0.f;
  ACK(cudaEventElapsedTime(&tot, ev_0, ev_b), "event");
  s->t_total_ms = tot;
  cudaEventDestroy(ev_a);
  cudaEventDestroy(ev_b);
  cudaEventDestroy(ev_0);
  cudaFree(save_f);
  cudaFree(save_phi);
  return CACL_OK;
}

cacl_status cacl_adjoint_stage(cacl_ctx* c, int stage, const float* in, float* out,
                               double* dparam, float* state) {
  if (!c || stage < CACL_ADJ_CORRECT || stage > CACL_ADJ_GHOST || !in || !out)
    return c ? afail(c, CACL_ERR_ARG, "invalid adjoint stage request") : CACL_ERR_ARG;
  AdjointState* s = c->adj;
  if (!s || !s->forward_done || s->outer != 0)
    return afail(c, CACL_ERR_STATE, "call cacl_adjoint_forward first (one level)");
  const Grid g = c->g;
  const int64_t N = g.N;
  const int W = s->W;
  const float eps = c->k.eps_phi;
  const double width = c->p.width;
  const float db4 = (float)(48.0 / width), dkp = (float)(1.5 * width);
  cudaStream_t st = c->stream;
  const size_t pb = sizeof(float) * N;
  // step 0 of the rollout, recomputed from checkpoint 0 into tape slot 0;
  // the context's state is saved and put back
  float* save_f = nullptr;
  float* save_phi = nullptr;
  ACK(alloc(&save_f, (size_t)Q * N), "alloc");
  ACK(alloc(&save_phi, N), "alloc");
  ACK(cudaMemcpyAsync(save_f, c->f[c->fcur], pb * Q, cudaMemcpyDeviceToDevice, st), "save");
  ACK(cudaMemcpyAsync(save_phi, c->phi[c->pcur], pb, cudaMemcpyDeviceToDevice, st), "save");
  const int save_fc = c->fcur, save_pc = c->pcur;
  MassScalars save_mass;
  ACK(cudaMemcpyAsync(&save_mass, c->mass, sizeof(MassScalars), cudaMemcpyDeviceToHost, st),
      "save");
  ACK(cudaStreamSynchronize(st), "sync");
  ACK(cudaMemcpyAsync(s->t_fprev[0], s->ck_f[0], pb * Q, cudaMemcpyDeviceToDevice, st),
      "restore");
  ACK(cudaMemcpyAsync(c->phi[c->pcur], s->ck_phi[0], pb, cudaMemcpyDeviceToDevice, st),
      "restore");
  ACK(cudaMemcpyAsync(c->mass, s->ck_mass, sizeof(MassScalars), cudaMemcpyDeviceToDevice, st),
      "restore");
  const cacl_status ts = taped_step(c, s, 0, 1);
  if (ts != CACL_OK) return ts;
  if (state) {  // the linearisation point
    float* o = state;
    const float* parts[] = {s->t_phipre[0], s->t_fprev[0], s->t_phig[0], s->t_u[0],
                            s->t_a[0], s->t_phis[0]};
    const size_t sizes[] = {1, Q, 1, 3, 3, 1};
    for (int i = 0; i < 6; ++i) {
      ACK(cudaMemcpyAsync(o, parts[i], pb * sizes[i], cudaMemcpyDeviceToDevice, st), "state");
      o += sizes[i] * N;
    }
  }
  const dim3 rows((g.nx + 127) / 128, g.ny, g.nz);
  // threads of a row block: 128, or the row rounded up to whole warps
  const int rt = std::min(128, (g.nx + 31) / 32 * 32);
  const bool small = !c->index64 && (int64_t)Q * N < (int64_t)INT32_MAX;
  const bool small15 = !c->index64 && (int64_t)15 * N < (int64_t)INT32_MAX;
  switch (stage) {
    case CACL_ADJ_CORRECT: {
      ACK(cudaMemcpyAsync(s->phib, in, pb, cudaMemcpyDeviceToDevice, st), "in");
      const int nparts = std::min(nblk(N, AT), 1024);
      adj_correct_sum<<<nparts, AT, 0, st>>>(s->phib, s->t_phis[0], c->flags, N, eps,
                                             s->partial);
      adj_correct_scalars<<<1, AT, 0, st>>>(s->partial, nparts, s->t_mass, s->scal);
      adj_correct_apply<<<nblk(N, AT), AT, 0, st>>>(s->phib, s->t_phis[0], c->flags, N,
                                                    eps, s->scal, s->phisb);
      ACK(cudaMemcpyAsync(out, s->phisb, pb, cudaMemcpyDeviceToDevice, st), "out");
      break;
    }
    case CACL_ADJ_PHASE:
      ACK(cudaMemcpyAsync(s->phisb, in, pb, cudaMemcpyDeviceToDevice, st), "in");
      if (small15) {
        adj_phase_faces<int><<<rows, rt, 0, st>>>(s->t_phig[0], s->t_u[0], c->flags,
                                                   s->phisb, s->face, g);
        adj_phase_gather<int><<<rows, rt, 0, st>>>(c->flags, s->phisb, s->face, s->phigb,
                                                    s->ub, s->ab, g, c->k);
      } else {
        adj_phase_faces<int64_t><<<rows, rt, 0, st>>>(s->t_phig[0], s->t_u[0], c->flags,
                                                       s->phisb, s->face, g);
        adj_phase_gather<int64_t><<<rows, rt, 0, st>>>(c->flags, s->phisb, s->face,
                                                        s->phigb, s->ub, s->ab, g, c->k);
      }
      ACK(cudaMemcpyAsync(out, s->phigb, pb, cudaMemcpyDeviceToDevice, st), "out");
      ACK(cudaMemcpyAsync(out + N, s->ub, 3 * pb, cudaMemcpyDeviceToDevice, st), "out");
      ACK(cudaMemcpyAsync(out + 4 * N, s->ab, 3 * pb, cudaMemcpyDeviceToDevice, st), "out");
      break;
    case CACL_ADJ_COLLIDE: {
      ACK(cudaMemcpyAsync(s->fb, in, pb * Q, cudaMemcpyDeviceToDevice, st), "in");
      ACK(cudaMemcpyAsync(s->ub, in + Q * N, 3 * pb, cudaMemcpyDeviceToDevice, st), "in");
      ACK(cudaMemcpyAsync(s->ab, in + (Q + 3) * N, 3 * pb, cudaMemcpyDeviceToDevice, st),
          "in");
      const int nbl_all = 4 * (int)(((g.nx + 127) / 128) * (int64_t)g.ny * g.nz);
      ACK(cudaMemsetAsync(s->sig_acc, 0, sizeof(double) * nbl_all, st), "zero");
      ACK(cudaMemsetAsync(s->phigb, 0, pb, st), "zero");
      if (small) {
        adj_lb_node<int><<<rows, rt, 0, st>>>(s->t_fprev[0], s->t_phig[0], c->flags, s->fb,
                                               s->ub, s->ab, s->fb2, s->nodeb, s->sig_acc,
                                               g, c->k, db4, dkp);
        adj_lb_gather<int><<<rows, rt, 0, st>>>(s->nodeb, s->phigb, g);
      } else {
        adj_lb_node<int64_t><<<rows, rt, 0, st>>>(s->t_fprev[0], s->t_phig[0], c->flags,
                                                   s->fb, s->ub, s->ab, s->fb2, s->nodeb,
                                                   s->sig_acc, g, c->k, db4, dkp);
        adj_lb_gather<int64_t><<<rows, rt, 0, st>>>(s->nodeb, s->phigb, g);
      }
      sum_partials<<<1, 128, 0, st>>>(s->sig_acc, nbl_all, s->sigmab);
      ACK(cudaMemcpyAsync(out, s->fb2, pb * Q, cudaMemcpyDeviceToDevice, st), "out");
      ACK(cudaMemcpyAsync(out + Q * N, s->phigb, pb, cudaMemcpyDeviceToDevice, st), "out");
      if (dparam)
        ACK(cudaMemcpyAsync(dparam, s->sigmab, sizeof(double), cudaMemcpyDeviceToDevice, st),
            "out");
      break;
    }
    default:  // CACL_ADJ_GHOST
      ACK(cudaMemcpyAsync(s->phigb, in, pb, cudaMemcpyDeviceToDevice, st), "in");
      ACK(cudaMemsetAsync(s->thetab, 0, sizeof(double) * (W > 0 ? W : 1), st), "zero");
      if (W > 0)
        adj_ghost_node<<<nblk(W, 128), 128, 0, st>>>(s->t_phipre[0], c->w_idx, c->w_donor,
                                                     c->w_q, c->w_nw, c->w_cot, c->w_theta,
                                                     s->phigb, s->wd, s->thetab, W, g);
      adj_ghost_gather<<<nblk(N, AT), AT, 0, st>>>(c->flags, s->phigb, s->row_start,
                                                   s->row_entry, s->wd, s->phib, N, nullptr,
                                                   eps, s->partial);
      ACK(cudaMemcpyAsync(out, s->phib, pb, cudaMemcpyDeviceToDevice, st), "out");
      if (dparam && W > 0)
        ACK(cudaMemcpyAsync(dparam, s->thetab, sizeof(double) * W, cudaMemcpyDeviceToDevice,
                            st), "out");
      break;
  }
  ACK(cudaGetLastError(), "adjoint stage");
  c->fcur = save_fc;
  c->pcur = save_pc;
  ACK(cudaMemcpyAsync(c->f[c->fcur], save_f, pb * Q, cudaMemcpyDeviceToDevice, st),
      "restore");
  ACK(cudaMemcpyAsync(c->phi[c->pcur], save_phi, pb, cudaMemcpyDeviceToDevice, st),
      "restore");
  ACK(cudaMemcpyAsync(c->mass, &save_mass, sizeof(MassScalars), cudaMemcpyHostToDevice, st),
      "restore");
  ACK(cudaStreamSynchronize(st), "sync");
  cudaFree(save_f);
  cudaFree(save_phi);
  return CACL_OK;
}

cacl_status cacl_adjoint_timing(const cacl_ctx* c, double* recompute_ms,
                                double* total_ms) {
  if (!c || !c->adj) return CACL_ERR_STATE;
  if (recompute_ms) *recompute_ms = c->adj->t_recompute_ms;
  if (total_ms) *total_ms = c->adj->t_total_ms;
  return CACL_OK;
}

}  // extern "C"
