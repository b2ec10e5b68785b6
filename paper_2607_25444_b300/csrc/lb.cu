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
// splits into a part even in c and a part odd in c:
//   E = k1 + 4.5 cu^2 + om45 cAc + 4.5 cu ca
//   O = cu (k2 + 4.5 cu^2 + 3 om45 cAc) - 2 om45 cAu + 1.5 ca
//   f*(+c) = w (E + O),  f*(-c) = w (E - O)
// with om45 = 4.5 (1 - omega), k1 = p* - 1.5 (u.u + u.a) - om45 tr / 3,
// k2 = 3 - 4.5 u.u - om45 tr.
#include "cacl_internal.cuh"

namespace cacl {
namespace {

constexpr int LB_BX = 128;
constexpr int LB_BY = 1;

struct NodeOut {
  float f[Q];
  float ux, uy, uz;
};

__device__ __forceinline__ void collide(const float (&f)[Q], float phi0,
                                        float gx, float gy, float gz, float lap,
                                        const Consts& k, NodeOut& o) {
  // moments over pairs of opposite directions (q < 13 has opposite 26 - q)
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
  const float muphi =
      k.beta4 * phi0 * (phi0 - 1.0f) * (phi0 - 0.5f) - k.kappa_phi * lap;
  const float p3 = p * (1.0f / 3.0f);
  const float rb = rho - k.rho_g;
  const float F0x = muphi * gx - p3 * grx + rb * k.gx;
  const float F0y = muphi * gy - p3 * gry + rb * k.gy;
  const float F0z = muphi * gz - p3 * grz + rb * k.gz;
  // predictor for the viscous correction (Eq. Fnu)
  const float a0x = F0x * inv_rho, a0y = F0y * inv_rho, a0z = F0z * inv_rho;
  const float u0x = jx + 0.5f * a0x, u0y = jy + 0.5f * a0y, u0z = jz + 0.5f * a0z;
  const float Q0xx = Pxx - p3 - u0x * u0x + u0x * a0x;
  const float Q0yy = Pyy - p3 - u0y * u0y + u0y * a0y;
  const float Q0zz = Pzz - p3 - u0z * u0z + u0z * a0z;
  const float Q0xy = Pxy - u0x * u0y + 0.5f * (u0x * a0y + a0x * u0y);
  const float Q0xz = Pxz - u0x * u0z + 0.5f * (u0x * a0z + a0x * u0z);
  const float Q0yz = Pyz - u0y * u0z + 0.5f * (u0y * a0z + a0y * u0z);
  const float cnu = -3.0f * nu * omega;
  const float Fx = F0x + cnu * (Q0xx * grx + Q0xy * gry + Q0xz * grz);
  const float Fy = F0y + cnu * (Q0xy * grx + Q0yy * gry + Q0yz * grz);
  const float Fz = F0z + cnu * (Q0xz * grx + Q0yz * gry + Q0zz * grz);
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
  const float uu = ux * ux + uy * uy + uz * uz;
  const float ua = ux * ax + uy * ay + uz * az;
  const float om45 = 4.5f * (1.0f - omega);
  const float k1 = p - 1.5f * (uu + ua) - om45 * tr * (1.0f / 3.0f);
  const float k2 = 3.0f - 4.5f * uu - om45 * tr;
  const float om3 = 3.0f * om45, om2 = 2.0f * om45;
#pragma unroll
  for (int q = 0; q < REST; ++q) {
    const int X = cx(q), Y = cy(q), Z = cz(q);
    const float cu = X * ux + Y * uy + Z * uz;
    const float ca = X * ax + Y * ay + Z * az;
    const float cAu = X * vx + Y * vy + Z * vz;
    const float cAc = (X * X) * Axx + (Y * Y) * Ayy + (Z * Z) * Azz +
                      2.0f * ((X * Y) * Axy + (X * Z) * Axz + (Y * Z) * Ayz);
    const float cu2 = cu * cu;
    const float E = k1 + 4.5f * cu2 + om45 * cAc + 4.5f * cu * ca;
    const float O = cu * (k2 + 4.5f * cu2 + om3 * cAc) - om2 * cAu + 1.5f * ca;
    o.f[q] = wq(q) * (E + O);
    o.f[opp(q)] = wq(q) * (E - O);
  }
  o.f[REST] = wq(REST) * k1;
  o.ux = ux;
  o.uy = uy;
  o.uz = uz;
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
    const float dv = (3.0f * wq(q)) * (vp - vm);
    gx += cx(q) * dv;
    gy += cy(q) * dv;
    gz += cz(q) * dv;
    ssum += wq(q) * (vp + vm);
  }
  const float lap = 6.0f * (ssum - (1.0f - wq(REST)) * phi0);
  float ax, ay, az;
  compressive(phi0, gx, gy, gz, ax, ay, az);
  a[n] = ax;
  a[N + n] = ay;
  a[2 * N + n] = az;

  NodeOut o;
  collide(f, phi0, gx, gy, gz, lap, k, o);
#pragma unroll
  for (int q = 0; q < Q; ++q) fout[q * N + n] = Store::encode(o.f[q], q);
  u[n] = o.ux;
  u[N + n] = o.uy;
  u[2 * N + n] = o.uz;
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

template <typename Store>
void launch_store(cacl_ctx* c, const void* fin, void* fout, const float* phi) {
  using T = typename Store::T;
  const Grid g = c->g;
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
