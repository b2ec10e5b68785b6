// phase.cu -- conservative Allen-Cahn update of phi at fluid nodes
// (Sect. 2.2: Eqs. phi_update_muscl, divF, face_flux_def, slope_minmod_x,
// minmod, recon_lr_x, upwind_select_x, source_sharp; Eq. lap_iso), plus the
// per-block partial sums of the volume correction (Sect. 2.4,
// Eqs. tentative_phase_field_mass, mass_correction_normalization).
//
// Each block owns a TX x TY column of nodes and marches up a chunk of ZC
// planes, one barrier per plane. Shared memory holds a ring of phi planes
// (with a halo of 2 in x and y, the reach of the minmod slopes) and of planes
// of the compressive vector a = phi (1 - phi) grad phi / |grad phi| (halo 1),
// which the collide-stream of the same step wrote. The own column's phi
// values, solid flags and the in-plane partial stencils are carried in
// registers from plane to plane.
//
// The D3Q27 weights factor as w(c) = s(cx) s(cy) s(cz) with s(0) = 2/3,
// s(+-1) = 1/6, so every isotropic stencil of Eqs. grad_iso / lap_iso is a
// product of 1D three-point operators: S f = (f- + 4 f0 + f+)/6 and
// Dd f = (f+ - f-)/6. Then
//   grad phi = 3 (Dd_x S_y S_z, S_x Dd_y S_z, S_x S_y Dd_z) phi,
//   lap phi  = 6 (S_x S_y S_z phi - phi),
//   div_iso a = 3 S_z (Dd_x S_y a_x + S_x Dd_y a_y) + 3 Dd_z (S_x S_y a_z),
// which is the same sum over the 27 links, evaluated in a different order.
//
// Partial sums are accumulated per thread as unevaluated float pairs
// (Knuth's two-sum), combined across the block the same way, and written as
// FP64 per block: FP64 arithmetic stays out of the per-node path.
#include "cacl_internal.cuh"

namespace cacl {
namespace {

constexpr int TX = 32;

struct DF {
  float hi, lo;
};

__device__ __forceinline__ void df_add(DF& s, float x) {
  const float t = s.hi + x;
  const float bb = t - s.hi;
  const float err = (s.hi - (t - bb)) + (x - bb);
  s.hi = t;
  s.lo += err;
}

__device__ __forceinline__ DF df_merge(DF a, DF b) {
  const float t = a.hi + b.hi;
  const float bb = t - a.hi;
  float err = (a.hi - (t - bb)) + (b.hi - bb);
  err += a.lo + b.lo;
  DF r;
  r.hi = t + err;
  r.lo = err - (r.hi - t);
  return r;
}

__device__ __forceinline__ DF df_shfl_down(DF v, int off) {
  DF r;
  r.hi = __shfl_down_sync(0xffffffffu, v.hi, off);
  r.lo = __shfl_down_sync(0xffffffffu, v.lo, off);
  return r;
}

// minmod(a, b) = 0 if a b <= 0, else sign(a) min(|a|, |b|) (Eq. minmod)
__device__ __forceinline__ float minmod(float a, float b) {
  const float m = fminf(fabsf(a), fabsf(b));
  return (a * b > 0.f) ? copysignf(m, a) : 0.f;
}

__device__ __forceinline__ int mod(int i, int n) {
  const int r = i % n;
  return r < 0 ? r + n : r;
}

// Net advective flux difference along one axis (Eqs. divF .. upwind_select):
// values at -2..+2 along the axis, solid flags at -1/+1, cell velocities at
// -1, 0, +1. Faces touching a solid carry no flux.
__device__ __forceinline__ float muscl_axis(float vm2, float vm1, float v0,
                                            float vp1, float vp2, bool solm,
                                            bool solp, float um, float uc,
                                            float up) {
  const float sm = minmod(vm1 - vm2, v0 - vm1);
  const float s0 = minmod(v0 - vm1, vp1 - v0);
  const float sp = minmod(vp1 - v0, vp2 - vp1);
  const float ufp = 0.5f * (uc + up);
  const float ufm = 0.5f * (um + uc);
  const float fp = ufp * ((ufp >= 0.f) ? fmaf(0.5f, s0, v0) : fmaf(-0.5f, sp, vp1));
  const float fm = ufm * ((ufm >= 0.f) ? fmaf(0.5f, sm, vm1) : fmaf(-0.5f, s0, v0));
  return (solp ? 0.f : fp) - (solm ? 0.f : fm);
}

// One block: TX x TY output nodes per plane, TX x TY/2 threads; each thread
// owns two vertically adjacent output nodes (rows 2 ty and 2 ty + 1), which
// share most of their stencil reads and all per-thread bookkeeping.
// One tile (bxi, byi, bzi) of one grid; its partial sums go to slot pb of
// partials (phi* sums) and nblocks + pb (chi sums).
template <int TY, int ZC>
__device__ __forceinline__ void phase_tile_body(
    int bxi, int byi, int bzi, int pb, const float* __restrict__ phi,
    const float* __restrict__ afld, float* __restrict__ phi_out,
    const float* __restrict__ u, const uint8_t* __restrict__ flags,
    double* __restrict__ partials, int nblocks, const Grid& g, const Consts& k) {
  constexpr int PX = TX + 4, PY = TY + 4, NP = PX * PY;  // phi plane, halo 2
  constexpr int AX = TX + 2, AY = TY + 2, NA = AX * AY;  // a plane, halo 1
  constexpr int THREADS = TX * TY / 2;
  constexpr int NLD = (NP + THREADS - 1) / THREADS;      // plane entries/thread
  constexpr int NLA = (NA + THREADS - 1) / THREADS;
  // Ring of four phi planes and two a planes, one barrier per plane: the
  // slots written at step kz (phi plane kz + 2, a plane kz + 1) were last
  // read at step kz - 2, before the barrier of step kz - 1.
  __shared__ float s_phi[4][NP];
  __shared__ uint8_t s_sol[4][NP];
  __shared__ float s_a[2][3][NA];
  __shared__ DF red[2][THREADS / 32];

  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = tx + TX * ty;
  const int x0 = bxi * TX, y0 = byi * TY, z0 = bzi * ZC;
  const int zend = min(z0 + ZC, g.nz);
  const int nxy = g.nx * g.ny;
  const int64_t N = g.N;

  int ld_off[NLD], la_off[NLA];
#pragma unroll
  for (int j = 0; j < NLD; ++j) {
    const int i = tid + j * THREADS;
    ld_off[j] = (i < NP) ? mod(x0 + i % PX - 2, g.nx) + g.nx * mod(y0 + i / PX - 2, g.ny) : -1;
  }
#pragma unroll
  for (int j = 0; j < NLA; ++j) {
    const int i = tid + j * THREADS;
    la_off[j] = (i < NA) ? mod(x0 + i % AX - 1, g.nx) + g.nx * mod(y0 + i / AX - 1, g.ny) : -1;
  }
  float pf_phi[NLD], pf_a[3][NLA];
  uint8_t pf_sol[NLD];
  auto fetch_phi = [&](int zw) {  // zw: wrapped plane index
    const float* pb = phi + (int64_t)zw * nxy;
    const uint8_t* fb = flags + (int64_t)zw * nxy;
#pragma unroll
    for (int j = 0; j < NLD; ++j) {
      if (ld_off[j] >= 0) {
        pf_phi[j] = __ldg(pb + ld_off[j]);
        pf_sol[j] = __ldg(fb + ld_off[j]) & FLAG_SOLID;
      }
    }
  };
  auto fetch_a = [&](int zw) {
    const float* ab = afld + (int64_t)zw * nxy;
#pragma unroll
    for (int j = 0; j < NLA; ++j) {
      if (la_off[j] >= 0) {
#pragma unroll
        for (int c = 0; c < 3; ++c) pf_a[c][j] = __ldg(ab + c * N + la_off[j]);
      }
    }
  };
  auto store_phi = [&](int kz) {
    float* sp = s_phi[kz & 3];
    uint8_t* ss = s_sol[kz & 3];
#pragma unroll
    for (int j = 0; j < NLD; ++j) {
      if (ld_off[j] >= 0) {
        sp[tid + j * THREADS] = pf_phi[j];
        ss[tid + j * THREADS] = pf_sol[j];
      }
    }
  };
  auto store_a = [&](int kz) {
#pragma unroll
    for (int j = 0; j < NLA; ++j) {
      if (la_off[j] >= 0) {
#pragma unroll
        for (int c = 0; c < 3; ++c) s_a[kz & 1][c][tid + j * THREADS] = pf_a[c][j];
      }
    }
  };

  // the two output rows of this thread
  const int x = x0 + tx;
  const int ya = y0 + 2 * ty, yb = ya + 1;
  const bool act_a = (x < g.nx) && (ya < g.ny);
  const bool act_b = (x < g.nx) && (yb < g.ny);
  const int xc = min(x, g.nx - 1);  // clamped: inactive threads load in bounds
  const int xm = wrap(xc, -1, g.nx), xp = wrap(xc, 1, g.nx);
  const int yam = wrap(min(ya, g.ny - 1), -1, g.ny);
  const int ybw = wrap(min(ya, g.ny - 1), 1, g.ny);  // row b, wrapped
  const int ybp = wrap(ybw, 1, g.ny);
  const int own_a = xc + g.nx * min(ya, g.ny - 1);
  const int own_b = xc + g.nx * ybw;
  const int cp = (tx + 2) + PX * (2 * ty + 2);  // row a in phi-plane coords
  const int ca = (tx + 1) + AX * (2 * ty + 1);  // row a in a-plane coords

  int zf = mod(z0 - 2, g.nz);
  fetch_phi(zf);
  store_phi(z0 - 2);
  zf = (zf + 1 == g.nz) ? 0 : zf + 1;
  fetch_phi(zf);
  store_phi(z0 - 1);
  const int za = zf;  // plane z0 - 1
  zf = (zf + 1 == g.nz) ? 0 : zf + 1;
  fetch_phi(zf);  // plane z0, stored at the first step
  fetch_a(za);    // plane z0 - 1
  __syncthreads();
  // own columns: phi at kz-2..kz+2, solid at kz-1..kz+1, rows a and b
  float ca5[5] = {0.f, 0.f, 0.f, s_phi[(z0 - 2) & 3][cp], s_phi[(z0 - 1) & 3][cp]};
  float cb5[5] = {0.f, 0.f, 0.f, s_phi[(z0 - 2) & 3][cp + PX], s_phi[(z0 - 1) & 3][cp + PX]};
  bool sa3[3] = {false, false, s_sol[(z0 - 2) & 3][cp] != 0};
  bool sb3[3] = {false, false, s_sol[(z0 - 2) & 3][cp + PX] != 0};
  float Ha[3] = {0.f, 0.f, 0.f}, Hb[3] = {0.f, 0.f, 0.f};
  float Va[3] = {0.f, 0.f, 0.f}, Vb[3] = {0.f, 0.f, 0.f};
  float La[3] = {0.f, 0.f, 0.f}, Lb[3] = {0.f, 0.f, 0.f};
  // z velocity of the own columns at kz-1, kz, kz+1 (rolled)
  const float* uz_ = u + 2 * N;
  float uza[3], uzb[3];
  {
    const int64_t zm = (int64_t)mod(z0 - 1, g.nz) * nxy;
    const int64_t zc = (int64_t)mod(z0, g.nz) * nxy;
    uza[0] = 0.f; uzb[0] = 0.f;
    uza[1] = __ldg(uz_ + zm + own_a);
    uzb[1] = __ldg(uz_ + zm + own_b);
    uza[2] = __ldg(uz_ + zc + own_a);
    uzb[2] = __ldg(uz_ + zc + own_b);
  }
  DF msum = {0.f, 0.f}, wsum = {0.f, 0.f};

  for (int kz = z0 - 2; kz < zend; ++kz) {
    store_phi(kz + 2);
    store_a(kz + 1);
    if (kz + 1 < zend) {
      const int zfa = zf;                     // plane kz + 2
      zf = (zf + 1 == g.nz) ? 0 : zf + 1;     // plane kz + 3
      fetch_phi(zf);
      fetch_a(zfa);
    }
    const bool out = kz >= z0;
    // velocities of the output plane: x and y components, and the z
    // component one plane ahead for the rolled column values
    float uxa[3], uxb[3], uy4[4];
    if (out) {
      const float* ux_ = u + (int64_t)kz * nxy;
      const float* uy_ = ux_ + N;
      const int zp = (kz == g.nz - 1) ? -(g.nz - 1) * nxy : nxy;
      const int ra = g.nx * min(ya, g.ny - 1), rb = g.nx * ybw;
      uxa[0] = __ldg(ux_ + ra + xm);
      uxa[1] = __ldg(ux_ + own_a);
      uxa[2] = __ldg(ux_ + ra + xp);
      uxb[0] = __ldg(ux_ + rb + xm);
      uxb[1] = __ldg(ux_ + own_b);
      uxb[2] = __ldg(ux_ + rb + xp);
      uy4[0] = __ldg(uy_ + g.nx * yam + xc);
      uy4[1] = __ldg(uy_ + own_a);
      uy4[2] = __ldg(uy_ + own_b);
      uy4[3] = __ldg(uy_ + g.nx * ybp + xc);
      const float* uzk = uz_ + (int64_t)kz * nxy + zp;
      uza[0] = uza[1]; uza[1] = uza[2]; uza[2] = __ldg(uzk + own_a);
      uzb[0] = uzb[1]; uzb[1] = uzb[2]; uzb[2] = __ldg(uzk + own_b);
    }
    __syncthreads();
    const float* P0 = s_phi[kz & 3];
    const float* P1 = s_phi[(kz + 1) & 3];
    // in-plane parts for plane kz + 1 at rows a and b:
    //   H = Dd_x S_y a_x + S_x Dd_y a_y, V = S_x S_y a_z, L = S_x S_y phi
    {
      const float* axp = s_a[(kz + 1) & 1][0];
      const float* ayp = s_a[(kz + 1) & 1][1];
      const float* azp = s_a[(kz + 1) & 1][2];
      float xm_[4], xp_[4], ym_[4][3], zz[4][3], pp[4][3];
#pragma unroll
      for (int r = 0; r < 4; ++r) {  // a-plane rows 2ty .. 2ty+3 (y-1 .. y+2)
        const int o = ca + (r - 1) * AX;
        xm_[r] = axp[o - 1];
        xp_[r] = axp[o + 1];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          ym_[r][d] = ayp[o + d - 1];
          zz[r][d] = azp[o + d - 1];
          pp[r][d] = P1[cp + (r - 1) * PX + d - 1];
        }
      }
      float H2[2], V2[2], L2[2];
#pragma unroll
      for (int j = 0; j < 2; ++j) {  // output row j uses rows j .. j+2
        const float sxp = xp_[j] + fmaf(4.f, xp_[j + 1], xp_[j + 2]);
        const float sxm = xm_[j] + fmaf(4.f, xm_[j + 1], xm_[j + 2]);
        const float d0 = ym_[j + 2][0] - ym_[j][0];
        const float d1 = ym_[j + 2][1] - ym_[j][1];
        const float d2 = ym_[j + 2][2] - ym_[j][2];
        H2[j] = (sxp - sxm + d0 + fmaf(4.f, d1, d2)) * (1.0f / 36.0f);
        float rz[3], rl[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          rz[r] = zz[j + r][0] + fmaf(4.f, zz[j + r][1], zz[j + r][2]);
          rl[r] = pp[j + r][0] + fmaf(4.f, pp[j + r][1], pp[j + r][2]);
        }
        V2[j] = (rz[0] + fmaf(4.f, rz[1], rz[2])) * (1.0f / 36.0f);
        L2[j] = (rl[0] + fmaf(4.f, rl[1], rl[2])) * (1.0f / 36.0f);
      }
      Ha[0] = Ha[1]; Ha[1] = Ha[2]; Ha[2] = H2[0];
      Hb[0] = Hb[1]; Hb[1] = Hb[2]; Hb[2] = H2[1];
      Va[0] = Va[1]; Va[1] = Va[2]; Va[2] = V2[0];
      Vb[0] = Vb[1]; Vb[1] = Vb[2]; Vb[2] = V2[1];
      La[0] = La[1]; La[1] = La[2]; La[2] = L2[0];
      Lb[0] = Lb[1]; Lb[1] = Lb[2]; Lb[2] = L2[1];
      const float* P2 = s_phi[(kz + 2) & 3];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        ca5[i] = ca5[i + 1];
        cb5[i] = cb5[i + 1];
      }
      ca5[4] = P2[cp];
      cb5[4] = P2[cp + PX];
      sa3[0] = sa3[1]; sa3[1] = sa3[2]; sa3[2] = s_sol[(kz + 1) & 3][cp] != 0;
      sb3[0] = sb3[1]; sb3[1] = sb3[2]; sb3[2] = s_sol[(kz + 1) & 3][cp + PX] != 0;
    }
    if (!out) continue;
    // output plane kz, rows a and b
    const uint8_t* sc = s_sol[kz & 3];
    // phi along y at rows ya-2 .. yb+2 of the own column
    const float py0 = P0[cp - 2 * PX], py1 = P0[cp - PX], py4 = P0[cp + 2 * PX],
                py5 = P0[cp + 3 * PX];
    const bool sy0 = sc[cp - PX] != 0, sy3 = sc[cp + 2 * PX] != 0;
    auto emit = [&](bool act, int own, int c, float v0, float cm2, float cm1,
                    float cp1, float cp2, bool solc, bool szm, bool szp,
                    float yv0, float yv1, float yv3, float yv4, bool sym, bool syp,
                    float ux0, float ux1, float ux2, float uy0, float uy1,
                    float uy2, float uz0, float uz1, float uz2, float h0,
                    float h1, float h2, float vv0, float vv2, float l0, float l1,
                    float l2) {
      if (!act) return;
      const int64_t n = own + (int64_t)kz * nxy;
      if (solc) {
        phi_out[n] = v0;
        return;
      }
      float div = muscl_axis(P0[c - 2], P0[c - 1], v0, P0[c + 1], P0[c + 2],
                             sc[c - 1] != 0, sc[c + 1] != 0, ux0, ux1, ux2);
      div += muscl_axis(yv0, yv1, v0, yv3, yv4, sym, syp, uy0, uy1, uy2);
      div += muscl_axis(cm2, cm1, v0, cp1, cp2, szm, szp, uz0, uz1, uz2);
      // lap = 6 (S_z L - phi), div_iso a = 3 S_z H + 3 Dd_z V
      const float lap = l0 + fmaf(4.f, l1, l2) - 6.f * v0;
      const float diva = 0.5f * (h0 + fmaf(4.f, h1, h2) + vv2 - vv0);
      const float vs = v0 - div + k.mobility * lap - k.kappa * diva;
      phi_out[n] = vs;
      df_add(msum, vs);
      const float chi = (vs > k.eps_phi && vs < 1.0f - k.eps_phi) ? vs * (1.0f - vs) : 0.f;
      df_add(wsum, chi);
    };
    emit(act_a, own_a, cp, ca5[2], ca5[0], ca5[1], ca5[3], ca5[4], sa3[1], sa3[0],
         sa3[2], py0, py1, cb5[2], py4, sy0, sb3[1], uxa[0], uxa[1], uxa[2],
         uy4[0], uy4[1], uy4[2], uza[0], uza[1], uza[2], Ha[0], Ha[1], Ha[2],
         Va[0], Va[2], La[0], La[1], La[2]);
    emit(act_b, own_b, cp + PX, cb5[2], cb5[0], cb5[1], cb5[3], cb5[4], sb3[1],
         sb3[0], sb3[2], py1, ca5[2], py4, py5, sa3[1], sy3, uxb[0], uxb[1],
         uxb[2], uy4[1], uy4[2], uy4[3], uzb[0], uzb[1], uzb[2], Hb[0], Hb[1],
         Hb[2], Vb[0], Vb[2], Lb[0], Lb[1], Lb[2]);
  }

  // block reduction of the two partial sums
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    msum = df_merge(msum, df_shfl_down(msum, off));
    wsum = df_merge(wsum, df_shfl_down(wsum, off));
  }
  const int lane = tid & 31, warp = tid >> 5;
  if (lane == 0) {
    red[0][warp] = msum;
    red[1][warp] = wsum;
  }
  __syncthreads();
  if (tid == 0) {
    double m = 0.0, w = 0.0;
    for (int i = 0; i < THREADS / 32; ++i) {
      m += (double)red[0][i].hi + (double)red[0][i].lo;
      w += (double)red[1][i].hi + (double)red[1][i].lo;
    }
    partials[pb] = m;
    partials[nblocks + pb] = w;
  }
}

template <int TY, int ZC, int MINB>
__global__ void __launch_bounds__(TX * TY / 2, MINB)
phase_update_march(const float* __restrict__ phi, const float* __restrict__ afld,
                   float* __restrict__ phi_out, const float* __restrict__ u,
                   const uint8_t* __restrict__ flags,
                   double* __restrict__ partials, int nblocks, Grid g,
                   Consts k) {
  const int pb = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
  phase_tile_body<TY, ZC>(blockIdx.x, blockIdx.y, blockIdx.z, pb, phi, afld,
                          phi_out, u, flags, partials, nblocks, g, k);
}

// Batched phi update: virtual block b is tile (bx, by, bz) of its case.
template <int TY, int ZC, int MINB>
__global__ void __launch_bounds__(TX * TY / 2, MINB)
phase_update_batch(const CaseDesc* __restrict__ cases, WorkList wl, int pc) {
  __shared__ CaseCursor cur;
  if (threadIdx.x == 0 && threadIdx.y == 0) cur.begin();
  __syncthreads();
  int b0, b1;
  block_range(wl, b0, b1);
  for (int b = b0; b < b1; ++b) {
    cur.seek(cases, wl, b);
    const CaseDesc& cd = cur.d;
    const int local = b - cur.cstart;
    const int nbx = (cd.g.nx + TX - 1) / TX, nby = (cd.g.ny + TY - 1) / TY;
    __syncthreads();  // the previous tile's shared-memory reads are done
    phase_tile_body<TY, ZC>(local % nbx, (local / nbx) % nby, local / (nbx * nby),
                            local, cd.phi[pc], cd.a, cd.phi[1 - pc], cd.u,
                            cd.flags, cd.partials, cd.phase_nb, cd.g, cd.k);
  }
}

// Compressive vector of phi at every node (0 at solid nodes), for a phi
// update run on its own: within a full step the collide-stream forms it.
__global__ void __launch_bounds__(256)
compressive_field(const float* __restrict__ phi, const uint8_t* __restrict__ flags,
                  float* __restrict__ a, Grid g) {
  const int x = blockIdx.x * 32 + (threadIdx.x & 31);
  const int y = blockIdx.y * 8 + (threadIdx.x >> 5);
  const int z = blockIdx.z;
  if (x >= g.nx || y >= g.ny) return;
  const int64_t nxy = (int64_t)g.nx * g.ny;
  const int64_t n = x + (int64_t)g.nx * y + nxy * z;
  float ax = 0.f, ay = 0.f, az = 0.f;
  if (!(flags[n] & FLAG_SOLID)) {
    const int xo[3] = {wrap(x, -1, g.nx), x, wrap(x, 1, g.nx)};
    const int yo[3] = {wrap(y, -1, g.ny) * g.nx, y * g.nx, wrap(y, 1, g.ny) * g.nx};
    const int64_t zo[3] = {wrap(z, -1, g.nz) * nxy, z * nxy, wrap(z, 1, g.nz) * nxy};
    float gx, gy, gz, ssum;
    phi_stencil(phi, xo, yo, zo, gx, gy, gz, ssum);
    compressive(__ldg(phi + n), gx, gy, gz, ax, ay, az);
  }
  a[n] = ax;
  a[g.N + n] = ay;
  a[2 * g.N + n] = az;
}

struct PhaseShape {
  int ty, zc;
};

PhaseShape phase_shape(int variant) {
  switch (variant) {
    case 1: return {8, 16};
    case 2: return {8, 32};
    case 3: return {16, 32};
    default: return {16, 16};
  }
}

dim3 phase_grid(const Grid& g, int variant) {
  const PhaseShape s = phase_shape(variant);
  return dim3((g.nx + TX - 1) / TX, (g.ny + s.ty - 1) / s.ty,
              (g.nz + s.zc - 1) / s.zc);
}

}  // namespace

int phase_blocks(const cacl_ctx* c) {
  // partial-sum storage is sized for the variant with the most blocks
  int nb = 0;
  for (int v = 0; v < 4; ++v) {
    const dim3 gr = phase_grid(c->g, v);
    nb = std::max(nb, (int)(gr.x * gr.y * gr.z));
  }
  return nb;
}

cudaError_t phase_init_attributes() { return cudaSuccess; }

void phase_tile(int variant, int& ty, int& zc) {
  const PhaseShape s = phase_shape(variant);
  ty = s.ty;
  zc = s.zc;
}

namespace {
void* phase_batch_kernel(int variant) {
  switch (variant) {
    case 1: return (void*)phase_update_batch<8, 16, 4>;
    case 2: return (void*)phase_update_batch<8, 32, 4>;
    case 3: return (void*)phase_update_batch<16, 32, 2>;
    default: return (void*)phase_update_batch<16, 16, 2>;
  }
}
}  // namespace

int phase_batch_occupancy(int variant) {
  int nb = 0;
  const PhaseShape s = phase_shape(variant);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, phase_batch_kernel(variant),
                                                TX * s.ty / 2, 0);
  return nb;
}

cudaError_t launch_phase_batch(const CaseDesc* cases, WorkList wl, int variant,
                               int grid, int pc, cudaStream_t st) {
  const PhaseShape s = phase_shape(variant);
  void* args[] = {(void*)&cases, (void*)&wl, (void*)&pc};
  return cudaLaunchKernel(phase_batch_kernel(variant), dim3(grid),
                          dim3(TX, s.ty / 2, 1), args, 0, st);
}

cudaError_t launch_compressive(cacl_ctx* c, const float* phi) {
  const Grid g = c->g;
  const dim3 grid((g.nx + 31) / 32, (g.ny + 7) / 8, g.nz);
  compressive_field<<<grid, 256, 0, c->stream>>>(phi, c->flags, c->a, g);
  return cudaGetLastError();
}

cudaError_t launch_phase(cacl_ctx* c, const float* phi_in, float* phi_out) {
  const int v = c->phase_variant;
  const dim3 grid = phase_grid(c->g, v);
  const int nb = (int)(grid.x * grid.y * grid.z);
  c->phase_nblocks = nb;
  const PhaseShape s = phase_shape(v);
  const dim3 block(TX, s.ty / 2, 1);
  switch (v) {
    case 1:
      phase_update_march<8, 16, 4><<<grid, block, 0, c->stream>>>(
          phi_in, c->a, phi_out, c->u, c->flags, c->partials, nb, c->g, c->k);
      break;
    case 2:
      phase_update_march<8, 32, 4><<<grid, block, 0, c->stream>>>(
          phi_in, c->a, phi_out, c->u, c->flags, c->partials, nb, c->g, c->k);
      break;
    case 3:
      phase_update_march<16, 32, 2><<<grid, block, 0, c->stream>>>(
          phi_in, c->a, phi_out, c->u, c->flags, c->partials, nb, c->g, c->k);
      break;
    default:
      phase_update_march<16, 16, 2><<<grid, block, 0, c->stream>>>(
          phi_in, c->a, phi_out, c->u, c->flags, c->partials, nb, c->g, c->k);
      break;
  }
  return cudaGetLastError();
}

}  // namespace cacl
