// phase.cu -- conservative Allen-Cahn update of phi at fluid nodes
// (Sect. 2.2: Eqs. phi_update_muscl, divF, face_flux_def, slope_minmod_x,
// minmod, recon_lr_x, upwind_select_x, source_sharp; Eq. lap_iso), plus the
// per-block partial sums of the volume correction (Sect. 2.4,
// Eqs. tentative_phase_field_mass, mass_correction_normalization).
//
// Each block owns a TX x TY x TZ tile. phi and the solid flags of the tile
// plus a halo of 2 (the reach of the minmod slopes of the neighbouring
// cells) are staged in shared memory; the compressive vector
// a = phi (1 - phi) grad phi / |grad phi| is formed once per node of the
// tile plus a halo of 1 and kept in shared memory, so its isotropic
// divergence costs 27 shared reads instead of 27 gradient evaluations.
// Face velocities are the mean of the two cell velocities and vanish on
// fluid-solid faces; the compressive vector is zero at solid nodes.
//
// Partial sums are accumulated per thread as unevaluated float pairs
// (Knuth's two-sum), combined across the block the same way, and written as
// FP64 per block: FP64 arithmetic stays out of the per-node path.
#include "cacl_internal.cuh"

namespace cacl {
namespace {

constexpr int TX = 32, TY = 8, TZ = 8;
constexpr int PX = TX + 4, PY = TY + 4, PZ = TZ + 4;  // phi tile, halo 2
constexpr int AX = TX + 2, AY = TY + 2, AZ = TZ + 2;  // a tile, halo 1
constexpr int PHASE_THREADS = TX * TY;
constexpr int NPHI = PX * PY * PZ;
constexpr int NA = AX * AY * AZ;
constexpr size_t PHASE_SMEM = sizeof(float) * (NPHI + 3 * NA) + NPHI;

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

__device__ __forceinline__ float minmod(float a, float b) {
  return (a * b <= 0.f) ? 0.f : (a > 0.f ? fminf(a, b) : fmaxf(a, b));
}

__device__ __forceinline__ int mod(int i, int n) {
  const int r = i % n;
  return r < 0 ? r + n : r;
}

__global__ void __launch_bounds__(PHASE_THREADS)
phase_update_tile(const float* __restrict__ phi, float* __restrict__ phi_out,
                  const float* __restrict__ u, const uint8_t* __restrict__ flags,
                  double* __restrict__ partials, int nblocks, Grid g, Consts k) {
  extern __shared__ float smem[];
  float* sphi = smem;                     // [PZ][PY][PX]
  float* sa = smem + NPHI;                // [3][AZ][AY][AX]
  uint8_t* ssol = (uint8_t*)(sa + 3 * NA);  // [PZ][PY][PX]

  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * TZ;
  const int tid = threadIdx.x + TX * threadIdx.y;
  const int64_t nxy = (int64_t)g.nx * g.ny;

  for (int i = tid; i < NPHI; i += PHASE_THREADS) {
    const int lx = i % PX, ly = (i / PX) % PY, lz = i / (PX * PY);
    const int gx = mod(x0 + lx - 2, g.nx), gy = mod(y0 + ly - 2, g.ny),
              gz = mod(z0 + lz - 2, g.nz);
    const int64_t n = gx + (int64_t)g.nx * gy + nxy * gz;
    sphi[i] = __ldg(phi + n);
    ssol[i] = __ldg(flags + n) & FLAG_SOLID;
  }
  __syncthreads();

  // compressive vector on the tile plus halo 1
  for (int i = tid; i < NA; i += PHASE_THREADS) {
    const int ax = i % AX, ay = (i / AX) % AY, az = i / (AX * AY);
    const int c = (ax + 1) + PX * ((ay + 1) + PY * (az + 1));
    float vx = 0.f, vy = 0.f, vz = 0.f;
    if (!ssol[c]) {
      float gx = 0.f, gy = 0.f, gz = 0.f;
#pragma unroll
      for (int q = 0; q < REST; ++q) {
        const int off = cx(q) + PX * (cy(q) + PY * cz(q));
        const float dv = (3.0f * wq(q)) * (sphi[c + off] - sphi[c - off]);
        gx += cx(q) * dv;
        gy += cy(q) * dv;
        gz += cz(q) * dv;
      }
      const float gm = sqrtf(gx * gx + gy * gy + gz * gz);
      if (gm >= 1e-12f) {
        const float v = sphi[c];
        const float s = v * (1.0f - v) / gm;
        vx = s * gx;
        vy = s * gy;
        vz = s * gz;
      }
    }
    sa[i] = vx;
    sa[NA + i] = vy;
    sa[2 * NA + i] = vz;
  }
  __syncthreads();

  DF msum = {0.f, 0.f}, wsum = {0.f, 0.f};
  const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
  const int64_t N = g.N;
  if (x < g.nx && y < g.ny) {
    const int xo[3] = {wrap(x, -1, g.nx), x, wrap(x, 1, g.nx)};
    const int yo[3] = {wrap(y, -1, g.ny) * g.nx, y * g.nx, wrap(y, 1, g.ny) * g.nx};
    for (int tz = 0; tz < TZ; ++tz) {
      const int z = z0 + tz;
      if (z >= g.nz) break;
      const int64_t zo[3] = {wrap(z, -1, g.nz) * nxy, z * nxy,
                             wrap(z, 1, g.nz) * nxy};
      const int64_t n = xo[1] + yo[1] + zo[1];
      const int c = (threadIdx.x + 2) + PX * ((threadIdx.y + 2) + PY * (tz + 2));
      const float v0 = sphi[c];
      if (ssol[c]) {
        phi_out[n] = v0;
        continue;
      }
      // MUSCL-minmod advective divergence, one axis at a time
      float div = 0.f;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const int st = (d == 0) ? 1 : (d == 1) ? PX : PX * PY;
        const float vm2 = sphi[c - 2 * st], vm1 = sphi[c - st];
        const float vp1 = sphi[c + st], vp2 = sphi[c + 2 * st];
        const float sm = minmod(vm1 - vm2, v0 - vm1);
        const float s0 = minmod(v0 - vm1, vp1 - v0);
        const float sp = minmod(vp1 - v0, vp2 - vp1);
        const float* ud = u + (int64_t)d * N;
        const int64_t np = (d == 0) ? xo[2] + yo[1] + zo[1]
                         : (d == 1) ? xo[1] + yo[2] + zo[1]
                                    : xo[1] + yo[1] + zo[2];
        const int64_t nm = (d == 0) ? xo[0] + yo[1] + zo[1]
                         : (d == 1) ? xo[1] + yo[0] + zo[1]
                                    : xo[1] + yo[1] + zo[0];
        const float uc = __ldg(ud + n);
        float fp = 0.f, fm = 0.f;
        if (!ssol[c + st]) {
          const float uf = 0.5f * (uc + __ldg(ud + np));
          fp = uf * ((uf >= 0.f) ? v0 + 0.5f * s0 : vp1 - 0.5f * sp);
        }
        if (!ssol[c - st]) {
          const float uf = 0.5f * (__ldg(ud + nm) + uc);
          fm = uf * ((uf >= 0.f) ? vm1 + 0.5f * sm : v0 - 0.5f * s0);
        }
        div += fp - fm;
      }
      // isotropic Laplacian and divergence of a, pairs of opposite links
      const int ca = (threadIdx.x + 1) + AX * ((threadIdx.y + 1) + AY * (tz + 1));
      float ssum = 0.f, diva = 0.f;
#pragma unroll
      for (int q = 0; q < REST; ++q) {
        const int off = cx(q) + PX * (cy(q) + PY * cz(q));
        ssum += wq(q) * (sphi[c + off] + sphi[c - off]);
        const int oa = cx(q) + AX * (cy(q) + AY * cz(q));
        const float dax = sa[ca + oa] - sa[ca - oa];
        const float day = sa[NA + ca + oa] - sa[NA + ca - oa];
        const float daz = sa[2 * NA + ca + oa] - sa[2 * NA + ca - oa];
        diva += (3.0f * wq(q)) * (cx(q) * dax + cy(q) * day + cz(q) * daz);
      }
      const float lap = 6.0f * (ssum - (1.0f - wq(REST)) * v0);
      const float vs = v0 - div + k.mobility * lap - k.kappa * diva;
      phi_out[n] = vs;
      df_add(msum, vs);
      const float chi = (vs > k.eps_phi && vs < 1.0f - k.eps_phi) ? vs * (1.0f - vs) : 0.f;
      df_add(wsum, chi);
    }
  }

  // block reduction of the two partial sums
  __shared__ DF red[2][PHASE_THREADS / 32];
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
    for (int i = 0; i < PHASE_THREADS / 32; ++i) {
      m += (double)red[0][i].hi + (double)red[0][i].lo;
      w += (double)red[1][i].hi + (double)red[1][i].lo;
    }
    const int b = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    partials[b] = m;
    partials[nblocks + b] = w;
  }
}

dim3 phase_grid(const Grid& g) {
  return dim3((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY, (g.nz + TZ - 1) / TZ);
}

}  // namespace

int phase_blocks(const cacl_ctx* c) {
  const dim3 gr = phase_grid(c->g);
  return (int)(gr.x * gr.y * gr.z);
}

cudaError_t phase_init_attributes() {
  return cudaFuncSetAttribute(phase_update_tile,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)PHASE_SMEM);
}

cudaError_t launch_phase(cacl_ctx* c, const float* phi_in, float* phi_out) {
  const dim3 grid = phase_grid(c->g);
  const int nb = (int)(grid.x * grid.y * grid.z);
  phase_update_tile<<<grid, dim3(TX, TY, 1), PHASE_SMEM, c->stream>>>(
      phi_in, phi_out, c->u, c->flags, c->partials, nb, c->g, c->k);
  return cudaGetLastError();
}

}  // namespace cacl
