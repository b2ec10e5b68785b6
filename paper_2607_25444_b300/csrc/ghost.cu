// ghost.cu -- ghost phi values at wall nodes (Sect. 2.2, Algorithm 1,
// Eqs. tangential_gradient_contact_angle .. contact_angle_localization).
//
// Jacobi semantics: ghost_eval computes every ghost from phi^n into a
// scratch array, ghost_scatter then writes them into phi^n. A wall node
// reads only its donor's 27-point neighbourhood and writes only its own
// scratch slot, so the pass is race-free without atomics.
#include "cacl_internal.cuh"

namespace cacl {
namespace {

constexpr int GHOST_THREADS = 128;

__device__ __forceinline__ void ghost_one(int w, const float* __restrict__ phi,
                                          const int32_t* __restrict__ donor,
                                          const int8_t* __restrict__ qstar,
                                          const float* __restrict__ nw,
                                          const float* __restrict__ cot_c,
                                          float* __restrict__ g_out, int W,
                                          const Grid& g) {
  const int d = donor[w];
  const int x = d % g.nx;
  const int r = d / g.nx;
  const int y = r % g.ny;
  const int z = r / g.ny;
  const int xo[3] = {wrap(x, -1, g.nx), x, wrap(x, 1, g.nx)};
  const int yo[3] = {wrap(y, -1, g.ny) * g.nx, y * g.nx, wrap(y, 1, g.ny) * g.nx};
  const int64_t nxy = (int64_t)g.nx * g.ny;
  const int64_t zo[3] = {wrap(z, -1, g.nz) * nxy, z * nxy, wrap(z, 1, g.nz) * nxy};
  // isotropic gradient at the donor (Eq. grad_iso), pairs of opposite links
  float gx = 0.f, gy = 0.f, gz = 0.f;
#pragma unroll
  for (int q = 0; q < REST; ++q) {
    const float vp = __ldg(phi + xo[1 + cx(q)] + yo[1 + cy(q)] + zo[1 + cz(q)]);
    const float vm = __ldg(phi + xo[1 - cx(q)] + yo[1 - cy(q)] + zo[1 - cz(q)]);
    const float dv = 3.0f * wq(q) * (vp - vm);
    gx += cx(q) * dv;
    gy += cy(q) * dv;
    gz += cz(q) * dv;
  }
  const float phi_f = __ldg(phi + d);
  const float nx_ = nw[w], ny_ = nw[W + w], nz_ = nw[2 * W + w];
  const float gn = gx * nx_ + gy * ny_ + gz * nz_;
  const float px = gx - gn * nx_, py = gy - gn * ny_, pz = gz - gn * nz_;
  const float t = sqrtf(px * px + py * py + pz * pz);
  const float dn = -t * cot_c[w];
  const float cgx = px + dn * nx_, cgy = py + dn * ny_, cgz = pz + dn * nz_;
  const float lam = sqrtf(fmaxf(0.f, 4.f * phi_f * (1.f - phi_f)));
  const int q = qstar[w];
  // r_fs = -c_{q*} (Eq. donor_to_solid)
  const float dot = -(cgx * (float)(q % 3 - 1) + cgy * (float)((q / 3) % 3 - 1) +
                      cgz * (float)(q / 9 - 1));
  g_out[w] = phi_f + lam * dot;
}

__global__ void __launch_bounds__(GHOST_THREADS)
ghost_eval(const float* __restrict__ phi, const int32_t* __restrict__ donor,
           const int8_t* __restrict__ qstar, const float* __restrict__ nw,
           const float* __restrict__ cot_c, float* __restrict__ g_out, int W,
           Grid g) {
  const int w = blockIdx.x * GHOST_THREADS + threadIdx.x;
  if (w < W) ghost_one(w, phi, donor, qstar, nw, cot_c, g_out, W, g);
}

// Batched ghost pass: virtual block b covers GHOST_THREADS wall nodes of
// its case. eval and scatter are separate launches (Jacobi semantics).
__global__ void __launch_bounds__(GHOST_THREADS)
ghost_eval_batch(const CaseDesc* __restrict__ cases, WorkList wl, int pc) {
  __shared__ CaseCursor cur;
  if (threadIdx.x == 0) cur.begin();
  __syncthreads();
  int b0, b1;
  block_range(wl, b0, b1);
  for (int b = b0; b < b1; ++b) {
    cur.seek(cases, wl, b);
    const CaseDesc& cd = cur.d;
    const int w = (b - cur.cstart) * GHOST_THREADS + threadIdx.x;
    if (w < cd.W)
      ghost_one(w, cd.phi[pc], cd.w_donor, cd.w_q, cd.w_nw, cd.w_cot, cd.w_g,
                cd.W, cd.g);
  }
}

__global__ void __launch_bounds__(GHOST_THREADS)
ghost_scatter_batch(const CaseDesc* __restrict__ cases, WorkList wl, int pc) {
  __shared__ CaseCursor cur;
  if (threadIdx.x == 0) cur.begin();
  __syncthreads();
  int b0, b1;
  block_range(wl, b0, b1);
  for (int b = b0; b < b1; ++b) {
    cur.seek(cases, wl, b);
    const CaseDesc& cd = cur.d;
    const int w = (b - cur.cstart) * GHOST_THREADS + threadIdx.x;
    if (w < cd.W) cd.phi[pc][cd.w_idx[w]] = cd.w_g[w];
  }
}

__global__ void __launch_bounds__(GHOST_THREADS)
ghost_scatter(float* __restrict__ phi, const int32_t* __restrict__ idx,
              const float* __restrict__ g_in, int W) {
  const int w = blockIdx.x * GHOST_THREADS + threadIdx.x;
  if (w < W) phi[idx[w]] = g_in[w];
}

}  // namespace

int ghost_batch_block() { return GHOST_THREADS; }

cudaError_t launch_ghost_batch(const CaseDesc* cases, WorkList wl, int grid,
                               int pc, cudaStream_t st) {
  if (wl.total == 0) return cudaSuccess;
  ghost_eval_batch<<<grid, GHOST_THREADS, 0, st>>>(cases, wl, pc);
  ghost_scatter_batch<<<grid, GHOST_THREADS, 0, st>>>(cases, wl, pc);
  return cudaGetLastError();
}

cudaError_t launch_ghost(cacl_ctx* c, float* phi) {
  const int W = c->wall_count;
  if (W == 0) return cudaSuccess;
  const int nb = (W + GHOST_THREADS - 1) / GHOST_THREADS;
  ghost_eval<<<nb, GHOST_THREADS, 0, c->stream>>>(phi, c->w_donor, c->w_q,
                                                   c->w_nw, c->w_cot, c->w_g,
                                                   W, c->g);
  ghost_scatter<<<nb, GHOST_THREADS, 0, c->stream>>>(phi, c->w_idx, c->w_g, W);
  return cudaGetLastError();
}

}  // namespace cacl
