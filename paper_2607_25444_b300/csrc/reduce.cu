// reduce.cu -- volume correction (Sect. 2.3, Eqs. mass_defect,
// interface_weight_mass_correction, mass_correction_normalization,
// mass_corrected_phi), the initial state (Eq. feq3 at p* = 0), the mass
// reference (Eq. phase_field_mass) and small state queries.
//
// The correction is deterministic: the phase update leaves one FP64 pair
// (sum phi*, sum chi) per block, and its last block to finish sums them in
// a fixed order and forms lambda = (M_ref - M*)/W (0 when W = 0; the
// batched path does the same in finalize_mass_batch); correct_phi applies
// phi = phi* + lambda chi(phi*) at fluid nodes.
#include "cacl_internal.cuh"

namespace cacl {
namespace {

constexpr int ELEM_THREADS = 256;

__global__ void __launch_bounds__(32)
finalize_mass_ref(const double* __restrict__ partials, int nb,
                  MassScalars* ms) {
  const double m = warp_sum_fixed(partials, nb, threadIdx.x);
  if (threadIdx.x == 0) {
    ms->m_ref = m;
    ms->m_star = m;
    ms->w_sum = 0.0;
    ms->lambda = 0.0;
    ms->lambda_f = 0.0f;
    ms->step = 0;
  }
}

// Batched finalize: block c (one warp) reduces case c's partials.
__global__ void __launch_bounds__(32)
finalize_mass_batch(const CaseDesc* __restrict__ cases) {
  const CaseDesc& cd = cases[blockIdx.x];
  mass_from_partials(cd.partials, cd.phase_nb, cd.mass, threadIdx.x);
}

// phi = phi* + lambda chi(phi*) at the fluid nodes of a group of four
// held in registers (v, their flags fl), rounded without bias; the rounding
// key of the group's first node is key0. Returns whether any node of the
// group is in the interface band (outside it chi = 0 and phi is unchanged).
__device__ __forceinline__ bool correct4(float4& v, uchar4 fl, float lam, uint32_t step,
                                         float eps, int64_t key0) {
  float* pv = &v.x;
  const uint8_t fa[4] = {fl.x, fl.y, fl.z, fl.w};
  bool band = false;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float s = pv[j];
    const bool in = (s > eps && s < 1.0f - eps) && !(fa[j] & FLAG_SOLID);
    if (in) pv[j] = add_unbiased(s, lam * (s * (1.0f - s)), step, key0 + j);
    band |= in;
  }
  return band;
}

// The same at the fluid nodes i4 .. i4 + 3 of a field of N nodes (i4 a
// multiple of 4, fewer at the end); the rounding key of node n is
// node_offset + n.
__device__ __forceinline__ void correct_group(float* __restrict__ phi,
                                              const uint8_t* __restrict__ flags,
                                              float lam, uint32_t step, float eps,
                                              int64_t N, int64_t i4,
                                              int64_t node_offset) {
  if (i4 + 3 < N) {
    float4 v = *reinterpret_cast<const float4*>(phi + i4);
    const uchar4 fl = *reinterpret_cast<const uchar4*>(flags + i4);
    if (correct4(v, fl, lam, step, eps, node_offset + i4))
      *reinterpret_cast<float4*>(phi + i4) = v;  // band nodes only
  } else {
    for (int64_t n = i4; n < N; ++n) {
      const float s = phi[n];
      if ((s > eps && s < 1.0f - eps) && !(flags[n] & FLAG_SOLID))
        phi[n] = add_unbiased(s, lam * (s * (1.0f - s)), step, node_offset + n);
    }
  }
}

// The correction over one field, four nodes per thread.
__global__ void __launch_bounds__(ELEM_THREADS)
correct_phi(float* __restrict__ phi, const uint8_t* __restrict__ flags,
            const MassScalars* __restrict__ ms, int64_t N, float eps,
            int64_t node_offset) {
  const int64_t i4 = ((int64_t)blockIdx.x * ELEM_THREADS + threadIdx.x) * 4;
  correct_group(phi, flags, ms->lambda_f, ms->step, eps, N, i4, node_offset);
}

// The correction right after a phi update, by the update's tiles (32 x ty x
// zc nodes from (32 bx, ty by, zc bz); ty, zc powers of two). chi is
// non-negative, so a tile's chi sum, which the update left in wsum, is zero
// only when no node of the tile is in the interface band; there phi = phi*
// is left as it is. A tile is split along z into `split` blocks (block
// (bx, by, bz') covers planes zc bz + tz s .. + tz - 1 of tile (bx, by, bz),
// tz = zc / split, s = bz' % split): many tiles take one block each, and
// the few tiles of a small grid spread their band work over several; a
// block of a tile without band nodes returns after one load. The nodes are
// corrected as in correct_phi (four per group when VEC, nx % 4 == 0), with
// the same rounding keys: the field is bit-identical to correct_phi's. A
// thread loads up to TB groups before it corrects and stores them.
template <bool VEC, int TB>
__global__ void __launch_bounds__(ELEM_THREADS)
correct_tiles(float* __restrict__ phi, const uint8_t* __restrict__ flags,
              const MassScalars* __restrict__ ms, const double* __restrict__ wsum,
              Grid g, int ty, int zc, int split, float eps, int64_t node_offset) {
  const int bz = blockIdx.z / split, sz = blockIdx.z % split;
  const int pb = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * bz);
  if (!(wsum[pb] > 0.0)) return;
  const float lam = ms->lambda_f;
  const uint32_t step = ms->step;
  const int tz = zc / split;
  const int x0 = 32 * blockIdx.x, y0 = ty * blockIdx.y, z0 = zc * bz + tz * sz;
  constexpr int PER_ROW = VEC ? 8 : 32;  // groups (or nodes) per tile row
  const int items = ty * tz * PER_ROW;
  for (int j0 = threadIdx.x; j0 < items; j0 += TB * ELEM_THREADS) {
    int64_t n[TB];
    bool ok[TB];
#pragma unroll
    for (int t = 0; t < TB; ++t) {
      const int j = j0 + t * ELEM_THREADS;
      const int r = j / PER_ROW, c = j % PER_ROW;
      const int x = x0 + (VEC ? 4 * c : c), y = y0 + r % ty, z = z0 + r / ty;
      ok[t] = j < items && x < g.nx && y < g.ny && z < g.nz;
      n[t] = x + (int64_t)g.nx * (y + (int64_t)g.ny * z);
    }
    if constexpr (VEC) {
      float4 v[TB];
      uchar4 fl[TB];
#pragma unroll
      for (int t = 0; t < TB; ++t)
        if (ok[t]) {
          v[t] = *reinterpret_cast<const float4*>(phi + n[t]);
          fl[t] = *reinterpret_cast<const uchar4*>(flags + n[t]);
        }
#pragma unroll
      for (int t = 0; t < TB; ++t)
        if (ok[t] && correct4(v[t], fl[t], lam, step, eps, node_offset + n[t]))
          *reinterpret_cast<float4*>(phi + n[t]) = v[t];
    } else {
      float v[TB];
      uint8_t fl[TB];
#pragma unroll
      for (int t = 0; t < TB; ++t)
        if (ok[t]) {
          v[t] = phi[n[t]];
          fl[t] = flags[n[t]];
        }
#pragma unroll
      for (int t = 0; t < TB; ++t) {
        const float s = v[t];
        if (ok[t] && (s > eps && s < 1.0f - eps) && !(fl[t] & FLAG_SOLID))
          phi[n[t]] = add_unbiased(s, lam * (s * (1.0f - s)), step, node_offset + n[t]);
      }
    }
  }
}

// Batched correction: virtual block b covers 4 * ELEM_THREADS nodes of its
// case, four per thread as in correct_phi.
__global__ void __launch_bounds__(ELEM_THREADS)
correct_phi_batch(const CaseDesc* __restrict__ cases, WorkList wl, int pc) {
  __shared__ CaseCursor cur;
  if (threadIdx.x == 0) cur.begin();
  __syncthreads();
  int b0, b1;
  block_range(wl, b0, b1);
  for (int b = b0; b < b1; ++b) {
    cur.seek(cases, wl, b);
    const CaseDesc& cd = cur.d;
    const int64_t i4 = ((int64_t)(b - cur.cstart) * ELEM_THREADS + threadIdx.x) * 4;
    correct_group(cd.phi[1 - pc], cd.flags, cd.mass->lambda_f, cd.mass->step,
                  cd.k.eps_phi, cd.g.N, i4, 0);
  }
}

// FP64 block partials of sum phi over fluid nodes (once per set_fields).
__global__ void __launch_bounds__(ELEM_THREADS)
fluid_sum(const float* __restrict__ phi, const uint8_t* __restrict__ flags,
          int64_t N, double* __restrict__ partials) {
  __shared__ double sh[ELEM_THREADS];
  double s = 0.0;
  const int64_t base = (int64_t)blockIdx.x * ELEM_THREADS * 8;
  for (int j = 0; j < 8; ++j) {
    const int64_t n = base + j * ELEM_THREADS + threadIdx.x;
    if (n < N && !(flags[n] & FLAG_SOLID)) s += (double)phi[n];
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = ELEM_THREADS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = sh[0];
}

// f = f^eq(p* = 0, u) (Eq. feq3) into both population buffers; u = 0 at
// solid nodes.
template <typename Store>
__global__ void __launch_bounds__(ELEM_THREADS)
init_populations(typename Store::T* __restrict__ f0,
                 typename Store::T* __restrict__ f1, float* __restrict__ u,
                 const uint8_t* __restrict__ flags, int64_t N) {
  const int64_t n = (int64_t)blockIdx.x * ELEM_THREADS + threadIdx.x;
  if (n >= N) return;
  float ux = u[n], uy = u[N + n], uz = u[2 * N + n];
  if (flags[n] & FLAG_SOLID) {
    ux = uy = uz = 0.f;
    u[n] = 0.f;
    u[N + n] = 0.f;
    u[2 * N + n] = 0.f;
  }
  const float uu = ux * ux + uy * uy + uz * uz;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const float cu = cx(q) * ux + cy(q) * uy + cz(q) * uz;
    const float v = wq(q) * (3.0f * cu + 4.5f * cu * cu - 1.5f * uu +
                             4.5f * cu * (cu * cu - uu));
    f0[(int64_t)q * N + n] = Store::encode(v, q);
    f1[(int64_t)q * N + n] = Store::encode(v, q);
  }
}

template <typename Store>
__global__ void __launch_bounds__(ELEM_THREADS)
pstar_kernel(const typename Store::T* __restrict__ f,
             const uint8_t* __restrict__ flags, int64_t N,
             float* __restrict__ out) {
  const int64_t n = (int64_t)blockIdx.x * ELEM_THREADS + threadIdx.x;
  if (n >= N) return;
  float s = 0.f;
#pragma unroll
  for (int q = 0; q < Q; ++q) s += Store::decode(f[(int64_t)q * N + n], q);
  out[n] = (flags[n] & FLAG_SOLID) ? 0.f : s;
}

// FP32 populations [q][n] <-> the storage type.
template <typename Store>
__global__ void __launch_bounds__(ELEM_THREADS)
to_storage(const float* __restrict__ src, typename Store::T* __restrict__ dst,
           int64_t N) {
  const int64_t n = (int64_t)blockIdx.x * ELEM_THREADS + threadIdx.x;
  if (n >= N) return;
#pragma unroll
  for (int q = 0; q < Q; ++q)
    dst[(int64_t)q * N + n] = Store::encode(src[(int64_t)q * N + n], q);
}

template <typename Store>
__global__ void __launch_bounds__(ELEM_THREADS)
from_storage(const typename Store::T* __restrict__ src, float* __restrict__ dst,
             int64_t N) {
  const int64_t n = (int64_t)blockIdx.x * ELEM_THREADS + threadIdx.x;
  if (n >= N) return;
#pragma unroll
  for (int q = 0; q < Q; ++q)
    dst[(int64_t)q * N + n] = Store::decode(src[(int64_t)q * N + n], q);
}

__global__ void __launch_bounds__(ELEM_THREADS)
finite_kernel(const float* __restrict__ phi, const float* __restrict__ u,
              const uint8_t* __restrict__ flags, int64_t N, int* bad) {
  const int64_t n = (int64_t)blockIdx.x * ELEM_THREADS + threadIdx.x;
  if (n >= N) return;
  if (flags[n] & FLAG_SOLID) return;
  const bool ok = isfinite(phi[n]) && isfinite(u[n]) && isfinite(u[N + n]) &&
                  isfinite(u[2 * N + n]);
  if (!ok) atomicOr(bad, 1);
}

int elem_blocks(int64_t N) { return (int)((N + ELEM_THREADS - 1) / ELEM_THREADS); }

}  // namespace

cudaError_t launch_correct(cacl_ctx* c, float* phi) {
  // lambda was formed by the last block of the phi update
  const int64_t N = c->g.N;
  const int nb = (int)((N + 4 * ELEM_THREADS - 1) / (4 * ELEM_THREADS));
  correct_phi<<<nb, ELEM_THREADS, 0, c->stream>>>(phi, c->flags, c->mass, N,
                                                 c->k.eps_phi, c->node_offset);
  return cudaGetLastError();
}

cudaError_t launch_correct_tiles(cacl_ctx* c, float* phi) {
  // the tiles and chi sums of the phi update that wrote phi
  int ty = 0, zc = 0;
  phase_tile(c->phase_variant, ty, zc);
  const Grid g = c->g;
  const int gx = (g.nx + 31) / 32, gy = (g.ny + ty - 1) / ty, gz = (g.nz + zc - 1) / zc;
  // at least about 2048 blocks (the tiles of 256^3), at most 4 planes each
  int split = 1;
  while (split < zc / 4 && (int64_t)gx * gy * gz * split < 2048) split *= 2;
  const dim3 grid(gx, gy, gz * split);
  const double* wsum = c->partials + c->phase_nblocks;
  const bool vec = g.nx % 4 == 0 && ((uintptr_t)phi & 15u) == 0;
  // groups in flight per thread: all of a whole tile's share, or two
  auto fn = vec ? (split == 1 ? correct_tiles<true, 8> : correct_tiles<true, 2>)
                : (split == 1 ? correct_tiles<false, 8> : correct_tiles<false, 2>);
  fn<<<grid, ELEM_THREADS, 0, c->stream>>>(phi, c->flags, c->mass, wsum, g, ty, zc, split,
                                           c->k.eps_phi, c->node_offset);
  return cudaGetLastError();
}

// lambda from partial sums gathered by the caller (nb phi* sums, then nb
// chi sums), in the fixed order of the phi update's own finalize.
__global__ void __launch_bounds__(32)
finalize_mass_from(const double* __restrict__ partials, int nb, MassScalars* ms) {
  mass_from_partials(partials, nb, ms, threadIdx.x);
}

cudaError_t launch_mass_from(cacl_ctx* c, const double* partials, int nb) {
  finalize_mass_from<<<1, 32, 0, c->stream>>>(partials, nb, c->mass);
  return cudaGetLastError();
}

int correct_batch_nodes() { return 4 * ELEM_THREADS; }

cudaError_t launch_correct_batch(const CaseDesc* cases, int ncases, WorkList wl,
                                 int grid, int pc, cudaStream_t st) {
  finalize_mass_batch<<<ncases, 32, 0, st>>>(cases);
  correct_phi_batch<<<grid, ELEM_THREADS, 0, st>>>(cases, wl, pc);
  return cudaGetLastError();
}

cudaError_t launch_mass_ref(cacl_ctx* c, const float* phi) {
  const int64_t N = c->g.N;
  const int nb = (int)((N + ELEM_THREADS * 8 - 1) / (ELEM_THREADS * 8));
  fluid_sum<<<nb, ELEM_THREADS, 0, c->stream>>>(phi, c->flags, N, c->partials);
  finalize_mass_ref<<<1, 32, 0, c->stream>>>(c->partials, nb, c->mass);
  return cudaGetLastError();
}

int mass_ref_blocks(int64_t N) {
  return (int)((N + ELEM_THREADS * 8 - 1) / (ELEM_THREADS * 8));
}

#define CACL_STORAGE_DISPATCH(c, KERNEL_CALL)                     \
  switch ((c)->p.storage) {                                       \
    case CACL_F16_SHIFTED: { using S = StoreF16; KERNEL_CALL; } break;  \
    case CACL_BF16_SHIFTED: { using S = StoreBF16; KERNEL_CALL; } break; \
    default: { using S = StoreF32; KERNEL_CALL; } break;          \
  }

cudaError_t launch_init_populations(cacl_ctx* c) {
  const int nb = elem_blocks(c->g.N);
  CACL_STORAGE_DISPATCH(c, (init_populations<S><<<nb, ELEM_THREADS, 0, c->stream>>>(
      (S::T*)c->f[0], (S::T*)c->f[1], c->u, c->flags, c->g.N)));
  return cudaGetLastError();
}

cudaError_t launch_pstar(cacl_ctx* c, const void* f, float* out) {
  const int nb = elem_blocks(c->g.N);
  CACL_STORAGE_DISPATCH(c, (pstar_kernel<S><<<nb, ELEM_THREADS, 0, c->stream>>>(
      (const S::T*)f, c->flags, c->g.N, out)));
  return cudaGetLastError();
}

cudaError_t launch_to_storage(cacl_ctx* c, const float* src, void* dst) {
  const int nb = elem_blocks(c->g.N);
  CACL_STORAGE_DISPATCH(c, (to_storage<S><<<nb, ELEM_THREADS, 0, c->stream>>>(
      src, (S::T*)dst, c->g.N)));
  return cudaGetLastError();
}

cudaError_t launch_from_storage(cacl_ctx* c, const void* src, float* dst) {
  const int nb = elem_blocks(c->g.N);
  CACL_STORAGE_DISPATCH(c, (from_storage<S><<<nb, ELEM_THREADS, 0, c->stream>>>(
      (const S::T*)src, dst, c->g.N)));
  return cudaGetLastError();
}

cudaError_t launch_check_finite(cacl_ctx* c, const float* phi, int* bad_dev) {
  finite_kernel<<<elem_blocks(c->g.N), ELEM_THREADS, 0, c->stream>>>(
      phi, c->u, c->flags, c->g.N, bad_dev);
  return cudaGetLastError();
}

}  // namespace cacl
