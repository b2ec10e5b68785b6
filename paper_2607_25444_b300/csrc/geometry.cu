// geometry.cu -- node flags and the wall list (Sect. 2.2,
// Eqs. local_wall_normal, wall_normal_weights, unit_wall_normal,
// donor_alignment_score, donor_selection, donor_to_solid).
//
// Once per geometry. Three launches: classify (flags + per-block wall
// counts), an exclusive scan of the counts, emit (wall entries in node
// order). All comparisons of the donor scores are exact integer arithmetic;
// the unit normal is the FP32 value n~6_k / sqrt(|n~6|^2) with correctly
// rounded division and square root.
#include "cacl_internal.cuh"

namespace cacl {
namespace {

constexpr int GEOM_THREADS = 256;

struct WallGeom {
  int n6[3];
  bool any_fluid;
  int qstar;
};

__device__ __forceinline__ bool solid_at(const uint8_t* solid, const Grid& g,
                                         int x, int y, int z) {
  return solid[(int64_t)x + (int64_t)g.nx * (y + (int64_t)g.ny * z)] != 0;
}

// Integer normal (6 w_q weights: 6, 3, 2) and exact donor argmax for the
// solid node at (x, y, z).
__device__ WallGeom wall_geometry(const uint8_t* solid, const Grid& g, int x,
                                  int y, int z) {
  WallGeom r;
  r.n6[0] = r.n6[1] = r.n6[2] = 0;
  r.any_fluid = false;
  r.qstar = -1;
  bool fluid[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    fluid[q] = false;
    if (q == REST) continue;
    const bool s = solid_at(solid, g, wrap(x, cx(q), g.nx), wrap(y, cy(q), g.ny),
                            wrap(z, cz(q), g.nz));
    if (!s) {
      fluid[q] = true;
      r.any_fluid = true;
      const int m = 6 / csq(q);
      r.n6[0] -= m * cx(q);
      r.n6[1] -= m * cy(q);
      r.n6[2] -= m * cz(q);
    }
  }
  if (!r.any_fluid) return r;
  // score a_q / sqrt(m_q) with a_q = -c_q . n~6, m_q = |c_q|^2
  long long ba = 0, bm = 1;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    if (!fluid[q]) continue;
    const long long a = -(long long)(cx(q) * r.n6[0] + cy(q) * r.n6[1] +
                                     cz(q) * r.n6[2]);
    const long long m = csq(q);
    bool better;
    if (r.qstar < 0) {
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
      r.qstar = q;
      ba = a;
      bm = m;
    }
  }
  return r;
}

__device__ __forceinline__ void coords(int64_t n, const Grid& g, int& x, int& y,
                                       int& z) {
  x = (int)(n % g.nx);
  const int64_t r = n / g.nx;
  y = (int)(r % g.ny);
  z = (int)(r / g.ny);
}

__global__ void __launch_bounds__(GEOM_THREADS)
geom_classify(const uint8_t* __restrict__ solid, uint8_t* __restrict__ flags,
              int* __restrict__ block_counts, Grid g) {
  const int64_t n = (int64_t)blockIdx.x * GEOM_THREADS + threadIdx.x;
  int wall = 0;
  if (n < g.N) {
    int x, y, z;
    coords(n, g, x, y, z);
    uint8_t fl = 0;
    if (solid[n]) {
      fl = FLAG_SOLID;
      const WallGeom w = wall_geometry(solid, g, x, y, z);
      if (w.any_fluid && (w.n6[0] | w.n6[1] | w.n6[2]) != 0) {
        fl |= FLAG_WALL;
        wall = 1;
      }
    } else {
      bool near = false;
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        if (q == REST) continue;
        near |= solid_at(solid, g, wrap(x, cx(q), g.nx), wrap(y, cy(q), g.ny),
                         wrap(z, cz(q), g.nz));
      }
      if (near) fl = FLAG_NEAR;
    }
    flags[n] = fl;
  }
  const int cnt = __syncthreads_count(wall);
  if (threadIdx.x == 0) block_counts[blockIdx.x] = cnt;
}

// Exclusive scan of nb counts in one block of 1024 threads: each thread sums
// a contiguous chunk, the chunk totals are scanned in shared memory, then
// each thread writes its chunk's offsets. counts[nb] receives the total.
__global__ void __launch_bounds__(1024) scan_counts(int* counts, int nb) {
  __shared__ int part[1024];
  const int t = threadIdx.x;
  const int chunk = (nb + 1023) / 1024;
  const int lo = min(t * chunk, nb), hi = min(lo + chunk, nb);
  int s = 0;
  for (int i = lo; i < hi; ++i) s += counts[i];
  part[t] = s;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    const int v = (t >= off) ? part[t - off] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  int run = part[t] - s;  // exclusive prefix of this chunk
  for (int i = lo; i < hi; ++i) {
    const int c = counts[i];
    counts[i] = run;
    run += c;
  }
  if (t == 1023) counts[nb] = part[1023];
}

__global__ void __launch_bounds__(GEOM_THREADS)
geom_emit(const uint8_t* __restrict__ solid, const uint8_t* __restrict__ flags,
          const int* __restrict__ offsets, Grid g, int32_t* __restrict__ w_idx,
          int32_t* __restrict__ w_donor, int8_t* __restrict__ w_q,
          int16_t* __restrict__ w_n6, float* __restrict__ w_nw, int W) {
  __shared__ int warp_tot[GEOM_THREADS / 32];
  const int64_t n = (int64_t)blockIdx.x * GEOM_THREADS + threadIdx.x;
  const bool wall = (n < g.N) && (flags[n] & FLAG_WALL);
  const unsigned ball = __ballot_sync(0xffffffffu, wall);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) warp_tot[warp] = __popc(ball);
  __syncthreads();
  int base = offsets[blockIdx.x];
  for (int i = 0; i < warp; ++i) base += warp_tot[i];
  if (!wall) return;
  const int slot = base + __popc(ball & ((1u << lane) - 1u));
  int x, y, z;
  coords(n, g, x, y, z);
  const WallGeom w = wall_geometry(solid, g, x, y, z);
  const int q = w.qstar;
  const int dx = wrap(x, cx(q), g.nx), dy = wrap(y, cy(q), g.ny),
            dz = wrap(z, cz(q), g.nz);
  w_idx[slot] = (int32_t)n;
  w_donor[slot] = (int32_t)(dx + (int64_t)g.nx * (dy + (int64_t)g.ny * dz));
  w_q[slot] = (int8_t)q;
  const int nn = w.n6[0] * w.n6[0] + w.n6[1] * w.n6[1] + w.n6[2] * w.n6[2];
  const float inv = __fsqrt_rn((float)nn);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    w_n6[a * W + slot] = (int16_t)w.n6[a];
    w_nw[a * W + slot] = __fdiv_rn((float)w.n6[a], inv);
  }
}

}  // namespace

// Builds flags and the wall list from a device copy of the occupancy.
// Allocates the wall arrays (sized after the count is known). Synchronises.
cudaError_t launch_geometry(cacl_ctx* c, const uint8_t* solid_dev) {
  const Grid g = c->g;
  const int nb = (int)((g.N + GEOM_THREADS - 1) / GEOM_THREADS);
  cudaError_t e;
  if (c->scan_blocks < nb + 1) {
    if (c->scan_scratch) cudaFree(c->scan_scratch);
    c->scan_scratch = nullptr;
    c->scan_blocks = 0;
    e = cudaMalloc(&c->scan_scratch, sizeof(int) * (nb + 1));
    if (e != cudaSuccess) return e;
    c->scan_blocks = nb + 1;
  }
  geom_classify<<<nb, GEOM_THREADS, 0, c->stream>>>(solid_dev, c->flags,
                                                     c->scan_scratch, g);
  scan_counts<<<1, 1024, 0, c->stream>>>(c->scan_scratch, nb);
  int W = 0;
  e = cudaMemcpyAsync(&W, c->scan_scratch + nb, sizeof(int),
                      cudaMemcpyDeviceToHost, c->stream);
  if (e != cudaSuccess) return e;
  e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return e;

  void** bufs[] = {(void**)&c->w_idx, (void**)&c->w_donor, (void**)&c->w_q,
                   (void**)&c->w_n6, (void**)&c->w_nw, (void**)&c->w_cot,
                   (void**)&c->w_theta, (void**)&c->w_g};
  for (void** b : bufs) {
    if (*b) cudaFree(*b);
    *b = nullptr;
  }
  c->wall_count = W;
  const size_t Wa = (size_t)(W > 0 ? W : 1);
  const size_t sizes[] = {4 * Wa, 4 * Wa, Wa, 2 * 3 * Wa, 4 * 3 * Wa,
                          4 * Wa, 4 * Wa, 4 * Wa};
  for (int i = 0; i < 8; ++i) {
    e = cudaMalloc(bufs[i], sizes[i]);
    if (e != cudaSuccess) return e;
  }
  geom_emit<<<nb, GEOM_THREADS, 0, c->stream>>>(
      solid_dev, c->flags, c->scan_scratch, g, c->w_idx, c->w_donor, c->w_q,
      c->w_n6, c->w_nw, W);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(c->stream);
}

}  // namespace cacl
