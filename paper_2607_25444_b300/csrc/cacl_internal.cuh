// cacl_internal.cuh -- shared device helpers and the context layout of the
// sm_103a CAC-LB wetting step.
//
// Lattice: D3Q27, direction q = 9(cz+1) + 3(cy+1) + (cx+1), rest q = 13,
// opposite direction 26 - q, weights 8/27, 2/27, 1/54, 1/216 by |c|^2
// (Sect. 2.1), c_s^2 = 1/3. Everything is derived from q at compile time.
#pragma once

#include <nvtx3/nvToolsExt.h>
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <string>

#include "../../include/cacl.h"

namespace cacl {

constexpr int Q = 27;
constexpr int REST = 13;

__host__ __device__ constexpr int cx(int q) { return q % 3 - 1; }
__host__ __device__ constexpr int cy(int q) { return (q / 3) % 3 - 1; }
__host__ __device__ constexpr int cz(int q) { return q / 9 - 1; }
__host__ __device__ constexpr int opp(int q) { return 26 - q; }
__host__ __device__ constexpr int csq(int q) {
  return cx(q) * cx(q) + cy(q) * cy(q) + cz(q) * cz(q);
}
__host__ __device__ constexpr float wq(int q) {
  return csq(q) == 0 ? 8.0f / 27.0f
       : csq(q) == 1 ? 2.0f / 27.0f
       : csq(q) == 2 ? 1.0f / 54.0f
                     : 1.0f / 216.0f;
}

// Population storage. FP32 stores f_i. The 16-bit forms store the
// weight-normalised deviation from the rest state, h_i = (f_i - w_i p*_ref)
// / w_i with p*_ref = 0 (the pressure gauge of the initial state), rounded
// to nearest even; 1/w_i is exact in FP32, so the scaling adds no rounding.
// All arithmetic stays FP32.
// Population storage: decode gives f_q, encode stores f_q, and encode_w
// stores the population w_q P given P = f_q / w_q.
struct StoreF32 {
  using T = float;
  using T2 = float2;  // two x-adjacent nodes
  __device__ __forceinline__ static float decode(T v, int q) { return v; }
  __device__ __forceinline__ static T encode(float v, int q) { return v; }
  __device__ __forceinline__ static T encode_w(float P, int q) { return wq(q) * P; }
  __device__ __forceinline__ static float2 decode2(T2 v, int q) { return v; }
  __device__ __forceinline__ static T2 encode_w2(float2 P, int q) {
    return __fmul2_rn(make_float2(wq(q), wq(q)), P);
  }
  __device__ __forceinline__ static T2 pack(T lo, T hi) { return make_float2(lo, hi); }
  __device__ __forceinline__ static T lo(T2 v) { return v.x; }
  __device__ __forceinline__ static T hi(T2 v) { return v.y; }
};

struct StoreF16 {
  using T = __half;
  using T2 = __half2;
  __device__ __forceinline__ static float decode(T v, int q) {
    return __fmul_rn(__half2float(v), wq(q));
  }
  __device__ __forceinline__ static T encode(float v, int q) {
    return __float2half_rn(v * (1.0f / wq(q)));
  }
  __device__ __forceinline__ static T encode_w(float P, int q) {
    return __float2half_rn(P);
  }
  __device__ __forceinline__ static float2 decode2(T2 v, int q) {
    const float2 h = __half22float2(v);
    return make_float2(__fmul_rn(h.x, wq(q)), __fmul_rn(h.y, wq(q)));
  }
  __device__ __forceinline__ static T2 encode_w2(float2 P, int q) {
    return __float22half2_rn(P);
  }
  // pair assembly on the bits (a byte permutation, a mask or a shift)
  __device__ __forceinline__ static uint32_t bits2(T2 v) {
    return *reinterpret_cast<const uint32_t*>(&v);
  }
  __device__ __forceinline__ static uint32_t bits1(T v) {
    return *reinterpret_cast<const uint16_t*>(&v);
  }
  __device__ __forceinline__ static T2 pack(T lo, T hi) {
    const uint32_t b = __byte_perm(bits1(lo), bits1(hi), 0x5410);
    return *reinterpret_cast<const T2*>(&b);
  }
  __device__ __forceinline__ static T lo(T2 v) {
    const uint16_t b = (uint16_t)(bits2(v) & 0xffffu);
    return *reinterpret_cast<const T*>(&b);
  }
  __device__ __forceinline__ static T hi(T2 v) {
    const uint16_t b = (uint16_t)(bits2(v) >> 16);
    return *reinterpret_cast<const T*>(&b);
  }
};

struct StoreBF16 {
  using T = __nv_bfloat16;
  using T2 = __nv_bfloat162;
  __device__ __forceinline__ static float decode(T v, int q) {
    return __fmul_rn(__bfloat162float(v), wq(q));
  }
  __device__ __forceinline__ static T encode(float v, int q) {
    return __float2bfloat16_rn(v * (1.0f / wq(q)));
  }
  __device__ __forceinline__ static T encode_w(float P, int q) {
    return __float2bfloat16_rn(P);
  }
  // a bf16 value is the upper half of the float it widens to: the pair
  // operations below work on the bits (exact, the same values as the
  // conversion intrinsics)
  __device__ __forceinline__ static uint32_t bits2(T2 v) {
    return *reinterpret_cast<const uint32_t*>(&v);
  }
  __device__ __forceinline__ static uint32_t bits1(T v) {
    return *reinterpret_cast<const uint16_t*>(&v);
  }
  __device__ __forceinline__ static float2 decode2(T2 v, int q) {
    const uint32_t b = bits2(v);
    return make_float2(__fmul_rn(__uint_as_float(b << 16), wq(q)),
                       __fmul_rn(__uint_as_float(b & 0xffff0000u), wq(q)));
  }
  __device__ __forceinline__ static T2 encode_w2(float2 P, int q) {
    return __float22bfloat162_rn(P);
  }
  __device__ __forceinline__ static T2 pack(T lo, T hi) {
    const uint32_t b = __byte_perm(bits1(lo), bits1(hi), 0x5410);
    return *reinterpret_cast<const T2*>(&b);
  }
  __device__ __forceinline__ static T lo(T2 v) {
    const uint16_t b = (uint16_t)(bits2(v) & 0xffffu);
    return *reinterpret_cast<const T*>(&b);
  }
  __device__ __forceinline__ static T hi(T2 v) {
    const uint16_t b = (uint16_t)(bits2(v) >> 16);
    return *reinterpret_cast<const T*>(&b);
  }
};

inline size_t storage_bytes(int storage) {
  return (storage == CACL_F32 || storage == CACL_F32_MOMENTS) ? 4 : 2;
}
// components per node of the population buffers: 27 populations, or the 17
// coefficients of the moment form
inline int pop_comps(int storage) { return storage == CACL_F32_MOMENTS ? 17 : 27; }

// Node flags (one byte per node).
constexpr uint8_t FLAG_SOLID = 1;  // node is solid
constexpr uint8_t FLAG_NEAR = 2;   // fluid node with a solid neighbour
constexpr uint8_t FLAG_WALL = 4;   // solid node that carries a ghost value

struct Grid {
  int nx, ny, nz;
  int64_t N;
};

// Wrapped neighbour coordinate along one axis (every axis wraps; closed axes
// have solid boundary layers, so a wrapped neighbour there is solid).
__device__ __forceinline__ int wrap(int i, int d, int n) {
  int j = i + d;
  j = (j < 0) ? j + n : j;
  return (j >= n) ? j - n : j;
}

// Arithmetic on one node (float) or on a pair of x-adjacent nodes (float2,
// the packed FP32 pair operations of sm_100 and later). Every operation is
// round-to-nearest, and a pair operation rounds each lane exactly as the
// scalar operation does, so a kernel that handles two nodes per thread
// gives the same bits as one that handles one. The scalar forms are never
// contracted; a packed product that feeds a packed sum directly is fused
// into one packed multiply-add by this toolchain (CUDA 13.0) even with
// explicit rounding (measured: __fadd2_rn(__fmul2_rn(a, b), c) equals
// fmaf lane by lane, and differs from the two rounded scalar operations in
// 14% of random lanes), so pair code keeps such a product apart from its sum
// (a select, or a use as an addend of vfma), and the pair kernels are
// checked bit for bit against the one-node kernels.
__device__ __forceinline__ float vfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) {
  return __ffma2_rn(a, b, c);
}
__device__ __forceinline__ float vmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float vadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float vneg(float a) { return -a; }
__device__ __forceinline__ float2 vneg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float vsub(float a, float b) { return __fadd_rn(a, -b); }
__device__ __forceinline__ float2 vsub(float2 a, float2 b) { return __fadd2_rn(a, vneg(b)); }
// 1 / a, correctly rounded, per lane
__device__ __forceinline__ float vrcp(float a) { return 1.0f / a; }
__device__ __forceinline__ float2 vrcp(float2 a) { return make_float2(1.0f / a.x, 1.0f / a.y); }
template <typename V> __device__ __forceinline__ V splat(float c);
template <> __device__ __forceinline__ float splat<float>(float c) { return c; }
template <> __device__ __forceinline__ float2 splat<float2>(float c) {
  return make_float2(c, c);
}

// One pair of opposite links (q, 26 - q) of the isotropic phi stencil (Eqs.
// grad_iso, lap_iso): phi at x + c_q (vp) and x - c_q (vm) added to the
// gradient and to sum_q w_q phi(x + c_q), in explicitly rounded operations.
template <typename V>
__device__ __forceinline__ void stencil_pair(int q, V vp, V vm, V& gx, V& gy, V& gz,
                                             V& ssum) {
  const V dv = vmul(splat<V>(3.0f * wq(q)), vadd(vp, vneg(vm)));
  if (cx(q) > 0) gx = vadd(gx, dv);
  if (cx(q) < 0) gx = vadd(gx, vneg(dv));
  if (cy(q) > 0) gy = vadd(gy, dv);
  if (cy(q) < 0) gy = vadd(gy, vneg(dv));
  if (cz(q) > 0) gz = vadd(gz, dv);
  if (cz(q) < 0) gz = vadd(gz, vneg(dv));
  ssum = vfma(splat<V>(wq(q)), vadd(vp, vm), ssum);
}

// Isotropic gradient (Eq. grad_iso) and the neighbour sum of Eq. lap_iso of
// phi at a node whose wrapped neighbour offsets are xo/yo/zo[0..2] (-1, 0,
// +1), summed over pairs of opposite links. lap = 6 (ssum - (1 - w_0) phi).
__device__ __forceinline__ void phi_stencil(const float* __restrict__ phi,
                                            const int (&xo)[3],
                                            const int (&yo)[3],
                                            const int64_t (&zo)[3], float& gx,
                                            float& gy, float& gz,
                                            float& ssum) {
  gx = 0.f;
  gy = 0.f;
  gz = 0.f;
  ssum = 0.f;
#pragma unroll
  for (int q = 0; q < REST; ++q) {
    const float vp = __ldg(phi + xo[1 + cx(q)] + yo[1 + cy(q)] + zo[1 + cz(q)]);
    const float vm = __ldg(phi + xo[1 - cx(q)] + yo[1 - cy(q)] + zo[1 - cz(q)]);
    stencil_pair(q, vp, vm, gx, gy, gz, ssum);
  }
}

// Compressive vector a = phi (1 - phi) grad phi / |grad phi| (Sect. 2.1.1),
// zero where |grad phi| < 1e-12.
__device__ __forceinline__ void compressive(float phi0, float gx, float gy,
                                            float gz, float& ax, float& ay,
                                            float& az) {
  const float g2 = fmaf(gz, gz, fmaf(gy, gy, __fmul_rn(gx, gx)));
  ax = ay = az = 0.f;
  if (g2 >= 1e-24f) {
    const float sc = __fmul_rn(__fmul_rn(phi0, __fadd_rn(1.0f, -phi0)), rsqrtf(g2));
    ax = __fmul_rn(sc, gx);
    ay = __fmul_rn(sc, gy);
    az = __fmul_rn(sc, gz);
  }
}

// The same for a pair of nodes, lane by lane.
__device__ __forceinline__ void compressive(float2 phi0, float2 gx, float2 gy,
                                            float2 gz, float2& ax, float2& ay,
                                            float2& az) {
  compressive(phi0.x, gx.x, gy.x, gz.x, ax.x, ay.x, az.x);
  compressive(phi0.y, gx.y, gy.y, gz.y, ax.y, ay.y, az.y);
}

// Scalar parameters uploaded once per context.
struct Consts {
  float rho_g, drho;      // rho = rho_g + drho * phi
  float mu_g, dmu;        // mu = mu_g + dmu * phi
  float beta4;            // 4 beta
  float kappa_phi;        // kappa_phi
  float gx, gy, gz;       // gravity
  float mobility;         // D
  float kappa;            // 4 D / delta
  float eps_phi;
};

// Reduction partials of the phase update: per block (sum phi*, sum chi) as
// doubles, plus the scalars formed from them.
struct MassScalars {
  double m_ref;
  double m_star;
  double w_sum;
  double lambda;
  float lambda_f;
  uint32_t step;  // corrections applied since set_fields (rounding key)
};

// phi + d rounded to FP32 without bias: the exact residual of the sum
// (Knuth's two-sum) decides, against a uniform number drawn from a
// counter-based hash of (step, node), whether to move one unit in the last
// place towards it, so the expected stored value is phi + d. A correction
// far below the resolution of phi is then applied on average instead of
// being rounded away every step.
__device__ __forceinline__ float add_unbiased(float s, float d, uint32_t step,
                                              uint64_t node) {
  // each operation rounded on its own (a product feeding d must not be
  // fused into the sum, or the residual is not that of fl(s + d))
  const float t = __fadd_rn(s, d);
  const float bb = __fsub_rn(t, s);
  const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bb)), __fsub_rn(d, bb));
  if (e == 0.f) return t;
  // splitmix64 finalizer of the key
  uint64_t z = ((uint64_t)step << 40) ^ node ^ 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  const float u = (float)(z >> 40) * (1.0f / 16777216.0f);
  const float nb = nextafterf(t, e > 0.f ? INFINITY : -INFINITY);
  return (u * fabsf(nb - t) < fabsf(e)) ? nb : t;
}

// Fixed-order sum of nb doubles by one warp: lane l adds src[l], src[l+32],
// ... in turn, then the lanes combine pairwise (offsets 16, 8, 4, 2, 1).
// The loads go through L2 (ld.global.cg): the values may have been written
// by other blocks of the same launch. The result is valid in lane 0.
__device__ __forceinline__ double warp_sum_fixed(const double* src, int nb,
                                                 int lane) {
  double s = 0.0;
#pragma unroll 8
  for (int i = lane; i < nb; i += 32) s += __ldcg(src + i);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  return s;
}

// lambda = (M_ref - M*) / W of the volume correction (Eq.
// mass_correction_normalization; 0 when W = 0) from the per-block partial
// sums of the phi update (nb phi* sums, then nb chi sums), by warp 0 of the
// calling block; the correction counter advances by one.
__device__ __forceinline__ void mass_from_partials(const double* partials,
                                                   int nb, MassScalars* ms,
                                                   int lane) {
  const double m = warp_sum_fixed(partials, nb, lane);
  const double w = warp_sum_fixed(partials + nb, nb, lane);
  if (lane == 0) {
    const double lam = (w > 0.0) ? (ms->m_ref - m) / w : 0.0;
    ms->m_star = m;
    ms->w_sum = w;
    ms->lambda = lam;
    ms->lambda_f = (float)lam;
    ms->step += 1;
  }
}

// One case of a batch as the batched kernels see it: grid, constants and
// the device buffers of the case's own context.
struct CaseDesc {
  Grid g;
  Consts k;
  void* f[2];
  float* phi[2];
  float* u;
  float* a;
  uint8_t* flags;
  int W;
  int32_t* w_idx;
  int32_t* w_donor;
  int8_t* w_q;
  float* w_nw;
  float* w_cot;
  float* w_g;
  double* partials;
  MassScalars* mass;
  int phase_nb;  // phase-update blocks of this case for the batch's tile
  int lbw;       // nodes per thread of the batched collide-stream (1, 2, 4)
};

// Virtual block b of a work-list belongs to case c when
// start[c] <= b < start[c + 1]; every thread of a block finds the same c.
__device__ __forceinline__ int find_case(const int* __restrict__ start,
                                         int ncases, int b) {
  int lo = 0, hi = ncases - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(start + mid) <= b)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// Work-list of one batched stage: per-case starts of its virtual blocks.
struct WorkList {
  const int* start;  // device, ncases + 1
  int ncases;
  int total;
};

// A persistent block of a batched stage walks the virtual blocks of the
// work-list in increasing order (a contiguous range [b0, b1), or every
// gridDim.x-th block); the descriptor of the current case sits in shared
// memory and is refreshed only when the walk crosses into a later case.
// Every thread of the block must call seek() (it synchronises).
struct CaseCursor {
  CaseDesc d;
  int c, cstart, cend;

  __device__ __forceinline__ void begin() { cend = -1; }
  // make the case of virtual block b current
  __device__ __forceinline__ void seek(const CaseDesc* __restrict__ cases,
                                       const WorkList& wl, int b) {
    if (b < cend) return;  // uniform across the block: cend is shared
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      c = find_case(wl.start, wl.ncases, b);
      cstart = __ldg(wl.start + c);
      cend = __ldg(wl.start + c + 1);
      d = cases[c];
    }
    __syncthreads();
  }
};

__device__ __forceinline__ void block_range(const WorkList& wl, int& b0,
                                            int& b1) {
  const int per = (wl.total + (int)gridDim.x - 1) / (int)gridDim.x;
  b0 = min((int)blockIdx.x * per, wl.total);
  b1 = min(b0 + per, wl.total);
}

}  // namespace cacl

struct AdjointState;

struct cacl_ctx {
  cacl_params p;
  cacl::Grid g;
  cacl::Consts k;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string err;
  bool has_geometry = false;
  bool has_fields = false;
  int geom_version = 0;  // bumped by every cacl_set_geometry

  // device state
  void* f[2] = {nullptr, nullptr};     // populations, [q][n], ping-pong,
                                        // in the storage type of p.storage
  float* phi[2] = {nullptr, nullptr};  // phi^n (with ghosts) and phi*
  float* u = nullptr;                  // [3][n]
  float* a = nullptr;                  // [3][n] compressive vector of phi^n
  uint8_t* flags = nullptr;
  int fcur = 0;                         // buffer holding the current f*
  int pcur = 0;                         // buffer holding the current phi

  // wall list
  int32_t wall_count = 0;
  int32_t* w_idx = nullptr;
  int32_t* w_donor = nullptr;
  int8_t* w_q = nullptr;
  int16_t* w_n6 = nullptr;  // [3][W]
  float* w_nw = nullptr;    // [3][W]
  float* w_cot = nullptr;   // cot(theta_c)
  float* w_theta = nullptr; // theta in degrees
  float* w_g = nullptr;     // ghost scratch

  // kernel shape choices (cacl_set_option)
  int phase_variant = 2;
  int phase_pipe = 0;      // 0 auto, 1 register staging, 2 cp.async staging
  int lb_pipe = 0;         // 0 two nodes per thread (else one), 1 bulk-copy
                           // staged rows, 2 one node per thread, 3 TMA-tiled
                           // (else two nodes per thread)
  int lb_grid = 1;         // blocks of the persistent staged collide-stream
  bool index64 = false;    // 64-bit offsets in every kernel that has both
                           // widths, whatever the size (CACL_OPT_INDEX64)
  // tensor maps of the TMA-tiled collide-stream (nx a multiple of 8):
  // population loads and stores per buffer, phi loads per buffer, u and a
  // stores; valid when lbt_ok
  bool lbt_ok = false;
  CUtensorMap lbt_fload[2], lbt_fstore[2], lbt_phi[2], lbt_u, lbt_a;
  int phase_nblocks = 0;   // blocks of the last phase-update launch

  // z slab of a decomposition (cacl_slab_create): the phi update covers
  // planes [zbase, zlim) (zlim 0 = every plane), lambda is formed from
  // gathered partials instead of by the phi update's last block, and the
  // rounding key of the correction uses global node indices (node_offset
  // added to the local index)
  int zbase = 0, zlim = 0;
  bool ext_finalize = false;
  int64_t node_offset = 0;
  int slab_z0 = 0, slab_nz = 0;  // first global plane and interior planes

  // reductions
  int part_blocks = 0;
  double* partials = nullptr;  // [2][part_blocks]
  cacl::MassScalars* mass = nullptr;
  int* scan_scratch = nullptr;
  int scan_blocks = 0;

  // one-step graphs, indexed by (fcur, pcur)
  cudaGraphExec_t graph[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  int* bad_flag = nullptr;  // device word for cacl_check_finite
  // [0] phase-update blocks done (the last one finalises), [1] set when a
  // bounded wait for asynchronous copies gave up, [2] test request that
  // makes the first copy waits of the staged and TMA-tiled collide-stream
  // run out
  unsigned* ticket = nullptr;
  AdjointState* adj = nullptr;  // checkpoints, tape and adjoint fields
  int64_t device_bytes = 0;
};

// Kernel launchers (defined in the .cu files). All enqueue on c->stream.
namespace cacl {
// An NVTX range around a host call: a profiler's timeline shows the step,
// batch step and adjoint calls by name.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

cudaError_t launch_geometry(cacl_ctx* c, const uint8_t* solid_dev);
cudaError_t launch_ghost(cacl_ctx* c, float* phi);
cudaError_t lb_init(cacl_ctx* c);
bool lb_staged_ok(const cacl_ctx* c, const void* fin, const void* fout,
                  const void* phi);
bool lb_pair_ok(const cacl_ctx* c, const void* fin, const void* fout,
                const void* phi);
bool lb_quad_ok(const cacl_ctx* c, const void* fin, const void* fout,
                const void* phi);
cudaError_t lb_tma_init(cacl_ctx* c);
bool lb_tma_ok(const cacl_ctx* c, const void* fin, const void* fout,
               const void* phi);
cudaError_t launch_lb(cacl_ctx* c, const void* fin, void* fout,
                      const float* phi);
cudaError_t launch_compressive(cacl_ctx* c, const float* phi);
cudaError_t phase_init_attributes();
cudaError_t launch_phase(cacl_ctx* c, const float* phi_in, float* phi_out);
cudaError_t launch_correct(cacl_ctx* c, float* phi);
// the correction right after launch_phase over the whole context (tiles
// without interface-band nodes skipped)
cudaError_t launch_correct_tiles(cacl_ctx* c, float* phi);
cudaError_t launch_mass_from(cacl_ctx* c, const double* partials, int nb);
cudaError_t launch_mass_ref(cacl_ctx* c, const float* phi);
cudaError_t launch_init_populations(cacl_ctx* c);
cudaError_t launch_moments_init(cacl_ctx* c);
cudaError_t launch_moments_expand(cacl_ctx* c, const void* C, float* f, float* pstar);
cudaError_t launch_pstar(cacl_ctx* c, const void* f, float* out);
cudaError_t launch_to_storage(cacl_ctx* c, const float* src, void* dst);
cudaError_t launch_from_storage(cacl_ctx* c, const void* src, float* dst);
cudaError_t launch_check_finite(cacl_ctx* c, const float* phi, int* bad_dev);
int phase_blocks(const cacl_ctx* c);
int phase_default_variant(const Grid& g);
int mass_ref_blocks(int64_t N);
void adjoint_free(AdjointState* s);

// Batched stages: one grid-strided launch runs the stage for every case of
// a work-list; fc / pc select each case's current population / phi buffer.
// collide-stream blocks of 64, 128, 256 threads, persistent (variants 0-2)
// or one block per work item (3-5); one launch per node width (1, 2, 4
// nodes per thread) over the cases of that width
constexpr int LB_BATCH_VARIANTS = 6;
int lb_batch_row(int variant);
bool lb_batch_persistent(int variant);
cudaError_t launch_lb_batch(const CaseDesc* cases, WorkList wl, int storage, int width,
                            int variant, int grid, int fc, int pc,
                            cudaStream_t st);
int lb_batch_occupancy(int storage, int width, int variant);
cudaError_t launch_ghost_batch(const CaseDesc* cases, WorkList wl, int grid,
                               int pc, cudaStream_t st);
int ghost_batch_block();
cudaError_t launch_phase_batch(const CaseDesc* cases, WorkList wl, int variant,
                               int grid, int pc, cudaStream_t st);
int phase_batch_occupancy(int variant);
// the same over cases that qualify for copy staging (phase_copy_ok): two
// nodes per thread along y (phase pipeline 2) or 2 x 2 (0 and 3)
cudaError_t launch_phase_batch_copy(const CaseDesc* cases, WorkList wl, int variant,
                                    int grid, int pc, bool aligned, cudaStream_t st);
int phase_batch_copy_occupancy(int variant, bool aligned);
cudaError_t launch_phase_batch_quad(const CaseDesc* cases, WorkList wl, int variant,
                                    int grid, int pc, cudaStream_t st);
int phase_batch_quad_occupancy(int variant);
bool phase_copy_ok(const Grid& g, const void* phi_in, const void* phi_out,
                   const void* a, const void* u, const void* flags);
void phase_tile(int variant, int& ty, int& zc);
cudaError_t launch_correct_batch(const CaseDesc* cases, int ncases, WorkList wl,
                                 int grid, int pc, cudaStream_t st);
int correct_batch_nodes();
}  // namespace cacl
