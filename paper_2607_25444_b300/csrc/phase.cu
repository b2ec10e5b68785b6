// phase.cu -- conservative Allen-Cahn update of phi at fluid nodes
// (Sect. 2.1.1: Eqs. phi_update_muscl, divF, face_flux_def, slope_minmod_x,
// minmod, recon_lr_x, upwind_select_x, source_sharp; Eq. lap_iso), plus the
// per-block partial sums of the volume correction (Sect. 2.3,
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
#include <type_traits>

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

// two independent compensated sums, one per lane of an x pair, advanced in
// packed pair operations (each lane as df_add)
struct DF2 {
  float2 hi, lo;
};

__device__ __forceinline__ void df2_add(DF2& s, float2 x) {
  const float2 t = vadd(s.hi, x);
  const float2 bb = vsub(t, s.hi);
  const float2 err = vadd(vsub(s.hi, vsub(t, bb)), vsub(x, bb));
  s.hi = t;
  s.lo = vadd(s.lo, err);
}
__device__ __forceinline__ DF lane_x(const DF2& s) { return {s.hi.x, s.lo.x}; }
__device__ __forceinline__ DF lane_y(const DF2& s) { return {s.hi.y, s.lo.y}; }

__device__ __forceinline__ DF df_shfl_down(DF v, int off) {
  DF r;
  r.hi = __shfl_down_sync(0xffffffffu, v.hi, off);
  r.lo = __shfl_down_sync(0xffffffffu, v.lo, off);
  return r;
}

// minmod(a, b) = 0 if a b <= 0, else sign(a) min(|a|, |b|) (Eq. minmod),
// which is the median of a, b and 0, evaluated as
// max(min(a, b), min(a, 0), min(b, 0)): for a, b > 0 it gives min(a, b),
// for a, b < 0 max(a, b), and 0 for opposite signs or a zero. min(d, 0) of
// a difference can serve both slopes next to it (minmod_m). Every step is
// exact, so any evaluation order gives the same bits.
__device__ __forceinline__ float max3(float a, float b, float c) {
  float r;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}
__device__ __forceinline__ float neg_part(float d) { return fminf(d, 0.f); }
// minmod from the differences and their neg_part
__device__ __forceinline__ float minmod_m(float a, float b, float ma, float mb) {
  return max3(fminf(a, b), ma, mb);
}
__device__ __forceinline__ float minmod(float a, float b) {
  return minmod_m(a, b, neg_part(a), neg_part(b));
}
__device__ __forceinline__ float2 minmod(float2 a, float2 b) {
  return make_float2(minmod(a.x, b.x), minmod(a.y, b.y));
}
__device__ __forceinline__ float2 neg_part(float2 d) {
  return make_float2(neg_part(d.x), neg_part(d.y));
}
__device__ __forceinline__ float2 minmod_m(float2 a, float2 b, float2 ma, float2 mb) {
  return make_float2(minmod_m(a.x, b.x, ma.x, mb.x), minmod_m(a.y, b.y, ma.y, mb.y));
}

__device__ __forceinline__ int mod(int i, int n) {
  const int r = i % n;
  return r < 0 ? r + n : r;
}

// i wrapped into [0, n) for i in [-n, 2n)
__device__ __forceinline__ int wrap1(int i, int n) {
  return i < 0 ? i + n : (i >= n ? i - n : i);
}

// The arithmetic of a node, shared by every phi-update kernel. Each
// operation rounds once, in the order written (vfma, vmul, vadd, vsub leave
// no contraction to the compiler), so kernels that evaluate one node or a
// packed pair of nodes at a time give the same bits at every node.

// upwind state: pl where uf >= 0, else pr (per lane)
__device__ __forceinline__ float upwind(float uf, float pl, float pr) {
  return uf >= 0.f ? pl : pr;
}
__device__ __forceinline__ float2 upwind(float2 uf, float2 pl, float2 pr) {
  return make_float2(uf.x >= 0.f ? pl.x : pr.x, uf.y >= 0.f ? pl.y : pr.y);
}

// Upwind flux u_f phi_f through the face between cells l and r (Eqs.
// face_flux_def, recon_lr_x, upwind_select_x): u_f = (u_l + u_r) / 2, and
// phi_f the left state phi_l + s_l / 2 when u_f >= 0, else the right state
// phi_r - s_r / 2 (s the minmod slopes).
template <typename V>
__device__ __forceinline__ V face_flux(V ul, V ur, V vl, V sl, V vr, V sr) {
  const V uf = vmul(splat<V>(0.5f), vadd(ul, ur));
  return vmul(uf, upwind(uf, vfma(splat<V>(0.5f), sl, vl), vfma(splat<V>(-0.5f), sr, vr)));
}

// a + 4 b + c, the three-point sum of the factored D3Q27 weights (times 6)
template <typename V>
__device__ __forceinline__ V sum141(V a, V b, V c) {
  return vadd(a, vfma(splat<V>(4.f), b, c));
}

// In-plane partial stencils of one output node (times 36 undone):
// H = Dd_x S_y a_x + S_x Dd_y a_y from S_y a_x at x + 1 and x - 1 and Dd_y
// a_y (times 6) at x - 1, x, x + 1; V or L = S_y of the S_x row sums.
template <typename V>
__device__ __forceinline__ V partial_h(V sxp, V sxm, V d0, V d1, V d2) {
  return vmul(splat<V>(1.0f / 36.0f),
              vadd(vadd(vsub(sxp, sxm), d0), vfma(splat<V>(4.f), d1, d2)));
}
template <typename V>
__device__ __forceinline__ V partial_s(V r0, V r1, V r2) {
  return vmul(splat<V>(1.0f / 36.0f), sum141(r0, r1, r2));
}

// Eq. phi_update_muscl with the isotropic diffusion and the compressive
// term: phi* = phi - div F + D lap phi - kappa div_iso a, with
// lap = 6 (S_z L - phi) and div_iso a = 3 S_z H + 3 Dd_z V written through
// the carried partials of planes kz-1 .. kz+1.
template <typename V>
__device__ __forceinline__ V node_update(V v0, V div, V l0, V l1, V l2, V h0, V h1,
                                         V h2, V vv0, V vv2, const Consts& k) {
  const V lap = vfma(splat<V>(-6.f), v0, sum141(l0, l1, l2));
  const V diva = vmul(splat<V>(0.5f), vsub(vadd(sum141(h0, h1, h2), vv2), vv0));
  return vfma(splat<V>(-k.kappa), diva, vfma(splat<V>(k.mobility), lap, vsub(v0, div)));
}

// chi(phi*) = phi* (1 - phi*) inside the band eps < phi* < 1 - eps (Eq.
// mass_correction_normalization), else 0
__device__ __forceinline__ float band_chi(float vs, const Consts& k) {
  return (vs > k.eps_phi && vs < 1.0f - k.eps_phi) ? __fmul_rn(vs, __fadd_rn(1.0f, -vs))
                                                     : 0.f;
}

// Net advective flux difference along one axis (Eqs. divF .. upwind_select):
// values at -2..+2 along the axis, solid flags at -1/+1, cell velocities at
// -1, 0, +1. Faces touching a solid carry no flux.
__device__ __forceinline__ float muscl_axis(float vm2, float vm1, float v0,
                                            float vp1, float vp2, bool solm,
                                            bool solp, float um, float uc,
                                            float up) {
  const float sm = minmod(vsub(vm1, vm2), vsub(v0, vm1));
  const float s0 = minmod(vsub(v0, vm1), vsub(vp1, v0));
  const float sp = minmod(vsub(vp1, v0), vsub(vp2, vp1));
  const float fp = face_flux(uc, up, v0, s0, vp1, sp);
  const float fm = face_flux(um, uc, vm1, sm, v0, s0);
  return vsub(solp ? 0.f : fp, solm ? 0.f : fm);
}

// Registers a thread carries up its pair of columns (output rows a and b)
// from plane to plane, at output plane kz: phi at kz..kz+2, solid flags at
// kz-1..kz+1, the z velocity at kz and kz+1, the z slope at kz+1 and the z
// face fluxes at kz-1/2 and kz+1/2 (each face and slope is formed once, by
// the plane below it, and is the same number the node-wise Eq. divF uses
// from either side), the in-plane partial stencils of planes kz-1..kz+1
//   H = Dd_x S_y a_x + S_x Dd_y a_y, V = S_x S_y a_z, L = S_x S_y phi,
// and the two partial sums.
struct March {
  float ca[3], cb[3];
  bool sa3[3], sb3[3];
  float Ha[3], Hb[3], Va[3], Vb[3], La[3], Lb[3];
  float uza[2], uzb[2];
  float sza, szb;               // z slope at kz + 1
  float fzma, fzmb, fzpa, fzpb;  // z fluxes at kz - 1/2 and kz + 1/2
  DF msum, wsum;
};

__device__ __forceinline__ void march_init(March& m) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    m.ca[i] = m.cb[i] = 0.f;
    m.sa3[i] = m.sb3[i] = false;
    m.Ha[i] = m.Hb[i] = m.Va[i] = m.Vb[i] = m.La[i] = m.Lb[i] = 0.f;
  }
  m.uza[0] = m.uza[1] = m.uzb[0] = m.uzb[1] = 0.f;
  m.sza = m.szb = 0.f;
  m.fzma = m.fzmb = m.fzpa = m.fzpb = 0.f;
  m.msum = {0.f, 0.f};
  m.wsum = {0.f, 0.f};
}

// Advance the carried registers by one plane: the in-plane partials of plane
// kz + 1 (phi plane P1 with row pitch PP, a planes with row pitch AP; cp and
// ca index row a of the thread), the own columns' phi at kz + 2 (P2), solid
// flags at kz + 1 (S1), then the z slope at kz + 1 and the z flux at
// kz + 1/2 (m.uz* must hold u_z at kz and kz + 1).
template <int PP, int AP>
__device__ __forceinline__ void march_roll(March& m, const float* P1,
                                           const float* P2, const uint8_t* S1,
                                           const float* axp, const float* ayp,
                                           const float* azp, int cp, int ca) {
  float xm_[4], xp_[4], ym_[4][3], zz[4][3], pp[4][3];
#pragma unroll
  for (int r = 0; r < 4; ++r) {  // a-plane rows y-1 .. y+2 of the pair
    const int o = ca + (r - 1) * AP;
    xm_[r] = axp[o - 1];
    xp_[r] = axp[o + 1];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      ym_[r][d] = ayp[o + d - 1];
      zz[r][d] = azp[o + d - 1];
      pp[r][d] = P1[cp + (r - 1) * PP + d - 1];
    }
  }
  float H2[2], V2[2], L2[2];
#pragma unroll
  for (int j = 0; j < 2; ++j) {  // output row j uses rows j .. j+2
    const float sxp = sum141(xp_[j], xp_[j + 1], xp_[j + 2]);
    const float sxm = sum141(xm_[j], xm_[j + 1], xm_[j + 2]);
    const float d0 = vsub(ym_[j + 2][0], ym_[j][0]);
    const float d1 = vsub(ym_[j + 2][1], ym_[j][1]);
    const float d2 = vsub(ym_[j + 2][2], ym_[j][2]);
    H2[j] = partial_h(sxp, sxm, d0, d1, d2);
    float rz[3], rl[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      rz[r] = sum141(zz[j + r][0], zz[j + r][1], zz[j + r][2]);
      rl[r] = sum141(pp[j + r][0], pp[j + r][1], pp[j + r][2]);
    }
    V2[j] = partial_s(rz[0], rz[1], rz[2]);
    L2[j] = partial_s(rl[0], rl[1], rl[2]);
  }
  m.Ha[0] = m.Ha[1]; m.Ha[1] = m.Ha[2]; m.Ha[2] = H2[0];
  m.Hb[0] = m.Hb[1]; m.Hb[1] = m.Hb[2]; m.Hb[2] = H2[1];
  m.Va[0] = m.Va[1]; m.Va[1] = m.Va[2]; m.Va[2] = V2[0];
  m.Vb[0] = m.Vb[1]; m.Vb[1] = m.Vb[2]; m.Vb[2] = V2[1];
  m.La[0] = m.La[1]; m.La[1] = m.La[2]; m.La[2] = L2[0];
  m.Lb[0] = m.Lb[1]; m.Lb[1] = m.Lb[2]; m.Lb[2] = L2[1];
  m.ca[0] = m.ca[1]; m.ca[1] = m.ca[2]; m.ca[2] = P2[cp];
  m.cb[0] = m.cb[1]; m.cb[1] = m.cb[2]; m.cb[2] = P2[cp + PP];
  m.sa3[0] = m.sa3[1]; m.sa3[1] = m.sa3[2]; m.sa3[2] = (S1[cp] & FLAG_SOLID) != 0;
  m.sb3[0] = m.sb3[1]; m.sb3[1] = m.sb3[2]; m.sb3[2] = (S1[cp + PP] & FLAG_SOLID) != 0;
  // z slope at kz + 1 and z flux at kz + 1/2, from the slope at kz
  const float sa1 = minmod(vsub(m.ca[1], m.ca[0]), vsub(m.ca[2], m.ca[1]));
  const float sb1 = minmod(vsub(m.cb[1], m.cb[0]), vsub(m.cb[2], m.cb[1]));
  m.fzma = m.fzpa;
  m.fzmb = m.fzpb;
  m.fzpa = face_flux(m.uza[0], m.uza[1], m.ca[0], m.sza, m.ca[1], sa1);
  m.fzpb = face_flux(m.uzb[0], m.uzb[1], m.cb[0], m.szb, m.cb[1], sb1);
  m.sza = sa1;
  m.szb = sb1;
}

// Rest of one output node: Eq. phi_update_muscl with the isotropic
// diffusion and the compressive term, written to *out, and its contribution
// to the partial sums (Eqs. tentative_phase_field_mass,
// mass_correction_normalization). c indexes the node in P0 / S0; dy and dz
// are the (masked) y and z flux differences, u* the x velocities at -1, 0,
// +1, h* / vv* / l* the in-plane partials of planes kz-1..kz+1.
__device__ __forceinline__ void march_node(
    DF& msum, DF& wsum, const float* P0, const uint8_t* S0, int c, float v0,
    bool solc, float dy, float dz, float ux0, float ux1, float ux2, float h0,
    float h1, float h2, float vv0, float vv2, float l0, float l1, float l2,
    float* out, const Consts& k) {
  if (solc) {
    *out = v0;
    return;
  }
  const float dx = muscl_axis(P0[c - 2], P0[c - 1], v0, P0[c + 1], P0[c + 2],
                              (S0[c - 1] & FLAG_SOLID) != 0,
                              (S0[c + 1] & FLAG_SOLID) != 0, ux0, ux1, ux2);
  const float vs = node_update(v0, vadd(vadd(dx, dy), dz), l0, l1, l2, h0, h1, h2,
                               vv0, vv2, k);
  *out = vs;
  df_add(msum, vs);
  df_add(wsum, band_chi(vs, k));
}

// Both output nodes of the pair at plane kz: P0 / S0 hold phi and the flags
// of plane kz (row pitch PP), ux* / uy4 the in-plane velocities (x
// component at x-1, x, x+1 of rows a and b; y component at rows ya-1, ya,
// yb, yb+1), outa / outb the destinations. The y faces ya-1/2, ya+1/2 and
// yb+1/2 are formed once for the pair.
template <int PP>
__device__ __forceinline__ void march_emit(March& m, const float* P0,
                                           const uint8_t* S0, int cp,
                                           const float (&uxa)[3],
                                           const float (&uxb)[3],
                                           const float (&uy4)[4], bool act_a,
                                           bool act_b, float* outa, float* outb,
                                           const Consts& k) {
  // phi along y at rows ya-2 .. yb+2 of the own column
  const float py0 = P0[cp - 2 * PP], py1 = P0[cp - PP], py4 = P0[cp + 2 * PP],
              py5 = P0[cp + 3 * PP];
  const float va = m.ca[0], vb = m.cb[0];
  const bool sy0 = (S0[cp - PP] & FLAG_SOLID) != 0;
  const bool sy3 = (S0[cp + 2 * PP] & FLAG_SOLID) != 0;
  const float s_m = minmod(vsub(py1, py0), vsub(va, py1));  // y slopes at ya-1 .. yb+1
  const float s_a = minmod(vsub(va, py1), vsub(vb, va));
  const float s_b = minmod(vsub(vb, va), vsub(py4, vb));
  const float s_p = minmod(vsub(py4, vb), vsub(py5, py4));
  const float fy_m = face_flux(uy4[0], uy4[1], py1, s_m, va, s_a);  // ya-1/2
  const float fy_c = face_flux(uy4[1], uy4[2], va, s_a, vb, s_b);   // ya+1/2
  const float fy_p = face_flux(uy4[2], uy4[3], vb, s_b, py4, s_p);  // yb+1/2
  if (act_a) {
    const float dy = vsub(m.sb3[1] ? 0.f : fy_c, sy0 ? 0.f : fy_m);
    const float dz = vsub(m.sa3[2] ? 0.f : m.fzpa, m.sa3[0] ? 0.f : m.fzma);
    march_node(m.msum, m.wsum, P0, S0, cp, va, m.sa3[1], dy, dz, uxa[0], uxa[1],
               uxa[2], m.Ha[0], m.Ha[1], m.Ha[2], m.Va[0], m.Va[2], m.La[0],
               m.La[1], m.La[2], outa, k);
  }
  if (act_b) {
    const float dy = vsub(sy3 ? 0.f : fy_p, m.sa3[1] ? 0.f : fy_c);
    const float dz = vsub(m.sb3[2] ? 0.f : m.fzpb, m.sb3[0] ? 0.f : m.fzmb);
    march_node(m.msum, m.wsum, P0, S0, cp + PP, vb, m.sb3[1], dy, dz, uxb[0],
               uxb[1], uxb[2], m.Hb[0], m.Hb[1], m.Hb[2], m.Vb[0], m.Vb[2],
               m.Lb[0], m.Lb[1], m.Lb[2], outb, k);
  }
}

// Block reduction of the two partial sums; thread 0 writes them as FP64 to
// slot pb of partials (phi* sums) and nblocks + pb (chi sums).
template <int THREADS>
__device__ __forceinline__ void block_partials(DF msum, DF wsum, int tid,
                                               double* __restrict__ partials,
                                               int pb, int nblocks) {
  __shared__ DF red[2][THREADS / 32];
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
    double mm = 0.0, ww = 0.0;
    for (int i = 0; i < THREADS / 32; ++i) {
      mm += (double)red[0][i].hi + (double)red[0][i].lo;
      ww += (double)red[1][i].hi + (double)red[1][i].lo;
    }
    partials[pb] = mm;
    partials[nblocks + pb] = ww;
  }
}

// After the block's partial sums are stored: the last block of the launch
// to finish (a ticket counter, no waiting) forms lambda from all partials
// and resets the counter for the next launch. Without a ticket (a slab of
// a z decomposition) nothing is formed here.
__device__ __forceinline__ void finish_mass(const double* partials, int nb,
                                            MassScalars* ms, unsigned* ticket,
                                            int tid) {
  if (!ticket) return;  // the caller forms lambda from gathered partials
  __shared__ bool last;
  if (tid == 0) {
    __threadfence();  // this block's partials before its ticket
    last = atomicAdd(ticket, 1u) == (unsigned)(nb - 1);
  }
  __syncthreads();
  if (!last || tid >= 32) return;
  __threadfence();
  mass_from_partials(partials, nb, ms, tid);
  if (tid == 0) *ticket = 0u;
}

// One block: TX x TY output nodes per plane, TX x TY/2 threads; each thread
// owns two vertically adjacent output nodes (rows 2 ty and 2 ty + 1), which
// share most of their stencil reads and all per-thread bookkeeping.
// One tile (bxi, byi, bzi) of one grid; its partial sums go to slot pb of
// partials (phi* sums) and nblocks + pb (chi sums).
// Staging through registers: each thread loads its share of the next planes
// one plane ahead and stores it to shared memory at the next step. Works for
// any grid size.
template <int TY, int ZC>
__device__ __forceinline__ void phase_tile_body(
    int bxi, int byi, int bzi, int pb, const float* __restrict__ phi,
    const float* __restrict__ afld, float* __restrict__ phi_out,
    const float* __restrict__ u, const uint8_t* __restrict__ flags,
    double* __restrict__ partials, int nblocks, const Grid& g, const Consts& k,
    int zbase, int zlim) {
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

  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = tx + TX * ty;
  const int x0 = bxi * TX, y0 = byi * TY, z0 = zbase + bzi * ZC;
  const int zend = min(z0 + ZC, zlim);
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
  March m;
  march_init(m);
  m.ca[1] = s_phi[(z0 - 2) & 3][cp];
  m.ca[2] = s_phi[(z0 - 1) & 3][cp];
  m.cb[1] = s_phi[(z0 - 2) & 3][cp + PX];
  m.cb[2] = s_phi[(z0 - 1) & 3][cp + PX];
  // z velocity of the own columns at kz, kz + 1 (rolled at the output
  // planes), with the next plane's in nza / nzb
  const float* uz_ = u + 2 * N;
  float nza, nzb;
  {
    const int64_t zm = (int64_t)mod(z0 - 1, g.nz) * nxy;
    const int64_t zc = (int64_t)mod(z0, g.nz) * nxy;
    const int64_t zn = (int64_t)mod(z0 + 1, g.nz) * nxy;
    m.uza[0] = __ldg(uz_ + zm + own_a);
    m.uzb[0] = __ldg(uz_ + zm + own_b);
    m.uza[1] = __ldg(uz_ + zc + own_a);
    m.uzb[1] = __ldg(uz_ + zc + own_b);
    nza = __ldg(uz_ + zn + own_a);
    nzb = __ldg(uz_ + zn + own_b);
  }
  // x and y velocities of the next output plane
  float nxa[3] = {0.f, 0.f, 0.f}, nxb[3] = {0.f, 0.f, 0.f};
  float ny4[4] = {0.f, 0.f, 0.f, 0.f};
  auto fetch_u = [&](int kz) {
    const float* ux_ = u + (int64_t)kz * nxy;
    const float* uy_ = ux_ + N;
    const int ra = g.nx * min(ya, g.ny - 1), rb = g.nx * ybw;
    nxa[0] = __ldg(ux_ + ra + xm);
    nxa[1] = __ldg(ux_ + own_a);
    nxa[2] = __ldg(ux_ + ra + xp);
    nxb[0] = __ldg(ux_ + rb + xm);
    nxb[1] = __ldg(ux_ + own_b);
    nxb[2] = __ldg(ux_ + rb + xp);
    ny4[0] = __ldg(uy_ + g.nx * yam + xc);
    ny4[1] = __ldg(uy_ + own_a);
    ny4[2] = __ldg(uy_ + own_b);
    ny4[3] = __ldg(uy_ + g.nx * ybp + xc);
  };

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
    // velocities of the output plane, fetched one plane ahead: x and y
    // components of plane kz (loaded at kz - 1), and the z component rolled
    // along the own columns
    float uxa[3], uxb[3], uy4[4];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      uxa[i] = nxa[i];
      uxb[i] = nxb[i];
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) uy4[i] = ny4[i];
    if (out) {
      m.uza[0] = m.uza[1]; m.uza[1] = nza;
      m.uzb[0] = m.uzb[1]; m.uzb[1] = nzb;
      const int z2 = (kz + 2 >= g.nz) ? kz + 2 - g.nz : kz + 2;
      nza = __ldg(uz_ + (int64_t)z2 * nxy + own_a);
      nzb = __ldg(uz_ + (int64_t)z2 * nxy + own_b);
    }
    if (kz + 1 >= z0 && kz + 1 < zend) fetch_u(kz + 1);
    __syncthreads();
    march_roll<PX, AX>(m, s_phi[(kz + 1) & 3], s_phi[(kz + 2) & 3],
                       s_sol[(kz + 1) & 3], s_a[(kz + 1) & 1][0],
                       s_a[(kz + 1) & 1][1], s_a[(kz + 1) & 1][2], cp, ca);
    if (!out) continue;
    float* po = phi_out + (int64_t)kz * nxy;
    march_emit<PX>(m, s_phi[kz & 3], s_sol[kz & 3], cp, uxa, uxb, uy4, act_a,
                   act_b, po + own_a, po + own_b, k);
  }
  block_partials<THREADS>(m.msum, m.wsum, tid, partials, pb, nblocks);
}

// cp.async copies global -> shared (16 bytes through L2 only, 4 bytes through
// L1), and their commit / wait.
__device__ __forceinline__ void cp_async16(void* s, const void* gsrc) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(s);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(a), "l"(gsrc)
               : "memory");
}
__device__ __forceinline__ void cp_async4(void* s, const void* gsrc) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(s);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(a), "l"(gsrc)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int NPEND>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(NPEND) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// Shared-memory layout of the copy-staged tile. Every plane window spans
// x0-4 .. x0+35 (CW = 40 columns, ten 16-byte chunks) so that each chunk is
// 16-byte aligned in global memory when nx is a multiple of 4. Per bundle of
// copies: phi and the flags of plane t+2 (rows y0-2 .. y0+TY+1), a of plane
// t+1 (rows y0-1 .. y0+TY), u_x of plane t (rows y0 .. y0+TY-1, all 40
// columns), u_y of plane t (rows y0-1 .. y0+TY, columns x0 .. x0+31) and u_z
// of plane t+1 (rows y0 .. y0+TY-1, columns x0 .. x0+31). Bundles are issued
// D planes ahead into rings of RP (phi, flags) and RA (a, u) slots.
constexpr int CW = TX + 8;
constexpr int NCH = CW / 4;

template <int TY, int D>
struct CopyTile {
  static constexpr int PR = TY + 4, AR = TY + 2;
  // ring sizes: at least 4 + D phi planes and 2 + D a / u planes, rounded
  // up to powers of two so that slots are plane counters masked
  static constexpr int RP = (4 + D <= 4) ? 4 : (4 + D <= 8 ? 8 : 16);
  static constexpr int RA = (2 + D <= 2) ? 2 : (2 + D <= 4 ? 4 : 8);
  static constexpr int PHI = PR * CW;               // floats per phi slot
  static constexpr int AC = AR * CW;                // floats per a component
  static constexpr int UX = TY * CW, UY = (TY + 2) * TX, UZ = TY * TX;
  static constexpr int ASLOT = 3 * AC + UX + UY + UZ;  // a and u of one plane
  static constexpr int FLG = PR * CW;               // bytes per flags slot
  static constexpr size_t bytes =
      sizeof(float) * ((size_t)RP * PHI + (size_t)RA * ASLOT) + (size_t)RP * FLG;
};

// The same tile as phase_tile_body with every plane staged by cp.async
// copies issued D planes ahead. AL (nx % 4 == 0, 16-byte aligned fields):
// one 16-byte copy per 4-node chunk, the flags by 4-byte copies. Otherwise
// (any nx): one 4-byte copy per element, consecutive threads on
// consecutive elements of a window, each at its own wrapped column; the
// flag bytes (whose rows are not 4-byte aligned) are loaded into registers
// when their plane's copies are issued and stored into shared memory one
// step later, before the barrier that publishes them. Requires nz >= 2.
// smem is the dynamic shared memory of CopyTile<TY, D>::bytes.
template <int TY, int ZC, int D, bool AL = true>
__device__ __forceinline__ void phase_tile_copy(
    int bxi, int byi, int bzi, int pb, const float* __restrict__ phi,
    const float* __restrict__ afld, float* __restrict__ phi_out,
    const float* __restrict__ u, const uint8_t* __restrict__ flags,
    double* __restrict__ partials, int nblocks, const Grid& g, const Consts& k,
    float* smem, int zbase, int zlim) {
  using L = CopyTile<TY, D>;
  constexpr int THREADS = TX * TY / 2;
  static_assert(L::PR * NCH <= THREADS && L::AR * NCH <= THREADS &&
                    L::UY / 4 <= THREADS,
                "one copy job of each kind per thread");
  float* s_phi = smem;                                  // [RP][PHI]
  float* s_au = smem + L::RP * L::PHI;                  // [RA][ASLOT]
  uint8_t* s_flg = (uint8_t*)(s_au + L::RA * L::ASLOT); // [RP][FLG]

  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = tx + TX * ty;
  const int x0 = bxi * TX, y0 = byi * TY, z0 = zbase + bzi * ZC;
  const int zend = min(z0 + ZC, zlim);
  const int nxy = g.nx * g.ny;
  const int64_t N = g.N;

  // this thread's copy jobs: plane offsets (global) and slot offsets (shared)
  const bool hp = tid < L::PR * NCH;  // phi + flags chunk
  const bool ha = tid < L::AR * NCH;  // a chunk (3 components)
  const bool hx = tid < TY * NCH;     // u_x chunk
  const bool hy = tid < L::UY / 4;    // u_y chunk
  const bool hz = tid < L::UZ / 4;    // u_z chunk
  const int cx_ = tid % NCH, rx_ = tid / NCH;       // 40-column windows
  const int c8 = tid % (TX / 4), r8 = tid / (TX / 4);  // 32-column windows
  const int wx = mod(x0 - 4 + 4 * cx_, g.nx);
  const int w8 = mod(x0 + 4 * c8, g.nx);
  const int gp = wx + g.nx * mod(y0 - 2 + rx_, g.ny), sp = rx_ * CW + 4 * cx_;
  const int ga = wx + g.nx * mod(y0 - 1 + rx_, g.ny);  // slot offset sp
  const int gx = wx + g.nx * mod(y0 + rx_, g.ny);      // slot offset sp
  const int gy = w8 + g.nx * mod(y0 - 1 + r8, g.ny), s8 = r8 * TX + 4 * c8;
  const int gz = w8 + g.nx * mod(y0 + r8, g.ny);       // slot offset s8

  // element jobs (!AL): element j = tid + i THREADS of each window (the
  // slot offset is j; consecutive threads copy consecutive elements), with
  // its global in-plane offset (-1: none)
  constexpr int WP = L::PR * CW, WA = L::AR * CW, WX = L::UX, WY = L::UY, WZ = L::UZ;
  constexpr int NPE = AL ? 1 : (WP + THREADS - 1) / THREADS;
  constexpr int NAE = AL ? 1 : (WA + THREADS - 1) / THREADS;
  constexpr int NXE = AL ? 1 : (WX + THREADS - 1) / THREADS;
  constexpr int NYE = AL ? 1 : (WY + THREADS - 1) / THREADS;
  constexpr int NZE = AL ? 1 : (WZ + THREADS - 1) / THREADS;
  int ope[NPE], oae[NAE], oxe[NXE], oye[NYE], oze[NZE];
  uint8_t fpend[NPE];  // flag bytes waiting for their shared-memory store
  int fslot = -1;      // ... and their slot (-1: none)
  if constexpr (!AL) {
    auto off40 = [&](int j, int w, int ylo) {  // 40-column window, rows from ylo
      return j < w ? mod(x0 - 4 + j % CW, g.nx) + g.nx * mod(ylo + j / CW, g.ny) : -1;
    };
    auto off32 = [&](int j, int w, int ylo) {  // 32-column window
      return j < w ? mod(x0 + j % TX, g.nx) + g.nx * mod(ylo + j / TX, g.ny) : -1;
    };
#pragma unroll
    for (int i = 0; i < NPE; ++i) ope[i] = off40(tid + i * THREADS, WP, y0 - 2);
#pragma unroll
    for (int i = 0; i < NAE; ++i) oae[i] = off40(tid + i * THREADS, WA, y0 - 1);
#pragma unroll
    for (int i = 0; i < NXE; ++i) oxe[i] = off40(tid + i * THREADS, WX, y0);
#pragma unroll
    for (int i = 0; i < NYE; ++i) oye[i] = off32(tid + i * THREADS, WY, y0 - 1);
#pragma unroll
    for (int i = 0; i < NZE; ++i) oze[i] = off32(tid + i * THREADS, WZ, y0);
  }
  // a window's elements into shared memory (!AL)
  auto elems = [&](float* dst, const float* plane, const int* off, int n) {
#pragma unroll
    for (int i = 0; i < n; ++i)
      if (off[i] >= 0) cp_async4(dst + tid + i * THREADS, plane + off[i]);
  };

  const int nb = zend - z0 + 2;  // bundles / steps: planes z0-2 .. zend-1
  // phi and flags of plane p; !AL with defer: the flag bytes are stored at
  // the next step
  auto issue_phi = [&](int p, int slot, bool defer) {
    const int64_t zo = (int64_t)wrap1(p, g.nz) * nxy;
    if constexpr (AL) {
      if (hp) {
        cp_async16(s_phi + slot * L::PHI + sp, phi + zo + gp);
        cp_async4(s_flg + slot * L::FLG + sp, flags + zo + gp);
      }
    } else {
      elems(s_phi + slot * L::PHI, phi + zo, ope, NPE);
      uint8_t* sf = s_flg + slot * L::FLG;
#pragma unroll
      for (int i = 0; i < NPE; ++i) {
        if (ope[i] < 0) continue;
        const uint8_t f = __ldg(flags + zo + ope[i]);
        if (defer)
          fpend[i] = f;
        else
          sf[tid + i * THREADS] = f;
      }
      if (defer) fslot = slot;
    }
  };
  auto issue = [&](int b, bool defer) {  // bundle b: step kz = z0 - 2 + b
    const int t = z0 - 2 + b;
    issue_phi(t + 2, (b + 2) & (L::RP - 1), defer);
    float* sa = s_au + (b & (L::RA - 1)) * L::ASLOT;
    const int64_t z1 = (int64_t)wrap1(t + 1, g.nz) * nxy;
    const int64_t z0o = (int64_t)wrap1(t, g.nz) * nxy;  // output plane t
    if constexpr (AL) {
      if (ha) {
#pragma unroll
        for (int c = 0; c < 3; ++c)
          cp_async16(sa + c * L::AC + sp, afld + c * N + z1 + ga);
      }
      if (hz) cp_async16(sa + 3 * L::AC + L::UX + L::UY + s8, u + 2 * N + z1 + gz);
      if (b >= 2) {
        if (hx) cp_async16(sa + 3 * L::AC + sp, u + z0o + gx);
        if (hy) cp_async16(sa + 3 * L::AC + L::UX + s8, u + N + z0o + gy);
      }
    } else {
#pragma unroll
      for (int c = 0; c < 3; ++c) elems(sa + c * L::AC, afld + c * N + z1, oae, NAE);
      elems(sa + 3 * L::AC + L::UX + L::UY, u + 2 * N + z1, oze, NZE);
      if (b >= 2) {
        elems(sa + 3 * L::AC, u + z0o, oxe, NXE);
        elems(sa + 3 * L::AC + L::UX, u + N + z0o, oye, NYE);
      }
    }
  };

  // the two output rows of this thread
  const int x = x0 + tx;
  const int ya = y0 + 2 * ty, yb = ya + 1;
  const bool act_a = (x < g.nx) && (ya < g.ny);
  const bool act_b = (x < g.nx) && (yb < g.ny);
  const int own_a = x + g.nx * ya;  // used only when active
  const int own_b = own_a + g.nx;
  const int cp = (tx + 4) + CW * (2 * ty + 2);  // row a in phi-window coords
  const int ca = (tx + 4) + CW * (2 * ty + 1);  // row a in a-window coords
  const int cxu = (tx + 4) + CW * (2 * ty);     // row a in the u_x window
  const int cyu = tx + TX * (2 * ty + 1);       // row a in the u_y window
  const int czu = tx + TX * (2 * ty);           // row a in the u_z window

  // prologue: phi planes z0-2, z0-1 with bundle 0, then bundles 1 .. D-1
  // (their flag bytes stored at once: the first barrier publishes them)
  issue_phi(z0 - 2, 0, false);
  issue_phi(z0 - 1, 1, false);
  issue(0, false);
  cp_async_commit();
#pragma unroll
  for (int b = 1; b < D; ++b) {
    if (b < nb) issue(b, false);
    cp_async_commit();
  }

  March m;
  march_init(m);
  for (int b = 0; b < nb; ++b) {
    if constexpr (!AL) {
      // the flag bytes loaded at the previous step: their slot was last read
      // before that step's barrier, and is next read D - 1 steps from now
      if (fslot >= 0) {
        uint8_t* sf = s_flg + fslot * L::FLG;
#pragma unroll
        for (int i = 0; i < NPE; ++i)
          if (ope[i] >= 0) sf[tid + i * THREADS] = fpend[i];
      }
      fslot = -1;
    }
    if (b + D < nb) issue(b + D, true);
    cp_async_commit();
    cp_async_wait<D>();
    __syncthreads();
    const float* P0 = s_phi + (b & (L::RP - 1)) * L::PHI;
    const float* P1 = s_phi + ((b + 1) & (L::RP - 1)) * L::PHI;
    const float* P2 = s_phi + ((b + 2) & (L::RP - 1)) * L::PHI;
    const uint8_t* S0 = s_flg + (b & (L::RP - 1)) * L::FLG;
    const uint8_t* S1 = s_flg + ((b + 1) & (L::RP - 1)) * L::FLG;
    const float* sa = s_au + (b & (L::RA - 1)) * L::ASLOT;
    const float* su = sa + 3 * L::AC;
    if (b == 0) {  // own columns at planes z0-2, z0-1
      m.ca[1] = P0[cp];
      m.cb[1] = P0[cp + CW];
      m.ca[2] = P1[cp];
      m.cb[2] = P1[cp + CW];
    }
    const float* suz = su + L::UX + L::UY;
    m.uza[0] = m.uza[1]; m.uza[1] = suz[czu];
    m.uzb[0] = m.uzb[1]; m.uzb[1] = suz[czu + TX];
    march_roll<CW, CW>(m, P1, P2, S1, sa, sa + L::AC, sa + 2 * L::AC, cp, ca);
    if (b < 2) continue;
    const float uxa[3] = {su[cxu - 1], su[cxu], su[cxu + 1]};
    const float uxb[3] = {su[cxu + CW - 1], su[cxu + CW], su[cxu + CW + 1]};
    const float* suy = su + L::UX;
    const float uy4[4] = {suy[cyu - TX], suy[cyu], suy[cyu + TX], suy[cyu + 2 * TX]};
    float* po = phi_out + (int64_t)(z0 - 2 + b) * nxy;
    march_emit<CW>(m, P0, S0, cp, uxa, uxb, uy4, act_a, act_b, po + own_a,
                   po + own_b, k);
  }
  cp_async_wait_all();
  block_partials<THREADS>(m.msum, m.wsum, tid, partials, pb, nblocks);
}

// ---- Copy-staged tile with 2 x 2 nodes per thread --------------------------
// The same tile (TX x TYN nodes of a plane, marching up ZC planes) and the
// same per-node arithmetic as phase_tile_copy, with each thread owning an x
// pair of nodes on each of two rows: (x, x + 1) x (ya, ya + 1), x even. The
// x pair is evaluated in packed pair operations (one instruction for both
// nodes, rounded per node as the scalar one), shared-memory reads of the
// pair are 8-byte, the x faces between the pair and the stencil sums of the
// pair share their operands, and the copy jobs (phi with its flags, a and
// u, the same windows as phase_tile_copy) are addressed from offsets fixed
// once per tile. Bit-identical to the other phi-update kernels at every
// node; the per-thread order of the partial sums differs, so M* and W
// agree to rounding of the sums.
constexpr int QTX = TX / 2;  // thread columns

template <int TYN, int D>
struct QuadTile {
  static constexpr int PR = TYN + 4, AR = TYN + 2;  // phi rows, a rows
  // the copies of step b + D are issued before the barrier of step b, while
  // a thread may still be at step b - 1: they must miss the phi slots of
  // planes t-1 .. t+1 and the a slot of plane t that it reads
  static constexpr int RP = 4 + D, RA = 2 + D;
  static constexpr int PHI = PR * CW;  // floats per phi slot
  static constexpr int AC = AR * CW;   // floats per a component
  // u_x of plane t (rows y0 .., all CW columns), u_y of plane t (rows
  // y0-1 .., columns x0 .. x0+31), u_z of plane t + 1 (rows y0 .., 32
  // columns), after a of plane t + 1
  static constexpr int UX = TYN * CW, UY = (TYN + 2) * TX, UZ = TYN * TX;
  static constexpr int ASLOT = 3 * AC + UX + UY + UZ;
  static constexpr int FLG = PR * CW;  // bytes per flags slot
  static constexpr int NPJ = PR * NCH, NAJ = AR * NCH;  // copy jobs per plane
  static constexpr int NXJ = TYN * NCH, NYJ = (TYN + 2) * (TX / 4), NZJ = TYN * (TX / 4);
  static constexpr size_t bytes =
      sizeof(float) * ((size_t)RP * PHI + (size_t)RA * ASLOT) + (size_t)RP * FLG;
};

// solid bit of node i (0: (x, ya), 1: (x+1, ya), 2: (x, yb), 3: (x+1, yb))
// of carried plane p (0: kz-1, 1: kz, 2: kz+1)
__device__ __forceinline__ bool qsolid(uint32_t bits, int p, int i) {
  return (bits >> (4 * p + i)) & 1u;
}
// the two solid flags of an x pair from two flag bytes read as one 16-bit
// word (low byte: x, high byte: x + 1)
__device__ __forceinline__ uint32_t pair_bits(const uint8_t* s) {
  static_assert(FLAG_SOLID == 1, "solid flag in bit 0");
  const uint32_t w = *reinterpret_cast<const uint16_t*>(s);
  return (w & 1u) | ((w >> 7) & 2u);
}
__device__ __forceinline__ bool lo_solid(const uint8_t* s) {
  return (*reinterpret_cast<const uint16_t*>(s) & FLAG_SOLID) != 0;
}
__device__ __forceinline__ bool hi_solid(const uint8_t* s) {
  return (*reinterpret_cast<const uint16_t*>(s) & (FLAG_SOLID << 8)) != 0;
}
__device__ __forceinline__ float2 masked(bool sx, bool sy, float2 f) {
  return make_float2(sx ? 0.f : f.x, sy ? 0.f : f.y);
}
__device__ __forceinline__ float2 ld2(const float* p) {
  return *reinterpret_cast<const float2*>(p);
}

// Registers a thread carries up its 2 x 2 columns (pairs A: row ya, B: row
// yb), as March does for a pair of rows.
struct QMarch {
  float2 cA[3], cB[3];  // phi at kz .. kz+2
  uint32_t sol;         // solid bits of planes kz-1 .. kz+1 (qsolid)
  float2 HA[3], HB[3], VA[3], VB[3], LA[3], LB[3];
  float2 uzA[2], uzB[2];  // u_z at kz, kz+1
  float2 szA, szB;        // z slope at kz + 1
  float2 fzmA, fzmB, fzpA, fzpB;
  DF2 msum, wsum;  // per lane of the x pair
};

// In-plane partials of one output row pair from rows r .. r+2 of the four
// columns x-1 .. x+2 (a_x, a_y, a_z, phi rows as read from shared memory).
__device__ __forceinline__ void quad_row_partials(const float (&ax)[4][4],
                                                  const float (&ay)[4][4],
                                                  const float2 (&rz)[4],
                                                  const float2 (&rl)[4], int r,
                                                  float2& H, float2& V, float2& L) {
  auto col = [](const float (&f)[4][4], int row, int c) {
    return make_float2(f[row][c], f[row][c + 1]);
  };
  // S_y a_x at (x-1, x) and (x+1, x+2)
  const float2 sxm = sum141(col(ax, r, 0), col(ax, r + 1, 0), col(ax, r + 2, 0));
  const float2 sxp = sum141(col(ax, r, 2), col(ax, r + 1, 2), col(ax, r + 2, 2));
  // Dd_y a_y (times 6) at (x-1, x), (x, x+1), (x+1, x+2)
  const float2 d0 = vsub(col(ay, r + 2, 0), col(ay, r, 0));
  const float2 d1 = vsub(col(ay, r + 2, 1), col(ay, r, 1));
  const float2 d2 = vsub(col(ay, r + 2, 2), col(ay, r, 2));
  H = partial_h(sxp, sxm, d0, d1, d2);
  V = partial_s(rz[r], rz[r + 1], rz[r + 2]);
  L = partial_s(rl[r], rl[r + 1], rl[r + 2]);
}

// Advance the carried registers by one plane (as march_roll): partials of
// plane kz + 1 (phi slot P1, a slot components ax / ay / az, all with row
// pitch CW; cp and ca index (x, ya) in the phi and a windows), own phi at
// kz + 2 (P2), solid flags at kz + 1 (S1), then the z slope at kz + 1 and
// the z flux at kz + 1/2 (m.uz* must hold u_z at kz and kz + 1).
__device__ __forceinline__ void quad_roll(QMarch& m, const float* P1, const float* P2,
                                          const uint8_t* S1, const float* axp,
                                          const float* ayp, const float* azp, int cp,
                                          int ca) {
  float ax[4][4], ay[4][4];
  float2 rz[4], rl[4];
  // columns x-1 .. x+2 of a row from the aligned pairs at x-2, x, x+2
  auto row4 = [](const float* p, float (&v)[4]) {
    const float2 l = ld2(p - 2), c = ld2(p), r = ld2(p + 2);
    v[0] = l.y;
    v[1] = c.x;
    v[2] = c.y;
    v[3] = r.x;
  };
#pragma unroll
  for (int r = 0; r < 4; ++r) {  // rows ya-1 .. yb+1, columns x-1 .. x+2
    const int o = ca + (r - 1) * CW;
    const int op = cp + (r - 1) * CW;
    float zz[4], pp[4];
    row4(axp + o, ax[r]);
    row4(ayp + o, ay[r]);
    row4(azp + o, zz);
    row4(P1 + op, pp);
    // S_x of the row at (x, x+1)
    rz[r] = sum141(make_float2(zz[0], zz[1]), make_float2(zz[1], zz[2]),
                   make_float2(zz[2], zz[3]));
    rl[r] = sum141(make_float2(pp[0], pp[1]), make_float2(pp[1], pp[2]),
                   make_float2(pp[2], pp[3]));
  }
  float2 HA, VA, LA, HB, VB, LB;
  quad_row_partials(ax, ay, rz, rl, 0, HA, VA, LA);
  quad_row_partials(ax, ay, rz, rl, 1, HB, VB, LB);
  m.HA[0] = m.HA[1]; m.HA[1] = m.HA[2]; m.HA[2] = HA;
  m.HB[0] = m.HB[1]; m.HB[1] = m.HB[2]; m.HB[2] = HB;
  m.VA[0] = m.VA[1]; m.VA[1] = m.VA[2]; m.VA[2] = VA;
  m.VB[0] = m.VB[1]; m.VB[1] = m.VB[2]; m.VB[2] = VB;
  m.LA[0] = m.LA[1]; m.LA[1] = m.LA[2]; m.LA[2] = LA;
  m.LB[0] = m.LB[1]; m.LB[1] = m.LB[2]; m.LB[2] = LB;
  m.cA[0] = m.cA[1]; m.cA[1] = m.cA[2]; m.cA[2] = ld2(P2 + cp);
  m.cB[0] = m.cB[1]; m.cB[1] = m.cB[2]; m.cB[2] = ld2(P2 + cp + CW);
  m.sol = (m.sol >> 4) | (pair_bits(S1 + cp) << 8) | (pair_bits(S1 + cp + CW) << 10);
  const float2 sA1 = minmod(vsub(m.cA[1], m.cA[0]), vsub(m.cA[2], m.cA[1]));
  const float2 sB1 = minmod(vsub(m.cB[1], m.cB[0]), vsub(m.cB[2], m.cB[1]));
  m.fzmA = m.fzpA;
  m.fzmB = m.fzpB;
  m.fzpA = face_flux(m.uzA[0], m.uzA[1], m.cA[0], m.szA, m.cA[1], sA1);
  m.fzpB = face_flux(m.uzB[0], m.uzB[1], m.cB[0], m.szB, m.cB[1], sB1);
  m.szA = sA1;
  m.szB = sB1;
}

// x faces of one row pair at plane kz: phi at x-2 .. x+3 (pm, pc, pp),
// u_x at x-1 (um), (x, x+1) (uc), x+2 (up), solid flags at x-1 .. x+2;
// returns the masked flux differences of nodes x and x + 1.
__device__ __forceinline__ float2 quad_x_faces(float2 pm, float2 pc, float2 pp,
                                               float um, float2 uc, float up,
                                               bool sm1, bool s0, bool s1, bool s2) {
  // differences at x-3/2 .. x+5/2
  const float dm3 = vsub(pm.y, pm.x), dm1 = vsub(pc.x, pm.y), d1 = vsub(pc.y, pc.x),
              d3 = vsub(pp.x, pc.y), d5 = vsub(pp.y, pp.x);
  const float mm3 = neg_part(dm3), mm1 = neg_part(dm1), m1 = neg_part(d1),
              m3 = neg_part(d3), m5 = neg_part(d5);
  const float sxm = minmod_m(dm3, dm1, mm3, mm1), sx0 = minmod_m(dm1, d1, mm1, m1),
              sx1 = minmod_m(d1, d3, m1, m3), sx2 = minmod_m(d3, d5, m3, m5);
  // faces (x-1/2, x+1/2) and (x+1/2, x+3/2)
  const float2 fl = face_flux(make_float2(um, uc.x), uc, make_float2(pm.y, pc.x),
                              make_float2(sxm, sx0), pc, make_float2(sx0, sx1));
  const float2 fr = face_flux(uc, make_float2(uc.y, up), pc, make_float2(sx0, sx1),
                              make_float2(pc.y, pp.x), make_float2(sx1, sx2));
  return vsub(masked(s1, s2, fr), masked(sm1, s0, fl));
}

// One output row pair: phi*, its store and its partial sums (as march_node
// per node; a node outside the grid or solid adds an exact zero, which
// leaves the compensated sums unchanged). act: the pair is inside the grid.
__device__ __forceinline__ void quad_nodes(DF2& msum, DF2& wsum, float2 v0, float2 div,
                                           const float2 (&L)[3], const float2 (&H)[3],
                                           const float2 (&Vz)[3], bool solx, bool soly,
                                           bool act, float* out, const Consts& k) {
  const float2 vs = node_update(v0, div, L[0], L[1], L[2], H[0], H[1], H[2], Vz[0],
                                Vz[2], k);
  if (act)
    *reinterpret_cast<float2*>(out) = make_float2(solx ? v0.x : vs.x, soly ? v0.y : vs.y);
  const float2 v = make_float2((act && !solx) ? vs.x : 0.f, (act && !soly) ? vs.y : 0.f);
  df2_add(msum, v);
  df2_add(wsum, make_float2(band_chi(v.x, k), band_chi(v.y, k)));
}

// The tile (bxi, byi, bzi) of one grid, 2 x 2 nodes per thread, staged by
// asynchronous copies issued D planes ahead. Requires nx % 4 == 0 (every
// 16-byte chunk of a plane row is aligned and the x pairs never straddle
// the wrap) and 16-byte aligned fields. smem: QuadTile<TYN, D>::bytes.
// Ring slots and plane offsets advance by one per step (no division); the
// first two steps, which only fill the carried registers, are peeled.
template <int TYN, int ZC, int D>
__device__ __forceinline__ void phase_tile_quad(
    int bxi, int byi, int bzi, int pb, const float* __restrict__ phi,
    const float* __restrict__ afld, float* __restrict__ phi_out,
    const float* __restrict__ u, const uint8_t* __restrict__ flags,
    double* __restrict__ partials, int nblocks, const Grid& g, const Consts& k,
    float* smem, int zbase, int zlim) {
  using L = QuadTile<TYN, D>;
  constexpr int THREADS = QTX * TYN / 2;
  static_assert(L::NPJ <= 2 * THREADS && L::NAJ <= 2 * THREADS && L::NXJ <= 2 * THREADS &&
                    L::NYJ <= 2 * THREADS && L::NZJ <= THREADS,
                "at most two copy jobs of a kind a thread");
  float* s_phi = smem;                                   // [RP][PHI]
  float* s_a = smem + L::RP * L::PHI;                    // [RA][3][AC]
  uint8_t* s_flg = (uint8_t*)(s_a + L::RA * L::ASLOT);   // [RP][FLG]

  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = tx + QTX * ty;
  const int x0 = bxi * TX, y0 = byi * TYN, z0 = zbase + bzi * ZC;
  const int zend = min(z0 + ZC, zlim);
  const int nx = g.nx, ny = g.ny, nxy = nx * ny;
  const int64_t N = g.N;
  const int64_t nzxy = (int64_t)g.nz * nxy;
  auto advance = [&](int64_t& off) {  // plane offset of the next plane (wraps)
    off += nxy;
    if (off >= nzxy) off -= nzxy;
  };

  // copy jobs j = tid, tid + THREADS: in-plane global offsets (wrapped) and
  // offsets in the slot; phi chunks cover rows y0-2 .., a chunks y0-1 ..
  int gp[2], ga[2], so[2], gux[2], guy[2], sy8[2];
  bool hp[2], ha[2], hx[2], hy[2];
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int j = tid + i * THREADS;
    const int row = j / NCH, ch = j % NCH;
    const int gx = mod(x0 - 4 + 4 * ch, nx);
    hp[i] = j < L::NPJ;
    ha[i] = j < L::NAJ;
    hx[i] = j < L::NXJ;
    gp[i] = gx + nx * mod(y0 - 2 + row, ny);
    ga[i] = gx + nx * mod(y0 - 1 + row, ny);
    gux[i] = gx + nx * mod(y0 + row, ny);
    so[i] = row * CW + 4 * ch;
    const int r8 = j / (TX / 4), c8 = j % (TX / 4);
    hy[i] = j < L::NYJ;
    guy[i] = mod(x0 + 4 * c8, nx) + nx * mod(y0 - 1 + r8, ny);
    sy8[i] = r8 * TX + 4 * c8;
  }
  const bool hz = tid < L::NZJ;
  const int guz = mod(x0 + 4 * (tid % (TX / 4)), nx) + nx * mod(y0 + tid / (TX / 4), ny);
  auto issue_phi = [&](int64_t zo, int slot) {  // phi and flags of one plane
    float* sp = s_phi + slot * L::PHI;
    uint8_t* sf = s_flg + slot * L::FLG;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      if (hp[i]) {
        cp_async16(sp + so[i], phi + zo + gp[i]);
        cp_async4(sf + so[i], flags + zo + gp[i]);
      }
    }
  };
  // a and u_z of the plane at zo, u_x and u_y of the plane before it (zu)
  auto issue_a = [&](int64_t zo, int64_t zu, int slot) {
    float* sa = s_a + slot * L::ASLOT;
    float* su = sa + 3 * L::AC;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      if (ha[i]) {
#pragma unroll
        for (int c = 0; c < 3; ++c)
          cp_async16(sa + c * L::AC + so[i], afld + c * N + zo + ga[i]);
      }
      if (hx[i]) cp_async16(su + so[i], u + zu + gux[i]);
      if (hy[i]) cp_async16(su + L::UX + sy8[i], u + N + zu + guy[i]);
    }
    if (hz) cp_async16(su + L::UX + L::UY + 4 * tid, u + 2 * N + zo + guz);
  };
  auto plane = [&](int p) { return (int64_t)wrap1(p, g.nz) * nxy; };

  // the 2 x 2 nodes of this thread (clamped copies for the global reads of
  // threads outside the grid)
  const int x = x0 + 2 * tx;
  const int ya = y0 + 2 * ty, yb = ya + 1;
  const bool act_a = (x < nx) && (ya < ny);
  const bool act_b = (x < nx) && (yb < ny);
  const int own_a = x + nx * ya, own_b = own_a + nx;  // stores, when active
  const int cp = (2 * tx + 4) + CW * (2 * ty + 2);  // (x, ya) in the phi window
  const int ca = (2 * tx + 4) + CW * (2 * ty + 1);  // (x, ya) in the a window
  const int cux = (2 * tx + 4) + CW * (2 * ty);     // (x, ya) in the u_x window
  const int cuy = 2 * tx + TX * (2 * ty + 1);       // (x, ya) in the u_y window
  const int cuz = 2 * tx + TX * (2 * ty);           // (x, ya) in the u_z window

  // prologue: phi planes z0-2, z0-1, then steps 0 .. D-1 (phi t+2, a t+1)
  const int nb = zend - z0 + 2;  // steps: planes z0-2 .. zend-1 (nb >= 3)
  issue_phi(plane(z0 - 2), 0);
  issue_phi(plane(z0 - 1), 1);
#pragma unroll
  for (int b = 0; b < D; ++b) {
    if (b < nb) {
      issue_phi(plane(z0 + b), (b + 2) % L::RP);
      issue_a(plane(z0 - 1 + b), plane(z0 - 2 + b), b % L::RA);
    }
    cp_async_commit();
  }
  // next issues: phi plane t + 2 + D, a plane t + 1 + D, u plane t + D
  int64_t zi_phi = plane(z0 + D), zi_a = plane(z0 - 1 + D), zi_u = plane(z0 - 2 + D);
  int spi = (2 + D) % L::RP, sai = D % L::RA;                 // their slots
  int sp0 = 0, sa0 = 0;  // phi slot of plane t, a slot of plane t + 1
  auto next = [](int s, int n) { return s + 1 == n ? 0 : s + 1; };

  QMarch m;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    m.cA[i] = m.cB[i] = make_float2(0.f, 0.f);
    m.HA[i] = m.HB[i] = m.VA[i] = m.VB[i] = m.LA[i] = m.LB[i] = make_float2(0.f, 0.f);
  }
  m.sol = 0u;
  m.uzA[0] = m.uzA[1] = m.uzB[0] = m.uzB[1] = make_float2(0.f, 0.f);
  m.szA = m.szB = m.fzmA = m.fzmB = m.fzpA = m.fzpB = make_float2(0.f, 0.f);
  m.msum = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
  m.wsum = m.msum;
  int64_t zo_u = (int64_t)z0 * nxy;  // output plane of the first emitting step

  // one step: issue the copies D planes ahead, wait for this step's planes,
  // roll the carried registers and (EMIT) write output plane t
  auto step = [&](int b, auto first_c, auto emit_c) {
    constexpr bool FIRST = decltype(first_c)::value;
    constexpr bool EMIT = decltype(emit_c)::value;
    if (b + D < nb) {
      issue_phi(zi_phi, spi);
      issue_a(zi_a, zi_u, sai);
    }
    cp_async_commit();
    advance(zi_phi);
    advance(zi_a);
    advance(zi_u);
    spi = next(spi, L::RP);
    sai = next(sai, L::RA);
    cp_async_wait<D>();
    __syncthreads();
    const int sp1 = next(sp0, L::RP), sp2 = next(sp1, L::RP);
    const float* P0 = s_phi + sp0 * L::PHI;
    const float* P1 = s_phi + sp1 * L::PHI;
    const float* P2 = s_phi + sp2 * L::PHI;
    const uint8_t* S0 = s_flg + sp0 * L::FLG;
    const uint8_t* S1 = s_flg + sp1 * L::FLG;
    const float* A1 = s_a + sa0 * L::ASLOT;
    const float* su = A1 + 3 * L::AC;  // u_x, u_y of plane t, u_z of plane t + 1
    m.uzA[0] = m.uzA[1];
    m.uzA[1] = ld2(su + L::UX + L::UY + cuz);
    m.uzB[0] = m.uzB[1];
    m.uzB[1] = ld2(su + L::UX + L::UY + cuz + TX);
    if constexpr (FIRST) {  // own columns at planes z0-2, z0-1
      m.cA[1] = ld2(P0 + cp);
      m.cB[1] = ld2(P0 + cp + CW);
      m.cA[2] = ld2(P1 + cp);
      m.cB[2] = ld2(P1 + cp + CW);
    }
    quad_roll(m, P1, P2, S1, A1, A1 + L::AC, A1 + 2 * L::AC, cp, ca);
    sp0 = sp1;
    sa0 = next(sa0, L::RA);
    if constexpr (EMIT) {
      // x faces of rows ya and yb
      const bool sAx = qsolid(m.sol, 1, 0), sAy = qsolid(m.sol, 1, 1);
      const bool sBx = qsolid(m.sol, 1, 2), sBy = qsolid(m.sol, 1, 3);
      const float2 dxA = quad_x_faces(ld2(P0 + cp - 2), m.cA[0], ld2(P0 + cp + 2),
                                      su[cux - 1], ld2(su + cux), su[cux + 2],
                                      hi_solid(S0 + cp - 2), sAx, sAy,
                                      lo_solid(S0 + cp + 2));
      const float2 dxB = quad_x_faces(ld2(P0 + cp + CW - 2), m.cB[0],
                                      ld2(P0 + cp + CW + 2), su[cux + CW - 1],
                                      ld2(su + cux + CW), su[cux + CW + 2],
                                      hi_solid(S0 + cp + CW - 2), sBx, sBy,
                                      lo_solid(S0 + cp + CW + 2));
      const float* suy = su + L::UX;
      const float2 uym = ld2(suy + cuy - TX), uyA = ld2(suy + cuy),
                   uyB = ld2(suy + cuy + TX), uyp = ld2(suy + cuy + 2 * TX);
      // y faces ya-1/2, ya+1/2, yb+1/2 of both columns
      const float2 qm2 = ld2(P0 + cp - 2 * CW), qm1 = ld2(P0 + cp - CW);
      const float2 qa = m.cA[0], qb = m.cB[0];
      const float2 qp1 = ld2(P0 + cp + 2 * CW), qp2 = ld2(P0 + cp + 3 * CW);
      const float2 e0 = vsub(qm1, qm2), e1 = vsub(qa, qm1), e2 = vsub(qb, qa),
                   e3 = vsub(qp1, qb), e4 = vsub(qp2, qp1);
      const float2 n0 = neg_part(e0), n1 = neg_part(e1), n2 = neg_part(e2),
                   n3 = neg_part(e3), n4 = neg_part(e4);
      const float2 sym = minmod_m(e0, e1, n0, n1), sya = minmod_m(e1, e2, n1, n2),
                   syb = minmod_m(e2, e3, n2, n3), syp = minmod_m(e3, e4, n3, n4);
      const float2 fym = face_flux(uym, uyA, qm1, sym, qa, sya);
      const float2 fyc = face_flux(uyA, uyB, qa, sya, qb, syb);
      const float2 fyp = face_flux(uyB, uyp, qb, syb, qp1, syp);
      const uint32_t sm1 = pair_bits(S0 + cp - CW), sp1b = pair_bits(S0 + cp + 2 * CW);
      const float2 dyA = vsub(masked(sBx, sBy, fyc), masked(sm1 & 1u, sm1 & 2u, fym));
      const float2 dyB = vsub(masked(sp1b & 1u, sp1b & 2u, fyp), masked(sAx, sAy, fyc));
      const float2 dzA = vsub(masked(qsolid(m.sol, 2, 0), qsolid(m.sol, 2, 1), m.fzpA),
                              masked(qsolid(m.sol, 0, 0), qsolid(m.sol, 0, 1), m.fzmA));
      const float2 dzB = vsub(masked(qsolid(m.sol, 2, 2), qsolid(m.sol, 2, 3), m.fzpB),
                              masked(qsolid(m.sol, 0, 2), qsolid(m.sol, 0, 3), m.fzmB));
      float* po = phi_out + zo_u;
      quad_nodes(m.msum, m.wsum, qa, vadd(vadd(dxA, dyA), dzA), m.LA, m.HA, m.VA, sAx,
                 sAy, act_a, po + own_a, k);
      quad_nodes(m.msum, m.wsum, qb, vadd(vadd(dxB, dyB), dzB), m.LB, m.HB, m.VB, sBx,
                 sBy, act_b, po + own_b, k);
      zo_u += nxy;
    }
  };
  step(0, std::true_type{}, std::false_type{});
  step(1, std::false_type{}, std::false_type{});
#pragma unroll 1
  for (int b = 2; b < nb; ++b) step(b, std::false_type{}, std::true_type{});
  cp_async_wait_all();
  block_partials<THREADS>(df_merge(lane_x(m.msum), lane_y(m.msum)),
                          df_merge(lane_x(m.wsum), lane_y(m.wsum)), tid, partials, pb,
                          nblocks);
}

template <int TYN, int ZC, int D, int MINB>
__global__ void __launch_bounds__(QTX * TYN / 2, MINB)
phase_update_quad(const float* __restrict__ phi, const float* __restrict__ afld,
                  float* __restrict__ phi_out, const float* __restrict__ u,
                  const uint8_t* __restrict__ flags,
                  double* __restrict__ partials, int nblocks, Grid g,
                  Consts k, MassScalars* ms, unsigned* ticket, int zbase, int zlim) {
  extern __shared__ __align__(16) float dsm[];
  const int pb = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
  phase_tile_quad<TYN, ZC, D>(blockIdx.x, blockIdx.y, blockIdx.z, pb, phi, afld, phi_out,
                              u, flags, partials, nblocks, g, k, dsm, zbase, zlim);
  finish_mass(partials, nblocks, ms, ticket, threadIdx.x + QTX * threadIdx.y);
}

template <int TY, int ZC, int MINB>
__global__ void __launch_bounds__(TX * TY / 2, MINB)
phase_update_march(const float* __restrict__ phi, const float* __restrict__ afld,
                   float* __restrict__ phi_out, const float* __restrict__ u,
                   const uint8_t* __restrict__ flags,
                   double* __restrict__ partials, int nblocks, Grid g,
                   Consts k, MassScalars* ms, unsigned* ticket, int zbase, int zlim) {
  const int pb = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
  phase_tile_body<TY, ZC>(blockIdx.x, blockIdx.y, blockIdx.z, pb, phi, afld,
                          phi_out, u, flags, partials, nblocks, g, k, zbase, zlim);
  finish_mass(partials, nblocks, ms, ticket, threadIdx.x + TX * threadIdx.y);
}

template <int TY, int ZC, int D, int MINB, bool AL = true>
__global__ void __launch_bounds__(TX * TY / 2, MINB)
phase_update_copy(const float* __restrict__ phi, const float* __restrict__ afld,
                  float* __restrict__ phi_out, const float* __restrict__ u,
                  const uint8_t* __restrict__ flags,
                  double* __restrict__ partials, int nblocks, Grid g,
                  Consts k, MassScalars* ms, unsigned* ticket, int zbase, int zlim) {
  extern __shared__ __align__(16) float dsm[];
  const int pb = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
  phase_tile_copy<TY, ZC, D, AL>(blockIdx.x, blockIdx.y, blockIdx.z, pb, phi, afld,
                                 phi_out, u, flags, partials, nblocks, g, k, dsm, zbase,
                                 zlim);
  finish_mass(partials, nblocks, ms, ticket, threadIdx.x + TX * threadIdx.y);
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
                            cd.flags, cd.partials, cd.phase_nb, cd.g, cd.k, 0,
                            cd.g.nz);
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

dim3 phase_grid(const Grid& g, int variant, int nzr) {
  const PhaseShape s = phase_shape(variant);
  return dim3((g.nx + TX - 1) / TX, (g.ny + s.ty - 1) / s.ty, (nzr + s.zc - 1) / s.zc);
}

}  // namespace

// The default tile shape: 32 x 8 x 32 (variant 2), or 32 x 8 x 16 (variant
// 1) when the deeper tiles would number fewer than 400, fewer than three
// per SM, and leave most of the GPU idle (measured per step: 64^3 45.4 ->
// 36.9 us, 96^3 87.0 -> 80.5, 128^3 130.6 -> 127.9; from 160^3 on the deeper
// tiles are faster).
int phase_default_variant(const Grid& g) {
  const dim3 gr = phase_grid(g, 2, g.nz);
  return (int64_t)gr.x * gr.y * gr.z < 400 ? 1 : 2;
}

int phase_blocks(const cacl_ctx* c) {
  // partial-sum storage is sized for the variant with the most blocks
  int nb = 0;
  for (int v = 0; v < 4; ++v) {
    const dim3 gr = phase_grid(c->g, v, c->g.nz);
    nb = std::max(nb, (int)(gr.x * gr.y * gr.z));
  }
  return nb;
}

namespace {
// copy-staged kernels of the four tile shapes, with their shared memory
// (plane indices are wrapped once, so nz >= 2)
constexpr int COPY_D = 2;  // planes of copies in flight ahead of the compute
struct CopyKernel {
  void* fn;
  size_t smem;
};
CopyKernel copy_kernel(int variant) {
  switch (variant) {
    case 1: return {(void*)phase_update_copy<8, 16, COPY_D, 4>, CopyTile<8, COPY_D>::bytes};
    case 2: return {(void*)phase_update_copy<8, 32, COPY_D, 4>, CopyTile<8, COPY_D>::bytes};
    case 3: return {(void*)phase_update_copy<16, 32, COPY_D, 2>, CopyTile<16, COPY_D>::bytes};
    default: return {(void*)phase_update_copy<16, 16, COPY_D, 2>, CopyTile<16, COPY_D>::bytes};
  }
}

// the same with element-wise staging (any nx)
CopyKernel copy_kernel_u(int variant) {
  switch (variant) {
    case 1:
      return {(void*)phase_update_copy<8, 16, COPY_D, 4, false>, CopyTile<8, COPY_D>::bytes};
    case 2:
      return {(void*)phase_update_copy<8, 32, COPY_D, 4, false>, CopyTile<8, COPY_D>::bytes};
    case 3:
      return {(void*)phase_update_copy<16, 32, COPY_D, 2, false>, CopyTile<16, COPY_D>::bytes};
    default:
      return {(void*)phase_update_copy<16, 16, COPY_D, 2, false>, CopyTile<16, COPY_D>::bytes};
  }
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// Batched phi update over cases that qualify for copy staging: virtual
// block b is tile (bx, by, bz) of its case, staged as in phase_update_copy.
template <int TY, int ZC, int MINB, bool AL = true>
__global__ void __launch_bounds__(TX * TY / 2, MINB)
phase_update_batch_copy(const CaseDesc* __restrict__ cases, WorkList wl, int pc) {
  extern __shared__ __align__(16) float dsm[];
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
    phase_tile_copy<TY, ZC, COPY_D, AL>(local % nbx, (local / nbx) % nby,
                                    local / (nbx * nby), local, cd.phi[pc], cd.a,
                                    cd.phi[1 - pc], cd.u, cd.flags, cd.partials,
                                    cd.phase_nb, cd.g, cd.k, dsm, 0, cd.g.nz);
  }
}

// 2 x 2 kernels of the four tile shapes (TYN = the tile's rows), with
// their shared memory
constexpr int QUAD_D = 1;
CopyKernel quad_kernel(int variant) {
  switch (variant) {
    case 1: return {(void*)phase_update_quad<8, 16, QUAD_D, 5>, QuadTile<8, QUAD_D>::bytes};
    case 2: return {(void*)phase_update_quad<8, 32, QUAD_D, 5>, QuadTile<8, QUAD_D>::bytes};
    case 3: return {(void*)phase_update_quad<16, 32, QUAD_D, 3>, QuadTile<16, QUAD_D>::bytes};
    default: return {(void*)phase_update_quad<16, 16, QUAD_D, 3>, QuadTile<16, QUAD_D>::bytes};
  }
}

// Batched phi update over cases that run the 2 x 2 kernel alone.
template <int TYN, int ZC, int MINB>
__global__ void __launch_bounds__(QTX * TYN / 2, MINB)
phase_update_batch_quad(const CaseDesc* __restrict__ cases, WorkList wl, int pc) {
  extern __shared__ __align__(16) float dsm[];
  __shared__ CaseCursor cur;
  if (threadIdx.x == 0 && threadIdx.y == 0) cur.begin();
  __syncthreads();
  int b0, b1;
  block_range(wl, b0, b1);
  for (int b = b0; b < b1; ++b) {
    cur.seek(cases, wl, b);
    const CaseDesc& cd = cur.d;
    const int local = b - cur.cstart;
    const int nbx = (cd.g.nx + TX - 1) / TX, nby = (cd.g.ny + TYN - 1) / TYN;
    __syncthreads();  // the previous tile's shared-memory reads are done
    phase_tile_quad<TYN, ZC, QUAD_D>(local % nbx, (local / nbx) % nby,
                                     local / (nbx * nby), local, cd.phi[pc], cd.a,
                                     cd.phi[1 - pc], cd.u, cd.flags, cd.partials,
                                     cd.phase_nb, cd.g, cd.k, dsm, 0, cd.g.nz);
  }
}

CopyKernel quad_batch_kernel(int variant) {
  switch (variant) {
    case 1: return {(void*)phase_update_batch_quad<8, 16, 5>, QuadTile<8, QUAD_D>::bytes};
    case 2: return {(void*)phase_update_batch_quad<8, 32, 5>, QuadTile<8, QUAD_D>::bytes};
    case 3: return {(void*)phase_update_batch_quad<16, 32, 3>, QuadTile<16, QUAD_D>::bytes};
    default: return {(void*)phase_update_batch_quad<16, 16, 3>, QuadTile<16, QUAD_D>::bytes};
  }
}

CopyKernel copy_batch_kernel(int variant, bool al = true) {
  switch (variant) {
    case 1:
      return {al ? (void*)phase_update_batch_copy<8, 16, 4>
                 : (void*)phase_update_batch_copy<8, 16, 4, false>,
              CopyTile<8, COPY_D>::bytes};
    case 2:
      return {al ? (void*)phase_update_batch_copy<8, 32, 4>
                 : (void*)phase_update_batch_copy<8, 32, 4, false>,
              CopyTile<8, COPY_D>::bytes};
    case 3:
      return {al ? (void*)phase_update_batch_copy<16, 32, 2>
                 : (void*)phase_update_batch_copy<16, 32, 2, false>,
              CopyTile<16, COPY_D>::bytes};
    default:
      return {al ? (void*)phase_update_batch_copy<16, 16, 2>
                 : (void*)phase_update_batch_copy<16, 16, 2, false>,
              CopyTile<16, COPY_D>::bytes};
  }
}
}  // namespace

cudaError_t phase_init_attributes() {
  for (int v = 0; v < 4; ++v) {
    for (const CopyKernel ck : {copy_kernel(v), copy_kernel_u(v), copy_batch_kernel(v),
                                copy_batch_kernel(v, false), quad_kernel(v),
                                quad_batch_kernel(v)}) {
      const cudaError_t e = cudaFuncSetAttribute(
          ck.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ck.smem);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

int phase_batch_copy_occupancy(int variant, bool aligned) {
  int nb = 0;
  const PhaseShape s = phase_shape(variant);
  const CopyKernel ck = copy_batch_kernel(variant, aligned);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, ck.fn, TX * s.ty / 2, ck.smem);
  return nb;
}

cudaError_t launch_phase_batch_copy(const CaseDesc* cases, WorkList wl, int variant,
                                    int grid, int pc, bool aligned, cudaStream_t st) {
  const PhaseShape s = phase_shape(variant);
  const CopyKernel ck = copy_batch_kernel(variant, aligned);
  void* args[] = {(void*)&cases, (void*)&wl, (void*)&pc};
  return cudaLaunchKernel(ck.fn, dim3(grid), dim3(TX, s.ty / 2, 1), args, ck.smem,
                          st);
}

int phase_batch_quad_occupancy(int variant) {
  int nb = 0;
  const PhaseShape s = phase_shape(variant);
  const CopyKernel ck = quad_batch_kernel(variant);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, ck.fn, QTX * s.ty / 2, ck.smem);
  return nb;
}

cudaError_t launch_phase_batch_quad(const CaseDesc* cases, WorkList wl, int variant,
                                    int grid, int pc, cudaStream_t st) {
  const PhaseShape s = phase_shape(variant);
  const CopyKernel ck = quad_batch_kernel(variant);
  void* args[] = {(void*)&cases, (void*)&wl, (void*)&pc};
  return cudaLaunchKernel(ck.fn, dim3(grid), dim3(QTX, s.ty / 2, 1), args, ck.smem,
                          st);
}

bool phase_copy_ok(const Grid& g, const void* phi_in, const void* phi_out,
                   const void* a, const void* u, const void* flags) {
  return g.nx % 4 == 0 && g.nz >= 2 && aligned16(phi_in) && aligned16(phi_out) &&
         aligned16(a) && aligned16(u) && ((uintptr_t)flags & 3u) == 0;
}

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

// The phi update over planes [zbase, zlim) of the context (every plane for
// an ordinary context, the interior planes of a slab).
cudaError_t launch_phase(cacl_ctx* c, const float* phi_in, float* phi_out) {
  const int v = c->phase_variant;
  const int zbase = c->zbase, zlim = c->zlim > 0 ? c->zlim : c->g.nz;
  const dim3 grid = phase_grid(c->g, v, zlim - zbase);
  const int nb = (int)(grid.x * grid.y * grid.z);
  c->phase_nblocks = nb;
  const PhaseShape s = phase_shape(v);
  const dim3 block(TX, s.ty / 2, 1);
  const bool copy_ok = phase_copy_ok(c->g, phi_in, phi_out, c->a, c->u, c->flags);
  // element-wise staging: any nx (nz >= 2), two nodes per thread along y
  const bool copy_u = !copy_ok && c->g.nz >= 2;
  unsigned* ticket = c->ext_finalize ? nullptr : c->ticket;
  if (c->phase_pipe == 3 && !copy_ok) return cudaErrorInvalidValue;
  if (c->phase_pipe == 2 && !copy_ok && !copy_u) return cudaErrorInvalidValue;
  if (c->phase_pipe != 1 && (copy_ok || copy_u)) {
    const bool two = c->phase_pipe == 2 || !copy_ok;  // two nodes per thread along y
    const CopyKernel ck = !copy_ok ? copy_kernel_u(v) : (two ? copy_kernel(v) : quad_kernel(v));
    const dim3 cblock = two ? block : dim3(QTX, s.ty / 2, 1);
    const float* a = c->a;
    const float* u = c->u;
    const uint8_t* fl = c->flags;
    double* part = c->partials;
    Grid g = c->g;
    Consts k = c->k;
    int nbk = nb;
    MassScalars* ms = c->mass;
    int zb = zbase, zl = zlim;
    void* args[] = {(void*)&phi_in, (void*)&a,    (void*)&phi_out,
                    (void*)&u,      (void*)&fl,   (void*)&part,
                    (void*)&nbk,    (void*)&g,    (void*)&k,
                    (void*)&ms,     (void*)&ticket, (void*)&zb, (void*)&zl};
    return cudaLaunchKernel(ck.fn, grid, cblock, args, ck.smem, c->stream);
  }
  switch (v) {
    case 1:
      phase_update_march<8, 16, 4><<<grid, block, 0, c->stream>>>(
          phi_in, c->a, phi_out, c->u, c->flags, c->partials, nb, c->g, c->k,
          c->mass, ticket, zbase, zlim);
      break;
    case 2:
      phase_update_march<8, 32, 4><<<grid, block, 0, c->stream>>>(
          phi_in, c->a, phi_out, c->u, c->flags, c->partials, nb, c->g, c->k,
          c->mass, ticket, zbase, zlim);
      break;
    case 3:
      phase_update_march<16, 32, 2><<<grid, block, 0, c->stream>>>(
          phi_in, c->a, phi_out, c->u, c->flags, c->partials, nb, c->g, c->k,
          c->mass, ticket, zbase, zlim);
      break;
    default:
      phase_update_march<16, 16, 2><<<grid, block, 0, c->stream>>>(
          phi_in, c->a, phi_out, c->u, c->flags, c->partials, nb, c->g, c->k,
          c->mass, ticket, zbase, zlim);
      break;
  }
  return cudaGetLastError();
}

}  // namespace cacl
