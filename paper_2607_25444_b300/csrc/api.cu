// api.cu -- the C ABI declared in include/cacl.h: context life cycle, host
// transfers, the step as a captured CUDA graph, and queries.
#include <cmath>
#include <cstring>
#include <vector>

#include "cacl_internal.cuh"

using namespace cacl;

namespace {

const double kPi = 3.14159265358979323846;

cacl_status fail(cacl_ctx* c, cacl_status st, const std::string& msg) {
  if (c) c->err = msg;
  return st;
}

cacl_status cuda_fail(cacl_ctx* c, cudaError_t e, const char* where) {
  return fail(c, CACL_ERR_CUDA,
              std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(expr, where)                       \
  do {                                        \
    cudaError_t e_ = (expr);                  \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, where); \
  } while (0)

void drop_graphs(cacl_ctx* c) {
  for (auto& row : c->graph)
    for (auto& gexec : row) {
      if (gexec) cudaGraphExecDestroy(gexec);
      gexec = nullptr;
    }
}

// cot(theta_c), theta_c = pi - theta (Eq. internal_contact_angle), with the
// regularisation near |sin theta_c| -> 0 (Sect. 2.2).
double cot_internal(double theta_deg) {
  const double thc = kPi - theta_deg * kPi / 180.0;
  const double s = std::sin(thc), co = std::cos(thc);
  if (std::fabs(s) < 1e-6) return (co >= 0.0 ? 1.0 : -1.0) * 1e6;
  return co / s;
}

cudaError_t enqueue_step(cacl_ctx* c, int fc, int pc) {
  cudaError_t e;
  if ((e = launch_ghost(c, c->phi[pc])) != cudaSuccess) return e;
  if ((e = launch_lb(c, c->f[fc], c->f[1 - fc], c->phi[pc])) != cudaSuccess)
    return e;
  if ((e = launch_phase(c, c->phi[pc], c->phi[1 - pc])) != cudaSuccess) return e;
  if (c->zbase == 0 && c->zlim == 0 && !c->ext_finalize)
    return launch_correct_tiles(c, c->phi[1 - pc]);
  return launch_correct(c, c->phi[1 - pc]);
}

cudaError_t build_graph(cacl_ctx* c, int fc, int pc) {
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  const cudaError_t el = enqueue_step(c, fc, pc);
  e = cudaStreamEndCapture(c->stream, &graph);
  if (el != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return el;
  }
  if (e != cudaSuccess) return e;
  e = cudaGraphInstantiate(&c->graph[fc][pc], graph, 0);
  cudaGraphDestroy(graph);
  return e;
}

cacl_status upload_angles(cacl_ctx* c, const float* theta_node) {
  const int W = c->wall_count;
  if (W == 0) return CACL_OK;
  std::vector<int32_t> idx(W);
  CK(cudaMemcpyAsync(idx.data(), c->w_idx, sizeof(int32_t) * W,
                     cudaMemcpyDeviceToHost, c->stream), "copy wall index");
  CK(cudaStreamSynchronize(c->stream), "sync");
  std::vector<float> th(W), ct(W);
  for (int w = 0; w < W; ++w) {
    const double t = theta_node ? (double)theta_node[idx[w]] : c->p.theta_deg;
    th[w] = (float)t;
    ct[w] = (float)cot_internal(t);
  }
  CK(cudaMemcpyAsync(c->w_theta, th.data(), sizeof(float) * W,
                     cudaMemcpyHostToDevice, c->stream), "upload theta");
  CK(cudaMemcpyAsync(c->w_cot, ct.data(), sizeof(float) * W,
                     cudaMemcpyHostToDevice, c->stream), "upload cot");
  CK(cudaStreamSynchronize(c->stream), "sync");
  return CACL_OK;
}

bool ready(cacl_ctx* c) {
  if (!c) return false;
  if (!c->has_fields) {
    c->err = "state not initialised: call cacl_set_geometry and cacl_set_fields";
    return false;
  }
  return true;
}

}  // namespace

extern "C" {

cacl_status cacl_create(const cacl_params* p, void* stream, cacl_ctx** out) {
  if (!p || !out) return CACL_ERR_ARG;
  *out = nullptr;
  if (p->nx < 1 || p->ny < 1 || p->nz < 1) return CACL_ERR_ARG;
  const int64_t N = (int64_t)p->nx * p->ny * p->nz;
  if (N > (int64_t)INT32_MAX) return CACL_ERR_ARG;  // wall list uses int32 nodes
  if (!(p->width > 0) || !(p->mobility >= 0) || !(p->rho_l > 0) ||
      !(p->rho_g > 0) || !(p->nu_l > 0) || !(p->nu_g > 0) ||
      !(p->eps_phi > 0 && p->eps_phi < 0.5) || !(p->sigma >= 0))
    return CACL_ERR_ARG;
  if (p->storage != CACL_F32 && p->storage != CACL_F16_SHIFTED &&
      p->storage != CACL_BF16_SHIFTED && p->storage != CACL_F32_MOMENTS)
    return CACL_ERR_ARG;
  cacl_ctx* c = new cacl_ctx();
  c->p = *p;
  c->g = {p->nx, p->ny, p->nz, N};
  Consts& k = c->k;
  k.rho_g = (float)p->rho_g;
  k.drho = (float)(p->rho_l - p->rho_g);
  k.mu_g = (float)(p->rho_g * p->nu_g);
  k.dmu = (float)(p->rho_l * p->nu_l - p->rho_g * p->nu_g);
  k.beta4 = (float)(4.0 * 12.0 * p->sigma / p->width);  // 4 beta, Eq. Fcap
  k.kappa_phi = (float)(1.5 * p->sigma * p->width);
  k.gx = (float)p->gravity[0];
  k.gy = (float)p->gravity[1];
  k.gz = (float)p->gravity[2];
  k.mobility = (float)p->mobility;
  k.kappa = (float)(4.0 * p->mobility / p->width);     // Eq. kappa_delta
  k.eps_phi = (float)p->eps_phi;

  cudaError_t e;
  auto bail = [&](const char* where) {
    c->err = std::string(where) + ": " + cudaGetErrorString(e);
    cacl_destroy(c);
    return CACL_ERR_CUDA;
  };
  if (stream) {
    c->stream = (cudaStream_t)stream;
  } else {
    // a blocking stream of our own: graph capture needs a non-default
    // stream, and a blocking stream still orders with the legacy stream
    if ((e = cudaStreamCreate(&c->stream)) != cudaSuccess) return bail("stream");
    c->own_stream = true;
  }
  if ((e = phase_init_attributes()) != cudaSuccess) return bail("attributes");
  if ((e = lb_init(c)) != cudaSuccess) return bail("collide-stream set-up");
  const size_t fbytes = storage_bytes(p->storage) * (size_t)pop_comps(p->storage) * N;
  for (int i = 0; i < 2; ++i) {
    if ((e = cudaMalloc(&c->f[i], fbytes)) != cudaSuccess) return bail("alloc f");
    if ((e = cudaMalloc(&c->phi[i], sizeof(float) * N)) != cudaSuccess)
      return bail("alloc phi");
  }
  if ((e = cudaMalloc(&c->u, sizeof(float) * 3 * N)) != cudaSuccess)
    return bail("alloc u");
  if ((e = cudaMalloc(&c->a, sizeof(float) * 3 * N)) != cudaSuccess)
    return bail("alloc a");
  if ((e = cudaMalloc(&c->flags, N)) != cudaSuccess) return bail("alloc flags");
  if ((e = lb_tma_init(c)) != cudaSuccess) return bail("collide-stream tensor maps");
  c->phase_variant = phase_default_variant(c->g);
  c->part_blocks = phase_blocks(c);
  const int pb = std::max(c->part_blocks, mass_ref_blocks(N));
  if ((e = cudaMalloc(&c->partials, sizeof(double) * 2 * pb)) != cudaSuccess)
    return bail("alloc partials");
  if ((e = cudaMalloc(&c->mass, sizeof(MassScalars))) != cudaSuccess)
    return bail("alloc mass");
  if ((e = cudaMalloc(&c->bad_flag, sizeof(int))) != cudaSuccess)
    return bail("alloc flag");
  if ((e = cudaMalloc(&c->ticket, 3 * sizeof(unsigned))) != cudaSuccess)
    return bail("alloc ticket");
  if ((e = cudaMemsetAsync(c->ticket, 0, 3 * sizeof(unsigned), c->stream)) !=
      cudaSuccess)
    return bail("memset");
  if ((e = cudaMemsetAsync(c->mass, 0, sizeof(MassScalars), c->stream)) !=
      cudaSuccess)
    return bail("memset");
  if ((e = cudaMemsetAsync(c->flags, 0, N, c->stream)) != cudaSuccess)
    return bail("memset");
  c->device_bytes = 2 * (int64_t)fbytes + 2 * 4 * N + 24 * N + N +
                    16 * (int64_t)pb + (int64_t)sizeof(MassScalars);
  *out = c;
  return CACL_OK;
}

void cacl_destroy(cacl_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  drop_graphs(c);
  adjoint_free(c->adj);
  void* bufs[] = {c->f[0], c->f[1], c->phi[0], c->phi[1], c->u, c->a, c->flags,
                  c->w_idx, c->w_donor, c->w_q, c->w_n6, c->w_nw, c->w_cot,
                  c->w_theta, c->w_g, c->partials, c->mass, c->scan_scratch,
                  c->bad_flag, c->ticket};
  for (void* b : bufs)
    if (b) cudaFree(b);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

const char* cacl_last_error(const cacl_ctx* c) { return c ? c->err.c_str() : ""; }

cacl_status cacl_set_geometry(cacl_ctx* c, const uint8_t* solid) {
  if (!c || !solid) return fail(c, CACL_ERR_ARG, "null argument");
  const Grid& g = c->g;
  const int ext[3] = {g.nx, g.ny, g.nz};
  for (int ax = 0; ax < 3; ++ax) {
    if (c->p.periodic[ax]) continue;
    if (ext[ax] < 2)
      return fail(c, CACL_ERR_GEOMETRY, "non-periodic axis shorter than 2");
    for (int64_t n = 0; n < g.N; ++n) {
      const int co[3] = {(int)(n % g.nx), (int)((n / g.nx) % g.ny),
                         (int)(n / ((int64_t)g.nx * g.ny))};
      if ((co[ax] == 0 || co[ax] == ext[ax] - 1) && !solid[n])
        return fail(c, CACL_ERR_GEOMETRY,
                    "non-periodic axis not closed by solid layers");
    }
  }
  drop_graphs(c);
  uint8_t* dsolid = nullptr;
  CK(cudaMalloc(&dsolid, g.N), "alloc occupancy");
  std::vector<uint8_t> bin(solid, solid + g.N);
  for (auto& b : bin) b = b ? 1 : 0;
  cudaError_t e = cudaMemcpyAsync(dsolid, bin.data(), g.N,
                                  cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = launch_geometry(c, dsolid);
  cudaFree(dsolid);
  if (e != cudaSuccess) return cuda_fail(c, e, "geometry");
  c->has_geometry = true;
  c->has_fields = false;
  c->geom_version++;
  return upload_angles(c, nullptr);
}

cacl_status cacl_set_wall_angles(cacl_ctx* c, const float* theta_w) {
  if (!c || !theta_w) return fail(c, CACL_ERR_ARG, "null argument");
  if (!c->has_geometry) return fail(c, CACL_ERR_STATE, "set_geometry first");
  const int W = c->wall_count;
  if (W == 0) return CACL_OK;
  std::vector<float> ct(W);
  for (int w = 0; w < W; ++w) ct[w] = (float)cot_internal(theta_w[w]);
  CK(cudaMemcpyAsync(c->w_theta, theta_w, sizeof(float) * W,
                     cudaMemcpyHostToDevice, c->stream), "upload theta");
  CK(cudaMemcpyAsync(c->w_cot, ct.data(), sizeof(float) * W,
                     cudaMemcpyHostToDevice, c->stream), "upload cot");
  CK(cudaStreamSynchronize(c->stream), "sync");
  return CACL_OK;
}

cacl_status cacl_set_sigma(cacl_ctx* c, double sigma) {
  if (!c || !(sigma >= 0)) return fail(c, CACL_ERR_ARG, "invalid surface tension");
  c->p.sigma = sigma;
  c->k.beta4 = (float)(4.0 * 12.0 * sigma / c->p.width);
  c->k.kappa_phi = (float)(1.5 * sigma * c->p.width);
  drop_graphs(c);  // the constants are launch arguments inside the graphs
  return CACL_OK;
}

cacl_status cacl_set_contact_angle(cacl_ctx* c, const float* theta) {
  if (!c) return CACL_ERR_ARG;
  if (!c->has_geometry) return fail(c, CACL_ERR_STATE, "set_geometry first");
  return upload_angles(c, theta);
}

cacl_status cacl_set_fields(cacl_ctx* c, const float* phi, const float* u) {
  if (!c || !phi) return fail(c, CACL_ERR_ARG, "null argument");
  if (!c->has_geometry) return fail(c, CACL_ERR_STATE, "set_geometry first");
  const int64_t N = c->g.N;
  CK(cudaMemcpyAsync(c->phi[0], phi, sizeof(float) * N, cudaMemcpyHostToDevice,
                     c->stream), "upload phi");
  CK(cudaMemcpyAsync(c->phi[1], c->phi[0], sizeof(float) * N, cudaMemcpyDeviceToDevice,
                     c->stream), "copy phi");
  if (u)
    CK(cudaMemcpyAsync(c->u, u, sizeof(float) * 3 * N, cudaMemcpyHostToDevice,
                       c->stream), "upload u");
  else
    CK(cudaMemsetAsync(c->u, 0, sizeof(float) * 3 * N, c->stream), "zero u");
  CK(cudaMemsetAsync(c->a, 0, sizeof(float) * 3 * N, c->stream), "zero a");
  if (c->p.storage == CACL_F32_MOMENTS)
    CK(launch_moments_init(c), "init moments");
  else
    CK(launch_init_populations(c), "init populations");
  CK(launch_mass_ref(c, c->phi[0]), "mass reference");
  CK(cudaStreamSynchronize(c->stream), "sync");
  c->fcur = 0;
  c->pcur = 0;
  c->has_fields = true;
  return CACL_OK;
}

cacl_status cacl_set_populations(cacl_ctx* c, const float* f) {
  if (!c || !f) return fail(c, CACL_ERR_ARG, "null argument");
  if (!ready(c)) return CACL_ERR_STATE;
  if (c->p.storage == CACL_F32_MOMENTS)
    return fail(c, CACL_ERR_ARG, "the moment form holds 17 coefficients per node, "
                                 "not arbitrary populations");
  const size_t bytes = sizeof(float) * Q * c->g.N;
  if (c->p.storage == CACL_F32) {
    CK(cudaMemcpyAsync(c->f[c->fcur], f, bytes, cudaMemcpyHostToDevice,
                       c->stream), "upload f");
  } else {
    float* tmp = nullptr;
    CK(cudaMalloc(&tmp, bytes), "alloc f staging");
    cudaError_t e = cudaMemcpyAsync(tmp, f, bytes, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = launch_to_storage(c, tmp, c->f[c->fcur]);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(tmp);
    if (e != cudaSuccess) return cuda_fail(c, e, "upload f");
  }
  CK(cudaStreamSynchronize(c->stream), "sync");
  return CACL_OK;
}

cacl_status cacl_set_phi(cacl_ctx* c, const float* phi) {
  if (!c || !phi) return fail(c, CACL_ERR_ARG, "null argument");
  if (!ready(c)) return CACL_ERR_STATE;
  CK(cudaMemcpyAsync(c->phi[c->pcur], phi, sizeof(float) * c->g.N,
                     cudaMemcpyHostToDevice, c->stream), "upload phi");
  CK(cudaStreamSynchronize(c->stream), "sync");
  return CACL_OK;
}

cacl_status cacl_set_velocity(cacl_ctx* c, const float* u) {
  if (!c || !u) return fail(c, CACL_ERR_ARG, "null argument");
  if (!ready(c)) return CACL_ERR_STATE;
  CK(cudaMemcpyAsync(c->u, u, sizeof(float) * 3 * c->g.N,
                     cudaMemcpyHostToDevice, c->stream), "upload u");
  CK(cudaStreamSynchronize(c->stream), "sync");
  return CACL_OK;
}

cacl_status cacl_set_mass_ref(cacl_ctx* c, double m) {
  if (!ready(c)) return c ? CACL_ERR_STATE : CACL_ERR_ARG;
  CK(cudaMemcpyAsync(&c->mass->m_ref, &m, sizeof(double),
                     cudaMemcpyHostToDevice, c->stream), "upload m_ref");
  CK(cudaStreamSynchronize(c->stream), "sync");
  return CACL_OK;
}

cacl_status cacl_step(cacl_ctx* c, int nsteps) {
  if (!c || nsteps < 0) return fail(c, CACL_ERR_ARG, "invalid step count");
  if (!ready(c)) return CACL_ERR_STATE;
  cacl::NvtxRange range("cacl_step");
  for (int s = 0; s < nsteps; ++s) {
    cudaGraphExec_t& gx = c->graph[c->fcur][c->pcur];
    if (!gx) CK(build_graph(c, c->fcur, c->pcur), "capture step");
    CK(cudaGraphLaunch(gx, c->stream), "launch step");
    c->fcur ^= 1;
    c->pcur ^= 1;
  }
  return CACL_OK;
}

namespace {
// Layout of a saved state: header, the current populations as stored, the
// current phi (with ghosts), u, the mass record (64 bytes), the wall angles.
struct StateHeader {
  char magic[8];
  int32_t nx, ny, nz, storage, comps, walls;
  int64_t nodes;
  int64_t reserved[3];
};
static_assert(sizeof(StateHeader) == 64, "64-byte header");
constexpr char STATE_MAGIC[8] = {'C', 'A', 'C', 'L', 'S', 'T', '0', '1'};
constexpr size_t MASS_SLOT = 64;
static_assert(sizeof(MassScalars) <= MASS_SLOT, "mass record fits its slot");

int64_t state_bytes(const cacl_ctx* c) {
  const int64_t N = c->g.N;
  return (int64_t)sizeof(StateHeader) +
         (int64_t)pop_comps(c->p.storage) * N * (int64_t)storage_bytes(c->p.storage) +
         4 * N * (int64_t)sizeof(float) + (int64_t)MASS_SLOT +
         (int64_t)c->wall_count * (int64_t)sizeof(float);
}
}  // namespace

int64_t cacl_state_bytes(const cacl_ctx* c) {
  if (!c || !c->has_geometry) return -1;
  return state_bytes(c);
}

cacl_status cacl_save_state(cacl_ctx* c, void* buf, int64_t bytes) {
  if (!c || !buf) return fail(c, CACL_ERR_ARG, "null argument");
  if (!ready(c)) return CACL_ERR_STATE;
  if (bytes < state_bytes(c)) return fail(c, CACL_ERR_ARG, "state buffer too small");
  const int64_t N = c->g.N;
  char* o = static_cast<char*>(buf);
  StateHeader h{};
  std::memcpy(h.magic, STATE_MAGIC, sizeof h.magic);
  h.nx = c->g.nx;
  h.ny = c->g.ny;
  h.nz = c->g.nz;
  h.storage = c->p.storage;
  h.comps = pop_comps(c->p.storage);
  h.walls = c->wall_count;
  h.nodes = N;
  std::memcpy(o, &h, sizeof h);
  o += sizeof h;
  const size_t fb = (size_t)h.comps * N * storage_bytes(c->p.storage);
  CK(cudaMemcpyAsync(o, c->f[c->fcur], fb, cudaMemcpyDeviceToHost, c->stream), "save f");
  o += fb;
  CK(cudaMemcpyAsync(o, c->phi[c->pcur], sizeof(float) * N, cudaMemcpyDeviceToHost,
                     c->stream), "save phi");
  o += sizeof(float) * N;
  CK(cudaMemcpyAsync(o, c->u, sizeof(float) * 3 * N, cudaMemcpyDeviceToHost, c->stream),
     "save u");
  o += sizeof(float) * 3 * N;
  std::memset(o, 0, MASS_SLOT);
  CK(cudaMemcpyAsync(o, c->mass, sizeof(MassScalars), cudaMemcpyDeviceToHost, c->stream),
     "save mass");
  o += MASS_SLOT;
  if (c->wall_count > 0)
    CK(cudaMemcpyAsync(o, c->w_theta, sizeof(float) * c->wall_count,
                       cudaMemcpyDeviceToHost, c->stream), "save angles");
  CK(cudaStreamSynchronize(c->stream), "sync");
  return CACL_OK;
}

cacl_status cacl_load_state(cacl_ctx* c, const void* buf, int64_t bytes) {
  if (!c || !buf) return fail(c, CACL_ERR_ARG, "null argument");
  if (!c->has_geometry) return fail(c, CACL_ERR_STATE, "set_geometry first");
  if (bytes < (int64_t)sizeof(StateHeader)) return fail(c, CACL_ERR_ARG, "no state header");
  StateHeader h;
  std::memcpy(&h, buf, sizeof h);
  if (std::memcmp(h.magic, STATE_MAGIC, sizeof h.magic) != 0)
    return fail(c, CACL_ERR_ARG, "not a saved state");
  if (h.nx != c->g.nx || h.ny != c->g.ny || h.nz != c->g.nz || h.storage != c->p.storage ||
      h.comps != pop_comps(c->p.storage) || h.walls != c->wall_count || h.nodes != c->g.N)
    return fail(c, CACL_ERR_ARG, "saved state of another grid, storage or geometry");
  if (bytes < state_bytes(c)) return fail(c, CACL_ERR_ARG, "state buffer too small");
  const int64_t N = c->g.N;
  const char* o = static_cast<const char*>(buf) + sizeof h;
  const size_t fb = (size_t)h.comps * N * storage_bytes(c->p.storage);
  CK(cudaMemcpyAsync(c->f[0], o, fb, cudaMemcpyHostToDevice, c->stream), "load f");
  o += fb;
  for (int i = 0; i < 2; ++i)
    CK(cudaMemcpyAsync(c->phi[i], o, sizeof(float) * N, cudaMemcpyHostToDevice,
                       c->stream), "load phi");
  o += sizeof(float) * N;
  CK(cudaMemcpyAsync(c->u, o, sizeof(float) * 3 * N, cudaMemcpyHostToDevice, c->stream),
     "load u");
  o += sizeof(float) * 3 * N;
  CK(cudaMemsetAsync(c->a, 0, sizeof(float) * 3 * N, c->stream), "zero a");
  CK(cudaMemcpyAsync(c->mass, o, sizeof(MassScalars), cudaMemcpyHostToDevice, c->stream),
     "load mass");
  o += MASS_SLOT;
  CK(cudaStreamSynchronize(c->stream), "sync");
  c->fcur = 0;
  c->pcur = 0;
  c->has_fields = true;
  if (c->wall_count > 0) {
    const cacl_status st = cacl_set_wall_angles(c, reinterpret_cast<const float*>(o));
    if (st != CACL_OK) return st;
  }
  return CACL_OK;
}

cacl_status cacl_inject_wait_timeout(cacl_ctx* c) {
  if (!c) return CACL_ERR_ARG;
  if (!c->ticket) return fail(c, CACL_ERR_STATE, "context without device state");
  const unsigned one = 1u;
  CK(cudaMemcpyAsync(c->ticket + 1, &one, sizeof one, cudaMemcpyHostToDevice, c->stream),
     "inject");
  CK(cudaStreamSynchronize(c->stream), "sync");
  return CACL_OK;
}

cacl_status cacl_inject_copy_stall(cacl_ctx* c, int on) {
  if (!c) return CACL_ERR_ARG;
  if (!c->ticket) return fail(c, CACL_ERR_STATE, "context without device state");
  const unsigned v = on ? 1u : 0u;
  CK(cudaMemcpyAsync(c->ticket + 2, &v, sizeof v, cudaMemcpyHostToDevice, c->stream),
     "inject");
  CK(cudaStreamSynchronize(c->stream), "sync");
  return CACL_OK;
}

cacl_status cacl_ghost_update(cacl_ctx* c) {
  if (!ready(c)) return c ? CACL_ERR_STATE : CACL_ERR_ARG;
  CK(launch_ghost(c, c->phi[c->pcur]), "ghost update");
  return CACL_OK;
}

cacl_status cacl_lb_collide(cacl_ctx* c) {
  if (!ready(c)) return c ? CACL_ERR_STATE : CACL_ERR_ARG;
  CK(launch_lb(c, c->f[c->fcur], c->f[1 - c->fcur], c->phi[c->pcur]),
     "collide-stream");
  c->fcur ^= 1;
  return CACL_OK;
}

cacl_status cacl_phase_update(cacl_ctx* c) {
  if (!ready(c)) return c ? CACL_ERR_STATE : CACL_ERR_ARG;
  CK(launch_compressive(c, c->phi[c->pcur]), "compressive vector");
  CK(launch_phase(c, c->phi[c->pcur], c->phi[1 - c->pcur]), "phase update");
  c->pcur ^= 1;
  return CACL_OK;
}

cacl_status cacl_volume_correct(cacl_ctx* c) {
  if (!ready(c)) return c ? CACL_ERR_STATE : CACL_ERR_ARG;
  CK(launch_correct(c, c->phi[c->pcur]), "volume correction");
  return CACL_OK;
}

cacl_status cacl_get_fields(cacl_ctx* c, float* phi, float* u, float* pstar,
                            int device_ptrs) {
  if (!ready(c)) return c ? CACL_ERR_STATE : CACL_ERR_ARG;
  const int64_t N = c->g.N;
  const cudaMemcpyKind kind =
      device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (phi)
    CK(cudaMemcpyAsync(phi, c->phi[c->pcur], sizeof(float) * N, kind, c->stream),
       "copy phi");
  if (u) CK(cudaMemcpyAsync(u, c->u, sizeof(float) * 3 * N, kind, c->stream), "copy u");
  if (pstar) {
    auto pst = [&](float* dst) {
      return c->p.storage == CACL_F32_MOMENTS
                 ? launch_moments_expand(c, c->f[c->fcur], nullptr, dst)
                 : launch_pstar(c, c->f[c->fcur], dst);
    };
    if (device_ptrs) {
      CK(pst(pstar), "p*");
    } else {
      float* tmp = nullptr;
      CK(cudaMalloc(&tmp, sizeof(float) * N), "alloc p*");
      cudaError_t e = pst(tmp);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(pstar, tmp, sizeof(float) * N,
                            cudaMemcpyDeviceToHost, c->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
      cudaFree(tmp);
      if (e != cudaSuccess) return cuda_fail(c, e, "p*");
    }
  }
  if (!device_ptrs) CK(cudaStreamSynchronize(c->stream), "sync");
  return CACL_OK;
}

cacl_status cacl_get_populations(cacl_ctx* c, float* f, int device_ptrs) {
  if (!ready(c)) return c ? CACL_ERR_STATE : CACL_ERR_ARG;
  if (!f) return fail(c, CACL_ERR_ARG, "null argument");
  const size_t bytes = sizeof(float) * Q * c->g.N;
  if (c->p.storage == CACL_F32) {
    CK(cudaMemcpyAsync(f, c->f[c->fcur], bytes,
                       device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                       c->stream), "copy f");
  } else if (device_ptrs) {
    if (c->p.storage == CACL_F32_MOMENTS)
      CK(launch_moments_expand(c, c->f[c->fcur], f, nullptr), "expand moments");
    else
      CK(launch_from_storage(c, c->f[c->fcur], f), "decode f");
  } else {
    float* tmp = nullptr;
    CK(cudaMalloc(&tmp, bytes), "alloc f staging");
    cudaError_t e = c->p.storage == CACL_F32_MOMENTS
                        ? launch_moments_expand(c, c->f[c->fcur], tmp, nullptr)
                        : launch_from_storage(c, c->f[c->fcur], tmp);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(f, tmp, bytes, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(tmp);
    if (e != cudaSuccess) return cuda_fail(c, e, "copy f");
  }
  if (!device_ptrs) CK(cudaStreamSynchronize(c->stream), "sync");
  return CACL_OK;
}

cacl_status cacl_get_wall_list(cacl_ctx* c, int32_t* idx, int8_t* qstar,
                               int16_t* ntilde6, float* nw, int32_t* count) {
  if (!c || !count) return fail(c, CACL_ERR_ARG, "null argument");
  if (!c->has_geometry) return fail(c, CACL_ERR_STATE, "set_geometry first");
  const int W = c->wall_count;
  *count = W;
  if (W == 0) return CACL_OK;
  if (idx)
    CK(cudaMemcpyAsync(idx, c->w_idx, 4 * W, cudaMemcpyDeviceToHost, c->stream),
       "copy idx");
  if (qstar)
    CK(cudaMemcpyAsync(qstar, c->w_q, W, cudaMemcpyDeviceToHost, c->stream),
       "copy qstar");
  std::vector<int16_t> n6(ntilde6 ? 3 * W : 0);
  std::vector<float> nwv(nw ? 3 * W : 0);
  if (ntilde6)
    CK(cudaMemcpyAsync(n6.data(), c->w_n6, 2 * 3 * W, cudaMemcpyDeviceToHost,
                       c->stream), "copy n6");
  if (nw)
    CK(cudaMemcpyAsync(nwv.data(), c->w_nw, 4 * 3 * W, cudaMemcpyDeviceToHost,
                       c->stream), "copy nw");
  CK(cudaStreamSynchronize(c->stream), "sync");
  for (int w = 0; w < W; ++w)
    for (int a = 0; a < 3; ++a) {
      if (ntilde6) ntilde6[3 * w + a] = n6[a * W + w];
      if (nw) nw[3 * w + a] = nwv[a * W + w];
    }
  return CACL_OK;
}

cacl_status cacl_get_mass(cacl_ctx* c, double* m_ref, double* m_star,
                          double* w_sum, double* lambda) {
  if (!ready(c)) return c ? CACL_ERR_STATE : CACL_ERR_ARG;
  MassScalars ms;
  CK(cudaMemcpyAsync(&ms, c->mass, sizeof(ms), cudaMemcpyDeviceToHost, c->stream),
     "copy mass");
  CK(cudaStreamSynchronize(c->stream), "sync");
  if (m_ref) *m_ref = ms.m_ref;
  if (m_star) *m_star = ms.m_star;
  if (w_sum) *w_sum = ms.w_sum;
  if (lambda) *lambda = ms.lambda;
  return CACL_OK;
}

cacl_status cacl_check_finite(cacl_ctx* c) {
  if (!ready(c)) return c ? CACL_ERR_STATE : CACL_ERR_ARG;
  int bad = 0;
  unsigned waited = 0;
  CK(cudaMemsetAsync(c->bad_flag, 0, sizeof(int), c->stream), "memset");
  CK(launch_check_finite(c, c->phi[c->pcur], c->bad_flag), "finite check");
  CK(cudaMemcpyAsync(&bad, c->bad_flag, sizeof(int), cudaMemcpyDeviceToHost,
                     c->stream), "copy flag");
  CK(cudaMemcpyAsync(&waited, c->ticket + 1, sizeof(unsigned),
                     cudaMemcpyDeviceToHost, c->stream), "copy flag");
  CK(cudaStreamSynchronize(c->stream), "sync");
  if (waited) return fail(c, CACL_ERR_TIMEOUT, "a wait for asynchronous copies gave up");
  if (bad) return fail(c, CACL_ERR_DIVERGED, "non-finite phi or u");
  return CACL_OK;
}

cacl_status cacl_set_option(cacl_ctx* c, int option, int value) {
  if (!c) return CACL_ERR_ARG;
  if (option == CACL_OPT_PHASE_TILE) {
    if (value < 0 || value > 3) return fail(c, CACL_ERR_ARG, "unknown phase tile");
    if (c->phase_variant != value) drop_graphs(c);
    c->phase_variant = value;
    return CACL_OK;
  }
  if (option == CACL_OPT_LB_PIPE) {
    if (value < 0 || value > 3) return fail(c, CACL_ERR_ARG, "unknown collide pipeline");
    if (value != 0 && c->p.storage == CACL_F32_MOMENTS)
      return fail(c, CACL_ERR_ARG, "the moment form has one collide-stream kernel");
    const int pf = 16 / (int)storage_bytes(c->p.storage);
    if (value == 1 && (c->g.nx % pf != 0 || c->g.nx % 4 != 0))
      return fail(c, CACL_ERR_ARG, "staged collide-stream needs nx a multiple of 16 bytes");
    if (c->lb_pipe != value) drop_graphs(c);
    c->lb_pipe = value;
    return CACL_OK;
  }
  if (option == CACL_OPT_PHASE_PIPE) {
    if (value < 0 || value > 3) return fail(c, CACL_ERR_ARG, "unknown phase pipeline");
    if (value >= 2 && c->g.nz < 2)
      return fail(c, CACL_ERR_ARG, "copy-staged phase update needs nz >= 2");
    if (value == 3 && c->g.nx % 4 != 0)
      return fail(c, CACL_ERR_ARG, "2 x 2 phase update needs nx % 4 == 0");
    if (c->phase_pipe != value) drop_graphs(c);
    c->phase_pipe = value;
    return CACL_OK;
  }
  if (option == CACL_OPT_INDEX64) {
    if (value != 0 && value != 1) return fail(c, CACL_ERR_ARG, "index64 is 0 or 1");
    if (c->index64 != (value != 0)) {
      drop_graphs(c);
      c->index64 = value != 0;
      CK(lb_init(c), "collide-stream setup");
    }
    return CACL_OK;
  }
  return fail(c, CACL_ERR_ARG, "unknown option");
}

cacl_status cacl_get_info(const cacl_ctx* c, int64_t* nodes,
                          int64_t* device_bytes, int32_t* wall_count) {
  if (!c) return CACL_ERR_ARG;
  if (nodes) *nodes = c->g.N;
  if (device_bytes) *device_bytes = c->device_bytes;
  if (wall_count) *wall_count = c->wall_count;
  return CACL_OK;
}

}  // extern "C"
