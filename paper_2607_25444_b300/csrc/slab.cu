// slab.cu -- one z slab of a decomposition of the grid along z, for running
// one problem on several GPUs (one slab per GPU) or for checking the
// decomposition on one GPU.
//
// A slab owning the global planes [z0, z0 + nz) is an ordinary context of
// nz + 4 planes, periodic in z: planes 0-1 and nz+2 .. nz+3 are halos that
// hold copies of the neighbouring slabs' planes (z0 - 2, z0 - 1 and
// z0 + nz, z0 + nz + 1, wrapped around the global grid). The reach of the
// step fixes the halo: the ghost update reads phi two planes from a wall
// node, the collide-stream pulls populations and reads phi one plane away,
// the phi update reads phi two planes and u, a one plane away. One step of
// the decomposition is, on every slab, with halo exchanges between:
//   ghost update; exchange phi (2 planes, ghosts included);
//   collide-stream; exchange f* (1 plane, 27 populations) and u, a (1 plane);
//   phi update over the interior planes only (block partial sums);
//   gather every slab's partial sums in slab order; correction with lambda
//   from them (the same fixed-order sum an undivided context forms);
//   exchange phi (2 planes) for the next step's ghost update.
// Halo planes are computed on as well, with wrapped data, and overwritten
// by the exchanges. When every slab's interior starts on a multiple of the
// phi update's tile depth (32 planes with the default tile) the gathered
// partial sums are those of an undivided context in its order, and the
// correction's rounding key uses global node indices, so the decomposition
// is bit-identical to the undivided step.
#include "cacl_internal.cuh"

using namespace cacl;

namespace {

constexpr int HALO = 2;

cacl_status sfail(cacl_ctx* c, cacl_status st, const char* m) {
  if (c) c->err = m;
  return st;
}

// planes and components moved by one exchange of `field`
void field_shape(const cacl_ctx* c, int field, int& planes, int& comps, size_t& esize) {
  switch (field) {
    case CACL_SLAB_PHI: planes = 2; comps = 1; esize = 4; break;
    case CACL_SLAB_F:
      planes = 1;
      comps = pop_comps(c->p.storage);
      esize = storage_bytes(c->p.storage);
      break;
    default: planes = 1; comps = 6; esize = 4; break;  // u (3), a (3)
  }
}

// base pointer and component stride (elements) of component j of `field`
void* field_comp(cacl_ctx* c, int field, int j, size_t esize) {
  const int64_t N = c->g.N;
  switch (field) {
    case CACL_SLAB_PHI: return c->phi[c->pcur];
    case CACL_SLAB_F: return (char*)c->f[c->fcur] + (size_t)j * N * esize;
    default:
      return j < 3 ? (void*)(c->u + (size_t)j * N) : (void*)(c->a + (size_t)(j - 3) * N);
  }
}

}  // namespace

extern "C" {

cacl_status cacl_slab_create(const cacl_params* global, int z0, int nz,
                             void* stream, cacl_ctx** out) {
  if (!global || !out) return CACL_ERR_ARG;
  *out = nullptr;
  if (nz < 1 || z0 < 0 || z0 + nz > global->nz) return CACL_ERR_ARG;
  cacl_params p = *global;
  p.nz = nz + 2 * HALO;
  p.periodic[2] = 1;  // the halos are fed by exchanges
  cacl_ctx* c = nullptr;
  const cacl_status st = cacl_create(&p, stream, &c);
  if (st != CACL_OK) return st;
  const int64_t nxy = (int64_t)p.nx * p.ny;
  c->zbase = HALO;
  c->zlim = HALO + nz;
  c->ext_finalize = true;
  c->node_offset = nxy * (int64_t)(z0 - HALO);
  c->slab_z0 = z0;
  c->slab_nz = nz;
  // the tile shape the undivided grid takes by default, so that the slabs'
  // tiles and partial sums match its own
  c->phase_variant = phase_default_variant(
      {global->nx, global->ny, global->nz,
       (int64_t)global->nx * global->ny * global->nz});
  *out = c;
  return CACL_OK;
}

cacl_status cacl_slab_stage(cacl_ctx* c, int stage) {
  if (!c) return CACL_ERR_ARG;
  if (!c->ext_finalize) return sfail(c, CACL_ERR_STATE, "not a slab context");
  if (!c->has_fields) return sfail(c, CACL_ERR_STATE, "set_fields first");
  cudaError_t e = cudaSuccess;
  switch (stage) {
    case CACL_SLAB_GHOST: e = launch_ghost(c, c->phi[c->pcur]); break;
    case CACL_SLAB_COLLIDE:
      e = launch_lb(c, c->f[c->fcur], c->f[1 - c->fcur], c->phi[c->pcur]);
      if (e == cudaSuccess) c->fcur ^= 1;
      break;
    case CACL_SLAB_PHASE:
      // the compressive vector is the one the collide-stream wrote
      e = launch_phase(c, c->phi[c->pcur], c->phi[1 - c->pcur]);
      if (e == cudaSuccess) c->pcur ^= 1;
      break;
    default: return sfail(c, CACL_ERR_ARG, "unknown slab stage");
  }
  if (e != cudaSuccess) {
    c->err = std::string("slab stage: ") + cudaGetErrorString(e);
    return CACL_ERR_CUDA;
  }
  return CACL_OK;
}

cacl_status cacl_slab_partials(cacl_ctx* c, double* dst, int* nblocks) {
  if (!c || !nblocks) return CACL_ERR_ARG;
  if (!c->ext_finalize) return sfail(c, CACL_ERR_STATE, "not a slab context");
  const int nb = c->phase_nblocks;
  *nblocks = nb;
  if (!dst) return CACL_OK;
  if (nb <= 0) return sfail(c, CACL_ERR_STATE, "no phi update since set_fields");
  cudaError_t e = cudaMemcpyAsync(dst, c->partials, sizeof(double) * nb,
                                  cudaMemcpyDeviceToDevice, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dst + nb, c->partials + nb, sizeof(double) * nb,
                        cudaMemcpyDeviceToDevice, c->stream);
  if (e != cudaSuccess) {
    c->err = std::string("slab partials: ") + cudaGetErrorString(e);
    return CACL_ERR_CUDA;
  }
  return CACL_OK;
}

cacl_status cacl_slab_correct(cacl_ctx* c, const double* all, int nb_total) {
  if (!c || !all || nb_total < 1) return CACL_ERR_ARG;
  if (!c->ext_finalize) return sfail(c, CACL_ERR_STATE, "not a slab context");
  cudaError_t e = launch_mass_from(c, all, nb_total);
  if (e == cudaSuccess) e = launch_correct(c, c->phi[c->pcur]);
  if (e != cudaSuccess) {
    c->err = std::string("slab correction: ") + cudaGetErrorString(e);
    return CACL_ERR_CUDA;
  }
  return CACL_OK;
}

cacl_status cacl_slab_halo(cacl_ctx* c, int field, int side, int direction,
                           void* buf) {
  if (!c || !buf) return CACL_ERR_ARG;
  if (!c->ext_finalize) return sfail(c, CACL_ERR_STATE, "not a slab context");
  if (field < CACL_SLAB_PHI || field > CACL_SLAB_UA || (side != 0 && side != 1) ||
      (direction != 0 && direction != 1))
    return sfail(c, CACL_ERR_ARG, "invalid halo request");
  int planes, comps;
  size_t es;
  field_shape(c, field, planes, comps, es);
  const int64_t nxy = (int64_t)c->g.nx * c->g.ny;
  const int nz = c->slab_nz;
  // interior planes next to the side (sent), halo planes on the side (received)
  const int zpack = side == 0 ? HALO : HALO + nz - planes;
  const int zhalo = side == 0 ? HALO - planes : HALO + nz;
  const size_t chunk = (size_t)planes * nxy * es;
  for (int j = 0; j < comps; ++j) {
    char* base = (char*)field_comp(c, field, j, es);
    char* b = (char*)buf + j * chunk;
    const cudaError_t e =
        direction == 0
            ? cudaMemcpyAsync(b, base + zpack * nxy * es, chunk, cudaMemcpyDeviceToDevice,
                              c->stream)
            : cudaMemcpyAsync(base + zhalo * nxy * es, b, chunk, cudaMemcpyDeviceToDevice,
                              c->stream);
    if (e != cudaSuccess) {
      c->err = std::string("slab halo: ") + cudaGetErrorString(e);
      return CACL_ERR_CUDA;
    }
  }
  return CACL_OK;
}

int64_t cacl_slab_halo_bytes(const cacl_ctx* c, int field) {
  if (!c || field < CACL_SLAB_PHI || field > CACL_SLAB_UA) return -1;
  int planes, comps;
  size_t es;
  field_shape(c, field, planes, comps, es);
  return (int64_t)planes * comps * c->g.nx * c->g.ny * (int64_t)es;
}

}  // extern "C"
