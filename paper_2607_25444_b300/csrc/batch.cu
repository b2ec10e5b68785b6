// batch.cu -- many CAC-LB cases of uneven size advanced together: every
// stage of the step is a grid-strided launch over a work-list that spans
// all cases of one kernel shape (the collide-stream one launch per node
// width, the phi update one per staging pipeline, as each case would run
// alone), the step is captured in a CUDA graph, and an autotuner picks the
// collide-stream block size and the phi-update tile.
//
// Each case keeps its own context (cacl_ctx) for set-up, queries and its
// device buffers; the batch holds a device table of per-case descriptors and
// the prefix-summed work-lists. Cases advance in lockstep, so one (f, phi)
// parity holds for all of them.
#include <vector>

#include "cacl_internal.cuh"

using namespace cacl;

struct cacl_batch {
  std::vector<cacl_ctx*> cases;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int storage = CACL_F32;
  int lb_variant = 1;
  int phase_variant = 2;
  CaseDesc* d_cases = nullptr;
  int* d_starts = nullptr;  // NLISTS lists of ncases + 1 starts
  // collide-stream: the cases of one, two and four nodes per thread
  // (wl_lb[w], w = 0, 1, 2); phi update: the cases of width class w staged
  // through registers (wl_ph[0][w]), by 16-byte copies with two nodes per
  // thread (wl_ph[1][w]), with 2 x 2 (wl_ph[2][w]) and by element copies
  // with two nodes per thread (wl_ph[3][w]); each as the case would run
  // alone
  WorkList wl_lb[3]{}, wl_ph[4][3]{}, wl_ghost{}, wl_corr{};
  int grid_lb[3] = {0, 0, 0};
  int grid_ph[4][3] = {};
  int grid_ghost = 0, grid_corr = 0;
  // the width classes touch disjoint cases: in the captured step each runs
  // its collide-stream and phi update as a branch of its own (side streams
  // joined by events), between the ghost update and the correction
  cudaStream_t side[2] = {nullptr, nullptr};
  cudaEvent_t ev_fork = nullptr, ev_join[2] = {nullptr, nullptr};
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  bool plan_ok = false;
  std::vector<int> geom_version;  // of each case when the plan was built
  std::vector<int> phase_nb;      // phase-update blocks of each case
  std::string err;
};

namespace {

constexpr int NLISTS = 17;  // ghost, correction, 3 collide-stream, 4 x 3 phi
constexpr int LB_WIDTH[3] = {1, 2, 4};

cacl_status bfail(cacl_batch* b, cacl_status st, const std::string& msg) {
  if (b) b->err = msg;
  return st;
}

#define BCK(expr, where)                                                   \
  do {                                                                     \
    cudaError_t e_ = (expr);                                               \
    if (e_ != cudaSuccess)                                                 \
      return bfail(b, CACL_ERR_CUDA, std::string(where) + ": " +          \
                                         cudaGetErrorString(e_));          \
  } while (0)

void drop_batch_graphs(cacl_batch* b) {
  for (auto& gx : b->graph) {
    if (gx) cudaGraphExecDestroy(gx);
    gx = nullptr;
  }
}

int sm_count() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

// Per-case descriptors and work-lists for the current launch shapes.
cacl_status build_plan(cacl_batch* b) {
  const int nc = (int)b->cases.size();
  std::vector<CaseDesc> desc(nc);
  b->phase_nb.assign(nc, 0);
  b->geom_version.assign(nc, -1);
  std::vector<int> starts(NLISTS * (nc + 1), 0);
  auto list = [&](int k) { return starts.data() + k * (nc + 1); };
  int* s_gh = list(0);
  int* s_cr = list(1);
  int* s_lb[3] = {list(2), list(3), list(4)};
  int* s_ph[4][3];
  for (int q = 0; q < 4; ++q)
    for (int w = 0; w < 3; ++w) s_ph[q][w] = list(5 + 3 * q + w);
  const int row = lb_batch_row(b->lb_variant);
  int ty = 16, zc = 16;
  phase_tile(b->phase_variant, ty, zc);
  for (int i = 0; i < nc; ++i) {
    cacl_ctx* c = b->cases[i];
    CaseDesc& d = desc[i];
    d.g = c->g;
    d.k = c->k;
    d.f[0] = c->f[0];
    d.f[1] = c->f[1];
    d.phi[0] = c->phi[0];
    d.phi[1] = c->phi[1];
    d.u = c->u;
    d.a = c->a;
    d.flags = c->flags;
    d.W = c->wall_count;
    d.w_idx = c->w_idx;
    d.w_donor = c->w_donor;
    d.w_q = c->w_q;
    d.w_nw = c->w_nw;
    d.w_cot = c->w_cot;
    d.w_g = c->w_g;
    d.partials = c->partials;
    d.mass = c->mass;
    const int nbx = (c->g.nx + 31) / 32, nby = (c->g.ny + ty - 1) / ty,
              nbz = (c->g.nz + zc - 1) / zc;
    d.phase_nb = nbx * nby * nbz;
    b->phase_nb[i] = d.phase_nb;
    b->geom_version[i] = c->geom_version;
    if (d.phase_nb > c->part_blocks)
      return bfail(b, CACL_ERR_STATE, "partial-sum storage too small");
    // nodes per thread of the collide-stream: the kernel the case gets alone
    // (four-node for 16-bit populations, two-node, one-node), for both
    // population buffers and both phi buffers
    const bool quad = lb_quad_ok(c, c->f[0], c->f[1], c->phi[0]) &&
                      lb_quad_ok(c, c->f[1], c->f[0], c->phi[1]);
    const bool pair = lb_pair_ok(c, c->f[0], c->f[1], c->phi[0]) &&
                      lb_pair_ok(c, c->f[1], c->f[0], c->phi[1]);
    d.lbw = quad ? 4 : (pair ? 2 : 1);
    const int wc = quad ? 2 : (pair ? 1 : 0);
    for (int w = 0; w < 3; ++w) {
      const int64_t units = c->g.N / d.lbw;
      s_lb[w][i + 1] = s_lb[w][i] + (w == wc ? (int)((units + row - 1) / row) : 0);
    }
    const bool copy = c->phase_pipe != 1 &&
                      phase_copy_ok(c->g, c->phi[0], c->phi[1], c->a, c->u, c->flags);
    const bool copy_u = c->phase_pipe != 1 && !copy && c->g.nz >= 2;
    const int pipe = copy_u ? 3 : (!copy ? 0 : (c->phase_pipe == 2 ? 1 : 2));
    for (int q = 0; q < 4; ++q)
      for (int w = 0; w < 3; ++w)
        s_ph[q][w][i + 1] = s_ph[q][w][i] + (q == pipe && w == wc ? d.phase_nb : 0);
    s_gh[i + 1] = s_gh[i] + (c->wall_count + ghost_batch_block() - 1) /
                                ghost_batch_block();
    const int64_t per = correct_batch_nodes();
    s_cr[i + 1] = s_cr[i] + (int)((c->g.N + per - 1) / per);
  }
  BCK(cudaMemcpyAsync(b->d_cases, desc.data(), sizeof(CaseDesc) * nc,
                      cudaMemcpyHostToDevice, b->stream), "upload cases");
  BCK(cudaMemcpyAsync(b->d_starts, starts.data(), sizeof(int) * starts.size(),
                      cudaMemcpyHostToDevice, b->stream), "upload work-lists");
  BCK(cudaStreamSynchronize(b->stream), "sync");
  auto dlist = [&](int k) { return b->d_starts + k * (nc + 1); };
  b->wl_ghost = {dlist(0), nc, s_gh[nc]};
  b->wl_corr = {dlist(1), nc, s_cr[nc]};
  for (int w = 0; w < 3; ++w) b->wl_lb[w] = {dlist(2 + w), nc, s_lb[w][nc]};
  for (int q = 0; q < 4; ++q)
    for (int w = 0; w < 3; ++w)
      b->wl_ph[q][w] = {dlist(5 + 3 * q + w), nc, s_ph[q][w][nc]};
  // persistent grids: as many blocks as stay resident, at most the work
  const int sms = sm_count();
  auto grid_for = [&](int total, int per_sm) {
    const int cap = sms * (per_sm > 0 ? per_sm : 1);
    return total < cap ? (total > 0 ? total : 1) : cap;
  };
  for (int w = 0; w < 3; ++w)
    b->grid_lb[w] =
        b->wl_lb[w].total == 0
            ? 0
            : (lb_batch_persistent(b->lb_variant)
                   ? grid_for(b->wl_lb[w].total,
                              lb_batch_occupancy(b->storage, LB_WIDTH[w], b->lb_variant))
                   : b->wl_lb[w].total);
  const int occ[4] = {phase_batch_occupancy(b->phase_variant),
                      phase_batch_copy_occupancy(b->phase_variant, true),
                      phase_batch_quad_occupancy(b->phase_variant),
                      phase_batch_copy_occupancy(b->phase_variant, false)};
  for (int q = 0; q < 4; ++q)
    for (int w = 0; w < 3; ++w) b->grid_ph[q][w] = grid_for(b->wl_ph[q][w].total, occ[q]);
  b->grid_ghost = grid_for(b->wl_ghost.total, 8);
  b->grid_corr = grid_for(b->wl_corr.total, 8);
  b->plan_ok = true;
  return CACL_OK;
}

// phi-update launch of pipeline q (0 registers, 1 two-node 16-byte copies,
// 2 2 x 2, 3 two-node element copies)
cudaError_t launch_phase_pipe(const CaseDesc* cases, WorkList wl, int q, int variant,
                              int grid, int pc, cudaStream_t st) {
  switch (q) {
    case 0: return launch_phase_batch(cases, wl, variant, grid, pc, st);
    case 1: return launch_phase_batch_copy(cases, wl, variant, grid, pc, true, st);
    case 3: return launch_phase_batch_copy(cases, wl, variant, grid, pc, false, st);
    default: return launch_phase_batch_quad(cases, wl, variant, grid, pc, st);
  }
}

cudaError_t enqueue_batch_step(cacl_batch* b, int par) {
  cudaError_t e;
  if ((e = launch_ghost_batch(b->d_cases, b->wl_ghost, b->grid_ghost, par,
                              b->stream)) != cudaSuccess)
    return e;
  // one branch per collide-stream width class: its collide-stream, then the
  // phi update of the same cases; the first branch on the batch's stream
  if ((e = cudaEventRecord(b->ev_fork, b->stream)) != cudaSuccess) return e;
  int nside = 0;
  bool main_used = false;
  for (int w = 0; w < 3; ++w) {
    if (b->wl_lb[w].total == 0) continue;
    cudaStream_t sw = b->stream;
    if (main_used) {
      sw = b->side[nside];
      if ((e = cudaStreamWaitEvent(sw, b->ev_fork, 0)) != cudaSuccess) return e;
    }
    if ((e = launch_lb_batch(b->d_cases, b->wl_lb[w], b->storage, LB_WIDTH[w],
                             b->lb_variant, b->grid_lb[w], par, par, sw)) != cudaSuccess)
      return e;
    for (int q = 0; q < 4; ++q)
      if (b->wl_ph[q][w].total > 0 &&
          (e = launch_phase_pipe(b->d_cases, b->wl_ph[q][w], q, b->phase_variant,
                                 b->grid_ph[q][w], par, sw)) != cudaSuccess)
        return e;
    if (main_used) {
      if ((e = cudaEventRecord(b->ev_join[nside], sw)) != cudaSuccess) return e;
      ++nside;
    }
    main_used = true;
  }
  for (int k = 0; k < nside; ++k)
    if ((e = cudaStreamWaitEvent(b->stream, b->ev_join[k], 0)) != cudaSuccess) return e;
  return launch_correct_batch(b->d_cases, (int)b->cases.size(), b->wl_corr,
                              b->grid_corr, par, b->stream);
}

cudaError_t build_batch_graph(cacl_batch* b, int par) {
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  const cudaError_t el = enqueue_batch_step(b, par);
  e = cudaStreamEndCapture(b->stream, &graph);
  if (el != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return el;
  }
  if (e != cudaSuccess) return e;
  e = cudaGraphInstantiate(&b->graph[par], graph, 0);
  cudaGraphDestroy(graph);
  return e;
}

}  // namespace

extern "C" {

cacl_status cacl_batch_create(const cacl_params* params, int ncases,
                              void* stream, cacl_batch** out) {
  if (!params || !out || ncases < 1) return CACL_ERR_ARG;
  *out = nullptr;
  for (int i = 1; i < ncases; ++i)
    if (params[i].storage != params[0].storage) return CACL_ERR_ARG;
  if (params[0].storage == CACL_F32_MOMENTS) return CACL_ERR_ARG;  // population forms only
  for (int i = 0; i < ncases; ++i) {  // the batched kernels index with 32 bits
    const int64_t n = (int64_t)params[i].nx * params[i].ny * params[i].nz;
    if (n > 0 && (int64_t)Q * n >= (int64_t)INT32_MAX) return CACL_ERR_TOO_LARGE;
  }
  cacl_batch* b = new cacl_batch();
  b->storage = params[0].storage;
  if (stream) {
    b->stream = (cudaStream_t)stream;
  } else {
    if (cudaStreamCreate(&b->stream) != cudaSuccess) {
      delete b;
      return CACL_ERR_CUDA;
    }
    b->own_stream = true;
  }
  for (int i = 0; i < ncases; ++i) {
    cacl_ctx* c = nullptr;
    const cacl_status st = cacl_create(&params[i], b->stream, &c);
    if (st != CACL_OK) {
      cacl_batch_destroy(b);
      return st;
    }
    b->cases.push_back(c);
  }
  for (int k = 0; k < 2; ++k) {
    if (cudaStreamCreateWithFlags(&b->side[k], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_join[k], cudaEventDisableTiming) != cudaSuccess) {
      cacl_batch_destroy(b);
      return CACL_ERR_CUDA;
    }
  }
  if (cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) != cudaSuccess) {
    cacl_batch_destroy(b);
    return CACL_ERR_CUDA;
  }
  if (cudaMalloc(&b->d_cases, sizeof(CaseDesc) * ncases) != cudaSuccess ||
      cudaMalloc(&b->d_starts, sizeof(int) * NLISTS * (ncases + 1)) != cudaSuccess) {
    cacl_batch_destroy(b);
    return CACL_ERR_CUDA;
  }
  *out = b;
  return CACL_OK;
}

void cacl_batch_destroy(cacl_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  drop_batch_graphs(b);
  for (cacl_ctx* c : b->cases) cacl_destroy(c);
  if (b->d_cases) cudaFree(b->d_cases);
  if (b->d_starts) cudaFree(b->d_starts);
  for (int k = 0; k < 2; ++k) {
    if (b->side[k]) cudaStreamDestroy(b->side[k]);
    if (b->ev_join[k]) cudaEventDestroy(b->ev_join[k]);
  }
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

const char* cacl_batch_last_error(const cacl_batch* b) {
  return b ? b->err.c_str() : "";
}

cacl_status cacl_batch_case(cacl_batch* b, int i, cacl_ctx** out) {
  if (!b || !out || i < 0 || i >= (int)b->cases.size())
    return bfail(b, CACL_ERR_ARG, "no such case");
  *out = b->cases[i];
  return CACL_OK;
}

cacl_status cacl_batch_set_option(cacl_batch* b, int lb_variant,
                                  int phase_variant) {
  if (!b || lb_variant < 0 || lb_variant >= LB_BATCH_VARIANTS ||
      phase_variant < 0 || phase_variant > 3)
    return bfail(b, CACL_ERR_ARG, "unknown launch shape");
  b->lb_variant = lb_variant;
  b->phase_variant = phase_variant;
  b->plan_ok = false;
  drop_batch_graphs(b);
  return CACL_OK;
}

cacl_status cacl_batch_step(cacl_batch* b, int nsteps) {
  if (!b || nsteps < 0) return bfail(b, CACL_ERR_ARG, "invalid step count");
  NvtxRange range("cacl_batch_step");
  const int par = b->cases[0]->fcur;
  for (cacl_ctx* c : b->cases) {
    if (!c->has_fields)
      return bfail(b, CACL_ERR_STATE, "every case needs geometry and fields");
    if (c->fcur != par || c->pcur != par)
      return bfail(b, CACL_ERR_STATE, "cases are not in lockstep");
  }
  for (size_t i = 0; i < b->cases.size() && b->plan_ok; ++i)
    if (b->geom_version[i] != b->cases[i]->geom_version) b->plan_ok = false;
  if (!b->plan_ok) {
    drop_batch_graphs(b);
    const cacl_status st = build_plan(b);
    if (st != CACL_OK) return st;
  }
  int p = par;
  for (int s = 0; s < nsteps; ++s) {
    if (!b->graph[p]) BCK(build_batch_graph(b, p), "capture batch step");
    BCK(cudaGraphLaunch(b->graph[p], b->stream), "launch batch step");
    p ^= 1;
  }
  for (size_t i = 0; i < b->cases.size(); ++i) {
    b->cases[i]->fcur = p;
    b->cases[i]->pcur = p;
    b->cases[i]->phase_nblocks = b->phase_nb[i];
  }
  return CACL_OK;
}

cacl_status cacl_batch_autotune(cacl_batch* b, int steps, int* lb_variant,
                                int* phase_variant, float* best_ms) {
  if (!b || steps < 1) return bfail(b, CACL_ERR_ARG, "invalid step count");
  cudaEvent_t e0, e1;
  BCK(cudaEventCreate(&e0), "event");
  BCK(cudaEventCreate(&e1), "event");
  float best = 1e30f;
  int bl = b->lb_variant, bp = b->phase_variant;
  for (int lv = 0; lv < LB_BATCH_VARIANTS; ++lv) {
    for (int pv = 0; pv < 4; ++pv) {
      cacl_status st = cacl_batch_set_option(b, lv, pv);
      if (st == CACL_OK) st = cacl_batch_step(b, 1);  // capture, warm
      if (st != CACL_OK) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return st;
      }
      cudaEventRecord(e0, b->stream);
      st = cacl_batch_step(b, steps);
      cudaEventRecord(e1, b->stream);
      if (st != CACL_OK) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return st;
      }
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      ms /= (float)steps;
      if (ms < best) {
        best = ms;
        bl = lv;
        bp = pv;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const cacl_status st = cacl_batch_set_option(b, bl, bp);
  if (lb_variant) *lb_variant = bl;
  if (phase_variant) *phase_variant = bp;
  if (best_ms) *best_ms = best;
  return st;
}

}  // extern "C"
