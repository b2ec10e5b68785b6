/*
 * cacl.h -- C ABI of the B300 (sm_103a) CAC-LB wetting step.
 *
 * One time step of the conservative Allen-Cahn lattice Boltzmann scheme with
 * the geometric wetting boundary condition of arXiv 2607.25444:
 *   1. ghost phi values at wall nodes from the reconstructed wall normal and
 *      a donor fluid node at the imposed contact angle (Sect. 2.2,
 *      Eqs. local_wall_normal .. contact_angle_localization, Algorithm 1);
 *   2. the D3Q27 pull collide-stream: third-order Hermite equilibrium,
 *      recursive regularisation, Guo forcing with the chemical-potential
 *      capillary force, the pressure and viscous corrections and gravity
 *      (Sect. 2.1, Eqs. lbe .. lap_iso);
 *   3. the conservative Allen-Cahn update with MUSCL-minmod advection,
 *      isotropic diffusion and the isotropic compressive divergence
 *      (Sect. 2.1.1, Eq. phi_update_muscl);
 *   4. the global volume correction over the interface band (Sect. 2.3,
 *      Eqs. tentative_phase_field_mass .. mass_corrected_phi).
 *
 * Conventions for every call:
 *   - Grid: nx * ny * nz nodes, node n = x + nx*(y + ny*z), x fastest.
 *   - Host pointers are read or written during the call only, never kept.
 *   - All device work is enqueued on the stream given to cacl_create (NULL =
 *     the legacy default stream). Calls that return data to host memory
 *     synchronise that stream before returning.
 *   - Every call returns a cacl_status. On error the context records a
 *     message, readable with cacl_last_error; the state is unchanged unless
 *     the message says otherwise.
 *   - Required order: cacl_create -> cacl_set_geometry ->
 *     [cacl_set_contact_angle] -> cacl_set_fields -> cacl_step ...
 *     A call out of order returns CACL_ERR_STATE.
 *   - The context owns all device memory it allocates; cacl_destroy frees it.
 *   - Errors of the CUDA runtime are returned as CACL_ERR_CUDA.
 */
#ifndef CACL_H
#define CACL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cacl_ctx cacl_ctx;

typedef enum {
  CACL_OK = 0,
  CACL_ERR_ARG = -1,       /* invalid argument or size */
  CACL_ERR_CUDA = -2,      /* CUDA runtime error */
  CACL_ERR_STATE = -3,     /* call out of the required order */
  CACL_ERR_GEOMETRY = -4,  /* non-periodic axis not closed by solid layers */
  CACL_ERR_DIVERGED = -5,  /* non-finite phi or u found by cacl_check_finite */
  CACL_ERR_TIMEOUT = -6,   /* a bounded device wait gave up (reported by
                              cacl_check_finite) */
  CACL_ERR_TOO_LARGE = -7  /* size above the fixed scratch of an
                              allocation-free entry point, or above the
                              32-bit indexing of a batch */
} cacl_status;

/* Storage of the populations; arithmetic is FP32 in every mode.
 *   CACL_F32           the 27 post-collision populations f*_q, FP32
 *   CACL_F16_SHIFTED   h_q = (f*_q - w_q p*_ref) / w_q with p*_ref = 0,
 *   CACL_BF16_SHIFTED  rounded to FP16 / BF16 (nearest even)
 *   CACL_F32_MOMENTS   the paper's thread-safe moment form (Sect. 2.1): each
 *                      node keeps the 17 coefficients of its post-collision
 *                      polynomial P (f*_q = w_q P(c_q)) in FP32, and the
 *                      collide-stream rebuilds the populations it pulls from
 *                      the neighbours' coefficients; bit-identical to
 *                      CACL_F32 at fluid nodes from a state at rest. Not
 *                      available to cacl_set_populations, the adjoint or
 *                      batches. */
typedef enum {
  CACL_F32 = 0,
  CACL_F16_SHIFTED = 1,
  CACL_BF16_SHIFTED = 2,
  CACL_F32_MOMENTS = 3
} cacl_storage;

/*
 * Problem statement (Sect. 2.1-2.3). All quantities in lattice units.
 *   width      interface thickness delta (Eq. kappa_delta); > 0
 *   mobility   interface diffusivity D; >= 0. kappa = 4 D / delta.
 *   sigma      surface tension; beta = 12 sigma/delta, kappa_phi = 3 sigma
 *              delta / 2 (Eq. Fcap)
 *   rho_l/g    densities of liquid (phi = 1) and gas (phi = 0)
 *   nu_l/g     kinematic viscosities; mu = rho nu mixes linearly
 *              (Eq. mu_mix_linear)
 *   gravity    g; the body force is F_ext = (rho(phi) - rho_g) g
 *   theta_deg  contact angle of every wall node until set_contact_angle
 *   eps_phi    band threshold of the volume correction weight chi
 *              (Eq. interface_weight_mass_correction), 0 < eps_phi < 1/2
 *   periodic   1 = periodic axis; 0 = axis closed by solid layers at 0 and
 *              n-1 (checked by cacl_set_geometry)
 */
typedef struct {
  int nx, ny, nz;
  int periodic[3];
  double width;
  double mobility;
  double sigma;
  double rho_l, rho_g;
  double nu_l, nu_g;
  double gravity[3];
  double theta_deg;
  double eps_phi;
  int storage; /* cacl_storage */
} cacl_params;

/* Validates *params and allocates the device state (populations x2, phi x2,
 * velocity, flags, reduction scratch) on the current CUDA device.
 * stream: a cudaStream_t or NULL. On success *out owns the state. */
cacl_status cacl_create(const cacl_params* params, void* stream,
                        cacl_ctx** out);

/* Frees everything the context owns. NULL is accepted. */
void cacl_destroy(cacl_ctx* ctx);

/* Text of the last error recorded on ctx ("" if none). */
const char* cacl_last_error(const cacl_ctx* ctx);

/* Occupancy (host, N bytes, 1 = solid) -> flags, wall list (Sect. 2.2,
 * Eqs. local_wall_normal .. donor_to_solid). For every solid node with fluid
 * neighbours: integer normal n~6 = sum over fluid links of 6 w_q (-c_q)
 * (w_q = 1, 1/2, 1/3), unit normal n_w = n~6/|n~6| rounded to FP32, donor
 * q* = argmax (-c_q . n_w)/|c_q| compared exactly (ties: lowest q with
 * q = 9(cz+1) + 3(cy+1) + (cx+1)). Nodes with n~6 = 0 are skipped. The wall
 * list is sorted by node index. Contact angles reset to params.theta_deg;
 * fields must be set again afterwards. Returns CACL_ERR_GEOMETRY when a
 * non-periodic axis is not closed by solid layers. Synchronises. */
cacl_status cacl_set_geometry(cacl_ctx* ctx, const uint8_t* solid);

/* Contact angle per node in degrees (host, N floats, read at wall nodes
 * only), or NULL for params.theta_deg everywhere (Eq.
 * internal_contact_angle: theta_c = pi - theta; cot theta_c replaced by
 * sign(cos theta_c) 1e6 when |sin theta_c| < 1e-6). */
cacl_status cacl_set_contact_angle(cacl_ctx* ctx, const float* theta_deg);

/* Contact angle per wall node, in wall-list order (host, W floats,
 * degrees); the parameters of the adjoint's dL/dtheta. */
cacl_status cacl_set_wall_angles(cacl_ctx* ctx, const float* theta_deg_wall);

/* Change the surface tension (beta = 12 sigma/delta, kappa_phi = 3 sigma
 * delta / 2, Eq. Fcap); the parameter of the adjoint's dL/dsigma. */
cacl_status cacl_set_sigma(cacl_ctx* ctx, double sigma);

/* Initial state from host arrays: phi (N floats, every node; values at
 * solid nodes seed the ghosts) and u (3N floats, component-major, or NULL
 * for rest). Populations become f^eq(p* = 0, u) (Eq. feq3); the mass
 * reference M_ref becomes the FP64 sum of phi over fluid nodes
 * (Eq. phase_field_mass). */
cacl_status cacl_set_fields(cacl_ctx* ctx, const float* phi, const float* u);

/* Replace parts of the state (host arrays), e.g. to resume from a
 * checkpoint: populations f* (27N floats, f[q*N + n]), phi (N), u (3N). */
cacl_status cacl_set_populations(cacl_ctx* ctx, const float* f);
cacl_status cacl_set_phi(cacl_ctx* ctx, const float* phi);
cacl_status cacl_set_velocity(cacl_ctx* ctx, const float* u);
cacl_status cacl_set_mass_ref(cacl_ctx* ctx, double m_ref);

/* Checkpoint and resume. cacl_save_state copies the complete dynamic state
 * of the context into a host buffer of at least cacl_state_bytes bytes: a
 * header (grid, storage, wall count), the current populations as stored,
 * phi with its ghost values, u, the mass record of the volume correction
 * (M_ref, the last M*, W and lambda, and the count of corrections, which
 * keys their unbiased rounding) and the contact angle of every wall node.
 * cacl_load_state restores it into a context of the same grid, storage and
 * geometry (cacl_set_geometry first); stepping on from there gives bit for
 * bit what the saved context gives. The caller owns the buffer and any
 * file it is written to. cacl_state_bytes returns -1 before
 * cacl_set_geometry; save returns CACL_ERR_STATE before cacl_set_fields,
 * CACL_ERR_ARG for a short buffer; load returns CACL_ERR_ARG for a buffer
 * that is not a saved state or belongs to another grid, storage or
 * geometry. Both synchronise the context stream. */
int64_t cacl_state_bytes(const cacl_ctx* ctx);
cacl_status cacl_save_state(cacl_ctx* ctx, void* host_buf, int64_t bytes);
cacl_status cacl_load_state(cacl_ctx* ctx, const void* host_buf, int64_t bytes);

/* Test hook for failure detection: sets the context's device error word as
 * a bounded wait for asynchronous copies that gave up would (no GPU fault
 * is made); the next cacl_check_finite then returns CACL_ERR_TIMEOUT. The
 * word stays set: the state is not trusted after such a failure. */
cacl_status cacl_inject_wait_timeout(cacl_ctx* ctx);

/* Test hook that makes a bounded wait run out (no GPU fault is made). While
 * on != 0, every block of the copy-staged collide-stream
 * (CACL_OPT_LB_PIPE = 1) registers 16 bytes more for the copies of its
 * first row segment than they deliver, so the wait for them cannot
 * complete: each thread gives up after 0.5 s of the GPU's global timer,
 * the block records it in the device error word, finishes its segment on
 * the stale stage, waits (bounded) for its copies still in flight and
 * returns. Every block of the TMA-tiled collide-stream
 * (CACL_OPT_LB_PIPE = 3) does the same with its one tile: it gives up
 * after 0.5 s, records it, waits once more (bounded, 0.5 s) and returns
 * without computing. The next cacl_check_finite returns CACL_ERR_TIMEOUT;
 * the word stays set and the state is not trusted. Other kernels ignore
 * the request. Synchronises the context stream. */
cacl_status cacl_inject_copy_stall(cacl_ctx* ctx, int on);

/* Advance nsteps >= 0 full steps (ghost update, collide-stream, phi update,
 * volume correction) on the context stream; does not synchronise. The
 * step's correction visits only the phi-update tiles whose chi sum is
 * positive (chi >= 0, so the others hold no interface-band node and keep
 * phi = phi*); the result is bit-identical to correcting every node. */
cacl_status cacl_step(cacl_ctx* ctx, int nsteps);

/* The four parts of one step, enqueued singly (for inspection and part by
 * part checks). cacl_lb_collide reads phi and writes populations, u and the
 * compressive vector of phi; cacl_phase_update forms that vector from the
 * current phi itself, then writes phi*, the block partial sums and, from
 * them, lambda; cacl_volume_correct writes
 * phi^{n+1} = phi* + lambda chi(phi*). */
cacl_status cacl_ghost_update(cacl_ctx* ctx);
cacl_status cacl_lb_collide(cacl_ctx* ctx);
cacl_status cacl_phase_update(cacl_ctx* ctx);
cacl_status cacl_volume_correct(cacl_ctx* ctx);

/* Copy out phi (N), u (3N), p* (N, sum of f* at fluid nodes, 0 at solids);
 * any pointer may be NULL. device_ptrs = 1: the pointers are device memory
 * (copied on the context stream, no synchronisation); 0: host memory
 * (synchronises). */
cacl_status cacl_get_fields(cacl_ctx* ctx, float* phi, float* u, float* pstar,
                            int device_ptrs);
cacl_status cacl_get_populations(cacl_ctx* ctx, float* f, int device_ptrs);

/* Wall list (host arrays sized by *count, which is always written):
 * idx (node), qstar (donor direction), ntilde6 (3 per node), nw (FP32 unit
 * normal, 3 per node). Pass NULL arrays to query the count. */
cacl_status cacl_get_wall_list(cacl_ctx* ctx, int32_t* idx, int8_t* qstar,
                               int16_t* ntilde6, float* nw, int32_t* count);

/* FP64 mass bookkeeping of the last correction: M_ref, M* (sum phi* over
 * fluid), W (sum chi), lambda. Synchronises. */
cacl_status cacl_get_mass(cacl_ctx* ctx, double* m_ref, double* m_star,
                          double* w_sum, double* lambda);

/* Returns CACL_ERR_TIMEOUT if a kernel's bounded wait for its asynchronous
 * copies gave up since the context was created (its results are then not
 * to be trusted), else CACL_ERR_DIVERGED if phi or u holds a NaN or Inf.
 * Synchronises. */
cacl_status cacl_check_finite(cacl_ctx* ctx);

/*
 * Adjoint (reverse mode, hand-written) of nsteps full steps with respect to
 * the contact angle of every wall node and the surface tension, for a loss
 * L(phi) of the final phase field (FP32 populations only).
 *   cacl_adjoint_forward advances the state by nsteps steps from the current
 *   state, storing a checkpoint (f*, phi) every ckpt_every steps;
 *   cacl_adjoint_backward takes dL/dphi of the final field (device, N
 *   floats), recomputes each segment from its checkpoint with a per-step
 *   tape, applies the transposed step in reverse (volume correction, phi
 *   update, collide-stream, ghost map) and writes dL/dtheta_deg per wall node
 *   (device, W doubles, wall-list order) and dL/dsigma (device, 1 double),
 *   both accumulated in FP64. The state after the call is the one the
 *   forward reached. At points where the step is not differentiable (minmod
 *   switches, upwind choice, band edges of chi) the derivative of the branch
 *   the forward took is used.
 */
cacl_status cacl_adjoint_forward(cacl_ctx* ctx, int nsteps, int ckpt_every);
cacl_status cacl_adjoint_backward(cacl_ctx* ctx, const float* dL_dphi,
                                  double* dL_dtheta, double* dL_dsigma);
/* One stage of the adjoint on its own (a test hook for the transposes):
 * step 0 of the rollout of the last cacl_adjoint_forward (one level) is
 * recomputed from its checkpoint, and the transpose of one of its maps is
 * applied to the cotangent `in` at that linearisation point. All pointers
 * are device pointers (FP32 unless stated), node-major as the fields:
 *   CACL_ADJ_CORRECT (Sect. 2.3, Eq. mass_corrected_phi with lambda of
 *     Eq. mass_correction_normalization): in = phi^{n+1}_bar (N) ->
 *     out = phi*_bar (N).
 *   CACL_ADJ_PHASE (Sect. 2.1.1, Eq. phi_update_muscl, the compressive
 *     vector a taken as an input): in = phi*_bar (N) -> out = [phi_g_bar
 *     (N) | u_bar (3N) | a_bar (3N)].
 *   CACL_ADJ_COLLIDE (Sect. 2.1, Eqs. lbe .. lap_iso, the compressive vector
 *     of the ghosted phi and the pull of the next step): in = [the next
 *     step's pulled populations' cotangent (27N) | u_bar (3N) | a_bar (3N)]
 *     -> out = [this step's pulled populations' cotangent (27N) |
 *     phi_g_bar (N)], dparam[0] = dL/dsigma (double).
 *   CACL_ADJ_GHOST (Sect. 2.2): in = phi_g_bar (N) -> out = phi^n_bar (N),
 *     dparam = dL/dtheta per wall node (W doubles, wall-list order).
 * state (optional, 36 N floats) receives the linearisation point: phi^n,
 * f*^{n-1} (27 N, as stored), the ghosted phi, u, a, phi*. The context's
 * state is left as it was. CACL_ERR_STATE without a one-level forward. */
typedef enum {
  CACL_ADJ_CORRECT = 0,
  CACL_ADJ_PHASE = 1,
  CACL_ADJ_COLLIDE = 2,
  CACL_ADJ_GHOST = 3
} cacl_adj_stage;
cacl_status cacl_adjoint_stage(cacl_ctx* ctx, int stage, const float* in, float* out,
                               double* dparam, float* state);

/* GPU time (CUDA events) of the last cacl_adjoint_backward: the taped
 * recomputes of its segments (and outer segments) and the whole call, in
 * milliseconds. CACL_ERR_STATE before any backward. */
cacl_status cacl_adjoint_timing(const cacl_ctx* ctx, double* recompute_ms,
                                double* total_ms);

/* Two-level checkpointing for long rollouts: as cacl_adjoint_forward, but
 * the forward keeps a checkpoint only every outer_every steps (a positive
 * multiple of ckpt_every; 0 = one level, the same as cacl_adjoint_forward).
 * cacl_adjoint_backward then recomputes each outer segment once from its
 * checkpoint to rebuild the checkpoints every ckpt_every steps inside it,
 * and proceeds as with one level; the gradients are bit-identical to the
 * one-level ones. Device memory: ceil(nsteps / outer_every) + outer_every /
 * ckpt_every checkpoints of 28 N floats, plus the tape of ckpt_every steps
 * (36 N floats each), instead of ceil(nsteps / ckpt_every) checkpoints;
 * every step is computed once more. Returns CACL_ERR_ARG when outer_every
 * is not a multiple of ckpt_every. */
cacl_status cacl_adjoint_forward_levels(cacl_ctx* ctx, int nsteps,
                                        int ckpt_every, int outer_every);

/*
 * Batches: many cases of uneven grid size advanced together (each stage of
 * the step is one grid-strided launch over a work-list spanning all cases,
 * the step is a captured CUDA graph). Every case is an ordinary context
 * owned by the batch: set it up and query it with the single-case calls on
 * the handle from cacl_batch_case (geometry, angles, fields, getters). All
 * cases must use the same storage; they advance in lockstep, so do not step
 * a case on its own between batch steps (cacl_batch_step then returns
 * CACL_ERR_STATE). Giving a case a new geometry is picked up at the next
 * cacl_batch_step.
 */
typedef struct cacl_batch cacl_batch;

/* ncases >= 1 parameter sets (same storage, not CACL_F32_MOMENTS); stream
 * as for cacl_create. CACL_ERR_TOO_LARGE when a case has 27 nx ny nz >=
 * 2^31 nodes (the batched kernels index with 32 bits). */
cacl_status cacl_batch_create(const cacl_params* params, int ncases,
                              void* stream, cacl_batch** out);
void cacl_batch_destroy(cacl_batch* batch);
const char* cacl_batch_last_error(const cacl_batch* batch);

/* The batch's context of case i (0 <= i < ncases); owned by the batch. */
cacl_status cacl_batch_case(cacl_batch* batch, int i, cacl_ctx** out);

/* Advance every case by nsteps full steps (ghost update, collide-stream,
 * phi update, volume correction with a per-case lambda). */
cacl_status cacl_batch_step(cacl_batch* batch, int nsteps);

/* Launch shapes of the batched stages: collide-stream blocks of 64, 128 or
 * 256 threads (each thread one, two or four consecutive nodes of a case, as
 * the case would run alone) with a resident-sized grid striding through the
 * work-list (lb_variant 0, 1, 2) or one block per work item (3, 4, 5), and
 * the phi-update tile (0..3, as CACL_OPT_PHASE_TILE). */
cacl_status cacl_batch_set_option(cacl_batch* batch, int lb_variant,
                                  int phase_variant);

/* Autotuner: times `steps` batch steps for every launch-shape pair, keeps
 * the fastest and returns it with its time per step. It runs real steps:
 * every case advances by 25 * steps steps (use it as the warm-up). */
cacl_status cacl_batch_autotune(cacl_batch* batch, int steps, int* lb_variant,
                                int* phase_variant, float* best_ms);

/* Launch-shape options (results do not depend on them beyond rounding
 * order). CACL_OPT_PHASE_TILE selects the tile of the phase update:
 * 0 = 32x16 nodes x 16 planes, 1 = 32x8 x 16, 2 = 32x8 x 32,
 * 3 = 32x16 x 32. CACL_OPT_PHASE_PIPE selects how the phase update stages
 * its planes in shared memory and how many nodes a thread evaluates:
 * 0 = automatic (3 when nx is a multiple of 4, nz >= 2 and the fields are
 * 16-byte aligned; else 2 when nz >= 2; else 1), 1 = staging through
 * registers, 2 = asynchronous copies (16-byte copies when nx is a multiple
 * of 4, else 4-byte copies element by element), two nodes per thread along
 * y, 3 = asynchronous 16-byte copies, 2 x 2 nodes per thread (an x pair on
 * two rows, packed pair arithmetic); 2 returns CACL_ERR_ARG when nz < 2, 3
 * also when nx is not a multiple of 4. All
 * give bit-identical phi*; the partial sums of the volume correction agree
 * to the rounding of their summation order, bit for bit between 1 and 2.
 * CACL_OPT_LB_PIPE selects how the collide-stream
 * reads its 27 pulled population rows and 9 phi rows: 0 = direct loads
 * through the cache with two x-adjacent nodes per thread, one aligned
 * access per pair and packed pair arithmetic (the default; when nx is odd
 * or 27 N >= 2^31 it runs one node per thread), 1 = row runs staged in
 * shared memory by bulk asynchronous copies through a two-stage ring of
 * persistent blocks (CACL_ERR_ARG unless nx is a multiple of 4 and of 16
 * bytes' worth of populations), 2 = direct loads, one node per thread,
 * 3 = tiles of 128 nodes copied into shared memory and stored back by the
 * tensor memory accelerator (when nx is a multiple of 8; else as 0); all
 * bit-identical at fluid nodes (the tiled form writes f* = 0 at solid
 * nodes, the others leave them). CACL_OPT_INDEX64 = 1 makes every
 * collide-stream and adjoint kernel that exists with 32- and 64-bit offsets
 * take its 64-bit form (and the collide-stream the one-node or staged
 * kernel, as when 27 N >= 2^31), whatever the grid size; the results are
 * bit-identical to pipeline 2 (or 1) and to the 32-bit adjoint. It exists so
 * that the path of grids above 2^31 / 27 nodes can be checked on small
 * ones. Defaults: tile 2 (tile 1 when the grid has fewer than 400 tiles
 * of 32 x 8 x 32 nodes), pipelines 0, index64 0.
 * Returns CACL_ERR_ARG for an unknown option or value. */
typedef enum {
  CACL_OPT_PHASE_TILE = 1,
  CACL_OPT_PHASE_PIPE = 2,
  CACL_OPT_LB_PIPE = 3,
  CACL_OPT_INDEX64 = 4
} cacl_option;
cacl_status cacl_set_option(cacl_ctx* ctx, int option, int value);

/* Grid size N and bytes of device memory the context holds. */
cacl_status cacl_get_info(const cacl_ctx* ctx, int64_t* nodes,
                          int64_t* device_bytes, int32_t* wall_count);

/*
 * z-slab decomposition: one problem split along z into slabs, one per GPU
 * (or several on one GPU), each an ordinary context with two halo planes on
 * each side. This is the parallel split of the step across devices that
 * the paper's large domains call for: per step one exchange of phi before
 * and after the ghost update, one of f* and of u, a after the
 * collide-stream, and one gather of the phi update's block partial sums for
 * the global volume correction (Sect. 2.3, Eqs. tentative_phase_field_mass
 * .. mass_corrected_phi).
 *
 * cacl_slab_create: a slab owning global planes [z0, z0 + nz) of the grid
 *   described by *global (0 <= z0, z0 + nz <= global->nz). Its context has
 *   nz + 4 planes, periodic in z: local plane l holds global plane
 *   z0 - 2 + l (wrapped around global->nz). Set its geometry, fields and
 *   angles with the ordinary calls on those nz + 4 planes (halo planes
 *   included), then set the global mass reference with cacl_set_mass_ref
 *   (cacl_set_fields sums the slab's own planes only).
 * cacl_slab_stage: one stage of the step on every local plane (ghost
 *   update, collide-stream) or on the interior planes (phi update: block
 *   partial sums only, no correction).
 * cacl_slab_partials: the last phi update's block partial sums, nb phi*
 *   sums then nb chi sums (device dst, 2 nb doubles; NULL dst queries nb).
 *   Blocks are ordered by their z tile last, so the slabs' arrays in slab
 *   order, phi* parts of all slabs first and then the chi parts, are the
 *   undivided context's array when every interior starts on a multiple of
 *   the phi update's tile depth (32 planes with the default tile).
 * cacl_slab_correct: lambda from such a gathered array (device, nb_total
 *   phi* sums then nb_total chi sums), in the fixed order an undivided
 *   context uses, then the correction; the rounding key uses global node
 *   indices.
 * cacl_slab_halo: direction 0 packs the interior planes next to side 0
 *   (low z) or 1 (high z) into buf, direction 1 unpacks buf into the halo
 *   planes on that side. field CACL_SLAB_PHI: 2 planes of phi (ghosts
 *   included); CACL_SLAB_F: 1 plane of the 27 current populations (storage
 *   type); CACL_SLAB_UA: 1 plane of u (3 components) then a (3). buf is a
 *   device buffer of cacl_slab_halo_bytes(ctx, field) bytes, component-major,
 *   then plane, y, x. A slab's low interior planes feed the halo of the
 *   slab below (its side 1) and its high ones the slab above (side 0).
 * Enqueued on the context's stream; CACL_ERR_STATE on an ordinary context.
 */
enum {
  CACL_SLAB_PHI = 0,
  CACL_SLAB_F = 1,
  CACL_SLAB_UA = 2
};
enum {
  CACL_SLAB_GHOST = 0,
  CACL_SLAB_COLLIDE = 1,
  CACL_SLAB_PHASE = 2
};
cacl_status cacl_slab_create(const cacl_params* global, int z0, int nz,
                             void* stream, cacl_ctx** out);
cacl_status cacl_slab_stage(cacl_ctx* ctx, int stage);
cacl_status cacl_slab_partials(cacl_ctx* ctx, double* dst, int* nblocks);
cacl_status cacl_slab_correct(cacl_ctx* ctx, const double* all, int nb_total);
cacl_status cacl_slab_halo(cacl_ctx* ctx, int field, int side, int direction,
                           void* buf);
int64_t cacl_slab_halo_bytes(const cacl_ctx* ctx, int field);

/*
 * Allocation-free volume correction (the paper has no counterpart: this is
 * a library service). Some callers cannot call cudaMalloc: a process whose
 * device memory already belongs to another allocator's pool, a host that
 * forbids device allocation once it is serving, or code that must not risk
 * the implicit device synchronisation of cudaFree. This call corrects a
 * phase field they own without allocating anything: its reduction scratch
 * is a fixed 256 KiB array compiled into the library, held on every GPU
 * that loads the library until the process exits.
 *
 *   phi     device, n floats, corrected in place at fluid nodes:
 *           phi += lambda chi(phi), chi = phi (1 - phi) inside
 *           (eps_phi, 1 - eps_phi), lambda = (m_ref - M*) / W (0 if W = 0),
 *           M* and W the FP64 sums of phi and chi over fluid nodes. The sum
 *           phi + lambda chi is rounded to FP32 without bias, as in the
 *           context's correction (cacl_volume_correct): the exact residual
 *           decides, against a hashed uniform number, whether to move one
 *           unit in the last place, so corrections below the FP32
 *           resolution of phi still hold the mass on average over repeated
 *           calls. The hash key is a per-device call counter the library
 *           keeps in the scratch array (zero when the library is loaded).
 *   solid   device, n bytes, nonzero = solid (left untouched)
 *   n       1 <= n <= 67,108,864 (4096 x 16384); larger n returns
 *           CACL_ERR_TOO_LARGE before any work is enqueued
 *   m_ref   target fluid mass; eps_phi in (0, 1/2)
 *   out     device, 3 doubles (M*, W, lambda) or NULL
 *   stream  cudaStream_t or NULL; the call enqueues and returns
 *
 * phi, solid, out and the stream must belong to the current CUDA device
 * (pointers on another device, or host pointers, return CACL_ERR_ARG).
 * The first call on a device looks up the scratch array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture. Every call shares the one scratch array, so
 * calls that overlap on the GPU (other streams, other host threads) race;
 * serialise them on one stream. Returns CACL_ERR_ARG for null pointers,
 * invalid sizes or pointers not on the current device, CACL_ERR_CUDA for a
 * launch or set-up failure.
 */
cacl_status cacl_volume_correct_noalloc(float* phi, const uint8_t* solid,
                                        int64_t n, double m_ref,
                                        double eps_phi, double* out,
                                        void* stream);

#ifdef __cplusplus
}
#endif
#endif /* CACL_H */
