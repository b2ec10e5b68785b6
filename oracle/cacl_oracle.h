/*
 * cacl_oracle.h -- TEST INFRASTRUCTURE, not part of the product.
 *
 * A plain, slow FP64 CPU restatement of one time step of the conservative
 * Allen-Cahn lattice Boltzmann (CAC-LB) scheme with the geometric wetting
 * boundary condition of arXiv 2607.25444 (Sects. 2.1-2.3).  It exists only to
 * check the CUDA path: only the tests, the smoke check and the bench's CPU
 * baseline leg may load it.  It shares no code, header, table or helper with
 * the CUDA library; its lattice tables, parameter struct and enumerations are
 * written out here independently.
 *
 * Layout of every field: node index n = x + nx*(y + ny*z), x fastest.
 * Populations are stored as f[q*N + n]; velocity as u[d*N + n].
 * Direction order q: (cz, cy, cx) in {-1,0,1}^3 lexicographic, cx fastest
 * (D2Q9: (cy, cx) in {-1,0,1}^2, cz = 0), so that q = 9(cz+1)+3(cy+1)+(cx+1).
 * That order is also the donor tie-break order (lowest q wins a tie).
 */
#ifndef CACL_ORACLE_H
#define CACL_ORACLE_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int dim;            /* 3 -> D3Q27, 2 -> D2Q9 (then nz must be 1) */
  int nx, ny, nz;
  int periodic[3];    /* non-periodic axes must be closed by solid layers */
  double width;       /* interface width delta (Sect. 2.1.1, Eq. kappa_delta) */
  double mobility;    /* interface diffusivity D */
  double sigma;       /* surface tension */
  double rho_l, rho_g;
  double nu_l, nu_g;  /* kinematic viscosities; mu = rho nu mixed linearly */
  double gravity[3];  /* F_ext = (rho(phi) - rho_g) g */
  double theta_deg;   /* default contact angle */
  double eps_phi;     /* chi band threshold of the volume correction */
} orc_params;

typedef struct orc_state orc_state;

/* Life cycle. Return 0 on success, negative on error (text via orc_error). */
orc_state* orc_create(const orc_params* p);
void orc_destroy(orc_state* s);
const char* orc_error(const orc_state* s);

int orc_set_geometry(orc_state* s, const uint8_t* solid);
int orc_set_contact_angle(orc_state* s, const double* theta_deg_per_node);
int orc_set_fields(orc_state* s, const double* phi, const double* u);
int orc_set_populations(orc_state* s, const double* f);
int orc_set_phi(orc_state* s, const double* phi);
int orc_set_velocity(orc_state* s, const double* u);
int orc_set_mass_ref(orc_state* s, double m_ref);

/* One full step: ghost update, LB collide-stream, phi update, correction. */
int orc_step(orc_state* s, int nsteps);
/* The four parts of the step, for part-by-part parity. */
int orc_ghost_update(orc_state* s);
int orc_lb_collide(orc_state* s);
int orc_phase_update(orc_state* s);   /* writes phi* into the phi array */
int orc_volume_correct(orc_state* s); /* from phi* and M_ref */

int orc_get_fields(const orc_state* s, double* phi, double* u, double* pstar);
int orc_get_populations(const orc_state* s, double* f);
int orc_get_wall_count(const orc_state* s);
int orc_get_wall_list(const orc_state* s, int32_t* idx, int8_t* qstar,
                      int16_t* ntilde6, float* nw_f32, double* nw_f64);
int orc_get_mass(const orc_state* s, double* m_ref, double* m_star,
                 double* w_sum, double* lambda);
double orc_fluid_mass(const orc_state* s);

/* Node-level pieces, exposed so tests can pin them in closed form. */
int orc_lattice(int dim, int* c /*Q*3*/, double* w /*Q*/);
int orc_feq(int dim, double pstar, const double* u, double* feq);
int orc_collide_node(const orc_state* s, const double* f_in, double phi,
                     const double* grad_phi, double lap_phi, double* f_out,
                     double* u_out, double* a_out, double* omega_out);
int orc_grad_lap(const orc_state* s, const double* field, double* grad,
                 double* lap);
double orc_ghost_value(double phi_f, const double* grad_f, const double* nw,
                       const double* r_fs, double theta_deg);

#ifdef __cplusplus
}
#endif
#endif
