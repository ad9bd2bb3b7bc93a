/* sph_oracle.h -- plain FP64 CPU oracle of the coupled fluid-solid-thermal
 * weakly-compressible SPH step (test infrastructure only).
 *
 * This is a slow, obviously-correct restatement of the paper's equations:
 * brute-force O(N^2) neighbour search, particles kept in id order, every sum
 * a plain loop in ascending neighbour id.  Only the test suite, the package
 * smoke check and the benchmark's CPU-baseline leg may call it; the CUDA
 * product path never does.  It shares no code with the CUDA library.
 *
 * Section / equation references are to the paper (arXiv 2512.09904):
 *   Sec. 2.1  mass/momentum equations Eq. (1), linear EoS Eq. (2)
 *   Sec. 2.3  Riemann-based continuity and momentum, Eqs. (10)-(13)
 *   Sec. 2.4  density re-initialisation, Eqs. (14)-(15)
 *   Sec. 2.5  wall dummy particles, one-sided Riemann, Eqs. (16)-(19)
 *   Sec. 2.6  Cleary heat conduction, Eqs. (20)-(22)
 *   Sec. 2.8  dual-criteria time stepping, Eqs. (25)-(26)
 */
#ifndef SPH_ORACLE_H
#define SPH_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    double origin[3], extent[3]; /* domain box (periodic axes wrap on it) */
    double dx, h_over_dx;        /* lattice spacing; h = h_over_dx * dx */
    double gravity[3];
    double c0, u_ref;            /* artificial sound speed; velocity floor */
    double cfl_ad, cfl_ac;       /* 0.25, 0.6 (Sec. 2.8) */
    int free_surface;            /* 1: Eq. (14) max() form; 0: Eq. (15) */
    int periodic_mask;           /* bit a: axis a periodic */
    int max_substeps;            /* acoustic sub-steps cap per advection step; 0 = default */
    int viscous_heating;         /* 1: add the viscous-dissipation heating 2 mu S:S (not in the
                                    paper's model, which omits it; default 0) */
    int vstar_literal;           /* 1: Eq. (13)'s interface velocity with its printed sign,
                                    v* = (U* - U~) e_ij + v~ (default 0: v* = -(U* - U~) e_ij + v~) */
    double cfl_T;                /* Eq. (26) coefficient (0.5 printed); 0: no thermal bound */
    int wall_pstar_printed;      /* 1: the wall interface pressure exactly as Eq. (19) prints it,
                                    the density-weighted mean of the fluid and mirror pressures
                                    (default 0: that mean plus Eq. (12)'s limiter term on the
                                    same one-sided states) */
} orc_config;

typedef struct { double rho0, mu, k, cp, T_init; int fixed_T; } orc_material;

typedef struct orc_sim orc_sim;

/* --- scalar pieces (pinned individually by the tests) -------------------- */
double orc_W(double r, double h);      /* Wendland C2, 3-D, support 2h */
double orc_dW(double r, double h);     /* dW/dr */
double orc_sigma0(double dx, double h);/* sum of W over an exact cubic lattice incl. self */
/* fluid-fluid Riemann (Sec. 2.3): returns U*, p* for states (rho,U,p) L/R */
void orc_riemann(double rhoL, double UL, double pL, double rhoR, double UR, double pR,
                 double c0, double* Ustar, double* pstar);
/* wall one-sided Riemann (Sec. 2.5): right state and interface values;
 * printed = 1 gives Eq. (19)'s p* without the limiter term */
void orc_wall_riemann(double rho_f, double UL, double p_f, double u_w, double g_dot_rfw,
                      double rho0, double c0, int printed, double* UR, double* PR, double* rhoR,
                      double* Ustar, double* pstar);
void orc_timesteps(double h, double vmax, double u_ref, double nu_max, double c0,
                   double cfl_ad, double cfl_ac, double* dt_ad, double* dt_ac);
double orc_dt_thermal(double cfl_T, double rho, double cp, double h, double k);  /* Eq. (26) */

/* brute-force pair list: pairs (i,j), 0 < |r_i - r_j|^2 < R2 (FP64, strict),
 * minimum image on periodic axes.  counts[i] = neighbours of i; if list is
 * non-NULL it receives, for each i in order, its neighbours in ascending j.
 * Returns total pair entries, or -1 if cap is too small. */
int64_t orc_neighbors_of(int64_t n, const double* pos, double R2, int periodic_mask, const double* extent,
                         int64_t m, const int64_t* idx, int64_t* counts, int32_t* list, int64_t cap);
int64_t orc_neighbors(int64_t n, const double* pos, double R2, int periodic_mask,
                      const double* extent, int64_t* counts, int32_t* list, int64_t cap);
/* passes D, V and T of the fluid particles idx[0..m) only, from the whole
 * state at the start of an advection step (brute force, any size):
 * av[3m] viscous accelerations (Eqs. 10, 18), dTdt[m] (Eq. 22), with the
 * re-initialised densities of Eq. (14) (free_surface = 1) or (15).  Returns
 * -1 if an index is out of range or not a fluid particle. */
int orc_sample_vt(int64_t n, const double* pos, const double* vel, const double* rho, const double* T,
                  const int* kind, const int* mat_id, const orc_material* mats, double dx, double h,
                  int free_surface, int periodic_mask, const double* extent, int64_t m, const int64_t* idx,
                  double* av, double* dTdt);
/* pass M of the fluid particles idx[0..m) for the first acoustic sub-step
 * (size dt) of an advection step, from the same state plus drho and the wall
 * normals: ap[3m] the pressure acceleration (Eqs. 10-12, 16-19; without the
 * held viscous term and gravity).  -1 as orc_sample_vt. */
int orc_sample_ap(int64_t n, const double* pos, const double* vel, const double* rho, const double* drho,
                  const double* nrm, const int* kind, const int* mat_id, const orc_material* mats, double dx,
                  double h, int free_surface, const double* gravity, double c0, int wall_pstar_printed, double dt,
                  int periodic_mask, const double* extent, int64_t m, const int64_t* idx, double* ap);
/* the first acoustic sub-step of an advection step for the fluid particles
 * idx[0..m) (non-periodic cases): from the state at the step's start, or any
 * part of it holding every particle within three support radii of each
 * sample, the kicked velocities v_new[3m] (pass M with the held viscous term
 * and g) and pass C's continuity rates drho_new[m].  -1 as orc_sample_vt,
 * -2 if host memory runs out. */
int orc_sample_substep(int64_t n, const double* pos, const double* vel, const double* rho, const double* drho,
                       const double* nrm, const int* kind, const int* mat_id, const orc_material* mats, double dx,
                       double h, int free_surface, const double* gravity, double c0, int wall_pstar_printed,
                       double dt, int64_t m, const int64_t* idx, double* v_new, double* drho_new);
/* expected cell order: key = linear cell index (x fastest) of
 * floor((x - origin)/w) per axis, clamped to the grid; particles sorted by
 * (key, id).  perm[k] = id at sorted position k; cell_start has ncell+1. */
void orc_cell_order(int64_t n, const double* pos, const double* origin, const double* cellw,
                    const int* ncell, int64_t* perm, int64_t* cell_start);

/* --- whole simulation ---------------------------------------------------- */
orc_sim* orc_create(const orc_config* cfg);
void orc_destroy(orc_sim*);
int orc_set_threads(int n);
int orc_set_material(orc_sim*, int id, const orc_material*);
int orc_set_rotation(orc_sim*, int body, const double c[3], const double axis[3], double omega);
/* kind: 0 fluid, 1 solid; body: -1 static; rho NaN -> material rho0 */
int orc_add_particles(orc_sim*, int64_t n, const int* kind, const int* mat, const int* body,
                      const double* pos, const double* vel, const double* normal,
                      const double* T, const double* rho);
int orc_step(orc_sim*, int n_adv);
/* fields (id order): 0 pos[3], 1 vel[3], 2 rho, 3 p, 4 T, 5 drho, 6 a_visc[3], 7 dTdt,
 * 8 sigma (kernel sum of pass D), 9 wall normal[3], 10 wall velocity[3],
 * 11 contact factor of rigid-body particles (Sec. 2.7; 0 for the others),
 * 12 fluid density right after pass D of the last advection step (Eq. 14 / 15;
 *    the material rho0 for solids) */
int orc_get_field(const orc_sim*, int field, double* out);

/* --- physics-driven particle relaxation (Sec. 2.2), a pre-processing step --- */
typedef struct {
    double dx, h_over_dx;          /* particle spacing, smoothing length h = h_over_dx dx */
    const double* phi;             /* level set (negative inside), nphi[0] x nphi[1] x nphi[2] nodes, x fastest */
    int nphi[3];
    double phi_origin[3], phi_spacing;
} orc_relax_config;
/* half-space kernel integral A(d) = 2 pi int_d^{2h} W(r) r dr (quadrature) */
double orc_relax_A(double d, double h);
/* level set and its unit gradient at x (trilinear) */
double orc_phi(const orc_relax_config* c, const double* x, double* n_out);
/* `iterations` relaxation steps of the n particles pos[n*3] (in place);
 * max_accel[k] = max |F_p| of step k (may be NULL) */
int orc_relax(const orc_relax_config* cfg, int64_t n, double* pos, int iterations, double* max_accel);
/* body: torque about its axis (last sub-step), dt-weighted average since
 * start, heat into fluid sum m cp (T - T0), mean fluid temperature */
int orc_torque_heat(const orc_sim*, int body, double* torque, double* torque_avg,
                    double* heat_into_fluid, double* mean_fluid_T);
/* body: total force of the fluid on the body (last sub-step; pressure + viscous) */
int orc_body_force(const orc_sim*, int body, double* force3);
int orc_time(const orc_sim*, double* t, int64_t* adv_steps, int64_t* substeps,
             double* last_dt_ad, int* last_nsub);
int64_t orc_count(const orc_sim*);

#ifdef __cplusplus
}
#endif
#endif
