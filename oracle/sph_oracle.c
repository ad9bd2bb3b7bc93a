/* sph_oracle.c -- plain FP64 CPU oracle (test infrastructure only).
 *
 * A direct restatement of the paper's method, written for checking by eye,
 * not for speed.  Particles stay in id order, the neighbour list is rebuilt
 * by brute force over all pairs once per advection step, and every sum runs
 * over neighbours in ascending id.  Compile with -ffp-contract=off so that
 * the squared distance that decides pair membership is the plain
 * ((dx*dx + dy*dy) + dz*dz) in round-to-nearest FP64.
 *
 * The step (Sec. 2.8, dual-criteria time stepping) is:
 *   advection step (size dt_ad, Eq. 25 first line, at most the thermal bound of Eq. 26):
 *     rigid bodies placed at angle omega*t; snapshot of all positions;
 *     neighbour list from the snapshot (kept for the whole advection step);
 *     pass D  density re-initialisation (Eq. 14 / Eq. 15);
 *     pass V  viscous acceleration (Eq. 10 second term, Eq. 18 second line),
 *             held through the acoustic sub-steps;
 *     pass T  dT/dt by the Cleary form (Eq. 22), applied with the step size;
 *     acoustic sub-steps (size dt_ac, Eq. 25 second line) until dt_ad:
 *       rho += dt/2 drho; p = EoS (Eq. 2); r += dt/2 v;
 *       pass M  Riemann pressure force (Eqs. 10-12) + wall pressure (Eqs. 16-19);
 *               v += dt (a_p + a_visc + g);
 *       r += dt/2 v;
 *       pass C  Riemann continuity (Eqs. 10-13) + wall continuity (Eqs. 16-17);
 *               rho += dt/2 drho.
 * Readings of points the paper leaves open are marked READING below.
 *
 * Parity unpinned by the paper: the magnitudes of long-run churning torque
 * and heat-up (the paper prints no values for them).  The torque and force
 * sums themselves are pinned by sign (drag opposes rotation) and by the still
 * tank's walls carrying the oil's weight.
 */
#include "sph_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAX_MAT 16
#define ORC_MAX_BODY 8
#define PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* Kernel.  READING: the paper names no kernel; Wendland C2 in 3-D with
 * support 2h:  W = a (1 - q/2)^4 (1 + 2q),  a = 21 / (16 pi h^3),  q = r/h. */
double orc_W(double r, double h) {
    double q = r / h;
    if (q >= 2.0) return 0.0;
    double a = 21.0 / (16.0 * PI * h * h * h);
    double t = 1.0 - 0.5 * q;
    return a * t * t * t * t * (1.0 + 2.0 * q);
}

/* d/dr of the above: (a/h) * (-5 q) (1 - q/2)^3 */
double orc_dW(double r, double h) {
    double q = r / h;
    if (q >= 2.0) return 0.0;
    double a = 21.0 / (16.0 * PI * h * h * h);
    double t = 1.0 - 0.5 * q;
    return (a / h) * (-5.0 * q) * t * t * t;
}

/* Reference kernel sum for Eq. (14): W summed over the full cubic lattice of
 * spacing dx around a particle, itself included. */
double orc_sigma0(double dx, double h) {
    int m = (int)ceil(2.0 * h / dx) + 1;
    double s = 0.0;
    for (int k = -m; k <= m; ++k)
        for (int j = -m; j <= m; ++j)
            for (int i = -m; i <= m; ++i) {
                double r = dx * sqrt((double)(i * i + j * j + k * k));
                s += orc_W(r, h);
            }
    return s;
}

/* Linearised Riemann solution with the dissipation limiter (Eq. 12).
 * READING: the sound speed c in Eq. (12) is c0; the bars are arithmetic means. */
void orc_riemann(double rhoL, double UL, double pL, double rhoR, double UR, double pR,
                 double c0, double* Ustar, double* pstar) {
    double dU = UL - UR;
    double beta = 3.0 * (dU > 0.0 ? dU : 0.0);
    if (beta > c0) beta = c0;
    *Ustar = 0.5 * (UL + UR) + (pL - pR) / (c0 * (rhoL + rhoR));
    *pstar = 0.5 * (pL + pR) + rhoL * rhoR * beta * dU / (rhoL + rhoR);
}

/* One-sided wall Riemann problem (Eqs. 16-17, 19).  Left state is the fluid
 * (rho_f, U_L = -n.v_f, p_f); right state U_R = -U_L + 2 u_w,
 * P_R = p_f + rho_f g.r_fw, rho_R from the EoS.  Interface velocity from
 * Eq. (12) with these states.
 * READING: the interface pressure is Eq. (19)'s density-weighted mean with
 * (p_w, rho_w) = (P_R, rho_R) plus the limiter term of Eq. (12) on the same
 * one-sided states, beta = min(3 max(U_L - U_R, 0), c0).  Eq. (19) alone has no
 * term that resists a particle approaching the wall, and with it fluid
 * particles drift into walls at edges and corners.  printed = 1 keeps Eq. (19)
 * exactly as printed (no limiter term), for comparison. */
void orc_wall_riemann(double rho_f, double UL, double p_f, double u_w, double g_dot_rfw,
                      double rho0, double c0, int printed, double* UR, double* PR, double* rhoR,
                      double* Ustar, double* pstar) {
    *UR = -UL + 2.0 * u_w;
    *PR = p_f + rho_f * g_dot_rfw;
    *rhoR = rho0 + *PR / (c0 * c0);
    *Ustar = 0.5 * (UL + *UR) + (p_f - *PR) / (c0 * (rho_f + *rhoR));
    /* Eq. (19): the density-weighted mean, with (p_w, rho_w) = (P_R, rho_R) */
    *pstar = (rho_f * *PR + *rhoR * p_f) / (rho_f + *rhoR);
    if (printed) return;
    double dU = UL - *UR;
    double beta = 3.0 * (dU > 0.0 ? dU : 0.0);
    if (beta > c0) beta = c0;
    *pstar += rho_f * *rhoR * beta * dU / (rho_f + *rhoR);
}

/* Eq. (25).  READING: |v|max is floored at u_ref = c0/10 (the anticipated
 * maximum speed of Eq. 2) so a fluid at rest still gets a finite step. */
void orc_timesteps(double h, double vmax, double u_ref, double nu_max, double c0,
                   double cfl_ad, double cfl_ac, double* dt_ad, double* dt_ac) {
    double U = vmax > u_ref ? vmax : u_ref;
    double a = h / U;
    if (nu_max > 0.0) {
        double b = h * h / nu_max;
        if (b < a) a = b;
    }
    *dt_ad = cfl_ad * a;
    *dt_ac = cfl_ac * h / (c0 + vmax);
}

/* Eq. (26), printed with cfl_T = 0.5 */
double orc_dt_thermal(double cfl_T, double rho, double cp, double h, double k) {
    return cfl_T * rho * cp * h * h / k;
}

/* ------------------------------------------------------------------------ */
/* Squared distance in FP64 with the minimum image on periodic axes.
 * vec receives r_i - r_j. */
static double dist2(const double* pi, const double* pj, int periodic_mask, const double* ext,
                    double vec[3]) {
    for (int a = 0; a < 3; ++a) {
        double d = pi[a] - pj[a];
        if (periodic_mask & (1 << a)) {
            double L = ext[a];
            if (d > 0.5 * L) d -= L;
            else if (d < -0.5 * L) d += L;
        }
        vec[a] = d;
    }
    double r2 = vec[0] * vec[0] + vec[1] * vec[1];
    r2 = r2 + vec[2] * vec[2];
    return r2;
}

int64_t orc_neighbors(int64_t n, const double* pos, double R2, int periodic_mask,
                      const double* extent, int64_t* counts, int32_t* list, int64_t cap) {
    #pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
        int64_t c = 0;
        double v[3];
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double r2 = dist2(pos + 3 * i, pos + 3 * j, periodic_mask, extent, v);
            if (r2 > 0.0 && r2 < R2) ++c;
        }
        counts[i] = c;
    }
    int64_t total = 0;
    for (int64_t i = 0; i < n; ++i) total += counts[i];
    if (!list) return total;
    if (total > cap) return -1;
    int64_t* start = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
    start[0] = 0;
    for (int64_t i = 0; i < n; ++i) start[i + 1] = start[i] + counts[i];
    #pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
        int64_t c = start[i];
        double v[3];
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double r2 = dist2(pos + 3 * i, pos + 3 * j, periodic_mask, extent, v);
            if (r2 > 0.0 && r2 < R2) list[c++] = (int32_t)j;
        }
    }
    free(start);
    return total;
}

/* Brute-force neighbour sets of the m particles idx[] only (same rule as
 * orc_neighbors): for checking a large case on a sample of its particles. */
int64_t orc_neighbors_of(int64_t n, const double* pos, double R2, int periodic_mask, const double* extent,
                         int64_t m, const int64_t* idx, int64_t* counts, int32_t* list, int64_t cap) {
    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t q = 0; q < m; ++q) {
        const int64_t i = idx[q];
        int64_t c = 0;
        double v[3];
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double r2 = dist2(pos + 3 * i, pos + 3 * j, periodic_mask, extent, v);
            if (r2 > 0.0 && r2 < R2) ++c;
        }
        counts[q] = c;
    }
    int64_t total = 0;
    for (int64_t q = 0; q < m; ++q) total += counts[q];
    if (!list) return total;
    if (total > cap) return -1;
    int64_t* start = (int64_t*)malloc(sizeof(int64_t) * (size_t)(m + 1));
    start[0] = 0;
    for (int64_t q = 0; q < m; ++q) start[q + 1] = start[q] + counts[q];
    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t q = 0; q < m; ++q) {
        const int64_t i = idx[q];
        int64_t c = start[q];
        double v[3];
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double r2 = dist2(pos + 3 * i, pos + 3 * j, periodic_mask, extent, v);
            if (r2 > 0.0 && r2 < R2) list[c++] = (int32_t)j;
        }
    }
    free(start);
    return total;
}

void orc_cell_order(int64_t n, const double* pos, const double* origin, const double* cellw,
                    const int* ncell, int64_t* perm, int64_t* cell_start) {
    int64_t nc = (int64_t)ncell[0] * ncell[1] * ncell[2];
    int64_t* key = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) {
        int64_t c[3];
        for (int a = 0; a < 3; ++a) {
            double f = floor((pos[3 * i + a] - origin[a]) / cellw[a]);
            if (f < 0.0) f = 0.0;
            if (f > (double)(ncell[a] - 1)) f = (double)(ncell[a] - 1);
            c[a] = (int64_t)f;
        }
        key[i] = (c[2] * ncell[1] + c[1]) * ncell[0] + c[0];
    }
    /* counting sort visiting ids in ascending order = sort by (key, id) */
    for (int64_t c = 0; c <= nc; ++c) cell_start[c] = 0;
    for (int64_t i = 0; i < n; ++i) cell_start[key[i] + 1]++;
    for (int64_t c = 0; c < nc; ++c) cell_start[c + 1] += cell_start[c];
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nc > 0 ? nc : 1));
    for (int64_t c = 0; c < nc; ++c) fill[c] = cell_start[c];
    for (int64_t i = 0; i < n; ++i) perm[fill[key[i]]++] = i;
    free(fill);
    free(key);
}

/* ------------------------------------------------------------------------ */
typedef struct { double c[3], a[3], omega; int set; } orc_body;

struct orc_sim {
    orc_config cfg;
    double h, R2, vol, sigma0, nu_max;
    double dt_T;  /* Eq. (26) over the particles whose temperature is integrated */
    int kcap;
    orc_material mat[ORC_MAX_MAT];
    int mat_set[ORC_MAX_MAT];
    orc_body body[ORC_MAX_BODY];
    int64_t n, cap;
    int *kind, *mat_id, *body_id;
    double *pos, *vel, *rho, *drho, *p, *T, *T0, *mass;
    double *ref_pos, *ref_nrm, *nrm, *wvel, *av, *dTdt, *acc, *sigma, *snap, *contact, *rho_D;
    int64_t* nb_start;
    int32_t* nb;
    int64_t nb_cap;
    double t, last_dt_ad;
    int64_t adv_steps, substeps;
    int last_nsub;
    double tq_visc[ORC_MAX_BODY], tq_p[ORC_MAX_BODY], tq_inst[ORC_MAX_BODY], tq_int[ORC_MAX_BODY];
    double f_visc[ORC_MAX_BODY][3], f_p[ORC_MAX_BODY][3];
    double time_int;
    int started;
};

int orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

orc_sim* orc_create(const orc_config* cfg) {
    orc_sim* S = (orc_sim*)calloc(1, sizeof(orc_sim));
    S->cfg = *cfg;
    S->h = cfg->h_over_dx * cfg->dx;
    double R = 2.0 * S->h;
    S->R2 = R * R;
    S->vol = cfg->dx * cfg->dx * cfg->dx;
    S->sigma0 = orc_sigma0(cfg->dx, S->h);
    if (cfg->max_substeps > 0) S->kcap = cfg->max_substeps;
    else {
        /* READING: at most ceil(cfl_ad/cfl_ac (c0/u_ref + 1)) + 2 acoustic
         * sub-steps per advection step; the advection step ends early if the cap
         * is reached. */
        S->kcap = (int)ceil(cfg->cfl_ad / cfg->cfl_ac * (cfg->c0 / cfg->u_ref + 1.0)) + 2;
    }
    return S;
}

void orc_destroy(orc_sim* S) {
    if (!S) return;
    void* ptrs[] = {S->kind, S->mat_id, S->body_id, S->pos, S->vel, S->rho, S->drho, S->p, S->T,
                    S->T0, S->mass, S->ref_pos, S->ref_nrm, S->nrm, S->wvel, S->av, S->dTdt,
                    S->acc, S->sigma, S->snap, S->contact, S->rho_D, S->nb_start, S->nb};
    for (size_t k = 0; k < sizeof(ptrs) / sizeof(ptrs[0]); ++k) free(ptrs[k]);
    free(S);
}

int orc_set_material(orc_sim* S, int id, const orc_material* m) {
    if (id < 0 || id >= ORC_MAX_MAT || S->started) return -1;
    S->mat[id] = *m;
    S->mat_set[id] = 1;
    return 0;
}

int orc_set_rotation(orc_sim* S, int b, const double c[3], const double axis[3], double omega) {
    if (b < 0 || b >= ORC_MAX_BODY) return -1;
    for (int a = 0; a < 3; ++a) { S->body[b].c[a] = c[a]; S->body[b].a[a] = axis[a]; }
    S->body[b].omega = omega;
    S->body[b].set = 1;
    return 0;
}

static void grow(orc_sim* S, int64_t need) {
    if (need <= S->cap) return;
    int64_t c = S->cap ? S->cap : 1024;
    while (c < need) c *= 2;
#define RE(p, T, k) p = (T*)realloc(p, sizeof(T) * (size_t)(c * (k)))
    RE(S->kind, int, 1); RE(S->mat_id, int, 1); RE(S->body_id, int, 1);
    RE(S->pos, double, 3); RE(S->vel, double, 3); RE(S->rho, double, 1); RE(S->drho, double, 1);
    RE(S->p, double, 1); RE(S->T, double, 1); RE(S->T0, double, 1); RE(S->mass, double, 1);
    RE(S->ref_pos, double, 3); RE(S->ref_nrm, double, 3); RE(S->nrm, double, 3);
    RE(S->wvel, double, 3); RE(S->av, double, 3); RE(S->dTdt, double, 1); RE(S->acc, double, 3);
    RE(S->sigma, double, 1); RE(S->snap, double, 3); RE(S->contact, double, 1);
    RE(S->rho_D, double, 1);
#undef RE
    S->cap = c;
}

int orc_add_particles(orc_sim* S, int64_t n, const int* kind, const int* mat, const int* body,
                      const double* pos, const double* vel, const double* normal,
                      const double* T, const double* rho) {
    if (S->started) return -1;
    grow(S, S->n + n);
    for (int64_t q = 0; q < n; ++q) {
        int64_t i = S->n + q;
        int m = mat[q];
        if (m < 0 || m >= ORC_MAX_MAT || !S->mat_set[m]) return -2;
        S->kind[i] = kind[q];
        S->mat_id[i] = m;
        S->body_id[i] = kind[q] == 0 ? -1 : body[q];
        for (int a = 0; a < 3; ++a) {
            S->pos[3 * i + a] = pos[3 * q + a];
            S->ref_pos[3 * i + a] = pos[3 * q + a];
            S->vel[3 * i + a] = (kind[q] == 0 && vel) ? vel[3 * q + a] : 0.0;
            S->ref_nrm[3 * i + a] = (kind[q] == 1 && normal) ? normal[3 * q + a] : 0.0;
            S->nrm[3 * i + a] = S->ref_nrm[3 * i + a];
            S->wvel[3 * i + a] = 0.0;
            S->av[3 * i + a] = 0.0;
            S->acc[3 * i + a] = 0.0;
        }
        double r0 = S->mat[m].rho0;
        S->rho[i] = (kind[q] == 0 && rho && !isnan(rho[q])) ? rho[q] : r0;
        S->drho[i] = 0.0;
        S->p[i] = S->cfg.c0 * S->cfg.c0 * (S->rho[i] - r0);
        S->T[i] = T ? T[q] : S->mat[m].T_init;
        S->T0[i] = S->T[i];
        S->mass[i] = r0 * S->vol;
        S->dTdt[i] = 0.0;
        S->sigma[i] = 0.0;
        S->contact[i] = 0.0;
        S->rho_D[i] = S->rho[i];
    }
    S->n += n;
    return 0;
}

/* Rodrigues rotation of d about unit axis a by (cos, sin) */
static void rotate(const double a[3], double cs, double sn, const double d[3], double out[3]) {
    double axd[3] = {a[1] * d[2] - a[2] * d[1], a[2] * d[0] - a[0] * d[2], a[0] * d[1] - a[1] * d[0]};
    double ad = a[0] * d[0] + a[1] * d[1] + a[2] * d[2];
    for (int k = 0; k < 3; ++k) out[k] = cs * d[k] + sn * axd[k] + (1.0 - cs) * ad * a[k];
}

static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* torque about the body axis of force F applied at point r */
static double axial_torque(const orc_body* B, const double* r, const double* F) {
    double d[3] = {r[0] - B->c[0], r[1] - B->c[1], r[2] - B->c[2]};
    double tq[3] = {d[1] * F[2] - d[2] * F[1], d[2] * F[0] - d[0] * F[2], d[0] * F[1] - d[1] * F[0]};
    return dot3(tq, B->a);
}

static void build_neighbors(orc_sim* S) {
    int64_t n = S->n;
    if (!S->nb_start) S->nb_start = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
    int64_t* counts = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t total = orc_neighbors(n, S->snap, S->R2, S->cfg.periodic_mask, S->cfg.extent, counts, NULL, 0);
    if (total > S->nb_cap) {
        free(S->nb);
        S->nb_cap = total + total / 4 + 16;
        S->nb = (int32_t*)malloc(sizeof(int32_t) * (size_t)S->nb_cap);
    }
    orc_neighbors(n, S->snap, S->R2, S->cfg.periodic_mask, S->cfg.extent, counts, S->nb, S->nb_cap);
    S->nb_start[0] = 0;
    for (int64_t i = 0; i < n; ++i) S->nb_start[i + 1] = S->nb_start[i] + counts[i];
    free(counts);
}

/* pair geometry from the frozen snapshot: r_ij = r_i - r_j, |r_ij|, e_ij, dW/dr */
static void pair_geom(const orc_sim* S, int64_t i, int64_t j, double rv[3], double* r, double e[3],
                      double* dW) {
    double r2 = dist2(S->snap + 3 * i, S->snap + 3 * j, S->cfg.periodic_mask, S->cfg.extent, rv);
    *r = sqrt(r2);
    for (int a = 0; a < 3; ++a) e[a] = rv[a] / *r;
    *dW = orc_dW(*r, S->h);
}

static double fluid_volume(const orc_sim* S, int64_t j) {
    return S->kind[j] == 0 ? S->mass[j] / S->rho[j] : S->vol;
}

int orc_step(orc_sim* S, int n_adv) {
    const orc_config* C = &S->cfg;
    const int64_t n = S->n;
    const double h = S->h, c0 = C->c0, c02 = c0 * c0;
    S->started = 1;
    S->nu_max = 0.0;
    for (int64_t i = 0; i < n; ++i)
        if (S->kind[i] == 0) {
            double nu = S->mat[S->mat_id[i]].mu / S->mat[S->mat_id[i]].rho0;
            if (nu > S->nu_max) S->nu_max = nu;
        }
    /* READING of Eq. (26): the thermal bound caps the advection step for every
     * conducting material whose temperature is integrated (fluid, free solids);
     * cfl_T = 0 turns it off */
    S->dt_T = INFINITY;
    for (int64_t i = 0; i < n && C->cfl_T > 0.0; ++i) {
        const orc_material* M = &S->mat[S->mat_id[i]];
        if ((S->kind[i] == 0 || !M->fixed_T) && M->k > 0.0) {
            double d = orc_dt_thermal(C->cfl_T, M->rho0, M->cp, h, M->k);
            if (d < S->dt_T) S->dt_T = d;
        }
    }
    for (int st = 0; st < n_adv; ++st) {
        /* periodic wrap of fluid positions into the domain box */
        for (int64_t i = 0; i < n; ++i)
            for (int a = 0; a < 3; ++a)
                if ((C->periodic_mask & (1 << a)) && S->kind[i] == 0) {
                    double L = C->extent[a], o = C->origin[a];
                    if (S->pos[3 * i + a] >= o + L) S->pos[3 * i + a] -= L;
                    else if (S->pos[3 * i + a] < o) S->pos[3 * i + a] += L;
                }
        /* advection step size, Eq. (25) */
        double vmax = 0.0;
        for (int64_t i = 0; i < n; ++i)
            if (S->kind[i] == 0) {
                double v = sqrt(dot3(S->vel + 3 * i, S->vel + 3 * i));
                if (v > vmax) vmax = v;
            }
        double dt_ad, dt_ac0;
        orc_timesteps(h, vmax, C->u_ref, S->nu_max, c0, C->cfl_ad, C->cfl_ac, &dt_ad, &dt_ac0);
        if (S->dt_T < dt_ad) dt_ad = S->dt_T;

        /* rigid bodies: prescribed rotation theta = omega t about (c, axis) */
        for (int64_t i = 0; i < n; ++i) {
            if (S->kind[i] != 1) continue;
            int b = S->body_id[i];
            if (b < 0 || !S->body[b].set) {
                for (int a = 0; a < 3; ++a) { S->pos[3 * i + a] = S->ref_pos[3 * i + a]; S->wvel[3 * i + a] = 0.0; }
                continue;
            }
            const orc_body* B = &S->body[b];
            double th = B->omega * S->t, cs = cos(th), sn = sin(th);
            double d[3] = {S->ref_pos[3 * i] - B->c[0], S->ref_pos[3 * i + 1] - B->c[1], S->ref_pos[3 * i + 2] - B->c[2]};
            double rd[3];
            rotate(B->a, cs, sn, d, rd);
            for (int a = 0; a < 3; ++a) S->pos[3 * i + a] = B->c[a] + rd[a];
            rotate(B->a, cs, sn, S->ref_nrm + 3 * i, S->nrm + 3 * i);
            double w[3] = {B->omega * B->a[0], B->omega * B->a[1], B->omega * B->a[2]};
            S->wvel[3 * i + 0] = w[1] * rd[2] - w[2] * rd[1];
            S->wvel[3 * i + 1] = w[2] * rd[0] - w[0] * rd[2];
            S->wvel[3 * i + 2] = w[0] * rd[1] - w[1] * rd[0];
        }
        /* snapshot: pair geometry is frozen for the advection step (Sec. 2.8) */
        memcpy(S->snap, S->pos, sizeof(double) * 3 * (size_t)n);
        build_neighbors(S);

        /* ---- pass D: density re-initialisation, Eqs. (14)/(15) ---------- */
        #pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            if (S->kind[i] != 0) continue;
            double s = orc_W(0.0, h);
            for (int64_t q = S->nb_start[i]; q < S->nb_start[i + 1]; ++q) {
                int64_t j = S->nb[q];
                double rv[3];
                double r2 = dist2(S->snap + 3 * i, S->snap + 3 * j, C->periodic_mask, C->extent, rv);
                s += orc_W(sqrt(r2), h);
            }
            S->sigma[i] = s;
            double r0 = S->mat[S->mat_id[i]].rho0;
            double rr = r0 * s / S->sigma0;
            S->rho[i] = C->free_surface ? (S->rho[i] > rr ? S->rho[i] : rr) : rr;
            S->rho_D[i] = S->rho[i];
        }

        /* ---- pass V: viscous acceleration, Eq. (10) and Eq. (18) ---------- */
        for (int b = 0; b < ORC_MAX_BODY; ++b) { S->tq_visc[b] = 0.0; S->f_visc[b][0] = S->f_visc[b][1] = S->f_visc[b][2] = 0.0; }
        #pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            if (S->kind[i] != 0) continue;
            double a[3] = {0, 0, 0};
            double mu_i = S->mat[S->mat_id[i]].mu;
            for (int64_t q = S->nb_start[i]; q < S->nb_start[i + 1]; ++q) {
                int64_t j = S->nb[q];
                double rv[3], r, e[3], dW;
                pair_geom(S, i, j, rv, &r, e, &dW);
                double eta, vj[3];
                if (S->kind[j] == 0) {
                    double mu_j = S->mat[S->mat_id[j]].mu;
                    eta = (mu_i + mu_j > 0.0) ? 2.0 * mu_i * mu_j / (mu_i + mu_j) : 0.0;
                    for (int k = 0; k < 3; ++k) vj[k] = S->vel[3 * j + k];
                } else {
                    /* READING: the wall takes the fluid's viscosity, so the
                     * harmonic mean of Eq. (18) reduces to eta_i */
                    eta = mu_i;
                    for (int k = 0; k < 3; ++k) vj[k] = S->wvel[3 * j + k];
                }
                double c = 2.0 * fluid_volume(S, j) / S->rho[i] * eta / r * dW;
                for (int k = 0; k < 3; ++k) a[k] += c * (S->vel[3 * i + k] - vj[k]);
            }
            for (int k = 0; k < 3; ++k) S->av[3 * i + k] = a[k];
        }
        /* viscous force of the fluid on each rigid body (reaction of Eq. 18) */
        for (int64_t i = 0; i < n; ++i) {
            if (S->kind[i] != 0) continue;
            double mu_i = S->mat[S->mat_id[i]].mu;
            for (int64_t q = S->nb_start[i]; q < S->nb_start[i + 1]; ++q) {
                int64_t j = S->nb[q];
                if (S->kind[j] != 1) continue;
                int b = S->body_id[j];
                if (b < 0 || !S->body[b].set) continue;
                double rv[3], r, e[3], dW;
                pair_geom(S, i, j, rv, &r, e, &dW);
                double c = 2.0 * S->vol / S->rho[i] * mu_i / r * dW;
                double F[3];
                for (int k = 0; k < 3; ++k) F[k] = -S->mass[i] * c * (S->vel[3 * i + k] - S->wvel[3 * j + k]);
                S->tq_visc[b] += axial_torque(&S->body[b], S->snap + 3 * j, F);
                for (int k = 0; k < 3; ++k) S->f_visc[b][k] += F[k];
            }
        }

        /* ---- contact factor of rigid-body particles (Sec. 2.7) -------- */
        /* READING: V_j = m_j / rho_j of the lubricant partners at the advection
         * step (densities after re-initialisation); the fully immersed reference
         * is the kernel sum over the full lattice of spacing dx around the
         * particle, the particle itself excluded: dx^3 (sigma0 - W(0)). */
        {
            const double full = S->vol * (S->sigma0 - orc_W(0.0, S->h));
            #pragma omp parallel for schedule(static)
            for (int64_t i = 0; i < n; ++i) {
                const int b = S->body_id[i];
                if (S->kind[i] != 1 || b < 0 || !S->body[b].set) { S->contact[i] = 0.0; continue; }
                double s = 0.0;
                for (int64_t q = S->nb_start[i]; q < S->nb_start[i + 1]; ++q) {
                    int64_t j = S->nb[q];
                    if (S->kind[j] != 0) continue;
                    double rv[3];
                    double r2 = dist2(S->snap + 3 * i, S->snap + 3 * j, C->periodic_mask, C->extent, rv);
                    s += fluid_volume(S, j) * orc_W(sqrt(r2), S->h);
                }
                S->contact[i] = s / full;
            }
        }

        /* ---- pass T: Cleary conduction, Eq. (22) ---------------------- */
        #pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            const orc_material* Mi = &S->mat[S->mat_id[i]];
            if (S->kind[i] == 1 && Mi->fixed_T) { S->dTdt[i] = 0.0; continue; }
            double s = 0.0;
            for (int64_t q = S->nb_start[i]; q < S->nb_start[i + 1]; ++q) {
                int64_t j = S->nb[q];
                double rv[3], r, e[3], dW;
                pair_geom(S, i, j, rv, &r, e, &dW);
                double kj = S->mat[S->mat_id[j]].k;
                double K = (Mi->k + kj > 0.0) ? 4.0 * Mi->k * kj / (Mi->k + kj) : 0.0;
                s += fluid_volume(S, j) * K * (S->T[i] - S->T[j]) / r * dW;
            }
            double rho_i = S->kind[i] == 0 ? S->rho[i] : Mi->rho0;
            S->dTdt[i] = s / (rho_i * Mi->cp);
            /* READING (an extension: the paper's thermal model omits it): viscous
             * dissipation Phi = 2 mu S:S, S the symmetric part of the SPH velocity
             * gradient sum_j V_j (v_j - v_i) (x) grad_i W_ij over fluid and wall
             * partners (walls with their no-slip velocity), from the velocities of
             * the advection step; dT/dt += Phi / (rho c_p). */
            if (C->viscous_heating && S->kind[i] == 0) {
                double G[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
                for (int64_t q = S->nb_start[i]; q < S->nb_start[i + 1]; ++q) {
                    int64_t j = S->nb[q];
                    double rv[3], r, e[3], dW;
                    pair_geom(S, i, j, rv, &r, e, &dW);
                    const double* vj = S->kind[j] == 0 ? S->vel + 3 * j : S->wvel + 3 * j;
                    for (int a = 0; a < 3; ++a)
                        for (int b = 0; b < 3; ++b)
                            G[a][b] += fluid_volume(S, j) * (vj[a] - S->vel[3 * i + a]) * e[b] * dW;
                }
                double ss = 0.0;
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) {
                        const double sab = 0.5 * (G[a][b] + G[b][a]);
                        ss += sab * sab;
                    }
                S->dTdt[i] += 2.0 * Mi->mu * ss / (rho_i * Mi->cp);
            }
        }

        /* ---- acoustic sub-steps ---------------------------------------- */
        double tau = 0.0;
        int s = 0, last = 0;
        while (!last) {
            double vm = 0.0;
            for (int64_t i = 0; i < n; ++i)
                if (S->kind[i] == 0) {
                    double v = sqrt(dot3(S->vel + 3 * i, S->vel + 3 * i));
                    if (v > vm) vm = v;
                }
            double dt_ac = C->cfl_ac * h / (c0 + vm);
            double rem = dt_ad - tau, dt;
            int reach = rem <= dt_ac;
            dt = reach ? rem : dt_ac;
            last = reach || (s + 1 >= S->kcap);
            /* half kick of density, EoS Eq. (2), half drift */
            for (int64_t i = 0; i < n; ++i) {
                if (S->kind[i] != 0) continue;
                S->rho[i] += 0.5 * dt * S->drho[i];
                S->p[i] = c02 * (S->rho[i] - S->mat[S->mat_id[i]].rho0);
                for (int k = 0; k < 3; ++k) S->pos[3 * i + k] += 0.5 * dt * S->vel[3 * i + k];
            }
            /* pass M: pressure acceleration, Eqs. (10)-(12), (18)-(19) */
            #pragma omp parallel for schedule(static)
            for (int64_t i = 0; i < n; ++i) {
                if (S->kind[i] != 0) continue;
                double a[3] = {0, 0, 0};
                const double rho_i = S->rho[i], p_i = S->p[i];
                const double r0i = S->mat[S->mat_id[i]].rho0;
                for (int64_t q = S->nb_start[i]; q < S->nb_start[i + 1]; ++q) {
                    int64_t j = S->nb[q];
                    double rv[3], r, e[3], dW, pstar, Ustar;
                    pair_geom(S, i, j, rv, &r, e, &dW);
                    if (S->kind[j] == 0) {
                        double UL = -dot3(S->vel + 3 * i, e), UR = -dot3(S->vel + 3 * j, e);
                        orc_riemann(rho_i, UL, p_i, S->rho[j], UR, S->p[j], c0, &Ustar, &pstar);
                    } else {
                        /* r_fw = r_w - r_f = -r_ij */
                        double g_rfw = -dot3(C->gravity, rv);
                        double UL = -dot3(S->nrm + 3 * j, S->vel + 3 * i);
                        double uw = -dot3(S->nrm + 3 * j, S->wvel + 3 * j);
                        double UR, PR, rhoR;
                        orc_wall_riemann(rho_i, UL, p_i, uw, g_rfw, r0i, c0, C->wall_pstar_printed, &UR, &PR, &rhoR, &Ustar, &pstar);
                    }
                    double c = -2.0 * fluid_volume(S, j) / rho_i * pstar * dW;
                    for (int k = 0; k < 3; ++k) a[k] += c * e[k];
                }
                for (int k = 0; k < 3; ++k) S->acc[3 * i + k] = a[k];
            }
            /* pressure force of the fluid on each rigid body */
            for (int b = 0; b < ORC_MAX_BODY; ++b) { S->tq_p[b] = 0.0; S->f_p[b][0] = S->f_p[b][1] = S->f_p[b][2] = 0.0; }
            for (int64_t i = 0; i < n; ++i) {
                if (S->kind[i] != 0) continue;
                const double rho_i = S->rho[i], p_i = S->p[i];
                const double r0i = S->mat[S->mat_id[i]].rho0;
                for (int64_t q = S->nb_start[i]; q < S->nb_start[i + 1]; ++q) {
                    int64_t j = S->nb[q];
                    if (S->kind[j] != 1) continue;
                    int b = S->body_id[j];
                    if (b < 0 || !S->body[b].set) continue;
                    double rv[3], r, e[3], dW, pstar, Ustar, UR, PR, rhoR;
                    pair_geom(S, i, j, rv, &r, e, &dW);
                    double g_rfw = -dot3(C->gravity, rv);
                    double UL = -dot3(S->nrm + 3 * j, S->vel + 3 * i);
                    double uw = -dot3(S->nrm + 3 * j, S->wvel + 3 * j);
                    orc_wall_riemann(rho_i, UL, p_i, uw, g_rfw, r0i, c0, C->wall_pstar_printed, &UR, &PR, &rhoR, &Ustar, &pstar);
                    double c = -2.0 * S->vol / rho_i * pstar * dW;
                    double F[3];
                    for (int k = 0; k < 3; ++k) F[k] = -S->mass[i] * c * e[k];
                    S->tq_p[b] += axial_torque(&S->body[b], S->snap + 3 * j, F);
                    for (int k = 0; k < 3; ++k) S->f_p[b][k] += F[k];
                }
            }
            /* kick of velocity, second half drift */
            for (int64_t i = 0; i < n; ++i) {
                if (S->kind[i] != 0) continue;
                for (int k = 0; k < 3; ++k) {
                    S->vel[3 * i + k] += dt * (S->acc[3 * i + k] + S->av[3 * i + k] + C->gravity[k]);
                    S->pos[3 * i + k] += 0.5 * dt * S->vel[3 * i + k];
                }
            }
            /* pass C: continuity, Eqs. (10)-(13) and the wall problem (16)-(17).
             * READING of Eq. (13): U is measured along -e_ij (Eq. 11), so the
             * interface velocity is v* = -(U* - U~) e_ij + v~ (U~, v~ the
             * density-weighted means); then (v_i - v*).e_ij = U* - U_L. */
            #pragma omp parallel for schedule(static)
            for (int64_t i = 0; i < n; ++i) {
                if (S->kind[i] != 0) continue;
                double d = 0.0;
                const double rho_i = S->rho[i], p_i = S->p[i];
                const double r0i = S->mat[S->mat_id[i]].rho0;
                for (int64_t q = S->nb_start[i]; q < S->nb_start[i + 1]; ++q) {
                    int64_t j = S->nb[q];
                    double rv[3], r, e[3], dW, pstar, Ustar;
                    pair_geom(S, i, j, rv, &r, e, &dW);
                    if (S->kind[j] == 0) {
                        double UL = -dot3(S->vel + 3 * i, e), UR = -dot3(S->vel + 3 * j, e);
                        orc_riemann(rho_i, UL, p_i, S->rho[j], UR, S->p[j], c0, &Ustar, &pstar);
                        if (C->vstar_literal) {
                            /* Eq. (13) with its printed sign: v* = (U* - U~) e_ij + v~,
                             * U~ and v~ the density-weighted means of the two states */
                            const double rho_j = S->rho[j], srho = rho_i + rho_j;
                            const double Ut = (rho_i * UL + rho_j * UR) / srho;
                            double dv[3];
                            for (int k = 0; k < 3; ++k) {
                                const double vt = (rho_i * S->vel[3 * i + k] + rho_j * S->vel[3 * j + k]) / srho;
                                dv[k] = S->vel[3 * i + k] - ((Ustar - Ut) * e[k] + vt);
                            }
                            d += 2.0 * rho_i * fluid_volume(S, j) * dot3(dv, e) * dW;
                        } else
                            d += 2.0 * rho_i * fluid_volume(S, j) * (Ustar - UL) * dW;
                    } else {
                        /* READING: wall interface velocity v* = -U* n_w plus the
                         * fluid's tangential velocity, so (v_i - v*).e = (U* - U_L) n_w.e */
                        double g_rfw = -dot3(C->gravity, rv);
                        const double* nw = S->nrm + 3 * j;
                        double UL = -dot3(nw, S->vel + 3 * i);
                        double uw = -dot3(nw, S->wvel + 3 * j);
                        double UR, PR, rhoR;
                        orc_wall_riemann(rho_i, UL, p_i, uw, g_rfw, r0i, c0, C->wall_pstar_printed, &UR, &PR, &rhoR, &Ustar, &pstar);
                        d += 2.0 * rho_i * S->vol * (Ustar - UL) * dot3(nw, e) * dW;
                    }
                }
                S->drho[i] = d;
            }
            for (int64_t i = 0; i < n; ++i)
                if (S->kind[i] == 0) S->rho[i] += 0.5 * dt * S->drho[i];

            for (int b = 0; b < ORC_MAX_BODY; ++b) {
                S->tq_inst[b] = S->tq_p[b] + S->tq_visc[b];
                S->tq_int[b] += dt * S->tq_inst[b];
            }
            S->time_int += dt;
            tau = reach ? dt_ad : tau + dt;
            ++s;
        }
        /* temperature update with the step actually taken */
        for (int64_t i = 0; i < n; ++i) S->T[i] += tau * S->dTdt[i];
        S->t += tau;
        S->last_dt_ad = dt_ad;
        S->last_nsub = s;
        S->adv_steps += 1;
        S->substeps += s;
    }
    return 0;
}

int orc_get_field(const orc_sim* S, int field, double* out) {
    const int64_t n = S->n;
    switch (field) {
    case 0: memcpy(out, S->pos, sizeof(double) * 3 * (size_t)n); return 0;
    case 1: memcpy(out, S->vel, sizeof(double) * 3 * (size_t)n); return 0;
    case 2: memcpy(out, S->rho, sizeof(double) * (size_t)n); return 0;
    case 3:
        for (int64_t i = 0; i < n; ++i)
            out[i] = S->kind[i] == 0 ? S->cfg.c0 * S->cfg.c0 * (S->rho[i] - S->mat[S->mat_id[i]].rho0) : 0.0;
        return 0;
    case 4: memcpy(out, S->T, sizeof(double) * (size_t)n); return 0;
    case 5: memcpy(out, S->drho, sizeof(double) * (size_t)n); return 0;
    case 6: memcpy(out, S->av, sizeof(double) * 3 * (size_t)n); return 0;
    case 7: memcpy(out, S->dTdt, sizeof(double) * (size_t)n); return 0;
    case 8: memcpy(out, S->sigma, sizeof(double) * (size_t)n); return 0;
    case 9: memcpy(out, S->nrm, sizeof(double) * 3 * (size_t)n); return 0;
    case 10: memcpy(out, S->wvel, sizeof(double) * 3 * (size_t)n); return 0;
    case 11: memcpy(out, S->contact, sizeof(double) * (size_t)n); return 0;
    case 12: memcpy(out, S->rho_D, sizeof(double) * (size_t)n); return 0;
    default: return -1;
    }
}

int orc_torque_heat(const orc_sim* S, int b, double* torque, double* torque_avg,
                    double* heat_into_fluid, double* mean_fluid_T) {
    if (b < 0 || b >= ORC_MAX_BODY) return -1;
    *torque = S->tq_inst[b];
    *torque_avg = S->time_int > 0.0 ? S->tq_int[b] / S->time_int : 0.0;
    double H = 0.0, mT = 0.0, m = 0.0;
    for (int64_t i = 0; i < S->n; ++i) {
        if (S->kind[i] != 0) continue;
        H += S->mass[i] * S->mat[S->mat_id[i]].cp * (S->T[i] - S->T0[i]);
        mT += S->mass[i] * S->T[i];
        m += S->mass[i];
    }
    *heat_into_fluid = H;
    *mean_fluid_T = m > 0.0 ? mT / m : 0.0;
    return 0;
}

int orc_body_force(const orc_sim* S, int b, double* f) {
    if (b < 0 || b >= ORC_MAX_BODY) return -1;
    for (int k = 0; k < 3; ++k) f[k] = S->f_p[b][k] + S->f_visc[b][k];
    return 0;
}

int orc_time(const orc_sim* S, double* t, int64_t* adv, int64_t* sub, double* dt_ad, int* nsub) {
    *t = S->t;
    *adv = S->adv_steps;
    *sub = S->substeps;
    *dt_ad = S->last_dt_ad;
    *nsub = S->last_nsub;
    return 0;
}

int64_t orc_count(const orc_sim* S) { return S->n; }

/* ------------------------------------------------------------------------ */
/* Pass D and passes V/T of sampled fluid particles at any size.  The whole
 * state at the start of an advection step is given (positions = the frozen
 * snapshot, solids already placed, their velocities the wall velocities;
 * fluid densities before re-initialisation).  For each sampled fluid particle
 * i: its partners by brute force over all particles (the strict FP64 rule);
 * the re-initialised density (Eq. 14, or Eq. 15 when free_surface = 0) of i
 * and of each fluid partner, each from its own kernel sum over its own
 * brute-force partners (self and walls included); then the viscous
 * acceleration (Eq. 10 second term; Eq. 18 with the fluid's viscosity on
 * walls) and dT/dt by the Cleary form (Eq. 22), exactly as orc_step's
 * passes D, V and T compute them.  O(samples x partners x n): for checking a
 * few particles of a workload far beyond the stepper's O(N^2). */
static double reinit_rho(int64_t n, const double* pos, const double* rho, const int* mat_id,
                         const orc_material* mats, double R2, double h, double sigma0, int free_surface,
                         int periodic_mask, const double* extent, int64_t i) {
    double s = orc_W(0.0, h);
    for (int64_t j = 0; j < n; ++j) {
        double rv[3];
        const double r2 = dist2(pos + 3 * i, pos + 3 * j, periodic_mask, extent, rv);
        if (r2 > 0.0 && r2 < R2) s += orc_W(sqrt(r2), h);
    }
    const double rr = mats[mat_id[i]].rho0 * s / sigma0;
    return free_surface ? (rho[i] > rr ? rho[i] : rr) : rr;
}

int orc_sample_vt(int64_t n, const double* pos, const double* vel, const double* rho, const double* T,
                  const int* kind, const int* mat_id, const orc_material* mats, double dx, double h,
                  int free_surface, int periodic_mask, const double* extent, int64_t m, const int64_t* idx,
                  double* av, double* dTdt) {
    const double R2 = 4.0 * h * h, vol = dx * dx * dx, sigma0 = orc_sigma0(dx, h);
    int bad = 0;
    #pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
    for (int64_t q = 0; q < m; ++q) {
        const int64_t i = idx[q];
        if (i < 0 || i >= n || kind[i] != 0) { bad = 1; continue; }
        const orc_material* Mi = &mats[mat_id[i]];
        const double rho_i = reinit_rho(n, pos, rho, mat_id, mats, R2, h, sigma0, free_surface, periodic_mask,
                                        extent, i);
        double a[3] = {0.0, 0.0, 0.0}, sT = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            double rv[3];
            const double r2 = dist2(pos + 3 * i, pos + 3 * j, periodic_mask, extent, rv);
            if (!(r2 > 0.0 && r2 < R2)) continue;
            const double r = sqrt(r2), dW = orc_dW(r, h);
            const orc_material* Mj = &mats[mat_id[j]];
            double Vj, eta;
            if (kind[j] == 0) {
                const double rho_j = reinit_rho(n, pos, rho, mat_id, mats, R2, h, sigma0, free_surface,
                                                periodic_mask, extent, j);
                Vj = Mj->rho0 * vol / rho_j;
                eta = (Mi->mu + Mj->mu > 0.0) ? 2.0 * Mi->mu * Mj->mu / (Mi->mu + Mj->mu) : 0.0;
            } else {
                Vj = vol;
                eta = Mi->mu; /* READING: the wall takes the fluid's viscosity (Eq. 18) */
            }
            const double c = 2.0 * Vj / rho_i * eta / r * dW;
            for (int k = 0; k < 3; ++k) a[k] += c * (vel[3 * i + k] - vel[3 * j + k]);
            const double K = (Mi->k + Mj->k > 0.0) ? 4.0 * Mi->k * Mj->k / (Mi->k + Mj->k) : 0.0;
            sT += Vj * K * (T[i] - T[j]) / r * dW;
        }
        for (int k = 0; k < 3; ++k) av[3 * q + k] = a[k];
        dTdt[q] = sT / (rho_i * Mi->cp);
    }
    return bad ? -1 : 0;
}

/* Pass M of sampled fluid particles at any size, for the first acoustic
 * sub-step of an advection step: the densities re-initialised (Eq. 14/15,
 * as orc_sample_vt) and half-kicked with the given drho (rho += dt/2 drho),
 * the EoS (Eq. 2), then the pressure acceleration of Eqs. (10)-(12) over
 * fluid partners and Eqs. (16)-(19) over wall partners (n_w the wall
 * normals, the wall velocities in vel), as orc_step's pass M computes it.
 * The held viscous acceleration and gravity are not included. */
int orc_sample_ap(int64_t n, const double* pos, const double* vel, const double* rho, const double* drho,
                  const double* nrm, const int* kind, const int* mat_id, const orc_material* mats, double dx,
                  double h, int free_surface, const double* gravity, double c0, int wall_pstar_printed, double dt,
                  int periodic_mask, const double* extent, int64_t m, const int64_t* idx, double* ap) {
    const double R2 = 4.0 * h * h, vol = dx * dx * dx, sigma0 = orc_sigma0(dx, h), c02 = c0 * c0;
    int bad = 0;
    #pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
    for (int64_t q = 0; q < m; ++q) {
        const int64_t i = idx[q];
        if (i < 0 || i >= n || kind[i] != 0) { bad = 1; continue; }
        const double r0i = mats[mat_id[i]].rho0;
        double rho_i = reinit_rho(n, pos, rho, mat_id, mats, R2, h, sigma0, free_surface, periodic_mask, extent, i);
        rho_i += 0.5 * dt * drho[i];
        const double p_i = c02 * (rho_i - r0i);
        double a[3] = {0.0, 0.0, 0.0};
        for (int64_t j = 0; j < n; ++j) {
            double rv[3];
            const double r2 = dist2(pos + 3 * i, pos + 3 * j, periodic_mask, extent, rv);
            if (!(r2 > 0.0 && r2 < R2)) continue;
            const double r = sqrt(r2), dW = orc_dW(r, h);
            double e[3];
            for (int k = 0; k < 3; ++k) e[k] = rv[k] / r;
            double pstar, Ustar, Vj;
            if (kind[j] == 0) {
                double rho_j = reinit_rho(n, pos, rho, mat_id, mats, R2, h, sigma0, free_surface, periodic_mask,
                                          extent, j);
                rho_j += 0.5 * dt * drho[j];
                const double p_j = c02 * (rho_j - mats[mat_id[j]].rho0);
                const double UL = -dot3(vel + 3 * i, e), UR = -dot3(vel + 3 * j, e);
                orc_riemann(rho_i, UL, p_i, rho_j, UR, p_j, c0, &Ustar, &pstar);
                Vj = mats[mat_id[j]].rho0 * vol / rho_j;
            } else {
                /* r_fw = r_w - r_f = -r_ij */
                const double g_rfw = -dot3(gravity, rv);
                const double UL = -dot3(nrm + 3 * j, vel + 3 * i), uw = -dot3(nrm + 3 * j, vel + 3 * j);
                double UR, PR, rhoR;
                orc_wall_riemann(rho_i, UL, p_i, uw, g_rfw, r0i, c0, wall_pstar_printed, &UR, &PR, &rhoR, &Ustar,
                                 &pstar);
                Vj = vol;
            }
            const double c = -2.0 * Vj / rho_i * pstar * dW;
            for (int k = 0; k < 3; ++k) a[k] += c * e[k];
        }
        for (int k = 0; k < 3; ++k) ap[3 * q + k] = a[k];
    }
    return bad ? -1 : 0;
}

/* The first acoustic sub-step of an advection step for sampled fluid
 * particles, at any size: from the whole state at the step's start, or any
 * part of it that holds every particle within three support radii of each
 * sample (a sample's pass C reads its partners' kicked velocities, their pass
 * M reads their own partners' half-kicked densities, and those densities'
 * re-initialisation reads the next ring's positions).  In the order of
 * orc_step: re-initialised densities (Eq. 14/15), held viscous accelerations
 * (Eqs. 10, 18), the half kick of density and the EoS (Eq. 2), the velocity
 * kick of pass M (Eqs. 10-12, 16-19, plus g), then pass C's continuity rate
 * (Eqs. 10, 13 in the adopted reading of v*; walls Eqs. 16-17).  Outputs per
 * sample: the kicked velocity v_new[3] and the rate drho_new.  Work: one
 * brute-force scan per particle of the three rings.  Non-periodic cases. */
static int64_t partners_of(int64_t n, const double* pos, double R2, int64_t i, int64_t** buf, int64_t* cap) {
    int64_t k = 0;
    for (int64_t j = 0; j < n; ++j) {
        double rv[3];
        const double r2 = dist2(pos + 3 * i, pos + 3 * j, 0, NULL, rv);
        if (!(r2 > 0.0 && r2 < R2)) continue;
        if (k == *cap) {
            *cap = *cap ? 2 * *cap : 256;
            int64_t* grown = (int64_t*)realloc(*buf, sizeof(int64_t) * (size_t)*cap);
            if (!grown) abort(); /* test infrastructure: out of host memory ends the run */
            *buf = grown;
        }
        (*buf)[k++] = j;
    }
    return k;
}

/* the members of ring r + 1 (flag bit r + 1) from the partners of ring r */
static void next_ring(int64_t n, const double* pos, const int* kind, double R2, unsigned char* ring, int r) {
    int64_t* buf = NULL;
    int64_t cap = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (!(ring[i] & (1u << r)) || kind[i] != 0) continue;
        const int64_t k = partners_of(n, pos, R2, i, &buf, &cap);
        for (int64_t q = 0; q < k; ++q) ring[buf[q]] |= (unsigned char)(1u << (r + 1));
    }
    free(buf);
}

int orc_sample_substep(int64_t n, const double* pos, const double* vel, const double* rho, const double* drho,
                       const double* nrm, const int* kind, const int* mat_id, const orc_material* mats, double dx,
                       double h, int free_surface, const double* gravity, double c0, int wall_pstar_printed,
                       double dt, int64_t m, const int64_t* idx, double* v_new, double* drho_new) {
    const double R2 = 4.0 * h * h, vol = dx * dx * dx, sigma0 = orc_sigma0(dx, h), c02 = c0 * c0;
    for (int64_t q = 0; q < m; ++q)
        if (idx[q] < 0 || idx[q] >= n || kind[idx[q]] != 0) return -1;
    unsigned char* ring = (unsigned char*)calloc((size_t)n, 1);
    double* rho_re = (double*)malloc(sizeof(double) * (size_t)n);  /* re-initialised density */
    double* rho_h = (double*)malloc(sizeof(double) * (size_t)n);   /* half-kicked density */
    double* vk = (double*)malloc(sizeof(double) * 3 * (size_t)n);  /* kicked velocity */
    if (!ring || !rho_re || !rho_h || !vk) {
        free(ring);
        free(rho_re);
        free(rho_h);
        free(vk);
        return -2;
    }
    for (int64_t q = 0; q < m; ++q) ring[idx[q]] |= 1u;
    next_ring(n, pos, kind, R2, ring, 0); /* partners of the samples */
    next_ring(n, pos, kind, R2, ring, 1); /* their partners */
    /* re-initialisation and half kick of every fluid particle of the three rings */
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        if (!ring[i] || kind[i] != 0) continue;
        rho_re[i] = reinit_rho(n, pos, rho, mat_id, mats, R2, h, sigma0, free_surface, 0, NULL, i);
        rho_h[i] = rho_re[i] + 0.5 * dt * drho[i];
    }
    /* viscous and pressure accelerations, velocity kick: samples and their partners */
    #pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < n; ++i) {
        if (!(ring[i] & 3u) || kind[i] != 0) continue;
        const orc_material* Mi = &mats[mat_id[i]];
        const double p_i = c02 * (rho_h[i] - Mi->rho0);
        double av[3] = {0, 0, 0}, ap[3] = {0, 0, 0};
        for (int64_t j = 0; j < n; ++j) {
            double rv[3];
            const double r2 = dist2(pos + 3 * i, pos + 3 * j, 0, NULL, rv);
            if (!(r2 > 0.0 && r2 < R2)) continue;
            const double r = sqrt(r2), dW = orc_dW(r, h);
            double e[3];
            for (int k = 0; k < 3; ++k) e[k] = rv[k] / r;
            double eta, Vre, Vh, pstar, Ustar;
            if (kind[j] == 0) {
                const orc_material* Mj = &mats[mat_id[j]];
                eta = (Mi->mu + Mj->mu > 0.0) ? 2.0 * Mi->mu * Mj->mu / (Mi->mu + Mj->mu) : 0.0;
                Vre = Mj->rho0 * vol / rho_re[j];
                Vh = Mj->rho0 * vol / rho_h[j];
                const double p_j = c02 * (rho_h[j] - Mj->rho0);
                orc_riemann(rho_h[i], -dot3(vel + 3 * i, e), p_i, rho_h[j], -dot3(vel + 3 * j, e), p_j, c0, &Ustar,
                            &pstar);
            } else {
                eta = Mi->mu; /* READING: the wall takes the fluid's viscosity (Eq. 18) */
                Vre = Vh = vol;
                double UR, PR, rhoR;
                orc_wall_riemann(rho_h[i], -dot3(nrm + 3 * j, vel + 3 * i), p_i, -dot3(nrm + 3 * j, vel + 3 * j),
                                 -dot3(gravity, rv), Mi->rho0, c0, wall_pstar_printed, &UR, &PR, &rhoR, &Ustar,
                                 &pstar);
            }
            const double cv = 2.0 * Vre / rho_re[i] * eta / r * dW, cp = -2.0 * Vh / rho_h[i] * pstar * dW;
            for (int k = 0; k < 3; ++k) {
                av[k] += cv * (vel[3 * i + k] - vel[3 * j + k]);
                ap[k] += cp * e[k];
            }
        }
        for (int k = 0; k < 3; ++k) vk[3 * i + k] = vel[3 * i + k] + dt * (ap[k] + av[k] + gravity[k]);
    }
    /* pass C of the samples, from the kicked velocities (walls keep theirs) */
    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t q = 0; q < m; ++q) {
        const int64_t i = idx[q];
        const orc_material* Mi = &mats[mat_id[i]];
        const double p_i = c02 * (rho_h[i] - Mi->rho0);
        double d = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            double rv[3];
            const double r2 = dist2(pos + 3 * i, pos + 3 * j, 0, NULL, rv);
            if (!(r2 > 0.0 && r2 < R2)) continue;
            const double r = sqrt(r2), dW = orc_dW(r, h);
            double e[3];
            for (int k = 0; k < 3; ++k) e[k] = rv[k] / r;
            double pstar, Ustar;
            const double UL = -dot3(vk + 3 * i, e);
            if (kind[j] == 0) {
                const orc_material* Mj = &mats[mat_id[j]];
                const double p_j = c02 * (rho_h[j] - Mj->rho0);
                orc_riemann(rho_h[i], UL, p_i, rho_h[j], -dot3(vk + 3 * j, e), p_j, c0, &Ustar, &pstar);
                d += 2.0 * rho_h[i] * (Mj->rho0 * vol / rho_h[j]) * (Ustar - UL) * dW;
            } else {
                /* READING: wall interface velocity -U* n_w plus the fluid's tangential velocity */
                const double* nw = nrm + 3 * j;
                const double ULw = -dot3(nw, vk + 3 * i), uw = -dot3(nw, vel + 3 * j);
                double UR, PR, rhoR;
                orc_wall_riemann(rho_h[i], ULw, p_i, uw, -dot3(gravity, rv), Mi->rho0, c0, wall_pstar_printed, &UR,
                                 &PR, &rhoR, &Ustar, &pstar);
                d += 2.0 * rho_h[i] * vol * (Ustar - ULw) * dot3(nw, e) * dW;
            }
        }
        drho_new[q] = d;
        for (int k = 0; k < 3; ++k) v_new[3 * q + k] = vk[3 * i + k];
    }
    free(ring);
    free(rho_re);
    free(rho_h);
    free(vk);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Physics-driven particle relaxation (Sec. 2.2).  Particles move under the
 * constant background pressure p0 (scale-free: p0 / rho0 = 1),
 *   F_p,i = -(2 / m_i) sum_j V_i V_j p0 grad_i W_ij = -2 sum_j V_j W'(r) e_ij,
 * with r += F_p dt^2 / 2 and dt = 0.25 sqrt(h / max |F_p|).
 * READING of the static level-set confinement the paper takes from its
 * reference: (i) the kernel volume missing beyond the surface is replaced by
 * the half space at the particle's depth d = -phi: sum over it of V grad_i W
 * = n A(d), n the outward unit normal grad phi / |grad phi|, A(d) =
 * 2 pi int_d^{2h} W(r) r dr; (ii) a particle that ends a step outside
 * (phi > 0) is moved back along n onto the surface, x -= phi n. */
double orc_relax_A(double d, double h) {
    if (d < 0.0) d = 0.0;
    const double R = 2.0 * h;
    if (d >= R) return 0.0;
    const int m = 2000; /* Simpson on [d, 2h] */
    const double a = d, b = R, dh = (b - a) / m;
    double s = orc_W(a, h) * a + orc_W(b, h) * b;
    for (int k = 1; k < m; ++k) {
        const double r = a + k * dh;
        s += (k % 2 ? 4.0 : 2.0) * orc_W(r, h) * r;
    }
    return 2.0 * PI * s * dh / 3.0;
}

static double phi_node(const orc_relax_config* c, int i, int j, int k) {
    if (i < 0) i = 0;
    if (j < 0) j = 0;
    if (k < 0) k = 0;
    if (i > c->nphi[0] - 1) i = c->nphi[0] - 1;
    if (j > c->nphi[1] - 1) j = c->nphi[1] - 1;
    if (k > c->nphi[2] - 1) k = c->nphi[2] - 1;
    return c->phi[((int64_t)k * c->nphi[1] + j) * c->nphi[0] + i];
}

/* central difference of phi along axis a at node (i, j, k) (one-sided at the
 * grid's faces) */
static double phi_grad_node(const orc_relax_config* c, int i, int j, int k, int a) {
    int lo[3] = {i, j, k}, hi[3] = {i, j, k};
    lo[a] -= 1;
    hi[a] += 1;
    const int idx[3] = {i, j, k};
    double span = 2.0;
    if (lo[a] < 0) { lo[a] = idx[a]; span -= 1.0; }
    if (hi[a] > c->nphi[a] - 1) { hi[a] = idx[a]; span -= 1.0; }
    return (phi_node(c, hi[0], hi[1], hi[2]) - phi_node(c, lo[0], lo[1], lo[2])) / (span * c->phi_spacing);
}

/* trilinear interpolation of phi; n_out = the normalised trilinear
 * interpolation of the nodes' central-difference gradients (continuous, so
 * mirror-image points get mirror-image normals) */
double orc_phi(const orc_relax_config* c, const double* x, double* n_out) {
    double u[3], f[3];
    int b[3];
    for (int a = 0; a < 3; ++a) {
        u[a] = (x[a] - c->phi_origin[a]) / c->phi_spacing;
        double fl = floor(u[a]);
        if (fl < 0.0) fl = 0.0;
        if (fl > c->nphi[a] - 2) fl = c->nphi[a] - 2;
        b[a] = (int)fl;
        f[a] = u[a] - fl;
    }
    double phi = 0.0, g[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < 2; ++k)
        for (int j = 0; j < 2; ++j)
            for (int i = 0; i < 2; ++i) {
                const double w = (i ? f[0] : 1.0 - f[0]) * (j ? f[1] : 1.0 - f[1]) * (k ? f[2] : 1.0 - f[2]);
                phi += w * phi_node(c, b[0] + i, b[1] + j, b[2] + k);
                for (int a = 0; a < 3; ++a) g[a] += w * phi_grad_node(c, b[0] + i, b[1] + j, b[2] + k, a);
            }
    if (n_out) {
        const double gn = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
        for (int a = 0; a < 3; ++a) n_out[a] = gn > 0.0 ? g[a] / gn : 0.0;
    }
    return phi;
}

int orc_relax(const orc_relax_config* cfg, int64_t n, double* pos, int iterations, double* max_accel) {
    const double dx = cfg->dx, h = cfg->h_over_dx * dx, R2 = 4.0 * h * h, V = dx * dx * dx;
    double* acc = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    for (int it = 0; it < iterations; ++it) {
        double amax = 0.0;
        #pragma omp parallel for schedule(dynamic, 64) reduction(max : amax)
        for (int64_t i = 0; i < n; ++i) {
            double a[3] = {0.0, 0.0, 0.0}, v[3];
            for (int64_t j = 0; j < n; ++j) {
                if (j == i) continue;
                const double r2 = dist2(pos + 3 * i, pos + 3 * j, 0, NULL, v);
                if (!(r2 > 0.0 && r2 < R2)) continue;
                const double r = sqrt(r2), c = -2.0 * V * orc_dW(r, h) / r;
                for (int k = 0; k < 3; ++k) a[k] += c * v[k];
            }
            double nrm[3];
            const double phi = orc_phi(cfg, pos + 3 * i, nrm);
            const double A = orc_relax_A(-phi, h);
            for (int k = 0; k < 3; ++k) a[k] += -2.0 * nrm[k] * A;
            for (int k = 0; k < 3; ++k) acc[3 * i + k] = a[k];
            const double am = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
            if (am > amax) amax = am;
        }
        if (max_accel) max_accel[it] = amax;
        if (!(amax > 0.0)) continue;
        const double dt = 0.25 * sqrt(h / amax);
        #pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            double* x = pos + 3 * i;
            for (int k = 0; k < 3; ++k) x[k] = x[k] + 0.5 * acc[3 * i + k] * dt * dt;
            double nrm[3];
            const double phi = orc_phi(cfg, x, nrm);
            if (phi > 0.0)
                for (int k = 0; k < 3; ++k) x[k] -= phi * nrm[k];
        }
    }
    free(acc);
    return 0;
}
