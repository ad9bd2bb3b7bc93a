/* sph.h -- C ABI of the B300 (sm_103a) coupled fluid-solid-thermal SPH library.
 *
 * One library call advances weakly-compressible SPH particles through the
 * method of arXiv 2512.09904 (Sec. 2): a cell-linked-list neighbour search,
 * Riemann-based continuity and pressure force, viscous force, fluid-wall and
 * rotating-rigid-body coupling, Cleary heat conduction, and dual-criteria
 * time integration.  Every step runs in this library's CUDA kernels; there is
 * no CPU fallback.
 *
 * Conventions (all entry points):
 *  - Every function returns sph_status and never throws.  On error,
 *    sph_last_error(ctx) gives a one-line message (per context).
 *  - Pointers documented as "host" are read (or written) before the call
 *    returns; the caller keeps ownership.  Pointers documented as "device"
 *    must be CUDA device allocations on the current device.
 *  - Device memory of a context is allocated by the library (cudaMalloc) at
 *    its first step and freed by sph_destroy; a batch allocates at
 *    sph_batch_create and frees at sph_batch_destroy.
 *  - Work is issued on the CUDA stream given at creation (NULL = legacy
 *    default stream).  Calls that return host data synchronise that stream.
 *  - One context must not be used by two host threads at the same time.
 *  - Particle ids are assigned in call order starting at 0; fields are read
 *    back in id order.  Particles may only be added before the first step
 *    (SPH_ESTATE afterwards).
 *  - Units are SI, temperatures in kelvin.
 */
#ifndef SPH_B300_H
#define SPH_B300_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sph_ctx sph_ctx;

typedef enum {
    SPH_OK = 0,
    SPH_EINVAL = -1,    /* bad argument (size, id, layout) */
    SPH_ENOMEM = -2,    /* device allocation or admission budget failed */
    SPH_ECUDA = -3,     /* a CUDA runtime call failed */
    SPH_EUNSTABLE = -4, /* NaN/Inf state or a fluid particle left the domain box */
    SPH_ETIMEOUT = -5,  /* reserved: a bounded device wait gave up */
    SPH_ESTATE = -6     /* call not valid in the current state */
} sph_status;

/* Case configuration.  The domain box holds every particle for the whole run;
 * it is cut into geometry cells of width >= 2h per axis, each split into 8
 * sort cells along x (width >= h/4) and 2 along y and z (width >= h): the
 * cell-linked list.  The neighbour search walks the rows of sort cells within
 * two of a particle's along y and z whose slab its 2h sphere reaches, and in
 * each row the sort cells the sphere reaches.  A periodic axis wraps particle
 * positions on this machine and needs at least 3 geometry cells along it. */
typedef struct {
    double origin[3], extent[3]; /* domain box, m */
    double dx;                   /* particle spacing, m (mass = rho0 dx^3, wall volume dx^3) */
    double h_over_dx;            /* smoothing length h = h_over_dx * dx (Wendland C2, support 2h) */
    double gravity[3];           /* m/s^2 */
    double c0;                   /* artificial sound speed of the EoS p = c0^2 (rho - rho0), Eq. (2) */
    double u_ref;                /* velocity floor of the advection criterion, normally c0/10 */
    double cfl_ad, cfl_ac;       /* 0.25 and 0.6 in the paper, Eq. (25) */
    int free_surface;            /* 1: re-initialise rho = max(rho, rho0 sumW/sumW0), Eq. (14); 0: Eq. (15) */
    int periodic_mask;           /* bit a set: axis a is periodic */
    int max_substeps;            /* cap on acoustic sub-steps per advection step; 0 = ceil(cfl_ad/cfl_ac (c0/u_ref + 1)) + 2 */
    int pair_precision;          /* 0: FP32 pair arithmetic, FP64 positions, temperatures and
                                    reductions (default); 1: FP64 pair arithmetic and particle
                                    state throughout (the plain FP64 method, for small cases;
                                    not admissible to a batch).  Other values: SPH_EINVAL. */
    int viscous_heating;         /* 1: add the viscous-dissipation heating Phi = 2 mu S:S to
                                    dT/dt (S from the SPH velocity gradient over fluid and wall
                                    partners); an extension: the paper's thermal model omits it
                                    (Sec. 2.6).  0 (default): the paper's model.  Other values:
                                    SPH_EINVAL. */
    int vstar_literal;           /* 0 (default): Eq. (13)'s interface velocity read with U measured
                                    along -e_ij as in Eq. (11), v* = -(U* - U~) e_ij + v~, so that
                                    (v_i - v*).e_ij = U* - U_L; 1: the sign as printed,
                                    v* = (U* - U~) e_ij + v~, which turns the pressure-difference
                                    term of the continuity sum anti-diffusive (for study; needs
                                    pair_precision = 1).  Other values, or 1 with FP32 pairs:
                                    SPH_EINVAL. */
    double cfl_T;                /* Eq. (26): dt_ad <= cfl_T rho c_p h^2 / k over every conducting
                                    material whose temperature is integrated (fluid, free
                                    solids); 0.5 as printed.  0: no thermal bound.  The printed
                                    0.5 keeps the Cleary update stable at h = 1.0 dx but not at
                                    h = 1.3 dx in 3-D, where about 0.2 is needed.  Negative or
                                    NaN: SPH_EINVAL. */
    int wall_pstar_printed;      /* 0 (default): the wall interface pressure of the one-sided
                                    problem (Sec. 2.5) is Eq. (19)'s density-weighted mean of
                                    the fluid and mirror pressures plus Eq. (12)'s limiter term
                                    rho_f rho_R beta (U_L - U_R) / (rho_f + rho_R) on the same
                                    states, so that a particle approaching a wall meets a
                                    rising pressure; 1: Eq. (19) exactly as printed, without
                                    that term (for study; needs pair_precision = 1).  Other
                                    values, or 1 with FP32 pairs: SPH_EINVAL. */
} sph_config;

/* Material table entry (Sec. 2.6 and the paper's property tables). */
typedef struct {
    double rho0;    /* reference density, kg/m^3 */
    double mu;      /* dynamic viscosity, Pa s (fluids) */
    double k;       /* thermal conductivity, W/(m K); 0 = adiabatic */
    double cp;      /* specific heat, J/(kg K) */
    double T_init;  /* default initial temperature, K */
    int fixed_T;    /* solids only: 1 = temperature held (heat source/sink) */
} sph_material;

/* Create a single-case context: the problem of Sec. 2.1 (weakly compressible
 * flow, Eq. 1, closed by the linear EoS of Eq. 2 with sound speed c0) on the
 * particle spacing dx and smoothing length h, stepped by the dual criteria of
 * Sec. 2.8 (Eq. 25 with cfl_ad, cfl_ac; Eq. 26 with cfl_T) and re-initialised
 * by Eq. (14) or (15) (Sec. 2.4, free_surface).  cfg: host, copied.
 * cuda_stream: a cudaStream_t or NULL.  *out receives the context, owned by
 * the caller until sph_destroy.
 * Errors: SPH_EINVAL (non-positive dx/h/extent, periodic axis with < 3 cells,
 * a switch out of range), SPH_ECUDA. */
sph_status sph_create(const sph_config* cfg, void* cuda_stream, sph_ctx** out);

/* Free the context and all its device memory.  NULL is accepted. */
sph_status sph_destroy(sph_ctx* ctx);

/* Set material `material_id` (0..15): the reference density rho0 of Eq. (2),
 * the dynamic viscosity eta of Eq. (10) and Eq. (18), and the conductivity k
 * and specific heat c_p of the Cleary conduction, Eq. (22) (Sec. 2.6); the
 * paper's values are its Table 3 (slabs) and Table 6 (lubricant and gears).
 * mat: host, copied.  Must precede the particles that use it and the first
 * step.  Errors: SPH_EINVAL (id out of range, NULL, rho0 or c_p not
 * positive, k or eta negative), SPH_ESTATE. */
sph_status sph_set_material(sph_ctx* ctx, int material_id, const sph_material* mat);

/* Append n fluid particles of material `material_id`.
 * pos: host double[n*3] (x,y,z per particle).  vel: host double[n*3] or NULL
 * (rest).  T: host double[n] or NULL (material T_init).  rho: host double[n]
 * or NULL (material rho0).  *first_id (may be NULL) receives the first id.
 * Errors: SPH_EINVAL, SPH_ESTATE (after the first step). */
sph_status sph_add_fluid(sph_ctx* ctx, int material_id, int64_t n, const double* pos,
                         const double* vel, const double* T, const double* rho, int64_t* first_id);

/* Append n solid (dummy wall) particles, Sec. 2.5.  body_id: -1 for a static
 * wall, 0..3 for a rigid body whose motion is set by sph_set_rotation.
 * pos: host double[n*3] reference positions (at time 0).  normal: host
 * double[n*3] unit wall normals pointing into the fluid.  T: host double[n] or
 * NULL.  Errors: SPH_EINVAL, SPH_ESTATE. */
sph_status sph_add_solid(sph_ctx* ctx, int body_id, int material_id, int64_t n, const double* pos,
                         const double* normal, const double* T, int64_t* first_id);

/* Prescribed rigid rotation of body `body_id` (0..3), as the gears of the
 * paper's gearbox runs are driven at set shaft speeds (Sec. 4.1, Table 5):
 * angle omega*t (rad/s) about the unit axis through center (host double[3]
 * each, m, copied); the body's dummy particles move with it and their wall
 * velocity omega x (r - center) enters the wall problem of Sec. 2.5.
 * Errors: SPH_EINVAL (id out of range, axis not unit), SPH_ESTATE. */
sph_status sph_set_rotation(sph_ctx* ctx, int body_id, const double center[3], const double axis[3],
                            double omega);

/* Advance n advection steps (each with its acoustic sub-steps, Sec. 2.8).
 * *sim_time_out (may be NULL) receives the simulated time.  The first call
 * uploads the particles and builds the step's CUDA graph.
 * Errors: SPH_EUNSTABLE (state no longer finite or a fluid particle left the
 * box; the case is frozen after the advection step that found it, so later
 * calls leave its state unchanged and return SPH_EUNSTABLE again, and the
 * context stays readable), SPH_ENOMEM, SPH_ECUDA. */
sph_status sph_step(sph_ctx* ctx, int n_advection_steps, double* sim_time_out);

/* Churning torque and heat-up.  torque_axis: torque of the fluid on body
 * `body_id` about its axis at the last acoustic sub-step (pressure + viscous
 * wall forces of Eq. 18, applied at the wall particles), N m.
 * torque_time_avg: its sub-step-weighted mean since the first step.
 * heat_into_fluid: sum over fluid of m cp (T - T_initial), J.
 * mean_fluid_T: mass-weighted mean fluid temperature, K.  Any output pointer
 * may be NULL.  All four are FP64 reductions in a fixed order.
 * Errors: SPH_EINVAL (body id), SPH_ESTATE (no step taken yet). */
sph_status sph_read_torque_heat(sph_ctx* ctx, int body_id, double* torque_axis,
                                double* torque_time_avg, double* heat_into_fluid,
                                double* mean_fluid_T);

/* Torque and heat-up history of the context: the last n (<= max_steps, <=
 * 4096) advection-step records, oldest first, 8 doubles each: simulated time
 * at the end of the step, torque of body 0 about its axis (as
 * sph_read_torque_heat), its running time average, heat into fluid, mean
 * fluid temperature, dt_ad of the step, acoustic sub-steps of the step, the
 * max fluid speed that set dt_ad.  out: host double[8 * max_steps], owned by the caller; n_out
 * may be NULL.  Errors: SPH_EINVAL (out NULL, max_steps < 0), SPH_ESTATE
 * (not started), SPH_ECUDA. */
sph_status sph_read_curve(sph_ctx* ctx, double* out, int64_t max_steps, int64_t* n_out);

/* Field ids for sph_read_fields (values as double, original id order). */
enum {
    SPH_FIELD_POS = 0,      /* n*3; solids: at the current simulation time */
    SPH_FIELD_VEL = 1,      /* n*3; solids: wall velocity at the current time */
    SPH_FIELD_RHO = 2,      /* n; rho0 for solids */
    SPH_FIELD_P = 3,        /* n; 0 for solids */
    SPH_FIELD_T = 4,        /* n */
    SPH_FIELD_DRHO = 5,     /* n; last continuity rate */
    SPH_FIELD_AVISC = 6,    /* n*3; viscous acceleration of the last advection step */
    SPH_FIELD_DTDT = 7,     /* n; conduction rate of the last advection step */
    SPH_FIELD_NORMAL = 9,   /* n*3; wall normal at the current time (solids) */
    SPH_FIELD_CONTACT = 11  /* n; contact factor of rigid-body particles (Sec. 2.7, Eq. 24):
                               sum of V_j W_ij over lubricant partners, V_j = m_j / rho_j,
                               over its fully immersed value dx^3 (sum of W over the full
                               lattice, the particle itself excluded); last advection
                               step; 0 for fluid and static walls */
};

/* Copy field `field` of all n particles (n must equal the particle count)
 * into host_dst (host double, n or n*3 values, owned by the caller), in
 * particle id order: the state of Eq. (1) (positions, velocities, densities
 * and the EoS pressure of Eq. 2), the temperature of Eq. (4), the rates of
 * the last step (continuity, Eq. 10; viscous acceleration; conduction,
 * Eq. 22) and the contact factor of Eq. (24).
 * Errors: SPH_EINVAL (unknown field, n mismatch, NULL), SPH_ESTATE. */
sph_status sph_read_fields(sph_ctx* ctx, int field, void* host_dst, int64_t n);

/* Neighbour pairs of the last advection step's frozen snapshot (pair
 * membership 0 < |r_i - r_j|^2 < (2h)^2 decided exactly as in FP64).  After
 * the first step: the pairs of the initial positions.
 * counts: host int64[n] (per id).  ids: host int32[cap] or NULL; receives,
 * for each id in order, its neighbour ids in ascending order.  *total gets the
 * number of entries.  Errors: SPH_EINVAL (cap too small), SPH_ESTATE. */
sph_status sph_read_neighbors(sph_ctx* ctx, int64_t* counts, int32_t* ids, int64_t cap,
                              int64_t* total);

/* Cell order of the last neighbour search: perm[k] = id at sorted position k
 * (sorted by cell index, x fastest, then id).  host int64[n].  Errors:
 * SPH_ESTATE before the first step. */
sph_status sph_read_cell_order(sph_ctx* ctx, int64_t* perm, int64_t n);

typedef struct {
    int64_t n_fluid, n_solid;
    double t;                 /* simulated time */
    int64_t adv_steps, substeps;
    double last_dt_ad;
    int last_nsub;
    int kcap;                 /* sub-step cap per advection step */
    int ncell[3];             /* sort cells per axis (8 per geometry cell along x, 2 along y, z) */
    double cell_width[3];     /* sort-cell width (>= h/4 along x, >= h along y, z) */
    int error_bits;           /* 1 NaN/Inf, 2 fluid left the box */
    int graph_launches;       /* kernels per advection step of the profiling graph (kcap sub-step slots) */
    int kernels_fixed;        /* kernels per advection step of the stepping graph: kernels_fixed + */
    int kernels_per_substep;  /* kernels_per_substep x (its sub-steps) */
    int info_bits;            /* 4: since creation, some particle had more partners than its
                                 128-entry list holds and took the 27-cell loop instead (results
                                 unchanged; informational) */
} sph_info;

/* Fill *info (host) with the context's sizes, grid, clock and flags; before the
 * first step only the static fields are set.  Errors: SPH_EINVAL (NULL),
 * SPH_ECUDA (reading the step state back). */
sph_status sph_get_info(sph_ctx* ctx, sph_info* info);

/* Directed neighbour pairs of fluid particles in the current snapshot, by
 * partner kind (fluid, wall).  Used to turn kernel times into pair rates.
 * Errors: SPH_ESTATE (no step yet), SPH_ECUDA. */
sph_status sph_pair_stats(sph_ctx* ctx, int64_t* fluid_fluid, int64_t* fluid_wall);

/* Work of the current snapshot's neighbour search (pass D): particles
 * searched, candidates tested (sum of their 27-cell populations) and
 * partners found.  Used to turn pass-D times into search rates.
 * Errors: SPH_ESTATE (no step yet), SPH_EINVAL (NULL output), SPH_ECUDA. */
sph_status sph_search_stats(sph_ctx* ctx, int64_t* searched, int64_t* candidates, int64_t* partners);

/* Measured FP32 throughput of the current device, the denominator of the
 * pair passes' ALU roofline (they are bound by FP32 issue, not by HBM or
 * tensor cores): a probe kernel in which every thread of one full wave of
 * resident blocks runs independent chains of FP32 fused multiply-adds
 * (2 flops each), timed with device events on `stream` after a warm-up
 * launch.  Stateless (no context).  tflops: host, TFLOP/s of the fastest of
 * `reps` launches; ms: host, may be NULL, that launch's duration.
 * Errors: SPH_EINVAL (NULL tflops, reps < 1), SPH_ENOMEM, SPH_ECUDA. */
sph_status sph_fma_peak(void* stream, int reps, double* tflops, double* ms);

/* Kernel-variant knobs of the pair passes (performance only).  List batch
 * and block size leave every result bitwise unchanged; two threads per
 * particle add each particle's pair terms in two interleaved halves, which
 * changes FP32 rounding only. */
enum {
    SPH_TUNE_LIST_BATCH = 0, /* neighbour-list entries each thread loads together: 1, 2 (default), 4 or 8 */
    SPH_TUNE_TPP = 1,        /* threads per particle in passes VT, M, C: 1 (default; 32 particles
                                per warp) or 2 (16 particles per warp) */
    SPH_TUNE_BLOCK = 2       /* threads per block of the pair passes: 64, 128 (default) or 256 */
};

/* Select a kernel variant; re-captures the step graph if the context has
 * started.  Errors: SPH_EINVAL (unknown key or value), SPH_ECUDA. */
sph_status sph_set_tuning(sph_ctx* ctx, int key, int value);
/* The variant in force for `key` into *value (host).  Errors: SPH_EINVAL. */
sph_status sph_get_tuning(sph_ctx* ctx, int key, int* value);

/* Autotuner result: the variant now in force and the model time it won on,
 * ms per advection step = (D + VT) per step + substeps_ref x (M + C) per
 * sub-step, measured with device events. */
typedef struct {
    int list_batch, tpp, block; /* chosen variant (set on return) */
    double ms_step_start;       /* model time of the variant in force before tuning */
    double ms_step_chosen;      /* model time of the chosen variant */
    double substeps_ref;        /* sub-steps per advection step of the first trial */
    int trials;                 /* variants timed */
    int64_t steps;              /* advection steps advanced while tuning */
} sph_tune_report;

/* Time the pair-pass variants on this context's own workload and keep the
 * fastest (coordinate descent: list batch, then threads per particle, then
 * block size; 1 + steps_per_trial real advection steps per variant, the
 * simulation advances by report->steps).  report: host, may be NULL.
 * Errors: SPH_EINVAL (steps_per_trial < 1), SPH_ESTATE (no particles, or
 * the case has finished), SPH_EUNSTABLE, SPH_ECUDA. */
sph_status sph_autotune(sph_ctx* ctx, int steps_per_trial, sph_tune_report* report);

/* Device-time profile of the advection step, by kernel group. */
enum {
    SPH_PROF_SORT = 0,     /* step set-up + cell hash, count, scan, scatter, id order, reorder */
    SPH_PROF_PASS_D = 1,   /* density re-initialisation */
    SPH_PROF_PASS_VT = 2,  /* viscous acceleration + heat conduction */
    SPH_PROF_PASS_M = 3,   /* Riemann pressure force + kick/drift (one per active sub-step) */
    SPH_PROF_PASS_C = 4,   /* Riemann continuity (one per active sub-step) */
    SPH_PROF_CONTROL = 5,  /* sub-step size + torque reduction */
    SPH_PROF_ADV_END = 6,  /* temperature update + heat reductions */
    SPH_PROF_IDLE = 7,     /* kernels of sub-step slots past the end of the advection step */
    SPH_PROF_NCLASS = 8
};

/* enable != 0: re-capture the step graph with CUDA event records between
 * kernel groups; sph_step then synchronises after every advection step and
 * adds each group's device time (cudaEventElapsedTime) to a per-group total.
 * enable == 0: plain graph again.  Counters are reset either way. */
sph_status sph_profile(sph_ctx* ctx, int enable);

/* ms: host double[SPH_PROF_NCLASS] accumulated device milliseconds;
 * launches: host int64[SPH_PROF_NCLASS] intervals counted.  reset != 0
 * clears the counters after reading. */
sph_status sph_profile_read(sph_ctx* ctx, double* ms, int64_t* launches, int reset);

/* Physics-driven particle relaxation (Sec. 2.2): pre-processing that moves
 * particles seeded on a lattice inside a body towards an isotropic,
 * body-fitted distribution under a constant background pressure p0
 * (scale-free, p0 / rho0 = 1), confined by the body's level set.  Per
 * iteration: F_p,i = -2 sum_j V_j W'(r) e_ij over partners within 2h, plus
 * -2 n A(d) for the kernel volume missing beyond the surface (n = unit
 * gradient of phi, d = -phi the depth, A(d) = 2 pi int_d^{2h} W(r) r dr);
 * dt = 0.25 sqrt(h / max |F_p|); r += F_p dt^2 / 2; a particle that ends
 * outside (phi > 0) is moved back along n by phi.  FP64 throughout. */
typedef struct {
    double dx, h_over_dx;    /* particle spacing (V = dx^3) and h = h_over_dx dx */
    const double* phi;       /* host: level set, negative inside, nphi[0] x nphi[1] x nphi[2]
                                nodes, x fastest; node (i, j, k) at phi_origin + (i, j, k) phi_spacing;
                                trilinear in between.  The particles stay inside this box. */
    int nphi[3];             /* >= 2 each */
    double phi_origin[3], phi_spacing;
} sph_relax_config;

/* Relax the n particles pos (host double[n*3], in place) for `iterations`
 * steps on `stream` (a cudaStream_t or NULL); device memory is allocated and
 * freed on that stream.  max_accel: host double[iterations] receiving
 * max |F_p| of each step, or NULL.  Errors: SPH_EINVAL (NULL arguments,
 * non-positive sizes, a level-set grid under 2 nodes on an axis), SPH_ENOMEM,
 * SPH_ECUDA; the message is in sph_last_error(NULL). */
sph_status sph_relax(const sph_relax_config* cfg, int64_t n, double* pos, int iterations, void* stream,
                     double* max_accel);

/* Message of the last failed call on ctx ("" if none).  With ctx == NULL:
 * the last failed context-free call (sph_cell_sort*) of this host thread.
 * Never NULL. */
const char* sph_last_error(const sph_ctx* ctx);

/* Stateless cell sort (the neighbour-search core of Sec. 2.8's per-advection
 * step update).  pos: device double[n*3].  Particle k goes to the cell
 * floor((pos - origin)/cellw) (clamped to the grid); particles are ordered by
 * (linear cell index with x fastest, k).  perm: device int32[n] receives the
 * particle index at each sorted position; cell_start: device int32[ncells+1]
 * receives each cell's first sorted position (last entry n).  Scratch of
 * about 12 n + 4 ncells bytes is allocated and freed on `stream` with
 * cudaMallocAsync.  Errors: SPH_EINVAL, SPH_ENOMEM, SPH_ECUDA. */
sph_status sph_cell_sort(const double* pos, int64_t n, const double origin[3], const double cellw[3],
                         const int ncell[3], int32_t* perm, int32_t* cell_start, void* stream);

/* ------------------------------------------------------------------------
 * Batched cases (sweeps and serving).  A batch is one packed particle array
 * on the device holding many independent cases (each built like a single
 * case: sph_create + sph_set_material + sph_add_* + sph_set_rotation, never
 * stepped).  One sph_batch_step advances every resident case by one
 * advection step in a single CUDA graph launch; each case keeps its own step
 * sizes, sub-step count, time, torque and heat, and its results do not depend
 * on which other cases are resident (no cross-case sums; fixed-order
 * per-case reductions).  Cases are admitted and retired between steps.
 * ------------------------------------------------------------------------ */
typedef struct sph_batch sph_batch;

typedef struct {
    int64_t max_particles; /* capacity of the packed array (all resident cases) */
    int max_cases;         /* case slots */
    int64_t max_cells;     /* capacity of the cell index space (sum of the cases' grids) */
    int history_steps;     /* per-case ring of advection-step records (sph_batch_read_curve) */
} sph_batch_config;

enum { SPH_BATCH_RUNNING = 0, SPH_BATCH_DONE = 1, SPH_BATCH_UNSTABLE = -4 };

/* Device bytes a batch of this configuration allocates (its HBM budget). */
int64_t sph_batch_bytes(const sph_batch_config* cfg);

/* Allocate a batch (all device memory up front).  Errors: SPH_EINVAL,
 * SPH_ENOMEM (message in sph_last_error(NULL)), SPH_ECUDA. */
sph_status sph_batch_create(const sph_batch_config* cfg, void* cuda_stream, sph_batch** out);
/* Free the batch and all its device memory; NULL is allowed. */
sph_status sph_batch_destroy(sph_batch* b);
/* Text of the batch's last error (empty if none), or with b = NULL of the last
 * failed call that had no batch (sph_batch_create); the pointer lives until
 * the next call on the batch. */
const char* sph_batch_last_error(const sph_batch* b);

/* Copy a staged case (never stepped; one fluid material) into the batch; it
 * runs n_steps advection steps (0 = until retired).  *slot receives its
 * slot id.  The staged context may be destroyed afterwards.  The case joins
 * at the next sph_batch_step.  Errors: SPH_ENOMEM (no free slot, particle,
 * cell or id capacity: the caller queues the request), SPH_EINVAL, SPH_ESTATE. */
sph_status sph_batch_admit(sph_batch* b, sph_ctx* staged, int64_t n_steps, int* slot);

/* Advance every running case n advection steps (finished cases stay
 * resident, unchanged, until retired).  A case that turns unstable (NaN/Inf
 * state or a fluid particle out of its box) is frozen after the advection
 * step that found it and polls as SPH_BATCH_UNSTABLE; the other cases go on
 * as if it were not there.  Errors: SPH_ECUDA. */
sph_status sph_batch_step(sph_batch* b, int n_advection_steps);

/* Steps done, simulated time and state (SPH_BATCH_*) of a resident case. */
sph_status sph_batch_poll(sph_batch* b, int slot, int64_t* steps_done, double* sim_time, int* state);

/* As sph_read_torque_heat, for a resident case. */
sph_status sph_batch_read_torque_heat(sph_batch* b, int slot, int body_id, double* torque_axis,
                                      double* torque_time_avg, double* heat_into_fluid, double* mean_fluid_T);

/* The last n (<= max_steps, <= history_steps) advection-step records of a
 * case, oldest first, 8 doubles each: time, torque of body 0, its running
 * time average, heat into fluid, mean fluid temperature, dt_ad, sub-steps,
 * max speed.  out: host double[8 * max_steps]. */
sph_status sph_batch_read_curve(sph_batch* b, int slot, double* out, int64_t max_steps, int64_t* n_out);

/* As sph_read_fields, for a resident case (n = its particle count). */
sph_status sph_batch_read_fields(sph_batch* b, int slot, int field, void* host_dst, int64_t n);

/* Remove a case; its particles, cells and ids are freed at the next step. */
sph_status sph_batch_retire(sph_batch* b, int slot);

/* Resident particles and cases, and kernels launched per advection step. */
sph_status sph_batch_info(sph_batch* b, int64_t* n_particles, int* n_cases, int* kernels_per_step);

/* sph_set_tuning for every case of the batch.  Errors: SPH_EINVAL, SPH_ECUDA. */
sph_status sph_batch_set_tuning(sph_batch* b, int key, int value);

/* sph_autotune for the resident cases of a batch (one variant for all). */
sph_status sph_batch_autotune(sph_batch* b, int steps_per_trial, sph_tune_report* report);
/* sph_profile and sph_profile_read for the batch's step graph. */
sph_status sph_batch_profile(sph_batch* b, int enable);
sph_status sph_batch_profile_read(sph_batch* b, double* ms, int64_t* launches, int reset);

/* Allocation-free variant of sph_cell_sort, for callers that cannot let a
 * library allocate device memory: a process whose free HBM is already held by
 * its own caching allocator, a latency-critical loop that cannot take the
 * device synchronisation of cudaMalloc/cudaFree, or a host whose memory
 * manager forbids outside allocations.  (The paper has no counterpart; this
 * is a deployment variant of the neighbour-search sort.)
 *
 * Same arguments, layout and result as sph_cell_sort.  Scratch lives in one
 * fixed device array of about 12 SPH_NOALLOC_MAX_N + 4 SPH_NOALLOC_MAX_CELLS
 * bytes (16 MiB).  It occupies a device from the first call there (from the
 * library's load instead when CUDA_MODULE_LOADING=EAGER) until the process
 * exits.  The call allocates nothing: no cudaMalloc, cudaFree or allocating
 * library routine.
 *  - n > SPH_NOALLOC_MAX_N or more than SPH_NOALLOC_MAX_CELLS cells:
 *    SPH_EINVAL, with the reason in sph_last_error(NULL).
 *  - The first call on a device looks up the scratch array's device address
 *    (cudaGetSymbolAddress, with that device current); make that first call
 *    outside any stream capture.  A failed lookup returns SPH_ECUDA.  The
 *    address is kept for the process: resetting the device (cudaDeviceReset
 *    or a primary-context reset) after the first call is not supported.
 *  - All calls share the one array (it keeps the last call's contents; the
 *    per-cell counters are cleared by each call).  Calls whose work overlaps
 *    on the GPU (different streams, or different host threads) race on it:
 *    serialise them on one stream.
 * Errors: SPH_EINVAL, SPH_ECUDA. */
#define SPH_NOALLOC_MAX_N (1 << 20)
#define SPH_NOALLOC_MAX_CELLS (1 << 20)
sph_status sph_cell_sort_noalloc(const double* pos, int64_t n, const double origin[3], const double cellw[3],
                                 const int ncell[3], int32_t* perm, int32_t* cell_start, void* stream);

#ifdef __cplusplus
}
#endif
#endif
