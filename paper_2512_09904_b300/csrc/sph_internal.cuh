// sph_internal.cuh -- device-side data layout and helpers of the SPH library.
//
// Layout in HBM (one engine = one packed particle array over all resident
// cases; a case's particles are contiguous after every cell sort):
//   X[3]   double, work positions (fluid drift target), slot order
//   Y[3]   double, frozen snapshot positions of the advection step, slot order
//   V[2]   float4 (vx, vy, vz, drho_rel = rho - rho0), ping-pong across passes;
//          for solids (wall velocity, 0)
//   DR[2]  float, continuity rate carried between sub-steps
//   T64[2] double temperature; T32 float (T - T_ref) for pair arithmetic
//   SNAP   float4 (offset of the snapshot position from its cell corner, tag)
//   CELLK  uint32 global cell index of each slot
//   AV     float4 (viscous acceleration held for the sub-steps, dT/dt)
//   NRM    float4 wall normal (solids)
//   per-id arrays (indexed by particle id, never reordered): reference
//   positions/normals of solids, per-solid torque contributions.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace sph {

constexpr int MAX_MAT = 16;
// Sort cells per geometry cell: 8 along x, 2 along y and z.  The search walks
// x-contiguous rows of sort cells, so narrow cells along x clip each row to
// the 2h sphere more tightly (fewer candidates) at no extra cost per row.
constexpr int SPLIT_X_SHIFT = 3, SPLIT_X = 1 << SPLIT_X_SHIFT, SPLIT_YZ = 2;
__host__ __device__ __forceinline__ int split_of(int axis) { return axis == 0 ? SPLIT_X : SPLIT_YZ; }
constexpr int MAX_BODY = 4;
constexpr int GCORNER_MAX = 512;  // geometry cells per axis with a tabulated corner
constexpr uint32_t KIND_FLUID = 0u, KIND_STATIC = 1u, KIND_ROT = 2u;
constexpr int ERR_NAN = 1, ERR_ESCAPE = 2, ERR_NB_OVERFLOW = 4;

// Per-particle neighbour lists, rebuilt once per advection step (the pair
// set is frozen for the step).  Entry = j | code << 26 (code: cell offset,
// see for_each_neighbor).  Fluid partners fill slots 0, 1, ... and wall
// partners slots NB_CAP-1, NB_CAP-2, ...; slot k of particle i lives at
// NB[k * stride + i] so a warp's loads of one slot are coalesced.
// NBC[i] = nf | nw << 8 | NB_HAS; NB_OVF marks a particle whose partners did
// not fit (its passes fall back to the 27-cell loop).
constexpr int NB_CAP = 128;
constexpr uint32_t NB_HAS = 1u << 30, NB_OVF = 1u << 31;
constexpr uint32_t NB_JMASK = (1u << 26) - 1u;
constexpr int MAX_PARTICLES = 1 << 26;

// particle tag: material (4 bits) | kind (2) | body (2) | case (24)
__host__ __device__ __forceinline__ uint32_t make_tag(uint32_t mat, uint32_t kind, uint32_t body,
                                                      uint32_t cs) {
    return mat | (kind << 4) | (body << 6) | (cs << 8);
}
__host__ __device__ __forceinline__ uint32_t tag_mat(uint32_t t) { return t & 15u; }
__host__ __device__ __forceinline__ uint32_t tag_kind(uint32_t t) { return (t >> 4) & 3u; }
__host__ __device__ __forceinline__ uint32_t tag_body(uint32_t t) { return (t >> 6) & 3u; }
__host__ __device__ __forceinline__ uint32_t tag_case(uint32_t t) { return t >> 8; }

struct MatDev {
    float rho0, mass, mu, k, cp, inv_rho0_cp;
    int fixed_T, pad;
};

// The same material in FP64 (pair arithmetic in FP64).
struct MatDev64 {
    double rho0, mass, mu, k, cp, inv_rho0_cp;
};

struct BodyDev {
    double c[3], axis[3], omega;
    int id_lo, id_hi;   // id range holding the body's particles
    int set, pad;
};

// Two grids per case: sort cells (cellw, ncell: width >= h/4 along x and >= h
// along y and z, the cell-linked list) and geometry cells of SPLIT_X x
// SPLIT_YZ x SPLIT_YZ sort cells (gcellw: width >= 2h),
// to whose corners the FP32 snapshot offsets refer; a partner's geometry
// cell is within one of the particle's on every axis.
struct CaseDev {
    double origin[3], ext[3], cellw[3], gcellw[3], inv_cellw[3];
    float gcellwf[3], scellwf[3], inv_scellwf[3];
    float originf[3];  // origin rounded to FP32 (the cell hash's estimate)
    float Rmargin;  // slack on the search sphere (FP32 rounding of the clipping)
    int ncell[3];
    int cell_base, ncells;
    int periodic;
    double R2;                    // (2h)^2 in FP64: the membership rule
    float R2lo, R2hi, R2eps;      // FP32 guard band around the rule
    float h, inv_h, w0, kw, kdw;  // W(0), alpha, -5 alpha / h
    float nhinv, kdwh;            // -1 / (2h) and kdw / h: (dW/dr) / r = kdwh (1 - r / 2h)^3
    float inv_sigma0, vol;
    float inv_contact_full;  // 1 / (dx^3 (sigma0 - W(0))): the fully immersed kernel volume sum
    float c0, c02, inv_c0, inv_c02;
    float g[3];
    double h64, c0_64, u_ref, cfl_ad, cfl_ac, nu_max;
    double dt_T;  // Eq. (26) thermal bound on dt_ad (infinite without conduction)
    double T_ref;
    // FP64 copies of the constants above (pair arithmetic in FP64)
    double kw64, kdw64, w0_64, inv_sigma0_64, vol64, c02_64, inv_c0_64, inv_c02_64, g64[3];
    double inv_contact_full64;
    int free_surface, kcap, n_body, fp64;
    int visc_heat;  // add the viscous-dissipation heating 2 mu S:S (extension; off in the paper)
    int vstar_lit;  // Eq. (13) with its printed sign (FP64 pairs only; off by default)
    int wall_printed;  // Eq. (19) without the limiter term (FP64 pairs only; off by default)
    MatDev fluid;   // the material of the case's fluid particles, when they all share one
    MatDev mat[MAX_MAT];
    MatDev64 mat64[MAX_MAT];
    BodyDev body[MAX_BODY];
    // origin + g w of geometry cell g on each axis (FP64), when every axis
    // has at most GCORNER_MAX geometry cells: the snapshot offset is then
    // one FP64 subtraction from the position
    int gcorner_ok;
    double gcorner[3][GCORNER_MAX];
};

// The constants the pair passes read per pair, for one case: a table of them
// over the resident cases fits a kernel's parameter block, where they are
// constant-bank operands instead of loads from the global case table.
// Materials and rigid bodies (read once per particle) stay in the case table.
// Field names follow CaseDev's, so the pair code takes either.
struct PairConst {
    float gcellwf[3], scellwf[3], inv_scellwf[3];
    float Rmargin, R2lo, R2hi, R2eps;
    float inv_h, w0, kw, kdw, inv_sigma0, vol, inv_contact_full;
    float nhinv, kdwh;
    float c0, c02, inv_c0, inv_c02;
    float g[3];
    int ncell[3];
    int cell_base, periodic, free_surface, visc_heat;
    MatDev fluid;         // the material of the case's fluid particles, when they all share one
    const MatDev* mat;    // the case's materials in the case table
    const BodyDev* body;  // the case's rigid bodies in the case table
};

// Pair-pass constants of up to PAIRTAB_MAX cases, indexed by case slot (one
// resident case: at index 0), passed by value to the pair passes.
constexpr int PAIRTAB_MAX = 64;
struct PairTab {
    PairConst c[PAIRTAB_MAX];
};

struct CaseState {
    double t, dt_ad, tau, dt;
    float dtf, hdtf;
    int active, last, nsub, reach;
    unsigned vmax_bits;
    int err;       // error bits that fail sph_step (NaN, particle escaped)
    int err_info;  // informational bits (neighbour list overflow)
    long long adv_steps, substeps;
    double cs[MAX_BODY], sn[MAX_BODY];
    double tq_p[MAX_BODY], tq_v[MAX_BODY], tq_inst[MAX_BODY], tq_int[MAX_BODY];
    double time_int;
    double sum_mcpT, sum_mT, sum_m, heat0;
    double heat, mean_T;
    int seg_lo, seg_hi;
    int chunk_lo, nchunks;
    int last_nsub, pad;
    double last_dt_ad;
    int alive;         // resident in the engine (dead: sorted out at the next step)
    int running;       // advancing (cleared when the requested steps are done)
    int init_pending;  // reference heat content still to be taken
    int pad2;
    long long steps_req;  // advection steps requested (0 = unlimited)
    unsigned long long vmax64_bits;  // FP64 pair arithmetic: bits of the (non-negative) max speed
};

// ---------------------------------------------------------------- kernel ---
// Wendland C2 (3-D, support 2h): W = alpha (1 - q/2)^4 (1 + 2q),
// dW/dr = -(5 alpha / h) q (1 - q/2)^3, q = r/h.
template <class CC>
__device__ __forceinline__ float kernel_W(const CC& C, float r) {
    float q = r * C.inv_h;
    float t = fmaf(-0.5f, q, 1.0f);
    float t2 = t * t;
    return C.kw * t2 * t2 * fmaf(2.0f, q, 1.0f);
}
template <class CC>
__device__ __forceinline__ float kernel_dW(const CC& C, float r) {
    float q = r * C.inv_h;
    float t = fmaf(-0.5f, q, 1.0f);
    return C.kdw * q * t * t * t;
}

// (dW/dr) / r as a function of r: (5 alpha / h) q (1 - q/2)^3 / r with
// q / r = 1 / h, so kdwh (1 - r / 2h)^3, kdwh = kdw / h.  The pair passes
// need dW/dr only times the unit vector r_ij / r, i.e. this times r_ij.
template <class CC>
__device__ __forceinline__ float kernel_dW_over_r(const CC& C, float r) {
    const float t = fmaf(C.nhinv, r, 1.0f);
    return C.kdwh * (t * t) * t;
}

__device__ __forceinline__ float dot3f(float ax, float ay, float az, float bx, float by, float bz) {
    return fmaf(az, bz, fmaf(ay, by, ax * bx));
}

// Exact pair-membership rule on the FP64 snapshot: 0 < r^2 < R2 with
// r^2 = ((dx*dx + dy*dy) + dz*dz) in round-to-nearest, no contraction, and
// the minimum image on periodic axes.  Cg is the case in the global case
// table (the periodic box and R2 are read from there only on this rare
// path).  Inlined: as an out-of-line call its register save made the
// search loop of pass D spill.
static __device__ __forceinline__ bool member_fp64(const CaseDev* __restrict__ Cg, const double* __restrict__ Yx,
                                                   const double* __restrict__ Yy, const double* __restrict__ Yz,
                                                   int i, int j) {
    const CaseDev& C = *Cg;
    double d[3] = {__dsub_rn(Yx[i], Yx[j]), __dsub_rn(Yy[i], Yy[j]), __dsub_rn(Yz[i], Yz[j])};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (C.periodic & (1 << a)) {
            double L = C.ext[a];
            if (d[a] > 0.5 * L) d[a] = __dsub_rn(d[a], L);
            else if (d[a] < -0.5 * L) d[a] = __dadd_rn(d[a], L);
        }
    }
    double r2 = __dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1]));
    r2 = __dadd_rn(r2, __dmul_rn(d[2], d[2]));
    return r2 > 0.0 && r2 < C.R2;
}

// Half-width of the x interval of the 2h sphere around a point at squared
// distance d2 (< R2) from a row's slab, plus Rmargin.  The square root is the
// hardware reciprocal estimate: its relative error (~1e-7) is far inside the
// margin, so the clipping stays conservative.
template <class CC>
__device__ __forceinline__ float row_half_width(const CC& C, float d2) {
    const float e2 = C.R2hi - d2;
    return fmaf(e2, rsqrtf(e2), C.Rmargin);
}

// Distance from a point at offset o inside its sort cell (width w) to the
// slab of the cell d sort cells away on that axis: d w - o ahead (d > 0),
// o - (d + 1) w behind (d < 0), 0 in its own cell, as one branch-free max.
__device__ __forceinline__ float slab_gap(int d, float w, float o) {
    return fmaxf(fmaxf(fmaf((float)d, w, -o), fmaf(-(float)(d + 1), w, o)), 0.f);
}

// Candidate runs of slot i (sort cell key_i, geometry offsets si): the rows
// of sort cells within two of i's on y and z whose slab the sphere of radius
// 2h around i reaches, and in each row the cells within two on x that the
// sphere reaches, cut where the geometry cell changes.  run(a, b, dcx, dcy,
// dcz) gets a slot range and its particles' geometry-cell offset from i's.
// The clipping is conservative (guard-band radius plus Rmargin): every
// partner of the FP64 rule is among the candidates.
template <class CC, class F>
__device__ __forceinline__ void for_each_run(const CC& C, const uint32_t* __restrict__ cstart, float4 si,
                                             uint32_t key_i, F&& run) {
    const int nx = C.ncell[0], ny = C.ncell[1], nz = C.ncell[2];
    const int cl = (int)key_i - C.cell_base;
    const int sx = cl % nx, sy = (cl / nx) % ny, sz = cl / (nx * ny);
    const float wx = C.scellwf[0], wy = C.scellwf[1], wz = C.scellwf[2];
    // position of i inside its sort cell
    const float ox = fmaf(-(float)(sx & (SPLIT_X - 1)), wx, si.x);
    const float oy = fmaf(-(float)(sy & 1), wy, si.y);
    const float oz = fmaf(-(float)(sz & 1), wz, si.z);
    const bool px = C.periodic & 1, py = C.periodic & 2, pz = C.periodic & 4;
    const float R2 = C.R2hi;
#pragma unroll 1
    for (int dz = -2; dz <= 2; ++dz) {
        int z = sz + dz;
        if (z < 0 || z >= nz) {
            if (!pz) continue;
            z = (z + nz) % nz;
        }
        const float gz = slab_gap(dz, wz, oz);
        if (gz * gz >= R2) continue;
        const int dcz = ((sz + dz) >> 1) - (sz >> 1);
#pragma unroll 1
        for (int dy = -2; dy <= 2; ++dy) {
            int y = sy + dy;
            if (y < 0 || y >= ny) {
                if (!py) continue;
                y = (y + ny) % ny;
            }
            const float gy = slab_gap(dy, wy, oy);
            const float d2 = fmaf(gy, gy, gz * gz);
            if (d2 >= R2) continue;
            const float ex = row_half_width(C, d2);
            int xl = sx + max(-SPLIT_X, (int)floorf((ox - ex) * C.inv_scellwf[0]));
            int xh = sx + min(SPLIT_X, (int)floorf((ox + ex) * C.inv_scellwf[0]));
            if (!px) {
                xl = max(xl, 0);
                xh = min(xh, nx - 1);
            }
            const int row = C.cell_base + (z * ny + y) * nx;
            const int dcy = ((sy + dy) >> 1) - (sy >> 1);
            // geometry cells along x: floor division by SPLIT_X (arithmetic shift, also below 0)
            for (int g = xl >> SPLIT_X_SHIFT; g <= (xh >> SPLIT_X_SHIFT); ++g) {
                const int a = max(xl, SPLIT_X * g), b = min(xh, SPLIT_X * g + SPLIT_X - 1);
                if (a > b) continue;
                // a..b lie in one geometry cell; nx is a multiple of SPLIT_X, so it
                // stays contiguous when wrapped
                const int aw = px ? ((a % nx) + nx) % nx : a;
                run((int)cstart[row + aw], (int)cstart[row + aw + (b - a) + 1], g - (sx >> SPLIT_X_SHIFT), dcy, dcz);
            }
        }
    }
}

// Every candidate j of slot i, in the order of for_each_run (rows by z, y;
// slots ascending), as f(j, ox, oy, oz, code): (ox, oy, oz) = i's offsets
// moved into j's geometry cell, so r_ij = o - (j's offsets), and code =
// (dcx+1) | (dcy+1) << 2 | (dcz+1) << 4 that cell's offset.  Without periodic
// axes a clipped row is one contiguous slot range, walked in a single loop
// that steps the geometry-cell offset at the first slot of each next cell:
// the threads of a warp then diverge per row, not per row and cell.
template <class CC, class F>
__device__ __forceinline__ void for_each_candidate(const CC& C, const uint32_t* __restrict__ cstart, float4 si,
                                                   uint32_t key_i, F&& f) {
    if (C.periodic) {
        for_each_run(C, cstart, si, key_i, [&](int a, int b, int dcx, int dcy, int dcz) {
            const float ox = fmaf(-(float)dcx, C.gcellwf[0], si.x);
            const float oy = fmaf(-(float)dcy, C.gcellwf[1], si.y);
            const float oz = fmaf(-(float)dcz, C.gcellwf[2], si.z);
            const uint32_t code = (uint32_t)((dcx + 1) | ((dcy + 1) << 2) | ((dcz + 1) << 4));
            for (int j = a; j < b; ++j) f(j, ox, oy, oz, code);
        });
        return;
    }
    const int nx = C.ncell[0], ny = C.ncell[1], nz = C.ncell[2];
    const int cl = (int)key_i - C.cell_base;
    const int sx = cl % nx, sy = (cl / nx) % ny, sz = cl / (nx * ny);
    const float wx = C.scellwf[0], wy = C.scellwf[1], wz = C.scellwf[2];
    const float cx = fmaf(-(float)(sx & (SPLIT_X - 1)), wx, si.x);
    const float cy = fmaf(-(float)(sy & 1), wy, si.y);
    const float cz = fmaf(-(float)(sz & 1), wz, si.z);
    const float R2 = C.R2hi, gw = C.gcellwf[0];
    // rows inside the grid, and the x range within SPLIT_X sort cells of i's
    const int dz0 = max(-2, -sz), dz1 = min(2, nz - 1 - sz), dy0 = max(-2, -sy), dy1 = min(2, ny - 1 - sy);
    const int xlo = max(0, sx - SPLIT_X), xhi = min(nx - 1, sx + SPLIT_X);
    const float cxi = cx * C.inv_scellwf[0];  // i's offset in sort-cell widths
#pragma unroll 1
    for (int dz = dz0; dz <= dz1; ++dz) {
        const int z = sz + dz;
        const float gz = slab_gap(dz, wz, cz);
        if (gz * gz >= R2) continue;
        const int dcz = ((sz + dz) >> 1) - (sz >> 1);
        const float oz = fmaf(-(float)dcz, C.gcellwf[2], si.z);
        const int rowz = C.cell_base + z * ny * nx;
#pragma unroll 1
        for (int dy = dy0; dy <= dy1; ++dy) {
            const int y = sy + dy;
            const float gy = slab_gap(dy, wy, cy);
            const float d2 = fmaf(gy, gy, gz * gz);
            if (d2 >= R2) continue;
            const float ex = row_half_width(C, d2);
            const int xl = max(xlo, sx + __float2int_rd(fmaf(-ex, C.inv_scellwf[0], cxi)));
            const int xh = min(xhi, sx + __float2int_rd(fmaf(ex, C.inv_scellwf[0], cxi)));
            if (xl > xh) continue;
            const int row = rowz + y * nx;
            const int dcy = ((sy + dy) >> 1) - (sy >> 1);
            const float oy = fmaf(-(float)dcy, C.gcellwf[1], si.y);
            const int dcx = (xl >> SPLIT_X_SHIFT) - (sx >> SPLIT_X_SHIFT);
            float ox = fmaf(-(float)dcx, gw, si.x);
            uint32_t code = (uint32_t)((dcx + 1) | ((dcy + 1) << 2) | ((dcz + 1) << 4));
            const int end = (int)cstart[row + xh + 1];
            int xb = (xl & ~(SPLIT_X - 1)) + SPLIT_X;  // first sort cell of the next geometry cell
            int jb = xb <= xh ? (int)cstart[row + xb] : end;
            for (int j = (int)cstart[row + xl]; j < end; ++j) {
                while (j == jb) {  // ends: jb = end > j once xb passes xh
                    ox -= gw;
                    ++code;
                    xb += SPLIT_X;
                    jb = xb <= xh ? (int)cstart[row + xb] : end;
                }
                f(j, ox, oy, oz, code);
            }
        }
    }
}

// Visit every neighbour j of slot i.  Pair geometry comes from the FP32
// geometry-cell offsets of the frozen snapshot: r_ij = off_i - off_j - dc w.
// Membership is decided in FP32 away from the cut-off and re-decided from
// the FP64 snapshot inside a relative guard band, so the pair set equals the
// FP64 rule exactly.  f(j, sj, rx, ry, rz, r2, code) receives r_ij = r_i - r_j
// and the geometry-cell offset packed as code = (dx+1) | (dy+1) << 2 | (dz+1) << 4.
// C may be a parameter-block copy of the case; Cg is the same case in the
// global table, for the rare FP64 re-check.
template <class CC, class F>
__device__ __forceinline__ void for_each_neighbor(const CC& C, const CaseDev* Cg,
                                                  const uint32_t* __restrict__ cstart,
                                                  const float4* __restrict__ snap,
                                                  const double* __restrict__ Yx,
                                                  const double* __restrict__ Yy,
                                                  const double* __restrict__ Yz, int i, float4 si,
                                                  uint32_t key_i, F&& f) {
    for_each_candidate(C, cstart, si, key_i, [&](int j, float ox, float oy, float oz, uint32_t code) {
        const float4 sj = __ldg(snap + j);
        const float rx = ox - sj.x, ry = oy - sj.y, rz = oz - sj.z;
        const float r2 = fmaf(rz, rz, fmaf(ry, ry, rx * rx));
        bool in;
        if (r2 >= C.R2hi) in = false;
        else if (r2 < C.R2lo && r2 > C.R2eps) in = true;
        else in = j != i && member_fp64(Cg, Yx, Yy, Yz, i, j);  // i itself: r2 = 0 lands here
        if (in) f(j, sj, rx, ry, rz, r2, (int)code);
    });
}

// Position of a solid particle at the current advection step: static walls
// sit at their reference position; rigid bodies are rotated by the step's
// angle about (c, axis) (Rodrigues' formula, FP64).
__device__ __forceinline__ void solid_position(const CaseDev& C, const CaseState& S, uint32_t tag,
                                               const double* __restrict__ RPx,
                                               const double* __restrict__ RPy,
                                               const double* __restrict__ RPz, int id, double p[3]) {
    p[0] = RPx[id];
    p[1] = RPy[id];
    p[2] = RPz[id];
    if (tag_kind(tag) == KIND_ROT) {
        const int b = tag_body(tag);
        const BodyDev& B = C.body[b];
        const double cs = S.cs[b], sn = S.sn[b];
        double d[3] = {p[0] - B.c[0], p[1] - B.c[1], p[2] - B.c[2]};
        double axd[3] = {B.axis[1] * d[2] - B.axis[2] * d[1], B.axis[2] * d[0] - B.axis[0] * d[2],
                         B.axis[0] * d[1] - B.axis[1] * d[0]};
        double ad = B.axis[0] * d[0] + B.axis[1] * d[1] + B.axis[2] * d[2];
#pragma unroll
        for (int k = 0; k < 3; ++k) p[k] = B.c[k] + (cs * d[k] + sn * axd[k] + (1.0 - cs) * ad * B.axis[k]);
    }
}

}  // namespace sph
