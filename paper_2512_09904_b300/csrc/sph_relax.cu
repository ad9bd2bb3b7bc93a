// sph_relax.cu -- physics-driven particle relaxation (Sec. 2.2), a
// pre-processing step that moves particles seeded on a lattice inside a body
// towards an isotropic, body-fitted distribution.
//
// Per iteration: cell sort of the positions (cells of width >= 2h), the
// background-pressure acceleration F_p,i = -2 sum_j V_j W'(r) e_ij (p0 / rho0
// = 1) plus the level-set confinement (the kernel volume missing beyond the
// surface, replaced by the half space at the particle's depth d = -phi:
// -2 n A(d), A(d) = 2 pi int_d^{2h} W(r) r dr in closed form), the step
// dt = 0.25 sqrt(h / max |F_p|), r += F_p dt^2 / 2, and particles that end
// outside moved back onto the surface along the level-set normal.  FP64
// arithmetic; B300's FP64 pipe is the bound, so candidates are rejected
// first from an FP32 copy of the positions with an error margin (the FP64
// membership rule still decides every pair that passes), and the kernel and
// level-set formulas multiply by precomputed reciprocals instead of dividing.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "sph.h"
#include "sph_kernels.cuh"

namespace sph {
void set_stateless_error(const char* msg);
}

namespace {

using namespace sph;

struct RelaxDev {
    double h, R2, vol;
    double inv_h;
    double kw, kdw;      // Wendland C2 alpha, -5 alpha / h
    double kdwh;         // kdw / h: (dW/dr) / r = kdwh (1 - r / 2h)^3
    float R2f;           // FP32 pre-test: no pair has r2 (from the FP32 copy) at or above this
    double aw;           // 2 pi alpha h^2: A(d) = aw (2/7 - F(d / h))
    const double* phi;
    int nphi[3];
    double phi_o[3], phi_inv, phi_dx;
    double inv_dx1, inv_dx2;  // 1 / phi_dx, 1 / (2 phi_dx): one- and two-sided differences
    double cell_o[3], cell_w[3];
    int ncell[3];
};

// (dW/dr) / r = (kdw / h) (1 - q/2)^3 with q = r / h
__device__ __forceinline__ double rx_dW_over_r(const RelaxDev& R, double r) {
    const double t = 1.0 - 0.5 * (r * R.inv_h);
    return R.kdwh * t * t * t;
}

// A(d) = 2 pi alpha h^2 (2/7 - F(q)), q = d / h, with F the antiderivative of
// (1 - q/2)^4 (1 + 2q) q: q^7/56 - 5 q^6/32 + q^5/2 - 5 q^4/8 + q^2/2
__device__ __forceinline__ double rx_A(const RelaxDev& R, double d) {
    double q = d * R.inv_h;
    if (q < 0.0) q = 0.0;
    if (q >= 2.0) return 0.0;
    const double q2 = q * q, q4 = q2 * q2;
    const double F = q4 * q2 * q / 56.0 - 5.0 * q4 * q2 / 32.0 + q4 * q / 2.0 - 5.0 * q4 / 8.0 + q2 / 2.0;
    return R.aw * (2.0 / 7.0 - F);
}

__device__ __forceinline__ double rx_node(const RelaxDev& R, int i, int j, int k) {
    i = min(max(i, 0), R.nphi[0] - 1);
    j = min(max(j, 0), R.nphi[1] - 1);
    k = min(max(k, 0), R.nphi[2] - 1);
    return R.phi[((long long)k * R.nphi[1] + j) * R.nphi[0] + i];
}

// central difference of phi along axis a at a node (one-sided at the grid's faces)
__device__ double rx_grad_node(const RelaxDev& R, int i, int j, int k, int a) {
    int id[3] = {i, j, k};
    int lo = id[a] - 1, hi = id[a] + 1;
    double span = 2.0;
    if (lo < 0) {
        lo = id[a];
        span -= 1.0;
    }
    if (hi > R.nphi[a] - 1) {
        hi = id[a];
        span -= 1.0;
    }
    int l[3] = {i, j, k}, u[3] = {i, j, k};
    l[a] = lo;
    u[a] = hi;
    return (rx_node(R, u[0], u[1], u[2]) - rx_node(R, l[0], l[1], l[2])) * (span > 1.5 ? R.inv_dx2 : R.inv_dx1);
}

// trilinear level set, and the normalised trilinear interpolation of the
// nodes' central-difference gradients (continuous across cells)
__device__ double rx_phi(const RelaxDev& R, const double x[3], double n[3]) {
    double f[3];
    int b[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double u = (x[a] - R.phi_o[a]) * R.phi_inv;
        double fl = floor(u);
        fl = fmin(fmax(fl, 0.0), (double)(R.nphi[a] - 2));
        b[a] = (int)fl;
        f[a] = u - fl;
    }
    double phi = 0.0, g[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < 2; ++k)
        for (int j = 0; j < 2; ++j)
            for (int i = 0; i < 2; ++i) {
                const double w = (i ? f[0] : 1.0 - f[0]) * (j ? f[1] : 1.0 - f[1]) * (k ? f[2] : 1.0 - f[2]);
                phi += w * rx_node(R, b[0] + i, b[1] + j, b[2] + k);
#pragma unroll
                for (int a = 0; a < 3; ++a) g[a] += w * rx_grad_node(R, b[0] + i, b[1] + j, b[2] + k, a);
            }
    const double gn = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
#pragma unroll
    for (int a = 0; a < 3; ++a) n[a] = gn > 0.0 ? g[a] / gn : 0.0;
    return phi;
}

// FP32 copy of a position, relative to the cell grid's corner
__device__ __forceinline__ float4 rx_f32(const RelaxDev& R, const double x[3]) {
    return make_float4((float)(x[0] - R.cell_o[0]), (float)(x[1] - R.cell_o[1]), (float)(x[2] - R.cell_o[2]), 0.f);
}

__global__ void k_rx_f32(RelaxDev R, int n, const double* __restrict__ pos, float4* pf) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double x[3] = {pos[3 * i], pos[3 * i + 1], pos[3 * i + 2]};
    pf[i] = rx_f32(R, x);
}

__global__ void k_rx_force(RelaxDev R, int n, const double* __restrict__ pos, const float4* __restrict__ pf,
                           const int* __restrict__ perm, const int* __restrict__ cs, double* acc,
                           unsigned long long* amax) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double xi[3] = {pos[3 * i], pos[3 * i + 1], pos[3 * i + 2]};
    const float4 fi = pf[i];
    int c[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double f = floor((xi[a] - R.cell_o[a]) / R.cell_w[a]);
        c[a] = (int)fmin(fmax(f, 0.0), (double)(R.ncell[a] - 1));
    }
    double ac[3] = {0.0, 0.0, 0.0};
    for (int z = max(c[2] - 1, 0); z <= min(c[2] + 1, R.ncell[2] - 1); ++z)
        for (int y = max(c[1] - 1, 0); y <= min(c[1] + 1, R.ncell[1] - 1); ++y)
            for (int x = max(c[0] - 1, 0); x <= min(c[0] + 1, R.ncell[0] - 1); ++x) {
                const int cell = (z * R.ncell[1] + y) * R.ncell[0] + x;
                for (int q = cs[cell]; q < cs[cell + 1]; ++q) {
                    const int j = perm[q];
                    if (j == i) continue;
                    const float4 fj = pf[j];
                    const float e0 = fi.x - fj.x, e1 = fi.y - fj.y, e2 = fi.z - fj.z;
                    if (fmaf(e2, e2, fmaf(e1, e1, e0 * e0)) >= R.R2f) continue;  // beyond 2h even with the FP32 error
                    const double d0 = __dsub_rn(xi[0], pos[3 * j]), d1 = __dsub_rn(xi[1], pos[3 * j + 1]),
                                 d2 = __dsub_rn(xi[2], pos[3 * j + 2]);
                    const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(d0, d0), __dmul_rn(d1, d1)), __dmul_rn(d2, d2));
                    if (!(r2 > 0.0 && r2 < R.R2)) continue;
                    const double k = -2.0 * R.vol * rx_dW_over_r(R, sqrt(r2));
                    ac[0] += k * d0;
                    ac[1] += k * d1;
                    ac[2] += k * d2;
                }
            }
    double nrm[3];
    const double phi = rx_phi(R, xi, nrm);
    const double A = rx_A(R, -phi);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        ac[a] += -2.0 * nrm[a] * A;
        acc[3 * i + a] = ac[a];
    }
    const double am = sqrt(ac[0] * ac[0] + ac[1] * ac[1] + ac[2] * ac[2]);
    atomicMax(amax, (unsigned long long)__double_as_longlong(am));  // non-negative: bit order = value order
}

__global__ void k_rx_move(RelaxDev R, int n, double* pos, float4* pf, const double* __restrict__ acc,
                          const unsigned long long* amax) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double am = __longlong_as_double((long long)*amax);
    if (!(am > 0.0)) return;
    const double dt = 0.25 * sqrt(R.h / am);
    double x[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) x[a] = pos[3 * i + a] + 0.5 * acc[3 * i + a] * dt * dt;
    double nrm[3];
    const double phi = rx_phi(R, x, nrm);
    if (phi > 0.0) {
#pragma unroll
        for (int a = 0; a < 3; ++a) x[a] -= phi * nrm[a];
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) pos[3 * i + a] = x[a];
    pf[i] = rx_f32(R, x);
}

}  // namespace

extern "C" sph_status sph_relax(const sph_relax_config* cfg, int64_t n, double* pos, int iterations, void* stream,
                                double* max_accel) {
    if (!cfg || n < 0 || (n > 0 && !pos) || iterations < 0 || !cfg->phi || !(cfg->dx > 0) ||
        !(cfg->h_over_dx > 0) || !(cfg->phi_spacing > 0) || cfg->nphi[0] < 2 || cfg->nphi[1] < 2 || cfg->nphi[2] < 2 ||
        n > ((int64_t)1 << 30)) {
        sph::set_stateless_error("sph_relax: invalid argument");
        return SPH_EINVAL;
    }
    if (n == 0 || iterations == 0) return SPH_OK;
    cudaStream_t s = (cudaStream_t)stream;
    RelaxDev R{};
    R.h = cfg->h_over_dx * cfg->dx;
    R.R2 = 4.0 * R.h * R.h;
    R.vol = cfg->dx * cfg->dx * cfg->dx;
    const double alpha = 21.0 / (16.0 * M_PI * R.h * R.h * R.h);
    R.kw = alpha;
    R.kdw = -5.0 * alpha / R.h;
    R.aw = 2.0 * M_PI * alpha * R.h * R.h;
    R.inv_h = 1.0 / R.h;
    R.kdwh = R.kdw / R.h;
    R.inv_dx1 = 1.0 / cfg->phi_spacing;
    R.inv_dx2 = 1.0 / (2.0 * cfg->phi_spacing);
    R.phi_inv = 1.0 / cfg->phi_spacing;
    R.phi_dx = cfg->phi_spacing;
    int64_t nphi = 1, ncells = 1;
    for (int a = 0; a < 3; ++a) {
        R.nphi[a] = cfg->nphi[a];
        R.phi_o[a] = cfg->phi_origin[a];
        nphi *= cfg->nphi[a];
        // the cell grid covers the level-set box; cells of width >= 2h
        const double ext = (cfg->nphi[a] - 1) * cfg->phi_spacing;
        int64_t m = (int64_t)std::floor(ext / (2.0 * R.h));
        if (m < 1) m = 1;
        R.ncell[a] = (int)m;
        R.cell_w[a] = ext / (double)m;
        R.cell_o[a] = cfg->phi_origin[a];
        ncells *= m;
    }
    if (ncells > ((int64_t)1 << 28)) {
        sph::set_stateless_error("sph_relax: level-set box too large for the cell grid");
        return SPH_EINVAL;
    }
    // FP32 pre-test margin.  An FP32 coordinate relative to the grid corner
    // is off by at most E 2^-24 (E bounds |x - corner|: the box, or a seed
    // outside it, doubled for the moves), an FP32 difference of two by
    // delta = 2 E 2^-24 plus its own rounding (differences within the 27
    // cells are below 8h), so a pair (r < 2h) has r_f32 < 2h + 2 delta; the
    // factor 1 + 1e-6 covers the FP32 rounding of r^2 and of the bound.
    double E = 0.0;
    for (int a = 0; a < 3; ++a) E = std::max(E, (R.nphi[a] - 1) * cfg->phi_spacing);
    for (int64_t i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) E = std::max(E, std::fabs(pos[3 * i + a] - R.cell_o[a]));
    E *= 2.0;
    const double delta = 2.0 * E * 0x1p-24 + 8.0 * R.h * 0x1p-24, rmax = 2.0 * R.h + 2.0 * delta;
    R.R2f = (float)(rmax * rmax * (1.0 + 1e-6));
    double *d_pos = nullptr, *d_acc = nullptr, *d_phi = nullptr;
    float4* d_pf = nullptr;
    unsigned long long* d_amax = nullptr;
    uint32_t *keys = nullptr, *rank = nullptr, *cnt = nullptr, *tmp = nullptr, *blk = nullptr;
    int32_t *perm = nullptr, *cs = nullptr;
    const size_t nb = scan_blocks((int)ncells) + 1;
    cudaError_t e = cudaSuccess;
#define RA(p, bytes) \
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&(p), (bytes), s)
    RA(d_pos, sizeof(double) * 3 * n);
    RA(d_acc, sizeof(double) * 3 * n);
    RA(d_pf, sizeof(float4) * n);
    RA(d_phi, sizeof(double) * nphi);
    RA(d_amax, sizeof(unsigned long long) * (size_t)iterations);
    RA(keys, sizeof(uint32_t) * n);
    RA(rank, sizeof(uint32_t) * n);
    RA(tmp, sizeof(uint32_t) * n);
    RA(perm, sizeof(int32_t) * n);
    RA(cnt, sizeof(uint32_t) * (ncells + 1));
    RA(cs, sizeof(int32_t) * (ncells + 1));
    RA(blk, sizeof(uint32_t) * nb);
#undef RA
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_pos, pos, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_phi, cfg->phi, sizeof(double) * nphi, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_amax, 0, sizeof(unsigned long long) * (size_t)iterations, s);
    R.phi = d_phi;
    const int g = (int)((n + 127) / 128);
    if (e == cudaSuccess) {
        k_rx_f32<<<g, 128, 0, s>>>(R, (int)n, d_pos, d_pf);
        e = cudaGetLastError();
    }
    for (int it = 0; it < iterations && e == cudaSuccess; ++it) {
        e = launch_cell_sort(d_pos, (int)n, R.cell_o, R.cell_w, R.ncell, keys, rank, cnt, tmp, blk, perm, cs, s);
        if (e == cudaSuccess) {
            k_rx_force<<<g, 128, 0, s>>>(R, (int)n, d_pos, d_pf, perm, cs, d_acc, d_amax + it);
            k_rx_move<<<g, 128, 0, s>>>(R, (int)n, d_pos, d_pf, d_acc, d_amax + it);
            e = cudaGetLastError();
        }
    }
    std::vector<unsigned long long> am(iterations, 0ull);
    if (e == cudaSuccess) e = cudaMemcpyAsync(pos, d_pos, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(am.data(), d_amax, sizeof(unsigned long long) * (size_t)iterations,
                            cudaMemcpyDeviceToHost, s);
    for (void* p : {(void*)d_pos, (void*)d_acc, (void*)d_pf, (void*)d_phi, (void*)d_amax, (void*)keys, (void*)rank, (void*)tmp,
                    (void*)perm, (void*)cnt, (void*)cs, (void*)blk})
        if (p) cudaFreeAsync(p, s);
    const cudaError_t e2 = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) {
        char msg[160];
        snprintf(msg, sizeof msg, "sph_relax: %s", cudaGetErrorString(e));
        sph::set_stateless_error(msg);
        return e == cudaErrorMemoryAllocation ? SPH_ENOMEM : SPH_ECUDA;
    }
    if (max_accel)
        for (int it = 0; it < iterations; ++it) {
            long long b = (long long)am[it];
            double v;
            memcpy(&v, &b, sizeof v);
            max_accel[it] = v;
        }
    return SPH_OK;
}
