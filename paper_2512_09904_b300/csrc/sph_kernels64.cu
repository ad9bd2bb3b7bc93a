// sph_kernels64.cu -- the pair passes with FP64 arithmetic (sph_config.pair_precision = 1).
//
// Same method and same neighbour lists as the FP32 passes; the pair
// geometry is the FP64 snapshot difference r_i - r_j (minimum image on
// periodic axes) with r^2 = ((x^2 + y^2) + z^2) rounded as the membership
// rule, and every pair term, accumulation and particle state is FP64.  This
// is the plain FP64 variant of the method for small cases; the FP32 passes
// are the fast path.
#include "sph_kernels.cuh"

namespace sph {

namespace {

__device__ __forceinline__ double geom64(const CaseDev& C, const Bufs& B, int i, int j, double& rx, double& ry,
                                         double& rz) {
    double d[3] = {__dsub_rn(B.Y[0][i], B.Y[0][j]), __dsub_rn(B.Y[1][i], B.Y[1][j]),
                   __dsub_rn(B.Y[2][i], B.Y[2][j])};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (C.periodic & (1 << a)) {
            const double L = C.ext[a];
            if (d[a] > 0.5 * L) d[a] = __dsub_rn(d[a], L);
            else if (d[a] < -0.5 * L) d[a] = __dadd_rn(d[a], L);
        }
    }
    rx = d[0];
    ry = d[1];
    rz = d[2];
    return __dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])), __dmul_rn(d[2], d[2]));
}

// Wendland C2, support 2h: W = alpha (1 - q/2)^4 (1 + 2q), dW/dr = -(5 alpha/h) q (1 - q/2)^3
__device__ __forceinline__ double W64(const CaseDev& C, double r) {
    const double q = r / C.h64;
    const double t = 1.0 - 0.5 * q;
    return C.kw64 * t * t * t * t * (1.0 + 2.0 * q);
}
__device__ __forceinline__ double dW64(const CaseDev& C, double r) {
    const double q = r / C.h64;
    const double t = 1.0 - 0.5 * q;
    return C.kdw64 * q * t * t * t;
}

__device__ __forceinline__ double harm2(double a, double b) {
    const double s = a + b;
    return s > 0.0 ? 2.0 * a * b / s : 0.0;
}

__device__ __forceinline__ double dot3(double ax, double ay, double az, double bx, double by, double bz) {
    return ax * bx + ay * by + az * bz;
}

constexpr int P_FLUID = 1, P_WALL = 2, P_ALL = 3;

// Partners of slot i: f(j, tag_j, rx, ry, rz, r2).  From the particle's list
// when it has one, else from the 27-cell loop (same pair set).
template <int PART, class F>
__device__ __forceinline__ void visit64(const CaseDev& C, const Bufs& B, int i, F&& f) {
    const uint32_t cnt = B.NBC[i];
    auto emit = [&](int j) {
        const uint32_t tj = __float_as_uint(B.SNAP[j].w);
        const bool fj = tag_kind(tj) == KIND_FLUID;
        if (!((fj && (PART & P_FLUID)) || (!fj && (PART & P_WALL)))) return;
        double rx, ry, rz;
        const double r2 = geom64(C, B, i, j, rx, ry, rz);
        f(j, tj, rx, ry, rz, r2);
    };
    if ((cnt & NB_HAS) && !(cnt & NB_OVF)) {
        const size_t stride = (size_t)B.nb_stride;
        if (PART & P_FLUID)
            for (uint32_t q = 0; q < (cnt & 255u); ++q) emit((int)(B.NB[(size_t)q * stride + i] & NB_JMASK));
        if (PART & P_WALL)
            for (uint32_t q = 0; q < ((cnt >> 8) & 255u); ++q)
                emit((int)(B.NB[(size_t)(NB_CAP - 1 - q) * stride + i] & NB_JMASK));
    } else {
        for_each_neighbor(C, &C, B.CSTART, B.SNAP, B.Y[0], B.Y[1], B.Y[2], i, B.SNAP[i], B.CELLK[i],
                          [&](int j, float4, float, float, float, float, int) { emit(j); });
    }
}

__device__ __forceinline__ double axial_torque64(const BodyDev& Bd, const Bufs& B, int i, double fx, double fy,
                                                 double fz) {
    const double dx = B.Y[0][i] - Bd.c[0], dy = B.Y[1][i] - Bd.c[1], dz = B.Y[2][i] - Bd.c[2];
    const double tx = dy * fz - dz * fy, ty = dz * fx - dx * fz, tz = dx * fy - dy * fx;
    return tx * Bd.axis[0] + ty * Bd.axis[1] + tz * Bd.axis[2];
}

// Pass D: neighbour lists (exact FP64 membership, as in the FP32 path) and the
// density re-initialisation of Eq. (14) / Eq. (15) with sum W in FP64.
__global__ void __launch_bounds__(128) k_passD64(Bufs B, int par) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B.n) return;
    const float4 si = B.SNAP[i];
    const uint32_t tag = __float_as_uint(si.w);
    const uint32_t kind = tag_kind(tag);
    const CaseDev& C = B.cases[tag_case(tag)];
    if ((kind == KIND_STATIC && C.mat[tag_mat(tag)].fixed_T) || !B.st[tag_case(tag)].active) {
        B.NBC[i] = 0u;
        return;
    }
    const size_t stride = (size_t)B.nb_stride;
    uint32_t* nb = B.NB + i;
    double sum = C.w0_64;
    uint32_t nf = 0, nw = 0;
    for_each_neighbor(C, &C, B.CSTART, B.SNAP, B.Y[0], B.Y[1], B.Y[2], i, si, B.CELLK[i],
                      [&](int j, float4 sj, float, float, float, float, int code) {
                          double rx, ry, rz;
                          sum += W64(C, sqrt(geom64(C, B, i, j, rx, ry, rz)));
                          const uint32_t e = (uint32_t)j | ((uint32_t)code << 26);
                          const bool room = nf + nw < (uint32_t)NB_CAP;
                          if (tag_kind(__float_as_uint(sj.w)) == KIND_FLUID) {
                              if (room) nb[(size_t)nf * stride] = e;
                              ++nf;
                          } else {
                              if (room) nb[(size_t)(NB_CAP - 1 - nw) * stride] = e;
                              ++nw;
                          }
                      });
    if (nf + nw > (uint32_t)NB_CAP) {
        B.NBC[i] = NB_HAS | NB_OVF;
        atomicOr(&B.st[tag_case(tag)].err_info, ERR_NB_OVERFLOW);
    } else {
        B.NBC[i] = NB_HAS | nf | (nw << 8);
    }
    if (kind != KIND_FLUID) return;
    double4_32a* V = B.V64[1 - par];
    const double rr = C.mat64[tag_mat(tag)].rho0 * (sum * C.inv_sigma0_64 - 1.0);
    const double d = V[i].w;
    V[i].w = C.free_surface ? fmax(d, rr) : rr;
}

// Pass VT: viscous acceleration (Eq. 10 second term, wall term of Eq. 18) and
// dT/dt by the Cleary form (Eq. 22); rigid-body particles record the viscous
// torque of their fluid partners.
__global__ void __launch_bounds__(128) k_passVT64(Bufs B, int par) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B.n) return;
    const int cur = 1 - par;
    const uint32_t tag = B.TAG[cur][i];
    if (!B.st[tag_case(tag)].active) return;
    if (!(B.NBC[i] & NB_HAS)) {
        B.AV64[i] = make_double4_32a(0.0, 0.0, 0.0, 0.0);
        return;
    }
    const CaseDev& C = B.cases[tag_case(tag)];
    const MatDev64& Mi = C.mat64[tag_mat(tag)];
    const double4_32a* V = B.V64[cur];
    const double* T = B.T64[cur];
    const double Ti = T[i];
    const uint32_t kind = tag_kind(tag);
    if (kind == KIND_FLUID) {
        const double4_32a vi = V[i];
        const double rho_i = Mi.rho0 + vi.w;
        double ax = 0.0, ay = 0.0, az = 0.0, dT = 0.0;
        double G[3][3] = {{0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}};
        auto grad = [&](double g, double4_32a vj, double rx, double ry, double rz) {
            const double dv[3] = {vj.x - vi.x, vj.y - vi.y, vj.z - vi.z}, rr[3] = {rx, ry, rz};
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) G[a][b] += g * dv[a] * rr[b];
        };
        visit64<P_FLUID>(C, B, i, [&](int j, uint32_t tj, double rx, double ry, double rz, double r2) {
            const double r = sqrt(r2), inv_r = 1.0 / r;
            const double dW = dW64(C, r);
            const MatDev64& Mj = C.mat64[tag_mat(tj)];
            const double4_32a vj = V[j];
            const double Vj = Mj.mass / (Mj.rho0 + vj.w);
            const double cv = 2.0 * Vj * harm2(Mi.mu, Mj.mu) * inv_r * dW;
            ax += cv * (vi.x - vj.x);
            ay += cv * (vi.y - vj.y);
            az += cv * (vi.z - vj.z);
            dT += Vj * 2.0 * harm2(Mi.k, Mj.k) * (Ti - T[j]) * inv_r * dW;
            if (C.visc_heat) grad(Vj * dW * inv_r, vj, rx, ry, rz);
        });
        visit64<P_WALL>(C, B, i, [&](int j, uint32_t tj, double rx, double ry, double rz, double r2) {
            const double r = sqrt(r2), inv_r = 1.0 / r;
            const double dW = dW64(C, r);
            const MatDev64& Mj = C.mat64[tag_mat(tj)];
            const double4_32a vw = V[j];
            const double cv = 2.0 * C.vol64 * Mi.mu * inv_r * dW;  // the wall takes the fluid's viscosity
            ax += cv * (vi.x - vw.x);
            ay += cv * (vi.y - vw.y);
            az += cv * (vi.z - vw.z);
            dT += C.vol64 * 2.0 * harm2(Mi.k, Mj.k) * (Ti - T[j]) * inv_r * dW;
            if (C.visc_heat) grad(C.vol64 * dW * inv_r, vw, rx, ry, rz);
        });
        if (C.visc_heat) {  // viscous-dissipation heating Phi = 2 mu S:S (extension)
            double ss = 0.0;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) {
                    const double sab = 0.5 * (G[a][b] + G[b][a]);
                    ss += sab * sab;
                }
            dT += 2.0 * Mi.mu * ss;
        }
        B.AV64[i] = make_double4_32a(ax / rho_i, ay / rho_i, az / rho_i, dT / (rho_i * Mi.cp));
        return;
    }
    const bool thermal = !C.mat[tag_mat(tag)].fixed_T;
    const bool rot = kind == KIND_ROT;
    const double4_32a vw = V[i];
    double dT = 0.0, fx = 0.0, fy = 0.0, fz = 0.0, cf = 0.0;
    visit64<P_ALL>(C, B, i, [&](int j, uint32_t tj, double, double, double, double r2) {
        const double r = sqrt(r2), inv_r = 1.0 / r;
        const double dW = dW64(C, r);
        const MatDev64& Mj = C.mat64[tag_mat(tj)];
        const bool fj = tag_kind(tj) == KIND_FLUID;
        double Vj = C.vol64, rho_j = 1.0;
        double4_32a vj = make_double4_32a(0.0, 0.0, 0.0, 0.0);
        if (fj) {
            vj = V[j];
            rho_j = Mj.rho0 + vj.w;
            Vj = Mj.mass / rho_j;
        }
        if (thermal) dT += Vj * 2.0 * harm2(Mi.k, Mj.k) * (Ti - T[j]) * inv_r * dW;
        if (rot && fj) {
            const double c = -Mj.mass * (2.0 * C.vol64 / rho_j) * Mj.mu * inv_r * dW;
            fx += c * (vj.x - vw.x);
            fy += c * (vj.y - vw.y);
            fz += c * (vj.z - vw.z);
            cf += Vj * W64(C, r);  // contact factor (Eq. 24)
        }
    });
    B.AV64[i] = make_double4_32a(0.0, 0.0, 0.0, thermal ? dT * Mi.inv_rho0_cp : 0.0);
    if (rot) {
        const int id = B.ID[cur][i];
        B.TORQV64[id] = axial_torque64(C.body[tag_body(tag)], B, i, fx, fy, fz);
        B.CF[id] = cf * C.inv_contact_full64;
    }
}

// Half kick of density for the sub-step into VH64 (input of pass M).
__global__ void k_halfkick64(Bufs B, int par) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < B.n; i += gridDim.x * blockDim.x) {
        const uint32_t tag = B.TAG[1 - par][i];
        const CaseState& S = B.st[tag_case(tag)];
        if (!S.active) continue;
        double4_32a v = B.V64[1 - par][i];
        if (tag_kind(tag) == KIND_FLUID) v.w += 0.5 * S.dt * B.DR64[1 - par][i];
        B.VH64[i] = v;
    }
}

// Pass M: Riemann pressure force (Eqs. 10-12), wall problem (Eqs. 16-19 with
// the dissipation term of Eq. 12), kick and both half drifts; pressure torque
// on rigid-body particles.
__global__ void __launch_bounds__(128) k_passM64(Bufs B, int par) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B.n) return;
    const uint32_t tag = B.TAG[1 - par][i];
    const CaseState& S = B.st[tag_case(tag)];
    const uint32_t kind = tag_kind(tag);
    const bool first = S.nsub == 0;  // first sub-step of the advection step
    if (!S.active) {
        if (first && kind == KIND_FLUID)
            for (int a = 0; a < 3; ++a) B.X[a][i] = B.Y[a][i];
        return;
    }
    const CaseDev& C = B.cases[tag_case(tag)];
    const MatDev64& Mi = C.mat64[tag_mat(tag)];
    const double4_32a* VH = B.VH64;
    const double4_32a vi = VH[i];
    const double dt = S.dt, hd = 0.5 * S.dt;
    if (kind == KIND_FLUID) {
        const double dh_i = vi.w;
        const double rho_i = Mi.rho0 + dh_i;
        const double p_i = C.c02_64 * dh_i;
        double ax = 0.0, ay = 0.0, az = 0.0;
        visit64<P_FLUID>(C, B, i, [&](int j, uint32_t tj, double rx, double ry, double rz, double r2) {
            const double r = sqrt(r2), inv_r = 1.0 / r;
            const double dW = dW64(C, r);
            const MatDev64& Mj = C.mat64[tag_mat(tj)];
            const double4_32a vj = VH[j];
            const double rho_j = Mj.rho0 + vj.w;
            const double p_j = C.c02_64 * vj.w;
            const double dU = -inv_r * dot3(vi.x - vj.x, vi.y - vj.y, vi.z - vj.z, rx, ry, rz);
            const double beta = fmin(3.0 * fmax(dU, 0.0), C.c0_64);
            const double pstar = 0.5 * (p_i + p_j) + rho_i * rho_j * beta * dU / (rho_i + rho_j);
            const double coef = Mj.mass / rho_j * pstar * dW * inv_r;
            ax += coef * rx;
            ay += coef * ry;
            az += coef * rz;
        });
        visit64<P_WALL>(C, B, i, [&](int j, uint32_t, double rx, double ry, double rz, double r2) {
            const double r = sqrt(r2), inv_r = 1.0 / r;
            const double dW = dW64(C, r);
            const double4_32a nw = B.NRM64[j];
            const double4_32a vw = VH[j];
            const double g_rfw = -dot3(C.g64[0], C.g64[1], C.g64[2], rx, ry, rz);
            const double PR = p_i + rho_i * g_rfw;
            const double rhoR = Mi.rho0 + PR * C.inv_c02_64;
            const double dUw = -2.0 * dot3(nw.x, nw.y, nw.z, vi.x - vw.x, vi.y - vw.y, vi.z - vw.z);
            // Eq. (19) plus the limiter term of Eq. (12); wall_printed: Eq. (19) alone
            const double beta = C.wall_printed ? 0.0 : fmin(3.0 * fmax(dUw, 0.0), C.c0_64);
            const double pstar = (rho_i * PR + rhoR * p_i + rho_i * rhoR * beta * dUw) / (rho_i + rhoR);
            const double coef = C.vol64 * pstar * dW * inv_r;
            ax += coef * rx;
            ay += coef * ry;
            az += coef * rz;
        });
        const double k = -2.0 / rho_i;
        const double4_32a av = B.AV64[i];
        const double nv[3] = {vi.x + dt * (k * ax + av.x + C.g64[0]), vi.y + dt * (k * ay + av.y + C.g64[1]),
                              vi.z + dt * (k * az + av.z + C.g64[2])};
        B.V64[par][i] = make_double4_32a(nv[0], nv[1], nv[2], dh_i);
        const double vo[3] = {vi.x, vi.y, vi.z};
        for (int a = 0; a < 3; ++a) {
            double x = first ? B.Y[a][i] : B.X[a][i];
            x = x + hd * vo[a];
            x = x + hd * nv[a];
            B.X[a][i] = x;
        }
        const double sp = sqrt(nv[0] * nv[0] + nv[1] * nv[1] + nv[2] * nv[2]);
        if (!(sp <= 1.0e300) || !(fabs(dh_i) <= 1.0e300)) {
            atomicOr(&B.st[tag_case(tag)].err, ERR_NAN);
        } else {
            atomicMax(&B.st[tag_case(tag)].vmax64_bits, (unsigned long long)__double_as_longlong(sp));
        }
        return;
    }
    B.V64[par][i] = vi;
    if (kind != KIND_ROT || !(B.NBC[i] & NB_HAS)) return;
    const double4_32a nwi = B.NRM64[i];
    double fx = 0.0, fy = 0.0, fz = 0.0;
    visit64<P_FLUID>(C, B, i, [&](int j, uint32_t tj, double rx, double ry, double rz, double r2) {
        const double r = sqrt(r2), inv_r = 1.0 / r;
        const double dW = dW64(C, r);
        const MatDev64& Mj = C.mat64[tag_mat(tj)];
        const double4_32a vj = VH[j];
        const double rho_j = Mj.rho0 + vj.w;
        const double p_j = C.c02_64 * vj.w;
        const double g_rfw = dot3(C.g64[0], C.g64[1], C.g64[2], rx, ry, rz);
        const double PR = p_j + rho_j * g_rfw;
        const double rhoR = Mj.rho0 + PR * C.inv_c02_64;
        const double dUw = -2.0 * dot3(nwi.x, nwi.y, nwi.z, vj.x - vi.x, vj.y - vi.y, vj.z - vi.z);
        const double beta = C.wall_printed ? 0.0 : fmin(3.0 * fmax(dUw, 0.0), C.c0_64);
        const double pstar = (rho_j * PR + rhoR * p_j + rho_j * rhoR * beta * dUw) / (rho_j + rhoR);
        const double cf = -Mj.mass * (2.0 * C.vol64 / rho_j) * pstar * dW * inv_r;
        fx += cf * rx;
        fy += cf * ry;
        fz += cf * rz;
    });
    B.TORQ64[B.ID[1 - par][i]] = axial_torque64(C.body[tag_body(tag)], B, i, fx, fy, fz);
}

// Pass C: Riemann continuity (Eq. 10 first line, v* of Eq. 13), wall problem
// of Eqs. 16-17, second half kick of density.
__global__ void __launch_bounds__(128) k_passC64(Bufs B, int par) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B.n) return;
    const uint32_t tag = B.TAG[1 - par][i];
    const CaseState& S = B.st[tag_case(tag)];
    if (!S.active) return;
    const double4_32a* Vin = B.V64[par];
    const double4_32a vi = Vin[i];
    if (tag_kind(tag) != KIND_FLUID) {
        B.V64[1 - par][i] = vi;
        return;
    }
    const CaseDev& C = B.cases[tag_case(tag)];
    const MatDev64& Mi = C.mat64[tag_mat(tag)];
    const double rho_i = Mi.rho0 + vi.w;
    double d = 0.0;
    visit64<P_FLUID>(C, B, i, [&](int j, uint32_t tj, double rx, double ry, double rz, double r2) {
        const double r = sqrt(r2), inv_r = 1.0 / r;
        const double dW = dW64(C, r);
        const MatDev64& Mj = C.mat64[tag_mat(tj)];
        const double4_32a vj = Vin[j];
        const double rho_j = Mj.rho0 + vj.w;
        // (v_i - v*).e_ij from U_R - U_L = (v_i - v_j).e_ij and p_i - p_j = c0^2 (drho_i - drho_j):
        // U* - U_L = (U_R - U_L)/2 + (p_i - p_j) / (c0 (rho_i + rho_j)); with Eq. (13)'s printed
        // sign it is 2 U~ - U_L - U* = (U_R - U_L)(1/2 - (rho_i - rho_j)/(rho_i + rho_j)) - (p_i - p_j) / (c0 (rho_i + rho_j))
        const double dU = inv_r * dot3(vi.x - vj.x, vi.y - vj.y, vi.z - vj.z, rx, ry, rz);
        const double dp = C.c0_64 * (vi.w - vj.w) / (rho_i + rho_j);
        const double du = C.vstar_lit ? dU * (0.5 - (rho_i - rho_j) / (rho_i + rho_j)) - dp : 0.5 * dU + dp;
        d += Mj.mass / rho_j * du * dW;
    });
    visit64<P_WALL>(C, B, i, [&](int j, uint32_t, double rx, double ry, double rz, double r2) {
        const double r = sqrt(r2), inv_r = 1.0 / r;
        const double dW = dW64(C, r);
        const double4_32a nw = B.NRM64[j];
        const double4_32a vw = Vin[j];
        const double g_rfw = -dot3(C.g64[0], C.g64[1], C.g64[2], rx, ry, rz);
        const double PR = rho_i * g_rfw + C.c02_64 * vi.w;
        const double rhoR = Mi.rho0 + PR * C.inv_c02_64;
        const double du = dot3(nw.x, nw.y, nw.z, vi.x - vw.x, vi.y - vw.y, vi.z - vw.z) -
                          rho_i * g_rfw * C.inv_c0_64 / (rho_i + rhoR);
        d += C.vol64 * du * dot3(nw.x, nw.y, nw.z, rx, ry, rz) * inv_r * dW;
    });
    const double drho = 2.0 * rho_i * d;
    B.V64[1 - par][i] = make_double4_32a(vi.x, vi.y, vi.z, vi.w + 0.5 * S.dt * drho);
    B.DR64[1 - par][i] = drho;
}

inline int blocks(int n, int t) { return n > 0 ? (n + t - 1) / t : 1; }

}  // namespace

cudaError_t launch_passD64(const Bufs& B, int par, cudaStream_t s) {
    k_passD64<<<blocks(B.n, 128), 128, 0, s>>>(B, par);
    return cudaGetLastError();
}

cudaError_t launch_passVT64(const Bufs& B, int par, cudaStream_t s) {
    k_passVT64<<<blocks(B.n, 128), 128, 0, s>>>(B, par);
    return cudaGetLastError();
}

cudaError_t launch_passM64(const Bufs& B, int par, cudaStream_t s) {
    k_halfkick64<<<blocks(B.n, 256), 256, 0, s>>>(B, par);
    k_passM64<<<blocks(B.n, 128), 128, 0, s>>>(B, par);
    return cudaGetLastError();
}

cudaError_t launch_passC64(const Bufs& B, int par, cudaStream_t s) {
    k_passC64<<<blocks(B.n, 128), 128, 0, s>>>(B, par);
    return cudaGetLastError();
}

}  // namespace sph
