// sph_kernels.cu -- CUDA kernels of the coupled SPH step (sm_103a).
//
// Per advection step (Sec. 2.8): adv_begin -> cell sort (hash, count, scan,
// scatter, id-order, reorder) -> pass D (Eq. 14/15) -> pass VT (viscous
// part of Eq. 10 and Eq. 18; conduction Eq. 22) -> acoustic sub-steps
// [sub_begin -> pass M (Eqs. 10-12, 16-19) -> pass C (Eqs. 10-13, 16-17) ->
// sub_end] x cap -> T update and fixed-order FP64 reductions.
//
// Pair arithmetic is FP32 on the frozen snapshot geometry; positions,
// temperatures, time and all reductions are FP64.  No kernel waits on
// another block, so no kernel can hang.
#include <cstdio>

#include <type_traits>

#include "sph_kernels.cuh"

namespace sph {

static int g_grid_cap = 148 * 8;
void set_grid_cap(int sms) { g_grid_cap = sms * 8; }

static inline int grid_stride_grid(int n, int block) {
    int g = (n + block - 1) / block;
    if (g > g_grid_cap) g = g_grid_cap;
    return g < 1 ? 1 : g;
}
static inline int grid_1to1(int n, int block) {
    int g = (n + block - 1) / block;
    return g < 1 ? 1 : g;
}

#define GSTRIDE_LOOP(i, n) for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += gridDim.x * blockDim.x)

// ------------------------------------------------------------- admission ---
// One staged block of a newly admitted case (ids idb.., all of one kind,
// material and body) into the packed arrays from slot `at`: positions to the
// work and reference arrays, velocity and density excess, reference normals,
// temperatures, ids and tags.  Missing inputs (null): zero velocity and
// normal, the material's T_init and rho0.
__global__ void k_admit_block(Bufs B, int par, int n, int at, int idb, uint32_t tag, int fluid, double rho0,
                              double T_init, const double* __restrict__ pos, const double* __restrict__ vel,
                              const double* __restrict__ nrm, const double* __restrict__ T,
                              const double* __restrict__ rho) {
    GSTRIDE_LOOP(q, n) {
        const int i = at + q, id = idb + q;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double x = pos[3 * q + a];
            B.X[a][i] = x;
            B.RP[a][id] = x;
        }
        const double v[3] = {vel && fluid ? vel[3 * q] : 0.0, vel && fluid ? vel[3 * q + 1] : 0.0,
                             vel && fluid ? vel[3 * q + 2] : 0.0};
        const double dr = fluid ? (rho ? rho[q] : rho0) - rho0 : 0.0;
        B.V[par][i] = make_float4((float)v[0], (float)v[1], (float)v[2], (float)dr);
        const double nv[3] = {nrm ? nrm[3 * q] : 0.0, nrm ? nrm[3 * q + 1] : 0.0, nrm ? nrm[3 * q + 2] : 0.0};
        B.RN[id] = make_float4((float)nv[0], (float)nv[1], (float)nv[2], 0.f);
        B.T64[par][i] = T ? T[q] : T_init;
        B.ID[par][i] = id;
        B.TAG[par][i] = tag;
        if (B.fp64) {
            B.V64[par][i] = make_double4_32a(v[0], v[1], v[2], dr);
            B.RN64[id] = make_double4_32a(nv[0], nv[1], nv[2], 0.0);
        }
    }
}

cudaError_t launch_admit_block(const Bufs& B, int par, int n, int at, int idb, uint32_t tag, int fluid, double rho0,
                               double T_init, const double* pos, const double* vel, const double* nrm, const double* T,
                               const double* rho, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_admit_block<<<grid_stride_grid(n, 256), 256, 0, s>>>(B, par, n, at, idb, tag, fluid, rho0, T_init, pos, vel, nrm,
                                                          T, rho);
    return cudaGetLastError();
}

// --------------------------------------------------------------- control ---
// Initial max speed of the particles in slots [lo, hi) (a newly admitted
// case): warp-aggregated atomics per case.
__global__ void k_vmax_init(Bufs B, int par, int lo, int hi) {
    const int stride = gridDim.x * blockDim.x;
    const int span = hi - lo;
    const int rounds = (span + stride - 1) / stride;
    for (int k = 0; k < rounds; ++k) {
        const int i = lo + k * stride + blockIdx.x * blockDim.x + threadIdx.x;
        int c = -1;
        unsigned bits = 0u;
        if (i < hi) {
            const uint32_t tag = B.TAG[par][i];
            if (tag_kind(tag) == KIND_FLUID) {
                c = (int)tag_case(tag);
                if (B.fp64) {
                    const double4_32a v = B.V64[par][i];
                    const double sp = sqrt(v.x * v.x + v.y * v.y + v.z * v.z);
                    atomicMax(&B.st[c].vmax64_bits, (unsigned long long)__double_as_longlong(sp));
                } else {
                    const float4 v = B.V[par][i];
                    bits = __float_as_uint(sqrtf(dot3f(v.x, v.y, v.z, v.x, v.y, v.z)));
                }
            }
        }
        const unsigned peers = __match_any_sync(0xffffffffu, c);
        const unsigned m = __reduce_max_sync(peers, bits);
        if (c >= 0 && (int)(threadIdx.x & 31) == __ffs(peers) - 1) atomicMax(&B.st[c].vmax_bits, m);
    }
}

// Eq. (25) first line: dt_ad = cfl_ad min(h / max(|v|max, u_ref), h^2 / nu),
// at most the thermal bound of Eq. (26).
__global__ void k_adv_begin(Bufs B) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= B.ncases) return;
    const CaseDev& C = B.cases[c];
    CaseState& S = B.st[c];
    double vmax = C.fp64 ? __longlong_as_double((long long)S.vmax64_bits) : (double)__uint_as_float(S.vmax_bits);
    double U = vmax > C.u_ref ? vmax : C.u_ref;
    double a = C.h64 / U;
    if (C.nu_max > 0.0) {
        double b = C.h64 * C.h64 / C.nu_max;
        if (b < a) a = b;
    }
    S.dt_ad = C.cfl_ad * a;
    if (C.dt_T < S.dt_ad) S.dt_ad = C.dt_T;  // Eq. (26)
    S.tau = 0.0;
    S.nsub = 0;
    S.active = (S.alive && S.running) ? 1 : 0;
    S.last = 0;
    for (int b = 0; b < MAX_BODY; ++b) {
        double th = C.body[b].omega * S.t;
        double sn, cs;
        sincos(th, &sn, &cs);
        S.cs[b] = cs;
        S.sn[b] = sn;
    }
}

// Eq. (25) second line, clipped to land exactly on dt_ad.
__global__ void k_sub_begin(Bufs B) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= B.ncases) return;
    const CaseDev& C = B.cases[c];
    CaseState& S = B.st[c];
    if (!S.active) {
        S.dt = 0.0;
        S.dtf = 0.0f;
        S.hdtf = 0.0f;
        return;
    }
    double vmax = C.fp64 ? __longlong_as_double((long long)S.vmax64_bits) : (double)__uint_as_float(S.vmax_bits);
    double dt_ac = C.cfl_ac * C.h64 / (C.c0_64 + vmax);
    double rem = S.dt_ad - S.tau;
    int reach = rem <= dt_ac;
    double dt = reach ? rem : dt_ac;
    S.reach = reach;
    S.last = reach || (S.nsub + 1 >= C.kcap);
    S.dt = dt;
    S.dtf = (float)dt;
    S.hdtf = (float)(0.5 * dt);
    S.vmax_bits = 0u;
    S.vmax64_bits = 0ull;
}

// fixed-order block reduction of doubles (blockDim = 256)
__device__ double block_sum_256(double v, double* sh) {
    int t = threadIdx.x;
    sh[t] = v;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (t < s) sh[t] += sh[t + s];
        __syncthreads();
    }
    double r = sh[0];
    __syncthreads();
    return r;
}

// Torque of the fluid on each rigid body: per-particle contributions summed
// over the body's id range (id order: independent of the sort and of other
// resident cases) in two fixed-order levels, chunks of TQ_CHUNK ids first.
__global__ void __launch_bounds__(256) k_torque_chunks(Bufs B) {
    __shared__ double sh[256];
    const int4 q = B.TQC[blockIdx.x];  // (case, body, id_lo, id_hi)
    const CaseDev& C = B.cases[q.x];
    const CaseState& S = B.st[q.x];
    if (!S.active) return;
    const bool first = S.nsub == 0;
    double acc = 0.0, accv = 0.0;
    for (int id = q.z + threadIdx.x; id < q.w; id += 256) {
        acc += C.fp64 ? B.TORQ64[id] : (double)B.TORQ[id];
        if (first) accv += C.fp64 ? B.TORQV64[id] : (double)B.TORQV[id];
    }
    acc = block_sum_256(acc, sh);
    accv = first ? block_sum_256(accv, sh) : 0.0;
    if (threadIdx.x == 0) {
        B.TQP[2 * blockIdx.x] = acc;
        B.TQP[2 * blockIdx.x + 1] = accv;
    }
}

// ... then the chunk sums of each body in order, and the sub-step's time
// bookkeeping (one thread per case).
__global__ void k_sub_end(Bufs B) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= B.ncases) return;
    const CaseDev& C = B.cases[c];
    CaseState& S = B.st[c];
    if (!S.active) return;
    const int first = S.nsub == 0;
    for (int b = 0; b < C.n_body; ++b) {
        if (!C.body[b].set) continue;
        const int2 r = B.TQR[c * MAX_BODY + b];  // (first chunk, chunks)
        double tq = 0.0, tqv = 0.0;
        for (int k = 0; k < r.y; ++k) {
            tq += B.TQP[2 * (r.x + k)];
            tqv += B.TQP[2 * (r.x + k) + 1];
        }
        S.tq_p[b] = tq;
        if (first) S.tq_v[b] = tqv;
        S.tq_inst[b] = S.tq_p[b] + S.tq_v[b];
        S.tq_int[b] += S.dt * S.tq_inst[b];
    }
    S.time_int += S.dt;
    S.tau = S.reach ? S.dt_ad : S.tau + S.dt;
    S.nsub += 1;
    S.substeps += 1;
    if (S.last) S.active = 0;
}

// Condition of the graph's sub-step loop (a WHILE conditional node): run
// another sub-step while any case has one left.  Every case stops after at
// most kcap sub-steps (k_sub_begin), so the loop always ends.
__global__ void k_sub_cond(Bufs B, cudaGraphConditionalHandle h) {
    int any = 0;
    for (int c = threadIdx.x; c < B.ncases; c += blockDim.x) any |= B.st[c].active;
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) cudaGraphSetConditional(h, any ? 1u : 0u);
}

// ------------------------------------------------------------ cell sort ---
// x rounded toward zero to FP32 with integer operations only (FP64
// arithmetic and conversions share the slow FP64 pipe): |error| < 2^-23 |x|
// in FP32's normal range, magnitudes below it give 0 (error < 2^-126).
// False for magnitudes above FP32's range, infinities and NaN.
__device__ __forceinline__ bool f64_to_f32_trunc(double x, float* out) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
    const int e = (int)((hi >> 20) & 0x7ffu) - 1023 + 127;
    if (e >= 255) return false;
    *out = e <= 0 ? 0.0f
                  : __uint_as_float((hi & 0x80000000u) | ((uint32_t)e << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29));
    return true;
}

// The conversion instructions for the rare operands of the two helpers
// below, out of line so that they are branched around rather than issued
// (predicated) for every operand.
__device__ __noinline__ float f64_to_f32_insn(double x) { return (float)x; }
__device__ __noinline__ double f32_to_f64_insn(float x) { return (double)x; }

// (float)x, the FP64 -> FP32 conversion rounding to nearest (ties to
// even), with integer operations when x lies in FP32's normal range; the
// conversion instruction (FP64 pipe) only for the rest (zero, subnormal
// results, overflow, infinities, NaN).
__device__ __forceinline__ float f64_to_f32_rn(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
    const int e = (int)((hi >> 20) & 0x7ffu) - 1023 + 127;
    if (e <= 0 || e >= 255) return f64_to_f32_insn(x);
    const uint32_t sign = hi & 0x80000000u;
    // 23 kept mantissa bits, 29 dropped ones; a carry out of the mantissa
    // moves into the exponent, which is the correct rounding
    uint32_t f = sign | ((uint32_t)e << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
    const uint32_t rest = lo & 0x1fffffffu, half = 0x10000000u;
    if (rest > half || (rest == half && (f & 1u))) f += 1u;
    return __uint_as_float(f);
}

// (double)x, exact, with integer operations for normal x and zeros; the
// conversion instruction (FP64 pipe) only for subnormals, infinities and NaN.
__device__ __forceinline__ double f32_to_f64(float x) {
    const uint32_t u = __float_as_uint(x);
    const uint32_t e = (u >> 23) & 0xffu;
    if ((u << 1) == 0u) return __hiloint2double((int)(u & 0x80000000u), 0);  // +-0
    if (e == 0u || e == 255u) return f32_to_f64_insn(x);
    const uint32_t hi = (u & 0x80000000u) | ((e + (1023u - 127u)) << 20) | ((u & 0x7fffffu) >> 3);
    return __hiloint2double((int)hi, (int)(u << 29));
}

// (double)g, exact, for an unsigned integer, with integer operations.
__device__ __forceinline__ double u32_to_f64(uint32_t g) {
    if (g == 0u) return 0.0;
    const int lz = __clz(g);  // the leading one is bit 31 - lz; move it to bit 52
    const unsigned long long m = (unsigned long long)g << (21 + lz);
    return __longlong_as_double(
        (long long)(((unsigned long long)(1023 + 31 - lz) << 52) | (m & 0xfffffffffffffull)));
}

__device__ __forceinline__ uint32_t cell_key(const CaseDev& C, const double p[3], bool* out) {
    int cc[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        // floor((p - o) / w) of the FP64 quotient.  An FP32 estimate from
        // FP32 copies of p and o decides when its fraction is farther from an
        // integer than a bound on its error: 2^-23 |p| + 2^-24 |o| from the
        // copies and three FP32 roundings, in units of w, well under the
        // margin below.  Else the FP64 product with 1/w (a few ulp off)
        // decides unless it lies within 1e-9 of an integer, and there the
        // division itself is taken.
        const int top = C.ncell[a] - 1;
        float pf;
        bool fast = f64_to_f32_trunc(p[a], &pf);
        int ci = 0;
        if (fast) {
            const float of = C.originf[a], iw = C.inv_scellwf[a];
            const float qf = (pf - of) * iw;
            const float ff = floorf(qf);
            const float mf = 1e-6f * (1.0f + fabsf(qf) + (fabsf(pf) + fabsf(of)) * iw);
            fast = qf - ff > mf && qf - ff < 1.0f - mf;
            ci = (int)ff;
        }
        if (fast) {
            if (ci < 0) {
                ci = 0;
                *out = true;
            } else if (ci > top) {
                ci = top;
                *out = true;
            }
        } else {
            const double d = p[a] - C.origin[a];
            double q = d * C.inv_cellw[a];
            if (fabs(q - rint(q)) < 1e-9 * fmax(1.0, fabs(q))) q = d / C.cellw[a];
            double f = floor(q);
            if (!(f >= 0.0)) {
                f = 0.0;
                *out = true;
            } else if (f > (double)top) {
                f = (double)top;
                *out = true;
            }
            ci = (int)f;
        }
        cc[a] = ci;
    }
    return (uint32_t)(C.cell_base + (cc[2] * C.ncell[1] + cc[1]) * C.ncell[0] + cc[0]);
}

__global__ void k_hash(Bufs B, int par) {
    GSTRIDE_LOOP(s, B.n) {
        const uint32_t tag = B.TAG[par][s];
        const int c = tag_case(tag);
        const CaseDev& C = B.cases[c];
        if (!B.st[c].alive) {  // retired case: its particles go to the last bucket
            B.KEYS[s] = (uint32_t)B.ncells;
            B.RANK[s] = atomicAdd(&B.CNT[B.ncells], 1u);
            continue;
        }
        double p[3];
        const bool fluid = tag_kind(tag) == KIND_FLUID;
        if (fluid) {
            p[0] = B.X[0][s];
            p[1] = B.X[1][s];
            p[2] = B.X[2][s];
            bool moved = false;
#pragma unroll
            for (int a = 0; a < 3; ++a)
                if (C.periodic & (1 << a)) {
                    double L = C.ext[a], o = C.origin[a];
                    if (p[a] >= o + L) { p[a] -= L; moved = true; }
                    else if (p[a] < o) { p[a] += L; moved = true; }
                }
            if (moved && B.st[c].running) {  // a finished case keeps its state untouched
                B.X[0][s] = p[0];
                B.X[1][s] = p[1];
                B.X[2][s] = p[2];
            }
        } else {
            solid_position(C, B.st[c], tag, B.RP[0], B.RP[1], B.RP[2], B.ID[par][s], p);
        }
        bool out = false;
        uint32_t key = cell_key(C, p, &out);
        if (out && fluid && B.st[c].running) atomicOr(&B.st[c].err, ERR_ESCAPE);
        B.KEYS[s] = key;
        B.RANK[s] = atomicAdd(&B.CNT[key], 1u);
    }
}

// exclusive scan of cnt[0..ncells) into cstart, tiles of SCAN_TILE cells
__global__ void __launch_bounds__(1024) k_scan_tiles(const uint32_t* __restrict__ cnt, uint32_t* cstart,
                                                     uint32_t* blk, int ncells) {
    __shared__ uint32_t wsum[32];
    const int t = threadIdx.x;
    const int base = blockIdx.x * SCAN_TILE + 2 * t;
    uint32_t a = base < ncells ? cnt[base] : 0u;
    uint32_t b = base + 1 < ncells ? cnt[base + 1] : 0u;
    uint32_t v = a + b;
    const int lane = t & 31, w = t >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
        uint32_t s = wsum[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        wsum[lane] = s;
    }
    __syncthreads();
    uint32_t excl = x - v + (w > 0 ? wsum[w - 1] : 0u);
    if (base < ncells) cstart[base] = excl;
    if (base + 1 < ncells) cstart[base + 1] = excl + a;
    if (t == 1023) blk[blockIdx.x] = wsum[31];
}

__global__ void __launch_bounds__(1024) k_scan_top(uint32_t* blk, int nblk, uint32_t* cstart, int ncells) {
    __shared__ uint32_t wsum[32];
    __shared__ uint32_t carry;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    if (t == 0) carry = 0u;
    __syncthreads();
    for (int base = 0; base < nblk; base += 1024) {
        uint32_t v = base + t < nblk ? blk[base + t] : 0u;
        uint32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[w] = x;
        __syncthreads();
        if (w == 0) {
            uint32_t s = wsum[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += y;
            }
            wsum[lane] = s;
        }
        __syncthreads();
        uint32_t excl = x - v + (w > 0 ? wsum[w - 1] : 0u) + carry;
        if (base + t < nblk) blk[base + t] = excl;
        __syncthreads();
        if (t == 1023) carry = excl + v;
        __syncthreads();
    }
    if (t == 0) cstart[ncells] = carry;
}

__global__ void k_scan_add(uint32_t* cstart, const uint32_t* __restrict__ blk, uint32_t* cnt, int ncells) {
    GSTRIDE_LOOP(i, ncells) {
        cstart[i] += blk[i / SCAN_TILE];
        cnt[i] = 0u;
    }
}

__global__ void k_scatter(int n, const uint32_t* __restrict__ keys, const uint32_t* __restrict__ rank,
                          const uint32_t* __restrict__ cstart, uint32_t* tmp) {
    GSTRIDE_LOOP(s, n) tmp[cstart[keys[s]] + rank[s]] = (uint32_t)s;
}

// Within a cell, order by particle id: rank = #{cell members with smaller id}.
// Particles in the bucket `dead` (retired cases, dropped after this sort) keep
// their arrival rank: their order does not matter and the bucket can be large.
__global__ void k_order(int n, const uint32_t* __restrict__ keys, const uint32_t* __restrict__ cstart,
                        const uint32_t* __restrict__ tmp, const int* __restrict__ ids, uint32_t* perm,
                        const uint32_t* __restrict__ rank, uint32_t dead) {
    GSTRIDE_LOOP(s, n) {
        const uint32_t key = keys[s];
        if (key == dead) {
            perm[cstart[key] + rank[s]] = (uint32_t)s;
            continue;
        }
        const uint32_t a = cstart[key], b = cstart[key + 1];
        const int my = ids ? ids[s] : s;
        uint32_t r = 0;
        for (uint32_t t = a; t < b; ++t) {
            const uint32_t o = tmp[t];
            const int id = ids ? ids[o] : (int)o;
            r += id < my;
        }
        perm[a + r] = (uint32_t)s;
    }
}

__device__ void solid_at(const CaseDev& C, const CaseState& S, uint32_t tag, const Bufs& B, int id, double p[3],
                         double n[3], double v[3]);

// Gather every per-particle field into cell order; build the frozen snapshot.
__global__ void k_reorder(Bufs B, int par) {
    const int in = par, out = 1 - par;
    GSTRIDE_LOOP(d, B.n) {
        const int s = (int)B.PERM[d];
        const uint32_t tag = B.TAG[in][s];
        const int id = B.ID[in][s];
        const int c = tag_case(tag);
        const CaseDev& C = B.cases[c];
        const uint32_t key = B.KEYS[s];
        const bool fluid = tag_kind(tag) == KIND_FLUID;
        if (key == (uint32_t)B.ncells) {  // retired case: carried to the end, then dropped
            B.SNAP[d] = make_float4(0.f, 0.f, 0.f, __uint_as_float(tag));
            B.CELLK[d] = key;
            B.ID[out][d] = id;
            B.TAG[out][d] = tag;
            continue;
        }
        double p[3];
        if (fluid) {
            p[0] = B.X[0][s];
            p[1] = B.X[1][s];
            p[2] = B.X[2][s];
        } else {
            solid_position(C, B.st[c], tag, B.RP[0], B.RP[1], B.RP[2], id, p);
        }
        B.Y[0][d] = p[0];
        B.Y[1][d] = p[1];
        B.Y[2][d] = p[2];
        int cl = (int)key - C.cell_base;
        // offsets from the corner of the geometry cell (SPLIT_X x 2 x 2 sort cells);
        // cc: the geometry cell per axis
        int cc[3] = {(cl % C.ncell[0]) / SPLIT_X, ((cl / C.ncell[0]) % C.ncell[1]) >> 1,
                     (cl / (C.ncell[0] * C.ncell[1])) >> 1};
        float off[3];
        if (C.gcorner_ok) {
#pragma unroll
            for (int a = 0; a < 3; ++a) off[a] = f64_to_f32_rn(p[a] - C.gcorner[a][cc[a]]);
        } else {
#pragma unroll
            for (int a = 0; a < 3; ++a)
                off[a] = f64_to_f32_rn((p[a] - C.origin[a]) - u32_to_f64((uint32_t)cc[a]) * C.gcellw[a]);
        }
        B.SNAP[d] = make_float4(off[0], off[1], off[2], __uint_as_float(tag));
        B.CELLK[d] = key;
        if (fluid) {
            if (C.fp64) {
                B.V64[out][d] = B.V64[in][s];
                B.DR64[out][d] = B.DR64[in][s];
            } else {
                B.V[out][d] = B.V[in][s];
                B.DR[out][d] = B.DR[in][s];
            }
        } else if (C.fp64) {
            double sp[3], sn[3], sv[3];
            solid_at(C, B.st[c], tag, B, id, sp, sn, sv);
            B.V64[out][d] = make_double4_32a(sv[0], sv[1], sv[2], 0.0);
            B.DR64[out][d] = 0.0;
            B.NRM64[d] = make_double4_32a(sn[0], sn[1], sn[2], 0.0);
        } else {
            float4 n0 = B.RN[id];
            float vw[3] = {0.f, 0.f, 0.f};
            float nn[3] = {n0.x, n0.y, n0.z};
            if (tag_kind(tag) == KIND_ROT) {
                const int b = tag_body(tag);
                const BodyDev& Bd = C.body[b];
                const float cs = (float)B.st[c].cs[b], sn = (float)B.st[c].sn[b];
                const float ax = (float)Bd.axis[0], ay = (float)Bd.axis[1], az = (float)Bd.axis[2];
                float an = ax * n0.x + ay * n0.y + az * n0.z;
                float axn[3] = {ay * n0.z - az * n0.y, az * n0.x - ax * n0.z, ax * n0.y - ay * n0.x};
                float A[3] = {ax, ay, az};
#pragma unroll
                for (int k = 0; k < 3; ++k) nn[k] = cs * nn[k] + sn * axn[k] + (1.0f - cs) * an * A[k];
                // v_w = omega axis x (r_w - c)
                float d0 = (float)(p[0] - Bd.c[0]), d1 = (float)(p[1] - Bd.c[1]), d2 = (float)(p[2] - Bd.c[2]);
                float w = (float)Bd.omega;
                vw[0] = w * (ay * d2 - az * d1);
                vw[1] = w * (az * d0 - ax * d2);
                vw[2] = w * (ax * d1 - ay * d0);
            }
            B.V[out][d] = make_float4(vw[0], vw[1], vw[2], 0.0f);
            B.DR[out][d] = 0.0f;
            B.NRM[d] = make_float4(nn[0], nn[1], nn[2], 0.0f);
        }
        const double T = B.T64[in][s];
        B.T64[out][d] = T;
        B.T32[d] = f64_to_f32_rn(T - C.T_ref);
        B.ID[out][d] = id;
        B.TAG[out][d] = tag;
    }
}

// Case segments and the fixed reduction-chunk table (one thread).
__global__ void k_segments(Bufs B) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int q = 0;
    for (int c = 0; c < B.ncases; ++c) {
        const CaseDev& C = B.cases[c];
        CaseState& S = B.st[c];
        if (!S.alive) {
            S.seg_lo = S.seg_hi = 0;
            S.chunk_lo = q;
            S.nchunks = 0;
            continue;
        }
        S.seg_lo = (int)B.CSTART[C.cell_base];
        S.seg_hi = (int)B.CSTART[C.cell_base + C.ncells];
        int nch = (S.seg_hi - S.seg_lo + RED_CHUNK - 1) / RED_CHUNK;
        S.chunk_lo = q;
        S.nchunks = nch;
        for (int k = 0; k < nch && q < B.max_chunks; ++k) B.CHUNK_CASE[q++] = c;
    }
    *B.nchunks = q;  // chunks in use this step
    *B.novf = 0;  // overflow list of this advection step's neighbour search
}

// --------------------------------------------------------- pair passes ----
#define PAIR_ARGS B.CSTART, B.SNAP, B.Y[0], B.Y[1], B.Y[2]

constexpr int PART_FLUID = 1, PART_WALL = 2, PART_ALL = 3;

// Walk `cnt` list slots starting at slot k0 with step ks (+1 fluid part,
// -1 wall part); geometry from the snapshot offsets and the packed cell code.
// A thread loads its list entries BATCH at a time, one batch ahead of their
// use, and prefetches the batch after that from DRAM into L2, so that the
// (DRAM-resident) list stream is in flight while partners are gathered and
// summed.  With TPP threads per particle, thread `sub` takes list slots sub,
// sub + TPP, ...
template <int BATCH, int TPP, class CC, class F>
__device__ __forceinline__ void list_walk(const CC& C, const Bufs& B, int i, float4 si, int k0, int ks,
                                          int cnt, int sub, F&& f) {
    const size_t stride = (size_t)B.nb_stride;
    const uint32_t* __restrict__ nb = B.NB + (size_t)k0 * stride + i;
    const ptrdiff_t step = ks * (ptrdiff_t)stride;
    const float sx = si.x + C.gcellwf[0], sy = si.y + C.gcellwf[1], sz = si.z + C.gcellwf[2];
    // list entries one batch ahead of their use: the next batch's loads are
    // in flight while the current batch's partners are gathered and summed
    uint32_t e[BATCH];
#pragma unroll
    for (int u = 0; u < BATCH; ++u) e[u] = (sub + TPP * u < cnt) ? __ldg(nb + (sub + TPP * u) * step) : 0u;
    for (int q0 = sub; q0 < cnt; q0 += TPP * BATCH) {
#pragma unroll
        for (int u = 0; u < BATCH; ++u) {
            const int q = q0 + TPP * (2 * BATCH + u);
            if (q < cnt) asm volatile("prefetch.global.L2 [%0];" ::"l"(nb + q * step));
        }
        uint32_t en[BATCH];
#pragma unroll
        for (int u = 0; u < BATCH; ++u) {
            const int q = q0 + TPP * (BATCH + u);
            en[u] = q < cnt ? __ldg(nb + q * step) : 0u;
        }
#pragma unroll
        for (int u = 0; u < BATCH; ++u) {
            if (q0 + TPP * u < cnt) {
                const int j = (int)(e[u] & NB_JMASK);
                const uint32_t d = e[u] >> 26;
                const float4 sj = __ldg(B.SNAP + j);
                const float rx = fmaf(-(float)(d & 3u), C.gcellwf[0], sx) - sj.x;
                const float ry = fmaf(-(float)((d >> 2) & 3u), C.gcellwf[1], sy) - sj.y;
                const float rz = fmaf(-(float)(d >> 4), C.gcellwf[2], sz) - sj.z;
                const float r2 = fmaf(rz, rz, fmaf(ry, ry, rx * rx));
                f(j, sj, rx, ry, rz, r2);
            }
        }
#pragma unroll
        for (int u = 0; u < BATCH; ++u) e[u] = en[u];
    }
}

// Neighbours of a particle from its list (the common case), walked by TPP
// adjacent threads; sum() adds the threads' partial sums (the same value on
// each) and lead() marks the thread that stores the particle's results.
template <int BATCH, int TPP, class CC>
struct ListVis {
    const CC& C;
    const Bufs& B;
    int i;
    float4 si;
    uint32_t cnt;
    int sub = 0;
    template <int PART, class F>
    __device__ __forceinline__ void run(F&& f) const {
        if (PART & PART_FLUID) list_walk<BATCH, TPP>(C, B, i, si, 0, 1, (int)(cnt & 255u), sub, f);
        if (PART & PART_WALL) list_walk<BATCH, TPP>(C, B, i, si, NB_CAP - 1, -1, (int)((cnt >> 8) & 255u), sub, f);
    }
    __device__ __forceinline__ float sum(float x) const {
        // the two threads of the particle (adjacent lanes) wait for each other here
        if (TPP == 2) x += __shfl_xor_sync(3u << ((threadIdx.x & 31u) & ~1u), x, 1);
        return x;
    }
    __device__ __forceinline__ bool lead() const { return sub == 0; }
};

// ... or, for a particle whose partners did not fit its list, from the
// 27-cell loop with the same exact membership rule.
struct CellVis {
    const CaseDev& C;
    const Bufs& B;
    int i;
    float4 si;
    __device__ __forceinline__ float sum(float x) const { return x; }
    __device__ __forceinline__ bool lead() const { return true; }
    template <int PART, class F>
    __device__ __forceinline__ void run(F&& f) const {
        // the overflow kernels read the case table: C is the global entry
        for_each_neighbor(C, &C, PAIR_ARGS, i, si, B.CELLK[i],
                          [&](int j, float4 sj, float rx, float ry, float rz, float r2, int) {
                              const bool fj = tag_kind(__float_as_uint(sj.w)) == KIND_FLUID;
                              if ((fj && (PART & PART_FLUID)) || (!fj && (PART & PART_WALL)))
                                  f(j, sj, rx, ry, rz, r2);
                          });
    }
};

__device__ __forceinline__ bool listed(uint32_t cnt) { return (cnt & NB_HAS) && !(cnt & NB_OVF); }

// Where the pair passes read a particle's case constants: the global case
// table, or the table of pair constants in the kernel's parameter block
// (indexed by case slot), or its entry 0 when a single case is resident.
enum { CM_GLOBAL = 0, CM_ONE = 1, CM_TAB = 2 };
// the pair passes' constant argument: the whole table only where it is read
template <int CM>
using PairArg = std::conditional_t<CM == CM_TAB, PairTab, PairConst>;
template <int CM, class F>
__device__ __forceinline__ void with_case(const Bufs& B, const PairArg<CM>& T, uint32_t tag, F&& f) {
    if constexpr (CM == CM_GLOBAL) f(B.cases[tag_case(tag)]);
    else if constexpr (CM == CM_ONE) f(T);
    else f(T.c[tag_case(tag)]);
}
template <int CM>
static inline const PairArg<CM>& pair_arg(const PairTab& T) {
    if constexpr (CM == CM_TAB) return T;
    else return T.c[0];
}
template <int BATCH, int TPP, class CC>
__device__ __forceinline__ ListVis<BATCH, TPP, CC> list_vis(const CC& C, const Bufs& B, int i, float4 si,
                                                           uint32_t cnt, int sub) {
    return ListVis<BATCH, TPP, CC>{C, B, i, si, cnt, sub};
}

// Pass D: the advection step's neighbour search (27-cell loop, exact FP64
// membership) writes every particle's partner list, and fluid particles get
// their density re-initialised, Eq. (14) (free surface) or Eq. (15); sum W
// runs over all partners (fluid and wall) plus the particle itself.  Static
// walls of fixed temperature have no pair sums of their own and get no list.
template <class CC>
__device__ __forceinline__ void d_particle(const Bufs& B, int par, int i, float4 si, uint32_t tag, const CC& C) {
    const uint32_t kind = tag_kind(tag);
    const MatDev& Mi = C.mat[tag_mat(tag)];
    if ((kind == KIND_STATIC && Mi.fixed_T) || !B.st[tag_case(tag)].active) {
        B.NBC[i] = 0u;
        return;
    }
    const size_t stride = (size_t)B.nb_stride;
    uint32_t* nb = B.NB + i;
    float sum = C.w0;
    uint32_t nf = 0, nw = 0;
    for_each_neighbor(C, B.cases + tag_case(tag), PAIR_ARGS, i, si, B.CELLK[i],
                      [&](int j, float4 sj, float, float, float, float r2, int code) {
        // r from the reciprocal root estimate; the add is kept unfused so that
        // every variant of the kernel rounds the sum alike
        sum = __fadd_rn(sum, kernel_W(C, r2 * rsqrtf(fmaxf(r2, 1e-30f))));
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
        B.OVFL[atomicAdd(B.novf, 1)] = i;
        atomicOr(&B.st[tag_case(tag)].err_info, ERR_NB_OVERFLOW);
    } else {
        B.NBC[i] = NB_HAS | nf | (nw << 8);
    }
    if (kind != KIND_FLUID) return;
    float4* V = B.V[1 - par];
    const float rr = Mi.rho0 * fmaf(sum, C.inv_sigma0, -1.0f);
    const float d = V[i].w;
    V[i].w = C.free_surface ? fmaxf(d, rr) : rr;
}

template <int CM>
__global__ void __launch_bounds__(256, 4) k_passD(Bufs B, int par, const PairArg<CM> T) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B.n) return;
    const float4 si = B.SNAP[i];
    const uint32_t tag = __float_as_uint(si.w);
    with_case<CM>(B, T, tag, [&](const auto& C) { d_particle(B, par, i, si, tag, C); });
}

__device__ __forceinline__ float axial_torque(const BodyDev& Bd, const double* __restrict__ Yx,
                                              const double* __restrict__ Yy, const double* __restrict__ Yz,
                                              int i, float fx, float fy, float fz) {
    float dx = (float)(Yx[i] - Bd.c[0]), dy = (float)(Yy[i] - Bd.c[1]), dz = (float)(Yz[i] - Bd.c[2]);
    float tx = dy * fz - dz * fy, ty = dz * fx - dx * fz, tz = dx * fy - dy * fx;
    return tx * (float)Bd.axis[0] + ty * (float)Bd.axis[1] + tz * (float)Bd.axis[2];
}

__device__ __forceinline__ float harmonic2(float a, float b) {
    const float s = a + b;
    return s > 0.f ? __fdividef(2.f * a * b, s) : 0.f;
}

// UNI: every fluid particle of a case has the same material, the case's
// `fluid` entry (a constant of the pair table), so neither a fluid particle's
// own material nor its fluid partners' need a table load.
template <bool UNI, class CC>
__device__ __forceinline__ const MatDev& fluid_mat(const CC& C, uint32_t tj) {
    if constexpr (UNI) return C.fluid;
    else return C.mat[tag_mat(tj)];
}

// Pass VT for one particle: viscous acceleration (Eq. 10 second term; wall
// term of Eq. 18), held for the sub-steps, and dT/dt by the Cleary form
// (Eq. 22).  Rigid-body particles also record the viscous torque on them.
// VH: also the viscous-dissipation heating Phi = 2 mu S:S (an extension the
// paper's thermal model omits; per case by its flag), S the symmetric part of
// the velocity gradient sum_j V_j (v_j - v_i) (x) grad_i W_ij over fluid and
// wall partners, added to dT/dt as Phi / (rho c_p).
template <bool UNI, class Vis, bool VH = false, class CC>
__device__ __forceinline__ void vt_particle(const Bufs& B, int par, int i, float4 si, uint32_t tag,
                                            const CC& C, const Vis& vis) {
    const uint32_t kind = tag_kind(tag);
    const MatDev& Mi = C.mat[tag_mat(tag)];
    const float4* __restrict__ V = B.V[1 - par];
    const float* __restrict__ T32 = B.T32;
    const float Ti = T32[i];
    if (kind == KIND_FLUID) {
        const MatDev& Mf = fluid_mat<UNI>(C, tag);
        const float4 vi = V[i];
        const float rho_i = Mf.rho0 + vi.w;
        float ax = 0.f, ay = 0.f, az = 0.f, dT = 0.f;
        float G[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
        const bool vh = VH && C.visc_heat;
        auto grad = [&](float g, float4 vj, float rx, float ry, float rz) {
            const float dv[3] = {vj.x - vi.x, vj.y - vi.y, vj.z - vi.z}, rr[3] = {rx, ry, rz};
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b) G[a][b] = fmaf(g * dv[a], rr[b], G[a][b]);
        };
        const float Kii = 2.f * harmonic2(Mf.k, Mf.k), eii = harmonic2(Mf.mu, Mf.mu);
        vis.template run<PART_FLUID>([&](int j, float4 sj, float rx, float ry, float rz, float r2) {
            const float s = kernel_dW_over_r(C, r2 * rsqrtf(r2));  // dW/dr / r
            const MatDev& Mj = fluid_mat<UNI>(C, __float_as_uint(sj.w));
            const float4 vj = __ldg(V + j);
            const float Vs = __fdividef(Mj.mass, Mj.rho0 + vj.w) * s;  // V_j dW/dr / r
            const float cv = 2.f * (UNI ? eii : harmonic2(Mf.mu, Mj.mu)) * Vs;
            ax = fmaf(cv, vi.x - vj.x, ax);
            ay = fmaf(cv, vi.y - vj.y, ay);
            az = fmaf(cv, vi.z - vj.z, az);
            const float K = UNI ? Kii : 2.f * harmonic2(Mf.k, Mj.k);
            dT = fmaf(K * (Ti - __ldg(T32 + j)), Vs, dT);
            if (VH && vh) grad(Vs, vj, rx, ry, rz);
        });
        vis.template run<PART_WALL>([&](int j, float4 sj, float rx, float ry, float rz, float r2) {
            const float Vs = C.vol * kernel_dW_over_r(C, r2 * rsqrtf(r2));  // V_w dW/dr / r
            const MatDev& Mj = C.mat[tag_mat(__float_as_uint(sj.w))];
            const float4 vw = __ldg(V + j);
            const float cv = 2.f * Mf.mu * Vs;  // the wall takes the fluid's viscosity
            ax = fmaf(cv, vi.x - vw.x, ax);
            ay = fmaf(cv, vi.y - vw.y, ay);
            az = fmaf(cv, vi.z - vw.z, az);
            const float K = 2.f * harmonic2(Mf.k, Mj.k);
            dT = fmaf(K * (Ti - __ldg(T32 + j)), Vs, dT);
            if (VH && vh) grad(Vs, vw, rx, ry, rz);
        });
        if (VH && vh) {
            // r_ij = r_i - r_j and grad_i W = W' r_ij / r, so the sums above carry
            // V_j W' / r (v_j - v_i)_a (r_ij)_b
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b) G[a][b] = vis.sum(G[a][b]);
            float ss = 0.f;
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    const float sab = 0.5f * (G[a][b] + G[b][a]);
                    ss = fmaf(sab, sab, ss);
                }
            dT = fmaf(2.f * Mf.mu, ss, dT);  // Phi, divided by rho_i c_p with the conduction sum below
        }
        ax = vis.sum(ax);
        ay = vis.sum(ay);
        az = vis.sum(az);
        dT = vis.sum(dT);
        const float inv_rho = 1.0f / rho_i;
        if (vis.lead()) B.AV[i] = make_float4(ax * inv_rho, ay * inv_rho, az * inv_rho, dT * inv_rho / Mf.cp);
        return;
    }
    const bool thermal = !Mi.fixed_T;
    const bool rot = kind == KIND_ROT;
    const float4 vw = V[i];
    float dT = 0.f, fx = 0.f, fy = 0.f, fz = 0.f, cf = 0.f;
    vis.template run<PART_ALL>([&](int j, float4 sj, float, float, float, float r2) {
        const float r = r2 * rsqrtf(r2);
        const float s = kernel_dW_over_r(C, r);  // dW/dr / r
        const uint32_t tj = __float_as_uint(sj.w);
        const MatDev& Mj = C.mat[tag_mat(tj)];
        const bool fj = tag_kind(tj) == KIND_FLUID;
        float Vj = C.vol;
        float rho_j = 1.f;
        float4 vj = make_float4(0.f, 0.f, 0.f, 0.f);
        if (fj) {
            vj = __ldg(V + j);
            rho_j = Mj.rho0 + vj.w;
            Vj = __fdividef(Mj.mass, rho_j);
        }
        if (thermal) {
            const float K = 2.f * harmonic2(Mi.k, Mj.k);
            dT = fmaf(Vj * K * (Ti - __ldg(T32 + j)), s, dT);
        }
        if (rot && fj) {
            // force of fluid j on this wall particle: -m_j a_jw, with
            // a_jw = 2 V_w / rho_j mu_j (v_j - v_w) / r dW/dr
            const float c = -Mj.mass * __fdividef(2.f * C.vol, rho_j) * Mj.mu * s;
            fx = fmaf(c, vj.x - vw.x, fx);
            fy = fmaf(c, vj.y - vw.y, fy);
            fz = fmaf(c, vj.z - vw.z, fz);
            // contact factor (Eq. 24): lubricant volume weighted by W
            cf = fmaf(Vj, kernel_W(C, r), cf);
        }
    });
    dT = vis.sum(dT);
    fx = vis.sum(fx);
    fy = vis.sum(fy);
    fz = vis.sum(fz);
    cf = vis.sum(cf);
    if (!vis.lead()) return;
    B.AV[i] = make_float4(0.f, 0.f, 0.f, thermal ? dT * Mi.inv_rho0_cp : 0.f);
    if (rot) {
        const BodyDev& Bd = C.body[tag_body(tag)];
        const int id = B.ID[1 - par][i];
        B.TORQV[id] = axial_torque(Bd, B.Y[0], B.Y[1], B.Y[2], i, fx, fy, fz);
        B.CF[id] = (double)(cf * C.inv_contact_full);
    }
}

template <bool UNI, int BATCH, int TPP, int CM, bool VH = false>
__global__ void __launch_bounds__(256) k_passVT(Bufs B, int par, const PairArg<CM> T) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = g / TPP, sub = g % TPP;
    if (i >= B.n) return;
    const uint32_t cnt = B.NBC[i];
    if (!listed(cnt)) {
        if (!(cnt & NB_HAS) && sub == 0) B.AV[i] = make_float4(0.f, 0.f, 0.f, 0.f);  // no pair sums: no heating
        return;                                                            // overflow: k_passVT_ovf
    }
    const float4 si = B.SNAP[i];
    const uint32_t tag = __float_as_uint(si.w);
    if (!B.st[tag_case(tag)].active) return;
    with_case<CM>(B, T, tag, [&](const auto& C) {
        const auto vis = list_vis<BATCH, TPP>(C, B, i, si, cnt, sub);
        vt_particle<UNI, decltype(vis), VH>(B, par, i, si, tag, C, vis);
    });
}

template <bool UNI, bool VH = false>
__global__ void __launch_bounds__(128) k_passVT_ovf(Bufs B, int par) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < *B.novf; k += gridDim.x * blockDim.x) {
        const int i = B.OVFL[k];
        const float4 si = B.SNAP[i];
        const uint32_t tag = __float_as_uint(si.w);
        const CaseDev& C = B.cases[tag_case(tag)];
        vt_particle<UNI, CellVis, VH>(B, par, i, si, tag, C, CellVis{C, B, i, si});
    }
}

// Half kick of density for the sub-step (rho += dt/2 drho), written with the
// velocity into VH, the input of pass M for the particle and its partners.
__global__ void k_halfkick(Bufs B, int par) {
    const float4* __restrict__ Vin = B.V[1 - par];
    const float* __restrict__ DR = B.DR[1 - par];
    GSTRIDE_LOOP(i, B.n) {
        const uint32_t tag = B.TAG[1 - par][i];
        const CaseState& S = B.st[tag_case(tag)];
        if (!S.active) continue;
        float4 v = Vin[i];
        if (tag_kind(tag) == KIND_FLUID) v.w = fmaf(S.hdtf, DR[i], v.w);
        B.VH[i] = v;
    }
}

// Pass M for one particle: Riemann pressure force (Eqs. 10-12) and the wall
// problem (Eqs. 16-19) with half-kicked densities and the EoS (Eq. 2),
// velocity kick, both half drifts of the position (FP64).  Rigid-body
// particles record the pressure torque of their fluid partners.
template <bool UNI, class Vis, class CC>
__device__ __forceinline__ void m_particle(const Bufs& B, int par, int first, int i, float4 si, uint32_t tag,
                                           const CC& C, const CaseState& S, const Vis& vis, int* case_out,
                                           unsigned* vbits_out) {
    const uint32_t kind = tag_kind(tag);
    const float4* __restrict__ VH = B.VH;
    float4* Vout = B.V[par];
    const float hdt = S.hdtf, dt = S.dtf;
    const float4 vi = VH[i];
    if (kind == KIND_FLUID) {
        const MatDev& Mi = fluid_mat<UNI>(C, tag);
        const float dh_i = vi.w;
        const float rho_i = Mi.rho0 + dh_i;
        const float p_i = C.c02 * dh_i;
        float ax = 0.f, ay = 0.f, az = 0.f;
        vis.template run<PART_FLUID>([&](int j, float4 sj, float rx, float ry, float rz, float r2) {
            const float inv_r = rsqrtf(r2);
            const float s = kernel_dW_over_r(C, r2 * inv_r);  // dW/dr / r
            const MatDev& Mj = fluid_mat<UNI>(C, __float_as_uint(sj.w));
            const float4 vj = __ldg(VH + j);
            const float rho_j = Mj.rho0 + vj.w;
            // U_L - U_R = -(v_i - v_j).e_ij
            const float dU = -inv_r * dot3f(vi.x - vj.x, vi.y - vj.y, vi.z - vj.z, rx, ry, rz);
            const float beta = fminf(3.f * fmaxf(dU, 0.f), C.c0);
            // V_j p* with V_j = m_j / rho_j and p* = (p_i + p_j)/2 + rho_i rho_j
            // beta dU / (rho_i + rho_j), over the one reciprocal of
            // rho_j (rho_i + rho_j); p_i + p_j with p_j = c0^2 (rho_j - rho0) fused
            const float srho = rho_i + rho_j;
            const float num = fmaf(rho_i * rho_j, beta * dU, 0.5f * fmaf(C.c02, vj.w, p_i) * srho);
            const float coef = __fdividef(Mj.mass * num, rho_j * srho) * s;
            ax = fmaf(coef, rx, ax);
            ay = fmaf(coef, ry, ay);
            az = fmaf(coef, rz, az);
        });
        vis.template run<PART_WALL>([&](int j, float4, float rx, float ry, float rz, float r2) {
            const float s = kernel_dW_over_r(C, r2 * rsqrtf(r2));  // dW/dr / r
            // one-sided wall problem: P_R = p_f + rho_f g.r_fw, r_fw = -r_ij;
            // U_L - U_R = 2 (U_L - u_w) = -2 n.(v_f - v_w)
            const float4 nw = __ldg(B.NRM + j);
            const float4 vw = __ldg(VH + j);
            const float g_rfw = -dot3f(C.g[0], C.g[1], C.g[2], rx, ry, rz);
            const float PR = fmaf(rho_i, g_rfw, p_i);
            const float rhoR = fmaf(PR, C.inv_c02, Mi.rho0);
            const float dUw = -2.f * dot3f(nw.x, nw.y, nw.z, vi.x - vw.x, vi.y - vw.y, vi.z - vw.z);
            const float beta = fminf(3.f * fmaxf(dUw, 0.f), C.c0);
            const float pstar = __fdividef(fmaf(rho_i * rhoR * beta, dUw, fmaf(rho_i, PR, rhoR * p_i)), rho_i + rhoR);
            const float coef = C.vol * pstar * s;
            ax = fmaf(coef, rx, ax);
            ay = fmaf(coef, ry, ay);
            az = fmaf(coef, rz, az);
        });
        ax = vis.sum(ax);
        ay = vis.sum(ay);
        az = vis.sum(az);
        const float k = -2.f / rho_i;
        const float4 av = B.AV[i];
        const float nvx = fmaf(dt, fmaf(k, ax, av.x) + C.g[0], vi.x);
        const float nvy = fmaf(dt, fmaf(k, ay, av.y) + C.g[1], vi.y);
        const float nvz = fmaf(dt, fmaf(k, az, av.z) + C.g[2], vi.z);
        const float sp = sqrtf(dot3f(nvx, nvy, nvz, nvx, nvy, nvz));
        *case_out = (int)tag_case(tag);
        *vbits_out = __float_as_uint(sp <= 3.0e38f ? sp : 3.0e38f);
        if (!vis.lead()) return;
        Vout[i] = make_float4(nvx, nvy, nvz, dh_i);
        // x + hd v with hd and v FP32 values: their product is exact in FP64,
        // so one fused operation rounds as the product-then-sum does
        const double hd = f32_to_f64(hdt);
        const double* Xs[3] = {first ? B.Y[0] : B.X[0], first ? B.Y[1] : B.X[1], first ? B.Y[2] : B.X[2]};
        const float vo[3] = {vi.x, vi.y, vi.z}, vn[3] = {nvx, nvy, nvz};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            double x = Xs[a][i];
            x = __fma_rn(hd, f32_to_f64(vo[a]), x);
            x = __fma_rn(hd, f32_to_f64(vn[a]), x);
            B.X[a][i] = x;
        }
        if (!(sp <= 3.0e38f) || !(fabsf(dh_i) <= 3.0e38f)) atomicOr(&B.st[tag_case(tag)].err, ERR_NAN);
        return;
    }
    if (vis.lead()) Vout[i] = vi;
    if (kind != KIND_ROT) return;
    // rigid-body particle: pressure force of its fluid neighbours on it
    const float4 nwi = B.NRM[i];
    float fx = 0.f, fy = 0.f, fz = 0.f;
    vis.template run<PART_FLUID>([&](int j, float4 sj, float rx, float ry, float rz, float r2) {
        const float s = kernel_dW_over_r(C, r2 * rsqrtf(r2));  // dW/dr / r
        const MatDev& Mj = fluid_mat<UNI>(C, __float_as_uint(sj.w));
        const float4 vj = __ldg(VH + j);
        const float rho_j = Mj.rho0 + vj.w;
        const float p_j = C.c02 * vj.w;
        // for fluid j: r_fw = r_w - r_j = r_ij (this thread is the wall)
        const float g_rfw = dot3f(C.g[0], C.g[1], C.g[2], rx, ry, rz);
        const float PR = fmaf(rho_j, g_rfw, p_j);
        const float rhoR = fmaf(PR, C.inv_c02, Mj.rho0);
        const float dUw = -2.f * dot3f(nwi.x, nwi.y, nwi.z, vj.x - vi.x, vj.y - vi.y, vj.z - vi.z);
        const float beta = fminf(3.f * fmaxf(dUw, 0.f), C.c0);
        const float pstar = __fdividef(fmaf(rho_j * rhoR * beta, dUw, fmaf(rho_j, PR, rhoR * p_j)), rho_j + rhoR);
        // a_jw = -2 V_w / rho_j p* dW e_jw with e_jw = -r_ij / r; force on wall = -m_j a_jw
        const float cf = -Mj.mass * __fdividef(2.f * C.vol, rho_j) * pstar * s;
        fx = fmaf(cf, rx, fx);
        fy = fmaf(cf, ry, fy);
        fz = fmaf(cf, rz, fz);
    });
    fx = vis.sum(fx);
    fy = vis.sum(fy);
    fz = vis.sum(fz);
    if (!vis.lead()) return;
    const BodyDev& Bd = C.body[tag_body(tag)];
    B.TORQ[B.ID[1 - par][i]] = axial_torque(Bd, B.Y[0], B.Y[1], B.Y[2], i, fx, fy, fz);
}

template <bool UNI, int BATCH, int TPP, int CM>
__global__ void __launch_bounds__(256) k_passM(Bufs B, int par, const PairArg<CM> T) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = g / TPP, sub = g % TPP;
    int c = -1;
    unsigned vb = 0u;
    if (i < B.n) {
        const uint32_t cnt = B.NBC[i];
        const float4 si = B.SNAP[i];
        const uint32_t tag = __float_as_uint(si.w);
        const CaseState& S = B.st[tag_case(tag)];
        const int first = S.nsub == 0;  // first sub-step of the advection step
        if (S.active && (listed(cnt) || !(cnt & NB_HAS))) {
            with_case<CM>(B, T, tag, [&](const auto& C) {
                m_particle<UNI>(B, par, first, i, si, tag, C, S, list_vis<BATCH, TPP>(C, B, i, si, cnt, sub), &c, &vb);
            });
        } else if (!S.active && first && tag_kind(tag) == KIND_FLUID && sub == 0) {
            // a case that does not advance still needs its work positions in the new order
            B.X[0][i] = B.Y[0][i];
            B.X[1][i] = B.Y[1][i];
            B.X[2][i] = B.Y[2][i];
        }
    }
    // per-case max speed for the next step sizes: warp-aggregated atomics
    const unsigned peers = __match_any_sync(0xffffffffu, c);
    const unsigned m = __reduce_max_sync(peers, vb);
    if (c >= 0 && (int)(threadIdx.x & 31) == __ffs(peers) - 1) atomicMax(&B.st[c].vmax_bits, m);
}

template <bool UNI>
__global__ void __launch_bounds__(128) k_passM_ovf(Bufs B, int par) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < *B.novf; k += gridDim.x * blockDim.x) {
        const int i = B.OVFL[k];
        const float4 si = B.SNAP[i];
        const uint32_t tag = __float_as_uint(si.w);
        const CaseState& S = B.st[tag_case(tag)];
        if (!S.active) continue;
        const CaseDev& C = B.cases[tag_case(tag)];
        int c = -1;
        unsigned vb = 0u;
        m_particle<UNI>(B, par, S.nsub == 0, i, si, tag, C, S, CellVis{C, B, i, si}, &c, &vb);
        if (c >= 0) atomicMax(&B.st[c].vmax_bits, vb);
    }
}

// Pass C for one particle: Riemann continuity (Eq. 10 first line with v* of
// Eq. 13) and the wall problem of Eqs. (16)-(17); second half kick.
template <bool UNI, class Vis, class CC>
__device__ __forceinline__ void c_particle(const Bufs& B, int par, int i, float4 si, uint32_t tag,
                                           const CC& C, const CaseState& S, const Vis& vis) {
    const float4* __restrict__ Vin = B.V[par];
    float4* Vout = B.V[1 - par];
    const float4 vi = Vin[i];
    if (tag_kind(tag) != KIND_FLUID) {
        if (vis.lead()) Vout[i] = vi;
        return;
    }
    const MatDev& Mi = fluid_mat<UNI>(C, tag);
    const float rho_i = Mi.rho0 + vi.w;
    float d = 0.f;
    vis.template run<PART_FLUID>([&](int j, float4 sj, float rx, float ry, float rz, float r2) {
        const float r = r2 * rsqrtf(r2);
        const float s = kernel_dW_over_r(C, r);  // dW/dr / r
        const MatDev& Mj = fluid_mat<UNI>(C, __float_as_uint(sj.w));
        const float4 vj = __ldg(Vin + j);
        const float rho_j = Mj.rho0 + vj.w;
        const float srho = rho_i + rho_j;
        // V_j (U* - U_L) dW/dr with U* - U_L = (U_R - U_L)/2 + (p_i - p_j) / (c0 (rho_i + rho_j)),
        // U_R - U_L = (v_i - v_j).e, p_i - p_j = c0^2 (drho_i - drho_j) and V_j = m_j / rho_j:
        // m_j s ((v_i - v_j).r_ij (rho_i + rho_j) / 2 + c0 (drho_i - drho_j) r) / (rho_j (rho_i + rho_j))
        const float num = fmaf(0.5f * srho, dot3f(vi.x - vj.x, vi.y - vj.y, vi.z - vj.z, rx, ry, rz),
                               C.c0 * (vi.w - vj.w) * r);
        d = fmaf(__fdividef(Mj.mass * num, rho_j * srho), s, d);
    });
    vis.template run<PART_WALL>([&](int j, float4, float rx, float ry, float rz, float r2) {
        const float s = kernel_dW_over_r(C, r2 * rsqrtf(r2));  // dW/dr / r
        const float4 nw = __ldg(B.NRM + j);
        const float4 vw = __ldg(Vin + j);
        const float g_rfw = -dot3f(C.g[0], C.g[1], C.g[2], rx, ry, rz);
        const float PR = fmaf(rho_i, g_rfw, C.c02 * vi.w);
        const float rhoR = fmaf(PR, C.inv_c02, Mi.rho0);
        // U*_w - U_L = n.(v_f - v_w) + (p_f - P_R) / (c0 (rho_f + rho_R))
        const float du = dot3f(nw.x, nw.y, nw.z, vi.x - vw.x, vi.y - vw.y, vi.z - vw.z) -
                         __fdividef(rho_i * g_rfw * C.inv_c0, rho_i + rhoR);
        d = fmaf(C.vol * du * dot3f(nw.x, nw.y, nw.z, rx, ry, rz), s, d);
    });
    d = vis.sum(d);
    if (!vis.lead()) return;
    const float drho = 2.f * rho_i * d;
    Vout[i] = make_float4(vi.x, vi.y, vi.z, fmaf(S.hdtf, drho, vi.w));
    B.DR[1 - par][i] = drho;
}

template <bool UNI, int BATCH, int TPP, int CM>
__global__ void __launch_bounds__(256) k_passC(Bufs B, int par, const PairArg<CM> T) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = g / TPP, sub = g % TPP;
    if (i >= B.n) return;
    const uint32_t cnt = B.NBC[i];
    if ((cnt & NB_HAS) && (cnt & NB_OVF)) return;  // k_passC_ovf
    const float4 si = B.SNAP[i];
    const uint32_t tag = __float_as_uint(si.w);
    const CaseState& S = B.st[tag_case(tag)];
    if (!S.active) return;
    with_case<CM>(B, T, tag, [&](const auto& C) {
        c_particle<UNI>(B, par, i, si, tag, C, S, list_vis<BATCH, TPP>(C, B, i, si, cnt, sub));
    });
}

template <bool UNI>
__global__ void __launch_bounds__(128) k_passC_ovf(Bufs B, int par) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < *B.novf; k += gridDim.x * blockDim.x) {
        const int i = B.OVFL[k];
        const float4 si = B.SNAP[i];
        const uint32_t tag = __float_as_uint(si.w);
        const CaseState& S = B.st[tag_case(tag)];
        if (!S.active) continue;
        const CaseDev& C = B.cases[tag_case(tag)];
        c_particle<UNI>(B, par, i, si, tag, C, S, CellVis{C, B, i, si});
    }
}

// -------------------------------------------------- end of advection step ---
__global__ void k_T_update(Bufs B, int par) {
    const int cur = 1 - par;
    GSTRIDE_LOOP(i, B.n) {
        const uint32_t tag = B.TAG[cur][i];
        const CaseState& S = B.st[tag_case(tag)];
        if (!S.running || !S.alive) continue;
        const double r = B.cases[tag_case(tag)].fp64 ? B.AV64[i].w : f32_to_f64(B.AV[i].w);
        if (r != 0.0) B.T64[cur][i] += S.tau * r;
    }
}

// fixed-order partial sums per chunk of a case segment (blockDim 256)
__global__ void __launch_bounds__(256) k_reduce_chunks(Bufs B, int cur) {
    __shared__ double sh[256];
    const int nq = *B.nchunks;
    for (int q = blockIdx.x; q < nq; q += gridDim.x) {
        const int c = B.CHUNK_CASE[q];
        const CaseState& S = B.st[c];
        const CaseDev& C = B.cases[c];
        const int lo = S.seg_lo + (q - S.chunk_lo) * RED_CHUNK;
        const int hi = min(lo + RED_CHUNK, S.seg_hi);
        double a = 0.0, b = 0.0, m = 0.0;
        for (int i = lo + threadIdx.x; i < hi; i += 256) {
            const uint32_t tag = B.TAG[cur][i];
            if (tag_kind(tag) != KIND_FLUID) continue;
            const MatDev& M = C.mat[tag_mat(tag)];
            const double T = B.T64[cur][i];
            const double mm = f32_to_f64(M.mass);
            a += mm * f32_to_f64(M.cp) * T;
            b += mm * T;
            m += mm;
        }
        a = block_sum_256(a, sh);
        b = block_sum_256(b, sh);
        m = block_sum_256(m, sh);
        if (threadIdx.x == 0) {
            B.PART[3 * q + 0] = a;
            B.PART[3 * q + 1] = b;
            B.PART[3 * q + 2] = m;
        }
    }
}

// one block per case: the case's chunk partials in a fixed order (thread t
// takes chunks t, t + 256, ..., then a fixed tree)
__global__ void __launch_bounds__(256) k_reduce_cases(Bufs B) {
    __shared__ double sh[256];
    const int c = blockIdx.x;
    CaseState& S = B.st[c];
    const bool live = S.running && S.alive;
    double a = 0.0, b = 0.0, m = 0.0;
    for (int k = threadIdx.x; k < S.nchunks; k += 256) {
        const int q = S.chunk_lo + k;
        a += B.PART[3 * q + 0];
        b += B.PART[3 * q + 1];
        m += B.PART[3 * q + 2];
    }
    a = block_sum_256(a, sh);
    b = block_sum_256(b, sh);
    m = block_sum_256(m, sh);
    if (threadIdx.x != 0 || !live) return;
    S.heat = a - S.heat0;
    S.sum_mcpT = a;
    S.sum_mT = b;
    S.sum_m = m;
    S.mean_T = m > 0.0 ? b / m : 0.0;
}

__global__ void k_adv_end_cases(Bufs B) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= B.ncases) return;
    CaseState& S = B.st[c];
    if (!S.running || !S.alive) return;
    S.t += S.tau;
    S.adv_steps += 1;
    S.last_nsub = S.nsub;
    S.last_dt_ad = S.dt_ad;
    if (B.HIST && B.hist_cap > 0) {
        double* h = B.HIST + ((size_t)c * B.hist_cap + (size_t)((S.adv_steps - 1) % B.hist_cap)) * 8;
        h[0] = S.t;
        h[1] = S.tq_inst[0];
        h[2] = S.time_int > 0.0 ? S.tq_int[0] / S.time_int : 0.0;
        h[3] = S.heat;
        h[4] = S.mean_T;
        h[5] = S.dt_ad;
        h[6] = (double)S.nsub;
        h[7] = B.cases[c].fp64 ? __longlong_as_double((long long)S.vmax64_bits) : (double)__uint_as_float(S.vmax_bits);
    }
    if (S.steps_req > 0 && S.adv_steps >= S.steps_req) S.running = 0;
    // an unstable case (NaN/Inf state, or a fluid particle out of the box) is
    // frozen after the step that found it: later steps leave its state as it
    // was, readable, and the other cases of a batch go on unaffected
    if (S.err) S.running = 0;
}

// ------------------------------------------------------------- readback ---
// Solid particle rotated by (cos, sin) of its body's angle: position, normal
// and velocity from its reference geometry (rigid rotation about (c, axis),
// Rodrigues' formula in FP64).
__device__ void solid_rotated(const CaseDev& C, uint32_t tag, const Bufs& B, int id, double cs, double sn,
                              double p[3], double n[3], double v[3]) {
    p[0] = B.RP[0][id];
    p[1] = B.RP[1][id];
    p[2] = B.RP[2][id];
    if (C.fp64) {
        const double4_32a n0 = B.RN64[id];
        n[0] = n0.x;
        n[1] = n0.y;
        n[2] = n0.z;
    } else {
        const float4 n0 = B.RN[id];
        n[0] = n0.x;
        n[1] = n0.y;
        n[2] = n0.z;
    }
    v[0] = v[1] = v[2] = 0.0;
    if (tag_kind(tag) != KIND_ROT) return;
    const BodyDev& Bd = C.body[tag_body(tag)];
    const double* a = Bd.axis;
    double d[3] = {p[0] - Bd.c[0], p[1] - Bd.c[1], p[2] - Bd.c[2]};
    double rd[3], rn[3];
    for (int pass = 0; pass < 2; ++pass) {
        const double* x = pass == 0 ? d : n;
        double* y = pass == 0 ? rd : rn;
        const double axx[3] = {a[1] * x[2] - a[2] * x[1], a[2] * x[0] - a[0] * x[2], a[0] * x[1] - a[1] * x[0]};
        const double ax = a[0] * x[0] + a[1] * x[1] + a[2] * x[2];
        for (int k = 0; k < 3; ++k) y[k] = cs * x[k] + sn * axx[k] + (1.0 - cs) * ax * a[k];
    }
    for (int k = 0; k < 3; ++k) {
        p[k] = Bd.c[k] + rd[k];
        n[k] = rn[k];
    }
    v[0] = Bd.omega * (a[1] * rd[2] - a[2] * rd[1]);
    v[1] = Bd.omega * (a[2] * rd[0] - a[0] * rd[2]);
    v[2] = Bd.omega * (a[0] * rd[1] - a[1] * rd[0]);
}

// ... at the case's current time
__device__ void solid_now(const CaseDev& C, const CaseState& S, uint32_t tag, const Bufs& B, int id, double p[3],
                          double n[3], double v[3]) {
    double sn = 0.0, cs = 1.0;
    if (tag_kind(tag) == KIND_ROT) sincos(C.body[tag_body(tag)].omega * S.t, &sn, &cs);
    solid_rotated(C, tag, B, id, cs, sn, p, n, v);
}

// ... at the angle of the current advection step
__device__ void solid_at(const CaseDev& C, const CaseState& S, uint32_t tag, const Bufs& B, int id, double p[3],
                         double n[3], double v[3]) {
    const int b = tag_body(tag);
    solid_rotated(C, tag, B, id, S.cs[b], S.sn[b], p, n, v);
}

__global__ void k_gather_field(Bufs B, int par, int field, int cs, int id_base, double* out) {
    const int cur = 1 - par;
    GSTRIDE_LOOP(i, B.n) {
        const uint32_t tag = B.TAG[cur][i];
        if ((int)tag_case(tag) != cs) continue;
        const int gid = B.ID[cur][i];
        const int id = gid - id_base;
        const CaseDev& C = B.cases[tag_case(tag)];
        const bool fluid = tag_kind(tag) == KIND_FLUID;
        const float4 vf = B.V[cur][i];
        const double4_32a v = C.fp64 ? B.V64[cur][i] : make_double4_32a(vf.x, vf.y, vf.z, vf.w);
        const double rho0 = C.fp64 ? C.mat64[tag_mat(tag)].rho0 : (double)C.mat[tag_mat(tag)].rho0;
        const double c02 = C.fp64 ? C.c02_64 : (double)C.c02;
        double sp[3], sn[3], sv[3];
        if (!fluid && (field == 0 || field == 1 || field == 9)) solid_now(C, B.st[cs], tag, B, gid, sp, sn, sv);
        switch (field) {
        case 0:
            out[3 * (size_t)id + 0] = fluid ? B.X[0][i] : sp[0];
            out[3 * (size_t)id + 1] = fluid ? B.X[1][i] : sp[1];
            out[3 * (size_t)id + 2] = fluid ? B.X[2][i] : sp[2];
            break;
        case 1:
            out[3 * (size_t)id + 0] = fluid ? v.x : sv[0];
            out[3 * (size_t)id + 1] = fluid ? v.y : sv[1];
            out[3 * (size_t)id + 2] = fluid ? v.z : sv[2];
            break;
        case 2: out[id] = fluid ? rho0 + v.w : rho0; break;
        case 3: out[id] = fluid ? c02 * v.w : 0.0; break;
        case 4: out[id] = B.T64[cur][i]; break;
        case 5: out[id] = fluid ? (C.fp64 ? B.DR64[cur][i] : (double)B.DR[cur][i]) : 0.0; break;
        case 6: {
            const float4 af = B.AV[i];
            const double4_32a a = C.fp64 ? B.AV64[i] : make_double4_32a(af.x, af.y, af.z, af.w);
            out[3 * (size_t)id + 0] = fluid ? a.x : 0.0;
            out[3 * (size_t)id + 1] = fluid ? a.y : 0.0;
            out[3 * (size_t)id + 2] = fluid ? a.z : 0.0;
            break;
        }
        case 7: out[id] = C.fp64 ? B.AV64[i].w : (double)B.AV[i].w; break;
        case 11: out[id] = tag_kind(tag) == KIND_ROT ? B.CF[gid] : 0.0; break;
        case 9:
            out[3 * (size_t)id + 0] = fluid ? 0.0 : sn[0];
            out[3 * (size_t)id + 1] = fluid ? 0.0 : sn[1];
            out[3 * (size_t)id + 2] = fluid ? 0.0 : sn[2];
            break;
        default: break;
        }
    }
}

// neighbour read-back: from the particle's list when it has one (what the
// passes use), else from the 27-cell loop (walls without pair sums)
template <class F>
__device__ __forceinline__ void visit_any(const CaseDev& C, const Bufs& B, int i, float4 si, F&& f) {
    const uint32_t cnt = B.NBC[i];
    auto g = [&](int j, float4, float, float, float, float) { f(j); };
    if (listed(cnt)) list_vis<1, 1>(C, B, i, si, cnt, 0).template run<PART_ALL>(g);
    else CellVis{C, B, i, si}.template run<PART_ALL>(g);
}

__global__ void __launch_bounds__(128) k_nb_count(Bufs B, int par, int cs, int id_base, int64_t* counts) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B.n) return;
    const float4 si = B.SNAP[i];
    if ((int)tag_case(__float_as_uint(si.w)) != cs) return;
    const CaseDev& C = B.cases[cs];
    int64_t k = 0;
    visit_any(C, B, i, si, [&](int) { ++k; });
    counts[B.ID[1 - par][i] - id_base] = k;
}

__global__ void __launch_bounds__(128) k_nb_list(Bufs B, int par, int cs, int id_base, const int64_t* start,
                                                 int32_t* list) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B.n) return;
    const float4 si = B.SNAP[i];
    if ((int)tag_case(__float_as_uint(si.w)) != cs) return;
    const CaseDev& C = B.cases[cs];
    const int* ID = B.ID[1 - par];
    int64_t k = start[ID[i] - id_base];
    visit_any(C, B, i, si, [&](int j) { list[k++] = ID[j] - id_base; });
}

// directed neighbour pairs of fluid particles by partner kind: [fluid, wall]
__global__ void __launch_bounds__(128) k_pair_stats(Bufs B, unsigned long long* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long ff = 0, fw = 0;
    if (i < B.n) {
        const float4 si = B.SNAP[i];
        const uint32_t tag = __float_as_uint(si.w);
        if (tag_kind(tag) == KIND_FLUID) {
            const CaseDev& C = B.cases[tag_case(tag)];
            const uint32_t cnt = B.NBC[i];
            if (listed(cnt)) {
                ff = cnt & 255u;
                fw = (cnt >> 8) & 255u;
            } else {
                CellVis{C, B, i, si}.template run<PART_FLUID>([&](int, float4, float, float, float, float) { ++ff; });
                CellVis{C, B, i, si}.template run<PART_WALL>([&](int, float4, float, float, float, float) { ++fw; });
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        ff += __shfl_down_sync(0xffffffffu, ff, o);
        fw += __shfl_down_sync(0xffffffffu, fw, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(out + 0, ff);
        atomicAdd(out + 1, fw);
    }
}

// Neighbour-search work of pass D: [particles searched, candidates tested
// (27-cell populations), partners found], over the particles with a search.
__global__ void __launch_bounds__(128) k_search_stats(Bufs B, unsigned long long* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long ns = 0, cand = 0, pairs = 0;
    if (i < B.n && (B.NBC[i] & NB_HAS)) {
        const float4 si = B.SNAP[i];
        const CaseDev& C = B.cases[tag_case(__float_as_uint(si.w))];
        ns = 1;
        for_each_run(C, B.CSTART, si, B.CELLK[i], [&](int a, int b, int, int, int) { cand += (unsigned)(b - a); });
        cand -= 1;  // the particle itself
        const uint32_t cnt = B.NBC[i];
        if (listed(cnt)) {
            pairs = (cnt & 255u) + ((cnt >> 8) & 255u);
        } else {
            CellVis{C, B, i, si}.template run<PART_ALL>([&](int, float4, float, float, float, float) { ++pairs; });
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        ns += __shfl_down_sync(0xffffffffu, ns, o);
        cand += __shfl_down_sync(0xffffffffu, cand, o);
        pairs += __shfl_down_sync(0xffffffffu, pairs, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(out + 0, ns);
        atomicAdd(out + 1, cand);
        atomicAdd(out + 2, pairs);
    }
}

cudaError_t launch_search_stats(const Bufs& B, unsigned long long* out, cudaStream_t s) {
    k_search_stats<<<grid_1to1(B.n, 128), 128, 0, s>>>(B, out);
    return cudaGetLastError();
}

cudaError_t launch_pair_stats(const Bufs& B, unsigned long long* out, cudaStream_t s) {
    k_pair_stats<<<grid_1to1(B.n, 128), 128, 0, s>>>(B, out);
    return cudaGetLastError();
}

// ----------------------------------------------------- stateless sort ----
__global__ void k_cs_hash(const double* __restrict__ pos, int n, double ox, double oy, double oz,
                          double wx, double wy, double wz, int nx, int ny, int nz, uint32_t* keys,
                          uint32_t* rank, uint32_t* cnt) {
    GSTRIDE_LOOP(s, n) {
        const double o[3] = {ox, oy, oz}, w[3] = {wx, wy, wz};
        const int nc[3] = {nx, ny, nz};
        int cc[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            double f = floor((pos[3 * (size_t)s + a] - o[a]) / w[a]);
            if (!(f >= 0.0)) f = 0.0;
            else if (f > (double)(nc[a] - 1)) f = (double)(nc[a] - 1);
            cc[a] = (int)f;
        }
        const uint32_t key = (uint32_t)((cc[2] * ny + cc[1]) * nx + cc[0]);
        keys[s] = key;
        rank[s] = atomicAdd(&cnt[key], 1u);
    }
}

// ------------------------------------------------------------ launchers ---
#define CK(x)                                   \
    do {                                        \
        cudaError_t e__ = (x);                  \
        if (e__ != cudaSuccess) return e__;     \
    } while (0)

size_t scan_blocks(int ncells) { return (size_t)((ncells + SCAN_TILE - 1) / SCAN_TILE); }

static cudaError_t launch_scan(uint32_t* cnt, uint32_t* cstart, uint32_t* blk, int ncells, cudaStream_t s) {
    const int nb = (int)scan_blocks(ncells);
    k_scan_tiles<<<nb, 1024, 0, s>>>(cnt, cstart, blk, ncells);
    k_scan_top<<<1, 1024, 0, s>>>(blk, nb, cstart, ncells);
    k_scan_add<<<grid_stride_grid(ncells, 256), 256, 0, s>>>(cstart, blk, cnt, ncells);
    return cudaGetLastError();
}

cudaError_t launch_vmax_init(const Bufs& B, int par, int lo, int hi, cudaStream_t s) {
    k_vmax_init<<<grid_stride_grid(hi - lo, 256), 256, 0, s>>>(B, par, lo, hi);
    return cudaGetLastError();
}

cudaError_t launch_adv_begin(const Bufs& B, cudaStream_t s) {
    k_adv_begin<<<(B.ncases + 63) / 64, 64, 0, s>>>(B);
    return cudaGetLastError();
}

cudaError_t launch_sort(const Bufs& B, int par, cudaStream_t s) {
    const int g = grid_stride_grid(B.n, 256);
    k_hash<<<g, 256, 0, s>>>(B, par);
    CK(launch_scan(B.CNT, B.CSTART, B.SCANBLK, B.ncells + 1, s));
    k_scatter<<<g, 256, 0, s>>>(B.n, B.KEYS, B.RANK, B.CSTART, B.TMP);
    k_order<<<g, 256, 0, s>>>(B.n, B.KEYS, B.CSTART, B.TMP, B.ID[par], B.PERM, B.RANK, (uint32_t)B.ncells);
    k_reorder<<<g, 256, 0, s>>>(B, par);
    k_segments<<<1, 32, 0, s>>>(B);
    return cudaGetLastError();
}

static const int kOvfGrid = 32;

static inline int pair_block(const Bufs& B) {
    return (B.tune_block == 64 || B.tune_block == 256) ? B.tune_block : 128;
}

// Case-constant source of the pair passes (see with_case).
static inline int case_mode(const Bufs& B) {
    if (B.one_case >= 0) return CM_ONE;
    return B.ncases <= PAIRTAB_MAX ? CM_TAB : CM_GLOBAL;
}

cudaError_t launch_passD(const Bufs& B, int par, const PairTab& T, cudaStream_t s) {
    if (B.fp64) return launch_passD64(B, par, s);
    const int blk = pair_block(B), grd = grid_1to1(B.n, blk);
    switch (case_mode(B)) {
    case CM_ONE: k_passD<CM_ONE><<<grd, blk, 0, s>>>(B, par, pair_arg<CM_ONE>(T)); break;
    case CM_TAB: k_passD<CM_TAB><<<grd, blk, 0, s>>>(B, par, pair_arg<CM_TAB>(T)); break;
    default: k_passD<CM_GLOBAL><<<grd, blk, 0, s>>>(B, par, pair_arg<CM_GLOBAL>(T)); break;
    }
    return cudaGetLastError();
}


// Pair-pass variant: list entries loaded together (B.tune_batch), threads per
// particle (B.tune_tpp), block size (B.tune_block) and the source of the case
// constants (case_mode).
#define DISPATCH_BT(KERNEL, UNI, CM, S, ...)                                                       \
    do {                                                                                           \
        const int tpp_ = B.tune_tpp == 2 ? 2 : 1;                                                  \
        const int blk_ = pair_block(B);                                                            \
        const int grd_ = grid_1to1(B.n * tpp_, blk_);                                              \
        switch (B.tune_batch * 4 + tpp_) {                                                         \
        case 1 * 4 + 1: KERNEL<UNI, 1, 1, CM><<<grd_, blk_, 0, S>>>(__VA_ARGS__, pair_arg<CM>(T)); break; \
        case 2 * 4 + 1: KERNEL<UNI, 2, 1, CM><<<grd_, blk_, 0, S>>>(__VA_ARGS__, pair_arg<CM>(T)); break; \
        case 4 * 4 + 1: KERNEL<UNI, 4, 1, CM><<<grd_, blk_, 0, S>>>(__VA_ARGS__, pair_arg<CM>(T)); break; \
        case 1 * 4 + 2: KERNEL<UNI, 1, 2, CM><<<grd_, blk_, 0, S>>>(__VA_ARGS__, pair_arg<CM>(T)); break; \
        case 2 * 4 + 2: KERNEL<UNI, 2, 2, CM><<<grd_, blk_, 0, S>>>(__VA_ARGS__, pair_arg<CM>(T)); break; \
        case 4 * 4 + 2: KERNEL<UNI, 4, 2, CM><<<grd_, blk_, 0, S>>>(__VA_ARGS__, pair_arg<CM>(T)); break; \
        case 8 * 4 + 2: KERNEL<UNI, 8, 2, CM><<<grd_, blk_, 0, S>>>(__VA_ARGS__, pair_arg<CM>(T)); break; \
        default: KERNEL<UNI, 8, 1, CM><<<grd_, blk_, 0, S>>>(__VA_ARGS__, pair_arg<CM>(T)); break;        \
        }                                                                                          \
    } while (0)
#define DISPATCH_PASS(KERNEL, UNI, S, ...)                                                         \
    do {                                                                                           \
        switch (case_mode(B)) {                                                                    \
        case CM_ONE: DISPATCH_BT(KERNEL, UNI, CM_ONE, S, __VA_ARGS__); break;                      \
        case CM_TAB: DISPATCH_BT(KERNEL, UNI, CM_TAB, S, __VA_ARGS__); break;                      \
        default: DISPATCH_BT(KERNEL, UNI, CM_GLOBAL, S, __VA_ARGS__); break;                       \
        }                                                                                          \
    } while (0)

template <bool UNI>
static void launch_passVT_heat(const Bufs& B, int par, const PairTab& T, cudaStream_t s) {
    const int blk = pair_block(B), grd = grid_1to1(B.n, blk);
    switch (case_mode(B)) {
    case CM_ONE: k_passVT<UNI, 2, 1, CM_ONE, true><<<grd, blk, 0, s>>>(B, par, pair_arg<CM_ONE>(T)); break;
    case CM_TAB: k_passVT<UNI, 2, 1, CM_TAB, true><<<grd, blk, 0, s>>>(B, par, pair_arg<CM_TAB>(T)); break;
    default: k_passVT<UNI, 2, 1, CM_GLOBAL, true><<<grd, blk, 0, s>>>(B, par, pair_arg<CM_GLOBAL>(T)); break;
    }
    k_passVT_ovf<UNI, true><<<kOvfGrid, 128, 0, s>>>(B, par);
}

cudaError_t launch_passVT(const Bufs& B, int par, const PairTab& T, cudaStream_t s) {
    if (B.fp64) return launch_passVT64(B, par, s);
    if (B.visc_heat) {
        // cases with viscous-dissipation heating: 2 entries per load and 1 thread
        // per particle (the list batch changes no result), case constants from
        // the parameter block where they fit
        if (B.uni_fluid) launch_passVT_heat<true>(B, par, T, s);
        else launch_passVT_heat<false>(B, par, T, s);
        return cudaGetLastError();
    }
    if (B.uni_fluid) {
        DISPATCH_PASS(k_passVT, true, s, B, par);
        k_passVT_ovf<true><<<kOvfGrid, 128, 0, s>>>(B, par);
    } else {
        DISPATCH_PASS(k_passVT, false, s, B, par);
        k_passVT_ovf<false><<<kOvfGrid, 128, 0, s>>>(B, par);
    }
    return cudaGetLastError();
}

cudaError_t launch_sub_begin(const Bufs& B, cudaStream_t s) {
    k_sub_begin<<<(B.ncases + 63) / 64, 64, 0, s>>>(B);
    return cudaGetLastError();
}

cudaError_t launch_passM(const Bufs& B, int par, const PairTab& T, cudaStream_t s) {
    if (B.fp64) return launch_passM64(B, par, s);
    k_halfkick<<<grid_stride_grid(B.n, 256), 256, 0, s>>>(B, par);
    if (B.uni_fluid) {
        DISPATCH_PASS(k_passM, true, s, B, par);
        k_passM_ovf<true><<<kOvfGrid, 128, 0, s>>>(B, par);
    } else {
        DISPATCH_PASS(k_passM, false, s, B, par);
        k_passM_ovf<false><<<kOvfGrid, 128, 0, s>>>(B, par);
    }
    return cudaGetLastError();
}

cudaError_t launch_passC(const Bufs& B, int par, const PairTab& T, cudaStream_t s) {
    if (B.fp64) return launch_passC64(B, par, s);
    if (B.uni_fluid) {
        DISPATCH_PASS(k_passC, true, s, B, par);
        k_passC_ovf<true><<<kOvfGrid, 128, 0, s>>>(B, par);
    } else {
        DISPATCH_PASS(k_passC, false, s, B, par);
        k_passC_ovf<false><<<kOvfGrid, 128, 0, s>>>(B, par);
    }
    return cudaGetLastError();
}

cudaError_t launch_sub_end(const Bufs& B, cudaStream_t s) {
    if (B.ntq > 0) k_torque_chunks<<<B.ntq, 256, 0, s>>>(B);
    k_sub_end<<<(B.ncases + 63) / 64, 64, 0, s>>>(B);
    return cudaGetLastError();
}

cudaError_t launch_reduce_heat(const Bufs& B, int par, cudaStream_t s) {
    int g = B.max_chunks_used < g_grid_cap ? B.max_chunks_used : g_grid_cap;
    k_reduce_chunks<<<g < 1 ? 1 : g, 256, 0, s>>>(B, 1 - par);
    k_reduce_cases<<<B.ncases, 256, 0, s>>>(B);
    return cudaGetLastError();
}

// Reference heat content of a newly admitted case from its appended block of
// slots [at, at+n) (id order), fixed-order: chunk partials, then their sum.
__global__ void __launch_bounds__(256) k_block_heat_chunks(Bufs B, int cur, int at, int n, double* part) {
    __shared__ double sh[256];
    const int nch = (n + RED_CHUNK - 1) / RED_CHUNK;
    for (int q = blockIdx.x; q < nch; q += gridDim.x) {
        const int lo = at + q * RED_CHUNK, hi = min(lo + RED_CHUNK, at + n);
        double a = 0.0;
        for (int i = lo + threadIdx.x; i < hi; i += 256) {
            const uint32_t tag = B.TAG[cur][i];
            if (tag_kind(tag) != KIND_FLUID) continue;
            const MatDev& M = B.cases[tag_case(tag)].mat[tag_mat(tag)];
            a += (double)M.mass * (double)M.cp * B.T64[cur][i];
        }
        a = block_sum_256(a, sh);
        if (threadIdx.x == 0) part[q] = a;
    }
}

__global__ void k_block_heat_final(Bufs B, int slot, int n, const double* part) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int nch = (n + RED_CHUNK - 1) / RED_CHUNK;
    double a = 0.0;
    for (int q = 0; q < nch; ++q) a += part[q];
    CaseState& S = B.st[slot];
    S.heat0 = a;
    S.heat = 0.0;
    S.init_pending = 0;
}

cudaError_t launch_block_heat0(const Bufs& B, int cur, int slot, int at, int n, double* part, cudaStream_t s) {
    const int nch = (n + RED_CHUNK - 1) / RED_CHUNK;
    int g = nch < g_grid_cap ? nch : g_grid_cap;
    k_block_heat_chunks<<<g < 1 ? 1 : g, 256, 0, s>>>(B, cur, at, n, part);
    k_block_heat_final<<<1, 32, 0, s>>>(B, slot, n, part);
    return cudaGetLastError();
}

cudaError_t launch_adv_end(const Bufs& B, int par, cudaStream_t s) {
    k_T_update<<<grid_stride_grid(B.n, 256), 256, 0, s>>>(B, par);
    CK(launch_reduce_heat(B, par, s));
    k_adv_end_cases<<<(B.ncases + 63) / 64, 64, 0, s>>>(B);
    return cudaGetLastError();
}

cudaError_t launch_sub_cond(const Bufs& B, cudaGraphConditionalHandle h, cudaStream_t s) {
    k_sub_cond<<<1, 256, 0, s>>>(B, h);
    return cudaGetLastError();
}

void kernels_in_step(bool fp64, bool torque, int* fixed, int* per_substep) {
    // adv_begin + sort (hash, 3 scan, scatter, order, reorder, segments) + D + VT (+ overflow)
    // + T update, 2 reductions, adv_end
    *fixed = 1 + 8 + 1 + (fp64 ? 1 : 2) + 4;
    // sub_begin, half kick, M (+ overflow), C (+ overflow), torque chunks, sub_end
    *per_substep = 1 + 1 + (fp64 ? 1 : 2) + (fp64 ? 1 : 2) + (torque ? 1 : 0) + 1;
}

int kernels_per_advection_step(int kcap, bool fp64) {
    int f = 0, k = 0;
    kernels_in_step(fp64, true, &f, &k);
    return f + kcap * k;
}

cudaError_t launch_gather_field(const Bufs& B, int par, int field, int cs, int id_base, double* out,
                                cudaStream_t s) {
    k_gather_field<<<grid_stride_grid(B.n, 256), 256, 0, s>>>(B, par, field, cs, id_base, out);
    return cudaGetLastError();
}

cudaError_t launch_neighbors(const Bufs& B, int par, int cs, int id_base, int64_t* counts, const int64_t* start,
                             int32_t* list, cudaStream_t s) {
    if (!list) k_nb_count<<<grid_1to1(B.n, 128), 128, 0, s>>>(B, par, cs, id_base, counts);
    else k_nb_list<<<grid_1to1(B.n, 128), 128, 0, s>>>(B, par, cs, id_base, start, list);
    return cudaGetLastError();
}

cudaError_t launch_cell_sort(const double* pos, int n, const double origin[3], const double cellw[3],
                             const int ncell[3], uint32_t* keys, uint32_t* rank, uint32_t* cnt, uint32_t* tmp,
                             uint32_t* scanblk, int32_t* perm, int32_t* cell_start, cudaStream_t s) {
    const int ncells = ncell[0] * ncell[1] * ncell[2];
    CK(cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * (size_t)ncells, s));
    const int g = grid_stride_grid(n, 256);
    k_cs_hash<<<g, 256, 0, s>>>(pos, n, origin[0], origin[1], origin[2], cellw[0], cellw[1], cellw[2], ncell[0],
                                ncell[1], ncell[2], keys, rank, cnt);
    uint32_t* cs = reinterpret_cast<uint32_t*>(cell_start);
    CK(launch_scan(cnt, cs, scanblk, ncells, s));
    k_scatter<<<g, 256, 0, s>>>(n, keys, rank, cs, tmp);
    k_order<<<g, 256, 0, s>>>(n, keys, cs, tmp, nullptr, reinterpret_cast<uint32_t*>(perm), rank, 0xffffffffu);
    return cudaGetLastError();
}

}  // namespace sph
