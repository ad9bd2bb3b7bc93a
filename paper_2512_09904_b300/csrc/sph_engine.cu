// sph_engine.cu -- host side of the C ABI (include/sph.h): validation,
// device allocation, upload, CUDA-graph capture of one advection step, and
// read-back.  The whole advection step (neighbour search, all passes, the
// acoustic sub-step loop and the reductions) is one CUDA graph launch with no
// host synchronisation; the sub-step count is data dependent and is handled
// on the device (sub-steps past the end of the advection step are no-ops).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "sph.h"
#include "sph_kernels.cuh"

namespace sph {
void set_grid_cap(int sms);

// message of the last failed call that has no context (sph_last_error(NULL))
static thread_local std::string g_stateless_err;
void set_stateless_error(const char* msg) { g_stateless_err = msg; }
}

using namespace sph;

struct sph_ctx {
    sph_config cfg{};
    cudaStream_t stream = nullptr;
    cudaStream_t cap = nullptr;  // private stream used only to capture the step graph
    std::string err;
    sph_material mats[MAX_MAT]{};
    bool mat_set[MAX_MAT]{};
    struct {
        double c[3], a[3], omega;
        bool set;
    } bodies[MAX_BODY]{};
    // host staging, id order
    std::vector<double> pos, vel, nrm, T, rho;
    std::vector<int> kind, mat, body;
    int64_t n_fluid = 0, n_solid = 0;
    bool started = false;
    // device
    Bufs B{};
    int parity = 0;  // index of the buffers holding the current state
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    std::vector<void*> allocs;
    double* d_field = nullptr;
    int kcap = 0;
    int ncell[3]{};
    double cellw[3]{};
    double sigma0 = 0.0;
    CaseState st_h{};
    // profiling: CUDA events recorded between kernel groups inside the graph
    bool prof = false;
    std::vector<cudaEvent_t> ev;
    std::vector<int> ev_class, ev_sub;  // per interval: group class and sub-step index (-1: not a sub-step)
    double prof_ms[SPH_PROF_NCLASS]{};
    int64_t prof_cnt[SPH_PROF_NCLASS]{};
};

static sph_status fail(sph_ctx* c, sph_status s, const char* fmt, ...) {
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return s;
}

#define CUDA_OR_FAIL(ctx, call)                                                                 \
    do {                                                                                        \
        cudaError_t e__ = (call);                                                               \
        if (e__ != cudaSuccess)                                                                 \
            return fail(ctx, SPH_ECUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e__), __FILE__, \
                        __LINE__);                                                              \
    } while (0)

// Kernel sum over the exact cubic lattice (spacing dx) including the centre:
// the reference value sum W0 of Eq. (14).  Wendland C2, support 2h.
static double lattice_sigma0(double dx, double h) {
    const double a = 21.0 / (16.0 * M_PI * h * h * h);
    const int m = (int)std::ceil(2.0 * h / dx) + 1;
    double s = 0.0;
    for (int k = -m; k <= m; ++k)
        for (int j = -m; j <= m; ++j)
            for (int i = -m; i <= m; ++i) {
                const double q = dx * std::sqrt((double)(i * i + j * j + k * k)) / h;
                if (q >= 2.0) continue;
                const double t = 1.0 - 0.5 * q;
                s += a * t * t * t * t * (1.0 + 2.0 * q);
            }
    return s;
}

template <class T>
static cudaError_t dalloc(sph_ctx* c, T** p, size_t count) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, sizeof(T) * (count ? count : 1));
    if (e != cudaSuccess) return e;
    c->allocs.push_back(q);
    *p = (T*)q;
    return cudaMemsetAsync(q, 0, sizeof(T) * (count ? count : 1), c->stream);
}

extern "C" {

const char* sph_last_error(const sph_ctx* ctx) { return ctx ? ctx->err.c_str() : sph::g_stateless_err.c_str(); }

sph_status sph_create(const sph_config* cfg, void* stream, sph_ctx** out) {
    if (!cfg || !out) return SPH_EINVAL;
    *out = nullptr;
    const double h = cfg->h_over_dx * cfg->dx;
    if (!(cfg->dx > 0) || !(cfg->h_over_dx > 0) || !(cfg->c0 > 0) || !(cfg->u_ref > 0) ||
        !(cfg->cfl_ad > 0) || !(cfg->cfl_ac > 0))
        return SPH_EINVAL;
    sph_ctx* c = new sph_ctx();
    c->cfg = *cfg;
    c->stream = (cudaStream_t)stream;
    const double R = 2.0 * h;
    int64_t total = 1;
    for (int a = 0; a < 3; ++a) {
        if (!(cfg->extent[a] > 0)) {
            delete c;
            return SPH_EINVAL;
        }
        int64_t n = (int64_t)std::floor(cfg->extent[a] / R);
        if (n < 1) n = 1;
        if ((cfg->periodic_mask & (1 << a)) && n < 3) {
            delete c;
            return SPH_EINVAL;
        }
        c->ncell[a] = (int)n;
        c->cellw[a] = cfg->extent[a] / (double)n;
        total *= n;
    }
    if (total > (int64_t)1 << 30) {
        delete c;
        return SPH_EINVAL;
    }
    c->kcap = cfg->max_substeps > 0
                  ? cfg->max_substeps
                  : (int)std::ceil(cfg->cfl_ad / cfg->cfl_ac * (cfg->c0 / cfg->u_ref + 1.0)) + 2;
    c->sigma0 = lattice_sigma0(cfg->dx, h);
    c->B.tune_batch = 8;
    *out = c;
    return SPH_OK;
}

sph_status sph_destroy(sph_ctx* c) {
    if (!c) return SPH_OK;
    for (int p = 0; p < 2; ++p)
        if (c->gexec[p]) cudaGraphExecDestroy(c->gexec[p]);
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    for (auto e : c->ev) cudaEventDestroy(e);
    if (c->cap) cudaStreamDestroy(c->cap);
    for (void* p : c->allocs) cudaFree(p);
    delete c;
    return SPH_OK;
}

sph_status sph_set_material(sph_ctx* c, int id, const sph_material* m) {
    if (!c) return SPH_EINVAL;
    if (c->started) return fail(c, SPH_ESTATE, "materials are fixed after the first step");
    if (id < 0 || id >= MAX_MAT || !m) return fail(c, SPH_EINVAL, "material id %d out of range 0..%d", id, MAX_MAT - 1);
    if (!(m->rho0 > 0) || !(m->cp > 0) || m->k < 0 || m->mu < 0)
        return fail(c, SPH_EINVAL, "material %d: rho0, cp must be > 0 and k, mu >= 0", id);
    c->mats[id] = *m;
    c->mat_set[id] = true;
    return SPH_OK;
}

static sph_status add_common(sph_ctx* c, int kind, int body, int mat, int64_t n, const double* pos,
                             const double* vel, const double* nrm, const double* T, const double* rho,
                             int64_t* first_id) {
    if (!c) return SPH_EINVAL;
    if (c->started) return fail(c, SPH_ESTATE, "particles can only be added before the first step");
    if (n < 0 || (n > 0 && !pos)) return fail(c, SPH_EINVAL, "n < 0 or pos is NULL");
    if (mat < 0 || mat >= MAX_MAT || !c->mat_set[mat]) return fail(c, SPH_EINVAL, "material %d not set", mat);
    if (kind == 1 && (body < -1 || body >= MAX_BODY)) return fail(c, SPH_EINVAL, "body id %d out of range", body);
    if (kind == 1 && n > 0 && !nrm) return fail(c, SPH_EINVAL, "solid particles need normals");
    const int64_t n0 = (int64_t)c->kind.size();
    if (n0 + n > (int64_t)MAX_PARTICLES - 1) return fail(c, SPH_EINVAL, "more than 2^26 - 1 particles");
    const sph_material& M = c->mats[mat];
    for (int64_t q = 0; q < 3 * n; ++q)
        if (!std::isfinite(pos[q])) return fail(c, SPH_EINVAL, "non-finite position");
    if (first_id) *first_id = n0;
    for (int64_t q = 0; q < n; ++q) {
        for (int a = 0; a < 3; ++a) {
            double p = pos[3 * q + a];
            c->pos.push_back(p);
            c->vel.push_back(vel ? vel[3 * q + a] : 0.0);
            c->nrm.push_back(nrm ? nrm[3 * q + a] : 0.0);
        }
        c->T.push_back(T ? T[q] : M.T_init);
        c->rho.push_back(rho && std::isfinite(rho[q]) ? rho[q] : M.rho0);
        c->kind.push_back(kind);
        c->mat.push_back(mat);
        c->body.push_back(kind == 0 ? -1 : body);
    }
    if (kind == 0) c->n_fluid += n;
    else c->n_solid += n;
    return SPH_OK;
}

sph_status sph_add_fluid(sph_ctx* c, int mat, int64_t n, const double* pos, const double* vel, const double* T,
                         const double* rho, int64_t* first_id) {
    return add_common(c, 0, -1, mat, n, pos, vel, nullptr, T, rho, first_id);
}

sph_status sph_add_solid(sph_ctx* c, int body, int mat, int64_t n, const double* pos, const double* normal,
                         const double* T, int64_t* first_id) {
    return add_common(c, 1, body, mat, n, pos, nullptr, normal, T, nullptr, first_id);
}

sph_status sph_set_rotation(sph_ctx* c, int b, const double center[3], const double axis[3], double omega) {
    if (!c) return SPH_EINVAL;
    if (c->started) return fail(c, SPH_ESTATE, "rotation is fixed after the first step");
    if (b < 0 || b >= MAX_BODY || !center || !axis) return fail(c, SPH_EINVAL, "body id %d out of range", b);
    const double L = std::sqrt(axis[0] * axis[0] + axis[1] * axis[1] + axis[2] * axis[2]);
    if (std::fabs(L - 1.0) > 1e-9 || !std::isfinite(omega)) return fail(c, SPH_EINVAL, "axis must be a unit vector");
    for (int a = 0; a < 3; ++a) {
        c->bodies[b].c[a] = center[a];
        c->bodies[b].a[a] = axis[a];
    }
    c->bodies[b].omega = omega;
    c->bodies[b].set = true;
    return SPH_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ upload --
static sph_status build_case(sph_ctx* c, CaseDev& C) {
    const sph_config& F = c->cfg;
    memset(&C, 0, sizeof C);
    const double h = F.h_over_dx * F.dx;
    const double R2 = (2.0 * h) * (2.0 * h);
    for (int a = 0; a < 3; ++a) {
        C.origin[a] = F.origin[a];
        C.ext[a] = F.extent[a];
        C.cellw[a] = c->cellw[a];
        C.cellwf[a] = (float)c->cellw[a];
        C.ncell[a] = c->ncell[a];
        C.g[a] = (float)F.gravity[a];
    }
    C.cell_base = 0;
    C.ncells = c->ncell[0] * c->ncell[1] * c->ncell[2];
    C.periodic = F.periodic_mask;
    C.R2 = R2;
    // FP32 guard band around the cut-off: inside it the FP64 rule decides
    C.R2lo = (float)(R2 * (1.0 - 1e-4));
    C.R2hi = (float)(R2 * (1.0 + 1e-4));
    C.R2eps = (float)(R2 * 1e-4);
    C.h = (float)h;
    C.inv_h = (float)(1.0 / h);
    const double alpha = 21.0 / (16.0 * M_PI * h * h * h);
    C.kw = (float)alpha;
    C.kdw = (float)(-5.0 * alpha / h);
    C.w0 = (float)alpha;
    C.inv_sigma0 = (float)(1.0 / c->sigma0);
    C.vol = (float)(F.dx * F.dx * F.dx);
    C.c0 = (float)F.c0;
    C.c02 = (float)(F.c0 * F.c0);
    C.inv_c0 = (float)(1.0 / F.c0);
    C.inv_c02 = (float)(1.0 / (F.c0 * F.c0));
    C.h64 = h;
    C.c0_64 = F.c0;
    C.u_ref = F.u_ref;
    C.cfl_ad = F.cfl_ad;
    C.cfl_ac = F.cfl_ac;
    C.free_surface = F.free_surface;
    C.kcap = c->kcap;
    double nu = 0.0, Tref = 0.0;
    int nfl = 0;
    for (size_t i = 0; i < c->kind.size(); ++i)
        if (c->kind[i] == 0) {
            const sph_material& M = c->mats[c->mat[i]];
            nu = std::max(nu, M.mu / M.rho0);
            if (nfl++ == 0) Tref = c->T[i];
        }
    if (nfl == 0 && !c->T.empty()) Tref = c->T[0];
    C.nu_max = nu;
    C.T_ref = Tref;
    for (int m = 0; m < MAX_MAT; ++m) {
        const sph_material& M = c->mats[m];
        if (!c->mat_set[m]) continue;
        C.mat[m].rho0 = (float)M.rho0;
        C.mat[m].mass = (float)(M.rho0 * F.dx * F.dx * F.dx);
        C.mat[m].mu = (float)M.mu;
        C.mat[m].k = (float)M.k;
        C.mat[m].cp = (float)M.cp;
        C.mat[m].inv_rho0_cp = (float)(1.0 / (M.rho0 * M.cp));
        C.mat[m].fixed_T = M.fixed_T;
    }
    int nb = 0;
    for (int b = 0; b < MAX_BODY; ++b) {
        BodyDev& Bd = C.body[b];
        Bd.id_lo = 0;
        Bd.id_hi = 0;
        if (!c->bodies[b].set) continue;
        nb = b + 1;
        Bd.set = 1;
        for (int a = 0; a < 3; ++a) {
            Bd.c[a] = c->bodies[b].c[a];
            Bd.axis[a] = c->bodies[b].a[a];
        }
        Bd.omega = c->bodies[b].omega;
        int lo = -1, hi = -1;
        for (size_t i = 0; i < c->kind.size(); ++i)
            if (c->kind[i] == 1 && c->body[i] == b) {
                if (lo < 0) lo = (int)i;
                hi = (int)i + 1;
            }
        Bd.id_lo = lo < 0 ? 0 : lo;
        Bd.id_hi = hi < 0 ? 0 : hi;
    }
    C.n_body = nb;
    return SPH_OK;
}

// Event k+1 closes interval k; intervals carry a group class (sph.h
// SPH_PROF_*) and the acoustic sub-step index they belong to.
static cudaError_t mark(sph_ctx* c, int cls, int sub) {
    if (!c->prof) return cudaSuccess;
    const size_t k = c->ev_class.size() + 1;
    if (k >= c->ev.size()) return cudaErrorInvalidValue;
    c->ev_class.push_back(cls);
    c->ev_sub.push_back(sub);
    return cudaEventRecordWithFlags(c->ev[k], c->cap, cudaEventRecordExternal);
}

static sph_status capture(sph_ctx* c) {
    for (int p = 0; p < 2; ++p) {
        if (c->gexec[p]) {
            cudaGraphExecDestroy(c->gexec[p]);
            c->gexec[p] = nullptr;
        }
    }
    // capture runs nothing; it needs a stream other than the legacy default one
    if (!c->cap) CUDA_OR_FAIL(c, cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking));
    if (c->prof && c->ev.empty()) {
        c->ev.resize(8 + 4 * (size_t)c->kcap + 8);
        for (auto& e : c->ev) CUDA_OR_FAIL(c, cudaEventCreate(&e));
    }
    for (int p = 0; p < 2; ++p) {
        cudaGraph_t g = nullptr;
        c->ev_class.clear();
        c->ev_sub.clear();
        CUDA_OR_FAIL(c, cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = c->prof ? cudaEventRecordWithFlags(c->ev[0], c->cap, cudaEventRecordExternal) : cudaSuccess;
        if (e == cudaSuccess) e = launch_adv_begin(c->B, c->cap);
        if (e == cudaSuccess) e = launch_sort(c->B, p, c->cap);
        if (e == cudaSuccess) e = mark(c, SPH_PROF_SORT, -1);
        if (e == cudaSuccess) e = launch_passD(c->B, p, c->cap);
        if (e == cudaSuccess) e = mark(c, SPH_PROF_PASS_D, -1);
        if (e == cudaSuccess) e = launch_passVT(c->B, p, c->cap);
        if (e == cudaSuccess) e = mark(c, SPH_PROF_PASS_VT, -1);
        for (int k = 0; k < c->kcap && e == cudaSuccess; ++k) {
            e = launch_sub_begin(c->B, c->cap);
            if (e == cudaSuccess) e = mark(c, SPH_PROF_CONTROL, k);
            if (e == cudaSuccess) e = launch_passM(c->B, p, k == 0, c->cap);
            if (e == cudaSuccess) e = mark(c, SPH_PROF_PASS_M, k);
            if (e == cudaSuccess) e = launch_passC(c->B, p, c->cap);
            if (e == cudaSuccess) e = mark(c, SPH_PROF_PASS_C, k);
            if (e == cudaSuccess) e = launch_sub_end(c->B, c->cap);
            if (e == cudaSuccess) e = mark(c, SPH_PROF_CONTROL, k);
        }
        if (e == cudaSuccess) e = launch_adv_end(c->B, p, c->cap);
        if (e == cudaSuccess) e = mark(c, SPH_PROF_ADV_END, -1);
        cudaError_t e2 = cudaStreamEndCapture(c->cap, &g);
        if (e != cudaSuccess || e2 != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return fail(c, SPH_ECUDA, "graph capture failed: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
        }
        e = cudaGraphInstantiate(&c->gexec[p], g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return fail(c, SPH_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
    }
    return SPH_OK;
}

static sph_status upload(sph_ctx* c) {
    const int64_t n = (int64_t)c->kind.size();
    if (n == 0) return fail(c, SPH_ESTATE, "no particles");
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    set_grid_cap(sms);
    CaseDev C;
    build_case(c, C);
    Bufs& B = c->B;
    B.n = (int)n;
    B.ncases = 1;
    B.ncells = C.ncells;
    B.max_chunks = (int)((n + RED_CHUNK - 1) / RED_CHUNK) + B.ncases + 1;
    B.hist_cap = 4096;
    cudaError_t e = cudaSuccess;
#define AL(p, cnt) \
    if (e == cudaSuccess) e = dalloc(c, &(p), (size_t)(cnt))
    AL(B.cases, 1);
    AL(B.st, 1);
    for (int a = 0; a < 3; ++a) {
        AL(B.X[a], n);
        AL(B.Y[a], n);
        AL(B.RP[a], n);
    }
    for (int p = 0; p < 2; ++p) {
        AL(B.V[p], n);
        AL(B.DR[p], n);
        AL(B.T64[p], n);
        AL(B.ID[p], n);
        AL(B.TAG[p], n);
    }
    AL(B.T32, n);
    AL(B.SNAP, n);
    AL(B.CELLK, n);
    AL(B.AV, n);
    AL(B.NRM, n);
    AL(B.RN, n);
    AL(B.TORQ, n);
    AL(B.TORQV, n);
    AL(B.KEYS, n);
    AL(B.RANK, n);
    AL(B.TMP, n);
    AL(B.PERM, n);
    AL(B.CNT, B.ncells);
    AL(B.CSTART, (size_t)B.ncells + 1);
    AL(B.SCANBLK, scan_blocks(B.ncells) + 1);
    AL(B.PART, (size_t)3 * B.max_chunks);
    AL(B.CHUNK_CASE, B.max_chunks);
    AL(B.HIST, (size_t)8 * B.hist_cap * B.ncases);
    AL(c->d_field, (size_t)3 * n);
    AL(B.NB, (size_t)NB_CAP * n);
    AL(B.NBC, n);
    AL(B.OVFL, n);
    AL(B.novf, 1);
    AL(B.VH, n);
    B.nb_stride = (int)n;
    {
        int fm = -1;
        bool uni = true;
        for (size_t i = 0; i < c->kind.size(); ++i)
            if (c->kind[i] == 0) {
                if (fm < 0) fm = c->mat[i];
                else if (c->mat[i] != fm) uni = false;
            }
        B.uni_fluid = uni ? 1 : 0;
    }
#undef AL
    if (e != cudaSuccess) return fail(c, e == cudaErrorMemoryAllocation ? SPH_ENOMEM : SPH_ECUDA,
                                      "device allocation: %s", cudaGetErrorString(e));
    // host images in id order
    std::vector<double> xs[3], rp[3];
    std::vector<float4> v(n), rn(n);
    std::vector<int> ids(n);
    std::vector<uint32_t> tags(n);
    for (int a = 0; a < 3; ++a) {
        xs[a].resize(n);
        rp[a].resize(n);
    }
    for (int64_t i = 0; i < n; ++i) {
        const int k = c->kind[i], m = c->mat[i], b = c->body[i];
        uint32_t kind = k == 0 ? KIND_FLUID : ((b >= 0 && c->bodies[b].set) ? KIND_ROT : KIND_STATIC);
        tags[i] = make_tag((uint32_t)m, kind, kind == KIND_ROT ? (uint32_t)b : 0u, 0u);
        ids[i] = (int)i;
        for (int a = 0; a < 3; ++a) {
            xs[a][i] = c->pos[3 * i + a];
            rp[a][i] = c->pos[3 * i + a];
        }
        if (k == 0)
            v[i] = make_float4((float)c->vel[3 * i], (float)c->vel[3 * i + 1], (float)c->vel[3 * i + 2],
                               (float)(c->rho[i] - c->mats[m].rho0));
        else
            v[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        rn[i] = make_float4((float)c->nrm[3 * i], (float)c->nrm[3 * i + 1], (float)c->nrm[3 * i + 2], 0.f);
    }
    CaseState S;
    memset(&S, 0, sizeof S);
    cudaStream_t s = c->stream;
    CUDA_OR_FAIL(c, cudaMemcpyAsync(B.cases, &C, sizeof C, cudaMemcpyHostToDevice, s));
    CUDA_OR_FAIL(c, cudaMemcpyAsync(B.st, &S, sizeof S, cudaMemcpyHostToDevice, s));
    for (int a = 0; a < 3; ++a) {
        CUDA_OR_FAIL(c, cudaMemcpyAsync(B.X[a], xs[a].data(), sizeof(double) * n, cudaMemcpyHostToDevice, s));
        CUDA_OR_FAIL(c, cudaMemcpyAsync(B.RP[a], rp[a].data(), sizeof(double) * n, cudaMemcpyHostToDevice, s));
    }
    CUDA_OR_FAIL(c, cudaMemcpyAsync(B.V[0], v.data(), sizeof(float4) * n, cudaMemcpyHostToDevice, s));
    CUDA_OR_FAIL(c, cudaMemcpyAsync(B.RN, rn.data(), sizeof(float4) * n, cudaMemcpyHostToDevice, s));
    CUDA_OR_FAIL(c, cudaMemcpyAsync(B.T64[0], c->T.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s));
    CUDA_OR_FAIL(c, cudaMemcpyAsync(B.ID[0], ids.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s));
    CUDA_OR_FAIL(c, cudaMemcpyAsync(B.TAG[0], tags.data(), sizeof(uint32_t) * n, cudaMemcpyHostToDevice, s));
    // initial speed, rotation at t = 0, first cell sort, reference heat content
    CUDA_OR_FAIL(c, launch_vmax_init(B, 0, s));
    CUDA_OR_FAIL(c, launch_adv_begin(B, s));
    CUDA_OR_FAIL(c, launch_sort(B, 0, s));
    CUDA_OR_FAIL(c, launch_init_heat0(B, s));
    for (int a = 0; a < 3; ++a)
        CUDA_OR_FAIL(c, cudaMemcpyAsync(B.X[a], B.Y[a], sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    c->parity = 1;
    CUDA_OR_FAIL(c, cudaStreamSynchronize(s));
    sph_status rs = capture(c);
    if (rs != SPH_OK) return rs;
    c->started = true;
    // host staging is no longer needed
    std::vector<double>().swap(c->vel);
    std::vector<double>().swap(c->rho);
    return SPH_OK;
}

static sph_status pull_state(sph_ctx* c) {
    CUDA_OR_FAIL(c, cudaMemcpyAsync(&c->st_h, c->B.st, sizeof(CaseState), cudaMemcpyDeviceToHost, c->stream));
    CUDA_OR_FAIL(c, cudaStreamSynchronize(c->stream));
    return SPH_OK;
}

extern "C" {

sph_status sph_step(sph_ctx* c, int n_steps, double* t_out) {
    if (!c) return SPH_EINVAL;
    if (n_steps < 0) return fail(c, SPH_EINVAL, "n_steps < 0");
    if (!c->started) {
        sph_status s = upload(c);
        if (s != SPH_OK) return s;
    }
    for (int k = 0; k < n_steps; ++k) {
        CUDA_OR_FAIL(c, cudaGraphLaunch(c->gexec[c->parity], c->stream));
        c->parity ^= 1;
        if (c->prof) {
            sph_status s = pull_state(c);
            if (s != SPH_OK) return s;
            const int nsub = c->st_h.last_nsub;
            for (size_t q = 0; q < c->ev_class.size(); ++q) {
                float ms = 0.f;
                CUDA_OR_FAIL(c, cudaEventElapsedTime(&ms, c->ev[q], c->ev[q + 1]));
                const int cls = (c->ev_sub[q] >= nsub) ? SPH_PROF_IDLE : c->ev_class[q];
                c->prof_ms[cls] += ms;
                c->prof_cnt[cls] += 1;
            }
        }
    }
    sph_status s = pull_state(c);
    if (s != SPH_OK) return s;
    if (t_out) *t_out = c->st_h.t;
    if (c->st_h.err)
        return fail(c, SPH_EUNSTABLE, "unstable state (error bits 0x%x: 1 = NaN/Inf, 2 = fluid left the box)",
                    c->st_h.err);
    return SPH_OK;
}

sph_status sph_read_torque_heat(sph_ctx* c, int b, double* tq, double* tq_avg, double* heat, double* meanT) {
    if (!c) return SPH_EINVAL;
    if (!c->started) return fail(c, SPH_ESTATE, "no step taken yet");
    if (b < 0 || b >= MAX_BODY) return fail(c, SPH_EINVAL, "body id %d out of range", b);
    sph_status s = pull_state(c);
    if (s != SPH_OK) return s;
    const CaseState& S = c->st_h;
    if (tq) *tq = S.tq_inst[b];
    if (tq_avg) *tq_avg = S.time_int > 0 ? S.tq_int[b] / S.time_int : 0.0;
    if (heat) *heat = S.heat;
    if (meanT) *meanT = S.mean_T;
    return SPH_OK;
}

sph_status sph_read_fields(sph_ctx* c, int field, void* dst, int64_t n) {
    if (!c) return SPH_EINVAL;
    if (!c->started) return fail(c, SPH_ESTATE, "no step taken yet");
    if (!dst || n != (int64_t)c->B.n) return fail(c, SPH_EINVAL, "n must equal the particle count %d", c->B.n);
    int k;
    switch (field) {
    case SPH_FIELD_POS: case SPH_FIELD_VEL: case SPH_FIELD_AVISC: case SPH_FIELD_NORMAL: k = 3; break;
    case SPH_FIELD_RHO: case SPH_FIELD_P: case SPH_FIELD_T: case SPH_FIELD_DRHO: case SPH_FIELD_DTDT: k = 1; break;
    default: return fail(c, SPH_EINVAL, "unknown field %d", field);
    }
    CUDA_OR_FAIL(c, launch_gather_field(c->B, c->parity ^ 1, field, c->d_field, c->stream));
    CUDA_OR_FAIL(c, cudaMemcpyAsync(dst, c->d_field, sizeof(double) * k * n, cudaMemcpyDeviceToHost, c->stream));
    CUDA_OR_FAIL(c, cudaStreamSynchronize(c->stream));
    return SPH_OK;
}

sph_status sph_read_neighbors(sph_ctx* c, int64_t* counts, int32_t* ids, int64_t cap, int64_t* total) {
    if (!c) return SPH_EINVAL;
    if (!c->started) return fail(c, SPH_ESTATE, "no step taken yet");
    if (!counts) return fail(c, SPH_EINVAL, "counts is NULL");
    const int64_t n = c->B.n;
    int64_t* d_cnt = nullptr;
    CUDA_OR_FAIL(c, cudaMalloc(&d_cnt, sizeof(int64_t) * (n + 1)));
    cudaError_t e = launch_neighbors(c->B, c->parity ^ 1, d_cnt, nullptr, nullptr, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(counts, d_cnt, sizeof(int64_t) * n, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        cudaFree(d_cnt);
        return fail(c, SPH_ECUDA, "neighbour count: %s", cudaGetErrorString(e));
    }
    std::vector<int64_t> start(n + 1, 0);
    for (int64_t i = 0; i < n; ++i) start[i + 1] = start[i] + counts[i];
    if (total) *total = start[n];
    if (!ids) {
        cudaFree(d_cnt);
        return SPH_OK;
    }
    if (cap < start[n]) {
        cudaFree(d_cnt);
        return fail(c, SPH_EINVAL, "cap %lld < %lld pair entries", (long long)cap, (long long)start[n]);
    }
    int32_t* d_list = nullptr;
    e = cudaMalloc(&d_list, sizeof(int32_t) * (start[n] + 1));
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_cnt, start.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = launch_neighbors(c->B, c->parity ^ 1, nullptr, d_cnt, d_list, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ids, d_list, sizeof(int32_t) * start[n], cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(d_list);
    cudaFree(d_cnt);
    if (e != cudaSuccess) return fail(c, SPH_ECUDA, "neighbour list: %s", cudaGetErrorString(e));
    for (int64_t i = 0; i < n; ++i) std::sort(ids + start[i], ids + start[i + 1]);
    return SPH_OK;
}

sph_status sph_read_cell_order(sph_ctx* c, int64_t* perm, int64_t n) {
    if (!c) return SPH_EINVAL;
    if (!c->started) return fail(c, SPH_ESTATE, "no step taken yet");
    if (!perm || n != (int64_t)c->B.n) return fail(c, SPH_EINVAL, "n must equal the particle count");
    std::vector<int> ids(n);
    CUDA_OR_FAIL(c, cudaMemcpyAsync(ids.data(), c->B.ID[c->parity], sizeof(int) * n, cudaMemcpyDeviceToHost, c->stream));
    CUDA_OR_FAIL(c, cudaStreamSynchronize(c->stream));
    for (int64_t k = 0; k < n; ++k) perm[k] = ids[k];
    return SPH_OK;
}

sph_status sph_get_info(sph_ctx* c, sph_info* info) {
    if (!c || !info) return SPH_EINVAL;
    memset(info, 0, sizeof *info);
    info->n_fluid = c->n_fluid;
    info->n_solid = c->n_solid;
    info->kcap = c->kcap;
    for (int a = 0; a < 3; ++a) {
        info->ncell[a] = c->ncell[a];
        info->cell_width[a] = c->cellw[a];
    }
    info->graph_launches = kernels_per_advection_step(c->kcap);
    if (c->started) {
        sph_status s = pull_state(c);
        if (s != SPH_OK) return s;
        info->t = c->st_h.t;
        info->adv_steps = c->st_h.adv_steps;
        info->substeps = c->st_h.substeps;
        info->last_dt_ad = c->st_h.last_dt_ad;
        info->last_nsub = c->st_h.last_nsub;
        info->error_bits = c->st_h.err;
    }
    return SPH_OK;
}

sph_status sph_pair_stats(sph_ctx* c, int64_t* fluid_fluid, int64_t* fluid_wall) {
    if (!c || !fluid_fluid || !fluid_wall) return SPH_EINVAL;
    if (!c->started) return fail(c, SPH_ESTATE, "no step taken yet");
    unsigned long long* d = nullptr;
    unsigned long long h[2] = {0, 0};
    CUDA_OR_FAIL(c, cudaMalloc(&d, sizeof h));
    cudaError_t e = cudaMemsetAsync(d, 0, sizeof h, c->stream);
    if (e == cudaSuccess) e = launch_pair_stats(c->B, d, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, d, sizeof h, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(d);
    if (e != cudaSuccess) return fail(c, SPH_ECUDA, "pair stats: %s", cudaGetErrorString(e));
    *fluid_fluid = (int64_t)h[0];
    *fluid_wall = (int64_t)h[1];
    return SPH_OK;
}

sph_status sph_set_tuning(sph_ctx* c, int key, int value) {
    if (!c) return SPH_EINVAL;
    switch (key) {
    case SPH_TUNE_LIST_BATCH:
        if (value != 1 && value != 2 && value != 4 && value != 8)
            return fail(c, SPH_EINVAL, "list batch must be 1, 2, 4 or 8");
        c->B.tune_batch = value;
        break;
    default: return fail(c, SPH_EINVAL, "unknown tuning key %d", key);
    }
    if (!c->started) return SPH_OK;
    CUDA_OR_FAIL(c, cudaStreamSynchronize(c->stream));
    return capture(c);
}

sph_status sph_get_tuning(sph_ctx* c, int key, int* value) {
    if (!c || !value) return SPH_EINVAL;
    switch (key) {
    case SPH_TUNE_LIST_BATCH: *value = c->B.tune_batch; return SPH_OK;
    default: return fail(c, SPH_EINVAL, "unknown tuning key %d", key);
    }
}

sph_status sph_profile(sph_ctx* c, int enable) {
    if (!c) return SPH_EINVAL;
    c->prof = enable != 0;
    for (int k = 0; k < SPH_PROF_NCLASS; ++k) {
        c->prof_ms[k] = 0.0;
        c->prof_cnt[k] = 0;
    }
    if (!c->started) return SPH_OK;
    CUDA_OR_FAIL(c, cudaStreamSynchronize(c->stream));
    return capture(c);
}

sph_status sph_profile_read(sph_ctx* c, double* ms, int64_t* launches, int reset) {
    if (!c || !ms || !launches) return SPH_EINVAL;
    for (int k = 0; k < SPH_PROF_NCLASS; ++k) {
        ms[k] = c->prof_ms[k];
        launches[k] = c->prof_cnt[k];
        if (reset) {
            c->prof_ms[k] = 0.0;
            c->prof_cnt[k] = 0;
        }
    }
    return SPH_OK;
}

sph_status sph_cell_sort(const double* pos, int64_t n, const double origin[3], const double cellw[3],
                         const int ncell[3], int32_t* perm, int32_t* cell_start, void* stream) {
    if (n < 0 || (n > 0 && (!pos || !perm)) || !origin || !cellw || !ncell || !cell_start) return SPH_EINVAL;
    if (n > ((int64_t)1 << 31) - 1) return SPH_EINVAL;
    int64_t nc = 1;
    for (int a = 0; a < 3; ++a) {
        if (ncell[a] < 1 || !(cellw[a] > 0)) return SPH_EINVAL;
        nc *= ncell[a];
    }
    if (nc > ((int64_t)1 << 30)) return SPH_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t nb = scan_blocks((int)nc) + 1;
    const size_t bytes = sizeof(uint32_t) * ((size_t)3 * (n > 0 ? n : 1) + (size_t)nc + nb);
    void* scratch = nullptr;
    if (cudaMallocAsync(&scratch, bytes, s) != cudaSuccess) return SPH_ENOMEM;
    uint32_t* keys = (uint32_t*)scratch;
    uint32_t* rank = keys + (n > 0 ? n : 1);
    uint32_t* tmp = rank + (n > 0 ? n : 1);
    uint32_t* cnt = tmp + (n > 0 ? n : 1);
    uint32_t* blk = cnt + nc;
    cudaError_t e = launch_cell_sort(pos, (int)n, origin, cellw, ncell, keys, rank, cnt, tmp, blk, perm,
                                     cell_start, s);
    cudaError_t e2 = cudaFreeAsync(scratch, s);
    if (e != cudaSuccess || e2 != cudaSuccess) return SPH_ECUDA;
    return SPH_OK;
}

}  // extern "C"
