// sph_engine.cu -- host side of the C ABI (include/sph.h).
//
// One Engine owns the device arrays of a packed particle array holding any
// number of resident cases (a single-case context is an Engine with one
// case).  A case occupies a contiguous segment of the array after every cell
// sort, its own range of the cell index space and of the particle id space,
// and one slot of the per-case parameter/state tables.  Admission appends the
// case's particles and re-sorts; retirement marks the case dead so the next
// sort carries its particles past the live ones, where they are dropped.
//
// The whole advection step (neighbour search, all passes, the acoustic
// sub-step loop and the reductions) of all resident cases is one CUDA graph
// launch with no host synchronisation; each case's data-dependent sub-step
// count is handled on the device (its sub-step slots past the end of its
// advection step are no-ops).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <sys/mman.h>

#include "sph.h"
#include "sph_kernels.cuh"

namespace sph {
void set_grid_cap(int sms);

// message of the last failed call that has no context (sph_last_error(NULL))
static thread_local std::string g_stateless_err;
void set_stateless_error(const char* msg) { g_stateless_err = msg; }
}  // namespace sph

using namespace sph;

namespace {

std::string vformat(const char* fmt, va_list ap) {
    char buf[512];
    vsnprintf(buf, sizeof buf, fmt, ap);
    return buf;
}

// First-fit allocator of [start, start+len) ranges in [0, cap).
struct RangeAlloc {
    std::vector<std::pair<int64_t, int64_t>> free_;  // (start, len), sorted by start
    void reset(int64_t cap) { free_.assign(1, {0, cap}); }
    bool alloc(int64_t len, int64_t* start) {
        if (len == 0) {
            *start = 0;
            return true;
        }
        for (size_t k = 0; k < free_.size(); ++k)
            if (free_[k].second >= len) {
                *start = free_[k].first;
                free_[k].first += len;
                free_[k].second -= len;
                if (free_[k].second == 0) free_.erase(free_.begin() + (long)k);
                return true;
            }
        return false;
    }
    void release(int64_t start, int64_t len) {
        if (len == 0) return;
        auto it = std::lower_bound(free_.begin(), free_.end(), std::make_pair(start, (int64_t)0));
        it = free_.insert(it, {start, len});
        size_t k = (size_t)(it - free_.begin());
        if (k + 1 < free_.size() && free_[k].first + free_[k].second == free_[k + 1].first) {
            free_[k].second += free_[k + 1].second;
            free_.erase(free_.begin() + (long)k + 1);
        }
        if (k > 0 && free_[k - 1].first + free_[k - 1].second == free_[k].first) {
            free_[k - 1].second += free_[k].second;
            free_.erase(free_.begin() + (long)k);
        }
    }
};

// Kernel sum over the exact cubic lattice (spacing dx) including the centre:
// the reference value sum W0 of Eq. (14).  Wendland C2, support 2h.
double lattice_sigma0(double dx, double h) {
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

struct HostCase {
    bool used = false, retiring = false, pending = false;
    bool dead = false;  // flagged dead on the device; compacted away by the next step's sort
    int64_t n = 0, n_fluid = 0, n_solid = 0;
    int64_t id_base = 0, cell_base = 0, ncells = 0;
    int kcap = 0;
    int ncell[3] = {0, 0, 0};
    double cellw[3] = {0, 0, 0};
    int64_t steps_req = 0;
    int body_lo[MAX_BODY] = {0, 0, 0, 0}, body_hi[MAX_BODY] = {0, 0, 0, 0};  // rigid-body id ranges
    bool visc_heat = false;
};

// device bytes per particle slot and per cell of an engine
constexpr int64_t kBytesPerParticle =
    3 * 8 * 2 /*X,Y*/ + 3 * 8 /*RP*/ + 16 * 2 /*V*/ + 4 * 2 /*DR*/ + 8 * 2 /*T64*/ + 4 * 2 /*ID*/ + 4 * 2 /*TAG*/ +
    4 /*T32*/ + 16 /*SNAP*/ + 4 /*CELLK*/ + 16 /*AV*/ + 16 /*NRM*/ + 16 /*RN*/ + 4 * 2 /*TORQ*/ + 8 /*CF*/ + 4 * 4 /*sort*/ +
    4 * NB_CAP /*NB*/ + 4 /*NBC*/ + 4 /*OVFL*/ + 16 /*VH*/ + 3 * 8 /*field*/ + 1 /*PART*/;
constexpr int64_t kBytesPerCell = 4 * 2 + 1;

}  // namespace

struct Engine {
    cudaStream_t stream = nullptr;
    cudaStream_t cap = nullptr;  // private stream used only to capture the step graph
    cudaStream_t cap2 = nullptr; // ... and the body of its sub-step loop
    std::string err;
    int64_t n_cap = 0, cells_cap = 0;
    int c_cap = 0, hist_cap = 0;
    bool allocated = false;
    Bufs B{};
    int parity = 0;  // index of the buffers holding the current state
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    bool graph_dirty = true;
    int kcap_max = 0;
    std::vector<void*> allocs;
    double* d_field = nullptr;
    std::vector<HostCase> cases;
    std::vector<CaseState> st_h;
    std::vector<CaseDev> cdev_h;  // host copies of the case table
    PairTab tab{};                // pair constants of the resident cases, passed to the pair passes
    RangeAlloc ids, cells;
    bool need_prepare = false;
    int64_t graph_steps = 0;  // advection steps launched so far
    int tq_cap = 0;           // capacity of the torque chunk table
    int64_t graph_instantiations = 0, graph_updates = 0;
    // profiling: CUDA events recorded between kernel groups inside the graph
    bool prof = false;
    std::vector<cudaEvent_t> ev;
    std::vector<int> ev_class, ev_sub;  // per interval: group class and sub-step index (-1: not a sub-step)
    double prof_ms[SPH_PROF_NCLASS]{};
    int64_t prof_cnt[SPH_PROF_NCLASS]{};

    sph_status fail(sph_status s, const char* fmt, ...) {
        va_list ap;
        va_start(ap, fmt);
        err = vformat(fmt, ap);
        va_end(ap);
        return s;
    }
    ~Engine() {
        for (int p = 0; p < 2; ++p)
            if (gexec[p]) cudaGraphExecDestroy(gexec[p]);
        if (allocated) cudaStreamSynchronize(stream);
        for (auto e : ev) cudaEventDestroy(e);
        if (cap) cudaStreamDestroy(cap);
        if (cap2) cudaStreamDestroy(cap2);
        for (void* p : allocs) cudaFree(p);
    }
};

#define E_CUDA(E, call)                                                                                      \
    do {                                                                                                     \
        cudaError_t e__ = (call);                                                                            \
        if (e__ != cudaSuccess)                                                                              \
            return (E).fail(SPH_ECUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e__), __FILE__, __LINE__); \
    } while (0)

// Page-locked host blocks for staging large particle arrays, kept by the
// process and handed from one context to the next: a staged array in such a
// block goes to the device at full DMA rate with no page-locking at admission
// (locking a large array page by page costs more than its copy).  Blocks are
// 2 MB multiples; at most kPinnedCap bytes are ever locked, beyond which (or
// where the runtime refuses, e.g. without a GPU) arrays fall back to
// ordinary host memory.
class PinnedPool {
  public:
    static PinnedPool& get() {
        static PinnedPool* p = new PinnedPool();  // never destroyed: blocks live until exit
        return *p;
    }
    // a block of at least `bytes` (its size in *cap), or nullptr
    void* take(size_t bytes, size_t* cap) {
        const size_t sz = round_up(bytes);
        std::lock_guard<std::mutex> lock(mu_);
        auto it = free_.lower_bound(sz);
        if (it != free_.end() && it->first <= 2 * sz) {
            void* p = it->second;
            *cap = it->first;
            free_.erase(it);
            return p;
        }
        if (disabled_ || locked_ + sz > kPinnedCap) return nullptr;
        void* p = nullptr;
        if (cudaHostAlloc(&p, sz, cudaHostAllocPortable) != cudaSuccess) {
            (void)cudaGetLastError();
            disabled_ = true;  // no device, or locked memory refused: stay with ordinary memory
            return nullptr;
        }
        locked_ += sz;
        *cap = sz;
        return p;
    }
    void give(void* p, size_t cap) {
        std::lock_guard<std::mutex> lock(mu_);
        free_.emplace(cap, p);
    }

  private:
    static constexpr size_t kBlock = (size_t)2 << 20;
    static constexpr size_t kPinnedCap = (size_t)8 << 30;
    static size_t round_up(size_t b) { return (b + kBlock - 1) / kBlock * kBlock; }
    std::mutex mu_;
    std::multimap<size_t, void*> free_;
    size_t locked_ = 0;
    bool disabled_ = false;
};

// Host staging array of doubles.  Arrays of 2 MB and more come from the
// page-locked pool when it can serve them, else sit on transparent huge pages
// where the kernel offers them (a 50 MB block then takes tens of page faults
// to fill instead of thousands).
class HostArray {
  public:
    HostArray() = default;
    HostArray(const HostArray&) = delete;
    HostArray& operator=(const HostArray&) = delete;
    HostArray(HostArray&& o) noexcept : p_(o.p_), n_(o.n_), pinned_cap_(o.pinned_cap_) {
        o.p_ = nullptr, o.n_ = 0, o.pinned_cap_ = 0;
    }
    HostArray& operator=(HostArray&& o) noexcept {
        if (this != &o) {
            release();
            p_ = o.p_, n_ = o.n_, pinned_cap_ = o.pinned_cap_;
            o.p_ = nullptr, o.n_ = 0, o.pinned_cap_ = 0;
        }
        return *this;
    }
    ~HostArray() { release(); }
    bool alloc(size_t n) {
        release();
        if (n == 0) return true;
        const size_t huge = (size_t)2 << 20, bytes = n * sizeof(double);
        if (bytes >= huge) {
            size_t cap = 0;
            p_ = (double*)PinnedPool::get().take(bytes, &cap);
            if (p_) {
                pinned_cap_ = cap;
            } else {
                p_ = (double*)std::aligned_alloc(huge, (bytes + huge - 1) / huge * huge);
                if (p_) madvise(p_, bytes, MADV_HUGEPAGE);  // advice only: failure is harmless
            }
        } else {
            p_ = (double*)std::malloc(bytes);
        }
        if (p_) n_ = n;
        return p_ != nullptr;
    }
    size_t size() const { return n_; }
    bool empty() const { return n_ == 0; }
    bool pinned() const { return pinned_cap_ != 0; }
    double* data() { return p_; }
    const double* data() const { return p_; }
    const double& operator[](size_t i) const { return p_[i]; }

  private:
    void release() {
        if (p_ && pinned_cap_) PinnedPool::get().give(p_, pinned_cap_);
        else std::free(p_);
        p_ = nullptr, n_ = 0, pinned_cap_ = 0;
    }
    double* p_ = nullptr;
    size_t n_ = 0;
    size_t pinned_cap_ = 0;  // size of the page-locked block holding p_, or 0
};

// dst = src[0..n), in up to 8 host threads for large arrays.  bad: how
// non-finite values are treated, 0 kept, 1 counted (the return value is the
// count), 2 replaced by `fill`.
static int64_t stage_copy(double* dst, const double* src, size_t n, int bad, double fill) {
    auto part = [=](size_t lo, size_t hi) -> int64_t {
        int64_t nb = 0;
        for (size_t q = lo; q < hi; ++q) {
            double v = src[q];
            if (bad != 0 && !std::isfinite(v)) {
                ++nb;
                if (bad == 2) v = fill;
            }
            dst[q] = v;
        }
        return nb;
    };
    const unsigned hw = std::thread::hardware_concurrency();
    const size_t nt = n < ((size_t)1 << 20) ? 1 : std::min<size_t>(8, std::max(1u, hw));
    if (nt == 1) return part(0, n);
    std::vector<int64_t> cnt(nt, 0);
    std::vector<std::thread> th;
    try {
        for (size_t t = 1; t < nt; ++t) th.emplace_back([&, t] { cnt[t] = part(n * t / nt, n * (t + 1) / nt); });
    } catch (...) {  // no thread to be had: this thread does the rest
        const size_t done = th.size() + 1;
        cnt[0] = part(n * done / nt, n);
    }
    cnt[0] += part(0, n / nt);
    for (auto& x : th) x.join();
    int64_t s = 0;
    for (int64_t v : cnt) s += v;
    return s;
}

// One sph_add_* call, staged on the host until the case is admitted: ids
// first .. first + n - 1, all of one kind (0 fluid, 1 solid), material and body.
struct PBlock {
    int kind = 0, body = -1, mat = 0;
    int64_t n = 0, first = 0;
    HostArray pos;       // 3n
    HostArray vel, nrm;  // 3n, or empty: zero
    HostArray T, rho;    // n, or empty: the material's T_init, rho0
};

struct sph_ctx {
    sph_config cfg{};
    cudaStream_t stream = nullptr;
    std::string err;
    sph_material mats[MAX_MAT]{};
    bool mat_set[MAX_MAT]{};
    struct {
        double c[3], a[3], omega;
        bool set;
    } bodies[MAX_BODY]{};
    // host staging: one block per sph_add_* call, in id order
    std::vector<PBlock> blocks;
    int64_t n_total = 0, n_fluid = 0, n_solid = 0;
    int ncell[3]{};
    double cellw[3]{};
    double sigma0 = 0.0;
    int kcap = 0;
    int tune_batch = 2, tune_tpp = 1, tune_block = 128;
    bool started = false;   // stepped as a single case
    bool admitted = false;  // handed to a batch
    Engine* eng = nullptr;
};

struct sph_batch {
    Engine eng;
};

static sph_status fail(sph_ctx* c, sph_status s, const char* fmt, ...) {
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        c->err = vformat(fmt, ap);
        va_end(ap);
    }
    return s;
}

// ----------------------------------------------------------------- engine ---
// The engine's device arrays are requested first and then carved out of one
// allocation (256-byte aligned each), zeroed by one memset: one cudaMalloc
// instead of one per array.
struct ArenaReq {
    void** slot;
    size_t bytes;
};
template <class T>
static void dreq(std::vector<ArenaReq>& R, T** p, size_t count) {
    R.push_back({(void**)p, sizeof(T) * (count ? count : 1)});
}
static cudaError_t arena_alloc(Engine& E, const std::vector<ArenaReq>& R) {
    auto span = [](size_t b) { return (b + 255) / 256 * 256; };
    size_t total = 0;
    for (const ArenaReq& r : R) total += span(r.bytes);
    void* base = nullptr;
    cudaError_t e = cudaMalloc(&base, total);
    if (e != cudaSuccess) return e;
    E.allocs.push_back(base);
    size_t off = 0;
    for (const ArenaReq& r : R) {
        *r.slot = (char*)base + off;
        off += span(r.bytes);
    }
    return cudaMemsetAsync(base, 0, total, E.stream);
}

static sph_status engine_alloc(Engine& E, int64_t n_cap, int c_cap, int64_t cells_cap, int hist_cap) {
    if (n_cap < 1 || n_cap > (int64_t)MAX_PARTICLES - 1 || c_cap < 1 || c_cap > (1 << 20) || cells_cap < 1 ||
        cells_cap > ((int64_t)1 << 30) || hist_cap < 0)
        return E.fail(SPH_EINVAL, "engine capacity out of range");
    int dev = 0, sms = 148;
    E_CUDA(E, cudaGetDevice(&dev));
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    set_grid_cap(sms);
    E.n_cap = n_cap;
    E.c_cap = c_cap;
    E.cells_cap = cells_cap;
    E.hist_cap = hist_cap;
    Bufs& B = E.B;
    const int64_t n = n_cap;
    B.n = 0;
    B.ncases = c_cap;
    B.ncells = (int)cells_cap;
    B.max_chunks = (int)((n + RED_CHUNK - 1) / RED_CHUNK) + c_cap + 1;
    B.hist_cap = hist_cap;
    B.one_case = -1;  // set when a step graph is captured over a single case
    std::vector<ArenaReq> reqs;
#define AL(p, cnt) dreq(reqs, &(p), (size_t)(cnt))
    AL(B.cases, c_cap);
    AL(B.st, c_cap);
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
    AL(B.CF, n);
    if (B.fp64) {
        for (int p = 0; p < 2; ++p) {
            AL(B.V64[p], n);
            AL(B.DR64[p], n);
        }
        AL(B.VH64, n);
        AL(B.AV64, n);
        AL(B.NRM64, n);
        AL(B.RN64, n);
        AL(B.TORQ64, n);
        AL(B.TORQV64, n);
    }
    AL(B.KEYS, n);
    AL(B.RANK, n);
    AL(B.TMP, n);
    AL(B.PERM, n);
    AL(B.CNT, cells_cap + 1);
    AL(B.CSTART, cells_cap + 2);
    AL(B.SCANBLK, scan_blocks((int)cells_cap + 1) + 1);
    AL(B.PART, (size_t)3 * B.max_chunks);
    AL(B.CHUNK_CASE, B.max_chunks);
    E.tq_cap = (int)((n + TQ_CHUNK - 1) / TQ_CHUNK) + c_cap * MAX_BODY;
    AL(B.TQC, E.tq_cap);
    AL(B.TQR, (size_t)c_cap * MAX_BODY);
    AL(B.TQP, (size_t)2 * E.tq_cap);
    AL(B.nchunks, 1);
    AL(B.HIST, (size_t)8 * (hist_cap > 0 ? hist_cap : 1) * c_cap);
    AL(E.d_field, (size_t)3 * n);
    AL(B.NB, (size_t)NB_CAP * n);
    AL(B.NBC, n);
    AL(B.OVFL, n);
    AL(B.novf, 1);
    AL(B.VH, n);
#undef AL
    const cudaError_t e = arena_alloc(E, reqs);
    if (e != cudaSuccess)
        return E.fail(e == cudaErrorMemoryAllocation ? SPH_ENOMEM : SPH_ECUDA, "device allocation: %s",
                      cudaGetErrorString(e));
    B.nb_stride = (int)n;
    if (B.tune_batch == 0) B.tune_batch = 2;
    if (B.tune_tpp == 0) B.tune_tpp = 1;
    if (B.tune_block == 0) B.tune_block = 128;
    E.cases.assign(c_cap, HostCase{});
    E.st_h.assign(c_cap, CaseState{});
    E.cdev_h.assign(c_cap, CaseDev{});
    E.ids.reset(n_cap);
    E.cells.reset(cells_cap);
    E.allocated = true;
    return SPH_OK;
}

// Per-case parameter table entry from a staged context.
static void build_case(const sph_ctx* c, const HostCase& H, CaseDev& C) {
    const sph_config& F = c->cfg;
    memset(&C, 0, sizeof C);
    const double h = F.h_over_dx * F.dx;
    const double R2 = (2.0 * h) * (2.0 * h);
    for (int a = 0; a < 3; ++a) {
        C.origin[a] = F.origin[a];
        C.ext[a] = F.extent[a];
        C.cellw[a] = c->cellw[a];
        C.inv_cellw[a] = 1.0 / c->cellw[a];
        C.gcellw[a] = split_of(a) * c->cellw[a];
        C.gcellwf[a] = (float)C.gcellw[a];
        C.scellwf[a] = (float)c->cellw[a];
        C.inv_scellwf[a] = (float)(1.0 / c->cellw[a]);
        C.originf[a] = (float)F.origin[a];
        C.ncell[a] = c->ncell[a];
        C.g[a] = (float)F.gravity[a];
    }
    C.cell_base = (int)H.cell_base;
    C.ncells = c->ncell[0] * c->ncell[1] * c->ncell[2];
    C.gcorner_ok = 1;
    for (int a = 0; a < 3; ++a) C.gcorner_ok &= (c->ncell[a] / split_of(a) <= GCORNER_MAX) ? 1 : 0;
    if (C.gcorner_ok)
        for (int a = 0; a < 3; ++a)
            for (int g = 0; g < c->ncell[a] / split_of(a); ++g) C.gcorner[a][g] = C.origin[a] + (double)g * C.gcellw[a];
    C.periodic = F.periodic_mask;
    C.R2 = R2;
    // FP32 guard band around the cut-off: inside it the FP64 rule decides
    C.R2lo = (float)(R2 * (1.0 - 1e-4));
    C.R2hi = (float)(R2 * (1.0 + 1e-4));
    C.R2eps = (float)(R2 * 1e-4);
    C.Rmargin = (float)(2.0 * h * 1e-4);
    C.h = (float)h;
    C.inv_h = (float)(1.0 / h);
    const double alpha = 21.0 / (16.0 * M_PI * h * h * h);
    C.kw = (float)alpha;
    C.kdw = (float)(-5.0 * alpha / h);
    C.nhinv = (float)(-0.5 / h);
    C.kdwh = (float)(-5.0 * alpha / (h * h));
    C.w0 = (float)alpha;
    C.inv_sigma0 = (float)(1.0 / c->sigma0);
    C.inv_contact_full = (float)(1.0 / (F.dx * F.dx * F.dx * (c->sigma0 - alpha)));
    C.inv_contact_full64 = 1.0 / (F.dx * F.dx * F.dx * (c->sigma0 - alpha));
    C.vol = (float)(F.dx * F.dx * F.dx);
    C.c0 = (float)F.c0;
    C.c02 = (float)(F.c0 * F.c0);
    C.inv_c0 = (float)(1.0 / F.c0);
    C.inv_c02 = (float)(1.0 / (F.c0 * F.c0));
    C.h64 = h;
    C.c0_64 = F.c0;
    C.kw64 = alpha;
    C.kdw64 = -5.0 * alpha / h;
    C.w0_64 = alpha;
    C.inv_sigma0_64 = 1.0 / c->sigma0;
    C.vol64 = F.dx * F.dx * F.dx;
    C.c02_64 = F.c0 * F.c0;
    C.inv_c0_64 = 1.0 / F.c0;
    C.inv_c02_64 = 1.0 / (F.c0 * F.c0);
    for (int a = 0; a < 3; ++a) C.g64[a] = F.gravity[a];
    C.fp64 = F.pair_precision == 1 ? 1 : 0;
    C.visc_heat = F.viscous_heating ? 1 : 0;
    C.vstar_lit = F.vstar_literal ? 1 : 0;
    C.wall_printed = F.wall_pstar_printed ? 1 : 0;
    C.u_ref = F.u_ref;
    C.cfl_ad = F.cfl_ad;
    C.cfl_ac = F.cfl_ac;
    C.free_surface = F.free_surface;
    C.kcap = c->kcap;
    double nu = 0.0, Tref = 0.0;
    int nfl = 0;
    auto T_first = [&](const PBlock& P) { return P.T.empty() ? c->mats[P.mat].T_init : P.T[0]; };
    for (const PBlock& P : c->blocks)
        if (P.kind == 0) {
            const sph_material& M = c->mats[P.mat];
            nu = std::max(nu, M.mu / M.rho0);
            if (nfl++ == 0) Tref = T_first(P);
        }
    if (nfl == 0 && !c->blocks.empty()) Tref = T_first(c->blocks[0]);
    C.nu_max = nu;
    C.T_ref = Tref;
    // Eq. (26): the thermal bound over every conducting material whose
    // temperature is integrated (fluid and free solids) caps dt_ad
    double dtT = INFINITY;
    const double hT = F.h_over_dx * F.dx;
    if (F.cfl_T > 0.0)
        for (const PBlock& P : c->blocks) {
            const sph_material& M = c->mats[P.mat];
            if ((P.kind == 0 || !M.fixed_T) && M.k > 0.0)
                dtT = std::min(dtT, F.cfl_T * M.rho0 * M.cp * hT * hT / M.k);
        }
    C.dt_T = dtT;
    for (int m = 0; m < MAX_MAT; ++m) {
        if (!c->mat_set[m]) continue;
        const sph_material& M = c->mats[m];
        C.mat[m].rho0 = (float)M.rho0;
        C.mat[m].mass = (float)(M.rho0 * F.dx * F.dx * F.dx);
        C.mat[m].mu = (float)M.mu;
        C.mat[m].k = (float)M.k;
        C.mat[m].cp = (float)M.cp;
        C.mat[m].inv_rho0_cp = (float)(1.0 / (M.rho0 * M.cp));
        C.mat[m].fixed_T = M.fixed_T;
        C.mat64[m].rho0 = M.rho0;
        C.mat64[m].mass = M.rho0 * F.dx * F.dx * F.dx;
        C.mat64[m].mu = M.mu;
        C.mat64[m].k = M.k;
        C.mat64[m].cp = M.cp;
        C.mat64[m].inv_rho0_cp = 1.0 / (M.rho0 * M.cp);
    }
    // the fluid particles' material (the pair passes' single-material path
    // reads it when every fluid particle of every resident case shares one)
    for (const PBlock& P : c->blocks)
        if (P.kind == 0) {
            C.fluid = C.mat[P.mat];
            break;
        }
    int nb = 0;
    for (int b = 0; b < MAX_BODY; ++b) {
        BodyDev& Bd = C.body[b];
        if (!c->bodies[b].set) continue;
        nb = b + 1;
        Bd.set = 1;
        for (int a = 0; a < 3; ++a) {
            Bd.c[a] = c->bodies[b].c[a];
            Bd.axis[a] = c->bodies[b].a[a];
        }
        Bd.omega = c->bodies[b].omega;
        int64_t lo = -1, hi = -1;
        for (const PBlock& P : c->blocks)
            if (P.kind == 1 && P.body == b) {
                if (lo < 0) lo = P.first;
                hi = P.first + P.n;
            }
        Bd.id_lo = (int)(H.id_base + (lo < 0 ? 0 : lo));
        Bd.id_hi = (int)(H.id_base + (hi < 0 ? 0 : hi));
    }
    C.n_body = nb;
}

static bool single_fluid_material(const sph_ctx* c) {
    int fm = -1;
    for (const PBlock& P : c->blocks)
        if (P.kind == 0) {
            if (fm < 0) fm = P.mat;
            else if (P.mat != fm) return false;
        }
    return true;
}

// Append a staged case's particles to the packed array (sorted in prepare()).
static sph_status engine_admit(Engine& E, const sph_ctx* c, int64_t steps_req, int* slot_out) {
    const int64_t n = c->n_total;
    if (n == 0) return E.fail(SPH_EINVAL, "case has no particles");
    int slot = -1;
    for (int k = 0; k < E.c_cap; ++k)
        if (!E.cases[k].used) {
            slot = k;
            break;
        }
    if (slot < 0) return E.fail(SPH_ENOMEM, "no free case slot (max_cases %d)", E.c_cap);
    if ((int64_t)E.B.n + n > E.n_cap)
        return E.fail(SPH_ENOMEM, "particle capacity exceeded (%lld resident + %lld > %lld)", (long long)E.B.n,
                      (long long)n, (long long)E.n_cap);
    const int64_t nc = (int64_t)c->ncell[0] * c->ncell[1] * c->ncell[2];
    HostCase H;
    if (!E.cells.alloc(nc, &H.cell_base)) return E.fail(SPH_ENOMEM, "cell index capacity exceeded");
    if (!E.ids.alloc(n, &H.id_base)) {
        E.cells.release(H.cell_base, nc);
        return E.fail(SPH_ENOMEM, "particle id capacity exceeded");
    }
    H.used = true;
    H.pending = true;
    H.n = n;
    H.n_fluid = c->n_fluid;
    H.n_solid = c->n_solid;
    H.ncells = nc;
    H.kcap = c->kcap;
    H.steps_req = steps_req;
    for (int a = 0; a < 3; ++a) {
        H.ncell[a] = c->ncell[a];
        H.cellw[a] = c->cellw[a];
    }
    CaseDev C;
    build_case(c, H, C);
    H.visc_heat = C.visc_heat != 0;
    for (int b = 0; b < MAX_BODY; ++b) {
        H.body_lo[b] = C.body[b].set ? C.body[b].id_lo : 0;
        H.body_hi[b] = C.body[b].set ? C.body[b].id_hi : 0;
    }
    CaseState S;
    memset(&S, 0, sizeof S);
    S.alive = 1;
    S.running = 1;
    S.init_pending = 1;
    S.steps_req = steps_req;
    Bufs& B = E.B;
    const int p = E.parity;
    const int64_t at = B.n;
    const int64_t idb = H.id_base;
    cudaStream_t s = E.stream;
    E_CUDA(E, cudaMemcpyAsync(B.cases + slot, &C, sizeof C, cudaMemcpyHostToDevice, s));
    E_CUDA(E, cudaMemcpyAsync(B.st + slot, &S, sizeof S, cudaMemcpyHostToDevice, s));
    E_CUDA(E, cudaMemsetAsync(B.DR[p] + at, 0, sizeof(float) * n, s));
    E_CUDA(E, cudaMemsetAsync(B.TORQ + idb, 0, sizeof(float) * n, s));
    E_CUDA(E, cudaMemsetAsync(B.TORQV + idb, 0, sizeof(float) * n, s));
    E_CUDA(E, cudaMemsetAsync(B.CF + idb, 0, sizeof(double) * n, s));
    if (B.fp64) {
        E_CUDA(E, cudaMemsetAsync(B.DR64[p] + at, 0, sizeof(double) * n, s));
        E_CUDA(E, cudaMemsetAsync(B.TORQ64 + idb, 0, sizeof(double) * n, s));
        E_CUDA(E, cudaMemsetAsync(B.TORQV64 + idb, 0, sizeof(double) * n, s));
    }
    // the staged blocks go up as they are (one device scratch holding them
    // all, so the copies and kernels of the blocks queue back to back) and a
    // kernel writes each into the packed layout
    size_t scratch = 0;
    for (const PBlock& P : c->blocks) scratch += P.pos.size() + P.vel.size() + P.nrm.size() + P.T.size() + P.rho.size();
    double* d = nullptr;
    E_CUDA(E, cudaMallocAsync((void**)&d, sizeof(double) * std::max<size_t>(scratch, 1), s));
    cudaError_t e = cudaSuccess;
    std::vector<void*> pinned;  // staging arrays page-locked here for their copies
    double* q = d;
    for (const PBlock& P : c->blocks) {
        auto up = [&](const HostArray& v) -> const double* {
            if (v.empty() || e != cudaSuccess) return nullptr;
            const size_t bytes = sizeof(double) * v.size();
            // large arrays not already in page-locked memory are locked for the
            // copy (full-rate DMA instead of the driver's pageable staging);
            // the pageable copy remains if that is refused
            if (bytes >= ((size_t)2 << 20) && !v.pinned()) {
                void* h = const_cast<double*>(v.data());
                if (cudaHostRegister(h, bytes, cudaHostRegisterDefault) == cudaSuccess) pinned.push_back(h);
                else (void)cudaGetLastError();
            }
            double* dst = q;
            e = cudaMemcpyAsync(dst, v.data(), bytes, cudaMemcpyHostToDevice, s);
            q += v.size();
            return dst;
        };
        const double* dpos = up(P.pos);
        const double* dvel = up(P.vel);
        const double* dnrm = up(P.nrm);
        const double* dT = up(P.T);
        const double* drho = up(P.rho);
        const uint32_t kind = P.kind == 0 ? KIND_FLUID
                                          : ((P.body >= 0 && c->bodies[P.body].set) ? KIND_ROT : KIND_STATIC);
        const uint32_t tag = make_tag((uint32_t)P.mat, kind, kind == KIND_ROT ? (uint32_t)P.body : 0u, (uint32_t)slot);
        const sph_material& M = c->mats[P.mat];
        if (e == cudaSuccess)
            e = launch_admit_block(B, p, (int)P.n, (int)(at + P.first), (int)(idb + P.first), tag, P.kind == 0 ? 1 : 0,
                                   M.rho0, M.T_init, dpos, dvel, dnrm, dT, drho, s);
        if (e != cudaSuccess) break;
    }
    // the copies are done before the staging arrays are unlocked or freed
    // (and, after an error, nothing is left in flight)
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    else (void)cudaStreamSynchronize(s);
    for (void* h : pinned) (void)cudaHostUnregister(h);
    cudaFreeAsync(d, s);
    if (e != cudaSuccess) return E.fail(SPH_ECUDA, "admission: %s", cudaGetErrorString(e));
    // reference heat content and initial max speed from the appended block
    E_CUDA(E, launch_block_heat0(B, p, slot, (int)at, (int)n, B.PART, s));
    E_CUDA(E, launch_vmax_init(B, p, (int)at, (int)(at + n), s));
    // the admitted particles are in place before the case can step
    E_CUDA(E, cudaStreamSynchronize(s));
    B.n = (int)(at + n);
    E.cases[slot] = H;
    E.st_h[slot] = S;
    E.cdev_h[slot] = C;
    E.need_prepare = true;
    E.graph_dirty = true;
    if (slot_out) *slot_out = slot;
    return SPH_OK;
}

// Event k+1 closes interval k; intervals carry a group class (SPH_PROF_*)
// and the acoustic sub-step index they belong to.
static cudaError_t mark(Engine& E, int cls, int sub) {
    if (!E.prof) return cudaSuccess;
    const size_t k = E.ev_class.size() + 1;
    if (k >= E.ev.size()) return cudaErrorInvalidValue;
    E.ev_class.push_back(cls);
    E.ev_sub.push_back(sub);
    return cudaEventRecordWithFlags(E.ev[k], E.cap, cudaEventRecordExternal);
}

// The pair constants of a case (host copy C) whose case-table entry is at
// device address dev.
static PairConst pair_const(const CaseDev& C, const CaseDev* dev) {
    PairConst P{};
    for (int a = 0; a < 3; ++a) {
        P.gcellwf[a] = C.gcellwf[a];
        P.scellwf[a] = C.scellwf[a];
        P.inv_scellwf[a] = C.inv_scellwf[a];
        P.g[a] = C.g[a];
        P.ncell[a] = C.ncell[a];
    }
    P.Rmargin = C.Rmargin;
    P.R2lo = C.R2lo;
    P.R2hi = C.R2hi;
    P.R2eps = C.R2eps;
    P.inv_h = C.inv_h;
    P.w0 = C.w0;
    P.kw = C.kw;
    P.kdw = C.kdw;
    P.nhinv = C.nhinv;
    P.kdwh = C.kdwh;
    P.inv_sigma0 = C.inv_sigma0;
    P.vol = C.vol;
    P.inv_contact_full = C.inv_contact_full;
    P.c0 = C.c0;
    P.c02 = C.c02;
    P.inv_c0 = C.inv_c0;
    P.inv_c02 = C.inv_c02;
    P.cell_base = C.cell_base;
    P.periodic = C.periodic;
    P.free_surface = C.free_surface;
    P.visc_heat = C.visc_heat;
    P.fluid = C.fluid;
    P.mat = reinterpret_cast<const MatDev*>(reinterpret_cast<const char*>(dev) + offsetof(CaseDev, mat));
    P.body = reinterpret_cast<const BodyDev*>(reinterpret_cast<const char*>(dev) + offsetof(CaseDev, body));
    return P;
}

static sph_status capture(Engine& E) {
    // capture runs nothing; it needs a stream other than the legacy default one
    if (!E.cap) E_CUDA(E, cudaStreamCreateWithFlags(&E.cap, cudaStreamNonBlocking));
    if (!E.cap2) E_CUDA(E, cudaStreamCreateWithFlags(&E.cap2, cudaStreamNonBlocking));
    E.kcap_max = 0;
    for (const HostCase& H : E.cases)
        if (H.used) E.kcap_max = std::max(E.kcap_max, H.kcap);
    // neighbour lists are rebuilt every step: lay them out for the resident
    // particles, not the capacity, so one particle's slots stay close together
    E.B.nb_stride = std::max(E.B.n, 1);
    E.B.max_chunks_used = (int)((E.B.n + RED_CHUNK - 1) / RED_CHUNK) + E.c_cap + 1;
    E.B.visc_heat = 0;
    for (const HostCase& H : E.cases)
        if (H.used && H.visc_heat) E.B.visc_heat = 1;
    // the pair passes' constants: entry 0 for a single resident case, else
    // one entry per case slot (when the slots fit the table)
    E.B.one_case = -1;
    E.tab = PairTab{};
    {
        int used = 0, k1 = -1;
        for (int k = 0; k < E.c_cap; ++k)
            if (E.cases[k].used) {
                ++used;
                k1 = k;
            }
        if (used == 1) {
            E.B.one_case = k1;
            E.tab.c[0] = pair_const(E.cdev_h[k1], E.B.cases + k1);
        } else if (E.c_cap <= PAIRTAB_MAX) {
            for (int k = 0; k < E.c_cap; ++k)
                if (E.cases[k].used) E.tab.c[k] = pair_const(E.cdev_h[k], E.B.cases + k);
        }
    }
    {
        // torque chunks of the resident rigid bodies (fixed TQ_CHUNK id blocks from each body's start)
        std::vector<int4> tqc;
        std::vector<int2> tqr((size_t)E.c_cap * MAX_BODY, make_int2(0, 0));
        for (int c = 0; c < E.c_cap; ++c) {
            const HostCase& H = E.cases[c];
            if (!H.used) continue;
            for (int b = 0; b < MAX_BODY; ++b) {
                const int lo = H.body_lo[b], hi = H.body_hi[b];
                if (hi <= lo) continue;
                tqr[(size_t)c * MAX_BODY + b] = make_int2((int)tqc.size(), (hi - lo + TQ_CHUNK - 1) / TQ_CHUNK);
                for (int a = lo; a < hi; a += TQ_CHUNK) tqc.push_back(make_int4(c, b, a, std::min(a + TQ_CHUNK, hi)));
            }
        }
        if ((int)tqc.size() > E.tq_cap) return E.fail(SPH_ECUDA, "torque chunk table overflow");
        E.B.ntq = (int)tqc.size();
        if (!tqc.empty())
            E_CUDA(E, cudaMemcpyAsync(E.B.TQC, tqc.data(), sizeof(int4) * tqc.size(), cudaMemcpyHostToDevice,
                                      E.stream));
        E_CUDA(E, cudaMemcpyAsync(E.B.TQR, tqr.data(), sizeof(int2) * tqr.size(), cudaMemcpyHostToDevice, E.stream));
        E_CUDA(E, cudaStreamSynchronize(E.stream));
    }
    const size_t nev = 8 + 4 * (size_t)E.kcap_max + 8;
    if (E.prof && E.ev.size() < nev) {
        for (auto e : E.ev) cudaEventDestroy(e);
        E.ev.assign(nev, nullptr);
        for (auto& e : E.ev) E_CUDA(E, cudaEventCreate(&e));
    }
    for (int p = 0; p < 2; ++p) {
        cudaGraph_t g = nullptr;
        E.ev_class.clear();
        E.ev_sub.clear();
        E_CUDA(E, cudaStreamBeginCapture(E.cap, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = E.prof ? cudaEventRecordWithFlags(E.ev[0], E.cap, cudaEventRecordExternal) : cudaSuccess;
        if (e == cudaSuccess) e = launch_adv_begin(E.B, E.cap);
        if (e == cudaSuccess) e = launch_sort(E.B, p, E.cap);
        if (e == cudaSuccess) e = mark(E, SPH_PROF_SORT, -1);
        if (e == cudaSuccess) e = launch_passD(E.B, p, E.tab, E.cap);
        if (e == cudaSuccess) e = mark(E, SPH_PROF_PASS_D, -1);
        if (e == cudaSuccess) e = launch_passVT(E.B, p, E.tab, E.cap);
        if (e == cudaSuccess) e = mark(E, SPH_PROF_PASS_VT, -1);
        if (E.prof) {
            // profiling: kcap unrolled sub-step slots with event records between
            // the kernel groups (slots past a step's last sub-step exit at once)
            for (int k = 0; k < E.kcap_max && e == cudaSuccess; ++k) {
                e = launch_sub_begin(E.B, E.cap);
                if (e == cudaSuccess) e = mark(E, SPH_PROF_CONTROL, k);
                if (e == cudaSuccess) e = launch_passM(E.B, p, E.tab, E.cap);
                if (e == cudaSuccess) e = mark(E, SPH_PROF_PASS_M, k);
                if (e == cudaSuccess) e = launch_passC(E.B, p, E.tab, E.cap);
                if (e == cudaSuccess) e = mark(E, SPH_PROF_PASS_C, k);
                if (e == cudaSuccess) e = launch_sub_end(E.B, E.cap);
                if (e == cudaSuccess) e = mark(E, SPH_PROF_CONTROL, k);
            }
        } else if (e == cudaSuccess) {
            // the sub-steps as a WHILE conditional node: its body is one
            // sub-step, and k_sub_cond clears the condition once no case has a
            // sub-step left, so only the sub-steps a step needs are launched
            cudaStreamCaptureStatus cst;
            cudaGraph_t cg = nullptr;
            const cudaGraphNode_t* deps = nullptr;
            size_t ndeps = 0;
            e = cudaStreamGetCaptureInfo(E.cap, &cst, nullptr, &cg, &deps, nullptr, &ndeps);
            cudaGraphConditionalHandle h = 0;
            if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h, cg, 1, cudaGraphCondAssignDefault);
            cudaGraphNodeParams np = {};
            np.type = cudaGraphNodeTypeConditional;
            np.conditional.handle = h;
            np.conditional.type = cudaGraphCondTypeWhile;
            np.conditional.size = 1;
            cudaGraphNode_t cn = nullptr;
            if (e == cudaSuccess) e = cudaGraphAddNode(&cn, cg, deps, nullptr, ndeps, &np);
            if (e == cudaSuccess) {
                e = cudaStreamBeginCaptureToGraph(E.cap2, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                                  cudaStreamCaptureModeThreadLocal);
                if (e == cudaSuccess) {
                    e = launch_sub_begin(E.B, E.cap2);
                    if (e == cudaSuccess) e = launch_passM(E.B, p, E.tab, E.cap2);
                    if (e == cudaSuccess) e = launch_passC(E.B, p, E.tab, E.cap2);
                    if (e == cudaSuccess) e = launch_sub_end(E.B, E.cap2);
                    if (e == cudaSuccess) e = launch_sub_cond(E.B, h, E.cap2);
                    cudaGraph_t bg = nullptr;
                    const cudaError_t e3 = cudaStreamEndCapture(E.cap2, &bg);
                    if (e == cudaSuccess) e = e3;
                }
            }
            if (e == cudaSuccess)
                e = cudaStreamUpdateCaptureDependencies(E.cap, &cn, nullptr, 1, cudaStreamSetCaptureDependencies);
        }
        if (e == cudaSuccess) e = launch_adv_end(E.B, p, E.cap);
        if (e == cudaSuccess) e = mark(E, SPH_PROF_ADV_END, -1);
        cudaError_t e2 = cudaStreamEndCapture(E.cap, &g);
        if (e != cudaSuccess || e2 != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return E.fail(SPH_ECUDA, "graph capture failed: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
        }
        // same kernels in the same order (only sizes and arguments changed):
        // patch the executable graph in place instead of instantiating anew
        if (E.gexec[p]) {
            cudaGraphExecUpdateResultInfo info;
            if (cudaGraphExecUpdate(E.gexec[p], g, &info) == cudaSuccess) {
                cudaGraphDestroy(g);
                ++E.graph_updates;
                continue;
            }
            (void)cudaGetLastError();
            cudaGraphExecDestroy(E.gexec[p]);
            E.gexec[p] = nullptr;
        }
        e = cudaGraphInstantiate(&E.gexec[p], g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return E.fail(SPH_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
        ++E.graph_instantiations;
    }
    E.graph_dirty = false;
    return SPH_OK;
}

static sph_status pull_state(Engine& E) {
    E_CUDA(E, cudaMemcpyAsync(E.st_h.data(), E.B.st, sizeof(CaseState) * E.c_cap, cudaMemcpyDeviceToHost, E.stream));
    E_CUDA(E, cudaStreamSynchronize(E.stream));
    return SPH_OK;
}

// Cells scanned per sort: up to the highest allocated cell range (the dead
// bucket sits just past it).
static void set_cell_high_water(Engine& E) {
    int64_t hw = 1;
    for (const HostCase& H : E.cases)
        if (H.used) hw = std::max(hw, H.cell_base + H.ncells);
    E.B.ncells = (int)hw;
}

// Apply pending retirements and admissions before the next step.  Nothing
// is re-sorted here: admitted particles sit unsorted past the resident ones
// and retired cases are flagged dead; the next step's cell sort places the
// former and carries the latter past all live particles, after which
// finish_retirements() drops them.
static sph_status prepare(Engine& E) {
    if (!E.need_prepare) return SPH_OK;
    Bufs& B = E.B;
    static const int zero = 0;
    for (int k = 0; k < E.c_cap; ++k) {
        HostCase& H = E.cases[k];
        if (!H.used || !H.retiring || H.dead) continue;
        E_CUDA(E, cudaMemcpyAsync(&B.st[k].alive, &zero, sizeof(int), cudaMemcpyHostToDevice, E.stream));
        E_CUDA(E, cudaMemcpyAsync(&B.st[k].running, &zero, sizeof(int), cudaMemcpyHostToDevice, E.stream));
        H.dead = true;
    }
    for (HostCase& H : E.cases) H.pending = false;
    set_cell_high_water(E);  // covers dead and newly admitted cases
    E.need_prepare = false;
    E.graph_dirty = true;
    return pull_state(E);
}

// After a step whose sort has carried the dead cases' particles past the live
// ones: shrink the particle count to the live ones and free their ranges.
static void finish_retirements(Engine& E) {
    int64_t live = 0;
    bool any = false;
    for (const HostCase& H : E.cases) {
        if (!H.used) continue;
        if (H.dead) any = true;
        else live += H.n;
    }
    if (!any) return;
    E.B.n = (int)live;
    for (HostCase& H : E.cases) {
        if (!H.used || !H.dead) continue;
        E.cells.release(H.cell_base, H.ncells);
        E.ids.release(H.id_base, H.n);
        H = HostCase{};
    }
    set_cell_high_water(E);
    E.graph_dirty = true;
}

static sph_status engine_step(Engine& E, int n_steps) {
    sph_status r = prepare(E);
    if (r != SPH_OK) return r;
    if (E.B.n == 0) return SPH_OK;
    if (E.graph_dirty) {
        r = capture(E);
        if (r != SPH_OK) return r;
    }
    for (int k = 0; k < n_steps; ++k) {
        if (E.graph_dirty) {
            r = capture(E);
            if (r != SPH_OK) return r;
        }
        E_CUDA(E, cudaGraphLaunch(E.gexec[E.parity], E.stream));
        E.parity ^= 1;
        ++E.graph_steps;
        finish_retirements(E);
        if (E.prof) {
            r = pull_state(E);
            if (r != SPH_OK) return r;
            int nsub = 0;
            for (int c = 0; c < E.c_cap; ++c)
                if (E.cases[c].used) nsub = std::max(nsub, E.st_h[c].last_nsub);
            for (size_t q = 0; q < E.ev_class.size(); ++q) {
                float ms = 0.f;
                E_CUDA(E, cudaEventElapsedTime(&ms, E.ev[q], E.ev[q + 1]));
                const int cls = (E.ev_sub[q] >= nsub) ? SPH_PROF_IDLE : E.ev_class[q];
                E.prof_ms[cls] += ms;
                E.prof_cnt[cls] += 1;
            }
        }
    }
    return pull_state(E);
}

static int engine_kernels_per_step(const Engine& E) {
    int kc = 0;
    for (const HostCase& H : E.cases)
        if (H.used) kc = std::max(kc, H.kcap);
    return kernels_per_advection_step(kc, E.B.fp64 != 0);
}

static sph_status read_fields(Engine& E, int slot, int field, void* dst, int64_t n) {
    const HostCase& H = E.cases[slot];
    if (!dst || n != H.n) return E.fail(SPH_EINVAL, "n must equal the case's particle count %lld", (long long)H.n);
    int k;
    switch (field) {
    case SPH_FIELD_POS: case SPH_FIELD_VEL: case SPH_FIELD_AVISC: case SPH_FIELD_NORMAL: k = 3; break;
    case SPH_FIELD_RHO: case SPH_FIELD_P: case SPH_FIELD_T: case SPH_FIELD_DRHO: case SPH_FIELD_DTDT:
    case SPH_FIELD_CONTACT: k = 1; break;
    default: return E.fail(SPH_EINVAL, "unknown field %d", field);
    }
    E_CUDA(E, launch_gather_field(E.B, E.parity ^ 1, field, slot, (int)H.id_base, E.d_field, E.stream));
    E_CUDA(E, cudaMemcpyAsync(dst, E.d_field, sizeof(double) * k * n, cudaMemcpyDeviceToHost, E.stream));
    E_CUDA(E, cudaStreamSynchronize(E.stream));
    return SPH_OK;
}

// The last n (<= max_steps, <= the ring's capacity) advection-step records
// of case `slot`, oldest first, 8 doubles each.
static sph_status read_curve(Engine& E, int slot, double* out, int64_t max_steps, int64_t* n_out) {
    if (!out || max_steps < 0) return E.fail(SPH_EINVAL, "out is NULL or max_steps < 0");
    const int64_t done = E.st_h[slot].adv_steps;
    const int64_t cap = E.hist_cap;
    const int64_t n = std::min(done, std::min(cap, max_steps));
    if (n > 0) {
        std::vector<double> ring((size_t)8 * (size_t)cap);
        E_CUDA(E, cudaMemcpyAsync(ring.data(), E.B.HIST + (size_t)slot * cap * 8, sizeof(double) * 8 * cap,
                                  cudaMemcpyDeviceToHost, E.stream));
        E_CUDA(E, cudaStreamSynchronize(E.stream));
        for (int64_t k = 0; k < n; ++k) {
            const int64_t step = done - n + k;  // 0-based advection step index
            memcpy(out + 8 * k, ring.data() + 8 * (step % cap), sizeof(double) * 8);
        }
    }
    if (n_out) *n_out = n;
    return SPH_OK;
}

static sph_status read_torque_heat(Engine& E, int slot, int b, double* tq, double* tq_avg, double* heat,
                                   double* meanT) {
    if (b < 0 || b >= MAX_BODY) return E.fail(SPH_EINVAL, "body id %d out of range", b);
    sph_status s = pull_state(E);
    if (s != SPH_OK) return s;
    const CaseState& S = E.st_h[slot];
    if (tq) *tq = S.tq_inst[b];
    if (tq_avg) *tq_avg = S.time_int > 0 ? S.tq_int[b] / S.time_int : 0.0;
    if (heat) *heat = S.heat;
    if (meanT) *meanT = S.mean_T;
    return SPH_OK;
}

// ----------------------------------------------------- single-case C ABI ---
extern "C" {

const char* sph_last_error(const sph_ctx* ctx) {
    if (!ctx) return sph::g_stateless_err.c_str();
    return ctx->err.c_str();
}

sph_status sph_create(const sph_config* cfg, void* stream, sph_ctx** out) {
    if (!cfg || !out) return SPH_EINVAL;
    *out = nullptr;
    const double h = cfg->h_over_dx * cfg->dx;
    if (!(cfg->dx > 0) || !(cfg->h_over_dx > 0) || !(cfg->c0 > 0) || !(cfg->u_ref > 0) || !(cfg->cfl_ad > 0) ||
        !(cfg->cfl_ac > 0) || (cfg->pair_precision != 0 && cfg->pair_precision != 1) ||
        (cfg->viscous_heating != 0 && cfg->viscous_heating != 1) ||
        (cfg->vstar_literal != 0 && !(cfg->vstar_literal == 1 && cfg->pair_precision == 1)) ||
        (cfg->wall_pstar_printed != 0 && !(cfg->wall_pstar_printed == 1 && cfg->pair_precision == 1)) ||
        !(cfg->cfl_T >= 0))
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
        // geometry cells of width >= 2h, each cut into split_of(a) sort cells
        // (8 of width >= h/4 along x, 2 of width >= h along y and z)
        int64_t n = (int64_t)std::floor(cfg->extent[a] / R);
        if (n < 1) n = 1;
        if ((cfg->periodic_mask & (1 << a)) && n < 3) {
            delete c;
            return SPH_EINVAL;
        }
        c->ncell[a] = (int)(split_of(a) * n);
        c->cellw[a] = cfg->extent[a] / (double)(split_of(a) * n);
        total *= split_of(a) * n;
    }
    if (total > (int64_t)1 << 30) {
        delete c;
        return SPH_EINVAL;
    }
    c->kcap = cfg->max_substeps > 0 ? cfg->max_substeps
                                    : (int)std::ceil(cfg->cfl_ad / cfg->cfl_ac * (cfg->c0 / cfg->u_ref + 1.0)) + 2;
    c->sigma0 = lattice_sigma0(cfg->dx, h);
    *out = c;
    return SPH_OK;
}

sph_status sph_destroy(sph_ctx* c) {
    if (!c) return SPH_OK;
    delete c->eng;
    delete c;
    return SPH_OK;
}

sph_status sph_set_material(sph_ctx* c, int id, const sph_material* m) {
    if (!c) return SPH_EINVAL;
    if (c->started || c->admitted) return fail(c, SPH_ESTATE, "materials are fixed after the first step");
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
    if (c->started || c->admitted) return fail(c, SPH_ESTATE, "particles can only be added before the first step");
    if (n < 0 || (n > 0 && !pos)) return fail(c, SPH_EINVAL, "n < 0 or pos is NULL");
    if (mat < 0 || mat >= MAX_MAT || !c->mat_set[mat]) return fail(c, SPH_EINVAL, "material %d not set", mat);
    if (kind == 1 && (body < -1 || body >= MAX_BODY)) return fail(c, SPH_EINVAL, "body id %d out of range", body);
    if (kind == 1 && n > 0 && !nrm) return fail(c, SPH_EINVAL, "solid particles need normals");
    const int64_t n0 = c->n_total;
    if (n0 + n > (int64_t)MAX_PARTICLES - 1) return fail(c, SPH_EINVAL, "more than 2^26 - 1 particles");
    const sph_material& M = c->mats[mat];
    if (n == 0) {
        if (first_id) *first_id = n0;
        return SPH_OK;
    }
    PBlock P;
    P.kind = kind;
    P.body = kind == 0 ? -1 : body;
    P.mat = mat;
    P.n = n;
    P.first = n0;
    const size_t n1 = (size_t)n, n3 = 3 * n1;
    if (!P.pos.alloc(n3) || (vel && !P.vel.alloc(n3)) || (nrm && !P.nrm.alloc(n3)) || (T && !P.T.alloc(n1)) ||
        (rho && !P.rho.alloc(n1)))
        return fail(c, SPH_ENOMEM, "host staging of %lld particles", (long long)n);
    // the positions are checked while they are copied; nothing is kept on failure
    if (stage_copy(P.pos.data(), pos, n3, 1, 0.0) != 0) return fail(c, SPH_EINVAL, "non-finite position");
    if (vel) stage_copy(P.vel.data(), vel, n3, 0, 0.0);
    if (nrm) stage_copy(P.nrm.data(), nrm, n3, 0, 0.0);
    if (T) stage_copy(P.T.data(), T, n1, 0, 0.0);
    if (rho) stage_copy(P.rho.data(), rho, n1, 2, M.rho0);
    if (first_id) *first_id = n0;
    c->blocks.push_back(std::move(P));
    c->n_total += n;
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
    if (c->started || c->admitted) return fail(c, SPH_ESTATE, "rotation is fixed after the first step");
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

// A single-case context is an engine with capacity for exactly its particles.
static sph_status single_engine(sph_ctx* c) {
    if (c->started) return SPH_OK;
    if (c->admitted) return fail(c, SPH_ESTATE, "this context was admitted to a batch");
    if (c->n_total == 0) return fail(c, SPH_ESTATE, "no particles");
    Engine* E = new Engine();
    E->stream = c->stream;
    E->B.tune_batch = c->tune_batch;
    E->B.tune_tpp = c->tune_tpp;
    E->B.tune_block = c->tune_block;
    E->B.uni_fluid = single_fluid_material(c) ? 1 : 0;
    E->B.fp64 = c->cfg.pair_precision == 1 ? 1 : 0;
    const int64_t nc = (int64_t)c->ncell[0] * c->ncell[1] * c->ncell[2];
    sph_status r = engine_alloc(*E, c->n_total, 1, nc, 4096);
    int slot = -1;
    if (r == SPH_OK) r = engine_admit(*E, c, 0, &slot);
    if (r == SPH_OK) r = prepare(*E);
    if (r == SPH_OK) r = capture(*E);
    if (r != SPH_OK) {
        c->err = E->err;
        delete E;
        return r;
    }
    c->eng = E;
    c->started = true;
    std::vector<PBlock>().swap(c->blocks);  // the engine holds the particles now
    return SPH_OK;
}

static sph_status relay(sph_ctx* c, sph_status s) {
    if (s != SPH_OK && c->eng) c->err = c->eng->err;
    return s;
}

#define STARTED_OR_STATE(c)                                                   \
    do {                                                                      \
        if (!(c)) return SPH_EINVAL;                                          \
        if (!(c)->started) return fail((c), SPH_ESTATE, "no step taken yet"); \
    } while (0)

extern "C" {

sph_status sph_step(sph_ctx* c, int n_steps, double* t_out) {
    if (!c) return SPH_EINVAL;
    if (n_steps < 0) return fail(c, SPH_EINVAL, "n_steps < 0");
    sph_status s = single_engine(c);
    if (s != SPH_OK) return s;
    Engine& E = *c->eng;
    s = engine_step(E, n_steps);
    if (s != SPH_OK) return relay(c, s);
    if (t_out) *t_out = E.st_h[0].t;
    if (E.st_h[0].err)
        return fail(c, SPH_EUNSTABLE, "unstable state (error bits 0x%x: 1 = NaN/Inf, 2 = fluid left the box)",
                    E.st_h[0].err);
    return SPH_OK;
}

sph_status sph_read_torque_heat(sph_ctx* c, int b, double* tq, double* tq_avg, double* heat, double* meanT) {
    STARTED_OR_STATE(c);
    return relay(c, read_torque_heat(*c->eng, 0, b, tq, tq_avg, heat, meanT));
}

sph_status sph_read_curve(sph_ctx* c, double* out, int64_t max_steps, int64_t* n_out) {
    STARTED_OR_STATE(c);
    return relay(c, read_curve(*c->eng, 0, out, max_steps, n_out));
}

sph_status sph_read_fields(sph_ctx* c, int field, void* dst, int64_t n) {
    STARTED_OR_STATE(c);
    return relay(c, read_fields(*c->eng, 0, field, dst, n));
}

sph_status sph_read_neighbors(sph_ctx* c, int64_t* counts, int32_t* ids, int64_t cap, int64_t* total) {
    STARTED_OR_STATE(c);
    if (c->eng->graph_steps == 0) return fail(c, SPH_ESTATE, "no neighbour search before the first step");
    if (!counts) return fail(c, SPH_EINVAL, "counts is NULL");
    Engine& E = *c->eng;
    const int64_t n = E.cases[0].n;
    const int idb = (int)E.cases[0].id_base;
    int64_t* d_cnt = nullptr;
    if (cudaMalloc(&d_cnt, sizeof(int64_t) * (n + 1)) != cudaSuccess) return fail(c, SPH_ENOMEM, "neighbour counts");
    cudaError_t e = launch_neighbors(E.B, E.parity ^ 1, 0, idb, d_cnt, nullptr, nullptr, E.stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(counts, d_cnt, sizeof(int64_t) * n, cudaMemcpyDeviceToHost, E.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(E.stream);
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
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_cnt, start.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, E.stream);
    if (e == cudaSuccess) e = launch_neighbors(E.B, E.parity ^ 1, 0, idb, nullptr, d_cnt, d_list, E.stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ids, d_list, sizeof(int32_t) * start[n], cudaMemcpyDeviceToHost, E.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(E.stream);
    cudaFree(d_list);
    cudaFree(d_cnt);
    if (e != cudaSuccess) return fail(c, SPH_ECUDA, "neighbour list: %s", cudaGetErrorString(e));
    for (int64_t i = 0; i < n; ++i) std::sort(ids + start[i], ids + start[i + 1]);
    return SPH_OK;
}

sph_status sph_read_cell_order(sph_ctx* c, int64_t* perm, int64_t n) {
    STARTED_OR_STATE(c);
    if (c->eng->graph_steps == 0) return fail(c, SPH_ESTATE, "no cell sort before the first step");
    Engine& E = *c->eng;
    if (!perm || n != E.cases[0].n) return fail(c, SPH_EINVAL, "n must equal the particle count");
    std::vector<int> ids(n);
    const int lo = E.st_h[0].seg_lo;
    if (cudaMemcpyAsync(ids.data(), E.B.ID[E.parity] + lo, sizeof(int) * n, cudaMemcpyDeviceToHost, E.stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(E.stream) != cudaSuccess)
        return fail(c, SPH_ECUDA, "cell order read-back failed");
    for (int64_t k = 0; k < n; ++k) perm[k] = ids[k] - E.cases[0].id_base;
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
    info->graph_launches = kernels_per_advection_step(c->kcap, c->cfg.pair_precision == 1);
    kernels_in_step(c->cfg.pair_precision == 1, true, &info->kernels_fixed, &info->kernels_per_substep);
    info->kernels_per_substep += 1;  // the loop condition
    if (c->started) {
        Engine& E = *c->eng;
        sph_status s = pull_state(E);
        if (s != SPH_OK) return relay(c, s);
        const CaseState& S = E.st_h[0];
        info->t = S.t;
        info->adv_steps = S.adv_steps;
        info->substeps = S.substeps;
        info->last_dt_ad = S.last_dt_ad;
        info->last_nsub = S.last_nsub;
        info->error_bits = S.err;
        info->info_bits = S.err_info;
    }
    return SPH_OK;
}

sph_status sph_pair_stats(sph_ctx* c, int64_t* fluid_fluid, int64_t* fluid_wall) {
    STARTED_OR_STATE(c);
    if (c->eng->graph_steps == 0) return fail(c, SPH_ESTATE, "no neighbour search before the first step");
    if (!fluid_fluid || !fluid_wall) return SPH_EINVAL;
    Engine& E = *c->eng;
    unsigned long long* d = nullptr;
    unsigned long long h[2] = {0, 0};
    if (cudaMalloc(&d, sizeof h) != cudaSuccess) return fail(c, SPH_ENOMEM, "pair stats");
    cudaError_t e = cudaMemsetAsync(d, 0, sizeof h, E.stream);
    if (e == cudaSuccess) e = launch_pair_stats(E.B, d, E.stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, d, sizeof h, cudaMemcpyDeviceToHost, E.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(E.stream);
    cudaFree(d);
    if (e != cudaSuccess) return fail(c, SPH_ECUDA, "pair stats: %s", cudaGetErrorString(e));
    *fluid_fluid = (int64_t)h[0];
    *fluid_wall = (int64_t)h[1];
    return SPH_OK;
}

sph_status sph_search_stats(sph_ctx* c, int64_t* searched, int64_t* candidates, int64_t* partners) {
    STARTED_OR_STATE(c);
    if (c->eng->graph_steps == 0) return fail(c, SPH_ESTATE, "no neighbour search before the first step");
    if (!searched || !candidates || !partners) return SPH_EINVAL;
    Engine& E = *c->eng;
    unsigned long long* d = nullptr;
    unsigned long long h[3] = {0, 0, 0};
    if (cudaMalloc(&d, sizeof h) != cudaSuccess) return fail(c, SPH_ENOMEM, "search stats");
    cudaError_t e = cudaMemsetAsync(d, 0, sizeof h, E.stream);
    if (e == cudaSuccess) e = launch_search_stats(E.B, d, E.stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, d, sizeof h, cudaMemcpyDeviceToHost, E.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(E.stream);
    cudaFree(d);
    if (e != cudaSuccess) return fail(c, SPH_ECUDA, "search stats: %s", cudaGetErrorString(e));
    *searched = (int64_t)h[0];
    *candidates = (int64_t)h[1];
    *partners = (int64_t)h[2];
    return SPH_OK;
}

// Kernel-variant knobs: validation and the engine field each one sets.
static const char* tuning_check(int key, int value) {
    switch (key) {
    case SPH_TUNE_LIST_BATCH:
        return (value == 1 || value == 2 || value == 4 || value == 8) ? nullptr : "list batch must be 1, 2, 4 or 8";
    case SPH_TUNE_TPP: return (value == 1 || value == 2) ? nullptr : "threads per particle must be 1 or 2";
    case SPH_TUNE_BLOCK:
        return (value == 64 || value == 128 || value == 256) ? nullptr : "block size must be 64, 128 or 256";
    default: return "unknown tuning key";
    }
}

static int* tuning_field(Bufs& B, int key) {
    return key == SPH_TUNE_LIST_BATCH ? &B.tune_batch : key == SPH_TUNE_TPP ? &B.tune_tpp : &B.tune_block;
}

sph_status sph_set_tuning(sph_ctx* c, int key, int value) {
    if (!c) return SPH_EINVAL;
    if (const char* m = tuning_check(key, value)) return fail(c, SPH_EINVAL, "%s (key %d, value %d)", m, key, value);
    int* f = key == SPH_TUNE_LIST_BATCH ? &c->tune_batch : key == SPH_TUNE_TPP ? &c->tune_tpp : &c->tune_block;
    *f = value;
    if (!c->started) return SPH_OK;
    Engine& E = *c->eng;
    *tuning_field(E.B, key) = value;
    if (cudaStreamSynchronize(E.stream) != cudaSuccess) return fail(c, SPH_ECUDA, "sync failed");
    return relay(c, capture(E));
}

sph_status sph_get_tuning(sph_ctx* c, int key, int* value) {
    if (!c || !value) return SPH_EINVAL;
    switch (key) {
    case SPH_TUNE_LIST_BATCH: *value = c->tune_batch; return SPH_OK;
    case SPH_TUNE_TPP: *value = c->tune_tpp; return SPH_OK;
    case SPH_TUNE_BLOCK: *value = c->tune_block; return SPH_OK;
    default: return fail(c, SPH_EINVAL, "unknown tuning key %d", key);
    }
}

static sph_status engine_profile(Engine& E, int enable) {
    E.prof = enable != 0;
    for (int k = 0; k < SPH_PROF_NCLASS; ++k) {
        E.prof_ms[k] = 0.0;
        E.prof_cnt[k] = 0;
    }
    E_CUDA(E, cudaStreamSynchronize(E.stream));
    return capture(E);
}

static void engine_profile_read(Engine& E, double* ms, int64_t* launches, int reset) {
    for (int k = 0; k < SPH_PROF_NCLASS; ++k) {
        ms[k] = E.prof_ms[k];
        launches[k] = E.prof_cnt[k];
        if (reset) {
            E.prof_ms[k] = 0.0;
            E.prof_cnt[k] = 0;
        }
    }
}

// Autotuner: coordinate descent over the pair-pass variants (list batch,
// threads per particle, block size), each timed over real advection steps
// with the profiling events: score = (D + VT) per advection step + the
// reference number of sub-steps x (M + C) per sub-step, so trials at
// different sub-step counts compare fairly.  The first step after each
// re-capture is not timed.
static sph_status engine_autotune(Engine& E, int steps_per_trial, sph_tune_report* rep) {
    if (steps_per_trial < 1) return E.fail(SPH_EINVAL, "steps per trial must be >= 1");
    const bool prof0 = E.prof;
    double nsub_ref = -1.0;
    int64_t steps = 0;
    int trials = 0;
    auto score = [&](double* out) -> sph_status {
        sph_status r = engine_profile(E, 1);
        if (r == SPH_OK) r = engine_step(E, 1);
        if (r != SPH_OK) return r;
        double ms[SPH_PROF_NCLASS];
        int64_t cnt[SPH_PROF_NCLASS];
        engine_profile_read(E, ms, cnt, 1);
        r = engine_step(E, steps_per_trial);
        if (r != SPH_OK) return r;
        engine_profile_read(E, ms, cnt, 1);
        steps += 1 + steps_per_trial;
        ++trials;
        if (cnt[SPH_PROF_PASS_M] == 0 || cnt[SPH_PROF_PASS_C] == 0)
            return E.fail(SPH_ESTATE, "no running case to time");
        if (nsub_ref < 0.0) nsub_ref = (double)cnt[SPH_PROF_PASS_M] / steps_per_trial;
        *out = (ms[SPH_PROF_PASS_D] + ms[SPH_PROF_PASS_VT]) / steps_per_trial +
               nsub_ref * (ms[SPH_PROF_PASS_M] / cnt[SPH_PROF_PASS_M] + ms[SPH_PROF_PASS_C] / cnt[SPH_PROF_PASS_C]);
        return SPH_OK;
    };
    static const int keys[3] = {SPH_TUNE_LIST_BATCH, SPH_TUNE_TPP, SPH_TUNE_BLOCK};
    static const int vals[3][4] = {{8, 4, 2, 1}, {1, 2, 0, 0}, {128, 64, 256, 0}};
    int best[3];
    for (int k = 0; k < 3; ++k) best[k] = *tuning_field(E.B, keys[k]);
    double s_start = 0.0, s_best = 0.0;
    sph_status r = score(&s_start);
    s_best = s_start;
    for (int k = 0; k < 3 && r == SPH_OK; ++k) {
        const int scored = best[k];  // this key's value in the best variant so far: already timed
        for (int v = 0; v < 4 && r == SPH_OK; ++v) {
            const int val = vals[k][v];
            if (val == 0 || val == scored) continue;
            for (int q = 0; q < 3; ++q) *tuning_field(E.B, keys[q]) = best[q];
            *tuning_field(E.B, keys[k]) = val;
            double sc = 0.0;
            r = score(&sc);
            if (r == SPH_OK && sc < s_best) {
                s_best = sc;
                best[k] = val;
            }
        }
    }
    for (int q = 0; q < 3; ++q) *tuning_field(E.B, keys[q]) = best[q];
    const sph_status r2 = engine_profile(E, prof0 ? 1 : 0);
    if (r != SPH_OK) return r;
    if (rep) {
        rep->list_batch = best[0];
        rep->tpp = best[1];
        rep->block = best[2];
        rep->ms_step_start = s_start;
        rep->ms_step_chosen = s_best;
        rep->substeps_ref = nsub_ref;
        rep->trials = trials;
        rep->steps = steps;
    }
    return r2;
}

sph_status sph_autotune(sph_ctx* c, int steps_per_trial, sph_tune_report* report) {
    if (!c) return SPH_EINVAL;
    sph_status r = single_engine(c);
    if (r != SPH_OK) return r;
    sph_tune_report rep{};
    r = relay(c, engine_autotune(*c->eng, steps_per_trial, &rep));
    c->tune_batch = c->eng->B.tune_batch;
    c->tune_tpp = c->eng->B.tune_tpp;
    c->tune_block = c->eng->B.tune_block;
    if (report) *report = rep;
    return r;
}

sph_status sph_profile(sph_ctx* c, int enable) {
    STARTED_OR_STATE(c);
    return relay(c, engine_profile(*c->eng, enable));
}

sph_status sph_profile_read(sph_ctx* c, double* ms, int64_t* launches, int reset) {
    if (!c || !ms || !launches) return SPH_EINVAL;
    STARTED_OR_STATE(c);
    engine_profile_read(*c->eng, ms, launches, reset);
    return SPH_OK;
}

sph_status sph_cell_sort(const double* pos, int64_t n, const double origin[3], const double cellw[3],
                         const int ncell[3], int32_t* perm, int32_t* cell_start, void* stream) {
    if (n < 0 || (n > 0 && (!pos || !perm)) || !origin || !cellw || !ncell || !cell_start) {
        sph::set_stateless_error("sph_cell_sort: null pointer or negative n");
        return SPH_EINVAL;
    }
    if (n > ((int64_t)1 << 31) - 1) {
        sph::set_stateless_error("sph_cell_sort: n >= 2^31");
        return SPH_EINVAL;
    }
    // the running product is checked after every factor, so it never overflows
    int64_t nc = 1;
    for (int a = 0; a < 3; ++a) {
        if (ncell[a] < 1 || !(cellw[a] > 0)) {
            sph::set_stateless_error("sph_cell_sort: ncell must be >= 1 and cellw > 0");
            return SPH_EINVAL;
        }
        nc *= ncell[a];
        if (nc > ((int64_t)1 << 30)) {
            sph::set_stateless_error("sph_cell_sort: more than 2^30 cells");
            return SPH_EINVAL;
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    const size_t nb = scan_blocks((int)nc) + 1;
    const size_t bytes = sizeof(uint32_t) * ((size_t)3 * (n > 0 ? n : 1) + (size_t)nc + nb);
    void* scratch = nullptr;
    if (cudaMallocAsync(&scratch, bytes, s) != cudaSuccess) {
        sph::set_stateless_error("sph_cell_sort: scratch allocation failed");
        return SPH_ENOMEM;
    }
    uint32_t* keys = (uint32_t*)scratch;
    uint32_t* rank = keys + (n > 0 ? n : 1);
    uint32_t* tmp = rank + (n > 0 ? n : 1);
    uint32_t* cnt = tmp + (n > 0 ? n : 1);
    uint32_t* blk = cnt + nc;
    cudaError_t e = launch_cell_sort(pos, (int)n, origin, cellw, ncell, keys, rank, cnt, tmp, blk, perm,
                                     cell_start, s);
    cudaError_t e2 = cudaFreeAsync(scratch, s);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        sph::set_stateless_error("sph_cell_sort: kernel launch failed");
        return SPH_ECUDA;
    }
    return SPH_OK;
}

// ----------------------------------------------------------- batch C ABI ---

int64_t sph_batch_bytes(const sph_batch_config* cfg) {
    if (!cfg) return -1;
    return cfg->max_particles * kBytesPerParticle + cfg->max_cells * kBytesPerCell +
           (int64_t)cfg->max_cases * (int64_t)(sizeof(CaseDev) + sizeof(CaseState) + 64 * (int64_t)cfg->history_steps);
}

sph_status sph_batch_create(const sph_batch_config* cfg, void* stream, sph_batch** out) {
    if (!cfg || !out) return SPH_EINVAL;
    *out = nullptr;
    sph_batch* b = new sph_batch();
    b->eng.stream = (cudaStream_t)stream;
    b->eng.B.tune_batch = 2;
    b->eng.B.uni_fluid = 1;  // batched cases carry a single fluid material
    sph_status s = engine_alloc(b->eng, cfg->max_particles, cfg->max_cases, cfg->max_cells, cfg->history_steps);
    if (s != SPH_OK) {
        sph::set_stateless_error(b->eng.err.c_str());
        delete b;
        return s;
    }
    *out = b;
    return SPH_OK;
}

sph_status sph_batch_destroy(sph_batch* b) {
    delete b;
    return SPH_OK;
}

const char* sph_batch_last_error(const sph_batch* b) { return b ? b->eng.err.c_str() : sph::g_stateless_err.c_str(); }

sph_status sph_batch_admit(sph_batch* b, sph_ctx* staged, int64_t n_steps, int* slot) {
    if (!b || !staged || n_steps < 0) return SPH_EINVAL;
    Engine& E = b->eng;
    if (staged->started || staged->admitted) return E.fail(SPH_ESTATE, "case was already stepped or admitted");
    if (!single_fluid_material(staged)) return E.fail(SPH_EINVAL, "batched cases need a single fluid material");
    if (staged->cfg.pair_precision != 0) return E.fail(SPH_EINVAL, "batched cases use FP32 pair arithmetic");
    sph_status s = engine_admit(E, staged, n_steps, slot);
    if (s == SPH_OK) staged->admitted = true;
    return s;
}

sph_status sph_batch_step(sph_batch* b, int n_steps) {
    if (!b || n_steps < 0) return SPH_EINVAL;
    return engine_step(b->eng, n_steps);
}

static sph_status batch_slot(sph_batch* b, int slot) {
    if (!b) return SPH_EINVAL;
    if (slot < 0 || slot >= b->eng.c_cap || !b->eng.cases[slot].used || b->eng.cases[slot].retiring)
        return b->eng.fail(SPH_EINVAL, "slot %d is not a resident case", slot);
    return SPH_OK;
}

sph_status sph_batch_poll(sph_batch* b, int slot, int64_t* steps_done, double* sim_time, int* state) {
    sph_status s = batch_slot(b, slot);
    if (s != SPH_OK) return s;
    const CaseState& S = b->eng.st_h[slot];
    if (steps_done) *steps_done = S.adv_steps;
    if (sim_time) *sim_time = S.t;
    if (state) *state = S.err ? SPH_BATCH_UNSTABLE : (S.running ? SPH_BATCH_RUNNING : SPH_BATCH_DONE);
    return SPH_OK;
}

sph_status sph_batch_read_torque_heat(sph_batch* b, int slot, int body, double* tq, double* tq_avg, double* heat,
                                      double* meanT) {
    sph_status s = batch_slot(b, slot);
    if (s != SPH_OK) return s;
    return read_torque_heat(b->eng, slot, body, tq, tq_avg, heat, meanT);
}

sph_status sph_batch_read_curve(sph_batch* b, int slot, double* out, int64_t max_steps, int64_t* n_out) {
    sph_status s = batch_slot(b, slot);
    if (s != SPH_OK) return s;
    return read_curve(b->eng, slot, out, max_steps, n_out);
}

sph_status sph_batch_read_fields(sph_batch* b, int slot, int field, void* host_dst, int64_t n) {
    sph_status s = batch_slot(b, slot);
    if (s != SPH_OK) return s;
    if (b->eng.need_prepare) return b->eng.fail(SPH_ESTATE, "step the batch after admitting or retiring");
    return read_fields(b->eng, slot, field, host_dst, n);
}

sph_status sph_batch_retire(sph_batch* b, int slot) {
    sph_status s = batch_slot(b, slot);
    if (s != SPH_OK) return s;
    Engine& E = b->eng;
    HostCase& H = E.cases[slot];
    if (H.pending) return E.fail(SPH_ESTATE, "step the batch once after admitting before retiring");
    H.retiring = true;
    E.need_prepare = true;
    return SPH_OK;
}

sph_status sph_batch_info(sph_batch* b, int64_t* n_particles, int* n_cases, int* kernels_per_step) {
    if (!b) return SPH_EINVAL;
    Engine& E = b->eng;
    int nc = 0;
    int64_t np = 0;
    for (const HostCase& H : E.cases)
        if (H.used && !H.retiring) {
            ++nc;
            np += H.n;
        }
    if (n_particles) *n_particles = np;
    if (n_cases) *n_cases = nc;
    if (kernels_per_step) *kernels_per_step = engine_kernels_per_step(E);
    return SPH_OK;
}

sph_status sph_batch_set_tuning(sph_batch* b, int key, int value) {
    if (!b) return SPH_EINVAL;
    Engine& E = b->eng;
    if (const char* m = tuning_check(key, value)) return E.fail(SPH_EINVAL, "%s (key %d, value %d)", m, key, value);
    *tuning_field(E.B, key) = value;
    E.graph_dirty = true;
    return SPH_OK;
}

sph_status sph_batch_autotune(sph_batch* b, int steps_per_trial, sph_tune_report* report) {
    if (!b) return SPH_EINVAL;
    sph_tune_report rep{};
    const sph_status r = engine_autotune(b->eng, steps_per_trial, &rep);
    if (report) *report = rep;
    return r;
}

sph_status sph_batch_profile(sph_batch* b, int enable) {
    if (!b) return SPH_EINVAL;
    return engine_profile(b->eng, enable);
}

sph_status sph_batch_profile_read(sph_batch* b, double* ms, int64_t* launches, int reset) {
    if (!b || !ms || !launches) return SPH_EINVAL;
    engine_profile_read(b->eng, ms, launches, reset);
    return SPH_OK;
}

}  // extern "C"
