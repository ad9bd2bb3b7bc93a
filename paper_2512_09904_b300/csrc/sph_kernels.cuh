// sph_kernels.cuh -- buffer table and launchers shared by the engine and the kernels.
#pragma once
#include "sph_internal.cuh"

namespace sph {

constexpr int RED_CHUNK = 4096;  // slots per fixed-order reduction chunk
constexpr int SCAN_TILE = 2048;  // cells per scan tile
constexpr int TQ_CHUNK = 2048;   // body ids per torque partial sum

// All device buffers of one engine (pointers only; passed by value).
struct Bufs {
    int n;             // particle slots in use
    int ncases;
    int ncells;        // cell index space of all cases; key ncells is the bucket of dead particles
    int max_chunks;       // capacity of the chunk table
    int max_chunks_used;  // chunks that the resident particles can need
    int hist_cap;
    CaseDev* cases;
    CaseState* st;
    double *X[3], *Y[3];
    float4* V[2];
    float* DR[2];
    double* T64[2];
    int* ID[2];
    uint32_t* TAG[2];
    float* T32;
    float4* SNAP;
    uint32_t* CELLK;
    float4* AV;
    float4* NRM;
    double* RP[3];
    float4* RN;
    float* TORQ;
    float* TORQV;
    double* CF;     // per-id contact factor of rigid-body particles (Eq. 24), last advection step
    uint32_t *KEYS, *RANK, *TMP, *PERM, *CNT, *CSTART, *SCANBLK;
    double* PART;
    int* CHUNK_CASE;
    int* nchunks;     // chunks in use (written by the cell sort)
    double* HIST;
    uint32_t* NB;   // neighbour lists, NB_CAP slots of nb_stride entries
    uint32_t* NBC;  // per-slot list counts
    int nb_stride;
    int* OVFL;      // slots whose partners overflowed their list (this step)
    int* novf;      // number of entries in OVFL
    float4* VH;     // (v, half-kicked drho) input of pass M
    int4* TQC;      // torque chunks: (case, body, id_lo, id_hi), TQ_CHUNK ids each
    int2* TQR;      // per (case, body): (first chunk, chunks)
    double* TQP;    // chunk partial sums (pressure, viscous)
    int ntq;        // chunks in use
    int uni_fluid;  // every case has a single fluid material
    int visc_heat;  // some resident case adds viscous-dissipation heating
    int tune_batch; // list entries loaded together per thread in the pair passes (1, 2, 4, 8)
    int tune_tpp;   // threads per particle in the list passes VT, M, C (1 or 2)
    int tune_block; // block size of the pair passes (64, 128, 256)
    // FP64 pair arithmetic (fp64 = 1): particle state in FP64 beside the
    // FP32 arrays above, which then only carry tags, snapshot offsets and lists
    int fp64;
    // the single resident case (its pair constants are entry 0 of the pair
    // passes' PairTab), or -1
    int one_case;
    double4_32a* V64[2];  // (vx, vy, vz, rho - rho0)
    double* DR64[2];
    double4_32a* VH64;
    double4_32a* AV64;    // (viscous acceleration, dT/dt)
    double4_32a* NRM64;   // wall normals at the advection step, slot order
    double4_32a* RN64;    // reference normals, by id
    double* TORQ64;   // per-id pressure torque
    double* TORQV64;  // per-id viscous torque
};

// launchers (stream-ordered; all return the launch error)
cudaError_t launch_vmax_init(const Bufs& B, int par, int lo, int hi, cudaStream_t s);
// a staged block of a new case into the packed arrays (device inputs; null = default)
cudaError_t launch_admit_block(const Bufs& B, int par, int n, int at, int idb, uint32_t tag, int fluid, double rho0,
                               double T_init, const double* pos, const double* vel, const double* nrm, const double* T,
                               const double* rho, cudaStream_t s);
cudaError_t launch_adv_begin(const Bufs& B, cudaStream_t s);
cudaError_t launch_sort(const Bufs& B, int par, cudaStream_t s);  // hash..reorder + segments
// pair passes: T holds the pair constants of the resident cases (PairTab)
cudaError_t launch_passD(const Bufs& B, int par, const PairTab& T, cudaStream_t s);
cudaError_t launch_passVT(const Bufs& B, int par, const PairTab& T, cudaStream_t s);
cudaError_t launch_sub_begin(const Bufs& B, cudaStream_t s);
cudaError_t launch_passM(const Bufs& B, int par, const PairTab& T, cudaStream_t s);  // first sub-step: decided on the device
cudaError_t launch_passC(const Bufs& B, int par, const PairTab& T, cudaStream_t s);
cudaError_t launch_sub_end(const Bufs& B, cudaStream_t s);
cudaError_t launch_adv_end(const Bufs& B, int par, cudaStream_t s);
cudaError_t launch_reduce_heat(const Bufs& B, int par, cudaStream_t s);
cudaError_t launch_block_heat0(const Bufs& B, int cur, int slot, int at, int n, double* part, cudaStream_t s);
cudaError_t launch_gather_field(const Bufs& B, int par, int field, int cs, int id_base, double* out,
                                cudaStream_t s);
cudaError_t launch_neighbors(const Bufs& B, int par, int cs, int id_base, int64_t* counts_by_id,
                             const int64_t* start_by_id, int32_t* list, cudaStream_t s);
int kernels_per_advection_step(int kcap, bool fp64);  // unrolled graph with kcap sub-step slots
// Kernels of one advection step: fixed part and per sub-step (the loop graph
// adds its condition kernel per sub-step).
void kernels_in_step(bool fp64, bool torque, int* fixed, int* per_substep);
cudaError_t launch_sub_cond(const Bufs& B, cudaGraphConditionalHandle h, cudaStream_t s);
cudaError_t launch_pair_stats(const Bufs& B, unsigned long long* out, cudaStream_t s);
cudaError_t launch_search_stats(const Bufs& B, unsigned long long* out, cudaStream_t s);

// FP64 pair passes (sph_kernels64.cu)
cudaError_t launch_passD64(const Bufs& B, int par, cudaStream_t s);
cudaError_t launch_passVT64(const Bufs& B, int par, cudaStream_t s);
cudaError_t launch_passM64(const Bufs& B, int par, cudaStream_t s);
cudaError_t launch_passC64(const Bufs& B, int par, cudaStream_t s);

// stateless cell sort (positions AoS)
cudaError_t launch_cell_sort(const double* pos, int n, const double origin[3], const double cellw[3],
                             const int ncell[3], uint32_t* keys, uint32_t* rank, uint32_t* cnt,
                             uint32_t* tmp, uint32_t* scanblk, int32_t* perm, int32_t* cell_start,
                             cudaStream_t s);
size_t scan_blocks(int ncells);

}  // namespace sph
