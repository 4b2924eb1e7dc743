// Internal declarations shared by the CUDA translation units of the library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstddef>
#include <utility>

#include "mdpd.h"

namespace mdpd {

// Device status bits, OR-ed by kernels into one word and mapped to MDPD_ERR_*.
enum : uint32_t {
    ST_NONFINITE = 1u,
    ST_OUT_OF_BOX = 2u,
    ST_OVERFLOW = 4u,
    ST_TIMEOUT = 8u,
    ST_BOUNDS = 16u,     // an index check of the debug build failed
};

// Index checks of the debug build (compiled with -DMDPD_DEBUG): a computed
// index outside its array sets ST_BOUNDS in the status word and the access is
// skipped (never a trap).  In the release build the check is the constant
// true and costs nothing.
#ifdef MDPD_DEBUG
#define MDPD_DBG_OK(cond, status) ((cond) ? true : (atomicOr((status), ::mdpd::ST_BOUNDS), false))
#else
#define MDPD_DBG_OK(cond, status) true
#endif

// Cell lattice and box (edge h >= r_c on every axis; x fastest).
struct Geo {
    int nc[3];
    int periodic[3];
    double lo[3], L[3], hi[3], h[3], inv_h[3];
    int64_t key_lo[3], key_hi[3];   // f64_key(lo), f64_key(hi): face comparisons in integers
    int64_t key_in[3];              // f64_key of a bound below hi: lo <= x below it implies
                                    //   0 <= RN(x - lo) < L (a loaded position needs no wrap)
    int64_t ncell;
};

// Constants derived from Phys and Geo in the precision of the pair
// arithmetic, computed once on the host (FP64 arithmetic runs at a small
// fraction of the FP32 rate on this part, so kernels must not rederive them
// per thread).
template <typename T>
struct Derived {
    T rc2, rd2, inv_rc, inv_rd;
    T cw_rho;        // 15 / (2 pi r_d^3): density weight normalisation (Sec. 2.1)
    T cw_phi;        // 15 / (2 pi r_c^3): wall-density weight normalisation
    T inv_sqrt_dt;   // random force scale 1 / sqrt(dt)
    T h[3];          // cell edges
    T hdt;           // dt / 2
    T g[3];          // body force
    T lo[3];         // box origin
    T inv_h[3];      // 1 / cell edge
    T c0[3];         // centre of cell 0: lo + h / 2
    T h_lo[3];       // FP32: h - h, c0 - c0 in FP64, rounded (h, c0 as FP32 pairs);
    T c0_lo[3];      //   FP64: zero
    T fix_scale;     // 2^e: density terms as integers (frozen split), with
    T fix_inv;       //   cw_rho * 2^e <= 2^31 (FP32) or 2^50 (FP64); and 2^-e
};

// Physical constants of Sec. 2.1 / Eq. 1, tables flattened [ti * 8 + tj].
struct Phys {
    double rc, rd, dt, hdt, kT;
    double g[3];
    uint32_t frozen;
    int ntypes;
    int xi_dist;
    int rho_self;
    int list_all;                 // 1: the density pass lists partners of frozen particles too
    int list_compact;             // 1: list column = block base + compacted mobile position
                                  //    (frozen-split density pass and rounds force pass)
    int prec32;                   // 1: FP32 pair arithmetic (kick increments formed in FP32)
    uint32_t fast_cell;           // bit k: axis k may take cell indices in FP32 (see k_bin_count)
    void* phi_out;                // wall density output (cell order, FP32/FP64), or nullptr
    uint32_t* dbg_status;         // the handle's status word (index checks of the debug build)
    uint32_t key0, key1;          // Philox key = (seed_lo, seed_hi)
    uint32_t rk[10][2];           // its ten round keys (key + r * Weyl increments; set_keys)
    Derived<float> df;
    Derived<double> dd;
    double A[64], B[64], gamma[64], sigma[64];   // keep last: a batch copies what precedes A
};

template <typename T>
__host__ __device__ __forceinline__ const Derived<T>& derived(const Phys& ph);
template <>
__host__ __device__ __forceinline__ const Derived<float>& derived<float>(const Phys& ph) { return ph.df; }
template <>
__host__ __device__ __forceinline__ const Derived<double>& derived<double>(const Phys& ph) { return ph.dd; }

// Fill ph.df and ph.dd from ph (rc, rd, dt) and the cell edges.
inline void fill_derived(Phys& ph, const Geo& geo)
{
    const double pi = 3.14159265358979323846;
    Derived<double>& d = ph.dd;
    d.rc2 = ph.rc * ph.rc;
    d.rd2 = ph.rd * ph.rd;
    d.inv_rc = 1.0 / ph.rc;
    d.inv_rd = 1.0 / ph.rd;
    d.cw_rho = 15.0 / (2.0 * pi * ph.rd * ph.rd * ph.rd);
    d.cw_phi = 15.0 / (2.0 * pi * ph.rc * ph.rc * ph.rc);
    d.inv_sqrt_dt = ph.dt > 0.0 ? 1.0 / std::sqrt(ph.dt) : 0.0;
    for (int k = 0; k < 3; ++k) d.h[k] = geo.h[k];
    d.hdt = 0.5 * ph.dt;
    ph.fast_cell = 0;
    for (int k = 0; k < 3; ++k) {
        d.g[k] = ph.g[k];
        d.lo[k] = geo.lo[k];
        d.inv_h[k] = geo.inv_h[k];
        d.c0[k] = geo.lo[k] + 0.5 * geo.h[k];
        // FP32 cell index: few cells and coordinates of moderate size in cell
        // units, so that the FP32 error stays below 4e-4 cell edges
        const double span = (std::fabs(geo.lo[k]) + geo.L[k]) * geo.inv_h[k];
        if (geo.nc[k] <= 1024 && span <= 2048.0) ph.fast_cell |= 1u << k;
    }
    // fixed-point scale of the frozen split's scattered density terms (each
    // at most cw_rho): a power of two, so the scaling is exact
    const int e64 = (int)std::floor(std::log2(std::ldexp(1.0, 50) / d.cw_rho));
    const int e32 = (int)std::floor(std::log2(std::ldexp(1.0, 31) / d.cw_rho));
    d.fix_scale = std::ldexp(1.0, e64);
    d.fix_inv = std::ldexp(1.0, -e64);
    Derived<float>& f = ph.df;
    f.fix_scale = (float)std::ldexp(1.0, e32);
    f.fix_inv = (float)std::ldexp(1.0, -e32);
    f.rc2 = (float)d.rc2;
    f.rd2 = (float)d.rd2;
    f.inv_rc = (float)d.inv_rc;
    f.inv_rd = (float)d.inv_rd;
    f.cw_rho = (float)d.cw_rho;
    f.cw_phi = (float)d.cw_phi;
    f.inv_sqrt_dt = (float)d.inv_sqrt_dt;
    for (int k = 0; k < 3; ++k) f.h[k] = (float)d.h[k];
    f.hdt = (float)d.hdt;
    for (int k = 0; k < 3; ++k) {
        f.g[k] = (float)d.g[k];
        f.lo[k] = (float)d.lo[k];
        f.inv_h[k] = (float)d.inv_h[k];
        f.c0[k] = (float)d.c0[k];
        f.h_lo[k] = (float)(d.h[k] - (double)f.h[k]);
        f.c0_lo[k] = (float)(d.c0[k] - (double)f.c0[k]);
        d.h_lo[k] = 0.0;
        d.c0_lo[k] = 0.0;
    }
}

// One member of a batch of independent systems: its box and cell lattice,
// the global index of its first cell and of its first particle, and its
// physical constants.  Kernels of a batch map each block to one chunk of one
// replica and copy the replica's record to shared memory.
struct alignas(16) Rep {
    Geo geo;
    int64_t cell0;      // first cell of the replica in the concatenated lattice
    uint32_t id0;       // first particle id (= first slot) of the replica
    uint32_t n;         // particles of the replica
    alignas(16) Phys ph;
};
static_assert(offsetof(Rep, ph) % 16 == 0 && sizeof(Rep) % 16 == 0, "Rep is copied in 16-byte words");

// Kernel-side view of a batch.  Particles of replica r always occupy the
// slots [reps[r].id0, reps[r].id0 + reps[r].n), in every ordering, so the
// work can be cut into chunks that never straddle two replicas:
//   chunks[b]  = (replica, first slot, count <= 128, 0)   for particle kernels
//   cchunks[b] = (replica, first cell, count <= 4, 0)     for cell kernels
struct Batch {
    const Rep* reps;
    const int4* chunks;
    const int4* cchunks;
    int nchunk, ncchunk;
};

constexpr int BATCH_CHUNK = 128;       // particles per chunk
constexpr int BATCH_CELL_CHUNK = 4;    // cells per chunk (warps of the cell kernel)

// Solid-voxel reflection mask (1 bit per voxel, x fastest); bits == nullptr
// means no mask.
struct MaskDev {
    const uint32_t* bits;
    int dim[3];
    double voxel;
    double inv_voxel;      // 1 / voxel
    int inv_voxel_exact;   // voxel is a power of two: t * inv_voxel == t / voxel
    double origin[3];
    // FP32 voxel index (see drift_reflect): allowed when the mask and the box
    // span at most 1024 voxels per axis and 2048 voxels from coordinate 0
    int fast;
    float origin_f[3];
    float inv_voxel_f;
};

// Master particle state, component-major: x[k * cap + i].
struct Master {
    double* x;
    double* v;
    double* a;
    uint32_t* id;
    uint8_t* type;
};

// Force-pass modes.
enum ForceMode : int {
    FM_EVAL = 0,    // write sum_j F_ij + g to `out`; no integration
    FM_LAST = 1,    // second half-kick: v(t+dt) = v + dt/2 a; store a
    FM_FUSED = 2,   // second half-kick, then the next step's half-kick,
                    // drift and reflection
};

// Programmatic dependent launch: every kernel of the time step is launched
// with programmatic stream serialisation, so it can be scheduled while the
// previous kernel drains; it waits for the previous grid's completion and
// memory (griddepcontrol.wait) before touching any data, then lets its own
// dependent be scheduled (griddepcontrol.launch_dependents).
__device__ __forceinline__ void pdl_enter()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl_smem(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                                   cudaStream_t st, Args&&... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, cudaStream_t st,
                              Args&&... args)
{
    return launch_pdl_smem(kern, grid, block, 0, st, std::forward<Args>(args)...);
}

// The replica record of this block's chunk, copied in part to dynamic shared
// memory (the launch provides REP_SMEM bytes): REP_GEO copies the geometry
// (everything before ph), REP_SCALARS also the scalar constants of ph (not the
// per-type-pair tables, which a kernel that needs them reads from reps[r]).
enum RepPart { REP_GEO = 0, REP_SCALARS = 1 };
__host__ __device__ constexpr size_t rep_part_bytes(int part)
{
    return ((part == REP_GEO ? offsetof(Rep, ph) : offsetof(Rep, ph) + offsetof(Phys, A)) + 15) / 16 * 16;
}
constexpr size_t REP_SMEM = rep_part_bytes(REP_SCALARS);

template <int PART>
__device__ __forceinline__ const Rep& block_rep(const Rep* __restrict__ reps, int r)
{
    extern __shared__ uint4 rep_smem[];
    constexpr int words = (int)(rep_part_bytes(PART) / sizeof(uint4));
    const uint4* src = reinterpret_cast<const uint4*>(reps + r);
    for (int k = threadIdx.x; k < words; k += blockDim.x) rep_smem[k] = src[k];
    __syncthreads();
    return *reinterpret_cast<const Rep*>(rep_smem);
}

constexpr int OBS_PARTIALS = 16;   // observable slots per partial (14 used)

// ---- launchers (binning / scan) -------------------------------------------
// Cell of every particle from the master positions m.x, and its arrival rank
// in the cell (atomic order); kick: first the step's first half-kick, drift
// and reflection.  tsum (scan_num_blocks(ncell) words, zero on entry) receives
// the scan's per-tile sums of the counts.
void launch_bin_count(cudaStream_t st, int n, int64_t cap, const Geo& geo, const Phys& ph,
                      const MaskDev& mk, const Master& m, bool kick, uint32_t* cellof,
                      uint32_t* slot, uint32_t* count, uint32_t* tsum, uint32_t* status);
int scan_num_blocks(int64_t n);
// Whether the binning of a lattice of n cells forms the scan's tile sums in
// its count kernel (few tiles) or in a launch of their own.
bool scan_fused_sums(int64_t n);
// Launches of the binning's scan.
int scan_num_launches(int64_t n);
// Exclusive scan of in[0..n) into out[0..n]; tmp holds scan_num_blocks(n) + 1
// words; zero_in clears in[] after it is read.
void launch_exclusive_scan(cudaStream_t st, uint32_t* in, int64_t n, uint32_t* out, uint32_t* tmp,
                           bool zero_in = false);
// The same for any n, as scans of segments of at most seg elements (seg within
// the two-level scan's limit) joined by a running carry: tmp holds
// scan_num_blocks(seg) + 1 words and carry one word.
void launch_exclusive_scan_long(cudaStream_t st, uint32_t* in, int64_t n, uint32_t* out,
                                uint32_t* tmp, uint32_t* carry, int64_t seg);
// The same in one launch, given the tile sums (from launch_bin_count); the
// counts are cleared as they are read, and so is zero_sums (the other tile-sum
// buffer, for the next binning).
void launch_scan_from_sums(cudaStream_t st, uint32_t* in, int64_t n, uint32_t* out,
                           const uint32_t* sums, uint32_t* zero_sums);
// For every scattered slot a: the particle's place s in its cell (rank of
// key[a] = frozen << 31 | id among the cell's keys), and the gather of master
// state in[src[a]] to out[s] with the cell-ordered compute arrays (pos4, vel4,
// cell_s).
void launch_rank_gather(cudaStream_t st, int precision, int n, int64_t cap,
                        const uint32_t* cellof, const uint32_t* start, const uint32_t* key,
                        const uint32_t* src, const Master& in, const Master& out, bool gather_a,
                        const Geo& geo, const Phys& ph, void* pos4, void* vel4, uint32_t* cell_s);
void launch_rank_gather_batch(cudaStream_t st, int precision, int64_t cap, const uint32_t* cellof,
                              const uint32_t* start, const uint32_t* key, const uint32_t* src,
                              const Master& in, const Master& out, bool gather_a, const Batch& bt,
                              void* pos4, void* vel4, uint32_t* cell_s);
void launch_bin_scatter(cudaStream_t st, int n, const uint32_t* cellof, const uint32_t* slot,
                        const uint32_t* start, const uint32_t* id, uint32_t* key, uint32_t* src,
                        uint32_t* status);
// Sorts each cell's slots by key and clears count[] for the next binning.
void launch_cell_sort(cudaStream_t st, int64_t ncell, const uint32_t* start, uint32_t* key,
                      uint32_t* src, uint32_t* count);

// ---- launchers (pair passes) -----------------------------------------------
void launch_density(cudaStream_t st, int precision, int n, const Geo& geo, const Phys& ph,
                    const void* pos4, const uint32_t* cell_s, const uint32_t* start, void* rho);
void launch_force(cudaStream_t st, int precision, ForceMode mode, int n, int64_t cap,
                  const Geo& geo, const Phys& ph, const MaskDev& mk, const void* pos4,
                  const void* vel4, const void* rho, const uint32_t* cell_s,
                  const uint32_t* start, const uint64_t* step_ptr, int step_offset,
                  const Master& m, double* out, double* partials, uint32_t* status);
// Blocks of a force launch over n particles at lpp lanes per particle, each
// block taking `rounds` rounds of its particles (see force_nl_rounds).
int force_num_blocks(int n, int lpp = 1, int rounds = 1);
// Number of per-warp observable partials the force pass writes for n particles.
int obs_num_partials(int n, int lpp = 1, int rounds = 1);
// Rounds per block of the list force pass of a single system (FORCE_ROUNDS
// with frozen particles at one lane per particle, else 1).
constexpr int FORCE_ROUNDS = 4;
int force_nl_rounds(const Phys& ph, int lpp);
// Density pass that also writes the force partners of mobile particles
// (entries (j << 5) | image code, slot-major: nl[k * cap + column] with the
// column of ph.list_compact; nl_count[i] by slot).
// fs (frozen split; id_s the cell-ordered ids, rho_ff cap values of the
// pass's type indexed by id, facc cap fixed-point accumulators in cell order,
// zero between passes): 0 full scans; 2 writes the frozen-frozen part of
// every frozen particle's density to rho_ff (-1 for mobile ids); 1 scans for
// mobile homes only, which scatter their terms to frozen candidates into
// facc, and a second launch forms the frozen densities and clears facc.
void launch_density_nl(cudaStream_t st, int precision, int n, int64_t cap, const Geo& geo,
                       const Phys& ph, const void* pos4, const uint32_t* cell_s,
                       const uint32_t* start, void* rho, uint32_t* nl, uint32_t* nl_count,
                       int fs = 0, unsigned long long* facc = nullptr,
                       const uint32_t* id_s = nullptr, void* rho_ff = nullptr, int shape = 0);
// Warp-per-cell variant of launch_density_nl (same outputs).
void launch_density_cell(cudaStream_t st, int precision, int64_t ncell, int64_t cap,
                         const Geo& geo, const Phys& ph, const void* pos4, const uint32_t* start,
                         void* rho, uint32_t* nl, uint32_t* nl_count);
// lpp: lanes per particle (1, 2 or 4).
void launch_force_nl(cudaStream_t st, int precision, ForceMode mode, int n, int64_t cap,
                     const Geo& geo, const Phys& ph, int lpp, const MaskDev& mk, const void* pos4,
                     const void* vel4, const void* rho, const uint32_t* cell_s,
                     const uint32_t* start, const uint32_t* nl, const uint32_t* nl_count,
                     const uint64_t* step_ptr, int step_offset, const Master& m, double* out,
                     double* partials, uint32_t* status);
constexpr int NL_SLOTS = 64;      // must equal NL_MAX of the kernels
// Level-one blocks of the observable reduction for nparts partials.
int reduce_l1_blocks(int nparts);
// Reduction of the per-warp partials (stored as FP32 when precision = 1, FP64
// otherwise; l1: NOBS * reduce_l1_blocks values of that type; ticket: one
// zero-initialised counter, left at zero).
void launch_reduce_obs(cudaStream_t st, int precision, const double* partials, int nparts,
                       double* l1, unsigned* ticket, double* obs, double* obs_sum,
                       double* obs_count, uint64_t* step_ptr, int advance);

// ---- launchers (batch of replicas; see Batch) ------------------------------
constexpr int OBS_STRIDE = 2 * MDPD_NUM_OBS + 2;   // per-replica observable record
void launch_load_state_batch(cudaStream_t st, int64_t cap, const double* pos3, const double* vel3,
                             const double* acc3, const Batch& bt, const Master& m,
                             const uint8_t* type_by_id, uint32_t* status);
void launch_bin_count_batch(cudaStream_t st, int64_t cap, const Batch& bt, const Master& m,
                            bool kick, uint32_t* cellof, uint32_t* slot, uint32_t* count,
                            uint32_t* tsum, uint32_t* status);
// shape: code shape of the thread-per-particle kernel (0 or 1; same results).
void launch_density_nl_batch(cudaStream_t st, int precision, int64_t cap, const Batch& bt,
                             const void* pos4, const uint32_t* cell_s, const uint32_t* start,
                             void* rho, uint32_t* nl, uint32_t* nl_count, int shape = 0);
void launch_density_cell_batch(cudaStream_t st, int precision, int64_t cap, const Batch& bt,
                               const void* pos4, const uint32_t* start, void* rho, uint32_t* nl,
                               uint32_t* nl_count);
// Partials: 4 per chunk (bt.nchunk * 4 in all).
void launch_force_nl_batch(cudaStream_t st, int precision, ForceMode mode, int64_t cap,
                           const Batch& bt, const void* pos4, const void* vel4, const void* rho,
                           const uint32_t* cell_s, const uint32_t* start, const uint32_t* nl,
                           const uint32_t* nl_count, const uint64_t* step_ptr, int step_offset,
                           const Master& m, double* out, double* partials, uint32_t* status);
// wr[r] = the range of partials of replica r; obs holds nrep * OBS_STRIDE doubles.
void launch_reduce_obs_batch(cudaStream_t st, int precision, const double* partials, int nparts,
                             const int2* wr, int nrep, unsigned* ticket, double* obs,
                             uint64_t* step_ptr, int advance);

// ---- launchers (adjoint) ---------------------------------------------------
// All take bt = nullptr for a single system (blocks of PAIR_BLOCK slots) or a
// batch (one block per chunk).  Vectors in id order are interleaved xyz;
// cell-ordered outputs are component-major [3][cap].
// Blocks of a VJP launch (entries of tpart / TB).
int vjp_num_blocks(int n, const Batch* bt);
// VJP of one force evaluation at the current cell-ordered state (lists built
// with list_all): abar (id order, may be NULL) the adjoint of the
// accelerations, wbar (6 per replica, may be NULL) weights of the virial
// components; xbar, ubar, rbar outputs in cell order; tpart[block][3 * 64]
// the blocks' parameter partials by (parameter, own type, partner type).
void launch_force_vjp(cudaStream_t st, int precision, int n, int64_t cap, const Geo& geo,
                      const Phys& ph, const Batch* bt, const void* pos4, const void* vel4,
                      const void* rho, const uint32_t* cell_s, const uint32_t* start,
                      const uint32_t* nl, const uint32_t* nl_count, const uint64_t* step_ptr,
                      const double* abar, const double* wbar, double* xbar, double* ubar,
                      double* rbar, double* tpart, uint32_t* status);
// The density chain: xbar (cell order, [3][cap]) += sum_j (rbar_i + rbar_j)
// w_rho'(r) e over partners within r_d (rbar in cell order).
void launch_density_vjp(cudaStream_t st, int precision, int n, int64_t cap, const Geo& geo,
                        const Phys& ph, const Batch* bt, const void* pos4,
                        const uint32_t* cell_s, const uint32_t* start, const uint32_t* nl,
                        const uint32_t* nl_count, const double* rbar, double* xbar,
                        uint32_t* status);
void launch_gather_by_id(cudaStream_t st, int n, const uint32_t* id, const double* in, double* out,
                         int add);
// *step_ptr = value, ordered on the stream.
void launch_set_step(cudaStream_t st, uint64_t* step_ptr, uint64_t value);
constexpr int THETA_SLOTS = 3 * 64;   // [parameter][type][type] of A, B, gamma
// Per replica: acc[r] (= or +=) the sum of its blocks' partials in block
// order; ranges[r] / scale = the replica's block range (NULL: all nblk).
void launch_theta_reduce(cudaStream_t st, int nrep, int nblk, const int2* ranges, int scale,
                         const double* tpart, double* acc, int add);
// Symmetric-table gradient [r][3][8][8] from the per-type-pair sums.
void launch_theta_symmetrise(cudaStream_t st, int nrep, const double* acc, double* out);
// Window checkpoints, start of the reverse sweep, and one reverse step's
// chain rule (see k_adjoint.cu).
void launch_win_record(cudaStream_t st, int n, int64_t cap, const Phys& ph, const Batch* bt,
                       const Master& m, double* X, double* VH);
void launch_win_init(cudaStream_t st, int n, const Phys& ph, const Batch* bt, const Master& m,
                     const double* xbar, const double* vbar, double* xb, double* vb, double* ab);
void launch_win_post(cudaStream_t st, int n, int64_t cap, const Phys& ph, const Batch* bt,
                     const Master& m, const double* gx, const double* gu, double* xb, double* vb,
                     double* ab, int first, int final, double* x0bar, double* v0bar);

// ---- launchers (walls) -----------------------------------------------------
void launch_mask_pack(cudaStream_t st, const uint8_t* mask, int64_t nvox, uint32_t* bits);
void launch_wall_count(cudaStream_t st, const uint8_t* mask, const int dim[3], const int per[3],
                       int R, int64_t R2, double lam, uint32_t key0, uint32_t key1,
                       uint32_t* count);
void launch_wall_emit(cudaStream_t st, const uint8_t* mask, const int dim[3],
                      const uint32_t* count, const uint32_t* offset, double voxel,
                      const double origin[3], uint32_t key0, uint32_t key1, int64_t base,
                      int64_t cap, const Master& m, uint8_t wall_type);

// ---- misc --------------------------------------------------------------------
void launch_scatter_by_id(cudaStream_t st, int n, int64_t cap, const uint32_t* id,
                          const double* vec3, double* out3);
void launch_scatter_scalar_by_id(cudaStream_t st, int precision, int n, const uint32_t* id,
                                 const void* rho_sorted, double* out);
void launch_scatter_type_by_id(cudaStream_t st, int n, const uint32_t* id, const uint8_t* type,
                               int32_t* out);
// Master state in id order from pos3, vel3 and (if not NULL) acc3, all
// interleaved xyz; periodic axes wrapped.
// Set *moved (device word, not cleared here) to 1 if a frozen particle's
// loaded position (master arrays indexed by id, as k_load_state leaves them)
// differs in any bit from ref (n x 3, by id), the positions the frozen-frozen
// density part was computed from.
void launch_frozen_moved(cudaStream_t st, int n, int64_t cap, const double* x, const double* ref,
                         const uint8_t* type_by_id, uint32_t frozen, uint32_t* moved);
void launch_load_state(cudaStream_t st, int n, int64_t cap, const double* pos3,
                       const double* vel3, const double* acc3, const Geo& geo, const Master& m,
                       const uint8_t* type_by_id, uint32_t* status);

}  // namespace mdpd
