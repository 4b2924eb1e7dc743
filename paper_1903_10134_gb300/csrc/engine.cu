// Host side of the C ABI (include/mdpd.h): owns the device state of one mDPD
// system, validates arguments, enqueues the kernels of a time step on the
// handle's stream (directly or as a captured CUDA graph) and moves data in
// and out in particle-id order.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "f64bits.cuh"
#include "mdpd_internal.cuh"
#include "philox.cuh"
#include "vec.cuh"

using namespace mdpd;

namespace {

constexpr int64_t MAX_PARTICLES = int64_t(1) << 27;   // neighbour-list entries hold j << 5
constexpr int64_t MAX_SCAN = int64_t(4096) * 4096;   // limit of the two-level scan
constexpr int EV_PER_STEP = 5;                        // profile events per step
constexpr int PAIR_BLOCK_WARPS = 4;                   // observable partials per force block

std::string g_create_error;

struct Graphs {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t ev_node[EV_PER_STEP] = {};
};

}  // namespace

struct mdpd_handle {
    mdpd_params p{};
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    // a step's observable reduction runs, deferred, on a side stream beside
    // the next step's binning and density pass
    cudaStream_t side = nullptr;
    cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
    bool pending = false;            // the last step's reduction is still to run
    uint64_t seed = 0;
    int precision = 1;
    int64_t n = 0, n_user = 0, cap = 0;
    Geo geo{};
    Phys ph{};
    MaskDev mk{};

    // master state, ping-pong between binnings
    double* x[2] = {};
    double* v[2] = {};
    double* a[2] = {};
    uint32_t* id[2] = {};
    uint8_t* type[2] = {};
    int cur = 0;
    // cell-ordered compute arrays
    void* pos4 = nullptr;
    void* vel4 = nullptr;
    void* rho = nullptr;
    uint32_t* cell_s = nullptr;
    // binning
    uint32_t *count = nullptr, *start = nullptr, *cellof = nullptr, *slot = nullptr;
    uint32_t *key = nullptr, *src = nullptr, *scan_tmp = nullptr;
    // the scan's per-tile sums of the counts, formed by the count kernel; two
    // buffers of scan_num_blocks(ncell) words used by binning parity (cur)
    uint32_t* tile_sums = nullptr;
    // frozen-frozen part of each frozen particle's density, by id (constant
    // while the frozen particles and r_d stay; recomputed when ff_dirty)
    void* rho_ff = nullptr;
    unsigned long long* facc = nullptr;  // cap fixed-point density sums of the frozen split
    bool ff_dirty = true;
    // positions (by id, n x 3) the frozen-frozen part was computed from, and a
    // device word that set_state raises when a loaded frozen position differs
    double* ffx = nullptr;
    uint32_t* ff_moved = nullptr;
    // misc
    uint32_t* status = nullptr;
    uint64_t* step = nullptr;
    double* partials = nullptr;
    double* red_l1 = nullptr;        // level-one partials of the reduction
    unsigned* red_ticket = nullptr;  // last-block ticket of the reduction
    double* obs = nullptr;       // MDPD_NUM_OBS current, then MDPD_NUM_OBS sums, then count
    double* fout = nullptr;      // 3 * cap staging / force output
    uint8_t* type_by_id = nullptr;
    uint32_t* mask_bits = nullptr;
    uint32_t* nl = nullptr;          // NL_SLOTS * cap neighbour-list entries
    uint32_t* nl_count = nullptr;    // cap
    void* phi = nullptr;             // cap wall densities (cell order)
    bool want_phi = false;
    int kernels = MDPD_KERNELS_NLIST;
    int force_lpp = 1;               // lanes per particle of the force pass (single system)
    int thread_shape = 0;            // code shape of the thread-per-particle density kernel
    bool walls_set = false;
    std::vector<int32_t> h_type;
    int64_t steps_host = 0;

    // graphs[profiled][mode: 0 fused, 1 last][cur][first half-kick in the binning]
    //       [previous step's reduction pending]
    bool use_graph = true;
    Graphs g[2][2][2][2][2];
    Graphs gm[2];                    // MULTI_STEPS fused steps in one graph, by cur
    cudaEvent_t tev[EV_PER_STEP] = {};

    // profiling ring
    int64_t prof_cap = 0, prof_used = 0;
    int64_t prof_every = 1, prof_tick = 0;   // record events on every prof_every-th step
    std::vector<cudaEvent_t> prof_ev;
    int64_t prof_launches = 0;

    // batch of independent replicas (nrep > 0; see Batch): host records,
    // device records and chunk tables, per-replica observable records
    int nrep = 0;
    std::vector<Rep> reps;
    std::vector<mdpd_params> rep_p;
    Rep* d_reps = nullptr;
    int4* d_chunks = nullptr;
    int4* d_cchunks = nullptr;
    int2* d_wr = nullptr;
    double* obs_b = nullptr;
    Rep* d_reps_all = nullptr;       // the same records with list_all set (adjoint lists)
    int nchunk = 0, ncchunk = 0;

    // adjoint: per-block parameter partials and per-replica sums, virial
    // weights, and a velocity-Verlet window's checkpoints (id order:
    // x_0..x_K, v'_0..v'_{K-1}, v_0) and reverse-sweep vectors (xb, vb, ab)
    double* vjp_tpart = nullptr;
    double* vjp_tacc = nullptr;
    double* vjp_wbar = nullptr;
    double* win_x = nullptr;
    double* win_vh = nullptr;
    double* win_v0 = nullptr;
    double* win_b = nullptr;
    int64_t win_alloc_steps = 0;     // steps the checkpoint arrays hold
    size_t win_vec = 0;              // 3N they were sized for
    int vjp_nblk = 0;                // blocks vjp_tpart was sized for
    int64_t win_k = 0, win_s0 = 0;
    bool win_valid = false;

    Batch batch(bool all = false) const
    {
        Batch b;
        b.reps = all && d_reps_all ? d_reps_all : d_reps;
        b.chunks = d_chunks;
        b.cchunks = d_cchunks;
        b.nchunk = nchunk;
        b.ncchunk = ncchunk;
        return b;
    }

    std::string err;

    int fail(int code, const std::string& msg)
    {
        err = msg;
        return code;
    }
};

#define CK(call)                                                                         \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return h->fail(MDPD_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

namespace {

template <typename P>
int dalloc(mdpd_handle* h, P** ptr, size_t bytes)
{
    *ptr = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc((void**)ptr, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *ptr = nullptr;
        return h->fail(MDPD_ERR_OOM, std::string("cudaMalloc(") + std::to_string(bytes) +
                                         "): " + cudaGetErrorString(e));
    }
    return MDPD_OK;
}

template <typename P>
void dfree(P*& ptr)
{
    if (ptr) cudaFree((void*)ptr);
    ptr = nullptr;
}

Master master(mdpd_handle* h, int k)
{
    Master m;
    m.x = h->x[k];
    m.v = h->v[k];
    m.a = h->a[k];
    m.id = h->id[k];
    m.type = h->type[k];
    return m;
}

void free_particles(mdpd_handle* h)
{
    for (int k = 0; k < 2; ++k) {
        dfree(h->x[k]);
        dfree(h->v[k]);
        dfree(h->a[k]);
        dfree(h->id[k]);
        dfree(h->type[k]);
    }
    dfree(h->pos4);
    dfree(h->vel4);
    dfree(h->rho);
    dfree(h->cell_s);
    dfree(h->cellof);
    dfree(h->slot);
    dfree(h->key);
    dfree(h->src);
    dfree(h->partials);
    dfree(h->red_l1);
    dfree(h->fout);
    dfree(h->type_by_id);
    dfree(h->nl);
    dfree(h->nl_count);
    dfree(h->phi);
    dfree(h->rho_ff);
    dfree(h->facc);
    dfree(h->ffx);
    dfree(h->ff_moved);
}

int alloc_particles(mdpd_handle* h, int64_t cap)
{
    const size_t c = (size_t)(cap > 0 ? cap : 1);
    const size_t tsz = h->precision == 0 ? sizeof(double) : sizeof(float);
    const size_t v4 = h->precision == 0 ? sizeof(D4) : sizeof(float4);
    int rc = MDPD_OK;
    for (int k = 0; k < 2 && rc == MDPD_OK; ++k) {
        if ((rc = dalloc(h, &h->x[k], 3 * c * sizeof(double)))) break;
        if ((rc = dalloc(h, &h->v[k], 3 * c * sizeof(double)))) break;
        if ((rc = dalloc(h, &h->a[k], 3 * c * sizeof(double)))) break;
        if ((rc = dalloc(h, &h->id[k], c * sizeof(uint32_t)))) break;
        if ((rc = dalloc(h, &h->type[k], c))) break;
    }
    if (!rc) rc = dalloc(h, &h->pos4, c * v4);
    if (!rc) rc = dalloc(h, &h->vel4, c * v4);
    if (!rc) rc = dalloc(h, &h->rho, c * tsz);
    if (!rc) rc = dalloc(h, &h->cell_s, c * sizeof(uint32_t));
    if (!rc) rc = dalloc(h, &h->cellof, c * sizeof(uint32_t));
    if (!rc) rc = dalloc(h, &h->slot, c * sizeof(uint32_t));
    if (!rc) rc = dalloc(h, &h->key, c * sizeof(uint32_t));
    if (!rc) rc = dalloc(h, &h->src, c * sizeof(uint32_t));
    const size_t nparts = std::max((size_t)obs_num_partials((int)c, 4), (size_t)h->nchunk * (PAIR_BLOCK_WARPS));
    if (!rc) rc = dalloc(h, &h->partials, nparts * OBS_PARTIALS * sizeof(double));
    if (!rc) rc = dalloc(h, &h->red_l1, (size_t)(reduce_l1_blocks(obs_num_partials((int)c, 4)) + 1) * OBS_PARTIALS * sizeof(double));
    if (!rc) rc = dalloc(h, &h->fout, 3 * c * sizeof(double));
    if (!rc) rc = dalloc(h, &h->type_by_id, c);
    if (!rc) rc = dalloc(h, &h->nl, (size_t)NL_SLOTS * c * sizeof(uint32_t));
    if (!rc) rc = dalloc(h, &h->nl_count, c * sizeof(uint32_t));
    if (!rc) rc = dalloc(h, &h->phi, c * tsz);
    if (!rc) rc = dalloc(h, &h->rho_ff, c * tsz);
    if (!rc) rc = dalloc(h, &h->facc, c * sizeof(unsigned long long));
    if (!rc && !h->nrep) rc = dalloc(h, &h->ffx, 3 * c * sizeof(double));
    if (!rc && h->ffx) rc = dalloc(h, &h->ff_moved, sizeof(uint32_t));
    if (!rc && cudaMemset(h->facc, 0, c * sizeof(unsigned long long)) != cudaSuccess)
        rc = h->fail(MDPD_ERR_CUDA, "cudaMemset of the frozen-split sums failed");
    if (!rc && cudaDeviceSynchronize() != cudaSuccess)
        rc = h->fail(MDPD_ERR_CUDA, "cudaDeviceSynchronize after allocation failed");
    if (!rc) h->cap = (int64_t)c;
    return rc;
}

// Exchange every per-particle array (and the capacity) of two handles.
void swap_particle_arrays(mdpd_handle* a, mdpd_handle* b)
{
    for (int k = 0; k < 2; ++k) {
        std::swap(a->x[k], b->x[k]);
        std::swap(a->v[k], b->v[k]);
        std::swap(a->a[k], b->a[k]);
        std::swap(a->id[k], b->id[k]);
        std::swap(a->type[k], b->type[k]);
    }
    std::swap(a->pos4, b->pos4);
    std::swap(a->vel4, b->vel4);
    std::swap(a->rho, b->rho);
    std::swap(a->cell_s, b->cell_s);
    std::swap(a->cellof, b->cellof);
    std::swap(a->slot, b->slot);
    std::swap(a->key, b->key);
    std::swap(a->src, b->src);
    std::swap(a->partials, b->partials);
    std::swap(a->red_l1, b->red_l1);
    std::swap(a->fout, b->fout);
    std::swap(a->type_by_id, b->type_by_id);
    std::swap(a->nl, b->nl);
    std::swap(a->nl_count, b->nl_count);
    std::swap(a->phi, b->phi);
    std::swap(a->rho_ff, b->rho_ff);
    std::swap(a->facc, b->facc);
    std::swap(a->ffx, b->ffx);
    std::swap(a->ff_moved, b->ff_moved);
    std::swap(a->cap, b->cap);
}

void destroy_graphs(mdpd_handle* h)
{
    for (auto& gg : h->gm) {
        if (gg.exec) cudaGraphExecDestroy(gg.exec);
        if (gg.graph) cudaGraphDestroy(gg.graph);
        gg = Graphs();
    }
    for (auto& a : h->g)
        for (auto& b : a)
            for (auto& c : b)
                for (auto& d : c)
                    for (auto& gg : d) {
                        if (gg.exec) cudaGraphExecDestroy(gg.exec);
                        if (gg.graph) cudaGraphDestroy(gg.graph);
                        gg = Graphs();
                    }
}

bool is_fin(double x) { return std::isfinite(x); }

int validate_params(const mdpd_params* p, std::string& why)
{
    if (!p) { why = "params is NULL"; return MDPD_ERR_INVALID_ARG; }
    if (p->ntypes < 1 || p->ntypes > MDPD_MAX_TYPES) { why = "ntypes must be in 1..8"; return MDPD_ERR_INVALID_ARG; }
    if (!(p->rc > 0) || !is_fin(p->rc)) { why = "rc must be > 0"; return MDPD_ERR_INVALID_ARG; }
    if (!(p->rd > 0) || !(p->rd <= p->rc)) { why = "rd must be in (0, rc]"; return MDPD_ERR_INVALID_ARG; }
    if (!(p->dt > 0) || !is_fin(p->dt)) { why = "dt must be > 0"; return MDPD_ERR_INVALID_ARG; }
    if (!(p->kT >= 0) || !is_fin(p->kT)) { why = "kT must be >= 0"; return MDPD_ERR_INVALID_ARG; }
    if (p->precision != 0 && p->precision != 1) { why = "precision must be 0 or 1"; return MDPD_ERR_INVALID_ARG; }
    if (p->xi_dist != 0 && p->xi_dist != 1) { why = "xi_dist must be 0 or 1"; return MDPD_ERR_INVALID_ARG; }
    for (int k = 0; k < 3; ++k) {
        if (!(p->box[k] > 0) || !is_fin(p->box[k]) || !is_fin(p->box_lo[k])) {
            why = "box lengths must be finite and > 0";
            return MDPD_ERR_INVALID_ARG;
        }
        if (p->periodic[k] && p->box[k] < 3.0 * p->rc) {
            why = "a periodic axis must be at least 3 rc long";
            return MDPD_ERR_INVALID_ARG;
        }
        if (!is_fin(p->g[k])) { why = "g must be finite"; return MDPD_ERR_INVALID_ARG; }
    }
    for (int a = 0; a < MDPD_MAX_TYPES; ++a)
        for (int b = 0; b < MDPD_MAX_TYPES; ++b) {
            if (!is_fin(p->A[a][b]) || !is_fin(p->B[a][b]) || !is_fin(p->gamma[a][b]) ||
                p->gamma[a][b] < 0) {
                why = "pair tables must be finite with gamma >= 0";
                return MDPD_ERR_INVALID_ARG;
            }
            if (a < p->ntypes && b < p->ntypes &&
                (p->A[a][b] != p->A[b][a] || p->B[a][b] != p->B[b][a] ||
                 p->gamma[a][b] != p->gamma[b][a])) {
                why = "pair tables must be symmetric";
                return MDPD_ERR_INVALID_ARG;
            }
        }
    return MDPD_OK;
}

void make_geo_phys(const mdpd_params& p, uint64_t seed, Geo& g, Phys& f)
{
    g.ncell = 1;
    for (int k = 0; k < 3; ++k) {
        int m = (int)std::floor(p.box[k] / p.rc);
        if (m < 1) m = 1;
        g.nc[k] = m;
        g.periodic[k] = p.periodic[k] ? 1 : 0;
        g.lo[k] = p.box_lo[k];
        g.L[k] = p.box[k];
        g.hi[k] = p.box_lo[k] + p.box[k];
        g.key_lo[k] = f64_key(g.lo[k]);
        g.key_hi[k] = f64_key(g.hi[k]);
        // below hi by twice the spacing of doubles near the larger face: for
        // lo <= x < hi_in the difference x - lo rounds to [0, L)
        const double big = std::max(std::fabs(g.lo[k]), std::fabs(g.hi[k]));
        const double hi_in = g.hi[k] - 2.0 * (std::nextafter(big, HUGE_VAL) - big);
        g.key_in[k] = f64_key(hi_in > g.lo[k] ? hi_in : g.lo[k]);
        g.h[k] = p.box[k] / m;
        g.inv_h[k] = 1.0 / g.h[k];
        g.ncell *= m;
    }
    f.rc = p.rc;
    f.rd = p.rd;
    f.dt = p.dt;
    f.hdt = 0.5 * p.dt;
    f.kT = p.kT;
    for (int k = 0; k < 3; ++k) f.g[k] = p.g[k];
    f.frozen = p.frozen_type_mask & 0xFFu;
    f.ntypes = p.ntypes;
    f.xi_dist = p.xi_dist;
    f.rho_self = p.rho_self ? 1 : 0;
    f.prec32 = p.precision == 1 ? 1 : 0;
    f.key0 = (uint32_t)seed;
    f.key1 = (uint32_t)(seed >> 32);
    philox_round_keys(f.key0, f.key1, f.rk);
    for (int a = 0; a < 8; ++a)
        for (int b = 0; b < 8; ++b) {
            f.A[a * 8 + b] = p.A[a][b];
            f.B[a * 8 + b] = p.B[a][b];
            f.gamma[a * 8 + b] = p.gamma[a][b];
            f.sigma[a * 8 + b] = std::sqrt(2.0 * p.gamma[a][b] * p.kT);
        }
    fill_derived(f, g);
}

void setup_geo_phys(mdpd_handle* h)
{
    const int list_all = h->ph.list_all;
    h->geo = Geo{};
    h->ph = Phys{};
    make_geo_phys(h->p, h->seed, h->geo, h->ph);
    h->ph.list_all = list_all;
    h->ph.dbg_status = h->status;
}

int status_to_code(uint32_t st)
{
    if (st & ST_BOUNDS) return MDPD_ERR_BOUNDS;      // (a failed check can cause the rest)
    if (st & ST_NONFINITE) return MDPD_ERR_NONFINITE;
    if (st & ST_OUT_OF_BOX) return MDPD_ERR_OUT_OF_BOX;
    if (st & ST_OVERFLOW) return MDPD_ERR_TILE_OVERFLOW;
    if (st & ST_TIMEOUT) return MDPD_ERR_TIMEOUT;
    return MDPD_OK;
}

// Synchronise the stream and turn the device status word into an error code
// (the word is cleared).
void flush_pending(mdpd_handle* h);

int sync_check(mdpd_handle* h)
{
    flush_pending(h);
    CK(cudaStreamSynchronize(h->stream));
    uint32_t st = 0;
    CK(cudaMemcpy(&st, h->status, sizeof(st), cudaMemcpyDeviceToHost));
    if (st) {
        CK(cudaMemset(h->status, 0, sizeof(uint32_t)));
        const int code = status_to_code(st);
        const char* what = code == MDPD_ERR_NONFINITE     ? "non-finite position, velocity or force"
                           : code == MDPD_ERR_OUT_OF_BOX   ? "a particle left a non-periodic box"
                           : code == MDPD_ERR_TILE_OVERFLOW ? "cell tile overflow"
                           : code == MDPD_ERR_BOUNDS ? "an index check of the debug build failed"
                                                            : "device wait timed out";
        return h->fail(code, what);
    }
    return MDPD_OK;
}

// ---- one time step, as a sequence of launches ---------------------------------

void record(mdpd_handle* h, cudaEvent_t* evs, int k)
{
    // external record: inside a stream capture this becomes an event-record node
    if (evs) cudaEventRecordWithFlags(evs[k], h->stream, cudaEventRecordExternal);
}

// Bin: (first half-kick and drift,) count, scan, scatter, rank inside each
// cell by id, gather into the other buffer.
void enqueue_bin(mdpd_handle* h, bool gather_a, bool kick = false)
{
    cudaStream_t st = h->stream;
    const int n = (int)h->n;
    // count[] and this parity's tile sums are zero here: cleared at creation
    // and by every scan (which clears the other parity's tile sums)
    const int64_t nb = scan_num_blocks(h->geo.ncell);
    const bool fused = scan_fused_sums(h->geo.ncell);
    uint32_t* tsum = fused ? h->tile_sums + (size_t)h->cur * nb : nullptr;
    uint32_t* tsum_next = h->tile_sums + (size_t)(1 - h->cur) * nb;
    if (h->nrep)
        launch_bin_count_batch(st, h->cap, h->batch(), master(h, h->cur), kick, h->cellof,
                               h->slot, h->count, tsum, h->status);
    else
        launch_bin_count(st, n, h->cap, h->geo, h->ph, h->mk, master(h, h->cur), kick, h->cellof,
                         h->slot, h->count, tsum, h->status);
    if (fused)
        launch_scan_from_sums(st, h->count, h->geo.ncell, h->start, tsum, tsum_next);
    else
        launch_exclusive_scan(st, h->count, h->geo.ncell, h->start, h->scan_tmp, true);
    launch_bin_scatter(st, n, h->cellof, h->slot, h->start, h->id[h->cur], h->key, h->src,
                       h->status);
    if (h->nrep)
        launch_rank_gather_batch(st, h->precision, h->cap, h->cellof, h->start, h->key, h->src,
                                 master(h, h->cur), master(h, 1 - h->cur), gather_a, h->batch(),
                                 h->pos4, h->vel4, h->cell_s);
    else
        launch_rank_gather(st, h->precision, n, h->cap, h->cellof, h->start, h->key, h->src,
                           master(h, h->cur), master(h, 1 - h->cur), gather_a, h->geo, h->ph,
                           h->pos4, h->vel4, h->cell_s);
    h->cur = 1 - h->cur;
}

bool use_split(const mdpd_handle* h);

// Kernel launches of one time step (enqueue_step): count, scan, scatter,
// rank + gather, density (two under the frozen split), force, reduction.
int step_launches(const mdpd_handle* h)
{
    return 6 + scan_num_launches(h->geo.ncell) + (use_split(h) ? 1 : 0);
}

// The thread-per-particle density pass of a system with frozen particles
// scans only mobile candidates for frozen homes (frozen split).
bool use_split(const mdpd_handle* h)
{
    return !h->nrep && h->ph.frozen != 0 && !h->ph.list_all &&
           (h->want_phi || h->kernels == MDPD_KERNELS_NLIST_THREAD);
}

// The frozen-frozen density part, from the last binning (the frozen
// particles have not moved since), when the split needs it and it is stale.
void ensure_ff(mdpd_handle* h)
{
    if (!use_split(h) || !h->ff_dirty) return;
    launch_density_nl(h->stream, h->precision, (int)h->n, h->cap, h->geo, h->ph, h->pos4,
                      h->cell_s, h->start, h->rho, h->nl, h->nl_count, 2, h->facc, h->id[h->cur],
                      h->rho_ff);
    // the positions it was computed from (set_state keeps the part while the
    // frozen particles are loaded unmoved)
    if (h->ffx) launch_scatter_by_id(h->stream, (int)h->n, h->cap, h->id[h->cur], h->x[h->cur], h->ffx);
    h->ff_dirty = false;
}

// Partner lists indexed by compacted mobile position (ph.list_compact): the
// frozen-split density pass and the force pass at one lane per particle use
// the same blocks of FORCE_ROUNDS * PAIR_BLOCK slots.
bool list_compact(const mdpd_handle* h) { return use_split(h) && h->force_lpp == 1; }

// all: partner lists for every particle, frozen ones too (the adjoint's;
// a single system takes it from ph.list_all).
void enqueue_density(mdpd_handle* h, bool all = false)
{
    const bool cell = h->kernels == MDPD_KERNELS_NLIST;
    if (h->nrep) {
        if (cell)
            launch_density_cell_batch(h->stream, h->precision, h->cap, h->batch(all), h->pos4,
                                      h->start, h->rho, h->nl, h->nl_count);
        else
            launch_density_nl_batch(h->stream, h->precision, h->cap, h->batch(all), h->pos4,
                                    h->cell_s, h->start, h->rho, h->nl, h->nl_count,
                                    h->thread_shape);
        return;
    }
    h->ph.phi_out = h->want_phi ? h->phi : nullptr;
    h->ph.list_compact = list_compact(h) ? 1 : 0;
    const int fs = use_split(h) ? 1 : 0;
    if (h->want_phi || h->kernels == MDPD_KERNELS_NLIST_THREAD)
        // (the wall density is accumulated by this variant only)
        launch_density_nl(h->stream, h->precision, (int)h->n, h->cap, h->geo, h->ph, h->pos4,
                          h->cell_s, h->start, h->rho, h->nl, h->nl_count, fs, h->facc,
                          h->id[h->cur], h->rho_ff, h->thread_shape);
    else if (cell)
        launch_density_cell(h->stream, h->precision, h->geo.ncell, h->cap, h->geo, h->ph, h->pos4,
                            h->start, h->rho, h->nl, h->nl_count);
    else
        launch_density(h->stream, h->precision, (int)h->n, h->geo, h->ph, h->pos4, h->cell_s,
                       h->start, h->rho);
}

void enqueue_force(mdpd_handle* h, ForceMode mode, int step_offset, double* out, int advance = 0)
{
    if (h->nrep)
        launch_force_nl_batch(h->stream, h->precision, mode, h->cap, h->batch(), h->pos4, h->vel4,
                              h->rho, h->cell_s, h->start, h->nl, h->nl_count, h->step,
                              step_offset, master(h, h->cur), out, h->partials, h->status);
    else if (h->kernels != MDPD_KERNELS_SCAN) {
        h->ph.list_compact = list_compact(h) ? 1 : 0;
        launch_force_nl(h->stream, h->precision, mode, (int)h->n, h->cap, h->geo, h->ph,
                        h->force_lpp, h->mk,
                        h->pos4, h->vel4, h->rho, h->cell_s, h->start, h->nl, h->nl_count,
                        h->step, step_offset, master(h, h->cur), out, h->partials, h->status);
    } else
        launch_force(h->stream, h->precision, mode, (int)h->n, h->cap, h->geo, h->ph, h->mk,
                     h->pos4, h->vel4, h->rho, h->cell_s, h->start, h->step, step_offset,
                     master(h, h->cur), out, h->partials, h->status);
}

void enqueue_reduce(mdpd_handle* h, int advance, cudaStream_t st = nullptr)
{
    if (!st) st = h->stream;
    if (h->nrep) {
        launch_reduce_obs_batch(st, h->precision, h->partials, h->nchunk * PAIR_BLOCK_WARPS,
                                h->d_wr, h->nrep, h->red_ticket, h->obs_b, h->step, advance);
        return;
    }
    const bool scan = h->kernels == MDPD_KERNELS_SCAN;
    const int lpp = scan ? 1 : h->force_lpp;
    const int rounds = scan ? 1 : force_nl_rounds(h->ph, lpp);
    launch_reduce_obs(st, h->precision, h->partials, obs_num_partials((int)h->n, lpp, rounds),
                      h->red_l1,
                      h->red_ticket, h->obs, h->obs + MDPD_NUM_OBS, h->obs + 2 * MDPD_NUM_OBS,
                      h->step, advance);
}

// The last step's observable reduction, if it has not run yet: enqueued
// before anything reads the observables or the step counter, or overwrites
// the force pass's partials outside the time-step loop.
void flush_pending(mdpd_handle* h)
{
    if (!h->pending) return;
    h->pending = false;
    enqueue_reduce(h, 1);
}

// One velocity-Verlet step: bin (after the first half-kick and drift when
// `kick`; otherwise the previous step's force pass did them), density, force
// (+ half-kick [+ next half-kick, drift]).  The step's own reduction is left
// pending.  With `pend` the previous step's reduction runs on the side stream
// beside this binning and density pass and joins before this force pass,
// which reads the step counter the reduction advances and overwrites the
// partials it reads.
void enqueue_step(mdpd_handle* h, ForceMode mode, bool kick, cudaEvent_t* evs, bool pend)
{
    record(h, evs, 0);
    if (pend) {
        cudaEventRecord(h->fork_ev, h->stream);
        cudaStreamWaitEvent(h->side, h->fork_ev, 0);
        enqueue_reduce(h, 1, h->side);
        cudaEventRecord(h->join_ev, h->side);
    }
    enqueue_bin(h, false, kick);
    record(h, evs, 1);
    enqueue_density(h);
    record(h, evs, 2);
    if (pend) cudaStreamWaitEvent(h->stream, h->join_ev, 0);
    enqueue_force(h, mode, 1, nullptr);
    record(h, evs, 3);
    record(h, evs, 4);
}

// Density and forces at the current state (no integration); the result goes
// to `out` (3 * cap doubles, cell order) or, if out is NULL, to the
// integration acceleration a.
int evaluate(mdpd_handle* h, double* out, bool keep_a)
{
    flush_pending(h);
    enqueue_bin(h, keep_a);
    ensure_ff(h);
    enqueue_density(h);
    enqueue_force(h, FM_EVAL, 0, out ? out : h->a[h->cur]);
    enqueue_reduce(h, 0);
    CK(cudaGetLastError());
    return MDPD_OK;
}

// Fused steps captured together (even, so the buffer parity returns to the
// starting one): the time-step loop runs as one graph launch per MULTI_STEPS
// steps when no per-step profiling events are pending.
constexpr int MULTI_STEPS = 8;

int capture_multi(mdpd_handle* h, int cur)
{
    Graphs& gg = h->gm[cur];
    const int saved = h->cur;
    h->cur = cur;
    CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    for (int k = 0; k < MULTI_STEPS; ++k) enqueue_step(h, FM_FUSED, false, nullptr, true);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(h->stream, &graph);
    h->cur = saved;
    if (e != cudaSuccess) return h->fail(MDPD_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        return h->fail(MDPD_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
    gg.graph = graph;
    gg.exec = exec;
    return MDPD_OK;
}

int capture_step(mdpd_handle* h, int prof, int mode, int cur, int kick, int pend)
{
    Graphs& gg = h->g[prof][mode][cur][kick][pend];
    const int saved = h->cur;
    h->cur = cur;
    CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    enqueue_step(h, mode == 0 ? FM_FUSED : FM_LAST, kick != 0, prof ? h->tev : nullptr,
                 pend != 0);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(h->stream, &graph);
    h->cur = saved;
    if (e != cudaSuccess) return h->fail(MDPD_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        return h->fail(MDPD_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
    gg.graph = graph;
    gg.exec = exec;
    if (prof) {
        size_t nn = 0;
        CK(cudaGraphGetNodes(graph, nullptr, &nn));
        std::vector<cudaGraphNode_t> nodes(nn);
        CK(cudaGraphGetNodes(graph, nodes.data(), &nn));
        for (auto nd : nodes) {
            cudaGraphNodeType t;
            CK(cudaGraphNodeGetType(nd, &t));
            if (t != cudaGraphNodeTypeEventRecord) continue;
            cudaEvent_t ev;
            CK(cudaGraphEventRecordNodeGetEvent(nd, &ev));
            for (int k = 0; k < EV_PER_STEP; ++k)
                if (ev == h->tev[k]) gg.ev_node[k] = nd;
        }
    }
    return MDPD_OK;
}

cudaEvent_t* next_prof_events(mdpd_handle* h)
{
    if (h->prof_used >= h->prof_cap) return nullptr;
    if (h->prof_every > 1 && (h->prof_tick++ % h->prof_every) != 0) return nullptr;
    cudaEvent_t* evs = &h->prof_ev[(size_t)h->prof_used * EV_PER_STEP];
    ++h->prof_used;
    return evs;
}

int run_step(mdpd_handle* h, ForceMode mode, bool kick)
{
    cudaEvent_t* evs = next_prof_events(h);
    h->prof_launches += step_launches(h);
    const bool pend = h->pending;
    h->pending = true;
    if (!h->use_graph) {
        enqueue_step(h, mode, kick, evs, pend);
        CK(cudaGetLastError());
        return MDPD_OK;
    }
    const int prof = evs ? 1 : 0;
    const int mi = mode == FM_FUSED ? 0 : 1;
    Graphs& gg = h->g[prof][mi][h->cur][kick ? 1 : 0][pend ? 1 : 0];
    if (!gg.exec) {
        int rc = capture_step(h, prof, mi, h->cur, kick ? 1 : 0, pend ? 1 : 0);
        if (rc) return rc;
    }
    if (prof)
        for (int k = 0; k < EV_PER_STEP; ++k)
            CK(cudaGraphExecEventRecordNodeSetEvent(gg.exec, gg.ev_node[k], evs[k]));
    CK(cudaGraphLaunch(gg.exec, h->stream));
    h->cur = 1 - h->cur;
    return MDPD_OK;
}

int check_ptr_kind(mdpd_handle* h, const void* p, bool want_device)
{
    if (!p) return MDPD_OK;
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return want_device ? h->fail(MDPD_ERR_INVALID_ARG, "pointer is not a device pointer") : MDPD_OK;
    }
    if (want_device && at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
        return h->fail(MDPD_ERR_INVALID_ARG, "pointer is not a device pointer");
    return MDPD_OK;
}

// Device setup shared by single systems and batches: stream, type check
// (particle i of replica r must have a type below ntypes[r]; replica r holds
// the ids [bounds[r], bounds[r + 1])), allocations, upload, loading and the
// first force evaluation.  Owns h: destroys it on failure.
int upload_reps(mdpd_handle* h);

int init_handle(mdpd_handle* h, const double* pos, const double* vel, const int32_t* type,
                void* stream, bool device_inputs, const std::vector<int64_t>& bounds,
                const std::vector<int>& ntypes, mdpd_handle** out)
{
    const int64_t n = h->n;
    int rc;
    auto bail = [&](int code) {
        g_create_error = h->err;
        mdpd_destroy(h);
        return code;
    };
    if (h->geo.ncell > MAX_SCAN) {
        h->err = "too many cells (box / rc exceeds 16.7M cells)";
        return bail(MDPD_ERR_INVALID_ARG);
    }
    if (cudaGetDevice(&h->device) != cudaSuccess) {
        h->err = "no CUDA device";
        return bail(MDPD_ERR_CUDA);
    }
    if (stream) {
        h->stream = (cudaStream_t)stream;
    } else {
        if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
            h->err = "cudaStreamCreate failed";
            return bail(MDPD_ERR_CUDA);
        }
        h->own_stream = true;
    }
    if (device_inputs) {
        if ((rc = check_ptr_kind(h, pos, true)) || (rc = check_ptr_kind(h, vel, true)) ||
            (rc = check_ptr_kind(h, type, true)))
            return bail(rc);
    }

    // types: validated on the host
    h->h_type.assign((size_t)n, 0);
    if (n > 0) {
        if (device_inputs) {
            if (cudaMemcpy(h->h_type.data(), type, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess) {
                h->err = "copy of types failed";
                return bail(MDPD_ERR_CUDA);
            }
        } else {
            std::memcpy(h->h_type.data(), type, (size_t)n * sizeof(int32_t));
        }
        for (size_t r = 0; r + 1 < bounds.size(); ++r)
            for (int64_t i = bounds[r]; i < bounds[r + 1]; ++i)
                if (h->h_type[i] < 0 || h->h_type[i] >= ntypes[r]) {
                    h->err = "type out of range at particle " + std::to_string(i);
                    return bail(MDPD_ERR_INVALID_ARG);
                }
    }
    if ((rc = alloc_particles(h, n))) return bail(rc);
    const int64_t nb = scan_num_blocks(h->geo.ncell);
    if ((rc = dalloc(h, &h->count, (size_t)h->geo.ncell * sizeof(uint32_t))) ||
        (rc = dalloc(h, &h->start, (size_t)(h->geo.ncell + 1) * sizeof(uint32_t))) ||
        (rc = dalloc(h, &h->scan_tmp, (size_t)(nb + 1) * sizeof(uint32_t))) ||
        (rc = dalloc(h, &h->tile_sums, (size_t)2 * nb * sizeof(uint32_t))) ||
        (rc = dalloc(h, &h->status, sizeof(uint32_t))) ||
        (rc = dalloc(h, &h->step, sizeof(uint64_t))) ||
        (rc = dalloc(h, &h->red_ticket, sizeof(unsigned))) ||
        (rc = dalloc(h, &h->obs, (2 * MDPD_NUM_OBS + 2) * sizeof(double))))
        return bail(rc);
    h->ph.dbg_status = h->status;
    if (h->nrep) {
        for (auto& R : h->reps) R.ph.dbg_status = h->status;
        if ((rc = upload_reps(h))) return bail(rc);
    }
    for (int k = 0; k < EV_PER_STEP; ++k)
        if (cudaEventCreate(&h->tev[k]) != cudaSuccess) {
            h->err = "cudaEventCreate failed";
            return bail(MDPD_ERR_CUDA);
        }
    if (cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->fork_ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->join_ev, cudaEventDisableTiming) != cudaSuccess) {
        h->err = "side stream or event creation failed";
        return bail(MDPD_ERR_CUDA);
    }

    // upload: positions to fout, velocities to x[1] (both 3n staging), types
    std::vector<uint8_t> t8((size_t)n);
    for (int64_t i = 0; i < n; ++i) t8[i] = (uint8_t)h->h_type[i];
    cudaStream_t st = h->stream;
    const cudaMemcpyKind kind = device_inputs ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    bool ok = cudaMemsetAsync(h->status, 0, sizeof(uint32_t), st) == cudaSuccess &&
              cudaMemsetAsync(h->step, 0, sizeof(uint64_t), st) == cudaSuccess &&
              cudaMemsetAsync(h->red_ticket, 0, sizeof(unsigned), st) == cudaSuccess &&
              cudaMemsetAsync(h->count, 0, (size_t)h->geo.ncell * sizeof(uint32_t), st) == cudaSuccess &&
              cudaMemsetAsync(h->tile_sums, 0,
                              (size_t)2 * scan_num_blocks(h->geo.ncell) * sizeof(uint32_t),
                              st) == cudaSuccess &&
              cudaMemsetAsync(h->obs, 0, (2 * MDPD_NUM_OBS + 2) * sizeof(double), st) == cudaSuccess;
    if (ok && n > 0)
        ok = cudaMemcpyAsync(h->fout, pos, (size_t)n * 3 * sizeof(double), kind, st) == cudaSuccess &&
             cudaMemcpyAsync(h->x[1], vel, (size_t)n * 3 * sizeof(double), kind, st) == cudaSuccess &&
             cudaMemcpyAsync(h->type_by_id, t8.data(), (size_t)n, cudaMemcpyHostToDevice, st) == cudaSuccess;
    if (!ok) {
        h->err = "initial upload failed";
        return bail(MDPD_ERR_CUDA);
    }
    h->cur = 0;
    if (h->nrep)
        launch_load_state_batch(st, h->cap, h->fout, h->x[1], nullptr, h->batch(), master(h, 0),
                                h->type_by_id, h->status);
    else
        launch_load_state(st, (int)n, h->cap, h->fout, h->x[1], nullptr, h->geo, master(h, 0),
                          h->type_by_id, h->status);
    if ((rc = evaluate(h, nullptr, false))) return bail(rc);
    if ((rc = sync_check(h))) return bail(rc);
    *out = h;
    return MDPD_OK;
}

int create_common(const mdpd_params* params, int64_t n, const double* pos, const double* vel,
                  const int32_t* type, uint64_t seed, void* stream, mdpd_handle** out,
                  bool device_inputs)
{
    g_create_error.clear();
    if (!out) { g_create_error = "out is NULL"; return MDPD_ERR_INVALID_ARG; }
    *out = nullptr;
    std::string why;
    int rc = validate_params(params, why);
    if (rc) { g_create_error = why; return rc; }
    if (n < 0 || n > MAX_PARTICLES) { g_create_error = "n out of range"; return MDPD_ERR_INVALID_ARG; }
    if (n > 0 && (!pos || !vel || !type)) { g_create_error = "pos, vel and type are required"; return MDPD_ERR_INVALID_ARG; }
    if (!device_inputs)
        for (int64_t i = 0; i < n; ++i)
            if (type[i] < 0 || type[i] >= params->ntypes) {
                g_create_error = "type out of range at particle " + std::to_string(i);
                return MDPD_ERR_INVALID_ARG;
            }

    mdpd_handle* h = new mdpd_handle();
    h->p = *params;
    h->seed = seed;
    h->precision = params->precision;
    h->n = h->n_user = n;
    setup_geo_phys(h);
    return init_handle(h, pos, vel, type, stream, device_inputs, { 0, n }, { params->ntypes }, out);
}

// The device copies of the replica records: as they are, and with list_all
// set (the adjoint's partner lists cover frozen particles too).
int upload_reps(mdpd_handle* h)
{
    const size_t bytes = sizeof(Rep) * (size_t)h->nrep;
    CK(cudaMemcpy(h->d_reps, h->reps.data(), bytes, cudaMemcpyHostToDevice));
    std::vector<Rep> all(h->reps);
    for (auto& R : all) R.ph.list_all = 1;
    CK(cudaMemcpy(h->d_reps_all, all.data(), bytes, cudaMemcpyHostToDevice));
    return MDPD_OK;
}

// Batch of nrep independent systems: replica r has its own parameters, seed
// and n[r] particles (the ids [sum_{q<r} n[q], ... + n[r]) of the inputs); its
// cells follow those of replica r - 1 in one lattice, so one launch of each
// kernel advances every replica.
int create_batch(int32_t nrep, const mdpd_params* params, const int64_t* n, const double* pos,
                 const double* vel, const int32_t* type, const uint64_t* seeds, void* stream,
                 mdpd_handle** out)
{
    g_create_error.clear();
    if (!out) { g_create_error = "out is NULL"; return MDPD_ERR_INVALID_ARG; }
    *out = nullptr;
    if (nrep < 1 || nrep > MDPD_MAX_REPLICAS || !params || !n || !seeds) {
        g_create_error = "nrep must be in 1..MDPD_MAX_REPLICAS with params, n and seeds given";
        return MDPD_ERR_INVALID_ARG;
    }
    std::vector<int64_t> bounds(1, 0);
    std::vector<int> ntypes;
    int64_t cells = 0;
    for (int r = 0; r < nrep; ++r) {
        std::string why;
        int rc = validate_params(&params[r], why);
        if (rc) { g_create_error = "replica " + std::to_string(r) + ": " + why; return rc; }
        if (params[r].precision != params[0].precision) {
            g_create_error = "all replicas must have the same precision";
            return MDPD_ERR_INVALID_ARG;
        }
        if (n[r] < 0 || bounds.back() + n[r] > MAX_PARTICLES) {
            g_create_error = "particle counts out of range";
            return MDPD_ERR_INVALID_ARG;
        }
        bounds.push_back(bounds.back() + n[r]);
        ntypes.push_back(params[r].ntypes);
    }
    const int64_t ntot = bounds.back();
    if (ntot > 0 && (!pos || !vel || !type)) { g_create_error = "pos, vel and type are required"; return MDPD_ERR_INVALID_ARG; }

    mdpd_handle* h = new mdpd_handle();
    h->nrep = nrep;
    h->p = params[0];
    h->seed = seeds[0];
    h->precision = params[0].precision;
    h->n = h->n_user = ntot;
    h->kernels = MDPD_KERNELS_NLIST;
    h->rep_p.assign(params, params + nrep);
    h->reps.resize((size_t)nrep);
    std::vector<int4> chunks, cchunks;
    std::vector<int2> wr((size_t)nrep);
    for (int r = 0; r < nrep; ++r) {
        Rep& R = h->reps[r];
        R = Rep{};
        make_geo_phys(params[r], seeds[r], R.geo, R.ph);
        R.cell0 = cells;
        R.id0 = (uint32_t)bounds[r];
        R.n = (uint32_t)n[r];
        cells += R.geo.ncell;
        if (cells > MAX_SCAN) {
            delete h;
            g_create_error = "too many cells in the batch (more than 16.7M)";
            return MDPD_ERR_INVALID_ARG;
        }
        wr[r].x = (int)chunks.size() * PAIR_BLOCK_WARPS;
        for (int64_t f = bounds[r]; f < bounds[r + 1]; f += BATCH_CHUNK)
            chunks.push_back(make_int4(r, (int)f, (int)std::min<int64_t>(BATCH_CHUNK, bounds[r + 1] - f), 0));
        wr[r].y = (int)chunks.size() * PAIR_BLOCK_WARPS;
        for (int64_t c = R.cell0; c < R.cell0 + R.geo.ncell; c += BATCH_CELL_CHUNK)
            cchunks.push_back(make_int4(r, (int)c, (int)std::min<int64_t>(BATCH_CELL_CHUNK, R.cell0 + R.geo.ncell - c), 0));
    }
    h->geo = h->reps[0].geo;
    h->geo.ncell = cells;                  // the concatenated lattice (scan and cell sort)
    h->ph = h->reps[0].ph;
    h->nchunk = (int)chunks.size();
    h->ncchunk = (int)cchunks.size();
    int rc;
    if ((rc = dalloc(h, &h->d_reps, sizeof(Rep) * (size_t)nrep)) ||
        (rc = dalloc(h, &h->d_reps_all, sizeof(Rep) * (size_t)nrep)) ||
        (rc = dalloc(h, &h->d_chunks, sizeof(int4) * chunks.size())) ||
        (rc = dalloc(h, &h->d_cchunks, sizeof(int4) * cchunks.size())) ||
        (rc = dalloc(h, &h->d_wr, sizeof(int2) * wr.size())) ||
        (rc = dalloc(h, &h->obs_b, sizeof(double) * OBS_STRIDE * (size_t)nrep))) {
        g_create_error = h->err;
        mdpd_destroy(h);
        return rc;
    }
    bool ok = upload_reps(h) == MDPD_OK &&
              (chunks.empty() || cudaMemcpy(h->d_chunks, chunks.data(), sizeof(int4) * chunks.size(), cudaMemcpyHostToDevice) == cudaSuccess) &&
              (cchunks.empty() || cudaMemcpy(h->d_cchunks, cchunks.data(), sizeof(int4) * cchunks.size(), cudaMemcpyHostToDevice) == cudaSuccess) &&
              cudaMemcpy(h->d_wr, wr.data(), sizeof(int2) * wr.size(), cudaMemcpyHostToDevice) == cudaSuccess &&
              cudaMemset(h->obs_b, 0, sizeof(double) * OBS_STRIDE * (size_t)nrep) == cudaSuccess;
    if (!ok) {
        g_create_error = "batch tables upload failed";
        mdpd_destroy(h);
        return MDPD_ERR_CUDA;
    }
    return init_handle(h, pos, vel, type, stream, false, bounds, ntypes, out);
}

}  // namespace

namespace mdpd {
// Error text for entry points that have no handle (read by mdpd_last_error(NULL)).
void set_global_error(const std::string& msg) { g_create_error = msg; }
}  // namespace mdpd

extern "C" {

int mdpd_create(const mdpd_params* params, int64_t n, const double* pos, const double* vel,
                const int32_t* type, uint64_t seed, void* cuda_stream, mdpd_handle** out)
{
    return create_common(params, n, pos, vel, type, seed, cuda_stream, out, false);
}

int mdpd_create_dev(const mdpd_params* params, int64_t n, const double* pos, const double* vel,
                    const int32_t* type, uint64_t seed, void* cuda_stream, mdpd_handle** out)
{
    return create_common(params, n, pos, vel, type, seed, cuda_stream, out, true);
}

int mdpd_create_batch(int32_t nrep, const mdpd_params* params, const int64_t* n,
                      const double* pos, const double* vel, const int32_t* type,
                      const uint64_t* seeds, void* cuda_stream, mdpd_handle** out)
{
    return create_batch(nrep, params, n, pos, vel, type, seeds, cuda_stream, out);
}

int mdpd_num_replicas(const mdpd_handle* h, int32_t* nrep)
{
    if (!h || !nrep) return MDPD_ERR_INVALID_ARG;
    *nrep = h->nrep ? h->nrep : 1;
    return MDPD_OK;
}

int mdpd_batch_observables(mdpd_handle* h, double* out, int32_t mean, int32_t reset)
{
    if (!h || !out) return MDPD_ERR_INVALID_ARG;
    if (!h->nrep) return h->fail(MDPD_ERR_INVALID_ARG, "not a batch handle");
    int rc = sync_check(h);
    if (rc) return rc;
    std::vector<double> buf((size_t)h->nrep * OBS_STRIDE);
    CK(cudaMemcpy(buf.data(), h->obs_b, buf.size() * sizeof(double), cudaMemcpyDeviceToHost));
    for (int r = 0; r < h->nrep; ++r) {
        const double* b = &buf[(size_t)r * OBS_STRIDE];
        const double cnt = b[2 * MDPD_NUM_OBS];
        for (int k = 0; k < MDPD_NUM_OBS; ++k)
            out[(size_t)r * MDPD_NUM_OBS + k] =
                mean ? (cnt > 0 ? b[MDPD_NUM_OBS + k] / cnt : 0.0) : b[k];
    }
    if (mean && reset) {
        for (int r = 0; r < h->nrep; ++r)
            for (int k = MDPD_NUM_OBS; k <= 2 * MDPD_NUM_OBS; ++k) buf[(size_t)r * OBS_STRIDE + k] = 0.0;
        CK(cudaMemcpy(h->obs_b, buf.data(), buf.size() * sizeof(double), cudaMemcpyHostToDevice));
    }
    return MDPD_OK;
}

int mdpd_batch_set_params(mdpd_handle* h, const mdpd_params* params)
{
    if (!h || !params) return MDPD_ERR_INVALID_ARG;
    if (!h->nrep) return h->fail(MDPD_ERR_INVALID_ARG, "not a batch handle");
    for (int r = 0; r < h->nrep; ++r) {
        std::string why;
        int rc = validate_params(&params[r], why);
        if (rc) return h->fail(rc, "replica " + std::to_string(r) + ": " + why);
        const mdpd_params& o = h->rep_p[r];
        for (int k = 0; k < 3; ++k)
            if (params[r].box[k] != o.box[k] || params[r].box_lo[k] != o.box_lo[k] ||
                params[r].periodic[k] != o.periodic[k])
                return h->fail(MDPD_ERR_INVALID_ARG, "the box of a replica cannot change");
        if (params[r].rc != o.rc || params[r].precision != o.precision || params[r].ntypes != o.ntypes)
            return h->fail(MDPD_ERR_INVALID_ARG, "rc, precision and ntypes cannot change");
    }
    int rc = sync_check(h);
    if (rc) return rc;
    for (int r = 0; r < h->nrep; ++r) {
        Rep& R = h->reps[r];
        const uint32_t k0 = R.ph.key0, k1 = R.ph.key1;
        Geo g{};
        R.ph = Phys{};
        make_geo_phys(params[r], 0, g, R.ph);
        R.ph.key0 = k0;
        R.ph.key1 = k1;
        R.ph.dbg_status = h->status;
        philox_round_keys(k0, k1, R.ph.rk);
        h->rep_p[r] = params[r];
    }
    // the records live in device memory: captured graphs stay valid
    h->win_valid = false;
    return upload_reps(h);
}

int mdpd_set_walls(mdpd_handle* h, const uint8_t* solid, int32_t nx, int32_t ny, int32_t nz,
                   double voxel, const double origin[3], double wall_density,
                   double shell_thickness, int32_t wall_type, uint64_t seed)
{
    if (!h) return MDPD_ERR_INVALID_ARG;
    if (h->nrep) return h->fail(MDPD_ERR_INVALID_ARG, "walls are not supported on a batch handle");
    if (h->walls_set) return h->fail(MDPD_ERR_INVALID_ARG, "walls already set");
    h->win_valid = false;
    if (!solid || !origin || nx <= 0 || ny <= 0 || nz <= 0 || !(voxel > 0) || !is_fin(voxel))
        return h->fail(MDPD_ERR_INVALID_ARG, "bad mask dimensions or voxel size");
    if (wall_type < 0 || wall_type >= h->p.ntypes)
        return h->fail(MDPD_ERR_INVALID_ARG, "wall_type out of range");
    if (!(wall_density >= 0) || !is_fin(wall_density) || !(shell_thickness >= 0) || !is_fin(shell_thickness))
        return h->fail(MDPD_ERR_INVALID_ARG, "wall_density and shell_thickness must be >= 0");
    const int dim[3] = { nx, ny, nz };
    const int64_t nvox = (int64_t)nx * ny * nz;
    if (nvox > (int64_t(1) << 31)) return h->fail(MDPD_ERR_INVALID_ARG, "mask larger than 2^31 voxels");
    for (int k = 0; k < 3; ++k) {
        if (!h->p.periodic[k]) continue;
        const double span = dim[k] * voxel;
        if (std::fabs(span - h->p.box[k]) > 1e-9 * h->p.box[k] ||
            std::fabs(origin[k] - h->p.box_lo[k]) > 1e-9 * (1.0 + std::fabs(h->p.box_lo[k])))
            return h->fail(MDPD_ERR_INVALID_ARG, "on a periodic axis the mask must span the box exactly");
    }
    int per[3];
    for (int k = 0; k < 3; ++k) per[k] = h->p.periodic[k] ? 1 : 0;
    cudaStream_t st = h->stream;
    int rc;
    uint8_t* dmask = nullptr;
    uint32_t *cnt = nullptr, *off = nullptr, *tmp = nullptr;
    auto cleanup = [&]() {
        dfree(dmask);
        dfree(cnt);
        dfree(off);
        dfree(tmp);
    };
    if ((rc = dalloc(h, &dmask, (size_t)nvox)) || (rc = dalloc(h, &cnt, (size_t)nvox * 4)) ||
        (rc = dalloc(h, &off, (size_t)(nvox + 1) * 4)) ||
        (rc = dalloc(h, &tmp, (size_t)(scan_num_blocks(std::min(nvox, MAX_SCAN)) + 2) * 4))) {
        cleanup();
        return rc;
    }
    uint32_t* bits = nullptr;
    if ((rc = dalloc(h, &bits, (size_t)((nvox + 31) / 32) * 4))) {
        cleanup();
        return rc;
    }
    const double rr = shell_thickness / voxel;
    const int R = (int)std::floor(rr + 1e-9);
    const int64_t R2 = (int64_t)std::floor(rr * rr + 1e-9);
    const double lam = wall_density * voxel * voxel * voxel;
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    uint32_t nw = 0;
    bool ok = cudaMemcpyAsync(dmask, solid, (size_t)nvox, cudaMemcpyHostToDevice, st) == cudaSuccess;
    if (ok) {
        launch_mask_pack(st, dmask, nvox, bits);
        launch_wall_count(st, dmask, dim, per, R, R2, lam, k0, k1, cnt);
        // (masks beyond the two-level scan's limit in segments; the last
        // word of tmp carries the running total)
        launch_exclusive_scan_long(st, cnt, nvox, off, tmp,
                                   tmp + scan_num_blocks(std::min(nvox, MAX_SCAN)) + 1, MAX_SCAN);
        ok = cudaMemcpyAsync(&nw, off + nvox, 4, cudaMemcpyDeviceToHost, st) == cudaSuccess &&
             cudaStreamSynchronize(st) == cudaSuccess;
    }
    if (!ok) {
        cleanup();
        dfree(bits);
        return h->fail(MDPD_ERR_CUDA, "wall sweep failed");
    }
    const int64_t n_old = h->n, n_new = h->n + (int64_t)nw;
    if (n_new > MAX_PARTICLES) {
        cleanup();
        dfree(bits);
        return h->fail(MDPD_ERR_INVALID_ARG, "too many particles with walls");
    }
    // fill arrays of the new capacity in a scratch handle, then swap them in
    mdpd_handle nh;
    nh.precision = h->precision;
    if ((rc = alloc_particles(&nh, n_new))) {
        free_particles(&nh);
        cleanup();
        dfree(bits);
        return h->fail(rc, nh.err);
    }
    const int64_t old_cap = h->cap;
    swap_particle_arrays(h, &nh);     // h: new arrays, nh: old arrays (old_cap)
    mdpd_handle& tmpH = nh;
    const int c = h->cur;
    ok = true;
    for (int k = 0; k < 3 && ok; ++k) {
        ok = cudaMemcpyAsync(h->x[0] + k * h->cap, tmpH.x[c] + k * old_cap, n_old * sizeof(double), cudaMemcpyDeviceToDevice, st) == cudaSuccess &&
             cudaMemcpyAsync(h->v[0] + k * h->cap, tmpH.v[c] + k * old_cap, n_old * sizeof(double), cudaMemcpyDeviceToDevice, st) == cudaSuccess &&
             cudaMemcpyAsync(h->a[0] + k * h->cap, tmpH.a[c] + k * old_cap, n_old * sizeof(double), cudaMemcpyDeviceToDevice, st) == cudaSuccess;
    }
    ok = ok && cudaMemcpyAsync(h->id[0], tmpH.id[c], n_old * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st) == cudaSuccess &&
         cudaMemcpyAsync(h->type[0], tmpH.type[c], (size_t)n_old, cudaMemcpyDeviceToDevice, st) == cudaSuccess &&
         cudaMemcpyAsync(h->type_by_id, tmpH.type_by_id, (size_t)n_old, cudaMemcpyDeviceToDevice, st) == cudaSuccess &&
         cudaMemsetAsync(h->type_by_id + n_old, wall_type, (size_t)nw, st) == cudaSuccess;
    h->cur = 0;
    // the scan's tile sums follow the buffer parity: with the parity reset,
    // clear both so the next binning starts from zero whichever it uses
    ok = ok && cudaMemsetAsync(h->tile_sums, 0,
                               (size_t)2 * scan_num_blocks(h->geo.ncell) * sizeof(uint32_t),
                               st) == cudaSuccess;
    if (ok) {
        launch_wall_emit(st, dmask, dim, cnt, off, voxel, origin, k0, k1, n_old, h->cap,
                         master(h, 0), (uint8_t)wall_type);
        ok = cudaStreamSynchronize(st) == cudaSuccess;
    }
    free_particles(&tmpH);
    cleanup();
    if (!ok) {
        dfree(bits);
        return h->fail(MDPD_ERR_CUDA, "wall emission failed");
    }
    h->n = n_new;
    h->h_type.resize((size_t)n_new, wall_type);
    dfree(h->mask_bits);
    h->mask_bits = bits;
    h->mk.bits = bits;
    for (int k = 0; k < 3; ++k) {
        h->mk.dim[k] = dim[k];
        h->mk.origin[k] = origin[k];
    }
    h->mk.voxel = voxel;
    h->mk.inv_voxel = 1.0 / voxel;
    {
        int ex = 0;
        h->mk.inv_voxel_exact = std::frexp(voxel, &ex) == 0.5 ? 1 : 0;
    }
    // FP32 voxel index: the FP32 error in voxels is at most about
    // 4 * 2^-24 * (|x| + |origin|) / voxel, below 5e-4 within these bounds
    h->mk.fast = 1;
    for (int k = 0; k < 3; ++k) {
        const double xmax = std::max(std::fabs(h->geo.lo[k]), std::fabs(h->geo.hi[k]));
        const double span = (xmax + std::fabs(origin[k])) / voxel;
        if (dim[k] > 1024 || !(span <= 2048.0)) h->mk.fast = 0;
        h->mk.origin_f[k] = (float)origin[k];
    }
    h->mk.inv_voxel_f = (float)(1.0 / voxel);
    h->walls_set = true;
    h->ff_dirty = true;
    destroy_graphs(h);
    if ((rc = evaluate(h, nullptr, false))) return rc;
    return sync_check(h);
}

int mdpd_step(mdpd_handle* h, int64_t nsteps)
{
    if (!h) return MDPD_ERR_INVALID_ARG;
    if (nsteps < 0) return h->fail(MDPD_ERR_INVALID_ARG, "nsteps < 0");
    if (nsteps == 0) return MDPD_OK;
    ensure_ff(h);
    // the first step's binning applies the first half-kick and drift; later
    // steps get them from the previous force pass (FM_FUSED)
    for (int64_t k = 0; k < nsteps; ++k) {
        // fused, no kick, with the previous step's reduction still pending
        const bool middle = k > 0 && k + MULTI_STEPS < nsteps && h->pending;
        if (middle && h->use_graph && h->prof_used >= h->prof_cap) {
            Graphs& gg = h->gm[h->cur];
            if (!gg.exec) {
                int rc = capture_multi(h, h->cur);
                if (rc) return rc;
            }
            CK(cudaGraphLaunch(gg.exec, h->stream));
            h->prof_launches += (int64_t)MULTI_STEPS * step_launches(h);
            k += MULTI_STEPS - 1;              // the parity is unchanged (even count)
            continue;
        }
        int rc = run_step(h, k + 1 < nsteps ? FM_FUSED : FM_LAST, k == 0);
        if (rc) return rc;
    }
    h->steps_host += nsteps;
    return MDPD_OK;
}

int mdpd_sync(mdpd_handle* h)
{
    if (!h) return MDPD_ERR_INVALID_ARG;
    return sync_check(h);
}

int mdpd_num_particles(const mdpd_handle* h, int64_t* n)
{
    if (!h || !n) return MDPD_ERR_INVALID_ARG;
    *n = h->n;
    return MDPD_OK;
}

int mdpd_step_count(const mdpd_handle* h, int64_t* steps)
{
    if (!h || !steps) return MDPD_ERR_INVALID_ARG;
    *steps = h->steps_host;
    return MDPD_OK;
}

static int get_state_impl(mdpd_handle* h, double* pos, double* vel, int32_t* type, double* rho,
                          bool dev)
{
    if (!h) return MDPD_ERR_INVALID_ARG;
    int rc = sync_check(h);
    if (rc) return rc;
    cudaStream_t st = h->stream;
    const int n = (int)h->n;
    const int c = h->cur;
    double* s_pos = h->fout;
    double* s_vel = h->x[1 - c];
    double* s_rho = h->v[1 - c];
    int32_t* s_type = (int32_t*)h->a[1 - c];
    if (dev) {
        s_pos = pos;
        s_vel = vel;
        s_rho = rho;
        s_type = type;
    }
    if (pos) launch_scatter_by_id(st, n, h->cap, h->id[c], h->x[c], s_pos);
    if (vel) launch_scatter_by_id(st, n, h->cap, h->id[c], h->v[c], s_vel);
    if (rho) launch_scatter_scalar_by_id(st, h->precision, n, h->id[c], h->rho, s_rho);
    if (type) launch_scatter_type_by_id(st, n, h->id[c], h->type[c], s_type);
    CK(cudaGetLastError());
    if (!dev) {
        if (pos) CK(cudaMemcpyAsync(pos, s_pos, (size_t)n * 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
        if (vel) CK(cudaMemcpyAsync(vel, s_vel, (size_t)n * 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
        if (rho) CK(cudaMemcpyAsync(rho, s_rho, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, st));
        if (type) CK(cudaMemcpyAsync(type, s_type, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    }
    return sync_check(h);
}

int mdpd_get_state(mdpd_handle* h, double* pos, double* vel, int32_t* type, double* rho)
{
    return get_state_impl(h, pos, vel, type, rho, false);
}

int mdpd_get_state_dev(mdpd_handle* h, double* pos, double* vel, int32_t* type, double* rho)
{
    if (h) {
        int rc;
        if ((rc = check_ptr_kind(h, pos, true)) || (rc = check_ptr_kind(h, vel, true)) ||
            (rc = check_ptr_kind(h, type, true)) || (rc = check_ptr_kind(h, rho, true)))
            return rc;
    }
    return get_state_impl(h, pos, vel, type, rho, true);
}

// acc (may be NULL): accelerations to restore instead of evaluating the
// forces at the loaded state (a checkpoint of a run resumes bit for bit).
static int set_state_impl(mdpd_handle* h, const double* pos, const double* vel, const double* acc,
                          bool dev)
{
    if (!h) return MDPD_ERR_INVALID_ARG;
    if (h->n > 0 && (!pos || !vel)) return h->fail(MDPD_ERR_INVALID_ARG, "pos and vel are required");
    int rc = sync_check(h);
    if (rc) return rc;
    if (dev && ((rc = check_ptr_kind(h, pos, true)) || (rc = check_ptr_kind(h, vel, true)))) return rc;
    cudaStream_t st = h->stream;
    const int n = (int)h->n;
    const int c = h->cur;
    const double* d_pos = pos;
    const double* d_vel = vel;
    const double* d_acc = nullptr;
    if (!dev && n > 0) {
        CK(cudaMemcpyAsync(h->fout, pos, (size_t)n * 3 * sizeof(double), cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(h->x[1 - c], vel, (size_t)n * 3 * sizeof(double), cudaMemcpyHostToDevice, st));
        d_pos = h->fout;
        d_vel = h->x[1 - c];
        if (acc) {
            CK(cudaMemcpyAsync(h->v[1 - c], acc, (size_t)n * 3 * sizeof(double), cudaMemcpyHostToDevice, st));
            d_acc = h->v[1 - c];
        }
    }
    if (h->nrep)
        launch_load_state_batch(st, h->cap, d_pos, d_vel, d_acc, h->batch(), master(h, c),
                                h->type_by_id, h->status);
    else
        launch_load_state(st, n, h->cap, d_pos, d_vel, d_acc, h->geo, master(h, c), h->type_by_id,
                          h->status);
    // the frozen-frozen density part stays valid if no frozen particle moved
    // (a caller that resumes or steps a state it read back loads the walls
    // unchanged): compared bit for bit with the positions it came from
    if (use_split(h) && !h->ff_dirty && h->ffx && n > 0) {
        CK(cudaMemsetAsync(h->ff_moved, 0, sizeof(uint32_t), st));
        launch_frozen_moved(st, n, h->cap, h->x[c], h->ffx, h->type_by_id, h->ph.frozen,
                            h->ff_moved);
        uint32_t moved = 1;
        CK(cudaMemcpyAsync(&moved, h->ff_moved, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        h->ff_dirty = moved != 0;
    } else {
        h->ff_dirty = true;
    }
    if (acc) {
        // no evaluation; when the frozen-frozen part must be recomputed, a
        // binning (the accelerations gathered along) gives it its cell order
        if (use_split(h) && h->ff_dirty) {
            enqueue_bin(h, true);
            ensure_ff(h);
        }
        CK(cudaGetLastError());
    } else if ((rc = evaluate(h, nullptr, false))) {
        return rc;
    }
    // host inputs are the caller's again when this returns (a copy from a
    // page-locked buffer runs asynchronously)
    if (!dev) CK(cudaStreamSynchronize(st));
    return MDPD_OK;
}

int mdpd_set_state(mdpd_handle* h, const double* pos, const double* vel)
{
    return set_state_impl(h, pos, vel, nullptr, false);
}

int mdpd_set_state_accel(mdpd_handle* h, const double* pos, const double* vel, const double* accel)
{
    if (h && h->n > 0 && !accel) return h->fail(MDPD_ERR_INVALID_ARG, "accel is required");
    return set_state_impl(h, pos, vel, accel, false);
}

int mdpd_get_accel(mdpd_handle* h, double* accel)
{
    if (!h || !accel) return MDPD_ERR_INVALID_ARG;
    int rc = sync_check(h);
    if (rc) return rc;
    double* tmp = h->x[1 - h->cur];
    launch_scatter_by_id(h->stream, (int)h->n, h->cap, h->id[h->cur], h->a[h->cur], tmp);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(accel, tmp, (size_t)h->n * 3 * sizeof(double), cudaMemcpyDeviceToHost,
                       h->stream));
    return sync_check(h);
}

int mdpd_set_state_dev(mdpd_handle* h, const double* pos, const double* vel)
{
    return set_state_impl(h, pos, vel, nullptr, true);
}

static int forces_impl(mdpd_handle* h, double* force, double* rho, bool dev)
{
    if (!h) return MDPD_ERR_INVALID_ARG;
    int rc = sync_check(h);
    if (rc) return rc;
    if (dev && ((rc = check_ptr_kind(h, force, true)) || (rc = check_ptr_kind(h, rho, true)))) return rc;
    if ((rc = evaluate(h, h->fout, true))) return rc;
    cudaStream_t st = h->stream;
    const int n = (int)h->n;
    const int c = h->cur;
    double* s_f = dev ? force : h->x[1 - c];
    double* s_rho = dev ? rho : h->v[1 - c];
    if (force) launch_scatter_by_id(st, n, h->cap, h->id[c], h->fout, s_f);
    if (rho) launch_scatter_scalar_by_id(st, h->precision, n, h->id[c], h->rho, s_rho);
    CK(cudaGetLastError());
    if (!dev) {
        if (force) CK(cudaMemcpyAsync(force, s_f, (size_t)n * 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
        if (rho) CK(cudaMemcpyAsync(rho, s_rho, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, st));
    }
    return sync_check(h);
}

int mdpd_forces(mdpd_handle* h, double* force, double* rho) { return forces_impl(h, force, rho, false); }

int mdpd_forces_dev(mdpd_handle* h, double* force, double* rho) { return forces_impl(h, force, rho, true); }

int mdpd_observables(mdpd_handle* h, double out[MDPD_NUM_OBS])
{
    if (!h || !out) return MDPD_ERR_INVALID_ARG;
    if (h->nrep) return h->fail(MDPD_ERR_INVALID_ARG, "batch handle: use mdpd_batch_observables");
    int rc = sync_check(h);
    if (rc) return rc;
    CK(cudaMemcpy(out, h->obs, MDPD_NUM_OBS * sizeof(double), cudaMemcpyDeviceToHost));
    return MDPD_OK;
}

int mdpd_observables_mean(mdpd_handle* h, double out[MDPD_NUM_OBS], int32_t reset)
{
    if (!h || !out) return MDPD_ERR_INVALID_ARG;
    if (h->nrep) return h->fail(MDPD_ERR_INVALID_ARG, "batch handle: use mdpd_batch_observables");
    int rc = sync_check(h);
    if (rc) return rc;
    double buf[MDPD_NUM_OBS + 1];
    CK(cudaMemcpy(buf, h->obs + MDPD_NUM_OBS, (MDPD_NUM_OBS + 1) * sizeof(double), cudaMemcpyDeviceToHost));
    const double cnt = buf[MDPD_NUM_OBS];
    for (int k = 0; k < MDPD_NUM_OBS; ++k) out[k] = cnt > 0 ? buf[k] / cnt : 0.0;
    if (reset) CK(cudaMemset(h->obs + MDPD_NUM_OBS, 0, (MDPD_NUM_OBS + 1) * sizeof(double)));
    return MDPD_OK;
}

int mdpd_pair_count(mdpd_handle* h, int64_t* pairs)
{
    if (!h || !pairs) return MDPD_ERR_INVALID_ARG;
    int rc = sync_check(h);
    if (rc) return rc;
    double v = 0.0;
    if (h->nrep) {
        std::vector<double> buf((size_t)h->nrep * OBS_STRIDE);
        CK(cudaMemcpy(buf.data(), h->obs_b, buf.size() * sizeof(double), cudaMemcpyDeviceToHost));
        for (int r = 0; r < h->nrep; ++r) v += buf[(size_t)r * OBS_STRIDE + 2 * MDPD_NUM_OBS + 1];
    } else {
        CK(cudaMemcpy(&v, h->obs + 2 * MDPD_NUM_OBS + 1, sizeof(double), cudaMemcpyDeviceToHost));
    }
    *pairs = (int64_t)v;
    return MDPD_OK;
}

int mdpd_set_option(mdpd_handle* h, int32_t option, int64_t value)
{
    if (!h) return MDPD_ERR_INVALID_ARG;
    flush_pending(h);      // the pending reduction reads the current partials layout
    switch (option) {
    case MDPD_OPT_GRAPH:
        h->use_graph = value != 0;
        return MDPD_OK;
    case MDPD_OPT_KERNELS:
        if (value != MDPD_KERNELS_NLIST && value != MDPD_KERNELS_SCAN &&
            value != MDPD_KERNELS_NLIST_THREAD)
            return h->fail(MDPD_ERR_INVALID_ARG, "unknown kernel variant");
        if (h->nrep && value == MDPD_KERNELS_SCAN)
            return h->fail(MDPD_ERR_INVALID_ARG, "a batch runs the neighbour-list kernels only");
        CK(cudaStreamSynchronize(h->stream));
        h->kernels = (int)value;
        destroy_graphs(h);
        return MDPD_OK;
    case MDPD_OPT_PROFILE: {
        if (value < 0 || value > (int64_t(1) << 20)) return h->fail(MDPD_ERR_INVALID_ARG, "profile steps out of range");
        CK(cudaStreamSynchronize(h->stream));
        const size_t need = (size_t)value * EV_PER_STEP;
        while (h->prof_ev.size() < need) {
            cudaEvent_t e;
            CK(cudaEventCreate(&e));
            h->prof_ev.push_back(e);
        }
        h->prof_cap = value;
        h->prof_used = 0;
        h->prof_launches = 0;
        h->prof_tick = 0;
        return MDPD_OK;
    }
    case MDPD_OPT_FORCE_LANES:
        if (value != 1 && value != 2 && value != 4)
            return h->fail(MDPD_ERR_INVALID_ARG, "lanes per particle must be 1, 2 or 4");
        if (h->nrep && value != 1)
            return h->fail(MDPD_ERR_INVALID_ARG, "a batch runs one lane per particle");
        CK(cudaStreamSynchronize(h->stream));
        h->force_lpp = (int)value;
        destroy_graphs(h);
        return MDPD_OK;
    case MDPD_OPT_DENSITY_SHAPE:
        if (value != 0 && value != 1)
            return h->fail(MDPD_ERR_INVALID_ARG, "the density code shape is 0 or 1");
        CK(cudaStreamSynchronize(h->stream));
        h->thread_shape = (int)value;
        destroy_graphs(h);
        return MDPD_OK;
    case MDPD_OPT_WALL_DENSITY:
        if (h->nrep) return h->fail(MDPD_ERR_INVALID_ARG, "a batch has no walls");
        CK(cudaStreamSynchronize(h->stream));
        h->want_phi = value != 0;
        destroy_graphs(h);
        return MDPD_OK;
    case MDPD_OPT_PROFILE_EVERY:
        if (value < 1) return h->fail(MDPD_ERR_INVALID_ARG, "profile interval must be >= 1");
        h->prof_every = value;
        h->prof_tick = 0;
        return MDPD_OK;
    default:
        return h->fail(MDPD_ERR_INVALID_ARG, "unknown option");
    }
}

int mdpd_profile(mdpd_handle* h, double ms[MDPD_NUM_KCLASS], int64_t* steps, int64_t* launches)
{
    if (!h || !ms) return MDPD_ERR_INVALID_ARG;
    CK(cudaStreamSynchronize(h->stream));
    for (int k = 0; k < MDPD_NUM_KCLASS; ++k) ms[k] = 0.0;
    for (int64_t s = 0; s < h->prof_used; ++s) {
        cudaEvent_t* e = &h->prof_ev[(size_t)s * EV_PER_STEP];
        for (int k = 0; k < MDPD_NUM_KCLASS; ++k) {
            float t = 0.f;
            CK(cudaEventElapsedTime(&t, e[k], e[k + 1]));
            ms[k] += t;
        }
    }
    if (steps) *steps = h->prof_used;
    if (launches) *launches = h->prof_launches;
    h->prof_used = 0;
    h->prof_launches = 0;
    return MDPD_OK;
}

int mdpd_set_params(mdpd_handle* h, const mdpd_params* p)
{
    if (!h) return MDPD_ERR_INVALID_ARG;
    if (h->nrep) return h->fail(MDPD_ERR_INVALID_ARG, "batch handle: use mdpd_batch_set_params");
    flush_pending(h);
    std::string why;
    int rc = validate_params(p, why);
    if (rc) return h->fail(rc, why);
    for (int k = 0; k < 3; ++k)
        if (p->box[k] != h->p.box[k] || p->box_lo[k] != h->p.box_lo[k] ||
            p->periodic[k] != h->p.periodic[k])
            return h->fail(MDPD_ERR_INVALID_ARG, "the box cannot change");
    if (p->rc != h->p.rc || p->rd != h->p.rd || p->precision != h->p.precision ||
        p->ntypes != h->p.ntypes)
        return h->fail(MDPD_ERR_INVALID_ARG, "rc, rd, precision and ntypes cannot change");
    if ((rc = sync_check(h))) return rc;
    h->win_valid = false;
    h->p = *p;
    setup_geo_phys(h);
    h->ff_dirty = true;                      // r_d or the frozen types may change
    destroy_graphs(h);
    return MDPD_OK;
}

int mdpd_set_step(mdpd_handle* h, int64_t step)
{
    if (!h || step < 0) return MDPD_ERR_INVALID_ARG;
    int rc = sync_check(h);
    if (rc) return rc;
    const uint64_t s = (uint64_t)step;
    CK(cudaMemcpy(h->step, &s, sizeof(s), cudaMemcpyHostToDevice));
    h->steps_host = step;
    return MDPD_OK;
}

int mdpd_get_accel_dev(mdpd_handle* h, double* accel)
{
    if (!h) return MDPD_ERR_INVALID_ARG;
    int rc = sync_check(h);
    if (rc) return rc;
    if ((rc = check_ptr_kind(h, accel, true))) return rc;
    if (accel) launch_scatter_by_id(h->stream, (int)h->n, h->cap, h->id[h->cur], h->a[h->cur], accel);
    CK(cudaGetLastError());
    return sync_check(h);
}

// ---- adjoint ---------------------------------------------------------------------

namespace {

int vjp_nrep(const mdpd_handle* h) { return h->nrep ? h->nrep : 1; }

// Parameter partials sized for the current particle count (which grows when
// walls are added).
int vjp_alloc(mdpd_handle* h)
{
    const Batch bt = h->batch();
    const int nblk = std::max(1, vjp_num_blocks((int)h->n, h->nrep ? &bt : nullptr));
    if (h->vjp_tpart && h->vjp_nblk >= nblk) return MDPD_OK;
    dfree(h->vjp_tpart);
    dfree(h->vjp_tacc);
    dfree(h->vjp_wbar);
    h->vjp_nblk = 0;
    int rc;
    if ((rc = dalloc(h, &h->vjp_tpart, (size_t)nblk * THETA_SLOTS * sizeof(double))) ||
        (rc = dalloc(h, &h->vjp_tacc, (size_t)vjp_nrep(h) * THETA_SLOTS * sizeof(double))) ||
        (rc = dalloc(h, &h->vjp_wbar, (size_t)vjp_nrep(h) * 6 * sizeof(double))))
        return rc;
    h->vjp_nblk = nblk;
    return MDPD_OK;
}

// Cell order and partner lists of every particle (frozen ones included) for
// the state in the master arrays: a binning and a density pass, no forces.
void vjp_prepare(mdpd_handle* h, bool gather_a)
{
    h->ph.list_all = 1;
    enqueue_bin(h, gather_a);
    enqueue_density(h, true);
    h->ph.list_all = 0;
}

// One VJP of the evaluation prepared by vjp_prepare: the force/virial part,
// the caller's density adjoint (id order, may be NULL) added to the density
// chain, the density chain, and the parameter partials summed per replica
// into vjp_tacc (stored, or added when add_theta).  Outputs in cell order in
// the spare master buffers: xbar in x[1 - cur], ubar in v[1 - cur].
void vjp_core(mdpd_handle* h, const double* abar, const double* wbar, const double* rhobar,
              int add_theta)
{
    cudaStream_t st = h->stream;
    const int n = (int)h->n;
    const int c = h->cur;
    const Batch bt = h->batch(true);
    const Batch* pb = h->nrep ? &bt : nullptr;
    double* xs = h->x[1 - c];
    double* us = h->v[1 - c];
    double* rs = h->a[1 - c];
    launch_force_vjp(st, h->precision, n, h->cap, h->geo, h->ph, pb, h->pos4, h->vel4, h->rho,
                     h->cell_s, h->start, h->nl, h->nl_count, h->step, abar, wbar, xs, us, rs,
                     h->vjp_tpart, h->status);
    if (rhobar) launch_gather_by_id(st, n, h->id[c], rhobar, rs, 1);
    launch_density_vjp(st, h->precision, n, h->cap, h->geo, h->ph, pb, h->pos4, h->cell_s,
                       h->start, h->nl, h->nl_count, rs, xs, h->status);
    launch_theta_reduce(st, vjp_nrep(h), vjp_num_blocks(n, pb), h->nrep ? h->d_wr : nullptr,
                        PAIR_BLOCK_WARPS, h->vjp_tpart, h->vjp_tacc, add_theta);
}

// Master state from device arrays in id order (no evaluation).
void load_state_dev(mdpd_handle* h, const double* pos, const double* vel)
{
    if (h->nrep)
        launch_load_state_batch(h->stream, h->cap, pos, vel, nullptr, h->batch(),
                                master(h, h->cur), h->type_by_id, h->status);
    else
        launch_load_state(h->stream, (int)h->n, h->cap, pos, vel, nullptr, h->geo,
                          master(h, h->cur), h->type_by_id, h->status);
    h->ff_dirty = true;
}

// A window needs differentiable steps: no reflection off walls or
// non-periodic faces.
bool window_allowed(const mdpd_handle* h, std::string& why)
{
    if (h->mk.bits || h->walls_set) { why = "reflection off walls is not differentiable"; return false; }
    const int nr = vjp_nrep(h);
    for (int r = 0; r < nr; ++r) {
        const mdpd_params& p = h->nrep ? h->rep_p[r] : h->p;
        for (int k = 0; k < 3; ++k)
            if (!p.periodic[k]) {
                why = "reflection at a non-periodic face is not differentiable";
                return false;
            }
    }
    return true;
}

}  // namespace

int mdpd_eval_vjp_dev(mdpd_handle* h, const double* abar, const double* cvir,
                      const double* rhobar, double* xbar, double* ubar, double* theta_bar)
{
    if (!h) return MDPD_ERR_INVALID_ARG;
    int rc = sync_check(h);
    if (rc) return rc;
    if ((rc = check_ptr_kind(h, abar, true)) || (rc = check_ptr_kind(h, cvir, true)) ||
        (rc = check_ptr_kind(h, rhobar, true)) || (rc = check_ptr_kind(h, xbar, true)) ||
        (rc = check_ptr_kind(h, ubar, true)) || (rc = check_ptr_kind(h, theta_bar, true)))
        return rc;
    if ((rc = vjp_alloc(h))) return rc;
    cudaStream_t st = h->stream;
    const int n = (int)h->n;
    vjp_prepare(h, true);
    vjp_core(h, abar, cvir, rhobar, 0);
    const int c = h->cur;
    if (xbar) launch_scatter_by_id(st, n, h->cap, h->id[c], h->x[1 - c], xbar);
    if (ubar) launch_scatter_by_id(st, n, h->cap, h->id[c], h->v[1 - c], ubar);
    if (theta_bar) launch_theta_symmetrise(st, vjp_nrep(h), h->vjp_tacc, theta_bar);
    CK(cudaGetLastError());
    return sync_check(h);
}

int mdpd_force_vjp_dev(mdpd_handle* h, const double* abar, double* xbar, double* ubar,
                       double* theta_bar)
{
    if (!h) return MDPD_ERR_INVALID_ARG;
    if (!abar) return h->fail(MDPD_ERR_INVALID_ARG, "abar is required");
    return mdpd_eval_vjp_dev(h, abar, nullptr, nullptr, xbar, ubar, theta_bar);
}

int mdpd_density_vjp_dev(mdpd_handle* h, const double* rhobar, double* xbar)
{
    if (!h) return MDPD_ERR_INVALID_ARG;
    if (!rhobar || !xbar) return h->fail(MDPD_ERR_INVALID_ARG, "rhobar and xbar are required");
    return mdpd_eval_vjp_dev(h, nullptr, nullptr, rhobar, xbar, nullptr, nullptr);
}

int mdpd_window_forward(mdpd_handle* h, int32_t nsteps)
{
    if (!h) return MDPD_ERR_INVALID_ARG;
    if (nsteps < 1) return h->fail(MDPD_ERR_INVALID_ARG, "nsteps must be >= 1");
    std::string why;
    if (!window_allowed(h, why)) return h->fail(MDPD_ERR_INVALID_ARG, why);
    int rc = sync_check(h);
    if (rc) return rc;
    flush_pending(h);
    const int n = (int)h->n;
    const size_t vec = (size_t)std::max(n, 1) * 3;
    if (h->win_alloc_steps < nsteps || h->win_vec != vec) {
        dfree(h->win_x);
        dfree(h->win_vh);
        dfree(h->win_v0);
        dfree(h->win_b);
        h->win_alloc_steps = 0;
        h->win_vec = 0;
        if ((rc = dalloc(h, &h->win_x, vec * (size_t)(nsteps + 1) * sizeof(double))) ||
            (rc = dalloc(h, &h->win_vh, vec * (size_t)nsteps * sizeof(double))) ||
            (rc = dalloc(h, &h->win_v0, vec * sizeof(double))) ||
            (rc = dalloc(h, &h->win_b, 3 * vec * sizeof(double))))
            return rc;
        h->win_alloc_steps = nsteps;
        h->win_vec = vec;
    }
    h->win_valid = false;
    cudaStream_t st = h->stream;
    const Batch bt = h->batch();
    const Batch* pb = h->nrep ? &bt : nullptr;
    h->win_s0 = h->steps_host;
    launch_win_record(st, n, h->cap, h->ph, pb, master(h, h->cur), h->win_x, nullptr);
    launch_scatter_by_id(st, n, h->cap, h->id[h->cur], h->v[h->cur], h->win_v0);
    for (int32_t k = 0; k < nsteps; ++k) {
        launch_win_record(st, n, h->cap, h->ph, pb, master(h, h->cur), h->win_x + vec * k,
                          h->win_vh + vec * k);
        ensure_ff(h);
        if ((rc = run_step(h, FM_LAST, true))) return rc;
        ++h->steps_host;
        launch_win_record(st, n, h->cap, h->ph, pb, master(h, h->cur), h->win_x + vec * (k + 1),
                          nullptr);
    }
    CK(cudaGetLastError());
    if ((rc = sync_check(h))) return rc;
    h->win_k = nsteps;
    h->win_valid = true;
    return MDPD_OK;
}

int mdpd_window_vjp_dev(mdpd_handle* h, const double* xbar, const double* vbar,
                        const double* cvir, const double* rhobar, double* x0bar, double* v0bar,
                        double* theta_bar)
{
    if (!h) return MDPD_ERR_INVALID_ARG;
    if (!h->win_valid) return h->fail(MDPD_ERR_INVALID_ARG, "no recorded window (mdpd_window_forward)");
    int rc = sync_check(h);
    if (rc) return rc;
    if ((rc = check_ptr_kind(h, xbar, true)) || (rc = check_ptr_kind(h, vbar, true)) ||
        (rc = check_ptr_kind(h, cvir, true)) || (rc = check_ptr_kind(h, rhobar, true)) ||
        (rc = check_ptr_kind(h, x0bar, true)) || (rc = check_ptr_kind(h, v0bar, true)) ||
        (rc = check_ptr_kind(h, theta_bar, true)))
        return rc;
    if ((rc = vjp_alloc(h))) return rc;
    const int n = (int)h->n;
    const size_t vec = (size_t)std::max(n, 1) * 3;
    if (vec != h->win_vec) return h->fail(MDPD_ERR_INVALID_ARG, "the window was recorded for another particle count");
    cudaStream_t st = h->stream;
    flush_pending(h);
    const Batch bt = h->batch();
    const Batch* pb = h->nrep ? &bt : nullptr;
    double* xb = h->win_b;
    double* vb = h->win_b + vec;
    double* ab = h->win_b + 2 * vec;
    const int64_t K = h->win_k, s0 = h->win_s0;
    launch_win_init(st, n, h->ph, pb, master(h, h->cur), xbar, vbar, xb, vb, ab);
    // reverse sweep: the force evaluation of step k + 1 at (x_{k+1}, v'_k);
    // the last one also produced the final densities and virial
    for (int64_t k = K - 1; k >= 0; --k) {
        load_state_dev(h, h->win_x + vec * (k + 1), h->win_vh + vec * k);
        launch_set_step(st, h->step, (uint64_t)(s0 + k + 1));
        vjp_prepare(h, false);
        const bool last = k == K - 1;
        vjp_core(h, ab, last ? cvir : nullptr, last ? rhobar : nullptr, last ? 0 : 1);
        const int c = h->cur;
        launch_win_post(st, n, h->cap, h->ph, pb, master(h, c), h->x[1 - c], h->v[1 - c], xb, vb,
                        ab, k == 0 ? 1 : 0, 0, nullptr, nullptr);
    }
    // a_0 = F(x_0, v_0) at step s0
    load_state_dev(h, h->win_x, h->win_v0);
    launch_set_step(st, h->step, (uint64_t)s0);
    vjp_prepare(h, false);
    vjp_core(h, ab, nullptr, nullptr, 1);
    {
        const int c = h->cur;
        launch_win_post(st, n, h->cap, h->ph, pb, master(h, c), h->x[1 - c], h->v[1 - c], xb, vb,
                        ab, 0, 1, x0bar, v0bar);
    }
    if (theta_bar) launch_theta_symmetrise(st, vjp_nrep(h), h->vjp_tacc, theta_bar);
    // the handle returns to the start of the window: (x_0, v_0), step s0,
    // accelerations re-evaluated
    load_state_dev(h, h->win_x, h->win_v0);
    if ((rc = evaluate(h, nullptr, false))) return rc;
    h->steps_host = s0;
    CK(cudaGetLastError());
    return sync_check(h);
}

int mdpd_get_wall_density(mdpd_handle* h, double* phi)
{
    if (!h || !phi) return MDPD_ERR_INVALID_ARG;
    if (!h->want_phi) return h->fail(MDPD_ERR_INVALID_ARG, "MDPD_OPT_WALL_DENSITY is off");
    int rc = sync_check(h);
    if (rc) return rc;
    double* tmp = h->v[1 - h->cur];
    launch_scatter_scalar_by_id(h->stream, h->precision, (int)h->n, h->id[h->cur], h->phi, tmp);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(phi, tmp, (size_t)h->n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    return sync_check(h);
}

int mdpd_autotune(mdpd_handle* h, int32_t reps, int32_t* chosen, double* ms)
{
    if (!h) return MDPD_ERR_INVALID_ARG;
    if (reps < 1) reps = 5;
    int rc = sync_check(h);
    if (rc) return rc;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    // mean time of reps launches of `run` after one warm-up, or < 0 on error
    auto time_it = [&](auto&& run) -> double {
        run();
        cudaEventRecord(e0, h->stream);
        for (int r = 0; r < reps; ++r) run();
        cudaEventRecord(e1, h->stream);
        float t = 0.f;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess)
            return -1.0;
        return (double)t / reps;
    };
    auto done = [&](int code, const char* what) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return code ? h->fail(code, std::string("autotune: ") + what) : MDPD_OK;
    };
    // 1) density variant (the thread-per-particle one in both code shapes;
    //    ms[1] is its faster shape)
    const int variants[3] = { MDPD_KERNELS_NLIST, MDPD_KERNELS_NLIST_THREAD,
                              MDPD_KERNELS_NLIST_THREAD };
    int best = h->kernels, best_shape = h->thread_shape;
    double best_ms = 1e300;
    enqueue_bin(h, true);                     // same positions: same order, state kept
    for (int v = 0; v < 3; ++v) {
        h->kernels = variants[v];
        h->thread_shape = v == 2 ? 1 : 0;
        ensure_ff(h);
        const double t = time_it([&] { enqueue_density(h); });
        if (t < 0) return done(MDPD_ERR_CUDA, cudaGetErrorString(cudaGetLastError()));
        if (ms) ms[v < 1 ? 0 : 1] = v == 2 ? std::min(ms[1], t) : t;
        if (t < best_ms) {
            best_ms = t;
            best = variants[v];
            best_shape = h->thread_shape;
        }
    }
    h->kernels = best;
    h->thread_shape = best_shape;
    enqueue_density(h);                       // rho and lists from the chosen variant
    // 2) lanes per particle of the force pass (evaluation only: the state is kept)
    const int lanes[3] = { 1, 2, 4 };
    int best_l = h->force_lpp;
    best_ms = 1e300;
    for (int v = 0; v < 3; ++v) {
        if (h->nrep && lanes[v] != 1) {
            if (ms) ms[2 + v] = -1.0;
            continue;
        }
        h->force_lpp = lanes[v];
        enqueue_density(h);                   // lists in this setting's layout (untimed)
        const double t = time_it([&] { enqueue_force(h, FM_EVAL, 0, h->fout); });
        if (t < 0) return done(MDPD_ERR_CUDA, cudaGetErrorString(cudaGetLastError()));
        if (ms) ms[2 + v] = t;
        if (t < best_ms) {
            best_ms = t;
            best_l = lanes[v];
        }
    }
    h->force_lpp = best_l;
    enqueue_density(h);                       // lists in the chosen layout
    destroy_graphs(h);
    if (chosen) {
        chosen[0] = best;
        chosen[1] = best_l;
        chosen[2] = h->thread_shape;
    }
    rc = done(MDPD_OK, "");
    if (rc) return rc;
    return sync_check(h);
}

int mdpd_describe(const mdpd_handle* h, int32_t ncell[3], int32_t* launches_per_step)
{
    if (!h) return MDPD_ERR_INVALID_ARG;
    if (ncell)
        for (int k = 0; k < 3; ++k) ncell[k] = h->geo.nc[k];
    if (launches_per_step) *launches_per_step = step_launches(h);
    return MDPD_OK;
}

void mdpd_destroy(mdpd_handle* h)
{
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    destroy_graphs(h);
    free_particles(h);
    dfree(h->count);
    dfree(h->start);
    dfree(h->scan_tmp);
    dfree(h->tile_sums);
    dfree(h->status);
    dfree(h->step);
    dfree(h->red_ticket);
    dfree(h->obs);
    dfree(h->mask_bits);
    dfree(h->d_reps);
    dfree(h->d_reps_all);
    dfree(h->vjp_tpart);
    dfree(h->vjp_tacc);
    dfree(h->vjp_wbar);
    dfree(h->win_x);
    dfree(h->win_vh);
    dfree(h->win_v0);
    dfree(h->win_b);
    dfree(h->d_chunks);
    dfree(h->d_cchunks);
    dfree(h->d_wr);
    dfree(h->obs_b);
    for (auto& e : h->tev)
        if (e) cudaEventDestroy(e);
    for (auto e : h->prof_ev) cudaEventDestroy(e);
    if (h->fork_ev) cudaEventDestroy(h->fork_ev);
    if (h->join_ev) cudaEventDestroy(h->join_ev);
    if (h->side) cudaStreamDestroy(h->side);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

const char* mdpd_last_error(const mdpd_handle* h)
{
    if (!h) return g_create_error.c_str();
    return h->err.c_str();
}

}  // extern "C"
