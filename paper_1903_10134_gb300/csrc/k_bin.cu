// Cell binning by a counting sort (per step): cell id of every particle (with
// the step's first half-kick and drift when asked), per-cell counts, an
// exclusive scan, a scatter in atomic order, and one kernel that ranks each
// particle inside its cell by (frozen, id) (so the order inside a cell does
// not depend on the order of the atomics, and a cell's mobile particles come
// first) and gathers the state into that order with positions re-expressed as
// offsets from the cell centre.
#include "pair.cuh"

namespace mdpd {

namespace {

constexpr int BLOCK = 256;

// exclusive scan of the cell counts: tiles of SCAN_TILE cells, one block each
constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

inline unsigned nblocks(int64_t n, int b = BLOCK) { return (unsigned)((n + b - 1) / b); }

// Batched kernels (BATCH = true) take their replica from the chunk of the
// block (see Batch); single-system kernels index by the global thread id.
// KICK: first apply the step's first half-kick, drift and reflection to the
// particle (the work of a separate kick launch at the start of mdpd_step).
// tsum (or nullptr): the scan's per-tile sums of the counts, added here (one
// atomic per tile and warp: consecutive particles mostly share a tile), so
// that the scan needs no launch of its own to form them.  Used for lattices
// of few tiles; with many, the atomics cost more than the launch they save.
template <bool BATCH, bool KICK>
__global__ void k_bin_count(int n, int64_t cap, Geo geo_p, Phys ph_p, Batch bt, MaskDev mk,
                            Master m, uint32_t* __restrict__ cellof, uint32_t* __restrict__ slot,
                            uint32_t* __restrict__ count, uint32_t* __restrict__ tsum,
                            uint32_t* __restrict__ status)
{
    pdl_enter();
    int i;
    bool valid;
    int64_t cell0 = 0;
    const Rep* rp = nullptr;
    if constexpr (BATCH) {
        const int4 ch = bt.chunks[blockIdx.x];
        rp = &block_rep<REP_SCALARS>(bt.reps, ch.x);     // the FP32 cell constants too
        i = ch.y + (int)threadIdx.x;
        valid = (int)threadIdx.x < ch.z;
        cell0 = rp->cell0;
    } else {
        i = blockIdx.x * blockDim.x + threadIdx.x;
        valid = i < n;
    }
    const unsigned act = __ballot_sync(0xffffffffu, valid);
    if (!valid) return;
    const Geo& geo = BATCH ? rp->geo : geo_p;
    const Phys& ph = BATCH ? rp->ph : ph_p;
    if constexpr (KICK) kick_drift_one(i, cap, geo, ph, mk, m, status);
    int q[3];
    uint32_t st = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const double xk = m.x[k * cap + i];
        // FP64 instructions run at 1/64 of the FP32 rate: the cell index is
        // taken in FP32 and recomputed in FP64 within 2e-3 cell edges of a
        // face, where FP32 rounding could pick the neighbour (on the axes
        // fill_derived marks, the FP32 error is below 4e-4 edges), so the
        // result is always the FP64 one
        const float t = (to_f32(xk) - ph.df.lo[k]) * ph.df.inv_h[k];
        if (!isfinite(t)) {
            st |= ST_NONFINITE;
            q[k] = 0;
            continue;
        }
        const float fl = floorf(t);
        int c = (int)fl;
        const bool exact = ((ph.fast_cell >> k) & 1u) && t - fl > 2e-3f && fl + 1.0f - t > 2e-3f;
        // the FP64 index behind a branch that a warp takes only when one of
        // its lanes needs it (if-converted, its four FP64 instructions ran
        // for every particle and were most of this kernel's time)
        if (__any_sync(__activemask(), !exact)) {
            if (!exact) c = (int)floor_index_f64(xk, geo.lo[k], geo.inv_h[k], 0.0, 0);
        }
        // the face test on order-preserving integer keys of the FP64 bits
        // (f64_key), under a uniform branch: as FP64 comparisons it cost
        // most of this kernel's time (FP64 runs at 1/64 of the FP32 rate)
        if (!geo.periodic[k]) {
            const int64_t kx = f64_key(xk);
            if (kx < geo.key_lo[k] || kx >= geo.key_hi[k]) st |= ST_OUT_OF_BOX;
        }
        c = c < 0 ? 0 : (c >= geo.nc[k] ? geo.nc[k] - 1 : c);
        q[k] = c;
    }
    if (st) atomicOr(status, st);
    const uint32_t c = (uint32_t)(cell0 + q[0] + geo.nc[0] * (q[1] + geo.nc[1] * q[2]));
    cellof[i] = c;
    // arrival slot, with the frozen flag in the top bit (it orders a cell's
    // frozen particles after its mobile ones)
    const uint32_t fz = (ph.frozen >> m.type[i]) & 1u;
    slot[i] = atomicAdd(&count[c], 1u) | (fz << 31);
    if (tsum != nullptr) {                     // uniform over the launch
        const uint32_t tile = c / (uint32_t)SCAN_TILE;
        const unsigned peers = __match_any_sync(act, tile);
        if ((threadIdx.x & 31) == (unsigned)(__ffs(peers) - 1))
            atomicAdd(&tsum[tile], (uint32_t)__popc(peers));
    }
}

// ---- exclusive scan ------------------------------------------------------------

// Exclusive prefix of v over the block; *total receives the block sum.
__device__ uint32_t block_exclusive(uint32_t v, uint32_t* total)
{
    __shared__ uint32_t wsum[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarp = blockDim.x >> 5;
    uint32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < nwarp ? wsum[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        wsum[lane] = w;
    }
    __syncthreads();
    const uint32_t base = warp > 0 ? wsum[warp - 1] : 0u;
    *total = wsum[nwarp - 1];
    __syncthreads();
    return base + incl - v;
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_blocks(const uint32_t* __restrict__ in,
                                                              int64_t n, uint32_t* __restrict__ sums)
{
    pdl_enter();
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k)
        if (base + k < n) s += in[base + k];
    uint32_t total;
    block_exclusive(s, &total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// Second pass: block b first adds the sums of the blocks before it (each
// block does this itself, so no third launch scans the block sums), then
// writes its tile's exclusive prefix.  Block 0 writes out[n], the total.
// zero_in: clear in[] after reading it.
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_apply(uint32_t* __restrict__ in,
                                                             int64_t n,
                                                             const uint32_t* __restrict__ sums,
                                                             int nb, uint32_t* __restrict__ out,
                                                             int zero_in,
                                                             uint32_t* __restrict__ zero_sums)
{
    pdl_enter();
    // the binning's tile sums alternate between two buffers: clear the other
    if (zero_sums && threadIdx.x == 0) zero_sums[blockIdx.x] = 0u;
    __shared__ uint32_t before_sh;
    const int b = (int)blockIdx.x;
    uint32_t mine = 0, all = 0;
    for (int q = threadIdx.x; q < nb; q += SCAN_THREADS) {
        const uint32_t t = sums[q];
        mine += q < b ? t : 0u;
        all += t;
    }
    uint32_t tot;
    block_exclusive(mine, &tot);
    if (threadIdx.x == 0) before_sh = tot;
    uint32_t grand;
    block_exclusive(all, &grand);
    const uint32_t before = before_sh;
    const int64_t base = (int64_t)b * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    uint32_t v[SCAN_ITEMS], s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        v[k] = base + k < n ? in[base + k] : 0u;
        s += v[k];
    }
    uint32_t total;
    uint32_t run = block_exclusive(s, &total) + before;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        if (base + k < n) {
            out[base + k] = run;
            if (zero_in) in[base + k] = 0u;
        }
        run += v[k];
    }
    if (b == 0 && threadIdx.x == 0) out[n] = grand;
}

__global__ void k_bin_scatter(int n, const uint32_t* __restrict__ cellof,
                              const uint32_t* __restrict__ slot, const uint32_t* __restrict__ start,
                              const uint32_t* __restrict__ id, uint32_t* __restrict__ key,
                              uint32_t* __restrict__ src, uint32_t* __restrict__ status)
{
    pdl_enter();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t sl = slot[i];
    const uint32_t dst = start[cellof[i]] + (sl & 0x7fffffffu);
    if (dst >= (uint32_t)n) {          // inconsistent counts: report, write nothing
        atomicOr(status, ST_OVERFLOW);
        return;
    }
    key[dst] = id[i] | (sl & 0x80000000u);
    src[dst] = (uint32_t)i;
}

// Insertion sort of each cell's slots by particle id; also clears the cell's
// count, so the counts are zero whenever a binning starts.
__global__ void k_cell_sort(int64_t ncell, const uint32_t* __restrict__ start,
                            uint32_t* __restrict__ key, uint32_t* __restrict__ src,
                            uint32_t* __restrict__ count)
{
    pdl_enter();
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    count[c] = 0u;      // the counts are consumed; leave them zero for the next binning
    const uint32_t b = start[c], e = start[c + 1];
    for (uint32_t a = b + 1; a < e; ++a) {
        const uint32_t k = key[a], s = src[a];
        uint32_t p = a;
        while (p > b && key[p - 1] > k) {
            key[p] = key[p - 1];
            src[p] = src[p - 1];
            --p;
        }
        key[p] = k;
        src[p] = s;
    }
}

// Order inside each cell by (frozen, particle id), fused with the gather into
// cell order.  The scatter filled slot a (in atomic order)
// with key[a] = frozen << 31 | id and
// src[a] = the particle's master index i; the particle's place in its cell c
// is s = start[c] + (number of keys of the cell below key[a]), and the thread
// copies particle i's master state to slot s of the other buffer and writes
// the compute arrays of slot s: position as FP32/FP64 offset from the cell
// centre with the type bits, velocity with the id (within the replica).
template <typename T, bool BATCH>
__global__ void k_rank_gather(int n, int64_t cap, const uint32_t* __restrict__ cellof,
                              const uint32_t* __restrict__ start, const uint32_t* __restrict__ key,
                              const uint32_t* __restrict__ src, Master in, Master out,
                              int gather_a, Geo geo_p, Phys ph_p, Batch bt,
                              typename Vec4<T>::type* __restrict__ pos4,
                              typename Vec4<T>::type* __restrict__ vel4,
                              uint32_t* __restrict__ cell_s)
{
    pdl_enter();
    int a;
    bool valid;
    int64_t cell0 = 0;
    uint32_t id0 = 0;
    const Rep* rp = nullptr;
    if constexpr (BATCH) {
        const int4 ch = bt.chunks[blockIdx.x];
        rp = &block_rep<REP_SCALARS>(bt.reps, ch.x);
        a = ch.y + (int)threadIdx.x;
        valid = (int)threadIdx.x < ch.z;
        cell0 = rp->cell0;
        id0 = rp->id0;
    } else {
        a = blockIdx.x * blockDim.x + threadIdx.x;
        valid = a < n;
    }
    if (!valid) return;
    const Geo& geo = BATCH ? rp->geo : geo_p;
    const Phys& ph_g = BATCH ? rp->ph : ph_p;
    const uint32_t i = src[a];
    if (i >= (uint32_t)cap) return;        // slot never written (counts inconsistent: reported)
    const uint32_t cg = cellof[i];
    const uint32_t b = start[cg], e = start[cg + 1];
    if (e > (uint32_t)cap || b > e) return;
    const uint32_t kk = key[a];
    uint32_t r = 0;
    for (uint32_t q = b; q < e; ++q) r += key[q] < kk ? 1u : 0u;
    const uint32_t s = b + r;
    const uint32_t c = cg - (uint32_t)cell0;      // cell within the replica
    const int q[3] = { (int)(c % (uint32_t)geo.nc[0]),
                       (int)((c / (uint32_t)geo.nc[0]) % (uint32_t)geo.nc[1]),
                       (int)(c / ((uint32_t)geo.nc[0] * (uint32_t)geo.nc[1])) };
    double xv[3], vv[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        xv[k] = in.x[k * cap + i];
        vv[k] = in.v[k * cap + i];
        out.x[k * cap + s] = xv[k];
        out.v[k * cap + s] = vv[k];
        if (gather_a) out.a[k * cap + s] = in.a[k * cap + i];
    }
    const uint32_t pid = in.id[i];
    const uint8_t pt = in.type[i];
    out.id[s] = pid;
    out.type[s] = pt;
    cell_s[s] = c;
    // offset from the cell centre lo + (q + 1/2) h, taken in FP64 (the
    // centre as one fused multiply-add on the host-made lo + h/2)
    // (FP32: no FP64 instruction, see cell_offset_f32; FP64: one fused
    // multiply-add and one subtraction)
    T off[3];
    bool done = false;
    if constexpr (sizeof(T) == 4) {
        const Derived<float>& f = ph_g.df;
        done = true;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            float o;
            done &= cell_offset_f32(xv[k], q[k], f.h[k], f.h_lo[k], f.c0[k], f.c0_lo[k], &o);
            off[k] = o;
        }
    }
    // FP64 pairs, or a coordinate outside the FP32 split's range (a
    // warp-voted branch: FP64 instructions cost 64 FP32 issue slots)
    if (__any_sync(__activemask(), !done)) {
        if (!done) {
#pragma unroll
            for (int k = 0; k < 3; ++k)
                off[k] = to_t<T>(xv[k] - fma((double)q[k], geo.h[k], ph_g.dd.c0[k]));
        }
    }
    pos4[s] = make4(off[0], off[1], off[2], pack_u32(T(0), (uint32_t)pt));
    // the random stream is keyed on ids within the replica
    vel4[s] = make4(to_t<T>(vv[0]), to_t<T>(vv[1]), to_t<T>(vv[2]), pack_u32(T(0), pid - id0));
}

// Load a state given in id order (pos/vel interleaved xyz) into the master
// arrays (index = id), wrapping periodic axes.
template <bool BATCH>
__global__ void k_load_state(int n, int64_t cap, const double* __restrict__ pos3,
                             const double* __restrict__ vel3, const double* __restrict__ acc3,
                             Geo geo_p, Batch bt, Master m,
                             const uint8_t* __restrict__ type_by_id, uint32_t* __restrict__ status)
{
    pdl_enter();
    int i;
    bool valid;
    const Rep* rp = nullptr;
    if constexpr (BATCH) {
        const int4 ch = bt.chunks[blockIdx.x];
        rp = &block_rep<REP_GEO>(bt.reps, ch.x);
        i = ch.y + (int)threadIdx.x;
        valid = (int)threadIdx.x < ch.z;
    } else {
        i = blockIdx.x * blockDim.x + threadIdx.x;
        valid = i < n;
    }
    if (!valid) return;
    const Geo& geo = BATCH ? rp->geo : geo_p;
    uint32_t st = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        double x = pos3[3 * i + k];
        const double v = vel3[3 * i + k];
        if (!isfinite(x) || !isfinite(v)) st |= ST_NONFINITE;
        // a position in [lo, key_in) is left as it is (there x - lo rounds to
        // [0, L), so the wrap below would not change it); the FP64 division
        // runs only for the others, under a branch a warp takes when one of
        // its lanes needs it (FP64 runs at 1/64 of the FP32 rate)
        const int64_t kx = f64_key(x);
        const bool wrap = geo.periodic[k] && isfinite(x) && (kx < geo.key_lo[k] || kx >= geo.key_in[k]);
        if (__any_sync(__activemask(), wrap)) {
            if (wrap) {
                const double w = floor((x - geo.lo[k]) / geo.L[k]);
                if (w != 0.0) x -= geo.L[k] * w;      // in-box positions stay bit-identical
                if (x >= geo.hi[k] || x < geo.lo[k]) x = geo.lo[k];
            }
        }
        m.x[k * cap + i] = x;
        m.v[k * cap + i] = v;
        m.a[k * cap + i] = acc3 ? acc3[3 * i + k] : 0.0;
    }
    if (st) atomicOr(status, st);
    m.id[i] = (uint32_t)i;
    m.type[i] = type_by_id[i];
}

__global__ void k_scatter_vec_by_id(int n, int64_t cap, const uint32_t* __restrict__ id,
                                    const double* __restrict__ v, double* __restrict__ out)
{
    pdl_enter();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const uint32_t d = id[s];
#pragma unroll
    for (int k = 0; k < 3; ++k) out[3 * (int64_t)d + k] = v[k * cap + s];
}

template <typename T>
__global__ void k_scatter_scalar_by_id(int n, const uint32_t* __restrict__ id,
                                       const T* __restrict__ r, double* __restrict__ out)
{
    pdl_enter();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    out[id[s]] = (double)r[s];
}

__global__ void k_scatter_type_by_id(int n, const uint32_t* __restrict__ id,
                                     const uint8_t* __restrict__ t, int32_t* __restrict__ out)
{
    pdl_enter();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    out[id[s]] = (int32_t)t[s];
}

}  // namespace

void launch_bin_count(cudaStream_t st, int n, int64_t cap, const Geo& geo, const Phys& ph,
                      const MaskDev& mk, const Master& m, bool kick, uint32_t* cellof,
                      uint32_t* slot, uint32_t* count, uint32_t* tsum, uint32_t* status)
{
    if (n <= 0) return;
    launch_pdl(kick ? k_bin_count<false, true> : k_bin_count<false, false>, dim3(nblocks(n)),
               dim3(BLOCK), st, n, cap, geo, ph, Batch{}, mk, m, cellof, slot, count, tsum,
               status);
}

void launch_bin_count_batch(cudaStream_t st, int64_t cap, const Batch& bt, const Master& m,
                            bool kick, uint32_t* cellof, uint32_t* slot, uint32_t* count,
                            uint32_t* tsum, uint32_t* status)
{
    if (bt.nchunk <= 0) return;
    launch_pdl_smem(kick ? k_bin_count<true, true> : k_bin_count<true, false>, dim3(bt.nchunk),
                    dim3(BATCH_CHUNK), REP_SMEM, st, 0, cap, Geo{}, Phys{}, bt, MaskDev{}, m,
                    cellof, slot, count, tsum, status);
}

int scan_num_blocks(int64_t n) { return (int)((n + SCAN_TILE - 1) / SCAN_TILE); }

int scan_num_launches(int64_t n) { return scan_fused_sums(n) ? 1 : 2; }

bool scan_fused_sums(int64_t n) { return scan_num_blocks(n) <= 64; }

void launch_exclusive_scan(cudaStream_t st, uint32_t* in, int64_t n, uint32_t* out, uint32_t* tmp,
                           bool zero_in)
{
    const int nb = scan_num_blocks(n);
    if (nb <= 0) return;
    launch_pdl(k_scan_blocks, dim3(nb), dim3(SCAN_THREADS), st, in, n, tmp);
    launch_pdl(k_scan_apply, dim3(nb), dim3(SCAN_THREADS), st, in, n, tmp, nb, out, (int)zero_in,
               (uint32_t*)nullptr);
}

__global__ void k_add_carry(uint32_t* __restrict__ out, int64_t len, const uint32_t* __restrict__ carry)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < len) out[i] += *carry;
}

void launch_exclusive_scan_long(cudaStream_t st, uint32_t* in, int64_t n, uint32_t* out,
                                uint32_t* tmp, uint32_t* carry, int64_t seg)
{
    for (int64_t s0 = 0; s0 < n; s0 += seg) {
        const int64_t len = n - s0 < seg ? n - s0 : seg;
        // the running total before s0 (written at out[s0] by the previous
        // segment's fix-up) is saved before this segment's scan overwrites it
        if (s0 > 0) cudaMemcpyAsync(carry, out + s0, sizeof(uint32_t), cudaMemcpyDeviceToDevice, st);
        launch_exclusive_scan(st, in + s0, len, out + s0, tmp, false);
        if (s0 > 0)
            k_add_carry<<<(unsigned)((len + 1 + 255) / 256), 256, 0, st>>>(out + s0, len + 1, carry);
    }
}

void launch_scan_from_sums(cudaStream_t st, uint32_t* in, int64_t n, uint32_t* out,
                           const uint32_t* sums, uint32_t* zero_sums)
{
    const int nb = scan_num_blocks(n);
    if (nb <= 0) return;
    launch_pdl(k_scan_apply, dim3(nb), dim3(SCAN_THREADS), st, in, n, sums, nb, out, 1, zero_sums);
}

void launch_bin_scatter(cudaStream_t st, int n, const uint32_t* cellof, const uint32_t* slot,
                        const uint32_t* start, const uint32_t* id, uint32_t* key, uint32_t* src,
                        uint32_t* status)
{
    if (n <= 0) return;
    launch_pdl(k_bin_scatter, dim3(nblocks(n)), dim3(BLOCK), st, n, cellof, slot, start, id, key, src,
               status);
}

void launch_cell_sort(cudaStream_t st, int64_t ncell, const uint32_t* start, uint32_t* key,
                      uint32_t* src, uint32_t* count)
{
    if (ncell <= 0) return;
    launch_pdl(k_cell_sort, dim3(nblocks(ncell)), dim3(BLOCK), st, ncell, start, key, src, count);
}

void launch_rank_gather(cudaStream_t st, int precision, int n, int64_t cap,
                        const uint32_t* cellof, const uint32_t* start, const uint32_t* key,
                        const uint32_t* src, const Master& in, const Master& out, bool gather_a,
                        const Geo& geo, const Phys& ph, void* pos4, void* vel4, uint32_t* cell_s)
{
    if (n <= 0) return;
    if (precision == 0)
        launch_pdl(k_rank_gather<double, false>, dim3(nblocks(n)), dim3(BLOCK), st, n, cap, cellof,
                   start, key, src, in, out, (int)gather_a, geo, ph, Batch{}, (D4*)pos4, (D4*)vel4,
                   cell_s);
    else
        launch_pdl(k_rank_gather<float, false>, dim3(nblocks(n)), dim3(BLOCK), st, n, cap, cellof,
                   start, key, src, in, out, (int)gather_a, geo, ph, Batch{}, (float4*)pos4,
                   (float4*)vel4, cell_s);
}

void launch_rank_gather_batch(cudaStream_t st, int precision, int64_t cap, const uint32_t* cellof,
                              const uint32_t* start, const uint32_t* key, const uint32_t* src,
                              const Master& in, const Master& out, bool gather_a, const Batch& bt,
                              void* pos4, void* vel4, uint32_t* cell_s)
{
    if (bt.nchunk <= 0) return;
    const dim3 g(bt.nchunk), b(BATCH_CHUNK);
    if (precision == 0)
        launch_pdl_smem(k_rank_gather<double, true>, g, b, REP_SMEM, st, 0, cap, cellof, start, key,
                        src, in, out, (int)gather_a, Geo{}, Phys{}, bt, (D4*)pos4, (D4*)vel4, cell_s);
    else
        launch_pdl_smem(k_rank_gather<float, true>, g, b, REP_SMEM, st, 0, cap, cellof, start, key,
                        src, in, out, (int)gather_a, Geo{}, Phys{}, bt, (float4*)pos4, (float4*)vel4,
                        cell_s);
}

__global__ void k_frozen_moved(int n, int64_t cap, const double* __restrict__ x,
                               const double* __restrict__ ref, const uint8_t* __restrict__ type_by_id,
                               uint32_t frozen, uint32_t* __restrict__ moved)
{
    pdl_enter();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !((frozen >> type_by_id[i]) & 1u)) return;
    bool diff = false;
#pragma unroll
    for (int k = 0; k < 3; ++k)
        diff |= __double_as_longlong(x[k * cap + i]) != __double_as_longlong(ref[3 * i + k]);
    if (diff) atomicOr(moved, 1u);
}

void launch_frozen_moved(cudaStream_t st, int n, int64_t cap, const double* x, const double* ref,
                         const uint8_t* type_by_id, uint32_t frozen, uint32_t* moved)
{
    if (n <= 0) return;
    launch_pdl(k_frozen_moved, dim3(nblocks(n)), dim3(BLOCK), st, n, cap, x, ref, type_by_id,
               frozen, moved);
}

void launch_load_state(cudaStream_t st, int n, int64_t cap, const double* pos3,
                       const double* vel3, const double* acc3, const Geo& geo, const Master& m,
                       const uint8_t* type_by_id, uint32_t* status)
{
    if (n <= 0) return;
    launch_pdl(k_load_state<false>, dim3(nblocks(n)), dim3(BLOCK), st, n, cap, pos3, vel3, acc3,
               geo, Batch{}, m, type_by_id, status);
}

void launch_load_state_batch(cudaStream_t st, int64_t cap, const double* pos3, const double* vel3,
                             const double* acc3, const Batch& bt, const Master& m,
                             const uint8_t* type_by_id, uint32_t* status)
{
    if (bt.nchunk <= 0) return;
    launch_pdl_smem(k_load_state<true>, dim3(bt.nchunk), dim3(BATCH_CHUNK), REP_SMEM, st, 0, cap,
                    pos3, vel3, acc3, Geo{}, bt, m, type_by_id, status);
}

void launch_scatter_by_id(cudaStream_t st, int n, int64_t cap, const uint32_t* id,
                          const double* vec3, double* out3)
{
    if (n <= 0) return;
    launch_pdl(k_scatter_vec_by_id, dim3(nblocks(n)), dim3(BLOCK), st, n, cap, id, vec3, out3);
}

void launch_scatter_scalar_by_id(cudaStream_t st, int precision, int n, const uint32_t* id,
                                 const void* r, double* out)
{
    if (n <= 0) return;
    if (precision == 0)
        launch_pdl(k_scatter_scalar_by_id<double>, dim3(nblocks(n)), dim3(BLOCK), st, n, id, (const double*)r, out);
    else
        launch_pdl(k_scatter_scalar_by_id<float>, dim3(nblocks(n)), dim3(BLOCK), st, n, id, (const float*)r, out);
}

void launch_scatter_type_by_id(cudaStream_t st, int n, const uint32_t* id, const uint8_t* type,
                               int32_t* out)
{
    if (n <= 0) return;
    launch_pdl(k_scatter_type_by_id, dim3(nblocks(n)), dim3(BLOCK), st, n, id, type, out);
}

}  // namespace mdpd
