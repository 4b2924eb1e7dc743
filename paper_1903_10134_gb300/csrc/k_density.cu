// Density pass that also records each mobile particle's force partners
// (arXiv:1903.10134, Sec. 2.1, Algorithm 1 step 4).
//
// Why lists: in a one-thread-per-particle scan of the 27 neighbour cells only
// about 15 % of the candidates lie within r_c, so a force pass scanning cells
// would execute the ~100 operations of a pair force for nearly every
// candidate with most lanes idle.  The density pass already computes every
// candidate distance; it records the candidates within r_c, and the force
// pass (k_force.cu) runs the pair force only for real partners.  A list entry
// is (j << 5) | image code, where the code (0..26) names the neighbour cell
// offset (ox, oy, oz) that fixes the periodic image of j; so j < 2^27.
// Lists are slot-major (nl[k * cap + column]) so consecutive particles store
// consecutive words; the column is the particle's slot, or, under
// ph.list_compact (frozen-split pass), its block's first slot plus its place
// among the block's mobile particles.  Particles with more than NL_MAX
// partners keep only the count, and the force pass scans their cells
// directly.
#include "pair.cuh"

namespace mdpd {

namespace {

__device__ __forceinline__ int image_code(int ox, int oy, int oz)
{
    return (ox + 1) + 3 * (oy + 1) + 9 * (oz + 1);
}

// A scaled density term (at most 2^31 in FP32, 2^50 in FP64) rounded to the
// nearest integer, and a fixed-point sum back in the pair precision.
__device__ __forceinline__ unsigned long long to_fixed(float v)
{
    return (unsigned long long)__float2uint_rn(v);
}
__device__ __forceinline__ unsigned long long to_fixed(double v) { return __double2ull_rn(v); }
__device__ __forceinline__ float from_fixed(unsigned long long a, float inv)
{
    const float hi = __uint2float_rn((uint32_t)(a >> 32));
    const float lo = __uint2float_rn((uint32_t)a);
    return fmaf(hi, 4294967296.0f, lo) * inv;
}
__device__ __forceinline__ double from_fixed(unsigned long long a, double inv)
{
    return __ull2double_rn(a) * inv;
}

// Densities of the frozen particles under the frozen split (see
// k_density_nl): rho = frozen-frozen part + the mobile homes' scattered terms.
template <typename T>
__global__ void __launch_bounds__(PAIR_BLOCK)
k_frozen_rho(int n, Phys ph, const uint32_t* __restrict__ id_s, const T* __restrict__ rho_ff,
             unsigned long long* __restrict__ facc, T* __restrict__ rho_out)
{
    pdl_enter();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const T f = rho_ff[id_s[s]];
    if (f < T(0)) return;                       // a mobile particle
    const unsigned long long a = facc[s];
    rho_out[s] = f + from_fixed(a, derived<T>(ph).fix_inv);
    if (a) facc[s] = 0ull;
}

// Thread-per-particle variant: each thread scans its 27 neighbour cells and
// stores its partners straight to the slot-major list (no shared-memory
// staging, so occupancy is set by registers alone).  The density term is
// evaluated under a branch: on the large porous systems this variant is picked
// for, most warps have no candidate within r_d in an iteration, and a
// branch-free weight (a reciprocal square root per candidate) measured slower.
//
// Frozen split (FS, single systems with frozen particles).  Frozen particles
// never move, so the part of a frozen particle's density that comes from
// frozen neighbours is a constant: FS = 2 computes it once (frozen homes,
// frozen candidates only) into rho_ff[id] (-1 for mobile ids).  FS = 1 then
// scans for mobile homes only: a mobile home adds each frozen candidate's
// share w_rho(r_ij) of that candidate's density (the same term it adds to its
// own) to facc[j] as a fixed-point integer (Derived::fix_scale), by atomic
// addition, so the sum does not depend on the order; k_frozen_rho then forms
// rho_j = rho_ff + facc * fix_inv and clears facc.  Each FS = 1 block gathers
// the mobile homes of FS_ROUNDS * PAIR_BLOCK slots and runs them in rounds of
// PAIR_BLOCK, so no warp is spent on frozen homes.  Homes with partner lists
// (mobile, or every home under list_all) scan everything.
//
// Two code shapes (SH, picked by the autotuner): 0 = candidate loop not
// unrolled, registers as the compiler likes (faster on the porous rock);
// 1 = unrolled by two with at least 8 resident blocks (faster on the batch of
// slabs).  Their results are identical.
// Slots per block of the frozen-split pass, in units of PAIR_BLOCK: a block
// gathers the mobile homes of FS_ROUNDS * PAIR_BLOCK slots and runs them in
// rounds of PAIR_BLOCK, so its warps are full of mobile homes (on a porous
// rock about 45 % of the slots are mobile, and a block of one PAIR_BLOCK
// would keep most of its warps idle while holding its resident-block slot).
constexpr int FS_ROUNDS = FORCE_ROUNDS;      // the same blocks as the force pass's rounds

// The density and partner list of the home in slot s (see k_density_nl).
template <typename T, bool WANT_PHI, int FS, int SH>
__device__ __forceinline__ void density_home(
    int s, int64_t cap, const Geo& geo, const Phys& ph, int64_t cell0,
    const typename Vec4<T>::type* __restrict__ pos4, const uint32_t* __restrict__ cell_s,
    const uint32_t* __restrict__ start, T* __restrict__ rho_out, uint32_t* __restrict__ nl,
    uint32_t* __restrict__ nl_count, unsigned long long* __restrict__ facc,
    const uint32_t* __restrict__ id_s, T* __restrict__ rho_ff, int64_t lcol)
{
    const Derived<T>& dc = derived<T>(ph);
    const T rd2 = dc.rd2, rc2 = dc.rc2;
    const T inv_rd = dc.inv_rd;
    const T cw = dc.cw_rho;
    const auto pi = pos4[s];
    const bool mob_true = ((ph.frozen >> unpack_u32(pi.w)) & 1u) == 0u;
    const bool mobile = ph.list_all || mob_true;
    if (FS == 2 && mobile) {                    // the frozen-frozen part only
        rho_ff[id_s[s]] = T(-1);
        return;
    }
    if (FS == 1 && !mobile) {                   // k_frozen_rho forms the density
        nl_count[s] = 0;
        if (WANT_PHI) ((T*)ph.phi_out)[s] = T(0);
        return;
    }
    // wall density of a mobile particle (WANT_PHI): sum over frozen partners
    // within r_c of 15/(2 pi r_c^3) (1 - r/r_c)^2
    const bool want_phi = WANT_PHI && mob_true;
    const T inv_rc = dc.inv_rc;
    const T cphi = dc.cw_phi;
    T phi = T(0);
    int q0, q1, q2;
    cell_coords(cell_s[s], geo, q0, q1, q2);
    // the scan meets the home itself (r = 0, weight w(0)); that term is taken
    // off at the end unless the self term is asked for
    T acc = T(0);
    uint32_t cnt = 0;
    uint32_t* lp = nl + lcol;                   // next list entry: nl[cnt * cap + lcol]
    for (int oz = -1; oz <= 1; ++oz) {
        const int z = neighbour_index(q2, oz, geo.nc[2], geo.periodic[2]);
        if (z < 0) continue;
        const T sz = pi.z - (T)oz * dc.h[2];
        for (int oy = -1; oy <= 1; ++oy) {
            const int y = neighbour_index(q1, oy, geo.nc[1], geo.periodic[1]);
            if (y < 0) continue;
            const T sy = pi.y - (T)oy * dc.h[1];
            for (int ox = -1; ox <= 1; ++ox) {
                const int x = neighbour_index(q0, ox, geo.nc[0], geo.periodic[0]);
                if (x < 0) continue;
                const T sx = pi.x - (T)ox * dc.h[0];
                const uint32_t code = (uint32_t)image_code(ox, oy, oz);
                const uint32_t nc = (uint32_t)(cell0 + x + geo.nc[0] * (y + geo.nc[1] * z));
                uint32_t b = start[nc], e = start[nc + 1];
                if (!MDPD_DBG_OK(b <= e && e <= (uint32_t)cap, ph.dbg_status)) e = b;
                // the common path is one distance test: r_d <= r_c, so the
                // density term and the list append sit inside the r < r_c
                // branch (about 15 % of the candidates); inside it the density
                // weight is branch-free (zero beyond r_d)
#pragma unroll(SH ? 2 : 1)
                for (uint32_t j = b; j < e; ++j) {
                    const auto pj = pos4[j];
                    const T dx = sx - pj.x, dy = sy - pj.y, dz = sz - pj.z;
                    const T r2 = dx * dx + dy * dy + dz * dz;
                    // (FS = 2 takes frozen candidates only, by type, so it does not
                    // depend on the frozen types the binning ordered by)
                    if (r2 < rc2 && (FS != 2 || ((ph.frozen >> unpack_u32(pj.w)) & 1u))) {
                        const T w = max(T(1) - sqrt_fast(r2) * inv_rd, T(0));
                        const T term = cw * w * w;      // r = 0 gives w(0)
                        acc += term;
                        if (FS == 1 && term > T(0) && ((ph.frozen >> unpack_u32(pj.w)) & 1u))
                            atomicAdd(facc + j, to_fixed(term * dc.fix_scale));
                        if (mobile && r2 > T(0)) {      // not the home, not coincident
                            if (cnt < NL_MAX) {
                                *lp = (j << 5) | code;
                                lp += cap;
                            }
                            ++cnt;
                            if (want_phi && ((ph.frozen >> unpack_u32(pj.w)) & 1u)) {
                                const T wq = T(1) - sqrt_t(r2) * inv_rc;
                                phi += cphi * wq * wq;
                            }
                        }
                    }
                }
            }
        }
    }
    if (!ph.rho_self) acc -= cw;
    if constexpr (FS == 2) {
        rho_ff[id_s[s]] = acc;
        return;
    }
    rho_out[s] = acc;
    nl_count[s] = cnt;
    if (WANT_PHI) ((T*)ph.phi_out)[s] = phi;
}

template <typename T, bool BATCH, bool WANT_PHI, int FS, int SH>
__global__ void __launch_bounds__(PAIR_BLOCK, SH ? 8 : 12)
k_density_nl(int n, int64_t cap, Geo geo_p, Phys ph_p, Batch bt,
             const typename Vec4<T>::type* __restrict__ pos4, const uint32_t* __restrict__ cell_s,
             const uint32_t* __restrict__ start, T* __restrict__ rho_out,
             uint32_t* __restrict__ nl, uint32_t* __restrict__ nl_count,
             unsigned long long* __restrict__ facc, const uint32_t* __restrict__ id_s,
             T* __restrict__ rho_ff)
{
    static_assert(FS == 0 || !BATCH, "the frozen split is for single systems");
    pdl_enter();
    if constexpr (FS == 1) {
        // the mobile homes of the block's FS_ROUNDS * PAIR_BLOCK slots, in
        // slot order; frozen homes only clear their count (k_frozen_rho forms
        // their density)
        __shared__ int act[FS_ROUNDS * PAIR_BLOCK];
        __shared__ uint32_t wcnt[FS_ROUNDS][PAIR_BLOCK / 32];
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        const unsigned lt = (1u << lane) - 1u;
        const int64_t base = (int64_t)blockIdx.x * (FS_ROUNDS * PAIR_BLOCK);
        unsigned bm[FS_ROUNDS];
#pragma unroll
        for (int r = 0; r < FS_ROUNDS; ++r) {
            const int64_t t = base + r * PAIR_BLOCK + threadIdx.x;
            const bool valid = t < n;
            bool mob = false;
            if (valid) {
                mob = ph_p.list_all || ((ph_p.frozen >> unpack_u32(pos4[t].w)) & 1u) == 0u;
                if (!mob) {
                    nl_count[t] = 0;
                    if (WANT_PHI) ((T*)ph_p.phi_out)[t] = T(0);
                }
            }
            bm[r] = __ballot_sync(0xffffffffu, mob);
            if (lane == 0) wcnt[r][warp] = (uint32_t)__popc(bm[r]);
        }
        __syncthreads();
        uint32_t nmob = 0;
#pragma unroll
        for (int r = 0; r < FS_ROUNDS; ++r) {
            uint32_t off = nmob;
#pragma unroll
            for (int w = 0; w < PAIR_BLOCK / 32; ++w) {
                off += w < warp ? wcnt[r][w] : 0u;
                nmob += wcnt[r][w];
            }
            if ((bm[r] >> lane) & 1u)
                act[off + __popc(bm[r] & lt)] = (int)(base + r * PAIR_BLOCK + threadIdx.x);
        }
        __syncthreads();
        // list column: the home's slot, or (list_compact) the block's first
        // slot plus the home's place among its mobile homes, which the force
        // pass's rounds blocks form the same way (consecutive columns for a
        // warp's homes: coalesced list stores and loads)
        for (uint32_t q = threadIdx.x; q < nmob; q += PAIR_BLOCK)
            density_home<T, WANT_PHI, FS, SH>(act[q], cap, geo_p, ph_p, 0, pos4, cell_s, start,
                                              rho_out, nl, nl_count, facc, id_s, rho_ff,
                                              ph_p.list_compact ? base + q : (int64_t)act[q]);
        return;
    }
    int s;
    bool valid;
    int64_t cell0 = 0;
    const Rep* rp = nullptr;
    if constexpr (BATCH) {
        const int4 ch = bt.chunks[blockIdx.x];
        rp = &block_rep<REP_SCALARS>(bt.reps, ch.x);
        s = ch.y + (int)threadIdx.x;
        valid = (int)threadIdx.x < ch.z;
        cell0 = rp->cell0;
    } else {
        s = blockIdx.x * blockDim.x + threadIdx.x;
        valid = s < n;
    }
    if (!valid) return;
    density_home<T, WANT_PHI, FS, SH>(s, cap, BATCH ? rp->geo : geo_p, BATCH ? rp->ph : ph_p,
                                      cell0, pos4, cell_s, start, rho_out, nl, nl_count, facc,
                                      id_s, rho_ff, s);
}

// Warp-cooperative density pass: one warp per home cell.  The 27 neighbour
// cells' particles form one candidate sequence (a warp prefix sum over the
// cells' counts); each lane takes one candidate per round of 32 and tests it
// against up to DC_GROUP home particles broadcast from shared memory, so all
// lanes run the same trip count.  Density terms accumulate per lane and are
// summed with a fixed shuffle tree; partners within r_c of mobile home
// particles are appended by warp ballot to per-particle lists staged in
// shared memory, then written slot-major (nl[k * cap + i]).
constexpr int DC_WARPS = 4;
constexpr int DC_GROUP = 8;
// Candidate sequences up to this length get a table from candidate position
// to neighbour cell, built once per home cell; longer ones (dense regions)
// search the cells' prefix sums instead.
constexpr int DC_MAP = 384;

// The work of one warp on home cell c (global index; cell0 = first cell of
// its replica).  Shared memory is per warp (index w).
template <typename T>
__device__ __forceinline__ void density_cell_warp(int64_t c, int64_t cell0, const Geo& geo,
                                                  const Phys& ph,
                                                  const typename Vec4<T>::type* __restrict__ pos4,
                                                  const uint32_t* __restrict__ start,
                                                  T* __restrict__ rho_out, int64_t cap,
                                                  uint32_t* __restrict__ nl,
                                                  uint32_t* __restrict__ nl_count)
{
    using V = typename Vec4<T>::type;
    __shared__ V hpos[DC_WARPS][DC_GROUP];
    __shared__ uint32_t pre[DC_WARPS][28];
    __shared__ uint32_t cbase[DC_WARPS][27];
    __shared__ uint32_t ccnt[DC_WARPS][DC_GROUP];
    __shared__ uint32_t lst[DC_WARPS][NL_MAX][DC_GROUP];
    __shared__ uint8_t cellmap[DC_WARPS][DC_MAP];
    __shared__ V cshift[DC_WARPS][27];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t hb = start[c], he = start[c + 1];
    if (hb == he) return;                         // whole warp: empty cell
    int q0, q1, q2;
    cell_coords((uint32_t)(c - cell0), geo, q0, q1, q2);
    uint32_t cb = 0, cn = 0;
    if (lane < 27) {
        const int x = neighbour_index(q0, lane % 3 - 1, geo.nc[0], geo.periodic[0]);
        const int y = neighbour_index(q1, (lane / 3) % 3 - 1, geo.nc[1], geo.periodic[1]);
        const int z = neighbour_index(q2, lane / 9 - 1, geo.nc[2], geo.periodic[2]);
        if (x >= 0 && y >= 0 && z >= 0) {
            const uint32_t nc = (uint32_t)(cell0 + x + geo.nc[0] * (y + geo.nc[1] * z));
            cb = start[nc];
            const uint32_t ce = start[nc + 1];
            cn = MDPD_DBG_OK(cb <= ce && ce <= (uint32_t)cap, ph.dbg_status) ? ce - cb : 0u;
        }
    }
    uint32_t inc = cn;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    const uint32_t C = __shfl_sync(0xffffffffu, inc, 31);
    const Derived<T>& dc = derived<T>(ph);
    const T rc2 = dc.rc2;
    const T inv_rd = dc.inv_rd;
    const T cw = dc.cw_rho;
    const unsigned lt = (1u << lane) - 1u;
    const bool use_map = C <= (uint32_t)DC_MAP;   // warp-uniform
    if (lane < 27) {
        pre[w][lane] = inc - cn;
        cbase[w][lane] = cb;
        // the neighbour cell's image shift into the home cell's frame
        cshift[w][lane] = make4((T)(lane % 3 - 1) * dc.h[0], (T)((lane / 3) % 3 - 1) * dc.h[1],
                                (T)(lane / 9 - 1) * dc.h[2], T(0));
        if (use_map)
            for (uint32_t t = inc - cn; t < inc; ++t) cellmap[w][t] = (uint8_t)lane;
    }
    if (lane == 27) pre[w][27] = C;
    __syncwarp();

    // far-away stand-in for the candidate slots past the end of the last round:
    // beyond r_c and r_d of every home particle, finite in FP32
    const T far = T(1e15);
    for (uint32_t g0 = hb; g0 < he; g0 += DC_GROUP) {
        const int ng = (int)min((uint32_t)DC_GROUP, he - g0);
        bool mob_l = false;
        if (lane < ng) {
            const V ph_i = pos4[g0 + lane];
            hpos[w][lane] = ph_i;
            mob_l = ph.list_all || ((ph.frozen >> unpack_u32(ph_i.w)) & 1u) == 0u;
        }
        // home particles that take partner lists (warp-uniform)
        const unsigned mobmask = __ballot_sync(0xffffffffu, mob_l);
        __syncwarp();
        T acc[DC_GROUP];
        uint32_t cnt[DC_GROUP];
#pragma unroll
        for (int i = 0; i < DC_GROUP; ++i) {
            acc[i] = T(0);
            cnt[i] = 0;
        }
        for (uint32_t t0 = 0; t0 < C; t0 += 32) {
            const uint32_t t = t0 + lane;
            const bool valid = t < C;
            int lo = 0;
            if (use_map) {
                lo = valid ? (int)cellmap[w][t] : 0;
            } else {
                int hi = 27;
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (pre[w][mid] <= t) lo = mid;
                    else hi = mid;
                }
            }
            const uint32_t j = valid ? cbase[w][lo] + (t - pre[w][lo]) : hb;
            const V pj = pos4[j];
            // the candidate in the home cell's frame (its image across the
            // neighbour cell offset)
            const V sh = cshift[w][lo];
            const T cx = valid ? pj.x + sh.x : far;
            const T cy = valid ? pj.y + sh.y : far;
            const T cz = valid ? pj.z + sh.z : far;
            const uint32_t entry = (j << 5) | (uint32_t)lo;
#pragma unroll
            for (int i = 0; i < DC_GROUP; ++i) {
                if (i < ng) {
                    const V pi = hpos[w][i];
                    const T dx = pi.x - cx;
                    const T dy = pi.y - cy;
                    const T dz = pi.z - cz;
                    const T r2 = dx * dx + dy * dy + dz * dz;
                    // branch-free weight; the home particle's own r = 0 term is
                    // removed after the loop
                    const T wr = max(T(1) - sqrt_fast(r2) * inv_rd, T(0));
                    acc[i] += cw * wr * wr;
                    if ((mobmask >> i) & 1u) {
                        const bool hc = r2 < rc2 && r2 > T(0);
                        const unsigned m = __ballot_sync(0xffffffffu, hc);
                        if (m) {
                            const uint32_t slot = cnt[i] + (uint32_t)__popc(m & lt);
                            if (hc && slot < (uint32_t)NL_MAX) lst[w][slot][i] = entry;
                            cnt[i] += (uint32_t)__popc(m);
                        }
                    }
                }
            }
        }
        uint32_t maxc = 0;
#pragma unroll
        for (int i = 0; i < DC_GROUP; ++i) {
            if (i < ng) {
                T v = acc[i];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane == 0) {
                    rho_out[g0 + i] = v - (ph.rho_self ? T(0) : cw);
                    nl_count[g0 + i] = cnt[i];
                }
                const uint32_t kept = cnt[i] < (uint32_t)NL_MAX ? cnt[i] : (uint32_t)NL_MAX;
                if (lane == i) ccnt[w][i] = kept;
                maxc = kept > maxc ? kept : maxc;
            }
        }
        __syncwarp();
        for (uint32_t e = lane; e < maxc * DC_GROUP; e += 32) {
            const uint32_t slot = e / DC_GROUP, i = e % DC_GROUP;
            if ((int)i < ng && slot < ccnt[w][i]) nl[(int64_t)slot * cap + g0 + i] = lst[w][slot][i];
        }
        __syncwarp();
    }
}

// One warp per home cell (a block per cell chunk of a batch).  The loops let
// a grid smaller than the lattice walk it; a persistent grid of 16 blocks per
// SM measured no faster than one warp per cell on the porous rock, the batch
// of slabs or the slab.
template <typename T, bool BATCH>
__global__ void __launch_bounds__(DC_WARPS * 32)
k_density_cell(int64_t ncell, int64_t cap, Geo geo_p, Phys ph_p, Batch bt,
               const typename Vec4<T>::type* __restrict__ pos4,
               const uint32_t* __restrict__ start, T* __restrict__ rho_out,
               uint32_t* __restrict__ nl, uint32_t* __restrict__ nl_count)
{
    pdl_enter();
    static_assert(DC_WARPS == BATCH_CELL_CHUNK, "a cell chunk is one block");
    const int w = threadIdx.x >> 5;
    if constexpr (BATCH) {
        for (int b = blockIdx.x; b < bt.ncchunk; b += gridDim.x) {
            const int4 ch = bt.cchunks[b];
            const Rep& rp = block_rep<REP_SCALARS>(bt.reps, ch.x);
            if (w < ch.z)
                density_cell_warp<T>((int64_t)ch.y + w, rp.cell0, rp.geo, rp.ph, pos4, start,
                                     rho_out, cap, nl, nl_count);
            __syncthreads();              // the record is overwritten by the next chunk
        }
    } else {
        for (int64_t c = (int64_t)blockIdx.x * DC_WARPS + w; c < ncell;
             c += (int64_t)gridDim.x * DC_WARPS)
            density_cell_warp<T>(c, 0, geo_p, ph_p, pos4, start, rho_out, cap, nl, nl_count);
    }
}

}  // namespace

template <typename T, int SH>
void density_nl_t(cudaStream_t st, int n, int64_t cap, const Geo& geo, const Phys& ph,
                  const void* pos4, const uint32_t* cell_s, const uint32_t* start, void* rho,
                  uint32_t* nl, uint32_t* nl_count, int fs, unsigned long long* facc,
                  const uint32_t* id_s, void* rho_ff)
{
    using V = typename Vec4<T>::type;
    const int nb = (n + PAIR_BLOCK - 1) / PAIR_BLOCK;
    const int nb1 = (n + FS_ROUNDS * PAIR_BLOCK - 1) / (FS_ROUNDS * PAIR_BLOCK);
    const bool phi = ph.phi_out != nullptr;
    auto k = phi ? k_density_nl<T, false, true, 0, SH> : k_density_nl<T, false, false, 0, SH>;
    if (fs == 1) k = phi ? k_density_nl<T, false, true, 1, SH> : k_density_nl<T, false, false, 1, SH>;
    if (fs == 2) k = k_density_nl<T, false, false, 2, SH>;
    launch_pdl(k, dim3(fs == 1 ? nb1 : nb), dim3(PAIR_BLOCK), st, n, cap, geo, ph, Batch{},
               (const V*)pos4, cell_s, start, (T*)rho, nl, nl_count, facc, id_s, (T*)rho_ff);
    if (fs == 1)
        launch_pdl(k_frozen_rho<T>, dim3(nb), dim3(PAIR_BLOCK), st, n, ph, id_s,
                   (const T*)rho_ff, facc, (T*)rho);
}

void launch_density_nl(cudaStream_t st, int precision, int n, int64_t cap, const Geo& geo,
                       const Phys& ph, const void* pos4, const uint32_t* cell_s,
                       const uint32_t* start, void* rho, uint32_t* nl, uint32_t* nl_count,
                       int fs, unsigned long long* facc, const uint32_t* id_s, void* rho_ff,
                       int shape)
{
    if (n <= 0) return;
    auto f = precision == 0 ? (shape ? density_nl_t<double, 1> : density_nl_t<double, 0>)
                            : (shape ? density_nl_t<float, 1> : density_nl_t<float, 0>);
    f(st, n, cap, geo, ph, pos4, cell_s, start, rho, nl, nl_count, fs, facc, id_s, rho_ff);
}

void launch_density_nl_batch(cudaStream_t st, int precision, int64_t cap, const Batch& bt,
                             const void* pos4, const uint32_t* cell_s, const uint32_t* start,
                             void* rho, uint32_t* nl, uint32_t* nl_count, int shape)
{
    if (bt.nchunk <= 0) return;
    const dim3 g(bt.nchunk), b(PAIR_BLOCK);
    if (precision == 0)
        launch_pdl_smem(shape ? k_density_nl<double, true, false, 0, 1>
                              : k_density_nl<double, true, false, 0, 0>,
                        g, b, REP_SMEM, st, 0, cap, Geo{}, Phys{}, bt, (const D4*)pos4, cell_s,
                        start, (double*)rho, nl, nl_count, nullptr, nullptr, nullptr);
    else
        launch_pdl_smem(shape ? k_density_nl<float, true, false, 0, 1>
                              : k_density_nl<float, true, false, 0, 0>,
                        g, b, REP_SMEM, st, 0, cap, Geo{}, Phys{}, bt, (const float4*)pos4, cell_s,
                        start, (float*)rho, nl, nl_count, nullptr, nullptr, nullptr);
}

void launch_density_cell(cudaStream_t st, int precision, int64_t ncell, int64_t cap,
                         const Geo& geo, const Phys& ph, const void* pos4, const uint32_t* start,
                         void* rho, uint32_t* nl, uint32_t* nl_count)
{
    if (ncell <= 0) return;
    const unsigned nb = (unsigned)((ncell + DC_WARPS - 1) / DC_WARPS);
    if (precision == 0)
        launch_pdl(k_density_cell<double, false>, dim3(nb), dim3(DC_WARPS * 32), st, ncell, cap,
                   geo, ph, Batch{}, (const D4*)pos4, start, (double*)rho, nl, nl_count);
    else
        launch_pdl(k_density_cell<float, false>, dim3(nb), dim3(DC_WARPS * 32), st, ncell, cap,
                   geo, ph, Batch{}, (const float4*)pos4, start, (float*)rho, nl, nl_count);
}

void launch_density_cell_batch(cudaStream_t st, int precision, int64_t cap, const Batch& bt,
                               const void* pos4, const uint32_t* start, void* rho, uint32_t* nl,
                               uint32_t* nl_count)
{
    if (bt.ncchunk <= 0) return;
    const dim3 g(bt.ncchunk), b(DC_WARPS * 32);
    if (precision == 0)
        launch_pdl_smem(k_density_cell<double, true>, g, b, REP_SMEM, st, 0, cap, Geo{}, Phys{},
                        bt, (const D4*)pos4, start, (double*)rho, nl, nl_count);
    else
        launch_pdl_smem(k_density_cell<float, true>, g, b, REP_SMEM, st, 0, cap, Geo{}, Phys{},
                        bt, (const float4*)pos4, start, (float*)rho, nl, nl_count);
}

}  // namespace mdpd
