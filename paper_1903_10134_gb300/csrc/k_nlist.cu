// Density pass that also records each mobile particle's force partners, and
// the force pass that walks those lists (arXiv:1903.10134, Sec. 2.1, Eq. 1,
// Algorithm 1 steps 4 and 6).
//
// Why: in a one-thread-per-particle scan of the 27 neighbour cells only about
// 15 % of the candidates lie within r_c, so a warp would execute the ~100
// operations of a pair force for nearly every candidate with most lanes idle.
// The density pass already computes every candidate distance; it appends the
// candidates within r_c to a per-thread list in shared memory (conflict-free,
// column per thread) and writes the list out slot by slot, so consecutive
// threads store consecutive words.  The force pass then runs the pair force
// only for real partners.  A list entry is (j << 5) | image code, where the
// code (0..26) names the neighbour cell offset (ox, oy, oz) that fixes the
// periodic image of j; so j < 2^27.  Particles with more than NL_MAX partners
// are scanned directly by the force pass.
#include "pair.cuh"

namespace mdpd {

namespace {

__device__ __forceinline__ int image_code(int ox, int oy, int oz)
{
    return (ox + 1) + 3 * (oy + 1) + 9 * (oz + 1);
}

// Thread-per-particle variant: each thread scans its 27 neighbour cells and
// stores its partners straight to the slot-major list (no shared-memory
// staging, so occupancy is set by registers alone).  The density term is
// evaluated under a branch: on the large porous systems this variant is picked
// for, most warps have no candidate within r_d in an iteration, and a
// branch-free weight (a reciprocal square root per candidate) measured slower.
template <typename T, bool BATCH, bool WANT_PHI>
__global__ void __launch_bounds__(PAIR_BLOCK, 12)
k_density_nl(int n, int64_t cap, Geo geo_p, Phys ph_p, Batch bt,
             const typename Vec4<T>::type* __restrict__ pos4, const uint32_t* __restrict__ cell_s,
             const uint32_t* __restrict__ start, T* __restrict__ rho_out,
             uint32_t* __restrict__ nl, uint32_t* __restrict__ nl_count)
{
    pdl_enter();
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
    const Geo& geo = BATCH ? rp->geo : geo_p;
    const Phys& ph = BATCH ? rp->ph : ph_p;
    const Derived<T>& dc = derived<T>(ph);
    const T rd2 = dc.rd2, rc2 = dc.rc2;
    const T inv_rd = dc.inv_rd;
    const T cw = dc.cw_rho;
    const auto pi = pos4[s];
    const bool mob_true = ((ph.frozen >> unpack_u32(pi.w)) & 1u) == 0u;
    const bool mobile = ph.list_all || mob_true;
    // wall density of a mobile particle (WANT_PHI): sum over frozen partners
    // within r_c of 15/(2 pi r_c^3) (1 - r/r_c)^2
    const bool want_phi = WANT_PHI && mob_true;
    const T inv_rc = dc.inv_rc;
    const T cphi = dc.cw_phi;
    T phi = T(0);
    int q0, q1, q2;
    cell_coords(cell_s[s], geo, q0, q1, q2);
    T acc = ph.rho_self ? cw : T(0);
    uint32_t cnt = 0;
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
                const uint32_t b = start[nc], e = start[nc + 1];
                for (uint32_t j = b; j < e; ++j) {
                    const auto pj = pos4[j];
                    const T dx = sx - pj.x, dy = sy - pj.y, dz = sz - pj.z;
                    const T r2 = dx * dx + dy * dy + dz * dz;
                    const bool other = j != (uint32_t)s;
                    if (other && r2 < rd2) {
                        const T w = T(1) - sqrt_t(r2) * inv_rd;
                        acc += cw * w * w;
                    }
                    if (other && mobile && r2 < rc2 && r2 > T(0)) {
                        if (cnt < NL_MAX) nl[(int64_t)cnt * cap + s] = (j << 5) | code;
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
    rho_out[s] = acc;
    nl_count[s] = cnt;
    if (WANT_PHI) ((T*)ph.phi_out)[s] = phi;
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

template <typename T, bool BATCH>
__global__ void __launch_bounds__(DC_WARPS * 32)
k_density_cell(int64_t ncell, int64_t cap, Geo geo_p, Phys ph_p, Batch bt,
               const typename Vec4<T>::type* __restrict__ pos4,
               const uint32_t* __restrict__ start, T* __restrict__ rho_out,
               uint32_t* __restrict__ nl, uint32_t* __restrict__ nl_count)
{
    pdl_enter();
    using V = typename Vec4<T>::type;
    static_assert(DC_WARPS == BATCH_CELL_CHUNK, "a cell chunk is one block");
    __shared__ V hpos[DC_WARPS][DC_GROUP];
    __shared__ uint32_t pre[DC_WARPS][28];
    __shared__ uint32_t cbase[DC_WARPS][27];
    __shared__ uint32_t ccnt[DC_WARPS][DC_GROUP];
    __shared__ uint32_t lst[DC_WARPS][NL_MAX][DC_GROUP];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t c, cell0 = 0;           // global cell, first cell of the replica
    bool valid;
    const Rep* rp = nullptr;
    if constexpr (BATCH) {
        const int4 ch = bt.cchunks[blockIdx.x];
        rp = &block_rep<REP_SCALARS>(bt.reps, ch.x);
        c = (int64_t)ch.y + w;
        valid = w < ch.z;
        cell0 = rp->cell0;
    } else {
        c = (int64_t)blockIdx.x * DC_WARPS + w;
        valid = c < ncell;
    }
    if (!valid) return;                           // whole warp
    const Geo& geo = BATCH ? rp->geo : geo_p;
    const Phys& ph = BATCH ? rp->ph : ph_p;
    const uint32_t hb = start[c], he = start[c + 1];
    if (hb == he) return;                         // whole warp
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
            cn = start[nc + 1] - cb;
        }
    }
    uint32_t inc = cn;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    const uint32_t C = __shfl_sync(0xffffffffu, inc, 31);
    if (lane < 27) {
        pre[w][lane] = inc - cn;
        cbase[w][lane] = cb;
    }
    if (lane == 27) pre[w][27] = C;
    __syncwarp();

    const Derived<T>& dc = derived<T>(ph);
    const T rc2 = dc.rc2;
    const T inv_rd = dc.inv_rd;
    const T cw = dc.cw_rho;
    const T hx = dc.h[0], hy = dc.h[1], hz = dc.h[2];
    const unsigned lt = (1u << lane) - 1u;

    for (uint32_t g0 = hb; g0 < he; g0 += DC_GROUP) {
        const int ng = (int)min((uint32_t)DC_GROUP, he - g0);
        if (lane < ng) hpos[w][lane] = pos4[g0 + lane];
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
            int lo = 0, hi = 27;
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (pre[w][mid] <= t) lo = mid;
                else hi = mid;
            }
            const uint32_t j = valid ? cbase[w][lo] + (t - pre[w][lo]) : hb;
            const V pj = pos4[j];
            const T shx = (T)(lo % 3 - 1) * hx;
            const T shy = (T)((lo / 3) % 3 - 1) * hy;
            const T shz = (T)(lo / 9 - 1) * hz;
            const uint32_t entry = (j << 5) | (uint32_t)lo;
#pragma unroll
            for (int i = 0; i < DC_GROUP; ++i) {
                if (i < ng) {
                    const V pi = hpos[w][i];
                    const T dx = pi.x - shx - pj.x;
                    const T dy = pi.y - shy - pj.y;
                    const T dz = pi.z - shz - pj.z;
                    const T r2 = dx * dx + dy * dy + dz * dz;
                    // branch-free weight; the home particle's own r = 0 term is
                    // removed after the loop
                    const T wr = valid ? max(T(1) - sqrt0_t(r2) * inv_rd, T(0)) : T(0);
                    acc[i] += cw * wr * wr;
                    const bool mob = ph.list_all || ((ph.frozen >> unpack_u32(pi.w)) & 1u) == 0u;
                    const bool hc = valid && mob && r2 < rc2 && r2 > T(0);
                    const unsigned m = __ballot_sync(0xffffffffu, hc);
                    if (m) {
                        const uint32_t slot = cnt[i] + (uint32_t)__popc(m & lt);
                        if (hc && slot < (uint32_t)NL_MAX) lst[w][slot][i] = entry;
                        cnt[i] += (uint32_t)__popc(m);
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

// Force pass over the partner lists.  The particles of a block (128
// consecutive in cell order) are first compacted so that the mobile ones sit
// on the leading lanes (frozen wall particles need no force), then each of
// those lanes walks its list with a two-stage software prefetch: list entries
// two ahead, partner data one ahead.
// Minimum resident blocks per SM asked of the FP32 force kernel (0: the
// compiler's default, kept for FP64).  The pair loop is latency-bound on its
// partner gathers, so occupancy pays more than the few registers it costs: 8
// blocks (64 registers, a 12-byte spill) measured 13 % faster than the
// default 94 registers on the 4.4M-particle rock, and 8 beat 4 to 12 on a
// batch (whose scalar constants sit in shared memory and take registers).
#ifndef MDPD_FORCE_BATCH_MIN_BLOCKS
#define MDPD_FORCE_BATCH_MIN_BLOCKS 8
#endif
#ifndef MDPD_FORCE_MIN_BLOCKS
#define MDPD_FORCE_MIN_BLOCKS 8
#endif
template <typename T, bool BATCH, int LPP>
constexpr int force_min_blocks()
{
    // several lanes per particle hold the group reduction's values too: 4 blocks
    return sizeof(T) != 4 ? 0
                          : (BATCH ? MDPD_FORCE_BATCH_MIN_BLOCKS
                                   : (LPP > 1 ? 4 : MDPD_FORCE_MIN_BLOCKS));
}

// LPP lanes share one particle: lane `sub` of the group takes the list
// entries sub, sub + LPP, ...; the group's sums are combined with a fixed
// butterfly.  LPP > 1 multiplies the warps of a small system (a 48k-particle
// slab fills only 2.5 blocks per SM at one lane per particle).
template <typename T, int MODE, bool BATCH, int LPP>
__global__ void __launch_bounds__(PAIR_BLOCK, (force_min_blocks<T, BATCH, LPP>()))
k_force_nl(int n, int64_t cap, Geo geo_p, Phys ph_p, Batch bt, MaskDev mk,
           const typename Vec4<T>::type* __restrict__ pos4,
           const typename Vec4<T>::type* __restrict__ vel4, const T* __restrict__ rho,
           const uint32_t* __restrict__ cell_s, const uint32_t* __restrict__ start,
           const uint32_t* __restrict__ nl, const uint32_t* __restrict__ nl_count,
           const uint64_t* __restrict__ step_ptr, int step_offset, Master m,
           double* __restrict__ out, double* __restrict__ partials, uint32_t* __restrict__ status)
{
    pdl_enter();
    using V = typename Vec4<T>::type;
    static_assert(LPP == 1 || LPP == 2 || LPP == 4, "lanes per particle");
    static_assert(!BATCH || LPP == 1, "a batch chunk is one particle per lane");
    constexpr int PPB = PAIR_BLOCK / LPP;        // particles per block
    __shared__ PairTables<T> tab;
    __shared__ T shift[27][3];
    __shared__ int act[PAIR_BLOCK];
    __shared__ int wsum[PAIR_BLOCK / 32];
    int s0;
    bool in_range;
    int64_t cell0 = 0;
    const Rep* rp = nullptr;
    int rep_r = 0;
    if constexpr (BATCH) {
        const int4 ch = bt.chunks[blockIdx.x];
        rp = &block_rep<REP_SCALARS>(bt.reps, ch.x);
        rep_r = ch.x;
        s0 = ch.y + (int)threadIdx.x;
        in_range = (int)threadIdx.x < ch.z;
        cell0 = rp->cell0;
    } else {
        s0 = blockIdx.x * PPB + threadIdx.x;
        in_range = (int)threadIdx.x < PPB && s0 < n;
    }
    const Geo& geo = BATCH ? rp->geo : geo_p;
    const Phys& ph = BATCH ? rp->ph : ph_p;      // in a batch: scalars only (see block_rep)
    load_tables(tab, BATCH ? bt.reps[rep_r].ph : ph_p);
    if (threadIdx.x < 27) {
        const int c = threadIdx.x;
        const Derived<T>& dc = derived<T>(ph);
        shift[c][0] = (T)(c % 3 - 1) * dc.h[0];
        shift[c][1] = (T)((c / 3) % 3 - 1) * dc.h[1];
        shift[c][2] = (T)(c / 9 - 1) * dc.h[2];
    }
    // compact the block's mobile particles onto the first lanes, in cell order
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool mob0 = in_range && ((ph.frozen >> m.type[s0]) & 1u) == 0u;
    const unsigned bal = __ballot_sync(0xffffffffu, mob0);
    if (lane == 0) wsum[warp] = __popc(bal);
    __syncthreads();
    int woff = 0, nact = 0;
#pragma unroll
    for (int w = 0; w < PAIR_BLOCK / 32; ++w) {
        woff += w < warp ? wsum[w] : 0;
        nact += wsum[w];
    }
    if (mob0) act[woff + __popc(bal & ((1u << lane) - 1u))] = s0;
    if (MODE == FM_EVAL && in_range && !mob0) {
#pragma unroll
        for (int k = 0; k < 3; ++k) out[k * cap + s0] = 0.0;
    }
    __syncthreads();

    const uint64_t step = *step_ptr + (uint64_t)step_offset;
    T obs[NOBS];
#pragma unroll
    for (int k = 0; k < NOBS; ++k) obs[k] = T(0);
    const int slot = (int)threadIdx.x / LPP, sub = (int)threadIdx.x % LPP;
    const bool active = slot < nact;
    const int s = active ? act[slot] : 0;
    T f[3] = { T(0), T(0), T(0) };
    T W[6] = { T(0), T(0), T(0), T(0), T(0), T(0) };
    int npair = 0;
    if (active) {
        const PairConst<T> c(ph);
        const V pi = pos4[s];
        const V vi = vel4[s];
        const T rho_i = rho[s];
        const uint32_t ti = unpack_u32(pi.w);
        const uint32_t id_i = unpack_u32(vi.w);
        const T* tA = tab.A + ti * 8;
        const T* tB = tab.B + ti * 8;
        const T* tG = tab.G + ti * 8;
        const T* tS = tab.S + ti * 8;
        const uint32_t cnt = nl_count[s];
        if (cnt <= (uint32_t)NL_MAX) {
            const uint32_t k0 = (uint32_t)sub;
            uint32_t e0 = k0 < cnt ? nl[(int64_t)k0 * cap + s] : 0u;
            uint32_t e1 = k0 + LPP < cnt ? nl[(int64_t)(k0 + LPP) * cap + s] : 0u;
            V pj = pos4[e0 >> 5];
            V vj = vel4[e0 >> 5];
            T rj = rho[e0 >> 5];
            for (uint32_t k = k0; k < cnt; k += LPP) {
                const uint32_t e2 = k + 2 * LPP < cnt ? nl[(int64_t)(k + 2 * LPP) * cap + s] : 0u;
                const V pn = pos4[e1 >> 5];
                const V vn = vel4[e1 >> 5];
                const T rn = rho[e1 >> 5];
                const uint32_t code = e0 & 31u;
                const T dx = pi.x - shift[code][0] - pj.x;
                const T dy = pi.y - shift[code][1] - pj.y;
                const T dz = pi.z - shift[code][2] - pj.z;
                const T r2 = dx * dx + dy * dy + dz * dz;
                pair_term(c, tA, tB, tG, tS, dx, dy, dz, r2, vi, vj, rho_i, rj,
                          unpack_u32(pj.w), id_i, unpack_u32(vj.w), step, ph, f, W);
                e0 = e1;
                e1 = e2;
                pj = pn;
                vj = vn;
                rj = rn;
            }
            npair = sub == 0 ? (int)cnt : 0;
        } else if (sub == 0) {
            // more partners than list slots: scan the 27 neighbour cells
            int q0, q1, q2;
            cell_coords(cell_s[s], geo, q0, q1, q2);
            for (int oz = -1; oz <= 1; ++oz) {
                const int z = neighbour_index(q2, oz, geo.nc[2], geo.periodic[2]);
                if (z < 0) continue;
                for (int oy = -1; oy <= 1; ++oy) {
                    const int y = neighbour_index(q1, oy, geo.nc[1], geo.periodic[1]);
                    if (y < 0) continue;
                    for (int ox = -1; ox <= 1; ++ox) {
                        const int x = neighbour_index(q0, ox, geo.nc[0], geo.periodic[0]);
                        if (x < 0) continue;
                        const int code = image_code(ox, oy, oz);
                        const uint32_t nc = (uint32_t)(cell0 + x + geo.nc[0] * (y + geo.nc[1] * z));
                        const uint32_t b = start[nc], e = start[nc + 1];
                        for (uint32_t j = b; j < e; ++j) {
                            const V pj = pos4[j];
                            const T dx = pi.x - shift[code][0] - pj.x;
                            const T dy = pi.y - shift[code][1] - pj.y;
                            const T dz = pi.z - shift[code][2] - pj.z;
                            const T r2 = dx * dx + dy * dy + dz * dz;
                            if (r2 < c.rc2 && r2 > T(0)) {
                                const V vj = vel4[j];
                                pair_term(c, tA, tB, tG, tS, dx, dy, dz, r2, vi, vj, rho_i,
                                          rho[j], unpack_u32(pj.w), id_i, unpack_u32(vj.w),
                                          step, ph, f, W);
                                ++npair;
                            }
                        }
                    }
                }
            }
        }
    }
    if constexpr (LPP > 1) {
        // every lane of the warp takes part (inactive groups add zeros)
#pragma unroll
        for (int o = 1; o < LPP; o <<= 1) {
#pragma unroll
            for (int k = 0; k < 3; ++k) f[k] += __shfl_xor_sync(0xffffffffu, f[k], o);
#pragma unroll
            for (int k = 0; k < 6; ++k) W[k] += __shfl_xor_sync(0xffffffffu, W[k], o);
            npair += __shfl_xor_sync(0xffffffffu, npair, o);
        }
    }
    if (active && sub == 0)
        force_finish<T, MODE>(s, true, f, W, npair, cap, geo, ph, mk, m, out, obs, status);
    warp_obs_store(obs, partials, (int64_t)gridDim.x * (PAIR_BLOCK / 32));
}

template <typename T, bool BATCH, int LPP>
void launch_force_nl_t(cudaStream_t st, ForceMode mode, int n, int64_t cap, const Geo& geo,
                       const Phys& ph, const Batch& bt, const MaskDev& mk, const void* pos4,
                       const void* vel4, const void* rho, const uint32_t* cell_s,
                       const uint32_t* start, const uint32_t* nl, const uint32_t* nl_count,
                       const uint64_t* step_ptr, int step_offset, const Master& m, double* out,
                       double* partials, uint32_t* status)
{
    using V = typename Vec4<T>::type;
    const int nb = BATCH ? bt.nchunk : force_num_blocks(n, LPP);
    const size_t smem = BATCH ? REP_SMEM : 0;
    const V* p = (const V*)pos4;
    const V* v = (const V*)vel4;
    const T* r = (const T*)rho;
#define MDPD_FNL(MODE_)                                                                    \
    launch_pdl_smem(k_force_nl<T, MODE_, BATCH, LPP>, dim3(nb), dim3(PAIR_BLOCK), smem, st, n, \
                    cap, geo, ph, bt, mk, p, v, r, cell_s, start, nl, nl_count, step_ptr,    \
                    step_offset, m, out, partials, status)
    if (mode == FM_EVAL) MDPD_FNL(FM_EVAL);
    else if (mode == FM_LAST) MDPD_FNL(FM_LAST);
    else MDPD_FNL(FM_FUSED);
#undef MDPD_FNL
}

template <typename T>
void launch_force_nl_lpp(cudaStream_t st, ForceMode mode, int n, int64_t cap, const Geo& geo,
                         const Phys& ph, int lpp, const MaskDev& mk, const void* pos4,
                         const void* vel4, const void* rho, const uint32_t* cell_s,
                         const uint32_t* start, const uint32_t* nl, const uint32_t* nl_count,
                         const uint64_t* step_ptr, int step_offset, const Master& m, double* out,
                         double* partials, uint32_t* status)
{
    if (lpp == 4)
        launch_force_nl_t<T, false, 4>(st, mode, n, cap, geo, ph, Batch{}, mk, pos4, vel4, rho,
                                       cell_s, start, nl, nl_count, step_ptr, step_offset, m, out,
                                       partials, status);
    else if (lpp == 2)
        launch_force_nl_t<T, false, 2>(st, mode, n, cap, geo, ph, Batch{}, mk, pos4, vel4, rho,
                                       cell_s, start, nl, nl_count, step_ptr, step_offset, m, out,
                                       partials, status);
    else
        launch_force_nl_t<T, false, 1>(st, mode, n, cap, geo, ph, Batch{}, mk, pos4, vel4, rho,
                                       cell_s, start, nl, nl_count, step_ptr, step_offset, m, out,
                                       partials, status);
}

}  // namespace

void launch_density_nl(cudaStream_t st, int precision, int n, int64_t cap, const Geo& geo,
                       const Phys& ph, const void* pos4, const uint32_t* cell_s,
                       const uint32_t* start, void* rho, uint32_t* nl, uint32_t* nl_count)
{
    if (n <= 0) return;
    const int nb = (n + PAIR_BLOCK - 1) / PAIR_BLOCK;
    const bool phi = ph.phi_out != nullptr;
    if (precision == 0)
        launch_pdl(phi ? k_density_nl<double, false, true> : k_density_nl<double, false, false>,
                   dim3(nb), dim3(PAIR_BLOCK), st, n, cap, geo, ph, Batch{}, (const D4*)pos4,
                   cell_s, start, (double*)rho, nl, nl_count);
    else
        launch_pdl(phi ? k_density_nl<float, false, true> : k_density_nl<float, false, false>,
                   dim3(nb), dim3(PAIR_BLOCK), st, n, cap, geo, ph, Batch{}, (const float4*)pos4,
                   cell_s, start, (float*)rho, nl, nl_count);
}

void launch_density_nl_batch(cudaStream_t st, int precision, int64_t cap, const Batch& bt,
                             const void* pos4, const uint32_t* cell_s, const uint32_t* start,
                             void* rho, uint32_t* nl, uint32_t* nl_count)
{
    if (bt.nchunk <= 0) return;
    const dim3 g(bt.nchunk), b(PAIR_BLOCK);
    if (precision == 0)
        launch_pdl_smem(k_density_nl<double, true, false>, g, b, REP_SMEM, st, 0, cap, Geo{}, Phys{},
                        bt, (const D4*)pos4, cell_s, start, (double*)rho, nl, nl_count);
    else
        launch_pdl_smem(k_density_nl<float, true, false>, g, b, REP_SMEM, st, 0, cap, Geo{}, Phys{},
                        bt, (const float4*)pos4, cell_s, start, (float*)rho, nl, nl_count);
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

void launch_force_nl(cudaStream_t st, int precision, ForceMode mode, int n, int64_t cap,
                     const Geo& geo, const Phys& ph, int lpp, const MaskDev& mk, const void* pos4,
                     const void* vel4, const void* rho, const uint32_t* cell_s,
                     const uint32_t* start, const uint32_t* nl, const uint32_t* nl_count,
                     const uint64_t* step_ptr, int step_offset, const Master& m, double* out,
                     double* partials, uint32_t* status)
{
    if (precision == 0)
        launch_force_nl_lpp<double>(st, mode, n, cap, geo, ph, lpp, mk, pos4, vel4, rho, cell_s,
                                    start, nl, nl_count, step_ptr, step_offset, m, out, partials,
                                    status);
    else
        launch_force_nl_lpp<float>(st, mode, n, cap, geo, ph, lpp, mk, pos4, vel4, rho, cell_s,
                                   start, nl, nl_count, step_ptr, step_offset, m, out, partials,
                                   status);
}

void launch_force_nl_batch(cudaStream_t st, int precision, ForceMode mode, int64_t cap,
                           const Batch& bt, const void* pos4, const void* vel4, const void* rho,
                           const uint32_t* cell_s, const uint32_t* start, const uint32_t* nl,
                           const uint32_t* nl_count, const uint64_t* step_ptr, int step_offset,
                           const Master& m, double* out, double* partials, uint32_t* status)
{
    const MaskDev none{};
    if (bt.nchunk <= 0) return;
    if (precision == 0)
        launch_force_nl_t<double, true, 1>(st, mode, 0, cap, Geo{}, Phys{}, bt, none, pos4, vel4, rho,
                                        cell_s, start, nl, nl_count, step_ptr, step_offset, m,
                                        out, partials, status);
    else
        launch_force_nl_t<float, true, 1>(st, mode, 0, cap, Geo{}, Phys{}, bt, none, pos4, vel4, rho,
                                       cell_s, start, nl, nl_count, step_ptr, step_offset, m,
                                       out, partials, status);
}

}  // namespace mdpd
