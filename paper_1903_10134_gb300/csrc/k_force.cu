// Force pass over the partner lists written by the density pass (k_density.cu),
// fused with the velocity-Verlet epilogue (arXiv:1903.10134, Sec. 2.1, Eq. 1,
// Algorithm 1 steps 6 and 7).  A list entry is (j << 5) | image code (see
// k_density.cu); particles with more than NL_MAX partners are scanned directly.
#include "pair.cuh"

namespace mdpd {

namespace {

__device__ __forceinline__ int image_code(int ox, int oy, int oz)
{
    return (ox + 1) + 3 * (oy + 1) + 9 * (oz + 1);
}

// Force pass over the partner lists.  The particles of a block (FR * 128
// consecutive in cell order) are first compacted so that the mobile ones sit
// on the leading lanes (frozen wall particles need no force), then each of
// those lanes walks its list with a two-stage software prefetch: list entries
// two ahead, partner data one ahead.  With frozen particles (FR = FORCE_ROUNDS)
// a block gathers the mobile particles of several blocks' worth of slots and
// runs them in rounds of 128, so its warps stay full instead of idling beside
// the wall particles while they hold the block's resident slot.
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
template <typename T, int MODE, bool BATCH, int LPP, int FR>
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
    static_assert(FR == 1 || (LPP == 1 && !BATCH), "rounds: one lane per particle, one system");
    constexpr int PPB = PAIR_BLOCK / LPP;        // particles per round
    __shared__ PairTables<T> tab;
    __shared__ V shift[27];                      // image shift of neighbour-cell code (xyz)
    __shared__ int act[FR * PAIR_BLOCK];
    __shared__ int wsum[FR][PAIR_BLOCK / 32];
    __shared__ T robs[FR > 1 ? NOBS : 1][PAIR_BLOCK];   // observables summed over rounds
    int64_t cell0 = 0;
    const Rep* rp = nullptr;
    int rep_r = 0;
    int4 ch = make_int4(0, 0, 0, 0);
    if constexpr (BATCH) {
        ch = bt.chunks[blockIdx.x];
        rp = &block_rep<REP_SCALARS>(bt.reps, ch.x);
        rep_r = ch.x;
        cell0 = rp->cell0;
    }
    const Geo& geo = BATCH ? rp->geo : geo_p;
    const Phys& ph = BATCH ? rp->ph : ph_p;      // in a batch: scalars only (see block_rep)
    load_tables(tab, BATCH ? bt.reps[rep_r].ph : ph_p);
    if (threadIdx.x < 27) {
        const int c = threadIdx.x;
        const Derived<T>& dc = derived<T>(ph);
        shift[c] = make4((T)(c % 3 - 1) * dc.h[0], (T)((c / 3) % 3 - 1) * dc.h[1],
                         (T)(c / 9 - 1) * dc.h[2], T(0));
    }
    // compact the block's mobile particles onto the first lanes, in cell order
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int s0[FR];
    unsigned bal[FR];
#pragma unroll
    for (int r = 0; r < FR; ++r) {
        bool in_range;
        if constexpr (BATCH) {
            s0[r] = ch.y + (int)threadIdx.x;
            in_range = (int)threadIdx.x < ch.z;
        } else {
            s0[r] = (blockIdx.x * FR + r) * PPB + threadIdx.x;
            in_range = (int)threadIdx.x < PPB && s0[r] < n;
        }
        const bool mob0 = in_range && ((ph.frozen >> m.type[s0[r]]) & 1u) == 0u;
        bal[r] = __ballot_sync(0xffffffffu, mob0);
        if (lane == 0) wsum[r][warp] = __popc(bal[r]);
        if (MODE == FM_EVAL && in_range && !mob0) {
#pragma unroll
            for (int k = 0; k < 3; ++k) out[k * cap + s0[r]] = 0.0;
        }
    }
    __syncthreads();
    int nact = 0;
#pragma unroll
    for (int r = 0; r < FR; ++r) {
        int woff = nact;
#pragma unroll
        for (int w = 0; w < PAIR_BLOCK / 32; ++w) {
            woff += w < warp ? wsum[r][w] : 0;
            nact += wsum[r][w];
        }
        if ((bal[r] >> lane) & 1u) act[woff + __popc(bal[r] & ((1u << lane) - 1u))] = s0[r];
    }
    __syncthreads();

    const uint64_t step = *step_ptr + (uint64_t)step_offset;
    T obs[NOBS];
#pragma unroll
    for (int k = 0; k < NOBS; ++k) obs[k] = T(0);
    if constexpr (FR > 1) {
#pragma unroll
        for (int k = 0; k < NOBS; ++k) robs[k][threadIdx.x] = T(0);
    }
    const int sub = (int)threadIdx.x % LPP;
    // rounds of PPB particles (block-uniform count, so every lane joins the
    // group reductions of every round)
    const int nround = FR == 1 ? 1 : (nact + PPB - 1) / PPB;
    for (int round = 0; round < nround; ++round) {
        const int slot = round * PPB + (int)threadIdx.x / LPP;
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
            const V* tP = tab.P + ti * 8;
            const uint32_t cnt = nl_count[s];
            // list column (see k_density_nl): the slot, or under list_compact
            // (rounds blocks only) the block's first slot plus the place among
            // its mobile particles, which the density pass formed the same way
            const int64_t lcol = (FR > 1 && ph.list_compact)
                                     ? (int64_t)blockIdx.x * (FR * PPB) + slot : (int64_t)s;
            if (cnt <= (uint32_t)NL_MAX) {
                const uint32_t k0 = (uint32_t)sub;
                // (debug build: an entry naming a slot beyond the arrays or a code
                // beyond 26 is reported and replaced by entry 0, so the access
                // stays inside the arrays; the result is then wrong and flagged)
                auto entry = [&](uint32_t k) -> uint32_t {
                    if (k >= cnt) return 0u;
                    const uint32_t e = nl[(int64_t)k * cap + lcol];
                    return MDPD_DBG_OK((e >> 5) < (uint32_t)cap && (e & 31u) < 27u, ph.dbg_status)
                               ? e : 0u;
                };
                uint32_t e0 = entry(k0);
                uint32_t e1 = entry(k0 + LPP);
                V pj = pos4[e0 >> 5];
                V vj = vel4[e0 >> 5];
                T rj = rho[e0 >> 5];
                for (uint32_t k = k0; k < cnt; k += LPP) {
                    const uint32_t e2 = entry(k + 2 * LPP);
                    const V pn = pos4[e1 >> 5];
                    const V vn = vel4[e1 >> 5];
                    const T rn = rho[e1 >> 5];
                    const V sh = shift[e0 & 31u];
                    const T dx = pi.x - sh.x - pj.x;
                    const T dy = pi.y - sh.y - pj.y;
                    const T dz = pi.z - sh.z - pj.z;
                    const T r2 = dx * dx + dy * dy + dz * dz;
                    pair_term<T, !BATCH>(c, tP[unpack_u32(pj.w)], dx, dy, dz, r2, vi, vj, rho_i, rj,
                                         id_i, unpack_u32(vj.w), step, ph, f, W);
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
                            const uint32_t b = start[nc];
                            uint32_t e = start[nc + 1];
                            if (!MDPD_DBG_OK(b <= e && e <= (uint32_t)cap, ph.dbg_status)) e = b;
                            for (uint32_t j = b; j < e; ++j) {
                                const V pj = pos4[j];
                                const V sh = shift[code];
                                const T dx = pi.x - sh.x - pj.x;
                                const T dy = pi.y - sh.y - pj.y;
                                const T dz = pi.z - sh.z - pj.z;
                                const T r2 = dx * dx + dy * dy + dz * dz;
                                if (r2 < c.rc2 && r2 > T(0)) {
                                    const V vj = vel4[j];
                                    pair_term<T, !BATCH>(c, tP[unpack_u32(pj.w)], dx, dy, dz, r2, vi,
                                                         vj, rho_i, rho[j], id_i, unpack_u32(vj.w),
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
        if (active && sub == 0) {
            if constexpr (FR == 1) {
                force_finish<T, MODE>(s, true, f, W, npair, cap, geo, ph, mk, m, out, obs, status);
            } else {
                // force_finish sets one particle's observables; the rounds are
                // added in the thread's shared-memory column (registers held
                // across the rounds would spill)
                force_finish<T, MODE>(s, true, f, W, npair, cap, geo, ph, mk, m, out, obs, status);
#pragma unroll
                for (int k = 0; k < NOBS; ++k) {
                    robs[k][threadIdx.x] += obs[k];
                    obs[k] = T(0);
                }
            }
        }
    }
    if constexpr (FR > 1) {
#pragma unroll
        for (int k = 0; k < NOBS; ++k) obs[k] = robs[k][threadIdx.x];
    }
    warp_obs_store(obs, partials, (int64_t)gridDim.x * (PAIR_BLOCK / 32));
}

template <typename T, bool BATCH, int LPP, int FR = 1>
void launch_force_nl_t(cudaStream_t st, ForceMode mode, int n, int64_t cap, const Geo& geo,
                       const Phys& ph, const Batch& bt, const MaskDev& mk, const void* pos4,
                       const void* vel4, const void* rho, const uint32_t* cell_s,
                       const uint32_t* start, const uint32_t* nl, const uint32_t* nl_count,
                       const uint64_t* step_ptr, int step_offset, const Master& m, double* out,
                       double* partials, uint32_t* status)
{
    using V = typename Vec4<T>::type;
    const int nb = BATCH ? bt.nchunk : force_num_blocks(n, LPP, FR);
    const size_t smem = BATCH ? REP_SMEM : 0;
    const V* p = (const V*)pos4;
    const V* v = (const V*)vel4;
    const T* r = (const T*)rho;
#define MDPD_FNL(MODE_)                                                                    \
    launch_pdl_smem(k_force_nl<T, MODE_, BATCH, LPP, FR>, dim3(nb), dim3(PAIR_BLOCK), smem, st, n, \
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
    else if (force_nl_rounds(ph, 1) > 1)
        launch_force_nl_t<T, false, 1, FORCE_ROUNDS>(st, mode, n, cap, geo, ph, Batch{}, mk, pos4,
                                                     vel4, rho, cell_s, start, nl, nl_count,
                                                     step_ptr, step_offset, m, out, partials,
                                                     status);
    else
        launch_force_nl_t<T, false, 1>(st, mode, n, cap, geo, ph, Batch{}, mk, pos4, vel4, rho,
                                       cell_s, start, nl, nl_count, step_ptr, step_offset, m, out,
                                       partials, status);
}

}  // namespace

int force_nl_rounds(const Phys& ph, int lpp) { return lpp == 1 && ph.frozen ? FORCE_ROUNDS : 1; }

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
