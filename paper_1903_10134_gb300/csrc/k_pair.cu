// Pair passes of the mDPD step (arXiv:1903.10134):
//   density pass  rho_i = sum_{j != i, r < r_d} 15/(2 pi r_d^3)(1 - r/r_d)^2   (Sec. 2.1)
//   force pass    F_i = sum_{j, 0 < r < r_c} [A w_C + B (rho_i + rho_j) w_d
//                       - gamma w_C^2 (e.v_ij) + sigma w_C xi_ij / sqrt(dt)] e  (Sec. 2.1, Eq. 1)
// fused with the velocity-Verlet half-kicks, the drift and the wall reflection
// (Algorithm 1), plus per-block FP64 partial sums of the observables.
// One thread per particle in cell order; neighbours are the particles of the
// 27 surrounding cells (edge >= r_c), read through the read-only data cache.
#include "pair.cuh"

namespace mdpd {

namespace {

template <typename T>
__global__ void __launch_bounds__(PAIR_BLOCK)
k_density(int n, Geo geo, Phys ph, const typename Vec4<T>::type* __restrict__ pos4,
          const uint32_t* __restrict__ cell_s, const uint32_t* __restrict__ start,
          T* __restrict__ rho_out)
{
    pdl_enter();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const Derived<T>& dc = derived<T>(ph);
    const T rd2 = dc.rd2;
    const T inv_rd = dc.inv_rd;
    const T cw = dc.cw_rho;
    const auto pi = pos4[s];
    const uint32_t c = cell_s[s];
    const int q0 = (int)(c % (uint32_t)geo.nc[0]);
    const int q1 = (int)((c / (uint32_t)geo.nc[0]) % (uint32_t)geo.nc[1]);
    const int q2 = (int)(c / ((uint32_t)geo.nc[0] * (uint32_t)geo.nc[1]));
    T acc = ph.rho_self ? cw : T(0);
    for (int oz = -1; oz <= 1; ++oz) {
        int z = q2 + oz;
        if (z < 0 || z >= geo.nc[2]) {
            if (!geo.periodic[2]) continue;
            z = z < 0 ? z + geo.nc[2] : z - geo.nc[2];
        }
        const T sz = pi.z - (T)oz * derived<T>(ph).h[2];
        for (int oy = -1; oy <= 1; ++oy) {
            int y = q1 + oy;
            if (y < 0 || y >= geo.nc[1]) {
                if (!geo.periodic[1]) continue;
                y = y < 0 ? y + geo.nc[1] : y - geo.nc[1];
            }
            const T sy = pi.y - (T)oy * derived<T>(ph).h[1];
            for (int ox = -1; ox <= 1; ++ox) {
                int x = q0 + ox;
                if (x < 0 || x >= geo.nc[0]) {
                    if (!geo.periodic[0]) continue;
                    x = x < 0 ? x + geo.nc[0] : x - geo.nc[0];
                }
                const T sx = pi.x - (T)ox * derived<T>(ph).h[0];
                const uint32_t nc = (uint32_t)(x + geo.nc[0] * (y + geo.nc[1] * z));
                const uint32_t b = start[nc];
                uint32_t e = start[nc + 1];
                if (!MDPD_DBG_OK(b <= e && e <= (uint32_t)n, ph.dbg_status)) e = b;
                for (uint32_t j = b; j < e; ++j) {
                    if (j == (uint32_t)s) continue;
                    const auto pj = pos4[j];
                    const T dx = sx - pj.x, dy = sy - pj.y, dz = sz - pj.z;
                    const T r2 = dx * dx + dy * dy + dz * dz;
                    if (r2 < rd2) {
                        const T r = sqrt(r2);
                        const T w = T(1) - r * inv_rd;
                        acc += cw * w * w;
                    }
                }
            }
        }
    }
    rho_out[s] = acc;
}

// Direct-scan force pass: each thread tests the particles of its 27 neighbour
// cells itself.  Kept as the baseline variant and for rows of cells too dense
// for a neighbour list.
template <typename T, int MODE>
__global__ void __launch_bounds__(PAIR_BLOCK)
k_force(int n, int64_t cap, Geo geo, Phys ph, MaskDev mk,
        const typename Vec4<T>::type* __restrict__ pos4,
        const typename Vec4<T>::type* __restrict__ vel4, const T* __restrict__ rho,
        const uint32_t* __restrict__ cell_s, const uint32_t* __restrict__ start,
        const uint64_t* __restrict__ step_ptr, int step_offset, Master m,
        double* __restrict__ out, double* __restrict__ partials, uint32_t* __restrict__ status)
{
    pdl_enter();
    __shared__ PairTables<T> tab;
    load_tables(tab, ph);
    __syncthreads();
    const uint64_t step = *step_ptr + (uint64_t)step_offset;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    T obs[NOBS];
#pragma unroll
    for (int k = 0; k < NOBS; ++k) obs[k] = T(0);
    if (s < n) {
        const PairConst<T> c(ph);
        const auto pi = pos4[s];
        const auto vi = vel4[s];
        const T rho_i = rho[s];
        const uint32_t ti = unpack_u32(pi.w);
        const uint32_t id_i = unpack_u32(vi.w);
        const bool mobile = ((ph.frozen >> ti) & 1u) == 0u;
        T f[3] = { T(0), T(0), T(0) };
        T W[6] = { T(0), T(0), T(0), T(0), T(0), T(0) };
        int npair = 0;
        if (mobile) {
            int q0, q1, q2;
            cell_coords(cell_s[s], geo, q0, q1, q2);
            const auto* tP = tab.P + ti * 8;
            for (int oz = -1; oz <= 1; ++oz) {
                const int z = neighbour_index(q2, oz, geo.nc[2], geo.periodic[2]);
                if (z < 0) continue;
                const T sz = pi.z - (T)oz * derived<T>(ph).h[2];
                for (int oy = -1; oy <= 1; ++oy) {
                    const int y = neighbour_index(q1, oy, geo.nc[1], geo.periodic[1]);
                    if (y < 0) continue;
                    const T sy = pi.y - (T)oy * derived<T>(ph).h[1];
                    for (int ox = -1; ox <= 1; ++ox) {
                        const int x = neighbour_index(q0, ox, geo.nc[0], geo.periodic[0]);
                        if (x < 0) continue;
                        const T sx = pi.x - (T)ox * derived<T>(ph).h[0];
                        const uint32_t nc = (uint32_t)(x + geo.nc[0] * (y + geo.nc[1] * z));
                        const uint32_t b = start[nc];
                        uint32_t e = start[nc + 1];
                        if (!MDPD_DBG_OK(b <= e && e <= (uint32_t)n, ph.dbg_status)) e = b;
                        for (uint32_t j = b; j < e; ++j) {
                            const auto pj = pos4[j];
                            const T dx = sx - pj.x, dy = sy - pj.y, dz = sz - pj.z;
                            const T r2 = dx * dx + dy * dy + dz * dz;
                            if (r2 < c.rc2 && r2 > T(0)) {
                                const auto vj = vel4[j];
                                pair_term<T, true>(c, tP[unpack_u32(pj.w)], dx, dy, dz, r2, vi, vj,
                                                   rho_i, rho[j], id_i, unpack_u32(vj.w), step,
                                                   ph, f, W);
                                ++npair;
                            }
                        }
                    }
                }
            }
        }
        force_finish<T, MODE>(s, mobile, f, W, npair, cap, geo, ph, mk, m, out, obs, status);
    }
    warp_obs_store(obs, partials, (int64_t)gridDim.x * (PAIR_BLOCK / 32));
}

// Reduction of the per-warp observable partials (type P: the pair
// arithmetic's precision).  FP64 additions, and conversions from FP64, cost
// 64 FP32 operations on this part, so the partials are added in P with the
// block's threads in parallel and only the 16 column sums per observable are
// widened to FP64.  Every addition happens in a fixed order, so the result is
// reproducible.
constexpr int RED_THREADS = 256;
constexpr int RED_CHUNK = RED_THREADS * 16;   // partials per level-one block

// res[k] = sum over q in [q0, q1) of data[k * stride + q], for the NOBS
// observables: thread t adds q = q0 + t, q0 + t + RED_THREADS, ...; then 16
// threads per observable add 16 columns each; then one thread per observable
// adds the 16 results in FP64.  The two counts (mobile particles, pairs) are
// added as 64-bit integers, so they stay exact at any size.  res is valid
// for every thread on return.
template <typename P>
__device__ void block_sum_obs(const P* __restrict__ data, int64_t stride, int64_t q0, int64_t q1,
                              double* res)
{
    constexpr int NV = NOBS - 2;
    __shared__ P sh[NV][RED_THREADS + 1];
    __shared__ unsigned long long shc[2][RED_THREADS + 1];
    __shared__ P s16[NV][16];
    __shared__ unsigned long long s16c[2][16];
    P v[NV];
    unsigned long long c[2] = { 0ull, 0ull };
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = P(0);
    for (int64_t q = q0 + threadIdx.x; q < q1; q += RED_THREADS) {
#pragma unroll
        for (int k = 0; k < NV; ++k) v[k] += __ldcg(&data[(int64_t)k * stride + q]);
#pragma unroll
        for (int k = 0; k < 2; ++k)
            c[k] += bits_count<P>(__ldcg(&data[(int64_t)(NV + k) * stride + q]));
    }
#pragma unroll
    for (int k = 0; k < NV; ++k) sh[k][threadIdx.x] = v[k];
    shc[0][threadIdx.x] = c[0];
    shc[1][threadIdx.x] = c[1];
    __syncthreads();
    if (threadIdx.x < NOBS * 16) {
        const int k = threadIdx.x >> 4, part = threadIdx.x & 15;
        if (k < NV) {
            P a = P(0);
#pragma unroll
            for (int l = 0; l < RED_THREADS / 16; ++l) a += sh[k][part * (RED_THREADS / 16) + l];
            s16[k][part] = a;
        } else {
            unsigned long long a = 0ull;
#pragma unroll
            for (int l = 0; l < RED_THREADS / 16; ++l) a += shc[k - NV][part * (RED_THREADS / 16) + l];
            s16c[k - NV][part] = a;
        }
    }
    __syncthreads();
    if (threadIdx.x < NOBS) {
        const int k = threadIdx.x;
        if (k < NV) {
            double a = 0.0;
#pragma unroll
            for (int l = 0; l < 16; ++l) a += (double)s16[k][l];
            res[k] = a;
        } else {
            unsigned long long a = 0ull;
#pragma unroll
            for (int l = 0; l < 16; ++l) a += s16c[k - NV][l];
            res[k] = (double)a;
        }
    }
    __syncthreads();
}

// One block over all nparts partials.
template <typename P>
__global__ void __launch_bounds__(RED_THREADS)
k_reduce_obs_small(const P* __restrict__ partials, int nparts, double* __restrict__ obs,
                   double* __restrict__ obs_sum, double* __restrict__ obs_count,
                   uint64_t* __restrict__ step_ptr, int advance)
{
    pdl_enter();
    __shared__ double res[NOBS];
    block_sum_obs<P>(partials, nparts, 0, nparts, res);
    if (threadIdx.x == 0) {
        double t[NOBS];
        for (int k = 0; k < NOBS; ++k) t[k] = res[k];
        const uint64_t step = *step_ptr + (advance ? 1u : 0u);
        finish_obs(t, step, obs, obs_sum, obs_count, advance);
        if (advance) *step_ptr = step;
    }
}

// Two levels in one launch: block b reduces the partials
// [b * RED_CHUNK, (b + 1) * RED_CHUNK) to a level-one partial l1[k * nb + b]
// and takes a ticket; the block with the last ticket reduces the level-one
// partials, derives the observables, accumulates the running sums, advances
// the step counter when asked and resets the ticket.
template <typename P>
__global__ void __launch_bounds__(RED_THREADS)
k_reduce_obs(const P* __restrict__ partials, int nparts, P* __restrict__ l1,
             unsigned* __restrict__ ticket, double* __restrict__ obs,
             double* __restrict__ obs_sum, double* __restrict__ obs_count,
             uint64_t* __restrict__ step_ptr, int advance)
{
    pdl_enter();
    __shared__ double res[NOBS];
    __shared__ bool last;
    const int64_t q0 = (int64_t)blockIdx.x * RED_CHUNK;
    const int64_t q1 = q0 + RED_CHUNK < nparts ? q0 + RED_CHUNK : nparts;
    block_sum_obs<P>(partials, nparts, q0, q1, res);
    if (threadIdx.x < NOBS) {
        // counts keep the integer bit pattern (at most RED_CHUNK * 2048 < 2^32)
        const int k = threadIdx.x;
        l1[(int64_t)k * gridDim.x + blockIdx.x] =
            k < NOBS - 2 ? (P)res[k] : count_bits<P>((unsigned)res[k]);
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    block_sum_obs<P>(l1, gridDim.x, 0, gridDim.x, res);
    if (threadIdx.x == 0) {
        double t[NOBS];
        for (int k = 0; k < NOBS; ++k) t[k] = res[k];
        const uint64_t step = *step_ptr + (advance ? 1u : 0u);
        finish_obs(t, step, obs, obs_sum, obs_count, advance);
        if (advance) *step_ptr = step;
        *ticket = 0u;
    }
}

// Per-replica reduction of a batch: block r reduces the partials of replica
// r's chunks, [wr[r].x, wr[r].y), and writes the replica's observables to
// obs[r * OBS_STRIDE ...] (current values, running sums, count, pairs: the
// layout of a single system).  The block holding the last ticket advances the
// shared step counter.
template <typename P>
__global__ void __launch_bounds__(RED_THREADS)
k_reduce_obs_batch(const P* __restrict__ partials, int nparts, const int2* __restrict__ wr,
                   unsigned* __restrict__ ticket, double* __restrict__ obs,
                   uint64_t* __restrict__ step_ptr, int advance)
{
    pdl_enter();
    __shared__ double res[NOBS];
    const int2 w = wr[blockIdx.x];
    block_sum_obs<P>(partials, nparts, w.x, w.y, res);
    if (threadIdx.x == 0) {
        double t[NOBS];
        for (int k = 0; k < NOBS; ++k) t[k] = res[k];
        const uint64_t step = *step_ptr + (advance ? 1u : 0u);
        double* o = obs + (int64_t)blockIdx.x * OBS_STRIDE;
        finish_obs(t, step, o, o + MDPD_NUM_OBS, o + 2 * MDPD_NUM_OBS, advance);
        __threadfence();
        const bool last = atomicAdd(ticket, 1u) == gridDim.x - 1;
        if (last) {
            if (advance) *step_ptr = step;
            *ticket = 0u;
        }
    }
}

template <typename T>
void launch_force_t(cudaStream_t st, ForceMode mode, int n, int64_t cap, const Geo& geo,
                    const Phys& ph, const MaskDev& mk, const void* pos4, const void* vel4,
                    const void* rho, const uint32_t* cell_s, const uint32_t* start,
                    const uint64_t* step_ptr, int step_offset, const Master& m, double* out,
                    double* partials, uint32_t* status)
{
    using V = typename Vec4<T>::type;
    const int nb = force_num_blocks(n);
    const V* p = (const V*)pos4;
    const V* v = (const V*)vel4;
    const T* r = (const T*)rho;
    switch (mode) {
    case FM_EVAL:
        launch_pdl(k_force<T, FM_EVAL>, dim3(nb), dim3(PAIR_BLOCK), st, n, cap, geo, ph, mk, p, v, r, cell_s,
                                                       start, step_ptr, step_offset, m, out,
                                                       partials, status);
        break;
    case FM_LAST:
        launch_pdl(k_force<T, FM_LAST>, dim3(nb), dim3(PAIR_BLOCK), st, n, cap, geo, ph, mk, p, v, r, cell_s,
                                                       start, step_ptr, step_offset, m, out,
                                                       partials, status);
        break;
    default:
        launch_pdl(k_force<T, FM_FUSED>, dim3(nb), dim3(PAIR_BLOCK), st, n, cap, geo, ph, mk, p, v, r, cell_s,
                                                        start, step_ptr, step_offset, m, out,
                                                        partials, status);
        break;
    }
}

}  // namespace

int force_num_blocks(int n, int lpp, int rounds)
{
    const int per = PAIR_BLOCK / lpp * rounds;
    return n > 0 ? (n + per - 1) / per : 1;
}

int obs_num_partials(int n, int lpp, int rounds)
{
    return force_num_blocks(n, lpp, rounds) * (PAIR_BLOCK / 32);
}

void launch_density(cudaStream_t st, int precision, int n, const Geo& geo, const Phys& ph,
                    const void* pos4, const uint32_t* cell_s, const uint32_t* start, void* rho)
{
    if (n <= 0) return;
    const int nb = (n + PAIR_BLOCK - 1) / PAIR_BLOCK;
    if (precision == 0)
        launch_pdl(k_density<double>, dim3(nb), dim3(PAIR_BLOCK), st, n, geo, ph, (const D4*)pos4, cell_s, start,
                                                     (double*)rho);
    else
        launch_pdl(k_density<float>, dim3(nb), dim3(PAIR_BLOCK), st, n, geo, ph, (const float4*)pos4, cell_s,
                                                    start, (float*)rho);
}

void launch_force(cudaStream_t st, int precision, ForceMode mode, int n, int64_t cap,
                  const Geo& geo, const Phys& ph, const MaskDev& mk, const void* pos4,
                  const void* vel4, const void* rho, const uint32_t* cell_s,
                  const uint32_t* start, const uint64_t* step_ptr, int step_offset,
                  const Master& m, double* out, double* partials, uint32_t* status)
{
    if (precision == 0)
        launch_force_t<double>(st, mode, n, cap, geo, ph, mk, pos4, vel4, rho, cell_s, start,
                               step_ptr, step_offset, m, out, partials, status);
    else
        launch_force_t<float>(st, mode, n, cap, geo, ph, mk, pos4, vel4, rho, cell_s, start,
                              step_ptr, step_offset, m, out, partials, status);
}

int reduce_l1_blocks(int nparts) { return (nparts + RED_CHUNK - 1) / RED_CHUNK; }

void launch_reduce_obs(cudaStream_t st, int precision, const double* partials, int nparts,
                       double* l1, unsigned* ticket, double* obs, double* obs_sum,
                       double* obs_count, uint64_t* step_ptr, int advance)
{
    // one block when its threads add at most 32 (FP32) or 4 (FP64) partials each
    const int small_max = precision == 1 ? RED_THREADS * 32 : RED_THREADS * 4;
    if (nparts <= small_max) {
        if (precision == 1)
            launch_pdl(k_reduce_obs_small<float>, dim3(1), dim3(RED_THREADS), st,
                       (const float*)partials, nparts, obs, obs_sum, obs_count, step_ptr, advance);
        else
            launch_pdl(k_reduce_obs_small<double>, dim3(1), dim3(RED_THREADS), st, partials, nparts,
                       obs, obs_sum, obs_count, step_ptr, advance);
        return;
    }
    const int nb = reduce_l1_blocks(nparts);
    if (precision == 1)
        launch_pdl(k_reduce_obs<float>, dim3(nb), dim3(RED_THREADS), st, (const float*)partials,
                   nparts, (float*)l1, ticket, obs, obs_sum, obs_count, step_ptr, advance);
    else
        launch_pdl(k_reduce_obs<double>, dim3(nb), dim3(RED_THREADS), st, partials, nparts, l1,
                   ticket, obs, obs_sum, obs_count, step_ptr, advance);
}

void launch_reduce_obs_batch(cudaStream_t st, int precision, const double* partials, int nparts,
                             const int2* wr, int nrep, unsigned* ticket, double* obs,
                             uint64_t* step_ptr, int advance)
{
    if (nrep <= 0) return;
    if (precision == 1)
        launch_pdl(k_reduce_obs_batch<float>, dim3(nrep), dim3(RED_THREADS), st,
                   (const float*)partials, nparts, wr, ticket, obs, step_ptr, advance);
    else
        launch_pdl(k_reduce_obs_batch<double>, dim3(nrep), dim3(RED_THREADS), st, partials, nparts,
                   wr, ticket, obs, step_ptr, advance);
}

}  // namespace mdpd
