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
    const T rd2 = (T)(ph.rd * ph.rd);
    const T inv_rd = (T)(1.0 / ph.rd);
    const T cw = (T)(15.0 / (2.0 * 3.14159265358979323846 * ph.rd * ph.rd * ph.rd));
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
        const T sz = pi.z - (T)oz * (T)geo.h[2];
        for (int oy = -1; oy <= 1; ++oy) {
            int y = q1 + oy;
            if (y < 0 || y >= geo.nc[1]) {
                if (!geo.periodic[1]) continue;
                y = y < 0 ? y + geo.nc[1] : y - geo.nc[1];
            }
            const T sy = pi.y - (T)oy * (T)geo.h[1];
            for (int ox = -1; ox <= 1; ++ox) {
                int x = q0 + ox;
                if (x < 0 || x >= geo.nc[0]) {
                    if (!geo.periodic[0]) continue;
                    x = x < 0 ? x + geo.nc[0] : x - geo.nc[0];
                }
                const T sx = pi.x - (T)ox * (T)geo.h[0];
                const uint32_t nc = (uint32_t)(x + geo.nc[0] * (y + geo.nc[1] * z));
                const uint32_t b = start[nc], e = start[nc + 1];
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
    double obs[NOBS];
#pragma unroll
    for (int k = 0; k < NOBS; ++k) obs[k] = 0.0;
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
            const T* tA = tab.A + ti * 8;
            const T* tB = tab.B + ti * 8;
            const T* tG = tab.G + ti * 8;
            const T* tS = tab.S + ti * 8;
            for (int oz = -1; oz <= 1; ++oz) {
                const int z = neighbour_index(q2, oz, geo.nc[2], geo.periodic[2]);
                if (z < 0) continue;
                const T sz = pi.z - (T)oz * (T)geo.h[2];
                for (int oy = -1; oy <= 1; ++oy) {
                    const int y = neighbour_index(q1, oy, geo.nc[1], geo.periodic[1]);
                    if (y < 0) continue;
                    const T sy = pi.y - (T)oy * (T)geo.h[1];
                    for (int ox = -1; ox <= 1; ++ox) {
                        const int x = neighbour_index(q0, ox, geo.nc[0], geo.periodic[0]);
                        if (x < 0) continue;
                        const T sx = pi.x - (T)ox * (T)geo.h[0];
                        const uint32_t nc = (uint32_t)(x + geo.nc[0] * (y + geo.nc[1] * z));
                        const uint32_t b = start[nc], e = start[nc + 1];
                        for (uint32_t j = b; j < e; ++j) {
                            const auto pj = pos4[j];
                            const T dx = sx - pj.x, dy = sy - pj.y, dz = sz - pj.z;
                            const T r2 = dx * dx + dy * dy + dz * dz;
                            if (r2 < c.rc2 && r2 > T(0)) {
                                const auto vj = vel4[j];
                                pair_term(c, tA, tB, tG, tS, dx, dy, dz, r2, vi, vj, rho_i, rho[j],
                                          unpack_u32(pj.w), id_i, unpack_u32(vj.w), step, ph, f, W);
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

template <bool BATCH>
__global__ void k_kick_drift(int n, int64_t cap, Geo geo_p, Phys ph_p, Batch bt, MaskDev mk,
                             Master m, uint32_t* __restrict__ status)
{
    pdl_enter();
    int s;
    bool valid;
    const Rep* rp = nullptr;
    if constexpr (BATCH) {
        const int4 ch = bt.chunks[blockIdx.x];
        rp = &block_rep<REP_SCALARS>(bt.reps, ch.x);
        s = ch.y + (int)threadIdx.x;
        valid = (int)threadIdx.x < ch.z;
    } else {
        s = blockIdx.x * blockDim.x + threadIdx.x;
        valid = s < n;
    }
    if (!valid) return;
    const Geo& geo = BATCH ? rp->geo : geo_p;
    const Phys& ph = BATCH ? rp->ph : ph_p;
    if ((ph.frozen >> m.type[s]) & 1u) return;
    double x[3], v[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        x[k] = m.x[k * cap + s];
        v[k] = __dadd_rn(m.v[k * cap + s], __dmul_rn(ph.hdt, m.a[k * cap + s]));
    }
    drift_reflect(x, v, geo, mk, ph.dt);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        m.x[k * cap + s] = x[k];
        m.v[k * cap + s] = v[k];
    }
    if (!isfinite(v[0]) || !isfinite(v[1]) || !isfinite(v[2])) atomicOr(status, ST_NONFINITE);
}

// Final reduction of the observables, one launch in two levels.  FP64 adds
// run at a small fraction of the FP32 rate on this part, so the sums are laid
// out to do few of them: block b takes the per-warp partials
// [b * RED_CHUNK, (b + 1) * RED_CHUNK), one per thread, transposes them
// through shared memory, and 16 threads per observable add 16 values each
// before one thread adds those 16 results; the block writes its level-one
// partial and takes a ticket.  The block holding the last ticket adds the
// level-one partials in block order, derives the observables, accumulates the
// running sums, advances the step counter when asked and resets the ticket.
// Every addition happens in a fixed order, so the result is reproducible.
constexpr int RED_CHUNK = 256;
constexpr int RED_THREADS = RED_CHUNK;

// Observables from the summed partials t (momentum 3, sum v^2 3, virial 6,
// mobile count, pairs): o = momentum, kinetic energy, kT, virial, sum v^2,
// mobile count, step; obs[2 * MDPD_NUM_OBS + 1] = the directed pair count.
__device__ void finish_obs(const double (&t)[NOBS], uint64_t step, double* __restrict__ obs,
                           double* __restrict__ obs_sum, double* __restrict__ obs_count,
                           int advance)
{
    double o[MDPD_NUM_OBS];
    for (int k = 0; k < 3; ++k) o[k] = t[k];
    o[3] = 0.5 * (t[3] + t[4] + t[5]);
    const double nm = t[12];
    o[4] = nm > 1.0 ? 2.0 * o[3] / (3.0 * (nm - 1.0)) : 0.0;
    for (int k = 0; k < 6; ++k) o[5 + k] = t[6 + k];
    for (int k = 0; k < 3; ++k) o[11 + k] = t[3 + k];
    o[14] = nm;
    o[15] = (double)step;
    for (int k = 0; k < MDPD_NUM_OBS; ++k) obs[k] = o[k];
    obs[2 * MDPD_NUM_OBS + 1] = t[13];     // directed pairs with r < r_c
    if (advance) {
        for (int k = 0; k < MDPD_NUM_OBS; ++k) obs_sum[k] += o[k];
        *obs_count += 1.0;
    }
}

__global__ void __launch_bounds__(RED_THREADS)
k_reduce_obs(const double* __restrict__ partials, int nparts, double* __restrict__ l1,
             unsigned* __restrict__ ticket, double* __restrict__ obs,
             double* __restrict__ obs_sum, double* __restrict__ obs_count,
             uint64_t* __restrict__ step_ptr, int advance)
{
    pdl_enter();
    __shared__ double sh[NOBS][RED_CHUNK + 1];
    __shared__ double s16[NOBS][17];
    __shared__ bool last;
    const int b = blockIdx.x * RED_CHUNK + threadIdx.x;
#pragma unroll
    for (int k = 0; k < NOBS; ++k)
        sh[k][threadIdx.x] = b < nparts ? partials[(int64_t)k * nparts + b] : 0.0;
    __syncthreads();
    if (threadIdx.x < NOBS * 16) {
        const int k = threadIdx.x >> 4, part = threadIdx.x & 15;
        double v = 0.0;
#pragma unroll
        for (int l = 0; l < RED_CHUNK / 16; ++l) v += sh[k][part * (RED_CHUNK / 16) + l];
        s16[k][part] = v;
    }
    __syncthreads();
    if (threadIdx.x < NOBS) {
        double v = 0.0;
#pragma unroll
        for (int l = 0; l < 16; ++l) v += s16[threadIdx.x][l];
        l1[(int64_t)threadIdx.x * gridDim.x + blockIdx.x] = v;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (threadIdx.x < NOBS) {
        double v = 0.0;
        for (unsigned q = 0; q < gridDim.x; ++q) v += __ldcg(&l1[(int64_t)threadIdx.x * gridDim.x + q]);
        s16[threadIdx.x][16] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t[NOBS];
        for (int k = 0; k < NOBS; ++k) t[k] = s16[k][16];
        const uint64_t step = *step_ptr + (advance ? 1u : 0u);
        finish_obs(t, step, obs, obs_sum, obs_count, advance);
        if (advance) *step_ptr = step;
        *ticket = 0u;
    }
}

// Per-replica reduction of a batch: block r adds the per-warp partials of
// replica r's chunks, [wr[r].x, wr[r].y), in a fixed order (a strided sum per
// thread, then 16 partial sums per observable, then one), and writes the
// replica's observables to obs[r * OBS_STRIDE ...] (current values, running
// sums, count, pairs: the layout of a single system).  The block holding the
// last ticket advances the shared step counter.
__global__ void __launch_bounds__(RED_THREADS)
k_reduce_obs_batch(const double* __restrict__ partials, int nparts, const int2* __restrict__ wr,
                   unsigned* __restrict__ ticket, double* __restrict__ obs,
                   uint64_t* __restrict__ step_ptr, int advance)
{
    pdl_enter();
    __shared__ double sh[NOBS][RED_THREADS + 1];
    __shared__ double s16[NOBS][17];
    const int2 w = wr[blockIdx.x];
#pragma unroll
    for (int k = 0; k < NOBS; ++k) {
        double v = 0.0;
        for (int q = w.x + (int)threadIdx.x; q < w.y; q += RED_THREADS)
            v += partials[(int64_t)k * nparts + q];
        sh[k][threadIdx.x] = v;
    }
    __syncthreads();
    if (threadIdx.x < NOBS * 16) {
        const int k = threadIdx.x >> 4, part = threadIdx.x & 15;
        double v = 0.0;
#pragma unroll
        for (int l = 0; l < RED_THREADS / 16; ++l) v += sh[k][part * (RED_THREADS / 16) + l];
        s16[k][part] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t[NOBS];
        for (int k = 0; k < NOBS; ++k) {
            double v = 0.0;
            for (int l = 0; l < 16; ++l) v += s16[k][l];
            t[k] = v;
        }
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

int force_num_blocks(int n) { return n > 0 ? (n + PAIR_BLOCK - 1) / PAIR_BLOCK : 1; }

int obs_num_partials(int n) { return force_num_blocks(n) * (PAIR_BLOCK / 32); }

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

void launch_kick_drift(cudaStream_t st, int n, int64_t cap, const Geo& geo, const Phys& ph,
                       const MaskDev& mk, const Master& m, uint32_t* status)
{
    if (n <= 0) return;
    launch_pdl(k_kick_drift<false>, dim3((n + 255) / 256), dim3(256), st, n, cap, geo, ph, Batch{},
               mk, m, status);
}

void launch_kick_drift_batch(cudaStream_t st, int64_t cap, const Batch& bt, const Master& m,
                             uint32_t* status)
{
    if (bt.nchunk <= 0) return;
    launch_pdl_smem(k_kick_drift<true>, dim3(bt.nchunk), dim3(BATCH_CHUNK), REP_SMEM, st, 0, cap,
                    Geo{}, Phys{}, bt, MaskDev{}, m, status);
}

void launch_reduce_obs_batch(cudaStream_t st, const double* partials, int nparts, const int2* wr,
                             int nrep, unsigned* ticket, double* obs, uint64_t* step_ptr,
                             int advance)
{
    if (nrep <= 0) return;
    launch_pdl(k_reduce_obs_batch, dim3(nrep), dim3(RED_THREADS), st, partials, nparts, wr, ticket,
               obs, step_ptr, advance);
}

int reduce_l1_blocks(int nparts) { return (nparts + RED_CHUNK - 1) / RED_CHUNK; }

void launch_reduce_obs(cudaStream_t st, const double* partials, int nparts, double* l1,
                       unsigned* ticket, double* obs, double* obs_sum, double* obs_count,
                       uint64_t* step_ptr, int advance)
{
    const int nb = reduce_l1_blocks(nparts) > 0 ? reduce_l1_blocks(nparts) : 1;
    launch_pdl(k_reduce_obs, dim3(nb), dim3(RED_THREADS), st, partials, nparts, l1, ticket, obs, obs_sum,
                                             obs_count, step_ptr, advance);
}

}  // namespace mdpd
