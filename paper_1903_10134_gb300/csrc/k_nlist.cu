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

template <typename T>
__global__ void __launch_bounds__(PAIR_BLOCK)
k_density_nl(int n, int64_t cap, Geo geo, Phys ph,
             const typename Vec4<T>::type* __restrict__ pos4, const uint32_t* __restrict__ cell_s,
             const uint32_t* __restrict__ start, T* __restrict__ rho_out,
             uint32_t* __restrict__ nl, uint32_t* __restrict__ nl_count)
{
    __shared__ uint32_t lst[NL_MAX][PAIR_BLOCK];
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const T rd2 = (T)(ph.rd * ph.rd), rc2 = (T)(ph.rc * ph.rc);
    const T inv_rd = (T)(1.0 / ph.rd);
    const T cw = (T)(15.0 / (2.0 * 3.14159265358979323846 * ph.rd * ph.rd * ph.rd));
    const auto pi = pos4[s];
    const bool mobile = ((ph.frozen >> unpack_u32(pi.w)) & 1u) == 0u;
    int q0, q1, q2;
    cell_coords(cell_s[s], geo, q0, q1, q2);
    T acc = ph.rho_self ? cw : T(0);
    uint32_t cnt = 0;
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
                const uint32_t code = (uint32_t)image_code(ox, oy, oz);
                const uint32_t nc = (uint32_t)(x + geo.nc[0] * (y + geo.nc[1] * z));
                const uint32_t b = start[nc], e = start[nc + 1];
                for (uint32_t j = b; j < e; ++j) {
                    const auto pj = pos4[j];
                    const T dx = sx - pj.x, dy = sy - pj.y, dz = sz - pj.z;
                    const T r2 = dx * dx + dy * dy + dz * dz;
                    if (j == (uint32_t)s) continue;
                    if (r2 < rd2) {
                        const T w = T(1) - sqrt(r2) * inv_rd;
                        acc += cw * w * w;
                    }
                    if (mobile && r2 < rc2 && r2 > T(0)) {
                        if (cnt < NL_MAX) lst[cnt][threadIdx.x] = (j << 5) | code;
                        ++cnt;
                    }
                }
            }
        }
    }
    rho_out[s] = acc;
    nl_count[s] = cnt;
    const uint32_t m = cnt < NL_MAX ? cnt : NL_MAX;
    for (uint32_t k = 0; k < m; ++k) nl[(int64_t)k * cap + s] = lst[k][threadIdx.x];
}

template <typename T, int MODE>
__global__ void __launch_bounds__(PAIR_BLOCK)
k_force_nl(int n, int64_t cap, Geo geo, Phys ph, MaskDev mk,
           const typename Vec4<T>::type* __restrict__ pos4,
           const typename Vec4<T>::type* __restrict__ vel4, const T* __restrict__ rho,
           const uint32_t* __restrict__ cell_s, const uint32_t* __restrict__ start,
           const uint32_t* __restrict__ nl, const uint32_t* __restrict__ nl_count,
           const uint64_t* __restrict__ step_ptr, int step_offset, Master m,
           double* __restrict__ out, double* __restrict__ partials, uint32_t* __restrict__ status)
{
    __shared__ PairTables<T> tab;
    __shared__ T shift[27][3];
    load_tables(tab, ph);
    if (threadIdx.x < 27) {
        const int c = threadIdx.x;
        shift[c][0] = (T)(c % 3 - 1) * (T)geo.h[0];
        shift[c][1] = (T)((c / 3) % 3 - 1) * (T)geo.h[1];
        shift[c][2] = (T)(c / 9 - 1) * (T)geo.h[2];
    }
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
            const T* tA = tab.A + ti * 8;
            const T* tB = tab.B + ti * 8;
            const T* tG = tab.G + ti * 8;
            const T* tS = tab.S + ti * 8;
            const uint32_t cnt = nl_count[s];
            if (cnt <= (uint32_t)NL_MAX) {
                for (uint32_t k = 0; k < cnt; ++k) {
                    const uint32_t e = nl[(int64_t)k * cap + s];
                    const uint32_t j = e >> 5, code = e & 31u;
                    const auto pj = pos4[j];
                    const T dx = pi.x - shift[code][0] - pj.x;
                    const T dy = pi.y - shift[code][1] - pj.y;
                    const T dz = pi.z - shift[code][2] - pj.z;
                    const T r2 = dx * dx + dy * dy + dz * dz;
                    const auto vj = vel4[j];
                    pair_term(c, tA, tB, tG, tS, dx, dy, dz, r2, vi, vj, rho_i, rho[j],
                              unpack_u32(pj.w), id_i, unpack_u32(vj.w), step, ph, f, W);
                }
                npair = (int)cnt;
            } else {
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
                            const uint32_t nc = (uint32_t)(x + geo.nc[0] * (y + geo.nc[1] * z));
                            const uint32_t b = start[nc], e = start[nc + 1];
                            for (uint32_t j = b; j < e; ++j) {
                                const auto pj = pos4[j];
                                const T dx = pi.x - shift[code][0] - pj.x;
                                const T dy = pi.y - shift[code][1] - pj.y;
                                const T dz = pi.z - shift[code][2] - pj.z;
                                const T r2 = dx * dx + dy * dy + dz * dz;
                                if (r2 < c.rc2 && r2 > T(0)) {
                                    const auto vj = vel4[j];
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
        force_finish<T, MODE>(s, mobile, f, W, npair, cap, geo, ph, mk, m, out, obs, status);
    }
    block_obs_store(obs, partials);
}

template <typename T>
void launch_force_nl_t(cudaStream_t st, ForceMode mode, int n, int64_t cap, const Geo& geo,
                       const Phys& ph, const MaskDev& mk, const void* pos4, const void* vel4,
                       const void* rho, const uint32_t* cell_s, const uint32_t* start,
                       const uint32_t* nl, const uint32_t* nl_count, const uint64_t* step_ptr,
                       int step_offset, const Master& m, double* out, double* partials,
                       uint32_t* status)
{
    using V = typename Vec4<T>::type;
    const int nb = force_num_blocks(n);
    const V* p = (const V*)pos4;
    const V* v = (const V*)vel4;
    const T* r = (const T*)rho;
#define MDPD_FNL(MODE_)                                                                    \
    k_force_nl<T, MODE_><<<nb, PAIR_BLOCK, 0, st>>>(n, cap, geo, ph, mk, p, v, r, cell_s, \
                                                    start, nl, nl_count, step_ptr,        \
                                                    step_offset, m, out, partials, status)
    if (mode == FM_EVAL) MDPD_FNL(FM_EVAL);
    else if (mode == FM_LAST) MDPD_FNL(FM_LAST);
    else MDPD_FNL(FM_FUSED);
#undef MDPD_FNL
}

}  // namespace

void launch_density_nl(cudaStream_t st, int precision, int n, int64_t cap, const Geo& geo,
                       const Phys& ph, const void* pos4, const uint32_t* cell_s,
                       const uint32_t* start, void* rho, uint32_t* nl, uint32_t* nl_count)
{
    if (n <= 0) return;
    const int nb = (n + PAIR_BLOCK - 1) / PAIR_BLOCK;
    if (precision == 0)
        k_density_nl<double><<<nb, PAIR_BLOCK, 0, st>>>(n, cap, geo, ph, (const D4*)pos4, cell_s,
                                                        start, (double*)rho, nl, nl_count);
    else
        k_density_nl<float><<<nb, PAIR_BLOCK, 0, st>>>(n, cap, geo, ph, (const float4*)pos4,
                                                       cell_s, start, (float*)rho, nl, nl_count);
}

void launch_force_nl(cudaStream_t st, int precision, ForceMode mode, int n, int64_t cap,
                     const Geo& geo, const Phys& ph, const MaskDev& mk, const void* pos4,
                     const void* vel4, const void* rho, const uint32_t* cell_s,
                     const uint32_t* start, const uint32_t* nl, const uint32_t* nl_count,
                     const uint64_t* step_ptr, int step_offset, const Master& m, double* out,
                     double* partials, uint32_t* status)
{
    if (precision == 0)
        launch_force_nl_t<double>(st, mode, n, cap, geo, ph, mk, pos4, vel4, rho, cell_s, start,
                                  nl, nl_count, step_ptr, step_offset, m, out, partials, status);
    else
        launch_force_nl_t<float>(st, mode, n, cap, geo, ph, mk, pos4, vel4, rho, cell_s, start,
                                 nl, nl_count, step_ptr, step_offset, m, out, partials, status);
}

}  // namespace mdpd
