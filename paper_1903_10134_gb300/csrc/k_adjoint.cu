// Vector-Jacobian product of one force evaluation (Sec. 2.1, Eq. 1 of
// arXiv:1903.10134): given abar (the adjoint of the accelerations, id order),
// the gradient of L = sum_{i mobile} abar_i . a_i with respect to positions,
// the velocities u the dissipative term sees, and the symmetric pair
// parameters A, B, gamma, with the random draws of the step held fixed.
//
// For a pair (i, j), d = x_i - x_j, r = |d|, e = d / r, w = e . u_ij and
// f_ij = s e with
//   s = A wc + B (rho_i + rho_j) wd [r < r_d] - gamma wc^2 w + sigma wc xi / sqrt(dt).
// Frozen particles contribute no acceleration, so their abar counts as zero;
// with q = abar_i - abar_j the pair's term of L is q . f_ij and, since the
// partner lists hold every pair from both sides, each thread adds its own
// particle's share without atomics:
//   xbar_i += (q.e)(s_r e + s_w (u_ij - w e) / r) + s (q - (q.e) e) / r
//   ubar_i += (q.e) s_w e,         rhobar_i += (q.e) B wd [r < r_d]
// (s_r = ds/dr at fixed w and rho, s_w = -gamma wc^2).  A second pass sends
// rhobar back to positions: xbar_i += (rhobar_i + rhobar_j) w_rho'(r) e over
// partners within r_d.  Parameter gradients (each pair seen twice: factor 1/2)
// are summed per block in shared memory and added to the output with atomics.
#include "pair.cuh"

namespace mdpd {

namespace {

template <typename T>
__global__ void __launch_bounds__(PAIR_BLOCK)
k_force_vjp(int n, int64_t cap, Geo geo, Phys ph, const typename Vec4<T>::type* __restrict__ pos4,
            const typename Vec4<T>::type* __restrict__ vel4, const T* __restrict__ rho,
            const uint32_t* __restrict__ nl, const uint32_t* __restrict__ nl_count,
            const uint64_t* __restrict__ step_ptr, const double* __restrict__ abar,
            double* __restrict__ xbar, double* __restrict__ ubar, double* __restrict__ rbar,
            double* __restrict__ tbar, uint32_t* __restrict__ status)
{
    using V = typename Vec4<T>::type;
    __shared__ double tsh[3 * 64];
    __shared__ T shift[27][3];
    for (int k = threadIdx.x; k < 3 * 64; k += blockDim.x) tsh[k] = 0.0;
    if (threadIdx.x < 27) {
        const int c = threadIdx.x;
        shift[c][0] = (T)(c % 3 - 1) * derived<T>(ph).h[0];
        shift[c][1] = (T)((c / 3) % 3 - 1) * derived<T>(ph).h[1];
        shift[c][2] = (T)(c / 9 - 1) * derived<T>(ph).h[2];
    }
    __syncthreads();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < n) {
        const uint64_t step = *step_ptr;
        const Derived<T>& dc = derived<T>(ph);
        const T inv_rc = dc.inv_rc, inv_rd = dc.inv_rd;
        const T rd = (T)ph.rd;
        const T inv_sqrt_dt = dc.inv_sqrt_dt;
        const V pi = pos4[s];
        const V vi = vel4[s];
        const T rho_i = rho[s];
        const uint32_t ti = unpack_u32(pi.w), id_i = unpack_u32(vi.w);
        const bool mob_i = ((ph.frozen >> ti) & 1u) == 0u;
        T ai[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) ai[k] = mob_i ? (T)abar[3 * (int64_t)id_i + k] : T(0);
        T gx[3] = { T(0), T(0), T(0) }, gu[3] = { T(0), T(0), T(0) };
        T gr = T(0);
        const uint32_t cnt = nl_count[s];
        if (cnt > (uint32_t)NL_MAX) atomicOr(status, ST_OVERFLOW);
        const uint32_t m = cnt < (uint32_t)NL_MAX ? cnt : (uint32_t)NL_MAX;
        for (uint32_t k = 0; k < m; ++k) {
            const uint32_t e = nl[(int64_t)k * cap + s];
            const uint32_t j = e >> 5, code = e & 31u;
            const V pj = pos4[j];
            const V vj = vel4[j];
            const T rho_j = rho[j];
            const uint32_t tj = unpack_u32(pj.w), id_j = unpack_u32(vj.w);
            const bool mob_j = ((ph.frozen >> tj) & 1u) == 0u;
            T q[3];
#pragma unroll
            for (int c = 0; c < 3; ++c)
                q[c] = ai[c] - (mob_j ? (T)abar[3 * (int64_t)id_j + c] : T(0));
            const T dx = pi.x - shift[code][0] - pj.x;
            const T dy = pi.y - shift[code][1] - pj.y;
            const T dz = pi.z - shift[code][2] - pj.z;
            const T r2 = dx * dx + dy * dy + dz * dz;
            const T r = sqrt(r2);
            const T ex = dx / r, ey = dy / r, ez = dz / r;
            const T ux = vi.x - vj.x, uy = vi.y - vj.y, uz = vi.z - vj.z;
            const T w = ex * ux + ey * uy + ez * uz;
            const T wc = T(1) - r * inv_rc;
            const bool near = r < rd;
            const T wd = near ? T(1) - r * inv_rd : T(0);
            const int pidx = ti * 8 + tj;
            const T A = (T)ph.A[pidx], B = (T)ph.B[pidx], G = (T)ph.gamma[pidx];
            const T sig = (T)ph.sigma[pidx];
            const U4 wr = pair_draw(id_i, id_j, step, ph.key0, ph.key1);
            const T xi = xi_of<T>(wr, ph.xi_dist);
            const T rsum = rho_i + rho_j;
            const T sval = A * wc + B * rsum * wd - G * wc * wc * w + sig * wc * xi * inv_sqrt_dt;
            const T s_r = -A * inv_rc - (near ? B * rsum * inv_rd : T(0)) +
                          T(2) * G * wc * w * inv_rc - sig * xi * inv_sqrt_dt * inv_rc;
            const T s_w = -G * wc * wc;
            const T qe = q[0] * ex + q[1] * ey + q[2] * ez;
            const T e3[3] = { ex, ey, ez }, u3[3] = { ux, uy, uz };
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                gx[c] += qe * (s_r * e3[c] + s_w * (u3[c] - w * e3[c]) / r) +
                         sval * (q[c] - qe * e3[c]) / r;
                gu[c] += qe * s_w * e3[c];
            }
            gr += qe * B * wd;
            const int a = ti < tj ? (int)ti : (int)tj, b = ti < tj ? (int)tj : (int)ti;
            const double dsig = ph.gamma[pidx] > 0.0 ? ph.kT / ph.sigma[pidx] : 0.0;
            atomicAdd(&tsh[0 * 64 + a * 8 + b], 0.5 * (double)(qe * wc));
            atomicAdd(&tsh[1 * 64 + a * 8 + b], 0.5 * (double)(qe * rsum * wd));
            atomicAdd(&tsh[2 * 64 + a * 8 + b],
                      0.5 * (double)(qe * (-wc * wc * w)) +
                          0.5 * (double)qe * dsig * (double)(wc * xi * inv_sqrt_dt));
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            xbar[c * cap + s] = (double)gx[c];
            ubar[c * cap + s] = (double)gu[c];
        }
        rbar[s] = (double)gr;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < 3 * 64; k += blockDim.x)
        if (tsh[k] != 0.0) atomicAdd(&tbar[k], tsh[k]);
}

template <typename T>
__global__ void __launch_bounds__(PAIR_BLOCK)
k_density_vjp(int n, int64_t cap, Geo geo, Phys ph, const typename Vec4<T>::type* __restrict__ pos4,
              const uint32_t* __restrict__ nl, const uint32_t* __restrict__ nl_count,
              const double* __restrict__ rbar, double* __restrict__ xbar,
              uint32_t* __restrict__ status)
{
    using V = typename Vec4<T>::type;
    __shared__ T shift[27][3];
    if (threadIdx.x < 27) {
        const int c = threadIdx.x;
        shift[c][0] = (T)(c % 3 - 1) * derived<T>(ph).h[0];
        shift[c][1] = (T)((c / 3) % 3 - 1) * derived<T>(ph).h[1];
        shift[c][2] = (T)(c / 9 - 1) * derived<T>(ph).h[2];
    }
    __syncthreads();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const Derived<T>& dc = derived<T>(ph);
    const T rd = (T)ph.rd, inv_rd = dc.inv_rd;
    const T cw = dc.cw_rho;
    const V pi = pos4[s];
    const T rb_i = (T)rbar[s];
    T g[3] = { T(0), T(0), T(0) };
    const uint32_t cnt = nl_count[s];
    if (cnt > (uint32_t)NL_MAX) atomicOr(status, ST_OVERFLOW);
    const uint32_t m = cnt < (uint32_t)NL_MAX ? cnt : (uint32_t)NL_MAX;
    for (uint32_t k = 0; k < m; ++k) {
        const uint32_t e = nl[(int64_t)k * cap + s];
        const uint32_t j = e >> 5, code = e & 31u;
        const V pj = pos4[j];
        const T dx = pi.x - shift[code][0] - pj.x;
        const T dy = pi.y - shift[code][1] - pj.y;
        const T dz = pi.z - shift[code][2] - pj.z;
        const T r = sqrt(dx * dx + dy * dy + dz * dz);
        if (!(r < rd)) continue;
        const T dw = T(-2) * cw * (T(1) - r * inv_rd) * inv_rd;   // w_rho'(r)
        const T f = (rb_i + (T)rbar[j]) * dw / r;
        g[0] += f * dx;
        g[1] += f * dy;
        g[2] += f * dz;
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) xbar[c * cap + s] += (double)g[c];
}

// rbar in cell order from the caller's rhobar in id order.
__global__ void k_gather_by_id(int n, const uint32_t* __restrict__ id,
                               const double* __restrict__ in, double* __restrict__ out)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < n) out[s] = in[id[s]];
}

}  // namespace

void launch_density_vjp(cudaStream_t st, int precision, int n, int64_t cap, const Geo& geo,
                        const Phys& ph, const void* pos4, const uint32_t* nl,
                        const uint32_t* nl_count, const uint32_t* id, const double* rhobar,
                        double* rbar, double* xbar, uint32_t* status)
{
    if (n <= 0) return;
    const int nb = (n + PAIR_BLOCK - 1) / PAIR_BLOCK;
    k_gather_by_id<<<nb, PAIR_BLOCK, 0, st>>>(n, id, rhobar, rbar);
    cudaMemsetAsync(xbar, 0, 3 * (size_t)cap * sizeof(double), st);
    if (precision == 0)
        k_density_vjp<double><<<nb, PAIR_BLOCK, 0, st>>>(n, cap, geo, ph, (const D4*)pos4, nl,
                                                         nl_count, rbar, xbar, status);
    else
        k_density_vjp<float><<<nb, PAIR_BLOCK, 0, st>>>(n, cap, geo, ph, (const float4*)pos4, nl,
                                                        nl_count, rbar, xbar, status);
}

void launch_force_vjp(cudaStream_t st, int precision, int n, int64_t cap, const Geo& geo,
                      const Phys& ph, const void* pos4, const void* vel4, const void* rho,
                      const uint32_t* nl, const uint32_t* nl_count, const uint64_t* step_ptr,
                      const double* abar, double* xbar, double* ubar, double* rbar, double* tbar,
                      uint32_t* status)
{
    if (n <= 0) return;
    const int nb = (n + PAIR_BLOCK - 1) / PAIR_BLOCK;
    if (precision == 0) {
        k_force_vjp<double><<<nb, PAIR_BLOCK, 0, st>>>(n, cap, geo, ph, (const D4*)pos4,
                                                       (const D4*)vel4, (const double*)rho, nl,
                                                       nl_count, step_ptr, abar, xbar, ubar, rbar,
                                                       tbar, status);
        k_density_vjp<double><<<nb, PAIR_BLOCK, 0, st>>>(n, cap, geo, ph, (const D4*)pos4, nl,
                                                         nl_count, rbar, xbar, status);
    } else {
        k_force_vjp<float><<<nb, PAIR_BLOCK, 0, st>>>(n, cap, geo, ph, (const float4*)pos4,
                                                      (const float4*)vel4, (const float*)rho, nl,
                                                      nl_count, step_ptr, abar, xbar, ubar, rbar,
                                                      tbar, status);
        k_density_vjp<float><<<nb, PAIR_BLOCK, 0, st>>>(n, cap, geo, ph, (const float4*)pos4, nl,
                                                        nl_count, rbar, xbar, status);
    }
}

}  // namespace mdpd
