// Device pieces shared by the density and force kernels: the pair force of
// Sec. 2.1 / Eq. 1 (arXiv:1903.10134), the velocity-Verlet epilogue of
// Algorithm 1 with the wall reflection, and the FP64 block reduction of the
// observables.
#pragma once

#include "f64bits.cuh"
#include "mdpd_internal.cuh"
#include "philox.cuh"
#include "vec.cuh"

namespace mdpd {

constexpr int PAIR_BLOCK = 128;
constexpr int NOBS = 14;     // momentum 3, sum v^2 3, virial 6, mobile count 1, pairs 1
constexpr int NL_MAX = NL_SLOTS;   // neighbour-list slots per particle (more: direct scan)

__device__ __forceinline__ float rsqrt_t(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_t(double x) { return 1.0 / sqrt(x); }
// r from r^2 (> 0) for the density weight: FP32 through the hardware reciprocal
// square root (about 2 ulp), FP64 correctly rounded.
__device__ __forceinline__ float sqrt_t(float x) { return x * rsqrtf(x); }
__device__ __forceinline__ double sqrt_t(double x) { return sqrt(x); }
// Same for r^2 >= 0, giving 0 at 0.
__device__ __forceinline__ float sqrt0_t(float x) { return x * rsqrtf(fmaxf(x, 1e-30f)); }
__device__ __forceinline__ double sqrt0_t(double x) { return sqrt(x); }
// r from r^2 >= 0 in one instruction: the PTX approximate square root (its
// FP32 error is within the density pass's FP32 tolerance; the density parity
// tests bound it), FP64 correctly rounded.
__device__ __forceinline__ float sqrt_fast(float x)
{
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ double sqrt_fast(double x) { return sqrt(x); }

template <typename T>
__device__ __forceinline__ T xi_of(U4 w, int dist)
{
    if (dist == 0) return xi_uniform<T>(w.x);
    if constexpr (sizeof(T) == 4) return xi_gauss_f(w.x, w.y);
    else return xi_gauss_d(w.x, w.y);
}

// Per-type-pair tables in shared memory, row ti: A, B, gamma, sigma.
template <typename T>
struct PairTables {
    typename Vec4<T>::type P[64];     // (A, B, gamma, sigma) of type pair [ti * 8 + tj]
};

template <typename T>
__device__ __forceinline__ void load_tables(PairTables<T>& t, const Phys& ph)
{
    for (int k = threadIdx.x; k < 64; k += blockDim.x)
        t.P[k] = make4((T)ph.A[k], (T)ph.B[k], (T)ph.gamma[k], (T)ph.sigma[k]);
}

template <typename T>
struct PairConst {
    T rc2, rd2, inv_rc, inv_rd, inv_sqrt_dt;
    __device__ explicit PairConst(const Phys& ph)
        : rc2(derived<T>(ph).rc2), rd2(derived<T>(ph).rd2), inv_rc(derived<T>(ph).inv_rc),
          inv_rd(derived<T>(ph).inv_rd), inv_sqrt_dt(derived<T>(ph).inv_sqrt_dt)
    {
    }
};

// Add the force of j on i (separation d = r_i - r_j, 0 < r2 < r_c^2) to f and
// the conservative virial 0.5 d_a F^C e_b to W:
//   F = [A w_C + B (rho_i + rho_j) w_d [r < r_d] - gamma w_C^2 (e.v_ij)
//        + sigma w_C xi_ij / sqrt(dt)] e,   w_C = 1 - r/r_c, w_d = 1 - r/r_d.
template <typename T, bool RK, typename V4>
__device__ __forceinline__ void pair_term(const PairConst<T>& c, const V4& prm, T dx, T dy, T dz,
                                          T r2, const V4& vi, const V4& vj, T rho_i, T rho_j,
                                          uint32_t id_i, uint32_t id_j, uint64_t step,
                                          const Phys& ph, T (&f)[3], T (&W)[6])
{
    // prm = (A, B, gamma, sigma) of the pair's types
    const T rinv = rsqrt_t(r2);
    const T r = r2 * rinv;
    const T wc = T(1) - r * c.inv_rc;
    T fc = prm.x * wc;
    if (r2 < c.rd2) fc += prm.y * (rho_i + rho_j) * (T(1) - r * c.inv_rd);
    const T ev = (dx * (vi.x - vj.x) + dy * (vi.y - vj.y) + dz * (vi.z - vj.z)) * rinv;
    const T fd = -prm.z * wc * wc * ev;
    const U4 w = RK ? pair_draw_rk(id_i, id_j, step, ph.rk)
                    : pair_draw(id_i, id_j, step, ph.key0, ph.key1);
    const T fr = prm.w * wc * xi_of<T>(w, ph.xi_dist) * c.inv_sqrt_dt;
    const T fp = (fc + fd + fr) * rinv;
    f[0] += fp * dx;
    f[1] += fp * dy;
    f[2] += fp * dz;
    const T fv = T(0.5) * fc * rinv;      // 0.5 d_a F^C e_b = 0.5 fc d_a d_b / r
    W[0] += fv * dx * dx;
    W[1] += fv * dy * dy;
    W[2] += fv * dz * dz;
    W[3] += fv * dx * dy;
    W[4] += fv * dx * dz;
    W[5] += fv * dy * dz;
}

// floor((x - lo) * s) or floor((x - lo) / d) in FP64 (div: d used), the exact
// cell or voxel index for the rare coordinates near a face.  Not inlined, so
// that the compiler cannot execute its FP64 instructions speculatively for
// every particle (FP64 runs at 1/64 of the FP32 rate on this part).
static __device__ __noinline__ double floor_index_f64(double x, double lo, double s, double d, int div)
{
    const double t = __dsub_rn(x, lo);
    return floor(div ? __ddiv_rn(t, d) : __dmul_rn(t, s));
}

// Drift by dt with velocity v, wrap periodic axes, and undo the drift with a
// negated velocity if the new position is beyond a non-periodic face or in a
// solid voxel.  Explicit round-to-nearest operations keep each product and
// sum separately rounded.
__device__ __forceinline__ void drift_reflect(double (&x)[3], double (&v)[3], const Geo& geo,
                                              const MaskDev& mk, double dt)
{
    double xn[3];
    bool blocked = false;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        xn[k] = __dadd_rn(x[k], __dmul_rn(dt, v[k]));
        // the comparisons with the box faces on integer keys of the bits
        // (f64_key orders like the FP64 comparison, off the FP64 pipe)
        const int64_t kx = f64_key(xn[k]);
        if (geo.periodic[k]) {
            // the rare wrap behind a warp-voted branch (FP64 adds)
            const bool up = kx >= geo.key_hi[k], down = kx < geo.key_lo[k];
            if (__any_sync(__activemask(), up || down)) {
                if (up) xn[k] = __dsub_rn(xn[k], geo.L[k]);
                else if (down) xn[k] = __dadd_rn(xn[k], geo.L[k]);
            }
        } else if (kx < geo.key_lo[k] || kx >= geo.key_hi[k]) {
            blocked = true;
        }
    }
    if (!blocked && mk.bits != nullptr) {
        bool inside = true;
        int64_t q[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            // voxel index in FP32 when that cannot differ from the FP64 one
            // (mk.fast: FP32 error below 4e-4 voxels; the index is taken only
            // 2e-3 voxels or more from a face), in FP64 otherwise; the FP64
            // path sits behind a branch that a warp takes only when one of
            // its lanes needs it (if-converted, it ran on the 1/64-rate FP64
            // pipe for every particle)
            bool done = false;
            if (mk.fast) {
                const float t = (to_f32(xn[k]) - mk.origin_f[k]) * mk.inv_voxel_f;
                const float fl = floorf(t);
                if (t - fl > 2e-3f && fl + 1.0f - t > 2e-3f) {
                    if (!(fl >= 0.0f) || fl >= (float)mk.dim[k]) inside = false;
                    q[k] = inside ? (int64_t)fl : 0;
                    done = true;
                }
            }
            if (__any_sync(__activemask(), !done)) {
                if (!done) {
                    // for a power-of-two voxel t * (1/voxel) is exactly t / voxel
                    const double f = floor_index_f64(xn[k], mk.origin[k], mk.inv_voxel,
                                                     mk.voxel, !mk.inv_voxel_exact);
                    if (!(f >= 0.0) || f >= (double)mk.dim[k]) inside = false;
                    q[k] = inside ? (int64_t)f : 0;
                }
            }
        }
        if (inside) {
            const int64_t idx = q[0] + (int64_t)mk.dim[0] * (q[1] + (int64_t)mk.dim[1] * q[2]);
            blocked = (mk.bits[idx >> 5] >> (idx & 31)) & 1u;
        }
    }
    if (blocked) {
#pragma unroll
        for (int k = 0; k < 3; ++k) v[k] = -v[k];
    } else {
#pragma unroll
        for (int k = 0; k < 3; ++k) x[k] = xn[k];
    }
}

// First half-kick, drift and reflection of the particle in master slot s
// (Algorithm 1: v += dt/2 a, x += dt v); frozen particles stay.
// With FP32 pair arithmetic the stored acceleration is an FP32 value and the
// increment is formed in FP32 as in force_finish.
__device__ __forceinline__ void kick_drift_one(int s, int64_t cap, const Geo& geo, const Phys& ph,
                                               const MaskDev& mk, const Master& m,
                                               uint32_t* status)
{
    if ((ph.frozen >> m.type[s]) & 1u) return;
    double x[3], v[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        x[k] = m.x[k * cap + s];
        const double a = m.a[k * cap + s];
        const double d = ph.prec32 ? to_f64(ph.df.hdt * to_f32(a)) : __dmul_rn(ph.hdt, a);
        v[k] = __dadd_rn(m.v[k * cap + s], d);
    }
    drift_reflect(x, v, geo, mk, ph.dt);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        m.x[k * cap + s] = x[k];
        m.v[k * cap + s] = v[k];
    }
    if (!isfinite(v[0]) || !isfinite(v[1]) || !isfinite(v[2])) atomicOr(status, ST_NONFINITE);
}

// Everything after the pair sum of mobile-or-frozen particle s: acceleration,
// the half-kick(s), drift and reflection by MODE, and the observables (in T).
//
// FP64 pair arithmetic (T = double) takes every step in FP64 with separately
// rounded products and sums.  With FP32 pair arithmetic the forces carry FP32
// rounding anyway, so the kick increment dv = (dt/2) a is formed in FP32 and
// applied to the FP64 master velocity with one conversion and one add per
// component; FP64 instructions run at 1/64 of the FP32 rate on this part,
// and this keeps the epilogue close to the drift's cost.
template <typename T, int MODE>
__device__ __forceinline__ void force_finish(int s, bool mobile, const T (&f)[3],
                                             const T (&W)[6], int npair, int64_t cap,
                                             const Geo& geo, const Phys& ph, const MaskDev& mk,
                                             const Master& m, double* __restrict__ out,
                                             T (&obs)[NOBS], uint32_t* status)
{
    uint32_t st = 0;
    if constexpr (sizeof(T) == 8) {
        double a[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) a[k] = mobile ? (double)f[k] + ph.g[k] : 0.0;
        if (!isfinite(a[0]) || !isfinite(a[1]) || !isfinite(a[2])) st |= ST_NONFINITE;
        double v[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) v[k] = m.v[k * cap + s];
        if (MODE == FM_EVAL) {
#pragma unroll
            for (int k = 0; k < 3; ++k) out[k * cap + s] = a[k];
        } else if (mobile) {
#pragma unroll
            for (int k = 0; k < 3; ++k) v[k] = __dadd_rn(v[k], __dmul_rn(ph.hdt, a[k]));
        }
        if (mobile) {
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                obs[k] = v[k];
                obs[3 + k] = v[k] * v[k];
            }
        }
        if (MODE == FM_LAST && mobile) {
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                m.v[k * cap + s] = v[k];
                m.a[k * cap + s] = a[k];
            }
        }
        if (MODE == FM_FUSED && mobile) {
            double x[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                x[k] = m.x[k * cap + s];
                v[k] = __dadd_rn(v[k], __dmul_rn(ph.hdt, a[k]));
            }
            drift_reflect(x, v, geo, mk, ph.dt);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                m.x[k * cap + s] = x[k];
                m.v[k * cap + s] = v[k];
            }
        }
        if (MODE != FM_EVAL && (!isfinite(v[0]) || !isfinite(v[1]) || !isfinite(v[2])))
            st |= ST_NONFINITE;
    } else {
        const Derived<float>& dc = ph.df;
        float af[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) af[k] = mobile ? f[k] + dc.g[k] : 0.f;
        if (!isfinite(af[0]) || !isfinite(af[1]) || !isfinite(af[2])) st |= ST_NONFINITE;
        double v[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) v[k] = m.v[k * cap + s];
        // (conversions between FP32 and FP64 in integer arithmetic, off the
        // FP64 pipe: see f64bits.cuh)
        if (MODE == FM_EVAL) {
#pragma unroll
            for (int k = 0; k < 3; ++k) out[k * cap + s] = to_f64(af[k]);
        }
        if (mobile) {
            float dv[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                dv[k] = MODE == FM_EVAL ? 0.f : dc.hdt * af[k];
                const float v1 = to_f32(v[k]) + dv[k];          // v(t + dt)
                obs[k] = v1;
                obs[3 + k] = v1 * v1;
            }
            if (MODE == FM_LAST) {
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    m.v[k * cap + s] = __dadd_rn(v[k], to_f64(dv[k]));
                    m.a[k * cap + s] = to_f64(af[k]);
                }
            }
            if (MODE == FM_FUSED) {
                // the same two adds as FM_LAST followed by the next step's
                // first kick (kick_drift_one), so split and fused steps agree
                double x[3];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    x[k] = m.x[k * cap + s];
                    const double d = to_f64(dv[k]);
                    v[k] = __dadd_rn(__dadd_rn(v[k], d), d);
                }
                drift_reflect(x, v, geo, mk, ph.dt);
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    m.x[k * cap + s] = x[k];
                    m.v[k * cap + s] = v[k];
                }
            }
        }
    }
    if (mobile) {
#pragma unroll
        for (int k = 0; k < 6; ++k) obs[6 + k] = W[k];
        obs[12] = T(1);
        obs[13] = (T)npair;
    }
    if (st) atomicOr(status, st);
}

// Per-warp partial sums of the observables, written as T to
// partials[k * nparts + global warp index] with no block-wide barrier,
// so a warp that finishes early does not hold its block.  The values are
// transposed through shared memory and summed serially by a few lanes (16
// values per lane, then one combining add) instead of a shuffle tree in which
// every lane adds at every level; with FP32 pair arithmetic these 32-term
// sums and the stored partials are FP32 (FP64 instructions, conversions
// included, are slow on this part).  The two integer counts use the warp
// integer reduction and are stored as integer bit patterns.
// The order of the additions is fixed, so the result is reproducible.
constexpr int NOBS_F = 12;   // momentum 3, sum v^2 3, virial 6

// The two count partials travel as the bit pattern of an unsigned integer in
// a T slot (no conversion instructions; read back with bits_count).
template <typename T>
__device__ __forceinline__ T count_bits(unsigned c)
{
    if constexpr (sizeof(T) == 4) return __uint_as_float(c);
    else return __longlong_as_double((long long)c);
}
template <typename T>
__device__ __forceinline__ unsigned long long bits_count(T x)
{
    if constexpr (sizeof(T) == 4) return (unsigned long long)__float_as_uint(x);
    else return (unsigned long long)__double_as_longlong(x);
}

template <typename T>
__device__ __forceinline__ void warp_obs_store(const T (&o)[NOBS], double* __restrict__ partials,
                                               int64_t nparts)
{
    __shared__ T sh[PAIR_BLOCK / 32][NOBS_F][33];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NOBS_F; ++k) sh[warp][k][lane] = o[k];
    const unsigned nm = __reduce_add_sync(0xffffffffu, (unsigned)o[12]);
    const unsigned np = __reduce_add_sync(0xffffffffu, (unsigned)o[13]);
    __syncwarp();
    const int k = lane & 15, half = lane >> 4;
    T v = T(0);
    if (k < NOBS_F) {
#pragma unroll
        for (int l = 0; l < 16; ++l) v += sh[warp][k][16 * half + l];
    }
    v += __shfl_down_sync(0xffffffffu, v, 16);
    const int64_t gw = (int64_t)blockIdx.x * (PAIR_BLOCK / 32) + warp;
    T* p = reinterpret_cast<T*>(partials);
    if (lane < NOBS_F) p[(int64_t)lane * nparts + gw] = v;
    if (lane == 0) {
        p[(int64_t)12 * nparts + gw] = count_bits<T>(nm);
        p[(int64_t)13 * nparts + gw] = count_bits<T>(np);
    }
}

// Observables from the summed partials t (momentum 3, sum v^2 3, virial 6,
// mobile count, pairs): o = momentum, kinetic energy, kT, virial, sum v^2,
// mobile count, step; obs[2 * MDPD_NUM_OBS + 1] = the directed pair count.
__device__ __forceinline__ void finish_obs(const double (&t)[NOBS], uint64_t step,
                                           double* __restrict__ obs, double* __restrict__ obs_sum,
                                           double* __restrict__ obs_count, int advance)
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

// Decompose a cell id into lattice coordinates.
__device__ __forceinline__ void cell_coords(uint32_t c, const Geo& geo, int& q0, int& q1, int& q2)
{
    q0 = (int)(c % (uint32_t)geo.nc[0]);
    q1 = (int)((c / (uint32_t)geo.nc[0]) % (uint32_t)geo.nc[1]);
    q2 = (int)(c / ((uint32_t)geo.nc[0] * (uint32_t)geo.nc[1]));
}

// Neighbour cell along one axis: -1 if it falls off a non-periodic face.
__device__ __forceinline__ int neighbour_index(int q, int o, int nc, int periodic)
{
    int z = q + o;
    if (z < 0 || z >= nc) {
        if (!periodic) return -1;
        z = z < 0 ? z + nc : z - nc;
    }
    return z;
}

}  // namespace mdpd
