// Adjoint (vector-Jacobian products) of one mDPD force evaluation and of a
// velocity-Verlet window (Sec. 2.1, Eq. 1 and Algorithm 1 of
// arXiv:1903.10134), for single systems and batches of replicas.
//
// One force evaluation maps (x, u, theta) to a_i = sum_j f_ij (i mobile),
// with rho_i = sum_j w_rho(r_ij) recomputed from x, u the velocities the
// dissipative term sees and theta = (A, B, gamma).  Its conservative virial is
// W_ab = 1/2 sum_{i mobile} sum_j d_a F^C_b.  Given abar (the adjoint of the
// accelerations, id order) and, optionally, weights c of the six virial
// components (per replica), the kernels return the gradient of
//     L = sum_i abar_i . a_i + sum_k c_k W_k
// with respect to positions, to u and to the symmetric tables A, B, gamma,
// the random draws of the step held fixed.
//
// For a pair (i, j): d = x_i - x_j, r = |d|, e = d / r, w = e . u_ij,
//   s   = A wc + B (rho_i + rho_j) wd [r < r_d] - gamma wc^2 w + sigma wc xi / sqrt(dt)
//   s_c = A wc + B (rho_i + rho_j) wd [r < r_d]            (conservative part)
// Force part, q = abar_i - abar_j (frozen particles have no acceleration, so
// their abar counts as zero):
//   xbar_i += (q.e)(s_r e + s_w (u_ij - w e) / r) + s (q - (q.e) e) / r
//   ubar_i += (q.e) s_w e,     rhobar_i += (q.e) B wd [r < r_d]
// (s_r = ds/dr at fixed w and rho, s_w = -gamma wc^2).  Virial part, with the
// quadratic form Q(d) = c_xx d_x^2 + c_yy d_y^2 + c_zz d_z^2 + c_xy d_x d_y +
// c_xz d_x d_z + c_yz d_y d_z and m = [i mobile] + [j mobile] (the ordered
// pairs of W that contain the pair):
//   xbar_i += m/2 (s_c (grad Q / r - Q d / r^3) + (Q / r) s_c' e),
//   rhobar_i += m/2 (Q / r) B wd [r < r_d],  s_c' = ds_c/dr at fixed rho.
// The partner lists hold every pair from both sides, so each thread adds its
// own particle's share without atomics (a particle with more partners than
// list slots scans its neighbour cells instead, as the force pass does).  A second pass sends rhobar back to
// positions: xbar_i += (rhobar_i + rhobar_j) w_rho'(r) e over partners within
// r_d.
//
// Parameter gradients are deterministic: each thread accumulates its pairs'
// terms in its own shared-memory column, indexed by (parameter, partner
// type); the block then adds the columns of its threads in thread order for
// every (parameter, own type, partner type), and a per-replica kernel adds the
// blocks in block order.  Each unordered pair is seen from both sides, so each
// side adds half its term.
#include "pair.cuh"

namespace mdpd {

namespace {

constexpr int TB = 3 * 64;         // parameter slots [q][a][b], q = A, B, gamma
constexpr int TCOL = 3 * 8;        // per-thread columns [q][partner type]

// The block's particle slot, replica record and validity (see Batch).
template <bool BATCH>
struct BlockSite {
    int s;
    bool valid;
    int r;
    const Rep* rp;
};

template <bool BATCH>
__device__ __forceinline__ BlockSite<BATCH> block_site(int n, const Batch& bt)
{
    BlockSite<BATCH> b;
    if constexpr (BATCH) {
        const int4 ch = bt.chunks[blockIdx.x];
        b.rp = &block_rep<REP_SCALARS>(bt.reps, ch.x);
        b.r = ch.x;
        b.s = ch.y + (int)threadIdx.x;
        b.valid = (int)threadIdx.x < ch.z;
    } else {
        b.rp = nullptr;
        b.r = 0;
        b.s = blockIdx.x * PAIR_BLOCK + threadIdx.x;
        b.valid = b.s < n;
    }
    return b;
}

// Visit the partners within r_c (0 < r) of particle s: from its list, or, for
// a particle with more partners than list slots, by a scan of its 27
// neighbour cells (the same partners, in cell order), as the force pass does.
template <typename T, typename V, typename F>
__device__ __forceinline__ void for_partners(int s, uint32_t cnt, int64_t cap,
                                             const uint32_t* __restrict__ nl, const Geo& geo,
                                             int64_t cell0, const uint32_t* __restrict__ cell_s,
                                             const uint32_t* __restrict__ start,
                                             const V* __restrict__ pos4, const V& pi,
                                             const T (&shift)[27][3], T rc2,
                                             uint32_t* __restrict__ dbg, F&& partner)
{
    if (cnt <= (uint32_t)NL_MAX) {
        for (uint32_t k = 0; k < cnt; ++k) {
            const uint32_t e = nl[(int64_t)k * cap + s];
            if (MDPD_DBG_OK((e >> 5) < (uint32_t)cap && (e & 31u) < 27u, dbg))
                partner(e >> 5, e & 31u);
        }
        return;
    }
    int q0, q1, q2;
    cell_coords(cell_s[s], geo, q0, q1, q2);      // (the cell within the replica)
    for (int oz = -1; oz <= 1; ++oz) {
        const int z = neighbour_index(q2, oz, geo.nc[2], geo.periodic[2]);
        if (z < 0) continue;
        for (int oy = -1; oy <= 1; ++oy) {
            const int y = neighbour_index(q1, oy, geo.nc[1], geo.periodic[1]);
            if (y < 0) continue;
            for (int ox = -1; ox <= 1; ++ox) {
                const int x = neighbour_index(q0, ox, geo.nc[0], geo.periodic[0]);
                if (x < 0) continue;
                const uint32_t code = (uint32_t)((ox + 1) + 3 * (oy + 1) + 9 * (oz + 1));
                const uint32_t nc = (uint32_t)(cell0 + x + geo.nc[0] * (y + geo.nc[1] * z));
                const uint32_t b = start[nc];
                uint32_t e = start[nc + 1];
                if (!MDPD_DBG_OK(b <= e && e <= (uint32_t)cap, dbg)) e = b;
                for (uint32_t j = b; j < e; ++j) {
                    const V pj = pos4[j];
                    const T dx = pi.x - shift[code][0] - pj.x;
                    const T dy = pi.y - shift[code][1] - pj.y;
                    const T dz = pi.z - shift[code][2] - pj.z;
                    const T r2 = dx * dx + dy * dy + dz * dz;
                    if (r2 < rc2 && r2 > T(0)) partner(j, code);
                }
            }
        }
    }
}

template <typename T, bool BATCH>
__global__ void __launch_bounds__(PAIR_BLOCK)
k_force_vjp(int n, int64_t cap, Geo geo_p, Phys ph_p, Batch bt,
            const typename Vec4<T>::type* __restrict__ pos4,
            const typename Vec4<T>::type* __restrict__ vel4, const T* __restrict__ rho,
            const uint32_t* __restrict__ cell_s, const uint32_t* __restrict__ start,
            const uint32_t* __restrict__ nl, const uint32_t* __restrict__ nl_count,
            const uint64_t* __restrict__ step_ptr, const double* __restrict__ abar,
            const double* __restrict__ wbar, double* __restrict__ xbar,
            double* __restrict__ ubar, double* __restrict__ rbar, double* __restrict__ tpart,
            uint32_t* __restrict__ status)
{
    using V = typename Vec4<T>::type;
    __shared__ double col[PAIR_BLOCK][TCOL + 1];
    __shared__ uint8_t ty[PAIR_BLOCK];
    __shared__ T shift[27][3];
    const BlockSite<BATCH> b = block_site<BATCH>(n, bt);
    const Phys& ph = BATCH ? b.rp->ph : ph_p;             // scalars (and tables if single)
    const Phys& tabs = BATCH ? bt.reps[b.r].ph : ph_p;    // per-type-pair tables
    const uint32_t id0 = BATCH ? b.rp->id0 : 0u;
    const int tid = threadIdx.x;
#pragma unroll
    for (int k = 0; k < TCOL; ++k) col[tid][k] = 0.0;
    if (tid < 27) {
        shift[tid][0] = (T)(tid % 3 - 1) * derived<T>(ph).h[0];
        shift[tid][1] = (T)((tid / 3) % 3 - 1) * derived<T>(ph).h[1];
        shift[tid][2] = (T)(tid / 9 - 1) * derived<T>(ph).h[2];
    }
    const int s = b.s;
    ty[tid] = b.valid ? (uint8_t)unpack_u32(pos4[s].w) : (uint8_t)0xFF;
    __syncthreads();
    if (b.valid) {
        const uint64_t step = *step_ptr;
        const Derived<T>& dc = derived<T>(ph);
        const T inv_rc = dc.inv_rc, inv_rd = dc.inv_rd;
        const T rd = (T)ph.rd;
        const T inv_sqrt_dt = dc.inv_sqrt_dt;
        // virial weights of this replica (c_xx c_yy c_zz c_xy c_xz c_yz)
        T cw[6] = { T(0), T(0), T(0), T(0), T(0), T(0) };
        const bool vir = wbar != nullptr;
        if (vir)
#pragma unroll
            for (int k = 0; k < 6; ++k) cw[k] = (T)wbar[6 * b.r + k];
        const V pi = pos4[s];
        const V vi = vel4[s];
        const T rho_i = rho[s];
        const uint32_t ti = unpack_u32(pi.w), id_i = unpack_u32(vi.w);
        const bool mob_i = ((ph.frozen >> ti) & 1u) == 0u;
        T ai[3] = { T(0), T(0), T(0) };
        if (abar && mob_i)
#pragma unroll
            for (int k = 0; k < 3; ++k) ai[k] = (T)abar[3 * (int64_t)(id0 + id_i) + k];
        T gx[3] = { T(0), T(0), T(0) }, gu[3] = { T(0), T(0), T(0) };
        T gr = T(0);
        // one partner j in the image of neighbour-cell code `code`
        auto partner = [&](uint32_t j, uint32_t code) {
            const V pj = pos4[j];
            const V vj = vel4[j];
            const T rho_j = rho[j];
            const uint32_t tj = unpack_u32(pj.w), id_j = unpack_u32(vj.w);
            const bool mob_j = ((ph.frozen >> tj) & 1u) == 0u;
            const T dx = pi.x - shift[code][0] - pj.x;
            const T dy = pi.y - shift[code][1] - pj.y;
            const T dz = pi.z - shift[code][2] - pj.z;
            const T r2 = dx * dx + dy * dy + dz * dz;
            const T r = sqrt(r2);
            const T ex = dx / r, ey = dy / r, ez = dz / r;
            const T e3[3] = { ex, ey, ez };
            const T wc = T(1) - r * inv_rc;
            const bool near = r < rd;
            const T wd = near ? T(1) - r * inv_rd : T(0);
            const int pidx = ti * 8 + tj;
            const T A = (T)tabs.A[pidx], B = (T)tabs.B[pidx];
            const T rsum = rho_i + rho_j;
            double* cl = col[tid];
            if (abar) {
                T q[3];
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    q[c] = ai[c] - (mob_j ? (T)abar[3 * (int64_t)(id0 + id_j) + c] : T(0));
                const T ux = vi.x - vj.x, uy = vi.y - vj.y, uz = vi.z - vj.z;
                const T u3[3] = { ux, uy, uz };
                const T w = ex * ux + ey * uy + ez * uz;
                const T G = (T)tabs.gamma[pidx];
                const T sig = (T)tabs.sigma[pidx];
                const U4 wr = pair_draw(id_i, id_j, step, ph.key0, ph.key1);
                const T xi = xi_of<T>(wr, ph.xi_dist);
                const T sval = A * wc + B * rsum * wd - G * wc * wc * w + sig * wc * xi * inv_sqrt_dt;
                const T s_r = -A * inv_rc - (near ? B * rsum * inv_rd : T(0)) +
                              T(2) * G * wc * w * inv_rc - sig * xi * inv_sqrt_dt * inv_rc;
                const T s_w = -G * wc * wc;
                const T qe = q[0] * ex + q[1] * ey + q[2] * ez;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    gx[c] += qe * (s_r * e3[c] + s_w * (u3[c] - w * e3[c]) / r) +
                             sval * (q[c] - qe * e3[c]) / r;
                    gu[c] += qe * s_w * e3[c];
                }
                gr += qe * B * wd;
                const double dsig = tabs.gamma[pidx] > 0.0 ? ph.kT / tabs.sigma[pidx] : 0.0;
                cl[0 * 8 + tj] += 0.5 * (double)(qe * wc);
                cl[1 * 8 + tj] += 0.5 * (double)(qe * rsum * wd);
                cl[2 * 8 + tj] += 0.5 * (double)(qe * (-wc * wc * w)) +
                                  0.5 * (double)qe * dsig * (double)(wc * xi * inv_sqrt_dt);
            }
            if (vir) {
                const T mm = T((mob_i ? 1 : 0) + (mob_j ? 1 : 0));
                if (mm > T(0)) {
                    const T Q = cw[0] * dx * dx + cw[1] * dy * dy + cw[2] * dz * dz +
                                cw[3] * dx * dy + cw[4] * dx * dz + cw[5] * dy * dz;
                    const T gQ[3] = { T(2) * cw[0] * dx + cw[3] * dy + cw[4] * dz,
                                      T(2) * cw[1] * dy + cw[3] * dx + cw[5] * dz,
                                      T(2) * cw[2] * dz + cw[4] * dx + cw[5] * dy };
                    const T sc = A * wc + B * rsum * wd;
                    const T sc_r = -A * inv_rc - (near ? B * rsum * inv_rd : T(0));
                    const T Qr = Q / r;
                    const T d3[3] = { dx, dy, dz };
#pragma unroll
                    for (int c = 0; c < 3; ++c)
                        gx[c] += T(0.5) * mm *
                                 (sc * (gQ[c] / r - Q * d3[c] / (r2 * r)) + Qr * sc_r * e3[c]);
                    gr += T(0.5) * mm * Qr * B * wd;
                    cl[0 * 8 + tj] += 0.25 * (double)(mm * Qr * wc);
                    cl[1 * 8 + tj] += 0.25 * (double)(mm * Qr * rsum * wd);
                }
            }
        };
        const Geo& geo = BATCH ? b.rp->geo : geo_p;
        for_partners<T>(s, nl_count[s], cap, nl, geo, BATCH ? b.rp->cell0 : 0, cell_s, start, pos4,
                        pi, shift, derived<T>(ph).rc2, ph.dbg_status, partner);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            xbar[c * cap + s] = (double)gx[c];
            ubar[c * cap + s] = (double)gu[c];
        }
        rbar[s] = (double)gr;
    }
    __syncthreads();
    // slot (q, a, b): the columns (q, b) of the block's threads of type a, in
    // thread order
    for (int k = tid; k < TB; k += PAIR_BLOCK) {
        const int q = k / 64, a = (k / 8) % 8, bb = k % 8;
        double acc = 0.0;
        for (int t = 0; t < PAIR_BLOCK; ++t)
            if (ty[t] == a) acc += col[t][q * 8 + bb];
        tpart[(int64_t)blockIdx.x * TB + k] = acc;
    }
}

template <typename T, bool BATCH>
__global__ void __launch_bounds__(PAIR_BLOCK)
k_density_vjp(int n, int64_t cap, Geo geo_p, Phys ph_p, Batch bt,
              const typename Vec4<T>::type* __restrict__ pos4,
              const uint32_t* __restrict__ cell_s, const uint32_t* __restrict__ start,
              const uint32_t* __restrict__ nl, const uint32_t* __restrict__ nl_count,
              const double* __restrict__ rbar, double* __restrict__ xbar,
              uint32_t* __restrict__ status)
{
    using V = typename Vec4<T>::type;
    __shared__ T shift[27][3];
    const BlockSite<BATCH> b = block_site<BATCH>(n, bt);
    const Phys& ph = BATCH ? b.rp->ph : ph_p;
    if (threadIdx.x < 27) {
        const int c = threadIdx.x;
        shift[c][0] = (T)(c % 3 - 1) * derived<T>(ph).h[0];
        shift[c][1] = (T)((c / 3) % 3 - 1) * derived<T>(ph).h[1];
        shift[c][2] = (T)(c / 9 - 1) * derived<T>(ph).h[2];
    }
    __syncthreads();
    if (!b.valid) return;
    const int s = b.s;
    const Derived<T>& dc = derived<T>(ph);
    const T rd = (T)ph.rd, inv_rd = dc.inv_rd;
    const T cw = dc.cw_rho;
    const V pi = pos4[s];
    const T rb_i = (T)rbar[s];
    T g[3] = { T(0), T(0), T(0) };
    auto partner = [&](uint32_t j, uint32_t code) {
        const V pj = pos4[j];
        const T dx = pi.x - shift[code][0] - pj.x;
        const T dy = pi.y - shift[code][1] - pj.y;
        const T dz = pi.z - shift[code][2] - pj.z;
        const T r = sqrt(dx * dx + dy * dy + dz * dz);
        if (!(r < rd)) return;
        const T dw = T(-2) * cw * (T(1) - r * inv_rd) * inv_rd;   // w_rho'(r)
        const T f = (rb_i + (T)rbar[j]) * dw / r;
        g[0] += f * dx;
        g[1] += f * dy;
        g[2] += f * dz;
    };
    const Geo& geo = BATCH ? b.rp->geo : geo_p;
    for_partners<T>(s, nl_count[s], cap, nl, geo, BATCH ? b.rp->cell0 : 0, cell_s, start, pos4, pi,
                    shift, derived<T>(ph).rc2, ph.dbg_status, partner);
#pragma unroll
    for (int c = 0; c < 3; ++c) xbar[c * cap + s] += (double)g[c];
}

// rbar in cell order from the caller's rhobar in id order (stored, or added
// to what the force VJP left there).
__global__ void k_gather_by_id(int n, const uint32_t* __restrict__ id,
                               const double* __restrict__ in, double* __restrict__ out, int add)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < n) out[s] = add ? out[s] + in[id[s]] : in[id[s]];
}

// Per replica (one block each, TB threads): the sum of its blocks' parameter
// partials in block order, stored (add = 0) or added (add = 1) to acc.
// ranges[r] = (first, end) of replica r's blocks (x4 for warp ranges: scale).
__global__ void k_theta_reduce(int nrep, int nblk, const int2* __restrict__ ranges, int scale,
                               const double* __restrict__ tpart, double* __restrict__ acc, int add)
{
    const int r = blockIdx.x, k = threadIdx.x;
    if (r >= nrep || k >= TB) return;
    int lo = 0, hi = nblk;
    if (ranges) {
        lo = ranges[r].x / scale;
        hi = ranges[r].y / scale;
    }
    double sum = 0.0;
    for (int b = lo; b < hi; ++b) sum += tpart[(int64_t)b * TB + k];
    acc[(int64_t)r * TB + k] = add ? acc[(int64_t)r * TB + k] + sum : sum;
}

// Gradient of the symmetric tables from the per-(own type, partner type) sums
// S: out[q][a][b] = out[q][b][a] = S[q][a][b] + S[q][b][a] for a != b and
// S[q][a][a] on the diagonal.
__global__ void k_theta_symmetrise(int nrep, const double* __restrict__ acc, double* __restrict__ out)
{
    const int r = blockIdx.x, k = threadIdx.x;
    if (r >= nrep || k >= TB) return;
    const int q = k / 64, a = (k / 8) % 8, b = k % 8;
    const double* S = acc + (int64_t)r * TB + q * 64;
    out[(int64_t)r * TB + k] = a == b ? S[a * 8 + a] : S[a * 8 + b] + S[b * 8 + a];
}

// ---- velocity-Verlet window ------------------------------------------------
// Each kernel walks the slots of the current binning (chunks of a batch), so
// that the particle's type, replica and id are at hand; vectors in id order
// are interleaved xyz (element 3 * id + k).

template <bool BATCH>
struct SlotSite {
    int s;
    bool valid;
    const Rep* rp;
};

template <bool BATCH>
__device__ __forceinline__ SlotSite<BATCH> slot_site(int n, const Batch& bt)
{
    SlotSite<BATCH> b;
    if constexpr (BATCH) {
        const int4 ch = bt.chunks[blockIdx.x];
        b.rp = &block_rep<REP_SCALARS>(bt.reps, ch.x);
        b.s = ch.y + (int)threadIdx.x;
        b.valid = (int)threadIdx.x < ch.z;
    } else {
        b.rp = nullptr;
        b.s = blockIdx.x * blockDim.x + threadIdx.x;
        b.valid = b.s < n;
    }
    return b;
}

// Checkpoint of step k of a window: X = x_k and, if VH is given, the
// half-step velocity v'_k = v_k + (dt/2) a_k of mobile particles formed with
// the same arithmetic as the integrator's first half-kick (kick_drift_one;
// frozen particles keep v).
template <bool BATCH>
__global__ void __launch_bounds__(BATCH_CHUNK)
k_win_record(int n, int64_t cap, Phys ph_p, Batch bt, Master m, double* __restrict__ X,
             double* __restrict__ VH)
{
    const SlotSite<BATCH> b = slot_site<BATCH>(n, bt);
    if (!b.valid) return;
    const Phys& ph = BATCH ? b.rp->ph : ph_p;
    const int s = b.s;
    const int64_t i = m.id[s];
    const bool mob = ((ph.frozen >> m.type[s]) & 1u) == 0u;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        X[3 * i + k] = m.x[k * cap + s];
        if (VH) {
            const double v = m.v[k * cap + s];
            const double a = m.a[k * cap + s];
            const double d = ph.prec32 ? to_f64(ph.df.hdt * to_f32(a)) : __dmul_rn(ph.hdt, a);
            VH[3 * i + k] = mob ? __dadd_rn(v, d) : v;
        }
    }
}

// Start of the reverse sweep: xb = xbar_K, vb = vbar_K, ab = (dt/2) vb
// (mobile), the adjoint of the last half-kick.
template <bool BATCH>
__global__ void __launch_bounds__(BATCH_CHUNK)
k_win_init(int n, Phys ph_p, Batch bt, Master m, const double* __restrict__ xbar,
           const double* __restrict__ vbar, double* __restrict__ xb, double* __restrict__ vb,
           double* __restrict__ ab)
{
    const SlotSite<BATCH> b = slot_site<BATCH>(n, bt);
    if (!b.valid) return;
    const Phys& ph = BATCH ? b.rp->ph : ph_p;
    const int s = b.s;
    const int64_t i = m.id[s];
    const double mob = ((ph.frozen >> m.type[s]) & 1u) == 0u ? 1.0 : 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const double x = xbar ? xbar[3 * i + k] : 0.0;
        const double v = vbar ? vbar[3 * i + k] : 0.0;
        xb[3 * i + k] = x;
        vb[3 * i + k] = v;
        ab[3 * i + k] = __dmul_rn(__dmul_rn(ph.hdt, v), mob);
    }
}

// After the force VJP of step k (outputs gx, gu in cell order, [3][cap]):
//   xb += gx;  vhb = vb + gu + dt xb (mobile);  vb = vhb;
//   ab = (dt/2) vhb (mobile), plus (dt/2) vb once more unless this was the
//   window's first step (the next step's half-kick adjoint).
// final = 1 (the VJP of a_0 = F(x_0, v_0)): x0bar = xb + gx, v0bar = vb + gu.
template <bool BATCH>
__global__ void __launch_bounds__(BATCH_CHUNK)
k_win_post(int n, int64_t cap, Phys ph_p, Batch bt, Master m, const double* __restrict__ gx,
           const double* __restrict__ gu, double* __restrict__ xb, double* __restrict__ vb,
           double* __restrict__ ab, int first, int final, double* __restrict__ x0bar,
           double* __restrict__ v0bar)
{
    const SlotSite<BATCH> b = slot_site<BATCH>(n, bt);
    if (!b.valid) return;
    const Phys& ph = BATCH ? b.rp->ph : ph_p;
    const int s = b.s;
    const int64_t i = m.id[s];
    const double mob = ((ph.frozen >> m.type[s]) & 1u) == 0u ? 1.0 : 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const double g = gx[k * cap + s], u = gu[k * cap + s];
        if (final) {
            if (x0bar) x0bar[3 * i + k] = __dadd_rn(xb[3 * i + k], g);
            if (v0bar) v0bar[3 * i + k] = __dadd_rn(vb[3 * i + k], u);
            continue;
        }
        const double x = __dadd_rn(xb[3 * i + k], g);
        const double vh = __dadd_rn(__dadd_rn(vb[3 * i + k], u), __dmul_rn(__dmul_rn(ph.dt, x), mob));
        const double t = __dmul_rn(__dmul_rn(ph.hdt, vh), mob);
        xb[3 * i + k] = x;
        vb[3 * i + k] = vh;
        ab[3 * i + k] = first ? t : __dadd_rn(t, t);
    }
}

inline unsigned pair_blocks(int n) { return (unsigned)((n + PAIR_BLOCK - 1) / PAIR_BLOCK); }

}  // namespace

int vjp_num_blocks(int n, const Batch* bt)
{
    return bt ? bt->nchunk : (int)pair_blocks(n);
}

void launch_force_vjp(cudaStream_t st, int precision, int n, int64_t cap, const Geo& geo,
                      const Phys& ph, const Batch* bt, const void* pos4, const void* vel4,
                      const void* rho, const uint32_t* cell_s, const uint32_t* start,
                      const uint32_t* nl, const uint32_t* nl_count, const uint64_t* step_ptr,
                      const double* abar, const double* wbar, double* xbar, double* ubar,
                      double* rbar, double* tpart, uint32_t* status)
{
    const int nb = vjp_num_blocks(n, bt);
    if (nb <= 0) return;
    const Batch bb = bt ? *bt : Batch{};
    const size_t smem = bt ? REP_SMEM : 0;
#define MDPD_FVJP(T_, B_)                                                                       \
    k_force_vjp<T_, B_><<<nb, PAIR_BLOCK, smem, st>>>(                                        \
        n, cap, geo, ph, bb, (const typename Vec4<T_>::type*)pos4,                                \
        (const typename Vec4<T_>::type*)vel4, (const T_*)rho, cell_s, start, nl, nl_count,        \
        step_ptr, abar, wbar, xbar, ubar, rbar, tpart, status)
    if (precision == 0) {
        if (bt) MDPD_FVJP(double, true);
        else MDPD_FVJP(double, false);
    } else {
        if (bt) MDPD_FVJP(float, true);
        else MDPD_FVJP(float, false);
    }
#undef MDPD_FVJP
}

void launch_density_vjp(cudaStream_t st, int precision, int n, int64_t cap, const Geo& geo,
                        const Phys& ph, const Batch* bt, const void* pos4,
                        const uint32_t* cell_s, const uint32_t* start, const uint32_t* nl,
                        const uint32_t* nl_count, const double* rbar, double* xbar,
                        uint32_t* status)
{
    const int nb = vjp_num_blocks(n, bt);
    if (nb <= 0) return;
    const Batch bb = bt ? *bt : Batch{};
    const size_t smem = bt ? REP_SMEM : 0;
#define MDPD_DVJP(T_, B_)                                                                       \
    k_density_vjp<T_, B_><<<nb, PAIR_BLOCK, smem, st>>>(                                      \
        n, cap, geo, ph, bb, (const typename Vec4<T_>::type*)pos4, cell_s, start, nl, nl_count,  \
        rbar, xbar, status)
    if (precision == 0) {
        if (bt) MDPD_DVJP(double, true);
        else MDPD_DVJP(double, false);
    } else {
        if (bt) MDPD_DVJP(float, true);
        else MDPD_DVJP(float, false);
    }
#undef MDPD_DVJP
}

void launch_gather_by_id(cudaStream_t st, int n, const uint32_t* id, const double* in, double* out,
                         int add)
{
    if (n <= 0) return;
    k_gather_by_id<<<pair_blocks(n), PAIR_BLOCK, 0, st>>>(n, id, in, out, add);
}

__global__ void k_set_u64(uint64_t* __restrict__ p, uint64_t v) { *p = v; }

void launch_set_step(cudaStream_t st, uint64_t* step_ptr, uint64_t value)
{
    k_set_u64<<<1, 1, 0, st>>>(step_ptr, value);
}

void launch_theta_reduce(cudaStream_t st, int nrep, int nblk, const int2* ranges, int scale,
                         const double* tpart, double* acc, int add)
{
    if (nrep <= 0) return;
    k_theta_reduce<<<nrep, TB, 0, st>>>(nrep, nblk, ranges, scale, tpart, acc, add);
}

void launch_theta_symmetrise(cudaStream_t st, int nrep, const double* acc, double* out)
{
    if (nrep <= 0) return;
    k_theta_symmetrise<<<nrep, TB, 0, st>>>(nrep, acc, out);
}

void launch_win_record(cudaStream_t st, int n, int64_t cap, const Phys& ph, const Batch* bt,
                       const Master& m, double* X, double* VH)
{
    if (bt) {
        if (bt->nchunk > 0)
            k_win_record<true><<<bt->nchunk, BATCH_CHUNK, REP_SMEM, st>>>(n, cap, ph, *bt, m, X, VH);
    } else if (n > 0) {
        k_win_record<false><<<(n + BATCH_CHUNK - 1) / BATCH_CHUNK, BATCH_CHUNK, 0, st>>>(
            n, cap, ph, Batch{}, m, X, VH);
    }
}

void launch_win_init(cudaStream_t st, int n, const Phys& ph, const Batch* bt, const Master& m,
                     const double* xbar, const double* vbar, double* xb, double* vb, double* ab)
{
    if (bt) {
        if (bt->nchunk > 0)
            k_win_init<true><<<bt->nchunk, BATCH_CHUNK, REP_SMEM, st>>>(n, ph, *bt, m, xbar, vbar,
                                                                        xb, vb, ab);
    } else if (n > 0) {
        k_win_init<false><<<(n + BATCH_CHUNK - 1) / BATCH_CHUNK, BATCH_CHUNK, 0, st>>>(
            n, ph, Batch{}, m, xbar, vbar, xb, vb, ab);
    }
}

void launch_win_post(cudaStream_t st, int n, int64_t cap, const Phys& ph, const Batch* bt,
                     const Master& m, const double* gx, const double* gu, double* xb, double* vb,
                     double* ab, int first, int final, double* x0bar, double* v0bar)
{
    if (bt) {
        if (bt->nchunk > 0)
            k_win_post<true><<<bt->nchunk, BATCH_CHUNK, REP_SMEM, st>>>(
                n, cap, ph, *bt, m, gx, gu, xb, vb, ab, first, final, x0bar, v0bar);
    } else if (n > 0) {
        k_win_post<false><<<(n + BATCH_CHUNK - 1) / BATCH_CHUNK, BATCH_CHUNK, 0, st>>>(
            n, cap, ph, Batch{}, m, gx, gu, xb, vb, ab, first, final, x0bar, v0bar);
    }
}

}  // namespace mdpd
