/*
 * mdpd_oracle.c -- plain, slow, obviously-correct FP64 CPU oracle of the
 * many-body DPD (mDPD) hot path of arXiv:1903.10134.
 *
 * TEST INFRASTRUCTURE.  Only the test-suite, the package smoke check and the
 * benchmark's CPU-baseline leg load this library.  The product (the CUDA
 * library under paper_1903_10134_gb300/) never calls it and shares no code,
 * header, table or constant generator with it.
 *
 * What it computes, with the passage of the paper that defines each piece:
 *   pair force  F_ij = F^C + F^D + F^R, central, r_ij = r_i - r_j     Sec. 2.1
 *   F^D = -gamma w_D(r) (e.v_ij) e,  F^R = sigma w_R(r) xi_ij e        Sec. 2.1
 *   sigma^2 = 2 gamma kT,  w_D = w_R^2,  w_C = w_R = 1 - r/r_c          Sec. 2.1
 *   F^C = A w_C(r) e + B (rho_i + rho_j) w_d(r) e,  w_d = 1 - r/r_d     Eq. 1
 *   rho_i = sum_{j != i} w_rho(r_ij),
 *   w_rho = 15/(2 pi r_d^3) (1 - r/r_d)^2, int 4 pi r^2 w_rho = 1       Sec. 2.1
 *   velocity-Verlet step: x(t+dt), then rho, then f(t+dt), then
 *   v(t+dt)                                                  Algorithm 1
 *   walls: fluid may not enter solid voxels of the pore image (no-slip,
 *   non-penetration)                                        Sec. 2.2, 3.2
 *   wall particles fill the solid voxels within a shell of given
 *   thickness of the pore space                                   Sec. 2.3
 *   wall density phi_i of solid particles within a fluid particle's
 *   support                                         Sec. 3.2, Algorithm 1
 *
 * Where the paper is silent the oracle takes these readings (each is stated
 * again at the code that uses it):
 *   - the random force is divided by sqrt(dt) (standard DPD time discretisation);
 *   - xi_ij is uniform with unit variance: xi = sqrt(3) * m * 2^-24 with the odd
 *     integer m = 2*(w0 >> 8) + 1 - 2^24, where w0 is word 0 of
 *     Philox-4x32-10 (Salmon et al., SC'11) with key (seed_lo, seed_hi) and
 *     counter (min id, max id, step_lo, step_hi); a Box-Muller Gaussian option
 *     uses words 0 and 1;
 *   - pairs interact for 0 < r < r_c (force) and r < r_d (density; r = 0
 *     contributes w_rho(0));
 *   - the half-kick / drift / reflect / rho / force / half-kick order, with the
 *     dissipative force seeing v(t + dt/2);
 *   - reflection: a drift that lands in a solid voxel or beyond a non-periodic
 *     box face is undone (x <- x(t)) and the half-step velocity is negated;
 *   - the virial is taken over the conservative force only.
 *
 * All arithmetic is FP64.  The library is compiled with -ffp-contract=off so
 * that every a*b+c rounds twice, exactly as written.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXT 8

typedef struct orc_sys {
    double lo[3];                 /* box lower corner                       */
    double L[3];                  /* box edge lengths                       */
    int32_t periodic[3];          /* 1 = periodic, 0 = reflecting faces     */
    int32_t ntypes;
    double rc, rd, dt, kT;
    double A[ORC_MAXT][ORC_MAXT];     /* attractive amplitude, Eq. 1         */
    double B[ORC_MAXT][ORC_MAXT];     /* many-body repulsion, Eq. 1          */
    double gamma[ORC_MAXT][ORC_MAXT]; /* dissipation, Sec. 2.1               */
    double g[3];                  /* body acceleration on mobile particles  */
    uint32_t frozen_mask;         /* bit t set: particles of type t frozen  */
    int32_t xi_dist;              /* 0 uniform (unit variance), 1 Gaussian  */
    int32_t rho_self;             /* 1: add w_rho(0) for j = i (off by default) */
    int32_t use_cells;            /* 0: all pairs O(N^2); 1: cell list      */
    uint64_t seed;
    const uint8_t *mask;          /* solid voxels (x fastest), NULL = none  */
    int32_t mdim[3];
    int32_t pad_;
    double voxel;
    double morigin[3];
} orc_sys;

/* ------------------------------------------------------------------------ */
/* Philox-4x32-10, from its published definition (Salmon, Moraes, Dror and   */
/* Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11): ten rounds of */
/* a 2x(32x32->64) multiply S-box on a 4-word counter; the 2-word key is      */
/* bumped by the Weyl constants between rounds.                               */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                       uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += W0; k1 += W1; }
        uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* The pair random variable xi_ij of F^R (Sec. 2.1).  It must be the same     */
/* number seen from i and from j, so the counter holds (min id, max id).      */
double orc_xi(uint64_t seed, uint64_t step, uint32_t id_i, uint32_t id_j,
              int32_t dist)
{
    uint32_t a = id_i < id_j ? id_i : id_j;
    uint32_t b = id_i < id_j ? id_j : id_i;
    uint32_t ctr[4] = { a, b, (uint32_t)step, (uint32_t)(step >> 32) };
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    uint32_t w[4];
    orc_philox4x32_10(ctr, key, w);
    if (dist == 0) {
        /* uniform on (-sqrt3, sqrt3): mean 0, variance 1 */
        int32_t m = (int32_t)((w[0] >> 8) << 1) + 1 - (1 << 24);
        return sqrt(3.0) * ((double)m * (1.0 / 16777216.0));
    }
    /* Box-Muller standard normal from words 0 and 1 */
    double u1 = ((double)(w[0] >> 8) + 0.5) * (1.0 / 16777216.0);
    double u2 = ((double)(w[1] >> 8) + 0.5) * (1.0 / 16777216.0);
    const double two_pi = 6.283185307179586476925286766559;
    return sqrt(-2.0 * log(u1)) * cos(two_pi * u2);
}

/* w_rho of Sec. 2.1 (the paper's "w_d(r) = 15/(2 pi r_d^3)(1-r/r_d)^2" is    */
/* the density weight; w_d itself stays 1 - r/r_d in Eq. 1).                 */
double orc_w_rho(double r, double rd)
{
    if (r >= rd) return 0.0;
    const double pi = 3.14159265358979323846264338327950288;
    double q = 1.0 - r / rd;
    return 15.0 / (2.0 * pi * rd * rd * rd) * q * q;
}

static double min_image(double d, double L, int periodic)
{
    if (periodic) d -= L * nearbyint(d / L);
    return d;
}

static void pair_vec(const orc_sys *s, const double *xi, const double *xj,
                     double d[3])
{
    for (int k = 0; k < 3; ++k)
        d[k] = min_image(xi[k] - xj[k], s->L[k], s->periodic[k]);
}

static int is_frozen(const orc_sys *s, int32_t t)
{
    return (int)((s->frozen_mask >> (uint32_t)t) & 1u);
}

/* Pair force on i from j, Sec. 2.1 and Eq. 1.  Writes the total pair force   */
/* f[3] and the conservative virial terms 0.5 * d_a * F^C_b (xx yy zz xy xz  */
/* yz).  Returns 0 if the pair is outside 0 < r < r_c.                        */
int orc_pair_force(const orc_sys *s, const double d[3], const double vij[3],
                   int32_t ti, int32_t tj, double rho_i, double rho_j,
                   double xi, double f[3], double vir[6])
{
    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    if (!(r2 < s->rc * s->rc) || !(r2 > 0.0)) return 0;
    double r = sqrt(r2);
    double e[3] = { d[0] / r, d[1] / r, d[2] / r };
    double wc = 1.0 - r / s->rc;                       /* w_C = w_R */
    double fc = s->A[ti][tj] * wc;
    if (r < s->rd) fc += s->B[ti][tj] * (rho_i + rho_j) * (1.0 - r / s->rd);
    double ev = e[0] * vij[0] + e[1] * vij[1] + e[2] * vij[2];
    double fd = -s->gamma[ti][tj] * (wc * wc) * ev;    /* w_D = w_R^2 */
    double sigma = sqrt(2.0 * s->gamma[ti][tj] * s->kT);
    double fr = sigma * wc * xi / sqrt(s->dt);
    double ftot = fc + fd + fr;
    for (int k = 0; k < 3; ++k) f[k] = ftot * e[k];
    if (vir) {
        vir[0] = 0.5 * d[0] * (fc * e[0]);
        vir[1] = 0.5 * d[1] * (fc * e[1]);
        vir[2] = 0.5 * d[2] * (fc * e[2]);
        vir[3] = 0.5 * d[0] * (fc * e[1]);
        vir[4] = 0.5 * d[0] * (fc * e[2]);
        vir[5] = 0.5 * d[1] * (fc * e[2]);
    }
    return 1;
}

/* ------------------------------------------------------------------------ */
/* Neighbour enumeration.  use_cells = 0 walks every j in index order.       */
/* use_cells = 1 finds the same j through a cell lattice of edge >= r_c and   */
/* then visits them in ascending j, so both modes add the same terms in the   */
/* same order and give bit-identical sums.                                    */
/* ------------------------------------------------------------------------ */
typedef struct {
    int nc[3];
    double h[3];
    int64_t *head;   /* first particle of each cell, -1 if empty */
    int64_t *next;   /* next particle in the same cell           */
} orc_cells;

static int cells_build(const orc_sys *s, int64_t n, const double *x,
                       orc_cells *c)
{
    int64_t ncell = 1;
    for (int k = 0; k < 3; ++k) {
        int m = (int)floor(s->L[k] / s->rc);
        if (m < 1) m = 1;
        if (s->periodic[k] && m < 3) return -1;
        c->nc[k] = m;
        c->h[k] = s->L[k] / m;
        ncell *= m;
    }
    c->head = (int64_t *)malloc(sizeof(int64_t) * (size_t)ncell);
    c->next = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!c->head || !c->next) return -2;
    for (int64_t q = 0; q < ncell; ++q) c->head[q] = -1;
    for (int64_t i = n - 1; i >= 0; --i) {
        int q[3];
        for (int k = 0; k < 3; ++k) {
            q[k] = (int)floor((x[3 * i + k] - s->lo[k]) / c->h[k]);
            if (q[k] < 0) q[k] = 0;
            if (q[k] >= c->nc[k]) q[k] = c->nc[k] - 1;
        }
        int64_t id = q[0] + (int64_t)c->nc[0] * (q[1] + (int64_t)c->nc[1] * q[2]);
        c->next[i] = c->head[id];
        c->head[id] = i;
    }
    return 0;
}

static void cells_free(orc_cells *c)
{
    free(c->head);
    free(c->next);
}

/* Collect the j (j != i) that could be within r_c of i, in ascending order. */
typedef struct { int64_t *j; int64_t n, cap; } orc_list;

static void list_push(orc_list *l, int64_t j)
{
    if (l->n == l->cap) {
        l->cap = l->cap ? 2 * l->cap : 256;
        l->j = (int64_t *)realloc(l->j, sizeof(int64_t) * (size_t)l->cap);
    }
    l->j[l->n++] = j;
}

static int cmp_i64(const void *a, const void *b)
{
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return (x > y) - (x < y);
}

static void candidates(const orc_sys *s, const orc_cells *c, int64_t n,
                       const double *x, int64_t i, orc_list *out)
{
    out->n = 0;
    if (!s->use_cells) {
        for (int64_t j = 0; j < n; ++j)
            if (j != i) list_push(out, j);
        return;
    }
    int q[3];
    for (int k = 0; k < 3; ++k) {
        q[k] = (int)floor((x[3 * i + k] - s->lo[k]) / c->h[k]);
        if (q[k] < 0) q[k] = 0;
        if (q[k] >= c->nc[k]) q[k] = c->nc[k] - 1;
    }
    for (int oz = -1; oz <= 1; ++oz)
        for (int oy = -1; oy <= 1; ++oy)
            for (int ox = -1; ox <= 1; ++ox) {
                int o[3] = { ox, oy, oz }, p[3], ok = 1;
                for (int k = 0; k < 3; ++k) {
                    p[k] = q[k] + o[k];
                    if (p[k] < 0 || p[k] >= c->nc[k]) {
                        if (!s->periodic[k]) { ok = 0; break; }
                        p[k] = (p[k] + c->nc[k]) % c->nc[k];
                    }
                }
                if (!ok) continue;
                int64_t id = p[0] + (int64_t)c->nc[0] * (p[1] + (int64_t)c->nc[1] * p[2]);
                for (int64_t j = c->head[id]; j >= 0; j = c->next[j])
                    if (j != i) list_push(out, j);
            }
    qsort(out->j, (size_t)out->n, sizeof(int64_t), cmp_i64);
}

/* ------------------------------------------------------------------------ */
/* Local density, Sec. 2.1: rho_i = sum_{j != i, r < r_d} w_rho(r_ij).        */
/* ------------------------------------------------------------------------ */
int orc_density(const orc_sys *s, int64_t n, const double *x, double *rho)
{
    orc_cells c = { { 0, 0, 0 }, { 0, 0, 0 }, NULL, NULL };
    if (s->use_cells && cells_build(s, n, x, &c) != 0) { cells_free(&c); return -1; }
    const double rd2 = s->rd * s->rd;
#pragma omp parallel
    {
        orc_list lst = { NULL, 0, 0 };
#pragma omp for schedule(dynamic, 64)
        for (int64_t i = 0; i < n; ++i) {
            candidates(s, &c, n, x, i, &lst);
            double acc = s->rho_self ? orc_w_rho(0.0, s->rd) : 0.0;
            for (int64_t k = 0; k < lst.n; ++k) {
                int64_t j = lst.j[k];
                double d[3];
                pair_vec(s, &x[3 * i], &x[3 * j], d);
                double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                if (r2 < rd2) acc += orc_w_rho(sqrt(r2), s->rd);
            }
            rho[i] = acc;
        }
        free(lst.j);
    }
    if (s->use_cells) cells_free(&c);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Wall-particle density, Sec. 3.2 and Algorithm 1 (the phi step): for each   */
/* fluid (mobile) particle i, the number density of solid (frozen) particles  */
/* inside its support, phi_i = sum_{j frozen, 0 < r_ij < r_c} w_phi(r_ij),    */
/* with the density weight of Sec. 2.1 normalised over the support radius r_c */
/* instead of r_d: w_phi = 15/(2 pi r_c^3) (1 - r/r_c)^2.  phi_i = 0 for      */
/* frozen i.                                                                  */
/* ------------------------------------------------------------------------ */
int orc_wall_density(const orc_sys *s, int64_t n, const double *x,
                     const int32_t *type, double *phi)
{
    orc_cells c = { { 0, 0, 0 }, { 0, 0, 0 }, NULL, NULL };
    if (s->use_cells && cells_build(s, n, x, &c) != 0) { cells_free(&c); return -1; }
    const double rc2 = s->rc * s->rc;
#pragma omp parallel
    {
        orc_list lst = { NULL, 0, 0 };
#pragma omp for schedule(dynamic, 64)
        for (int64_t i = 0; i < n; ++i) {
            double acc = 0.0;
            if (!is_frozen(s, type[i])) {
                candidates(s, &c, n, x, i, &lst);
                for (int64_t k = 0; k < lst.n; ++k) {
                    int64_t j = lst.j[k];
                    if (!is_frozen(s, type[j])) continue;
                    double d[3];
                    pair_vec(s, &x[3 * i], &x[3 * j], d);
                    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                    if (r2 > 0.0 && r2 < rc2) acc += orc_w_rho(sqrt(r2), s->rc);
                }
            }
            phi[i] = acc;
        }
        free(lst.j);
    }
    if (s->use_cells) cells_free(&c);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Forces, Sec. 2.1 + Eq. 1.  a_i = sum_j F_ij / m + g for mobile i (m = 1),  */
/* a_i = 0 for frozen i.  virial (may be NULL) receives the conservative      */
/* virial tensor 0.5 sum_{i mobile} sum_j d_a F^C_b (xx yy zz xy xz yz).      */
/* ------------------------------------------------------------------------ */
int orc_forces(const orc_sys *s, int64_t n, const double *x, const double *v,
               const int32_t *type, const uint32_t *id, const double *rho,
               uint64_t step, double *a, double *virial)
{
    orc_cells c = { { 0, 0, 0 }, { 0, 0, 0 }, NULL, NULL };
    if (s->use_cells && cells_build(s, n, x, &c) != 0) { cells_free(&c); return -1; }
    double *vir_i = virial ? (double *)calloc((size_t)(n > 0 ? n : 1) * 6, sizeof(double)) : NULL;
#pragma omp parallel
    {
        orc_list lst = { NULL, 0, 0 };
#pragma omp for schedule(dynamic, 64)
        for (int64_t i = 0; i < n; ++i) {
            double F[3] = { 0.0, 0.0, 0.0 }, W[6] = { 0, 0, 0, 0, 0, 0 };
            if (!is_frozen(s, type[i])) {
                candidates(s, &c, n, x, i, &lst);
                for (int64_t k = 0; k < lst.n; ++k) {
                    int64_t j = lst.j[k];
                    double d[3], vij[3], f[3], w[6];
                    pair_vec(s, &x[3 * i], &x[3 * j], d);
                    for (int q = 0; q < 3; ++q) vij[q] = v[3 * i + q] - v[3 * j + q];
                    double xi = orc_xi(s->seed, step, id[i], id[j], s->xi_dist);
                    if (orc_pair_force(s, d, vij, type[i], type[j], rho[i], rho[j],
                                       xi, f, w)) {
                        for (int q = 0; q < 3; ++q) F[q] += f[q];
                        for (int q = 0; q < 6; ++q) W[q] += w[q];
                    }
                }
                for (int q = 0; q < 3; ++q) F[q] += s->g[q];   /* m = 1 */
            }
            for (int q = 0; q < 3; ++q) a[3 * i + q] = F[q];
            if (vir_i) for (int q = 0; q < 6; ++q) vir_i[6 * i + q] = W[q];
        }
        free(lst.j);
    }
    if (virial) {
        for (int q = 0; q < 6; ++q) virial[q] = 0.0;
        for (int64_t i = 0; i < n; ++i)
            for (int q = 0; q < 6; ++q) virial[q] += vir_i[6 * i + q];
        free(vir_i);
    }
    if (s->use_cells) cells_free(&c);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Reflection rule for the no-slip, non-penetrating walls (Sec. 2.2, 3.2):    */
/* a position is blocked if it lies beyond a non-periodic face or inside a   */
/* solid voxel of the pore image.                                              */
/* ------------------------------------------------------------------------ */
int orc_blocked(const orc_sys *s, const double xn[3])
{
    for (int k = 0; k < 3; ++k)
        if (!s->periodic[k] && (xn[k] < s->lo[k] || xn[k] >= s->lo[k] + s->L[k]))
            return 1;
    if (!s->mask) return 0;
    int64_t q[3];
    for (int k = 0; k < 3; ++k) {
        double f = floor((xn[k] - s->morigin[k]) / s->voxel);
        if (f < 0.0 || f >= (double)s->mdim[k]) return 0;
        q[k] = (int64_t)f;
    }
    return s->mask[q[0] + (int64_t)s->mdim[0] * (q[1] + (int64_t)s->mdim[1] * q[2])] != 0;
}

/* Observables of the state (v at a full step, virial of that step's forces): */
/* out[0..2] momentum (m = 1), out[3] kinetic energy, out[4] kT estimate       */
/* 2 KE / (3 (N_mobile - 1)), out[5..10] virial (xx yy zz xy xz yz),           */
/* out[11..13] sum v_a^2, out[14] N_mobile, out[15] step.                      */
void orc_observables(const orc_sys *s, int64_t n, const double *v,
                     const int32_t *type, const double *virial, uint64_t step,
                     double out[16])
{
    for (int q = 0; q < 16; ++q) out[q] = 0.0;
    double nm = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        if (is_frozen(s, type[i])) continue;
        nm += 1.0;
        for (int q = 0; q < 3; ++q) {
            out[q] += v[3 * i + q];
            out[11 + q] += v[3 * i + q] * v[3 * i + q];
        }
    }
    out[3] = 0.5 * (out[11] + out[12] + out[13]);
    out[4] = nm > 1.0 ? 2.0 * out[3] / (3.0 * (nm - 1.0)) : 0.0;
    for (int q = 0; q < 6; ++q) out[5 + q] = virial ? virial[q] : 0.0;
    out[14] = nm;
    out[15] = (double)step;
}

/* ------------------------------------------------------------------------ */
/* Velocity-Verlet, Algorithm 1 without its communication lines.              */
/* On entry a holds a(t) and step the index of the force evaluation that      */
/* produced it.  Each step:                                                    */
/*   v <- v + (dt/2) a ; x' <- x + dt v ; wrap periodic axes ;                 */
/*   if x' is blocked: keep x, v <- -v  (reflection) ; else x <- x' ;          */
/*   step <- step + 1 ; rho <- density(x) ; a <- forces(x, v, rho, step) ;      */
/*   v <- v + (dt/2) a.                                                        */
/* obs_last gets the observables after the last step, obs_sum their sum over  */
/* the steps (both may be NULL).                                               */
/* ------------------------------------------------------------------------ */
int orc_run(const orc_sys *s, int64_t n, double *x, double *v,
            const int32_t *type, const uint32_t *id, double *a, double *rho,
            uint64_t *step, int64_t nsteps, double *obs_last, double *obs_sum)
{
    const double hdt = 0.5 * s->dt;
    double vir[6], obs[16];
    if (obs_sum) for (int q = 0; q < 16; ++q) obs_sum[q] = 0.0;
    for (int64_t it = 0; it < nsteps; ++it) {
        for (int64_t i = 0; i < n; ++i) {
            if (is_frozen(s, type[i])) continue;
            double xn[3];
            for (int k = 0; k < 3; ++k) v[3 * i + k] = v[3 * i + k] + hdt * a[3 * i + k];
            for (int k = 0; k < 3; ++k) {
                xn[k] = x[3 * i + k] + s->dt * v[3 * i + k];
                if (s->periodic[k]) {
                    if (xn[k] >= s->lo[k] + s->L[k]) xn[k] -= s->L[k];
                    else if (xn[k] < s->lo[k]) xn[k] += s->L[k];
                }
            }
            if (orc_blocked(s, xn)) {
                for (int k = 0; k < 3; ++k) v[3 * i + k] = -v[3 * i + k];
            } else {
                for (int k = 0; k < 3; ++k) x[3 * i + k] = xn[k];
            }
        }
        *step += 1;
        if (orc_density(s, n, x, rho) != 0) return -1;
        if (orc_forces(s, n, x, v, type, id, rho, *step, a, vir) != 0) return -1;
        for (int64_t i = 0; i < n; ++i) {
            if (is_frozen(s, type[i])) continue;
            for (int k = 0; k < 3; ++k) v[3 * i + k] = v[3 * i + k] + hdt * a[3 * i + k];
        }
        if (obs_last || obs_sum) {
            orc_observables(s, n, v, type, vir, *step, obs);
            if (obs_last) memcpy(obs_last, obs, sizeof(obs));
            if (obs_sum) for (int q = 0; q < 16; ++q) obs_sum[q] += obs[q];
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Wall-particle packing from a voxel image, Sec. 2.3: one sweep marks the    */
/* solid voxels within `shell` of a pore voxel (centre-to-centre distance in  */
/* voxel units, squared, <= (shell/voxel)^2); a second sweep fills each such  */
/* voxel with particles at number density rho_w.  The paper's locally        */
/* equilibrated database is not published, so each voxel gets                */
/* floor(rho_w voxel^3 + u) particles at uniform random points, u and the     */
/* points drawn from Philox-4x32-10 with key (seed_lo, seed_hi) and counter   */
/* (voxel id, k, 0x57414C4C, 0): k = 0 for the count, k = 1.. for particle    */
/* k-1's three coordinates.  Particles are listed by ascending voxel id, then */
/* k.  Returns the count (positions beyond cap are not written); shell_out    */
/* (optional) receives 1 for each shell voxel.                                */
/* ------------------------------------------------------------------------ */
int64_t orc_place_walls(const uint8_t *mask, const int32_t dim[3],
                        const int32_t periodic[3], double voxel,
                        const double origin[3], double rho_w, double shell,
                        uint64_t seed, double *out, int64_t cap,
                        uint8_t *shell_out)
{
    const uint32_t TAG = 0x57414C4Cu;
    const uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    const int nx = dim[0], ny = dim[1], nz = dim[2];
    const double rr = shell / voxel;
    const int R = (int)floor(rr + 1e-9);
    const int64_t R2 = (int64_t)floor(rr * rr + 1e-9);
    const double lam = rho_w * voxel * voxel * voxel;
    int64_t count = 0;
    for (int iz = 0; iz < nz; ++iz)
        for (int iy = 0; iy < ny; ++iy)
            for (int ix = 0; ix < nx; ++ix) {
                int64_t vid = ix + (int64_t)nx * (iy + (int64_t)ny * iz);
                int in_shell = 0;
                if (mask[vid]) {
                    for (int dz = -R; dz <= R && !in_shell; ++dz)
                        for (int dy = -R; dy <= R && !in_shell; ++dy)
                            for (int dx = -R; dx <= R && !in_shell; ++dx) {
                                if ((int64_t)dx * dx + (int64_t)dy * dy + (int64_t)dz * dz > R2)
                                    continue;
                                int p[3] = { ix + dx, iy + dy, iz + dz };
                                const int m[3] = { nx, ny, nz };
                                int ok = 1;
                                for (int k = 0; k < 3; ++k) {
                                    if (p[k] < 0 || p[k] >= m[k]) {
                                        if (!periodic[k]) { ok = 0; break; }
                                        p[k] = (p[k] % m[k] + m[k]) % m[k];
                                    }
                                }
                                if (!ok) continue;
                                if (!mask[p[0] + (int64_t)nx * (p[1] + (int64_t)ny * p[2])])
                                    in_shell = 1;
                            }
                }
                if (shell_out) shell_out[vid] = (uint8_t)in_shell;
                if (!in_shell) continue;
                uint32_t w[4];
                uint32_t c0[4] = { (uint32_t)vid, 0u, TAG, 0u };
                orc_philox4x32_10(c0, key, w);
                double u = ((double)w[0] + 0.5) * (1.0 / 4294967296.0);
                int64_t nv = (int64_t)floor(lam + u);
                for (int64_t k = 0; k < nv; ++k) {
                    uint32_t ck[4] = { (uint32_t)vid, (uint32_t)(k + 1), TAG, 0u };
                    orc_philox4x32_10(ck, key, w);
                    if (count < cap && out) {
                        const int iq[3] = { ix, iy, iz };
                        for (int q = 0; q < 3; ++q) {
                            double uq = ((double)w[q] + 0.5) * (1.0 / 4294967296.0);
                            out[3 * count + q] = origin[q] + ((double)iq[q] + uq) * voxel;
                        }
                    }
                    ++count;
                }
            }
    return count;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads used by later calls (n >= 1); the sums are gather-only, so results */
/* do not depend on it.                                                        */
void orc_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* Forces on a subset of particles (indices idx[0..m-1]) of the whole system,  */
/* with rho given for every particle; same definition as orc_forces.          */
int orc_forces_subset(const orc_sys *s, int64_t n, const double *x, const double *v,
                      const int32_t *type, const uint32_t *id, const double *rho,
                      uint64_t step, int64_t m, const int64_t *idx, double *a)
{
    orc_cells c = { { 0, 0, 0 }, { 0, 0, 0 }, NULL, NULL };
    if (s->use_cells && cells_build(s, n, x, &c) != 0) { cells_free(&c); return -1; }
#pragma omp parallel
    {
        orc_list lst = { NULL, 0, 0 };
#pragma omp for schedule(dynamic, 16)
        for (int64_t q = 0; q < m; ++q) {
            const int64_t i = idx[q];
            double F[3] = { 0.0, 0.0, 0.0 };
            if (!is_frozen(s, type[i])) {
                candidates(s, &c, n, x, i, &lst);
                for (int64_t k = 0; k < lst.n; ++k) {
                    int64_t j = lst.j[k];
                    double d[3], vij[3], f[3];
                    pair_vec(s, &x[3 * i], &x[3 * j], d);
                    for (int r = 0; r < 3; ++r) vij[r] = v[3 * i + r] - v[3 * j + r];
                    double xi = orc_xi(s->seed, step, id[i], id[j], s->xi_dist);
                    if (orc_pair_force(s, d, vij, type[i], type[j], rho[i], rho[j], xi, f, NULL))
                        for (int r = 0; r < 3; ++r) F[r] += f[r];
                }
                for (int r = 0; r < 3; ++r) F[r] += s->g[r];
            }
            for (int r = 0; r < 3; ++r) a[3 * q + r] = F[r];
        }
        free(lst.j);
    }
    if (s->use_cells) cells_free(&c);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Vector-Jacobian product of one evaluation.                                */
/* The evaluation maps (x, u, theta) to the accelerations a_i = sum_j f_ij of */
/* mobile i (Sec. 2.1, Eq. 1), to the conservative virial                     */
/* W_ab = 1/2 sum_{i mobile} sum_j d_a F^C_b (the pressure tensor of Sec.     */
/* 4.1) and to the local densities rho_i = sum_j w_rho(r_ij) (Sec. 2.1), with */
/* u the velocities the dissipative term sees.  Given abar (3n), cvir (the    */
/* six weights of W in the order xx yy zz xy xz yz) and rhobar (n), each may   */
/* be NULL for zero, it returns the gradient of                               */
/*   L = sum_i abar_i . a_i + sum_k cvir_k W_k + sum_i rhobar_i rho_i         */
/* with respect to x (xbar), u (ubar) and the symmetric parameters A, B,      */
/* gamma (tbar[3][8][8], entry [a][b] = [b][a] = dL/dP_ab).  The random       */
/* draws xi_ij of the given step are held fixed.  Written from the chain rule */
/* on each ordered pair (i mobile, j): with d = x_i - x_j, r = |d|, e = d/r,  */
/* w = e.u_ij and f_ij = s e,                                                  */
/*   s = A wc + B (rho_i + rho_j) wd [r < r_d] - gamma wc^2 w                  */
/*       + sigma wc xi / sqrt(dt),                                             */
/*   d(abar_i.f_ij)/dd = (abar_i.e)(s_r e + s_w (u_ij - w e)/r)               */
/*                       + s (abar_i - (abar_i.e) e)/r,                        */
/* s_r the r-derivative of s at fixed w and rho, s_w = -gamma wc^2; the       */
/* virial term of the pair, 1/2 (s_c / r) Q(d) with s_c = A wc + B (rho_i +   */
/* rho_j) wd and Q(d) = sum_k cvir_k d_a d_b, has the d-gradient              */
/*   1/2 [ (Q/r) s_c' e + s_c (grad Q / r - Q d / r^3) ];                      */
/* then the density chain rho_bar_k = dL/drho_k sent back through w_rho'(r) e.*/
/* ------------------------------------------------------------------------ */
int orc_eval_vjp(const orc_sys *s, int64_t n, const double *x, const double *u,
                 const int32_t *type, const uint32_t *id, uint64_t step,
                 const double *abar, const double *cvir, const double *rhobar,
                 double *xbar, double *ubar, double *tbar);

int orc_force_vjp(const orc_sys *s, int64_t n, const double *x, const double *u,
                  const int32_t *type, const uint32_t *id, uint64_t step,
                  const double *abar, double *xbar, double *ubar, double *tbar)
{
    return orc_eval_vjp(s, n, x, u, type, id, step, abar, NULL, NULL, xbar, ubar, tbar);
}

int orc_eval_vjp(const orc_sys *s, int64_t n, const double *x, const double *u,
                 const int32_t *type, const uint32_t *id, uint64_t step,
                 const double *abar, const double *cvir, const double *rhobar,
                 double *xbar, double *ubar, double *tbar)
{
    double *rho = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *rbar = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    if (!rho || !rbar) { free(rho); free(rbar); return -2; }
    if (orc_density(s, n, x, rho) != 0) { free(rho); free(rbar); return -1; }
    for (int64_t k = 0; k < 3 * n; ++k) { xbar[k] = 0.0; ubar[k] = 0.0; }
    for (int k = 0; k < 3 * ORC_MAXT * ORC_MAXT; ++k) tbar[k] = 0.0;
    if (rhobar) for (int64_t k = 0; k < n; ++k) rbar[k] = rhobar[k];
    const double rc = s->rc, rd = s->rd;
    const double sq_dt = sqrt(s->dt);
    const double pi = 3.14159265358979323846264338327950288;
    const double cw = 15.0 / (2.0 * pi * rd * rd * rd);
    /* force part (serial, plain) */
    for (int64_t i = 0; i < n; ++i) {
        if (is_frozen(s, type[i])) continue;
        const double zero3[3] = { 0.0, 0.0, 0.0 };
        const double *ab = abar ? &abar[3 * i] : zero3;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double d[3];
            pair_vec(s, &x[3 * i], &x[3 * j], d);
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (!(r2 < rc * rc) || !(r2 > 0.0)) continue;
            const int32_t ti = type[i], tj = type[j];
            double r = sqrt(r2), e[3], uij[3];
            for (int k = 0; k < 3; ++k) { e[k] = d[k] / r; uij[k] = u[3 * i + k] - u[3 * j + k]; }
            double w = e[0] * uij[0] + e[1] * uij[1] + e[2] * uij[2];
            double wc = 1.0 - r / rc;
            double A = s->A[ti][tj], B = s->B[ti][tj], g = s->gamma[ti][tj];
            double sig = sqrt(2.0 * g * s->kT);
            double xi = orc_xi(s->seed, step, id[i], id[j], s->xi_dist);
            int near = r < rd;
            double wd = near ? 1.0 - r / rd : 0.0;
            double sval = A * wc + B * (rho[i] + rho[j]) * wd - g * wc * wc * w + sig * wc * xi / sq_dt;
            double s_r = -A / rc - (near ? B * (rho[i] + rho[j]) / rd : 0.0)
                         + 2.0 * g * wc * w / rc - sig * xi / (sq_dt * rc);
            double s_w = -g * wc * wc;
            double ae = ab[0] * e[0] + ab[1] * e[1] + ab[2] * e[2];
            for (int k = 0; k < 3; ++k) {
                double gd = ae * (s_r * e[k] + s_w * (uij[k] - w * e[k]) / r)
                            + sval * (ab[k] - ae * e[k]) / r;
                xbar[3 * i + k] += gd;
                xbar[3 * j + k] -= gd;
                double gu = ae * s_w * e[k];
                ubar[3 * i + k] += gu;
                ubar[3 * j + k] -= gu;
            }
            if (near) {
                rbar[i] += ae * B * wd;
                rbar[j] += ae * B * wd;
            }
            int a = ti < tj ? ti : tj, b = ti < tj ? tj : ti;
            double dsig = g > 0.0 ? s->kT / sig : 0.0;
            double gA = ae * wc, gB = ae * (rho[i] + rho[j]) * wd;
            double gG = ae * (-wc * wc * w + dsig * wc * xi / sq_dt);
            tbar[0 * 64 + a * 8 + b] += gA;
            tbar[1 * 64 + a * 8 + b] += gB;
            tbar[2 * 64 + a * 8 + b] += gG;
            if (cvir) {
                /* virial term 1/2 (s_c / r) Q(d) of this ordered pair */
                double Q = cvir[0] * d[0] * d[0] + cvir[1] * d[1] * d[1] + cvir[2] * d[2] * d[2]
                           + cvir[3] * d[0] * d[1] + cvir[4] * d[0] * d[2] + cvir[5] * d[1] * d[2];
                double gQ[3] = { 2.0 * cvir[0] * d[0] + cvir[3] * d[1] + cvir[4] * d[2],
                                 2.0 * cvir[1] * d[1] + cvir[3] * d[0] + cvir[5] * d[2],
                                 2.0 * cvir[2] * d[2] + cvir[4] * d[0] + cvir[5] * d[1] };
                double sc = A * wc + B * (rho[i] + rho[j]) * wd;
                double sc_r = -A / rc - (near ? B * (rho[i] + rho[j]) / rd : 0.0);
                for (int k = 0; k < 3; ++k) {
                    double gd = 0.5 * ((Q / r) * sc_r * e[k] + sc * (gQ[k] / r - Q * d[k] / (r2 * r)));
                    xbar[3 * i + k] += gd;
                    xbar[3 * j + k] -= gd;
                }
                if (near) {
                    rbar[i] += 0.5 * (Q / r) * B * wd;
                    rbar[j] += 0.5 * (Q / r) * B * wd;
                }
                tbar[0 * 64 + a * 8 + b] += 0.5 * (Q / r) * wc;
                tbar[1 * 64 + a * 8 + b] += 0.5 * (Q / r) * (rho[i] + rho[j]) * wd;
            }
        }
    }
    /* density part: rho_k = sum_m w_rho(r_km) */
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double d[3];
            pair_vec(s, &x[3 * i], &x[3 * j], d);
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (!(r2 < rd * rd) || !(r2 > 0.0)) continue;
            double r = sqrt(r2);
            double dw = -2.0 * cw * (1.0 - r / rd) / rd;      /* w_rho'(r) */
            for (int k = 0; k < 3; ++k) {
                double gk = rbar[i] * dw * d[k] / r;          /* d rho_i / d x_i */
                xbar[3 * i + k] += gk;
                xbar[3 * j + k] -= gk;
            }
        }
    }
    for (int q = 0; q < 3; ++q)
        for (int a = 0; a < 8; ++a)
            for (int b = a + 1; b < 8; ++b) tbar[q * 64 + b * 8 + a] = tbar[q * 64 + a * 8 + b];
    free(rho);
    free(rbar);
    return 0;
}
