/*
 * at_oracle.c -- plain FP64 CPU oracle for the weakly-synchronous AT method.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * execute this file; only the tests, the smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code, header, table or constant
 * generator with the CUDA library: the two are checked against each other.
 *
 * What it computes (arXiv 1911.05769):
 *   - viscous Burgers' equation u_t + u u_x = nu u_xx (Eq. BS, one velocity
 *     component, one dimension), optionally with a time-independent forcing
 *     F(x) = A sin(x), or the linear advection-diffusion equation
 *     u_t + c u_x = nu u_xx used for the accuracy demonstration of Fig. 2;
 *   - forward-Euler time integration (Sec. 3.2);
 *   - standard central differences at interior points I_i (Sec. 3.2);
 *   - asynchrony-tolerant (AT) differences at process-boundary points I_b,
 *     Eq. AT1 / Eq. AT2, in the "split" form of Sec. 5.2: every halo value is
 *     first approximated from the delayed levels n-k, n-k-1 (the
 *     "approximate" step of Algorithm 2), then the unchanged central stencil
 *     is applied;
 *   - delays k <= L per (time level n, subdomain p, face), prescribed by a
 *     counter-based generator (SplitMix64), replayed from an array, or zero
 *     (the synchronous algorithm, Algorithm 1).
 *
 * The domain [x0, x0 + N dx) is split into P subdomains of M = N/P points.
 * Readings of the paper used here (the paper is silent or ambiguous):
 *   - k ranges over {0..L}: Algorithm 2 lets the receive time lag the send
 *     time by L (Sec. 2 writes n-L+1 as the oldest level; Alg. 2 allows n-L).
 *   - Start-up: k is clamped to n-s+1 so that no level below 0 is read; this
 *     is the "synchronize during initialisation" branch of Algorithm 2.
 *   - 4th order: the paper gives only the 2nd-order AT formulas; the 4th-order
 *     variant extrapolates each delayed halo value quadratically in time from
 *     three levels (a wider stencil in time, Sec. 2) and then applies the
 *     standard 4th-order central stencil.
 *   - Delays are drawn independently per face (one message per face per step,
 *     Sec. 5.1); the per_subdomain flag uses one draw for both faces.
 *
 * Everything is FP64, evaluated in the written order; compile with
 * -O2 -ffp-contract=off and no fast-math.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EARG (-1)
#define ORC_ENOMEM (-2)
#define ORC_EDELAY (-3)

/* ------------------------------------------------------------------------ */
/* Counter-based generator for prescribed delays.                           */
/* SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number    */
/* generators", OOPSLA 2014): state advances by the golden-ratio increment  */
/* and each state is passed through the 64-bit finaliser with shift/multiply */
/* constants (30, 0xBF58476D1CE4E5B9), (27, 0x94D049BB133111EB), 31.         */
/* at_oracle_splitmix64(seed, i) is the i-th (0-based) output of the        */
/* sequence started from state `seed`.                                       */
/* ------------------------------------------------------------------------ */
uint64_t at_oracle_splitmix64(uint64_t seed, uint64_t i)
{
    uint64_t z = seed + (i + 1u) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Raw prescribed delay in {0..L} for (level n, subdomain p, face f) of a
 * decomposition into P subdomains with F faces each: the generator output at
 * counter (n*P + p)*F + f, upper 32 bits mapped to {0..L} by multiply-shift. */
int at_oracle_seeded_delay(uint64_t seed, int64_t n, int64_t p, int64_t P,
                           int face, int F, int L)
{
    uint64_t ctr = ((uint64_t)n * (uint64_t)P + (uint64_t)p) * (uint64_t)F
                   + (uint64_t)face;
    uint64_t h = at_oracle_splitmix64(seed, ctr) >> 32;
    return (int)((h * (uint64_t)(L + 1)) >> 32);
}

/* ------------------------------------------------------------------------ */
/* Halo approximation weights (Eq. AT1 / AT2; split form, Sec. 5.2).        */
/* The value at level n is extrapolated from the s levels n-k, ..., n-k-s+1 */
/* by the Lagrange polynomial through times -k-m (m = 0..s-1) evaluated at  */
/* time 0:  w_m = prod_{j != m} (0 - t_j) / (t_m - t_j),  t_j = -k-j.       */
/* For s = 2 this gives w = (k+1, -k), the coefficients of Eq. AT1 / AT2.   */
/* With at_weights == 0 the delayed value is used as is, w = (1, 0, ...):   */
/* the "standard schemes under asynchrony" configuration of Fig. 2.         */
/* ------------------------------------------------------------------------ */
int at_oracle_weights(int s, int k, int at_weights, double *w)
{
    if (s < 1 || s > 8 || k < 0) return ORC_EARG;
    for (int m = 0; m < s; ++m) {
        if (!at_weights) { w[m] = (m == 0) ? 1.0 : 0.0; continue; }
        double num = 1.0, den = 1.0;
        for (int j = 0; j < s; ++j) {
            if (j == m) continue;
            double tj = (double)(-k - j), tm = (double)(-k - m);
            num *= (0.0 - tj);
            den *= (tm - tj);
        }
        w[m] = num / den;
    }
    return ORC_OK;
}

/* Approximate one halo value from its delayed levels lev[m] = f^{n-k-m}.   */
/* Terms with a zero weight are skipped, so that k = 0 returns lev[0]       */
/* exactly (Sec. 3.2: for k = 0 the AT schemes are the standard schemes).   */
double at_oracle_extrapolate(int s, int k, int at_weights, const double *lev)
{
    double w[8];
    at_oracle_weights(s, k, at_weights, w);
    double acc = 0.0;
    for (int m = 0; m < s; ++m)
        if (w[m] != 0.0) acc += w[m] * lev[m];
    return acc;
}

/* Central differences of order 2 or 4 at the middle of v[0..2R]
 * (v[R] is the point itself).  Sec. 3.2 (order 2); order 4 is the standard
 * five-point formula. */
int at_oracle_derivs(int order, const double *v, double dx, double *d1, double *d2)
{
    if (order == 2) {
        const double *c = v + 1;
        *d1 = (c[1] - c[-1]) / (2.0 * dx);
        *d2 = (c[1] - 2.0 * c[0] + c[-1]) / (dx * dx);
        return ORC_OK;
    }
    if (order == 4) {
        const double *c = v + 2;
        *d1 = (-c[2] + 8.0 * c[1] - 8.0 * c[-1] + c[-2]) / (12.0 * dx);
        *d2 = (-c[2] + 16.0 * c[1] - 30.0 * c[0] + 16.0 * c[-1] - c[-2])
              / (12.0 * dx * dx);
        return ORC_OK;
    }
    return ORC_EARG;
}

/* ------------------------------------------------------------------------ */
/* One run of the method.                                                    */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t N;          /* grid points of the whole domain                   */
    int64_t P;          /* subdomains of the whole domain                    */
    int64_t p_lo;       /* first simulated subdomain (window), 0 = all       */
    int64_t p_count;    /* simulated subdomains; the window wraps around     */
    int32_t order;      /* 2 or 4                                            */
    int32_t L;          /* maximal allowable delay                           */
    double nu, dt;      /* viscosity, time step                              */
    double x0, dx;      /* x_i = x0 + i dx                                   */
    double forcing_amp; /* F(x) = A sin(x)                                   */
    int32_t eq;         /* 0: Burgers, 1: linear advection-diffusion         */
    int32_t bc;         /* 0: periodic, 1: exact tanh travelling wave ghosts */
    double adv_c;       /* advection speed of the linear equation            */
    double tanh_a, tanh_c, tanh_xc; /* u = c - a tanh(a (x - xc - c t)/(2 nu)) */
    int32_t delay_mode; /* 0: synchronous, 1: seeded, 2: replay              */
    int32_t per_subdomain; /* one delay draw for both faces                  */
    int32_t at_weights;    /* 1: AT extrapolation, 0: standard (negative ctl) */
    int32_t pad_;
    uint64_t seed;
} at_oracle_cfg;

static int64_t wrap(int64_t a, int64_t b) { int64_t r = a % b; return r < 0 ? r + b : r; }

static double tanh_wave(const at_oracle_cfg *c, double x, double t)
{
    return c->tanh_c - c->tanh_a * tanh(c->tanh_a * (x - c->tanh_xc - c->tanh_c * t) / (2.0 * c->nu));
}

/* Runs n_steps forward-Euler steps from level 0.
 *   u0     [p_count*M]   initial field of the window (level 0)
 *   u_out  [p_count*M]   field at level n_steps
 *   replay [n_steps][p_count][2]   delays for delay_mode 2 (else ignored)
 *   hist   [L+1]         counts of the delays used (after the start-up clamp)
 *   k_used [n_steps][p_count][2]   delays used (may be NULL)
 * The window p_lo .. p_lo+p_count-1 is taken modulo P (it may run past the
 * last subdomain).  When it is smaller than the domain its two ends are glued
 * together; values within n_steps*R points of its ends are then meaningless,
 * the rest exact. */
int at_oracle_run(const at_oracle_cfg *c, int64_t n_steps, const int8_t *replay,
                  const double *u0, double *u_out, int64_t *hist, int8_t *k_used)
{
    if (!c || c->N <= 0 || c->P <= 0 || c->N % c->P != 0) return ORC_EARG;
    if (c->order != 2 && c->order != 4) return ORC_EARG;
    if (c->L < 0 || c->L > 64 || n_steps < 0) return ORC_EARG;
    if (c->p_count <= 0 || c->p_lo < 0 || c->p_lo >= c->P || c->p_count > c->P) return ORC_EARG;
    const int64_t M = c->N / c->P;
    const int R = c->order / 2;        /* stencil radius                     */
    const int s = c->order / 2 + 1;    /* time levels per halo approximation */
    if (M < 2 * R) return ORC_EARG;
    if (c->bc == 1 && (c->p_lo != 0 || c->p_count != c->P)) return ORC_EARG;
    const int64_t W = c->p_count * M;  /* points simulated                   */
    const int depth = c->L + s + 1;    /* levels n-L-s+1 .. n+1              */

    double *H = (double *)calloc((size_t)depth * (size_t)W, sizeof(double));
    if (!H) return ORC_ENOMEM;
    memcpy(H, u0, (size_t)W * sizeof(double));
    if (hist) memset(hist, 0, (size_t)(c->L + 1) * sizeof(int64_t));

    int *K = (int *)malloc((size_t)c->p_count * 2 * sizeof(int));
    if (!K) { free(H); return ORC_ENOMEM; }
    for (int64_t n = 0; n < n_steps; ++n) {
        const double *cur = H + (size_t)(n % depth) * W;
        double *nxt = H + (size_t)((n + 1) % depth) * W;
        const double tn = (double)n * c->dt;
        /* delays of the two faces of every subdomain at this level
         * (0: left neighbour p-1, 1: right p+1) */
        for (int64_t pl = 0; pl < c->p_count; ++pl) {
            const int64_t pg = (c->p_lo + pl) % c->P;   /* windows wrap */
            for (int f = 0; f < 2; ++f) {
                int kr = 0;
                if (c->delay_mode == 1)
                    kr = at_oracle_seeded_delay(c->seed, n, pg, c->P,
                                                c->per_subdomain ? 0 : f, 2, c->L);
                else if (c->delay_mode == 2)
                    kr = replay[((size_t)n * c->p_count + pl) * 2 + f];
                if (kr < 0 || kr > c->L) { free(H); free(K); return ORC_EDELAY; }
                /* start-up: never read a level below 0 */
                int64_t kmax = n - s + 1; if (kmax < 0) kmax = 0;
                K[pl * 2 + f] = (kr < kmax) ? kr : (int)kmax;
                if (hist) hist[K[pl * 2 + f]] += 1;
                if (k_used) k_used[((size_t)n * c->p_count + pl) * 2 + f] = (int8_t)K[pl * 2 + f];
            }
        }
        /* the points of every subdomain (independent of one another: the
         * subdomains may be taken by several threads, each point's arithmetic
         * is the same whatever the thread count) */
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
        for (int64_t pl = 0; pl < c->p_count; ++pl) {
            const int64_t pg = (c->p_lo + pl) % c->P;
            const int *k = K + pl * 2;
            double v[5], lev[4];
            for (int64_t m = 0; m < M; ++m) {
                const int64_t il = pl * M + m;   /* index in the window */
                const int64_t ig = pg * M + m;   /* index in the domain */
                for (int j = -R; j <= R; ++j) {
                    const int64_t mj = m + j;
                    if (mj >= 0 && mj < M) {     /* same subdomain: level n  */
                        v[j + R] = cur[il + j];
                        continue;
                    }
                    const int64_t gj = ig + j;
                    if (c->bc == 1 && (gj < 0 || gj >= c->N)) {
                        /* domain boundary: exact ghost value, undelayed */
                        v[j + R] = tanh_wave(c, c->x0 + (double)gj * c->dx, tn);
                        continue;
                    }
                    /* halo point across face f, approximated from n-k-m */
                    const int f = (mj < 0) ? 0 : 1;
                    const int64_t src = wrap(il + j, W);
                    for (int q = 0; q < s; ++q) {
                        const int64_t lv = n - k[f] - q;
                        lev[q] = (lv >= 0) ? H[(size_t)(lv % depth) * W + src] : 0.0;
                    }
                    v[j + R] = at_oracle_extrapolate(s, k[f], c->at_weights, lev);
                }
                double d1, d2;
                at_oracle_derivs(c->order, v, c->dx, &d1, &d2);
                const double a = (c->eq == 0) ? v[R] : c->adv_c;
                double rhs = -a * d1 + c->nu * d2;
                if (c->forcing_amp != 0.0)
                    rhs += c->forcing_amp * sin(c->x0 + (double)ig * c->dx);
                nxt[il] = cur[il] + c->dt * rhs;
            }
        }
    }
    free(K);
    memcpy(u_out, H + (size_t)(n_steps % depth) * W, (size_t)W * sizeof(double));
    free(H);
    return ORC_OK;
}

/* Threads the point loops of the runs use (OpenMP over subdomains / planes;
 * every point's arithmetic is the same whatever the count, so results do not
 * depend on it).  n <= 0 leaves the setting alone.  Returns the count now in
 * force (1 when the oracle was built without OpenMP). */
int at_oracle_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* Size of the configuration struct, so the caller can check its layout. */
int64_t at_oracle_cfg_size(void) { return (int64_t)sizeof(at_oracle_cfg); }

/* ------------------------------------------------------------------------ */
/* Discrete adjoint of the method (reverse-mode differentiation of the run  */
/* above, for Burgers' equation on the whole periodic domain).              */
/*                                                                          */
/* The run maps (u^0, nu) to u^{n_steps}.  For a scalar J that depends on   */
/* the run only through u^{n_steps}, given lam_T = dJ/du^{n_steps} this      */
/* returns lam_0 = dJ/du^0 and dJ/dnu.  It stores every level, then walks    */
/* the levels backwards.  Each update                                       */
/*     u^{n+1}_i = u^n_i + dt (-v_0 D1(v) + nu D2(v) + F(x_i))              */
/* (Sec. 3.2, Eq. BS) reads stencil values v_j, each a stored value: the    */
/* point itself or a neighbour at level n, or across a subdomain face the   */
/* extrapolation sum_m w_m(k) f^{n-k-m} of Eq. AT1/AT2 over delayed levels.  */
/* The derivative of the update with respect to v_j,                         */
/*     dt (-v_0 dD1/dv_j + nu dD2/dv_j) - dt D1 [j = 0],                     */
/* times lam^{n+1}_i, is added to the adjoint of every stored value v_j is   */
/* made of (weight w_m(k) for a delayed level); the identity term adds      */
/* lam^{n+1}_i to lam^n_i; dJ/dnu collects dt D2(v) lam^{n+1}_i.             */
/* Contributions reach levels n, n-1, ..., so lam^n is complete once every  */
/* update above level n has been processed.                                  */
/* ------------------------------------------------------------------------ */

/* Coefficients of D1 (times dx) and D2 (times dx^2) at offsets -R..R. */
static void deriv_coeffs(int order, double *a1, double *a2)
{
    if (order == 2) {
        a1[0] = -0.5; a1[1] = 0.0; a1[2] = 0.5;
        a2[0] = 1.0; a2[1] = -2.0; a2[2] = 1.0;
    } else {
        a1[0] = 1.0 / 12.0; a1[1] = -8.0 / 12.0; a1[2] = 0.0; a1[3] = 8.0 / 12.0; a1[4] = -1.0 / 12.0;
        a2[0] = -1.0 / 12.0; a2[1] = 16.0 / 12.0; a2[2] = -30.0 / 12.0; a2[3] = 16.0 / 12.0; a2[4] = -1.0 / 12.0;
    }
}

/* Stencil value j (offset -R..R) of point il at level n, as a combination of
 * stored values: levels lv[q], indices ix[q], weights wt[q], q < *cnt. */
static void stencil_sources(const at_oracle_cfg *c, int64_t M, int R, int s, int64_t n, int64_t il,
                            const int k[2], int j, int64_t *lv, int64_t *ix, double *wt, int *cnt)
{
    const int64_t m = il % M;
    const int64_t mj = m + j;
    *cnt = 0;
    if (mj >= 0 && mj < M) {
        lv[0] = n; ix[0] = il + j; wt[0] = 1.0; *cnt = 1;
        return;
    }
    const int f = (mj < 0) ? 0 : 1;
    const int64_t src = wrap(il + j, c->N);
    double w[8];
    at_oracle_weights(s, k[f], c->at_weights, w);
    (void)R;
    for (int q = 0; q < s; ++q) {
        if (w[q] == 0.0) continue;
        lv[*cnt] = n - k[f] - q; ix[*cnt] = src; wt[*cnt] = w[q]; ++*cnt;
    }
}

int at_oracle_adjoint(const at_oracle_cfg *c, int64_t n_steps, const int8_t *replay, const double *u0,
                      const double *lam_T, double *u_T, double *lam_0, double *dnu)
{
    if (!c || c->N <= 0 || c->P <= 0 || c->N % c->P != 0) return ORC_EARG;
    if (c->order != 2 && c->order != 4) return ORC_EARG;
    if (c->L < 0 || c->L > 64 || n_steps < 0) return ORC_EARG;
    if (c->eq != 0 || c->bc != 0 || c->p_lo != 0 || c->p_count != c->P) return ORC_EARG;
    const int64_t N = c->N, M = c->N / c->P;
    const int R = c->order / 2, s = c->order / 2 + 1;
    if (M < 2 * R) return ORC_EARG;
    const size_t lvls = (size_t)n_steps + 1;
    double *U = (double *)malloc(lvls * (size_t)N * sizeof(double));
    double *G = (double *)calloc(lvls * (size_t)N, sizeof(double));
    int8_t *K = (int8_t *)malloc(((size_t)n_steps * (size_t)c->P * 2 + 1) * sizeof(int8_t));
    if (!U || !G || !K) { free(U); free(G); free(K); return ORC_ENOMEM; }
    double a1[5], a2[5], v[5], wt[3];
    int64_t lv[3], ix[3];
    int cnt;
    deriv_coeffs(c->order, a1, a2);

    /* forward: every level, every delay */
    memcpy(U, u0, (size_t)N * sizeof(double));
    for (int64_t n = 0; n < n_steps; ++n) {
        for (int64_t p = 0; p < c->P; ++p) {
            for (int f = 0; f < 2; ++f) {
                int kr = 0;
                if (c->delay_mode == 1)
                    kr = at_oracle_seeded_delay(c->seed, n, p, c->P, c->per_subdomain ? 0 : f, 2, c->L);
                else if (c->delay_mode == 2)
                    kr = replay[((size_t)n * c->P + p) * 2 + f];
                if (kr < 0 || kr > c->L) { free(U); free(G); free(K); return ORC_EDELAY; }
                int64_t kmax = n - s + 1; if (kmax < 0) kmax = 0;
                K[((size_t)n * c->P + p) * 2 + f] = (int8_t)((kr < kmax) ? kr : kmax);
            }
        }
        for (int64_t i = 0; i < N; ++i) {
            const int64_t p = i / M;
            const int k[2] = {K[((size_t)n * c->P + p) * 2], K[((size_t)n * c->P + p) * 2 + 1]};
            for (int j = -R; j <= R; ++j) {
                stencil_sources(c, M, R, s, n, i, k, j, lv, ix, wt, &cnt);
                double acc = 0.0;
                for (int q = 0; q < cnt; ++q) acc += wt[q] * U[(size_t)lv[q] * N + ix[q]];
                v[j + R] = acc;
            }
            double d1, d2;
            at_oracle_derivs(c->order, v, c->dx, &d1, &d2);
            double rhs = -v[R] * d1 + c->nu * d2;
            if (c->forcing_amp != 0.0) rhs += c->forcing_amp * sin(c->x0 + (double)i * c->dx);
            U[(size_t)(n + 1) * N + i] = U[(size_t)n * N + i] + c->dt * rhs;
        }
    }
    if (u_T) memcpy(u_T, U + (size_t)n_steps * N, (size_t)N * sizeof(double));

    /* backward */
    memcpy(G + (size_t)n_steps * N, lam_T, (size_t)N * sizeof(double));
    double gnu = 0.0;
    for (int64_t n = n_steps - 1; n >= 0; --n) {
        for (int64_t i = 0; i < N; ++i) {
            const double g = G[(size_t)(n + 1) * N + i];
            const int64_t p = i / M;
            const int k[2] = {K[((size_t)n * c->P + p) * 2], K[((size_t)n * c->P + p) * 2 + 1]};
            for (int j = -R; j <= R; ++j) {
                stencil_sources(c, M, R, s, n, i, k, j, lv, ix, wt, &cnt);
                double acc = 0.0;
                for (int q = 0; q < cnt; ++q) acc += wt[q] * U[(size_t)lv[q] * N + ix[q]];
                v[j + R] = acc;
            }
            double d1, d2;
            at_oracle_derivs(c->order, v, c->dx, &d1, &d2);
            G[(size_t)n * N + i] += g;                       /* u^n_i itself */
            gnu += g * c->dt * d2;
            for (int j = -R; j <= R; ++j) {
                double dv = c->dt * (-v[R] * a1[j + R] / c->dx + c->nu * a2[j + R] / (c->dx * c->dx));
                if (j == 0) dv -= c->dt * d1;
                stencil_sources(c, M, R, s, n, i, k, j, lv, ix, wt, &cnt);
                for (int q = 0; q < cnt; ++q) G[(size_t)lv[q] * N + ix[q]] += g * dv * wt[q];
            }
        }
    }
    memcpy(lam_0, G, (size_t)N * sizeof(double));
    if (dnu) *dnu = gnu;
    free(U); free(G); free(K);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Three dimensions: u_t + u (u_x + u_y + u_z) = nu (u_xx + u_yy + u_zz)    */
/* (the scalar 3D form of Eq. BS), periodic box of n0 x n1 x n2 points      */
/* (index (k n1 + j) n0 + i, x fastest), split into P0 x P1 x P2 subdomains  */
/* of m0 x m1 x m2 points; subdomain index (p2 P1 + p1) P0 + p0.  Order-2    */
/* central differences along each axis (Sec. 3.2); a stencil point across   */
/* one of the six faces (0: -x, 1: +x, 2: -y, 3: +y, 4: -z, 5: +z) takes the */
/* neighbour's value extrapolated from levels n-k, n-k-1 with that face's   */
/* delay (Eq. AT1/AT2, split form).  Delays per (level, subdomain, face):    */
/* seeded with counter (n P + p) 6 + face, replayed, or zero.                */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t n[3];       /* points per axis                                    */
    int64_t P[3];       /* subdomains per axis                                */
    int32_t L;          /* maximal delay                                      */
    int32_t delay_mode; /* 0: synchronous, 1: seeded, 2: replay               */
    double nu, dt;
    double dx[3];       /* spacing per axis                                   */
    uint64_t seed;
} at_oracle_cfg3;

int at_oracle_run3d(const at_oracle_cfg3 *c, int64_t n_steps, const int8_t *replay,
                    const double *u0, double *u_out, int64_t *hist)
{
    if (!c || n_steps < 0 || c->L < 0 || c->L > 64) return ORC_EARG;
    int64_t m[3], NP = 1, N = 1;
    for (int a = 0; a < 3; ++a) {
        if (c->n[a] <= 0 || c->P[a] <= 0 || c->n[a] % c->P[a] != 0) return ORC_EARG;
        m[a] = c->n[a] / c->P[a];
        if (m[a] < 2) return ORC_EARG;
        NP *= c->P[a];
        N *= c->n[a];
    }
    const int s = 2;                   /* levels per halo approximation     */
    const int depth = c->L + s + 1;
    double *H = (double *)calloc((size_t)depth * (size_t)N, sizeof(double));
    int8_t *K = (int8_t *)malloc((size_t)NP * 6);
    if (!H || !K) { free(H); free(K); return ORC_ENOMEM; }
    memcpy(H, u0, (size_t)N * sizeof(double));
    if (hist) memset(hist, 0, (size_t)(c->L + 1) * sizeof(int64_t));
    const int64_t n0 = c->n[0], n1 = c->n[1], n2 = c->n[2];
    for (int64_t n = 0; n < n_steps; ++n) {
        const double *cur = H + (size_t)(n % depth) * N;
        double *nxt = H + (size_t)((n + 1) % depth) * N;
        /* the six delays of every subdomain at this level */
        for (int64_t p = 0; p < NP; ++p) {
            for (int f = 0; f < 6; ++f) {
                int kr = 0;
                if (c->delay_mode == 1) kr = at_oracle_seeded_delay(c->seed, n, p, NP, f, 6, c->L);
                else if (c->delay_mode == 2) kr = replay[((size_t)n * NP + p) * 6 + f];
                if (kr < 0 || kr > c->L) { free(H); free(K); return ORC_EDELAY; }
                int64_t kmax = n - s + 1; if (kmax < 0) kmax = 0;
                K[p * 6 + f] = (int8_t)((kr < kmax) ? kr : kmax);
                if (hist) hist[K[p * 6 + f]] += 1;
            }
        }
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
        for (int64_t k = 0; k < n2; ++k)
            for (int64_t j = 0; j < n1; ++j)
                for (int64_t i = 0; i < n0; ++i) {
                    const int64_t idx[3] = {i, j, k};
                    const int64_t p = ((k / m[2]) * c->P[1] + j / m[1]) * c->P[0] + i / m[0];
                    const double u = cur[(k * n1 + j) * n0 + i];
                    double d1 = 0.0, d2 = 0.0;
                    for (int a = 0; a < 3; ++a) {
                        double v[2];    /* neighbour below and above along axis a */
                        for (int side = 0; side < 2; ++side) {
                            int64_t q[3] = {i, j, k};
                            q[a] = wrap(idx[a] + (side ? 1 : -1), c->n[a]);
                            const int64_t src = (q[2] * n1 + q[1]) * n0 + q[0];
                            const int64_t loc = idx[a] % m[a] + (side ? 1 : -1);
                            if (loc >= 0 && loc < m[a]) {      /* same subdomain: level n */
                                v[side] = cur[src];
                                continue;
                            }
                            const int kf = K[p * 6 + 2 * a + side];
                            double lev[2];
                            for (int t = 0; t < s; ++t) {
                                const int64_t lv = n - kf - t;
                                lev[t] = (lv >= 0) ? H[(size_t)(lv % depth) * N + src] : 0.0;
                            }
                            v[side] = at_oracle_extrapolate(s, kf, 1, lev);
                        }
                        d1 += (v[1] - v[0]) / (2.0 * c->dx[a]);
                        d2 += (v[1] - 2.0 * u + v[0]) / (c->dx[a] * c->dx[a]);
                    }
                    nxt[(k * n1 + j) * n0 + i] = u + c->dt * (-u * d1 + c->nu * d2);
                }
    }
    memcpy(u_out, H + (size_t)(n_steps % depth) * N, (size_t)N * sizeof(double));
    free(H); free(K);
    return ORC_OK;
}

int64_t at_oracle_cfg3_size(void) { return (int64_t)sizeof(at_oracle_cfg3); }

/* ------------------------------------------------------------------------ */
/* The system of Eq. BS in three dimensions: velocity components q_0, q_1,  */
/* q_2 (u, v, w) and passive scalars q_3 .. q_{nf-1}, each                  */
/*     d_t q_f + u d_x q_f + v d_y q_f + w d_z q_f = kappa_f lap q_f         */
/* (kappa = nu for the velocity components, the scalar's diffusivity alpha  */
/* for the scalars), same grid, decomposition, stencils and AT halos as     */
/* at_oracle_run3d; one delay per (level, subdomain, face) serves every      */
/* field (one message per face carries all of them).  Fields are stored one  */
/* after another: q[f][k][j][i].                                             */
/* ------------------------------------------------------------------------ */
int at_oracle_run3d_system(const at_oracle_cfg3 *c, int nf, const double *kappa, int64_t n_steps,
                           const int8_t *replay, const double *q0, double *q_out, int64_t *hist)
{
    if (!c || nf < 3 || nf > 8 || !kappa || n_steps < 0 || c->L < 0 || c->L > 64) return ORC_EARG;
    int64_t m[3], NP = 1, N = 1;
    for (int a = 0; a < 3; ++a) {
        if (c->n[a] <= 0 || c->P[a] <= 0 || c->n[a] % c->P[a] != 0) return ORC_EARG;
        m[a] = c->n[a] / c->P[a];
        if (m[a] < 2) return ORC_EARG;
        NP *= c->P[a];
        N *= c->n[a];
    }
    const int s = 2;
    const int depth = c->L + s + 1;
    const size_t lvl = (size_t)nf * (size_t)N;     /* words per level (all fields) */
    double *H = (double *)calloc((size_t)depth * lvl, sizeof(double));
    int8_t *K = (int8_t *)malloc((size_t)NP * 6);
    if (!H || !K) { free(H); free(K); return ORC_ENOMEM; }
    memcpy(H, q0, lvl * sizeof(double));
    if (hist) memset(hist, 0, (size_t)(c->L + 1) * sizeof(int64_t));
    const int64_t n0 = c->n[0], n1 = c->n[1], n2 = c->n[2];
    for (int64_t n = 0; n < n_steps; ++n) {
        const double *cur = H + (size_t)(n % depth) * lvl;
        double *nxt = H + (size_t)((n + 1) % depth) * lvl;
        for (int64_t p = 0; p < NP; ++p) {
            for (int f = 0; f < 6; ++f) {
                int kr = 0;
                if (c->delay_mode == 1) kr = at_oracle_seeded_delay(c->seed, n, p, NP, f, 6, c->L);
                else if (c->delay_mode == 2) kr = replay[((size_t)n * NP + p) * 6 + f];
                if (kr < 0 || kr > c->L) { free(H); free(K); return ORC_EDELAY; }
                int64_t kmax = n - s + 1; if (kmax < 0) kmax = 0;
                K[p * 6 + f] = (int8_t)((kr < kmax) ? kr : kmax);
                if (hist) hist[K[p * 6 + f]] += 1;
            }
        }
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
        for (int64_t k = 0; k < n2; ++k)
            for (int64_t j = 0; j < n1; ++j)
                for (int64_t i = 0; i < n0; ++i) {
                    const int64_t idx[3] = {i, j, k};
                    const int64_t p = ((k / m[2]) * c->P[1] + j / m[1]) * c->P[0] + i / m[0];
                    const int64_t pt = (k * n1 + j) * n0 + i;
                    const double vel[3] = {cur[pt], cur[(size_t)N + pt], cur[2 * (size_t)N + pt]};
                    for (int fld = 0; fld < nf; ++fld) {
                        const double *cf = cur + (size_t)fld * N;
                        const double q = cf[pt];
                        double adv = 0.0, lap = 0.0;
                        for (int a = 0; a < 3; ++a) {
                            double v[2];
                            for (int side = 0; side < 2; ++side) {
                                int64_t qq[3] = {i, j, k};
                                qq[a] = wrap(idx[a] + (side ? 1 : -1), c->n[a]);
                                const int64_t src = (qq[2] * n1 + qq[1]) * n0 + qq[0];
                                const int64_t loc = idx[a] % m[a] + (side ? 1 : -1);
                                if (loc >= 0 && loc < m[a]) { v[side] = cf[src]; continue; }
                                const int kf = K[p * 6 + 2 * a + side];
                                double lev[2];
                                for (int t = 0; t < s; ++t) {
                                    const int64_t lv = n - kf - t;
                                    lev[t] = (lv >= 0) ? H[(size_t)(lv % depth) * lvl + (size_t)fld * N + src] : 0.0;
                                }
                                v[side] = at_oracle_extrapolate(s, kf, 1, lev);
                            }
                            adv += vel[a] * (v[1] - v[0]) / (2.0 * c->dx[a]);
                            lap += (v[1] - 2.0 * q + v[0]) / (c->dx[a] * c->dx[a]);
                        }
                        nxt[(size_t)fld * N + pt] = q + c->dt * (-adv + kappa[fld] * lap);
                    }
                }
    }
    memcpy(q_out, H + (size_t)(n_steps % depth) * lvl, lvl * sizeof(double));
    free(H); free(K);
    return ORC_OK;
}
