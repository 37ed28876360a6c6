/*
 * oracle/geer_oracle.c -- plain, single-threaded FP64 reference ("oracle")
 * of the GEER query of "Efficient Estimation of Pairwise Effective
 * Resistance" (Yang & Tang, arXiv 2312.06123).
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load this file. It shares no code,
 * header, table or helper with the CUDA path; the two are written
 * independently from the paper and from the walk-RNG specification below.
 *
 * Every function follows the paper step by step, with no blocking, fusion
 * or reordering beyond what the paper states:
 *   - transition matrix P = D^-1 A (Section 2.1), (Px)(v) = mean of x over
 *     the neighbours of v, summed in ascending CSR order;
 *   - truncation length l, Eq. (6) (Theorem 1); Peng et al.'s l, Eq. (5);
 *   - spectral bound lambda = max(|lambda_2|, |lambda_n|) of P (Section 3.1),
 *     by Lanczos with full re-orthogonalisation on D^-1/2 A D^-1/2 deflated
 *     by its top eigenvector, and Sturm-sequence bisection on the
 *     tridiagonal matrix;
 *   - SMM, Algorithm 2, with the support sets V_s, V_t of Eq. (17) taken
 *     structurally (nodes reachable by a walk of exactly i steps);
 *   - AMC, Algorithm 1, with psi from Eq. (9), eta* from Eq. (8) (natural
 *     log) and the empirical Bernstein test of Lemma 2 / Eq. (7) at
 *     delta/tau;
 *   - GEER, Algorithm 3, with the greedy switch of Eq. (17).
 *
 * Walk randomness (the paper fixes none; this is the project's
 * specification, implemented independently on both sides):
 *   Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
 *   easy as 1, 2, 3", SC'11), key = (seed low 32 bits, seed high 32 bits),
 *   counter = (k, 2(b-1)+sigma, q_index, (j-1) >> 2) for walk k of batch b
 *   (sigma = 0: walk from s, 1: walk from t), step j = 1..l_f; the draw is
 *   word (j-1) & 3 of the output; the next node is
 *   col_idx[row_ptr[w] + ((uint64)draw * d(w) >> 32)].
 *
 * Walk checksum (for bit-exact comparison of walk endpoints): the wrapping
 * 64-bit sum, over every walk of every batch run, of splitmix64-finalise(x)
 * with x = endpoint + 0x9E3779B97F4A7C15 * (2k + sigma + 1) + (b << 58).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* Philox4x32-10                                                        */
/* ------------------------------------------------------------------ */
void og_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    /* round multipliers and Weyl key increments as published by Salmon et
       al. for Philox4x32 */
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)M0 * (uint64_t)x0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += W0;
        k1 += W1;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* splitmix64 finaliser (Steele, Lea, Flood, OOPSLA'14) */
static uint64_t og_mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

uint64_t og_walk_hash(int32_t endpoint, int64_t k, int sigma, int b)
{
    uint64_t x = (uint64_t)(uint32_t)endpoint
               + 0x9E3779B97F4A7C15ull * (uint64_t)(2 * k + sigma + 1)
               + ((uint64_t)b << 58);
    return og_mix64(x);
}

/* One step of a simple random walk (Section 2.1: move to a uniformly chosen
   neighbour) under the project's RNG specification. */
static int32_t og_walk_step(const int64_t *row_ptr, const int32_t *col_idx, int32_t w,
                            uint64_t seed, int64_t k, int lane, int64_t q_index, int j)
{
    uint32_t ctr[4] = {(uint32_t)k, (uint32_t)lane, (uint32_t)q_index, (uint32_t)((j - 1) >> 2)};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    og_philox4x32_10(ctr, key, out);
    uint32_t draw = out[(j - 1) & 3];
    uint64_t d = (uint64_t)(row_ptr[w + 1] - row_ptr[w]);
    uint64_t pick = ((uint64_t)draw * d) >> 32;
    return col_idx[row_ptr[w] + (int64_t)pick];
}

/* Walk of l_f steps from `start`; writes w_1..w_lf into nodes[0..lf-1]. */
void og_walk(const int64_t *row_ptr, const int32_t *col_idx, int32_t start, int lf,
             uint64_t seed, int64_t q_index, int b, int sigma, int64_t k, int32_t *nodes)
{
    int32_t w = start;
    for (int j = 1; j <= lf; ++j) {
        w = og_walk_step(row_ptr, col_idx, w, seed, k, 2 * (b - 1) + sigma, q_index, j);
        nodes[j - 1] = w;
    }
}

/* ------------------------------------------------------------------ */
/* Truncation length                                                   */
/* ------------------------------------------------------------------ */

/* Eq. (6): l = ceil( log((2/d(s) + 2/d(t)) / (eps (1 - lambda))) / log(1/lambda) - 1 ),
   clamped at 0 (a negative value means the zeroth term alone is within
   eps/2). lambda == 0 gives l = 0; lambda >= 1 is rejected (-1). */
int64_t og_ell(double ds, double dt, double eps, double lambda)
{
    if (!(lambda < 1.0) || !(eps > 0.0))
        return -1; /* Theorem 1 needs lambda < 1 (connected, non-bipartite) */
    if (lambda <= 0.0)
        return 0;
    double num = log((2.0 / ds + 2.0 / dt) / (eps * (1.0 - lambda)));
    double v = ceil(num / log(1.0 / lambda) - 1.0);
    return v < 0.0 ? 0 : (int64_t)v;
}

/* Eq. (5), Peng et al.'s degree-free truncation length. */
int64_t og_ell_peng(double eps, double lambda)
{
    if (!(lambda < 1.0) || !(eps > 0.0))
        return -1;
    if (lambda <= 0.0)
        return 0;
    double v = ceil(log(4.0 / (eps - eps * lambda)) / log(1.0 / lambda) - 1.0);
    return v < 0.0 ? 0 : (int64_t)v;
}

/* Eq. (8): eta* = 2 psi^2 log(2 tau / delta) / eps^2 (natural log; the
   Hoeffding step of Theorem 2's proof fixes the base). tau is a double
   only so that tests can evaluate variants of the log argument. */
double og_eta_star(double psi, double eps, double delta, double tau)
{
    return 2.0 * psi * psi * log(2.0 * tau / delta) / (eps * eps);
}

/* Eq. (7) at failure probability delta_b: f(n, var, psi, delta_b) */
double og_bernstein(double n, double var, double psi, double delta_b)
{
    double L = log(3.0 / delta_b);
    return sqrt(2.0 * var * L / n) + 3.0 * psi * L / n;
}

/* ------------------------------------------------------------------ */
/* Vector helpers                                                      */
/* ------------------------------------------------------------------ */

/* (P x)(v) = (1/d(v)) * sum_{u in N(v)} x(u), P = D^-1 A (Section 2.1). */
void og_apply_P(int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                const double *x, double *y)
{
    for (int64_t v = 0; v < n; ++v) {
        double acc = 0.0;
        for (int64_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e)
            acc += x[col_idx[e]];
        y[v] = acc / (double)(row_ptr[v + 1] - row_ptr[v]);
    }
}

/* Support of P x given the support of x: V' = N(V). */
static void og_expand_support(int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                              const uint8_t *in, uint8_t *out)
{
    for (int64_t v = 0; v < n; ++v) {
        uint8_t any = 0;
        for (int64_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e)
            any |= in[col_idx[e]];
        out[v] = any;
    }
}

/* max_1 and max_2 of a vector: the first and second elements of its
   entries sorted descending as a multiset (so a tie gives max2 == max1). */
void og_top2(int64_t n, const double *x, double *max1, double *max2)
{
    double a = -INFINITY, b = -INFINITY;
    for (int64_t v = 0; v < n; ++v) {
        double z = x[v];
        if (z > a) {
            b = a;
            a = z;
        } else if (z > b) {
            b = z;
        }
    }
    if (n < 2)
        b = 0.0;
    *max1 = a;
    *max2 = b;
}

/* Eq. (9) */
double og_psi(int64_t lf, double s_max1, double s_max2, double t_max1, double t_max2,
              double ds, double dt)
{
    double up = (double)((lf + 1) / 2), dn = (double)(lf / 2);
    return 2.0 * up * (s_max1 / ds + t_max1 / dt) + 2.0 * dn * (s_max2 / ds + t_max2 / dt);
}

static double og_series_term(const double *xs, const double *xt, int32_t s, int32_t t,
                             double ds, double dt)
{
    /* the four terms of Algorithm 2 / Algorithm 3 */
    return xs[s] / ds + xt[t] / dt - xs[t] / ds - xt[s] / dt;
}

/* SMM series terms for i = 0..L (Eq. (4) summands, computed by Algorithm
   2's iteration). terms has L+1 entries. */
int og_smm_terms(int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                 int32_t s, int32_t t, int64_t L, double *terms)
{
    double *xs = calloc((size_t)n, sizeof(double));
    double *xt = calloc((size_t)n, sizeof(double));
    double *ys = calloc((size_t)n, sizeof(double));
    double *yt = calloc((size_t)n, sizeof(double));
    if (!xs || !xt || !ys || !yt) {
        free(xs); free(xt); free(ys); free(yt);
        return -1;
    }
    double ds = (double)(row_ptr[s + 1] - row_ptr[s]);
    double dt = (double)(row_ptr[t + 1] - row_ptr[t]);
    xs[s] = 1.0;
    xt[t] = 1.0;
    terms[0] = og_series_term(xs, xt, s, t, ds, dt);
    for (int64_t i = 1; i <= L; ++i) {
        og_apply_P(n, row_ptr, col_idx, xs, ys);
        og_apply_P(n, row_ptr, col_idx, xt, yt);
        double *tmp;
        tmp = xs; xs = ys; ys = tmp;
        tmp = xt; xt = yt; yt = tmp;
        terms[i] = og_series_term(xs, xt, s, t, ds, dt);
    }
    free(xs); free(xt); free(ys); free(yt);
    return 0;
}

/* ------------------------------------------------------------------ */
/* AMC, Algorithm 1                                                    */
/* ------------------------------------------------------------------ */

typedef struct {
    double psi;           /* Eq. (9) */
    double eta_star;      /* Eq. (8) */
    int64_t eta0;         /* walks in the first batch */
    int32_t batches;      /* batches run */
    int32_t free_batches; /* first batch whose Bernstein test passed (0: none) */
    int64_t walks;        /* walk pairs run over all batches */
    int64_t walk_steps;   /* single-walk steps over all batches */
    double r_f;           /* returned estimate Z */
    double f_last;        /* Bernstein error of the last batch */
    double var_last;      /* empirical variance of the last batch */
    uint64_t checksum;    /* walk checksum (see header) */
} og_amc_out;

/* forced_eta0 <= 0: eta0 = ceil(eta_star / 2^(tau-1)); forced_batches <= 0: stop
   at the first batch whose test passes (or after tau batches). */
int og_amc(int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
           int32_t s, int32_t t, const double *xs, const double *xt, int64_t lf,
           double eps, int tau, double delta, uint64_t seed, int64_t q_index,
           int64_t forced_eta0, int forced_batches, og_amc_out *o)
{
    memset(o, 0, sizeof(*o));
    if (lf <= 0)
        return 0; /* nothing left to estimate: r_f = 0 */
    double ds = (double)(row_ptr[s + 1] - row_ptr[s]);
    double dt = (double)(row_ptr[t + 1] - row_ptr[t]);
    double s1, s2, t1, t2;
    og_top2(n, xs, &s1, &s2);
    og_top2(n, xt, &t1, &t2);
    o->psi = og_psi(lf, s1, s2, t1, t2, ds, dt);
    o->eta_star = og_eta_star(o->psi, eps, delta, (double)tau);
    int64_t eta = (int64_t)ceil(o->eta_star / ldexp(1.0, tau - 1));
    if (eta < 1)
        eta = 1;
    if (forced_eta0 > 0)
        eta = forced_eta0;
    o->eta0 = eta;
    int32_t *nodes = malloc((size_t)lf * sizeof(int32_t));
    if (!nodes)
        return -1;
    double Z = 0.0;
    for (int b = 1; b <= tau; ++b) {
        double sumZ = 0.0, sumZ2 = 0.0;
        for (int64_t k = 0; k < eta; ++k) {
            double Zk = 0.0;
            /* walk S_k from s */
            og_walk(row_ptr, col_idx, s, (int)lf, seed, q_index, b, 0, k, nodes);
            for (int64_t j = 0; j < lf; ++j)
                Zk += xs[nodes[j]] / ds - xt[nodes[j]] / dt;
            o->checksum += og_walk_hash(nodes[lf - 1], k, 0, b);
            /* walk T_k from t */
            og_walk(row_ptr, col_idx, t, (int)lf, seed, q_index, b, 1, k, nodes);
            for (int64_t j = 0; j < lf; ++j)
                Zk += xt[nodes[j]] / dt - xs[nodes[j]] / ds;
            o->checksum += og_walk_hash(nodes[lf - 1], k, 1, b);
            sumZ += Zk;
            sumZ2 += Zk * Zk;
        }
        o->walks += eta;
        o->walk_steps += 2 * eta * lf;
        Z = sumZ / (double)eta;
        double var = sumZ2 / (double)eta - Z * Z;
        if (var < 0.0)
            var = 0.0;
        double f = og_bernstein((double)eta, var, o->psi, delta / (double)tau);
        o->f_last = f;
        o->var_last = var;
        o->batches = b;
        int pass = f <= eps / 2.0;
        if (pass && o->free_batches == 0)
            o->free_batches = b;
        int stop = forced_batches > 0 ? (b >= forced_batches) : pass;
        if (stop)
            break;
        eta *= 2;
    }
    free(nodes);
    o->r_f = Z;
    return 0;
}

/* ------------------------------------------------------------------ */
/* GEER, Algorithm 3                                                   */
/* ------------------------------------------------------------------ */

typedef struct {
    double r;            /* r'(s,t) = r_b + r_f */
    double r_b, r_f;
    int64_t ell;         /* Eq. (6) */
    int64_t ell_b;       /* SMM iterations run */
    int64_t free_ell_b;  /* first iteration whose switch test held (0: none run) */
    double volume;       /* sum_{V_s} d + sum_{V_t} d at the switch */
    double h;            /* h(l - l_b) at the switch */
    og_amc_out amc;
} og_geer_out;

/* forced_ell_b < 0: free-running switch (Eq. (17) or l_b >= l).
   trace (nullable) receives, per SMM iteration i = 1..l_b, the 6-tuple
   (r_b after i, volume, h(l - i), psi(l - i), max_1(s*)/d(s) + max_1(t*)/d(t),
   volume of the union V_s u V_t) at trace[6(i-1) ..]: Eq. (17)'s quantities,
   Eq. (9)'s leading term and the next push's size (the learned switch's
   features and cost). */
int og_geer(int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
            int32_t s, int32_t t, double eps, double delta, int tau, uint64_t seed,
            double lambda, int64_t q_index, int64_t forced_ell_b, int64_t forced_eta0,
            int forced_batches, int use_peng_ell, og_geer_out *o, double *trace)
{
    memset(o, 0, sizeof(*o));
    if (s == t)
        return 0; /* r(s,s) = 0 (Definition 1) */
    double ds = (double)(row_ptr[s + 1] - row_ptr[s]);
    double dt = (double)(row_ptr[t + 1] - row_ptr[t]);
    int64_t ell = use_peng_ell ? og_ell_peng(eps, lambda) : og_ell(ds, dt, eps, lambda);
    if (ell < 0)
        return -3;
    o->ell = ell;
    double *xs = calloc((size_t)n, sizeof(double));
    double *xt = calloc((size_t)n, sizeof(double));
    double *ys = calloc((size_t)n, sizeof(double));
    double *yt = calloc((size_t)n, sizeof(double));
    uint8_t *vs = calloc((size_t)n, 1), *vt = calloc((size_t)n, 1);
    uint8_t *ws = calloc((size_t)n, 1), *wt = calloc((size_t)n, 1);
    if (!xs || !xt || !ys || !yt || !vs || !vt || !ws || !wt) {
        free(xs); free(xt); free(ys); free(yt); free(vs); free(vt); free(ws); free(wt);
        return -1;
    }
    xs[s] = 1.0;
    xt[t] = 1.0;
    vs[s] = 1;
    vt[t] = 1;
    double rb = og_series_term(xs, xt, s, t, ds, dt);
    int64_t lb = 0;
    const int64_t h_mult = ((int64_t)1 << tau) - 1;
    int run_smm = forced_ell_b >= 0 ? (forced_ell_b > 0) : (ell >= 1);
    while (run_smm) {
        og_apply_P(n, row_ptr, col_idx, xs, ys);
        og_apply_P(n, row_ptr, col_idx, xt, yt);
        double *tmp;
        tmp = xs; xs = ys; ys = tmp;
        tmp = xt; xt = yt; yt = tmp;
        og_expand_support(n, row_ptr, col_idx, vs, ws);
        og_expand_support(n, row_ptr, col_idx, vt, wt);
        uint8_t *tb;
        tb = vs; vs = ws; ws = tb;
        tb = vt; vt = wt; wt = tb;
        rb += og_series_term(xs, xt, s, t, ds, dt);
        lb += 1;
        /* Eq. (17): volume of the supports against h(l - l_b) = (2^tau - 1) eta */
        double vol = 0.0;
        for (int64_t v = 0; v < n; ++v) {
            double d = (double)(row_ptr[v + 1] - row_ptr[v]);
            if (vs[v]) vol += d;
            if (vt[v]) vol += d;
        }
        double vol_union = 0.0;
        for (int64_t v = 0; v < n; ++v)
            if (vs[v] || vt[v])
                vol_union += (double)(row_ptr[v + 1] - row_ptr[v]);
        int64_t lf = ell - lb;
        double psi = 0.0, h = 0.0;
        double s1, s2, t1, t2;
        og_top2(n, xs, &s1, &s2);
        og_top2(n, xt, &t1, &t2);
        if (lf > 0) {
            psi = og_psi(lf, s1, s2, t1, t2, ds, dt);
            int64_t eta = (int64_t)ceil(og_eta_star(psi, eps, delta, (double)tau) / ldexp(1.0, tau - 1));
            if (eta < 1)
                eta = 1;
            h = (double)(h_mult * eta);
        }
        o->volume = vol;
        o->h = h;
        if (trace) {
            trace[6 * (lb - 1) + 0] = rb;
            trace[6 * (lb - 1) + 1] = vol;
            trace[6 * (lb - 1) + 2] = h;
            trace[6 * (lb - 1) + 3] = psi;
            trace[6 * (lb - 1) + 4] = s1 / ds + t1 / dt;
            trace[6 * (lb - 1) + 5] = vol_union;
        }
        int free_stop = (vol > h) || (lb >= ell);
        if (free_stop && o->free_ell_b == 0)
            o->free_ell_b = lb;
        int stop = forced_ell_b >= 0 ? (lb >= forced_ell_b) : free_stop;
        if (stop)
            break;
    }
    o->ell_b = lb;
    o->r_b = rb;
    int64_t lf = ell - lb;
    int rc = 0;
    if (lf > 0)
        rc = og_amc(n, row_ptr, col_idx, s, t, xs, xt, lf, eps, tau, delta, seed, q_index,
                    forced_eta0, forced_batches, &o->amc);
    o->r_f = o->amc.r_f;
    o->r = o->r_b + o->r_f;
    free(xs); free(xt); free(ys); free(yt); free(vs); free(vt); free(ws); free(wt);
    return rc;
}

/* ------------------------------------------------------------------ */
/* Spectral bound (Section 3.1)                                        */
/* ------------------------------------------------------------------ */

/* number of eigenvalues of the symmetric tridiagonal (a, b) below x
   (Sturm sequence count of the LDL^T pivots) */
static int64_t og_sturm_count(int64_t k, const double *a, const double *b, double x)
{
    int64_t cnt = 0;
    double q = a[0] - x;
    if (q < 0.0) cnt++;
    for (int64_t i = 1; i < k; ++i) {
        double qq = q == 0.0 ? 1e-300 : q;
        q = (a[i] - x) - b[i - 1] * b[i - 1] / qq;
        if (q < 0.0) cnt++;
    }
    return cnt;
}

/* the idx-th smallest eigenvalue (0-based) of the tridiagonal matrix */
static double og_tridiag_eig(int64_t k, const double *a, const double *b, int64_t idx)
{
    double lo = INFINITY, hi = -INFINITY;
    for (int64_t i = 0; i < k; ++i) {
        double r = (i > 0 ? fabs(b[i - 1]) : 0.0) + (i + 1 < k ? fabs(b[i]) : 0.0);
        if (a[i] - r < lo) lo = a[i] - r;
        if (a[i] + r > hi) hi = a[i] + r;
    }
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi)
            break;
        if (og_sturm_count(k, a, b, mid) > idx)
            hi = mid;
        else
            lo = mid;
    }
    return 0.5 * (lo + hi);
}

static double og_dot(int64_t n, const double *x, const double *y)
{
    double acc = 0.0;
    for (int64_t i = 0; i < n; ++i)
        acc += x[i] * y[i];
    return acc;
}

/* lambda_2 and lambda_n of P via Lanczos on N = D^-1/2 A D^-1/2 (similar
   to P) restricted to the complement of its top eigenvector sqrt(d/2m),
   with full re-orthogonalisation. Runs until the extreme Ritz values move
   by less than tol over 10 steps, the Krylov space is exhausted, or
   max_steps. Returns the number of Lanczos steps taken (< 0 on error). */
int64_t og_spectral_bound(int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                          int64_t max_steps, double tol, double *lam2, double *lamn)
{
    if (n < 2)
        return -1;
    int64_t kmax = max_steps < n - 1 ? max_steps : n - 1;
    double *Q = malloc((size_t)(kmax + 1) * (size_t)n * sizeof(double));
    double *phi = malloc((size_t)n * sizeof(double));
    double *isd = malloc((size_t)n * sizeof(double));
    double *w = malloc((size_t)n * sizeof(double));
    double *a = calloc((size_t)(kmax + 1), sizeof(double));
    double *b = calloc((size_t)(kmax + 1), sizeof(double));
    if (!Q || !phi || !isd || !w || !a || !b) {
        free(Q); free(phi); free(isd); free(w); free(a); free(b);
        return -2;
    }
    double two_m = (double)row_ptr[n];
    for (int64_t v = 0; v < n; ++v) {
        double d = (double)(row_ptr[v + 1] - row_ptr[v]);
        phi[v] = sqrt(d / two_m);
        isd[v] = 1.0 / sqrt(d);
    }
    /* deterministic start vector, orthogonal to phi */
    double *q0 = Q;
    uint64_t st = 0x243F6A8885A308D3ull;
    for (int64_t v = 0; v < n; ++v) {
        st = og_mix64(st + 0x9E3779B97F4A7C15ull);
        q0[v] = (double)(st >> 11) * (1.0 / 9007199254740992.0) - 0.5;
    }
    for (int pass = 0; pass < 2; ++pass) {
        double c = og_dot(n, phi, q0);
        for (int64_t v = 0; v < n; ++v) q0[v] -= c * phi[v];
    }
    double nrm = sqrt(og_dot(n, q0, q0));
    for (int64_t v = 0; v < n; ++v) q0[v] /= nrm;

    int64_t k = 0;
    double prev_hi = 0.0, prev_lo = 0.0;
    for (int64_t j = 0; j < kmax; ++j) {
        const double *qj = Q + (size_t)j * (size_t)n;
        /* w = N q_j */
        for (int64_t v = 0; v < n; ++v) {
            double acc = 0.0;
            for (int64_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e)
                acc += qj[col_idx[e]] * isd[col_idx[e]];
            w[v] = acc * isd[v];
        }
        a[j] = og_dot(n, qj, w);
        /* full re-orthogonalisation (twice) against phi and q_0..q_j */
        for (int pass = 0; pass < 2; ++pass) {
            double c = og_dot(n, phi, w);
            for (int64_t v = 0; v < n; ++v) w[v] -= c * phi[v];
            for (int64_t i = 0; i <= j; ++i) {
                const double *qi = Q + (size_t)i * (size_t)n;
                double ci = og_dot(n, qi, w);
                for (int64_t v = 0; v < n; ++v) w[v] -= ci * qi[v];
            }
        }
        k = j + 1;
        double beta = sqrt(og_dot(n, w, w));
        b[j] = beta;
        if ((j + 1) % 10 == 0 || beta < 1e-12 || j + 1 == kmax) {
            double hi = og_tridiag_eig(k, a, b, k - 1);
            double lo = og_tridiag_eig(k, a, b, 0);
            if (beta < 1e-12 || j + 1 == kmax)
                break;
            if (j + 1 >= 20 && fabs(hi - prev_hi) < tol && fabs(lo - prev_lo) < tol)
                break;
            prev_hi = hi;
            prev_lo = lo;
        }
        double *qn = Q + (size_t)(j + 1) * (size_t)n;
        for (int64_t v = 0; v < n; ++v) qn[v] = w[v] / beta;
    }
    *lam2 = og_tridiag_eig(k, a, b, k - 1);
    *lamn = og_tridiag_eig(k, a, b, 0);
    free(Q); free(phi); free(isd); free(w); free(a); free(b);
    return k;
}
