/*
 * geer.h -- C ABI of the GB300 GEER engine: epsilon-approximate pairwise
 * effective resistance (Yang & Tang, "Efficient Estimation of Pairwise
 * Effective Resistance", arXiv 2312.06123).
 *
 * The engine answers the query of Definition 2: for node pairs (s, t) of an
 * undirected, unweighted, connected, non-bipartite graph (Section 2.1), it
 * returns r'(s,t) with |r(s,t) - r'(s,t)| <= eps with probability >= 1-delta,
 * r(s,t) being the effective resistance of Definition 1 / Eq. (1). It runs
 * GEER (Algorithm 3): the truncation length l of Eq. (6), then SMM
 * iterations (Algorithm 2) until the greedy switch of Eq. (17), then AMC
 * (Algorithm 1) for the remaining l - l_b steps, r' = r_b + r_f.
 *
 * Conventions shared by every entry point:
 *   - Return value: GER_OK (0) or a negative GER_ERR_* code; on error no
 *     output is written and ger_last_error() describes the failure.
 *   - No C++ exception crosses this boundary.
 *   - Node ids are int32 in [0, n). Host pointers unless the name ends in
 *     _dev (device pointers on the graph's device).
 *   - A ger_graph handle is not thread-safe; separate handles are.
 *   - Results are deterministic for a given (graph, lambda, options, seed,
 *     query index in the batch, eps): the walk random numbers are keyed by
 *     (seed, query index, batch, walk, step) with Philox4x32-10.
 */
#ifndef GEER_H
#define GEER_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define GER_OK                 0
#define GER_ERR_INVALID       -1  /* bad argument (null pointer, eps <= 0, q < 0, ...) */
#define GER_ERR_NODE_RANGE    -2  /* a query node outside [0, n) */
#define GER_ERR_CSR           -3  /* CSR not canonical: unsorted, self-loop, duplicate, asymmetric */
#define GER_ERR_DISCONNECTED  -4  /* graph not connected (Section 2.1 assumes it is) */
#define GER_ERR_BIPARTITE     -5  /* bipartite graph: lambda_n = -1 and Eq. (6) is undefined */
#define GER_ERR_OOM           -6  /* device or host allocation failed */
#define GER_ERR_CUDA          -7  /* a CUDA runtime call failed */
#define GER_ERR_TIMEOUT       -8  /* a bounded device-side wait gave up (reserved: no entry point
                                     of this version has such a wait, so none returns it) */
#define GER_ERR_CAPACITY      -9  /* a query outgrew a workspace limit (see ger_options) */
#define GER_ERR_NO_LAMBDA    -10  /* spectral bound neither computed nor set */

/* precision of the SMM vectors (series and statistics are FP64 always) */
#define GER_FP64 0
#define GER_FP32 1

/* switch policy between SMM and AMC */
#define GER_SWITCH_RULE  0  /* Eq. (17): stop SMM once the support volume exceeds h(l - l_b) */
#define GER_SWITCH_MLP   1  /* the learned switch installed by ger_set_switch_mlp (stops no later than
                               Eq. (17)); Eq. (17) alone if none is installed */
#define GER_SWITCH_FIXED 2  /* run exactly min(fixed_ell_b, l) SMM iterations; fixed_ell_b < 0 means l */

/* engine of the SMM iterations */
#define GER_ENGINE_SPARSE 0 /* per-query frontier tables, push (fits the small frontiers of Eq. (17)'s switch) */
#define GER_ENGINE_DENSE  1 /* blocks of query vectors, pull SpMM over all rows (deep SMM) */
#define GER_ENGINE_HYBRID 2 /* sparse push first; a query whose next push reaches dense_switch pairs
                               moves to a dense column (as many as dense_budget_mb holds) */

/* truncation length formula */
#define GER_ELL_REFINED 0   /* Eq. (6), Theorem 1 */
#define GER_ELL_PENG    1   /* Eq. (5), Peng et al. */

typedef struct ger_graph ger_graph; /* opaque; owns the device copy of the graph */

typedef struct ger_options {
    double   delta;         /* failure probability delta (paper default 0.01) */
    int32_t  tau;           /* maximum number of AMC batches tau (paper default 5), 1..20;
                               0: the graph's autotuned tau (ger_autotune), else 5 */
    int32_t  precision;     /* GER_FP32 (default) or GER_FP64 */
    int32_t  per_query;     /* 0: all queries of the batch together; 1: one query at a time */
    int32_t  switch_policy; /* GER_SWITCH_RULE (default), GER_SWITCH_MLP or GER_SWITCH_FIXED */
    int32_t  fixed_ell_b;   /* used by GER_SWITCH_FIXED */
    int32_t  ell_formula;   /* GER_ELL_REFINED (default) or GER_ELL_PENG */
    uint64_t seed;          /* walk RNG seed */
    int64_t  sparse_cap;    /* max SMM push pairs of one query iteration (0: no limit beyond the pool) */
    int32_t  smm_engine;    /* GER_ENGINE_SPARSE (default), GER_ENGINE_DENSE or GER_ENGINE_HYBRID */
    int32_t  dense_width;   /* dense engine: columns per block (2 per query); 0: autotuned per graph */
    int64_t  dense_switch;  /* hybrid engine: push pairs at which a query moves to the SpMM; 0: autotuned, else nnz / 16 */
    int32_t  dense_budget_mb; /* hybrid engine: device memory for dense columns (MiB); 0: half the free memory */
    int32_t  mlp_at_start;  /* GER_SWITCH_MLP: 1 also consults the network before the first SMM
                               iteration (l_b = 0: AMC alone); 0 (default): after iterations only */
} ger_options;

/* Per-query statistics (all optional outputs). */
typedef struct ger_query_stats {
    int32_t  ell;        /* truncation length l, Eq. (6) (or Eq. (5)) */
    int32_t  ell_b;      /* SMM iterations run (Algorithm 3) */
    int32_t  batches;    /* AMC batches run (Algorithm 1), 0 if l_f = 0 */
    int32_t  flags;      /* reserved, 0 */
    int64_t  eta0;       /* walk pairs in the first AMC batch */
    int64_t  walks;      /* walk pairs over all batches */
    int64_t  walk_steps; /* single-walk steps over all batches */
    double   r_b;        /* SMM part, Eq. (16) r*_b */
    double   r_f;        /* AMC estimate of Eq. (16) r*_f */
    double   psi;        /* Eq. (9) at l_f = l - l_b */
    double   f_last;     /* empirical Bernstein error of the last batch, Eq. (7) */
    double   volume;     /* sum_{V_s} d + sum_{V_t} d after the last SMM iteration, Eq. (17) */
    double   h;          /* h(l - l_b) at the last SMM iteration */
    uint64_t checksum;   /* wrapping sum over all walks of a hash of (endpoint, walk, batch) */
} ger_query_stats;

/* Fill *opt with the defaults: delta 0.01, tau 5, FP32, batched, rule, refined l, seed 3. */
void ger_default_options(ger_options *opt);

/*
 * Load a graph given as canonical CSR: row_ptr[0..n] (int64, row_ptr[0] == 0),
 * col_idx[0..row_ptr[n]) with every neighbour list sorted ascending, no
 * self-loops, no duplicates, and every edge stored in both rows (the
 * undirected, unweighted graph of Section 2.1). The graph must be connected
 * and non-bipartite (Section 2.1). The arrays are copied to `device`; the
 * caller keeps ownership of its inputs. On success *out owns the device copy
 * until ger_free().
 * Errors: GER_ERR_INVALID, GER_ERR_CSR, GER_ERR_DISCONNECTED,
 * GER_ERR_BIPARTITE, GER_ERR_OOM, GER_ERR_CUDA.
 */
int ger_load_csr(int64_t n, const int64_t *row_ptr, const int32_t *col_idx, int device,
                 ger_graph **out);

/* Release the handle and every device buffer it owns. Null is a no-op. */
void ger_free(ger_graph *g);

/* Graph size: n and the number of stored (directed) entries 2m. */
int ger_graph_size(const ger_graph *g, int64_t *n, int64_t *nnz);

/*
 * Spectral bound lambda = max(|lambda_2|, |lambda_n|) of P = D^-1 A, the
 * once-per-graph preprocessing of Section 3.1 that Eq. (6) needs. Computed on
 * the device (FP64 Lanczos with full re-orthogonalisation on D^-1/2 A D^-1/2,
 * deflated by its top eigenvector) on first call and cached; lam2 and lamn
 * (nullable) receive lambda_2 and lambda_n.
 */
int ger_spectral_bound(ger_graph *g, double *lambda, double *lam2, double *lamn);

/* Inject lambda (0 <= lambda < 1) instead of computing it (e.g. to share one
   value between runs). */
int ger_set_spectral_bound(ger_graph *g, double lambda);

/*
 * How the graph's lambda (Section 3.1) was obtained. steps: Lanczos steps
 * taken (0 when lambda was set with ger_set_spectral_bound). converged: 1
 * when the extreme Ritz values settled to 1e-13 over 10 steps, or the Krylov
 * space was exhausted, within 300 steps. When they did not, an unconverged
 * Ritz value lies inside the spectrum and would underestimate lambda (Eq. (6)
 * would then give too short an l, voiding Theorem 1's eps/2 tail bound), so
 * ger_spectral_bound's lambda is widened to
 * max(|lambda_2| + resid_hi, |lambda_n| + resid_lo), resid_* being the
 * residual bounds beta_k |s_k| of the two extreme Ritz pairs (an eigenvalue
 * of P lies within each). Any output pointer may be null.
 * Errors: GER_ERR_INVALID, GER_ERR_NO_LAMBDA (nothing computed or set yet).
 */
int ger_spectral_bound_info(const ger_graph *g, int32_t *converged, int32_t *steps, double *resid_hi,
                            double *resid_lo);

/*
 * Answer q queries r_out[i] ~ r(s[i], t[i]) at error eps (Algorithm 3).
 * s, t: q node ids each (host); r_out: q doubles (host); stats: q entries
 * (host, nullable); opt: nullable (defaults). s[i] == t[i] gives exactly 0
 * (Definition 1). The query's index i keys its walk random numbers.
 * Errors: GER_ERR_INVALID, GER_ERR_NODE_RANGE, GER_ERR_NO_LAMBDA (cannot
 * happen: lambda is computed on demand), GER_ERR_CAPACITY, GER_ERR_OOM,
 * GER_ERR_CUDA.
 */
int ger_query_batch(ger_graph *g, int64_t q, const int32_t *s, const int32_t *t, double eps,
                    const ger_options *opt, double *r_out, ger_query_stats *stats);

/* As ger_query_batch, with a per-query error eps[i] (host). */
int ger_query_batch_eps(ger_graph *g, int64_t q, const int32_t *s, const int32_t *t,
                        const double *eps, const ger_options *opt, double *r_out,
                        ger_query_stats *stats);

/*
 * Device-resident variant: s_dev, t_dev, eps_dev (q entries each), r_dev (q
 * doubles) and stats_dev (q ger_query_stats, nullable) live on the graph's
 * device; work is issued on `stream` (a cudaStream_t, null = default
 * stream) and the call returns once it has completed. Node ids are checked
 * on the device; an out-of-range id yields GER_ERR_NODE_RANGE.
 */
int ger_query_batch_dev(ger_graph *g, int64_t q, const int32_t *s_dev, const int32_t *t_dev,
                        const double *eps_dev, const ger_options *opt, double *r_dev,
                        ger_query_stats *stats_dev, void *stream);

/*
 * ger_query_batch_dev with no allocation: the paper has no counterpart; this
 * entry point exists for callers that cannot call cudaMalloc -- a serving
 * loop that must never block on the device (cudaMalloc/cudaFree may
 * synchronise it), or a process whose device memory is reserved up front or
 * owned by another allocator. It allocates nothing (no cudaMalloc, cudaFree,
 * pinned buffer or allocating library call): all scratch comes from one
 * static 32 MiB device array that every GPU loading the library holds until
 * the process exits. Arguments are those of ger_query_batch_dev, with these
 * limits:
 *   - q <= 64 queries per call;
 *   - 524288 frontier-table slots per call, shared by the tables of every SMM
 *     iteration of every query (each a power of two at least twice the
 *     iteration's push volume), so one table holds at most 262144 push pairs;
 *   - options.sparse_cap, when set, bounds one table as in the other entry
 *     points;
 *   - high-degree frontier nodes are pushed in chunks through a list of 4096
 *     chunk records; beyond it they are pushed by single warps (slower, the
 *     same result).
 * Beyond the first three it returns GER_ERR_CAPACITY. Options it rejects with
 * GER_ERR_INVALID: switch_policy GER_SWITCH_MLP (the learned switch) and
 * smm_engine GER_ENGINE_DENSE or GER_ENGINE_HYBRID (their dense blocks are
 * far larger than the array); per_query, dense_width, dense_switch and
 * dense_budget_mb are ignored (queries run as one batch, sparse engine). The
 * spectral bound must already be available
 * (ger_spectral_bound or ger_set_spectral_bound), else GER_ERR_NO_LAMBDA.
 * The first call on a device looks up the array's device address; make that
 * first call before any stream capture. Every call shares the one array and
 * resets what must start at zero; calls that overlap on the GPU (other
 * streams, other threads) race on it and must be serialised by the caller.
 * Returns once the work has completed.
 */
int ger_query_batch_dev_noalloc(ger_graph *g, int64_t q, const int32_t *s_dev, const int32_t *t_dev,
                                const double *eps_dev, const ger_options *opt, double *r_dev,
                                ger_query_stats *stats_dev, void *stream);

/* Thread-local description of the last error of this thread. */
const char *ger_last_error(void);

/* Testing hook for the out-of-memory paths (no counterpart in the paper):
 * the countdown-th next device allocation of a graph's query workspace
 * (countdown >= 1; 0 disarms) reports failure without allocating, so the
 * call that needed it returns GER_ERR_OOM. The handle stays usable: a later
 * call allocates again. Process-wide; not thread-safe against concurrent
 * queries. Errors: GER_ERR_INVALID for countdown < 0. */
int ger_test_fail_alloc(int64_t countdown);

/* Number of kernels this library has launched in this process (every node
   of a replayed CUDA graph counts). */
int64_t ger_launch_count(void);

/* Per-kernel-family timing, measured with CUDA events recorded on the
   stream each kernel is launched on. */
typedef struct ger_kernel_profile {
    char     name[32];   /* kernel family, e.g. "amc_walk" */
    int64_t  launches;   /* launches timed since the last enable */
    double   total_ms;   /* summed launch durations */
} ger_kernel_profile;

/* on != 0: start timing every launch from now on (accumulators reset);
   on == 0: stop timing. Timing adds two event records per launch. */
int ger_profile_enable(int on);

/* Copy up to max_entries family records into out; returns the number of
   families with at least one timed launch (>= 0), or GER_ERR_INVALID. */
int ger_profile_read(ger_kernel_profile *out, int max_entries);

/* Autotuning of the SMM engines (no counterpart in the paper; the choices
 * change run time only, never a result). Times, on graph g and the given
 * queries (host pointers, per-query eps), with the given options:
 *  1. the dense block width: standalone SMM (4 iterations) of up to 64 of the
 *     queries on the dense engine at every width the precision allows;
 *  2. the hybrid engine's switch size: the whole batch at nnz/64, nnz/16,
 *     nnz/4, nnz push pairs and without moves.
 *  3. tau, the number of AMC batches of Algorithm 1: the whole batch with the
 *     caller's options at tau = 1..8 (Theorem 2's guarantee holds at delta /
 *     tau for any tau, so the choice changes the walks drawn and the run
 *     time, not the eps guarantee; Section 5.4 measures the same range).
 * The fastest of each is stored on g and used whenever an option leaves the
 * value at 0 (dense_width, dense_switch, tau). out (nullable) receives the
 * choices and the median batch times.
 * Errors: as ger_query_batch_eps. */
typedef struct ger_tuning {
    int32_t dense_width;            /* chosen block width (0: no dense engine on this graph) */
    int32_t reserved;
    int64_t dense_switch;           /* chosen hybrid switch size (push pairs) */
    float   width_ms[3];            /* widths 32, 64, 128 (FP64: 32, 64) */
    float   switch_ms[5];
    int64_t switch_candidates[5];
    int32_t tau;                    /* chosen tau (used by options with tau = 0) */
    float   tau_ms[8];              /* median batch time at tau = 1..8 */
} ger_tuning;

int ger_autotune(ger_graph *g, int64_t q, const int32_t *s, const int32_t *t, const double *eps,
                 const ger_options *opt, ger_tuning *out);

/* ------------------------------------------------------------------------
 * The learned SMM -> AMC switch (no counterpart in the paper; it replaces
 * the cost comparison of Eq. (17), Section 4.3, by a small network; the
 * truncation length l of Eq. (6) is unchanged, so Theorem 2's eps guarantee
 * holds whatever it decides).
 *
 * Network: 6 -> 64 -> 64 -> 1, ReLU, FP16 weights (IEEE binary16 bit
 * patterns), FP32 arithmetic. Parameter order, GER_MLP_PARAMS values:
 * W1[64][6], b1[64], W2[64][64] (W2[j][k] multiplies hidden unit k of the
 * first layer), b2[64], W3[64], b3. Inputs after SMM iteration l_b, each
 * normalised as (f - mean) / std: log d(s), log d(t), l - l_b,
 * log(Eq. 17's volume), log h(l - l_b), max_1(s*)/d(s) + max_1(t*)/d(t).
 * Output: predicted log C(l_b + 1) - log C(l_b), C(j) being the query's
 * cost when it switches after j iterations; the query switches when the
 * output is >= 0, when Eq. (17) says to switch (the network can stop a
 * query earlier than the rule, never later, so its SMM work is bounded by
 * the rule's), and always once l_b = l. The network is consulted where the
 * rule continues: after each SMM iteration, and, with options.mlp_at_start,
 * also before the first one (l_b = 0: AMC alone, Algorithm 1), with the
 * inputs of s* = e_s, t* = e_t (log d(s), log d(t), l, log(d(s) + d(t)),
 * log h(l), 1/d(s) + 1/d(t)). One thread per query evaluates it inside the
 * decision kernels.
 * ------------------------------------------------------------------------ */
#define GER_MLP_INPUTS 6
#define GER_MLP_HIDDEN 64
#define GER_MLP_PARAMS 4673
#define GER_LOG_WIDTH  8   /* columns of one cost-log row, see ger_smm_trace */

/* Install (weights != NULL) or remove (weights == NULL) the learned switch
 * of graph g. norm = {mean[6], std[6]} (std > 0), weights = GER_MLP_PARAMS
 * FP16 values; both are copied. Queries with switch_policy GER_SWITCH_MLP use
 * it from the next call on.
 * Errors: GER_ERR_INVALID, GER_ERR_OOM, GER_ERR_CUDA. */
int ger_set_switch_mlp(ger_graph *g, const float *norm, const uint16_t *weights);

/*
 * Algorithm 3 with the greedy switch of Eq. (17) replaced, per query, by a
 * given number of SMM iterations: the experiment of Section 5.4 (Fig. 10)
 * that varies l_b around the switch point l*_b Eq. (17) picks. Query i runs
 * min(ell_b[i], l) SMM iterations (ell_b[i] = 0: AMC alone, Algorithm 1;
 * ell_b[i] >= l: SMM alone, Algorithm 2), then AMC for the remaining
 * l - l_b steps; ell_b[i] < 0 leaves query i to opt's switch policy. Theorem
 * 2's eps guarantee holds for every l_b (the truncation length l is
 * unchanged). Host pointers (ell_b: q int32); other arguments and errors as
 * ger_query_batch_eps.
 */
int ger_query_batch_lb(ger_graph *g, int64_t q, const int32_t *s, const int32_t *t, const double *eps,
                       const int32_t *ell_b, const ger_options *opt, double *r_out, ger_query_stats *stats);

/* Cost log of the learned switch: runs the batch with min(max_steps, l)
 * SMM iterations (GER_SWITCH_FIXED; the other options are used as given)
 * and writes, for query i and iteration j = 1..ell_b(i),
 * log_out[(i * max_steps + j - 1) * GER_LOG_WIDTH + k] =
 *   k = 0..5: the six raw (unnormalised) network inputs after iteration j,
 *   k = 6:    sum of d(v) over V_s u V_t after iteration j (the size of the
 *             push that computes iteration j + 1),
 *   k = 7:    Eq. (17)'s volume after iteration j.
 * Rows past ell_b(i) are zero. stats (nullable) as for ger_query_batch.
 * Host pointers. Errors: as ger_query_batch_eps; GER_ERR_INVALID for
 * max_steps outside 1..4096. */
int ger_smm_trace(ger_graph *g, int64_t q, const int32_t *s, const int32_t *t, const double *eps,
                  const ger_options *opt, int32_t max_steps, float *log_out, ger_query_stats *stats);

/* Network output for `rows` normalised input rows x[rows][6] (host
 * pointers), on the current device. Errors: GER_ERR_INVALID, GER_ERR_OOM,
 * GER_ERR_CUDA. */
int ger_mlp_forward(int64_t rows, const float *x, const uint16_t *weights, float *y);

/* Gradient of L = (1/rows) sum_i (y_i - target_i)^2 with respect to the
 * GER_MLP_PARAMS parameters (FP32, same order), and L (nullable), at the
 * given FP16 weights. Host pointers; current device. */
int ger_mlp_gradient(int64_t rows, const float *x, const float *target, const uint16_t *weights, float *grad,
                     float *loss);

typedef struct ger_mlp_train_options {
    int32_t  epochs;     /* passes over the rows (default 60) */
    int32_t  batch;      /* rows per Adam step (default 1024) */
    float    lr;         /* Adam step size (default 2e-3) */
    float    beta1, beta2, adam_eps;  /* Adam moments (0.9, 0.999, 1e-8) */
    uint64_t seed;       /* row shuffling */
} ger_mlp_train_options;

void ger_default_mlp_train_options(ger_mlp_train_options *o);

/* Train the network on the GPU (current device): minibatch Adam on FP32
 * master weights, FP16 weights in every forward and backward pass, the
 * mean squared error of the rows x[rows][6] (normalised) against target.
 * weights: initial values in, trained values out (FP16). loss_per_epoch
 * (nullable, epochs entries): mean loss over each epoch's minibatches before
 * their updates. Errors: GER_ERR_INVALID, GER_ERR_OOM, GER_ERR_CUDA. */
int ger_mlp_train(int64_t rows, const float *x, const float *target, const ger_mlp_train_options *o,
                  uint16_t *weights, float *loss_per_epoch);

#ifdef __cplusplus
}
#endif

#endif /* GEER_H */
