// geer_kernels.h -- launch arguments and kernel declarations of the GEER
// CUDA library (internal).
#pragma once

#include <vector>

#include "geer_internal.cuh"

namespace geer {

struct SmmArgs {
    DevGraph g;
    int32_t nq;            // queries handled by this launch
    int32_t q_index_base;  // batch index of query 0 of this launch
    QState* st;            // nq records
    QSmm* sm;              // nq records
    const int32_t* s;
    const int32_t* t;
    const double* eps;     // nullable: eps_scalar for every query
    double eps_scalar;
    double lambda, delta;
    double log_inv_lambda;  // log(1 / lambda) (used for 0 < lambda < 1): Eq. (6)'s denominator
    double log_2tau_delta;  // log(2 tau / delta): Eq. (8)'s logarithm at delta / tau
    int32_t tau, ell_formula, policy, fixed_lb;
    int64_t max_table;     // largest table a query may request (slots)
    // table pool: slots of every query-iteration table of the batch
    GEntry* ent;
    unsigned long long* sum_s;
    unsigned long long* sum_t;
    void* ys;              // T per slot
    void* yt;              // T per slot
    int64_t pool_cap;
    int64_t* heavy;        // per chunk of a high-degree frontier node: slot << 20 | chunk index
    int64_t heavy_cap;
    // dense engine (all queries of the launch when dense_engine != 0)
    int32_t dense_engine;
    int32_t dense_width;   // columns per dense block (2 per query)
    int32_t dense_fp64;
    void* dense_X[2];      // value buffers: block b at b * n * dense_width
    SmmCtl* ctl;
    int* err_flag;
    // hybrid engine: a sparse query whose next push has >= migrate_at pairs
    // moves to a free dense column (of dense_cap)
    int32_t hybrid = 0;
    int32_t dense_cap = 0;
    int64_t migrate_at = 0;
    int32_t* dense_block_q = nullptr;  // column -> query
    int32_t* mig_list = nullptr;       // queries moved by the current decision
    // learned switch (policy 1): input normalisation (mean[6], std[6]) and FP16 weights
    const float* mlp_norm = nullptr;
    const unsigned short* mlp_w = nullptr;  // null: no network, the rule of Eq. (17) decides
    const float* mlp_wt = nullptr;          // the same weights in FP32, W1 and W2 transposed (mlp_stage's layout)
    int32_t mlp_at_start = 0;               // also consult the network before the first SMM iteration
    // cost log: per query and SMM iteration 1..trace_steps, kTraceWidth floats
    float* trace = nullptr;
    int32_t trace_steps = 0;
    WalkQ* wq = nullptr;  // walk records, packed for the queries that enter AMC
    // per-query SMM length (nullable): query q runs min(lb_force[q], l) SMM
    // iterations when lb_force[q] >= 0, overriding the policy
    const int32_t* lb_force = nullptr;
};

// Columns of one cost-log row: the six switch inputs, the union frontier's
// volume (the next push's size) and Eq. (17)'s volume.
constexpr int kTraceWidth = 8;

// Per-warp partial sums of the dense SpMM epilogue, per query.
struct DensePartial {
    unsigned long long vp, vu, cnt;
    double s1, s2, t1, t2;
};

struct DenseArgs {
    DevGraph g;
    int32_t nblocks;
    int32_t width;          // columns per block (B)
    void* X[2];             // values (sign bit: support), nblocks * n * width each
    const int32_t* block_q; // nblocks * width/2: query of each column pair, -1: none
    int32_t* block_run;     // per block: 0 idle, 1 running, 2 running with full supports
    QState* st;
    QSmm* sm;
    DensePartial* part;     // nblocks * part_warps * width/2
    int32_t part_warps;     // warps of the SpMM grid per block (grid.x = part_warps / 8)
    SmmCtl* ctl;
    // balanced work units of the graph (built once per graph)
    const int4* units;      // light: {first row, end row, first edge, end edge}; heavy piece: {-h-1, piece, edges}
    int32_t nunits;
    const int4* heavy;      // per heavy row h: {row, first piece slot, pieces, degree}
    int32_t nheavy;
    int32_t nslots;         // piece slots per block
    unsigned int* unit_ctr; // per block: next unit
    unsigned int* heavy_ctr;// per block and heavy row: pieces done (reset by the finishing warp)
    void* pieces;           // per block: nslots * width partial sums
    int32_t fp64;           // element type of X
};

struct AmcArgs {
    DevGraph g;
    int32_t nq;
    QState* st;
    int64_t* chunk_begin;  // nq + 1: chunk prefix of the next walk launch (above kSmemChunkBegin - 1 queries)
    int32_t* chunk_count;  // nq: chunks per query of the next walk launch (up to kSmemChunkBegin - 1 queries)
    WalkQ* wq;             // nq walk records, packed by the schedule
    unsigned long long* walk_ctr;  // next chunk of the batch (reset by the schedule)
    unsigned int* done;    // CTA counter of the reduce (its last CTA lays out large batches)
    Partial* partial;
    int64_t partial_cap;
    const GEntry* pool;
    uint64_t seed;
    int32_t tau;
    int32_t batch;         // 1-based index b of the launch's first batch
    int32_t* group;        // batches walked by the first launch (set by the first schedule)
    int32_t dense_fp64;    // element type of dense-engine values
    double delta;
    double log_3tau_delta;  // log(3 tau / delta): Eq. (7)'s logarithm at delta / tau
    int* err_flag;
    // the first walk launch lays out its own chunks (batches of up to
    // kSmemChunkBegin - 1 queries; no schedule launch)
    int32_t fused_schedule = 0;
    // the last statistics launch (batch tau) also writes every query's outputs
    // (null: a separate finalize launch does)
    double* out_r = nullptr;
    ger_query_stats* out_stats = nullptr;
};

// host launchers (one per kernel)
// SMM phase, level-synchronous over the batch. The iteration number lives
// in the control block (device memory), so the launches of an iteration are
// the same every time and can sit in a graph's while loop.
//   start     : iteration 0 in closed form (sparse and hybrid engines): set-up,
//               the F_0 tables, the first decision, the F_1 tables
//   setup     : set-up alone (dense engine, whose F_0 lives in its blocks)
//   iteration : push (+ heavy push), finish, top2, decide (+ next tables)
//   advance   : clears the tables just handed out, iteration += 1, and
//               optionally sets the graph's while condition
void launch_smm_setup(const SmmArgs& a, cudaStream_t st);
void launch_smm_push(bool fp64, const SmmArgs& a, int grid, cudaStream_t st);
void launch_smm_finish(bool fp64, const SmmArgs& a, int grid, cudaStream_t st);
void launch_smm_top2(bool fp64, const SmmArgs& a, int grid, cudaStream_t st);
void launch_smm_decide(const SmmArgs& a, cudaStream_t st, bool first = false);
void launch_smm_advance(const SmmArgs& a, int grid, cudaGraphConditionalHandle h, bool use_handle, cudaStream_t st);
void launch_smm_start(bool fp64, const SmmArgs& a, cudaStream_t st);
void launch_smm_iteration(bool fp64, const SmmArgs& a, int grid, cudaStream_t st);
// the sparse part of one iteration (push .. top2), without the decision
void launch_smm_body(bool fp64, const SmmArgs& a, int grid, cudaStream_t st);
// the dense engine: iteration 0 and one pull-SpMM iteration (+ its epilogue)
bool dense_width_ok(int width, bool fp64);
int dense_prepare();  // cudaError_t of the shared-memory opt-in
void build_dense_units(int64_t n, const int64_t* row_ptr, std::vector<int4>* units, std::vector<int4>* heavy,
                       int32_t* nslots);
void launch_dense_map(const DenseArgs& d, int64_t nq, cudaStream_t st);
void launch_dense_init(bool fp64, const DenseArgs& d, cudaStream_t st);
void launch_dense_iteration(bool fp64, const DenseArgs& d, cudaStream_t st);
// hybrid engine: zero newly used dense blocks, then scatter the frontier
// tables of the queries the last decision moved into their dense columns
void launch_dense_migrate(bool fp64, const DenseArgs& d, const SmmArgs& a, cudaStream_t st);
void launch_amc_schedule(const AmcArgs& a, cudaStream_t st);
// edge e -> {col_idx[e], node_info[col_idx[e]], 0}
void launch_edge_records(const int32_t* col_idx, const uint2* node_info, int64_t nnz, uint4* out, cudaStream_t st);
// col_idx -> k entries of pack_bits(k) bits per 16-byte unit
void launch_pack_cols(const int32_t* col_idx, int64_t nnz, int k, uint4* out, cudaStream_t st);
// one persistent grid (as many CTAs as fit on the GPU) over the batch's chunks
void launch_amc_walk(const AmcArgs& a, int sm_count, cudaStream_t st);
// batch statistics of the launch's batches and the next launch's layout
void launch_amc_reduce(const AmcArgs& a, cudaStream_t st);

}  // namespace geer

namespace geer {

// host-side launch accounting (ger_launch_count)
void note_launches(int k);

// kernel families timed by the profiler
enum Family : int { FAM_SMM_SETUP = 0, FAM_SMM_ADVANCE, FAM_SMM_PUSH, FAM_SMM_PUSH_HEAVY, FAM_SMM_FINISH,
                    FAM_SMM_TOP2, FAM_SMM_DECIDE, FAM_DENSE_SPMM, FAM_AMC_SCHEDULE, FAM_AMC_WALK, FAM_AMC_REDUCE,
                    FAM_FINALIZE, FAM_LANCZOS, FAM_MLP_TRAIN, FAM_COUNT };
// bracket one launch on stream st with profiler events (no-op when off)
void prof_begin(int fam, cudaStream_t st);
void prof_end(int fam, cudaStream_t st);
// fold the recorded events of completed launches into the accumulators
void prof_collect();

// Convergence record of the spectral bound: whether the extreme Ritz values
// settled (or the Krylov space was exhausted) before the step limit, and the
// residual bounds beta_k |s_k| of the two extreme Ritz pairs.
struct LanczosInfo {
    int converged = 0;
    double resid_hi = 0.0, resid_lo = 0.0;
};

// Spectral bound of P on the device (Section 3.1). Returns 0 on success.
int lanczos_spectral_bound(const DevGraph& g, int max_steps, double tol, cudaStream_t st, double* lam2,
                           double* lamn, int* steps, LanczosInfo* info = nullptr);

}  // namespace geer

struct ger_graph;

namespace geer {

// accessors of api.cu for entry points in other translation units
int graph_view(const ger_graph* g, DevGraph* dg, double* lambda, bool* has_lambda, int* device, int* sm_count);
int set_error(int code, const char* msg);
// The FP32 copy of a switch network's FP16 weights that the decisions read.
void launch_mlp_expand(const unsigned short* w, float* out, cudaStream_t st);
void launch_finalize(const QState* st, int64_t nq, double* r, ger_query_stats* stats, cudaStream_t s);

}  // namespace geer
