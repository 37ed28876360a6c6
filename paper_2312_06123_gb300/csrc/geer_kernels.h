// geer_kernels.h -- launch arguments and kernel declarations of the GEER
// CUDA library (internal).
#pragma once

#include "geer_internal.cuh"

namespace geer {

struct SmmArgs {
    DevGraph g;
    int32_t nq;            // queries handled by this launch
    int32_t q_index_base;  // batch index of query 0 of this launch
    QState* st;            // nq records
    const int32_t* s;
    const int32_t* t;
    const double* eps;     // nullable: eps_scalar for every query
    double eps_scalar;
    double lambda, delta;
    int32_t tau, ell_formula, policy, fixed_lb;
    int32_t nbits;         // bits of the largest node id (radix passes)
    int64_t cap;           // push pairs per query iteration (sparse capacity)
    int32_t* scr_i32;      // per CTA: 5 cap + 3 (cap + 2) + 2 int32
    void* scr_val;         // per CTA: 4 (cap + 2) values
    uint8_t* scr_bits;     // per CTA: 2 (cap + 2) bytes
    GEntry* pool;          // lookup tables
    int64_t pool_cap;
    unsigned long long* pool_used;
    int* work_counter;
    int* err_flag;
};

struct AmcArgs {
    DevGraph g;
    int32_t nq;
    QState* st;
    int64_t* chunk_begin;  // nq + 1
    Partial* partial;
    int64_t partial_cap;
    const GEntry* pool;
    uint64_t seed;
    int32_t tau;
    int32_t batch;         // 1-based batch index b
    double delta;
    int* err_flag;
};

// host launchers (one per kernel)
void launch_smm_sparse(bool fp64, const SmmArgs& a, int grid, cudaStream_t st);
void launch_amc_schedule(const AmcArgs& a, cudaStream_t st);
void launch_amc_walk(const AmcArgs& a, int grid, cudaStream_t st);
void launch_amc_reduce(const AmcArgs& a, int grid, cudaStream_t st);

}  // namespace geer

namespace geer {

// host-side launch accounting (ger_launch_count)
void note_launches(int k);

// kernel families timed by the profiler
enum Family : int { FAM_SMM_SPARSE = 0, FAM_AMC_SCHEDULE, FAM_AMC_WALK, FAM_AMC_REDUCE, FAM_FINALIZE,
                    FAM_LANCZOS, FAM_COUNT };
// bracket one launch on stream st with profiler events (no-op when off)
void prof_begin(int fam, cudaStream_t st);
void prof_end(int fam, cudaStream_t st);
// fold the recorded events of completed launches into the accumulators
void prof_collect();

// Spectral bound of P on the device (Section 3.1). Returns 0 on success.
int lanczos_spectral_bound(const DevGraph& g, int max_steps, double tol, cudaStream_t st, double* lam2,
                           double* lamn, int* steps);

}  // namespace geer

struct ger_graph;
struct ger_query_stats;

namespace geer {

// accessors of api.cu for entry points in other translation units
int graph_view(const ger_graph* g, DevGraph* dg, double* lambda, bool* has_lambda, int* device, int* sm_count);
int set_error(int code, const char* msg);
void launch_finalize(const QState* st, int64_t nq, double* r, ger_query_stats* stats, cudaStream_t s);

}  // namespace geer
