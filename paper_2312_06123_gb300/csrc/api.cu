// api.cu -- the C ABI of include/geer.h: graph loading and validation,
// workspace management, and the launch sequence of a GEER query batch
// (Algorithm 3): SMM iterations on the sparse push, dense pull SpMM or hybrid
// engine with the switch of Eq. (17) (or the learned switch), then the AMC
// rounds of schedule -> walks -> batch statistics, then the per-query
// outputs; one batch shape is captured once as a CUDA graph. Also the
// autotuner and the learned switch's installation and cost log.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/geer.h"
#include "geer_internal.cuh"
#include "geer_kernels.h"

namespace geer {

static std::atomic<int64_t> g_launches{0};
static bool g_capturing = false;    // graph capture: launches are counted per replay instead
static int64_t g_captured = 0;      // kernels captured so far
constexpr int64_t kHeavyCap = 1 << 16;     // initial heavy-push list (chunk records)
constexpr int64_t kHeavyCapMax = 1 << 26;
void note_launches(int k) {
    if (g_capturing) g_captured += k;
    else g_launches.fetch_add(k, std::memory_order_relaxed);
}

// ---------------------------------------------------------------------------
// profiler: CUDA events around launches, on the launch stream
// ---------------------------------------------------------------------------
static const char* kFamilyNames[] = {"smm_setup", "smm_advance", "smm_push",
                                              "smm_push_heavy", "smm_finish", "smm_top2", "smm_decide", "dense_spmm",
                                              "amc_schedule", "amc_walk", "amc_reduce", "finalize", "lanczos",
                                     "mlp_train"};
static_assert(sizeof(kFamilyNames) / sizeof(kFamilyNames[0]) == FAM_COUNT, "one name per kernel family");
struct ProfRec {
    int fam;
    cudaEvent_t a, b;
};
static bool g_prof_on = false;
static bool g_prof_suspend = false;             // inside a graph's while body: no event records
static std::vector<ProfRec>* g_prof_sink = nullptr;  // graph capture: keep the records with the graph
static std::vector<ProfRec> g_prof_pending;
static std::vector<cudaEvent_t> g_prof_free;
static cudaEvent_t g_prof_open[FAM_COUNT];
static int64_t g_prof_launches[FAM_COUNT];
static double g_prof_ms[FAM_COUNT];

static cudaEvent_t prof_event() {
    if (!g_prof_free.empty()) {
        cudaEvent_t e = g_prof_free.back();
        g_prof_free.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Inside a graph capture the record must be an external event-record node,
// so that the event is really recorded each time the graph runs.
static void prof_record(cudaEvent_t e, cudaStream_t st) {
    if (g_prof_sink) cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
    else cudaEventRecord(e, st);
}

void prof_begin(int fam, cudaStream_t st) {
    if (!g_prof_on || g_prof_suspend) return;
    g_prof_open[fam] = prof_event();
    prof_record(g_prof_open[fam], st);
}

void prof_end(int fam, cudaStream_t st) {
    if (!g_prof_on || g_prof_suspend || !g_prof_open[fam]) return;
    cudaEvent_t b = prof_event();
    prof_record(b, st);
    (g_prof_sink ? *g_prof_sink : g_prof_pending).push_back({fam, g_prof_open[fam], b});
    g_prof_open[fam] = nullptr;
}

// fold the records kept by a replayed graph (after it has completed)
static void prof_collect_graph(const std::vector<ProfRec>& recs) {
    if (!g_prof_on) return;
    for (const ProfRec& r : recs) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            g_prof_ms[r.fam] += ms;
            g_prof_launches[r.fam] += 1;
        } else {
            cudaGetLastError();
        }
    }
}

void prof_collect() {
    for (const ProfRec& r : g_prof_pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            g_prof_ms[r.fam] += ms;
            g_prof_launches[r.fam] += 1;
        }
        g_prof_free.push_back(r.a);
        g_prof_free.push_back(r.b);
    }
    g_prof_pending.clear();
}

static thread_local char g_err[512] = "";

static int fail(int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

static int cuda_fail(cudaError_t e, const char* what) {
    return fail(GER_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define GER_CUDA(call)                                          \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);     \
    } while (0)

// ---------------------------------------------------------------------------
// workspace
// ---------------------------------------------------------------------------
struct Workspace {
    int64_t q_cap = 0;
    QState* st = nullptr;
    int32_t* s = nullptr;
    int32_t* t = nullptr;
    double* eps = nullptr;
    double* r = nullptr;
    ger_query_stats* stats = nullptr;
    int64_t* chunk_begin = nullptr;
    int32_t* chunk_count = nullptr;
    int32_t* lbf = nullptr;       // per-query forced SMM lengths (ger_query_batch_lb)
    WalkQ* wq = nullptr;
    Partial* partial = nullptr;
    int64_t partial_cap = 0;
    // SMM phase
    QSmm* qsmm = nullptr;
    int64_t* heavy = nullptr;     // heavy_cap chunk records of the heavy push
    int64_t heavy_cap = 0;
    SmmCtl* ctl = nullptr;
    // frontier-table pool (also the walk lookup tables)
    GEntry* ent = nullptr;
    unsigned long long* sums = nullptr;  // 2 pool_cap
    double* yvals = nullptr;             // 2 pool_cap values (T = float or double)
    int64_t pool_cap = 0;
    // dense engine
    void* dX[2] = {nullptr, nullptr};
    int32_t* dblock_q = nullptr;
    int32_t* dblock_run = nullptr;
    unsigned int* dunit_ctr = nullptr;
    unsigned int* dheavy_ctr = nullptr;
    void* dpieces = nullptr;
    DensePartial* dpart = nullptr;
    size_t dX_bytes = 0, dpart_n = 0, dpieces_bytes = 0, dheavy_ctr_n = 0;
    int64_t dblock_q_n = 0;
    int32_t* dmig = nullptr;          // hybrid engine: queries moved by one decision
    int64_t dmig_n = 0;
    int64_t dblock_n = 0;             // blocks the per-block arrays hold
    uint64_t gen = 0;                 // bumped by every (re)allocation: captured graphs go stale
    // counters: [1] error flag (int), [2] AMC done counter
    int* counters = nullptr;
    // pinned readback
    int64_t* host_rb = nullptr;
};

}  // namespace geer

namespace geer {
// The captured launch sequence of one batch shape (see run_batch).
struct BatchGraph {
    bool valid = false;
    int64_t nq = 0;
    bool fp64 = false;
    ger_options o{};
    double lambda = 0;
    const void* pool = nullptr;
    const void* state = nullptr;
    const void* dense = nullptr;
    int dense_w = 0;
    bool prof = false;
    int64_t launches = 0;       // kernels outside the while body
    int64_t body_launches = 0;  // kernels per pass of the while body
    bool mlp = false;           // captured with the learned switch's kernel
    int64_t dense_cols = 0;     // dense columns of the captured engine
    const void* dense_dev = nullptr;  // dense column map and move list the capture uses
    const void* mig = nullptr;
    uint64_t gen = 0;                 // workspace generation the capture saw
    bool forced = false;              // captured with per-query SMM lengths
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<ProfRec> prof_recs;
};
}  // namespace geer

struct ger_graph {
    int device = 0;
    int sm_count = 0;
    int64_t n = 0, nnz = 0;
    int64_t* row_ptr = nullptr;
    int32_t* col_idx = nullptr;
    uint2* node_info = nullptr;  // {first edge, degree} per node when nnz < 2^32
    uint4* edge_rec = nullptr;   // {neighbour, its first edge, its degree, 0} per edge (walks)
    uint4* cols_packed = nullptr; // the walks' packed copy of col_idx (pack_k entries per 16 B)
    int pack_k = 0;
    bool has_lambda = false;
    double lambda = 0, lam2 = 0, lamn = 0;
    // how lambda was obtained: Lanczos steps (0: set by the caller), whether
    // the extreme Ritz values converged, and their residual bounds
    int lam_steps = 0, lam_converged = 1;
    double lam_resid_hi = 0.0, lam_resid_lo = 0.0;
    cudaStream_t stream = nullptr;
    cudaStream_t stream2 = nullptr;  // captures the SMM while body
    int dense_tuned[2] = {0, 0};     // autotuned dense block width (FP32, FP64), 0: not tuned
    int64_t hybrid_tuned = 0;        // autotuned hybrid switch size (push pairs), 0: not tuned
    int tau_tuned = 0;               // autotuned tau (AMC batches), 0: not tuned
    int dense_ctas = 0;              // dense SpMM CTAs per SM and block, 0: default
    int4* dense_units = nullptr;     // dense SpMM work units (null when nnz >= 2^32)
    int4* dense_heavy = nullptr;     // dense SpMM heavy rows
    int32_t dense_nunits = 0, dense_nheavy = 0, dense_nslots = 0;
    bool dense_ready = false;        // SpMM kernels opted into their shared memory
    unsigned short* mlp_w = nullptr; // learned switch: FP16 weights (null: none installed)
    float* mlp_wt = nullptr;         // learned switch: the same weights in FP32, as the decisions read them
    float* mlp_norm = nullptr;       // learned switch: input mean[6], std[6]
    geer::Workspace ws;
    geer::BatchGraph bg;
};

namespace geer {

// The device view of a loaded graph.
static DevGraph dev_graph(const ger_graph* g) {
    DevGraph d{g->n, g->nnz, g->row_ptr, g->col_idx, g->node_info, g->edge_rec};
    d.cols_packed = g->cols_packed;
    d.pack_k = g->cols_packed ? g->pack_k : 0;
    return d;
}

static void free_ws(Workspace& w) {
    cudaFree(w.st); cudaFree(w.s); cudaFree(w.t); cudaFree(w.eps); cudaFree(w.r); cudaFree(w.stats);
    cudaFree(w.chunk_begin); cudaFree(w.partial); cudaFree(w.qsmm);
    cudaFree(w.wq); cudaFree(w.chunk_count); cudaFree(w.lbf);
    cudaFree(w.ctl); cudaFree(w.ent); cudaFree(w.sums); cudaFree(w.yvals); cudaFree(w.counters);
    cudaFree(w.heavy);
    cudaFree(w.dX[0]); cudaFree(w.dX[1]);
    cudaFree(w.dblock_q); cudaFree(w.dblock_run); cudaFree(w.dunit_ctr); cudaFree(w.dheavy_ctr);
    cudaFree(w.dpieces); cudaFree(w.dpart); cudaFree(w.dmig);
    if (w.host_rb) cudaFreeHost(w.host_rb);
    w = Workspace();
}

// Testing hook (ger_test_fail_alloc): the countdown-th next workspace
// allocation reports failure without calling cudaMalloc.
static std::atomic<int64_t> g_fail_alloc_countdown{0};

template <typename T>
static cudaError_t alloc(T** p, size_t count) {
    if (g_fail_alloc_countdown.load(std::memory_order_relaxed) > 0 &&
        g_fail_alloc_countdown.fetch_sub(1) == 1) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T) + 16);
}

// Make room for q queries and a frontier-table pool of at least pool_cap slots.
static int ensure_ws(ger_graph* g, int64_t q, int64_t pool_cap) {
    Workspace& w = g->ws;
    if (!w.counters) {
        GER_CUDA(alloc(&w.counters, 8));  // [1] error flag, [2] reduce CTA counter, [4..5] walk ticket, [6] AMC group
        GER_CUDA(alloc(&w.ctl, 1));
        GER_CUDA(alloc(&w.heavy, kHeavyCap));
        w.heavy_cap = kHeavyCap;
        GER_CUDA(cudaMallocHost(reinterpret_cast<void**>(&w.host_rb), 4 * sizeof(int64_t)));
    }
    if (q > w.q_cap) {
        cudaFree(w.st); cudaFree(w.s); cudaFree(w.t); cudaFree(w.eps); cudaFree(w.r); cudaFree(w.stats);
        cudaFree(w.chunk_begin); cudaFree(w.partial); cudaFree(w.qsmm);
        cudaFree(w.wq); cudaFree(w.chunk_count); cudaFree(w.lbf);
        w.lbf = nullptr;
        w.st = nullptr; w.s = nullptr; w.t = nullptr; w.eps = nullptr; w.r = nullptr; w.stats = nullptr;
        w.chunk_begin = nullptr; w.partial = nullptr; w.qsmm = nullptr;
        w.wq = nullptr; w.chunk_count = nullptr;
        w.q_cap = 0;
        const int64_t qc = std::max<int64_t>(q, 64);
        const int64_t pc = qc * kMaxChunksPerQuery;
        if (alloc(&w.st, qc) || alloc(&w.s, qc) || alloc(&w.t, qc) || alloc(&w.eps, qc) || alloc(&w.r, qc) ||
            alloc(&w.stats, qc) || alloc(&w.chunk_begin, qc + 1) || alloc(&w.partial, pc) ||
            alloc(&w.qsmm, qc) || alloc(&w.wq, qc) ||
            alloc(&w.chunk_count, qc) || alloc(&w.lbf, qc)) {
            cudaGetLastError();
            return fail(GER_ERR_OOM, "workspace for %lld queries", (long long)q);
        }
        w.q_cap = qc;
        ++w.gen;
        w.partial_cap = pc;
    }
    if (pool_cap > w.pool_cap) {
        cudaFree(w.ent); cudaFree(w.sums); cudaFree(w.yvals);
        w.ent = nullptr; w.sums = nullptr; w.yvals = nullptr; w.pool_cap = 0;
        if (alloc(&w.ent, pool_cap) || alloc(&w.sums, 2 * pool_cap) || alloc(&w.yvals, 2 * pool_cap)) {
            cudaGetLastError();
            return fail(GER_ERR_OOM, "frontier-table pool of %lld slots", (long long)pool_cap);
        }
        w.pool_cap = pool_cap;
        ++w.gen;
    }
    return GER_OK;
}

// ---------------------------------------------------------------------------
// outputs
// ---------------------------------------------------------------------------
__global__ void finalize_kernel(const QState* st, int64_t nq, double* r, ger_query_stats* stats) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nq; q += (int64_t)gridDim.x * blockDim.x)
        store_outputs(st[q], q, r, stats);
}

// ---------------------------------------------------------------------------
// graph validation (host)
// ---------------------------------------------------------------------------
static int validate_csr(int64_t n, const int64_t* rp, const int32_t* ci) {
    if (n < 3) return fail(GER_ERR_INVALID, "n = %lld: a connected non-bipartite graph needs n >= 3", (long long)n);
    if (rp[0] != 0) return fail(GER_ERR_CSR, "row_ptr[0] != 0");
    for (int64_t v = 0; v < n; ++v)
        if (rp[v + 1] < rp[v]) return fail(GER_ERR_CSR, "row_ptr decreases at %lld", (long long)v);
    // sorted, in range, no self-loop, no duplicate
    for (int64_t v = 0; v < n; ++v) {
        for (int64_t e = rp[v]; e < rp[v + 1]; ++e) {
            const int64_t u = ci[e];
            if (u < 0 || u >= n) return fail(GER_ERR_CSR, "col_idx[%lld] = %lld out of range", (long long)e, (long long)u);
            if (u == v) return fail(GER_ERR_CSR, "self-loop at node %lld", (long long)v);
            if (e > rp[v] && ci[e - 1] >= u)
                return fail(GER_ERR_CSR, "row %lld not strictly increasing (unsorted or duplicate)", (long long)v);
        }
    }
    // symmetry: scanning rows in ascending order, the entries below the
    // diagonal of each row v must be exactly the rows u < v that list v
    std::vector<int64_t> cursor(rp, rp + n);
    for (int64_t u = 0; u < n; ++u) {
        for (int64_t e = rp[u]; e < rp[u + 1]; ++e) {
            const int64_t v = ci[e];
            if (v <= u) continue;
            const int64_t c = cursor[v];
            if (c >= rp[v + 1] || ci[c] != u)
                return fail(GER_ERR_CSR, "edge (%lld,%lld) has no reverse entry", (long long)u, (long long)v);
            cursor[v] = c + 1;
        }
    }
    for (int64_t v = 0; v < n; ++v)
        if (cursor[v] < rp[v + 1] && ci[cursor[v]] < v)
            return fail(GER_ERR_CSR, "edge (%lld,%d) has no reverse entry", (long long)v, ci[cursor[v]]);
    // connectivity and bipartiteness by breadth-first two-colouring
    std::vector<int8_t> colour(n, -1);
    std::vector<int32_t> queue(n);
    int64_t head = 0, tail = 0;
    colour[0] = 0;
    queue[tail++] = 0;
    bool odd_cycle = false;
    while (head < tail) {
        const int32_t v = queue[head++];
        for (int64_t e = rp[v]; e < rp[v + 1]; ++e) {
            const int32_t u = ci[e];
            if (colour[u] < 0) {
                colour[u] = (int8_t)(1 - colour[v]);
                queue[tail++] = u;
            } else if (colour[u] == colour[v]) {
                odd_cycle = true;
            }
        }
    }
    if (tail != n) return fail(GER_ERR_DISCONNECTED, "graph is not connected (%lld of %lld nodes reachable from 0)",
                               (long long)tail, (long long)n);
    if (!odd_cycle) return fail(GER_ERR_BIPARTITE, "graph is bipartite: lambda_n = -1 and Eq. (6) is undefined");
    return GER_OK;
}

static int ensure_lambda(ger_graph* g) {
    if (g->has_lambda) return GER_OK;
    DevGraph dg = dev_graph(g);
    double l2 = 0, ln = 0;
    int steps = 0;
    LanczosInfo info;
    const int rc = lanczos_spectral_bound(dg, 300, 1e-13, g->stream, &l2, &ln, &steps, &info);
    if (rc == -2) return fail(GER_ERR_OOM, "spectral bound workspace");
    if (rc != 0) return fail(GER_ERR_CUDA, "spectral bound: %s", cudaGetErrorString(cudaGetLastError()));
    g->lam2 = l2;
    g->lamn = ln;
    g->lam_steps = steps;
    g->lam_converged = info.converged;
    g->lam_resid_hi = info.resid_hi;
    g->lam_resid_lo = info.resid_lo;
    if (info.converged) {
        g->lambda = std::max(std::fabs(l2), std::fabs(ln));
    } else {
        // Ritz values lie inside the spectrum (Cauchy interlacing), so an
        // unconverged one underestimates |lambda_2| or |lambda_n| and Eq. (6)
        // would give too short an l: widen each by its residual bound (an
        // eigenvalue lies within it)
        g->lambda = std::max(std::fabs(l2) + info.resid_hi, std::fabs(ln) + info.resid_lo);
    }
    if (!(g->lambda < 1.0)) return fail(GER_ERR_BIPARTITE, "spectral bound lambda = %.17g >= 1", g->lambda);
    g->has_lambda = true;
    return GER_OK;
}

// ---------------------------------------------------------------------------
// the query batch
// ---------------------------------------------------------------------------
struct Plan {
    ger_options o;
    int64_t q;
    const int32_t* s;     // device
    const int32_t* t;     // device
    const double* eps;    // device, nullable
    double eps_scalar;
    double* r;            // device
    ger_query_stats* stats;  // device, nullable
    cudaStream_t st;
    float* trace = nullptr;  // device cost log (stream-ordered runs only), nullable
    int32_t trace_steps = 0;
    const int32_t* lb_force = nullptr;  // device per-query SMM lengths, nullable
};


static int map_device_error(int e) {
    switch (e) {
        case DERR_NODE_RANGE: return fail(GER_ERR_NODE_RANGE, "a query node is outside [0, n) or eps <= 0");
        case DERR_CAPACITY: return fail(GER_ERR_CAPACITY, "an SMM iteration needs a frontier table beyond the limit");
        case DERR_TABLE: return fail(GER_ERR_CAPACITY, "frontier-table pool exhausted");
        case DERR_ELL: return fail(GER_ERR_INVALID, "truncation length undefined (lambda >= 1)");
        case DERR_FULL: return fail(GER_ERR_CAPACITY, "a frontier table ran out of free slots (load factor broken)");
        case DERR_CHUNKS: return fail(GER_ERR_CUDA, "a walk launch's chunk layout exceeded the partial-sum array");
        default: return fail(GER_ERR_CUDA, "device error %d", e);
    }
}

// Dense-engine block width: the option, else the autotuned choice of the
// graph, else the widest block.
static int dense_width_for(ger_graph* g, const ger_options& o) {
    const bool fp64 = o.precision == GER_FP64;
    if (o.dense_width) return o.dense_width;
    const int tuned = fp64 ? g->dense_tuned[1] : g->dense_tuned[0];
    return tuned ? tuned : (fp64 ? 64 : 128);
}

// Warps of the dense SpMM grid per block (one partial slot each).
static int dense_part_warps(const ger_graph* g) {
    int c = g->dense_ctas;
    if (c <= 0) {
        const char* v = std::getenv("GEER_DENSE_CTAS");
        c = v ? std::atoi(v) : 0;
    }
    if (c <= 0 || c > 8) c = 2;
    return g->sm_count * c * 8;
}

// Make room for the dense engine's blocks (nq queries at `width` columns).
static int ensure_dense(ger_graph* g, int64_t nq, int width, bool fp64) {
    Workspace& w = g->ws;
    if (!g->dense_units) return fail(GER_ERR_INVALID, "the dense engine needs fewer than 2^32 stored edges");
    if (!g->dense_ready) {
        const int e = dense_prepare();
        if (e) return cuda_fail((cudaError_t)e, "dense SpMM shared-memory opt-in");
        g->dense_ready = true;
    }
    const int64_t qpb = width / 2;
    const int64_t nblocks = (nq + qpb - 1) / qpb;
    const size_t esz = fp64 ? 8 : 4;
    const size_t xb = (size_t)nblocks * (size_t)g->n * (size_t)width * esz;
    const int part_warps = dense_part_warps(g);
    const size_t pn = (size_t)nblocks * (size_t)part_warps * (size_t)qpb;
    const size_t pb = std::max<size_t>((size_t)nblocks * (size_t)g->dense_nslots * (size_t)width * esz, 16);
    const size_t hn = std::max<size_t>((size_t)nblocks * (size_t)g->dense_nheavy, 1);
    if (xb > w.dX_bytes) {
        cudaFree(w.dX[0]); cudaFree(w.dX[1]);
        w.dX[0] = w.dX[1] = nullptr;
        w.dX_bytes = 0;
        if (cudaMalloc(&w.dX[0], xb) != cudaSuccess || cudaMalloc(&w.dX[1], xb) != cudaSuccess) {
            cudaGetLastError();
            return fail(GER_ERR_OOM, "dense blocks (%zu bytes each)", xb);
        }
        w.dX_bytes = xb;
        ++w.gen;
    }
    if (pb > w.dpieces_bytes) {
        cudaFree(w.dpieces);
        w.dpieces = nullptr;
        w.dpieces_bytes = 0;
        if (cudaMalloc(&w.dpieces, pb) != cudaSuccess) {
            cudaGetLastError();
            return fail(GER_ERR_OOM, "dense heavy-row pieces");
        }
        w.dpieces_bytes = pb;
        ++w.gen;
    }
    if (hn > w.dheavy_ctr_n) {
        cudaFree(w.dheavy_ctr);
        w.dheavy_ctr = nullptr;
        w.dheavy_ctr_n = 0;
        // zero once: the warp that finishes a heavy row resets its counter
        if (alloc(&w.dheavy_ctr, hn) || cudaMemset(w.dheavy_ctr, 0, hn * sizeof(unsigned int))) {
            cudaGetLastError();
            return fail(GER_ERR_OOM, "dense heavy-row counters");
        }
        w.dheavy_ctr_n = hn;
        ++w.gen;
    }
    if (pn > w.dpart_n) {
        cudaFree(w.dpart);
        w.dpart = nullptr;
        w.dpart_n = 0;
        if (alloc(&w.dpart, pn)) {
            cudaGetLastError();
            return fail(GER_ERR_OOM, "dense partials");
        }
        w.dpart_n = pn;
        ++w.gen;
    }
    const int64_t nbq = nblocks * qpb;
    if (nbq > w.dblock_q_n || nblocks > w.dblock_n) {
        const int64_t nq_alloc = std::max(nbq, w.dblock_q_n), nb_alloc = std::max<int64_t>(nblocks, w.dblock_n);
        cudaFree(w.dblock_q); cudaFree(w.dblock_run); cudaFree(w.dunit_ctr);
        w.dblock_q = nullptr; w.dblock_run = nullptr; w.dunit_ctr = nullptr; w.dblock_q_n = 0; w.dblock_n = 0;
        if (alloc(&w.dblock_q, nq_alloc) || alloc(&w.dblock_run, nb_alloc) || alloc(&w.dunit_ctr, nb_alloc)) {
            cudaGetLastError();
            return fail(GER_ERR_OOM, "dense block map");
        }
        w.dblock_q_n = nq_alloc;
        w.dblock_n = nb_alloc;
        ++w.gen;
    }
    return GER_OK;
}

static DenseArgs make_dense_args(ger_graph* g, int64_t q0, int64_t nq, int width, bool fp64) {
    Workspace& w = g->ws;
    DenseArgs d;
    d.g = dev_graph(g);
    d.width = width;
    d.nblocks = (int32_t)((nq + width / 2 - 1) / (width / 2));
    d.X[0] = w.dX[0];
    d.X[1] = w.dX[1];
    d.block_q = w.dblock_q;
    d.block_run = w.dblock_run;
    d.st = w.st + q0;
    d.sm = w.qsmm + q0;
    d.part = w.dpart;
    d.part_warps = dense_part_warps(g);
    d.ctl = w.ctl;
    d.units = g->dense_units;
    d.nunits = g->dense_nunits;
    d.heavy = g->dense_heavy;
    d.nheavy = g->dense_nheavy;
    d.nslots = g->dense_nslots;
    d.unit_ctr = w.dunit_ctr;
    d.heavy_ctr = w.dheavy_ctr;
    d.pieces = w.dpieces;
    d.fp64 = fp64 ? 1 : 0;

    return d;
}

// Start of the dense engine for nq queries: empty blocks, the column map,
// iteration 0 (stream-ordered; capturable).
static void issue_dense_start(ger_graph* g, const DenseArgs& d, bool fp64, int64_t nq, cudaStream_t st) {
    Workspace& w = g->ws;
    const size_t xb = (size_t)d.nblocks * (size_t)g->n * (size_t)d.width * (fp64 ? 8 : 4);
    // buffer 0 starts as zeros plus e_s, e_t; buffer 1 is written in full by
    // iteration 1 in every column that is ever read
    cudaMemsetAsync(w.dX[0], 0, xb, st);
    launch_dense_map(d, nq, st);
    launch_dense_init(fp64, d, st);
}

// Launch arguments of the SMM and AMC phases for queries [q0, q0 + nq).
static void make_args(ger_graph* g, const Plan& p, int64_t q0, int64_t nq, bool fp64, SmmArgs* pa, AmcArgs* pm) {
    Workspace& w = g->ws;
    DevGraph dg = dev_graph(g);
    SmmArgs& a = *pa;
    a.g = dg;
    a.nq = (int32_t)nq;
    a.q_index_base = (int32_t)q0;
    a.st = w.st + q0;
    a.sm = w.qsmm + q0;
    a.s = p.s + q0;
    a.t = p.t + q0;
    a.eps = p.eps ? p.eps + q0 : nullptr;
    a.eps_scalar = p.eps_scalar;
    a.lambda = g->lambda;
    a.log_inv_lambda = a.lambda > 0.0 && a.lambda < 1.0 ? std::log(1.0 / a.lambda) : 0.0;
    a.delta = p.o.delta;
    a.tau = p.o.tau;
    a.log_2tau_delta = std::log(2.0 * (double)a.tau / a.delta);
    a.ell_formula = p.o.ell_formula;
    a.policy = p.o.switch_policy;
    a.fixed_lb = p.o.fixed_ell_b;
    if (p.o.sparse_cap > 0) {
        int64_t cap = 16;
        while (cap < 2 * p.o.sparse_cap) cap <<= 1;
        a.max_table = cap;
    } else {
        // a table holds at most n nodes (capacity < 4n); a pool too small for it
        // grows and the batch reruns, so only sparse_cap bounds a table
        a.max_table = (int64_t)1 << 40;
    }
    a.ent = w.ent;
    a.sum_s = w.sums;
    a.sum_t = w.sums + w.pool_cap;
    a.ys = w.yvals;
    a.yt = fp64 ? (void*)(w.yvals + w.pool_cap) : (void*)(reinterpret_cast<float*>(w.yvals) + w.pool_cap);
    a.pool_cap = w.pool_cap;
    a.heavy = w.heavy;
    a.heavy_cap = w.heavy_cap;
    a.dense_engine = p.o.smm_engine == GER_ENGINE_DENSE;
    a.dense_width = a.dense_engine ? dense_width_for(g, p.o) : 2;
    a.dense_fp64 = fp64;
    a.dense_X[0] = w.dX[0];
    a.dense_X[1] = w.dX[1];
    a.ctl = w.ctl;
    a.err_flag = w.counters + 1;
    a.wq = w.wq + q0;
    a.mlp_norm = g->mlp_norm;
    a.mlp_w = p.o.switch_policy == GER_SWITCH_MLP ? g->mlp_w : nullptr;
    a.mlp_wt = g->mlp_wt;
    a.mlp_at_start = p.o.mlp_at_start != 0;
    a.trace = p.trace ? p.trace + q0 * (int64_t)p.trace_steps * kTraceWidth : nullptr;
    a.trace_steps = p.trace_steps;
    a.lb_force = p.lb_force ? p.lb_force + q0 : nullptr;
    AmcArgs& m = *pm;
    m.g = dg;
    m.nq = (int32_t)nq;
    m.st = w.st + q0;
    m.chunk_begin = w.chunk_begin;
    m.chunk_count = w.chunk_count;
    m.wq = w.wq + q0;
    m.walk_ctr = reinterpret_cast<unsigned long long*>(w.counters + 4);
    m.group = w.counters + 6;
    m.done = reinterpret_cast<unsigned int*>(w.counters + 2);
    m.partial = w.partial;
    m.partial_cap = w.partial_cap;
    m.pool = w.ent;
    m.seed = p.o.seed;
    m.tau = p.o.tau;
    m.delta = p.o.delta;
    m.log_3tau_delta = std::log(3.0 * (double)m.tau / m.delta);
    m.dense_fp64 = fp64;
    m.err_flag = w.counters + 1;
}

// The tau AMC rounds (schedule -> walks -> batch statistics).
// The AMC rounds: one walk launch and one statistics launch per batch; the
// first schedule may fold the first batches into the first launch (the later
// launches of those batches then return at once).
// Batches of up to 4,095 queries need no schedule launch: the first walk
// launch lays out its own chunks. With m.out_r set, the last statistics
// launch writes the outputs.
static void issue_amc(ger_graph* g, AmcArgs m, int64_t nq, cudaStream_t st) {
    m.batch = 1;
    m.fused_schedule = nq + 1 <= 4096 ? 1 : 0;
    if (!m.fused_schedule) {
        launch_amc_schedule(m, st);
        note_launches(1);
    }
    for (int b = 1; b <= m.tau; ++b) {
        m.batch = b;
        launch_amc_walk(m, g->sm_count, st);
        launch_amc_reduce(m, st);  // it also lays out the next launch
    }
    note_launches(2 * m.tau);
}

// Dense columns of the hybrid engine for a batch of nq queries: as many
// query column pairs as the memory budget holds, at most nq.
static int64_t hybrid_columns(const ger_graph* g, const ger_options& o, int64_t nq) {
    int64_t budget = (int64_t)o.dense_budget_mb << 20;
    if (budget <= 0) {
        // default: half of the free device memory (dense buffers already held count as free)
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
            cudaGetLastError();
            fr = 0;
        }
        budget = ((int64_t)fr + 2 * (int64_t)g->ws.dX_bytes) / 2;
    }
    // a query holds two columns (s*, t*) in each of the two buffers
    const int64_t per = 4 * g->n * (o.precision == GER_FP64 ? 8 : 4);
    return std::min<int64_t>(nq, budget / std::max<int64_t>(per, 1));
}

// Launch arguments of one batch (or one query) and its SMM engine.
struct Engine {
    SmmArgs a;
    AmcArgs m;
    DenseArgs d{};
    bool dense = false, hybrid = false;
    int grid = 0;
    int64_t cols = 0;  // dense columns
};

static int prepare_engine(ger_graph* g, const Plan& p, int64_t q0, int64_t nq, bool fp64, Engine* E) {
    Workspace& w = g->ws;
    make_args(g, p, q0, nq, fp64, &E->a, &E->m);
    E->grid = g->sm_count * 8;
    E->dense = p.o.smm_engine == GER_ENGINE_DENSE;
    E->hybrid = p.o.smm_engine == GER_ENGINE_HYBRID;
    SmmArgs& a = E->a;
    if (!E->dense && !E->hybrid) return GER_OK;
    a.dense_width = dense_width_for(g, p.o);
    E->cols = E->dense ? nq : hybrid_columns(g, p.o, nq);
    if (E->hybrid && (E->cols == 0 || !g->dense_units)) {
        a.hybrid = 0;  // no room (or no work units) for dense columns: sparse only
        E->hybrid = false;
        return GER_OK;
    }
    int rc = ensure_dense(g, E->cols, a.dense_width, fp64);
    if (rc) return rc;
    if (E->hybrid) {
        if (nq > w.dmig_n) {
            cudaFree(w.dmig);
            w.dmig = nullptr;
            w.dmig_n = 0;
            if (alloc(&w.dmig, nq)) {
                cudaGetLastError();
                return fail(GER_ERR_OOM, "hybrid move list");
            }
            w.dmig_n = nq;
            ++w.gen;
        }
        a.hybrid = 1;
        a.dense_cap = (int32_t)E->cols;
        a.migrate_at = p.o.dense_switch > 0 ? p.o.dense_switch
                       : g->hybrid_tuned > 0 ? g->hybrid_tuned
                                             : std::max<int64_t>(g->nnz / 16, 1);
        a.dense_block_q = w.dblock_q;
        a.mig_list = w.dmig;
    }
    a.dense_X[0] = w.dX[0];
    a.dense_X[1] = w.dX[1];
    E->d = make_dense_args(g, q0, E->cols, a.dense_width, fp64);
    return GER_OK;
}

// Iteration 0 of the SMM phase (everything before the first advance).
static void issue_smm_start(ger_graph* g, Engine& E, bool fp64, cudaStream_t st) {
    if (E.dense) {
        launch_smm_setup(E.a, st);
        issue_dense_start(g, E.d, fp64, E.cols, st);
        launch_smm_decide(E.a, st, true);
    } else {
        if (E.hybrid) cudaMemsetAsync(g->ws.dblock_q, 0xff, E.d.nblocks * (size_t)(E.d.width / 2) * sizeof(int32_t), st);
        launch_smm_start(fp64, E.a, st);
        if (E.hybrid) launch_dense_migrate(fp64, E.d, E.a, st);
    }
}

// One further SMM iteration (everything before its advance).
static void issue_smm_iteration(Engine& E, bool fp64, cudaStream_t st) {
    if (E.dense) {
        launch_dense_iteration(fp64, E.d, st);
        launch_smm_decide(E.a, st);
    } else if (E.hybrid) {
        launch_smm_body(fp64, E.a, E.grid, st);
        launch_dense_iteration(fp64, E.d, st);
        launch_smm_decide(E.a, st);
        launch_dense_migrate(fp64, E.d, E.a, st);
    } else {
        launch_smm_iteration(fp64, E.a, E.grid, st);
    }
}

// The GEER launch sequence for queries [q0, q0 + nq), stream-ordered, with
// one host round trip per SMM iteration to learn whether any query
// continues; with `outputs`, its last launch writes r and the statistics.
static int run_queries(ger_graph* g, const Plan& p, int64_t q0, int64_t nq, bool fp64, bool outputs) {
    Workspace& w = g->ws;
    Engine E;
    int rc = prepare_engine(g, p, q0, nq, fp64, &E);
    if (rc) return rc;
    issue_smm_start(g, E, fp64, p.st);
    launch_smm_advance(E.a, E.grid, 0, false, p.st);
    int32_t* n_go = reinterpret_cast<int32_t*>(w.host_rb + 2);
    for (int iter = 1; iter < 100000; ++iter) {
        GER_CUDA(cudaMemcpyAsync(n_go, &w.ctl->n_go, sizeof(int32_t), cudaMemcpyDeviceToHost, p.st));
        GER_CUDA(cudaStreamSynchronize(p.st));
        if (*n_go == 0) break;
        issue_smm_iteration(E, fp64, p.st);
        launch_smm_advance(E.a, E.grid, 0, false, p.st);
    }
    if (outputs) {
        E.m.out_r = p.r + q0;
        E.m.out_stats = p.stats ? p.stats + q0 : nullptr;
    }
    issue_amc(g, E.m, nq, p.st);
    return GER_OK;
}

static void destroy_graph(BatchGraph& bg) {
    if (bg.exec) cudaGraphExecDestroy(bg.exec);
    if (bg.graph) cudaGraphDestroy(bg.graph);
    for (const ProfRec& r : bg.prof_recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    bg = BatchGraph();
}

static bool same_key(const BatchGraph& bg, const Plan& p, bool fp64, const ger_graph* g) {
    return bg.valid && bg.nq == p.q && bg.fp64 == fp64 && std::memcmp(&bg.o, &p.o, sizeof(ger_options)) == 0 &&
           bg.lambda == g->lambda && bg.pool == g->ws.ent && bg.state == g->ws.st && bg.prof == g_prof_on &&
           bg.dense == g->ws.dX[0] && bg.dense_w == (p.o.smm_engine ? dense_width_for(const_cast<ger_graph*>(g), p.o) : 0) &&
           bg.dense_dev == g->ws.dblock_q && bg.mig == g->ws.dmig && bg.gen == g->ws.gen &&
           bg.mlp == (g->mlp_w != nullptr) && bg.forced == (p.lb_force != nullptr);
}

// Capture the whole batch as one graph: the initial SMM iteration, a
// conditional while node over the further SMM iterations (its condition
// set on the device by the advance kernel), the tau AMC rounds and the
// outputs. The plan must read its inputs from, and write its outputs to,
// the workspace buffers, so that one capture serves every batch of the
// same shape.
static int build_graph(ger_graph* g, const Plan& p, bool fp64) {
    BatchGraph& bg = g->bg;
    destroy_graph(bg);
    Workspace& w = g->ws;
    cudaStream_t st = g->stream, st2 = g->stream2;
    Engine E;
    int rc = prepare_engine(g, p, 0, p.q, fp64, &E);
    if (rc) return rc;
    SmmArgs& a = E.a;
    AmcArgs& m = E.m;
    const bool dense = E.dense || E.hybrid;
    cudaGraph_t graph = nullptr;
    GER_CUDA(cudaGraphCreate(&graph, 0));
    cudaGraphConditionalHandle handle;
    cudaError_t e = cudaGraphConditionalHandleCreate(&handle, graph, 0, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        return cuda_fail(e, "cudaGraphConditionalHandleCreate");
    }
    g_prof_sink = &bg.prof_recs;
    g_capturing = true;
    g_captured = 0;
    int64_t body_launches = 0;
    e = cudaStreamBeginCaptureToGraph(st, graph, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
        cudaMemsetAsync(w.counters, 0, 8 * sizeof(int), st);
        cudaMemsetAsync(w.ctl, 0, sizeof(SmmCtl), st);
        issue_smm_start(g, E, fp64, st);
        launch_smm_advance(a, E.grid, handle, true, st);
        cudaStreamCaptureStatus cs;
        const cudaGraphNode_t* deps = nullptr;
        size_t ndeps = 0;
        cudaGraph_t cap = nullptr;
        e = cudaStreamGetCaptureInfo(st, &cs, nullptr, &cap, &deps, nullptr, &ndeps);
        cudaGraphNode_t cnode = nullptr;
        cudaGraphNodeParams cp = {};
        if (e == cudaSuccess) {
            cp.type = cudaGraphNodeTypeConditional;
            cp.conditional.handle = handle;
            cp.conditional.type = cudaGraphCondTypeWhile;
            cp.conditional.size = 1;
            e = cudaGraphAddNode(&cnode, cap, deps, nullptr, ndeps, &cp);
        }
        if (e == cudaSuccess)
            e = cudaStreamUpdateCaptureDependencies(st, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies);
        if (e == cudaSuccess) {
            cudaGraph_t body = cp.conditional.phGraph_out[0];
            e = cudaStreamBeginCaptureToGraph(st2, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
            if (e == cudaSuccess) {
                g_prof_suspend = true;  // no event records inside a conditional body
                const int64_t before = g_captured;
                issue_smm_iteration(E, fp64, st2);
                launch_smm_advance(a, E.grid, handle, true, st2);
                body_launches = g_captured - before;
                g_captured = before;
                g_prof_suspend = false;
                e = cudaStreamEndCapture(st2, &body);
            }
        }
        if (e == cudaSuccess) {
            m.out_r = p.r;  // the last statistics launch writes the outputs
            m.out_stats = p.stats;
            issue_amc(g, m, p.q, st);
        }
        cudaGraph_t done = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(st, &done);
        if (e == cudaSuccess) e = e2;
    }
    g_prof_sink = nullptr;
    g_capturing = false;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&bg.exec, graph, 0);
    bg.graph = graph;
    if (e != cudaSuccess) {
        destroy_graph(bg);
        cudaGetLastError();
        return cuda_fail(e, "capturing the batch graph");
    }
    bg.valid = true;
    bg.nq = p.q;
    bg.fp64 = fp64;
    bg.o = p.o;
    bg.lambda = g->lambda;
    bg.pool = w.ent;
    bg.state = w.st;
    bg.dense = w.dX[0];
    bg.dense_w = dense ? a.dense_width : 0;
    bg.dense_cols = E.cols;
    bg.dense_dev = w.dblock_q;
    bg.mig = w.dmig;
    bg.gen = w.gen;
    bg.prof = g_prof_on;
    bg.launches = g_captured;  // kernels outside the while body, once per replay
    bg.body_launches = body_launches;
    bg.mlp = g->mlp_w != nullptr;
    bg.forced = p.lb_force != nullptr;
    return GER_OK;
}

static bool graphs_enabled() {
    const char* v = std::getenv("GEER_NO_GRAPH");
    return !(v && v[0] && v[0] != '0');
}

// One batch. Batched plans run as a captured graph (built on first use for
// each batch shape, replayed after) and must use the workspace buffers for
// s, t, eps, r and stats; one-query-at-a-time plans run stream-ordered. A
// frontier-table pool overflow grows the pool and reruns the batch.
static int run_batch(ger_graph* g, Plan& p) {
    if (p.q == 0) return GER_OK;
    int rc = ensure_lambda(g);
    if (rc) return rc;
    const bool per_query = p.o.per_query != 0;
    const bool fp64 = p.o.precision == GER_FP64;
    const bool use_graph = !per_query && !p.trace && graphs_enabled();
    // the F_0 tables (8 slots per query) and room for the later ones
    int64_t pool = std::max<int64_t>({g->ws.pool_cap, (int64_t)1 << 22, (int64_t)kF0Slots * p.q + ((int64_t)1 << 20)});
    for (int attempt = 0; attempt < 6; ++attempt) {
        rc = ensure_ws(g, p.q, pool);
        if (rc) return rc;
        Workspace& w = g->ws;
        if (use_graph) {
            if (!same_key(g->bg, p, fp64, g)) {
                rc = build_graph(g, p, fp64);
                if (rc) return rc;
            }
            GER_CUDA(cudaGraphLaunch(g->bg.exec, p.st));
            note_launches((int)g->bg.launches);
        } else {
            GER_CUDA(cudaMemsetAsync(w.counters, 0, 8 * sizeof(int), p.st));
            GER_CUDA(cudaMemsetAsync(w.ctl, 0, sizeof(SmmCtl), p.st));
            if (per_query) {
                // each query's launches write its own outputs
                for (int64_t i = 0; i < p.q; ++i) {
                    rc = run_queries(g, p, i, 1, fp64, true);
                    if (rc) return rc;
                }
            } else {
                rc = run_queries(g, p, 0, p.q, fp64, true);
                if (rc) return rc;
            }
        }
        GER_CUDA(cudaGetLastError());
        GER_CUDA(cudaMemcpyAsync(w.host_rb, w.counters + 1, sizeof(int), cudaMemcpyDeviceToHost, p.st));
        GER_CUDA(cudaMemcpyAsync(w.host_rb + 1, &w.ctl->cursor, sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                                 p.st));
        GER_CUDA(cudaMemcpyAsync(w.host_rb + 3, &w.ctl->iter, sizeof(int32_t), cudaMemcpyDeviceToHost, p.st));
        GER_CUDA(cudaMemcpyAsync(reinterpret_cast<int32_t*>(w.host_rb + 3) + 1, &w.ctl->heavy_max, sizeof(int32_t),
                                 cudaMemcpyDeviceToHost, p.st));
        GER_CUDA(cudaStreamSynchronize(p.st));
        {
            // heavy pushes that did not fit ran on single warps (correct, slow):
            // give the next batches a list that holds them
            const int64_t need = reinterpret_cast<int32_t*>(w.host_rb + 3)[1];
            if (need > w.heavy_cap && w.heavy_cap < kHeavyCapMax) {
                int64_t cap = w.heavy_cap;
                while (cap < 2 * need && cap < kHeavyCapMax) cap <<= 1;
                int64_t* nh = nullptr;
                if (alloc(&nh, cap) == cudaSuccess) {
                    cudaFree(w.heavy);
                    w.heavy = nh;
                    w.heavy_cap = cap;
                    ++w.gen;
                } else {
                    cudaGetLastError();
                }
            }
        }
        if (use_graph) {
            prof_collect_graph(g->bg.prof_recs);
            // the while body ran iter - 1 times
            const int32_t iters = *reinterpret_cast<int32_t*>(w.host_rb + 3);
            if (iters > 1) note_launches((int)(g->bg.body_launches * (iters - 1)));
        }
        prof_collect();
        const int derr = (int)(reinterpret_cast<int*>(w.host_rb)[0]);
        if (derr == DERR_NONE) return GER_OK;
        if (derr == DERR_TABLE) {
            const int64_t used = w.host_rb[1] + (int64_t)kF0Slots * p.q;  // handed-out slots and the F_0 tables
            pool = std::max<int64_t>(2 * used, 2 * w.pool_cap);
            continue;
        }
        return map_device_error(derr);
    }
    return fail(GER_ERR_CAPACITY, "frontier-table pool did not fit after retries");
}

// Read-only view of a loaded graph, for entry points defined in other
// translation units.
int graph_view(const ger_graph* g, DevGraph* dg, double* lambda, bool* has_lambda, int* device, int* sm_count) {
    if (!g) return fail(GER_ERR_INVALID, "null graph");
    *dg = dev_graph(g);
    *lambda = g->lambda;
    *has_lambda = g->has_lambda;
    *device = g->device;
    *sm_count = g->sm_count;
    return GER_OK;
}

int set_error(int code, const char* msg) { return fail(code, "%s", msg); }

void launch_finalize(const QState* st, int64_t nq, double* r, ger_query_stats* stats, cudaStream_t s) {
    const int fg = query_grid(nq);
    prof_begin(FAM_FINALIZE, s);
    finalize_kernel<<<fg, kQueryCta, 0, s>>>(st, nq, r, stats);
    prof_end(FAM_FINALIZE, s);
}

}  // namespace geer

using namespace geer;

extern "C" {

void ger_default_options(ger_options* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->delta = 0.01;
    o->tau = 5;
    o->precision = GER_FP32;
    o->per_query = 0;
    o->switch_policy = GER_SWITCH_RULE;
    o->fixed_ell_b = -1;
    o->ell_formula = GER_ELL_REFINED;
    o->seed = 3;
    o->sparse_cap = 0;
    o->smm_engine = GER_ENGINE_SPARSE;
    o->dense_width = 0;
    o->dense_switch = 0;
    o->dense_budget_mb = 0;
}

const char* ger_last_error(void) { return g_err; }

int ger_test_fail_alloc(int64_t countdown) {
    if (countdown < 0) return fail(GER_ERR_INVALID, "countdown must be >= 0");
    g_fail_alloc_countdown.store(countdown);
    return GER_OK;
}

int64_t ger_launch_count(void) { return g_launches.load(); }

int ger_profile_enable(int on) {
    prof_collect();
    g_prof_on = on != 0;
    if (g_prof_on) {
        for (int f = 0; f < FAM_COUNT; ++f) {
            g_prof_launches[f] = 0;
            g_prof_ms[f] = 0.0;
            g_prof_open[f] = nullptr;
        }
    }
    return GER_OK;
}

int ger_profile_read(ger_kernel_profile* out, int max_entries) {
    if (max_entries < 0 || (max_entries > 0 && !out)) return fail(GER_ERR_INVALID, "bad profile buffer");
    prof_collect();
    int k = 0;
    for (int f = 0; f < FAM_COUNT; ++f) {
        if (g_prof_launches[f] == 0) continue;
        if (k < max_entries) {
            std::memset(&out[k], 0, sizeof(out[k]));
            std::snprintf(out[k].name, sizeof(out[k].name), "%s", kFamilyNames[f]);
            out[k].launches = g_prof_launches[f];
            out[k].total_ms = g_prof_ms[f];
        }
        ++k;
    }
    return k;
}

int ger_load_csr(int64_t n, const int64_t* row_ptr, const int32_t* col_idx, int device, ger_graph** out) {
    if (!out || !row_ptr || (!col_idx && n > 0)) return fail(GER_ERR_INVALID, "null argument");
    *out = nullptr;
    int rc = validate_csr(n, row_ptr, col_idx);
    if (rc) return rc;
    ger_graph* g = new (std::nothrow) ger_graph();
    if (!g) return fail(GER_ERR_OOM, "host allocation");
    g->device = device;
    g->n = n;
    g->nnz = row_ptr[n];
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) {
        delete g;
        return cuda_fail(e, "cudaSetDevice");
    }
    cudaDeviceGetAttribute(&g->sm_count, cudaDevAttrMultiProcessorCount, device);
    if (cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&g->stream2, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMalloc(&g->row_ptr, (n + 1) * sizeof(int64_t)) != cudaSuccess ||
        cudaMalloc(&g->col_idx, std::max<int64_t>(g->nnz, 1) * sizeof(int32_t)) != cudaSuccess) {
        cudaGetLastError();
        ger_free(g);
        return fail(GER_ERR_OOM, "device copy of the graph");
    }
    if (cudaMemcpy(g->row_ptr, row_ptr, (n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(g->col_idx, col_idx, g->nnz * sizeof(int32_t), cudaMemcpyHostToDevice) != cudaSuccess) {
        ger_free(g);
        return fail(GER_ERR_CUDA, "copying the graph");
    }
    if (g->nnz < ((int64_t)1 << 32)) {
        // one 8-byte record per node for the walks: {first edge, degree}
        std::vector<uint2> info(n);
        for (int64_t v = 0; v < n; ++v)
            info[v] = make_uint2((uint32_t)row_ptr[v], (uint32_t)(row_ptr[v + 1] - row_ptr[v]));
        if (cudaMalloc(&g->node_info, n * sizeof(uint2)) != cudaSuccess ||
            cudaMemcpy(g->node_info, info.data(), n * sizeof(uint2), cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaGetLastError();
            ger_free(g);
            return fail(GER_ERR_OOM, "device copy of the node records");
        }
        // the walks' edge records: 16 B per stored edge; without them the
        // walks take two dependent loads per step instead of one
        // opt-in (GEER_EDGE_RECORDS=1): a walk reads edges uniformly and node
        // records in proportion to degree, so col_idx plus the node records
        // hit L2 more often than one edge-record array; measured slower on the
        // 1M- and 4M-node power-law graphs
        const char* rec_env = std::getenv("GEER_EDGE_RECORDS");
        const bool want_rec = rec_env && rec_env[0] && rec_env[0] != '0';
        if (!want_rec) {
            g->edge_rec = nullptr;
        } else if (cudaMalloc(&g->edge_rec, (size_t)std::max<int64_t>(g->nnz, 1) * sizeof(uint4)) == cudaSuccess) {
            launch_edge_records(g->col_idx, g->node_info, g->nnz, g->edge_rec, g->stream);
            if (cudaStreamSynchronize(g->stream) != cudaSuccess) {
                cudaGetLastError();
                ger_free(g);
                return fail(GER_ERR_CUDA, "building the edge records");
            }
        } else {
            cudaGetLastError();
            g->edge_rec = nullptr;
        }
        // the walks' packed neighbour lists (GEER_PACKED_COLS=0 keeps col_idx);
        // their entries are addressed from the node records' 32-bit first
        // edge, so they exist only with the node records (nnz < 2^32)
        const char* pk_env = std::getenv("GEER_PACKED_COLS");
        const int pk = pack_k_for(n);
        if (pk > 0 && g->node_info && !(pk_env && pk_env[0] == '0')) {
            const int64_t units = (g->nnz + pk - 1) / pk;
            if (cudaMalloc(&g->cols_packed, (size_t)std::max<int64_t>(units, 1) * sizeof(uint4)) == cudaSuccess) {
                launch_pack_cols(g->col_idx, g->nnz, pk, g->cols_packed, g->stream);
                if (cudaStreamSynchronize(g->stream) != cudaSuccess) {
                    cudaGetLastError();
                    ger_free(g);
                    return fail(GER_ERR_CUDA, "packing the neighbour lists");
                }
                g->pack_k = pk;
            } else {
                cudaGetLastError();
                g->cols_packed = nullptr;
            }
        }
        if (n < INT32_MAX) {
            std::vector<int4> units, heavy;
            int32_t nslots = 0;
            build_dense_units(n, row_ptr, &units, &heavy, &nslots);
            if (cudaMalloc(&g->dense_units, units.size() * sizeof(int4) + 16) != cudaSuccess ||
                cudaMalloc(&g->dense_heavy, heavy.size() * sizeof(int4) + 16) != cudaSuccess ||
                cudaMemcpy(g->dense_units, units.data(), units.size() * sizeof(int4), cudaMemcpyHostToDevice) !=
                    cudaSuccess ||
                cudaMemcpy(g->dense_heavy, heavy.data(), heavy.size() * sizeof(int4), cudaMemcpyHostToDevice) !=
                    cudaSuccess) {
                cudaGetLastError();
                ger_free(g);
                return fail(GER_ERR_OOM, "device copy of the dense work units");
            }
            g->dense_nunits = (int32_t)units.size();
            g->dense_nheavy = (int32_t)heavy.size();
            g->dense_nslots = nslots;
        }
    }
    *out = g;
    return GER_OK;
}

void ger_free(ger_graph* g) {
    if (!g) return;
    cudaSetDevice(g->device);
    if (g->stream) cudaStreamSynchronize(g->stream);
    destroy_graph(g->bg);
    free_ws(g->ws);
    cudaFree(g->row_ptr);
    cudaFree(g->col_idx);
    cudaFree(g->node_info);
    cudaFree(g->edge_rec);
    cudaFree(g->cols_packed);
    cudaFree(g->dense_units);
    cudaFree(g->dense_heavy);
    cudaFree(g->mlp_w);
    cudaFree(g->mlp_wt);
    cudaFree(g->mlp_norm);
    if (g->stream) cudaStreamDestroy(g->stream);
    if (g->stream2) cudaStreamDestroy(g->stream2);
    delete g;
}

int ger_graph_size(const ger_graph* g, int64_t* n, int64_t* nnz) {
    if (!g) return fail(GER_ERR_INVALID, "null graph");
    if (n) *n = g->n;
    if (nnz) *nnz = g->nnz;
    return GER_OK;
}

int ger_spectral_bound(ger_graph* g, double* lambda, double* lam2, double* lamn) {
    if (!g) return fail(GER_ERR_INVALID, "null graph");
    cudaSetDevice(g->device);
    int rc = ensure_lambda(g);
    if (rc) return rc;
    if (lambda) *lambda = g->lambda;
    if (lam2) *lam2 = g->lam2;
    if (lamn) *lamn = g->lamn;
    return GER_OK;
}

int ger_set_spectral_bound(ger_graph* g, double lambda) {
    if (!g) return fail(GER_ERR_INVALID, "null graph");
    if (!(lambda >= 0.0 && lambda < 1.0)) return fail(GER_ERR_INVALID, "lambda must be in [0, 1)");
    g->lambda = lambda;
    g->lam2 = g->lamn = std::nan("");
    g->has_lambda = true;
    g->lam_steps = 0;
    g->lam_converged = 1;
    g->lam_resid_hi = g->lam_resid_lo = 0.0;
    return GER_OK;
}

int ger_spectral_bound_info(const ger_graph* g, int32_t* converged, int32_t* steps, double* resid_hi,
                            double* resid_lo) {
    if (!g) return fail(GER_ERR_INVALID, "null graph");
    if (!g->has_lambda) return fail(GER_ERR_NO_LAMBDA, "spectral bound neither computed nor set");
    if (converged) *converged = g->lam_converged;
    if (steps) *steps = g->lam_steps;
    if (resid_hi) *resid_hi = g->lam_resid_hi;
    if (resid_lo) *resid_lo = g->lam_resid_lo;
    return GER_OK;
}

static int check_opts(const ger_options* opt, ger_options* o) {
    if (opt) *o = *opt; else ger_default_options(o);
    if (!(o->delta > 0.0 && o->delta < 1.0)) return fail(GER_ERR_INVALID, "delta must be in (0, 1)");
    if (o->tau < 0 || o->tau > 20) return fail(GER_ERR_INVALID, "tau must be in 1..20 (0: the autotuned value)");
    if (o->precision != GER_FP32 && o->precision != GER_FP64) return fail(GER_ERR_INVALID, "bad precision");
    if (o->switch_policy != GER_SWITCH_RULE && o->switch_policy != GER_SWITCH_FIXED &&
        o->switch_policy != GER_SWITCH_MLP)
        return fail(GER_ERR_INVALID, "bad switch policy");
    if (o->ell_formula != GER_ELL_REFINED && o->ell_formula != GER_ELL_PENG) return fail(GER_ERR_INVALID, "bad ell formula");
    if (o->smm_engine != GER_ENGINE_SPARSE && o->smm_engine != GER_ENGINE_DENSE && o->smm_engine != GER_ENGINE_HYBRID)
        return fail(GER_ERR_INVALID, "bad smm engine");
    if (o->dense_width != 0 && !dense_width_ok(o->dense_width, o->precision == GER_FP64))
        return fail(GER_ERR_INVALID, "dense_width must be 32, 64 or 128 (FP32) or 32 or 64 (FP64)");
    if (o->dense_switch < 0 || o->dense_budget_mb < 0) return fail(GER_ERR_INVALID, "negative dense option");
    return GER_OK;
}

// tau = 0 in the options: the graph's autotuned tau, else the paper's 5
static void resolve_tau(const ger_graph* g, ger_options* o) {
    if (o->tau == 0) o->tau = g->tau_tuned > 0 ? g->tau_tuned : 5;
}

static int host_batch(ger_graph* g, int64_t q, const int32_t* s, const int32_t* t, const double* eps_arr,
                      double eps, const ger_options* opt, double* r_out, ger_query_stats* stats,
                      float* trace_out = nullptr, int32_t trace_steps = 0, const int32_t* lb_arr = nullptr) {
    if (!g || q < 0 || (q > 0 && (!s || !t || !r_out))) return fail(GER_ERR_INVALID, "null argument or q < 0");
    if (q > 0x7fffffff) return fail(GER_ERR_INVALID, "q too large");
    Plan p;
    int rc = check_opts(opt, &p.o);
    if (rc) return rc;
    resolve_tau(g, &p.o);
    for (int64_t i = 0; i < q; ++i) {
        if (s[i] < 0 || s[i] >= g->n || t[i] < 0 || t[i] >= g->n)
            return fail(GER_ERR_NODE_RANGE, "query %lld: node outside [0, %lld)", (long long)i, (long long)g->n);
        const double e = eps_arr ? eps_arr[i] : eps;
        if (!(e > 0.0)) return fail(GER_ERR_INVALID, "query %lld: eps must be > 0", (long long)i);
    }
    cudaSetDevice(g->device);
    if (q == 0) return GER_OK;
    rc = ensure_ws(g, q, std::max<int64_t>(g->ws.pool_cap, (int64_t)1 << 22));
    if (rc) return rc;
    Workspace& w = g->ws;
    cudaStream_t st = g->stream;
    GER_CUDA(cudaMemcpyAsync(w.s, s, q * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    GER_CUDA(cudaMemcpyAsync(w.t, t, q * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    if (eps_arr) {
        GER_CUDA(cudaMemcpyAsync(w.eps, eps_arr, q * sizeof(double), cudaMemcpyHostToDevice, st));
    } else {
        std::vector<double> ev((size_t)q, eps);
        GER_CUDA(cudaMemcpyAsync(w.eps, ev.data(), q * sizeof(double), cudaMemcpyHostToDevice, st));
        GER_CUDA(cudaStreamSynchronize(st));
    }
    if (lb_arr) {
        GER_CUDA(cudaMemcpyAsync(w.lbf, lb_arr, q * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        p.lb_force = w.lbf;
    }
    p.q = q;
    p.s = w.s;
    p.t = w.t;
    p.eps = w.eps;
    p.eps_scalar = 0.0;
    p.r = w.r;
    p.stats = w.stats;
    p.st = st;
    float* tr = nullptr;
    const size_t tr_bytes = trace_out ? (size_t)q * (size_t)trace_steps * kTraceWidth * sizeof(float) : 0;
    if (trace_out) {
        if (cudaMalloc(&tr, tr_bytes) != cudaSuccess) {
            cudaGetLastError();
            return fail(GER_ERR_OOM, "cost log (%zu bytes)", tr_bytes);
        }
        p.trace = tr;
        p.trace_steps = trace_steps;
        cudaMemsetAsync(tr, 0, tr_bytes, st);
    }
    rc = run_batch(g, p);
    if (!rc && trace_out) {
        const cudaError_t e = cudaMemcpyAsync(trace_out, tr, tr_bytes, cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) rc = cuda_fail(e, "reading the cost log");
        cudaStreamSynchronize(st);
    }
    cudaFree(tr);
    if (rc) return rc;
    GER_CUDA(cudaMemcpyAsync(r_out, w.r, q * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (stats) GER_CUDA(cudaMemcpyAsync(stats, w.stats, q * sizeof(ger_query_stats), cudaMemcpyDeviceToHost, st));
    GER_CUDA(cudaStreamSynchronize(st));
    return GER_OK;
}

int ger_query_batch(ger_graph* g, int64_t q, const int32_t* s, const int32_t* t, double eps,
                    const ger_options* opt, double* r_out, ger_query_stats* stats) {
    if (!(eps > 0.0)) return fail(GER_ERR_INVALID, "eps must be > 0");
    return host_batch(g, q, s, t, nullptr, eps, opt, r_out, stats);
}

int ger_query_batch_eps(ger_graph* g, int64_t q, const int32_t* s, const int32_t* t, const double* eps,
                        const ger_options* opt, double* r_out, ger_query_stats* stats) {
    if (q > 0 && !eps) return fail(GER_ERR_INVALID, "null eps");
    return host_batch(g, q, s, t, eps, 0.0, opt, r_out, stats);
}

int ger_query_batch_lb(ger_graph* g, int64_t q, const int32_t* s, const int32_t* t, const double* eps,
                       const int32_t* ell_b, const ger_options* opt, double* r_out, ger_query_stats* stats) {
    if (q > 0 && (!eps || !ell_b)) return fail(GER_ERR_INVALID, "null eps or ell_b");
    return host_batch(g, q, s, t, eps, 0.0, opt, r_out, stats, nullptr, 0, ell_b);
}

int ger_smm_trace(ger_graph* g, int64_t q, const int32_t* s, const int32_t* t, const double* eps,
                  const ger_options* opt, int32_t max_steps, float* log_out, ger_query_stats* stats) {
    if (q > 0 && (!eps || !log_out)) return fail(GER_ERR_INVALID, "null eps or log");
    if (max_steps < 1 || max_steps > 4096) return fail(GER_ERR_INVALID, "max_steps must be in 1..4096");
    ger_options o;
    if (opt) o = *opt; else ger_default_options(&o);
    o.switch_policy = GER_SWITCH_FIXED;
    o.fixed_ell_b = max_steps;
    o.per_query = 0;
    std::vector<double> r((size_t)std::max<int64_t>(q, 1));
    return host_batch(g, q, s, t, eps, 0.0, &o, r.data(), stats, log_out, max_steps);
}

// Wall time (ms) of one host-buffer batch on the graph's stream, after one
// untimed call with the same options (which also builds its graph).
static int timed_batch(ger_graph* g, int64_t q, const int32_t* s, const int32_t* t, const double* eps,
                       const ger_options* o, int reps, float* ms_out) {
    std::vector<double> r((size_t)q);
    int rc = host_batch(g, q, s, t, eps, 0.0, o, r.data(), nullptr);
    if (rc) return rc;
    cudaEvent_t a, b;
    GER_CUDA(cudaEventCreate(&a));
    GER_CUDA(cudaEventCreate(&b));
    std::vector<float> ms;
    for (int i = 0; i < reps && !rc; ++i) {
        cudaEventRecord(a, g->stream);
        rc = host_batch(g, q, s, t, eps, 0.0, o, r.data(), nullptr);
        cudaEventRecord(b, g->stream);
        cudaEventSynchronize(b);
        float x = 0.f;
        cudaEventElapsedTime(&x, a, b);
        ms.push_back(x);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (rc) return rc;
    std::sort(ms.begin(), ms.end());
    *ms_out = ms[ms.size() / 2];
    return GER_OK;
}

int ger_autotune(ger_graph* g, int64_t q, const int32_t* s, const int32_t* t, const double* eps,
                 const ger_options* opt, ger_tuning* out) {
    if (!g || q <= 0 || !s || !t || !eps) return fail(GER_ERR_INVALID, "null argument or no queries");
    ger_options base;
    int rc = check_opts(opt, &base);
    if (rc) return rc;
    resolve_tau(g, &base);
    const bool fp64 = base.precision == GER_FP64;
    ger_tuning res;
    std::memset(&res, 0, sizeof(res));
    // 1. dense block width: standalone SMM (min(l, 4) iterations) of up to 64
    //    queries per width on the dense engine; cost per query
    if (g->dense_units) {
        const int64_t qs = std::min<int64_t>(q, 64);
        const int widths32[3] = {32, 64, 128}, widths64[2] = {32, 64};
        const int* widths = fp64 ? widths64 : widths32;
        const int nw = fp64 ? 2 : 3;
        float best = 0.f;
        for (int i = 0; i < nw; ++i) {
            ger_options o = base;
            o.smm_engine = GER_ENGINE_DENSE;
            o.dense_width = widths[i];
            o.switch_policy = GER_SWITCH_FIXED;
            o.fixed_ell_b = 4;
            o.per_query = 0;
            float ms = 0.f;
            rc = timed_batch(g, qs, s, t, eps, &o, 3, &ms);
            if (rc) return rc;
            // queries share a block up to width / 2: the cost of qs queries at this width
            res.width_ms[i] = ms;
            if (i == 0 || ms < best) {
                best = ms;
                res.dense_width = widths[i];
            }
        }
        g->dense_tuned[fp64 ? 1 : 0] = res.dense_width;
    }
    // 2. hybrid switch size: the whole batch with the caller's options on the
    //    hybrid engine at a few sizes (and without moves), the fastest wins
    const int64_t cands[5] = {g->nnz / 64, g->nnz / 16, g->nnz / 4, g->nnz, (int64_t)1 << 62};
    float best = 0.f;
    for (int i = 0; i < 5; ++i) {
        ger_options o = base;
        o.smm_engine = GER_ENGINE_HYBRID;
        o.dense_switch = std::max<int64_t>(cands[i], 1);
        float ms = 0.f;
        rc = timed_batch(g, q, s, t, eps, &o, 3, &ms);
        if (rc) return rc;
        res.switch_ms[i] = ms;
        res.switch_candidates[i] = o.dense_switch;
        if (i == 0 || ms < best) {
            best = ms;
            res.dense_switch = o.dense_switch;
        }
    }
    g->hybrid_tuned = res.dense_switch;
    // 3. tau (Algorithm 1's batch count): the whole batch with the caller's
    //    options at tau = 1..8; Theorem 2 holds at delta / tau for every tau,
    //    so the choice changes the walks drawn and the time, never the guarantee
    float best_tau = 0.f;
    for (int tau = 1; tau <= 8; ++tau) {
        ger_options o = base;
        o.tau = tau;
        float ms = 0.f;
        rc = timed_batch(g, q, s, t, eps, &o, 3, &ms);
        if (rc) return rc;
        res.tau_ms[tau - 1] = ms;
        if (tau == 1 || ms < best_tau) {
            best_tau = ms;
            res.tau = tau;
        }
    }
    g->tau_tuned = res.tau;
    if (out) *out = res;
    return GER_OK;
}

int ger_set_switch_mlp(ger_graph* g, const float* norm, const uint16_t* weights) {
    if (!g) return fail(GER_ERR_INVALID, "null graph");
    cudaSetDevice(g->device);
    if (!weights) {
        if (g->stream) cudaStreamSynchronize(g->stream);
        cudaFree(g->mlp_w);
        cudaFree(g->mlp_wt);
        cudaFree(g->mlp_norm);
        g->mlp_w = nullptr;
        g->mlp_wt = nullptr;
        g->mlp_norm = nullptr;
        return GER_OK;
    }
    if (!norm) return fail(GER_ERR_INVALID, "null normalisation");
    for (int k = 0; k < kMlpIn; ++k)
        if (!(norm[kMlpIn + k] > 0.f) || !std::isfinite(norm[k])) return fail(GER_ERR_INVALID, "bad normalisation");
    if (!g->mlp_w) {
        if (cudaMalloc(&g->mlp_w, kMlpParams * sizeof(uint16_t) + 16) != cudaSuccess ||
            cudaMalloc(&g->mlp_wt, kMlpStaged * sizeof(float)) != cudaSuccess ||
            cudaMalloc(&g->mlp_norm, 2 * kMlpIn * sizeof(float)) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(g->mlp_w);
            cudaFree(g->mlp_wt);
            g->mlp_w = nullptr;
            g->mlp_wt = nullptr;
            return fail(GER_ERR_OOM, "switch network");
        }
    }
    if (g->stream) cudaStreamSynchronize(g->stream);
    GER_CUDA(cudaMemcpy(g->mlp_w, weights, kMlpParams * sizeof(uint16_t), cudaMemcpyHostToDevice));
    GER_CUDA(cudaMemcpy(g->mlp_norm, norm, 2 * kMlpIn * sizeof(float), cudaMemcpyHostToDevice));
    launch_mlp_expand(g->mlp_w, g->mlp_wt, g->stream);
    GER_CUDA(cudaGetLastError());
    GER_CUDA(cudaStreamSynchronize(g->stream));
    return GER_OK;
}

int ger_query_batch_dev(ger_graph* g, int64_t q, const int32_t* s_dev, const int32_t* t_dev, const double* eps_dev,
                        const ger_options* opt, double* r_dev, ger_query_stats* stats_dev, void* stream) {
    if (!g || q < 0 || (q > 0 && (!s_dev || !t_dev || !eps_dev || !r_dev)))
        return fail(GER_ERR_INVALID, "null argument or q < 0");
    if (q > 0x7fffffff) return fail(GER_ERR_INVALID, "q too large");
    Plan p;
    int rc = check_opts(opt, &p.o);
    if (rc) return rc;
    resolve_tau(g, &p.o);
    cudaSetDevice(g->device);
    if (q == 0) return GER_OK;
    rc = ensure_ws(g, q, std::max<int64_t>(g->ws.pool_cap, (int64_t)1 << 22));
    if (rc) return rc;
    Workspace& w = g->ws;
    cudaStream_t st = stream ? reinterpret_cast<cudaStream_t>(stream) : (cudaStream_t)0;
    GER_CUDA(cudaMemcpyAsync(w.s, s_dev, q * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
    GER_CUDA(cudaMemcpyAsync(w.t, t_dev, q * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
    GER_CUDA(cudaMemcpyAsync(w.eps, eps_dev, q * sizeof(double), cudaMemcpyDeviceToDevice, st));
    p.q = q;
    p.s = w.s;
    p.t = w.t;
    p.eps = w.eps;
    p.eps_scalar = 0.0;
    p.r = w.r;
    p.stats = w.stats;
    p.st = st;
    rc = run_batch(g, p);
    if (rc) return rc;
    GER_CUDA(cudaMemcpyAsync(r_dev, w.r, q * sizeof(double), cudaMemcpyDeviceToDevice, st));
    if (stats_dev) GER_CUDA(cudaMemcpyAsync(stats_dev, w.stats, q * sizeof(ger_query_stats), cudaMemcpyDeviceToDevice, st));
    GER_CUDA(cudaStreamSynchronize(st));
    return GER_OK;
}

}  // extern "C"
