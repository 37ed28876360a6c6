// noalloc.cu -- ger_query_batch_dev_noalloc: the batched GEER query of
// ger_query_batch_dev, for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: a serving loop that must never block
// on the device (cudaMalloc and cudaFree may synchronise it), a process
// whose device memory is owned by another allocator or reserved up front
// under a hard budget, or code that must keep its memory footprint fixed
// from start-up. This entry point takes all of its scratch from one
// statically sized device array (g_noalloc_scratch below) and allocates
// nothing: no cudaMalloc, no cudaFree, no pinned host buffer, no library
// routine that allocates. The caller passes the inputs and outputs.
//
// Limits: at most kNoAllocMaxQueries queries per call and kNoAllocPool
// frontier-table slots per call (the tables of every SMM iteration of every
// query, each a power of two at least twice the iteration's push volume);
// beyond them the call fails with GER_ERR_CAPACITY. The array lives in every
// GPU that loads this module, until the process exits.
#include <cmath>
#include <mutex>

#include "../../include/geer.h"

#include "geer_internal.cuh"
#include "geer_kernels.h"

namespace geer {

namespace {

constexpr int64_t kNoAllocMaxQueries = 64;
constexpr int64_t kNoAllocPool = 1 << 19;    // frontier-table slots per call
constexpr size_t kNoAllocBytes = 32u << 20;  // 32 MiB per GPU

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// byte offsets of the regions inside the array
constexpr size_t kOffCounters = 0;  // error flag (int) and spare words
constexpr size_t kOffCtl = align256(kOffCounters + 64);
constexpr size_t kOffState = align256(kOffCtl + sizeof(SmmCtl));
constexpr size_t kOffQSmm = align256(kOffState + sizeof(QState) * kNoAllocMaxQueries);
constexpr int64_t kNoAllocHeavy = 4096;
constexpr size_t kOffHeavy = align256(kOffQSmm + sizeof(QSmm) * kNoAllocMaxQueries);
constexpr size_t kOffChunk = align256(kOffHeavy + sizeof(int64_t) * kNoAllocHeavy);
constexpr size_t kOffWalkQ = align256(kOffChunk + sizeof(int64_t) * (kNoAllocMaxQueries + 1));
constexpr size_t kOffCount = align256(kOffWalkQ + sizeof(WalkQ) * kNoAllocMaxQueries);
constexpr size_t kOffPartial = align256(kOffCount + sizeof(int32_t) * kNoAllocMaxQueries);
constexpr size_t kOffEnt = align256(kOffPartial + sizeof(Partial) * kNoAllocMaxQueries * kMaxChunksPerQuery);
constexpr size_t kOffSums = align256(kOffEnt + sizeof(GEntry) * kNoAllocPool);
constexpr size_t kOffY = align256(kOffSums + sizeof(uint64_t) * 2 * kNoAllocPool);
constexpr size_t kEnd = kOffY + sizeof(double) * 2 * kNoAllocPool;
static_assert(kEnd <= kNoAllocBytes, "no-alloc layout exceeds its array");

// The scratch array. In host code this name is only a stand-in for the
// symbol, never a device address: its address comes from
// cudaGetSymbolAddress, once per device.
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_mu;
constexpr int kMaxDevices = 64;
void* g_scratch_dev[kMaxDevices] = {};

// Device address of the array on `device` (current). Looked up on the first
// call per device.
int scratch_address(int device, unsigned char** out) {
    if (device < 0 || device >= kMaxDevices) return set_error(GER_ERR_INVALID, "device id out of range");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_dev[device]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return set_error(GER_ERR_CUDA, "cudaGetSymbolAddress of the no-alloc scratch array failed");
        }
        g_scratch_dev[device] = p;
    }
    *out = static_cast<unsigned char*>(g_scratch_dev[device]);
    return GER_OK;
}

// Status of the launches issued so far (cudaGetLastError: a launch that could
// not start reports here, not through the kernel's error flag).
int check_launches() {
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(GER_ERR_CUDA, cudaGetErrorString(e));
    return GER_OK;
}

int sync_read_int(const void* dev, int* out, cudaStream_t st) {
    if (cudaMemcpyAsync(out, dev, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return set_error(GER_ERR_CUDA, cudaGetErrorString(cudaGetLastError()));
    return GER_OK;
}

}  // namespace

}  // namespace geer

using namespace geer;

extern "C" int ger_query_batch_dev_noalloc(ger_graph* g, int64_t q, const int32_t* s_dev, const int32_t* t_dev,
                                           const double* eps_dev, const ger_options* opt, double* r_dev,
                                           ger_query_stats* stats_dev, void* stream) {
    if (!g || q < 0 || (q > 0 && (!s_dev || !t_dev || !eps_dev || !r_dev)))
        return set_error(GER_ERR_INVALID, "null argument or q < 0");
    if (q > kNoAllocMaxQueries)
        return set_error(GER_ERR_CAPACITY, "ger_query_batch_dev_noalloc takes at most 64 queries per call");
    ger_options o;
    if (opt) o = *opt; else ger_default_options(&o);
    if (o.switch_policy == GER_SWITCH_MLP)
        return set_error(GER_ERR_INVALID, "the no-alloc entry point does not run the learned switch");
    if (!(o.delta > 0.0 && o.delta < 1.0) || o.tau < 1 || o.tau > 20 ||
        (o.precision != GER_FP32 && o.precision != GER_FP64) ||
        (o.switch_policy != GER_SWITCH_RULE && o.switch_policy != GER_SWITCH_FIXED) ||
        (o.ell_formula != GER_ELL_REFINED && o.ell_formula != GER_ELL_PENG))
        return set_error(GER_ERR_INVALID, "invalid options");
    if (o.smm_engine != GER_ENGINE_SPARSE)
        return set_error(GER_ERR_INVALID, "the no-alloc entry point runs the sparse SMM engine only");
    DevGraph dg;
    double lambda;
    bool has_lambda;
    int device, sm_count;
    int rc = graph_view(g, &dg, &lambda, &has_lambda, &device, &sm_count);
    if (rc) return rc;
    if (!has_lambda)
        return set_error(GER_ERR_NO_LAMBDA,
                         "spectral bound not available: call ger_spectral_bound or ger_set_spectral_bound first");
    if (q == 0) return GER_OK;
    if (cudaSetDevice(device) != cudaSuccess) return set_error(GER_ERR_CUDA, "cudaSetDevice failed");
    unsigned char* base = nullptr;
    rc = scratch_address(device, &base);
    if (rc) return rc;
    cudaStream_t st = stream ? reinterpret_cast<cudaStream_t>(stream) : (cudaStream_t)0;
    const bool fp64 = o.precision == GER_FP64;
    cudaGetLastError();  // a non-sticky error left by earlier work is not this call's

    int* counters = reinterpret_cast<int*>(base + kOffCounters);
    SmmCtl* ctl = reinterpret_cast<SmmCtl*>(base + kOffCtl);
    QState* qs = reinterpret_cast<QState*>(base + kOffState);
    // the array keeps the previous call's contents: reset what must start at zero
    if (cudaMemsetAsync(base + kOffCounters, 0, kOffState - kOffCounters, st) != cudaSuccess) {
        cudaGetLastError();
        return set_error(GER_ERR_CUDA, "cudaMemsetAsync of the no-alloc control words failed");
    }
    SmmArgs a;
    a.g = dg;
    a.nq = (int32_t)q;
    a.q_index_base = 0;
    a.st = qs;
    a.sm = reinterpret_cast<QSmm*>(base + kOffQSmm);
    a.s = s_dev;
    a.t = t_dev;
    a.eps = eps_dev;
    a.eps_scalar = 0.0;
    a.lambda = lambda;
    a.log_inv_lambda = a.lambda > 0.0 && a.lambda < 1.0 ? std::log(1.0 / a.lambda) : 0.0;
    a.delta = o.delta;
    a.tau = o.tau;
    a.log_2tau_delta = std::log(2.0 * (double)a.tau / a.delta);
    a.ell_formula = o.ell_formula;
    a.policy = o.switch_policy;
    a.fixed_lb = o.fixed_ell_b;
    int64_t max_table = kNoAllocPool;
    if (o.sparse_cap > 0) {
        int64_t cap = 16;
        while (cap < 2 * o.sparse_cap) cap <<= 1;
        max_table = cap < kNoAllocPool ? cap : kNoAllocPool;
    }
    a.max_table = max_table;
    a.ent = reinterpret_cast<GEntry*>(base + kOffEnt);
    a.sum_s = reinterpret_cast<unsigned long long*>(base + kOffSums);
    a.sum_t = a.sum_s + kNoAllocPool;
    a.ys = base + kOffY;
    a.yt = fp64 ? (void*)(reinterpret_cast<double*>(base + kOffY) + kNoAllocPool)
                : (void*)(reinterpret_cast<float*>(base + kOffY) + kNoAllocPool);
    a.pool_cap = kNoAllocPool;
    a.dense_engine = 0;
    a.dense_width = 2;
    a.dense_fp64 = fp64;
    a.dense_X[0] = a.dense_X[1] = nullptr;
    a.heavy = reinterpret_cast<int64_t*>(base + kOffHeavy);
    a.heavy_cap = kNoAllocHeavy;
    a.ctl = ctl;
    a.err_flag = counters + 1;
    a.wq = reinterpret_cast<WalkQ*>(base + kOffWalkQ);
    const int grid = sm_count * 8;
    launch_smm_start(fp64, a, st);
    launch_smm_advance(a, grid, 0, false, st);
    // a launch that failed to start (bad configuration, missing kernel image)
    // leaves the control words at their zeros: catch it before reading them
    rc = check_launches();
    if (rc) return rc;
    for (int iter = 1; iter < 100000; ++iter) {
        int n_go = 0;
        rc = sync_read_int(&ctl->n_go, &n_go, st);
        if (rc) return rc;
        if (n_go == 0) break;
        launch_smm_iteration(fp64, a, grid, st);
        launch_smm_advance(a, grid, 0, false, st);
        rc = check_launches();
        if (rc) return rc;
    }
    AmcArgs m;
    m.g = dg;
    m.nq = (int32_t)q;
    m.st = qs;
    m.chunk_begin = reinterpret_cast<int64_t*>(base + kOffChunk);
    m.wq = reinterpret_cast<WalkQ*>(base + kOffWalkQ);
    m.chunk_count = reinterpret_cast<int32_t*>(base + kOffCount);
    m.walk_ctr = reinterpret_cast<unsigned long long*>(counters + 4);  // inside the 64-byte counter region
    m.done = reinterpret_cast<unsigned int*>(counters + 2);
    m.partial = reinterpret_cast<Partial*>(base + kOffPartial);
    m.partial_cap = kNoAllocMaxQueries * kMaxChunksPerQuery;
    m.pool = a.ent;
    m.seed = o.seed;
    m.tau = o.tau;
    m.delta = o.delta;
    m.log_3tau_delta = std::log(3.0 * (double)m.tau / m.delta);
    m.dense_fp64 = fp64;
    m.err_flag = counters + 1;
    m.group = counters + 6;  // inside the 64-byte counter region
    m.batch = 1;
    launch_amc_schedule(m, st);
    for (int b = 1; b <= o.tau; ++b) {
        m.batch = b;
        launch_amc_walk(m, sm_count, st);
        launch_amc_reduce(m, st);  // it also lays out the next launch
    }
    launch_finalize(qs, q, r_dev, stats_dev, st);
    note_launches(2 + 2 * o.tau);
    rc = check_launches();
    if (rc) return rc;
    int derr = 0;
    rc = sync_read_int(counters + 1, &derr, st);
    if (rc) return rc;
    switch (derr) {
        case DERR_NONE: return GER_OK;
        case DERR_NODE_RANGE: return set_error(GER_ERR_NODE_RANGE, "a query node is outside [0, n) or eps <= 0");
        case DERR_CAPACITY:
            if (o.sparse_cap > 0 && max_table < kNoAllocPool)
                return set_error(GER_ERR_CAPACITY,
                                 "an SMM iteration needs a frontier table beyond options.sparse_cap push pairs");
            return set_error(GER_ERR_CAPACITY,
                             "an SMM iteration needs a frontier table beyond the no-alloc limit of 524288 slots");
        case DERR_TABLE:
            return set_error(GER_ERR_CAPACITY,
                             "the frontier tables of the call exceeded the no-alloc pool of 524288 slots");
        case DERR_FULL:
            return set_error(GER_ERR_CAPACITY, "a frontier table ran out of free slots (load factor broken)");
        case DERR_ELL: return set_error(GER_ERR_INVALID, "truncation length undefined (lambda >= 1)");
        case DERR_CHUNKS: return set_error(GER_ERR_CUDA, "a walk launch's chunk layout exceeded the partial-sum array");
        default: return set_error(GER_ERR_CUDA, "unknown device error");
    }
}
