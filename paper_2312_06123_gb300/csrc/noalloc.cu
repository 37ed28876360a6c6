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
// Limits: at most kNoAllocMaxQueries queries per call, at most kNoAllocCap
// push pairs per SMM iteration of a query, kNoAllocPool lookup entries per
// call; beyond them the call fails with GER_ERR_CAPACITY. The array lives
// in every GPU that loads this module, until the process exits.
#include <mutex>

#include "../../include/geer.h"
#include "geer_internal.cuh"
#include "geer_kernels.h"

namespace geer {

namespace {

constexpr int64_t kNoAllocMaxQueries = 64;
constexpr int kNoAllocSlots = 4;            // CTAs of the SMM kernel
constexpr int64_t kNoAllocCap = 1 << 16;    // push pairs per SMM iteration
constexpr int64_t kNoAllocPool = 1 << 19;   // lookup-table entries per call
constexpr size_t kNoAllocBytes = 32u << 20; // 32 MiB per GPU

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// byte offsets of the regions inside the array
constexpr size_t kOffCounters = 0;  // work counter, error flag (int), pool cursor (u64)
constexpr size_t kOffState = align256(kOffCounters + 64);
constexpr size_t kOffChunk = align256(kOffState + sizeof(QState) * kNoAllocMaxQueries);
constexpr size_t kOffPartial = align256(kOffChunk + sizeof(int64_t) * (kNoAllocMaxQueries + 1));
constexpr size_t kOffI32 = align256(kOffPartial + sizeof(Partial) * kNoAllocMaxQueries * kMaxChunksPerQuery);
constexpr size_t kF = kNoAllocCap + 2;
constexpr size_t kOffVal = align256(kOffI32 + sizeof(int32_t) * kNoAllocSlots * (5 * kNoAllocCap + 3 * kF + 2));
constexpr size_t kOffBits = align256(kOffVal + sizeof(double) * kNoAllocSlots * 4 * kF);
constexpr size_t kOffPool = align256(kOffBits + kNoAllocSlots * 2 * kF);
constexpr size_t kEnd = kOffPool + sizeof(GEntry) * kNoAllocPool;
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
    if (!(o.delta > 0.0 && o.delta < 1.0) || o.tau < 1 || o.tau > 20 ||
        (o.precision != GER_FP32 && o.precision != GER_FP64) ||
        (o.switch_policy != GER_SWITCH_RULE && o.switch_policy != GER_SWITCH_FIXED) ||
        (o.ell_formula != GER_ELL_REFINED && o.ell_formula != GER_ELL_PENG))
        return set_error(GER_ERR_INVALID, "invalid options");
    if (o.sparse_cap > kNoAllocCap)
        return set_error(GER_ERR_CAPACITY, "sparse_cap above the no-alloc limit of 65536 pairs");
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
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return set_error(GER_ERR_CUDA, "cudaSetDevice failed");
    unsigned char* base = nullptr;
    rc = scratch_address(device, &base);
    if (rc) return rc;
    cudaStream_t st = stream ? reinterpret_cast<cudaStream_t>(stream) : (cudaStream_t)0;

    int* counters = reinterpret_cast<int*>(base + kOffCounters);
    unsigned long long* pool_used = reinterpret_cast<unsigned long long*>(base + kOffCounters + 16);
    QState* qs = reinterpret_cast<QState*>(base + kOffState);
    // the array keeps the previous call's contents: reset the counters
    if (cudaMemsetAsync(base + kOffCounters, 0, 64, st) != cudaSuccess) {
        cudaGetLastError();
        return set_error(GER_ERR_CUDA, "cudaMemsetAsync of the no-alloc counters failed");
    }
    SmmArgs a;
    a.g = dg;
    a.nq = (int32_t)q;
    a.q_index_base = 0;
    a.st = qs;
    a.s = s_dev;
    a.t = t_dev;
    a.eps = eps_dev;
    a.eps_scalar = 0.0;
    a.lambda = lambda;
    a.delta = o.delta;
    a.tau = o.tau;
    a.ell_formula = o.ell_formula;
    a.policy = o.switch_policy;
    a.fixed_lb = o.fixed_ell_b;
    int nbits = 0;
    for (int64_t x = dg.n - 1; x > 0; x >>= 1) ++nbits;
    a.nbits = nbits < 1 ? 1 : nbits;
    a.cap = o.sparse_cap > 0 ? o.sparse_cap : kNoAllocCap;
    a.scr_i32 = reinterpret_cast<int32_t*>(base + kOffI32);
    a.scr_val = base + kOffVal;
    a.scr_bits = base + kOffBits;
    a.pool = reinterpret_cast<GEntry*>(base + kOffPool);
    a.pool_cap = kNoAllocPool;
    a.pool_used = pool_used;
    a.work_counter = counters;
    a.err_flag = counters + 1;
    const int grid = (int)(q < kNoAllocSlots ? q : kNoAllocSlots);
    launch_smm_sparse(o.precision == GER_FP64, a, grid, st);
    AmcArgs m;
    m.g = dg;
    m.nq = (int32_t)q;
    m.st = qs;
    m.chunk_begin = reinterpret_cast<int64_t*>(base + kOffChunk);
    m.partial = reinterpret_cast<Partial*>(base + kOffPartial);
    m.partial_cap = kNoAllocMaxQueries * kMaxChunksPerQuery;
    m.pool = a.pool;
    m.seed = o.seed;
    m.tau = o.tau;
    m.delta = o.delta;
    m.err_flag = counters + 1;
    for (int b = 1; b <= o.tau; ++b) {
        m.batch = b;
        launch_amc_schedule(m, st);
        launch_amc_walk(m, sm_count * 8, st);
        launch_amc_reduce(m, (int)q, st);
    }
    launch_finalize(qs, q, r_dev, stats_dev, st);
    note_launches(2 + 3 * o.tau);
    int derr = 0;
    if (cudaMemcpyAsync(&derr, counters + 1, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        return set_error(GER_ERR_CUDA, cudaGetErrorString(cudaGetLastError()));
    }
    switch (derr) {
        case DERR_NONE: return GER_OK;
        case DERR_NODE_RANGE: return set_error(GER_ERR_NODE_RANGE, "a query node is outside [0, n) or eps <= 0");
        case DERR_CAPACITY:
            return set_error(GER_ERR_CAPACITY, "an SMM iteration exceeded the no-alloc limit of 65536 push pairs");
        case DERR_TABLE:
            return set_error(GER_ERR_CAPACITY, "lookup tables exceeded the no-alloc limit of 524288 entries");
        default: return set_error(GER_ERR_INVALID, "truncation length undefined (lambda >= 1)");
    }
}
