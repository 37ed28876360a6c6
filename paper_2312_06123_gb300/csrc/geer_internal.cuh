// geer_internal.cuh -- device-side building blocks and the state shared by
// the GEER kernels (sparse SMM, AMC walks, spectral bound). Internal to the
// CUDA library; nothing here is visible through include/geer.h.
#pragma once

#include <cstdint>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "../../include/geer.h"

namespace geer {

constexpr int kCta = 256;          // threads per CTA of the SMM / reduction kernels
constexpr int kWarps = kCta / 32;
// CTA of the one-CTA table allocation, which walks every query in order:
// one tile covers 1,024 queries, so their loads go out together and one scan
// orders them. (Not for kernels with per-query FP64 work: the FP64 pipe of
// one SM is narrow, so those spread their queries over many SMs.)
constexpr int kSerialCta = 1024;
constexpr int kSerialWarps = kSerialCta / 32;
// CTA of the kernels with one thread per query (set-up, decision, outputs):
// each thread writes its query's few hundred bytes of state with scattered
// stores, so the queries are spread over many SMs
constexpr int kQueryCta = 32;
__host__ __device__ constexpr int query_grid(int64_t nq) {
    return (int)((nq + kQueryCta - 1) / kQueryCta < 8192 ? (nq + kQueryCta - 1) / kQueryCta : 8192);
}
constexpr int kPairsPerWarpRound = 16;  // walk pairs per warp per round (2 lanes per pair)
constexpr int kMaxChunksPerQuery = 4096;

// query lifecycle
enum : int32_t { ST_SMM = 0, ST_AMC = 1, ST_DONE = 2, ST_ERROR = 3 };

// device error codes (mirrored into the host status codes)
// DERR_FULL: a frontier table had no free slot left, which the load factor
// (capacity >= twice the push pairs) rules out; the probe gives up instead of
// looping.
// DERR_CHUNKS: a walk launch's chunk layout outgrew the partial-sum array
// (at most kMaxChunksPerQuery per query); the launch walks nothing.
enum : int32_t { DERR_NONE = 0, DERR_NODE_RANGE = 1, DERR_CAPACITY = 2, DERR_TABLE = 3, DERR_ELL = 4, DERR_FULL = 5,
                 DERR_CHUNKS = 6 };

// Per-query state, one record per query of a batch (device memory).
struct QState {
    int32_t s, t;
    int32_t qidx, pad0;       // index in the caller's batch (walk RNG key)
    double eps;
    int32_t ds, dt;
    int32_t ell, ell_b, lf, status;
    int32_t batch, err;       // batches completed; device error code
    double r_b, r_f, r;
    double psi, volume, h, f_last;
    int64_t eta0, eta;        // walk pairs: first batch, current batch
    int64_t walks, walk_steps;
    uint64_t checksum;
    int64_t ppc;              // walk pairs per chunk in the current batch
    int64_t nchunks;          // chunks in the current batch
    int64_t table_off;        // entry offset of this query's lookup table
    int32_t table_mask;       // capacity - 1 (power of two), -1: no table
    int32_t front;            // |V_s u V_t| after the last SMM iteration
    const void* dense_vals;   // dense engine: (s*, t*) of node v at dense_vals + v * dense_stride
    int32_t dense_stride;     // values per row of the query's dense block
    int32_t pad1;
};

// One slot of a query's frontier table (open addressing, linear probing):
// node v, its support bits (1: in V_s, 2: in V_t) and
// g(v) = s*(v)/d(s) - t*(v)/d(t), the per-visit term of Z_k (Eq. 11). The
// table of a query's last SMM iteration is the lookup table of its walks.
struct __align__(16) GEntry {
    int32_t v;      // -1: empty
    uint32_t bits;  // support bits (low 2) | owning query index << 2
    double g;
};

// Per-query scratch of the SMM phase (device memory), reset by each decision.
struct __align__(16) QSmm {
    int32_t run;                 // 1 while SMM iterations continue
    int32_t shift_s, shift_t;    // fixed-point scales 2^shift of s*, t*
    int32_t lb_target;           // iterations wanted by a fixed policy, -1: rule
    int32_t want;                // slots requested for the next table, 0: none
    int32_t dense;               // 1: this query's SMM runs on the dense engine
    int32_t dgo;                 // dense engine: 1 while iterations continue
    int32_t dblock, dcol;        // dense block and column pair
    int32_t pad_m;
    int64_t tab_off, tab_cap;    // table of the current frontier
    int64_t ntab_off, ntab_cap;  // table being filled
    unsigned long long vol_paper;  // sum_{V_s} d + sum_{V_t} d (Eq. 17)
    unsigned long long vol_union;  // sum_{V_s u V_t} d: push pairs of the next iteration
    unsigned long long count;      // |V_s u V_t|
    unsigned long long max1s, max1t, max2s, max2t;  // bit patterns of non-negative doubles
    unsigned long long cnt1s, cnt1t;                // entries equal to max1
    double sval[4];              // s*(s), t*(s), s*(t), t*(t)
    double inv_ds, inv_dt;       // 1/d(s), 1/d(t)
    // membership filters of the tables of iterations with parity 0 and 1
    // (tables of at most kFilterSlots slots; see filter_bit)
    uint32_t filt[2][32];
};

// Control block of the SMM phase (device memory, zeroed before a batch).
// Table slots: the F_0 tables of queries 0..nq-1 sit at [0, 8 nq); every
// later table is handed out by an atomic bump of `cursor` from 8 nq on, in
// the decision that asks for it. The advance after a decision clears the
// slots handed out since `mark` and records them as the next iteration's
// table range.
struct SmmCtl {
    unsigned long long cursor;   // slots handed out beyond the F_0 tables
    unsigned long long mark;     // cursor at the last advance
    int64_t lo[2], hi[2];        // slot range of the tables of iterations with this parity
    int32_t n_want;              // queries of the current decision that continue
    int32_t n_go;                // n_want of the last decision (the host loop reads it)
    int32_t n_heavy;             // chunks of high-degree frontier nodes left to the heavy push
    int32_t iter;                // current SMM iteration (0: the initial frontier)
    // hybrid engine: dense columns handed out, queries moved by the last
    // decision, dense blocks already zeroed
    int32_t dense_next, n_mig, dense_open;
    int32_t heavy_max;           // largest heavy-push chunk count of any iteration
    uint32_t adv_done;           // CTAs of the advance kernel finished (last one keeps the books)
    int32_t pad;
};

// slots of one query's F_0 table (F_0 = {s, t}; load 1/4)
constexpr int kF0Slots = 8;

// What a walk chunk needs of its query, packed by the batch schedule (one
// record per query in AMC).
struct __align__(16) WalkQ {
    int32_t s, t;
    uint2 s_info, t_info;     // {first edge, degree} of s and t
    int32_t lf, qidx;
    int64_t eta, ppc;         // walk pairs of this batch, pairs per chunk
    int64_t table_off;        // lookup table (mask >= 0) ...
    int32_t mask, dstride;
    const void* dvals;        // ... or the query's dense column (mask < 0)
    double inv_ds, inv_dt;
    const uint32_t* filt;     // membership filter of the lookup table (null: none)
};

// Per-chunk partial sums of the walk kernel.
struct Partial {
    double sz, sz2;
    uint64_t cs;
};

// Graph arrays on the device.
struct DevGraph {
    int64_t n, nnz;
    const int64_t* row_ptr;
    const int32_t* col_idx;
    const uint2* node_info;  // per node {first edge, degree} when nnz < 2^32, else null
    // per edge e = (u, v): {v, first edge of v, degree of v, 0} (null when absent): a walk
    // step's one load brings the next step's row as well
    const uint4* edge_rec = nullptr;
    // the walks' copy of col_idx packed at kPackBits(pack_k) bits per entry,
    // pack_k entries per 16-byte unit (entry e in unit e / pack_k); null with
    // pack_k = 0 when not built (the walks then read col_idx)
    const uint4* cols_packed = nullptr;
    int32_t pack_k = 0;
};

// Entries per 16-byte unit of the packed neighbour lists and their width:
// ids below 2^16 in 16 bits (8 per unit), below 2^21 in 21 bits (6 per
// unit), below 2^25 in 25 bits (5 per unit); larger graphs keep col_idx.
__host__ __device__ constexpr int pack_bits(int k) { return k == 8 ? 16 : (k == 6 ? 21 : (k == 5 ? 25 : 32)); }
__host__ __device__ constexpr int pack_k_for(int64_t n) {
    return n <= (int64_t)1 << 16 ? 8 : (n <= (int64_t)1 << 21 ? 6 : (n <= (int64_t)1 << 25 ? 5 : 0));
}

// Entry e of the packed neighbour lists (one 16-byte load through L2 only:
// a walk reads edges uniformly, so these loads almost never hit L1 and would
// only evict the node records and lookup tables there; the entry may
// straddle two 32-bit words of its unit, never the unit).
template <int K>
__device__ __forceinline__ int32_t packed_col(const uint4* cols, uint32_t e) {
    constexpr int B = pack_bits(K);
    const uint32_t u = e / K, j = e - u * K;
    const uint4 w = __ldcg(cols + u);
    const uint32_t o = j * B, wi = o >> 5, sh = o & 31;
    const uint32_t lo = wi == 0 ? w.x : (wi == 1 ? w.y : (wi == 2 ? w.z : w.w));
    const uint32_t hi = wi == 0 ? w.y : (wi == 1 ? w.z : (wi == 2 ? w.w : 0u));
    return (int32_t)(__funnelshift_r(lo, hi, sh) & ((1u << B) - 1u));
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11)
// ---------------------------------------------------------------------------
#ifndef GEER_PHILOX_UNROLL
#define GEER_PHILOX_UNROLL 10
#endif
constexpr int kPhiloxUnroll = GEER_PHILOX_UNROLL;  // rounds unrolled (code size of the walk loop)
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
    constexpr uint32_t kMul0 = 0xD2511F53u, kMul1 = 0xCD9E8D57u;
    constexpr uint32_t kWeyl0 = 0x9E3779B9u, kWeyl1 = 0xBB67AE85u;
#pragma unroll kPhiloxUnroll
    for (int r = 0; r < 10; ++r) {
        uint32_t lo0 = kMul0 * c.x, hi0 = __umulhi(kMul0, c.x);
        uint32_t lo1 = kMul1 * c.z, hi1 = __umulhi(kMul1, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += kWeyl0;
        k.y += kWeyl1;
    }
    return c;
}

// splitmix64 finaliser (Steele, Lea, Flood, OOPSLA'14), for walk checksums
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t walk_hash(int32_t endpoint, int64_t k, int sigma, int b) {
    uint64_t x = (uint64_t)(uint32_t)endpoint + 0x9E3779B97F4A7C15ull * (uint64_t)(2 * k + sigma + 1) +
                 ((uint64_t)b << 58);
    return mix64(x);
}

// murmur3 32-bit finaliser, for the lookup tables
__device__ __forceinline__ uint32_t hash32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return h;
}

// Membership filter of a small frontier table: 1,024 bits, one 32-bit word
// per lane of a warp, with bit filter_bit(v) set for every node v of the
// table. A walk step whose node's bit is clear skips the lookup (g = 0: the
// node is outside the support) -- most of a short SMM's walk nodes are. The
// bit comes from the top ten bits of the node's hash, the table slot from
// its low bits (tables with a filter have at most 2^12 slots).
constexpr int kFilterWords = 32;
constexpr int64_t kFilterSlots = 4096;
__device__ __forceinline__ uint32_t filter_bit(uint32_t hash) { return hash >> 22; }

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// ---------------------------------------------------------------------------
// CTA-wide helpers (blockDim.x == kCta)
// ---------------------------------------------------------------------------

// Inclusive warp scan of a 64-bit value.
__device__ __forceinline__ int64_t warp_incl_scan(int64_t x) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// Exclusive CTA scan of one value per thread; returns the prefix and writes
// the CTA total to *total (all threads). smem: kWarps + 1 int64.
// Exclusive scan over a CTA of NW warps (NW <= 32); smem holds NW + 1
// values. Returns x's exclusive prefix and the CTA total.
template <int NW>
__device__ __forceinline__ int64_t cta_excl_scan_w(int64_t x, int64_t* smem, int64_t* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t inc = warp_incl_scan(x);
    if (lane == 31) smem[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int64_t w = lane < NW ? smem[lane] : 0;
        int64_t wi = warp_incl_scan(w);
        if (lane < NW) smem[lane] = wi - w;
        if (lane == NW - 1) smem[NW] = wi;
    }
    __syncthreads();
    int64_t r = smem[warp] + inc - x;
    *total = smem[NW];
    __syncthreads();
    return r;
}

__device__ __forceinline__ int64_t cta_excl_scan(int64_t x, int64_t* smem, int64_t* total) {
    return cta_excl_scan_w<kWarps>(x, smem, total);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// merge two (max1, max2) pairs of a multiset
__device__ __forceinline__ void top2_merge(double& a, double& b, double a2, double b2) {
    double hi = fmax(a, a2), lo = fmin(a, a2);
    b = fmax(lo, fmax(b, b2));
    a = hi;
}

__device__ __forceinline__ void warp_top2(double& a, double& b) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        double a2 = __shfl_xor_sync(0xffffffffu, a, o);
        double b2 = __shfl_xor_sync(0xffffffffu, b, o);
        top2_merge(a, b, a2, b2);
    }
}

// ---------------------------------------------------------------------------
// switch quantities (Eqs. 8, 9, 17) and the learned switch's inputs
// ---------------------------------------------------------------------------

// psi (Eq. 9), eta0 = max(1, ceil(eta*/2^(tau-1))) with eta* from Eq. (8),
// h = (2^tau - 1) eta0; log_2tau_delta = log(2 tau / delta), the same for
// every query (computed on the host)
__device__ __forceinline__ void switch_quantities(int64_t lf, double s1, double s2, double t1, double t2, double ds,
                                                  double dt, double eps, double log_2tau_delta, int tau, double* psi,
                                                  int64_t* eta0, double* h) {
    const double up = (double)((lf + 1) / 2), dn = (double)(lf / 2);
    const double p = 2.0 * up * (s1 / ds + t1 / dt) + 2.0 * dn * (s2 / ds + t2 / dt);
    const double es = 2.0 * p * p * log_2tau_delta / (eps * eps);
    int64_t e0 = (int64_t)ceil(es * ldexp(1.0, 1 - tau));  // (scaling by a power of two is exact)
    if (e0 < 1) e0 = 1;
    *psi = p;
    *eta0 = e0;
    *h = (double)((((int64_t)1 << tau) - 1) * e0);
}

// max_1, max_2 of s* and t* after an SMM iteration (entries outside the
// frontier are zero, so accumulators starting at 0.0 already include them)
__device__ __forceinline__ void smm_maxima(const QSmm* M, double* s1, double* s2, double* t1, double* t2) {
    *s1 = __longlong_as_double((long long)M->max1s);
    *t1 = __longlong_as_double((long long)M->max1t);
    *s2 = M->cnt1s >= 2 ? *s1 : __longlong_as_double((long long)M->max2s);
    *t2 = M->cnt1t >= 2 ? *t1 : __longlong_as_double((long long)M->max2t);
}

// The learned switch: a 6 -> 64 -> 64 -> 1 ReLU network with FP16 weights and
// FP32 arithmetic. Parameter order (one FP16 array): W1[64][6], b1[64],
// W2[64][64] (W2[j][k] multiplies hidden unit k of layer 1), b2[64], W3[64], b3.
constexpr int kMlpIn = 6;
constexpr int kMlpH = 64;
constexpr int kMlpOffW1 = 0;
constexpr int kMlpOffB1 = kMlpOffW1 + kMlpH * kMlpIn;
constexpr int kMlpOffW2 = kMlpOffB1 + kMlpH;
constexpr int kMlpOffB2 = kMlpOffW2 + kMlpH * kMlpH;
constexpr int kMlpOffW3 = kMlpOffB2 + kMlpH;
constexpr int kMlpOffB3 = kMlpOffW3 + kMlpH;
constexpr int kMlpParams = kMlpOffB3 + 1;  // 4673

// Raw inputs of the learned switch (the network's inputs are FP32, so they
// are computed in FP32): log d(s), log d(t), l - l_b, log(volume), log h(l -
// l_b) (0 when no walk is left), max_1(s*)/d(s) + max_1(t*)/d(t), from
// Eq. (17)'s state after iteration l_b (h from switch_quantities).
__device__ __forceinline__ void switch_features(int32_t ds, int32_t dt, int64_t lf, unsigned long long vol, double h,
                                                double s1, double t1, float f[kMlpIn]) {
    const float fds = (float)ds, fdt = (float)dt;
    f[0] = logf(fds);
    f[1] = logf(fdt);
    f[2] = (float)lf;
    f[3] = logf((float)vol);
    f[4] = h > 0.0 ? logf((float)h) : 0.0f;
    f[5] = (float)s1 / fds + (float)t1 / fdt;
}

// Floats of the network's FP32 weight copy (a whole number of 16-byte FP16
// vectors).
constexpr int kMlpStaged = (kMlpParams + 7) / 8 * 8;

// Where parameter p sits in the staged copy: W1 and W2 transposed (input k
// of unit j at k * 64 + j), so the lanes of a warp evaluating units j and
// j + 32 read consecutive floats; biases and W3 in place.
__device__ __forceinline__ int mlp_staged_index(int p) {
    if (p < kMlpOffB1) return kMlpOffW1 + ((p - kMlpOffW1) % kMlpIn) * kMlpH + (p - kMlpOffW1) / kMlpIn;
    if (p >= kMlpOffW2 && p < kMlpOffB2) return kMlpOffW2 + ((p - kMlpOffW2) % kMlpH) * kMlpH + (p - kMlpOffW2) / kMlpH;
    return p;
}

// The whole CTA converts the network's FP16 weights into the FP32 copy the
// decisions read (16-byte loads; the weight buffer is allocated with 16
// bytes to spare, so the last vector stays inside it; the padding lands past
// the parameters).
// A thread's loads are issued in groups of kMlpStageGroup before any is
// converted, so the staging waits for a few round trips, not one per vector.
constexpr int kMlpStageGroup = 10;
__device__ __forceinline__ void mlp_stage(float* sw, const unsigned short* w) {
    constexpr int kVecs = kMlpStaged / 8;
    const uint4* src = reinterpret_cast<const uint4*>(w);
    for (int i0 = threadIdx.x; i0 < kVecs; i0 += blockDim.x * kMlpStageGroup) {
        uint4 v[kMlpStageGroup];
#pragma unroll
        for (int g = 0; g < kMlpStageGroup; ++g) {
            const int i = i0 + g * (int)blockDim.x;
            if (i < kVecs) v[g] = __ldg(src + i);
        }
#pragma unroll
        for (int g = 0; g < kMlpStageGroup; ++g) {
            const int i = i0 + g * (int)blockDim.x;
            if (i >= kVecs) break;
            const uint32_t u[4] = {v[g].x, v[g].y, v[g].z, v[g].w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&u[e]));
                sw[mlp_staged_index(8 * i + 2 * e)] = f.x;
                sw[mlp_staged_index(8 * i + 2 * e + 1)] = f.y;
            }
        }
    }
}

// TF32 bits of x, rounded to nearest (ties away)
__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// d += a * b on the tensor cores: one 16x8 tile, k = 8, TF32 operands, FP32
// accumulation (mma.sync m16n8k8: lane (g, t) = (lane / 4, lane % 4) holds
// A rows g, g + 8 at columns t, t + 4; B rows t, t + 4 at column g; D rows
// g, g + 8 at columns 2t, 2t + 1)
__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// position of the n-th (0-based) set bit of m, -1 when m has fewer
__device__ __forceinline__ int nth_set_bit(unsigned m, int n) {
    for (int i = 0; i < n; ++i) m &= m - 1;
    return m ? __ffs(m) - 1 : -1;
}

// The network's output for the query of every lane with `ask` set (the
// lane's raw inputs in raw[]), the whole warp evaluating 16 queries per
// pass; the lane gets its own query's output (0 where it did not ask).
// Every lane of the warp must call it. Weights: the FP32 copy in global
// memory (mlp_stage's layout). The first layer and the output in FP32 on
// the CUDA cores; the 64 x 64 second layer on the tensor cores (TF32 mma):
// the FP16 weights are exact in TF32, and each first-layer activation is
// split into a TF32 part and a TF32 remainder, so the products are those of
// FP32 arithmetic (only the order of the sums differs).
__device__ __forceinline__ float mlp_eval_asked(const float* wt, const float* norm, const float (&raw)[kMlpIn],
                                                bool ask) {
    const int lane = threadIdx.x & 31, gq = lane >> 2, tq = lane & 3;
    unsigned pend = __ballot_sync(0xffffffffu, ask);
    float mine = 0.f;
    while (pend) {
        const int cnt = __popc(pend) < 16 ? __popc(pend) : 16;
        // the lanes of this pass's rows gq and gq + 8 (a repeat of row 0 past the last)
        const int first = __ffs(pend) - 1;
        int sg = nth_set_bit(pend, gq), sh = nth_set_bit(pend, gq + 8);
        if (gq >= cnt || sg < 0) sg = first;
        if (gq + 8 >= cnt || sh < 0) sh = first;
        float xg[kMlpIn], xh[kMlpIn];
#pragma unroll
        for (int k = 0; k < kMlpIn; ++k) {
            const float mean = __ldg(norm + k), sd = __ldg(norm + kMlpIn + k);
            xg[k] = (__shfl_sync(0xffffffffu, raw[k], sg) - mean) / sd;
            xh[k] = (__shfl_sync(0xffffffffu, raw[k], sh) - mean) / sd;
        }
        // first layer, straight into the A fragments of the second (k-tile n:
        // hidden units 8n + tq and 8n + tq + 4), as TF32 part and remainder
        uint32_t ahi[8][4], alo[8][4];
#pragma unroll
        for (int n = 0; n < 8; ++n) {
            const int c0 = 8 * n + tq, c1 = c0 + 4;
            float v[4] = {__ldg(wt + kMlpOffB1 + c0), __ldg(wt + kMlpOffB1 + c0), __ldg(wt + kMlpOffB1 + c1),
                          __ldg(wt + kMlpOffB1 + c1)};
#pragma unroll
            for (int k = 0; k < kMlpIn; ++k) {
                const float w0 = __ldg(wt + kMlpOffW1 + k * kMlpH + c0), w1 = __ldg(wt + kMlpOffW1 + k * kMlpH + c1);
                v[0] = fmaf(w0, xg[k], v[0]);
                v[1] = fmaf(w0, xh[k], v[1]);
                v[2] = fmaf(w1, xg[k], v[2]);
                v[3] = fmaf(w1, xh[k], v[3]);
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float h = fmaxf(v[e], 0.f);
                ahi[n][e] = to_tf32(h);
                alo[n][e] = to_tf32(h - __uint_as_float(ahi[n][e]));
            }
        }
        // second layer tile by tile (units 8 nt .. 8 nt + 7), then the output
        // layer's terms of this lane's two units per row
        float yg = 0.f, yh = 0.f;
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            float d[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int kt = 0; kt < 8; ++kt) {
                // B rows = inputs 8 kt + tq (+ 4), column = unit 8 nt + gq: W2[unit][input]
                const uint32_t b0 = to_tf32(__ldg(wt + kMlpOffW2 + (8 * kt + tq) * kMlpH + 8 * nt + gq));
                const uint32_t b1 = to_tf32(__ldg(wt + kMlpOffW2 + (8 * kt + tq + 4) * kMlpH + 8 * nt + gq));
                mma_tf32(d, ahi[kt], b0, b1);
                mma_tf32(d, alo[kt], b0, b1);
            }
            const int c = 8 * nt + 2 * tq;
            const float b2a = __ldg(wt + kMlpOffB2 + c), b2b = __ldg(wt + kMlpOffB2 + c + 1);
            const float w3a = __ldg(wt + kMlpOffW3 + c), w3b = __ldg(wt + kMlpOffW3 + c + 1);
            yg = fmaf(w3a, fmaxf(d[0] + b2a, 0.f), yg);
            yg = fmaf(w3b, fmaxf(d[1] + b2b, 0.f), yg);
            yh = fmaf(w3a, fmaxf(d[2] + b2a, 0.f), yh);
            yh = fmaf(w3b, fmaxf(d[3] + b2b, 0.f), yh);
        }
        // the sums over the quad's 64 units, plus the output bias
        yg += __shfl_xor_sync(0xffffffffu, yg, 1);
        yg += __shfl_xor_sync(0xffffffffu, yg, 2);
        yh += __shfl_xor_sync(0xffffffffu, yh, 1);
        yh += __shfl_xor_sync(0xffffffffu, yh, 2);
        const float b3 = __ldg(wt + kMlpOffB3);
        // each asking lane of this pass takes its row's output (row r: quad r mod 8)
        const bool in_pass = ((pend >> lane) & 1u) && __popc(pend & ((1u << lane) - 1u)) < cnt;
        const int r = in_pass ? __popc(pend & ((1u << lane) - 1u)) : 0;
        const float vg = __shfl_sync(0xffffffffu, yg, (r & 7) * 4);
        const float vh = __shfl_sync(0xffffffffu, yh, (r & 7) * 4);
        if (in_pass) mine = (r < 8 ? vg : vh) + b3;
        // drop this pass's rows
        const int last = nth_set_bit(pend, cnt - 1);
        pend = last >= 31 ? 0u : pend & ~((2u << last) - 1u);
    }
    return mine;
}

// The outputs of one query (its record of the batch state): r' and, when
// asked for, the statistics record of include/geer.h.
__device__ __forceinline__ void store_outputs(const QState& Q, int64_t q, double* r, ger_query_stats* stats) {
    r[q] = Q.r;
    if (stats) {
        ger_query_stats o;
        o.ell = Q.ell;
        o.ell_b = Q.ell_b;
        o.batches = Q.batch;
        o.flags = Q.err;
        o.eta0 = Q.eta0;
        o.walks = Q.walks;
        o.walk_steps = Q.walk_steps;
        o.r_b = Q.r_b;
        o.r_f = Q.r_f;
        o.psi = Q.psi;
        o.f_last = Q.f_last;
        o.volume = Q.volume;
        o.h = Q.h;
        o.checksum = Q.checksum;
        stats[q] = o;
    }
}

}  // namespace geer
