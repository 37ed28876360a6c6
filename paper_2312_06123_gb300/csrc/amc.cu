// amc.cu -- AMC phase of GEER (Algorithm 1 with the residual vectors s*, t*
// of Algorithm 3): batches of walk pairs, the per-query sums of Z_k and
// Z_k^2, and the empirical-Bernstein stop of Lemma 2 / Eq. (7) at delta/tau.
//
// Work layout of one batch b: query q runs eta_q walk pairs, cut into
// chunks of ppc pairs (a multiple of 16 W, at most kMaxChunksPerQuery
// chunks). A warp owns one chunk at a time: lanes 2i and 2i+1 walk pairs
// k0 + i + 16 w (w < W walks per lane), lane 2i from s (sigma = 0), lane
// 2i+1 from t (sigma = 1). Each walk step
// draws one 32-bit word of Philox4x32-10 keyed by (seed) with counter
// (k, 2(b-1)+sigma, query index, (j-1) >> 2), word (j-1) & 3, and moves to
// neighbour floor(draw * d(w) / 2^32) in CSR order -- the same specification
// the CPU oracle implements, so walk endpoints agree bit for bit.
// Z_k = sum over the S walk of g(w_j) - sum over the T walk of g(w_j) with
// g(v) = s*(v)/d(s) - t*(v)/d(t) read from the query's lookup table (Eq. 11;
// the start node w_0 is not counted, as E[Z_k] = q(s,t) of Eqs. 12-13 requires).
// Per-chunk sums go to a partial array; the reduce kernel adds a query's
// chunks in a fixed order, so results do not depend on scheduling. When the
// first three batches' walks are few, they share the first launch (the
// chunks of a query are its batch-1, then batch-2, then batch-3 chunks) and
// the reduce evaluates them in order, ignoring batches after a stop.
// A launch's chunks are numbered query by query. For batches of up to
// kSmemChunkBegin - 1 queries the schedule and the reduce write per-query
// chunk counts and every walk CTA builds the prefix in shared memory (CTA 0
// also stores it for the reduce); larger batches get the prefix from a
// one-CTA layout.
#include "geer_internal.cuh"
#include "geer_kernels.h"

namespace geer {

#ifndef GEER_WALKS_PER_LANE
#define GEER_WALKS_PER_LANE 1
#endif
constexpr int kWalksPerLane = GEER_WALKS_PER_LANE;
// chunks a warp takes per ticket (one atomic on the shared ticket counter each)
#ifndef GEER_CHUNKS_PER_TICKET
#define GEER_CHUNKS_PER_TICKET 1
#endif
constexpr int kChunksPerTicket = GEER_CHUNKS_PER_TICKET;

// Row start and degree of node w.
__device__ __forceinline__ uint2 node_row(const DevGraph& g, int32_t w) {
    if (g.node_info) return __ldg(g.node_info + w);
    const int64_t rs = __ldg(g.row_ptr + w);
    return make_uint2((uint32_t)rs, (uint32_t)(__ldg(g.row_ptr + w + 1) - rs));
}

// node_row when the node records are known to exist (the packed neighbour
// lists, K > 0, are built only with them)
template <int K>
__device__ __forceinline__ uint2 node_row_k(const DevGraph& g, int32_t w) {
    if constexpr (K > 0) return __ldg(g.node_info + w);
    else return node_row(g, w);
}

__device__ __forceinline__ const int32_t* row_base(const DevGraph& g, int32_t w, uint2 info) {
    // node_info holds the low 32 bits of the row start (nnz < 2^32); otherwise
    // re-read the full 64-bit start
    return g.node_info ? g.col_idx + info.x : g.col_idx + __ldg(g.row_ptr + w);
}

// Chunks per query and batch when a launch walks nb batches (the common
// counts without a run-time 64-bit division).
__device__ __forceinline__ int64_t max_chunks(int nb) {
    return nb == 1 ? kMaxChunksPerQuery
                   : (nb == 2 ? kMaxChunksPerQuery / 2 : (nb == 3 ? kMaxChunksPerQuery / 3 : kMaxChunksPerQuery / nb));
}

// Walk pairs per chunk and chunk count of a batch of eta walk pairs, at
// most maxc chunks (a chunk is a whole number of warp rounds).
__device__ __forceinline__ void chunk_layout(int64_t eta, int64_t maxc, int64_t* ppc, int64_t* nch) {
    const int64_t unit = kWalksPerLane * kPairsPerWarpRound;
    const int64_t units = (eta + unit - 1) / unit;
    if (units <= maxc) {  // one warp round a chunk (the general case below, without its divisions)
        *ppc = unit;
        *nch = units;
        return;
    }
    const int64_t c = maxc;
    *ppc = unit * ((units + c - 1) / c);
    *nch = (eta + *ppc - 1) / *ppc;
}

// Chunk layout of the next walk launch (batches b .. b + nb - 1, batch i of
// a query having eta * 2^(i - b) pairs) for every query still in AMC, by one
// CTA, for batches too large for a walk CTA's shared-memory prefix: per query
// its chunk count over the launch's batches, and their prefix in
// chunk_begin. Reads the query state through the L2 (it was written by
// other CTAs of the same kernel).
__device__ void schedule_cta(const AmcArgs& a, int nb) {
    __shared__ int64_t scan[kWarps + 1];
    __shared__ int64_t carry;
    const int tid = threadIdx.x;
    if (tid == 0) carry = 0;
    __syncthreads();
    const int64_t maxc = max_chunks(nb);
    for (int64_t tile = 0; tile < a.nq; tile += kCta) {
        const int64_t q = tile + tid;
        int64_t nch = 0;
        if (q < a.nq) {
            QState* Q = a.st + q;
            if (__ldcg(&Q->status) == ST_AMC) {
                const int64_t eta = __ldcg(&Q->eta);
                for (int i = 0; i < nb; ++i) {
                    int64_t ppc, n;
                    chunk_layout(eta << i, maxc, &ppc, &n);
                    if (i == 0) Q->ppc = ppc;
                    nch += n;
                }
                // the rest of the walk record was packed when the query entered AMC
                a.wq[q].eta = eta;
            }
            Q->nchunks = nch;
        }
        int64_t tot;
        const int64_t ex = cta_excl_scan(nch, scan, &tot);
        if (q < a.nq) a.chunk_begin[q] = carry + ex;
        __syncthreads();
        if (tid == 0) carry += tot;
        __syncthreads();
    }
    if (tid == 0) {
        a.chunk_begin[a.nq] = carry;
        *a.walk_ctr = 0ull;
    }
}

// chunk prefix entries a walk CTA holds in shared memory (int32: a small
// batch has at most 4095 x kMaxChunksPerQuery chunks)
constexpr int kSmemChunkBegin = 4096;

// Chunk counts of the next walk launch, for batches whose prefix each walk
// CTA builds itself (up to kSmemChunkBegin - 1 queries): the count of every
// query in AMC over the launch's batches (nb of them), its walk record's
// eta, and a fresh ticket counter.
__device__ void count_cta(const AmcArgs& a, int nb) {
    const int64_t maxc = max_chunks(nb);
    for (int64_t q = threadIdx.x; q < a.nq; q += blockDim.x) {
        int32_t nch = 0;
        const QState* Q = a.st + q;
        if (Q->status == ST_AMC) {
            const int64_t eta = Q->eta;
            for (int i = 0; i < nb; ++i) {
                int64_t ppc, n;
                chunk_layout(eta << i, maxc, &ppc, &n);
                nch += (int32_t)n;
            }
            a.wq[q].eta = eta;
        }
        a.chunk_count[q] = nch;
    }
    if (threadIdx.x == 0) *a.walk_ctr = 0ull;
}

__device__ void schedule_first(const AmcArgs& a, int nb) {
    if (a.nq + 1 <= kSmemChunkBegin) count_cta(a, nb);
    else schedule_cta(a, nb);
}

// Batches walked together at the start (when cheap), and the walk steps
// below which they are: the speculative batches cost at most this much, the
// launches they save are latency-bound.
#ifndef GEER_AMC_GROUP
#define GEER_AMC_GROUP 3
#endif
constexpr int kAmcGroup = GEER_AMC_GROUP;
constexpr int64_t kAmcGroupSteps = (int64_t)1 << 25;

// First layout of a batch's AMC: walk batches 1..kAmcGroup in one launch
// when their walk steps (if no query stopped early) stay below
// kAmcGroupSteps -- most queries need several batches, so little is wasted
// and two latency-bound launch pairs are saved; else batch 1 alone. The
// choice goes to *a.group for the launches that follow.
__global__ void __launch_bounds__(kCta) amc_schedule_kernel(AmcArgs a) {
    __shared__ unsigned long long tot;
    if (threadIdx.x == 0) tot = 0ull;
    __syncthreads();
    const int nb = a.tau < kAmcGroup ? a.tau : kAmcGroup;
    unsigned long long mine = 0ull;
    for (int64_t q = threadIdx.x; q < a.nq; q += blockDim.x) {
        const QState* Q = a.st + q;
        if (Q->status == ST_AMC) mine += (unsigned long long)(((1ll << nb) - 1) * Q->eta * 2 * (int64_t)Q->lf);
    }
    atomicAdd(&tot, mine);
    __syncthreads();
    const int group = tot <= (unsigned long long)kAmcGroupSteps ? nb : 1;
    if (threadIdx.x == 0) *a.group = group;
    schedule_first(a, group);
}

// g of a node whose first probe `p` (slot h) is already loaded; a node absent
// from the table (outside the support) has g = 0. A full cycle of probes
// without v or an empty slot cannot happen while the load stays at most 1/2:
// it raises DERR_FULL and counts 0.
__device__ __forceinline__ double resolve_g(const GEntry* tab, int32_t mask, int32_t v, int4 p, uint32_t h,
                                            int* err_flag) {
    for (uint32_t probe = 0; probe <= (uint32_t)mask; ++probe) {
        if (p.x == v) return __hiloint2double(p.w, p.z);
        if (p.x == -1) return 0.0;
        h = (h + 1) & (uint32_t)mask;
        p = __ldg(reinterpret_cast<const int4*>(tab + h));
    }
    atomicCAS(err_flag, 0, DERR_FULL);
    return 0.0;
}

// resolve_g for a step whose lookup runs: g is added to z only where v is
// in the table (no FP64 addition of the zero of an absent node).
__device__ __forceinline__ void resolve_add(const GEntry* tab, int32_t mask, int32_t v, int4 p, uint32_t h,
                                            int* err_flag, double& z) {
    for (uint32_t probe = 0; probe <= (uint32_t)mask; ++probe) {
        if (p.x == v) {
            z += __hiloint2double(p.w, p.z);
            return;
        }
        if (p.x == -1) return;
        h = (h + 1) & (uint32_t)mask;
        p = __ldg(reinterpret_cast<const int4*>(tab + h));
    }
    atomicCAS(err_flag, 0, DERR_FULL);
}

// W walk pairs per lane pair and round: lanes 2i, 2i+1 walk pairs
// k0 + i + 16 w (w < W), from s and from t. The W walks of a lane advance in
// lockstep so that their loads overlap; each step issues the next node's
// row record and its first lookup probe together.
#ifndef GEER_WALK_MINB
#define GEER_WALK_MINB 4
#endif

// Walks of chunk L of query WQ in a launch that walks its batches batch0 ..
// batch0 + nbatch - 1 (eta pairs in batch0, doubling), chunked by chunk_layout at
// max_chunks(nbatch) chunks per batch. Returns the chunk's sums of
// Z_k, Z_k^2 and the walk checksum, reduced over the warp.
template <int W, bool REC, int K>
__device__ __forceinline__ void walk_chunk(const AmcArgs& a, const WalkQ* WQ, int64_t L, int64_t eta, int batch0,
                                           int nbatch, int lane, double* out_sz, double* out_sz2, uint64_t* out_cs) {
    const int sigma = lane & 1;
    const uint2 key = make_uint2((uint32_t)a.seed, (uint32_t)(a.seed >> 32));
    const DevGraph g = a.g;
    const int64_t maxc = max_chunks(nbatch);
    // which of the unit's batches this chunk belongs to, and its place in it
    int64_t ppc, nchb;
    int bi = 0;
    for (;;) {
        chunk_layout(eta, maxc, &ppc, &nchb);
        if (L < nchb || bi == nbatch - 1) break;
        L -= nchb;
        eta <<= 1;
        ++bi;
    }
    const int batch = batch0 + bi;
    const uint32_t lane_ctr = (uint32_t)(2 * (batch - 1) + sigma);
    const int32_t lf = WQ->lf, qidx = WQ->qidx;
    const int32_t start = sigma ? WQ->t : WQ->s;
    const GEntry* tab = a.pool + WQ->table_off;
    const int32_t mask = WQ->mask;
    const uint32_t* filt = WQ->filt;
    // dense-engine queries: (s*, t*) read directly from their block column
    const char* dvals = reinterpret_cast<const char*>(WQ->dvals);
    const int64_t dstride = WQ->dstride;
    const double inv_ds = WQ->inv_ds, inv_dt = WQ->inv_dt;
    const uint2 start_info = sigma ? WQ->t_info : WQ->s_info;
    const int64_t k_lo = L * ppc;
    const int64_t k_hi = min(k_lo + ppc, eta);
    double sz = 0.0, sz2 = 0.0;
    uint64_t cs = 0;
    for (int64_t k0 = k_lo; k0 < k_hi; k0 += W * kPairsPerWarpRound) {
        int64_t k[W];
        bool act[W];
        double z[W];
        int32_t w[W];
        uint2 inf[W];
        uint4 r[W];
#pragma unroll
        for (int i = 0; i < W; ++i) {
            k[i] = k0 + (lane >> 1) + i * kPairsPerWarpRound;
            act[i] = k[i] < k_hi;
            z[i] = 0.0;
            w[i] = start;
            inf[i] = start_info;
            r[i] = make_uint4(0, 0, 0, 0);
        }
        // every lane of the warp takes the same branch (REC and mask are the
        // chunk's), so warp-wide shuffles inside it are converged; lanes past
        // the chunk's last pair (act false) only predicate their loads off
        if (REC && mask >= 0) {
            // one dependent load per step: the edge record of the chosen
            // neighbour carries that neighbour's row; the lookup probe of
            // step j is resolved during step j + 1's load. The W walks of
            // the lane advance together so that their loads overlap.
            uint2 cur[W];
            int32_t pnx[W];
            uint32_t phh[W];
            int4 ppr[W];
#pragma unroll
            for (int i = 0; i < W; ++i) {
                cur[i] = start_info;
                pnx[i] = start;
                phh[i] = 0;
                ppr[i] = make_int4(0, 0, 0, 0);
            }
            for (int j = 1; j <= lf; ++j) {
                const int sub = (j - 1) & 3;
                uint4 rec[W];
#pragma unroll
                for (int i = 0; i < W; ++i) {
                    if (sub == 0)
                        r[i] = philox4x32_10(
                            make_uint4((uint32_t)k[i], lane_ctr, (uint32_t)qidx, (uint32_t)((j - 1) >> 2)), key);
                    const uint32_t d = sub == 0 ? r[i].x : (sub == 1 ? r[i].y : (sub == 2 ? r[i].z : r[i].w));
                    rec[i] = act[i] ? __ldg(g.edge_rec + cur[i].x + __umulhi(d, cur[i].y))
                                    : make_uint4((uint32_t)start, start_info.x, start_info.y, 0u);
                }
#pragma unroll
                for (int i = 0; i < W; ++i)
                    if (j > 1 && act[i]) z[i] += resolve_g(tab, mask, pnx[i], ppr[i], phh[i], a.err_flag);
#pragma unroll
                for (int i = 0; i < W; ++i) {
                    pnx[i] = (int32_t)rec[i].x;
                    cur[i] = make_uint2(rec[i].y, rec[i].z);
                    phh[i] = hash32(rec[i].x) & (uint32_t)mask;
                    ppr[i] = __ldg(reinterpret_cast<const int4*>(tab + phh[i]));
                }
            }
#pragma unroll
            for (int i = 0; i < W; ++i) {
                if (lf > 0 && act[i]) z[i] += resolve_g(tab, mask, pnx[i], ppr[i], phh[i], a.err_flag);
                w[i] = pnx[i];
                if (act[i]) cs += walk_hash(w[i], k[i], sigma, batch);
            }
        } else {
            // step j: Philox word (j-1)&3 (one generator call per 4 steps) picks the
            // next node among the current node's neighbours
            auto pick = [&](int j, int32_t (&nx)[W]) {
                const int sub = (j - 1) & 3;
#pragma unroll
                for (int i = 0; i < W; ++i) {
                    if (sub == 0 && act[i])
                        r[i] = philox4x32_10(
                            make_uint4((uint32_t)k[i], lane_ctr, (uint32_t)qidx, (uint32_t)((j - 1) >> 2)), key);
                    const uint32_t d = sub == 0 ? r[i].x : (sub == 1 ? r[i].y : (sub == 2 ? r[i].z : r[i].w));
                    if constexpr (K > 0)  // packed neighbour lists: entry first edge + pick
                        nx[i] = act[i] ? packed_col<K>(g.cols_packed, inf[i].x + __umulhi(d, inf[i].y)) : start;
                    else
                        nx[i] = act[i] ? __ldg(row_base(g, w[i], inf[i]) + __umulhi(d, inf[i].y)) : start;
                }
            };
            // one loop per value source, so the loop the warp runs holds only its own code
            if (mask >= 0) {
                // lane l holds word l of the lookup table's membership filter
                const uint32_t fw = filt ? __ldg(filt + lane) : 0xffffffffu;
                // one step with draw d[i]: the neighbour, then its row record
                // and, where its filter bit is set, the first lookup probe
                // (independent loads), then g of it
                auto step = [&](const uint32_t (&d)[W]) {
                    int32_t nx[W];
                    uint32_t hh[W];
                    int4 pr[W];
                    bool look[W];
#pragma unroll
                    for (int i = 0; i < W; ++i) {
                        if constexpr (K > 0)
                            nx[i] = act[i] ? packed_col<K>(g.cols_packed, inf[i].x + __umulhi(d[i], inf[i].y)) : start;
                        else
                            nx[i] = act[i] ? __ldg(row_base(g, w[i], inf[i]) + __umulhi(d[i], inf[i].y)) : start;
                    }
#pragma unroll
                    for (int i = 0; i < W; ++i) {
                        const uint32_t hv = hash32((uint32_t)nx[i]);
                        hh[i] = hv & (uint32_t)mask;
                        const uint32_t fb = filter_bit(hv);
                        const uint32_t fword = __shfl_sync(0xffffffffu, fw, (int)(fb >> 5));
                        look[i] = act[i] && ((fword >> (fb & 31u)) & 1u);
                        pr[i] = look[i] ? __ldg(reinterpret_cast<const int4*>(tab + hh[i])) : make_int4(-1, 0, 0, 0);
                        if (act[i]) inf[i] = node_row_k<K>(g, nx[i]);
                    }
#pragma unroll
                    for (int i = 0; i < W; ++i) {
                        if (look[i]) resolve_add(tab, mask, nx[i], pr[i], hh[i], a.err_flag, z[i]);
                        w[i] = nx[i];
                    }
                };
                auto block = [&](int j) {  // the Philox block of steps j .. j + 3
#pragma unroll
                    for (int i = 0; i < W; ++i)
                        if (act[i])
                            r[i] = philox4x32_10(
                                make_uint4((uint32_t)k[i], lane_ctr, (uint32_t)qidx, (uint32_t)((j - 1) >> 2)), key);
                };
                uint32_t d[W];
                // four steps per block, each taking its word of the block
                int j = 1;
                for (; j + 3 <= lf; j += 4) {
                    block(j);
#pragma unroll
                    for (int i = 0; i < W; ++i) d[i] = r[i].x;
                    step(d);
#pragma unroll
                    for (int i = 0; i < W; ++i) d[i] = r[i].y;
                    step(d);
#pragma unroll
                    for (int i = 0; i < W; ++i) d[i] = r[i].z;
                    step(d);
#pragma unroll
                    for (int i = 0; i < W; ++i) d[i] = r[i].w;
                    step(d);
                }
                if (j <= lf) {  // the last 1-3 steps
                    block(j);
#pragma unroll
                    for (int i = 0; i < W; ++i) d[i] = r[i].x;
                    step(d);
                    if (j + 1 <= lf) {
#pragma unroll
                        for (int i = 0; i < W; ++i) d[i] = r[i].y;
                        step(d);
                    }
                    if (j + 2 <= lf) {
#pragma unroll
                        for (int i = 0; i < W; ++i) d[i] = r[i].z;
                        step(d);
                    }
                }
            } else {
                for (int j = 1; j <= lf; ++j) {
                    int32_t nx[W];
                    pick(j, nx);
#pragma unroll
                    for (int i = 0; i < W; ++i) {
                        double xs, xt;
                        if (a.dense_fp64) {
                            const double2 p2 = __ldg(reinterpret_cast<const double2*>(dvals + (size_t)nx[i] * dstride * 8));
                            xs = fabs(p2.x);  // the sign bit carries the support
                            xt = fabs(p2.y);
                        } else {
                            const float2 p2 = __ldg(reinterpret_cast<const float2*>(dvals + (size_t)nx[i] * dstride * 4));
                            xs = (double)fabsf(p2.x);
                            xt = (double)fabsf(p2.y);
                        }
                        if (act[i]) {
                            inf[i] = node_row(g, nx[i]);
                            z[i] += xs * inv_ds - xt * inv_dt;
                        }
                        w[i] = nx[i];
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < W; ++i)
                if (act[i]) cs += walk_hash(w[i], k[i], sigma, batch);
        }
#pragma unroll
        for (int i = 0; i < W; ++i) {
            const double o = __shfl_xor_sync(0xffffffffu, z[i], 1);
            if (sigma == 0 && act[i]) {
                const double zk = z[i] - o;
                sz += zk;
                sz2 += zk * zk;
            }
        }
    }
    sz = warp_sum(sz);
    sz2 = warp_sum(sz2);
    cs = warp_sum(cs);
    *out_sz = sz;
    *out_sz2 = sz2;
    *out_cs = cs;
}

// Launch-per-batch walks: a persistent grid whose warps take chunks of the
// launch's layout (chunk_begin) from a ticket counter.
template <int W, bool REC, int K>
__global__ void __launch_bounds__(256, GEER_WALK_MINB) amc_walk_kernel(AmcArgs a) {
    // the launch's chunk prefix (nq + 1 entries, staged batches only): dynamic
    // shared memory sized to the batch, so the rest of the SM's unified L1
    // keeps caching the lookup tables and node records the walks read
    extern __shared__ int32_t cbeg[];
    __shared__ int64_t scan[kWarps + 1];
    __shared__ unsigned long long s_steps;
    // batches of this launch: the first launch walks *a.group batches, the
    // launches of batches it covered have nothing to do
    int group;
    const bool fused = a.batch == 1 && a.fused_schedule;
    if (fused) {
        // the first launch lays out its own chunks: batches 1..kAmcGroup walk
        // together when their walk steps (had no query stopped) stay below
        // kAmcGroupSteps (each CTA decides the same from the walk records)
        const int nb = a.tau < kAmcGroup ? a.tau : kAmcGroup;
        if (threadIdx.x == 0) s_steps = 0ull;
        __syncthreads();
        unsigned long long mine = 0ull;
        for (int64_t q = threadIdx.x; q < a.nq; q += blockDim.x) {
            const WalkQ* wr = a.wq + q;
            const int64_t eta = wr->eta;  // 0 unless the query is in AMC
            if (eta > 0) mine += (unsigned long long)(((1ll << nb) - 1) * eta * 2 * (int64_t)wr->lf);
        }
        mine = warp_sum(mine);
        if ((threadIdx.x & 31) == 0) atomicAdd(&s_steps, mine);
        __syncthreads();
        group = s_steps <= (unsigned long long)kAmcGroupSteps ? nb : 1;
        if (blockIdx.x == 0 && threadIdx.x == 0) *a.group = group;
    } else {
        group = *a.group;
    }
    if (a.batch > 1 && a.batch <= group) return;
    const int nbatch = a.batch == 1 ? group : 1;
    // chunk prefix over the queries: built here from the per-query counts
    // (small batches), else laid out by the schedule
    const bool staged = a.nq + 1 <= kSmemChunkBegin;
    if (staged) {
        const int64_t maxc = max_chunks(nbatch);
        int64_t carry = 0;
        for (int64_t tile = 0; tile < a.nq; tile += kCta) {
            const int64_t q = tile + threadIdx.x;
            int64_t cnt = 0;
            if (q < a.nq) {
                if (fused) {
                    const int64_t eta = a.wq[q].eta;
                    for (int i = 0; eta > 0 && i < nbatch; ++i) {
                        int64_t ppc, n;
                        chunk_layout(eta << i, maxc, &ppc, &n);
                        cnt += n;
                    }
                    // every query's count, zeros included: the statistics launches
                    // update only the queries still in AMC, and later walk launches
                    // build their prefix from these counts
                    if (blockIdx.x == 0) a.chunk_count[q] = (int32_t)cnt;
                } else {
                    cnt = a.chunk_count[q];
                }
            }
            int64_t tot;
            const int64_t ex = cta_excl_scan(cnt, scan, &tot);
            if (q < a.nq) cbeg[q] = (int32_t)(carry + ex);
            carry += tot;
        }
        if (threadIdx.x == 0) cbeg[a.nq] = (int32_t)carry;
        __syncthreads();
        if (blockIdx.x == 0)  // for the statistics launch that follows
            for (int i = threadIdx.x; i <= a.nq; i += blockDim.x) a.chunk_begin[i] = cbeg[i];
    }
    const int64_t* cb_glob = a.chunk_begin;
    auto cb_arr = [&](int i) -> int64_t { return staged ? (int64_t)cbeg[i] : cb_glob[i]; };
    const int lane = threadIdx.x & 31;
    const int64_t total = cb_arr(a.nq);
    if (total > a.partial_cap) {  // cannot happen with a valid layout; never write past the partials
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicCAS(a.err_flag, 0, DERR_CHUNKS);
        return;
    }
    for (;;) {
        // chunks are handed out in order by a ticket counter, kChunksPerTicket at a time
        unsigned long long ticket = 0;
        if (lane == 0) ticket = atomicAdd(a.walk_ctr, (unsigned long long)kChunksPerTicket);
        const int64_t c0 = (int64_t)__shfl_sync(0xffffffffu, ticket, 0);
        if (c0 >= total) break;
      for (int64_t c = c0; c < c0 + kChunksPerTicket && c < total; ++c) {
        // owning query: the last q with chunk_begin[q] <= c, by a 32-way warp
        // search (two rounds for up to 1,024 queries): the answer lies in
        // [lo, lo + span); each round the lanes test 32 evenly spaced entries
        // (non-decreasing, so the passing lanes are a prefix) and keep the
        // interval after the last passing one
        int lo = 0, span = (int)a.nq;
        while (span > 1) {
            const int step = (span + 31) >> 5;
            const int pos = lo + (lane + 1) * step;
            const bool ok = pos < lo + span && cb_arr(pos) <= c;
            const int pass = __popc(__ballot_sync(0xffffffffu, ok));
            const int nlo = lo + pass * step;
            span = min(step, lo + span - nlo);
            lo = nlo;
        }
        const int owner = lo;
        const WalkQ* WQ = a.wq + owner;
        double sz, sz2;
        uint64_t cs;
        walk_chunk<W, REC, K>(a, WQ, c - cb_arr(owner), WQ->eta, a.batch, nbatch, lane, &sz, &sz2, &cs);
        if (lane == 0) {
            Partial p;
            p.sz = sz;
            p.sz2 = sz2;
            p.cs = cs;
            a.partial[c] = p;
        }
      }
    }
}

// Queries per CTA of the statistics kernel, one per warp for the partial
// sums (their loads are a latency chain per query); the per-query scalar FP64
// work (Eq. (7): divisions, a logarithm, a square root) then runs one query
// per lane of warp 0, since a single-lane FP64 instruction holds the SM's
// narrow FP64 pipe as long as a full warp's.
constexpr int kReduceQ = kWarps;

// Launch-per-batch statistics (Algorithm 1: Z, the empirical variance, f of
// Eq. (7) at delta/tau) and the stop / doubling decision of each query in
// AMC, for the launch's batches in order until the query stops (the walks of
// later batches of the launch are then not used). A CTA takes kReduceQ
// queries: its warps add the queries' chunk partials, then warp 0 decides,
// one query per lane. For small batches it also writes the next launch's
// chunk counts; for large ones the last CTA to finish lays out the next
// launch (one batch).
__global__ void __launch_bounds__(kCta) amc_reduce_kernel(AmcArgs a) {
    __shared__ double s_sz[kAmcGroup][kReduceQ], s_sz2[kAmcGroup][kReduceQ];
    __shared__ unsigned long long s_cs[kAmcGroup][kReduceQ];
    __shared__ bool last;
    const int group = *a.group;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t q0 = (int64_t)blockIdx.x * kReduceQ;
    // the last launch writes every query's outputs (warp 0, one query per lane)
    const bool outputs = a.out_r != nullptr && a.batch == a.tau;
    if (a.batch > 1 && a.batch <= group) {  // walked and evaluated with batch 1
        if (outputs && warp == 0 && lane < kReduceQ && q0 + lane < a.nq)
            store_outputs(a.st[q0 + lane], q0 + lane, a.out_r, a.out_stats);
        return;
    }
    const int nbatch = a.batch == 1 ? group : 1;
    const int64_t maxc = max_chunks(nbatch);
    const bool staged = a.nq + 1 <= kSmemChunkBegin;
    // the batches' sums, one query per warp at a time; the first partial of
    // every lane and batch is loaded before any is added (one round trip for
    // the usual batch of at most 32 chunks), the rest lane-strided, then a
    // warp reduction per batch
    for (int j = warp; j < kReduceQ; j += kWarps) {
        const int64_t q = q0 + j;
        if (q >= a.nq || a.st[q].status != ST_AMC) continue;
        int64_t begin[kAmcGroup], nch[kAmcGroup];
        {
            int64_t b = a.chunk_begin[q], eta = a.st[q].eta;
#pragma unroll
            for (int bi = 0; bi < kAmcGroup; ++bi) {
                int64_t ppc = 0, n = 0;
                if (bi < nbatch) chunk_layout(eta, maxc, &ppc, &n);
                begin[bi] = b;
                nch[bi] = n;
                b += n;
                eta *= 2;
            }
        }
        Partial first[kAmcGroup];
#pragma unroll
        for (int bi = 0; bi < kAmcGroup; ++bi) {
            first[bi].sz = first[bi].sz2 = 0.0;
            first[bi].cs = 0ull;
            if (lane < nch[bi]) first[bi] = a.partial[begin[bi] + lane];
        }
#pragma unroll
        for (int bi = 0; bi < kAmcGroup; ++bi) {
            if (bi >= nbatch) break;
            double x = first[bi].sz, x2 = first[bi].sz2;
            uint64_t c = first[bi].cs;
            for (int64_t i = lane + 32; i < nch[bi]; i += 32) {
                const Partial p = a.partial[begin[bi] + i];
                x += p.sz;
                x2 += p.sz2;
                c += p.cs;
            }
            x = warp_sum(x);
            x2 = warp_sum(x2);
            c = warp_sum(c);
            if (lane == 0) {
                s_sz[bi][j] = x;
                s_sz2[bi][j] = x2;
                s_cs[bi][j] = c;
            }
        }
    }
    __syncthreads();
    if (warp == 0 && lane < kReduceQ) {
        const int64_t q = q0 + lane;
        QState* Q = a.st + q;
        if (q < a.nq && Q->status == ST_AMC) {
            const double Lg = a.log_3tau_delta;  // log(3 / (delta / tau)), Eq. (7) at delta / tau
            const double psi = Q->psi, qeps = Q->eps, r_b = Q->r_b;
            const int32_t lf = Q->lf;
            int64_t eta = Q->eta, walks = Q->walks, steps = Q->walk_steps;
            uint64_t chk = Q->checksum;
            bool stop = false;
            for (int bi = 0; bi < nbatch && !stop; ++bi) {
                const int batch = a.batch + bi;
                const double inv = 1.0 / (double)eta;
                const double Z = s_sz[bi][lane] * inv;
                double var = s_sz2[bi][lane] * inv - Z * Z;
                if (var < 0.0) var = 0.0;
                const double f = sqrt(2.0 * var * Lg * inv) + 3.0 * psi * Lg * inv;
                walks += eta;
                steps += 2 * eta * (int64_t)lf;
                chk += s_cs[bi][lane];
                Q->batch = batch;
                Q->f_last = f;
                if (f <= qeps / 2.0 || batch >= a.tau) {
                    Q->r_f = Z;
                    Q->r = r_b + Z;
                    Q->status = ST_DONE;
                    stop = true;
                } else {
                    eta *= 2;
                }
            }
            Q->walks = walks;
            Q->walk_steps = steps;
            Q->checksum = chk;
            Q->eta = eta;  // the next batch's pairs, or the last batch's on a stop
            if (staged && a.batch + nbatch <= a.tau) {
                // the next launch's chunks of the query (one batch)
                int32_t nch = 0;
                if (!stop) {
                    int64_t ppc, n;
                    chunk_layout(eta, kMaxChunksPerQuery, &ppc, &n);
                    nch = (int32_t)n;
                    a.wq[q].eta = eta;
                }
                a.chunk_count[q] = nch;
            }
        }
        if (outputs && q < a.nq) store_outputs(*Q, q, a.out_r, a.out_stats);
    }
    const int next = a.batch + nbatch;
    if (staged) {
        // each walk CTA builds the prefix; only the ticket counter is reset here,
        // after the last batch too: the next AMC phase on the same workspace (the
        // next query of a one-query-at-a-time batch) starts from ticket 0
        if (blockIdx.x == 0 && threadIdx.x == 0) *a.walk_ctr = 0ull;
        return;
    }
    if (next > a.tau) return;  // no next batch to lay out
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(a.done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    schedule_cta(a, 1);
    if (threadIdx.x == 0) *a.done = 0u;
}

void launch_amc_schedule(const AmcArgs& a, cudaStream_t st) {
    prof_begin(FAM_AMC_SCHEDULE, st);
    amc_schedule_kernel<<<1, kCta, 0, st>>>(a);
    prof_end(FAM_AMC_SCHEDULE, st);
}

__global__ void edge_records_kernel(const int32_t* col_idx, const uint2* node_info, int64_t nnz, uint4* out) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = col_idx[e];
        const uint2 inf = node_info[v];
        out[e] = make_uint4((uint32_t)v, inf.x, inf.y, 0u);
    }
}

// unit u of the packed neighbour lists: entries u*k .. u*k + k - 1 of col_idx,
// entry j at bits [j * B, j * B + B) of the 128-bit unit (B = pack_bits(k))
__global__ void pack_cols_kernel(const int32_t* col_idx, int64_t nnz, int k, uint4* out) {
    const int B = pack_bits(k);
    const int64_t units = (nnz + k - 1) / k;
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < units; u += (int64_t)gridDim.x * blockDim.x) {
        uint32_t w[5] = {0u, 0u, 0u, 0u, 0u};
        for (int j = 0; j < k; ++j) {
            const int64_t e = u * k + j;
            if (e >= nnz) break;
            const uint32_t v = (uint32_t)col_idx[e];
            const int o = j * B, wi = o >> 5, sh = o & 31;
            w[wi] |= v << sh;
            if (sh + B > 32) w[wi + 1] |= v >> (32 - sh);
        }
        out[u] = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

void launch_pack_cols(const int32_t* col_idx, int64_t nnz, int k, uint4* out, cudaStream_t st) {
    const int64_t units = (nnz + k - 1) / k;
    if (units <= 0) return;
    pack_cols_kernel<<<(int)std::min<int64_t>((units + 255) / 256, 152 * 32), 256, 0, st>>>(col_idx, nnz, k, out);
    note_launches(1);
}

void launch_edge_records(const int32_t* col_idx, const uint2* node_info, int64_t nnz, uint4* out, cudaStream_t st) {
    if (nnz <= 0) return;
    edge_records_kernel<<<(int)std::min<int64_t>((nnz + 255) / 256, 152 * 32), 256, 0, st>>>(col_idx, node_info, nnz,
                                                                                           out);
    note_launches(1);
}

// One walk kernel per neighbour-list layout: edge records, or col_idx
// packed k to a 16-byte unit (k = 8, 6, 5), or plain col_idx.
template <bool REC, int K>
static void launch_walk_variant(const AmcArgs& a, int sm_count, cudaStream_t st) {
    // the chunk prefix: nq + 1 int32 for batches up to kSmemChunkBegin - 1 queries
    const size_t smem = a.nq + 1 <= kSmemChunkBegin ? (size_t)(a.nq + 1) * sizeof(int32_t) : 0;
    static int per_sm = 0;  // resident CTAs per SM (register bound; the prefix is at most 16 KB)
    if (per_sm == 0) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, amc_walk_kernel<kWalksPerLane, REC, K>, 256,
                                                          kSmemChunkBegin * sizeof(int32_t)) != cudaSuccess ||
            b < 1) {
            cudaGetLastError();
            b = 1;
        }
        per_sm = b;
    }
    amc_walk_kernel<kWalksPerLane, REC, K><<<sm_count * per_sm, 256, smem, st>>>(a);
}

void launch_amc_walk(const AmcArgs& a, int sm_count, cudaStream_t st) {
    prof_begin(FAM_AMC_WALK, st);
    if (a.g.edge_rec) launch_walk_variant<true, 0>(a, sm_count, st);
    else if (a.g.cols_packed && a.g.pack_k == 8) launch_walk_variant<false, 8>(a, sm_count, st);
    else if (a.g.cols_packed && a.g.pack_k == 6) launch_walk_variant<false, 6>(a, sm_count, st);
    else if (a.g.cols_packed && a.g.pack_k == 5) launch_walk_variant<false, 5>(a, sm_count, st);
    else launch_walk_variant<false, 0>(a, sm_count, st);
    prof_end(FAM_AMC_WALK, st);
}

void launch_amc_reduce(const AmcArgs& a, cudaStream_t st) {
    const int grid = (int)((a.nq + kReduceQ - 1) / kReduceQ);
    prof_begin(FAM_AMC_REDUCE, st);
    amc_reduce_kernel<<<grid, kCta, 0, st>>>(a);
    prof_end(FAM_AMC_REDUCE, st);
}

}  // namespace geer
