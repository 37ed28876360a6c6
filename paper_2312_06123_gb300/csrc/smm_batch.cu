// smm_batch.cu -- SMM phase of GEER (Algorithm 3 with the iteration of
// Algorithm 2), level-synchronous over a whole batch of queries.
//
// A query keeps s* and t* (Eq. 15: s*(v) = p_i(v,s), t*(v) = p_i(v,t)) in a
// frontier table: an open-addressing hash table, in a pool shared by the
// batch, whose occupied slots are the nodes of V_s u V_t with both values
// and two support bits. One SMM iteration builds the query's next table by
// push: every node u of the current table sends x(u) to each v in N(u) --
// exactly the cost sum_{u in V} d(u) that Eq. (17) charges -- and then
// y(v) = (sum received) / d(v), the support bits OR-ed (V' = N(V),
// structurally). Contributions are added as 64-bit fixed-point integers
// with atomics at scale 2^S_s for s* (S_s = 61 - ceil(log2(d(s)+1))) and
// 2^S_t for t*: integer addition is associative, so the sums do not depend
// on thread scheduling, and the scale has headroom since
// sum_{u in N(v)} p_i(u,s) = d(s) p_{i+1}(s,v) <= d(s) (reversibility). A
// contribution carries at most 2^-(S+1) absolute rounding.
//
// Every kernel covers every query of the batch; one iteration is
//   alloc  (1 CTA)  : tables for the queries that continue, from the pool;
//   clear           : empty those tables;
//   seed | push     : F_0 = {s, t} with s* = e_s, t* = e_t | the push above;
//   finish          : y values, g(v) = s*(v)/d(s) - t*(v)/d(t), and the
//                     per-query sums of Eq. (17)'s volume, |V|, max_1;
//   top2            : max_2 (second element of the descending multiset);
//   decide          : the four series terms of Algorithm 2 added to r_b in
//                     FP64, psi (Eq. 9), eta* (Eq. 8), h(l - l_b) and the
//                     switch (Eq. 17, or a fixed policy).
// The last table of a query is its walk lookup table (Algorithm 1).
#include "geer_internal.cuh"
#include "geer_kernels.h"

namespace geer {

namespace {

// x * 2^S rounded to nearest (ties to even), for 0 <= x, from the bits of x
// (integer operations only).
__device__ __forceinline__ unsigned long long to_fixed(float x, int S) {
    const uint32_t b = __float_as_uint(x);
    const int e = (int)((b >> 23) & 0xff);
    uint64_t mant = b & 0x7fffffu;
    int ex;
    if (e == 0) {
        ex = -149;
    } else {
        mant |= 0x800000u;
        ex = e - 150;
    }
    const int sh = ex + S;
    if (sh >= 0) return mant << sh;
    const int r = -sh;
    if (r >= 64) return 0ull;
    const uint64_t q = mant >> r;
    const uint64_t rem = mant & ((1ull << r) - 1);
    const uint64_t half = 1ull << (r - 1);
    return q + ((rem > half || (rem == half && (q & 1))) ? 1 : 0);
}

__device__ __forceinline__ unsigned long long to_fixed(double x, int S) {
    const uint64_t b = (uint64_t)__double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7ff);
    uint64_t mant = b & 0xfffffffffffffull;
    int ex;
    if (e == 0) {
        ex = -1074;
    } else {
        mant |= 1ull << 52;
        ex = e - 1075;
    }
    const int sh = ex + S;
    if (sh >= 0) return sh >= 11 ? ~0ull : (mant << sh);  // x <= 1 never reaches sh >= 11
    const int r = -sh;
    if (r >= 64) return 0ull;
    const uint64_t q = mant >> r;
    const uint64_t rem = mant & ((1ull << r) - 1);
    const uint64_t half = 1ull << (r - 1);
    return q + ((rem > half || (rem == half && (q & 1))) ? 1 : 0);
}

// y = sum * 2^-S / d in T. FP32: the 64-bit integer is rounded to float
// through its two 32-bit halves (FP32 pipe only); FP64: one conversion.
template <typename T>
__device__ __forceinline__ T from_fixed(unsigned long long sum, int S, int64_t d);

template <>
__device__ __forceinline__ float from_fixed<float>(unsigned long long sum, int S, int64_t d) {
    const float hi = __uint2float_rn((uint32_t)(sum >> 32));
    const float lo = __uint2float_rn((uint32_t)sum);
    const float x = __fmaf_rn(hi, 4294967296.0f, lo);
    return ldexpf(x, -S) / (float)d;
}

template <>
__device__ __forceinline__ double from_fixed<double>(unsigned long long sum, int S, int64_t d) {
    return ldexp((double)sum, -S) / (double)d;
}

__device__ __forceinline__ int fixed_shift(int64_t d) {
    int b = 0;
    for (uint64_t x = (uint64_t)d; x > 0; x >>= 1) ++b;  // ceil(log2(d + 1))
    return 61 - b;
}

constexpr uint32_t kNoSlot = 0xffffffffu;

// insert v into a table (capacity mask+1); returns its slot, or kNoSlot
// (and raises DERR_FULL) when a full cycle of probes finds neither v nor a
// free slot -- impossible while the table's load stays at most 1/2
__device__ __forceinline__ uint32_t table_insert(GEntry* tab, uint32_t mask, int32_t v, int* err_flag) {
    uint32_t h = hash32((uint32_t)v) & mask;
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        const int32_t prev = atomicCAS(&tab[h].v, -1, v);
        if (prev == -1 || prev == v) return h;
        h = (h + 1) & mask;
    }
    atomicCAS(err_flag, 0, DERR_FULL);
    return kNoSlot;
}

}  // namespace

// ---------------------------------------------------------------------------
// set-up: validation and l (Eq. 6 or Eq. 5) of one query
// ---------------------------------------------------------------------------
// Resets the query's state; returns true when the query enters the SMM loop
// (s != t, valid input, l defined).
__device__ __forceinline__ bool setup_query(const SmmArgs& a, int64_t q) {
    const int64_t* row_ptr = a.g.row_ptr;
    QState* Q = a.st + q;
    QSmm* M = a.sm + q;
    const int32_t s = a.s[q], t = a.t[q];
    const double eps = a.eps ? a.eps[q] : a.eps_scalar;
    Q->s = s; Q->t = t; Q->eps = eps; Q->qidx = a.q_index_base + (int32_t)q;
    Q->batch = 0; Q->err = 0; Q->r_b = 0; Q->r_f = 0; Q->r = 0; Q->psi = 0;
    Q->volume = 0; Q->h = 0; Q->f_last = 0; Q->eta0 = 0; Q->eta = 0; Q->walks = 0;
    Q->walk_steps = 0; Q->checksum = 0; Q->ppc = 0; Q->nchunks = 0; Q->table_off = 0;
    Q->table_mask = -1; Q->front = 0; Q->ell = 0; Q->ell_b = 0; Q->lf = 0; Q->ds = 0; Q->dt = 0;
    M->run = 0; M->want = 0;
    M->tab_off = M->tab_cap = M->ntab_off = M->ntab_cap = 0;
    M->dense = a.dense_engine ? 1 : 0;
    M->dgo = 0;
    M->dblock = a.dense_engine ? (int32_t)(q / (a.dense_width / 2)) : -1;
    M->dcol = a.dense_engine ? (int32_t)(q % (a.dense_width / 2)) : -1;
    Q->dense_vals = nullptr;
    Q->dense_stride = 0;
    M->vol_paper = M->vol_union = M->count = 0;
    M->max1s = M->max1t = M->max2s = M->max2t = M->cnt1s = M->cnt1t = 0;
    M->sval[0] = M->sval[1] = M->sval[2] = M->sval[3] = 0.0;
    a.wq[q].eta = 0;  // no walks unless the query enters AMC
    if (s < 0 || s >= a.g.n || t < 0 || t >= a.g.n || !(eps > 0.0)) {
        Q->status = ST_ERROR;
        Q->err = DERR_NODE_RANGE;
        atomicCAS(a.err_flag, 0, DERR_NODE_RANGE);
        return false;
    }
    if (s == t) {  // r(s,s) = 0 (Definition 1)
        Q->status = ST_DONE;
        return false;
    }
    const int64_t dsi = row_ptr[s + 1] - row_ptr[s], dti = row_ptr[t + 1] - row_ptr[t];
    const double ds = (double)dsi, dt = (double)dti;
    int64_t ell;
    const double lam = a.lambda;
    if (!(lam < 1.0)) {
        ell = -1;
    } else if (lam <= 0.0) {
        ell = 0;
    } else {
        // (log(1 / lambda) is the same for every query: computed on the host)
        const double v = a.ell_formula == 1
                             ? ceil(log(4.0 / (eps - eps * lam)) / a.log_inv_lambda - 1.0)
                             : ceil(log((2.0 / ds + 2.0 / dt) / (eps * (1.0 - lam))) / a.log_inv_lambda - 1.0);
        ell = v < 0.0 ? 0 : (int64_t)v;
    }
    if (ell < 0) {
        Q->status = ST_ERROR;
        Q->err = DERR_ELL;
        atomicCAS(a.err_flag, 0, DERR_ELL);
        return false;
    }
    Q->status = ST_SMM;
    Q->ds = (int32_t)dsi;
    Q->dt = (int32_t)dti;
    Q->ell = (int32_t)ell;
    M->shift_s = fixed_shift(dsi);
    M->shift_t = fixed_shift(dti);
    M->inv_ds = 1.0 / ds;
    M->inv_dt = 1.0 / dt;
    M->lb_target = a.policy == 2 ? (a.fixed_lb < 0 ? (int32_t)ell : min(a.fixed_lb, (int32_t)ell)) : -1;
    if (a.lb_force && a.lb_force[q] >= 0) M->lb_target = min(a.lb_force[q], (int32_t)ell);
    return true;
}

// Set-up alone (dense engine: F_0 = {s, t} is written into the query's
// block column by the dense engine, and its first decision follows).
__global__ void smm_setup_kernel(SmmArgs a) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.ctl->iter = 0;
        a.ctl->lo[0] = a.ctl->hi[0] = 0;
    }
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < a.nq; q += (int64_t)gridDim.x * blockDim.x) {
        if (setup_query(a, q) && a.sm[q].dense) {
            a.sm[q].dgo = 1;
            a.sm[q].run = 1;
        }
    }
}

// A query leaves SMM after iteration lb (Algorithm 3's switch): its state of
// Eq. (17) (psi, volume, h, eta_0) is kept for the statistics, and it enters
// AMC with the lookup table of its last frontier (or its dense column), or,
// with no walk left (l_f = 0), finishes with r = r_b.
__device__ __forceinline__ void leave_smm(const SmmArgs& a, int64_t q, QState* Q, QSmm* M, int iter, int64_t lb,
                                          int64_t lf, double psi, double vol, double h, int64_t eta0,
                                          int64_t count) {
    M->run = 0;
    M->dgo = 0;
    Q->ell_b = (int32_t)lb;
    Q->lf = (int32_t)lf;
    Q->psi = psi;
    Q->volume = vol;
    Q->h = h;
    Q->eta0 = eta0;
    Q->eta = eta0;
    Q->front = (int32_t)count;
    if (M->dense) {
        // the values of the last iteration sit in dense buffer (iter & 1)
        const size_t esz = a.dense_fp64 ? sizeof(double) : sizeof(float);
        const char* base = reinterpret_cast<const char*>(a.dense_X[iter & 1]);
        Q->dense_vals = base + ((size_t)M->dblock * (size_t)a.g.n * (size_t)a.dense_width + 2 * (size_t)M->dcol) * esz;
        Q->dense_stride = a.dense_width;
        Q->table_off = 0;
        Q->table_mask = -1;
    } else {
        Q->table_off = M->tab_off;
        Q->table_mask = (int32_t)(M->tab_cap - 1);
    }
    if (lf > 0) {
        Q->status = ST_AMC;
        // the query's walk record
        WalkQ* wr = a.wq + q;
        wr->s = Q->s;
        wr->t = Q->t;
        if (a.g.node_info) {
            wr->s_info = a.g.node_info[Q->s];
            wr->t_info = a.g.node_info[Q->t];
        } else {
            const int64_t rs = a.g.row_ptr[Q->s], rt = a.g.row_ptr[Q->t];
            wr->s_info = make_uint2((uint32_t)rs, (uint32_t)Q->ds);
            wr->t_info = make_uint2((uint32_t)rt, (uint32_t)Q->dt);
        }
        wr->lf = (int32_t)lf;
        wr->qidx = Q->qidx;
        wr->eta = eta0;
        wr->table_off = Q->table_off;
        wr->mask = Q->table_mask;
        wr->dstride = Q->dense_stride;
        wr->dvals = Q->dense_vals;
        wr->inv_ds = M->inv_ds;
        wr->inv_dt = M->inv_dt;
        wr->filt = (!M->dense && M->tab_cap <= kFilterSlots) ? M->filt[lb & 1] : nullptr;
    } else {
        Q->status = ST_DONE;
        Q->r = Q->r_b;
    }
}

// A query continues into the next iteration: on the hybrid engine a free
// dense column when its next push has >= migrate_at pairs, else a frontier
// table for at most min(push pairs, n) nodes at load <= 1/2, bump-allocated
// from the pool. Returns false (query failed) when the table is beyond the
// option's limit or the pool.
#ifndef GEER_TABLE_SPREAD
#define GEER_TABLE_SPREAD 4
#endif
constexpr int64_t kTableSpread = GEER_TABLE_SPREAD;  // slots per possible entry of a small table
constexpr int64_t kSpreadMost = 1024;                // tables of at most this many entries are spread

__device__ __forceinline__ bool continue_smm(const SmmArgs& a, int64_t q, QState* Q, QSmm* M, int64_t lb,
                                             unsigned long long push_pairs) {
    if (M->dense) {
        M->dgo = 1;
        M->run = 1;
        atomicAdd(&a.ctl->n_want, 1);
        return true;
    }
    if (a.hybrid && (int64_t)push_pairs >= a.migrate_at) {
        int col = atomicAdd(&a.ctl->dense_next, 1);
        if (col < a.dense_cap) {
            const int qpb = a.dense_width / 2;
            M->dense = 1;
            M->dgo = 1;
            M->run = 1;
            M->dblock = col / qpb;
            M->dcol = col % qpb;
            a.dense_block_q[col] = (int32_t)q;
            a.mig_list[atomicAdd(&a.ctl->n_mig, 1)] = (int32_t)q;
            atomicAdd(&a.ctl->n_want, 1);
            return true;
        }
    }
    int64_t cap = 16;
    const int64_t most = min((int64_t)push_pairs, (int64_t)a.g.n);
    // small tables are spread to a lower load: the walks look up mostly
    // absent nodes, and an unsuccessful linear-probing search takes about
    // (1 + 1/(1 - load)^2) / 2 probes (a warp waits for its longest one)
    const int64_t spread = most <= kSpreadMost ? kTableSpread : 2;
    while (cap < spread * most) cap <<= 1;
    if (cap > a.max_table && spread > 2) {
        cap = 16;
        while (cap < 2 * most) cap <<= 1;
    }
    if (cap > a.max_table) {
        Q->status = ST_ERROR;
        Q->err = DERR_CAPACITY;
        Q->ell_b = (int32_t)lb;
        M->run = 0;
        atomicCAS(a.err_flag, 0, DERR_CAPACITY);
        return false;
    }
    const int64_t off = (int64_t)kF0Slots * a.nq + (int64_t)atomicAdd(&a.ctl->cursor, (unsigned long long)cap);
    if (off + cap > a.pool_cap) {  // the pool is too small for this batch: the host grows it and reruns
        Q->status = ST_ERROR;
        Q->err = DERR_TABLE;
        M->run = 0;
        atomicCAS(a.err_flag, 0, DERR_TABLE);
        return false;
    }
    M->ntab_off = off;
    M->ntab_cap = cap;
    M->run = 1;
    // the next table's filter starts empty (its finish sets the bits)
    uint4* fz = reinterpret_cast<uint4*>(M->filt[(lb + 1) & 1]);
#pragma unroll
    for (int k = 0; k < kFilterWords / 4; ++k) fz[k] = make_uint4(0u, 0u, 0u, 0u);
    atomicAdd(&a.ctl->n_want, 1);
    return true;
}

// Iteration 0 of the sparse and hybrid engines, in closed form (Algorithm 3
// before its first SMM step), one thread per query: set-up; the query's
// F_0 table at slots [8q, 8q + 8): F_0 = {s, t}, s* = e_s, t* = e_t, g(s) =
// 1/d(s), g(t) = -1/d(t) (the push source of iteration 1, and the walks'
// lookup table when no SMM step runs); Algorithm 2's four terms at i = 0,
// r_b = 1/d(s) + 1/d(t); the first decision (the loop runs once when
// l >= 1, or as a fixed policy says); and the table of F_1 (whose push has
// d(s) + d(t) pairs). Eq. (17)'s volume is d(s) + d(t) and max_1 = 1,
// max_2 = 0 for both vectors (one non-zero entry each).
// What the start kernel knows of a query before its first decision.
struct StartState {
    bool smm = false;  // the query enters the SMM loop
    bool go = false;   // its first decision: one SMM iteration (else AMC alone)
    bool ask = false;  // the learned switch takes that decision
    double psi = 0.0, h = 0.0;
    int64_t eta0 = 0, ell = 0;
    unsigned long long vol = 0;
    float f[kMlpIn];   // the learned switch's inputs at l_b = 0 (when ask)
};

template <typename T>
__device__ __forceinline__ StartState start_query(const SmmArgs& a, int64_t q, bool learned) {
    StartState S;
    S.smm = setup_query(a, q);
    // every F_0 table is written, so the push of iteration 1 reads no stale slot
    const int64_t off = (int64_t)kF0Slots * q;
    GEntry* tab = a.ent + off;
    GEntry empty;
    empty.v = -1;
    empty.bits = 0u;
    empty.g = 0.0;
#pragma unroll
    for (int k = 0; k < kF0Slots; ++k) tab[k] = empty;
    if (!S.smm) return S;
    T* ys = reinterpret_cast<T*>(a.ys);
    T* yt = reinterpret_cast<T*>(a.yt);
    QState* Q = a.st + q;
    QSmm* M = a.sm + q;
    const double ds = (double)Q->ds, dt = (double)Q->dt;
    // linear probing in an 8-slot table, as table_insert would place them
    const uint32_t hs = hash32((uint32_t)Q->s) & (kF0Slots - 1);
    uint32_t ht = hash32((uint32_t)Q->t) & (kF0Slots - 1);
    if (ht == hs) ht = (ht + 1) & (kF0Slots - 1);
    GEntry es, et;
    es.v = Q->s;
    es.bits = 1u | ((uint32_t)q << 2);
    es.g = 1.0 * M->inv_ds - 0.0 * M->inv_dt;
    et.v = Q->t;
    et.bits = 2u | ((uint32_t)q << 2);
    et.g = 0.0 * M->inv_ds - 1.0 * M->inv_dt;
    tab[hs] = es;
    tab[ht] = et;
    ys[off + hs] = T(1);
    yt[off + hs] = T(0);
    ys[off + ht] = T(0);
    yt[off + ht] = T(1);
    M->tab_off = off;
    M->tab_cap = kF0Slots;
    // F_0's filter: s and t
    uint4* fz = reinterpret_cast<uint4*>(M->filt[0]);
#pragma unroll
    for (int k = 0; k < kFilterWords / 4; ++k) fz[k] = make_uint4(0u, 0u, 0u, 0u);
    const uint32_t bs = filter_bit(hash32((uint32_t)Q->s)), bt = filter_bit(hash32((uint32_t)Q->t));
    M->filt[0][bs >> 5] |= 1u << (bs & 31u);
    M->filt[0][bt >> 5] |= 1u << (bt & 31u);
    // Algorithm 2 at i = 0: s*(s)/d(s) + t*(t)/d(t) - s*(t)/d(s) - t*(s)/d(t)
    // (1/d(s), 1/d(t) by the set-up's divisions; the zero terms subtract +0)
    Q->r_b = M->inv_ds + M->inv_dt;
    S.ell = Q->ell;
    S.vol = (unsigned long long)Q->ds + (unsigned long long)Q->dt;
    // Eq. (9) and h(l) at l_b = 0: max_1 = 1 and max_2 = 0 for both vectors
    if (S.ell > 0)
        switch_quantities(S.ell, 1.0, 0.0, 1.0, 0.0, ds, dt, Q->eps, a.log_2tau_delta, a.tau, &S.psi, &S.eta0,
                          &S.h);
    S.go = M->lb_target >= 0 ? (M->lb_target > 0) : (S.ell >= 1);  // the loop runs once when l >= 1
    if (S.go && M->lb_target < 0 && learned) {
        // the learned switch may stop before any SMM step (AMC alone, Algorithm 1):
        // its inputs at l_b = 0 (those switch_features gives after an iteration)
        S.ask = true;
        switch_features(Q->ds, Q->dt, S.ell, S.vol, S.h, 1.0, 1.0, S.f);
    }
    return S;
}

template <typename T>
__global__ void smm_start_kernel(SmmArgs a) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.ctl->iter = 0;
        a.ctl->lo[0] = 0;
        a.ctl->hi[0] = (int64_t)kF0Slots * a.nq;
    }
    const bool learned = a.policy == 1 && a.mlp_w != nullptr && a.mlp_at_start;
    // a loop of the same trip count for every thread: the network is evaluated by the whole warp
    static_assert(kQueryCta == 32, "one warp per CTA");
    for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < a.nq; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = base + threadIdx.x;
        StartState S;
        if (q < a.nq) S = start_query<T>(a, q, learned);
        if (learned) {
            const float y = mlp_eval_asked(a.mlp_wt, a.mlp_norm, S.f, S.ask);
            if (S.ask) S.go = y < 0.f;
        }
        if (!S.smm) continue;
        QState* Q = a.st + q;
        QSmm* M = a.sm + q;
        if (S.go) continue_smm(a, q, Q, M, 0, S.vol);
        else leave_smm(a, q, Q, M, 0, 0, S.ell, S.psi, (double)S.vol, S.h, S.eta0, 2);
    }
}

// The FP32 copy of the switch network's weights (one CTA).
__global__ void mlp_expand_kernel(const unsigned short* w, float* out) { mlp_stage(out, w); }

void launch_mlp_expand(const unsigned short* w, float* out, cudaStream_t st) {
    mlp_expand_kernel<<<1, 256, 0, st>>>(w, out);
    note_launches(1);
}

constexpr int64_t kLightMax = 128;  // neighbours a single warp pushes
constexpr int64_t kHeavyChunk = 512;

// push the values of table slot j (node u of query q) to neighbours
// [pb, pe) of u; called by `nthreads` cooperating threads with rank `rank`
template <typename T>
__device__ __forceinline__ void push_range(const SmmArgs& a, int64_t j, int q, int64_t pb, int64_t pe, int rank,
                                           int nthreads) {
    const T* ys = reinterpret_cast<const T*>(a.ys);
    const T* yt = reinterpret_cast<const T*>(a.yt);
    const QSmm* M = a.sm + q;
    GEntry* ntab = a.ent + M->ntab_off;
    const uint32_t nmask = (uint32_t)(M->ntab_cap - 1);
    const T xs = ys[j], xt = yt[j];
    const unsigned long long fs = xs != T(0) ? to_fixed(xs, M->shift_s) : 0ull;
    const unsigned long long ft = xt != T(0) ? to_fixed(xt, M->shift_t) : 0ull;
    const uint32_t bits = a.ent[j].bits;  // support bits and the owner, unchanged
    unsigned long long* ss = a.sum_s + M->ntab_off;
    unsigned long long* tt = a.sum_t + M->ntab_off;
    const int32_t* col_idx = a.g.col_idx;
    for (int64_t p = pb + rank; p < pe; p += nthreads) {
        const int32_t v = col_idx[p];
        const uint32_t h = table_insert(ntab, nmask, v, a.err_flag);
        if (h == kNoSlot) continue;
        if (fs) atomicAdd(&ss[h], fs);
        if (ft) atomicAdd(&tt[h], ft);
        atomicOr(&ntab[h].bits, bits);
    }
}

// push: every node of a continuing query's current table sends its values
// to its neighbours in the query's next table. One warp per table slot; a
// node with more than kLightMax neighbours goes to the heavy list instead.
template <typename T>
__global__ void __launch_bounds__(256) smm_push_kernel(SmmArgs a) {
    const int parity_cur = (a.ctl->iter & 1) ^ 1;
    const int lane = threadIdx.x & 31;
    const int64_t lo = a.ctl->lo[parity_cur], hi = a.ctl->hi[parity_cur];
    const int64_t* row_ptr = a.g.row_ptr;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t j = lo + (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5); j < hi; j += nwarps) {
        const GEntry e = a.ent[j];
        if (e.v < 0) continue;
        const int q = (int)(e.bits >> 2);
        if (!a.sm[q].run || a.sm[q].dense) continue;  // dense queries iterate in the SpMM
        const int64_t rb = row_ptr[e.v], re = row_ptr[e.v + 1];
        if (re - rb > kLightMax) {
            // hand the node's neighbour list, in chunks, to the heavy push
            const int nch = (int)((re - rb + kHeavyChunk - 1) / kHeavyChunk);
            int first = 0;
            if (lane == 0) first = atomicAdd(&a.ctl->n_heavy, nch);
            first = __shfl_sync(0xffffffffu, first, 0);
            if ((int64_t)first + nch <= a.heavy_cap) {
                for (int c = lane; c < nch; c += 32) a.heavy[first + c] = (j << 20) | (int64_t)c;
                continue;
            }
            // the list is full: mark the reserved records that fit as empty, push here
            for (int64_t c = (int64_t)first + lane; c < a.heavy_cap && c < (int64_t)first + nch; c += 32)
                a.heavy[c] = -1;
        }
        push_range<T>(a, j, q, rb, re, lane, 32);
    }
}

// heavy push: one CTA per chunk of kHeavyChunk neighbours of a node with
// more than kLightMax neighbours
template <typename T>
__global__ void __launch_bounds__(256) smm_push_heavy_kernel(SmmArgs a) {
    const int64_t nc = min((int64_t)a.ctl->n_heavy, a.heavy_cap);
    const int64_t* row_ptr = a.g.row_ptr;
    for (int64_t c = blockIdx.x; c < nc; c += gridDim.x) {
        const int64_t rec = a.heavy[c];
        if (rec < 0) continue;
        const int64_t j = rec >> 20, part = rec & 0xfffff;
        const GEntry e = a.ent[j];
        const int q = (int)(e.bits >> 2);
        const int64_t rb = row_ptr[e.v], re = row_ptr[e.v + 1];
        const int64_t pb = rb + part * kHeavyChunk;
        push_range<T>(a, j, q, pb, min(pb + kHeavyChunk, re), threadIdx.x, blockDim.x);
    }
}

// finish: y(v) = sum / d(v) in T, g(v), and the per-query sums (vol of
// Eq. 17, the next push volume, |V|, max_1), aggregated per warp
template <typename T>
__global__ void __launch_bounds__(256) smm_finish_kernel(SmmArgs a) {
    const int parity = a.ctl->iter & 1;
    const int64_t lo = a.ctl->lo[parity], hi = a.ctl->hi[parity];
    T* ys = reinterpret_cast<T*>(a.ys);
    T* yt = reinterpret_cast<T*>(a.yt);
    const int64_t* row_ptr = a.g.row_ptr;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // warp-uniform trip count so that every lane reaches the warp reductions
    for (int64_t base = lo + (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < hi; base += stride) {
        const int64_t j = base + (threadIdx.x & 31);
        int q = -1;
        unsigned long long vp = 0, vu = 0, cnt = 0, m1s = 0, m1t = 0;
        if (j < hi) {
            const GEntry e = a.ent[j];
            const int32_t v = e.v;
            if (v >= 0) {
                q = (int)(e.bits >> 2);
                QSmm* M = a.sm + q;
                if (M->run) {
                    const QState* Q = a.st + q;
                    const int64_t dv = row_ptr[v + 1] - row_ptr[v];
                    const T s_v = from_fixed<T>(a.sum_s[j], M->shift_s, dv);
                    const T t_v = from_fixed<T>(a.sum_t[j], M->shift_t, dv);
                    ys[j] = s_v;
                    yt[j] = t_v;
                    a.ent[j].g = (double)s_v * M->inv_ds - (double)t_v * M->inv_dt;
                    const uint32_t bits = e.bits & 3u;
                    if (M->ntab_cap <= kFilterSlots) {  // the table's membership filter
                        const uint32_t fb = filter_bit(hash32((uint32_t)v));
                        atomicOr(&M->filt[parity][fb >> 5], 1u << (fb & 31u));
                    }
                    vp = (unsigned long long)(dv * (int64_t)((bits & 1u) + ((bits >> 1) & 1u)));
                    vu = (unsigned long long)dv;
                    cnt = 1;
                    m1s = (unsigned long long)__double_as_longlong((double)s_v);
                    m1t = (unsigned long long)__double_as_longlong((double)t_v);
                    if (v == Q->s) {
                        M->sval[0] = (double)s_v;
                        M->sval[1] = (double)t_v;
                    }
                    if (v == Q->t) {
                        M->sval[2] = (double)s_v;
                        M->sval[3] = (double)t_v;
                    }
                } else {
                    q = -1;
                }
            }
        }
        const int q0 = __shfl_sync(0xffffffffu, q, 0);
        const bool uniform = __all_sync(0xffffffffu, q == q0 || q < 0);
        int qa = q;
        if (uniform) {
            // q0 may be -1 when lane 0's slot is empty: take any valid lane's query
            const unsigned has = __ballot_sync(0xffffffffu, q >= 0);
            qa = has ? __shfl_sync(0xffffffffu, q, __ffs(has) - 1) : -1;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                vp += __shfl_xor_sync(0xffffffffu, vp, o);
                vu += __shfl_xor_sync(0xffffffffu, vu, o);
                cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
                m1s = max(m1s, __shfl_xor_sync(0xffffffffu, m1s, o));
                m1t = max(m1t, __shfl_xor_sync(0xffffffffu, m1t, o));
            }
            if ((threadIdx.x & 31) != 0) qa = -1;
        }
        if (qa >= 0 && cnt > 0) {
            QSmm* M = a.sm + qa;
            atomicAdd(&M->vol_paper, vp);
            atomicAdd(&M->vol_union, vu);
            atomicAdd(&M->count, cnt);
            atomicMax(&M->max1s, m1s);
            atomicMax(&M->max1t, m1t);
        }
    }
}

// top2: max_2 of each vector = the largest value below max_1, or max_1 itself
// when it occurs twice (the multiset's second element); aggregated per warp
template <typename T>
__global__ void __launch_bounds__(256) smm_top2_kernel(SmmArgs a) {
    const int parity = a.ctl->iter & 1;
    const int64_t lo = a.ctl->lo[parity], hi = a.ctl->hi[parity];
    const T* ys = reinterpret_cast<const T*>(a.ys);
    const T* yt = reinterpret_cast<const T*>(a.yt);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = lo + (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < hi; base += stride) {
        const int64_t j = base + (threadIdx.x & 31);
        int q = -1;
        unsigned long long m2s = 0, m2t = 0, c1s = 0, c1t = 0;
        const GEntry e = j < hi ? a.ent[j] : GEntry{-1, 0u, 0.0};
        if (e.v >= 0) {
            q = (int)(e.bits >> 2);
            const QSmm* M = a.sm + q;
            if (M->run) {
                const unsigned long long bs = (unsigned long long)__double_as_longlong((double)ys[j]);
                const unsigned long long bt = (unsigned long long)__double_as_longlong((double)yt[j]);
                if (bs < M->max1s) m2s = bs; else c1s = 1;
                if (bt < M->max1t) m2t = bt; else c1t = 1;
            } else {
                q = -1;
            }
        }
        const int q0 = __shfl_sync(0xffffffffu, q, 0);
        const bool uniform = __all_sync(0xffffffffu, q == q0 || q < 0);
        int qa = q;
        if (uniform) {
            const unsigned has = __ballot_sync(0xffffffffu, q >= 0);
            qa = has ? __shfl_sync(0xffffffffu, q, __ffs(has) - 1) : -1;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                m2s = max(m2s, __shfl_xor_sync(0xffffffffu, m2s, o));
                m2t = max(m2t, __shfl_xor_sync(0xffffffffu, m2t, o));
                c1s += __shfl_xor_sync(0xffffffffu, c1s, o);
                c1t += __shfl_xor_sync(0xffffffffu, c1t, o);
            }
            if ((threadIdx.x & 31) != 0) qa = -1;
        }
        if (qa >= 0) {
            QSmm* M = a.sm + qa;
            if (m2s) atomicMax(&M->max2s, m2s);
            if (m2t) atomicMax(&M->max2t, m2t);
            if (c1s) atomicAdd(&M->cnt1s, c1s);
            if (c1t) atomicAdd(&M->cnt1t, c1t);
        }
    }
}

// decide: one thread per query whose table was just finished; a query that
// continues gets its next table (or dense column) here. With a learned
// switch, the CTA stages the network's weights in shared memory once some
// query of it needs the network (where Eq. (17) continues).
__global__ void smm_decide_kernel(SmmArgs a) {
    const int iter = a.ctl->iter;
    const bool learned = iter > 0 && a.policy == 1 && a.mlp_w != nullptr;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // a loop of the same trip count for every thread of the CTA (the network is evaluated by the whole warp)
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < a.nq; base += stride) {
        const int64_t q = base + threadIdx.x;
        const bool active = q < a.nq && a.sm[q].run && a.st[q].status == ST_SMM;
        QSmm* M = a.sm + (active ? q : 0);
        QState* Q = a.st + (active ? q : 0);
        const int64_t lb = iter;
        double psi = 0.0, h = 0.0, vol = 0.0;
        int64_t eta0 = 0, ell = 0, lf = 0;
        bool go = false, need = false;
        float f[kMlpIn];
        if (active) {
            const double ds = (double)Q->ds, dt = (double)Q->dt;
            // Algorithm 2: r_b += s*(s)/d(s) + t*(t)/d(t) - s*(t)/d(s) - t*(s)/d(t)
            Q->r_b += M->sval[0] / ds + M->sval[3] / dt - M->sval[2] / ds - M->sval[1] / dt;
            ell = Q->ell;
            double s1, s2, t1, t2;
            smm_maxima(M, &s1, &s2, &t1, &t2);
            vol = (double)M->vol_paper;
            lf = ell - lb;
            if (lf > 0)
                switch_quantities(lf, s1, s2, t1, t2, ds, dt, Q->eps, a.log_2tau_delta, a.tau, &psi, &eta0, &h);
            if (iter == 0) {
                go = M->lb_target >= 0 ? (M->lb_target > 0) : (ell >= 1);  // the loop runs once when l >= 1
            } else {
                // Eq. (17); a learned switch may stop a query earlier than Eq. (17)
                // does, never later (the rule bounds its SMM work): its network is
                // consulted only where the rule continues
                const bool rule_stop = (lb >= ell) || vol > h;
                go = M->lb_target >= 0 ? (lb < M->lb_target) : !rule_stop;
                need = learned && M->lb_target < 0 && !rule_stop;
                if (need || (a.trace && lb <= a.trace_steps))
                    switch_features(Q->ds, Q->dt, lf, M->vol_paper, h, s1, t1, f);
                if (a.trace && lb <= a.trace_steps) {
                    // cost log of the learned switch: its inputs and the next push's size
                    float* row = a.trace + ((int64_t)q * a.trace_steps + (lb - 1)) * kTraceWidth;
#pragma unroll
                    for (int k = 0; k < kMlpIn; ++k) row[k] = f[k];
                    row[6] = (float)M->vol_union;
                    row[7] = (float)M->vol_paper;
                }
            }
        }
        if (learned) {
            // the network of each query that needs it, by the whole warp (the CTA)
            const float y = mlp_eval_asked(a.mlp_wt, a.mlp_norm, f, need);
            if (need && y >= 0.f) go = false;
        }
        if (!active) continue;
        // the table just finished holds the current frontier
        M->tab_off = M->ntab_off;
        M->tab_cap = M->ntab_cap;
        if (go) continue_smm(a, q, Q, M, lb, M->vol_union);
        else leave_smm(a, q, Q, M, iter, lb, lf, psi, vol, h, eta0, (int64_t)M->count);
        M->vol_paper = M->vol_union = M->count = 0;
        M->max1s = M->max1t = M->max2s = M->max2t = M->cnt1s = M->cnt1t = 0;
        M->sval[0] = M->sval[1] = M->sval[2] = M->sval[3] = 0.0;
    }
}

// advance: clears the tables handed out since the last advance (by the
// start kernel or the decision just taken) and, in the CTA that finishes
// last, keeps the books: their slot range for the next iteration's kernels,
// iteration += 1, the count of continuing queries for the host loop and, in
// a captured graph, the while condition (another iteration while some query
// continues).
__global__ void __launch_bounds__(256) smm_advance_kernel(SmmArgs a, cudaGraphConditionalHandle h, int use_handle) {
    __shared__ bool last;
    SmmCtl* C = a.ctl;
    const int64_t base = (int64_t)kF0Slots * a.nq;
    const int64_t lo = base + (int64_t)C->mark;
    const int64_t hi = min(base + (int64_t)C->cursor, a.pool_cap);
    for (int64_t j = lo + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < hi;
         j += (int64_t)gridDim.x * blockDim.x) {
        GEntry e;
        e.v = -1;
        e.bits = 0;
        e.g = 0.0;
        a.ent[j] = e;
        a.sum_s[j] = 0ull;
        a.sum_t[j] = 0ull;
    }
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&C->adv_done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last || threadIdx.x != 0) return;
    // every other CTA has read mark and cursor (before counting itself done)
    const int next = C->iter + 1;
    C->lo[next & 1] = lo;
    C->hi[next & 1] = hi > lo ? hi : lo;
    C->mark = C->cursor;
    C->iter = next;
    C->n_go = C->n_want;
    C->n_want = 0;
    if (C->n_heavy > C->heavy_max) C->heavy_max = C->n_heavy;
    C->n_heavy = 0;
    C->adv_done = 0u;
    if (a.hybrid) {
        // the moved queries' columns are filled; their blocks are zeroed
        const int qpb = a.dense_width / 2;
        const int used = min(C->dense_next, a.dense_cap);
        C->dense_open = (used + qpb - 1) / qpb;
        C->n_mig = 0;
    }
    if (use_handle) cudaGraphSetConditional(h, C->n_go > 0 ? 1u : 0u);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
void launch_smm_setup(const SmmArgs& a, cudaStream_t st) {
    const int grid = query_grid(a.nq);
    prof_begin(FAM_SMM_SETUP, st);
    smm_setup_kernel<<<grid, kQueryCta, 0, st>>>(a);
    prof_end(FAM_SMM_SETUP, st);
    note_launches(1);
}

void launch_smm_start(bool fp64, const SmmArgs& a, cudaStream_t st) {
    const int grid = query_grid(a.nq);
    prof_begin(FAM_SMM_SETUP, st);
    if (fp64) smm_start_kernel<double><<<grid, kQueryCta, 0, st>>>(a);
    else smm_start_kernel<float><<<grid, kQueryCta, 0, st>>>(a);
    prof_end(FAM_SMM_SETUP, st);
    note_launches(1);
}

void launch_smm_push(bool fp64, const SmmArgs& a, int grid, cudaStream_t st) {
    prof_begin(FAM_SMM_PUSH, st);
    if (fp64) smm_push_kernel<double><<<grid, 256, 0, st>>>(a);
    else smm_push_kernel<float><<<grid, 256, 0, st>>>(a);
    prof_end(FAM_SMM_PUSH, st);
    prof_begin(FAM_SMM_PUSH_HEAVY, st);
    if (fp64) smm_push_heavy_kernel<double><<<grid, 256, 0, st>>>(a);
    else smm_push_heavy_kernel<float><<<grid, 256, 0, st>>>(a);
    prof_end(FAM_SMM_PUSH_HEAVY, st);
    note_launches(2);
}

void launch_smm_finish(bool fp64, const SmmArgs& a, int grid, cudaStream_t st) {
    prof_begin(FAM_SMM_FINISH, st);
    if (fp64) smm_finish_kernel<double><<<grid, 256, 0, st>>>(a);
    else smm_finish_kernel<float><<<grid, 256, 0, st>>>(a);
    prof_end(FAM_SMM_FINISH, st);
    note_launches(1);
}

void launch_smm_top2(bool fp64, const SmmArgs& a, int grid, cudaStream_t st) {
    prof_begin(FAM_SMM_TOP2, st);
    if (fp64) smm_top2_kernel<double><<<grid, 256, 0, st>>>(a);
    else smm_top2_kernel<float><<<grid, 256, 0, st>>>(a);
    prof_end(FAM_SMM_TOP2, st);
    note_launches(1);
}

void launch_smm_decide(const SmmArgs& a, cudaStream_t st, bool first) {
    const int grid = query_grid(a.nq);
    (void)first;
    prof_begin(FAM_SMM_DECIDE, st);
    smm_decide_kernel<<<grid, kQueryCta, 0, st>>>(a);
    prof_end(FAM_SMM_DECIDE, st);
    note_launches(1);
}

void launch_smm_advance(const SmmArgs& a, int grid, cudaGraphConditionalHandle h, bool use_handle, cudaStream_t st) {
    prof_begin(FAM_SMM_ADVANCE, st);
    smm_advance_kernel<<<grid, 256, 0, st>>>(a, h, use_handle ? 1 : 0);
    prof_end(FAM_SMM_ADVANCE, st);
    note_launches(1);
}

void launch_smm_body(bool fp64, const SmmArgs& a, int grid, cudaStream_t st) {
    launch_smm_push(fp64, a, grid, st);
    launch_smm_finish(fp64, a, grid, st);
    launch_smm_top2(fp64, a, grid, st);
}

void launch_smm_iteration(bool fp64, const SmmArgs& a, int grid, cudaStream_t st) {
    launch_smm_body(fp64, a, grid, st);
    launch_smm_decide(a, st);
}

}  // namespace geer
