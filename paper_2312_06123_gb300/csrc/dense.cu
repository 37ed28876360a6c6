// dense.cu -- the SMM iteration of GEER (Algorithm 2 inside Algorithm 3) as
// a dense pull SpMM over blocks of query vectors, for queries whose
// frontiers cover much of the graph (deep SMM: small eps, low degrees, or a
// fixed l_b such as the standalone SMM of Section 4.1.1).
//
// A dense block holds B = 32 * VEC columns, the (s*, t*) pairs of B/2
// queries, row-major: X[v * B + c], double-buffered across iterations. Lane
// l of a warp owns columns [l * VEC, (l + 1) * VEC), so one gathered row is
// one coalesced B * sizeof(T) load. Per row v:
//   y(v, c) = (sum over u in N(v) of x(u, c)) / d(v),
//   support(v, c) = OR over u in N(v) of support(u, c),
// with support kept structurally (Eq. 17's V_s, V_t) in the sign bit of the
// stored value: every value is >= 0, a stored -y means "y, in the support".
// Once every running column of a block covers all n nodes (support at i
// steps then stays full, the graph being connected), the kernel stops
// tracking it.
//
// Work is split into units built once per graph: runs of up to 32 light rows
// (at most kUnitEdges edges), and pieces of kPieceEdges edges of the heavy
// rows (degree > kHeavyDeg), handed out by an atomic counter per block,
// heavy pieces first. A warp walks the edges of its unit with G row gathers
// in flight; a heavy row's pieces write partial sums, and the warp that
// completes a row's last piece adds them in piece order and finishes the
// row, so every sum has a fixed order and the result is deterministic.
//
// Columns of queries that left SMM keep their last values (the walks read
// them). The epilogue is fused: per query, Eq. 17's volume, the support
// union's volume and size, max_1/max_2 of s* and t* (per-warp partials
// merged in a fixed order) and the values at s and t for the series terms.
#include <algorithm>
#include <vector>

#include "geer_internal.cuh"
#include "geer_kernels.h"

namespace geer {

namespace {

constexpr int kHeavyDeg = 512;    // rows above this degree are split into pieces
constexpr int kPieceEdges = 512;  // edges per heavy-row piece
constexpr int kUnitRows = 32;     // rows per light unit (one node record per lane)
constexpr int kUnitEdges = 512;   // edges per light unit
constexpr unsigned kFull = 0xffffffffu;

template <typename T, int VEC>
struct Pack {
    T e[VEC];
};

// One lane's VEC consecutive values of a row, read-only path (the gathers).
template <typename T, int VEC>
__device__ __forceinline__ Pack<T, VEC> ld_row(const T* p) {
    Pack<T, VEC> r;
    if constexpr (sizeof(T) == 4 && VEC == 4) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(p));
        r.e[0] = v.x; r.e[1] = v.y; r.e[2] = v.z; r.e[3] = v.w;
    } else if constexpr (sizeof(T) == 4 && VEC == 2) {
        const float2 v = __ldg(reinterpret_cast<const float2*>(p));
        r.e[0] = v.x; r.e[1] = v.y;
    } else if constexpr (sizeof(T) == 8 && VEC == 2) {
        const double2 v = __ldg(reinterpret_cast<const double2*>(p));
        r.e[0] = v.x; r.e[1] = v.y;
    } else {
        static_assert(VEC == 1, "unsupported lane width");
        r.e[0] = __ldg(p);
    }
    return r;
}

// Same, through L2 only (pieces written by other warps of the same launch).
template <typename T, int VEC>
__device__ __forceinline__ Pack<T, VEC> ld_l2(const T* p) {
    Pack<T, VEC> r;
    if constexpr (sizeof(T) == 4 && VEC == 4) {
        const float4 v = __ldcg(reinterpret_cast<const float4*>(p));
        r.e[0] = v.x; r.e[1] = v.y; r.e[2] = v.z; r.e[3] = v.w;
    } else if constexpr (sizeof(T) == 4 && VEC == 2) {
        const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
        r.e[0] = v.x; r.e[1] = v.y;
    } else if constexpr (sizeof(T) == 8 && VEC == 2) {
        const double2 v = __ldcg(reinterpret_cast<const double2*>(p));
        r.e[0] = v.x; r.e[1] = v.y;
    } else {
        r.e[0] = __ldcg(p);
    }
    return r;
}

// Vector store; `streaming` marks it evict-first (the next iteration's rows),
// else it stays in L2 (piece partials).
template <typename T, int VEC, bool streaming>
__device__ __forceinline__ void st_row(T* p, const Pack<T, VEC>& r) {
    if constexpr (sizeof(T) == 4 && VEC == 4) {
        const float4 v = make_float4(r.e[0], r.e[1], r.e[2], r.e[3]);
        if constexpr (streaming) __stcs(reinterpret_cast<float4*>(p), v);
        else __stcg(reinterpret_cast<float4*>(p), v);
    } else if constexpr (sizeof(T) == 4 && VEC == 2) {
        const float2 v = make_float2(r.e[0], r.e[1]);
        if constexpr (streaming) __stcs(reinterpret_cast<float2*>(p), v);
        else __stcg(reinterpret_cast<float2*>(p), v);
    } else if constexpr (sizeof(T) == 8 && VEC == 2) {
        const double2 v = make_double2(r.e[0], r.e[1]);
        if constexpr (streaming) __stcs(reinterpret_cast<double2*>(p), v);
        else __stcg(reinterpret_cast<double2*>(p), v);
    } else {
        if constexpr (streaming) __stcs(p, r.e[0]);
        else __stcg(p, r.e[0]);
    }
}

// High 32 bits of a value: bit 31 is its sign, i.e. its support bit.
__device__ __forceinline__ uint32_t hiword(float x) { return __float_as_uint(x); }
__device__ __forceinline__ uint32_t hiword(double x) { return (uint32_t)__double2hiint(x); }
// y >= 0 with the support bit (bit 31 of s) as its sign.
__device__ __forceinline__ float with_support(float y, uint32_t s) {
    return __uint_as_float(__float_as_uint(y) | (s & 0x80000000u));
}
__device__ __forceinline__ double with_support(double y, uint32_t s) { return (s & 0x80000000u) ? -y : y; }

template <typename T>
__device__ __forceinline__ void top2_push(T& a, T& b, T v) {
    if (v > a) {
        b = a;
        a = v;
    } else if (v > b) {
        b = v;
    }
}

// What one lane knows about its columns, and its epilogue accumulators.
template <typename T, int VEC>
struct Lane {
    static constexpr int QPL = VEC >= 2 ? VEC / 2 : 1;  // queries per lane
    int32_t q[QPL];
    bool act[QPL];
    int32_t s_node[QPL], t_node[QPL];
    bool all_act;
    // per-warp sums stay below the stored edge count, < 2^32 for this engine
    uint32_t vol[VEC];  // sum of d(v) over support rows, per column
    T m1[VEC], m2[VEC]; // top-2 of the column's values
    uint32_t vu[QPL], cnt[QPL];
};

template <int VEC>
__device__ __forceinline__ int lane_query(int e) {
    return VEC >= 2 ? e / 2 : 0;
}

// Finish row v: y = acc / d(v), the support bits, the store of the running
// columns and the epilogue. Called by the whole warp.
template <typename T, int VEC, bool SUP>
__device__ __forceinline__ void flush_row(Lane<T, VEC>& L, const DenseArgs& d, T* xrow, int64_t v, uint32_t deg,
                                          const T (&acc)[VEC], const uint32_t (&sg)[VEC], int lane) {
    const T inv = deg ? T(1) / (T)deg : T(0);
    Pack<T, VEC> out;
    uint32_t bit[VEC];
    T y[VEC];
#pragma unroll
    for (int e = 0; e < VEC; ++e) {
        bit[e] = SUP ? (sg[e] >> 31) : 1u;
        y[e] = acc[e] * inv;
        out.e[e] = with_support(y[e], bit[e] << 31);
    }
    if (L.all_act) {
        st_row<T, VEC, true>(xrow, out);
    } else {
#pragma unroll
        for (int e = 0; e < VEC; ++e)
            if (L.act[lane_query<VEC>(e)]) __stcs(xrow + e, out.e[e]);
    }
#pragma unroll
    for (int e = 0; e < VEC; ++e) {
        const int i = lane_query<VEC>(e);
        const int which = VEC >= 2 ? (e & 1) : (lane & 1);  // 0: s*, 1: t*
        if (!L.act[i]) continue;
        L.vol[e] += deg * bit[e];
        top2_push(L.m1[e], L.m2[e], y[e]);
        if (v == L.s_node[i]) d.sm[L.q[i]].sval[which] = (double)y[e];
        if (v == L.t_node[i]) d.sm[L.q[i]].sval[2 + which] = (double)y[e];
    }
#pragma unroll
    for (int i = 0; i < Lane<T, VEC>::QPL; ++i) {
        uint32_t both;
        if constexpr (VEC >= 2) both = bit[2 * i] | bit[2 * i + 1];
        else both = bit[0] | __shfl_xor_sync(kFull, bit[0], 1);
        if (L.act[i]) {
            L.vu[i] += deg * both;
            L.cnt[i] += both;
        }
    }
}

// Asynchronous copy of one lane's VEC values of a gathered row into its
// shared-memory ring slot (cp.async; completion tracked per thread by
// commit/wait groups, so each lane later reads only bytes it copied itself).
template <int BYTES>
__device__ __forceinline__ void cp_async_lane(uint32_t dst, const void* src) {
    if constexpr (BYTES == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(dst), "l"(src), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

template <typename T, int VEC>
__device__ __forceinline__ Pack<T, VEC> ld_ring(const T* p) {
    Pack<T, VEC> r;
    if constexpr (sizeof(T) == 4 && VEC == 4) {
        const float4 v = *reinterpret_cast<const float4*>(p);
        r.e[0] = v.x; r.e[1] = v.y; r.e[2] = v.z; r.e[3] = v.w;
    } else if constexpr (sizeof(T) == 4 && VEC == 2) {
        const float2 v = *reinterpret_cast<const float2*>(p);
        r.e[0] = v.x; r.e[1] = v.y;
    } else if constexpr (sizeof(T) == 8 && VEC == 2) {
        const double2 v = *reinterpret_cast<const double2*>(p);
        r.e[0] = v.x; r.e[1] = v.y;
    } else {
        r.e[0] = *p;
    }
    return r;
}

#ifndef GEER_DENSE_RING_BYTES
#define GEER_DENSE_RING_BYTES 12288
#endif
constexpr int kRingBytes = GEER_DENSE_RING_BYTES;  // shared-memory gather ring per warp
#ifndef GEER_DENSE_GROUP
#define GEER_DENSE_GROUP 8
#endif
constexpr int kGroup = GEER_DENSE_GROUP;           // row gathers per cp.async group

// Process the work units of block `blk` until they run out. Gathered rows
// stream through the warp's ring: RING slots of one row each, D = RING / 8
// groups of 8 rows in flight ahead of the consumer.
template <typename T, int VEC, bool SUP>
__device__ __forceinline__ void run_units(Lane<T, VEC>& L, const DenseArgs& d, int blk, int lane, T* ring) {
    constexpr int B = 32 * VEC;
    constexpr int LB = VEC * (int)sizeof(T);  // bytes per lane and row
    constexpr int RING = kRingBytes / (B * (int)sizeof(T));
    constexpr int D = RING / kGroup;
    static_assert(D >= 2, "ring too small");
    const int64_t n = d.g.n;
    const int iter = d.ctl->iter;
    const T* Xc = reinterpret_cast<const T*>(d.X[(iter & 1) ^ 1]) + (int64_t)blk * n * B + lane * VEC;
    T* Xn = reinterpret_cast<T*>(d.X[iter & 1]) + (int64_t)blk * n * B + lane * VEC;
    const int32_t* col = d.g.col_idx;
    T* my = ring + lane * VEC;
    const uint32_t my_s = (uint32_t)__cvta_generic_to_shared(my);

    unsigned u = 0;
    if (lane == 0) u = atomicAdd(d.unit_ctr + blk, 1u);
    u = __shfl_sync(kFull, u, 0);
    while (u < (unsigned)d.nunits) {
        unsigned nu = 0;
        if (lane == 0) nu = atomicAdd(d.unit_ctr + blk, 1u);  // next unit, used at the end
        const int4 U = __ldg(d.units + u);
        const bool heavy = U.x < 0;
        const uint32_t e0 = (uint32_t)U.z, e1 = (uint32_t)U.w;
        int nr = 0;
        uint2 ni = make_uint2(0u, 0u);
        if (!heavy) {
            nr = U.y - U.x;
            if (lane < nr) ni = __ldcs(d.g.node_info + U.x + lane);
        }
        // producer state: next edge to gather, its ring slot, the index chunk holding it
        uint32_t ie = e0;
        int islot = 0;
        uint32_t icb = e0;
        int32_t cid = e0 + lane < e1 ? __ldcs(col + e0 + lane) : 0;
        int32_t cid_next = e0 + 32 + lane < e1 ? __ldcs(col + e0 + 32 + lane) : 0;
        auto issue_group = [&]() {
#pragma unroll
            for (int j = 0; j < kGroup; ++j) {
                if (ie < e1) {
                    if (ie == icb + 32) {
                        icb += 32;
                        cid = cid_next;
                        cid_next = icb + 32 + lane < e1 ? __ldcs(col + icb + 32 + lane) : 0;
                    }
                    const int32_t nb = __shfl_sync(kFull, cid, (int)(ie - icb));
                    cp_async_lane<LB>(my_s + islot * (B * (int)sizeof(T)), Xc + (int64_t)nb * B);
                    ++ie;
                    islot = islot + 1 == RING ? 0 : islot + 1;
                }
            }
            cp_async_commit();
        };
#pragma unroll 1
        for (int g = 0; g < D; ++g) issue_group();

        int ri = 0;
        uint32_t row_end = heavy ? 0xffffffffu : __shfl_sync(kFull, ni.x + ni.y, 0);
        T acc[VEC];
        uint32_t sg[VEC];
#pragma unroll
        for (int e = 0; e < VEC; ++e) {
            acc[e] = T(0);
            sg[e] = 0u;
        }
        uint32_t ce = e0;
        int cslot = 0;
        while (ce < e1) {
            cp_async_wait<D - 1>();  // the oldest group in flight has landed
#pragma unroll
            for (int j = 0; j < kGroup; ++j) {
                if (ce < e1) {
                    const Pack<T, VEC> v = ld_ring<T, VEC>(my + cslot * B);
#pragma unroll
                    for (int e = 0; e < VEC; ++e) {
                        acc[e] += fabs(v.e[e]);
                        if (SUP) sg[e] |= hiword(v.e[e]);
                    }
                    if (ce + 1 == row_end) {
                        const int64_t row = (int64_t)U.x + ri;
                        const uint32_t deg = __shfl_sync(kFull, ni.y, ri);
                        flush_row<T, VEC, SUP>(L, d, Xn + row * B, row, deg, acc, sg, lane);
#pragma unroll
                        for (int e = 0; e < VEC; ++e) {
                            acc[e] = T(0);
                            sg[e] = 0u;
                        }
                        ++ri;
                        const uint32_t nxt = __shfl_sync(kFull, ni.x + ni.y, ri & 31);
                        row_end = ri < nr ? nxt : 0xffffffffu;
                    }
                    ++ce;
                    cslot = cslot + 1 == RING ? 0 : cslot + 1;
                }
            }
            issue_group();  // refill the slots just read (empty past the unit's end)
        }
        cp_async_wait<0>();
        if (heavy) {
            // a piece of a heavy row: store its partial sum; the last piece done finishes the row
            const int h = -U.x - 1, p = U.y;
            const int4 H = __ldg(d.heavy + h);  // {row, first slot, pieces, degree}
            T* P = reinterpret_cast<T*>(d.pieces) + ((int64_t)blk * d.nslots + H.y) * B + lane * VEC;
            Pack<T, VEC> out;
#pragma unroll
            for (int e = 0; e < VEC; ++e) out.e[e] = with_support(acc[e], SUP ? sg[e] : 0x80000000u);
            st_row<T, VEC, false>(P + (int64_t)p * B, out);
            __threadfence();
            unsigned old = 0;
            unsigned* ctr = d.heavy_ctr + (int64_t)blk * d.nheavy + h;
            if (lane == 0) old = atomicAdd(ctr, 1u);
            old = __shfl_sync(kFull, old, 0);
            if (old + 1 == (unsigned)H.z) {
                __threadfence();
#pragma unroll
                for (int e = 0; e < VEC; ++e) {
                    acc[e] = T(0);
                    sg[e] = 0u;
                }
                constexpr int G = 8;
                for (int p0 = 0; p0 < H.z; p0 += G) {
                    Pack<T, VEC> w[G];
#pragma unroll
                    for (int j = 0; j < G; ++j)
                        if (p0 + j < H.z) w[j] = ld_l2<T, VEC>(P + (int64_t)(p0 + j) * B);
#pragma unroll
                    for (int j = 0; j < G; ++j)
                        if (p0 + j < H.z) {
#pragma unroll
                            for (int e = 0; e < VEC; ++e) {
                                acc[e] += fabs(w[j].e[e]);
                                if (SUP) sg[e] |= hiword(w[j].e[e]);
                            }
                        }
                }
                flush_row<T, VEC, SUP>(L, d, Xn + (int64_t)H.x * B, H.x, (uint32_t)H.w, acc, sg, lane);
                if (lane == 0) *ctr = 0u;  // every piece of this launch has counted
            }
        }
        u = __shfl_sync(kFull, nu, 0);
    }
}

}  // namespace

// Iteration 0 of the dense queries: columns e_s, e_t (in the support) in
// buffer 0 and the per-query sums of the initial frontier {s, t}.
template <typename T>
__global__ void dense_init_kernel(DenseArgs d) {
    const int nq_block = d.width / 2;
    const int64_t total = (int64_t)d.nblocks * nq_block;
    T* X0 = reinterpret_cast<T*>(d.X[0]);
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(k / nq_block), j = (int)(k % nq_block);
        const int q = d.block_q[k];
        if (q < 0) continue;
        const QState* Q = d.st + q;
        QSmm* M = d.sm + q;
        if (Q->status != ST_SMM) continue;
        const int64_t base = (int64_t)b * d.g.n;
        X0[(base + Q->s) * d.width + 2 * j] = T(-1);  // 1, in the support
        X0[(base + Q->t) * d.width + 2 * j + 1] = T(-1);
        M->vol_paper = (unsigned long long)(Q->ds + Q->dt);
        M->vol_union = (unsigned long long)(Q->ds + Q->dt);
        M->count = 2;
        M->max1s = M->max1t = (unsigned long long)__double_as_longlong(1.0);
        M->max2s = M->max2t = 0ull;
        M->cnt1s = M->cnt1t = 1;
        M->sval[0] = 1.0;  // s*(s)
        M->sval[1] = 0.0;  // t*(s)
        M->sval[2] = 0.0;  // s*(t)
        M->sval[3] = 1.0;  // t*(t)
    }
}

// One pull SpMM iteration over every dense block with a running query.
// grid.y = dense block; grid.x * 8 = part_warps persistent warps per block.
#ifndef GEER_DENSE_MINB
#define GEER_DENSE_MINB 2
#endif
template <typename T, int VEC>
__global__ void __launch_bounds__(256, GEER_DENSE_MINB) dense_spmm_kernel(DenseArgs d) {
    constexpr int B = 32 * VEC;
    using L_t = Lane<T, VEC>;
    constexpr int QPL = L_t::QPL;
    const int blk = blockIdx.y;
    const int run = d.block_run[blk];
    if (!run) return;
    const int lane = threadIdx.x & 31;
    L_t L;
    L.all_act = true;
#pragma unroll
    for (int i = 0; i < QPL; ++i) {
        const int j = VEC >= 2 ? lane * QPL + i : lane / 2;
        L.q[i] = d.block_q[blk * (B / 2) + j];
        L.act[i] = L.q[i] >= 0 && d.sm[L.q[i]].run && d.sm[L.q[i]].dense;
        L.s_node[i] = L.act[i] ? d.st[L.q[i]].s : -1;
        L.t_node[i] = L.act[i] ? d.st[L.q[i]].t : -1;
        L.all_act &= L.act[i];
        L.vu[i] = L.cnt[i] = 0u;
    }
#pragma unroll
    for (int e = 0; e < VEC; ++e) {
        L.vol[e] = 0u;
        L.m1[e] = L.m2[e] = T(0);  // entries are >= 0; zeros are in the multiset
    }
    extern __shared__ __align__(16) unsigned char dense_smem[];
    T* ring = reinterpret_cast<T*>(dense_smem + (threadIdx.x >> 5) * kRingBytes);
    if (run == 1) run_units<T, VEC, true>(L, d, blk, lane, ring);
    else run_units<T, VEC, false>(L, d, blk, lane, ring);

    // one partial per warp and query
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    DensePartial* base = d.part + ((int64_t)blk * d.part_warps + warp) * (B / 2);
    if constexpr (VEC >= 2) {
#pragma unroll
        for (int i = 0; i < QPL; ++i) {
            DensePartial* p = base + lane * QPL + i;
            p->vp = (unsigned long long)L.vol[2 * i] + L.vol[2 * i + 1];
            p->vu = L.vu[i];
            p->cnt = L.cnt[i];
            p->s1 = (double)L.m1[2 * i];
            p->s2 = (double)L.m2[2 * i];
            p->t1 = (double)L.m1[2 * i + 1];
            p->t2 = (double)L.m2[2 * i + 1];
        }
    } else {
        const uint32_t ovol = __shfl_xor_sync(kFull, L.vol[0], 1);
        const T om1 = __shfl_xor_sync(kFull, L.m1[0], 1), om2 = __shfl_xor_sync(kFull, L.m2[0], 1);
        if ((lane & 1) == 0) {
            DensePartial* p = base + lane / 2;
            p->vp = (unsigned long long)L.vol[0] + ovol;
            p->vu = L.vu[0];
            p->cnt = L.cnt[0];
            p->s1 = (double)L.m1[0];
            p->s2 = (double)L.m2[0];
            p->t1 = (double)om1;
            p->t2 = (double)om2;
        }
    }
}

// Merge the per-warp partials of every running dense query (fixed order)
// into its SMM accumulators; one warp per query.
__global__ void __launch_bounds__(256) dense_reduce_kernel(DenseArgs d) {
    const int lane = threadIdx.x & 31;
    const int nq_block = d.width / 2;
    const int64_t total = (int64_t)d.nblocks * nq_block;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= total) return;
    const int blk = (int)(w / nq_block), j = (int)(w % nq_block);
    const int q = d.block_q[w];
    if (q < 0 || !d.block_run[blk]) return;
    QSmm* M = d.sm + q;
    if (!M->run || !M->dense) return;
    unsigned long long vp = 0, vu = 0, cnt = 0;
    double a1 = 0.0, a2 = 0.0, b1 = 0.0, b2 = 0.0;
    for (int64_t k = lane; k < d.part_warps; k += 32) {
        const DensePartial& p = d.part[((int64_t)blk * d.part_warps + k) * nq_block + j];
        vp += p.vp;
        vu += p.vu;
        cnt += p.cnt;
        top2_merge(a1, a2, p.s1, p.s2);
        top2_merge(b1, b2, p.t1, p.t2);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        vp += __shfl_xor_sync(kFull, vp, o);
        vu += __shfl_xor_sync(kFull, vu, o);
        cnt += __shfl_xor_sync(kFull, cnt, o);
        top2_merge(a1, a2, __shfl_xor_sync(kFull, a1, o), __shfl_xor_sync(kFull, a2, o));
        top2_merge(b1, b2, __shfl_xor_sync(kFull, b1, o), __shfl_xor_sync(kFull, b2, o));
    }
    if (lane == 0) {
        M->vol_paper = vp;
        M->vol_union = vu;
        M->count = cnt;
        M->max1s = (unsigned long long)__double_as_longlong(a1);
        M->max2s = (unsigned long long)__double_as_longlong(a2);
        M->max1t = (unsigned long long)__double_as_longlong(b1);
        M->max2t = (unsigned long long)__double_as_longlong(b2);
        M->cnt1s = M->cnt1t = 0;  // max2 is exact (ties included)
    }
}

// Column map: column pair j of block b serves query b * (width/2) + j.
__global__ void dense_map_kernel(DenseArgs d, int64_t nq) {
    const int64_t total = (int64_t)d.nblocks * (d.width / 2);
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x)
        const_cast<int32_t*>(d.block_q)[k] = k < nq ? (int32_t)k : -1;
}

// Per block: 0 when no query is still in SMM, 1 when one is, 2 when, in
// addition, every such query's support covers all n nodes after the last
// iteration. Resets the blocks' unit counters.
__global__ void dense_block_flags_kernel(DenseArgs d) {
    const int nq_block = d.width / 2;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < d.nblocks; b += gridDim.x * blockDim.x) {
        int any = 0, partial = 0;
        for (int j = 0; j < nq_block; ++j) {
            const int q = d.block_q[b * nq_block + j];
            if (q >= 0 && d.sm[q].run && d.sm[q].dense) {
                any = 1;
                if (d.sm[q].count < (unsigned long long)d.g.n) partial = 1;
            }
        }
        d.block_run[b] = any ? (partial ? 1 : 2) : 0;
        d.unit_ctr[b] = 0u;
    }
}

// Hybrid engine: blocks that received their first column in this decision
// start as zeros in both buffers (columns are handed out in order, so the
// new blocks are [dense_open, ceil(used / (width/2)))).
__global__ void dense_open_kernel(DenseArgs d, int cap) {
    const int qpb = d.width / 2;
    const int b0 = d.ctl->dense_open;
    const int b1 = (min(d.ctl->dense_next, cap) + qpb - 1) / qpb;
    if (b1 <= b0) return;
    const size_t esz = d.fp64 ? 8 : 4;
    const int64_t per = d.g.n * (int64_t)d.width * (int64_t)esz / 16;  // uint4 per block and buffer
    const int64_t total = (int64_t)(b1 - b0) * per;
    for (int buf = 0; buf < 2; ++buf) {
        uint4* X = reinterpret_cast<uint4*>(d.X[buf]) + (int64_t)b0 * per;
        for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total;
             k += (int64_t)gridDim.x * blockDim.x)
            X[k] = make_uint4(0u, 0u, 0u, 0u);
    }
}

// Hybrid engine: each query the last decision moved writes its frontier
// table (F_l_b with s*, t* and the support bits of V_s, V_t) into its
// column pair of the buffer the next SpMM reads. One CTA per moved query.
template <typename T>
__global__ void dense_migrate_kernel(DenseArgs d, SmmArgs a) {
    const int nm = a.ctl->n_mig;
    const int iter = a.ctl->iter;
    T* X = reinterpret_cast<T*>(d.X[iter & 1]);
    const T* ys = reinterpret_cast<const T*>(a.ys);
    const T* yt = reinterpret_cast<const T*>(a.yt);
    for (int k = blockIdx.x; k < nm; k += gridDim.x) {
        const int q = a.mig_list[k];
        const QSmm* M = a.sm + q;
        const int64_t off = M->tab_off, cap = M->tab_cap;
        T* col = X + (int64_t)M->dblock * d.g.n * d.width + 2 * M->dcol;
        for (int64_t j = threadIdx.x; j < cap; j += blockDim.x) {
            const GEntry e = a.ent[off + j];
            if (e.v < 0) continue;
            col[(int64_t)e.v * d.width] = with_support(ys[off + j], (e.bits & 1u) ? 0x80000000u : 0u);
            col[(int64_t)e.v * d.width + 1] = with_support(yt[off + j], (e.bits & 2u) ? 0x80000000u : 0u);
        }
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
void launch_dense_migrate(bool fp64, const DenseArgs& d, const SmmArgs& a, cudaStream_t st) {
    dense_open_kernel<<<1024, 256, 0, st>>>(d, a.dense_cap);
    if (fp64) dense_migrate_kernel<double><<<256, 256, 0, st>>>(d, a);
    else dense_migrate_kernel<float><<<256, 256, 0, st>>>(d, a);
    note_launches(2);
}

bool dense_width_ok(int width, bool fp64) {
    return fp64 ? (width == 32 || width == 64) : (width == 32 || width == 64 || width == 128);
}

void build_dense_units(int64_t n, const int64_t* row_ptr, std::vector<int4>* units, std::vector<int4>* heavy,
                       int32_t* nslots) {
    units->clear();
    heavy->clear();
    std::vector<int32_t> big;
    for (int64_t v = 0; v < n; ++v)
        if (row_ptr[v + 1] - row_ptr[v] > kHeavyDeg) big.push_back((int32_t)v);
    std::stable_sort(big.begin(), big.end(), [&](int32_t a, int32_t b) {
        return row_ptr[a + 1] - row_ptr[a] > row_ptr[b + 1] - row_ptr[b];
    });
    int32_t slot = 0;
    for (size_t h = 0; h < big.size(); ++h) {
        const int32_t v = big[h];
        const int64_t deg = row_ptr[v + 1] - row_ptr[v];
        const int32_t np = (int32_t)((deg + kPieceEdges - 1) / kPieceEdges);
        heavy->push_back(make_int4(v, slot, np, (int32_t)deg));
        for (int32_t p = 0; p < np; ++p) {
            const int64_t a = row_ptr[v] + (int64_t)p * kPieceEdges;
            const int64_t b = std::min<int64_t>(a + kPieceEdges, row_ptr[v + 1]);
            units->push_back(make_int4(-(int32_t)h - 1, p, (int32_t)(uint32_t)a, (int32_t)(uint32_t)b));
        }
        slot += np;
    }
    int64_t v = 0;
    while (v < n) {
        if (row_ptr[v + 1] - row_ptr[v] > kHeavyDeg) {
            ++v;
            continue;
        }
        const int64_t r0 = v;
        int64_t edges = 0;
        while (v < n && v - r0 < kUnitRows) {
            const int64_t dv = row_ptr[v + 1] - row_ptr[v];
            if (dv > kHeavyDeg || (v > r0 && edges + dv > kUnitEdges)) break;
            edges += dv;
            ++v;
        }
        units->push_back(
            make_int4((int32_t)r0, (int32_t)v, (int32_t)(uint32_t)row_ptr[r0], (int32_t)(uint32_t)row_ptr[v]));
    }
    *nslots = slot;
}

void launch_dense_map(const DenseArgs& d, int64_t nq, cudaStream_t st) {
    const int64_t total = (int64_t)d.nblocks * (d.width / 2);
    dense_map_kernel<<<(int)std::min<int64_t>((total + 255) / 256, 1024), 256, 0, st>>>(d, nq);
    note_launches(1);
}

void launch_dense_init(bool fp64, const DenseArgs& d, cudaStream_t st) {
    const int64_t total = (int64_t)d.nblocks * (d.width / 2);
    const int grid = (int)std::min<int64_t>((total + 255) / 256, 1024);
    if (fp64) dense_init_kernel<double><<<grid, 256, 0, st>>>(d);
    else dense_init_kernel<float><<<grid, 256, 0, st>>>(d);
    note_launches(1);
}

constexpr int kSpmmSmem = 8 * kRingBytes;  // 8 warps per CTA

template <typename T, int VEC>
static void launch_spmm(const DenseArgs& d, cudaStream_t st) {
    dense_spmm_kernel<T, VEC><<<dim3(d.part_warps / 8, d.nblocks), 256, kSpmmSmem, st>>>(d);
}

// Opt the SpMM kernels into their shared-memory rings (current device;
// called before any launch, outside stream capture).
int dense_prepare() {
    cudaError_t e = cudaSuccess;
    auto set = [&](const void* f) {
        if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, kSpmmSmem);
    };
    set((const void*)dense_spmm_kernel<float, 1>);
    set((const void*)dense_spmm_kernel<float, 2>);
    set((const void*)dense_spmm_kernel<float, 4>);
    set((const void*)dense_spmm_kernel<double, 1>);
    set((const void*)dense_spmm_kernel<double, 2>);
    return (int)e;
}

void launch_dense_iteration(bool fp64, const DenseArgs& d, cudaStream_t st) {
    dense_block_flags_kernel<<<1, 256, 0, st>>>(d);
    prof_begin(FAM_DENSE_SPMM, st);
    if (fp64) {
        if (d.width == 64) launch_spmm<double, 2>(d, st);
        else launch_spmm<double, 1>(d, st);
    } else {
        if (d.width == 128) launch_spmm<float, 4>(d, st);
        else if (d.width == 64) launch_spmm<float, 2>(d, st);
        else launch_spmm<float, 1>(d, st);
    }
    prof_end(FAM_DENSE_SPMM, st);
    const int64_t total = (int64_t)d.nblocks * (d.width / 2);
    dense_reduce_kernel<<<(int)((total * 32 + 255) / 256), 256, 0, st>>>(d);
    note_launches(3);
}

}  // namespace geer
