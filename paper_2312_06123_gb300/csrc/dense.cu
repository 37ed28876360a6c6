// dense.cu -- the SMM iteration of GEER (Algorithm 2 inside Algorithm 3) as
// a dense pull SpMM over blocks of query vectors, for queries whose
// frontiers cover much of the graph (deep SMM: small eps, low degrees, or a
// fixed l_b such as the standalone SMM of Section 4.1.1).
//
// A dense block holds B = LPR * VEC columns, the (s*, t*) pairs of B/2
// queries, row-major: X[v * B + c], double-buffered across iterations, and
// one support bit per column and row (Eq. 17's V_s, V_t, kept
// structurally). Per row v of the graph, LPR lanes each own VEC columns:
//   y(v, c) = (sum over u in N(v), in CSR order, of x(u, c)) / d(v),
//   support(v, c) = OR over u in N(v) of support(u, c),
// so each column's sum is sequential in CSR order, as in the oracle's pull.
// Columns of queries that left SMM keep their last values (the walks read
// them). The epilogue is fused: per query, Eq. 17's volume, the next
// push volume, |V|, max_1/max_2 of s* and t* (per-warp partials merged in a
// fixed order) and the values at s and t for the series terms.
#include "geer_internal.cuh"
#include "geer_kernels.h"

namespace geer {

namespace {

template <typename T> struct Vec;
template <> struct Vec<float> {
    using type = float4;
    static constexpr int n = 4;
};
template <> struct Vec<double> {
    using type = double2;
    static constexpr int n = 2;
};

template <typename T>
__device__ __forceinline__ void vadd(typename Vec<T>::type& a, const typename Vec<T>::type& b);
template <>
__device__ __forceinline__ void vadd<float>(float4& a, const float4& b) {
    a.x += b.x; a.y += b.y; a.z += b.z; a.w += b.w;
}
template <>
__device__ __forceinline__ void vadd<double>(double2& a, const double2& b) {
    a.x += b.x; a.y += b.y;
}

template <typename T>
__device__ __forceinline__ T vget(const typename Vec<T>::type& a, int i);
template <>
__device__ __forceinline__ float vget<float>(const float4& a, int i) {
    return i == 0 ? a.x : (i == 1 ? a.y : (i == 2 ? a.z : a.w));
}
template <>
__device__ __forceinline__ double vget<double>(const double2& a, int i) {
    return i == 0 ? a.x : a.y;
}

__device__ __forceinline__ void top2_push(double& a, double& b, double v) {
    if (v > a) {
        b = a;
        a = v;
    } else if (v > b) {
        b = v;
    }
}

}  // namespace

// Iteration 0 of the dense queries: columns e_s, e_t in buffer 0 and the
// per-query sums of the initial frontier {s, t}.
template <typename T>
__global__ void dense_init_kernel(DenseArgs d) {
    const int nq_block = d.width / 2;
    const int64_t total = (int64_t)d.nblocks * nq_block;
    T* X0 = reinterpret_cast<T*>(d.X[0]);
    uint32_t* S0 = d.S[0];
    const int words = d.width >= 32 ? d.width / 32 : 1;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(k / nq_block), j = (int)(k % nq_block);
        const int q = d.block_q[k];
        if (q < 0) continue;
        const QState* Q = d.st + q;
        QSmm* M = d.sm + q;
        if (Q->status != ST_SMM) continue;
        const int64_t base = (int64_t)b * d.g.n;
        const int cs = 2 * j, ct = 2 * j + 1;
        X0[(base + Q->s) * d.width + cs] = T(1);
        X0[(base + Q->t) * d.width + ct] = T(1);
        atomicOr(&S0[(base + Q->s) * words + cs / 32], 1u << (cs % 32));
        atomicOr(&S0[(base + Q->t) * words + ct / 32], 1u << (ct % 32));
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
// grid.y = dense block; LPR lanes per row, 32/LPR rows per warp.
template <typename T, int LPR>
__global__ void __launch_bounds__(256) dense_spmm_kernel(DenseArgs d) {
    using V = typename Vec<T>::type;
    constexpr int VEC = Vec<T>::n;
    constexpr int B = LPR * VEC;
    constexpr int RPW = 32 / LPR;  // rows per warp
    const int blk = blockIdx.y;
    if (!d.block_run[blk]) return;
    const int iter = d.ctl->iter;
    const T* Xc = reinterpret_cast<const T*>(d.X[(iter & 1) ^ 1]);
    T* Xn = reinterpret_cast<T*>(d.X[iter & 1]);
    const uint32_t* Sc = d.S[(iter & 1) ^ 1];
    uint32_t* Sn = d.S[iter & 1];
    constexpr int WORDS = B >= 32 ? B / 32 : 1;
    const int lane = threadIdx.x & 31;
    const int sub = lane % LPR;       // column group of this lane
    const int rsub = lane / LPR;      // row of this lane within the warp's rows
    const unsigned gmask = LPR == 32 ? 0xffffffffu : (((1u << LPR) - 1) << (rsub * LPR));
    const int64_t n = d.g.n;
    const int64_t boff = (int64_t)blk * n;
    // the queries of this lane's columns: VEC/2 per lane
    constexpr int QPL = VEC / 2;
    int qs[QPL];
    bool act[QPL];
    int32_t s_node[QPL], t_node[QPL];
#pragma unroll
    for (int i = 0; i < QPL; ++i) {
        const int j = sub * QPL + i;
        qs[i] = d.block_q[blk * (B / 2) + j];
        act[i] = qs[i] >= 0 && d.sm[qs[i]].run && d.sm[qs[i]].dense;
        s_node[i] = act[i] ? d.st[qs[i]].s : -1;
        t_node[i] = act[i] ? d.st[qs[i]].t : -1;
    }
    // per-lane epilogue accumulators
    unsigned long long vp[QPL], vu[QPL], cnt[QPL];
    double a1[QPL], a2[QPL], b1[QPL], b2[QPL];
#pragma unroll
    for (int i = 0; i < QPL; ++i) {
        vp[i] = vu[i] = cnt[i] = 0;
        a1[i] = a2[i] = b1[i] = b2[i] = 0.0;  // entries are >= 0; zeros are in the multiset
    }
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r0 = warp * RPW; r0 < n; r0 += nwarps * RPW) {
        const int64_t v = r0 + rsub;
        const bool row_ok = v < n;
        int64_t start = 0;
        uint32_t deg = 0;
        if (row_ok) {
            if (d.g.node_info) {
                const uint2 inf = __ldg(d.g.node_info + v);
                start = inf.x;
                deg = inf.y;
            } else {
                start = __ldg(d.g.row_ptr + v);
                deg = (uint32_t)(__ldg(d.g.row_ptr + v + 1) - start);
            }
        }
        V acc;
        if constexpr (VEC == 4) acc = make_float4(0.f, 0.f, 0.f, 0.f);
        else acc = make_double2(0.0, 0.0);
        uint32_t nib = 0;
        // the rows of a warp may differ in degree: loop to the warp's largest
        uint32_t dmax = deg;
#pragma unroll
        for (int o = LPR; o < 32; o <<= 1) dmax = max(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
        for (uint32_t base = 0; base < dmax; base += LPR) {
            const uint32_t e = base + sub;
            const int32_t u_l = (row_ok && e < deg) ? __ldg(d.g.col_idx + start + e) : -1;
            const uint32_t lim = deg > base ? min((uint32_t)LPR, deg - base) : 0u;
#pragma unroll 4
            for (uint32_t k = 0; k < (uint32_t)LPR; ++k) {
                const int32_t u = __shfl_sync(0xffffffffu, u_l, (int)k, LPR);
                if (k < lim) {
                    const int64_t ru = boff + u;
                    vadd<T>(acc, __ldg(reinterpret_cast<const V*>(Xc + ru * B) + sub));
                    const uint32_t wd = __ldg(Sc + ru * WORDS + (sub * VEC) / 32);
                    nib |= (wd >> ((sub * VEC) % 32)) & ((1u << VEC) - 1);
                }
            }
        }
        if (row_ok) {
            const T dv = (T)deg;
            V y;
            if constexpr (VEC == 4) y = make_float4(acc.x / dv, acc.y / dv, acc.z / dv, acc.w / dv);
            else y = make_double2(acc.x / dv, acc.y / dv);
            const int64_t rv = boff + v;
            V* dst = reinterpret_cast<V*>(Xn + rv * B) + sub;
            // keep the frozen columns of queries that left SMM
            bool all_act = true;
#pragma unroll
            for (int i = 0; i < QPL; ++i) all_act &= act[i];
            if (all_act) {
                *dst = y;
            } else {
#pragma unroll
                for (int i = 0; i < QPL; ++i)
                    if (act[i]) {
                        T* p = Xn + rv * B + sub * VEC + 2 * i;
                        p[0] = vget<T>(y, 2 * i);
                        p[1] = vget<T>(y, 2 * i + 1);
                    }
            }
#pragma unroll
            for (int i = 0; i < QPL; ++i) {
                if (!act[i]) continue;
                const uint32_t bs = (nib >> (2 * i)) & 1u, bt = (nib >> (2 * i + 1)) & 1u;
                const double ys = (double)vget<T>(y, 2 * i), yt = (double)vget<T>(y, 2 * i + 1);
                vp[i] += (unsigned long long)deg * (bs + bt);
                vu[i] += (unsigned long long)deg * (bs | bt);
                cnt[i] += (bs | bt);
                top2_push(a1[i], a2[i], ys);
                top2_push(b1[i], b2[i], yt);
                if (v == s_node[i]) {
                    d.sm[qs[i]].sval[0] = ys;
                    d.sm[qs[i]].sval[1] = yt;
                }
                if (v == t_node[i]) {
                    d.sm[qs[i]].sval[2] = ys;
                    d.sm[qs[i]].sval[3] = yt;
                }
            }
        }
        // support word(s) of the row: OR the lanes' nibbles
        uint32_t wv = row_ok ? (nib << ((sub * VEC) % 32)) : 0u;
        constexpr int LPW = 32 / VEC;  // lanes per support word
#pragma unroll
        for (int o = 1; o < LPW && o < LPR; o <<= 1) wv |= __shfl_xor_sync(0xffffffffu, wv, o);
        if (row_ok && (sub % LPW) == 0) Sn[(boff + v) * WORDS + (sub * VEC) / 32] = wv;
    }
    // merge the row groups of the warp, then one partial per warp and query
#pragma unroll
    for (int i = 0; i < QPL; ++i) {
#pragma unroll
        for (int o = LPR; o < 32; o <<= 1) {
            vp[i] += __shfl_xor_sync(0xffffffffu, vp[i], o);
            vu[i] += __shfl_xor_sync(0xffffffffu, vu[i], o);
            cnt[i] += __shfl_xor_sync(0xffffffffu, cnt[i], o);
            top2_merge(a1[i], a2[i], __shfl_xor_sync(0xffffffffu, a1[i], o), __shfl_xor_sync(0xffffffffu, a2[i], o));
            top2_merge(b1[i], b2[i], __shfl_xor_sync(0xffffffffu, b1[i], o), __shfl_xor_sync(0xffffffffu, b2[i], o));
        }
    }
    (void)gmask;
    if (rsub == 0) {
#pragma unroll
        for (int i = 0; i < QPL; ++i) {
            const int j = sub * QPL + i;
            DensePartial* p = d.part + ((int64_t)blk * d.part_warps + warp) * (B / 2) + j;
            p->vp = vp[i];
            p->vu = vu[i];
            p->cnt = cnt[i];
            p->s1 = a1[i];
            p->s2 = a2[i];
            p->t1 = b1[i];
            p->t2 = b2[i];
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
        vp += __shfl_xor_sync(0xffffffffu, vp, o);
        vu += __shfl_xor_sync(0xffffffffu, vu, o);
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        top2_merge(a1, a2, __shfl_xor_sync(0xffffffffu, a1, o), __shfl_xor_sync(0xffffffffu, a2, o));
        top2_merge(b1, b2, __shfl_xor_sync(0xffffffffu, b1, o), __shfl_xor_sync(0xffffffffu, b2, o));
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

// Blocks with at least one query still in SMM.
__global__ void dense_block_flags_kernel(DenseArgs d) {
    const int nq_block = d.width / 2;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < d.nblocks; b += gridDim.x * blockDim.x) {
        int any = 0;
        for (int j = 0; j < nq_block; ++j) {
            const int q = d.block_q[b * nq_block + j];
            if (q >= 0 && d.sm[q].run && d.sm[q].dense) any = 1;
        }
        d.block_run[b] = any;
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
int dense_lanes_per_row(int width, bool fp64) { return width / (fp64 ? 2 : 4); }

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

void launch_dense_iteration(bool fp64, const DenseArgs& d, cudaStream_t st) {
    dense_block_flags_kernel<<<1, 256, 0, st>>>(d);
    const dim3 grid(d.part_warps / 8, d.nblocks);
    prof_begin(FAM_DENSE_SPMM, st);
    const int lpr = dense_lanes_per_row(d.width, fp64);
    if (fp64) {
        if (lpr == 32) dense_spmm_kernel<double, 32><<<grid, 256, 0, st>>>(d);
        else if (lpr == 16) dense_spmm_kernel<double, 16><<<grid, 256, 0, st>>>(d);
        else dense_spmm_kernel<double, 8><<<grid, 256, 0, st>>>(d);
    } else {
        if (lpr == 32) dense_spmm_kernel<float, 32><<<grid, 256, 0, st>>>(d);
        else if (lpr == 16) dense_spmm_kernel<float, 16><<<grid, 256, 0, st>>>(d);
        else dense_spmm_kernel<float, 8><<<grid, 256, 0, st>>>(d);
    }
    prof_end(FAM_DENSE_SPMM, st);
    const int64_t total = (int64_t)d.nblocks * (d.width / 2);
    dense_reduce_kernel<<<(int)((total * 32 + 255) / 256), 256, 0, st>>>(d);
    note_launches(3);
}

}  // namespace geer
