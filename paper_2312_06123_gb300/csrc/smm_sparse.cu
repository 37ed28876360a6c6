// smm_sparse.cu -- SMM phase of GEER (Algorithm 3, lines with SMM steps,
// and Algorithm 2) on sparse frontiers, one CTA per query.
//
// A query keeps s* and t* (Eq. 15: s*(v) = p_i(v,s), t*(v) = p_i(v,t)) as a
// sorted list F of the nodes of V_s u V_t with both values and two support
// bits. One SMM iteration is a sparse matrix times sparse vector product in
// expand-sort-compress form:
//   expand  : every u in F emits (v, rank(u)) for v in N(u)  -- the push
//             cost sum_{u in F} d(u) that Eq. (17) charges to the iteration;
//   sort    : a stable CTA radix sort by v, so the contributions to each v
//             stay in ascending u order, i.e. CSR order of N(v);
//   compress: y(v) = (sum of x(u) over the contributions) / d(v), the
//             support bits OR-ed (V' = N(V), structurally).
// The sum order equals a CSR-order pull over N(v) with the zero terms left
// out, so the FP64 instantiation reproduces (Px)(v) bit for bit; the result
// does not depend on thread scheduling.
// The epilogue of each iteration is fused: the four series terms of
// Algorithm 2 added to r_b in FP64, the support volume of Eq. (17), max_1 and
// max_2 of s* and t*, psi (Eq. 9), eta* (Eq. 8), h(l - l_b) and the switch.
// At the switch the query's lookup table g(v) = s*(v)/d(s) - t*(v)/d(t) is
// built for the AMC walks (Algorithm 1, the Z_k of Eq. 11).
#include "geer_internal.cuh"
#include "geer_kernels.h"

namespace geer {

namespace {

__device__ __forceinline__ int64_t upper_bound_i32(const int32_t* a, int64_t n, int64_t x) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if ((int64_t)a[mid] <= x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

struct SmemSmm {
    int64_t scan[kWarps + 1];
    int hist[256];
    int base[256];
    int wcount[kWarps][256];
    double red_a[kWarps], red_b[kWarps], red_c[kWarps], red_d[kWarps];
    int64_t red_v[kWarps];
    double sval[4];  // s*(s), t*(s), s*(t), t*(t)
    int q;
    int flag;
    int64_t carry;
};

// Stable LSD radix sort of (key, val), N items, 8-bit digits over the low
// `nbits` bits of the keys. Sorts between (k0,v0) and (k1,v1); returns 0 if
// the result is in (k0,v0), 1 otherwise.
__device__ int cta_radix_sort(int32_t* k0, int32_t* v0, int32_t* k1, int32_t* v1, int64_t N, int nbits,
                              SmemSmm& sm) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int cur = 0;
    for (int i = tid; i < kWarps * 256; i += kCta) (&sm.wcount[0][0])[i] = 0;
    for (int shift = 0; shift < nbits; shift += 8) {
        const int32_t* ki = cur ? k1 : k0;
        const int32_t* vi = cur ? v1 : v0;
        int32_t* ko = cur ? k0 : k1;
        int32_t* vo = cur ? v0 : v1;
        for (int i = tid; i < 256; i += kCta) sm.hist[i] = 0;
        __syncthreads();
        for (int64_t i = tid; i < N; i += kCta) atomicAdd(&sm.hist[(ki[i] >> shift) & 255], 1);
        __syncthreads();
        {
            int64_t tot;
            int64_t x = sm.hist[tid];  // kCta == 256 digits
            int64_t ex = cta_excl_scan(x, sm.scan, &tot);
            sm.base[tid] = (int)ex;
        }
        __syncthreads();
        for (int64_t tile = 0; tile < N; tile += kCta) {
            const int64_t i = tile + tid;
            const bool valid = i < N;
            const int32_t key = valid ? ki[i] : 0;
            const int32_t val = valid ? vi[i] : 0;
            const int d = valid ? ((key >> shift) & 255) : 256;
            const unsigned peers = __match_any_sync(0xffffffffu, d);
            const int rank = __popc(peers & lanemask_lt());
            if (valid && rank == 0) sm.wcount[warp][d] = __popc(peers);
            __syncthreads();
            if (valid) {
                int off = sm.base[d] + rank;
                for (int w = 0; w < warp; ++w) off += sm.wcount[w][d];
                ko[off] = key;
                vo[off] = val;
            }
            __syncthreads();
            {
                int acc = 0;
                for (int w = 0; w < kWarps; ++w) {
                    acc += sm.wcount[w][tid];
                    sm.wcount[w][tid] = 0;
                }
                sm.base[tid] += acc;
            }
            __syncthreads();
        }
        cur ^= 1;
    }
    return cur;
}

// psi (Eq. 9), eta0 = max(1, ceil(eta*/2^(tau-1))) with eta* from Eq. (8),
// h = (2^tau - 1) eta0. Same expression order as the definitions.
__device__ void switch_quantities(int64_t lf, double s1, double s2, double t1, double t2, double ds,
                                  double dt, double eps, double delta, int tau, double* psi,
                                  int64_t* eta0, double* h) {
    double up = (double)((lf + 1) / 2), dn = (double)(lf / 2);
    double p = 2.0 * up * (s1 / ds + t1 / dt) + 2.0 * dn * (s2 / ds + t2 / dt);
    double es = 2.0 * p * p * log(2.0 * (double)tau / delta) / (eps * eps);
    int64_t e0 = (int64_t)ceil(es / ldexp(1.0, tau - 1));
    if (e0 < 1) e0 = 1;
    *psi = p;
    *eta0 = e0;
    *h = (double)((((int64_t)1 << tau) - 1) * e0);
}

}  // namespace

template <typename T>
__global__ void __launch_bounds__(kCta) smm_sparse_kernel(SmmArgs a) {
    __shared__ SmemSmm sm;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t P = a.cap;
    const int64_t F = a.cap + 2;
    // per-slot scratch
    int32_t* base_i = a.scr_i32 + (size_t)blockIdx.x * (size_t)(5 * P + 3 * F + 2);
    int32_t* pk0 = base_i;
    int32_t* pv0 = pk0 + P;
    int32_t* pk1 = pv0 + P;
    int32_t* pv1 = pk1 + P;
    int32_t* fk[2] = {pv1 + P, pv1 + P + F};
    int32_t* pre = fk[1] + F;       // F + 1
    int32_t* seg = pre + F + 1;     // P + 1
    T* base_v = reinterpret_cast<T*>(a.scr_val) + (size_t)blockIdx.x * (size_t)(4 * F);
    T* fxs[2] = {base_v, base_v + 2 * F};
    T* fxt[2] = {base_v + F, base_v + 3 * F};
    uint8_t* fb[2] = {a.scr_bits + (size_t)blockIdx.x * (size_t)(2 * F),
                      a.scr_bits + (size_t)blockIdx.x * (size_t)(2 * F) + F};
    const int64_t* row_ptr = a.g.row_ptr;
    const int32_t* col_idx = a.g.col_idx;
    const int64_t n = a.g.n;

    for (;;) {
        if (tid == 0) sm.q = atomicAdd(a.work_counter, 1);
        __syncthreads();
        const int q = sm.q;
        __syncthreads();
        if (q >= a.nq) break;
        QState* Q = a.st + q;
        const int32_t s = a.s[q], t = a.t[q];
        const double eps = a.eps ? a.eps[q] : a.eps_scalar;
        if (tid == 0) {
            Q->s = s; Q->t = t; Q->eps = eps; Q->qidx = a.q_index_base + q;
            Q->batch = 0; Q->err = 0; Q->r_b = 0; Q->r_f = 0; Q->r = 0; Q->psi = 0;
            Q->volume = 0; Q->h = 0; Q->f_last = 0; Q->eta0 = 0; Q->eta = 0; Q->walks = 0;
            Q->walk_steps = 0; Q->checksum = 0; Q->ppc = 0; Q->nchunks = 0; Q->table_off = 0;
            Q->table_mask = -1; Q->front = 0; Q->ell = 0; Q->ell_b = 0; Q->lf = 0; Q->ds = 0; Q->dt = 0;
        }
        if (s < 0 || s >= n || t < 0 || t >= n || !(eps > 0.0)) {
            if (tid == 0) {
                Q->status = ST_ERROR;
                Q->err = DERR_NODE_RANGE;
                atomicCAS(a.err_flag, 0, DERR_NODE_RANGE);
            }
            __syncthreads();
            continue;
        }
        if (s == t) {  // r(s,s) = 0 (Definition 1)
            if (tid == 0) Q->status = ST_DONE;
            __syncthreads();
            continue;
        }
        const double ds = (double)(row_ptr[s + 1] - row_ptr[s]);
        const double dt = (double)(row_ptr[t + 1] - row_ptr[t]);
        // truncation length: Eq. (6) (refined) or Eq. (5) (Peng et al.)
        int64_t ell;
        {
            const double lam = a.lambda;
            if (!(lam < 1.0)) ell = -1;
            else if (lam <= 0.0) ell = 0;
            else {
                double v = a.ell_formula == 1
                               ? ceil(log(4.0 / (eps - eps * lam)) / log(1.0 / lam) - 1.0)
                               : ceil(log((2.0 / ds + 2.0 / dt) / (eps * (1.0 - lam))) / log(1.0 / lam) - 1.0);
                ell = v < 0.0 ? 0 : (int64_t)v;
            }
        }
        if (ell < 0) {
            if (tid == 0) {
                Q->status = ST_ERROR;
                Q->err = DERR_ELL;
                atomicCAS(a.err_flag, 0, DERR_ELL);
            }
            __syncthreads();
            continue;
        }
        int64_t lb_target;  // SMM iterations wanted by the policy (-1: rule)
        if (a.policy == 2) {
            lb_target = a.fixed_lb < 0 ? ell : (a.fixed_lb < ell ? a.fixed_lb : ell);
        } else {
            lb_target = -1;
        }
        // F_0 = {s, t}, s* = e_s, t* = e_t (Algorithm 3 initialisation)
        int cur = 0;
        int64_t nf = 2;
        if (tid == 0) {
            const int lo = s < t ? s : t, hi = s < t ? t : s;
            fk[0][0] = lo; fk[0][1] = hi;
            fxs[0][0] = (lo == s) ? T(1) : T(0); fxt[0][0] = (lo == t) ? T(1) : T(0);
            fxs[0][1] = (hi == s) ? T(1) : T(0); fxt[0][1] = (hi == t) ? T(1) : T(0);
            fb[0][0] = (lo == s) ? 1 : 2;
            fb[0][1] = (hi == s) ? 1 : 2;
        }
        // the zeroth term of r_b: s*(s)/d(s) + t*(t)/d(t) - s*(t)/d(s) - t*(s)/d(t)
        double rb = 1.0 / ds + 1.0 / dt - 0.0 / ds - 0.0 / dt;
        int64_t lb = 0;
        double vol = ds + dt;
        double s1 = 1.0, s2 = 0.0, t1 = 1.0, t2 = 0.0;  // max_1, max_2 of e_s and e_t
        bool run = lb_target >= 0 ? (lb_target > 0) : (ell >= 1);
        bool failed = false;
        double psi = 0.0, h = 0.0;
        int64_t eta0 = 0;
        __syncthreads();
        while (run) {
            // ---- expand: degree prefix over F, then one (v, rank(u)) pair per edge
            if (tid == 0) sm.carry = 0;
            __syncthreads();
            for (int64_t tile = 0; tile < nf; tile += kCta) {
                const int64_t i = tile + tid;
                int64_t d = 0;
                if (i < nf) {
                    const int32_t u = fk[cur][i];
                    d = row_ptr[u + 1] - row_ptr[u];
                }
                int64_t tot;
                const int64_t ex = cta_excl_scan(d, sm.scan, &tot);
                if (i < nf) {
                    const int64_t pv = sm.carry + ex;
                    pre[i] = (int32_t)(pv < 0x7fffffff ? pv : 0x7fffffff);
                }
                __syncthreads();
                if (tid == 0) sm.carry += tot;
                __syncthreads();
            }
            const int64_t npairs = sm.carry;
            if (npairs > P) {
                failed = true;
                break;
            }
            if (tid == 0) pre[nf] = (int32_t)npairs;
            __syncthreads();
            for (int64_t p = tid; p < npairs; p += kCta) {
                const int64_t r = upper_bound_i32(pre, nf + 1, p) - 1;
                const int32_t u = fk[cur][r];
                pk0[p] = col_idx[row_ptr[u] + (p - pre[r])];
                pv0[p] = (int32_t)r;
            }
            __syncthreads();
            // ---- sort by v (stable)
            const int rbuf = cta_radix_sort(pk0, pv0, pk1, pv1, npairs, a.nbits, sm);
            const int32_t* kr = rbuf ? pk1 : pk0;
            const int32_t* vr = rbuf ? pv1 : pv0;
            int32_t* spare = rbuf ? pk0 : pk1;  // free for the head scan
            // ---- segment heads
            if (tid == 0) sm.carry = 0;
            __syncthreads();
            for (int64_t tile = 0; tile < npairs; tile += kCta) {
                const int64_t i = tile + tid;
                const int64_t head = (i < npairs && (i == 0 || kr[i] != kr[i - 1])) ? 1 : 0;
                int64_t tot;
                const int64_t ex = cta_excl_scan(head, sm.scan, &tot);
                if (head) seg[sm.carry + ex] = (int32_t)i;
                __syncthreads();
                if (tid == 0) sm.carry += tot;
                __syncthreads();
            }
            (void)spare;
            const int64_t nseg = sm.carry;
            if (tid == 0) {
                seg[nseg] = (int32_t)npairs;
                sm.sval[0] = sm.sval[1] = sm.sval[2] = sm.sval[3] = 0.0;
            }
            __syncthreads();
            // ---- compress: y(v) = sum x(u) / d(v); epilogue contributions
            const int nxt = cur ^ 1;
            int64_t my_vol = 0;
            double as = -INFINITY, bs = -INFINITY, at = -INFINITY, bt = -INFINITY;
            auto finish = [&](int64_t j, int32_t v, T ys, T yt, uint8_t bits) {
                const int64_t dv = row_ptr[v + 1] - row_ptr[v];
                ys = ys / (T)dv;
                yt = yt / (T)dv;
                fk[nxt][j] = v;
                fxs[nxt][j] = ys;
                fxt[nxt][j] = yt;
                fb[nxt][j] = bits;
                my_vol += dv * (int64_t)((bits & 1) + ((bits >> 1) & 1));
                top2_merge(as, bs, (double)ys, -INFINITY);
                top2_merge(at, bt, (double)yt, -INFINITY);
                if (v == s) { sm.sval[0] = (double)ys; sm.sval[1] = (double)yt; }
                if (v == t) { sm.sval[2] = (double)ys; sm.sval[3] = (double)yt; }
            };
            // short segments: one thread each, sequential in CSR order
            for (int64_t j = tid; j < nseg; j += kCta) {
                const int32_t b0 = seg[j], e0 = seg[j + 1];
                if (e0 - b0 > 32) continue;
                T ys = T(0), yt = T(0);
                uint8_t bits = 0;
                for (int32_t p = b0; p < e0; ++p) {
                    const int32_t r = vr[p];
                    ys += fxs[cur][r];
                    yt += fxt[cur][r];
                    bits |= fb[cur][r];
                }
                finish(j, kr[b0], ys, yt, bits);
            }
            // long segments: one warp each, lane-strided then a fixed xor tree
            for (int64_t base = (int64_t)warp * 32; base < nseg; base += (int64_t)kWarps * 32) {
                const int64_t j = base + lane;
                const bool lng = j < nseg && (seg[j + 1] - seg[j]) > 32;
                unsigned mask = __ballot_sync(0xffffffffu, lng);
                while (mask) {
                    const int l = __ffs(mask) - 1;
                    mask &= mask - 1;
                    const int64_t jj = base + l;
                    const int32_t b0 = seg[jj], e0 = seg[jj + 1];
                    T ys = T(0), yt = T(0);
                    unsigned bits = 0;
                    for (int32_t p = b0 + lane; p < e0; p += 32) {
                        const int32_t r = vr[p];
                        ys += fxs[cur][r];
                        yt += fxt[cur][r];
                        bits |= fb[cur][r];
                    }
                    ys = warp_sum(ys);
                    yt = warp_sum(yt);
                    bits = __reduce_or_sync(0xffffffffu, bits);
                    if (lane == 0) finish(jj, kr[b0], ys, yt, (uint8_t)bits);
                }
            }
            // ---- CTA reductions: volume and top-2 of s*, t*
            {
                int64_t v = my_vol;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                warp_top2(as, bs);
                warp_top2(at, bt);
                if (lane == 0) {
                    sm.red_v[warp] = v;
                    sm.red_a[warp] = as; sm.red_b[warp] = bs;
                    sm.red_c[warp] = at; sm.red_d[warp] = bt;
                }
                __syncthreads();
                if (tid == 0) {
                    int64_t tv = 0;
                    double A = -INFINITY, B = -INFINITY, C = -INFINITY, D = -INFINITY;
                    for (int w = 0; w < kWarps; ++w) {
                        tv += sm.red_v[w];
                        top2_merge(A, B, sm.red_a[w], sm.red_b[w]);
                        top2_merge(C, D, sm.red_c[w], sm.red_d[w]);
                    }
                    sm.red_v[0] = tv;
                    sm.red_a[0] = A; sm.red_b[0] = B; sm.red_c[0] = C; sm.red_d[0] = D;
                }
                __syncthreads();
            }
            vol = (double)sm.red_v[0];
            s1 = sm.red_a[0]; s2 = sm.red_b[0]; t1 = sm.red_c[0]; t2 = sm.red_d[0];
            // entries outside F are zero: they join the multisets when F < n
            if (nseg < n) {
                s1 = fmax(s1, 0.0); s2 = fmax(s2, 0.0); t1 = fmax(t1, 0.0); t2 = fmax(t2, 0.0);
            }
            rb += sm.sval[0] / ds + sm.sval[3] / dt - sm.sval[2] / ds - sm.sval[1] / dt;
            lb += 1;
            nf = nseg;
            cur = nxt;
            const int64_t lf = ell - lb;
            psi = 0.0; h = 0.0; eta0 = 0;
            if (lf > 0) switch_quantities(lf, s1, s2, t1, t2, ds, dt, eps, a.delta, a.tau, &psi, &eta0, &h);
            // Eq. (17), or the iteration target of a fixed policy
            const bool free_stop = (vol > h) || (lb >= ell);
            run = lb_target >= 0 ? (lb < lb_target) : !free_stop;
            __syncthreads();
        }
        if (failed) {
            if (tid == 0) {
                Q->status = ST_ERROR;
                Q->err = DERR_CAPACITY;
                Q->ell = (int32_t)ell;
                Q->ell_b = (int32_t)lb;
                atomicCAS(a.err_flag, 0, DERR_CAPACITY);
            }
            __syncthreads();
            continue;
        }
        const int64_t lf = ell - lb;
        if (lb == 0 && lf > 0)
            switch_quantities(lf, s1, s2, t1, t2, ds, dt, eps, a.delta, a.tau, &psi, &eta0, &h);
        // ---- lookup table of g(v) = s*(v)/d(s) - t*(v)/d(t) for the walks
        if (lf > 0) {
            if (tid == 0) {
                int64_t cap = 16;
                while (cap < 2 * nf) cap <<= 1;
                const unsigned long long off = atomicAdd(a.pool_used, (unsigned long long)cap);
                sm.carry = (off + (unsigned long long)cap <= (unsigned long long)a.pool_cap) ? (int64_t)off : -1;
                sm.flag = (int)(cap - 1);
            }
            __syncthreads();
            const int64_t off = sm.carry;
            const int32_t mask = sm.flag;
            if (off < 0) {
                if (tid == 0) {
                    Q->status = ST_ERROR;
                    Q->err = DERR_TABLE;
                    atomicCAS(a.err_flag, 0, DERR_TABLE);
                }
                __syncthreads();
                continue;
            }
            GEntry* tab = a.pool + off;
            for (int64_t i = tid; i <= mask; i += kCta) tab[i].v = -1;
            __syncthreads();
            for (int64_t i = tid; i < nf; i += kCta) {
                const double g = (double)fxs[cur][i] / ds - (double)fxt[cur][i] / dt;
                if (g == 0.0) continue;  // absent entries read as 0
                const int32_t v = fk[cur][i];
                uint32_t hsh = hash32((uint32_t)v) & (uint32_t)mask;
                for (;;) {
                    const int32_t prev = atomicCAS(&tab[hsh].v, -1, v);
                    if (prev == -1) {
                        tab[hsh].g = g;
                        break;
                    }
                    hsh = (hsh + 1) & (uint32_t)mask;
                }
            }
            if (tid == 0) {
                Q->table_off = off;
                Q->table_mask = mask;
            }
        }
        if (tid == 0) {
            Q->ds = (int32_t)ds;
            Q->dt = (int32_t)dt;
            Q->ell = (int32_t)ell;
            Q->ell_b = (int32_t)lb;
            Q->lf = (int32_t)lf;
            Q->r_b = rb;
            Q->psi = psi;
            Q->volume = vol;
            Q->h = h;
            Q->eta0 = eta0;
            Q->eta = eta0;
            Q->front = (int32_t)nf;
            if (lf > 0) {
                Q->status = ST_AMC;
            } else {
                Q->status = ST_DONE;
                Q->r = rb;
            }
        }
        __syncthreads();
    }
}

void launch_smm_sparse(bool fp64, const SmmArgs& a, int grid, cudaStream_t st) {
    prof_begin(FAM_SMM_SPARSE, st);
    if (fp64) smm_sparse_kernel<double><<<grid, kCta, 0, st>>>(a);
    else smm_sparse_kernel<float><<<grid, kCta, 0, st>>>(a);
    prof_end(FAM_SMM_SPARSE, st);
}

}  // namespace geer
