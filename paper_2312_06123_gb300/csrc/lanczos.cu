// lanczos.cu -- the spectral bound lambda = max(|lambda_2|, |lambda_n|) of
// P = D^-1 A (Section 3.1), the once-per-graph preprocessing that Eq. (6)
// needs. P is similar to N = D^-1/2 A D^-1/2, whose top eigenvector is
// phi(v) = sqrt(d(v)/2m) with eigenvalue 1. Lanczos runs on N restricted to
// the complement of phi, with full re-orthogonalisation (classical
// Gram-Schmidt applied twice), in FP64; lambda_2 and lambda_n are the
// extreme eigenvalues of the tridiagonal matrix, found by Sturm-sequence
// bisection. Every reduction has a fixed shape, so the result does not
// depend on scheduling.
#include <algorithm>
#include <cmath>
#include <vector>

#include "geer_internal.cuh"
#include "geer_kernels.h"

namespace geer {

namespace {

constexpr int kLzCtas = 304;  // partial-sum CTAs (2 per SM of a GB300)

__global__ void lz_init_kernel(DevGraph g, double* isd, double* phi, double* q0) {
    const double two_m = (double)g.nnz;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < g.n; v += (int64_t)gridDim.x * blockDim.x) {
        const double d = (double)(g.row_ptr[v + 1] - g.row_ptr[v]);
        isd[v] = 1.0 / sqrt(d);
        phi[v] = sqrt(d / two_m);
        // deterministic start vector with entries in [-0.5, 0.5)
        uint64_t z = mix64(0xD1B54A32D192ED03ull * (uint64_t)(v + 1));
        q0[v] = (double)(z >> 11) * (1.0 / 9007199254740992.0) - 0.5;
    }
}

// w = N x, one warp per row (rows of degree <= heavy cut)
__global__ void lz_spmv_kernel(DevGraph g, const double* isd, const double* x, double* w) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < g.n; v += nw) {
        const int64_t b = g.row_ptr[v], e = g.row_ptr[v + 1];
        double acc = 0.0;
        for (int64_t p = b + lane; p < e; p += 32) {
            const int32_t u = g.col_idx[p];
            acc += x[u] * isd[u];
        }
        acc = warp_sum(acc);
        if (lane == 0) w[v] = acc * isd[v];
    }
}

// partial dot products of vectors vec[0..m) with y, one slot per CTA:
// part[i * gridDim.x + cta]
__global__ void __launch_bounds__(kCta) lz_dots_kernel(const double* const* vec, int m, const double* y, int64_t n,
                                                      double* part) {
    __shared__ double red[kWarps];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
    const int64_t lo = blockIdx.x * chunk, hi = min(n, lo + chunk);
    for (int i = 0; i < m; ++i) {
        const double* x = vec[i];
        double acc = 0.0;
        for (int64_t v = lo + tid; v < hi; v += kCta) acc += x[v] * y[v];
        acc = warp_sum(acc);
        if (lane == 0) red[warp] = acc;
        __syncthreads();
        if (tid == 0) {
            double s = 0.0;
            for (int w = 0; w < kWarps; ++w) s += red[w];
            part[(int64_t)i * gridDim.x + blockIdx.x] = s;
        }
        __syncthreads();
    }
}

// out[i] = sum over CTAs of part[i * nparts + c], fixed order; one CTA per i
__global__ void __launch_bounds__(kCta) lz_dots_final_kernel(const double* part, int nparts, double* out) {
    __shared__ double red[kWarps];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double acc = 0.0;
    for (int c = tid; c < nparts; c += kCta) acc += part[(int64_t)blockIdx.x * nparts + c];
    acc = warp_sum(acc);
    if (lane == 0) red[warp] = acc;
    __syncthreads();
    if (tid == 0) {
        double s = 0.0;
        for (int w = 0; w < kWarps; ++w) s += red[w];
        out[blockIdx.x] = s;
    }
}

// y -= sum_i coef[i] vec[i]
__global__ void lz_subtract_kernel(const double* const* vec, int m, const double* coef, double* y, int64_t n) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        double acc = y[v];
        for (int i = 0; i < m; ++i) acc -= coef[i] * vec[i][v];
        y[v] = acc;
    }
}

__global__ void lz_scale_kernel(const double* x, const double* nrm2, double* y, int64_t n) {
    const double inv = 1.0 / sqrt(*nrm2);
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        y[v] = x[v] * inv;
}

// b2: squared off-diagonal entries
__device__ int64_t sturm_count(int64_t k, const double* a, const double* b2, double x) {
    int64_t cnt = 0;
    double q = a[0] - x;
    if (q < 0.0) ++cnt;
    for (int64_t i = 1; i < k; ++i) {
        const double qq = (q == 0.0) ? 1e-300 : q;
        q = (a[i] - x) - b2[i - 1] / qq;
        if (q < 0.0) ++cnt;
    }
    return cnt;
}

// thread 0: largest eigenvalue, thread 1: smallest, of the k x k tridiagonal
// matrix with diagonal a and squared off-diagonal b2
__global__ void lz_ritz_kernel(int64_t k, const double* a, const double* b2, double* out) {
    const int which = threadIdx.x;
    if (which > 1) return;
    double lo = INFINITY, hi = -INFINITY;
    for (int64_t i = 0; i < k; ++i) {
        const double r = (i > 0 ? sqrt(b2[i - 1]) : 0.0) + (i + 1 < k ? sqrt(b2[i]) : 0.0);
        lo = fmin(lo, a[i] - r);
        hi = fmax(hi, a[i] + r);
    }
    const int64_t idx = which == 0 ? k - 1 : 0;
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (!(mid > lo && mid < hi)) break;
        if (sturm_count(k, a, b2, mid) > idx) hi = mid; else lo = mid;
    }
    out[which] = 0.5 * (lo + hi);
}

}  // namespace

// Residual bound of a Ritz value theta of the k x k Lanczos tridiagonal
// matrix T (diagonal a, squared off-diagonal b2[0..k-2]): the Ritz pair
// (theta, V s) of N has residual |N V s - theta V s| = beta_k |s_k| with s
// the unit eigenvector of T for theta and beta_k^2 = b2[k-1]. s comes from
// inverse iteration: (T - sigma I) x = y solved by Gaussian elimination with
// partial pivoting on the tridiagonal band, sigma a hair off theta.
static double ritz_residual(int64_t k, const std::vector<double>& a, const std::vector<double>& b2, double theta) {
    if (k <= 0) return 0.0;
    const double beta_k = std::sqrt(std::max(b2[k - 1], 0.0));
    if (k == 1) return beta_k;
    std::vector<double> off(k - 1);
    double scale = 0.0;
    for (int64_t i = 0; i < k; ++i) scale = std::max(scale, std::fabs(a[i]));
    for (int64_t i = 0; i + 1 < k; ++i) {
        off[i] = std::sqrt(std::max(b2[i], 0.0));
        scale = std::max(scale, off[i]);
    }
    const double sigma = theta + 1e-12 * std::max(scale, 1.0);
    std::vector<double> x(k, 1.0 / std::sqrt((double)k));
    // band LU of T - sigma I with partial pivoting: rows keep diagonal d,
    // first and second super-diagonals u1, u2, and the multipliers
    std::vector<double> d(k), u1(k, 0.0), u2(k, 0.0), mult(k, 0.0);
    std::vector<char> swapped(k, 0);
    for (int64_t i = 0; i < k; ++i) d[i] = a[i] - sigma;
    for (int64_t i = 0; i + 1 < k; ++i) u1[i] = off[i];
    std::vector<double> lower(off);  // sub-diagonal
    for (int64_t i = 0; i + 1 < k; ++i) {
        if (std::fabs(lower[i]) > std::fabs(d[i])) {
            // swap rows i and i + 1 (row i + 1: lower[i], d[i+1], u1[i+1])
            std::swap(d[i], lower[i]);
            std::swap(u1[i], d[i + 1]);
            std::swap(u2[i], u1[i + 1]);
            swapped[i] = 1;
        }
        const double piv = d[i] != 0.0 ? d[i] : 1e-300;
        mult[i] = lower[i] / piv;
        d[i + 1] -= mult[i] * u1[i];
        u1[i + 1] -= mult[i] * u2[i];
    }
    if (d[k - 1] == 0.0) d[k - 1] = 1e-300;
    for (int it = 0; it < 3; ++it) {
        std::vector<double> y(x);
        for (int64_t i = 0; i + 1 < k; ++i) {
            if (swapped[i]) std::swap(y[i], y[i + 1]);
            y[i + 1] -= mult[i] * y[i];
        }
        for (int64_t i = k - 1; i >= 0; --i) {
            double v = y[i];
            if (i + 1 < k) v -= u1[i] * y[i + 1];
            if (i + 2 < k) v -= u2[i] * y[i + 2];
            y[i] = v / (d[i] != 0.0 ? d[i] : 1e-300);
        }
        double nrm = 0.0;
        for (int64_t i = 0; i < k; ++i) nrm += y[i] * y[i];
        nrm = std::sqrt(nrm);
        if (!(nrm > 0.0) || !std::isfinite(nrm)) break;
        for (int64_t i = 0; i < k; ++i) x[i] = y[i] / nrm;
    }
    return beta_k * std::fabs(x[k - 1]);
}

int lanczos_spectral_bound(const DevGraph& g, int max_steps, double tol, cudaStream_t st, double* lam2,
                           double* lamn, int* steps, LanczosInfo* info) {
    const int64_t n = g.n;
    if (n < 3) return -1;
    const int64_t kmax = max_steps < n - 1 ? max_steps : n - 1;
    double *V = nullptr, *isd = nullptr, *phi = nullptr, *w = nullptr, *part = nullptr, *coef = nullptr;
    double *alpha = nullptr, *beta2 = nullptr, *ritz = nullptr;
    const double** vptrs = nullptr;
    auto cleanup = [&]() {
        cudaFree(V); cudaFree(isd); cudaFree(phi); cudaFree(w); cudaFree(part); cudaFree(coef);
        cudaFree(alpha); cudaFree(beta2); cudaFree(ritz); cudaFree(vptrs);
    };
    if (cudaMalloc(&V, (size_t)(kmax + 1) * (size_t)n * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&isd, n * sizeof(double)) != cudaSuccess || cudaMalloc(&phi, n * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&w, n * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&part, (size_t)(kmax + 2) * kLzCtas * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&coef, (kmax + 2) * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&alpha, (kmax + 1) * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&beta2, (kmax + 1) * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&ritz, 2 * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&vptrs, (kmax + 3) * sizeof(double*)) != cudaSuccess) {
        cleanup();
        cudaGetLastError();
        return -2;
    }
    // pointer table: [phi, q_0, q_1, ..., q_kmax, w]
    std::vector<const double*> hp(kmax + 3);
    hp[0] = phi;
    for (int64_t i = 0; i <= kmax; ++i) hp[i + 1] = V + (size_t)i * (size_t)n;
    hp[kmax + 2] = w;
    cudaMemcpyAsync(vptrs, hp.data(), hp.size() * sizeof(double*), cudaMemcpyHostToDevice, st);
    const int grid = 1216, blk = 256;
    lz_init_kernel<<<grid, blk, 0, st>>>(g, isd, phi, V);
    note_launches(1);
    // orthogonalise the start vector against phi (twice), normalise
    for (int pass = 0; pass < 2; ++pass) {
        lz_dots_kernel<<<kLzCtas, kCta, 0, st>>>(vptrs, 1, V, n, part);
        lz_dots_final_kernel<<<1, kCta, 0, st>>>(part, kLzCtas, coef);
        lz_subtract_kernel<<<grid, blk, 0, st>>>(vptrs, 1, coef, V, n);
        note_launches(3);
    }
    lz_dots_kernel<<<kLzCtas, kCta, 0, st>>>(vptrs + 1, 1, V, n, part);
    lz_dots_final_kernel<<<1, kCta, 0, st>>>(part, kLzCtas, coef);
    lz_scale_kernel<<<grid, blk, 0, st>>>(V, coef, V, n);
    note_launches(3);

    double prev_hi = 0.0, prev_lo = 0.0, hr[2] = {0.0, 0.0};
    int64_t k = 0;
    bool converged = false;
    for (int64_t j = 0; j < kmax; ++j) {
        double* qj = V + (size_t)j * (size_t)n;
        lz_spmv_kernel<<<grid * 4, blk, 0, st>>>(g, isd, qj, w);
        // alpha_j = q_j . w
        lz_dots_kernel<<<kLzCtas, kCta, 0, st>>>(vptrs + 1 + j, 1, w, n, part);
        lz_dots_final_kernel<<<1, kCta, 0, st>>>(part, kLzCtas, alpha + j);
        note_launches(3);
        // full re-orthogonalisation against phi, q_0..q_j, twice
        for (int pass = 0; pass < 2; ++pass) {
            const int m = (int)(j + 2);
            lz_dots_kernel<<<kLzCtas, kCta, 0, st>>>(vptrs, m, w, n, part);
            lz_dots_final_kernel<<<m, kCta, 0, st>>>(part, kLzCtas, coef);
            lz_subtract_kernel<<<grid, blk, 0, st>>>(vptrs, m, coef, w, n);
            note_launches(3);
        }
        // beta_j^2 = w . w
        lz_dots_kernel<<<kLzCtas, kCta, 0, st>>>(vptrs + kmax + 2, 1, w, n, part);
        lz_dots_final_kernel<<<1, kCta, 0, st>>>(part, kLzCtas, beta2 + j);
        note_launches(2);
        k = j + 1;
        double b2 = 0.0;
        cudaMemcpyAsync(&b2, beta2 + j, sizeof(double), cudaMemcpyDeviceToHost, st);
        if (cudaStreamSynchronize(st) != cudaSuccess) {
            cleanup();
            return -3;
        }
        const double beta = std::sqrt(b2);
        const bool last = beta < 1e-12 || k == kmax;
        if (k % 10 == 0 || last) {
            lz_ritz_kernel<<<1, 32, 0, st>>>(k, alpha, beta2, ritz);
            note_launches(1);
            cudaMemcpyAsync(hr, ritz, 2 * sizeof(double), cudaMemcpyDeviceToHost, st);
            if (cudaStreamSynchronize(st) != cudaSuccess) {
                cleanup();
                return -3;
            }
            if (last) {
                converged = beta < 1e-12;  // the Krylov space is exhausted: the Ritz values are exact
                break;
            }
            if (k >= 20 && std::fabs(hr[0] - prev_hi) < tol && std::fabs(hr[1] - prev_lo) < tol) {
                converged = true;
                break;
            }
            prev_hi = hr[0];
            prev_lo = hr[1];
        }
        lz_scale_kernel<<<grid, blk, 0, st>>>(w, beta2 + j, V + (size_t)(j + 1) * (size_t)n, n);
        note_launches(1);
    }
    *lam2 = hr[0];
    *lamn = hr[1];
    *steps = (int)k;
    if (info) {
        // residual bounds of the two extreme Ritz pairs, from the tridiagonal matrix
        std::vector<double> ha(k > 0 ? k : 1), hb(k > 0 ? k : 1);
        if (k > 0 && (cudaMemcpyAsync(ha.data(), alpha, k * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                      cudaMemcpyAsync(hb.data(), beta2, k * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                      cudaStreamSynchronize(st) != cudaSuccess)) {
            cleanup();
            return -3;
        }
        info->converged = converged ? 1 : 0;
        info->resid_hi = ritz_residual(k, ha, hb, hr[0]);
        info->resid_lo = ritz_residual(k, ha, hb, hr[1]);
    }
    cleanup();
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

}  // namespace geer
