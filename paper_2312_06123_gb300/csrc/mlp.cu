// mlp.cu -- the learned SMM -> AMC switch: a 6 -> 64 -> 64 -> 1 ReLU network
// with FP16 weights and FP32 arithmetic that, after each SMM iteration of
// Algorithm 3, predicts log C(l_b + 1) - log C(l_b), the change of a query's
// total cost (SMM pushes + AMC walk steps) from running one more iteration;
// the query switches to AMC when the prediction is >= 0. The total
// truncation length l is fixed, so the choice changes run time only, never
// the eps guarantee of Theorem 2. Without a network, Eq. (17) decides.
//
// Kernels: the per-query call inside the SMM loop (one warp per query),
// batched inference, and training: forward + backward over chunks of 64 rows
// (per-chunk gradient partials reduced in a fixed order, so training is
// deterministic) and Adam on FP32 master weights with an FP16 copy. The
// layers are 64 wide: every product is a few thousand FMAs, latency- not
// throughput-bound, so they run on the CUDA cores.
#include <cuda_fp16.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "../../include/geer.h"
#include "geer_internal.cuh"
#include "geer_kernels.h"

namespace geer {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kRowsPerChunk = 64;  // rows per CTA of the training kernel
constexpr int kPartWidth = kMlpParams + 1;  // gradient partial + loss partial

// shared-memory copy of the network for inference: W1, b1, W2 transposed
// (W2T[k][j] = W2[j][k], so a warp's 32 output units read consecutive words),
// b2, W3, b3
constexpr int kSwW1 = 0, kSwB1 = kSwW1 + kMlpH * kMlpIn, kSwW2T = kSwB1 + kMlpH, kSwB2 = kSwW2T + kMlpH * kMlpH,
              kSwW3 = kSwB2 + kMlpH, kSwB3 = kSwW3 + kMlpH, kSwSize = kSwB3 + 1;

__device__ __forceinline__ float h2f(unsigned short b) { return __half2float(__ushort_as_half(b)); }

__device__ void mlp_load_inference(float* sw, const unsigned short* w) {
    for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) {
        const float v = h2f(w[i]);
        if (i >= kMlpOffW2 && i < kMlpOffB2) {
            const int j = (i - kMlpOffW2) / kMlpH, k = (i - kMlpOffW2) % kMlpH;
            sw[kSwW2T + k * kMlpH + j] = v;
        } else {
            sw[i] = v;  // the other blocks keep their offsets
        }
    }
}

// One network evaluation by a whole warp: lane l owns hidden units l, l + 32.
__device__ __forceinline__ float mlp_eval_warp(const float* sw, const float (&x)[kMlpIn], int lane) {
    float h1a = sw[kSwB1 + lane], h1b = sw[kSwB1 + lane + 32];
#pragma unroll
    for (int k = 0; k < kMlpIn; ++k) {
        h1a = fmaf(sw[kSwW1 + lane * kMlpIn + k], x[k], h1a);
        h1b = fmaf(sw[kSwW1 + (lane + 32) * kMlpIn + k], x[k], h1b);
    }
    h1a = fmaxf(h1a, 0.f);
    h1b = fmaxf(h1b, 0.f);
    float z2a = sw[kSwB2 + lane], z2b = sw[kSwB2 + lane + 32];
#pragma unroll 8
    for (int k = 0; k < 32; ++k) {
        const float a = __shfl_sync(kFull, h1a, k), b = __shfl_sync(kFull, h1b, k);
        z2a = fmaf(sw[kSwW2T + k * kMlpH + lane], a, z2a);
        z2b = fmaf(sw[kSwW2T + k * kMlpH + lane + 32], a, z2b);
        z2a = fmaf(sw[kSwW2T + (k + 32) * kMlpH + lane], b, z2a);
        z2b = fmaf(sw[kSwW2T + (k + 32) * kMlpH + lane + 32], b, z2b);
    }
    float p = sw[kSwW3 + lane] * fmaxf(z2a, 0.f) + sw[kSwW3 + lane + 32] * fmaxf(z2b, 0.f);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) p += __shfl_xor_sync(kFull, p, o);
    return p + sw[kSwB3];
}

}  // namespace

// Batched inference: one warp per row of normalised inputs.
__global__ void __launch_bounds__(256) mlp_forward_kernel(const float* x, int64_t rows, const unsigned short* w,
                                                          float* y) {
    __shared__ float sw[kSwSize];
    mlp_load_inference(sw, w);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (r >= rows) return;
    float f[kMlpIn];
#pragma unroll
    for (int k = 0; k < kMlpIn; ++k) f[k] = x[r * kMlpIn + k];
    const float v = mlp_eval_warp(sw, f, lane);
    if (lane == 0) y[r] = v;
}

// Forward and backward of the mean squared error over `count` rows
// (rows perm[base .. base + count) of x, t), one CTA per 64 rows; writes
// this chunk's gradient and loss partial sums to part[blockIdx.x].
//   z1 = W1 x + b1, h1 = relu(z1), z2 = W2 h1 + b2, h2 = relu(z2),
//   y = W3 h2 + b3, L = (1/count) sum (y - t)^2.
__global__ void __launch_bounds__(256) mlp_grad_kernel(const float* x, const float* t, const int32_t* perm,
                                                       int64_t base, int64_t count, const unsigned short* w,
                                                       float* part) {
    extern __shared__ float sm[];
    float* W1 = sm;                          // [64][6]
    float* b1 = W1 + kMlpH * kMlpIn;         // [64]
    float* W2 = b1 + kMlpH;                  // [64][64], row j: output unit j
    float* W2T = W2 + kMlpH * kMlpH;         // [64][64], W2T[k][j] = W2[j][k]
    float* b2 = W2T + kMlpH * kMlpH;         // [64]
    float* W3 = b2 + kMlpH;                  // [64]
    float* b3 = W3 + kMlpH;                  // [1]
    float* X = b3 + 4;                       // [R][6]
    float* H1 = X + kRowsPerChunk * kMlpIn;  // [R][64]
    float* H2 = H1 + kRowsPerChunk * kMlpH;  // [R][64], later dL/dz2
    float* D1 = H2 + kRowsPerChunk * kMlpH;  // [R][64]: dL/dz1
    float* Y = D1 + kRowsPerChunk * kMlpH;   // [R]: y, later dL/dy
    float* red = Y + kRowsPerChunk;          // [8] warp partials of the loss
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    for (int i = tid; i < kMlpParams; i += blockDim.x) {
        const float v = h2f(w[i]);
        if (i < kMlpOffB1) W1[i] = v;
        else if (i < kMlpOffW2) b1[i - kMlpOffB1] = v;
        else if (i < kMlpOffB2) {
            const int j = (i - kMlpOffW2) / kMlpH, k = (i - kMlpOffW2) % kMlpH;
            W2[j * kMlpH + k] = v;
            W2T[k * kMlpH + j] = v;
        } else if (i < kMlpOffW3) b2[i - kMlpOffB2] = v;
        else if (i < kMlpOffB3) W3[i - kMlpOffW3] = v;
        else b3[0] = v;
    }
    const int64_t r0 = (int64_t)blockIdx.x * kRowsPerChunk;
    const int nr = (int)std::min<int64_t>(kRowsPerChunk, count - r0);
    for (int i = tid; i < kRowsPerChunk * kMlpIn; i += blockDim.x) {
        const int r = i / kMlpIn, k = i % kMlpIn;
        float v = 0.f;
        if (r < nr) {
            const int64_t row = perm ? perm[base + r0 + r] : base + r0 + r;
            v = x[row * kMlpIn + k];
        }
        X[i] = v;
    }
    __syncthreads();
    const int jj = tid & 63, rr = tid >> 6;  // 64 columns x 4 row phases
    // layer 1
    for (int r = rr; r < kRowsPerChunk; r += 4) {
        float z = b1[jj];
#pragma unroll
        for (int k = 0; k < kMlpIn; ++k) z = fmaf(W1[jj * kMlpIn + k], X[r * kMlpIn + k], z);
        H1[r * kMlpH + jj] = fmaxf(z, 0.f);
    }
    __syncthreads();
    // layer 2
    for (int r = rr; r < kRowsPerChunk; r += 4) {
        float z = b2[jj];
        for (int k = 0; k < kMlpH; ++k) z = fmaf(W2T[k * kMlpH + jj], H1[r * kMlpH + k], z);
        H2[r * kMlpH + jj] = fmaxf(z, 0.f);
    }
    __syncthreads();
    // output and dL/dy: one warp per 8 rows
    float lsum = 0.f;
    for (int r = wid; r < kRowsPerChunk; r += 8) {
        float p = W3[lane] * H2[r * kMlpH + lane] + W3[lane + 32] * H2[r * kMlpH + lane + 32];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) p += __shfl_xor_sync(kFull, p, o);
        if (lane == 0) {
            float dy = 0.f;
            if (r < nr) {
                const int64_t row = perm ? perm[base + r0 + r] : base + r0 + r;
                const float e = p + b3[0] - t[row];
                lsum += e * e;
                dy = 2.f * e / (float)count;
            }
            Y[r] = dy;
        }
    }
    if (lane == 0) red[wid] = lsum;
    __syncthreads();
    float* P = part + (int64_t)blockIdx.x * kPartWidth;
    // dW3, db3
    if (tid < kMlpH) {
        float g = 0.f;
        for (int r = 0; r < kRowsPerChunk; ++r) g = fmaf(Y[r], H2[r * kMlpH + tid], g);
        P[kMlpOffW3 + tid] = g;
    } else if (tid == kMlpH) {
        float g = 0.f;
        for (int r = 0; r < kRowsPerChunk; ++r) g += Y[r];
        P[kMlpOffB3] = g;
        float l = 0.f;
        for (int i = 0; i < 8; ++i) l += red[i];
        P[kMlpParams] = l;
    }
    __syncthreads();
    // dL/dz2 in place of h2
    for (int r = rr; r < kRowsPerChunk; r += 4) {
        const float h = H2[r * kMlpH + jj];
        H2[r * kMlpH + jj] = h > 0.f ? Y[r] * W3[jj] : 0.f;
    }
    __syncthreads();
    // dW2[j][k] = sum_r dz2[r][j] h1[r][k]; db2
    for (int j = rr; j < kMlpH; j += 4) {
        float g = 0.f;
        for (int r = 0; r < kRowsPerChunk; ++r) g = fmaf(H2[r * kMlpH + j], H1[r * kMlpH + jj], g);
        P[kMlpOffW2 + j * kMlpH + jj] = g;
    }
    if (tid < kMlpH) {
        float g = 0.f;
        for (int r = 0; r < kRowsPerChunk; ++r) g += H2[r * kMlpH + tid];
        P[kMlpOffB2 + tid] = g;
    }
    // dL/dz1 = (W2^T dz2) * [h1 > 0]
    for (int r = rr; r < kRowsPerChunk; r += 4) {
        float g = 0.f;
        for (int j = 0; j < kMlpH; ++j) g = fmaf(W2[j * kMlpH + jj], H2[r * kMlpH + j], g);
        D1[r * kMlpH + jj] = H1[r * kMlpH + jj] > 0.f ? g : 0.f;
    }
    __syncthreads();
    // dW1[j][k] = sum_r dz1[r][j] x[r][k]; db1
    for (int i = tid; i < kMlpH * kMlpIn; i += blockDim.x) {
        const int j = i / kMlpIn, k = i % kMlpIn;
        float g = 0.f;
        for (int r = 0; r < kRowsPerChunk; ++r) g = fmaf(D1[r * kMlpH + j], X[r * kMlpIn + k], g);
        P[kMlpOffW1 + i] = g;
    }
    if (tid < kMlpH) {
        float g = 0.f;
        for (int r = 0; r < kRowsPerChunk; ++r) g += D1[r * kMlpH + tid];
        P[kMlpOffB1 + tid] = g;
    }
}

// grad[p] = sum over chunks of part[chunk][p], in chunk order.
__global__ void mlp_reduce_kernel(const float* part, int chunks, float* grad) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= kPartWidth) return;
    double g = 0.0;
    for (int c = 0; c < chunks; ++c) g += (double)part[(int64_t)c * kPartWidth + p];
    grad[p] = (float)g;
}

// Adam (Kingma and Ba) on the FP32 master weights; refreshes the FP16 copy.
__global__ void mlp_adam_kernel(float* master, float* m, float* v, const float* grad, unsigned short* w16, float lr,
                                float b1, float b2, float eps, float c1, float c2) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= kMlpParams) return;
    const float g = grad[p];
    const float mm = b1 * m[p] + (1.f - b1) * g;
    const float vv = b2 * v[p] + (1.f - b2) * g * g;
    m[p] = mm;
    v[p] = vv;
    const float wn = master[p] - lr * (mm / c1) / (sqrtf(vv / c2) + eps);
    master[p] = wn;
    w16[p] = __half_as_ushort(__float2half_rn(wn));
}

__global__ void mlp_master_kernel(const unsigned short* w16, float* master) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < kMlpParams) master[p] = h2f(w16[p]);
}


}  // namespace geer

using namespace geer;

namespace {

constexpr size_t kGradSmem = sizeof(float) * (kMlpH * kMlpIn + kMlpH + 2 * kMlpH * kMlpH + kMlpH + kMlpH + 4 +
                                              kRowsPerChunk * kMlpIn + 3 * kRowsPerChunk * kMlpH + kRowsPerChunk + 8);

// Device buffers of one training / gradient call (freed on return).
struct MlpBuffers {
    float* x = nullptr;
    float* t = nullptr;
    int32_t* perm = nullptr;
    float* part = nullptr;
    float* grad = nullptr;
    float* master = nullptr;
    float* m = nullptr;
    float* v = nullptr;
    unsigned short* w16 = nullptr;
    ~MlpBuffers() {
        cudaFree(x); cudaFree(t); cudaFree(perm); cudaFree(part); cudaFree(grad);
        cudaFree(master); cudaFree(m); cudaFree(v); cudaFree(w16);
    }
};

int mlp_cuda(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return GER_OK;
    cudaGetLastError();
    return set_error(e == cudaErrorMemoryAllocation ? GER_ERR_OOM : GER_ERR_CUDA, what);
}

int mlp_upload(MlpBuffers& b, int64_t rows, const float* x, const float* t, const uint16_t* w, int64_t chunks) {
    int rc;
    if ((rc = mlp_cuda(cudaMalloc(&b.x, rows * kMlpIn * sizeof(float) + 16), "mlp inputs"))) return rc;
    if (t && (rc = mlp_cuda(cudaMalloc(&b.t, rows * sizeof(float) + 16), "mlp targets"))) return rc;
    if ((rc = mlp_cuda(cudaMalloc(&b.w16, kMlpParams * sizeof(unsigned short) + 16), "mlp weights"))) return rc;
    if (chunks > 0) {
        if ((rc = mlp_cuda(cudaMalloc(&b.part, chunks * kPartWidth * sizeof(float)), "mlp partials"))) return rc;
        if ((rc = mlp_cuda(cudaMalloc(&b.grad, kPartWidth * sizeof(float)), "mlp gradient"))) return rc;
    }
    if ((rc = mlp_cuda(cudaMemcpy(b.x, x, rows * kMlpIn * sizeof(float), cudaMemcpyHostToDevice), "mlp inputs")))
        return rc;
    if (t && (rc = mlp_cuda(cudaMemcpy(b.t, t, rows * sizeof(float), cudaMemcpyHostToDevice), "mlp targets")))
        return rc;
    return mlp_cuda(cudaMemcpy(b.w16, w, kMlpParams * sizeof(unsigned short), cudaMemcpyHostToDevice), "mlp weights");
}

int mlp_grad_prepare() {
    static bool done = false;
    if (done) return GER_OK;
    int rc = mlp_cuda(cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)kGradSmem),
                      "mlp shared-memory opt-in");
    if (!rc) done = true;
    return rc;
}

// gradient (and loss) of the mean squared error over rows [base, base+count)
// of the (permuted) data into b.grad; stream-ordered
void mlp_grad_launch(MlpBuffers& b, int64_t base, int64_t count, cudaStream_t st) {
    const int chunks = (int)((count + kRowsPerChunk - 1) / kRowsPerChunk);
    prof_begin(FAM_MLP_TRAIN, st);
    mlp_grad_kernel<<<chunks, 256, kGradSmem, st>>>(b.x, b.t, b.perm, base, count, b.w16, b.part);
    mlp_reduce_kernel<<<(kPartWidth + 255) / 256, 256, 0, st>>>(b.part, chunks, b.grad);
    prof_end(FAM_MLP_TRAIN, st);
    note_launches(2);
}

uint64_t splitmix64(uint64_t& s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

}  // namespace

extern "C" {

void ger_default_mlp_train_options(ger_mlp_train_options* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->epochs = 60;
    o->batch = 1024;
    o->lr = 2e-3f;
    o->beta1 = 0.9f;
    o->beta2 = 0.999f;
    o->adam_eps = 1e-8f;
    o->seed = 7;
}

int ger_mlp_forward(int64_t rows, const float* x, const uint16_t* w, float* y) {
    if (rows < 0 || (rows > 0 && (!x || !y)) || !w) return set_error(GER_ERR_INVALID, "null argument");
    if (rows == 0) return GER_OK;
    MlpBuffers b;
    int rc = mlp_upload(b, rows, x, nullptr, w, 0);
    if (rc) return rc;
    float* yd = nullptr;
    if ((rc = mlp_cuda(cudaMalloc(&yd, rows * sizeof(float)), "mlp outputs"))) return rc;
    mlp_forward_kernel<<<(unsigned)((rows * 32 + 255) / 256), 256>>>(b.x, rows, b.w16, yd);
    note_launches(1);
    rc = mlp_cuda(cudaGetLastError(), "mlp forward launch");
    if (!rc) rc = mlp_cuda(cudaMemcpy(y, yd, rows * sizeof(float), cudaMemcpyDeviceToHost), "mlp forward");
    cudaFree(yd);
    return rc;
}

int ger_mlp_gradient(int64_t rows, const float* x, const float* t, const uint16_t* w, float* grad, float* loss) {
    if (rows <= 0 || !x || !t || !w || !grad) return set_error(GER_ERR_INVALID, "null argument or no rows");
    int rc = mlp_grad_prepare();
    if (rc) return rc;
    MlpBuffers b;
    const int64_t chunks = (rows + kRowsPerChunk - 1) / kRowsPerChunk;
    if ((rc = mlp_upload(b, rows, x, t, w, chunks))) return rc;
    mlp_grad_launch(b, 0, rows, 0);
    std::vector<float> g(kPartWidth);
    rc = mlp_cuda(cudaMemcpy(g.data(), b.grad, kPartWidth * sizeof(float), cudaMemcpyDeviceToHost), "mlp gradient");
    if (rc) return rc;
    std::memcpy(grad, g.data(), kMlpParams * sizeof(float));
    if (loss) *loss = g[kMlpParams] / (float)rows;
    return GER_OK;
}

int ger_mlp_train(int64_t rows, const float* x, const float* t, const ger_mlp_train_options* o, uint16_t* w,
                  float* loss_per_epoch) {
    if (rows <= 0 || !x || !t || !w || !o) return set_error(GER_ERR_INVALID, "null argument or no rows");
    if (o->epochs < 0 || o->batch <= 0 || !(o->lr > 0.f)) return set_error(GER_ERR_INVALID, "bad training options");
    int rc = mlp_grad_prepare();
    if (rc) return rc;
    MlpBuffers b;
    const int64_t mb = std::min<int64_t>(o->batch, rows);
    const int64_t chunks = (mb + kRowsPerChunk - 1) / kRowsPerChunk;
    if ((rc = mlp_upload(b, rows, x, t, w, chunks))) return rc;
    if ((rc = mlp_cuda(cudaMalloc(&b.perm, rows * sizeof(int32_t)), "mlp permutation"))) return rc;
    if ((rc = mlp_cuda(cudaMalloc(&b.master, kMlpParams * sizeof(float)), "mlp master weights"))) return rc;
    if ((rc = mlp_cuda(cudaMalloc(&b.m, kMlpParams * sizeof(float)), "mlp moments"))) return rc;
    if ((rc = mlp_cuda(cudaMalloc(&b.v, kMlpParams * sizeof(float)), "mlp moments"))) return rc;
    cudaMemset(b.m, 0, kMlpParams * sizeof(float));
    cudaMemset(b.v, 0, kMlpParams * sizeof(float));
    mlp_master_kernel<<<(kMlpParams + 255) / 256, 256>>>(b.w16, b.master);
    std::vector<int32_t> perm(rows);
    std::vector<float> gl(1);
    uint64_t rs = o->seed;
    int64_t step = 0;
    for (int ep = 0; ep < o->epochs; ++ep) {
        // a fresh shuffle per epoch (Fisher-Yates over splitmix64 draws)
        for (int64_t i = 0; i < rows; ++i) perm[i] = (int32_t)i;
        for (int64_t i = rows - 1; i > 0; --i) std::swap(perm[i], perm[splitmix64(rs) % (uint64_t)(i + 1)]);
        if ((rc = mlp_cuda(cudaMemcpy(b.perm, perm.data(), rows * sizeof(int32_t), cudaMemcpyHostToDevice),
                           "mlp permutation")))
            return rc;
        double lsum = 0.0;
        for (int64_t base = 0; base < rows; base += mb) {
            const int64_t cnt = std::min<int64_t>(mb, rows - base);
            mlp_grad_launch(b, base, cnt, 0);
            ++step;
            const float c1 = 1.f - powf(o->beta1, (float)step), c2 = 1.f - powf(o->beta2, (float)step);
            mlp_adam_kernel<<<(kMlpParams + 255) / 256, 256>>>(b.master, b.m, b.v, b.grad, b.w16, o->lr, o->beta1,
                                                                o->beta2, o->adam_eps, c1, c2);
            note_launches(1);
            if ((rc = mlp_cuda(cudaMemcpy(gl.data(), b.grad + kMlpParams, sizeof(float), cudaMemcpyDeviceToHost),
                               "mlp loss")))
                return rc;
            lsum += gl[0];
        }
        if (loss_per_epoch) loss_per_epoch[ep] = (float)(lsum / (double)rows);
    }
    return mlp_cuda(cudaMemcpy(w, b.w16, kMlpParams * sizeof(unsigned short), cudaMemcpyDeviceToHost),
                    "mlp weights");
}

}  // extern "C"
