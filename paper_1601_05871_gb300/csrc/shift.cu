// Learned diagonal shift: matrix features and the shift-predictor MLP.
//
// IC(k) of a matrix that is not an M-matrix can break down (a pivot <= 0 once fill is
// dropped); factoring B + alpha * diag(B) restores positive pivots for a large enough
// alpha at the price of a weaker preconditioner.  A small network reads 8 features of
// the matrix and predicts log10 alpha, so the first attempt is usually the last; the
// doubling retry (api.cpp, ic_numeric_shifted) remains the fallback and has the last word.
//
// Features (FP64, deterministic two-stage reductions), for row i with d = B_ii,
// s = sum_{j != i} |B_ij| and r = ||row i||_2:  dd_i = d / max(s, d / 1000),
// rn_i = r / d;  out = [min dd, mean dd, mean rn, max rn, positive fraction of the
// off-diagonal entries, k, log10 n, nu].
//
// MLP (FP32): z = (x - mean) / std, h1 = relu(z W1 + b1), h2 = relu(h1 W2 + b2),
// y = h2 . w3 + b3 with 32 hidden units; loss (1 / 2N) sum (y - t)^2.  One warp per
// sample, lane h owning hidden unit h; the per-sample gradient is written by each lane
// into its own slots of a per-warp shared-memory buffer (no atomics), the warps'
// buffers are summed in a fixed order per block, and the blocks' partial sums in a
// fixed order by a second kernel, so training is deterministic.  Adam: one thread per
// parameter.  Flat parameter order: W1 (8 x 32, row-major), b1, W2 (32 x 32,
// row-major, input g to unit h at g * 32 + h), b2, w3, b3.
#include <cmath>
#include <cstdint>

#include "ick_internal.h"

namespace ick {
namespace {

constexpr int kFeatThreads = 256;
constexpr int kFeatBlocks = 256;

struct FeatPart {
    double dd_min, dd_sum, rn_sum, rn_max, pos, off, bad;
};

__global__ void __launch_bounds__(kFeatThreads)
features_rows(int n, const long long* __restrict__ rp, const int* __restrict__ ci, const double* __restrict__ v,
              FeatPart* part) {
    double dd_min = INFINITY, dd_sum = 0.0, rn_sum = 0.0, rn_max = 0.0, pos = 0.0, off = 0.0, bad = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double d = 0.0, s = 0.0, sq = 0.0;
        bool has_d = false;
        for (long long e = rp[i]; e < rp[i + 1]; ++e) {
            const int j = ci[e];
            const double x = v[e];
            sq = fma(x, x, sq);
            if (j == i) {
                d = x;
                has_d = true;
            } else {
                s += fabs(x);
                off += 1.0;
                pos += x > 0.0 ? 1.0 : 0.0;
            }
        }
        if (!has_d || !(d > 0.0)) {
            bad += 1.0;
            continue;
        }
        const double dd = d / fmax(s, d / kShiftDdCap);
        const double rn = sqrt(sq) / d;
        dd_min = fmin(dd_min, dd);
        dd_sum += dd;
        rn_sum += rn;
        rn_max = fmax(rn_max, rn);
    }
    // block reduction in a fixed order: warp shuffles, then warp 0 over the warps
    __shared__ FeatPart w[kFeatThreads / 32];
    for (int o = 16; o > 0; o >>= 1) {
        dd_min = fmin(dd_min, __shfl_xor_sync(0xffffffffu, dd_min, o));
        dd_sum += __shfl_xor_sync(0xffffffffu, dd_sum, o);
        rn_sum += __shfl_xor_sync(0xffffffffu, rn_sum, o);
        rn_max = fmax(rn_max, __shfl_xor_sync(0xffffffffu, rn_max, o));
        pos += __shfl_xor_sync(0xffffffffu, pos, o);
        off += __shfl_xor_sync(0xffffffffu, off, o);
        bad += __shfl_xor_sync(0xffffffffu, bad, o);
    }
    if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = FeatPart{dd_min, dd_sum, rn_sum, rn_max, pos, off, bad};
    __syncthreads();
    if (threadIdx.x == 0) {
        FeatPart t = w[0];
        for (int q = 1; q < kFeatThreads / 32; ++q) {
            t.dd_min = fmin(t.dd_min, w[q].dd_min);
            t.dd_sum += w[q].dd_sum;
            t.rn_sum += w[q].rn_sum;
            t.rn_max = fmax(t.rn_max, w[q].rn_max);
            t.pos += w[q].pos;
            t.off += w[q].off;
            t.bad += w[q].bad;
        }
        part[blockIdx.x] = t;
    }
}

__global__ void features_finish(int n, int nparts, const FeatPart* part, int k, double nu, double* out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    FeatPart t = part[0];
    for (int q = 1; q < nparts; ++q) {
        t.dd_min = fmin(t.dd_min, part[q].dd_min);
        t.dd_sum += part[q].dd_sum;
        t.rn_sum += part[q].rn_sum;
        t.rn_max = fmax(t.rn_max, part[q].rn_max);
        t.pos += part[q].pos;
        t.off += part[q].off;
        t.bad += part[q].bad;
    }
    out[0] = t.dd_min;
    out[1] = t.dd_sum / n;
    out[2] = t.rn_sum / n;
    out[3] = t.rn_max;
    out[4] = t.off > 0.0 ? t.pos / t.off : 0.0;
    out[5] = double(k);
    out[6] = log10(double(n));
    out[7] = nu;
    out[8] = t.bad;  // rows whose diagonal is missing or not positive
}

// ------------------------------------------------------------------------ MLP
constexpr int H = kMlpHidden;
constexpr int F = kMlpFeatures;
constexpr int OFF_W1 = 0, OFF_B1 = F * H, OFF_W2 = OFF_B1 + H, OFF_B2 = OFF_W2 + H * H, OFF_W3 = OFF_B2 + H,
              OFF_B3 = OFF_W3 + H, NPARAM = OFF_B3 + 1;
static_assert(NPARAM == kMlpParams, "parameter layout");
constexpr int kMlpWarps = 4;  // the gradient kernel keeps one parameter-sized buffer per warp

__device__ __forceinline__ float warp_sum_f(float v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// One sample on one warp: fills the activations lane h needs (z of all features,
// a1_h, h1_h, a2_h, h2_h) and returns y on every lane.
struct Act {
    float z[F];
    float a1, h1, a2, h2, y;
};

__device__ __forceinline__ void forward_one(const float* th, const float* mean, const float* rstd, const float* x,
                                            Act& A) {
    const int h = threadIdx.x & 31;
#pragma unroll
    for (int f = 0; f < F; ++f) A.z[f] = (x[f] - mean[f]) * rstd[f];
    float a1 = th[OFF_B1 + h];
#pragma unroll
    for (int f = 0; f < F; ++f) a1 = fmaf(A.z[f], th[OFF_W1 + f * H + h], a1);
    A.a1 = a1;
    A.h1 = fmaxf(a1, 0.0f);
    float a2 = th[OFF_B2 + h];
#pragma unroll
    for (int g = 0; g < H; ++g) a2 = fmaf(__shfl_sync(0xffffffffu, A.h1, g), th[OFF_W2 + g * H + h], a2);
    A.a2 = a2;
    A.h2 = fmaxf(a2, 0.0f);
    A.y = warp_sum_f(A.h2 * th[OFF_W3 + h]) + th[OFF_B3];
}

__global__ void __launch_bounds__(32 * kMlpWarps)
mlp_forward_kernel(const float* __restrict__ theta, const float* __restrict__ mean, const float* __restrict__ rstd,
                   const float* __restrict__ X, long long n, float* __restrict__ y) {
    __shared__ float th[NPARAM];
    for (int p = threadIdx.x; p < NPARAM; p += blockDim.x) th[p] = theta[p];
    __syncthreads();
    const int warp = threadIdx.x >> 5;
    for (long long s = (long long)blockIdx.x * kMlpWarps + warp; s < n; s += (long long)gridDim.x * kMlpWarps) {
        Act A;
        forward_one(th, mean, rstd, X + s * F, A);
        if ((threadIdx.x & 31) == 0) y[s] = A.y;
    }
}

// Per-block partial gradient and loss; see the file header for the accumulation order.
__global__ void __launch_bounds__(32 * kMlpWarps)
mlp_grad_kernel(const float* __restrict__ theta, const float* __restrict__ mean, const float* __restrict__ rstd,
                const float* __restrict__ X, const float* __restrict__ t, long long n, float* __restrict__ part,
                float* __restrict__ loss_part) {
    __shared__ float th[NPARAM];
    __shared__ float acc[kMlpWarps][NPARAM];
    __shared__ float lacc[kMlpWarps];
    for (int p = threadIdx.x; p < NPARAM; p += blockDim.x) th[p] = theta[p];
    for (int p = threadIdx.x; p < kMlpWarps * NPARAM; p += blockDim.x) (&acc[0][0])[p] = 0.0f;
    __syncthreads();
    const int warp = threadIdx.x >> 5, h = threadIdx.x & 31;
    float* g = acc[warp];
    float loss = 0.0f;
    const float inv_n = 1.0f / float(n);
    for (long long s = (long long)blockIdx.x * kMlpWarps + warp; s < n; s += (long long)gridDim.x * kMlpWarps) {
        Act A;
        forward_one(th, mean, rstd, X + s * F, A);
        const float res = A.y - t[s];
        loss = fmaf(res, res, loss);
        const float r = res * inv_n;                            // dL/dy
        g[OFF_W3 + h] += r * A.h2;
        if (h == 0) g[OFF_B3] += r;
        const float d2 = A.a2 > 0.0f ? r * th[OFF_W3 + h] : 0.0f;  // dL/da2_h
        g[OFF_B2 + h] += d2;
        float d1 = 0.0f;                                        // dL/dh1 for unit h
#pragma unroll
        for (int q = 0; q < H; ++q) {
            const float h1q = __shfl_sync(0xffffffffu, A.h1, q);
            const float d2q = __shfl_sync(0xffffffffu, d2, q);
            g[OFF_W2 + q * H + h] += h1q * d2;                 // input q -> unit h
            d1 = fmaf(th[OFF_W2 + h * H + q], d2q, d1);         // unit h feeds q
        }
        d1 = A.a1 > 0.0f ? d1 : 0.0f;                           // dL/da1_h
        g[OFF_B1 + h] += d1;
#pragma unroll
        for (int f = 0; f < F; ++f) g[OFF_W1 + f * H + h] += A.z[f] * d1;
    }
    if (h == 0) lacc[warp] = loss;
    __syncthreads();
    for (int p = threadIdx.x; p < NPARAM; p += blockDim.x) {
        float v = 0.0f;
        for (int w = 0; w < kMlpWarps; ++w) v += acc[w][p];
        part[(size_t)blockIdx.x * NPARAM + p] = v;
    }
    if (threadIdx.x == 0) {
        float v = 0.0f;
        for (int w = 0; w < kMlpWarps; ++w) v += lacc[w];
        loss_part[blockIdx.x] = v;
    }
}

__global__ void mlp_grad_sum(const float* __restrict__ part, const float* __restrict__ loss_part, int nblocks,
                             long long n, float* __restrict__ grad, float* __restrict__ loss) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < NPARAM) {
        float v = 0.0f;
        for (int b = 0; b < nblocks; ++b) v += part[(size_t)b * NPARAM + p];
        grad[p] = v;
    }
    if (p == 0) {
        float v = 0.0f;
        for (int b = 0; b < nblocks; ++b) v += loss_part[b];
        *loss = 0.5f * v / float(n);
    }
}

__global__ void adam_kernel(float* __restrict__ theta, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ g, float lr, float c1, float c2) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NPARAM) return;
    const float mp = 0.9f * m[p] + 0.1f * g[p];
    const float vp = 0.999f * v[p] + 0.001f * g[p] * g[p];
    m[p] = mp;
    v[p] = vp;
    theta[p] -= lr * (mp * c1) / (sqrtf(vp * c2) + 1e-8f);
}

}  // namespace

int mlp_grad_blocks(long long n) {
    const long long b = (n + kMlpWarps - 1) / kMlpWarps;
    return int(b < 1 ? 1 : (b > kMlpMaxBlocks ? kMlpMaxBlocks : b));
}

cudaError_t launch_features(int n, const long long* rp, const int* ci, const double* v, int k, double nu,
                            void* scratch, double* out, cudaStream_t s) {
    FeatPart* part = static_cast<FeatPart*>(scratch);
    const int blocks = (n + kFeatThreads - 1) / kFeatThreads < kFeatBlocks ? (n + kFeatThreads - 1) / kFeatThreads
                                                                           : kFeatBlocks;
    const int nb = blocks < 1 ? 1 : blocks;
    features_rows<<<nb, kFeatThreads, 0, s>>>(n, rp, ci, v, part);
    features_finish<<<1, 32, 0, s>>>(n, nb, part, k, nu, out);
    return cudaGetLastError();
}

size_t features_scratch_bytes() { return kFeatBlocks * sizeof(FeatPart); }

cudaError_t launch_mlp_forward(const MlpDev& M, const float* X, long long n, float* y, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const long long b = (n + kMlpWarps - 1) / kMlpWarps;
    mlp_forward_kernel<<<int(b < 4096 ? b : 4096), 32 * kMlpWarps, 0, s>>>(M.theta, M.mean, M.rstd, X, n, y);
    return cudaGetLastError();
}

cudaError_t launch_mlp_grad(const MlpDev& M, const float* X, const float* t, long long n, cudaStream_t s) {
    const int nb = mlp_grad_blocks(n);
    mlp_grad_kernel<<<nb, 32 * kMlpWarps, 0, s>>>(M.theta, M.mean, M.rstd, X, t, n, M.part, M.loss_part);
    mlp_grad_sum<<<(NPARAM + 255) / 256, 256, 0, s>>>(M.part, M.loss_part, nb, n, M.grad, M.loss);
    return cudaGetLastError();
}

cudaError_t launch_mlp_adam(const MlpDev& M, float lr, int step, cudaStream_t s) {
    const float c1 = 1.0f / (1.0f - powf(0.9f, float(step)));
    const float c2 = 1.0f / (1.0f - powf(0.999f, float(step)));
    adam_kernel<<<(NPARAM + 255) / 256, 256, 0, s>>>(M.theta, M.m, M.v, M.grad, lr, c1, c2);
    return cudaGetLastError();
}

}  // namespace ick
