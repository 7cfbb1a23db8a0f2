// Batched PCG kernels: many independent systems stored as one block-diagonal system
// (rows of system s are [row_off[s], row_off[s+1])).  Every system keeps its own PCG
// scalars and stops on its own tolerance: a converged system's step length is forced
// to zero, so its iterate and residual no longer change while the others continue.
// Reductions use one CTA per system and a fixed order, so results are reproducible.
#include <cstdint>

#include "ick_internal.h"

namespace ick {
namespace {

constexpr int kBT = 256;

__device__ __forceinline__ double bsum(double v) {
    __shared__ double s[kBT / 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) s[w] = v;
    __syncthreads();
    double t = 0.0;
    if (w == 0) {
        t = lane < kBT / 32 ? s[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    return t;
}

// out[s] = a_s . b_s for every system s (one CTA per system, grid-stride over systems)
__global__ void __launch_bounds__(kBT)
seg_dot(const long long* __restrict__ row_off, int count, const double* __restrict__ a,
        const double* __restrict__ b, double* __restrict__ out) {
    for (int s = blockIdx.x; s < count; s += gridDim.x) {
        const long long r0 = row_off[s], r1 = row_off[s + 1];
        double acc = 0.0;
        for (long long i = r0 + threadIdx.x; i < r1; i += kBT) acc = fma(a[i], b[i], acc);
        acc = bsum(acc);
        if (threadIdx.x == 0) out[s] = acc;
        __syncthreads();
    }
}

// Per-system scalar updates.  op 0: alpha = active ? rz / pq : 0.
// op 1: relres = sqrt(rr)/|b|; a system whose relres <= tol becomes inactive and keeps
//       its iteration count; counts the systems still active.
// op 2: beta = rz_new / rz, rz = rz_new (inactive: beta = 0).
// op 3: rz = v.  op 4: |b| = sqrt(v) (1 for a zero right-hand side), all systems active.
// The iteration number lives on the device (*B.iter, advanced by batch_bump at the top
// of every iteration) so that one captured iteration can be replayed as a graph.
__global__ void seg_scalars(BatchScalars B, int count, int op, double tol) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < count; s += gridDim.x * blockDim.x) {
        const double v = B.tmp[s];
        switch (op) {
            case 0: B.alpha[s] = B.active[s] ? B.rz[s] / v : 0.0; break;
            case 1: {
                const double rel = sqrt(v) / B.bnorm[s];
                if (B.active[s]) {
                    B.relres[s] = rel;
                    B.iters[s] = *B.iter;
                    if (rel <= tol) B.active[s] = 0;
                    else atomicAdd(B.nactive, 1);
                }
                break;
            }
            case 2: {
                const double beta = B.active[s] ? v / B.rz[s] : 0.0;
                B.beta[s] = beta;
                if (B.active[s]) B.rz[s] = v;
                break;
            }
            case 3: B.rz[s] = v; break;
            case 4:
                B.bnorm[s] = v > 0.0 ? sqrt(v) : 1.0;
                B.active[s] = 1;
                B.iters[s] = 0;
                B.relres[s] = v > 0.0 ? 1.0 : 0.0;
                if (!(v > 0.0)) B.active[s] = 0;
                break;
            default: break;
        }
    }
}

// x += alpha_s p, r -= alpha_s q (rows of system s)
__global__ void seg_xr(int n, const int* __restrict__ sys, const double* __restrict__ alpha,
                       double* __restrict__ x, double* __restrict__ r, const double* __restrict__ p,
                       const double* __restrict__ q) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double a = alpha[sys[i]];
        x[i] = fma(a, p[i], x[i]);
        r[i] = fma(-a, q[i], r[i]);
    }
}

// p = z + beta_s p for active systems
__global__ void seg_p(int n, const int* __restrict__ sys, const double* __restrict__ beta,
                      const int* __restrict__ active, double* __restrict__ p, const double* __restrict__ z) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int s = sys[i];
        if (active[s]) p[i] = fma(beta[s], p[i], z[i]);
    }
}

__global__ void zero_int(int* p) { *p = 0; }
__global__ void bump_int(int* p) { *p += 1; }

int vgrid(int n) {
    int g = (n + kBT - 1) / kBT;
    return g < 1 ? 1 : (g > 4096 ? 4096 : g);
}

}  // namespace

cudaError_t batch_dot(const long long* row_off, int count, const double* a, const double* b,
                      double* out, cudaStream_t s) {
    const int g = count < 4096 ? count : 4096;
    seg_dot<<<g < 1 ? 1 : g, kBT, 0, s>>>(row_off, count, a, b, out);
    return cudaGetLastError();
}

cudaError_t batch_scalars(const BatchScalars& B, int count, int op, double tol, cudaStream_t s) {
    if (op == 1 || op == 4) {
        zero_int<<<1, 1, 0, s>>>(op == 1 ? B.nactive : B.iter);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    const int g = (count + 127) / 128;
    seg_scalars<<<g < 1 ? 1 : g, 128, 0, s>>>(B, count, op, tol);
    return cudaGetLastError();
}

cudaError_t batch_bump(const BatchScalars& B, cudaStream_t s) {
    bump_int<<<1, 1, 0, s>>>(B.iter);
    return cudaGetLastError();
}

cudaError_t batch_xr(int n, const int* sys, const double* alpha, double* x, double* r, const double* p,
                     const double* q, cudaStream_t s) {
    seg_xr<<<vgrid(n), kBT, 0, s>>>(n, sys, alpha, x, r, p, q);
    return cudaGetLastError();
}

cudaError_t batch_p(int n, const int* sys, const double* beta, const int* active, double* p,
                    const double* z, cudaStream_t s) {
    seg_p<<<vgrid(n), kBT, 0, s>>>(n, sys, beta, active, p, z);
    return cudaGetLastError();
}

}  // namespace ick
