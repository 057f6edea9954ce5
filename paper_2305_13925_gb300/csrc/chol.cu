// chol.cu -- the direct RZF of the Appendix on the GPU: P = L L^H (Cholesky),
// then X = P^{-1} B by forward substitution (L Y = B) and back substitution
// (L^H X = Y); B = I gives the inverse the RZF of Eq. 7 multiplies by.  It is
// the comparator the paper measures Jac-PCG against (its operation counts,
// Appendix), run as one more variant of the batched path: the Gram and
// W = H X phases are the path's own kernels, this kernel replaces the
// iteration.
//
// One CTA per instance.  The factorisation is right-looking: for each pivot
// column j, the pivot is checked (P must be positive definite: a pivot <= 0
// flags the instance NOTHPD and leaves X = 0), column j below the diagonal is
// scaled by 1 / l_jj, and the trailing lower triangle takes the rank-one
// update a_ik -= l_ij conj(l_kj); one barrier after each of the two steps.
// For the 8 ... 128 classes L lives in shared memory (K x (K + 1) complex,
// at most 129 KB); for the 256 class (512 KB) it is factorised in place in
// the instance's workspace A, which the L2 holds (the direct variant keeps no
// other use for A after the Gram phase: refinement is not offered with it).
// The solves give each warp whole right-hand-side columns: lane l holds rows
// l, l + 32, ... of its column in registers, the pivot row's value is
// broadcast by a shuffle, and every lane updates its rows -- column-oriented
// substitution, so L is read by columns in the forward solve (conflict-free)
// and by rows in the back solve.
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"

namespace jacpcg {
namespace {

constexpr int CH_THREADS = 512;

template <int KC, bool SMEM>
__global__ void __launch_bounds__(CH_THREADS) chol_kernel(const DevInst *__restrict__ insts,
                                                         const int *__restrict__ list, DevAccum acc) {
    constexpr int LD = SMEM ? KC + 1 : KC;   // padded rows in shared memory
    constexpr int RPL = KC >= 32 ? KC / 32 : 1;
    extern __shared__ __align__(16) float2 lsm[];
    __shared__ int bad;
    const int id = list[blockIdx.x];
    const DevInst &in = insts[id];
    const int K = in.K;
    float2 *L = SMEM ? lsm : in.A;
    if (threadIdx.x == 0) bad = 0;
    if (SMEM) {
        for (int e = threadIdx.x; e < K * K; e += CH_THREADS) {
            const int i = e % K, j = e / K;
            L[i + j * LD] = in.A[i + (size_t)j * KC];
        }
    }
    __syncthreads();

    // ---- factorisation, right-looking ----
    for (int j = 0; j < K; ++j) {
        const float d = L[j + j * LD].x;
        if (!(d > 0.f)) {   // uniform: every thread reads the same pivot
            if (threadIdx.x == 0) bad = 1;
            break;
        }
        const float inv = rsqrtf(d);
        for (int i = j + 1 + threadIdx.x; i < K; i += CH_THREADS) {
            const float2 v = L[i + j * LD];
            L[i + j * LD] = make_float2(v.x * inv, v.y * inv);
        }
        __syncthreads();
        if (threadIdx.x == 0) L[j + j * LD] = make_float2(d * inv, 0.f);   // l_jj = sqrt(d)
        const int n = K - j - 1;
        for (int e = threadIdx.x; e < n * n; e += CH_THREADS) {
            const int i = j + 1 + e % n, k = j + 1 + e / n;
            if (i < k) continue;   // lower triangle only
            const float2 a = L[i + j * LD], b = L[k + j * LD];
            float2 &t = L[i + k * LD];
            t.x -= a.x * b.x + a.y * b.y;   // a_ik -= l_ij conj(l_kj)
            t.y -= a.y * b.x - a.x * b.y;
        }
        __syncthreads();
    }
    __syncthreads();
    const bool failed = bad != 0;

    // ---- solves, one warp per right-hand-side column ----
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ncols = in.ncols;
    for (int c = warp; c < ncols; c += CH_THREADS / 32) {
        float2 y[RPL];
#pragma unroll
        for (int r = 0; r < RPL; ++r) {
            const int i = lane + 32 * r;
            float2 b = make_float2(0.f, 0.f);
            if (i < K) {
                if (!in.B) b.x = (i == c) ? 1.f : 0.f;
                else b = in.B[i + (size_t)c * in.ldb];
            }
            y[r] = b;
        }
        if (!failed) {
            // L y = b: y_k = b_k / l_kk, then b_i -= l_ik y_k for i > k
            for (int k = 0; k < K; ++k) {
                const int ok = k & 31, rk = k >> 5;
                float2 yk = make_float2(0.f, 0.f);
#pragma unroll
                for (int r = 0; r < RPL; ++r)
                    if (r == rk) yk = y[r];
                yk.x = __shfl_sync(0xffffffffu, yk.x, ok);
                yk.y = __shfl_sync(0xffffffffu, yk.y, ok);
                const float inv = 1.f / L[k + k * LD].x;
                yk = make_float2(yk.x * inv, yk.y * inv);
#pragma unroll
                for (int r = 0; r < RPL; ++r) {
                    const int i = lane + 32 * r;
                    if (i == k) y[r] = yk;
                    else if (i > k && i < K) {
                        const float2 l = L[i + k * LD];
                        y[r].x -= l.x * yk.x - l.y * yk.y;
                        y[r].y -= l.x * yk.y + l.y * yk.x;
                    }
                }
            }
            // L^H x = y: x_k = y_k / l_kk, then y_i -= conj(l_ki) x_k for i < k
            for (int k = K - 1; k >= 0; --k) {
                const int ok = k & 31, rk = k >> 5;
                float2 xk = make_float2(0.f, 0.f);
#pragma unroll
                for (int r = 0; r < RPL; ++r)
                    if (r == rk) xk = y[r];
                xk.x = __shfl_sync(0xffffffffu, xk.x, ok);
                xk.y = __shfl_sync(0xffffffffu, xk.y, ok);
                const float inv = 1.f / L[k + k * LD].x;
                xk = make_float2(xk.x * inv, xk.y * inv);
#pragma unroll
                for (int r = 0; r < RPL; ++r) {
                    const int i = lane + 32 * r;
                    if (i == k) y[r] = xk;
                    else if (i < k) {
                        const float2 l = L[k + i * LD];   // conj(l_ki)
                        y[r].x -= l.x * xk.x + l.y * xk.y;
                        y[r].y -= l.x * xk.y - l.y * xk.x;
                    }
                }
            }
        }
#pragma unroll
        for (int r = 0; r < RPL; ++r) {
            const int i = lane + 32 * r;
            if (i >= KC) continue;
            const float2 v = (failed || i >= K) ? make_float2(0.f, 0.f) : y[r];
            in.X[i + (size_t)c * KC] = v;
            if (in.Xout && i < K) in.Xout[i + (size_t)c * K] = v;
        }
    }
    if (threadIdx.x == 0 && failed) atomicOr(acc.flags + id, FLAG_NOTHPD);
}

template <int KC, bool SMEM>
cudaError_t launch_class(const DevInst *insts, const int *list, int n, DevAccum acc, cudaStream_t s) {
    const size_t smem = SMEM ? sizeof(float2) * (size_t)KC * (KC + 1) : 0;
    auto kern = chol_kernel<KC, SMEM>;
    if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<n, CH_THREADS, smem, s>>>(insts, list, acc);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_chol(int KC, const DevInst *insts, const int *list, int n, DevAccum acc, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    switch (KC) {
        case 8: return launch_class<8, true>(insts, list, n, acc, s);
        case 16: return launch_class<16, true>(insts, list, n, acc, s);
        case 32: return launch_class<32, true>(insts, list, n, acc, s);
        case 64: return launch_class<64, true>(insts, list, n, acc, s);
        case 128: return launch_class<128, true>(insts, list, n, acc, s);
        case 256: return launch_class<256, false>(insts, list, n, acc, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace jacpcg
