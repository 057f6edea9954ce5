// refine.cu -- the true residual of iterative refinement, R = B - A X (B = I
// for the RZF precoder, else the caller's right-hand sides), and its
// per-instance norm history.  Two evaluations, both far more accurate than
// the FP32 iteration they correct:
//   FP64: every product and sum in FP64 (A and X are FP32, so each product
//         is exact in FP64);
//   DOT2: FP32 error-free transformations (TwoProduct by FMA, TwoSum), the
//         compensated dot product of Ogita, Rump and Oishi ("Accurate sum and
//         dot product", SIAM J. Sci. Comput. 26(6), 2005), whose result is as
//         accurate as if computed in twice the working precision; it runs on
//         the FP32 pipes, which on this GPU are far faster than FP64.
// No passage of the paper: the paper solves Eq. 16 by the iteration alone;
// refinement is the system layer that wins back accuracy lost to FP32 and
// to bfloat16 inputs.
#include "common.cuh"
#include "kernels.h"

namespace jacpcg {

namespace {

__device__ __forceinline__ double block_sum256(double v, double *red) {
    const int i = threadIdx.x;
    red[i] = v;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (i < o) red[i] += red[i + o];
        __syncthreads();
    }
    const double s = red[0];
    __syncthreads();
    return s;
}

// One block per (instance, column j), one thread per row i (K <= 256).
template <bool FP64>
__global__ void __launch_bounds__(256) residual_kernel(const DevInst *__restrict__ insts,
                                                       const int2 *__restrict__ blocks) {
    __shared__ double red[256];
    const int2 blk = blocks[blockIdx.x];
    const DevInst &in = insts[blk.x];
    const int K = in.K, KC = in.KC, j = blk.y, i = threadIdx.x;
    const float2 *__restrict__ A = in.A;
    const float2 *__restrict__ X = in.X;
    const int ldx = KC;
    float2 b = make_float2(0.f, 0.f);
    if (i < K) {
        if (in.B) b = in.B[i + (size_t)j * in.ldb];
        else if (i == j) b.x = 1.f;
    }
    double re = 0.0, im = 0.0;
    if (i < K) {
        if (FP64) {
            for (int k = 0; k < K; ++k) {
                const float2 a = A[i + (size_t)k * KC];
                const float2 x = X[k + (size_t)j * ldx];
                re = fma((double)a.x, (double)x.x, re);
                re = fma(-(double)a.y, (double)x.y, re);
                im = fma((double)a.x, (double)x.y, im);
                im = fma((double)a.y, (double)x.x, im);
            }
            re = (double)b.x - re;
            im = (double)b.y - im;
        } else {
            // (s, c) pairs: s the rounded sum, c the accumulated error terms
            Comp cr = {b.x, 0.f}, ci = {b.y, 0.f};
            for (int k = 0; k < K; ++k) {
                const float2 a = A[i + (size_t)k * KC];
                const float2 x = X[k + (size_t)j * ldx];
                comp_fma(cr, -a.x, x.x);
                comp_fma(cr, a.y, x.y);
                comp_fma(ci, -a.x, x.y);
                comp_fma(ci, -a.y, x.x);
            }
            re = (double)cr.s + (double)cr.c;
            im = (double)ci.s + (double)ci.c;
        }
    }
    if (i < KC) in.R[i + (size_t)j * KC] = make_float2((float)re, (float)im);
    const double rn = block_sum256(re * re + im * im, red);
    if (i == 0) in.rnorm[j] = (float)rn;
}

// One warp per instance: fixed-order sum of the column norms.
__global__ void resid_hist_kernel(const DevInst *__restrict__ insts, int n_inst, int sweep) {
    const int inst = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (inst >= n_inst) return;
    const DevInst &in = insts[inst];
    if (!in.resid_hist) return;
    double s = 0.0;
    for (int j = lane; j < in.ncols; j += 32) s += (double)in.rnorm[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) in.resid_hist[sweep] = (float)sqrt(s / in.ncols);
}

}  // namespace

cudaError_t launch_residual(const DevInst *insts, const int2 *blocks, int n_blocks, cudaStream_t s,
                            bool fp64) {
    if (n_blocks <= 0) return cudaSuccess;
    if (fp64)
        residual_kernel<true><<<n_blocks, 256, 0, s>>>(insts, blocks);
    else
        residual_kernel<false><<<n_blocks, 256, 0, s>>>(insts, blocks);
    return cudaGetLastError();
}

cudaError_t launch_resid_hist(const DevInst *insts, int n_inst, int sweep, cudaStream_t s) {
    if (n_inst <= 0) return cudaSuccess;
    resid_hist_kernel<<<(n_inst + 7) / 8, 256, 0, s>>>(insts, n_inst, sweep);
    return cudaGetLastError();
}

}  // namespace jacpcg
