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
// Each evaluation also decides, per instance, whether refinement goes on:
// it stops once the largest relative column residual is at most refine_tol
// or no longer halves (the FP32 floor), and stopped instances skip the
// remaining correction solves and evaluations.
// No passage of the paper: the paper solves Eq. 16 by the iteration alone;
// refinement is the system layer that wins back accuracy lost to FP32 and
// to bfloat16 inputs.
#include "common.cuh"
#include "kernels.h"

namespace jacpcg {

namespace {

// One block per (instance, block of RES_CB columns j0 ..), one thread per row
// i (K <= 256).  Each thread carries the RES_CB residual entries of its row;
// rows k of X are staged in shared memory RES_KCH at a time and read as
// broadcasts, so A is read once per column block instead of once per column.
// Column norms: per-warp xor-butterfly sums, then the eight warp totals in a
// fixed order.
constexpr int RES_KCH = 32;

template <bool FP64>
__global__ void __launch_bounds__(256) residual_kernel(const DevInst *__restrict__ insts,
                                                       const int2 *__restrict__ blocks, int sweep) {
    constexpr int CB = RES_CB;
    __shared__ float2 Xs[RES_KCH][CB];
    __shared__ double red[2][8][CB];
    const int2 blk = blocks[blockIdx.x];
    const DevInst &in = insts[blk.x];
    if (sweep > 0 && in.rctl[1] != 0.f) return;   // stopped refining: R and its norms stand
    const int K = in.K, KC = in.KC, j0 = blk.y, i = threadIdx.x;
    const int nj = min(CB, in.ncols - j0);
    const float2 *__restrict__ A = in.A;
    const float2 *__restrict__ X = in.X;
    const int ldx = KC;
    float2 b[CB];
#pragma unroll
    for (int c = 0; c < CB; ++c) {
        b[c] = make_float2(0.f, 0.f);
        if (i < K && c < nj) {
            if (in.B) b[c] = in.B[i + (size_t)(j0 + c) * in.ldb];
            else if (i == j0 + c) b[c].x = 1.f;
        }
    }
    // FP64: plain FP64 sums; DOT2: (s, c) pairs, s the rounded sum, c the accumulated errors
    double dre[FP64 ? CB : 1], dim[FP64 ? CB : 1];
    Comp cre[FP64 ? 1 : CB], cim[FP64 ? 1 : CB];
#pragma unroll
    for (int c = 0; c < CB; ++c) {
        if (FP64) {
            dre[c] = 0.0;
            dim[c] = 0.0;
        } else {
            cre[c] = Comp{b[c].x, 0.f};
            cim[c] = Comp{b[c].y, 0.f};
        }
    }
    for (int k0 = 0; k0 < K; k0 += RES_KCH) {
        const int nk = min(RES_KCH, K - k0);
        __syncthreads();   // the previous chunk has been read
        for (int e = threadIdx.x; e < RES_KCH * CB; e += blockDim.x) {
            const int kk = e / CB, c = e % CB;
            Xs[kk][c] = (kk < nk && c < nj) ? X[(k0 + kk) + (size_t)(j0 + c) * ldx] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        if (i < K) {
#pragma unroll 4
            for (int kk = 0; kk < nk; ++kk) {
                const float2 a = A[i + (size_t)(k0 + kk) * KC];
#pragma unroll
                for (int c = 0; c < CB; ++c) {
                    const float2 x = Xs[kk][c];
                    if (FP64) {
                        dre[c] = fma((double)a.x, (double)x.x, dre[c]);
                        dre[c] = fma(-(double)a.y, (double)x.y, dre[c]);
                        dim[c] = fma((double)a.x, (double)x.y, dim[c]);
                        dim[c] = fma((double)a.y, (double)x.x, dim[c]);
                    } else {
                        comp_fma(cre[c], -a.x, x.x);
                        comp_fma(cre[c], a.y, x.y);
                        comp_fma(cim[c], -a.x, x.y);
                        comp_fma(cim[c], -a.y, x.x);
                    }
                }
            }
        }
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int c = 0; c < CB; ++c) {
        double re = 0.0, im = 0.0;
        if (i < K) {
            if (FP64) {
                re = (double)b[c].x - dre[c];
                im = (double)b[c].y - dim[c];
            } else {
                re = (double)cre[c].s + (double)cre[c].c;
                im = (double)cim[c].s + (double)cim[c].c;
            }
        }
        if (i < KC && c < nj) in.R[i + (size_t)(j0 + c) * KC] = make_float2((float)re, (float)im);
        double rn = re * re + im * im;
        double bn = (double)b[c].x * b[c].x + (double)b[c].y * b[c].y;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            rn += __shfl_xor_sync(0xffffffffu, rn, o);
            bn += __shfl_xor_sync(0xffffffffu, bn, o);
        }
        if (lane == 0) {
            red[0][warp][c] = rn;
            red[1][warp][c] = bn;
        }
    }
    __syncthreads();
    if (threadIdx.x < nj) {
        const int c = threadIdx.x, nw = blockDim.x >> 5;
        double rn = 0.0, bn = 0.0;
        for (int w = 0; w < nw; ++w) {
            rn += red[0][w][c];
            bn += red[1][w][c];
        }
        in.rnorm[j0 + c] = (float)rn;
        in.rnorm[KC + j0 + c] = (float)bn;
    }
}

// One warp per instance: fixed-order sum of the column norms for the history,
// and the stop decision.  An instance stops refining once its largest relative
// column residual (squared) is at most rtol2, or is above a quarter of its value
// at the previous evaluation (the residual norm did not halve: the FP32
// iteration's floor is reached, further sweeps only repeat the work).
__global__ void resid_hist_kernel(const DevInst *__restrict__ insts, int n_inst, int sweep) {
    const int inst = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (inst >= n_inst) return;
    const DevInst &in = insts[inst];
    if (in.no_refine) {   // selective policy: never evaluated, no correction solves
        if (lane == 0 && sweep == 0) {
            in.rctl[0] = 0.f;
            in.rctl[1] = 1.f;
        }
        return;
    }
    double s = 0.0;
    float rel = 0.f;
    for (int j = lane; j < in.ncols; j += 32) {
        const float rn = in.rnorm[j], bn = in.rnorm[in.KC + j];
        s += (double)rn;
        rel = fmaxf(rel, bn > 0.f ? rn / bn : rn);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        rel = fmaxf(rel, __shfl_xor_sync(0xffffffffu, rel, o));
    }
    if (lane != 0) return;
    if (in.resid_hist) in.resid_hist[sweep] = (float)sqrt(s / in.ncols);
    float *c = in.rctl;
    if (sweep == 0) {
        c[1] = (in.rtol2 > 0.f && rel <= in.rtol2) ? 1.f : 0.f;
        c[0] = rel;
    } else if (c[1] == 0.f) {
        if (in.rtol2 > 0.f && (rel <= in.rtol2 || rel > 0.25f * c[0])) c[1] = 1.f;
        c[0] = rel;
    }
}

}  // namespace

cudaError_t launch_residual(const DevInst *insts, const int2 *blocks, int n_blocks, int sweep,
                            cudaStream_t s, bool fp64) {
    if (n_blocks <= 0) return cudaSuccess;
    if (fp64)
        residual_kernel<true><<<n_blocks, 256, 0, s>>>(insts, blocks, sweep);
    else
        residual_kernel<false><<<n_blocks, 256, 0, s>>>(insts, blocks, sweep);
    return cudaGetLastError();
}

cudaError_t launch_resid_hist(const DevInst *insts, int n_inst, int sweep, cudaStream_t s) {
    if (n_inst <= 0) return cudaSuccess;
    resid_hist_kernel<<<(n_inst + 7) / 8, 256, 0, s>>>(insts, n_inst, sweep);
    return cudaGetLastError();
}

}  // namespace jacpcg
