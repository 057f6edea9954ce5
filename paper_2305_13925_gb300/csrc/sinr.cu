// sinr.cu -- per-user SINR of the precoder just formed (Eq. 9 in its
// centralised form for single-antenna users, G = beta W):
//   gamma_k = beta^2 |h_k^H w_k|^2 / (beta^2 sum_{j != k} |h_k^H w_j|^2 + sigma^2),
// from which the sum SE of Eq. 10 is sum_k log2(1 + gamma_k).  An optional
// output of the batched path (instance field `sinr`, B = I only), run after
// W = H X and the power factor, so the SE comes from the GPU's own W.
//
// One CTA per (instance, block of 8 users); warp u owns user k = 8 b + u and
// lane l the precoder columns j = l, l + 32, ...  Tiles of TM antennas of the
// 8 users' channels and of all K columns of W are staged in shared memory
// (W column-major with padded rows, so lane reads are conflict-free), and the
// products h_k^H w_j accumulate as compensated (Dot2) sums.  W is re-read
// from L2 once per user block.  beta is recomputed from the instance's
// ||W||_F^2 partials exactly as the finalise kernel sums them.
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"

namespace jacpcg {
namespace {

constexpr int SU = 8;     // users per CTA (one warp each)
constexpr int STM = 32;   // antennas per staged tile

template <int KC>
__global__ void __launch_bounds__(SU * 32) sinr_kernel(const DevInst *__restrict__ insts,
                                                      const int2 *__restrict__ jobs) {
    constexpr int NJ = KC >= 32 ? KC / 32 : 1;   // columns per lane
    constexpr int WLD = STM + 1;
    __shared__ float2 Hs[SU][STM];
    extern __shared__ float2 Ws[];               // KC x WLD
    const int2 job = jobs[blockIdx.x];
    const DevInst &in = insts[job.x];
    const int K = in.K, M = in.M;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int k = job.y * SU + warp;

    Comp gr[NJ], gi[NJ];
#pragma unroll
    for (int c = 0; c < NJ; ++c) gr[c] = gi[c] = Comp{0.f, 0.f};
    for (int m0 = 0; m0 < M; m0 += STM) {
        for (int e = threadIdx.x; e < SU * STM; e += SU * 32) {
            const int r = e % STM, u = e / STM, kk = job.y * SU + u;
            Hs[u][r] = (kk < K && m0 + r < M) ? load_h(in.H, in.h_bf16, (size_t)(m0 + r) + (size_t)kk * in.ldh)
                                              : make_float2(0.f, 0.f);
        }
        for (int e = threadIdx.x; e < KC * STM; e += SU * 32) {
            const int r = e % STM, j = e / STM;
            Ws[j * WLD + r] = (j < K && m0 + r < M) ? in.W[(size_t)(m0 + r) + (size_t)j * in.ldw]
                                                    : make_float2(0.f, 0.f);
        }
        __syncthreads();
#pragma unroll 4
        for (int r = 0; r < STM; ++r) {
            const float2 h = Hs[warp][r];
#pragma unroll
            for (int c = 0; c < NJ; ++c) {
                const int j = lane + 32 * c;
                if (KC < 32 && j >= KC) continue;
                const float2 w = Ws[j * WLD + r];
                // conj(h) w = (hr wr + hi wi) + i (hr wi - hi wr)
                comp_fma(gr[c], h.x, w.x);
                comp_fma(gr[c], h.y, w.y);
                comp_fma(gi[c], h.x, w.y);
                comp_fma(gi[c], -h.y, w.x);
            }
        }
        __syncthreads();
    }
    // signal and interference powers of user k
    float sig = 0.f;
    Comp intf = {0.f, 0.f};
#pragma unroll
    for (int c = 0; c < NJ; ++c) {
        const int j = lane + 32 * c;
        if (j >= K) continue;
        const float a = gr[c].s + gr[c].c, b = gi[c].s + gi[c].c;
        if (j == k) {
            sig = fmaf(a, a, b * b);
        } else {
            comp_fma(intf, a, a);
            comp_fma(intf, b, b);
        }
    }
    intf = comp_warp_allreduce(intf);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sig += __shfl_xor_sync(0xffffffffu, sig, o);   // one lane holds it
    // ||W||_F^2 as the finalise kernel sums it, then beta^2 = P / ||W||_F^2
    double s = 0.0;
    for (int e = lane; e < in.n_wpart; e += 32) s += (double)in.wpart[e];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane != 0 || k >= K) return;
    const double P = in.power > 0.f ? (double)in.power : 1.0;
    const double b2 = (s > 0.0 && isfinite(s)) ? P / s : 0.0;
    const double sigma2 = in.noise > 0.f ? (double)in.noise : 1.0;
    in.sinr[k] = (float)(b2 * (double)sig / (b2 * ((double)intf.s + (double)intf.c) + sigma2));
}

template <int KC>
cudaError_t launch_class(const DevInst *insts, const int2 *jobs, int n, cudaStream_t s) {
    const size_t smem = sizeof(float2) * (size_t)KC * (STM + 1);
    auto kern = sinr_kernel<KC>;
    if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<n, SU * 32, smem, s>>>(insts, jobs);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_sinr(int KC, const DevInst *insts, const int2 *jobs, int n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    switch (KC) {
        case 8: return launch_class<8>(insts, jobs, n, s);
        case 16: return launch_class<16>(insts, jobs, n, s);
        case 32: return launch_class<32>(insts, jobs, n, s);
        case 64: return launch_class<64>(insts, jobs, n, s);
        case 128: return launch_class<128>(insts, jobs, n, s);
        case 256: return launch_class<256>(insts, jobs, n, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace jacpcg
