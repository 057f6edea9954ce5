// hx_simt.cu -- the precoder W = H X on the FP32 SIMT pipes (Eq. 7 without
// the power factor; Eq. 15 per symbol) and the finalise step that turns the
// per-tile ||W||_F^2 partials into beta = sqrt(P / ||W||_F^2) (Sec. II after
// Eq. 7) and the per-instance status.
//
// One CTA computes one TM x TN tile of W (TM = 64 rows of antennas, TN
// columns of users) of one instance, reducing over the K rows of X in
// chunks of KCH.  256 threads form a 16 (rows) x 16 (columns) grid, each
// owning a 4 x (TN / 16) complex micro-tile.  H chunks are staged without
// transposition (column-major chunks match the read pattern); X chunks
// are staged transposed.  The tile's contribution to ||W||_F^2 goes to its
// own slot, so the final sum runs in a fixed order.
#include "common.cuh"
#include "kernels.h"

namespace jacpcg {

namespace {

constexpr int TM = 64;
constexpr int KCH = 16;

template <int TN>
__global__ void __launch_bounds__(256) hx_simt_kernel(const DevInst *__restrict__ insts,
                                                      const int4 *__restrict__ tiles) {
    constexpr int UM = TM / 16, UN = TN / 16;
    __shared__ __align__(16) float2 Sh[KCH][TM];
    __shared__ __align__(16) float2 Sx[KCH][TN + 2];
    __shared__ float red[8];

    const int4 t = tiles[blockIdx.x];        // (instance, m tile, n tile, slot)
    const DevInst &in = insts[t.x];
    const int M = in.M, K = in.K, ldh = in.ldh, KC = in.KC, NCOL = in.ncols;
    const float2 *__restrict__ H = in.H;
    const float2 *__restrict__ X = in.X;
    const bool bf16 = in.h_bf16 != 0;
    const int m0 = t.y * TM, j0 = t.z * TN;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;

    float2 acc[UM][UN];
#pragma unroll
    for (int u = 0; u < UM; ++u)
#pragma unroll
        for (int v = 0; v < UN; ++v) acc[u][v] = make_float2(0.f, 0.f);

    // H chunk: KCH columns x TM rows = 1024 complex, 4 per thread (row-contiguous)
    // X chunk: KCH rows x TN columns, TN * KCH / 256 per thread
    constexpr int XL = TN * KCH / 256;
    float2 rh[4], rx[XL];
    auto fetch = [&](int k0) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = threadIdx.x + 256 * q;
            const int kk = e / TM, mm = e % TM;
            const int m = m0 + mm, k = k0 + kk;
            rh[q] = (m < M && k < K) ? load_h(H, bf16, m + (size_t)k * ldh) : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int q = 0; q < XL; ++q) {
            const int e = threadIdx.x + 256 * q;
            const int n = e / KCH, kk = e % KCH;
            const int k = k0 + kk, j = j0 + n;
            rx[q] = (k < K && j < NCOL) ? __ldg(X + k + (size_t)j * KC) : make_float2(0.f, 0.f);
        }
    };
    fetch(0);
    for (int k0 = 0; k0 < K; k0 += KCH) {
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = threadIdx.x + 256 * q;
            Sh[e / TM][e % TM] = rh[q];
        }
#pragma unroll
        for (int q = 0; q < XL; ++q) {
            const int e = threadIdx.x + 256 * q;
            Sx[e % KCH][e / KCH] = rx[q];
        }
        __syncthreads();
        if (k0 + KCH < K) fetch(k0 + KCH);
#pragma unroll
        for (int kk = 0; kk < KCH; ++kk) {
            float2 a[UM], b[UN];
#pragma unroll
            for (int u = 0; u < UM; ++u) a[u] = Sh[kk][ty * UM + u];
#pragma unroll
            for (int v = 0; v < UN; ++v) b[v] = Sx[kk][tx * UN + v];
#pragma unroll
            for (int u = 0; u < UM; ++u)
#pragma unroll
                for (int v = 0; v < UN; ++v) cfma(acc[u][v], a[u], b[v]);
        }
    }

    // store W and this tile's share of ||W||_F^2
    float2 *__restrict__ W = in.W;
    const int ldw = in.ldw;
    float nrm = 0.f;
#pragma unroll
    for (int v = 0; v < UN; ++v) {
        const int j = j0 + tx * UN + v;
#pragma unroll
        for (int u = 0; u < UM; ++u) {
            const int m = m0 + ty * UM + u;
            if (m < M && j < NCOL) {
                W[m + (size_t)j * ldw] = acc[u][v];
                nrm = fmaf(acc[u][v].x, acc[u][v].x, nrm);
                nrm = fmaf(acc[u][v].y, acc[u][v].y, nrm);
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = nrm;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.f;
#pragma unroll
        for (int w = 0; w < 8; ++w) s += red[w];
        in.wpart[t.w] = s;
    }
}

// One warp per instance: fixed-order sum of the tile partials, beta, status.
__global__ void finalize_kernel(const DevInst *__restrict__ insts, int n_inst, DevAccum acc,
                                DevOut out) {
    const int inst = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (inst >= n_inst) return;
    const DevInst &in = insts[inst];
    double s = 0.0;
    for (int e = lane; e < in.n_wpart; e += 32) s += (double)in.wpart[e];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane != 0) return;
    const int f = acc.flags[inst];
    int32_t st = 0;                                  // JACPCG_OK
    if (f & FLAG_TIMEOUT) st = 7;                    // JACPCG_ETIMEOUT
    else if (!isfinite(s)) st = 6;                   // JACPCG_ENONFINITE
    else if (f & FLAG_NOTHPD) st = 5;                // JACPCG_ENOTHPD
    else if (f & FLAG_NOTCONV) st = 4;               // JACPCG_ENOTCONV
    // Eq. 7: beta = sqrt(P / ||W||_F^2); for a block of n symbol vectors
    // (Eq. 15) the block's mean transmit power is normalised to P
    const double P = (in.power > 0.f ? (double)in.power : 1.0) * (in.B ? (double)in.ncols : 1.0);
    if (out.status) out.status[inst] = st;
    if (out.iters) out.iters[inst] = acc.iters[inst];
    if (out.resid) out.resid[inst] = __uint_as_float(acc.resid_bits[inst]);
    if (out.beta) out.beta[inst] = (s > 0.0 && isfinite(s)) ? (float)sqrt(P / s) : 0.f;
}

}  // namespace

cudaError_t launch_hx_simt(int TN, const DevInst *insts, const int4 *tiles, int n_tiles,
                           cudaStream_t s) {
    if (n_tiles <= 0) return cudaSuccess;
    switch (TN) {
        case 16: hx_simt_kernel<16><<<n_tiles, 256, 0, s>>>(insts, tiles); break;
        case 32: hx_simt_kernel<32><<<n_tiles, 256, 0, s>>>(insts, tiles); break;
        case 64: hx_simt_kernel<64><<<n_tiles, 256, 0, s>>>(insts, tiles); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_finalize(const DevInst *insts, int n_inst, DevAccum acc, DevOut out,
                            cudaStream_t s) {
    if (n_inst <= 0) return cudaSuccess;
    const int per = 8;   // warps per CTA
    finalize_kernel<<<(n_inst + per - 1) / per, per * 32, 0, s>>>(insts, n_inst, acc, out);
    return cudaGetLastError();
}

}  // namespace jacpcg
