// gram_simt.cu -- A = H^H H + xi I and the Jacobi diagonal 1 / A_kk on the
// FP32 SIMT pipes (Sec. II, definition of P_i after Eq. 7; the splitting
// P = D + L + L^H of Eq. 21 needs only D).
//
// One CTA computes one TB x TB tile (bi, bj), bi >= bj, of one instance's
// lower triangle, reducing over all M rows of H, and writes the tile and
// its conjugate transpose (A is Hermitian; a diagonal tile writes each pair
// (i, j), (j, i) from the i >= j entry, so A is exactly Hermitian and its
// diagonal exactly real).  256 threads form a 16 x 16 grid, each owning a
// U x U complex micro-tile (U = TB / 16).  H is staged through shared
// memory in chunks of MC rows, prefetched into registers one chunk ahead.
// Each stage's products are summed into a fresh partial that is then added
// to the running total (two-level summation: the rounding error grows with
// MC + M / MC terms rather than with M).
// ACC: every real product is accumulated as a compensated pair (TwoProduct
// by FMA and TwoSum; Ogita, Rump and Oishi 2005) and xi is added in FP64, so
// each entry of A is the exactly rounded FP32 value of H^H H + xi I up to a
// few units.  Refinement uses it for channels with few antennas per user,
// whose Jacobi-scaled condition numbers reach the thousands and would turn
// the rounding of a plain FP32 Gram into an error floor near 1e-5 in W.
#include "common.cuh"
#include "kernels.h"

namespace jacpcg {

namespace {

constexpr int MC = 32;  // H rows per stage

template <int TB, bool ACC>
__global__ void __launch_bounds__(256) gram_simt_kernel(const DevInst *__restrict__ insts,
                                                        const int4 *__restrict__ tiles,
                                                        DevAccum acc_out) {
    constexpr int U = TB / 16;
    constexpr int PITCH = TB + 2;       // complex per staged row
    constexpr int LOADS = MC * TB / 256; // complex per thread per stage and column set
    __shared__ __align__(16) float2 Si[MC][PITCH];
    __shared__ __align__(16) float2 Sj[MC][PITCH];

    const int4 t = tiles[blockIdx.x];
    const DevInst &in = insts[t.x];
    const int M = in.M, K = in.K, ldh = in.ldh, KC = in.KC;
    const float2 *__restrict__ H = in.H;
    const bool bf16 = in.h_bf16 != 0;
    const int i0 = t.y * TB, j0 = t.z * TB;
    const bool diag = (t.y == t.z);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;

    if (t.y == 0 && t.z == 0 && threadIdx.x == 0) {   // reset per-instance accumulators
        acc_out.flags[t.x] = 0;
        acc_out.iters[t.x] = 0;
        acc_out.resid_bits[t.x] = 0u;
    }

    float2 acc[U][U];
    Comp cre[ACC ? U : 1][ACC ? U : 1], cim[ACC ? U : 1][ACC ? U : 1];
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
        for (int v = 0; v < U; ++v) {
            acc[u][v] = make_float2(0.f, 0.f);
            if (ACC) cre[u][v] = cim[u][v] = Comp{0.f, 0.f};
        }

    // staging map: element e = threadIdx.x + 256 q -> column c = e / MC, row r = e % MC
    float2 ri[LOADS], rj[LOADS];
    auto fetch = [&](int m0) {
#pragma unroll
        for (int q = 0; q < LOADS; ++q) {
            const int e = threadIdx.x + 256 * q;
            const int c = e / MC, r = e % MC;
            const int m = m0 + r;
            const int ci = i0 + c, cj = j0 + c;
            ri[q] = (m < M && ci < K) ? load_h(H, bf16, m + (size_t)ci * ldh) : make_float2(0.f, 0.f);
            if (!diag)
                rj[q] = (m < M && cj < K) ? load_h(H, bf16, m + (size_t)cj * ldh) : make_float2(0.f, 0.f);
        }
    };
    const int Mloop = (i0 < K) ? M : 0;   // tiles wholly in the zero padding skip the reduction
    if (Mloop) fetch(0);
    for (int m0 = 0; m0 < Mloop; m0 += MC) {
        __syncthreads();
#pragma unroll
        for (int q = 0; q < LOADS; ++q) {
            const int e = threadIdx.x + 256 * q;
            const int c = e / MC, r = e % MC;
            Si[r][c] = ri[q];
            if (!diag) Sj[r][c] = rj[q];
        }
        __syncthreads();
        if (m0 + MC < Mloop) fetch(m0 + MC);
        float2(*Sb)[PITCH] = diag ? Si : Sj;
        if constexpr (ACC) {   // compensated: conj(a) b = (ar br + ai bi) + i (ar bi - ai br)
#pragma unroll 2
            for (int r = 0; r < MC; ++r) {
                float2 a[U], b[U];
#pragma unroll
                for (int u = 0; u < U; ++u) a[u] = Si[r][ty * U + u];
#pragma unroll
                for (int v = 0; v < U; ++v) b[v] = Sb[r][tx * U + v];
#pragma unroll
                for (int u = 0; u < U; ++u)
#pragma unroll
                    for (int v = 0; v < U; ++v) {
                        comp_fma(cre[u][v], a[u].x, b[v].x);
                        comp_fma(cre[u][v], a[u].y, b[v].y);
                        comp_fma(cim[u][v], a[u].x, b[v].y);
                        comp_fma(cim[u][v], -a[u].y, b[v].x);
                    }
            }
        } else {
            // two-level sum: a fresh partial per stage of MC rows, added to the total
            float2 part[U][U];
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int v = 0; v < U; ++v) part[u][v] = make_float2(0.f, 0.f);
#pragma unroll 4
            for (int r = 0; r < MC; ++r) {
                float2 a[U], b[U];
#pragma unroll
                for (int u = 0; u < U; ++u) a[u] = Si[r][ty * U + u];
#pragma unroll
                for (int v = 0; v < U; ++v) b[v] = Sb[r][tx * U + v];
#pragma unroll
                for (int u = 0; u < U; ++u)
#pragma unroll
                    for (int v = 0; v < U; ++v) cfma_conj(part[u][v], a[u], b[v]);
            }
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int v = 0; v < U; ++v) {
                    acc[u][v].x += part[u][v].x;
                    acc[u][v].y += part[u][v].y;
                }
        }
    }

    // write the tile (workspace has leading dimension KC, caller's A has K)
    float2 *__restrict__ A = in.A;
    float2 *__restrict__ Aout = in.Aout;
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int i = i0 + ty * U + u;
#pragma unroll
        for (int v = 0; v < U; ++v) {
            const int j = j0 + tx * U + v;
            if (i >= KC || j >= KC || i < j) continue;
            float2 a = acc[u][v];
            double dre = 0.0;   // ACC: the compensated sum, rounded once
            if (ACC) {
                dre = (double)cre[u][v].s + (double)cre[u][v].c;
                a = make_float2((float)dre, (float)((double)cim[u][v].s + (double)cim[u][v].c));
            }
            if (i == j) {
                a.y = 0.f;
                if (i < K) {
                    a.x = ACC ? (float)(dre + (double)in.xi) : a.x + in.xi;
                    in.dinv[i] = 1.0f / a.x;
                } else {
                    in.dinv[i] = 0.f;
                }
            }
            A[i + (size_t)j * KC] = a;
            A[j + (size_t)i * KC] = make_float2(a.x, -a.y);
            if (Aout && i < K && j < K) {
                Aout[i + (size_t)j * K] = a;
                Aout[j + (size_t)i * K] = make_float2(a.x, -a.y);
            }
        }
    }
}

}  // namespace

cudaError_t launch_gram_simt(int TB, const DevInst *insts, const int4 *tiles, int n_tiles,
                             DevAccum acc, cudaStream_t s, bool accurate) {
    if (n_tiles <= 0) return cudaSuccess;
    switch (TB * 2 + (accurate ? 1 : 0)) {
        case 32: gram_simt_kernel<16, false><<<n_tiles, 256, 0, s>>>(insts, tiles, acc); break;
        case 64: gram_simt_kernel<32, false><<<n_tiles, 256, 0, s>>>(insts, tiles, acc); break;
        case 128: gram_simt_kernel<64, false><<<n_tiles, 256, 0, s>>>(insts, tiles, acc); break;
        case 33: gram_simt_kernel<16, true><<<n_tiles, 256, 0, s>>>(insts, tiles, acc); break;
        case 65: gram_simt_kernel<32, true><<<n_tiles, 256, 0, s>>>(insts, tiles, acc); break;
        case 129: gram_simt_kernel<64, true><<<n_tiles, 256, 0, s>>>(insts, tiles, acc); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace jacpcg
