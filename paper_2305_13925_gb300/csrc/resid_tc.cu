// resid_tc.cu -- the refinement residual R = B - A X on the tcgen05 tensor
// cores for the K = 128 and 256 classes, with error-free sliced products (the
// Ozaki scheme on tensor cores: Mukunoki, Ozaki, Ogita and Imamura, "DGEMM
// using Tensor Cores, and Its Accurate and Reproducible Versions", ISC 2020).
//
// The products are balanced first, with the same exact powers of two as the
// tensor-core iteration: Ah = E^-1 A E^-1 and Xh = E X E, E = diag(2^e_i),
// 2^e_i <= sqrt(A_ii) < 2^(e_i + 1), so that A X = E (Ah Xh) E^-1 and every
// entry of Ah and of the columns of Xh is of order one whatever the users'
// gains (slicing A and X directly, on grids set by their own rows and columns,
// left errors of order sqrt(A_ii / A_jj) too coarse).  Every row i of Ah and
// every column j of Xh is then cut into five 8-bit integer slices on a
// fixed-point grid of its own:
//   Ah_ik = 2^ga_i (a0 2^-7 + a1 2^-15 + ... + a4 2^-39 + ...),
//   Xh_kj = 2^gx_j (x0 2^-7 + x1 2^-15 + ...),   |a_s|, |x_t| <= 128,
// 2^ga_i above row i's largest |Re|, |Im| (and 2^gx_j above column j's), each
// slice the rounding of what the previous ones leave.  The slices are exact
// FP16 integers and a slice product an integer of at most 2^14; the classes
// c = s + t = 0..4 (fifteen slice pairs) are kept, each summed over k in one
// TMEM accumulator.  For c <= 3 the sum of at most four pairs over K <= 256
// terms stays within 2^24, so the tensor core's FP32 accumulation is exact
// whatever its order or truncation; the top class (five pairs) could round one
// unit, 2^-46 of the grid.  The first dropped class weighs 2^-48 of the
// leading products; on the bench channels the residual comes out within 1e-4
// of its own size (four slices: 2e-2).  The classes leave TMEM as integers and
// are combined, with B, by TwoSum in FP32 pairs (the compensated sums of
// Ogita, Rump and Oishi, 2005), rounded once into R.
//
// Complex products as planar real MMAs, as in the tensor-core iteration:
// U_c = Ar^(s) [Xr^(t) | Xi^(t)] and V_c = Ai^(s) [Xr^(t) | Xi^(t)] summed over
// the pairs of class c, Re AX = U[.., Xr] - V[.., Xi], Im AX = U[.., Xi] + V[.., Xr].
//
// A job is (instance, 24 columns).  Once per execute a prep kernel stores Ah's
// slices as MMA-ready FP16 stages (row tile rt, slice s, k-step ks: [Ar^(s) |
// Ai^(s)], 128 x 16 each, canonical no-swizzle K-major, 8 KB); the job's five
// Xh slices (B operand: 48 rows [Xr^T ; Xi^T] x KC, 120 KB at K = 256) are
// built by the epilogue warps at the start of the job.  Per row tile the A
// stages stream slice by slice through a ring of bulk copies; after slice s,
// class s is complete, so the epilogue drains it while the next slice streams.
// The five classes hold 2 x 5 x 48 TMEM columns (all U, then all V); the
// X slices' B rows follow each other, so slice s of A meets X slices 1 ..
// NSL - s in one MMA of N = 48 (NSL - s) into classes s .. 4 (one for U, one
// for V: two MMAs per k-step instead of ten).
//
// Roles: warps 0-7 build B, then drain the classes (TMEM lanes 32 (w mod 4)
// .., columns 12 (w / 4) .. of the job) and write R and the column norms;
// warp 8 lane 0 issues the bulk copies; warp 9 allocates TMEM, lane 0 issues
// the MMAs.  Every wait is bounded; a timeout flags the CTA's instances with
// FLAG_TIMEOUT, and the CTA still drains and frees its TMEM.
#include <cuda_fp16.h>

#include "common.cuh"
#include "kernels.h"
#include "tc.cuh"

namespace jacpcg {

namespace {

constexpr int NB = 24;                 // columns per job
constexpr int BR = 2 * NB;             // B rows: Xr^T then Xi^T (MMA N = 48)
constexpr int NSL = 5;                 // slices per row of Ah and per column of Xh
constexpr int NCLS = NSL;              // classes s + t = 0 .. 4
constexpr int CPT = NB / 2;            // columns per epilogue thread
constexpr int TILE = 128 * 16 * 2;     // one 128 x 16 FP16 tile (4 KB)
constexpr int STAGE = 2 * TILE;        // [Ar^(s) | Ai^(s)] of one k-step
constexpr int SUB = 4;                 // k-steps per bulk copy (ring slot)
constexpr int SLOT = SUB * STAGE;      // 32 KB
constexpr int RING = 3;
constexpr int NEW = 8;                 // epilogue warps
constexpr int TMA_WARP = NEW, MMA_WARP = NEW + 1;
constexpr int NTHREADS = (NEW + 2) * 32;
constexpr int TMEM_COLS = 512;         // NCLS x (U | V) = 480 used
constexpr uint32_t WAIT_LIMIT = 1u << 21;
constexpr int BAR_EPI = 1;

template <int KC>
struct RCfg {
    static_assert(KC / 16 % SUB == 0, "whole slots per slice");
    static constexpr int RT = KC / 128;                  // row tiles
    static constexpr int KS = KC / 16;                   // k-steps per row tile
    static constexpr uint32_t SBO_B = (KC / 8) * 128;    // bytes between 8-row groups of B
    static constexpr int BSL = BR * KC * 2;              // one X slice of B (32 KB at K = 256)
};

struct __align__(128) RSmem {
    unsigned char B[NSL][BR * 256 * 2];    // sized for K = 256
    unsigned char ring[RING][SLOT];
    float cmax[NEW][NB];                   // column maxima of E X, per epilogue warp
    float xs[NB];                          // 2^-(gx_j - e_j): the column's output scale, inverted
    float xsi[NB];                         // 2^(gx_j - e_j)
    float xe[NB];                          // 2^e_j
    float nr[4][NB], nb[4][NB];            // column norm partials per TMEM lane quarter
    uint64_t full[RING], empty[RING];
    uint64_t accf[NCLS], tfree[NCLS];
    uint64_t bready, fin;
    uint32_t tmem;
    volatile int err;
};
static_assert(sizeof(RSmem) <= 227 * 1024, "shared memory");
static_assert(NCLS * 2 * BR <= TMEM_COLS, "tensor memory");

// 2^v, v in [-126, 127]
__device__ __forceinline__ float p2(int v) { return __uint_as_float((uint32_t)(v + 127) << 23); }
// the grid exponent of a row / column whose largest magnitude is m: 2^e > m
// (e in [-100, 100]; 0 for an all-zero row)
__device__ __forceinline__ int grid_exp(float m) {
    if (!(m > 0.f)) return 0;
    const int e = (int)((__float_as_uint(m) >> 23) & 0xFFu) - 126;   // m < 2^e
    return max(-100, min(100, e));
}
// 2^e <= sqrt(aii) < 2^(e + 1): the balancing exponent of row i (0 for padding rows)
__device__ __forceinline__ int bal_exp(float aii) {
    if (!(aii >= 1.2e-38f) || !(aii < 3.0e38f)) return 0;
    return (int)((__float_as_uint(sqrtf(aii)) >> 23) & 0xFFu) - 127;
}
// v (|v| < 2^e) -> five 8-bit integer slices of v 2^-e on the grid 2^-7, 2^-15, ...
__device__ __forceinline__ void slice5(float v, float s_inv_lo, float s_inv_hi, __half (&o)[NSL]) {
    float x = (v * s_inv_lo) * s_inv_hi * 128.f;   // v 2^(7 - e), |x| < 128: exact
#pragma unroll
    for (int s = 0; s < NSL; ++s) {
        const float q = rintf(x);
        o[s] = __float2half_rn(q);                 // an integer of magnitude <= 128: exact
        x = (x - q) * 256.f;                       // exact
    }
}
__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float b) {
    const float s = hi + b, z = s - hi;
    lo += (hi - (s - z)) + (b - z);
    hi = s;
}

__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(tc::smem_u32(bar))
        : "memory");
}

// ---------------------------------------------------------------------------
// Ah's slices: one CTA per (instance, row tile); per row i DevInst::rexp holds
// e_i + ga_i (the row's output scale) and rexp[KC + i] holds e_i; the stages
// (rt, s, ks) go to DevInst::Asl.
template <int KC>
__global__ void __launch_bounds__(256) rtc_prep_kernel(const DevInst *__restrict__ insts, const int *__restrict__ list) {
    using C = RCfg<KC>;
    __shared__ float m2[2][128];
    __shared__ float cinv[KC];   // 2^-e_k of every column
    __shared__ int ga[128], eb[128];
    const int id = list[blockIdx.x / C::RT], rt = blockIdx.x % C::RT;
    const DevInst &in = insts[id];
    const float2 *__restrict__ A = in.A;
    const int t = threadIdx.x, r = t & 127, half = t >> 7;
    for (int k = t; k < KC; k += 256) cinv[k] = p2(-bal_exp(A[(size_t)k * (KC + 1)].x));
    __syncthreads();
    const int gi = rt * 128 + r;
    const float ri = p2(-bal_exp(A[(size_t)gi * (KC + 1)].x));
    float m = 0.f;
#pragma unroll 8
    for (int k = half * (KC / 2); k < (half + 1) * (KC / 2); ++k) {
        const float2 v = A[(size_t)gi + (size_t)k * KC];
        m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)) * ri * cinv[k]);   // exact scalings
    }
    m2[half][r] = m;
    __syncthreads();
    if (t < 128) {
        const int e = bal_exp(A[(size_t)(rt * 128 + t) * (KC + 1)].x);
        ga[t] = grid_exp(fmaxf(m2[0][t], m2[1][t]));
        eb[t] = e;
        in.rexp[rt * 128 + t] = (float)(e + ga[t]);
        in.rexp[KC + rt * 128 + t] = (float)e;
    }
    __syncthreads();
    // thread t: row rr = t mod 128 and the 8 columns 8 kh .. of each 16-column
    // k-step, one 16-byte store per slice and part (rows of a core matrix)
    char *dst0 = reinterpret_cast<char *>(in.Asl) + (size_t)rt * NSL * C::KS * STAGE;
    const int rr = t & 127, kh = t >> 7;
    const float rs0 = p2(-eb[rr]), g = p2(-ga[rr]);
    const uint32_t o = (uint32_t)(rr >> 3) * 256u + (uint32_t)kh * 128u + (uint32_t)(rr & 7) * 16u;
    for (int ks = 0; ks < C::KS; ++ks) {
        uint32_t wr[NSL][4], wi[NSL][4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int k0 = ks * 16 + 8 * kh + 2 * q;
            const float2 v0 = A[(size_t)(rt * 128 + rr) + (size_t)k0 * KC];
            const float2 v1 = A[(size_t)(rt * 128 + rr) + (size_t)(k0 + 1) * KC];
            const float s0 = rs0 * cinv[k0], s1 = rs0 * cinv[k0 + 1];   // 2^(-e_i - e_k)
            __half a0[NSL], a1[NSL], b0[NSL], b1[NSL];
            slice5(v0.x * s0, g, 1.f, a0);
            slice5(v1.x * s1, g, 1.f, a1);
            slice5(v0.y * s0, g, 1.f, b0);
            slice5(v1.y * s1, g, 1.f, b1);
#pragma unroll
            for (int s = 0; s < NSL; ++s) {
                wr[s][q] = (uint32_t)__half_as_ushort(a0[s]) | ((uint32_t)__half_as_ushort(a1[s]) << 16);
                wi[s][q] = (uint32_t)__half_as_ushort(b0[s]) | ((uint32_t)__half_as_ushort(b1[s]) << 16);
            }
        }
#pragma unroll
        for (int s = 0; s < NSL; ++s) {
            char *st = dst0 + ((size_t)s * C::KS + ks) * STAGE + o;
            *reinterpret_cast<uint4 *>(st) = make_uint4(wr[s][0], wr[s][1], wr[s][2], wr[s][3]);
            *reinterpret_cast<uint4 *>(st + TILE) = make_uint4(wi[s][0], wi[s][1], wi[s][2], wi[s][3]);
        }
    }
}

template <int KC>
__global__ void __launch_bounds__(NTHREADS, 1) resid_tc_kernel(const DevInst *__restrict__ insts,
                                                               const int2 *__restrict__ jobs, int n_jobs, int sweep,
                                                               DevAccum acc_out) {
    using C = RCfg<KC>;
    extern __shared__ unsigned char smem_raw[];
    const uint32_t pad = (128u - (tc::smem_u32(smem_raw) & 127u)) & 127u;
    RSmem &S = *reinterpret_cast<RSmem *>(smem_raw + pad);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int i = 0; i < RING; ++i) {
            tc::mbar_init(&S.full[i], 1);
            tc::mbar_init(&S.empty[i], 1);
        }
        for (int c = 0; c < NCLS; ++c) {
            tc::mbar_init(&S.accf[c], 1);
            tc::mbar_init(&S.tfree[c], NEW);
        }
        tc::mbar_init(&S.bready, NEW);
        tc::mbar_init(&S.fin, 1);
        S.err = 0;
        tc::mbar_init_fence();
    }
    if (warp == MMA_WARP) {
        tc::tmem_alloc(&S.tmem, TMEM_COLS);
        tc::tmem_relinquish();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = S.tmem;
    const uint32_t b0 = tc::smem_u32(S.B[0]), ring0 = tc::smem_u32(S.ring[0]);

    if (warp < NEW) {
        // ---------------- B from X, then the class drains and R ----------------
        const int t = threadIdx.x, quad = warp & 3, part = warp >> 2;
        uint32_t use = 0;   // (job, row tile) passes drained so far
        // every epilogue warp walks every job and row tile (named barriers)
        for (int jj = blockIdx.x; jj < n_jobs; jj += gridDim.x) {
            const int2 job = jobs[jj];
            const DevInst &in = insts[job.x];
            if (sweep > 0 && in.rctl[1] != 0.f) continue;   // uniform: every role skips it
            const int K = in.K, ncols = in.ncols, j0 = job.y;
            const float2 *__restrict__ X = in.X;
            const float *__restrict__ eks = in.rexp + KC;   // e_k of every row
            // column maxima of E X over the K rows (the job's columns): thread t takes
            // rows t, t + 256, ... of every column (coalesced), then the warp's and
            // the eight warps' maxima
            {
                float m[NB];
#pragma unroll
                for (int jl = 0; jl < NB; ++jl) m[jl] = 0.f;
                for (int k = t; k < K; k += NEW * 32) {
                    const float ek = p2((int)eks[k]);
#pragma unroll
                    for (int jl = 0; jl < NB; ++jl)
                        if (j0 + jl < ncols) {
                            const float2 v = X[k + (size_t)(j0 + jl) * KC];
                            m[jl] = fmaxf(m[jl], fmaxf(fabsf(v.x), fabsf(v.y)) * ek);
                        }
                }
#pragma unroll
                for (int jl = 0; jl < NB; ++jl) {
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) m[jl] = fmaxf(m[jl], __shfl_xor_sync(0xffffffffu, m[jl], o));
                    if (lane == 0) S.cmax[warp][jl] = m[jl];
                }
            }
            asm volatile("bar.sync %0, %1;\n" ::"r"(BAR_EPI), "r"(NEW * 32) : "memory");
            if (t < NB) {
                float m = 0.f;
#pragma unroll
                for (int w = 0; w < NEW; ++w) m = fmaxf(m, S.cmax[w][t]);
                const int ej = (j0 + t < KC) ? (int)eks[j0 + t] : 0;
                const int gx = grid_exp(m * p2(ej));   // grid of column j of Xh = E X E
                S.xs[t] = p2(ej - gx);                  // Xh's grid unit 2^-gx, applied to E X
                S.xsi[t] = p2(gx - ej);
            }
            asm volatile("bar.sync %0, %1;\n" ::"r"(BAR_EPI), "r"(NEW * 32) : "memory");
            // the slices: item (row n of B, 8 values k); 16 bytes per slice
            for (int e = t; e < NB * (KC / 8); e += NEW * 32) {
                const int r8 = e & 7, kg = (e >> 3) % (KC / 8), ng = (e >> 3) / (KC / 8);
                const int nl = 8 * ng + r8, n = j0 + nl;
                uint32_t wr[NSL][4], wi[NSL][4];
                const float sx = S.xs[nl];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                    const int k = 8 * kg + 2 * q;
                    float e0 = 0.f, e1 = 0.f;   // 2^e_k of the two rows
                    if (n < ncols && k < K) {
                        v = *reinterpret_cast<const float4 *>(X + k + (size_t)n * KC);
                        e0 = p2((int)eks[k]);
                        if (k + 1 >= K) v.z = v.w = 0.f;
                        else e1 = p2((int)eks[k + 1]);
                    }
                    __half r0[NSL], r1[NSL], i0[NSL], i1[NSL];
                    slice5(v.x * e0, sx, 1.f, r0);
                    slice5(v.z * e1, sx, 1.f, r1);
                    slice5(v.y * e0, sx, 1.f, i0);
                    slice5(v.w * e1, sx, 1.f, i1);
#pragma unroll
                    for (int s = 0; s < NSL; ++s) {
                        wr[s][q] = (uint32_t)__half_as_ushort(r0[s]) | ((uint32_t)__half_as_ushort(r1[s]) << 16);
                        wi[s][q] = (uint32_t)__half_as_ushort(i0[s]) | ((uint32_t)__half_as_ushort(i1[s]) << 16);
                    }
                }
#pragma unroll
                for (int s = 0; s < NSL; ++s) {
                    const uint32_t base = b0 + s * C::BSL + kg * 128 + r8 * 16;
                    const uint32_t ar = base + ng * C::SBO_B, ai = base + (NB / 8 + ng) * C::SBO_B;
                    asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};\n" ::"r"(ar), "r"(wr[s][0]), "r"(wr[s][1]),
                                 "r"(wr[s][2]), "r"(wr[s][3])
                                 : "memory");
                    asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};\n" ::"r"(ai), "r"(wi[s][0]), "r"(wi[s][1]),
                                 "r"(wi[s][2]), "r"(wi[s][3])
                                 : "memory");
                }
            }
            tc::fence_proxy_async_smem();   // the tensor core reads B
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&S.bready);

            for (int rt = 0; rt < C::RT; ++rt, ++use) {
                const int row = rt * 128 + 32 * quad + lane;
                const int ee = (int)in.rexp[row];   // e_i + ga_i
                const float sa_lo = p2(-(ee / 2)), sa_hi = p2(-(ee - ee / 2));   // 2^-ea, in two factors
                // scaled domain: acc = B 2^-(ea + ex) - sum_c 2^(-14 - 8 (c - 2)) (class c)
                auto bval = [&](int i) {
                    const int j = j0 + CPT * part + i;
                    float2 b = make_float2(0.f, 0.f);
                    if (j < ncols && row < K) {
                        if (in.B) b = in.B[row + (size_t)j * in.ldb];
                        else if (row == j) b.x = 1.f;
                    }
                    return b;
                };
                float hr[CPT], lr[CPT], hi_[CPT], li[CPT];
#pragma unroll
                for (int i = 0; i < CPT; ++i) {
                    const int jl = CPT * part + i;
                    const float2 b = bval(i);
                    const float sx = S.xs[jl];
                    hr[i] = ((b.x * sa_lo) * sa_hi) * sx;
                    hi_[i] = ((b.y * sa_lo) * sa_hi) * sx;
                    lr[i] = li[i] = 0.f;
                }
#pragma unroll 1
                for (int ci = 0; ci < NCLS; ++ci) {
                    bool ok = !S.err;
                    if (ok && !tc::mbar_wait(&S.accf[ci], use & 1, WAIT_LIMIT)) {
                        S.err = 1;
                        ok = false;
                    }
                    ok = __all_sync(0xffffffffu, ok);
                    if (!ok) continue;
                    tc::tc_fence_after();
                    // 16 columns from the thread's first (the last 4 belong to the neighbour)
                    // U of class ci at columns ci BR .., V at (NCLS + ci) BR ..
                    const uint32_t ta = tmem + ((uint32_t)(32 * quad) << 16) + ci * BR + CPT * part;
                    const uint32_t tv = ta + NCLS * BR;
                    const float w = p2(-14 - 8 * ci);
                    float u[16], v[16];
                    tc::tmem_ld16(ta, u);               // Ar Xr
                    tc::tmem_ld16(tv + NB, v);          // Ai Xi
                    tc::tmem_ld_wait();
#pragma unroll
                    for (int i = 0; i < CPT; ++i) {     // Re: acc -= w (Ar Xr - Ai Xi), terms exact
                        two_sum_acc(hr[i], lr[i], -w * u[i]);
                        two_sum_acc(hr[i], lr[i], w * v[i]);
                    }
                    tc::tmem_ld16(ta + NB, u);          // Ar Xi
                    tc::tmem_ld16(tv, v);               // Ai Xr
                    tc::tmem_ld_wait();
                    tc::tc_fence_before();
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(&S.tfree[ci]);
#pragma unroll
                    for (int i = 0; i < CPT; ++i) {     // Im: acc -= w (Ar Xi + Ai Xr)
                        two_sum_acc(hi_[i], li[i], -w * u[i]);
                        two_sum_acc(hi_[i], li[i], -w * v[i]);
                    }
                }
                const float ua_lo = p2(ee / 2), ua_hi = p2(ee - ee / 2);
#pragma unroll
                for (int i = 0; i < CPT; ++i) {
                    const int jl = CPT * part + i, j = j0 + jl;
                    const float sxi = S.xsi[jl];
                    const float re = (((hr[i] + lr[i]) * ua_lo) * ua_hi) * sxi;
                    const float im = (((hi_[i] + li[i]) * ua_lo) * ua_hi) * sxi;
                    if (j < ncols) in.R[row + (size_t)j * KC] = make_float2(re, im);
                    const float2 b = bval(i);
                    // column norms of this row tile (sums of nonnegative terms: FP32
                    // pairwise, accurate to a few units; FP64 is slow on this GPU): the
                    // warp's 32 rows, added to the lane quarter's sums in row-tile order
                    float nr = (j < ncols) ? fmaf(re, re, im * im) : 0.f;
                    float nb = fmaf(b.x, b.x, b.y * b.y);
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        nr += __shfl_xor_sync(0xffffffffu, nr, o);
                        nb += __shfl_xor_sync(0xffffffffu, nb, o);
                    }
                    if (lane == 0) {
                        S.nr[quad][jl] = rt == 0 ? nr : S.nr[quad][jl] + nr;
                        S.nb[quad][jl] = rt == 0 ? nb : S.nb[quad][jl] + nb;
                    }
                }
            }
            asm volatile("bar.sync %0, %1;\n" ::"r"(BAR_EPI), "r"(NEW * 32) : "memory");
            if (t < NB && j0 + t < ncols) {
                float rn = 0.f, bn = 0.f;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    rn += S.nr[q][t];
                    bn += S.nb[q][t];
                }
                in.rnorm[j0 + t] = rn;
                in.rnorm[KC + j0 + t] = bn;
            }
            if (S.err && t == 0) atomicOr(acc_out.flags + job.x, FLAG_TIMEOUT);
            // S.cmax, S.xs, S.nr are rewritten by the next job after this barrier
            asm volatile("bar.sync %0, %1;\n" ::"r"(BAR_EPI), "r"(NEW * 32) : "memory");
        }
    } else if (warp == TMA_WARP) {
        if (lane == 0) {
            uint32_t seq = 0;
            for (int jj = blockIdx.x; jj < n_jobs && !S.err; jj += gridDim.x) {
                const int2 job = jobs[jj];
                const DevInst &in = insts[job.x];
                if (sweep > 0 && in.rctl[1] != 0.f) continue;
                const char *src = reinterpret_cast<const char *>(in.Asl);
                // (rt, s, ks) order, SUB consecutive k-steps per copy
                for (int st = 0; st < C::RT * NSL * C::KS / SUB && !S.err; ++st, ++seq) {
                    const int slot = seq % RING;
                    if (seq >= RING && !tc::mbar_wait(&S.empty[slot], ((seq / RING) - 1) & 1, WAIT_LIMIT)) {
                        S.err = 1;
                        break;
                    }
                    tc::mbar_arrive_expect_tx(&S.full[slot], SLOT);
                    bulk_load(ring0 + slot * SLOT, src + (size_t)st * SLOT, SLOT, &S.full[slot]);
                }
            }
            for (uint32_t q = seq > RING ? seq - RING : 0; q < seq; ++q)
                tc::mbar_wait(&S.full[q % RING], (q / RING) & 1, WAIT_LIMIT);
        }
    } else {
        if (lane == 0) {

            uint32_t seq = 0, use = 0, njob = 0;
            for (int jj = blockIdx.x; jj < n_jobs && !S.err; jj += gridDim.x) {
                const int2 job = jobs[jj];
                const DevInst &in = insts[job.x];
                if (sweep > 0 && in.rctl[1] != 0.f) continue;
                if (!tc::mbar_wait(&S.bready, njob & 1, WAIT_LIMIT)) {
                    S.err = 1;
                    break;
                }
                ++njob;
                tc::tc_fence_after();
                for (int rt = 0; rt < C::RT && !S.err; ++rt, ++use) {
                    for (int s = 0; s < NSL && !S.err; ++s) {          // slice s + 1 of A
                        const uint32_t idn = tc::idesc_f16(128, BR * (NSL - s), false);
                        for (int kq = 0; kq < C::KS / SUB && !S.err; ++kq, ++seq) {
                            const int slot = seq % RING;
                            if (!tc::mbar_wait(&S.full[slot], (seq / RING) & 1, WAIT_LIMIT)) {
                                S.err = 1;
                                break;
                            }
                            tc::tc_fence_after();
                            for (int u = 0; u < SUB; ++u) {
                            const int ks = kq * SUB + u;
                            const uint32_t a = ring0 + slot * SLOT + u * STAGE;
                            const uint64_t ad = tc::smem_desc(a, 128, 256), vd = tc::smem_desc(a + TILE, 128, 256);
                            const bool first = s == 0 && ks == 0;   // initialises every class
                            if (first && use > 0)                    // the classes' previous pass is drained
                                for (int ci = 0; ci < NCLS; ++ci)
                                    if (!tc::mbar_wait(&S.tfree[ci], (use - 1) & 1, WAIT_LIMIT)) S.err = 1;
                            tc::tc_fence_after();
                            // X slices 1 .. NSL - s stacked along N (their B rows follow each
                            // other): one MMA into classes s .. NCLS - 1 for U, one for V
                            const uint64_t bd = tc::smem_desc(b0 + ks * 256, 128, C::SBO_B);
                            const uint32_t accum = first ? 0u : 1u;
                            tc::mma_bf16(tmem + s * BR, ad, bd, idn, accum);              // FP16 by the descriptor
                            tc::mma_bf16(tmem + (NCLS + s) * BR, vd, bd, idn, accum);
                            }
                            tc::mma_commit(&S.empty[slot]);
                        }
                        tc::mma_commit(&S.accf[s]);   // class s + 2 has all its pairs (slice s + 1 done)
                    }
                }
            }
            tc::mma_commit(&S.fin);
            tc::mbar_wait(&S.fin, 0, WAIT_LIMIT);
        }
    }

    tc::tc_fence_before();
    __syncthreads();
    if (S.err && threadIdx.x == 0)
        for (int jj = blockIdx.x; jj < n_jobs; jj += gridDim.x) atomicOr(acc_out.flags + jobs[jj].x, FLAG_TIMEOUT);
    if (warp == MMA_WARP) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, TMEM_COLS);
    }
}

template <int KC>
cudaError_t launch_main(const DevInst *insts, const int2 *jobs, int n, int sweep, DevAccum acc, cudaStream_t s) {
    const size_t smem = sizeof(RSmem) + 128;
    cudaError_t e = cudaFuncSetAttribute(resid_tc_kernel<KC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    resid_tc_kernel<KC><<<n < sms ? n : sms, NTHREADS, smem, s>>>(insts, jobs, n, sweep, acc);
    return cudaGetLastError();
}

}  // namespace

size_t resid_tc_slice_bytes(int KC) { return (size_t)(KC / 128) * NSL * (KC / 16) * STAGE; }

cudaError_t launch_rtc_prep(int KC, const DevInst *insts, const int *list, int n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    if (KC == 128) rtc_prep_kernel<128><<<n * RCfg<128>::RT, 256, 0, s>>>(insts, list);
    else if (KC == 256) rtc_prep_kernel<256><<<n * RCfg<256>::RT, 256, 0, s>>>(insts, list);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_resid_tc(int KC, const DevInst *insts, const int2 *jobs, int n, int sweep, DevAccum acc,
                            cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    if (KC == 128) return launch_main<128>(insts, jobs, n, sweep, acc, s);
    if (KC == 256) return launch_main<256>(insts, jobs, n, sweep, acc, s);
    return cudaErrorInvalidValue;
}

}  // namespace jacpcg
