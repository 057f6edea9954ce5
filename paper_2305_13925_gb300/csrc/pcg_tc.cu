// pcg_tc.cu -- the Jac-PCG iteration with the product Q = A P on the tcgen05
// tensor cores, K = 64 class (Sec. III-B Steps 1-4, Eqs. 12-14 and 19-21;
// standard and plain-CG forms; right-hand side B = I or the refinement
// residual, as the SIMT kernel in pcg_kernel.cuh).
//
// Complex product as one real MMA: A is expanded once per instance into the
// 128 x 128 real matrix whose 2 x 2 blocks are [[Ar, -Ai], [Ai, Ar]] (real
// row 2i + s is part s of complex row i), P into the 128 x 64 real matrix
// with rows 2k + t, so Q_real = A_real P_real has Re q_i in row 2i and Im q_i
// in row 2i + 1 -- two adjacent TMEM lanes of one warp.  3xTF32 as in
// gram_tc.cu; the head*head product is accumulated in two TMEM buffers (one
// per half of the reduction) and the correction products in a third, so no
// truncating accumulation chain is longer than 16 MMAs.
//
// One persistent CTA per SM walks its instances.  16 warps (four per SM
// sub-partition, 128 registers each) own the state: thread (warp w, lane l)
// holds complex row i = 16 (w mod 4) + l / 2 and the 8 columns starting at
// 16 (w / 4) + 8 (l mod 2) of x, r, p in registers for all iterations.  Per iteration they write P (TF32 head and tail) into
// shared memory, vote on continuing (a barrier reduction), thread 0 issues
// 48 MMAs and commits, and all warps read
// Q from TMEM, pair Re / Im with one shuffle, and reduce the per-column dot
// products (compensated, fixed order: warp shuffles, then the four row
// quarters through shared memory).  Core matrices along K are 144 bytes
// apart (16 bytes of padding) so that the P and A stores hit distinct banks.
#include "common.cuh"
#include "kernels.h"
#include "tc.cuh"

namespace jacpcg {

namespace {

constexpr int KCP = 64;                     // K class
constexpr int RR = 2 * KCP;                 // real rows = real reduction length
constexpr int NC = KCP;                     // right-hand sides (MMA N)
constexpr uint32_t LBO = 144;               // K-adjacent core matrices (128 + 16 padding)
constexpr uint32_t SBO = (RR / 4) * LBO;    // 8-row groups
constexpr int APART = (RR / 8) * SBO;       // one of A_hi, A_lo
constexpr int BPART = (NC / 8) * SBO;       // one of P_hi, P_lo
constexpr int NSW = 16;                     // state warps (thread 0 also issues the MMAs)
constexpr int NTHREADS = NSW * 32;
constexpr int CPT = 8;                      // columns owned per thread
constexpr int TMEM_COLS = 256;              // [0,64) head*head k<64, [64,128) k>=64, [128,192) corrections
constexpr uint32_t WAIT_LIMIT = 1u << 21;

struct __align__(128) PcgSmem {
    unsigned char A[2 * APART];
    unsigned char B[2 * BPART];
    float2 red[3][4][NC];                   // compensated partials per quantity, row quarter, column
    float2 tot[3][NC];                      // column totals per quantity
    uint64_t qfull;
    uint64_t fin;
    uint32_t tmem;
    int err;                                // a bounded wait ran out (sticky)
};

__device__ __forceinline__ void st_shared_v4(uint32_t addr, float a, float b, float c, float d) {
    asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};\n" ::"r"(addr), "f"(a), "f"(b), "f"(c),
                 "f"(d)
                 : "memory");
}
__device__ __forceinline__ void st_shared_v2(uint32_t addr, float a, float b) {
    asm volatile("st.shared.v2.f32 [%0], {%1, %2};\n" ::"r"(addr), "f"(a), "f"(b) : "memory");
}
// Sum, over the 64 rows, of one compensated partial per column for the
// thread's 8 columns, for NQ quantities at once.  Within a warp the 16 lanes
// of equal parity hold the 16 rows of a quarter: a butterfly
// reduce-scatter (offsets 2, 4, 8, halving the values each round, then a
// pairwise add at offset 16) leaves each lane the quarter sum of one column;
// the four quarters meet in shared memory, one lane per column adds them,
// and every thread reads back the totals of its 8 columns (fixed order).
template <int NQ>
__device__ __forceinline__ void column_sum(Comp (&v)[NQ][CPT], float2 (*red)[4][NC], float2 (*tot)[NC],
                                           int quad, int jb, int lane) {
    Comp d[NQ];
#pragma unroll
    for (int qn = 0; qn < NQ; ++qn) {
        Comp a[4], b[2];
#pragma unroll
        for (int k = 0; k < 4; ++k) {   // offset 2: keep half by lane bit 1
            const bool hi = (lane >> 1) & 1;
            const Comp send = hi ? v[qn][k] : v[qn][k + 4];
            Comp keep = hi ? v[qn][k + 4] : v[qn][k];
            Comp got;
            got.s = __shfl_xor_sync(0xffffffffu, send.s, 2);
            got.c = __shfl_xor_sync(0xffffffffu, send.c, 2);
            comp_add(keep, got);
            a[k] = keep;
        }
#pragma unroll
        for (int k = 0; k < 2; ++k) {   // offset 4: lane bit 2
            const bool hi = (lane >> 2) & 1;
            const Comp send = hi ? a[k] : a[k + 2];
            Comp keep = hi ? a[k + 2] : a[k];
            Comp got;
            got.s = __shfl_xor_sync(0xffffffffu, send.s, 4);
            got.c = __shfl_xor_sync(0xffffffffu, send.c, 4);
            comp_add(keep, got);
            b[k] = keep;
        }
        Comp c1;
        {                               // offset 8: lane bit 3
            const bool hi = (lane >> 3) & 1;
            const Comp send = hi ? b[0] : b[1];
            Comp keep = hi ? b[1] : b[0];
            Comp got;
            got.s = __shfl_xor_sync(0xffffffffu, send.s, 8);
            got.c = __shfl_xor_sync(0xffffffffu, send.c, 8);
            comp_add(keep, got);
            c1 = keep;
        }
        {                               // offset 16: both lanes hold the same column
            Comp got;
            got.s = __shfl_xor_sync(0xffffffffu, c1.s, 16);
            got.c = __shfl_xor_sync(0xffffffffu, c1.c, 16);
            // fixed order: the lane with bit 4 clear adds its partner's value second
            Comp lo = ((lane >> 4) & 1) ? got : c1, hi = ((lane >> 4) & 1) ? c1 : got;
            comp_add(lo, hi);
            d[qn] = lo;
        }
    }
    // this lane now holds column jb + 4 b1 + 2 b2 + b3 (b_n = lane bit n)
    const int col = jb + 4 * ((lane >> 1) & 1) + 2 * ((lane >> 2) & 1) + ((lane >> 3) & 1);
    if (((lane >> 4) & 1) == 0) {
#pragma unroll
        for (int qn = 0; qn < NQ; ++qn) red[qn][quad][col] = make_float2(d[qn].s, d[qn].c);
    }
    asm volatile("bar.sync 2, 512;\n" ::: "memory");
    if (quad == 0 && ((lane >> 4) & 1) == 0) {   // one lane per column adds the four quarters
#pragma unroll
        for (int qn = 0; qn < NQ; ++qn) {
            Comp t = {red[qn][0][col].x, red[qn][0][col].y};
#pragma unroll
            for (int qq = 1; qq < 4; ++qq) comp_add(t, Comp{red[qn][qq][col].x, red[qn][qq][col].y});
            tot[qn][col] = make_float2(t.s + t.c, 0.f);
        }
    }
    asm volatile("bar.sync 2, 512;\n" ::: "memory");
#pragma unroll
    for (int qn = 0; qn < NQ; ++qn)
#pragma unroll
        for (int c = 0; c < CPT; ++c) v[qn][c] = Comp{tot[qn][jb + c].x, 0.f};
}

template <int VAR>
__global__ void __launch_bounds__(NTHREADS, 1) pcg_tc64_kernel(const DevInst *__restrict__ insts,
                                                               const int *__restrict__ list, int n_list,
                                                               DevAccum acc_out, int mode) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    PcgSmem &S = *reinterpret_cast<PcgSmem *>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        tc::mbar_init(&S.qfull, 1);
        tc::mbar_init(&S.fin, 1);
        S.err = 0;
        tc::mbar_init_fence();
    }
    if (warp == 0) {
        tc::tmem_alloc(&S.tmem, TMEM_COLS);
        tc::tmem_relinquish();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = S.tmem;
    const uint32_t a_hi = tc::smem_u32(S.A), a_lo = a_hi + APART;
    const uint32_t b_hi = tc::smem_u32(S.B), b_lo = b_hi + BPART;

    // state-thread geometry
    const int quad = warp & 3, part = warp >> 2;     // TMEM lane quarter, column quarter
    const int i = 16 * quad + (lane >> 1);          // complex row
    const int s = lane & 1;                          // 0: Re lane, 1: Im lane
    const int jb = 16 * part + CPT * s;              // first of the owned columns
    uint32_t phase = 0;
    int err = 0;

    for (int jj = blockIdx.x; jj < n_list; jj += gridDim.x) {
        const int id = list[jj];
        const DevInst &in = insts[id];
        const int K = in.K, T = in.max_iter;
        const float tol2 = in.tol > 0.f ? in.tol * in.tol : -1.f;

        float2 x[CPT], r[CPT], p[CPT];
        float rho[CPT], res2[CPT], btol[CPT];
        uint32_t done = 0;                 // bit c: column jb + c stopped (or beyond K)
        int itmax = 0;                     // iterations in which an owned column updated
        float dv = 0.f;
        int notHPD = 0;
        {
            // ---- A in the real 2 x 2-block layout, TF32 head and tail ----
            const float2 *__restrict__ Ag = in.A;   // ld 64, zero beyond K
            for (int e = threadIdx.x; e < 64 * 32; e += NTHREADS) {
                const int ii = e & 63, kp = e >> 6;   // row, pair of columns (2 kp, 2 kp + 1)
                const float2 a0 = Ag[ii + (size_t)(2 * kp) * 64];
                const float2 a1 = Ag[ii + (size_t)(2 * kp + 1) * 64];
                const float re[4] = {a0.x, -a0.y, a1.x, -a1.y};   // real row 2 ii
                const float im[4] = {a0.y, a0.x, a1.y, a1.x};     // real row 2 ii + 1
                float rh[4], rl[4], ih[4], il[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    tc::split_tf32(re[u], rh[u], rl[u]);
                    tc::split_tf32(im[u], ih[u], il[u]);
                }
                const int a = 2 * ii;
                const uint32_t o0 = (uint32_t)(a >> 3) * SBO + kp * LBO + (a & 7) * 16;
                const uint32_t o1 = (uint32_t)((a + 1) >> 3) * SBO + kp * LBO + ((a + 1) & 7) * 16;
                st_shared_v4(a_hi + o0, rh[0], rh[1], rh[2], rh[3]);
                st_shared_v4(a_lo + o0, rl[0], rl[1], rl[2], rl[3]);
                st_shared_v4(a_hi + o1, ih[0], ih[1], ih[2], ih[3]);
                st_shared_v4(a_lo + o1, il[0], il[1], il[2], il[3]);
            }
            // ---- state init (Step 1; x = 0, r = b, p = D^{-1} r) ----
            dv = (i < K) ? (VAR == 2 ? 1.f : in.dinv[i]) : 0.f;
            Comp qv[3][CPT];
#pragma unroll
            for (int c = 0; c < CPT; ++c) {
                const int j = jb + c;
                float2 b = make_float2(0.f, 0.f);
                if (mode == 0) {
                    if (i < K && i == j) b.x = 1.f;
                } else if (i < K && j < K) {
                    b = in.R[i + (size_t)j * 64];
                }
                x[c] = make_float2(0.f, 0.f);
                r[c] = b;
                p[c] = make_float2(dv * b.x, dv * b.y);
                qv[0][c] = {0.f, 0.f};
                qv[1][c] = {0.f, 0.f};
                qv[2][c] = {0.f, 0.f};
                comp_fma(qv[0][c], r[c].x, p[c].x);     // r^H z
                comp_fma(qv[0][c], r[c].y, p[c].y);
                comp_fma(qv[1][c], r[c].x, r[c].x);     // ||r||^2
                comp_fma(qv[1][c], r[c].y, r[c].y);
                comp_fma(qv[2][c], b.x, b.x);           // ||b||^2
                comp_fma(qv[2][c], b.y, b.y);
            }
            column_sum<3>(qv, S.red, S.tot, quad, jb, lane);
#pragma unroll
            for (int c = 0; c < CPT; ++c) {
                rho[c] = qv[0][c].s;
                res2[c] = qv[1][c].s;
                btol[c] = tol2 * qv[2][c].s;
                if (jb + c >= K) done |= 1u << c;
            }
        }

        for (int t = 0;; ++t) {
            int any = 0;
            {
                // Step 2: stopping test, then publish P = [Re p; Im p] (head, tail)
#pragma unroll
                for (int c = 0; c < CPT; ++c)
                    if (tol2 > 0.f && res2[c] <= btol[c]) done |= 1u << c;
                any = done != (1u << CPT) - 1u;
                if (t >= T) any = 0;
#pragma unroll
                for (int c = 0; c < CPT; ++c) {
                    const int j = jb + c;
                    float ph, pl, qh, ql;
                    tc::split_tf32(p[c].x, ph, pl);
                    tc::split_tf32(p[c].y, qh, ql);
                    const uint32_t o = (uint32_t)(j >> 3) * SBO + (i >> 1) * LBO + (j & 7) * 16 + (i & 1) * 8;
                    st_shared_v2(b_hi + o, ph, qh);
                    st_shared_v2(b_lo + o, pl, ql);
                }
                tc::fence_proxy_async_smem();
                tc::tc_fence_before();
            }
            const int cont = __syncthreads_or(any) && !S.err;
            if (!cont) break;
            {
                if (threadIdx.x == 0) {
                    tc::tc_fence_after();
                    constexpr uint32_t idesc = tc::idesc_tf32(RR, NC);
#pragma unroll 4
                    for (int kk = 0; kk < RR / 8; ++kk) {
                        const uint32_t off = (uint32_t)(2 * kk) * LBO;
                        const uint64_t ah = tc::smem_desc(a_hi + off, LBO, SBO);
                        const uint64_t al = tc::smem_desc(a_lo + off, LBO, SBO);
                        const uint64_t bh = tc::smem_desc(b_hi + off, LBO, SBO);
                        const uint64_t bl = tc::smem_desc(b_lo + off, LBO, SBO);
                        const uint32_t d1 = tmem + (kk < RR / 16 ? 0u : 64u);
                        tc::mma_tf32(d1, ah, bh, idesc, (kk % (RR / 16)) ? 1u : 0u);
                        tc::mma_tf32(tmem + 128u, ah, bl, idesc, kk ? 1u : 0u);
                        tc::mma_tf32(tmem + 128u, al, bh, idesc, 1u);
                    }
                    tc::mma_commit(&S.qfull);
                }
                __syncwarp();
            }
            // ---- Q = A P from TMEM ----
            if (!tc::mbar_wait(&S.qfull, phase & 1, WAIT_LIMIT)) {
                err = 1;
                S.err = 1;   // seen by every thread after the next vote
            }
            ++phase;
            tc::tc_fence_after();
            float v[16];
            {
                const uint32_t ta = tmem + ((uint32_t)(32 * quad) << 16) + 16 * part;
                float u0[16], u1[16], u2[16];
                tc::tmem_ld16(ta, u0);
                tc::tmem_ld16(ta + 64, u1);
                tc::tmem_ld16(ta + 128, u2);
                tc::tmem_ld_wait();
#pragma unroll
                for (int e = 0; e < 16; ++e) v[e] = (u0[e] + u1[e]) + u2[e];
            }
            // pair Re (even lane) and Im (odd lane) of q[i][j] for the owned columns
            float2 q[CPT];
#pragma unroll
            for (int c = 0; c < CPT; ++c) {
                const float mine_own = s ? v[CPT + c] : v[c];    // my part of my column
                const float send = s ? v[c] : v[CPT + c];        // my part of the partner's column
                const float got = __shfl_xor_sync(0xffffffffu, send, 1);
                q[c] = s ? make_float2(got, mine_own) : make_float2(mine_own, got);
            }
            // lambda = r^H z / p^H A p
            // one row's term per column (plain FMA); the 64-row sums are compensated
            Comp pq[2][CPT];
#pragma unroll
            for (int c = 0; c < CPT; ++c) pq[0][c] = {fmaf(p[c].x, q[c].x, p[c].y * q[c].y), 0.f};
            column_sum<1>(*reinterpret_cast<Comp(*)[1][CPT]>(&pq[0]), S.red, S.tot, quad, jb, lane);
            const bool upd = (done != (1u << CPT) - 1u);
#pragma unroll
            for (int c = 0; c < CPT; ++c) {
                const float pAp = pq[0][c].s;
                const bool dn = (done >> c) & 1u;
                float lam = 0.f;
                if (pAp > 0.f) lam = rho[c] / pAp;
                else if (res2[c] != 0.f && !dn) notHPD = 1;
                if (dn) lam = 0.f;
                x[c].x = fmaf(lam, p[c].x, x[c].x);
                x[c].y = fmaf(lam, p[c].y, x[c].y);
                r[c].x = fmaf(-lam, q[c].x, r[c].x);
                r[c].y = fmaf(-lam, q[c].y, r[c].y);
                const float rr2 = fmaf(r[c].x, r[c].x, r[c].y * r[c].y);
                pq[0][c] = {dv * rr2, 0.f};          // r^H z with z = D^{-1} r
                pq[1][c] = {rr2, 0.f};               // ||r||^2
            }
            column_sum<2>(pq, S.red, S.tot, quad, jb, lane);
#pragma unroll
            for (int c = 0; c < CPT; ++c) {
                const float rz_new = pq[0][c].s;
                const float beta = rho[c] != 0.f ? rz_new / rho[c] : 0.f;
                if (!((done >> c) & 1u)) {
                    p[c].x = fmaf(beta, p[c].x, dv * r[c].x);
                    p[c].y = fmaf(beta, p[c].y, dv * r[c].y);
                    rho[c] = rz_new;
                    res2[c] = pq[1][c].s;
                }
            }
            if (upd) itmax = t + 1;
        }

        {
            // ---- outputs ----
#pragma unroll
            for (int c = 0; c < CPT; ++c) {
                const int j = jb + c;
                if (j >= K) continue;
                float2 val = x[c];
                if (mode == 1) {
                    const float2 o = in.X[i + (size_t)j * 64];
                    val = make_float2(o.x + val.x, o.y + val.y);
                }
                in.X[i + (size_t)j * 64] = val;
                if (in.Xout && i < K) in.Xout[i + (size_t)j * K] = val;
            }
            if (mode == 0) {
                float resmax = 0.f;
                bool notconv = false;
#pragma unroll
                for (int c = 0; c < CPT; ++c) {
                    if (jb + c >= K) continue;
                    resmax = fmaxf(resmax, sqrtf(fmaxf(res2[c], 0.f)));
                    if (tol2 > 0.f && !(res2[c] <= btol[c])) notconv = true;
                }
                if (i == 0) {   // one thread per 8 columns: quarter-0 warps, lanes 0 and 1
                    if (itmax > 0) atomicMax(acc_out.iters + id, itmax);
                    if (resmax > 0.f) atomicMax(acc_out.resid_bits + id, __float_as_uint(resmax));
                }
                const int f = (notHPD ? FLAG_NOTHPD : 0) | (notconv && i == 0 ? FLAG_NOTCONV : 0) |
                              (err ? FLAG_TIMEOUT : 0);
                if (f) atomicOr(acc_out.flags + id, f);
            }
        }
    }

    if (threadIdx.x == 0) {
        tc::mma_commit(&S.fin);
        tc::mbar_wait(&S.fin, 0, WAIT_LIMIT);
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, TMEM_COLS);
    }
}

}  // namespace

cudaError_t launch_pcg_tc64(int variant, const DevInst *insts, const int *list, int n, DevAccum acc,
                            cudaStream_t s, int mode) {
    if (n <= 0) return cudaSuccess;
    const size_t smem = sizeof(PcgSmem);
    int dev = 0, sms = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const int grid = n < sms ? n : sms;
    auto go = [&](auto kern) -> cudaError_t {
        cudaError_t r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (r != cudaSuccess) return r;
        kern<<<grid, NTHREADS, smem, s>>>(insts, list, n, acc, mode);
        return cudaGetLastError();
    };
    if (variant == 2) return go(pcg_tc64_kernel<2>);   // plain CG
    return go(pcg_tc64_kernel<0>);
}

}  // namespace jacpcg
