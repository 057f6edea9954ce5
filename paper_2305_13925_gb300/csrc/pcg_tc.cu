// pcg_tc.cu -- the Jac-PCG iteration with the product Q = A P on the tcgen05
// tensor cores, K = 64 class (Sec. III-B Steps 1-4, Eqs. 12-14 and 19-21;
// standard and plain-CG forms; right-hand side B = I or the refinement
// residual, as the SIMT kernel in pcg_kernel.cuh).
//
// Complex product as one real MMA: A is expanded once per instance into the
// 128 x 128 real matrix whose 2 x 2 blocks are [[Ar, -Ai], [Ai, Ar]] (real
// row 2i + s is part s of complex row i), P into the 128 x 64 real matrix
// with rows 2k + t, so Q_real = A_real P_real has Re q_i in row 2i and Im q_i
// in row 2i + 1.  3xTF32 as in gram_tc.cu: per k-step the A head multiplies
// [P head | P tail] in one N = 128 MMA (the tail tile follows the head tile in
// shared memory, so the two form one 128-row B operand; TMEM columns 0-63
// take head*head, 64-127 head*tail), and the A tail multiplies the P head in
// an N = 64 MMA into columns 128-191 -- 32 MMAs per iteration instead of 48
// (0.277 vs 0.315 ms per 2048-channel batch), no truncating accumulation
// chain longer than 16 MMAs.  The expanded A (head and tail) lives in tensor
// memory and is the MMAs' A operand there: per iteration the MMAs read only
// the 1 KB P tiles from shared memory instead of re-reading a 4 KB A tile for
// every MMA.  The next instance's A is prefetched into a shared staging tile
// while the current one iterates: one tiled TMA copy (cp.async.bulk.tensor)
// through a tensor map over the library's workspace arena, whose rows of 256
// bytes hold A (64 x 64 complex, ld 64) at a row boundary, completion counted
// in bytes on an mbarrier.
//
// The columns of P are independent systems that share A, so the 64 columns
// may form NG groups, each a team of warps with its own MMAs (N = 64 / NG),
// TMEM buffers, mbarrier and named barrier; with two teams the tensor core
// multiplies one team's P while the other updates its vectors, but every
// team issues its own full set of MMAs per iteration.  With A in tensor
// memory one team of 8 warps (N = 64) measures faster on GB300 (0.31 vs 0.34
// ms per 2048-channel batch), and only one team lets the head products fuse
// into one N = 128 MMA, so NG = 1.  Per iteration the team
//   1. writes P (TF32 head and tail) into the MMA's K-major layout and votes
//      on continuing (barrier reduction); its first thread issues 32 MMAs;
//   2. copies Q from TMEM (warp w reads TMEM lanes 32 (w mod 4) ..) into a
//      padded shared-memory tile, then a team barrier;
//   3. works column-wise: thread (warp w, lane l) owns column 8 w + (l mod 8)
//      and the 16 complex rows g, g + 4, .., g + 60 with g = l / 8, holding
//      x, r, p for them in registers; the step denominator p^H A p, whose
//      terms can cancel, is compensated (Dot2: in-thread error-free sums over
//      its 16 rows in a tree, then two xor shuffles across the four lanes of
//      the column, combined with commutative or exact operations only); the
//      squared norms r^H D^{-1} r and ||r||^2 sum nonnegative terms, where
//      pairwise summation is already accurate to a few units, and are summed
//      so (Dot2 on all three measured 0.368 against 0.318 ms per 2048-channel
//      batch).  All four lanes obtain bit-identical totals and take identical
//      decisions.
// The tile strides (128-byte core matrices, 68-float rows of the Q tile) make
// every P store, Q store and Q load free of shared-memory bank conflicts.
#include "common.cuh"
#include "kernels.h"
#include "tc.cuh"

namespace jacpcg {

namespace {

constexpr int KCP = 64;                     // K class
constexpr int RR = 2 * KCP;                 // real rows = real reduction length
constexpr int NC = KCP;                     // right-hand sides
constexpr int NG = 1;                       // column groups (teams): 1 or 2
constexpr int GC = NC / NG;                 // columns per group (MMA N)
constexpr uint32_t LBO = 128;               // K-adjacent core matrices
constexpr uint32_t SBO = (RR / 4) * LBO;    // 8-row groups
constexpr int BPART = (NC / 8) * SBO;       // one of P_hi, P_lo
constexpr int QLD = NC + 4;                 // floats per row of the Q tile
constexpr int NW = 8;                       // warps: two teams of four
constexpr int NTHREADS = NW * 32;
constexpr int TEAM = NTHREADS / NG;
constexpr int PARTS = (NW / NG) / 4;        // warps of a team per TMEM lane quarter
constexpr int TEAM_COLS = NG == 1 ? 256 : 128;   // TMEM columns per team: head*head, head*tail, tail*head
constexpr int RPT = KCP / 4;                // complex rows per thread
constexpr int TMEM_COLS = 512;              // [0, 192): head*head, head*tail, tail*head;
                                            // [256, 384): A head, [384, 512): A tail (128 lanes x 128 K)
constexpr uint32_t TA_HI = 256, TA_LO = 384;
constexpr uint32_t WAIT_LIMIT = 1u << 21;

struct __align__(128) PcgSmem {
    float2 Ast[KCP * KCP];                  // the next instance's A (complex, ld 64), prefetched
    unsigned char B[2 * BPART];
    float Q[RR * QLD];
    uint64_t qfull[NG];
    uint64_t fin[NG];
    uint64_t abar;                          // the staging tile's copy has landed
    uint32_t tmem;
    volatile int err;                       // a bounded wait ran out (sticky)
    volatile int aerr;                      // ... the wait for a staging copy (no further copies)
};
static_assert(sizeof(PcgSmem) <= 227 * 1024, "shared memory");

__device__ __forceinline__ void st_shared_v4(uint32_t addr, float a, float b, float c, float d) {
    asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};\n" ::"r"(addr), "f"(a), "f"(b), "f"(c),
                 "f"(d)
                 : "memory");
}
__device__ __forceinline__ void st_shared_v2(uint32_t addr, float a, float b) {
    asm volatile("st.shared.v2.f32 [%0], {%1, %2};\n" ::"r"(addr), "f"(a), "f"(b) : "memory");
}
__device__ __forceinline__ void team_sync(int id) {
    asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(TEAM) : "memory");
}
// OR of pred over the team's threads (every one of them receives the result)
__device__ __forceinline__ int team_or(int id, int pred) {
    int r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.s32 p, %1, 0;\n\t"
        "bar.red.or.pred q, %2, %3, p;\n\t"
        "selp.s32 %0, 1, 0, q;\n\t}\n"
        : "=r"(r)
        : "r"(pred), "r"(id), "r"(TEAM)
        : "memory");
    return r;
}
// Compensated per-column dot products (Dot2: each product split exactly by
// an FMA, each addition by TwoSum; Ogita, Rump and Oishi 2005).  A thread
// accumulates its 16 rows in order; the four lanes that share a column (lane
// bits 3 and 4) then combine as (s_a + s_b, (c_a + c_b) + e): every operation
// is commutative or exact, so all four lanes hold bit-identical totals.
__device__ __forceinline__ Comp col_total(Comp v) {
#pragma unroll
    for (int o = 8; o <= 16; o <<= 1) {
        const float ws = __shfl_xor_sync(0xffffffffu, v.s, o);
        const float wc = __shfl_xor_sync(0xffffffffu, v.c, o);
        float s, e;
        two_sum(v.s, ws, s, e);
        v.s = s;
        v.c = (v.c + wc) + e;
    }
    return v;
}
__device__ __forceinline__ float comp_value(Comp v) { return v.s + v.c; }
// Re sum_k conj(a_k) b_k over the thread's 16 rows, compensated and in a tree:
// every product is split exactly by an FMA (TwoProduct), the 16 partial sums
// are combined pairwise by TwoSum in 4 levels, and the errors are summed
// alongside.  The same error-free steps as a sequential Dot2, but with no
// chain of 32 dependent TwoSums on the iteration's critical path.
// Sum over the thread's rows of Re conj(a_k) b_k when every term is >= 0
// (||r||^2 and r^H D^{-1} r): no cancellation can occur, so plain pairwise
// summation is already accurate to a few units in the last place, and the
// lanes of a column combine by commutative additions (bit-identical totals).
__device__ __forceinline__ float sumsq_col(const float2 (&a)[RPT], const float2 (&b)[RPT]) {
    float s[RPT];
#pragma unroll
    for (int k = 0; k < RPT; ++k) s[k] = fmaf(a[k].x, b[k].x, a[k].y * b[k].y);
#pragma unroll
    for (int h = RPT / 2; h > 0; h >>= 1)
#pragma unroll
        for (int k = 0; k < h; ++k) s[k] += s[k + h];
    float v = s[0];
    v += __shfl_xor_sync(0xffffffffu, v, 8);
    v += __shfl_xor_sync(0xffffffffu, v, 16);
    return v;
}
__device__ __forceinline__ Comp dot2_rows(const float2 (&a)[RPT], const float2 (&b)[RPT]) {
    float s[RPT], c[RPT];
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
        const float p1 = a[k].x * b[k].x, p2 = a[k].y * b[k].y;
        const float e1 = fmaf(a[k].x, b[k].x, -p1), e2 = fmaf(a[k].y, b[k].y, -p2);
        float e;
        two_sum(p1, p2, s[k], e);
        c[k] = (e1 + e2) + e;
    }
#pragma unroll
    for (int h = RPT / 2; h > 0; h >>= 1) {
#pragma unroll
        for (int k = 0; k < h; ++k) {
            float sk, e;
            two_sum(s[k], s[k + h], sk, e);
            s[k] = sk;
            c[k] = (c[k] + c[k + h]) + e;
        }
    }
    return Comp{s[0], c[0]};
}

// MODE 0 solves A X = B from X0 (or 0); MODE 1 is a refinement correction
// solve (right-hand side R, X += dX, instances that stopped refining skipped).
// The form is a template parameter so the main solve carries none of the
// refinement code.
template <int VAR, int MODE>
__global__ void __launch_bounds__(NTHREADS, 1) pcg_tc64_kernel(const DevInst *__restrict__ insts,
                                                               const int *__restrict__ list, int n_list,
                                                               DevAccum acc_out,
                                                               const __grid_constant__ CUtensorMap amap,
                                                               const char *arena) {
    constexpr int mode = MODE;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    PcgSmem &S = *reinterpret_cast<PcgSmem *>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int team = warp / (NW / NG), quad = warp & 3;
    const int col_off = 32 * ((warp >> 2) % PARTS);   // this warp's 32 of its team's columns
    const int bar_id = 1 + team;

    if (threadIdx.x == 0) {
        for (int t = 0; t < NG; ++t) {
            tc::mbar_init(&S.qfull[t], 1);
            tc::mbar_init(&S.fin[t], 1);
        }
        tc::mbar_init(&S.abar, 1);
        S.err = 0;
        S.aerr = 0;
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
    const uint32_t b_hi = tc::smem_u32(S.B), b_lo = b_hi + BPART;
    const uint32_t ast = tc::smem_u32(S.Ast);
    // A of the instance at list position jj -> staging tile: the 128 arena rows
    // from A's row on, one tiled copy issued by thread 0 (A lies 256-byte aligned
    // in the arena, so its row index is exact and the copy starts at x = 0)
    auto prefetch_a = [&](int jj) {
        if (threadIdx.x == 0 && jj < n_list && !S.aerr) {
            const char *src = reinterpret_cast<const char *>(insts[list[jj]].A);
            tc::fence_proxy_async_smem();   // the staging tile's earlier reads come first
            tc::mbar_arrive_expect_tx(&S.abar, (uint32_t)sizeof(S.Ast));
            tc::tma_load_2d(ast, &amap, 0, (int)((src - arena) / 256), &S.abar);
        }
    };
    prefetch_a(blockIdx.x);
    const uint32_t q_base = tc::smem_u32(S.Q);
    const bool issuer = (threadIdx.x == team * TEAM);
    const uint32_t tq = tmem + team * TEAM_COLS;            // this team's TMEM columns

    // column-wise geometry: column j, complex rows g + 4 k
    const int jl = lane & 7, g = lane >> 3;
    const int j = 8 * warp + jl;
    // byte offset of (column j, row g) in P_hi / P_lo; row g + 4 k adds 2 k core matrices
    const uint32_t p_off = (uint32_t)warp * SBO + (uint32_t)(g >> 1) * LBO + jl * 16 + (g & 1) * 8;
    uint32_t phase = 0, aphase = 0;
    uint32_t a_lost = ~0u;   // parity of a staging copy whose wait ran out
    int err = 0;

    for (int jj = blockIdx.x; jj < n_list; jj += gridDim.x) {
        const int id = list[jj];
        const DevInst &in = insts[id];
        const int K = in.K, T = in.max_iter, NCOL = in.ncols;
        const bool warm = mode == 0 && in.X0 != nullptr;   // start from X0: one extra product A X0
        const float tl = (mode == 1 && in.rsolve_tol > 0.f) ? in.rsolve_tol : in.tol;   // correction solves
        const float tol2 = tl > 0.f ? tl * tl : -1.f;

        // ---- A in the real 2 x 2-block layout, TF32 head and tail, into TMEM ----
        // staging tile complete (every thread observes the copy; the vote makes a
        // timeout uniform); both teams are done with the previous instance
        const bool a_skip = S.aerr;   // set before an earlier barrier: uniform
        const bool a_ok = !a_skip && tc::mbar_wait(&S.abar, aphase & 1, WAIT_LIMIT);
        if (__syncthreads_or(!a_ok)) {
            if (!a_skip) a_lost = aphase;   // this copy may still land
            err = 1;
            S.err = 1;
            S.aerr = 1;
        }
        ++aphase;
        if constexpr (MODE == 1) {
            if (in.rctl[1] != 0.f) {   // the instance stopped refining (uniform)
                prefetch_a(jj + gridDim.x);
                continue;
            }
        }
        {
            // warp w writes TMEM lanes 32 (w mod 4) .. (real rows), K columns 64 (w / 4) ..
            const int rho = 32 * quad + lane, ii = rho >> 1, sp = rho & 1;
            const int half = warp >> 2;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                float hv[16], lv[16];
#pragma unroll
                for (int kk = 0; kk < 8; ++kk) {
                    const float2 a = S.Ast[ii + (size_t)(32 * half + 8 * c + kk) * 64];
                    const float v0 = sp ? a.y : a.x;      // column 2k of real row 2i + sp
                    const float v1 = sp ? a.x : -a.y;     // column 2k + 1
                    tc::split_tf32(v0, hv[2 * kk], lv[2 * kk]);
                    tc::split_tf32(v1, hv[2 * kk + 1], lv[2 * kk + 1]);
                }
                const uint32_t ta = tmem + ((uint32_t)(32 * quad) << 16) + 64 * half + 16 * c;
                tc::tmem_st16(ta + TA_HI, hv);
                tc::tmem_st16(ta + TA_LO, lv);
            }
            tc::tmem_st_wait();
        }
        tc::tc_fence_before();
        __syncthreads();   // A is in TMEM for both teams; the staging tile is free
        tc::tc_fence_after();
        prefetch_a(jj + gridDim.x);

        // ---- state init (Step 1; x = 0, r = b, p = D^{-1} r) ----
        float2 x[RPT], r[RPT], p[RPT];
        float dv[RPT];
        float rho, res2, btol, bn2c;
        bool done = j >= NCOL;             // column stopped (or beyond the right-hand sides)
        int itmax = 0;                     // iterations in which the column updated
        int notHPD = 0;
        {
#pragma unroll
            for (int k = 0; k < RPT; ++k) {
                const int i = g + 4 * k;
                dv[k] = (i < K) ? (VAR == 2 ? 1.f : in.dinv[i]) : 0.f;
                float2 b = make_float2(0.f, 0.f);
                if (mode == 0) {
                    if (!in.B) {
                        if (i < K && i == j) b.x = 1.f;                       // B = I
                    } else if (i < K && j < NCOL) {
                        b = in.B[i + (size_t)j * in.ldb];                     // symbol vectors
                    }
                } else if (i < K && j < NCOL) {
                    b = in.R[i + (size_t)j * 64];                             // refinement residual
                }
                x[k] = (warm && i < K && j < NCOL) ? in.X0[i + (size_t)j * K] : make_float2(0.f, 0.f);
                r[k] = b;
                p[k] = make_float2(dv[k] * b.x, dv[k] * b.y);
            }
            rho = sumsq_col(r, p);    // r^H z (terms d |r|^2 >= 0)
            res2 = sumsq_col(r, r);   // ||r||^2 = ||b||^2
            bn2c = res2;                   // stopping and reporting stay relative to ||b||
            btol = tol2 * bn2c;
        }

        for (int t = warm ? -1 : 0;; ++t) {
            const bool init = t < 0;   // the warm start's pass: Q = A X0, no update
            // Step 2: stopping test, then publish P = [Re p; Im p] (head, tail)
            if (!init && tol2 > 0.f && res2 <= btol) done = true;
            const int any = (init || (!done && t < T)) ? 1 : 0;
#pragma unroll
            for (int k = 0; k < RPT; ++k) {
                const float2 v = init ? x[k] : p[k];
                float ph, pl, qh, ql;
                tc::split_tf32(v.x, ph, pl);
                tc::split_tf32(v.y, qh, ql);
                const uint32_t o = p_off + (uint32_t)(2 * k) * LBO;
                st_shared_v2(b_hi + o, ph, qh);
                st_shared_v2(b_lo + o, pl, ql);
            }
            tc::fence_proxy_async_smem();
            tc::tc_fence_before();
            // the error flag enters the vote, so the team's decision is uniform
            const int cont = team_or(bar_id, any && !S.err);
            if (!cont) break;
            if (issuer) {
                tc::tc_fence_after();
                constexpr uint32_t idesc = tc::idesc_tf32(RR, GC);
                constexpr uint32_t idesc2 = tc::idesc_tf32(RR, 2 * GC);
                static_assert(NG == 1 && BPART == (GC / 8) * (int)SBO, "P tail tile directly after the head tile");
                const uint32_t bh0 = b_hi + (uint32_t)team * (GC / 8) * SBO;
#pragma unroll 4
                for (int kk = 0; kk < RR / 8; ++kk) {
                    const uint32_t off = (uint32_t)(2 * kk) * LBO;
                    const uint32_t ah = tmem + TA_HI + 8 * kk, al = tmem + TA_LO + 8 * kk;
                    const uint64_t bh = tc::smem_desc(bh0 + off, LBO, SBO);
                    // head x [P head | P tail] as one N = 128 MMA (the tail tile follows the head)
                    tc::mma_tf32_tmem_a(tq, ah, bh, idesc2, kk ? 1u : 0u);
                    tc::mma_tf32_tmem_a(tq + 2u * GC, al, bh, idesc, kk ? 1u : 0u);
                }
                tc::mma_commit(&S.qfull[team]);
            }
            __syncwarp();
            // ---- Q = A P: TMEM -> shared tile (real row 32 quad + lane) ----
            if (!tc::mbar_wait(&S.qfull[team], phase & 1, WAIT_LIMIT)) {
                err = 1;
                S.err = 1;   // seen by every thread after its team's next vote
            }
            ++phase;
            tc::tc_fence_after();
            {
                const uint32_t ta = tq + ((uint32_t)(32 * quad) << 16) + col_off;
                const uint32_t qrow = q_base + (uint32_t)((32 * quad + lane) * QLD + GC * team + col_off) * 4;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    float u0[16], u1[16], u2[16];
                    tc::tmem_ld16(ta + 16 * h, u0);
                    tc::tmem_ld16(ta + GC + 16 * h, u1);
                    tc::tmem_ld16(ta + 2 * GC + 16 * h, u2);
                    tc::tmem_ld_wait();
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        float v[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e) v[e] = (u0[4 * m + e] + u1[4 * m + e]) + u2[4 * m + e];
                        st_shared_v4(qrow + (16 * h + 4 * m) * 4, v[0], v[1], v[2], v[3]);
                    }
                }
            }
            team_sync(bar_id);
            float2 q[RPT];
#pragma unroll
            for (int k = 0; k < RPT; ++k) {
                const int i = g + 4 * k;
                q[k] = make_float2(S.Q[(2 * i) * QLD + j], S.Q[(2 * i + 1) * QLD + j]);
            }
            if (init) {   // r = b - A X0, then Step 1 from there
#pragma unroll
                for (int k = 0; k < RPT; ++k) {
                    r[k] = make_float2(r[k].x - q[k].x, r[k].y - q[k].y);
                    p[k] = make_float2(dv[k] * r[k].x, dv[k] * r[k].y);
                }
                rho = sumsq_col(r, p);
                res2 = sumsq_col(r, r);
                continue;
            }
            // lambda = r^H z / p^H A p (p^H A p is real for Hermitian A: Re part only)
            const float pAp = comp_value(col_total(dot2_rows(p, q)));
            float lam = 0.f;
            if (pAp > 0.f) lam = rho / pAp;
            else if (res2 != 0.f && !done) notHPD = 1;
            if (done) lam = 0.f;
            float2 z[RPT];
#pragma unroll
            for (int k = 0; k < RPT; ++k) {
                x[k].x = fmaf(lam, p[k].x, x[k].x);
                x[k].y = fmaf(lam, p[k].y, x[k].y);
                r[k].x = fmaf(-lam, q[k].x, r[k].x);
                r[k].y = fmaf(-lam, q[k].y, r[k].y);
                z[k] = make_float2(dv[k] * r[k].x, dv[k] * r[k].y);   // z = D^{-1} r
            }
            const float rz_new = sumsq_col(r, z);
            const float rr_new = sumsq_col(r, r);
            if (!done) {
                const float beta = rho != 0.f ? rz_new / rho : 0.f;
#pragma unroll
                for (int k = 0; k < RPT; ++k) {
                    p[k].x = fmaf(beta, p[k].x, z[k].x);
                    p[k].y = fmaf(beta, p[k].y, z[k].y);
                }
                rho = rz_new;
                res2 = rr_new;
                itmax = t + 1;
            }
        }

        // ---- outputs ----
        if (j < NCOL) {
#pragma unroll
            for (int k = 0; k < RPT; ++k) {
                const int i = g + 4 * k;
                float2 val = x[k];
                if (mode == 1) {   // X += dX
                    const float2 o = in.X[i + (size_t)j * 64];
                    val = make_float2(o.x + val.x, o.y + val.y);
                }
                in.X[i + (size_t)j * 64] = val;
                if (in.Xout && i < K) in.Xout[i + (size_t)j * K] = val;
            }
        }
        if (mode == 0 && g == 0) {   // one thread per column
            int f = err ? FLAG_TIMEOUT : 0;
            if (j < NCOL) {
                if (itmax > 0) atomicMax(acc_out.iters + id, itmax);
                const float rr = fmaxf(res2, 0.f);
                const float res = sqrtf(bn2c > 0.f ? rr / bn2c : rr);   // relative to ||b||
                if (res > 0.f) atomicMax(acc_out.resid_bits + id, __float_as_uint(res));
                if (notHPD) f |= FLAG_NOTHPD;
                if (tol2 > 0.f && !(res2 <= btol)) f |= FLAG_NOTCONV;
            }
            if (f) atomicOr(acc_out.flags + id, f);
        }
    }

    // every copy issued was waited for, except one whose wait ran out
    if (threadIdx.x == 0 && a_lost != ~0u) tc::mbar_wait(&S.abar, a_lost & 1, WAIT_LIMIT);
    if (issuer) {
        tc::mma_commit(&S.fin[team]);
        tc::mbar_wait(&S.fin[team], 0, WAIT_LIMIT);
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
                            const CUtensorMap *amap, const char *arena, cudaStream_t s, int mode) {
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
        kern<<<grid, NTHREADS, smem, s>>>(insts, list, n, acc, *amap, arena);
        return cudaGetLastError();
    };
    if (variant == 2) return mode ? go(pcg_tc64_kernel<2, 1>) : go(pcg_tc64_kernel<2, 0>);   // plain CG
    return mode ? go(pcg_tc64_kernel<0, 1>) : go(pcg_tc64_kernel<0, 0>);
}

}  // namespace jacpcg
