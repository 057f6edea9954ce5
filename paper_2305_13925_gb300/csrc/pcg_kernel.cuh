// pcg_kernel.cuh -- the Jac-PCG iteration for A X = I_K, all T iterations in one
// kernel (Sec. III-B Steps 1-4, Eqs. 12-14 and 19-21; Algorithm 1).
//
// Columns of X are independent right-hand sides (Eq. 16 per column), so a
// CTA owns a block of NW * CW columns of one instance and needs no data
// from any other CTA.  Warp w owns CW columns; lane l owns rows
// l, l + 32, ... (RPL rows; K classes below 32 leave lanes idle).  The
// iterate x, the residual r and the direction p of the owned entries live
// in registers for the whole solve.  The only heavy product per iteration,
// q = A p (8 K^2 flops per column), reads A from shared memory (resident
// for K <= 128; streamed in column chunks from L2 for K = 256) and the
// warp's own p columns from shared memory (broadcast).  The per-column dot
// products are compensated (Dot2) and reduced with warp shuffles in a
// fixed order, so every column's result is independent of the batch and of
// the launch shape.
//
// Variants (template VAR):
//   0 standard Jac-PCG in residual form: z = D^{-1} r, lambda = r^H z / p^H A p,
//     x += lambda p, r -= lambda A p, beta = r'^H z' / r^H z, p = z' + beta p;
//   1 Algorithm 1 as printed: r = D^{-1} b, m = r, alpha = r^H r / m^H D^{-1} A m
//     (complex), w += alpha m, r -= alpha D^{-1} A m, b = r'^H r' / r^H r,
//     m = r' + b m;
//   2 plain CG (variant 0 with D = I);
//   3 JOR (Sec. III-A), w^{t+1} = (I - omega D^{-1} A) w^t + omega D^{-1} b in
//     residual form: p = omega D^{-1} r, x += p, r -= A p (no step or direction
//     ratios; only ||r|| is reduced, for the stopping test).
// Stopping (tol > 0): a column stops before an update once
// ||r||^2 <= tol^2 ||b||^2 (Alg. 1: ||D r||^2).
// Right-hand side (mode): 0 solves A X = B (B = I_K, or the instance's
// symbol vectors, Eq. 16) and writes X -- from the initial point X0 when the
// instance has one (Sec. III-B Step 1: a pass before the first update forms
// A X0 with the iteration's own product, r = b - A X0, Alg. 1 scaling it by
// D^{-1}; the stopping test stays relative to ||b||); 1 solves A dX = R for the
// refinement residual R of the instance's workspace and adds dX to X
// (iterative refinement); only mode 0 reports iterations, residuals and
// non-convergence.
#pragma once

#include "common.cuh"
#include "kernels.h"

namespace jacpcg {
namespace pcgk {

template <int KC, int CW, int NW, bool RESIDENT, int VAR>
__global__ void __launch_bounds__(NW * 32) pcg_kernel(const DevInst *__restrict__ insts,
                                                      const int2 *__restrict__ blocks,
                                                      DevAccum acc_out, int mode) {
    constexpr int RPL = KC >= 32 ? KC / 32 : 1;  // rows per lane
    constexpr int KCH = 32;                       // A columns per streamed chunk (K = 256)
    extern __shared__ __align__(16) float2 smem[];
    float2 *A_s = smem;                                   // KC x KC (resident) or 2 x KC x KCH
    float2 *P_s = smem + (RESIDENT ? KC * KC : 2 * KC * KCH);  // NW x KC x CW

    const int2 blk = blocks[blockIdx.x];
    const DevInst &in = insts[blk.x];
    if (mode == 1 && in.rctl[1] != 0.f) return;   // the instance stopped refining
    const int K = in.K;
    const int T = in.max_iter;
    const bool warm = mode == 0 && in.X0 != nullptr;   // start from X0 (one extra product A X0)
    const float tl = (mode == 1 && in.rsolve_tol > 0.f) ? in.rsolve_tol : in.tol;   // correction solves
    const float tol2 = tl > 0.f ? tl * tl : -1.f;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const float2 *__restrict__ Ag = in.A;
    const float om = VAR == 3 ? in.omega : 1.f;   // JOR relaxation factor

    if (RESIDENT) {  // whole A into shared memory, 16 bytes per access
        const float4 *src = reinterpret_cast<const float4 *>(Ag);
        float4 *dst = reinterpret_cast<float4 *>(A_s);
        for (int e = threadIdx.x; e < KC * KC / 2; e += NW * 32) dst[e] = __ldg(src + e);
    }

    // owned rows and columns
    int row[RPL];
    bool rvalid[RPL];
    float dv[RPL], dd[RPL];
#pragma unroll
    for (int i = 0; i < RPL; ++i) {
        row[i] = lane + 32 * i;
        rvalid[i] = row[i] < K;
        const float di = rvalid[i] ? in.dinv[row[i]] : 0.f;
        dv[i] = (VAR == 2) ? (rvalid[i] ? 1.f : 0.f) : di;
        dd[i] = (VAR == 1 && rvalid[i]) ? 1.0f / di : 0.f;    // D for the Alg. 1 stopping test
    }
    int col[CW];
    bool cvalid[CW];
#pragma unroll
    for (int c = 0; c < CW; ++c) {
        col[c] = blk.y + warp * CW + c;
        cvalid[c] = col[c] < in.ncols;
    }

    // state: x (iterate), r (residual), p (direction; m in Alg. 1)
    float2 x[RPL][CW], r[RPL][CW], p[RPL][CW];
    float rho[CW];      // r^H z (standard / CG) or r^H r (Alg. 1)
    float res2[CW];     // squared stopping residual
    float btol[CW];     // tol^2 ||b||^2
    float bn2c[CW];     // ||b||^2 (the reported residual is relative to it)
    bool done[CW];
    int its[CW];
#pragma unroll
    for (int c = 0; c < CW; ++c) {
        Comp rz = {0.f, 0.f}, rs = {0.f, 0.f}, bb = {0.f, 0.f};
#pragma unroll
        for (int i = 0; i < RPL; ++i) {
            float2 b = make_float2(0.f, 0.f);
            if (mode == 0) {
                if (!in.B) {
                    if (rvalid[i] && row[i] == col[c]) b.x = 1.f;           // B = I
                } else if (rvalid[i] && cvalid[c]) {
                    b = in.B[row[i] + (size_t)col[c] * in.ldb];               // symbol vectors
                }
            } else if (rvalid[i] && cvalid[c]) {
                b = in.R[row[i] + (size_t)col[c] * KC];                       // refinement residual
            }
            comp_fma(bb, b.x, b.x);
            comp_fma(bb, b.y, b.y);
            x[i][c] = (warm && rvalid[i] && cvalid[c]) ? in.X0[row[i] + (size_t)col[c] * K]
                                                       : make_float2(0.f, 0.f);
            // a warm start keeps b in r until the first pass has formed A X0
            r[i][c] = (VAR == 1 && !warm) ? make_float2(dv[i] * b.x, dv[i] * b.y) : b;
            p[i][c] = make_float2(dv[i] * b.x, dv[i] * b.y);   // z = D^{-1} r (standard, CG); m = r (Alg. 1)
            if (VAR == 3) p[i][c] = make_float2(om * p[i][c].x, om * p[i][c].y);   // omega D^{-1} r
            const float2 z = make_float2(dv[i] * r[i][c].x, dv[i] * r[i][c].y);
            if (VAR == 1) {
                comp_fma(rz, r[i][c].x, r[i][c].x);
                comp_fma(rz, r[i][c].y, r[i][c].y);
                comp_fma(rs, dd[i] * r[i][c].x, dd[i] * r[i][c].x);
                comp_fma(rs, dd[i] * r[i][c].y, dd[i] * r[i][c].y);
            } else {
                comp_fma(rz, r[i][c].x, z.x);
                comp_fma(rz, r[i][c].y, z.y);
                comp_fma(rs, r[i][c].x, r[i][c].x);
                comp_fma(rs, r[i][c].y, r[i][c].y);
            }
        }
        rz = comp_warp_allreduce(rz);
        rs = comp_warp_allreduce(rs);
        bb = comp_warp_allreduce(bb);
        rho[c] = rz.s + rz.c;
        res2[c] = rs.s + rs.c;
        bn2c[c] = bb.s + bb.c;
        btol[c] = tol2 * bn2c[c];
        done[c] = !cvalid[c];
        its[c] = 0;
    }
    int notHPD = 0;

    float2 *Pw = P_s + (size_t)warp * KC * CW;   // this warp's p columns, [k][c]
    if (RESIDENT) __syncthreads();

    for (int t = warm ? -1 : 0; t < T; ++t) {
        const bool init = t < 0;   // the warm start's pass: q = A X0, no update
        // Step 2: stopping test before the update
        bool any = init;
#pragma unroll
        for (int c = 0; c < CW; ++c) {
            if (!init && !done[c] && tol2 > 0.f && res2[c] <= btol[c]) done[c] = true;
            any |= !done[c];
        }
        if (RESIDENT) {
            if (!any) break;              // warp-uniform: the warp's columns are all done
        } else {
            if (!__syncthreads_or(any)) break;   // every warp takes part in the chunk loop
        }

        // publish p for the product
#pragma unroll
        for (int i = 0; i < RPL; ++i)
#pragma unroll
            for (int c = 0; c < CW; ++c)
                if (row[i] < KC) Pw[row[i] * CW + c] = init ? x[i][c] : p[i][c];
        __syncwarp();

        // q = A p
        float2 q[RPL][CW];
#pragma unroll
        for (int i = 0; i < RPL; ++i)
#pragma unroll
            for (int c = 0; c < CW; ++c) q[i][c] = make_float2(0.f, 0.f);
        if (RESIDENT) {
#pragma unroll 4
            for (int k = 0; k < K; ++k) {
                float2 pk[CW];
#pragma unroll
                for (int c = 0; c < CW; ++c) pk[c] = Pw[k * CW + c];
#pragma unroll
                for (int i = 0; i < RPL; ++i) {
                    const float2 a = (KC >= 32 || row[i] < KC) ? A_s[k * KC + row[i]]
                                                               : make_float2(0.f, 0.f);
#pragma unroll
                    for (int c = 0; c < CW; ++c) cfma(q[i][c], a, pk[c]);
                }
            }
        } else {
            // A streamed from global (L2) in chunks of KCH columns, double buffered
            const int nch = (K + KCH - 1) / KCH;
            auto issue = [&](int ch, int buf) {
                const float4 *src = reinterpret_cast<const float4 *>(Ag + (size_t)ch * KCH * KC);
                float2 *dstb = A_s + (size_t)buf * KC * KCH;
                for (int e = threadIdx.x; e < KC * KCH / 2; e += NW * 32) {
                    const unsigned dst = (unsigned)__cvta_generic_to_shared(dstb + 2 * e);
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst),
                                 "l"(src + e));
                }
                asm volatile("cp.async.commit_group;\n" ::);
            };
            issue(0, 0);
            for (int ch = 0; ch < nch; ++ch) {
                if (ch + 1 < nch) {
                    issue(ch + 1, (ch + 1) & 1);
                    asm volatile("cp.async.wait_group 1;\n" ::);
                } else {
                    asm volatile("cp.async.wait_group 0;\n" ::);
                }
                __syncthreads();
                const float2 *Ab = A_s + (size_t)(ch & 1) * KC * KCH;
                const int kend = min(KCH, K - ch * KCH);
#pragma unroll 4
                for (int kk = 0; kk < kend; ++kk) {
                    const int k = ch * KCH + kk;
                    float2 pk[CW];
#pragma unroll
                    for (int c = 0; c < CW; ++c) pk[c] = Pw[k * CW + c];
#pragma unroll
                    for (int i = 0; i < RPL; ++i) {
                        const float2 a = Ab[kk * KC + row[i]];
#pragma unroll
                        for (int c = 0; c < CW; ++c) cfma(q[i][c], a, pk[c]);
                    }
                }
                __syncthreads();   // buffer (ch & 1) is refilled two chunks later
            }
        }
        __syncwarp();

        if (init) {
            // r = b - A X0 (Alg. 1: D^{-1} (b - A X0)), then Step 1 from there
#pragma unroll
            for (int c = 0; c < CW; ++c) {
                Comp rz = {0.f, 0.f}, rs = {0.f, 0.f};
#pragma unroll
                for (int i = 0; i < RPL; ++i) {
                    float2 rw = make_float2(r[i][c].x - q[i][c].x, r[i][c].y - q[i][c].y);
                    if (VAR == 1) {
                        rw = make_float2(dv[i] * rw.x, dv[i] * rw.y);
                        r[i][c] = rw;
                        p[i][c] = rw;
                        comp_fma(rz, rw.x, rw.x);
                        comp_fma(rz, rw.y, rw.y);
                        comp_fma(rs, dd[i] * rw.x, dd[i] * rw.x);
                        comp_fma(rs, dd[i] * rw.y, dd[i] * rw.y);
                    } else {
                        r[i][c] = rw;
                        const float2 z = make_float2(dv[i] * rw.x, dv[i] * rw.y);
                        p[i][c] = VAR == 3 ? make_float2(om * z.x, om * z.y) : z;
                        comp_fma(rz, rw.x, z.x);
                        comp_fma(rz, rw.y, z.y);
                        comp_fma(rs, rw.x, rw.x);
                        comp_fma(rs, rw.y, rw.y);
                    }
                }
                rz = comp_warp_allreduce(rz);
                rs = comp_warp_allreduce(rs);
                rho[c] = rz.s + rz.c;
                res2[c] = rs.s + rs.c;
            }
            __syncwarp();   // p columns in shared memory are rewritten next pass
            continue;
        }

        // scalars and vector updates, column by column
#pragma unroll
        for (int c = 0; c < CW; ++c) {
            if (VAR == 3) {
                // JOR: x += p, r -= A p, p = omega D^{-1} r
                const bool upd = !done[c];
                Comp rs = {0.f, 0.f};
#pragma unroll
                for (int i = 0; i < RPL; ++i) {
                    if (upd) {
                        x[i][c].x += p[i][c].x;
                        x[i][c].y += p[i][c].y;
                        r[i][c].x -= q[i][c].x;
                        r[i][c].y -= q[i][c].y;
                        p[i][c] = make_float2(om * (dv[i] * r[i][c].x), om * (dv[i] * r[i][c].y));
                    }
                    comp_fma(rs, r[i][c].x, r[i][c].x);
                    comp_fma(rs, r[i][c].y, r[i][c].y);
                }
                rs = comp_warp_allreduce(rs);
                if (upd) {
                    res2[c] = rs.s + rs.c;
                    ++its[c];
                }
            } else if (VAR == 1) {
                // u = D^{-1} A m, den = m^H u (complex)
                Comp dr = {0.f, 0.f}, di = {0.f, 0.f};
#pragma unroll
                for (int i = 0; i < RPL; ++i) {
                    q[i][c].x *= dv[i];
                    q[i][c].y *= dv[i];
                    comp_fma(dr, p[i][c].x, q[i][c].x);
                    comp_fma(dr, p[i][c].y, q[i][c].y);
                    comp_fma(di, p[i][c].x, q[i][c].y);
                    comp_fma(di, -p[i][c].y, q[i][c].x);
                }
                dr = comp_warp_allreduce(dr);
                di = comp_warp_allreduce(di);
                const float denr = dr.s + dr.c, deni = di.s + di.c;
                float2 alpha = make_float2(0.f, 0.f);
                const float den2 = denr * denr + deni * deni;
                if (den2 > 0.f) {
                    alpha = make_float2(rho[c] * denr / den2, -rho[c] * deni / den2);
                } else if (rho[c] != 0.f && !done[c]) {
                    notHPD = 1;
                }
                if (done[c]) alpha = make_float2(0.f, 0.f);
                Comp rr = {0.f, 0.f}, rs = {0.f, 0.f};
#pragma unroll
                for (int i = 0; i < RPL; ++i) {
                    cfma(x[i][c], alpha, p[i][c]);
                    cfma(r[i][c], make_float2(-alpha.x, -alpha.y), q[i][c]);
                    comp_fma(rr, r[i][c].x, r[i][c].x);
                    comp_fma(rr, r[i][c].y, r[i][c].y);
                    comp_fma(rs, dd[i] * r[i][c].x, dd[i] * r[i][c].x);
                    comp_fma(rs, dd[i] * r[i][c].y, dd[i] * r[i][c].y);
                }
                rr = comp_warp_allreduce(rr);
                rs = comp_warp_allreduce(rs);
                const float rr_new = rr.s + rr.c;
                const float bt = rho[c] != 0.f ? rr_new / rho[c] : 0.f;
                if (!done[c]) {
#pragma unroll
                    for (int i = 0; i < RPL; ++i) {
                        p[i][c].x = fmaf(bt, p[i][c].x, r[i][c].x);
                        p[i][c].y = fmaf(bt, p[i][c].y, r[i][c].y);
                    }
                    rho[c] = rr_new;
                    res2[c] = rs.s + rs.c;
                    ++its[c];
                }
            } else {
                Comp pq = {0.f, 0.f};
#pragma unroll
                for (int i = 0; i < RPL; ++i) {
                    comp_fma(pq, p[i][c].x, q[i][c].x);
                    comp_fma(pq, p[i][c].y, q[i][c].y);
                }
                pq = comp_warp_allreduce(pq);
                const float pAp = pq.s + pq.c;
                float lambda = 0.f;
                if (pAp > 0.f) {
                    lambda = rho[c] / pAp;
                } else if (res2[c] != 0.f && !done[c]) {
                    notHPD = 1;
                }
                if (done[c]) lambda = 0.f;
                Comp rz = {0.f, 0.f}, rs = {0.f, 0.f};
                float2 z[RPL];
#pragma unroll
                for (int i = 0; i < RPL; ++i) {
                    x[i][c].x = fmaf(lambda, p[i][c].x, x[i][c].x);
                    x[i][c].y = fmaf(lambda, p[i][c].y, x[i][c].y);
                    r[i][c].x = fmaf(-lambda, q[i][c].x, r[i][c].x);
                    r[i][c].y = fmaf(-lambda, q[i][c].y, r[i][c].y);
                    z[i] = make_float2(dv[i] * r[i][c].x, dv[i] * r[i][c].y);
                    comp_fma(rz, r[i][c].x, z[i].x);
                    comp_fma(rz, r[i][c].y, z[i].y);
                    comp_fma(rs, r[i][c].x, r[i][c].x);
                    comp_fma(rs, r[i][c].y, r[i][c].y);
                }
                rz = comp_warp_allreduce(rz);
                rs = comp_warp_allreduce(rs);
                const float rz_new = rz.s + rz.c;
                const float beta = rho[c] != 0.f ? rz_new / rho[c] : 0.f;
                if (!done[c]) {
#pragma unroll
                    for (int i = 0; i < RPL; ++i) {
                        p[i][c].x = fmaf(beta, p[i][c].x, z[i].x);
                        p[i][c].y = fmaf(beta, p[i][c].y, z[i].y);
                    }
                    rho[c] = rz_new;
                    res2[c] = rs.s + rs.c;
                    ++its[c];
                }
            }
        }
        __syncwarp();   // p columns in shared memory are rewritten next iteration
    }

    // outputs: X (workspace ld KC; caller's ld K), per-instance accumulators
#pragma unroll
    for (int c = 0; c < CW; ++c) {
        if (!cvalid[c]) continue;
#pragma unroll
        for (int i = 0; i < RPL; ++i) {
            if (row[i] >= KC) continue;
            float2 v = x[i][c];
            if (mode == 1) {   // X += dX
                const float2 o = in.X[row[i] + (size_t)col[c] * KC];
                v = make_float2(o.x + v.x, o.y + v.y);
            }
            in.X[row[i] + (size_t)col[c] * KC] = v;
            if (in.Xout && rvalid[i]) in.Xout[row[i] + (size_t)col[c] * K] = v;
        }
    }
    if (mode != 0) return;
    int itmax = 0;
    float resmax = 0.f;
    bool notconv = false;
#pragma unroll
    for (int c = 0; c < CW; ++c) {
        if (!cvalid[c]) continue;
        itmax = max(itmax, its[c]);
        const float rr = fmaxf(res2[c], 0.f);
        resmax = fmaxf(resmax, sqrtf(bn2c[c] > 0.f ? rr / bn2c[c] : rr));
        if (tol2 > 0.f && !(res2[c] <= btol[c])) notconv = true;
    }
    if (lane == 0) {
        if (itmax > 0) atomicMax(acc_out.iters + blk.x, itmax);
        if (resmax > 0.f) atomicMax(acc_out.resid_bits + blk.x, __float_as_uint(resmax));
        const int f = (notHPD ? FLAG_NOTHPD : 0) | (notconv ? FLAG_NOTCONV : 0);
        if (f) atomicOr(acc_out.flags + blk.x, f);
    }
}

template <int KC, int CW, int NW, bool RES>
cudaError_t launch_cfg(int variant, const DevInst *insts, const int2 *blocks, int n_blocks,
                       DevAccum acc, cudaStream_t s, int mode) {
    constexpr int KCH = 32;
    const size_t smem = sizeof(float2) * ((RES ? KC * KC : 2 * KC * KCH) + (size_t)NW * KC * CW);
    cudaError_t e = cudaSuccess;
    auto go = [&](auto kern) {
        if (smem > 48 * 1024) {
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return;
        }
        kern<<<n_blocks, NW * 32, smem, s>>>(insts, blocks, acc, mode);
        e = cudaGetLastError();
    };
    switch (variant) {
        case 0: go(pcg_kernel<KC, CW, NW, RES, 0>); break;
        case 1: go(pcg_kernel<KC, CW, NW, RES, 1>); break;
        case 2: go(pcg_kernel<KC, CW, NW, RES, 2>); break;
        case 3: go(pcg_kernel<KC, CW, NW, RES, 3>); break;
        default: return cudaErrorInvalidValue;
    }
    return e;
}

}  // namespace pcgk
}  // namespace jacpcg
