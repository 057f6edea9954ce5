// hx_bf16.cu -- the precoder W = H X on the tcgen05 tensor cores for bfloat16
// channels of the K = 128 and 256 classes (Eq. 7 without the power factor;
// Eq. 15 per symbol), the tensor core reading H as it lies in memory.
//
// H's memory read as a real 2M x K matrix U (column a = (Re h_0a, Im h_0a,
// Re h_1a, ...)) is the MMAs' A operand, MN-major.  D1 = U Xr and D2 = U Xi
// give, for antenna m,
//   Re W[m, n] = D1[2m, n] - D2[2m + 1, n],  Im W[m, n] = D1[2m + 1, n] + D2[2m, n],
// the two rows of an antenna sitting in adjacent TMEM lanes (one shuffle).
// X is FP32; it enters as three bfloat16 terms X = X1 + X2 + X3, each the
// rounding of what the previous ones leave, which sum to X exactly, so every
// product is exact in FP32.
//
// A job is (instance, output group g): the 32 columns 32 g .. 32 g + 31 of W.
// B = [Xr^T ; Xi^T] of those columns (64 rows, K-major, no swizzle, three
// terms: 96 KB for K = 256) stays in shared memory for the whole job; H
// streams through a ring of stages of 128 rows of U x 128 users, two tiled
// TMA copies each (128-byte swizzle, zero-filled past M and K).  The three
// terms' rows of B follow each other, so one N = 192 MMA per 16 users forms
// the X1, X2 and X3 products side by side in TMEM: three accumulation chains
// of K / 16 MMAs per 128-row tile (the tensor core's FP32 accumulation
// truncates; no chain is longer than the Gram's), added by the epilogue.
//
// Persistent, warp-specialised, one CTA per SM walking its jobs:
//   warps 0-7   at the start of a job (the previous job's MMAs done) build B
//               from X; then the epilogue: TMEM lanes 32 (w mod 4) .. (rows
//               of U), columns 16 (w / 4) .. of the group -> W (complex64,
//               column-major, coalesced) and the tile's ||W||_F^2 partial in
//               slot g * (row tiles) + tile;
//   warp 8      lane 0 issues the tensor copies, up to RING stages ahead;
//   warp 9      TMEM allocation (NBUF tiles of 192 columns); lane 0 issues
//               the MMAs and commits.
// Every wait is bounded; a timeout stops the CTA's pipeline, flags its
// instances with FLAG_TIMEOUT, and the CTA still drains and frees its TMEM.
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"
#include "tc.cuh"

namespace jacpcg {

namespace {

constexpr int NB = 32;                    // output columns per job
constexpr int BR = 2 * NB;                // B rows: Xr^T then Xi^T
constexpr int TR = 128;                   // rows of U (64 antennas) per tile: MMA M
constexpr int KU = 128;                   // users per stage: fewer, larger tensor copies (two per
                                          // stage) -- 64-user stages, twice the copies from one
                                          // issuing thread, took 1.34 against 1.17 ms on the XL batch
constexpr int BOX = KU * 128;             // one tensor copy: 128 users x 64 values (16 KB)
constexpr int UST = 2 * BOX;              // one stage: 128 rows of U x 128 users
constexpr int RING = 4;
constexpr int KCMAX = 256;
constexpr int BTERM = BR * KCMAX * 2;     // one bfloat16 term of B (32 KB)
constexpr int NBUF = 2;                   // TMEM tile buffers: X1 | X2 | X3 products, 64 columns each
constexpr int NEW = 8;                    // epilogue warps
constexpr int TMA_WARP = NEW, MMA_WARP = NEW + 1;
constexpr int NTHREADS = (NEW + 2) * 32;
constexpr int TMEM_COLS = 512;            // NBUF x 3 x BR = 384 used
constexpr uint32_t WAIT_LIMIT = 1u << 21;
constexpr int BAR_EPI = 1;                // named barrier of the epilogue warps

struct __align__(1024) HxBSmem {
    unsigned char ring[RING][UST];        // each 1024-byte aligned (the swizzle atom)
    unsigned char B[3][BTERM];
    uint64_t full[RING];                  // the stage's tensor copies landed
    uint64_t empty[RING];                 // its MMAs completed
    uint64_t accf[NBUF];                  // tile buffer complete
    uint64_t tfree[NBUF];                 // tile buffer read by the epilogue
    uint64_t bready;                      // B of the job built
    uint64_t fin;
    float red[2][NEW];
    uint32_t tmem;
    volatile int err;
};
static_assert(sizeof(HxBSmem) + 1024 <= 227 * 1024, "shared memory");

__device__ __forceinline__ int n_tiles(int M) { return (M + TR / 2 - 1) / (TR / 2); }

__device__ __forceinline__ uint32_t bf16_bits(float x) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }

// x = t1 + t2 + t3 exactly, each a bfloat16 (round to nearest)
__device__ __forceinline__ void split3(float x, uint32_t &t1, uint32_t &t2, uint32_t &t3) {
    const __nv_bfloat16 h1 = __float2bfloat16_rn(x);
    const float r1 = x - __bfloat162float(h1);
    const __nv_bfloat16 h2 = __float2bfloat16_rn(r1);
    const float r2 = r1 - __bfloat162float(h2);
    t1 = __bfloat16_as_ushort(h1);
    t2 = __bfloat16_as_ushort(h2);
    t3 = bf16_bits(r2);
}

__global__ void __launch_bounds__(NTHREADS, 1) hx_bf16_kernel(const DevInst *__restrict__ insts,
                                                              const int4 *__restrict__ jobs, int n_jobs,
                                                              const CUtensorMap *__restrict__ maps,
                                                              DevAccum acc_out) {
    extern __shared__ unsigned char smem_raw[];
    const uint32_t pad = (1024u - (tc::smem_u32(smem_raw) & 1023u)) & 1023u;
    HxBSmem &S = *reinterpret_cast<HxBSmem *>(smem_raw + pad);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < RING; ++s) {
            tc::mbar_init(&S.full[s], 1);
            tc::mbar_init(&S.empty[s], 1);
        }
        for (int b = 0; b < NBUF; ++b) {
            tc::mbar_init(&S.accf[b], 1);
            tc::mbar_init(&S.tfree[b], NEW);
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
    const uint32_t ring0 = tc::smem_u32(S.ring[0]);
    const uint32_t b0 = tc::smem_u32(S.B[0]);

    if (warp < NEW) {
        // ---------------- B from X, then the epilogue ----------------
        const int t = threadIdx.x, quad = warp & 3, part = warp >> 2;
        uint32_t seqt = 0;
        int red_p = 0;
        // The epilogue warps meet at a named barrier every tile, so they walk every
        // job and tile whatever happens; after a timeout they skip the waits.
        for (int j = blockIdx.x; j < n_jobs; j += gridDim.x) {
            const int4 job = jobs[j];
            const DevInst &in = insts[job.x];
            const int K = in.K, KC = in.KC, M = in.M, ncols = in.ncols, n0 = NB * job.y;
            const int nag = KC / 8;                  // 8-user groups along K
            const uint32_t sbo = nag * 128;
            // B term tt, row r (0..63), users a..a+7 (a = 8 ag): 16 bytes at
            // (8 tt + r / 8) * sbo + ag * 128 + (r % 8) * 16: the three terms' rows follow
            // each other, so one N = 192 MMA multiplies all three
            const float2 *__restrict__ X = in.X;
            for (int e = t; e < NB * nag; e += NEW * 32) {
                const int r8 = e & 7, ag = (e >> 3) % nag, ng = (e >> 3) / nag;
                const int nl = 8 * ng + r8, n = n0 + nl;
                uint32_t re[3][4], im[3][4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {   // users 8 ag + 2 q, + 1
                    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                    const int a = 8 * ag + 2 * q;
                    if (n < ncols && a < K) {
                        v = *reinterpret_cast<const float4 *>(X + a + (size_t)n * KC);
                        if (a + 1 >= K) v.z = v.w = 0.f;
                    }
                    uint32_t r0[3], r1[3], i0[3], i1[3];
                    split3(v.x, r0[0], r0[1], r0[2]);
                    split3(v.z, r1[0], r1[1], r1[2]);
                    split3(v.y, i0[0], i0[1], i0[2]);
                    split3(v.w, i1[0], i1[1], i1[2]);
#pragma unroll
                    for (int tt = 0; tt < 3; ++tt) {
                        re[tt][q] = r0[tt] | (r1[tt] << 16);
                        im[tt][q] = i0[tt] | (i1[tt] << 16);
                    }
                }
#pragma unroll
                for (int tt = 0; tt < 3; ++tt) {
                    const uint32_t base = b0 + tt * 8 * sbo + ag * 128 + r8 * 16;   // terms stacked along N
                    const uint32_t ar = base + ng * sbo, ai = base + (NB / 8 + ng) * sbo;
                    asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};\n" ::"r"(ar), "r"(re[tt][0]),
                                 "r"(re[tt][1]), "r"(re[tt][2]), "r"(re[tt][3])
                                 : "memory");
                    asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};\n" ::"r"(ai), "r"(im[tt][0]),
                                 "r"(im[tt][1]), "r"(im[tt][2]), "r"(im[tt][3])
                                 : "memory");
                }
            }
            tc::fence_proxy_async_smem();   // the tensor core reads B
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&S.bready);

            const int nmt = n_tiles(M);
            float *__restrict__ Wf = reinterpret_cast<float *>(in.W);
            const size_t ldw2 = 2 * (size_t)in.ldw;
            for (int mt = 0; mt < nmt; ++mt, ++seqt) {
                const int buf = seqt % NBUF;
                bool ok = !S.err;
                if (ok && !tc::mbar_wait(&S.accf[buf], (seqt / NBUF) & 1, WAIT_LIMIT)) {
                    S.err = 1;
                    ok = false;
                }
                ok = __all_sync(0xffffffffu, ok);
                float d1[16], d2[16], v[16], w[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) d1[i] = d2[i] = 0.f;
                if (ok) {
                    tc::tc_fence_after();
                    const uint32_t ta = tmem + ((uint32_t)(32 * quad) << 16) + buf * 3 * BR + 16 * part;
                    tc::tmem_ld16(ta, d1);               // X1 products, Xr columns
                    tc::tmem_ld16(ta + BR, v);           // X2
                    tc::tmem_ld16(ta + 2 * BR, w);       // X3
                    tc::tmem_ld_wait();
#pragma unroll
                    for (int i = 0; i < 16; ++i) d1[i] += v[i] + w[i];
                    tc::tmem_ld16(ta + NB, d2);          // X1 products, Xi columns
                    tc::tmem_ld16(ta + BR + NB, v);
                    tc::tmem_ld16(ta + 2 * BR + NB, w);
                    tc::tmem_ld_wait();
#pragma unroll
                    for (int i = 0; i < 16; ++i) d2[i] += v[i] + w[i];
                    tc::tc_fence_before();
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(&S.tfree[buf]);
                }
                const int row = TR * mt + 32 * quad + lane;   // 2 m + (0 re, 1 im)
                const bool odd = lane & 1, live = (row >> 1) < M;
                float s = 0.f;
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const float p = __shfl_xor_sync(0xffffffffu, d2[i], 1);
                    const float w = odd ? d1[i] + p : d1[i] - p;
                    const int n = n0 + 16 * part + i;
                    if (live && n < ncols) {
                        Wf[row + (size_t)n * ldw2] = w;
                        s = fmaf(w, w, s);
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                if (lane == 0) S.red[red_p][warp] = s;
                asm volatile("bar.sync %0, %1;\n" ::"r"(BAR_EPI), "r"(NEW * 32) : "memory");
                if (t == 0) {
                    float tot = 0.f;
#pragma unroll
                    for (int w = 0; w < NEW; ++w) tot += S.red[red_p][w];
                    in.wpart[job.y * nmt + mt] = tot;
                }
                red_p ^= 1;
            }
            if (S.err && t == 0) atomicOr(acc_out.flags + job.x, FLAG_TIMEOUT);
        }
    } else if (warp == TMA_WARP) {
        // ---------------- tensor copies ----------------
        if (lane == 0) {
            uint32_t seq = 0;
            for (int j = blockIdx.x; j < n_jobs && !S.err; j += gridDim.x) {
                const int4 job = jobs[j];
                const DevInst &in = insts[job.x];
                const CUtensorMap *map = maps + job.z;
                tc::tensormap_acquire(map);
                const int nmt = n_tiles(in.M), nkc = in.KC / KU;
                for (int mt = 0; mt < nmt && !S.err; ++mt) {
                    for (int kc = 0; kc < nkc; ++kc, ++seq) {
                        const int s = seq % RING;
                        if (seq >= RING && !tc::mbar_wait(&S.empty[s], ((seq / RING) - 1) & 1, WAIT_LIMIT)) {
                            S.err = 1;
                            break;
                        }
                        const uint32_t dst = ring0 + s * UST;
                        tc::mbar_arrive_expect_tx(&S.full[s], UST);
                        tc::tma_load_2d(dst, map, TR * mt, KU * kc, &S.full[s]);
                        tc::tma_load_2d(dst + BOX, map, TR * mt + TR / 2, KU * kc, &S.full[s]);
                    }
                }
            }
            // no copy may still be landing when the CTA exits
            for (uint32_t q = seq > RING ? seq - RING : 0; q < seq; ++q)
                tc::mbar_wait(&S.full[q % RING], (q / RING) & 1, WAIT_LIMIT);
        }
    } else {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            constexpr uint32_t idesc = tc::idesc_bf16(TR, 3 * BR, /*a_mn=*/true, /*b_mn=*/false);
            uint32_t seq = 0, seqt = 0, njob = 0;
            for (int j = blockIdx.x; j < n_jobs && !S.err; j += gridDim.x, ++njob) {
                const int4 job = jobs[j];
                const DevInst &in = insts[job.x];
                const int nmt = n_tiles(in.M), nkc = in.KC / KU;
                const uint32_t sbo = (in.KC / 8) * 128;
                if (!tc::mbar_wait(&S.bready, njob & 1, WAIT_LIMIT)) {
                    S.err = 1;
                    break;
                }
                tc::tc_fence_after();
                for (int mt = 0; mt < nmt && !S.err; ++mt, ++seqt) {
                    const int buf = seqt % NBUF;
                    if (seqt >= NBUF) {   // the epilogue has read the buffer's previous tile
                        if (!tc::mbar_wait(&S.tfree[buf], ((seqt / NBUF) - 1) & 1, WAIT_LIMIT)) {
                            S.err = 1;
                            break;
                        }
                        tc::tc_fence_after();
                    }
                    const uint32_t d = tmem + buf * 3 * BR;
                    for (int kc = 0; kc < nkc; ++kc, ++seq) {
                        const int s = seq % RING;
                        if (!tc::mbar_wait(&S.full[s], (seq / RING) & 1, WAIT_LIMIT)) {
                            S.err = 1;
                            break;
                        }
                        tc::tc_fence_after();
                        const uint32_t u = ring0 + s * UST;
#pragma unroll
                        for (int kk = 0; kk < KU / 16; ++kk) {
                            // 16 users: rows 16 kk .. of both boxes; B columns (8 kc + 2 kk) .. of 8 users
                            const uint64_t ad = tc::smem_desc_sw128(u + kk * 2048, BOX, 1024);
                            const uint32_t boff = ((KU / 8) * kc + 2 * kk) * 128;
                            const bool first = kc == 0 && kk == 0;
                            // all three terms (N = 192: X1 | X2 | X3 products side by side)
                            tc::mma_bf16(d, ad, tc::smem_desc(b0 + boff, 128, sbo), idesc, first ? 0u : 1u);
                        }
                        tc::mma_commit(&S.empty[s]);
                    }
                    tc::mma_commit(&S.accf[buf]);
                }
            }
            tc::mma_commit(&S.fin);
            tc::mbar_wait(&S.fin, 0, WAIT_LIMIT);   // no MMA in flight past this point
        }
    }

    tc::tc_fence_before();
    __syncthreads();
    if (S.err && threadIdx.x == 0) {
        for (int j = blockIdx.x; j < n_jobs; j += gridDim.x) atomicOr(acc_out.flags + jobs[j].x, FLAG_TIMEOUT);
    }
    if (warp == MMA_WARP) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, TMEM_COLS);
    }
}

}  // namespace

cudaError_t launch_hx_bf16(const DevInst *insts, const int4 *jobs, int n, const CUtensorMap *maps, DevAccum acc,
                           cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const size_t smem = sizeof(HxBSmem) + 1024;   // + alignment of the ring to the swizzle atom
    cudaError_t e = cudaFuncSetAttribute(hx_bf16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const int grid = n < sms ? n : sms;
    hx_bf16_kernel<<<grid, NTHREADS, smem, s>>>(insts, jobs, n, maps, acc);
    return cudaGetLastError();
}

}  // namespace jacpcg
