// gram_tc.cu -- A = H^H H + xi I on the tcgen05 tensor cores (Sec. II,
// definition of P_i after Eq. 7; diag for Eq. 21): the diagonal 64 x 64
// blocks.  A job is (instance, user group a): the Gram of the 64 users
// 64 a .. 64 a + 63 written into block (a, a) of A (leading dimension KC) with
// its 1/diag entries; for the K = 64 class that is all of A, for the 128 and
// 256 classes gram_tc_cross.cu computes the off-diagonal blocks.
//
// Complex arithmetic as one real GEMM: with Y = [Re H | Im H] (M x 2K real),
// D = Y^T Y (2K x 2K) gives Re A = D11 + D22 and Im A = D12 - D21.  For
// K = 64, D is one 128 x 128 tcgen05 tile (M = N = 128, FP32 in tensor memory).
//
// FP32 accuracy from TF32 units (3xTF32; Ootomo and Yokota, "Recovering
// single precision accuracy from Tensor Cores while surpassing the FP32
// theoretical peak performance", IJHPCA 2022): every staged value is split
// y = hi + lo (hi = y rounded to TF32, lo = exact remainder), and
// D = Yh^T Yh + Yh^T Yl + Yl^T Yh.  D is symmetric, so the two correction
// products are transposes of each other: the tile accumulates only
// E = Yh^T Yl and the epilogue adds E + E^T, two MMAs per k-step instead of
// three.  The tensor core's FP32 accumulation rounds toward zero, so long
// accumulation chains drift: the head product's reduction over M is cut into
// groups of G stages, each accumulated into one of two TMEM buffers from
// zero, and drain warps add the group results into FP32 registers while the
// next group accumulates into the other buffer.  E is about 2^-11 of D, so
// its drift stays far below FP32 rounding of D: it accumulates over the whole
// instance in a third buffer (two, alternating between instances).
//
// Persistent, warp-specialised: the CTA walks its share of the instances.
//   warps 0-7   producers: H streamed with per-thread asynchronous copies
//               (cp.async, 16 bytes, zero-filled past M and K) RAW - 1 stages
//               ahead into a ring of raw stages, then TF32 split into Y^T
//               stage tiles (hi, lo) in the canonical no-swizzle K-major
//               layout.  Warp w owns the 8 columns k = 8 i + ((w + i) mod 8),
//               i = 0..7, of every stage: each copy instruction reads whole
//               column pieces (two of 256 bytes), which streams H near the
//               HBM rate where scattered 64-byte pieces did not; the raw
//               chunks are XOR-swizzled by i, so copies, raw reads and split
//               stores are free of bank conflicts; a warp reads only what it
//               copied, so a __syncwarp after its own cp.async wait suffices;
//   warps 8-15  drain/epilogue: TMEM -> registers per group; at the end of an
//               instance head sums + E + E^T go through shared memory into A
//               (lower triangle mirrored, so A is exactly Hermitian) and
//               1/diag(A);
//   warp 16     TMEM allocation; lane 0 issues the MMAs and commits.
// Every wait is bounded; a timeout stops the CTA's pipeline, flags its
// instances with FLAG_TIMEOUT, and the CTA still drains and frees its TMEM.
#include "common.cuh"
#include "kernels.h"
#include "tc.cuh"

namespace jacpcg {

namespace {

constexpr int ROWS = 128;                     // 2K rows of Y^T for K = 64
constexpr int MCH = 32;                       // H rows (reduction values) per stage
// Three split stages and a 4-deep raw ring fill the shared memory next to the
// epilogue tile; against two split stages and a 6-deep ring this measured
// 0.294 vs 0.307 ms per 2048-channel batch: decoupling the producers from the
// MMA warp pays more than more loads in flight.
constexpr int STAGES = 3;                     // split stages shared with the MMA warp
constexpr int RAW = 4;                        // raw stages in flight per producer thread
constexpr int RAWB = MCH * 64 * 8;            // bytes of one raw stage (16 KB)
constexpr int G = 4;                          // stages per accumulation group
constexpr int PART = ROWS * MCH * 4;          // bytes of one part (hi or lo) of a stage
constexpr uint32_t LBO = 128;                 // K-adjacent core matrices
constexpr uint32_t SBO = (MCH / 4) * 128;     // 8-row groups
constexpr uint32_t WAIT_LIMIT = 1u << 21;
constexpr int DPITCH = ROWS + 1;              // floats per staged D row
constexpr int NPW = 8, NDW = 8;               // producer and drain warps
constexpr int MMA_WARP = NPW + NDW;
constexpr int NTHREADS = (NPW + NDW + 1) * 32;
constexpr int TMEM_COLS = 4 * ROWS;           // two head-group buffers, two correction buffers

struct __align__(128) GramSmem {
    unsigned char stage[STAGES][2 * PART];
    unsigned char raw[RAW][RAWB];               // [q][part][thread] 16-byte chunks
    float D[ROWS * DPITCH];
    uint64_t full[STAGES];
    uint64_t empty[STAGES];
    uint64_t accf[2];
    uint64_t acce[2];
    uint64_t core[2];                          // correction buffer drained
    uint64_t fin;
    uint32_t tmem;
    volatile int err;
};

static_assert(sizeof(GramSmem) <= 227 * 1024, "shared memory");

__device__ __forceinline__ void st_shared_v4(uint32_t addr, float a, float b, float c, float d) {
    asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};\n" ::"r"(addr), "f"(a), "f"(b), "f"(c),
                 "f"(d)
                 : "memory");
}

__global__ void __launch_bounds__(NTHREADS, 1) gram_tc64_kernel(const DevInst *__restrict__ insts,
                                                                const int2 *__restrict__ list, int n_list,
                                                                DevAccum acc_out) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    GramSmem &S = *reinterpret_cast<GramSmem *>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            tc::mbar_init(&S.full[s], NPW);
            tc::mbar_init(&S.empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            tc::mbar_init(&S.accf[b], 1);
            tc::mbar_init(&S.acce[b], NDW);
            tc::mbar_init(&S.core[b], NDW);
        }
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

    if (warp < NPW) {
        // ---------------- producers ----------------
        const uint32_t raw0 = tc::smem_u32(S.raw[0]);
        // stream cursor: (instance ordinal, stage) in this CTA's walk
        struct Cursor {
            int j, c, nch, M, K, ldh;   // K: users of the job's group that exist (K - 64 a)
            const char *H;              // column 64 a of H
            bool bf16;
        };
        auto cursor_load = [&](Cursor &u) {
            if (u.j < n_list) {
                const int2 job = list[u.j];
                const DevInst &in = insts[job.x];
                u.M = in.M;
                u.K = in.K - 64 * job.y;
                u.ldh = in.ldh;
                u.bf16 = in.h_bf16 != 0;
                u.H = reinterpret_cast<const char *>(in.H) + (size_t)64 * job.y * in.ldh * (u.bf16 ? 4 : 8);
                u.nch = (u.M + MCH - 1) / MCH;
            }
        };
        auto cursor_next = [&](Cursor &u) {
            if (++u.c >= u.nch) {
                u.c = 0;
                u.j += gridDim.x;
                cursor_load(u);
            }
        };
        // warp w's chunks of stage u into raw stage rs.  complex64: column slot i
        // holds 32 entries = 16 chunks pc of 2 entries at 16-byte slot pc ^ i;
        // bfloat16: 8 chunks of 4 entries at slot pc ^ i.
        auto issue = [&](const Cursor &u, int rs) {
            if (u.j < n_list) {
                const uint32_t wbase = raw0 + rs * RAWB + warp * 8 * 256;   // 8 column slots of 256 B
                if (u.bf16) {
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
                        const int i = 4 * q + (lane >> 3), pc = lane & 7;
                        const int k = 8 * i + ((warp + i) & 7);
                        const int m = u.c * MCH + 4 * pc;
                        const int left = k < u.K ? min(max(u.M - m, 0), 4) : 0;
                        const char *src = u.H + ((size_t)k * u.ldh + m) * 4;
                        tc::cp_async16(wbase + i * 128 + ((pc ^ i) & 7) * 16, left ? src : u.H, left * 4);
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int i = 2 * q + (lane >> 4), pc = lane & 15;
                        const int k = 8 * i + ((warp + i) & 7);
                        const int m = u.c * MCH + 2 * pc;
                        const int left = k < u.K ? min(max(u.M - m, 0), 2) : 0;
                        const char *src = u.H + ((size_t)k * u.ldh + m) * 8;
                        tc::cp_async16(wbase + i * 256 + (pc ^ i) * 16, left ? src : u.H, left * 8);
                    }
                }
            }
            tc::cp_async_commit();   // one group per stage, empty past the end
        };
        Cursor iu{(int)blockIdx.x, 0, 0, 0, 0, 0, nullptr, false};
        cursor_load(iu);
#pragma unroll 1
        for (int p = 0; p < RAW - 1; ++p) {
            issue(iu, p);
            cursor_next(iu);
        }
        uint32_t chunk = 0, sc = 0;
        for (int j = blockIdx.x; j < n_list && !S.err; j += gridDim.x) {
            const DevInst &in = insts[list[j].x];
            const int M = in.M;
            const bool bf16 = in.h_bf16 != 0;
            const int nch = (M + MCH - 1) / MCH;
            auto put = [&](const float4 (&buf)[2][2]) -> bool {
                const int s = chunk % STAGES;
                if (chunk >= STAGES &&
                    !tc::mbar_wait(&S.empty[s], ((chunk / STAGES) - 1) & 1, WAIT_LIMIT)) {
                    S.err = 1;
                    return false;
                }
                const uint32_t base = tc::smem_u32(S.stage[s]);
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const int i = lane & 7, mq = (lane >> 3) + 4 * q;
                    const int k = 8 * i + ((warp + i) & 7);
                    const float re[4] = {buf[q][0].x, buf[q][0].z, buf[q][1].x, buf[q][1].z};
                    const float im[4] = {buf[q][0].y, buf[q][0].w, buf[q][1].y, buf[q][1].w};
                    float rh[4], rl[4], ih[4], il[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        tc::split_tf32(re[i], rh[i], rl[i]);
                        tc::split_tf32(im[i], ih[i], il[i]);
                    }
                    const uint32_t o_re = (uint32_t)(k >> 3) * SBO + mq * LBO + (k & 7) * 16;
                    const uint32_t o_im = (uint32_t)((64 + k) >> 3) * SBO + mq * LBO + (k & 7) * 16;
                    st_shared_v4(base + o_re, rh[0], rh[1], rh[2], rh[3]);
                    st_shared_v4(base + o_im, ih[0], ih[1], ih[2], ih[3]);
                    st_shared_v4(base + PART + o_re, rl[0], rl[1], rl[2], rl[3]);
                    st_shared_v4(base + PART + o_im, il[0], il[1], il[2], il[3]);
                }
                tc::fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&S.full[s]);
                ++chunk;
                return true;
            };
            bool ok = true;
            for (int c = 0; c < nch && ok; ++c, ++sc) {
                tc::cp_async_wait<RAW - 2>();   // this thread's chunks of stage sc have landed
                __syncwarp();                   // ... and those of the rest of its warp
                const int rs = sc % RAW;
                float4 buf[2][2];
#pragma unroll
                for (int q = 0; q < 2; ++q) {   // entries 4 mq .. 4 mq + 3 of column slot i
                    const int i = lane & 7, mq = (lane >> 3) + 4 * q;
                    const unsigned char *wr = S.raw[rs] + warp * 8 * 256;
                    if (bf16) {
                        const uint4 u = *reinterpret_cast<const uint4 *>(wr + i * 128 + ((mq ^ i) & 7) * 16);
                        const float2 a = bf16x2_to_float2(u.x), b = bf16x2_to_float2(u.y);
                        const float2 c2 = bf16x2_to_float2(u.z), d = bf16x2_to_float2(u.w);
                        buf[q][0] = make_float4(a.x, a.y, b.x, b.y);
                        buf[q][1] = make_float4(c2.x, c2.y, d.x, d.y);
                    } else {
                        buf[q][0] = *reinterpret_cast<const float4 *>(wr + i * 256 + ((2 * mq) ^ i) * 16);
                        buf[q][1] = *reinterpret_cast<const float4 *>(wr + i * 256 + ((2 * mq + 1) ^ i) * 16);
                    }
                }
                issue(iu, (sc + RAW - 1) % RAW);   // refills the stage read one step ago
                cursor_next(iu);
                ok = put(buf);
            }
        }
        tc::cp_async_wait_all();   // no copy may still be landing when the CTA exits
    } else if (warp < MMA_WARP) {
        // ---------------- drain / epilogue ----------------
        const int dw = warp - NPW;                 // 0 .. 7
        const int quad = warp & 3;                 // TMEM lane quadrant of this warp
        const int half = dw >> 2;                  // columns [64 half, 64 half + 64)
        const int row = 32 * quad + lane;          // row of D owned by this thread
        const int dtid = threadIdx.x - NPW * 32;   // 0 .. 255
        uint32_t grp = 0, ninst = 0;
        for (int j = blockIdx.x; j < n_list; j += gridDim.x, ++ninst) {
            const int id = list[j].x;
            const int c0 = 64 * list[j].y;             // the job's users: c0 .. c0 + 63
            const DevInst &in = insts[id];
            const int nch = (in.M + MCH - 1) / MCH;
            const int ngrp = (nch + G - 1) / G;
            float sum[64];
#pragma unroll
            for (int i = 0; i < 64; ++i) sum[i] = 0.f;
            for (int g = 0; g < ngrp && !S.err; ++g, ++grp) {
                const int b = grp & 1;
                if (!tc::mbar_wait(&S.accf[b], (grp >> 1) & 1, WAIT_LIMIT)) {
                    S.err = 1;
                    break;
                }
                tc::tc_fence_after();
                const uint32_t ta = tmem + ((uint32_t)(32 * quad) << 16) + b * ROWS + half * 64;
#pragma unroll
                for (int c0 = 0; c0 < 64; c0 += 16) {
                    float v[16];
                    tc::tmem_ld16(ta + c0, v);
                    tc::tmem_ld_wait();
#pragma unroll
                    for (int i = 0; i < 16; ++i) sum[c0 + i] += v[i];
                }
                tc::tc_fence_before();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&S.acce[b]);
            }
            // D = head sums + E + E^T (the last group's commit covers every
            // correction MMA of the instance)
            const uint32_t te = tmem + ((uint32_t)(32 * quad) << 16) + (2 + (ninst & 1)) * ROWS + half * 64;
#pragma unroll
            for (int c0 = 0; c0 < 64; c0 += 16) {
                float v[16];
                tc::tmem_ld16(te + c0, v);
                tc::tmem_ld_wait();
#pragma unroll
                for (int i = 0; i < 16; ++i) S.D[row * DPITCH + half * 64 + c0 + i] = sum[c0 + i] + v[i];
            }
            asm volatile("bar.sync 1, 256;\n" ::: "memory");
#pragma unroll
            for (int c0 = 0; c0 < 64; c0 += 16) {   // element (c, row) takes E[row][c]: one writer each
                float v[16];
                tc::tmem_ld16(te + c0, v);
                tc::tmem_ld_wait();
#pragma unroll
                for (int i = 0; i < 16; ++i) S.D[(half * 64 + c0 + i) * DPITCH + row] += v[i];
            }
            tc::tc_fence_before();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&S.core[ninst & 1]);
            asm volatile("bar.sync 1, 256;\n" ::: "memory");
            const bool bad = S.err != 0;
            const int K = in.K, KC = in.KC;
            const float xi = in.xi;
            float2 *__restrict__ A = in.A;
            float2 *__restrict__ Aout = in.Aout;
            for (int e = dtid; e < 64 * 64; e += 256) {
                const int r = e & 63, c = e >> 6;
                const int k = max(r, c), jj = min(r, c);
                float re = S.D[k * DPITCH + jj] + S.D[(64 + k) * DPITCH + 64 + jj];
                float im = S.D[k * DPITCH + 64 + jj] - S.D[(64 + k) * DPITCH + jj];
                if (r < c) im = -im;
                const int gr = c0 + r, gc = c0 + c;        // position in A
                if (r == c) {
                    im = 0.f;
                    if (gr < K) {
                        re += xi;
                        in.dinv[gr] = 1.0f / re;
                    } else {
                        in.dinv[gr] = 0.f;
                    }
                }
                A[gr + (size_t)gc * KC] = make_float2(re, im);
                if (Aout && gr < K && gc < K) Aout[gr + (size_t)gc * K] = make_float2(re, im);
            }
            if (dtid == 0) {
                if (KC == 64) {   // the instance's only job resets its accumulators
                    acc_out.flags[id] = bad ? FLAG_TIMEOUT : 0;
                    acc_out.iters[id] = 0;
                    acc_out.resid_bits[id] = 0u;
                } else if (bad) {   // several jobs: reset before the launch, report only
                    atomicOr(acc_out.flags + id, FLAG_TIMEOUT);
                }
            }
            asm volatile("bar.sync 1, 256;\n" ::: "memory");   // D is rewritten by the next instance
        }
    } else if (lane == 0) {
        // ---------------- MMA issuer ----------------
        constexpr uint32_t idesc = tc::idesc_tf32(ROWS, ROWS);
        uint32_t chunk = 0, grp = 0, ninst = 0;
        for (int j = blockIdx.x; j < n_list && !S.err; j += gridDim.x, ++ninst) {
            const DevInst &in = insts[list[j].x];
            const int nch = (in.M + MCH - 1) / MCH;
            const uint32_t e = tmem + (2 + (ninst & 1)) * ROWS;
            if (ninst >= 2) {   // the correction buffer of two instances ago has been read
                if (!tc::mbar_wait(&S.core[ninst & 1], ((ninst >> 1) - 1) & 1, WAIT_LIMIT)) {
                    S.err = 1;
                    break;
                }
                tc::tc_fence_after();
            }
            for (int c = 0; c < nch; ++c, ++chunk) {
                const int b = grp & 1;
                if (c % G == 0 && grp >= 2) {
                    if (!tc::mbar_wait(&S.acce[b], ((grp >> 1) - 1) & 1, WAIT_LIMIT)) {
                        S.err = 1;
                        break;
                    }
                    tc::tc_fence_after();
                }
                const int s = chunk % STAGES;
                if (!tc::mbar_wait(&S.full[s], (chunk / STAGES) & 1, WAIT_LIMIT)) {
                    S.err = 1;
                    break;
                }
                tc::tc_fence_after();
                const uint32_t hi = tc::smem_u32(S.stage[s]), lo = hi + PART;
                const uint32_t d = tmem + b * ROWS;
#pragma unroll
                for (int kk = 0; kk < MCH / 8; ++kk) {
                    const uint32_t off = kk * 2 * LBO;   // 8 TF32 values = 2 core matrices along K
                    const uint64_t dh = tc::smem_desc(hi + off, LBO, SBO);
                    const uint64_t dl = tc::smem_desc(lo + off, LBO, SBO);
                    tc::mma_tf32(d, dh, dh, idesc, (c % G == 0 && kk == 0) ? 0u : 1u);
                    tc::mma_tf32(e, dh, dl, idesc, (c == 0 && kk == 0) ? 0u : 1u);
                }
                tc::mma_commit(&S.empty[s]);
                if (c % G == G - 1 || c == nch - 1) {
                    tc::mma_commit(&S.accf[b]);
                    ++grp;
                }
            }
        }
        tc::mma_commit(&S.fin);
        tc::mbar_wait(&S.fin, 0, WAIT_LIMIT);   // no MMA in flight past this point
    }

    tc::tc_fence_before();
    __syncthreads();
    if (S.err && threadIdx.x == 0) {
        for (int j = blockIdx.x; j < n_list; j += gridDim.x) atomicOr(acc_out.flags + list[j].x, FLAG_TIMEOUT);
    }
    if (warp == MMA_WARP) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, TMEM_COLS);
    }
}

}  // namespace

cudaError_t launch_gram_tc64(const DevInst *insts, const int2 *list, int n, DevAccum acc,
                             cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const size_t smem = sizeof(GramSmem);
    cudaError_t e = cudaFuncSetAttribute(gram_tc64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const int grid = n < sms ? n : sms;
    gram_tc64_kernel<<<grid, NTHREADS, smem, s>>>(insts, list, n, acc);
    return cudaGetLastError();
}

}  // namespace jacpcg
