// gram_tc_cross.cu -- the off-diagonal 64 x 64 blocks of A = H^H H + xi I
// on the tcgen05 tensor cores for the K = 128 and 256 classes (Sec. II,
// definition of P_i after Eq. 7).  A job is (instance, user groups a < b):
// block (a, b) = H_a^H H_b of the users 64 a .. 64 a + 63 and 64 b .. 64 b + 63,
// written with its conjugate transpose into block (b, a), so A stays exactly
// Hermitian; gram_tc.cu computes the diagonal blocks and 1/diag.
//
// As one real GEMM: with Y_a = [Re H_a | Im H_a] and Y_b likewise (M x 128
// each), D = Y_a^T Y_b (128 x 128) gives Re A_ab = D11 + D22 and
// Im A_ab = D12 - D21.  3xTF32 (Ootomo and Yokota, IJHPCA 2022): every staged
// value is split y = hi + lo, D = Yh_a^T Yh_b + Yh_a^T Yl_b + Yl_a^T Yh_b; D is
// not symmetric here, so both correction products are issued, accumulated
// over the whole instance in one TMEM buffer (their drift is 2^-11 of D's);
// the head product is drained from two alternating TMEM buffers every G
// stages (128 rows) into FP32 registers, as in gram_tc.cu.
//
// Persistent, warp-specialised, one CTA per SM walking its jobs:
//   warps 0-7   producers: a stage is 16 antennas x 128 users (both groups).
//               Per-thread asynchronous copies (cp.async, 16 bytes, zero-filled
//               past M and K) run RAW - 1 stages ahead into a ring of raw
//               stages; warp w copies 16 users (warps 0-3 group a, 4-7 group
//               b), whole 128-byte column pieces per copy instruction, chunks
//               XOR-swizzled so copies, raw reads and split stores are free of
//               bank conflicts, and converts exactly what it copied (a
//               __syncwarp after its own cp.async wait) into the TF32 head and
//               tail of its operand in the canonical no-swizzle K-major layout;
//   warps 8-15  drain/epilogue: head sums per group; at the end of a job the
//               sums plus corrections go through shared memory into A;
//   warp 16     TMEM allocation; lane 0 issues the MMAs and commits.
// Every wait is bounded; a timeout stops the CTA's pipeline, flags its
// instances with FLAG_TIMEOUT, and the CTA still drains and frees its TMEM.
#include "common.cuh"
#include "kernels.h"
#include "tc.cuh"

namespace jacpcg {

namespace {

constexpr int ROWS = 128;                     // real rows of one operand: 64 users x (Re, Im)
constexpr int MCH = 16;                       // H rows (reduction values) per stage
constexpr int STAGES = 2;                     // split stages shared with the MMA warp
constexpr int RAW = 6;                        // raw stages in flight per producer thread
constexpr int RAWB = MCH * 128 * 8;           // bytes of one raw stage (16 KB complex64)
constexpr int G = 8;                          // stages per head accumulation group (128 rows)
constexpr int PART = ROWS * MCH * 4;          // one operand part (hi or lo): 8 KB
constexpr uint32_t LBO = 128;                 // K-adjacent core matrices
constexpr uint32_t SBO = (MCH / 4) * 128;     // 8-row groups
constexpr uint32_t WAIT_LIMIT = 1u << 21;
constexpr int DPITCH = ROWS + 1;              // floats per staged D row
constexpr int NPW = 8, NDW = 8;               // producer and drain warps
constexpr int MMA_WARP = NPW + NDW;
constexpr int NTHREADS = (NPW + NDW + 1) * 32;
constexpr int TMEM_COLS = 4 * ROWS;           // two head-group buffers, two correction buffers

struct __align__(128) GramXSmem {
    unsigned char stage[STAGES][4 * PART];      // [A hi | A lo | B hi | B lo]
    unsigned char raw[RAW][RAWB];               // warp w: 2 KB, 16 column pieces
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
static_assert(sizeof(GramXSmem) <= 227 * 1024, "shared memory");

__device__ __forceinline__ void st_shared_v4(uint32_t addr, float a, float b, float c, float d) {
    asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};\n" ::"r"(addr), "f"(a), "f"(b), "f"(c),
                 "f"(d)
                 : "memory");
}

__global__ void __launch_bounds__(NTHREADS, 1) gram_tc_cross_kernel(const DevInst *__restrict__ insts,
                                                                    const int4 *__restrict__ list,
                                                                    int n_list, DevAccum acc_out) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    GramXSmem &S = *reinterpret_cast<GramXSmem *>(smem_raw);
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
        const int grp_b = warp >> 2;                 // 0: group a (A operand), 1: group b (B operand)
        // stream cursor: (job ordinal, stage) in this CTA's walk; this warp's group only
        struct Cursor {
            int j, c, nch, M, Kg, ldh;               // Kg: users of this warp's group that exist
            const char *H;                           // first column of this warp's group
            bool bf16;
        };
        auto cursor_load = [&](Cursor &u) {
            if (u.j < n_list) {
                const int4 job = list[u.j];
                const DevInst &in = insts[job.x];
                const int g = grp_b ? job.z : job.y;
                u.M = in.M;
                u.Kg = in.K - 64 * g;
                u.ldh = in.ldh;
                u.bf16 = in.h_bf16 != 0;
                u.H = reinterpret_cast<const char *>(in.H) + (size_t)64 * g * in.ldh * (u.bf16 ? 4 : 8);
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
        // warp w copies users 16 (w mod 4) + sl, sl = 0..15, of its group.  complex64:
        // column slot sl holds 16 entries = 8 chunks pc of 2 entries at 16-byte slot
        // pc ^ (sl mod 8); bfloat16: 4 chunks of 4 entries at slot pc ^ (sl mod 4).
        auto issue = [&](const Cursor &u, int rs) {
            if (u.j < n_list) {
                const uint32_t wbase = raw0 + rs * RAWB + warp * 2048;
                if (u.bf16) {
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
                        const int sl = 8 * q + (lane >> 2), pc = lane & 3;
                        const int k = 16 * (warp & 3) + sl;
                        const int m = u.c * MCH + 4 * pc;
                        const int left = k < u.Kg ? min(max(u.M - m, 0), 4) : 0;
                        const char *src = u.H + ((size_t)k * u.ldh + m) * 4;
                        tc::cp_async16(wbase + sl * 64 + ((pc ^ sl) & 3) * 16, left ? src : u.H, left * 4);
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int sl = 4 * q + (lane >> 3), pc = lane & 7;
                        const int k = 16 * (warp & 3) + sl;
                        const int m = u.c * MCH + 2 * pc;
                        const int left = k < u.Kg ? min(max(u.M - m, 0), 2) : 0;
                        const char *src = u.H + ((size_t)k * u.ldh + m) * 8;
                        tc::cp_async16(wbase + sl * 128 + ((pc ^ sl) & 7) * 16, left ? src : u.H, left * 8);
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
        const uint32_t opoff = grp_b ? 2 * PART : 0;   // this warp's operand in a stage
        for (int j = blockIdx.x; j < n_list && !S.err; j += gridDim.x) {
            const DevInst &in = insts[list[j].x];
            const bool bf16 = in.h_bf16 != 0;
            const int nch = (in.M + MCH - 1) / MCH;
            bool ok = true;
            for (int c = 0; c < nch && ok; ++c, ++sc) {
                tc::cp_async_wait<RAW - 2>();   // this thread's chunks of stage sc have landed
                __syncwarp();                   // ... and those of the rest of its warp
                const unsigned char *wr = S.raw[sc % RAW] + warp * 2048;
                float4 buf[2][2];
#pragma unroll
                for (int q = 0; q < 2; ++q) {   // entries 4 mq .. 4 mq + 3 of column slot sl
                    const int sl = lane & 15, mq = (lane >> 4) + 2 * q;
                    if (bf16) {
                        const uint4 u = *reinterpret_cast<const uint4 *>(wr + sl * 64 + ((mq ^ sl) & 3) * 16);
                        const float2 a = bf16x2_to_float2(u.x), b = bf16x2_to_float2(u.y);
                        const float2 c2 = bf16x2_to_float2(u.z), d = bf16x2_to_float2(u.w);
                        buf[q][0] = make_float4(a.x, a.y, b.x, b.y);
                        buf[q][1] = make_float4(c2.x, c2.y, d.x, d.y);
                    } else {
                        buf[q][0] = *reinterpret_cast<const float4 *>(wr + sl * 128 + (((2 * mq) ^ sl) & 7) * 16);
                        buf[q][1] = *reinterpret_cast<const float4 *>(wr + sl * 128 + (((2 * mq + 1) ^ sl) & 7) * 16);
                    }
                }
                issue(iu, (sc + RAW - 1) % RAW);   // refills the stage read one step ago
                cursor_next(iu);
                // put: the TF32 head and tail of this warp's operand rows into the split stage
                const int s = chunk % STAGES;
                if (chunk >= STAGES &&
                    !tc::mbar_wait(&S.empty[s], ((chunk / STAGES) - 1) & 1, WAIT_LIMIT)) {
                    S.err = 1;
                    ok = false;
                    break;
                }
                const uint32_t base = tc::smem_u32(S.stage[s]) + opoff;
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const int sl = lane & 15, mq = (lane >> 4) + 2 * q;
                    const int k = 16 * (warp & 3) + sl;   // user within the group
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
            }
            if (!ok) break;
        }
        tc::cp_async_wait_all();   // no copy may still be landing when the CTA exits
    } else if (warp < MMA_WARP) {
        // ---------------- drain / epilogue ----------------
        const int dw = warp - NPW;                 // 0 .. 7
        const int quad = warp & 3;                 // TMEM lane quadrant of this warp
        const int half = dw >> 2;                  // columns [64 half, 64 half + 64)
        const int row = 32 * quad + lane;          // row of D owned by this thread
        const int dtid = threadIdx.x - NPW * 32;   // 0 .. 255
        uint32_t grp = 0, njob = 0;
        for (int j = blockIdx.x; j < n_list; j += gridDim.x, ++njob) {
            const int4 job = list[j];
            const DevInst &in = insts[job.x];
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
            // D = head sums + corrections (the last group's commit covers every
            // correction MMA of the job)
            const uint32_t te = tmem + ((uint32_t)(32 * quad) << 16) + (2 + (njob & 1)) * ROWS + half * 64;
#pragma unroll
            for (int c0 = 0; c0 < 64; c0 += 16) {
                float v[16];
                tc::tmem_ld16(te + c0, v);
                tc::tmem_ld_wait();
#pragma unroll
                for (int i = 0; i < 16; ++i) S.D[row * DPITCH + half * 64 + c0 + i] = sum[c0 + i] + v[i];
            }
            tc::tc_fence_before();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&S.core[njob & 1]);
            asm volatile("bar.sync 1, 256;\n" ::: "memory");
            const bool bad = S.err != 0;
            const int K = in.K, KC = in.KC;
            const int a0 = 64 * job.y, b0 = 64 * job.z;
            float2 *__restrict__ A = in.A;
            float2 *__restrict__ Aout = in.Aout;
            // block (a, b): rows a0 + r, columns b0 + c (coalesced along r)
            for (int e = dtid; e < 64 * 64; e += 256) {
                const int r = e & 63, c = e >> 6;
                const float re = S.D[r * DPITCH + c] + S.D[(64 + r) * DPITCH + 64 + c];
                const float im = S.D[r * DPITCH + 64 + c] - S.D[(64 + r) * DPITCH + c];
                A[(a0 + r) + (size_t)(b0 + c) * KC] = make_float2(re, im);
                if (Aout && a0 + r < K && b0 + c < K) Aout[(a0 + r) + (size_t)(b0 + c) * K] = make_float2(re, im);
            }
            // block (b, a) = its conjugate transpose: rows b0 + c, columns a0 + r (coalesced along c)
            for (int e = dtid; e < 64 * 64; e += 256) {
                const int c = e & 63, r = e >> 6;
                const float re = S.D[r * DPITCH + c] + S.D[(64 + r) * DPITCH + 64 + c];
                const float im = S.D[r * DPITCH + 64 + c] - S.D[(64 + r) * DPITCH + c];
                A[(b0 + c) + (size_t)(a0 + r) * KC] = make_float2(re, -im);
                if (Aout && a0 + r < K && b0 + c < K) Aout[(b0 + c) + (size_t)(a0 + r) * K] = make_float2(re, -im);
            }
            if (dtid == 0 && bad) atomicOr(acc_out.flags + job.x, FLAG_TIMEOUT);
            asm volatile("bar.sync 1, 256;\n" ::: "memory");   // D is rewritten by the next job
        }
    } else if (lane == 0) {
        // ---------------- MMA issuer ----------------
        constexpr uint32_t idesc = tc::idesc_tf32(ROWS, ROWS);
        uint32_t chunk = 0, grp = 0, njob = 0;
        for (int j = blockIdx.x; j < n_list && !S.err; j += gridDim.x, ++njob) {
            const DevInst &in = insts[list[j].x];
            const int nch = (in.M + MCH - 1) / MCH;
            const uint32_t e = tmem + (2 + (njob & 1)) * ROWS;
            if (njob >= 2) {   // the correction buffer of two jobs ago has been read
                if (!tc::mbar_wait(&S.core[njob & 1], ((njob >> 1) - 1) & 1, WAIT_LIMIT)) {
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
                const uint32_t ah = tc::smem_u32(S.stage[s]), al = ah + PART;
                const uint32_t bh = ah + 2 * PART, bl = ah + 3 * PART;
                const uint32_t d = tmem + b * ROWS;
#pragma unroll
                for (int kk = 0; kk < MCH / 8; ++kk) {
                    const uint32_t off = kk * 2 * LBO;   // 8 TF32 values = 2 core matrices along K
                    const uint64_t dah = tc::smem_desc(ah + off, LBO, SBO);
                    const uint64_t dal = tc::smem_desc(al + off, LBO, SBO);
                    const uint64_t dbh = tc::smem_desc(bh + off, LBO, SBO);
                    const uint64_t dbl = tc::smem_desc(bl + off, LBO, SBO);
                    tc::mma_tf32(d, dah, dbh, idesc, (c % G == 0 && kk == 0) ? 0u : 1u);
                    tc::mma_tf32(e, dah, dbl, idesc, (c == 0 && kk == 0) ? 0u : 1u);
                    tc::mma_tf32(e, dal, dbh, idesc, 1u);
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

cudaError_t launch_gram_tc_cross(const DevInst *insts, const int4 *list, int n, DevAccum acc,
                                 cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const size_t smem = sizeof(GramXSmem);
    cudaError_t e = cudaFuncSetAttribute(gram_tc_cross_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const int grid = n < sms ? n : sms;
    gram_tc_cross_kernel<<<grid, NTHREADS, smem, s>>>(insts, list, n, acc);
    return cudaGetLastError();
}

}  // namespace jacpcg
