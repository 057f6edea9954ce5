// hx_tc_wide.cu -- the precoder W = H X on the tcgen05 tensor cores for the
// K = 128 and 256 classes (Eq. 7 without the power factor; Eq. 15 per
// symbol), 3xTF32.  A job is (instance, output group b): the 64 columns
// 64 b .. 64 b + 63 of W, all row tiles.  X is KC x KC, too large to stay
// resident in shared memory as in hx_tc.cu, so every stage brings the 16
// users' slice of X's group-b columns along with the 128 x 16 tile of H.
//
// Complex product as real MMAs over one 128-row tile of W, as in hx_tc.cu:
//   [Wr | Wi] = Hr [Xr | Xi] + Hi [-Xi | Xr],
// per stage with B = [-Xi^T ; Xr^T ; Xi^T] of the stage's 16 users (192 rows,
// K-major) in shared memory -- rows 64 .. 191 are [Xr^T ; Xi^T], rows 0 .. 127
// [-Xi^T ; Xr^T] -- and the H stage (Hr, Hi, TF32 head and tail) in tensor
// memory as the MMAs' A operand: two N = 128 MMAs per k-step and split
// product (hi*hi + hi*lo + lo*hi; Ootomo and Yokota, IJHPCA 2022), each
// reading only its B slice from shared memory (2.67 vs 3.16 ms for the
// 256-channel M = 4096, K = 256 batch with the H tile split into shared
// memory).  The tensor core's FP32 accumulation truncates, and a tile
// reduces over up to 32 stages, so the chain is cut as in gram_tc.cu: every G
// stages the MMAs switch between two TMEM buffers and the drain warps add
// the finished group into FP32 registers (no chain longer than the K = 64
// kernel's).
//
// Persistent, warp-specialised, one CTA per SM walking its jobs:
//   warps 0-7   producers: raw stages fetched RAW - 1 ahead with per-thread
//               asynchronous copies (cp.async, 16 bytes, zero-filled past M,
//               K and the instance's columns); warp w copies antennas
//               32 (w mod 4) .. + 31 (its TMEM lanes) of the stage's users
//               8 (w / 4) .. + 7 (whole 256-byte column pieces) and columns
//               8 w .. 8 w + 7 of the X slice (whole 128-byte column pieces,
//               chunks XOR-swizzled), converts exactly what it copied (a
//               __syncwarp after its own cp.async wait): H into its TMEM
//               lanes (tcgen05.st), X into B;
//   warps 8-15  drain: TMEM (two alternating 128-column accumulators, one
//               per group) -> FP32 registers summed over the tile's groups ->
//               W (complex64, column-major, coalesced) and the tile's
//               ||W||_F^2 partial in slot b * (row tiles) + tile;
//   warp 16     TMEM allocation; lane 0 issues MMAs and commits.
// Every wait is bounded; a timeout flags the CTA's instances with FLAG_TIMEOUT.
#include "common.cuh"
#include "kernels.h"
#include "tc.cuh"

namespace jacpcg {

namespace {

constexpr int TMR = 128;                      // W rows per tile
constexpr int KCH = 16;                       // users (reduction values) per stage
constexpr int STAGES = 2;                     // stages shared with the MMA warp
constexpr int RAW = 7;                        // raw stages in flight per producer thread
constexpr int RAWH = 16 * 1024;               // H part of a raw stage (warp w: 2 KB)
constexpr int RAWB = RAWH + 8 * 1024;         // + X slice (warp w: 1 KB)
constexpr int XPART = 192 * KCH * 4;          // one of B_hi, B_lo: rows -Xi^T, Xr^T, Xi^T, 12 KB
constexpr int SPLIT = 2 * XPART;              // one B stage: 24 KB
constexpr uint32_t LBO = 128;
constexpr uint32_t SBO = (KCH / 4) * 128;     // 512
constexpr uint32_t TS0 = 256;                 // H stages in TMEM: columns TS0 + 64 s + 16 part + user
constexpr uint32_t WAIT_LIMIT = 1u << 21;
constexpr int NPW = 8, NDW = 8;
constexpr int MMA_WARP = NPW + NDW;
constexpr int NTHREADS = (NPW + NDW + 1) * 32;
constexpr int TMEM_COLS = 512;                // two accumulators, two H stages
constexpr int G = 4;                          // stages per accumulation group

struct __align__(128) HxwSmem {
    unsigned char stage[STAGES][SPLIT];
    unsigned char raw[RAW][RAWB];
    float wsum[2][NDW];
    uint64_t full[STAGES];
    uint64_t empty[STAGES];
    uint64_t accf[2];
    uint64_t acce[2];
    uint64_t fin;
    uint32_t tmem;
    volatile int err;
};
static_assert(sizeof(HxwSmem) <= 227 * 1024, "shared memory");

// one warp stores 8 consecutive 32-bit columns of its 32 lanes
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const float (&v)[8]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};\n" ::"r"(taddr),
        "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
        "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
        "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7]))
        : "memory");
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, float a, float b, float c, float d) {
    asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};\n" ::"r"(addr), "f"(a), "f"(b), "f"(c),
                 "f"(d)
                 : "memory");
}

__global__ void __launch_bounds__(NTHREADS, 1) hx_tc_wide_kernel(const DevInst *__restrict__ insts,
                                                                 const int2 *__restrict__ list, int n_list,
                                                                 DevAccum acc_out) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    HxwSmem &S = *reinterpret_cast<HxwSmem *>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            tc::mbar_init(&S.full[s], NPW);
            tc::mbar_init(&S.empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            tc::mbar_init(&S.accf[b], 1);
            tc::mbar_init(&S.acce[b], NDW);
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
        // stream cursor: (job ordinal, stage t = tile t / nks, users 16 (t % nks) ..)
        struct Cursor {
            int j, t, nst, nks, M, K, ldh, ncols, KC, col0;
            const char *H;
            const char *X;
            bool bf16;
        };
        auto cursor_load = [&](Cursor &u) {
            if (u.j < n_list) {
                const int2 job = list[u.j];
                const DevInst &in = insts[job.x];
                u.M = in.M;
                u.K = in.K;
                u.ldh = in.ldh;
                u.ncols = in.ncols;
                u.KC = in.KC;
                u.col0 = 64 * job.y;
                u.H = reinterpret_cast<const char *>(in.H);
                u.X = reinterpret_cast<const char *>(in.X);
                u.bf16 = in.h_bf16 != 0;
                u.nks = (u.K + KCH - 1) / KCH;
                u.nst = ((u.M + TMR - 1) / TMR) * u.nks;
            }
        };
        auto cursor_next = [&](Cursor &u) {
            if (++u.t >= u.nst) {
                u.t = 0;
                u.j += gridDim.x;
                cursor_load(u);
            }
        };
        auto issue = [&](const Cursor &u, int rs) {
            if (u.j < n_list) {
                const uint32_t rb = raw0 + rs * RAWB;
                const int mt = u.t / u.nks, ks = u.t % u.nks;
                // warp w: antennas 32 (w mod 4) .. + 31 (its TMEM lanes) of the stage's
                // users 8 (w / 4) .. + 7, whole 256-byte (128-byte bfloat16) column pieces
                const uint32_t wb = rb + warp * 2048;
                const int m0 = mt * TMR + 32 * (warp & 3), k0 = ks * KCH + 8 * (warp >> 2);
                if (u.bf16) {
#pragma unroll
                    for (int c = 0; c < 2; ++c) {   // 8 columns x 8 chunks of 4 antennas
                        const int e = lane + 32 * c, uu = e >> 3, pc = e & 7;
                        const int k = k0 + uu, m = m0 + 4 * pc;
                        const int left = k < u.K ? min(max(u.M - m, 0), 4) : 0;
                        const char *src = u.H + ((size_t)k * u.ldh + m) * 4;
                        tc::cp_async16(wb + uu * 128 + pc * 16, left ? src : u.H, left * 4);
                    }
                } else {
#pragma unroll
                    for (int c = 0; c < 4; ++c) {   // 8 columns x 16 chunks of 2 antennas
                        const int e = lane + 32 * c, uu = e >> 4, pc = e & 15;
                        const int k = k0 + uu, m = m0 + 2 * pc;
                        const int left = k < u.K ? min(max(u.M - m, 0), 2) : 0;
                        const char *src = u.H + ((size_t)k * u.ldh + m) * 8;
                        tc::cp_async16(wb + uu * 256 + pc * 16, left ? src : u.H, left * 8);
                    }
                }
                // X slice: users ks*16 .. +15 of columns col0 + 8 w + cj, 8 chunks of 2 users
                const uint32_t xb = rb + RAWH + warp * 1024;
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const int cj = 4 * q + (lane >> 3), pc = lane & 7;
                    const int col = u.col0 + 8 * warp + cj, r = ks * KCH + 2 * pc;
                    const int left = col < u.ncols ? min(max(u.K - r, 0), 2) : 0;
                    const char *src = u.X + ((size_t)col * u.KC + r) * 8;
                    tc::cp_async16(xb + cj * 128 + ((pc ^ cj) & 7) * 16, left ? src : u.X, left * 8);
                }
            }
            tc::cp_async_commit();   // one group per stage, empty past the end
        };
        Cursor iu{(int)blockIdx.x, 0, 0, 0, 0, 0, 0, 0, 0, 0, nullptr, nullptr, false};
        cursor_load(iu);
#pragma unroll 1
        for (int p = 0; p < RAW - 1; ++p) {
            issue(iu, p);
            cursor_next(iu);
        }
        uint32_t chunk = 0, sc = 0;
        for (int j = blockIdx.x; j < n_list && !S.err; j += gridDim.x) {
            const DevInst &in = insts[list[j].x];
            const bool bf16 = in.h_bf16 != 0;
            const int T = ((in.M + TMR - 1) / TMR) * ((in.K + KCH - 1) / KCH);
            bool ok = true;
            for (int t = 0; t < T && ok; ++t, ++sc) {
                tc::cp_async_wait<RAW - 2>();   // this thread's chunks of the stage have landed
                __syncwarp();                   // ... and those of the rest of its warp
                const unsigned char *wr = S.raw[sc % RAW] + warp * 2048;
                const unsigned char *xr = S.raw[sc % RAW] + RAWH + warp * 1024;
                float2 h[8];   // antenna 32 (w mod 4) + lane of users 8 (w / 4) + uu
#pragma unroll
                for (int uu = 0; uu < 8; ++uu)
                    h[uu] = bf16 ? bf16x2_to_float2(*reinterpret_cast<const uint32_t *>(wr + uu * 128 + lane * 4))
                                 : *reinterpret_cast<const float2 *>(wr + uu * 256 + lane * 8);
                float4 xv[2];   // column 8 w + cj, users 4 kq .. 4 kq + 3
                {
                    const int cj = lane & 7, kq = lane >> 3;
                    xv[0] = *reinterpret_cast<const float4 *>(xr + cj * 128 + (((2 * kq) ^ cj) & 7) * 16);
                    xv[1] = *reinterpret_cast<const float4 *>(xr + cj * 128 + (((2 * kq + 1) ^ cj) & 7) * 16);
                }
                issue(iu, (sc + RAW - 1) % RAW);   // refills the stage read one step ago
                cursor_next(iu);
                // put: H (head and tail) into this warp's TMEM lanes, B into the shared stage
                const int s = chunk % STAGES;
                if (chunk >= STAGES &&
                    !tc::mbar_wait(&S.empty[s], ((chunk / STAGES) - 1) & 1, WAIT_LIMIT)) {
                    S.err = 1;
                    ok = false;
                    break;
                }
                tc::tc_fence_after();   // the MMAs that read this stage are complete
                {
                    float rh[8], rl[8], ih[8], il[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        tc::split_tf32(h[i].x, rh[i], rl[i]);
                        tc::split_tf32(h[i].y, ih[i], il[i]);
                    }
                    const uint32_t ts = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + TS0 + 64 * s + 8 * (warp >> 2);
                    tmem_st8(ts, rh);
                    tmem_st8(ts + 16, rl);
                    tmem_st8(ts + 32, ih);
                    tmem_st8(ts + 48, il);
                }
                const uint32_t base = tc::smem_u32(S.stage[s]);
                {
                    // B rows n: -Xi^T, 64 + n: Xr^T, 128 + n: Xi^T
                    const int n = 8 * warp + (lane & 7), kq = lane >> 3;
                    const float re[4] = {xv[0].x, xv[0].z, xv[1].x, xv[1].z};
                    const float im[4] = {xv[0].y, xv[0].w, xv[1].y, xv[1].w};
                    float rh[4], rl[4], ih[4], il[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        tc::split_tf32(re[i], rh[i], rl[i]);
                        tc::split_tf32(im[i], ih[i], il[i]);
                    }
                    const uint32_t o_n = (uint32_t)(n >> 3) * SBO + kq * LBO + (n & 7) * 16;
                    const uint32_t o_r = o_n + 8 * SBO, o_i = o_n + 16 * SBO;
                    st_shared_v4(base + o_n, -ih[0], -ih[1], -ih[2], -ih[3]);
                    st_shared_v4(base + o_r, rh[0], rh[1], rh[2], rh[3]);
                    st_shared_v4(base + o_i, ih[0], ih[1], ih[2], ih[3]);
                    st_shared_v4(base + XPART + o_n, -il[0], -il[1], -il[2], -il[3]);
                    st_shared_v4(base + XPART + o_r, rl[0], rl[1], rl[2], rl[3]);
                    st_shared_v4(base + XPART + o_i, il[0], il[1], il[2], il[3]);
                }
                tc::tmem_st_wait();
                tc::fence_proxy_async_smem();
                tc::tc_fence_before();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&S.full[s]);
                ++chunk;
            }
            if (!ok) break;
        }
        tc::cp_async_wait_all();   // no copy may still be landing when the CTA exits
    } else if (warp < MMA_WARP) {
        // ---------------- drain ----------------
        const int dw = warp - NPW;
        const int quad = warp & 3;
        const int half = dw >> 2;                  // columns [32 half, 32 half + 32) of the group
        const int row = 32 * quad + lane;
        uint32_t grp = 0, tile = 0;
        for (int j = blockIdx.x; j < n_list; j += gridDim.x) {
            const int2 job = list[j];
            const DevInst &in = insts[job.x];
            const int M = in.M, NCOL = in.ncols, ldw = in.ldw, col0 = 64 * job.y;
            float2 *__restrict__ W = in.W;
            const int nmt = (M + TMR - 1) / TMR;
            const int ngrp = ((in.K + KCH - 1) / KCH + G - 1) / G;
            for (int mt = 0; mt < nmt; ++mt, ++tile) {
                const int b = tile & 1;
                float wr[32], wi[32];
#pragma unroll
                for (int i = 0; i < 32; ++i) wr[i] = wi[i] = 0.f;
                bool ok = true;
                for (int g = 0; g < ngrp; ++g, ++grp) {
                    const int gb = grp & 1;
                    ok = ok && !S.err && tc::mbar_wait(&S.accf[gb], (grp >> 1) & 1, WAIT_LIMIT);
                    if (!ok) S.err = 1;
                    tc::tc_fence_after();
                    if (ok) {
                        const uint32_t ta = tmem + ((uint32_t)(32 * quad) << 16) + gb * 128 + 32 * half;
                        float v[16];
                        tc::tmem_ld16(ta, v);
                        tc::tmem_ld_wait();
#pragma unroll
                        for (int i = 0; i < 16; ++i) wr[i] += v[i];
                        tc::tmem_ld16(ta + 16, v);
                        tc::tmem_ld_wait();
#pragma unroll
                        for (int i = 0; i < 16; ++i) wr[16 + i] += v[i];
                        tc::tmem_ld16(ta + 64, v);
                        tc::tmem_ld_wait();
#pragma unroll
                        for (int i = 0; i < 16; ++i) wi[i] += v[i];
                        tc::tmem_ld16(ta + 80, v);
                        tc::tmem_ld_wait();
#pragma unroll
                        for (int i = 0; i < 16; ++i) wi[16 + i] += v[i];
                    }
                    tc::tc_fence_before();
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(&S.acce[gb]);
                }
                float nrm = 0.f;
                const int gm = mt * TMR + row;
                if (ok && gm < M) {
#pragma unroll
                    for (int i = 0; i < 32; ++i) {
                        const int jj = col0 + 32 * half + i;
                        if (jj < NCOL) {
                            W[gm + (size_t)jj * ldw] = make_float2(wr[i], wi[i]);
                            nrm = fmaf(wr[i], wr[i], nrm);
                            nrm = fmaf(wi[i], wi[i], nrm);
                        }
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
                if (lane == 0) S.wsum[b][dw] = nrm;
                asm volatile("bar.sync 1, 256;\n" ::: "memory");
                if (dw == 0 && lane == 0) {
                    float s = 0.f;
#pragma unroll
                    for (int w = 0; w < NDW; ++w) s += S.wsum[b][w];
                    in.wpart[job.y * nmt + mt] = s;
                }
            }
        }
    } else if (lane == 0) {
        // ---------------- MMA issuer ----------------
        constexpr uint32_t id128 = tc::idesc_tf32(TMR, 128);
        uint32_t chunk = 0, grp = 0;
        for (int j = blockIdx.x; j < n_list && !S.err; j += gridDim.x) {
            const DevInst &in = insts[list[j].x];
            const int nmt = (in.M + TMR - 1) / TMR;
            const int nks = (in.K + KCH - 1) / KCH;
            for (int mt = 0; mt < nmt && !S.err; ++mt) {
                for (int ks = 0; ks < nks; ++ks, ++chunk) {
                    const int b = grp & 1;
                    if (ks % G == 0 && grp >= 2) {   // this buffer's previous group has been drained
                        if (!tc::mbar_wait(&S.acce[b], ((grp >> 1) - 1) & 1, WAIT_LIMIT)) {
                            S.err = 1;
                            break;
                        }
                        tc::tc_fence_after();
                    }
                    const uint32_t d = tmem + b * 128;
                    const int s = chunk % STAGES;
                    if (!tc::mbar_wait(&S.full[s], (chunk / STAGES) & 1, WAIT_LIMIT)) {
                        S.err = 1;
                        break;
                    }
                    tc::tc_fence_after();
                    const uint32_t xh = tc::smem_u32(S.stage[s]), xl = xh + XPART;
                    const uint32_t ta = tmem + TS0 + 64 * s;
#pragma unroll
                    for (int kk = 0; kk < KCH / 8; ++kk) {
                        const uint32_t off = kk * 2 * LBO;
                        // [Xr; Xi] (rows 64 ..) for Hr, [-Xi; Xr] (rows 0 ..) for Hi
                        const uint64_t b1h = tc::smem_desc(xh + off + 8 * SBO, LBO, SBO);
                        const uint64_t b1l = tc::smem_desc(xl + off + 8 * SBO, LBO, SBO);
                        const uint64_t b2h = tc::smem_desc(xh + off, LBO, SBO);
                        const uint64_t b2l = tc::smem_desc(xl + off, LBO, SBO);
                        const uint32_t ak = ta + 8 * kk;
                        const uint32_t first = (ks % G == 0 && kk == 0) ? 0u : 1u;
                        tc::mma_tf32_tmem_a(d, ak, b1h, id128, first);        // Hr hi
                        tc::mma_tf32_tmem_a(d, ak, b1l, id128, 1u);
                        tc::mma_tf32_tmem_a(d, ak + 16, b1h, id128, 1u);      // Hr lo
                        tc::mma_tf32_tmem_a(d, ak + 32, b2h, id128, 1u);      // Hi hi
                        tc::mma_tf32_tmem_a(d, ak + 32, b2l, id128, 1u);
                        tc::mma_tf32_tmem_a(d, ak + 48, b2h, id128, 1u);      // Hi lo
                    }
                    tc::mma_commit(&S.empty[s]);
                    if (ks % G == G - 1 || ks == nks - 1) {
                        tc::mma_commit(&S.accf[b]);
                        ++grp;
                    }
                }
            }
        }
        tc::mma_commit(&S.fin);
        tc::mbar_wait(&S.fin, 0, WAIT_LIMIT);
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

cudaError_t launch_hx_tc_wide(const DevInst *insts, const int2 *list, int n, DevAccum acc,
                              cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const size_t smem = sizeof(HxwSmem);
    cudaError_t e = cudaFuncSetAttribute(hx_tc_wide_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const int grid = n < sms ? n : sms;
    hx_tc_wide_kernel<<<grid, NTHREADS, smem, s>>>(insts, list, n, acc);
    return cudaGetLastError();
}

}  // namespace jacpcg
