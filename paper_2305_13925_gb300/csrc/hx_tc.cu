// hx_tc.cu -- the precoder W = H X on the tcgen05 tensor cores for the K = 64
// class (Eq. 7 without the power factor; Eq. 15 per symbol), 3xTF32.
//
// Complex product as real MMAs over one 128-row tile of W (rows = antennas):
//   [Wr | Wi] = Hr [Xr | Xi] + Hi [-Xi | Xr].
// B = [-Xi^T ; Xr^T ; Xi^T] (192 rows of K values, K-major) is resident in
// shared memory per instance; its rows 64 .. 191 are [Xr^T ; Xi^T] and its
// rows 0 .. 127 are [-Xi^T ; Xr^T], so each reduction step is two N = 128
// MMAs, Hr against the first view and Hi against the second, each as
// hi*hi + hi*lo + lo*hi of the TF32 split (see gram_tc.cu).  The H stage
// (Hr and Hi, head and tail) lives in tensor memory as the MMAs' A operand:
// an MMA reads only its 4 KB B slice from shared memory (the stage never
// passes through shared memory after the raw copy), which cut the kernel from
// 0.436 to 0.375 ms per 2048-channel batch.  The reduction is only 2K long,
// so one TMEM accumulation per tile suffices.
//
// Persistent, warp-specialised, one CTA per SM walking its instances:
//   warps 0-7   producers: a stream of raw stages fetched RAW - 1 stages
//               ahead with per-thread asynchronous copies (cp.async, 16
//               bytes, zero-filled past M and K): per instance two stages of
//               the iterate X (each thread copies the chunks it converts into
//               B), then the H stages, where warp w copies antennas
//               32 (w mod 4) .. + 31 -- its TMEM lanes -- of the stage's users
//               8 (w / 4) .. + 7 as whole 256-byte column pieces, converts
//               exactly those entries and writes them to its lanes of the
//               tensor-memory stage (tcgen05.st), so a __syncwarp after its
//               own cp.async wait suffices.  Every raw stage keeps warp w's
//               bytes in its own 2 KB: the warps run unsynchronised, and a
//               warp refilling a stage must not overwrite bytes another warp
//               has yet to read;
//   warps 8-15  drain: TMEM (two alternating 128-column accumulators) ->
//               registers -> W (complex64, column-major, coalesced) and this
//               tile's ||W||_F^2 partial in its own slot;
//   warp 16     TMEM allocation; lane 0 issues the MMAs and commits.
// Every wait is bounded; a timeout flags the CTA's instances with FLAG_TIMEOUT.
#include "common.cuh"
#include "kernels.h"
#include "tc.cuh"

namespace jacpcg {

namespace {

constexpr int TMR = 128;                      // W rows per tile
constexpr int KCH = 16;                       // users (reduction values) per stage
constexpr int STAGES = 4;                     // H stages in tensor memory shared with the MMA warp
                                              // (4 measured 0.356 vs 0.366 ms with 2: they cost
                                              // no shared memory, and decouple the producers)
constexpr int RAW = 6;                        // raw stages in flight per producer thread
constexpr int RAWB = 16 * 1024;               // bytes of one raw stage
constexpr int BROWS = 192;                    // B rows: -Xi^T, Xr^T, Xi^T (64 each)
constexpr int BPART = BROWS * 64 * 4;         // one of B_hi, B_lo: 48 KB
constexpr uint32_t LBO = 128;
constexpr uint32_t SBO_B = (64 / 4) * 128;    // 2048
constexpr uint32_t TS0 = 256;                 // H stages: columns TS0 + 64 s + 16 part + user
constexpr uint32_t WAIT_LIMIT = 1u << 21;
constexpr int NPW = 8, NDW = 8;
constexpr int MMA_WARP = NPW + NDW;
constexpr int NTHREADS = (NPW + NDW + 1) * 32;
constexpr int TMEM_COLS = 512;                // two accumulators, four H stages (hi / lo of Hr, Hi)

struct __align__(128) HxSmem {
    unsigned char B[2 * BPART];
    unsigned char raw[RAW][RAWB];
    float wsum[2][NDW];
    uint64_t full[STAGES];
    uint64_t empty[STAGES];
    uint64_t bfull, bempty;
    uint64_t accf[2];
    uint64_t acce[2];
    uint64_t fin;
    uint32_t tmem;
    volatile int err;
};

static_assert(sizeof(HxSmem) <= 227 * 1024, "shared memory");

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

__global__ void __launch_bounds__(NTHREADS, 1) hx_tc64_kernel(const DevInst *__restrict__ insts,
                                                              const int *__restrict__ list, int n_list,
                                                              DevAccum acc_out) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    HxSmem &S = *reinterpret_cast<HxSmem *>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            tc::mbar_init(&S.full[s], NPW);
            tc::mbar_init(&S.empty[s], 1);
        }
        tc::mbar_init(&S.bfull, NPW);
        tc::mbar_init(&S.bempty, 1);
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
        const int tid = threadIdx.x;   // 0 .. 255
        const uint32_t bbase = tc::smem_u32(S.B);
        const uint32_t raw0 = tc::smem_u32(S.raw[0]);
        // stream cursor: (instance ordinal, stage) of this CTA's walk; per instance
        // stages 0 and 1 carry X (columns 32 t ..), then the H stages
        struct Cursor {
            int j, t, nst, nks, M, K, ldh, ncols;
            const char *H;
            const char *X;
            bool bf16;
        };
        auto cursor_load = [&](Cursor &u) {
            if (u.j < n_list) {
                const DevInst &in = insts[list[u.j]];
                u.M = in.M;
                u.K = in.K;
                u.ncols = in.ncols;
                u.ldh = in.ldh;
                u.H = reinterpret_cast<const char *>(in.H);
                u.X = reinterpret_cast<const char *>(in.X);
                u.bf16 = in.h_bf16 != 0;
                u.nks = (u.K + KCH - 1) / KCH;
                u.nst = 2 + ((u.M + TMR - 1) / TMR) * u.nks;
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
                if (u.t < 2) {
                    // X rows 4 rq .. 4 rq + 3 of column n, as two chunks of two rows
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int e = tid + 256 * (2 * u.t + h);
                        const int n = (e & 7) + 8 * (e >> 7), rq = (e >> 3) & 15;
#pragma unroll
                        for (int c = 0; c < 2; ++c) {
                            const int r = 4 * rq + 2 * c;
                            const int left = n < u.ncols ? min(max(u.K - r, 0), 2) : 0;
                            const char *src = u.X + ((size_t)n * 64 + r) * 8;
                            tc::cp_async16(rb + warp * 2048 + ((2 * h + c) * 32 + lane) * 16, left ? src : u.X,
                                           left * 8);
                        }
                    }
                } else {
                    // warp w: antennas 32 (w mod 4) .. + 31 (its TMEM lanes) of the stage's
                    // users 8 (w / 4) .. + 7, whole 256-byte (128-byte bfloat16) column pieces
                    const int st = u.t - 2, mt = st / u.nks, ks = st % u.nks;
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
                }
            }
            tc::cp_async_commit();   // one group per stage, empty past the end
        };
        Cursor iu{(int)blockIdx.x, 0, 0, 0, 0, 0, 0, 0, nullptr, nullptr, false};
        cursor_load(iu);
#pragma unroll 1
        for (int p = 0; p < RAW - 1; ++p) {
            issue(iu, p);
            cursor_next(iu);
        }
        uint32_t chunk = 0, ninst = 0, sc = 0;
        for (int j = blockIdx.x; j < n_list && !S.err; j += gridDim.x, ++ninst) {
            const DevInst &in = insts[list[j]];
            const int M = in.M, K = in.K;
            const bool bf16 = in.h_bf16 != 0;
            // B = [Xr^T ; Xi^T], rewritten once the previous instance's MMAs are done
            if (ninst > 0 && !tc::mbar_wait(&S.bempty, (ninst - 1) & 1, WAIT_LIMIT)) {
                S.err = 1;
                break;
            }
            for (int xs = 0; xs < 2; ++xs, ++sc) {
                tc::cp_async_wait<RAW - 2>();   // the chunks this thread copied have landed
                const unsigned char *rbuf = S.raw[sc % RAW];
                float2 v[2][4];
#pragma unroll
                for (int h = 0; h < 2; ++h)
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        const float4 w4 =
                            *reinterpret_cast<const float4 *>(rbuf + warp * 2048 + ((2 * h + c) * 32 + lane) * 16);
                        v[h][2 * c] = make_float2(w4.x, w4.y);
                        v[h][2 * c + 1] = make_float2(w4.z, w4.w);
                    }
                issue(iu, (sc + RAW - 1) % RAW);
                cursor_next(iu);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int e = tid + 256 * (2 * xs + h);
                    const int n = (e & 7) + 8 * (e >> 7), rq = (e >> 3) & 15;
                    float rh[4], rl[4], ih[4], il[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        tc::split_tf32(v[h][i].x, rh[i], rl[i]);
                        tc::split_tf32(v[h][i].y, ih[i], il[i]);
                    }
                    // rows n: -Xi^T, 64 + n: Xr^T, 128 + n: Xi^T
                    const uint32_t o_n = (uint32_t)(n >> 3) * SBO_B + rq * LBO + (n & 7) * 16;
                    const uint32_t o_r = o_n + 8 * SBO_B, o_i = o_n + 16 * SBO_B;
                    st_shared_v4(bbase + o_n, -ih[0], -ih[1], -ih[2], -ih[3]);
                    st_shared_v4(bbase + o_r, rh[0], rh[1], rh[2], rh[3]);
                    st_shared_v4(bbase + o_i, ih[0], ih[1], ih[2], ih[3]);
                    st_shared_v4(bbase + BPART + o_n, -il[0], -il[1], -il[2], -il[3]);
                    st_shared_v4(bbase + BPART + o_r, rl[0], rl[1], rl[2], rl[3]);
                    st_shared_v4(bbase + BPART + o_i, il[0], il[1], il[2], il[3]);
                }
            }
            tc::fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&S.bfull);
            // H tiles: stage t = (tile t / nks, users 16 (t % nks) ...)
            const int nmt = (M + TMR - 1) / TMR;
            const int nks = (K + KCH - 1) / KCH;
            const int T = nmt * nks;
            // H stage s in TMEM: thread (warp w, lane l) owns lane 32 (w mod 4) + l
            // (antenna) and columns 8 (w / 4) .. + 7 (users) of each part
            const uint32_t th = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + TS0 + 8 * (warp >> 2);
            auto put = [&](const float2 (&h)[8]) -> bool {
                const int s = chunk % STAGES;
                if (chunk >= STAGES &&
                    !tc::mbar_wait(&S.empty[s], ((chunk / STAGES) - 1) & 1, WAIT_LIMIT)) {
                    S.err = 1;
                    return false;
                }
                tc::tc_fence_after();   // the MMAs that read this stage are complete
                float rh[8], rl[8], ih[8], il[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    tc::split_tf32(h[i].x, rh[i], rl[i]);
                    tc::split_tf32(h[i].y, ih[i], il[i]);
                }
                const uint32_t ts = th + 64 * s;
                tmem_st8(ts, rh);
                tmem_st8(ts + 16, rl);
                tmem_st8(ts + 32, ih);
                tmem_st8(ts + 48, il);
                tc::tmem_st_wait();
                tc::tc_fence_before();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&S.full[s]);
                ++chunk;
                return true;
            };
            bool ok = true;
            for (int t = 0; t < T && ok; ++t, ++sc) {
                tc::cp_async_wait<RAW - 2>();   // this thread's chunks of the stage have landed
                __syncwarp();                   // ... and those of the rest of its warp
                const unsigned char *wr = S.raw[sc % RAW] + warp * 2048;
                float2 h[8];
#pragma unroll
                for (int uu = 0; uu < 8; ++uu)   // antenna 32 (w mod 4) + l of user uu
                    h[uu] = bf16 ? bf16x2_to_float2(*reinterpret_cast<const uint32_t *>(wr + uu * 128 + lane * 4))
                                 : *reinterpret_cast<const float2 *>(wr + uu * 256 + lane * 8);
                issue(iu, (sc + RAW - 1) % RAW);   // refills the stage read one step ago
                cursor_next(iu);
                ok = put(h);
            }
        }
        tc::cp_async_wait_all();   // no copy may still be landing when the CTA exits
    } else if (warp < MMA_WARP) {
        // ---------------- drain ----------------
        const int dw = warp - NPW;
        const int quad = warp & 3;
        const int half = dw >> 2;                  // users [32 half, 32 half + 32)
        const int row = 32 * quad + lane;
        uint32_t tile = 0;
        for (int j = blockIdx.x; j < n_list; j += gridDim.x) {
            const DevInst &in = insts[list[j]];
            const int M = in.M, NCOL = in.ncols, ldw = in.ldw;
            float2 *__restrict__ W = in.W;
            const int nmt = (M + TMR - 1) / TMR;
            for (int mt = 0; mt < nmt; ++mt, ++tile) {
                const int b = tile & 1;
                float wr[32], wi[32];
                bool ok = !S.err && tc::mbar_wait(&S.accf[b], (tile >> 1) & 1, WAIT_LIMIT);
                if (!ok) S.err = 1;
                tc::tc_fence_after();
                if (ok) {
                    const uint32_t ta = tmem + ((uint32_t)(32 * quad) << 16) + b * 128 + 32 * half;
                    float v[16];
                    tc::tmem_ld16(ta, v);
                    tc::tmem_ld_wait();
#pragma unroll
                    for (int i = 0; i < 16; ++i) wr[i] = v[i];
                    tc::tmem_ld16(ta + 16, v);
                    tc::tmem_ld_wait();
#pragma unroll
                    for (int i = 0; i < 16; ++i) wr[16 + i] = v[i];
                    tc::tmem_ld16(ta + 64, v);
                    tc::tmem_ld_wait();
#pragma unroll
                    for (int i = 0; i < 16; ++i) wi[i] = v[i];
                    tc::tmem_ld16(ta + 80, v);
                    tc::tmem_ld_wait();
#pragma unroll
                    for (int i = 0; i < 16; ++i) wi[16 + i] = v[i];
                }
                tc::tc_fence_before();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&S.acce[b]);
                float nrm = 0.f;
                const int gm = mt * TMR + row;
                if (ok && gm < M) {
#pragma unroll
                    for (int i = 0; i < 32; ++i) {
                        const int jj = 32 * half + i;
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
                    in.wpart[mt] = s;
                }
            }
        }
    } else if (lane == 0) {
        // ---------------- MMA issuer ----------------
        constexpr uint32_t id128 = tc::idesc_tf32(TMR, 128);
        const uint32_t bhi = tc::smem_u32(S.B), blo = bhi + BPART;
        uint32_t chunk = 0, tile = 0, ninst = 0;
        for (int j = blockIdx.x; j < n_list && !S.err; j += gridDim.x, ++ninst) {
            const DevInst &in = insts[list[j]];
            const int nmt = (in.M + TMR - 1) / TMR;
            const int nks = (in.K + KCH - 1) / KCH;
            if (!tc::mbar_wait(&S.bfull, ninst & 1, WAIT_LIMIT)) {
                S.err = 1;
                break;
            }
            tc::tc_fence_after();
            for (int mt = 0; mt < nmt && !S.err; ++mt, ++tile) {
                const int b = tile & 1;
                if (tile >= 2) {
                    if (!tc::mbar_wait(&S.acce[b], ((tile >> 1) - 1) & 1, WAIT_LIMIT)) {
                        S.err = 1;
                        break;
                    }
                    tc::tc_fence_after();
                }
                const uint32_t d = tmem + b * 128;
                for (int ks = 0; ks < nks; ++ks, ++chunk) {
                    const int s = chunk % STAGES;
                    if (!tc::mbar_wait(&S.full[s], (chunk / STAGES) & 1, WAIT_LIMIT)) {
                        S.err = 1;
                        break;
                    }
                    tc::tc_fence_after();
                    const uint32_t ta = tmem + TS0 + 64 * s;
#pragma unroll
                    for (int kk = 0; kk < KCH / 8; ++kk) {
                        const uint32_t bo = (uint32_t)(ks * KCH / 4 + 2 * kk) * LBO;
                        // [Xr; Xi] (rows 64 ..) for Hr, [-Xi; Xr] (rows 0 ..) for Hi
                        const uint64_t b1h = tc::smem_desc(bhi + bo + 8 * SBO_B, LBO, SBO_B);
                        const uint64_t b1l = tc::smem_desc(blo + bo + 8 * SBO_B, LBO, SBO_B);
                        const uint64_t b2h = tc::smem_desc(bhi + bo, LBO, SBO_B);
                        const uint64_t b2l = tc::smem_desc(blo + bo, LBO, SBO_B);
                        const uint32_t ak = ta + 8 * kk;
                        const uint32_t first = (ks == 0 && kk == 0) ? 0u : 1u;
                        tc::mma_tf32_tmem_a(d, ak, b1h, id128, first);        // Hr hi
                        tc::mma_tf32_tmem_a(d, ak, b1l, id128, 1u);
                        tc::mma_tf32_tmem_a(d, ak + 16, b1h, id128, 1u);      // Hr lo
                        tc::mma_tf32_tmem_a(d, ak + 32, b2h, id128, 1u);      // Hi hi
                        tc::mma_tf32_tmem_a(d, ak + 32, b2l, id128, 1u);
                        tc::mma_tf32_tmem_a(d, ak + 48, b2h, id128, 1u);      // Hi lo
                    }
                    tc::mma_commit(&S.empty[s]);
                }
                tc::mma_commit(&S.accf[b]);
            }
            tc::mma_commit(&S.bempty);
        }
        tc::mma_commit(&S.fin);
        tc::mbar_wait(&S.fin, 0, WAIT_LIMIT);
    }

    tc::tc_fence_before();
    __syncthreads();
    if (S.err && threadIdx.x == 0) {
        for (int j = blockIdx.x; j < n_list; j += gridDim.x) atomicOr(acc_out.flags + list[j], FLAG_TIMEOUT);
    }
    if (warp == MMA_WARP) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, TMEM_COLS);
    }
}

}  // namespace

cudaError_t launch_hx_tc64(const DevInst *insts, const int *list, int n, DevAccum acc,
                           cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const size_t smem = sizeof(HxSmem);
    cudaError_t e = cudaFuncSetAttribute(hx_tc64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const int grid = n < sms ? n : sms;
    hx_tc64_kernel<<<grid, NTHREADS, smem, s>>>(insts, list, n, acc);
    return cudaGetLastError();
}

}  // namespace jacpcg
