// gram_bf16.cu -- A = H^H H + xi I on the tcgen05 tensor cores for bfloat16
// channels of the K = 128 and 256 classes (Sec. II, definition of P_i after
// Eq. 7), the tensor core reading H as it lies in memory.  A bfloat16
// product is exact in FP32, so one kind::f16 MMA per k-step does what the
// three TF32 products of the 3xTF32 split do for complex64 channels, and no
// producer converts the operands.
//
// User a's channel column h_a, read as 2M real values y_a = (Re h_0a,
// Im h_0a, Re h_1a, ...), is one K-major row of the MMA operands; the
// reduction runs over those 2M values.  Then y_a . y_b = Re(h_a^H h_b), and
// with the rotated row z_b = (Im h_0b, -Re h_0b, Im h_1b, ...),
// y_a . z_b = Im(h_a^H h_b).  A job is (instance, user tiles ta <= tb of 128
// users): D = Y_ta [Y_tb ; Z_tb]^T, one N = 256 MMA per k-step, the real and
// imaginary parts of block (ta, tb) side by side in 256 TMEM columns.
//
// A stage is 32 antennas (64 real values) of the tiles' users: one tiled TMA
// copy per user tile (128 users x 128 bytes, 128-byte swizzle, zero-filled
// past M and K).  The rotation z = (y1, -y0) of each 4-byte (Re, Im) pair
// leaves the swizzled layout as it is, so two warps rotate the landed Y_tb
// word by word into the slot after it.  The tensor core's FP32 accumulation
// truncates, so as in the 3xTF32 kernels the chain is cut every G stages
// (128 antennas, 16 MMAs): the MMAs alternate between two TMEM buffers and
// the drain warps add each finished chain into FP32 registers.
//
// Persistent, warp-specialised, one CTA per SM walking its jobs:
//   warps 0-1   rotate Y_tb into Z_tb, stage by stage;
//   warp 2      lane 0 issues the tensor copies, up to RING stages ahead;
//   warp 3      TMEM allocation; lane 0 issues the MMAs and commits;
//   warps 4-19  drain: TMEM lanes 32 (w mod 4) .. (users of tile ta), users
//               32 ((w - 4) / 4) .. of tile tb; at the end of a job they
//               write block (ta, tb) and its conjugate transpose (a diagonal
//               job: its upper triangle, mirrored, so A is exactly
//               Hermitian), xi on the diagonal and 1 / diag.
// Every wait is bounded; a timeout stops the CTA's pipeline, flags its
// instances with FLAG_TIMEOUT, and the CTA still drains and frees its TMEM.
#include "common.cuh"
#include "kernels.h"
#include "tc.cuh"

namespace jacpcg {

namespace {

constexpr int TU = 128;                  // users per tile: MMA M, half of N
constexpr int TS = 64;                   // real values (32 antennas) per stage
constexpr int TILE = TU * TS * 2;        // one user tile of a stage: 16 KB
constexpr int SLOT = 3 * TILE;           // Y_ta | Y_tb | Z_tb (a diagonal job: Y_ta | Z_ta)
constexpr int RING = 4;
constexpr int G = 4;                     // stages per accumulation chain
constexpr uint32_t WAIT_LIMIT = 1u << 21;
constexpr int NROT = 2, TMA_WARP = 2, MMA_WARP = 3, NDW = 16;
constexpr int NTHREADS = (4 + NDW) * 32;
constexpr int TMEM_COLS = 4 * TU;        // two chain buffers of (Re | Im) x 128 users

struct __align__(1024) GramBSmem {
    unsigned char slot[RING][SLOT];      // each 1024-byte aligned (the swizzle atom)
    uint64_t full[RING];                 // the stage's tensor copies landed
    uint64_t zfull[RING];                // its rotated tile written
    uint64_t empty[RING];                // its MMAs completed
    uint64_t accf[2];                    // chain buffer complete
    uint64_t acce[2];                    // chain buffer drained
    uint64_t fin;
    uint32_t tmem;
    volatile int err;
};
static_assert(sizeof(GramBSmem) + 1024 <= 227 * 1024, "shared memory");

__device__ __forceinline__ uint32_t rot_pair(uint32_t w) {   // (re, im) -> (im, -re)
    return __byte_perm(w, 0u, 0x1032u) ^ 0x80000000u;
}

__device__ __forceinline__ int n_stages(int M) { return (M + TS / 2 - 1) / (TS / 2); }

__global__ void __launch_bounds__(NTHREADS, 1) gram_bf16_kernel(const DevInst *__restrict__ insts,
                                                                const int4 *__restrict__ jobs, int n_jobs,
                                                                const CUtensorMap *__restrict__ maps,
                                                                DevAccum acc_out) {
    extern __shared__ unsigned char smem_raw[];
    const uint32_t pad = (1024u - (tc::smem_u32(smem_raw) & 1023u)) & 1023u;
    GramBSmem &S = *reinterpret_cast<GramBSmem *>(smem_raw + pad);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < RING; ++s) {
            tc::mbar_init(&S.full[s], 1);
            tc::mbar_init(&S.zfull[s], NROT);
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
    const uint32_t slot0 = tc::smem_u32(S.slot[0]);

    if (warp < NROT) {
        // ---------------- rotation: Z = rot(Y) of the stage's second operand tile ----------------
        const uint32_t t = threadIdx.x;
        uint32_t seq = 0;
        for (int j = blockIdx.x; j < n_jobs && !S.err; j += gridDim.x) {
            const int4 job = jobs[j];
            const int nst = n_stages(insts[job.x].M);
            const uint32_t src_off = job.y == job.z ? 0u : (uint32_t)TILE;
            for (int c = 0; c < nst; ++c, ++seq) {
                const int s = seq % RING;
                if (!tc::mbar_wait(&S.full[s], (seq / RING) & 1, WAIT_LIMIT)) {
                    S.err = 1;
                    break;
                }
                const uint32_t src = slot0 + s * SLOT + src_off, dst = src + TILE;
#pragma unroll 4
                for (int i = 0; i < TILE / 16 / (NROT * 32); ++i) {
                    const uint32_t off = (i * NROT * 32 + t) * 16;
                    uint32_t x0, x1, x2, x3;
                    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];\n"
                                 : "=r"(x0), "=r"(x1), "=r"(x2), "=r"(x3)
                                 : "r"(src + off)
                                 : "memory");
                    asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};\n" ::"r"(dst + off), "r"(rot_pair(x0)),
                                 "r"(rot_pair(x1)), "r"(rot_pair(x2)), "r"(rot_pair(x3))
                                 : "memory");
                }
                tc::fence_proxy_async_smem();   // the tensor core reads what this thread wrote
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&S.zfull[s]);
            }
        }
    } else if (warp == TMA_WARP) {
        // ---------------- tensor copies ----------------
        if (lane == 0) {
            uint32_t seq = 0;
            for (int j = blockIdx.x; j < n_jobs && !S.err; j += gridDim.x) {
                const int4 job = jobs[j];
                const CUtensorMap *map = maps + job.w;
                tc::tensormap_acquire(map);
                const int nst = n_stages(insts[job.x].M);
                const bool diag = job.y == job.z;
                for (int c = 0; c < nst; ++c, ++seq) {
                    const int s = seq % RING;
                    if (seq >= RING && !tc::mbar_wait(&S.empty[s], ((seq / RING) - 1) & 1, WAIT_LIMIT)) {
                        S.err = 1;
                        break;
                    }
                    const uint32_t dst = slot0 + s * SLOT;
                    tc::mbar_arrive_expect_tx(&S.full[s], diag ? TILE : 2 * TILE);
                    tc::tma_load_2d(dst, map, c * TS, TU * job.y, &S.full[s]);
                    if (!diag) tc::tma_load_2d(dst + TILE, map, c * TS, TU * job.z, &S.full[s]);
                }
            }
            // no copy may still be landing when the CTA exits
            for (uint32_t q = seq > RING ? seq - RING : 0; q < seq; ++q)
                tc::mbar_wait(&S.full[q % RING], (q / RING) & 1, WAIT_LIMIT);
        }
    } else if (warp == MMA_WARP) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            constexpr uint32_t idesc = tc::idesc_bf16(TU, 2 * TU);
            uint32_t seq = 0, grp = 0;
            for (int j = blockIdx.x; j < n_jobs && !S.err; j += gridDim.x) {
                const int4 job = jobs[j];
                const int nst = n_stages(insts[job.x].M);
                const uint32_t b_off = job.y == job.z ? 0u : (uint32_t)TILE;
                for (int c = 0; c < nst; ++c, ++seq) {
                    const int b = grp & 1;
                    if (c % G == 0 && grp >= 2) {   // the buffer's previous chain has been drained
                        if (!tc::mbar_wait(&S.acce[b], ((grp >> 1) - 1) & 1, WAIT_LIMIT)) {
                            S.err = 1;
                            break;
                        }
                        tc::tc_fence_after();
                    }
                    const int s = seq % RING;
                    if (!tc::mbar_wait(&S.zfull[s], (seq / RING) & 1, WAIT_LIMIT)) {
                        S.err = 1;
                        break;
                    }
                    tc::tc_fence_after();
                    const uint32_t a0 = slot0 + s * SLOT, b0 = a0 + b_off;
                    const uint32_t d = tmem + b * 2 * TU;
#pragma unroll
                    for (int kk = 0; kk < TS / 16; ++kk) {   // 16 values (32 bytes) per k-step
                        const uint64_t ad = tc::smem_desc_sw128(a0 + kk * 32, 16, 1024);
                        const uint64_t bd = tc::smem_desc_sw128(b0 + kk * 32, 16, 1024);
                        tc::mma_bf16(d, ad, bd, idesc, (c % G == 0 && kk == 0) ? 0u : 1u);
                    }
                    tc::mma_commit(&S.empty[s]);
                    if (c % G == G - 1 || c == nst - 1) {
                        tc::mma_commit(&S.accf[b]);
                        ++grp;
                    }
                }
            }
            tc::mma_commit(&S.fin);
            tc::mbar_wait(&S.fin, 0, WAIT_LIMIT);   // no MMA in flight past this point
        }
    } else {
        // ---------------- drain and epilogue ----------------
        const int dw = warp - 4, quad = warp & 3, part = dw >> 2;
        const int row = 32 * quad + lane;   // user of tile ta
        uint32_t grp = 0;
        for (int j = blockIdx.x; j < n_jobs && !S.err; j += gridDim.x) {
            const int4 job = jobs[j];
            const DevInst &in = insts[job.x];
            const int nch = (n_stages(in.M) + G - 1) / G;
            float sr[32], si[32];
#pragma unroll
            for (int i = 0; i < 32; ++i) sr[i] = si[i] = 0.f;
            for (int g = 0; g < nch && !S.err; ++g, ++grp) {
                const int b = grp & 1;
                // the TMEM loads below are warp-collective: the warp agrees on the wait
                if (!__all_sync(0xffffffffu, tc::mbar_wait(&S.accf[b], (grp >> 1) & 1, WAIT_LIMIT))) {
                    S.err = 1;
                    break;
                }
                tc::tc_fence_after();
                const uint32_t ta = tmem + ((uint32_t)(32 * quad) << 16) + b * 2 * TU + 32 * part;
#pragma unroll
                for (int c0 = 0; c0 < 32; c0 += 16) {
                    float v[16];
                    tc::tmem_ld16(ta + c0, v);
                    tc::tmem_ld_wait();
#pragma unroll
                    for (int i = 0; i < 16; ++i) sr[c0 + i] += v[i];
                    tc::tmem_ld16(ta + TU + c0, v);
                    tc::tmem_ld_wait();
#pragma unroll
                    for (int i = 0; i < 16; ++i) si[c0 + i] += v[i];
                }
                tc::tc_fence_before();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&S.acce[b]);
            }
            const bool bad = S.err != 0;
            const int K = in.K, KC = in.KC;
            const bool diag = job.y == job.z;
            const int a = TU * job.y + row, b0 = TU * job.z + 32 * part;
            // element i: (a, b0 + i) down column b0 + i, and its mirror along row a
            float2 *__restrict__ pc = in.A + a + (size_t)b0 * KC;
            float2 *__restrict__ pr = in.A + (size_t)a * KC + b0;
            float2 *__restrict__ oc = in.Aout ? in.Aout + a + (size_t)b0 * K : nullptr;
            float2 *__restrict__ orow = in.Aout ? in.Aout + (size_t)a * K + b0 : nullptr;
            const bool user_a = a < K;
            // a diagonal job writes its strict upper triangle and the mirror, then the diagonal
            const int rel = diag ? row - 32 * part : -1;   // element rel lies on the diagonal
            float dre = 0.f;
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                if (i == rel) dre = sr[i];
                if (i > rel) {
                    pc[(size_t)i * KC] = make_float2(sr[i], si[i]);
                    if (oc && user_a && b0 + i < K) oc[(size_t)i * K] = make_float2(sr[i], si[i]);
                }
            }
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                if (i > rel) {
                    pr[i] = make_float2(sr[i], -si[i]);
                    if (orow && user_a && b0 + i < K) orow[i] = make_float2(sr[i], -si[i]);
                }
            }
            if (rel >= 0 && rel < 32) {
                const float re = user_a ? dre + in.xi : 0.f;
                in.dinv[a] = user_a ? 1.0f / re : 0.f;
                pc[(size_t)rel * KC] = make_float2(re, 0.f);
                if (oc && user_a) oc[(size_t)rel * K] = make_float2(re, 0.f);
            }
            if (bad && dw == 0 && lane == 0) atomicOr(acc_out.flags + job.x, FLAG_TIMEOUT);
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

cudaError_t launch_gram_bf16(const DevInst *insts, const int4 *jobs, int n, const CUtensorMap *maps, DevAccum acc,
                             cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const size_t smem = sizeof(GramBSmem) + 1024;   // + alignment of the ring to the swizzle atom
    cudaError_t e =
        cudaFuncSetAttribute(gram_bf16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const int grid = n < sms ? n : sms;
    gram_bf16_kernel<<<grid, NTHREADS, smem, s>>>(insts, jobs, n, maps, acc);
    return cudaGetLastError();
}

}  // namespace jacpcg
