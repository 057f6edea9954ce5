// pcg_tcw.cu -- the Jac-PCG iteration with Q = A P on the tcgen05 tensor
// cores for the K = 128 and K = 256 classes (Sec. III-B Steps 1-4, Eqs. 12-14
// and 19-21; standard and plain-CG forms; right-hand side B = I, the
// caller's symbol vectors, or the refinement residual; warm start from X0),
// as pcg_tc.cu does for the 64 class.
//
// At K = 256 A does not fit on one SM (512 KB complex), so it is streamed
// (at K = 128 its 128 KB of stages stay resident for a job).  Once per instance a prep kernel stores it as MMA-ready FP16
// tiles, for row tile rt (128 rows) and k-step ks (16 columns): Ar_h, Ai_h,
// Ar_t, Ai_t, each a 128 x 16 tile in the canonical no-swizzle K-major
// layout, in groups of SUB k-steps [heads of the group | tails of the group],
// of the scaled matrix
//   Ah = 2^13 E^-1 A E^-1,   E = diag(2^e_i),  2^e_i <= sqrt(A_ii) < 2^(e_i + 1),
// split into an FP16 head and the FP16 rounding of the rest.  Every scaling is
// a power of two (exact), and |A_ij| <= sqrt(A_ii A_jj) bounds |Ah_ij| below
// 2^15, inside FP16's range; head + tail carries 22 bits of every entry, as
// the TF32 head and tail of the 3xTF32 split do, in half the bytes, and the
// kind::f16 MMAs run at twice the kind::tf32 rate.  Each iteration streams the
// groups through a shared-memory ring with bulk copies (the TMA unit,
// cp.async.bulk), one 64 KB copy per group (a light correction: the heads of
// two groups), completion counted in bytes on an mbarrier.  Real and
// imaginary parts are kept apart (planar), so each byte of A is streamed once
// per iteration rather than twice as in the 2 x 2 real expansion.
//
// The columns of X are independent systems sharing A, so a CTA owns 32 of
// them (NB) for one instance, one CTA per SM.  Their P is resident in shared
// memory as the MMA's B operand, laid out as 4 NB rows [Pr_h | Pi_h | Pr_t | Pi_t] along N:
// FP16 head and tail of s_j E p_j, s_j a power of two per column that puts
// the column's largest entry in [2^14, 2^15).  Per k-step:
//   U += Ar_h [P_h | P_t]  (N = 4 NB),   U[2 NB..] += Ar_t P_h  (N = 2 NB),
//   V += Ai_h [P_h | P_t],               V[2 NB..] += Ai_t P_h,
// so U = Ar [Pr | Pi] and V = Ai [Pr | Pi] with every product exact (columns
// 0 .. 2 NB - 1 head x head, the rest both corrections), and
//   Re w = Ar Pr - Ai Pi,   Im w = Ai Pr + Ar Pi,   w = E^-1 A p,
// each scaled by 2^-13 / s_j on its way out of TMEM.  U and V of both row
// tiles take 2 x 2 x 4 NB TMEM columns (K = 256: all 512 of the SM's).  The
// accumulation chain of a row tile is its KC / 16 k-steps.  The iteration uses
// p as published (head + tail, 22 bits), in the product and everywhere else,
// so the recurrences stay consistent.
//
// Roles: 16 warps own the vectors; each iteration they publish P (split) into
// the B operand and vote on continuing (one barrier reduction), then thread 0
// streams the iteration's groups (waiting on `empty`), thread 32 issues the
// MMAs (waiting on `full`) and commits to `qfull`, and the epilogue -- idle
// while the product runs, so the roles take no warps of their own -- waits on
// `qfull`, moves U and V out of TMEM as Re w and Im w planes, column-major,
// into a staging area (ring slot 1, or after the ring when A stays resident),
// and works column-wise: thread (warp w, lane l) owns column 2 w + (l mod 2)
// and the complex row pairs 2 g + 32 n, 2 g + 32 n + 1 with g = l / 2 (16 rows
// at K = 256), so that its staging reads, B stores and reductions are two rows
// wide.  It works in the Jacobi-scaled variables of the product (r' = E^-1 r,
// u = s_j E p), where the row factors cancel from every step but the update
// of x.  r' and u (as published: head + tail, exact in FP32) live in
// registers; x lives in the instance's workspace X (which is also where a
// refinement correction X += dX lands) and takes x += lambda p as
// fire-and-forget reductions, so no thread waits on a global load inside the
// iteration.  The step denominator p^H A p, whose terms can cancel, is
// compensated (TwoProduct by FMA and TwoSum in a tree, then xor shuffles
// combined with commutative or exact operations); a light correction, which
// only has to cut the error by a fixed factor, sums it plainly.  The squared
// norms r^H D^{-1} r and ||r||^2 sum nonnegative terms, where pairwise
// summation is already accurate to a few units, and are summed so.  All lanes
// of a column hold bit-identical totals.  Every wait is bounded; a timeout
// sets the instance's ETIMEOUT flag and ends its iteration.
#include <cuda_fp16.h>

#include "common.cuh"
#include "kernels.h"
#include "tc.cuh"

namespace jacpcg {

namespace {

// One CTA per SM of 16 warps owning 32 columns, two ring slots of one 64 KB
// group each.  Measured on the XL batch's main solve (K = 256): two CTAs per
// SM of 8 warps and 16 columns each, 32 KB slots (one CTA's epilogue
// overlapping the other's product, but twice the bytes of A streamed per
// column): 3.41 ms; one CTA, 32 columns, 16 warps, four 32 KB slots: 3.29;
// two 64 KB slots: 3.09 (four 32 KB slots, even with a second copy-issuing
// thread, 3.28; eight 16 KB slots 3.75: the fewer, larger copies the
// better); the next iteration's first group copied during the epilogue:
// 2.84.  The three MMAs per k-step of the head / tail split take about 4 us
// of an iteration's 6 us product at the measured tensor peak.  16 warps (128
// registers, 16 rows per thread) rather than 8 (255, 32 rows) hide more of the
// epilogue's latency.
constexpr int NB = 32;                        // right-hand-side columns per CTA
constexpr int THREADS = 512;                  // 16 warps, up to 128 registers each
constexpr int CTAS_PER_SM = 1;
constexpr int EPI = THREADS;
constexpr int WARPS = THREADS / 32;
constexpr int CPW = NB / WARPS;               // columns per warp in the epilogue
constexpr int LPC = 32 / CPW;                 // lanes per column: lane bits log2(CPW) .. 4
constexpr int RCOLS = NB / (WARPS / 4);       // columns per warp in the TMEM readout
constexpr int STAGE = 16384;                  // bytes of one k-step: four 128 x 16 FP16 tiles
constexpr int SUB = 4;                        // k-steps per group: one bulk copy per ring slot
constexpr int SLOT = SUB * STAGE;
constexpr int RING = 2;                       // ring slots in flight per CTA
constexpr int TILE = 4096;
constexpr int SA = 13;                        // A is stored scaled by 2^SA (entries below 2^15)
constexpr int SP = 14;                        // a column of P is scaled to a largest entry in [2^14, 2^15)
constexpr uint32_t WAIT_LIMIT = 1u << 22;
constexpr int BAR_EPI = 1;                    // named barrier of the epilogue warps

template <int KC>
struct Cfg {
    static constexpr int RT = KC / 128;                      // row tiles
    static constexpr int KS = KC / 16;                       // k-steps per row tile
    static constexpr int NSTAGE = RT * KS;                   // stages per iteration
    static constexpr uint32_t SBO_B = (KC / 8) * 128;        // bytes between 8-row groups of B (N)
    static constexpr int B_BYTES = 4 * NB * KC * 2;          // the B operand
    static constexpr int MR = KC / LPC;                      // complex rows per epilogue thread
    static constexpr uint32_t TMEM_COLS = RT * 8 * NB;       // per row tile U | V, 4 NB columns each
    // A's stages fit the ring (K = 128: 128 KB): they stay resident for the job,
    // copied in by its first product, and the readout is staged after the ring
    static constexpr bool RES = NSTAGE * STAGE <= RING * SLOT;
    static constexpr int STG_BYTES = 2 * RT * NB * 128 * 4;   // Re, Im staging planes
    static constexpr int STG_OFF = RES ? B_BYTES + RING * SLOT : B_BYTES + SLOT;   // else ring slot 1
    static constexpr int TAB_OFF = B_BYTES + RING * SLOT + (RES ? STG_BYTES : 0);
    // B, ring, [staging], then per row {2^(2e) / A_ii, 2^(2e)} and {2^e, 2^-e}; per
    // column the readout factor
    static constexpr int SMEM = TAB_OFF + 4 * KC * 4 + NB * 4 + 256;
    static_assert(STG_BYTES <= SLOT, "the readout staging fits one ring slot");
    static_assert(KS % (2 * SUB) == 0, "whole slots in a row tile");
    static_assert(RING == 2, "group s of an iteration goes to slot s mod 2");
    static_assert(CTAS_PER_SM * (SMEM + 1024) <= 228 * 1024, "shared memory");
    static_assert(CTAS_PER_SM * TMEM_COLS <= 512, "tensor memory");
    static_assert(CPW * WARPS == NB && LPC * CPW == 32 && MR % 8 == 0, "whole columns per warp");
    static_assert(WARPS % 4 == 0 && RCOLS % 8 == 0, "the readout covers the TMEM lane quarters");
};

struct Ctl {
    uint64_t full[RING], empty[RING];
    uint64_t qfull;
    uint32_t tmem;
    volatile int err;
};

__device__ __forceinline__ void epi_sync() {
    asm volatile("bar.sync %0, %1;\n" ::"r"(BAR_EPI), "r"(EPI) : "memory");
}
__device__ __forceinline__ int epi_or(int pred) {
    int r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.s32 p, %1, 0;\n\t"
        "bar.red.or.pred q, %2, %3, p;\n\t"
        "selp.s32 %0, 1, 0, q;\n\t}\n"
        : "=r"(r)
        : "r"(pred), "r"(BAR_EPI), "r"(EPI)
        : "memory");
    return r;
}
// bulk copy global -> shared (both 16-byte aligned, bytes a multiple of 16),
// completion as transaction bytes on `bar`
__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(tc::smem_u32(bar))
        : "memory");
}

// byte offset of element (n, k) in the B operand (FP16, K-major, no swizzle)
template <int KC>
__device__ __forceinline__ uint32_t b_off(int n, int k) {
    return (uint32_t)(n >> 3) * Cfg<KC>::SBO_B + (uint32_t)(k >> 3) * 128u + (uint32_t)(n & 7) * 16u +
           (uint32_t)(k & 7) * 2u;
}

// 2^v as a float, v in [-126, 127]
__device__ __forceinline__ float pow2f(int v) { return __uint_as_float((uint32_t)(v + 127) << 23); }
// e with 2^e <= x < 2^(e + 1) for a normal x > 0
__device__ __forceinline__ int exp2_of(float x) { return (int)((__float_as_uint(x) >> 23) & 0xFFu) - 127; }
// the row exponent e_i of the scaling: 2^e_i <= sqrt(A_ii) < 2^(e_i + 1); 0 for
// padding rows (A_ii = 0) and anything not positive
__device__ __forceinline__ int row_exp(float aii) {
    if (!(aii >= 1.2e-38f) || !(aii < 3.0e38f)) return 0;
    return exp2_of(sqrtf(aii));
}
// x = h + t + (the rest), h and t FP16 (round to nearest); the FP32 sum h + t is exact
__device__ __forceinline__ void split_f16(float x, __half &h, __half &t) {
    h = __float2half_rn(x);
    t = __float2half_rn(x - __half2float(h));
}
// *dst = v as a relaxed store at GPU scope (8-byte aligned)
__device__ __forceinline__ void st_relaxed2(float2 *dst, float2 v) {
    asm volatile("st.relaxed.gpu.global.v2.f32 [%0], {%1, %2};" ::"l"(dst), "f"(v.x), "f"(v.y) : "memory");
}
// base[OFF / 16] += v in global memory (two complex values, 16-byte aligned)
// as one reduction that returns nothing: the issuing thread does not wait for
// it.  The byte offset is an immediate, so the unrolled rows share one address
// register.
template <int OFF>
__device__ __forceinline__ void red_add4(float2 *base, float4 v) {
    asm volatile("red.relaxed.gpu.global.add.v4.f32 [%0+%5], {%1, %2, %3, %4};" ::"l"(base), "f"(v.x), "f"(v.y),
                 "f"(v.z), "f"(v.w), "n"(OFF));
}
// red_add4 of f(n) at the row pairs n = M, M + 1, ..., N - 1 of base, STRIDE
// float2 apart
template <int M, int N, int STRIDE, typename F>
__device__ __forceinline__ void red_pairs(float2 *base, F f) {
    if constexpr (M < N) {
        red_add4<M * STRIDE * 8>(base, f(M));
        red_pairs<M + 1, N, STRIDE>(base, f);
    }
}
// keeps the compiler from moving memory accesses across this point: the row
// loops fence every 8 rows so that their loads are not all hoisted at once
// (with r and p resident, that would exceed the register file)
__device__ __forceinline__ void row_chunk_fence() { asm volatile("" ::: "memory"); }

// ---------------------------------------------------------------------------
// A (complex, workspace ld KC) -> the streamed FP16 stages of 2^SA E^-1 A E^-1:
// one CTA per (instance, stage); element (r, k) of a 128 x 16 tile at
// (r / 8) 256 + (k / 8) 128 + (r mod 8) 16 + (k mod 8) 2 bytes (LBO 128 along
// K, SBO 256 along M).
template <int KC>
__global__ void __launch_bounds__(256) tcw_prep_kernel(const DevInst *__restrict__ insts,
                                                      const int *__restrict__ list) {
    using C = Cfg<KC>;
    const int id = list[blockIdx.x / C::NSTAGE];
    const int s = blockIdx.x % C::NSTAGE, rt = s / C::KS, ks = s % C::KS;
    const DevInst &in = insts[id];
    // groups of SUB k-steps, [heads of the SUB k-steps | their tails], so that a
    // ring slot is one bulk copy, and a light correction's slot (heads only) two
    const int u0 = ks % SUB;
    char *dh = reinterpret_cast<char *>(in.As) + (size_t)(s - u0) * STAGE + (size_t)u0 * (STAGE / 2);
    char *dt = dh + SUB * (STAGE / 2);
    const float2 *__restrict__ A = in.A;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        const int e = threadIdx.x + 256 * u, r = e & 127, k = e >> 7;
        const int gi = rt * 128 + r, gk = ks * 16 + k;
        const float2 v = A[(size_t)gi + (size_t)gk * KC];
        // two factors, each inside the float exponent range; every product exact
        const float si = pow2f(SA - row_exp(A[(size_t)gi * (KC + 1)].x));
        const float sk = pow2f(-row_exp(A[(size_t)gk * (KC + 1)].x));
        __half rh, rl, ih, il;
        split_f16((v.x * si) * sk, rh, rl);
        split_f16((v.y * si) * sk, ih, il);
        const uint32_t o = (uint32_t)(r >> 3) * 256u + (uint32_t)(k >> 3) * 128u + (uint32_t)(r & 7) * 16u +
                           (uint32_t)(k & 7) * 2u;
        *reinterpret_cast<__half *>(dh + o) = rh;          // [Ar_h | Ai_h] of the k-step
        *reinterpret_cast<__half *>(dh + TILE + o) = ih;
        *reinterpret_cast<__half *>(dt + o) = rl;          // [Ar_t | Ai_t]
        *reinterpret_cast<__half *>(dt + TILE + o) = il;
    }
}

// Compensated sum over the thread's MR rows of Re conj(a_m) b_m: rows in
// chunks of 8, f(u, a, b) filling the operand pairs of chunk u, each chunk a
// TwoSum tree over the TwoProduct-split products, the chunks combined the same
// way, then the lanes of the column (lane bits log2(CPW) .. 4) by xor
// shuffles.  Only one chunk of operands is live at a time.
template <int MR, typename F>
__device__ __forceinline__ float col_sum2(F f) {
    constexpr int CH = 8;
    constexpr int NCH = MR / CH;
    static_assert(MR % CH == 0, "whole chunks");
    float S[NCH], Cc[NCH];
#pragma unroll
    for (int u = 0; u < NCH; ++u) {
        float2 a[CH], b[CH];
        f(u, a, b);
        float s[CH], c[CH];
#pragma unroll
        for (int k = 0; k < CH; ++k) {
            const float p1 = a[k].x * b[k].x, p2 = a[k].y * b[k].y;
            const float e1 = fmaf(a[k].x, b[k].x, -p1), e2 = fmaf(a[k].y, b[k].y, -p2);
            float e;
            two_sum(p1, p2, s[k], e);
            c[k] = (e1 + e2) + e;
        }
#pragma unroll
        for (int h = CH / 2; h > 0; h >>= 1) {
#pragma unroll
            for (int k = 0; k < h; ++k) {
                float sk, e;
                two_sum(s[k], s[k + h], sk, e);
                s[k] = sk;
                c[k] = (c[k] + c[k + h]) + e;
            }
        }
        S[u] = s[0];
        Cc[u] = c[0];
        row_chunk_fence();
    }
#pragma unroll
    for (int h = NCH / 2; h > 0; h >>= 1) {
#pragma unroll
        for (int k = 0; k < h; ++k) {
            float sk, e;
            two_sum(S[k], S[k + h], sk, e);
            S[k] = sk;
            Cc[k] = (Cc[k] + Cc[k + h]) + e;
        }
    }
    float vs = S[0], vc = Cc[0];
#pragma unroll
    for (int o = CPW; o <= 16; o <<= 1) {
        const float ws = __shfl_xor_sync(0xffffffffu, vs, o);
        const float wc = __shfl_xor_sync(0xffffffffu, vc, o);
        float sn, e;
        two_sum(vs, ws, sn, e);
        vs = sn;
        vc = (vc + wc) + e;
    }
    return vs + vc;
}

// Plain pairwise sum over the thread's MR rows of Re conj(a_m) b_m (chunks as
// in col_sum2), the lanes of the column combined commutatively: for the light
// correction solves, whose 1e-2 tolerance leaves FP32 rounding of the
// denominator far behind
template <int MR, typename F>
__device__ __forceinline__ float col_sum_plain(F f) {
    constexpr int CH = 8, NCH = MR / CH;
    float S[NCH];
#pragma unroll
    for (int u = 0; u < NCH; ++u) {
        float2 a[CH], b[CH];
        f(u, a, b);
        float s[CH];
#pragma unroll
        for (int k = 0; k < CH; ++k) s[k] = fmaf(a[k].x, b[k].x, a[k].y * b[k].y);
#pragma unroll
        for (int h = CH / 2; h > 0; h >>= 1)
#pragma unroll
            for (int k = 0; k < h; ++k) s[k] += s[k + h];
        S[u] = s[0];
        row_chunk_fence();
    }
#pragma unroll
    for (int h = NCH / 2; h > 0; h >>= 1)
#pragma unroll
        for (int k = 0; k < h; ++k) S[k] += S[k + h];
    float v = S[0];
#pragma unroll
    for (int o = CPW; o <= 16; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// MODE 0 solves A X = B from X0 (or 0); MODE 1 is a refinement correction
// solve (right-hand side R, X += dX; instances that stopped refining are
// skipped); MODE 2 is the same with the heads of A and P only (FP16, 11 bits:
// A off by 2^-12 of its entries, the correction's solution by about kappa
// 2^-12, far inside the loose tolerance such solves run to -- the host asks
// for it only when refine_solve_tol >= 5e-3): half the bytes streamed, two
// MMAs per k-step instead of four.  jobs: (instance, first column), NB
// columns each.
template <int KC, int VAR, int MODE>
__global__ void __launch_bounds__(THREADS, CTAS_PER_SM) pcg_tcw_kernel(const DevInst *__restrict__ insts,
                                                             const int2 *__restrict__ jobs, int n_jobs,
                                                             DevAccum acc_out) {
    using C = Cfg<KC>;
    constexpr int MR = C::MR;
    extern __shared__ __align__(1024) unsigned char smem[];
    // per row i: rowc = {d'_i = 2^(2 e_i) d_i, 2^(2 e_i)} (d_i the Jacobi factor
    // 1 / A_ii, or 1 for plain CG), rowe = {2^e_i, 2^-e_i}
    float *rowc = reinterpret_cast<float *>(smem + C::TAB_OFF);
    float *rowe = rowc + 2 * KC;
    float *colq = rowe + 2 * KC;   // per column 2^-SA / s_j: the readout's unscaling
    Ctl &S = *reinterpret_cast<Ctl *>(smem + C::TAB_OFF + 4 * KC * 4 + NB * 4);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int i = 0; i < RING; ++i) {
            tc::mbar_init(&S.full[i], 1);
            tc::mbar_init(&S.empty[i], 1);
        }
        tc::mbar_init(&S.qfull, 1);
        S.err = 0;
        tc::mbar_init_fence();
    }
    if (warp == 0) {
        tc::tmem_alloc(&S.tmem, C::TMEM_COLS);
        tc::tmem_relinquish();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = S.tmem;
    const uint32_t b_base = tc::smem_u32(smem), r_base = b_base + C::B_BYTES;
    // One iteration's A x P: thread 0 streams the KC / 128 x KC / 16 stages into
    // the ring, one group of SUB k-steps per bulk copy (a light correction: the
    // heads of two groups, two copies); thread 32 issues their MMAs (per k-step:
    // head x [P_h | P_t] and tail x P_h, Ar then Ai) and commits to qfull; the
    // other threads go on to wait.
    constexpr bool LIGHT = MODE == 2;
    constexpr int KPS = LIGHT ? 2 * SUB : SUB;       // k-steps per ring slot (heads: 8 KB each)
    auto first_kstep = [&](int s) {   // slot s -> (row tile, k-step of its first stage)
        const int g0 = s * KPS;
        return make_int2(g0 / C::KS, g0 % C::KS);
    };
    // Group s of an iteration goes to ring slot s mod 2, so that slot 0 can take
    // the next iteration's first group while the epilogue stages its readout in
    // slot 1.  fills[k] counts the fills of slot k (thread 0: issued; thread 32:
    // consumed), which gives the parity of each wait.
    // With A resident (C::RES) the job's first product fills the slots once and
    // later products multiply what is there.
    int fills[RING] = {0, 0};
    bool pref = false;   // group 0 (resident: all of A) of the current instance is already in the ring
    auto issue = [&](const char *src, int s) {   // thread 0: group s into slot s mod 2
        const int slot = s & 1;
        const int2 f = first_kstep(s);
        const char *st = src + (size_t)(f.x * C::KS + f.y) * STAGE;
        if (!tc::mbar_wait(&S.empty[slot], (fills[slot] & 1) ^ 1, WAIT_LIMIT)) S.err = 1;
        ++fills[slot];
        tc::mbar_arrive_expect_tx(&S.full[slot], SLOT);
        if (LIGHT) {   // the leading heads half of two groups
            bulk_load(r_base + slot * SLOT, st, SLOT / 2, &S.full[slot]);
            bulk_load(r_base + slot * SLOT + SLOT / 2, st + SLOT, SLOT / 2, &S.full[slot]);
        } else {
            bulk_load(r_base + slot * SLOT, st, SLOT, &S.full[slot]);
        }
    };
    auto product = [&](const char *src) {
        if (threadIdx.x == 0) {
            if (C::RES) {
                if (!pref)
                    for (int s = 0; s < C::NSTAGE / KPS; ++s) issue(src, s);
            } else {
                for (int s = pref ? 1 : 0; s < C::NSTAGE / KPS; ++s) issue(src, s);
                // the next iteration's first group, on the chance that the job goes
                // on: its copy then overlaps the epilogue
                issue(src, 0);
            }
        } else if (threadIdx.x == 32 && LIGHT) {
            constexpr uint32_t idN2 = tc::idesc_f16(128, 2 * NB, false);
            tc::tc_fence_after();
            for (int s = 0; s < C::NSTAGE / KPS; ++s) {
                const int slot = s & 1;
                if (!C::RES || !pref) {
                    if (!tc::mbar_wait(&S.full[slot], fills[slot] & 1, WAIT_LIMIT)) S.err = 1;
                    ++fills[slot];
                }
                tc::tc_fence_after();
                const int2 f = first_kstep(s);
#pragma unroll
                for (int u = 0; u < KPS; ++u) {
                    const int rt = f.x, ks = f.y + u;
                    const uint32_t a0 = r_base + slot * SLOT + u * (STAGE / 2);
                    const uint64_t bd = tc::smem_desc(b_base + ks * 256, 128, C::SBO_B);   // [Pr_h | Pi_h]
                    const uint32_t du = tmem + rt * 8 * NB, dvv = du + 4 * NB;
                    const uint32_t acc = ks > 0 ? 1u : 0u;
                    tc::mma_bf16(du, tc::smem_desc(a0, 128, 256), bd, idN2, acc);
                    tc::mma_bf16(dvv, tc::smem_desc(a0 + TILE, 128, 256), bd, idN2, acc);
                }
                if (!C::RES) tc::mma_commit(&S.empty[slot]);
            }
            tc::mma_commit(&S.qfull);
        } else if (threadIdx.x == 32) {
            constexpr uint32_t idN4 = tc::idesc_f16(128, 4 * NB, false);
            constexpr uint32_t idN2 = tc::idesc_f16(128, 2 * NB, false);
            tc::tc_fence_after();
            for (int s = 0; s < C::NSTAGE / SUB; ++s) {
                const int slot = s & 1;
                if (!C::RES || !pref) {
                    if (!tc::mbar_wait(&S.full[slot], fills[slot] & 1, WAIT_LIMIT)) S.err = 1;
                    ++fills[slot];
                }
                tc::tc_fence_after();
                const int2 f = first_kstep(s);
#pragma unroll
                for (int u = 0; u < SUB; ++u) {
                    const int rt = f.x, ks = f.y + u;
                    const uint32_t a0 = r_base + slot * SLOT + u * (STAGE / 2);   // [Ar_h | Ai_h]
                    const uint32_t a1 = a0 + SLOT / 2;                              // [Ar_t | Ai_t]
                    const uint64_t bd = tc::smem_desc(b_base + ks * 256, 128, C::SBO_B);
                    const uint32_t du = tmem + rt * 8 * NB, dvv = du + 4 * NB;
                    const uint32_t acc = ks > 0 ? 1u : 0u;
                    tc::mma_bf16(du, tc::smem_desc(a0, 128, 256), bd, idN4, acc);   // FP16 by the descriptors
                    tc::mma_bf16(du + 2 * NB, tc::smem_desc(a1, 128, 256), bd, idN2, 1u);
                    tc::mma_bf16(dvv, tc::smem_desc(a0 + TILE, 128, 256), bd, idN4, acc);
                    tc::mma_bf16(dvv + 2 * NB, tc::smem_desc(a1 + TILE, 128, 256), bd, idN2, 1u);
                }
                if (!C::RES) tc::mma_commit(&S.empty[slot]);   // the slot is free once these have read it
            }
            tc::mma_commit(&S.qfull);
        }
        pref = true;
        __syncwarp();
    };
    // the vote ended the job: the look-ahead group in slot 0 goes unused (resident:
    // A leaves the ring); thread 32 takes it off (its fill landed, the slot is free
    // again) and waits for the release to land before anything else may touch the
    // slot (or the CTA exit)
    auto release = [&](int k, bool landed) {
        if (!landed && !tc::mbar_wait(&S.full[k], fills[k] & 1, WAIT_LIMIT)) S.err = 1;
        if (!landed) ++fills[k];
        tc::tc_fence_after();
        tc::mma_commit(&S.empty[k]);
        if (!tc::mbar_wait(&S.empty[k], (fills[k] - 1) & 1, WAIT_LIMIT)) S.err = 1;   // phase fills - 1
    };
    auto discard = [&]() {
        if (pref && threadIdx.x == 32) {
            if (C::RES)
                for (int k = 0; k < RING && k < C::NSTAGE / KPS; ++k) release(k, true);
            else
                release(0, false);
        }
        pref = false;
        __syncwarp();
    };
    {
        // ---- epilogue: the vectors of the CTA's NB columns, column-wise ----
        // It works in the Jacobi-scaled variables of the product, E = diag(2^e_i):
        //   r' = E^-1 r,  w = E^-1 q (the readout),  u = s_j E p (P as published),
        // where the row factors cancel from every step but the update of x:
        //   p^H A p = Re u^H w / s_j,   r' -= lambda w,   x += (lambda / s_j) E^-1 u,
        //   r^H z = sum d'_i |r'_i|^2,  ||r||^2 = sum 2^(2 e_i) |r'_i|^2,  E z = d' r',
        //   E p_new = d' r' + (beta / s_j) u,      d'_i = 2^(2 e_i) d_i.
        // Every factor is a power of two, so the values are those of the unscaled
        // recurrences.
        const int cl = CPW * warp + (lane % CPW);   // local column
        const int g = lane / CPW;                    // row pairs 2 g + 2 LPC n, n < MR / 2
        const int qw = warp & 3, hh = warp >> 2;     // TMEM lane quarter and column group of the readout
        // the readout staging: ring slot 1 (slot 0 may hold the next iteration's
        // first group), or after the ring when A is resident; Re and Im planes, column c's row i at
        // (i / 128 NB + c) 128 + (i mod 128 xor 16 (c mod 2)), so that the two
        // columns of a warp's row-pair reads fall on disjoint banks
        float *Qre = reinterpret_cast<float *>(smem + C::STG_OFF);
        float *Qim = Qre + C::RT * NB * 128;
        unsigned char *Bop = smem;
        auto row = [&](int m) { return 2 * g + 2 * LPC * (m >> 1) + (m & 1); };   // the thread's row m
        // rows row(m), row(m) + 1 (m even) of B's plane pl: 0 Pr_h, 1 Pi_h, 2 Pr_t, 3 Pi_t
        auto bset2 = [&](int pl, int m, __half2 v) {
            *reinterpret_cast<__half2 *>(Bop + b_off<KC>(pl * NB + cl, row(m))) = v;
        };
        float2 r[MR];        // r' at the owned rows
        float2 u[MR];        // u at the owned rows, as published (head + tail, exact in FP32)
        float pinv = 1.f;    // 1 / s_j of the last publication
        float pmx = 0.f;     // the owned rows' largest |E p| as last published
        // the exponent ex for a column whose largest |E p| is at most mx, s_j =
        // 2^(SP - ex); clamped so that s_j, 1 / s_j and 2^-SA / s_j are floats
        auto exp_of = [&](float mx) {
            return (mx >= 1.2e-38f && mx < 3.0e38f) ? min(max(exp2_of(mx), SA + SP - 126), SP + 126) : SP;
        };
        auto col_max = [&](float mx) {   // over the column's lanes
#pragma unroll
            for (int o = CPW; o <= 16; o <<= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            return mx;
        };
        // store s_j v (v = f(m) = E p at row(m)) into B as FP16 head and tail, two
        // rows per 32-bit store, and keep u = s_j v as published
        auto publish_exp = [&](bool active, int ex, auto f) {
            if (!active) return;
            const float sj = pow2f(SP - ex);
            float mx = 0.f;
#pragma unroll
            for (int m = 0; m < MR; m += 2) {
                const float2 v0 = f(m), v1 = f(m + 1);
                mx = fmaxf(mx, fmaxf(fmaxf(fabsf(v0.x), fabsf(v0.y)), fmaxf(fabsf(v1.x), fabsf(v1.y))));
                const float ar = v0.x * sj, br = v1.x * sj, ai = v0.y * sj, bi = v1.y * sj;
                const __half2 hr = __floats2half2_rn(ar, br), hi = __floats2half2_rn(ai, bi);
                const float2 fr = __half22float2(hr), fi = __half22float2(hi);
                bset2(0, m, hr);
                bset2(1, m, hi);
                if (LIGHT) {   // a light correction uses the heads only
                    u[m] = make_float2(fr.x, fi.x);
                    u[m + 1] = make_float2(fr.y, fi.y);
                } else {
                    const __half2 tr = __floats2half2_rn(ar - fr.x, br - fr.y);
                    const __half2 ti = __floats2half2_rn(ai - fi.x, bi - fi.y);
                    const float2 gr = __half22float2(tr), gi = __half22float2(ti);
                    bset2(2, m, tr);
                    bset2(3, m, ti);
                    u[m] = make_float2(fr.x + gr.x, fi.x + gi.x);   // exact
                    u[m + 1] = make_float2(fr.y + gr.y, fi.y + gi.y);
                }
                if ((m & 7) == 6) row_chunk_fence();
            }
            pinv = pow2f(ex - SP);
            if (g == 0) colq[cl] = pow2f(ex - SP - SA);
            pmx = mx;
        };
        // a publication whose scale comes from the column's maximum (two passes
        // over f; all lanes take part)
        auto publish_all = [&](auto f) {
            float mx = 0.f;
#pragma unroll
            for (int m = 0; m < MR; ++m) {
                const float2 v = f(m);
                mx = fmaxf(mx, fmaxf(fabsf(v.x), fabsf(v.y)));
            }
            publish_exp(true, exp_of(col_max(mx)), f);
        };
        // w at rows row(m), row(m) + 1 (m even): {Re, Re}, {Im, Im}
        auto wpair = [&](int m, float2 &re, float2 &im) {
            const int i = row(m);
            const int o = ((i >> 7) * NB + cl) * 128 + ((i & 127) ^ ((cl & 1) << 4));
            re = *reinterpret_cast<const float2 *>(Qre + o);
            im = *reinterpret_cast<const float2 *>(Qim + o);
        };
        // rowc of rows row(m), row(m) + 1 (m even): {d', 2^2e, d', 2^2e}
        auto rcpair = [&](int m) { return *reinterpret_cast<const float4 *>(rowc + 2 * row(m)); };
        // the new r^H z and ||r||^2 (nonnegative terms, pairwise in chunks of 8
        // rows, then the chunks pairwise) and max |E z| over the owned rows
        auto norms = [&](float &rz, float &rr, float &mz) {
            float Sz[MR / 8], Sr[MR / 8];
            mz = 0.f;
#pragma unroll
            for (int c8 = 0; c8 < MR / 8; ++c8) {
                float sz[8], sr[8];
#pragma unroll
                for (int k = 0; k < 8; k += 2) {
                    const int m = 8 * c8 + k;
                    const float4 rc = rcpair(m);
                    const float zx0 = rc.x * r[m].x, zy0 = rc.x * r[m].y;
                    const float zx1 = rc.z * r[m + 1].x, zy1 = rc.z * r[m + 1].y;
                    sz[k] = fmaf(r[m].x, zx0, r[m].y * zy0);
                    sz[k + 1] = fmaf(r[m + 1].x, zx1, r[m + 1].y * zy1);
                    sr[k] = fmaf(r[m].x, r[m].x, r[m].y * r[m].y) * rc.y;
                    sr[k + 1] = fmaf(r[m + 1].x, r[m + 1].x, r[m + 1].y * r[m + 1].y) * rc.w;
                    mz = fmaxf(mz, fmaxf(fmaxf(fabsf(zx0), fabsf(zy0)), fmaxf(fabsf(zx1), fabsf(zy1))));
                }
#pragma unroll
                for (int h = 4; h > 0; h >>= 1)
#pragma unroll
                    for (int k = 0; k < h; ++k) {
                        sz[k] += sz[k + h];
                        sr[k] += sr[k + h];
                    }
                Sz[c8] = sz[0];
                Sr[c8] = sr[0];
                row_chunk_fence();
            }
#pragma unroll
            for (int h = MR / 16; h > 0; h >>= 1)
#pragma unroll
                for (int k = 0; k < h; ++k) {
                    Sz[k] += Sz[k + h];
                    Sr[k] += Sr[k + h];
                }
            rz = Sz[0];
            rr = Sr[0];
        };
        uint32_t qp = 0;
        int err = 0;
        for (int jj = blockIdx.x; jj < n_jobs; jj += gridDim.x) {
            const int2 job = jobs[jj];
            const int id = job.x;
            const DevInst &in = insts[id];
            if (MODE >= 1 && in.rctl[1] != 0.f) continue;   // uniform: every role skips it
            const int K = in.K, T = in.max_iter, NCOL = in.ncols;
            const int j = job.y + cl;
            const bool valid = j < NCOL;
            const bool warm = MODE == 0 && in.X0 != nullptr;
            const float tl = (MODE >= 1 && in.rsolve_tol > 0.f) ? in.rsolve_tol : in.tol;
            const float tol2 = tl > 0.f ? tl * tl : -1.f;
            float2 *X = in.X + (size_t)(valid ? j : 0) * KC;   // the iterate (workspace, ld KC)
            // the owned rows' right-hand side (and x0, kept in u until the first
            // publication reads it): loads in flight across the table build
#pragma unroll
            for (int m = 0; m < MR; ++m) {
                const int i = row(m);
                float2 b = make_float2(0.f, 0.f), x0 = make_float2(0.f, 0.f);
                if (valid && i < K) {
                    if (MODE >= 1) b = in.R[i + (size_t)j * KC];                    // refinement residual
                    else if (!in.B) b.x = (i == j) ? 1.f : 0.f;                      // B = I
                    else b = in.B[i + (size_t)j * in.ldb];                           // symbol vectors
                    if (warm) x0 = in.X0[i + (size_t)j * K];
                }
                r[m] = b;
                u[m] = x0;
            }
            epi_sync();   // the previous instance's readers of rowc and rowe are done
            for (int i = threadIdx.x; i < KC; i += EPI) {
                const int e = row_exp(in.A[(size_t)i * (KC + 1)].x);   // as the prep kernel scaled A
                const float d = (i < K) ? (VAR == 2 ? 1.f : in.dinv[i]) : 0.f;
                rowc[2 * i] = d * pow2f(2 * e);
                rowc[2 * i + 1] = pow2f(2 * e);
                rowe[2 * i] = pow2f(e);
                rowe[2 * i + 1] = pow2f(-e);
            }
            epi_sync();
            // ---- Step 1: r' = E^-1 b, x = x0 (mode 0; a correction adds to x as it
            // stands), p = D^{-1} r ----
#pragma unroll
            for (int m = 0; m < MR; ++m) {
                const int i = row(m);
                const float is = rowe[2 * i + 1];
                r[m] = make_float2(r[m].x * is, r[m].y * is);
                // x0 as a relaxed store at GPU scope, like the reductions that follow
                // it to the same address: the same thread's strong accesses to one
                // location are ordered without a fence
                if (MODE == 0 && valid) st_relaxed2(X + i, u[m]);
            }
            // the warm pass forms A X0 first; columns beyond the right-hand sides carry 0
            publish_all([&](int m) {
                const int i = row(m);
                if (!valid) return make_float2(0.f, 0.f);
                if (warm) {
                    const float sc = rowe[2 * i];
                    return make_float2(sc * u[m].x, sc * u[m].y);   // E x0
                }
                const float dp = rowc[2 * i];
                return make_float2(dp * r[m].x, dp * r[m].y);
            });
            float rho, res2, mz0;
            norms(rho, res2, mz0);
#pragma unroll
            for (int o = CPW; o <= 16; o <<= 1) {   // the lanes of the column, commutatively
                rho += __shfl_xor_sync(0xffffffffu, rho, o);
                res2 += __shfl_xor_sync(0xffffffffu, res2, o);
            }
            const float bn2 = res2;   // stopping and reporting stay relative to ||b||
            const float btol = tol2 * bn2;
            bool done = !valid;
            int itmax = 0, notHPD = 0;
            for (int t = warm ? -1 : 0;; ++t) {
                const bool init = t < 0;
                if (!init && tol2 > 0.f && res2 <= btol) done = true;
                const int any = (init || (!done && t < T)) ? 1 : 0;
                // P and the staging reads before the async proxy, the TMEM reads
                // before the next MMAs; one decision for the whole CTA
                tc::fence_proxy_async_smem();
                tc::tc_fence_before();
                const int cont = epi_or(any && !S.err);
                if (!cont) {
                    discard();
                    break;
                }
                product(reinterpret_cast<const char *>(in.As));
                // ---- w = E^-1 A p: U, V -> Re w, Im w staging planes ----
                if (!tc::mbar_wait(&S.qfull, qp & 1, WAIT_LIMIT)) {
                    err = 1;
                    S.err = 1;
                }
                ++qp;
                __syncwarp();   // the TMEM loads below are warp-collective
                tc::tc_fence_after();
                float cq[RCOLS];   // the readout's per-column unscaling 2^-SA / s_j
#pragma unroll
                for (int e = 0; e < RCOLS; ++e) cq[e] = colq[RCOLS * hh + e];
#pragma unroll
                for (int rt = 0; rt < C::RT; ++rt) {
                    const uint32_t tb = tmem + ((uint32_t)(32 * qw) << 16) + (uint32_t)(rt * 8 * NB + RCOLS * hh);
                    const int o = (rt * NB + RCOLS * hh) * 128;   // + column * 128 + row, swizzled
                    const int rl = 32 * qw + lane;
                    // Re w = (Ar Pr - Ai Pi) and Im w = (Ai Pr + Ar Pi) from U's and V's
                    // head products and corrections (a light correction has no
                    // corrections), 8 columns at a time
#pragma unroll
                    for (int h8 = 0; h8 < RCOLS; h8 += 8) {
                        float x[8], y[8], z[8];
                        if (LIGHT) {
                            tc::tmem_ld8(tb + h8, x);
                            tc::tmem_ld8(tb + 4 * NB + NB + h8, y);
                            tc::tmem_ld_wait();
#pragma unroll
                            for (int e = 0; e < 8; ++e) Qre[o + (h8 + e) * 128 + (rl ^ ((e & 1) << 4))] = (x[e] - y[e]) * cq[h8 + e];
                            tc::tmem_ld8(tb + 4 * NB + h8, x);
                            tc::tmem_ld8(tb + NB + h8, y);
                            tc::tmem_ld_wait();
#pragma unroll
                            for (int e = 0; e < 8; ++e) Qim[o + (h8 + e) * 128 + (rl ^ ((e & 1) << 4))] = (x[e] + y[e]) * cq[h8 + e];
                            continue;
                        }
                        tc::tmem_ld8(tb + h8, x);
                        tc::tmem_ld8(tb + 2 * NB + h8, y);
                        tc::tmem_ld_wait();
#pragma unroll
                        for (int e = 0; e < 8; ++e) x[e] += y[e];
                        tc::tmem_ld8(tb + 4 * NB + NB + h8, y);
                        tc::tmem_ld8(tb + 4 * NB + 3 * NB + h8, z);
                        tc::tmem_ld_wait();
#pragma unroll
                        for (int e = 0; e < 8; ++e) Qre[o + (h8 + e) * 128 + (rl ^ ((e & 1) << 4))] = (x[e] - (y[e] + z[e])) * cq[h8 + e];
                        tc::tmem_ld8(tb + 4 * NB + h8, x);
                        tc::tmem_ld8(tb + 4 * NB + 2 * NB + h8, y);
                        tc::tmem_ld_wait();
#pragma unroll
                        for (int e = 0; e < 8; ++e) x[e] += y[e];
                        tc::tmem_ld8(tb + NB + h8, y);
                        tc::tmem_ld8(tb + 3 * NB + h8, z);
                        tc::tmem_ld_wait();
#pragma unroll
                        for (int e = 0; e < 8; ++e) Qim[o + (h8 + e) * 128 + (rl ^ ((e & 1) << 4))] = (x[e] + (y[e] + z[e])) * cq[h8 + e];
                    }
                }
                epi_sync();
                if (init) {   // r = b - A X0, then Step 1 from there
#pragma unroll
                    for (int m = 0; m < MR; m += 2) {
                        float2 re, im;
                        wpair(m, re, im);
                        r[m] = make_float2(r[m].x - re.x, r[m].y - im.x);
                        r[m + 1] = make_float2(r[m + 1].x - re.y, r[m + 1].y - im.y);
                    }
                    publish_all([&](int m) {
                        const float dp = rowc[2 * row(m)];
                        return make_float2(dp * r[m].x, dp * r[m].y);
                    });
                    float mzi;
                    norms(rho, res2, mzi);
#pragma unroll
                    for (int o = CPW; o <= 16; o <<= 1) {
                        rho += __shfl_xor_sync(0xffffffffu, rho, o);
                        res2 += __shfl_xor_sync(0xffffffffu, res2, o);
                    }
                    continue;
                }
                // ---- Steps 2-4: lambda = r^H z / p^H A p, x += lambda p, r -= lambda q ----
                auto wchunk = [&](int c8, float2(&a)[8], float2(&b)[8]) {
#pragma unroll
                    for (int k = 0; k < 8; k += 2) {
                        const int m = 8 * c8 + k;
                        float2 re, im;
                        wpair(m, re, im);
                        a[k] = u[m];
                        a[k + 1] = u[m + 1];
                        b[k] = make_float2(re.x, im.x);
                        b[k + 1] = make_float2(re.y, im.y);
                    }
                };
                // p^H A p: compensated in the solve, plain in a light correction
                const float pAp = pinv * (LIGHT ? col_sum_plain<MR>(wchunk) : col_sum2<MR>(wchunk));
                float lam = 0.f;
                if (pAp > 0.f) lam = rho / pAp;
                else if (res2 != 0.f && !done) notHPD = 1;
                if (done) lam = 0.f;
                // x += lambda p = (lambda / s_j) E^-1 u as reductions into the
                // workspace, two rows each, which this thread does not wait for (it
                // reads X again only after a fence)
                if (!done) {
                    const float lp = lam * pinv;
                    red_pairs<0, MR / 2, 2 * LPC>(X + 2 * g, [&](int n) {
                        const float4 ee = *reinterpret_cast<const float4 *>(rowe + 2 * row(2 * n));
                        const float a0 = lp * ee.y, a1 = lp * ee.w;   // times 2^-e of the two rows
                        return make_float4(a0 * u[2 * n].x, a0 * u[2 * n].y, a1 * u[2 * n + 1].x, a1 * u[2 * n + 1].y);
                    });
                }
                // r' -= lambda w
#pragma unroll
                for (int m = 0; m < MR; m += 2) {
                    float2 re, im;
                    wpair(m, re, im);
                    r[m].x = fmaf(-lam, re.x, r[m].x);
                    r[m].y = fmaf(-lam, im.x, r[m].y);
                    r[m + 1].x = fmaf(-lam, re.y, r[m + 1].x);
                    r[m + 1].y = fmaf(-lam, im.y, r[m + 1].y);
                    if ((m & 7) == 6) row_chunk_fence();
                }
                float rz_new, rr_new, mz;
                norms(rz_new, rr_new, mz);
                // the lanes of the column: the sums commutatively, with the maxima
                // of |E z| and of the last published |E p| in the same independent
                // shuffle rounds
                float pm = pmx;
#pragma unroll
                for (int o = CPW; o <= 16; o <<= 1) {
                    rz_new += __shfl_xor_sync(0xffffffffu, rz_new, o);
                    rr_new += __shfl_xor_sync(0xffffffffu, rr_new, o);
                    mz = fmaxf(mz, __shfl_xor_sync(0xffffffffu, mz, o));
                    pm = fmaxf(pm, __shfl_xor_sync(0xffffffffu, pm, o));
                }
                // p = z + beta p, published for the next product, its scale from the
                // bound max |E p| <= max |E z| + beta max |E p_old| (< 2^(pex + 1), pex
                // the exponent of the maximum of what was published, so bounds do not
                // compound): one pass over the rows instead of two
                const float beta = (!done && rho != 0.f) ? rz_new / rho : 0.f;
                const int pex = exp_of(pm);
                const int exn = exp_of(fmaf(beta, pow2f(min(pex + 1, 127)), mz));
                const float bp = beta * pinv;
                publish_exp(!done, exn, [&](int m) {
                    const float dp = rowc[2 * row(m)];
                    return make_float2(fmaf(bp, u[m].x, dp * r[m].x), fmaf(bp, u[m].y, dp * r[m].y));
                });
                if (!done) {
                    rho = rz_new;
                    res2 = rr_new;
                    itmax = t + 1;
                }
            }
            // ---- outputs ----
            if (valid && in.Xout) {
                __threadfence();   // this thread's reductions into X are performed
#pragma unroll
                for (int m = 0; m < MR; ++m) {
                    const int i = row(m);
                    if (i < K) in.Xout[i + (size_t)j * K] = __ldcg(X + i);   // from L2, where they landed
                }
            }
            if (MODE == 0 && g == 0) {   // one thread per column
                int f = (err || S.err) ? FLAG_TIMEOUT : 0;
                if (valid) {
                    if (itmax > 0) atomicMax(acc_out.iters + id, itmax);
                    const float rr = fmaxf(res2, 0.f);
                    const float res = sqrtf(bn2 > 0.f ? rr / bn2 : rr);   // relative to ||b||
                    if (res > 0.f) atomicMax(acc_out.resid_bits + id, __float_as_uint(res));
                    if (notHPD) f |= FLAG_NOTHPD;
                    if (tol2 > 0.f && !(res2 <= btol)) f |= FLAG_NOTCONV;
                }
                if (f) atomicOr(acc_out.flags + id, f);
            }
        }
    }
    // the copies issued last have landed before the CTA may exit
    if (threadIdx.x == 0)
        for (int k = 0; k < RING; ++k)
            if (fills[k] > 0) (void)tc::mbar_wait(&S.full[k], (fills[k] - 1) & 1, WAIT_LIMIT);
    // every MMA has completed (each qfull was waited for) and every copy landed
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    if (warp == 0) tc::tmem_dealloc(tmem, C::TMEM_COLS);
}

int sm_count() {
    static int n = 0;
    if (!n) {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
            n = v;
        else
            n = 148;
    }
    return n;
}

template <int KC, int VAR, int MODE>
cudaError_t launch_main(const DevInst *insts, const int2 *jobs, int n, DevAccum acc, cudaStream_t s) {
    auto kern = pcg_tcw_kernel<KC, VAR, MODE>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg<KC>::SMEM);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    const int grid = CTAS_PER_SM * sm_count();
    kern<<<n < grid ? n : grid, THREADS, Cfg<KC>::SMEM, s>>>(insts, jobs, n, acc);
    return cudaGetLastError();
}

template <int KC>
cudaError_t launch_kc(int variant, const DevInst *insts, const int2 *jobs, int n, DevAccum acc, cudaStream_t s,
                      int mode) {
    if (variant == 0)
        return mode == 2 ? launch_main<KC, 0, 2>(insts, jobs, n, acc, s)
               : mode    ? launch_main<KC, 0, 1>(insts, jobs, n, acc, s)
                         : launch_main<KC, 0, 0>(insts, jobs, n, acc, s);
    if (variant == 2)
        return mode == 2 ? launch_main<KC, 2, 2>(insts, jobs, n, acc, s)
               : mode    ? launch_main<KC, 2, 1>(insts, jobs, n, acc, s)
                         : launch_main<KC, 2, 0>(insts, jobs, n, acc, s);
    return cudaErrorInvalidValue;
}

}  // namespace

int pcg_tcw_cols() { return NB; }

cudaError_t launch_tcw_prep(int KC, const DevInst *insts, const int *list, int n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    if (KC == 128) tcw_prep_kernel<128><<<n * Cfg<128>::NSTAGE, 256, 0, s>>>(insts, list);
    else if (KC == 256) tcw_prep_kernel<256><<<n * Cfg<256>::NSTAGE, 256, 0, s>>>(insts, list);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_pcg_tcw(int KC, int variant, const DevInst *insts, const int2 *jobs, int n, DevAccum acc,
                           cudaStream_t s, int mode) {
    if (n <= 0) return cudaSuccess;
    if (KC == 128) return launch_kc<128>(variant, insts, jobs, n, acc, s, mode);
    if (KC == 256) return launch_kc<256>(variant, insts, jobs, n, acc, s, mode);
    return cudaErrorInvalidValue;
}

}  // namespace jacpcg


