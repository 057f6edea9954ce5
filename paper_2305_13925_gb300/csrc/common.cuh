// common.cuh -- device-side data structures and helpers shared by the kernels
// of the Jac-PCG RZF precoder (arXiv 2305.13925).  Host code in api.cu builds
// the tables declared here; every kernel reads them.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace jacpcg {

// Per-instance flags accumulated by the kernels, turned into a status by the
// finalise kernel.
enum : int32_t { FLAG_NOTHPD = 1, FLAG_NOTCONV = 2, FLAG_TIMEOUT = 4 };

// One precoder instance as the kernels see it.  Workspace matrices (A, X)
// are KC x KC with leading dimension KC, where KC is the instance's K class
// (the next of 8, 16, 32, 64, 128, 256 at or above K); rows and columns
// from K to KC are zero.
struct DevInst {
    const float2 *H;      // M x K, leading dimension ldh (caller)
    float2 *W;            // M x ncols, leading dimension ldw (caller)
    float2 *Xout;         // optional K x ncols, ld K (caller)
    float2 *Aout;         // optional K x K, ld K (caller)
    float2 *A;            // workspace KC x KC: H^H H + xi I
    float *dinv;          // workspace KC: 1 / A_kk (0 beyond K)
    float2 *X;            // workspace KC x KC: the iterate
    float *wpart;         // workspace: one partial ||W||_F^2 per W = H X tile
    int M, K, ldh, ldw;
    int KC;               // K class
    int max_iter;
    int n_wpart;          // number of W = H X tiles of this instance
    int variant;          // JACPCG_STANDARD / ALG1 / CG / JOR
    float omega;          // JOR relaxation factor
    float xi, power, tol;
    int h_bf16;           // H holds bfloat16 (re, im) pairs instead of complex64
    float2 *R;            // workspace KC x KC: refinement residual I - A X (null without refinement)
    float *rnorm;         // workspace 2 KC: per-column ||R_j||^2 of the last residual, then ||B_j||^2
    float *rctl;          // workspace 2: largest column ||R_j||^2 / ||B_j||^2 at the last
                          // evaluation, and 1 once the instance has stopped refining
    float rtol2;          // refine_tol^2 (0: every sweep runs)
    float rsolve_tol;     // tolerance of the correction solves (0: tol)
    int no_refine;        // refinement is on but skips this instance (selective policy)
    float *resid_hist;    // caller's optional refinement history
    // right-hand sides (Eq. 16 per symbol vector): B == null means B = I_K
    const float2 *B;      // K x ncols, leading dimension ldb (caller)
    const float2 *X0;     // optional initial point, K x ncols, ld K (caller)
    int ldb;
    int ncols;            // right-hand sides: K for B = I, else n_rhs (<= KC)
    float *As;            // workspace: A as the streamed FP16 stages of the K = 128 and 256
                          // tensor-core iteration (null when that iteration is not used)
    float *sinr;          // optional per-user SINR out, K floats (caller); B = I only
    float noise;          // noise power sigma^2 of the SINR (0: 1)
    void *Asl;            // workspace: A's 8-bit slices as FP16 stages for the sliced tensor-core
                          // residual of the 128 and 256 classes (null when not used)
    float *rexp;          // workspace 2 KC: per row the slices' output exponent, then the
                          // balancing exponent e_i (2^e_i <= sqrt(A_ii) < 2^(e_i + 1))
};

// One entry of H as complex FP32 (bfloat16 converts exactly).
__device__ __forceinline__ float2 bf16x2_to_float2(uint32_t u) {
    return make_float2(__uint_as_float(u << 16), __uint_as_float(u & 0xFFFF0000u));
}
__device__ __forceinline__ float2 load_h(const float2 *H, bool bf16, size_t idx) {
    if (bf16) return bf16x2_to_float2(__ldg(reinterpret_cast<const uint32_t *>(H) + idx));
    return __ldg(H + idx);
}

// Per-instance results written by the kernels before finalisation.
struct DevAccum {
    int32_t *flags;       // FLAG_* bits
    int32_t *iters;       // largest per-column iteration count
    uint32_t *resid_bits; // largest per-column relative residual, float bits (>= 0)
};

// Caller-visible per-instance outputs (any may be null).
struct DevOut {
    int32_t *status;
    int32_t *iters;
    float *resid;
    float *beta;
};

// ---------------------------------------------------------------------------
// complex helpers (float2 = re, im)
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// acc += a * b
__device__ __forceinline__ void cfma(float2 &acc, float2 a, float2 b) {
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(a.y, b.x, acc.y);
}
// acc += conj(a) * b
__device__ __forceinline__ void cfma_conj(float2 &acc, float2 a, float2 b) {
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(-a.y, b.x, acc.y);
}

// ---------------------------------------------------------------------------
// Compensated summation (error-free transformations; Ogita, Rump and Oishi,
// "Accurate sum and dot product", SIAM J. Sci. Comput. 26(6), 2005).
// A value is carried as (s, c): the rounded sum and its accumulated error.
struct Comp {
    float s, c;
};
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    float z = s - a;
    e = (a - (s - z)) + (b - z);
}
// (s, c) += a * b exactly up to the final rounding of c (Dot2 step)
__device__ __forceinline__ void comp_fma(Comp &v, float a, float b) {
    float p = a * b;
    float pe = fmaf(a, b, -p);
    float s, e;
    two_sum(v.s, p, s, e);
    v.s = s;
    v.c += pe + e;
}
// warp-wide all-reduce of a compensated value (fixed xor butterfly order).
// Partners combine as (s_a + s_b, (c_a + c_b) + e): each operation is
// commutative or exact, so every lane ends with bit-identical totals and
// decisions taken on them (stopping tests) are warp-uniform.
__device__ __forceinline__ Comp comp_warp_allreduce(Comp v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float ws = __shfl_xor_sync(0xffffffffu, v.s, o);
        const float wc = __shfl_xor_sync(0xffffffffu, v.c, o);
        float s, e;
        two_sum(v.s, ws, s, e);
        v.s = s;
        v.c = (v.c + wc) + e;
    }
    return v;
}
__device__ __forceinline__ float warp_allreduce_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ int warp_allreduce_max_i(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

}  // namespace jacpcg
