// plain.cu -- the plain FP32 per-instance Jac-PCG precoder: the comparator
// the batched path is measured against.  Same mathematics as the batched
// path (Sec. II after Eq. 7; Sec. III-B Steps 1-4, Eqs. 19-21; Algorithm 1;
// Eq. 7 / Eq. 15), written the simple way: one instance at a time, one
// thread per output entry, one launch per step and per iteration (Gram,
// init, T x (A P, column update), W = H X, finalise), plain FP32 sums and
// tree reductions, no batching, no CUDA graphs, no tensor cores.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "../../include/jacpcg.h"

namespace {

// A = H^H H + xi I (K x K, ld K) and 1 / diag; one thread per entry.
__global__ void plain_gram(const float2 *__restrict__ H, int M, int K, int ldh, float xi,
                           float2 *__restrict__ A, float *__restrict__ dinv) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= K * K) return;
    const int i = e % K, j = e / K;
    float re = 0.f, im = 0.f;
    for (int m = 0; m < M; ++m) {
        const float2 a = H[m + (size_t)i * ldh], b = H[m + (size_t)j * ldh];
        re += a.x * b.x + a.y * b.y;
        im += a.x * b.y - a.y * b.x;
    }
    if (i == j) {
        re += xi;
        im = 0.f;
        dinv[i] = 1.0f / re;
    }
    A[i + (size_t)j * K] = make_float2(re, im);
}

// Column j of B = I: x = 0, r = e_j (Alg. 1: D^{-1} e_j), p = D^{-1} r (Alg. 1: r).
__global__ void plain_init(int K, int variant, const float *__restrict__ dinv, float2 *X, float2 *R,
                           float2 *P, float *rho, float *res2, int *its) {
    const int j = blockIdx.x, i = threadIdx.x;
    const float d = (variant == JACPCG_CG) ? 1.f : dinv[i];
    const float b = (i == j) ? 1.f : 0.f;
    X[i + (size_t)j * K] = make_float2(0.f, 0.f);
    const float r = (variant == JACPCG_ALG1) ? d * b : b;
    R[i + (size_t)j * K] = make_float2(r, 0.f);
    P[i + (size_t)j * K] = make_float2(d * b, 0.f);
    if (i == 0) {
        const float dj = (variant == JACPCG_CG) ? 1.f : dinv[j];
        rho[j] = (variant == JACPCG_ALG1) ? dj * dj : dj;
        res2[j] = 1.f;
        its[j] = 0;
    }
}

// Q = A P, one thread per entry.
__global__ void plain_matvec(int K, const float2 *__restrict__ A, const float2 *__restrict__ P,
                             float2 *__restrict__ Q) {
    const int j = blockIdx.x, i = threadIdx.x;
    float re = 0.f, im = 0.f;
    for (int k = 0; k < K; ++k) {
        const float2 a = A[i + (size_t)k * K], p = P[k + (size_t)j * K];
        re += a.x * p.x - a.y * p.y;
        im += a.x * p.y + a.y * p.x;
    }
    Q[i + (size_t)j * K] = make_float2(re, im);
}

__device__ float block_sum(float v, float *red) {
    red[threadIdx.x] = v;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    const float s = red[0];
    __syncthreads();
    return s;
}

// One iteration's scalars and vector updates for column j: block j, a power
// of two >= K threads (threads beyond K hold zeros in the reductions).
__global__ void plain_update(int K, int variant, float tol2, const float *__restrict__ dinv,
                             const float2 *__restrict__ Q, float2 *X, float2 *R, float2 *P, float *rho,
                             float *res2, int *its, int *flags) {
    extern __shared__ float red[];
    const int j = blockIdx.x, i = threadIdx.x;
    const bool act = i < K;
    const size_t o = i + (size_t)j * K;
    if (tol2 > 0.f && res2[j] <= tol2) return;   // column already converged (uniform per block)
    const float d = !act ? 0.f : (variant == JACPCG_CG ? 1.f : dinv[i]);
    const float2 zero = make_float2(0.f, 0.f);
    float2 x = act ? X[o] : zero, r = act ? R[o] : zero, p = act ? P[o] : zero, q = act ? Q[o] : zero;
    const float rh = rho[j];
    if (variant == JACPCG_ALG1) {
        q = make_float2(d * q.x, d * q.y);                       // u = D^{-1} A m
        const float dr = block_sum(p.x * q.x + p.y * q.y, red);  // m^H u
        const float di = block_sum(p.x * q.y - p.y * q.x, red);
        const float den = dr * dr + di * di;
        float ar = 0.f, ai = 0.f;
        if (den > 0.f) {
            ar = rh * dr / den;
            ai = -rh * di / den;
        } else if (rh != 0.f && i == 0) {
            atomicOr(flags, 1);
        }
        x = make_float2(x.x + ar * p.x - ai * p.y, x.y + ar * p.y + ai * p.x);
        r = make_float2(r.x - (ar * q.x - ai * q.y), r.y - (ar * q.y + ai * q.x));
        const float rr = block_sum(r.x * r.x + r.y * r.y, red);
        const float e = act ? 1.0f / d : 0.f;
        const float dres = block_sum(e * e * (r.x * r.x + r.y * r.y), red);
        const float bt = rh != 0.f ? rr / rh : 0.f;
        p = make_float2(r.x + bt * p.x, r.y + bt * p.y);
        if (i == 0) {
            rho[j] = rr;
            res2[j] = dres;
        }
    } else {
        const float pAp = block_sum(p.x * q.x + p.y * q.y, red);
        float lam = 0.f;
        if (pAp > 0.f) lam = rh / pAp;
        else if (res2[j] != 0.f && i == 0) atomicOr(flags, 1);
        x = make_float2(x.x + lam * p.x, x.y + lam * p.y);
        r = make_float2(r.x - lam * q.x, r.y - lam * q.y);
        const float2 z = make_float2(d * r.x, d * r.y);
        const float rz = block_sum(r.x * z.x + r.y * z.y, red);
        const float rr = block_sum(r.x * r.x + r.y * r.y, red);
        const float beta = rh != 0.f ? rz / rh : 0.f;
        p = make_float2(z.x + beta * p.x, z.y + beta * p.y);
        if (i == 0) {
            rho[j] = rz;
            res2[j] = rr;
        }
    }
    if (act) {
        X[o] = x;
        R[o] = r;
        P[o] = p;
    }
    if (i == 0) its[j] += 1;
}

// W = H X, one thread per entry.
__global__ void plain_hx(const float2 *__restrict__ H, int M, int K, int ldh,
                         const float2 *__restrict__ X, float2 *__restrict__ W, int ldw) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (size_t)M * K) return;
    const int m = (int)(e % M), j = (int)(e / M);
    float re = 0.f, im = 0.f;
    for (int k = 0; k < K; ++k) {
        const float2 h = H[m + (size_t)k * ldh], x = X[k + (size_t)j * K];
        re += h.x * x.x - h.y * x.y;
        im += h.x * x.y + h.y * x.x;
    }
    W[m + (size_t)j * ldw] = make_float2(re, im);
}

// ||W||_F^2 -> beta, status, iterations, residual (one block).
__global__ void plain_finalize(const float2 *__restrict__ W, int M, int K, int ldw, float power,
                               float tol2, const float *res2, const int *its, const int *flags, int idx,
                               int32_t *status, int32_t *iters, float *resid, float *beta) {
    extern __shared__ float red[];
    float s = 0.f;
    for (size_t e = threadIdx.x; e < (size_t)M * K; e += blockDim.x) {
        const float2 w = W[e % M + (e / M) * (size_t)ldw];
        s += w.x * w.x + w.y * w.y;
    }
    s = block_sum(s, red);
    int itmax = 0;
    float rmax = 0.f;
    bool notconv = false;
    for (int j = 0; j < K; ++j) {
        itmax = max(itmax, its[j]);
        rmax = fmaxf(rmax, sqrtf(fmaxf(res2[j], 0.f)));
        if (tol2 > 0.f && !(res2[j] <= tol2)) notconv = true;
    }
    if (threadIdx.x != 0) return;
    int st = JACPCG_OK;
    if (!isfinite(s)) st = JACPCG_ENONFINITE;
    else if (*flags) st = JACPCG_ENOTHPD;
    else if (notconv) st = JACPCG_ENOTCONV;
    if (status) status[idx] = st;
    if (iters) iters[idx] = itmax;
    if (resid) resid[idx] = rmax;
    if (beta) beta[idx] = (s > 0.f && isfinite(s)) ? sqrtf(power / s) : 0.f;
}

}  // namespace

extern "C" jacpcg_status jacpcg_precode_plain(const jacpcg_instance *inst, int n_inst, int variant,
                                              void *workspace, size_t workspace_bytes,
                                              int32_t *status_dev, int32_t *iters_dev,
                                              float *resid_dev, float *beta_dev, void *stream) {
    if (!inst || n_inst < 1 || variant < JACPCG_STANDARD || variant > JACPCG_CG || !workspace)
        return JACPCG_EINVAL;
    int maxK = 0;
    for (int i = 0; i < n_inst; ++i) {
        const jacpcg_instance &q = inst[i];
        if (q.K < 1 || q.K > 256 || q.M < 1 || q.ldh < q.M || q.ldw < q.M || !q.H || !q.W)
            return JACPCG_EINVAL;
        if (!std::isfinite(q.xi) || q.xi < 0.0 || (q.K > q.M && !(q.xi > 0.0))) return JACPCG_EINVAL;
        if (q.max_iter < 0 || q.max_iter > 4096 || !std::isfinite(q.tol)) return JACPCG_EINVAL;
        if (q.h_dtype != JACPCG_H_C64) return JACPCG_EINVAL;   // complex64 H only
        if (q.B || q.X0 || q.sinr) return JACPCG_EINVAL;      // B = I, zero start only, no SINR
        if (q.K > maxK) maxK = q.K;
    }
    // workspace: A, X, R, P, Q (K x K complex), dinv, rho, res2 (K floats), its (K ints), flags
    const size_t kk = (size_t)maxK * maxK * sizeof(float2);
    const size_t need = 5 * kk + 4 * (size_t)maxK * 4 + 256;
    if (workspace_bytes < need) return JACPCG_ENOMEM;
    char *w = static_cast<char *>(workspace);
    float2 *A = reinterpret_cast<float2 *>(w);
    float2 *X = reinterpret_cast<float2 *>(w + kk);
    float2 *R = reinterpret_cast<float2 *>(w + 2 * kk);
    float2 *P = reinterpret_cast<float2 *>(w + 3 * kk);
    float2 *Q = reinterpret_cast<float2 *>(w + 4 * kk);
    float *dinv = reinterpret_cast<float *>(w + 5 * kk);
    float *rho = dinv + maxK;
    float *res2 = rho + maxK;
    int *its = reinterpret_cast<int *>(res2 + maxK);
    int *flags = its + maxK;
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    for (int n = 0; n < n_inst; ++n) {
        const jacpcg_instance &q = inst[n];
        const int K = q.K, M = q.M;
        const float2 *H = static_cast<const float2 *>(q.H);
        float2 *W = static_cast<float2 *>(q.W);
        const float tol2 = q.tol > 0.f ? q.tol * q.tol : -1.f;
        if (cudaMemsetAsync(flags, 0, sizeof(int), s) != cudaSuccess) return JACPCG_ECUDA;
        plain_gram<<<(K * K + 255) / 256, 256, 0, s>>>(H, M, K, q.ldh, (float)q.xi, A, dinv);
        plain_init<<<K, K, 0, s>>>(K, variant, dinv, X, R, P, rho, res2, its);
        const int threads = K;
        int pow2 = 1;
        while (pow2 < threads) pow2 <<= 1;
        for (int t = 0; t < q.max_iter; ++t) {
            plain_matvec<<<K, K, 0, s>>>(K, A, P, Q);
            plain_update<<<K, pow2, pow2 * sizeof(float), s>>>(K, variant, tol2, dinv, Q, X, R, P, rho,
                                                              res2, its, flags);
        }
        if (q.X && cudaMemcpyAsync(q.X, X, (size_t)K * K * sizeof(float2), cudaMemcpyDeviceToDevice,
                                   s) != cudaSuccess)
            return JACPCG_ECUDA;
        plain_hx<<<(unsigned)(((size_t)M * K + 255) / 256), 256, 0, s>>>(H, M, K, q.ldh, X, W, q.ldw);
        plain_finalize<<<1, 256, 256 * sizeof(float), s>>>(W, M, K, q.ldw,
                                                          q.power > 0.0 ? (float)q.power : 1.f, tol2,
                                                          res2, its, flags, n, status_dev, iters_dev,
                                                          resid_dev, beta_dev);
        if (cudaGetLastError() != cudaSuccess) return JACPCG_ECUDA;
    }
    return JACPCG_OK;
}
