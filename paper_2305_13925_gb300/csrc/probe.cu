// probe.cu -- a measurement kernel for the FP32 roof the SIMT kernels are
// reported against: every thread runs 8 independent FMA chains (enough
// independent work to keep the FMA pipes issuing every cycle), and the
// caller times the launch with CUDA events.  Flops per launch =
// blocks * 256 threads * iters * 8 chains * 2.  The result is written so
// the chains are not optimised away.
#include <cuda_runtime.h>

#include "../../include/jacpcg.h"

namespace {

__global__ void __launch_bounds__(256) ffma_probe(int iters, float *out) {
    float a0 = threadIdx.x * 1e-7f, a1 = a0 + 1e-3f, a2 = a0 + 2e-3f, a3 = a0 + 3e-3f;
    float a4 = a0 + 4e-3f, a5 = a0 + 5e-3f, a6 = a0 + 6e-3f, a7 = a0 + 7e-3f;
    const float m = 0.999999f, c = 1e-7f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll 16
        for (int u = 0; u < 16; ++u) {
            a0 = fmaf(a0, m, c); a1 = fmaf(a1, m, c); a2 = fmaf(a2, m, c); a3 = fmaf(a3, m, c);
            a4 = fmaf(a4, m, c); a5 = fmaf(a5, m, c); a6 = fmaf(a6, m, c); a7 = fmaf(a7, m, c);
        }
    }
    const float s = ((a0 + a1) + (a2 + a3)) + ((a4 + a5) + (a6 + a7));
    if (s == 12345.f) out[blockIdx.x] = s;   // never true; keeps the chains live
}

}  // namespace

extern "C" jacpcg_status jacpcg_probe_fp32_fma(int blocks, int iters, float *scratch_dev, void *stream,
                                               double *flops) {
    if (blocks < 1 || iters < 1 || !scratch_dev) return JACPCG_EINVAL;
    ffma_probe<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(iters, scratch_dev);
    if (cudaGetLastError() != cudaSuccess) return JACPCG_ECUDA;
    if (flops) *flops = (double)blocks * 256.0 * (double)iters * 16.0 * 8.0 * 2.0;
    return JACPCG_OK;
}
