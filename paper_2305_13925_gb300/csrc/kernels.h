// kernels.h -- host-side launch wrappers for the device kernels (internal).
#pragma once

#include <cuda.h>   // CUtensorMap
#include <cuda_runtime.h>

#include "common.cuh"

namespace jacpcg {

// Launch shape of the iteration kernel for one K class.
struct PcgShape {
    int KC;   // K class
    int CW;   // columns per warp
    int NW;   // warps per CTA
};
// Candidate shapes per K class (8, 16, ..., 256), index 0 the default; the
// autotuner picks among them.  Each pcg_k<KC>.cu instantiates exactly these.
constexpr int PCG_MAX_SHAPES = 4;
constexpr PcgShape PCG_SHAPES[6][PCG_MAX_SHAPES] = {
    {{8, 4, 2}, {8, 8, 1}, {8, 2, 4}, {8, 4, 2}},
    {{16, 4, 4}, {16, 8, 2}, {16, 2, 8}, {16, 4, 4}},
    {{32, 4, 8}, {32, 8, 4}, {32, 2, 16}, {32, 4, 8}},
    {{64, 4, 16}, {64, 8, 8}, {64, 4, 8}, {64, 2, 16}},
    {{128, 4, 8}, {128, 2, 8}, {128, 2, 16}, {128, 4, 4}},
    {{256, 2, 8}, {256, 1, 8}, {256, 2, 4}, {256, 1, 16}},
};
constexpr int PCG_NSHAPES[6] = {3, 3, 3, 4, 4, 4};
inline int kc_index(int KC) {
    int i = 0;
    while ((8 << i) < KC) ++i;
    return i;
}
PcgShape pcg_shape(int KC, int shape = 0);

// Gram tile edge and W = H X tile width for a K class (SIMT kernels).
inline int gram_tb(int KC) { return KC <= 16 ? 16 : (KC >= 64 ? 64 : KC); }
inline int hx_tn(int KC) { return KC <= 16 ? 16 : (KC >= 64 ? 64 : KC); }
constexpr int HX_TM = 64;

// tiles: (instance, bi, bj, 0) with bi >= bj
cudaError_t launch_gram_simt(int TB, const DevInst *insts, const int4 *tiles, int n_tiles,
                             DevAccum acc, cudaStream_t s, bool accurate = false);
// tensor-core Gram (3xTF32), diagonal 64 x 64 blocks; list: (instance, user group) jobs
cudaError_t launch_gram_tc64(const DevInst *insts, const int2 *list, int n, DevAccum acc,
                             cudaStream_t s);
// tensor-core Gram, off-diagonal blocks (a, b), a < b, and their mirrors (K = 128 and
// 256 classes); list: (instance, a, b, 0) jobs
cudaError_t launch_gram_tc_cross(const DevInst *insts, const int4 *list, int n, DevAccum acc,
                                 cudaStream_t s);
// tensor-core Gram of bfloat16 channels of the K = 128 and 256 classes (kind::f16,
// H read by tiled tensor copies); jobs: (instance, user tile a, user tile b >= a,
// index into maps), 128-user tiles; maps: per instance a 2-D BF16 tensor map over
// H as K rows of 2M values, box 64 x 128, 128-byte swizzle
cudaError_t launch_gram_bf16(const DevInst *insts, const int4 *jobs, int n, const CUtensorMap *maps, DevAccum acc,
                             cudaStream_t s);
// tensor-core W = H X for bfloat16 channels of the K = 128 and 256 classes (kind::f16,
// X as three exact bfloat16 terms); jobs: (instance, 32-column output group, index
// into maps, 0); maps: per instance the same tensor over H with box 64 x 64
cudaError_t launch_hx_bf16(const DevInst *insts, const int4 *jobs, int n, const CUtensorMap *maps, DevAccum acc,
                           cudaStream_t s);
// tensor-core W = H X for the K = 64 class (3xTF32); list: instance ids
cudaError_t launch_hx_tc64(const DevInst *insts, const int *list, int n, DevAccum acc,
                           cudaStream_t s);
// tensor-core W = H X for the K = 128 and 256 classes (X streamed per stage);
// list: (instance, 64-column output group) jobs
cudaError_t launch_hx_tc_wide(const DevInst *insts, const int2 *list, int n, DevAccum acc,
                              cudaStream_t s);
// tensor-core iteration for the K = 64 class (standard or plain CG); list: instance ids;
// amap: 2-D FP32 tensor map over the arena holding every instance's A (rows of 64
// floats, box 64 x 128), arena: its base address
cudaError_t launch_pcg_tc64(int variant, const DevInst *insts, const int *list, int n, DevAccum acc,
                            const CUtensorMap *amap, const char *arena, cudaStream_t s, int mode);
// tensor-core iteration for the K = 128 and 256 classes (standard or plain CG):
// launch_tcw_prep stores each listed instance's A as the streamed FP16 stages
// (DevInst::As), launch_pcg_tcw iterates; jobs: (instance, first of
// pcg_tcw_cols() columns); mode 0 solve, 1 refinement correction, 2 correction
// with the FP16 heads only
int pcg_tcw_cols();
cudaError_t launch_tcw_prep(int KC, const DevInst *insts, const int *list, int n, cudaStream_t s);
cudaError_t launch_pcg_tcw(int KC, int variant, const DevInst *insts, const int2 *jobs, int n, DevAccum acc,
                           cudaStream_t s, int mode);
// direct solve (Cholesky, forward and back substitution) of the K = KC class;
// list: instance ids.  Replaces the iteration for the JACPCG_DIRECT variant.
cudaError_t launch_chol(int KC, const DevInst *insts, const int *list, int n, DevAccum acc, cudaStream_t s);
// per-user SINR (Eq. 9) from H, W and the power factor; jobs: (instance, block of 8 users)
cudaError_t launch_sinr(int KC, const DevInst *insts, const int2 *jobs, int n, cudaStream_t s);
// blocks: (instance, first column); mode 0: A X = I, mode 1: A dX = R, X += dX
cudaError_t launch_pcg(int KC, int variant, const DevInst *insts, const int2 *blocks,
                       int n_blocks, DevAccum acc, cudaStream_t s, int mode = 0);
cudaError_t launch_pcg_shape(int KC, int shape, int variant, const DevInst *insts, const int2 *blocks,
                             int n_blocks, DevAccum acc, cudaStream_t s, int mode);
#define JACPCG_DECLARE_PCG_CLASS(KC)                                                              \
    cudaError_t launch_pcg_k##KC(int shape, int variant, const DevInst *insts, const int2 *blocks, \
                                 int n_blocks, DevAccum acc, cudaStream_t s, int mode);
JACPCG_DECLARE_PCG_CLASS(8)
JACPCG_DECLARE_PCG_CLASS(16)
JACPCG_DECLARE_PCG_CLASS(32)
JACPCG_DECLARE_PCG_CLASS(64)
JACPCG_DECLARE_PCG_CLASS(128)
JACPCG_DECLARE_PCG_CLASS(256)
#undef JACPCG_DECLARE_PCG_CLASS
// refinement: R = B - A X (FP64 or Dot2) and per-column ||R_j||^2, ||B_j||^2 (blocks:
// (instance, first column), RES_CB columns each; from the second evaluation on,
// instances that stopped refining are skipped), then hist[sweep] = ||R||_F / sqrt(n)
// and the stop decision per instance
constexpr int RES_CB = 8;
cudaError_t launch_residual(const DevInst *insts, const int2 *blocks, int n_blocks, int sweep,
                            cudaStream_t s, bool fp64);
cudaError_t launch_resid_hist(const DevInst *insts, int n_inst, int sweep, cudaStream_t s);
// the same residual with sliced products on the tensor cores (K = 128 and 256
// classes): launch_rtc_prep slices A once per execute (list: instance ids;
// DevInst::Asl, resid_tc_slice_bytes(KC) bytes, and DevInst::rexp), then each
// evaluation runs launch_resid_tc over (instance, first of 24 columns) jobs
size_t resid_tc_slice_bytes(int KC);
cudaError_t launch_rtc_prep(int KC, const DevInst *insts, const int *list, int n, cudaStream_t s);
cudaError_t launch_resid_tc(int KC, const DevInst *insts, const int2 *jobs, int n, int sweep, DevAccum acc,
                            cudaStream_t s);
// tiles: (instance, m tile, n tile, partial slot)
cudaError_t launch_hx_simt(int TN, const DevInst *insts, const int4 *tiles, int n_tiles,
                           cudaStream_t s);
cudaError_t launch_finalize(const DevInst *insts, int n_inst, DevAccum acc, DevOut out,
                            cudaStream_t s);

}  // namespace jacpcg
