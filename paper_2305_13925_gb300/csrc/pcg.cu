// pcg.cu -- launch-shape table and dispatch of the Jac-PCG iteration kernel
// (the kernel itself is in pcg_kernel.cuh, instantiated per K class in
// pcg_k<KC>.cu so that the classes compile in parallel).
#include "kernels.h"

namespace jacpcg {

PcgShape pcg_shape(int KC, int shape) {
    const int c = kc_index(KC);
    if (c < 0 || c > 5) return {KC, 1, 1};
    if (shape < 0 || shape >= PCG_NSHAPES[c]) shape = 0;
    return PCG_SHAPES[c][shape];
}

cudaError_t launch_pcg_shape(int KC, int shape, int variant, const DevInst *insts, const int2 *blocks,
                             int n_blocks, DevAccum acc, cudaStream_t s, int mode) {
    if (n_blocks <= 0) return cudaSuccess;
    switch (KC) {
        case 8: return launch_pcg_k8(shape, variant, insts, blocks, n_blocks, acc, s, mode);
        case 16: return launch_pcg_k16(shape, variant, insts, blocks, n_blocks, acc, s, mode);
        case 32: return launch_pcg_k32(shape, variant, insts, blocks, n_blocks, acc, s, mode);
        case 64: return launch_pcg_k64(shape, variant, insts, blocks, n_blocks, acc, s, mode);
        case 128: return launch_pcg_k128(shape, variant, insts, blocks, n_blocks, acc, s, mode);
        case 256: return launch_pcg_k256(shape, variant, insts, blocks, n_blocks, acc, s, mode);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_pcg(int KC, int variant, const DevInst *insts, const int2 *blocks, int n_blocks,
                       DevAccum acc, cudaStream_t s, int mode) {
    return launch_pcg_shape(KC, 0, variant, insts, blocks, n_blocks, acc, s, mode);
}

}  // namespace jacpcg
