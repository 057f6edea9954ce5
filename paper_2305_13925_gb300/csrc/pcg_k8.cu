// pcg_k8.cu -- the Jac-PCG iteration kernel instantiated for the K = 8
// class in each candidate launch shape (see PCG_SHAPES in kernels.h).
#include "pcg_kernel.cuh"

namespace jacpcg {

static_assert(PCG_SHAPES[0][0].CW == 4 && PCG_SHAPES[0][0].NW == 2, "shape table");
static_assert(PCG_SHAPES[0][1].CW == 8 && PCG_SHAPES[0][1].NW == 1, "shape table");
static_assert(PCG_SHAPES[0][2].CW == 2 && PCG_SHAPES[0][2].NW == 4, "shape table");
cudaError_t launch_pcg_k8(int shape, int variant, const DevInst *insts, const int2 *blocks,
                            int n_blocks, DevAccum acc, cudaStream_t s, int mode) {
    switch (shape) {
        case 0: return pcgk::launch_cfg<8, 4, 2, true>(variant, insts, blocks, n_blocks, acc, s, mode);
        case 1: return pcgk::launch_cfg<8, 8, 1, true>(variant, insts, blocks, n_blocks, acc, s, mode);
        case 2: return pcgk::launch_cfg<8, 2, 4, true>(variant, insts, blocks, n_blocks, acc, s, mode);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace jacpcg
