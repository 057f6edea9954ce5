// pcg_k128.cu -- the Jac-PCG iteration kernel instantiated for the K = 128
// class in each candidate launch shape (see PCG_SHAPES in kernels.h).
#include "pcg_kernel.cuh"

namespace jacpcg {

static_assert(PCG_SHAPES[4][0].CW == 4 && PCG_SHAPES[4][0].NW == 8, "shape table");
static_assert(PCG_SHAPES[4][1].CW == 2 && PCG_SHAPES[4][1].NW == 8, "shape table");
static_assert(PCG_SHAPES[4][2].CW == 2 && PCG_SHAPES[4][2].NW == 16, "shape table");
static_assert(PCG_SHAPES[4][3].CW == 4 && PCG_SHAPES[4][3].NW == 4, "shape table");
cudaError_t launch_pcg_k128(int shape, int variant, const DevInst *insts, const int2 *blocks,
                            int n_blocks, DevAccum acc, cudaStream_t s, int mode) {
    switch (shape) {
        case 0: return pcgk::launch_cfg<128, 4, 8, true>(variant, insts, blocks, n_blocks, acc, s, mode);
        case 1: return pcgk::launch_cfg<128, 2, 8, true>(variant, insts, blocks, n_blocks, acc, s, mode);
        case 2: return pcgk::launch_cfg<128, 2, 16, true>(variant, insts, blocks, n_blocks, acc, s, mode);
        case 3: return pcgk::launch_cfg<128, 4, 4, true>(variant, insts, blocks, n_blocks, acc, s, mode);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace jacpcg
