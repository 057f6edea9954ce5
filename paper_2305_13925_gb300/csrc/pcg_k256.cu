// pcg_k256.cu -- the Jac-PCG iteration kernel instantiated for the K = 256
// class in each candidate launch shape (see PCG_SHAPES in kernels.h).
#include "pcg_kernel.cuh"

namespace jacpcg {

static_assert(PCG_SHAPES[5][0].CW == 2 && PCG_SHAPES[5][0].NW == 8, "shape table");
static_assert(PCG_SHAPES[5][1].CW == 1 && PCG_SHAPES[5][1].NW == 8, "shape table");
static_assert(PCG_SHAPES[5][2].CW == 2 && PCG_SHAPES[5][2].NW == 4, "shape table");
static_assert(PCG_SHAPES[5][3].CW == 1 && PCG_SHAPES[5][3].NW == 16, "shape table");
cudaError_t launch_pcg_k256(int shape, int variant, const DevInst *insts, const int2 *blocks,
                            int n_blocks, DevAccum acc, cudaStream_t s, int mode) {
    switch (shape) {
        case 0: return pcgk::launch_cfg<256, 2, 8, false>(variant, insts, blocks, n_blocks, acc, s, mode);
        case 1: return pcgk::launch_cfg<256, 1, 8, false>(variant, insts, blocks, n_blocks, acc, s, mode);
        case 2: return pcgk::launch_cfg<256, 2, 4, false>(variant, insts, blocks, n_blocks, acc, s, mode);
        case 3: return pcgk::launch_cfg<256, 1, 16, false>(variant, insts, blocks, n_blocks, acc, s, mode);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace jacpcg
