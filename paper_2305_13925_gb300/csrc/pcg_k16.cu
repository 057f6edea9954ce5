// pcg_k16.cu -- the Jac-PCG iteration kernel instantiated for the K = 16
// class in each candidate launch shape (see PCG_SHAPES in kernels.h).
#include "pcg_kernel.cuh"

namespace jacpcg {

static_assert(PCG_SHAPES[1][0].CW == 4 && PCG_SHAPES[1][0].NW == 4, "shape table");
static_assert(PCG_SHAPES[1][1].CW == 8 && PCG_SHAPES[1][1].NW == 2, "shape table");
static_assert(PCG_SHAPES[1][2].CW == 2 && PCG_SHAPES[1][2].NW == 8, "shape table");
cudaError_t launch_pcg_k16(int shape, int variant, const DevInst *insts, const int2 *blocks,
                            int n_blocks, DevAccum acc, cudaStream_t s, int mode) {
    switch (shape) {
        case 0: return pcgk::launch_cfg<16, 4, 4, true>(variant, insts, blocks, n_blocks, acc, s, mode);
        case 1: return pcgk::launch_cfg<16, 8, 2, true>(variant, insts, blocks, n_blocks, acc, s, mode);
        case 2: return pcgk::launch_cfg<16, 2, 8, true>(variant, insts, blocks, n_blocks, acc, s, mode);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace jacpcg
