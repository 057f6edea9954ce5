// pcg_k32.cu -- the Jac-PCG iteration kernel instantiated for the K = 32
// class in each candidate launch shape (see PCG_SHAPES in kernels.h).
#include "pcg_kernel.cuh"

namespace jacpcg {

static_assert(PCG_SHAPES[2][0].CW == 4 && PCG_SHAPES[2][0].NW == 8, "shape table");
static_assert(PCG_SHAPES[2][1].CW == 8 && PCG_SHAPES[2][1].NW == 4, "shape table");
static_assert(PCG_SHAPES[2][2].CW == 2 && PCG_SHAPES[2][2].NW == 16, "shape table");
cudaError_t launch_pcg_k32(int shape, int variant, const DevInst *insts, const int2 *blocks,
                            int n_blocks, DevAccum acc, cudaStream_t s, int mode) {
    switch (shape) {
        case 0: return pcgk::launch_cfg<32, 4, 8, true>(variant, insts, blocks, n_blocks, acc, s, mode);
        case 1: return pcgk::launch_cfg<32, 8, 4, true>(variant, insts, blocks, n_blocks, acc, s, mode);
        case 2: return pcgk::launch_cfg<32, 2, 16, true>(variant, insts, blocks, n_blocks, acc, s, mode);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace jacpcg
