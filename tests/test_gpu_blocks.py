"""GPU parity of the per-subarray block precoder (Eq. 7 with the block
structure of Eq. 6) through jacpcg_blocks + jacpcg_precode, against the
oracle's block extraction."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2305_13925_gb300 import channels as C

from gpu_util import rel_fro

pytestmark = pytest.mark.gpu

# the paper's three blocks on the 8 x 128-antenna array: group-1 users (first
# half) on subarrays 0-2, every user on subarrays 3-4, group-2 users on 5-7
PAPER_BLOCKS = [(0, 384, 0, 32), (384, 256, 0, 64), (640, 384, 32, 32)]


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_13925_gb300 import build
    build.build()


@pytest.mark.parametrize("precision", ["fp32", "tf32x3"])
def test_paper_blocks_against_oracle(precision):
    import torch
    from paper_2305_13925_gb300 import binding
    n = 12
    Hst, xi = C.generate_batch_device_layout("batched_1024x64", n, 5)
    Hd = torch.from_numpy(Hst).cuda()
    Wd = torch.zeros_like(Hd)                       # zero blocks of G stay zero
    insts = []
    for i in range(n):
        full = binding.instance(Hd[i], Wd[i], float(xi[i]), 6, power=3.0)
        insts += binding.jacpcg_blocks(full, PAPER_BLOCKS)
    st = torch.full((len(insts),), -1, dtype=torch.int32, device="cuda")
    beta = torch.zeros(len(insts), dtype=torch.float32, device="cuda")
    with binding.Precoder(max_instances=len(insts), max_M=1024, max_K=64, precision=precision) as prec:
        prec.precode(insts, st, beta=beta)
        torch.cuda.synchronize()
    assert (st.cpu().numpy() == 0).all()
    b = beta.cpu().numpy()
    for i in range(n):
        H = Hst[i].T.astype(np.complex128)
        G, betas = O.precode_blocks(H, xi[i], PAPER_BLOCKS, "standard", max_iter=6, power=3.0)
        Wg = Wd[i].T.cpu().numpy().astype(np.complex128)
        assert np.count_nonzero(Wg[0:384, 32:]) == 0 and np.count_nonzero(Wg[640:, :32]) == 0
        for k, (r0, nr, c0, nc) in enumerate(PAPER_BLOCKS):
            blk = Wg[r0:r0 + nr, c0:c0 + nc]
            assert rel_fro(blk, G[r0:r0 + nr, c0:c0 + nc]) <= 1e-5, (i, k)
            assert abs(b[3 * i + k] - betas[k]) <= 1e-5 * betas[k], (i, k)
