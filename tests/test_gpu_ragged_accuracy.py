"""The ragged workload's accuracy bar, through the C ABI: a batch drawn from
the ragged distribution (K uniform over {8, ..., 256}, M over {256, ...,
4096}, 8 subarrays, SNR in {0, 10, 20} dB) in tolerance mode -- tol 1e-5,
with Dot2 refinement that stops each instance at relative residual 1e-7 --
must put every precoder within 1e-5 (relative Frobenius) of the direct RZF
of Eq. 7, including the near-square 256-user channels whose Jacobi-scaled
condition numbers reach the thousands.  Marked gpu."""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

from oracle import oracle as O
from paper_2305_13925_gb300 import channels as C

from gpu_util import rel_fro, run

pytestmark = pytest.mark.gpu

TOL_W = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_13925_gb300 import build
    build.build()


@pytest.mark.parametrize("precision,selective", [("tf32x3", False), ("fp32", False), ("tf32x3", True)])
def test_ragged_batch_every_instance_within_1e5_of_direct_rzf(precision, selective):
    """selective: refinement (and the compensated Gram) only for the channels
    with M <= 2 K, the policy of the ragged and serving workloads."""
    insts = C.generate_ragged(40, 3)
    # and the hardest corner of the distribution: square 256-user channels at 20 dB
    hard = C.ChannelSpec(M=256, S=8, K=256, r=(0.3, 0.9), n_vis=(2, 6), snr_db=(20.0,))
    insts += [C.generate_instance(hard, 3, 5000 + i) for i in range(4)]
    Hs = [C.round_complex64(i.H) for i in insts]
    xis = [i.xi for i in insts]
    out = run(Hs, xis, T=1000, tol=1e-5, precision=precision, refine_sweeps=3, refine_tol=1e-7,
              refine_solve_tol=1e-2, refine_selective=selective, want_hist=True)
    with ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as ex:
        direct = list(ex.map(lambda a: O.rzf_direct(a[0], a[1])[0], zip(Hs, xis)))
    errs = [rel_fro(out["W"][i], direct[i]) for i in range(len(Hs))]
    worst = int(np.argmax(errs))
    assert (out["status"] == 0).all(), out["status"]
    assert errs[worst] <= TOL_W, (worst, Hs[worst].shape, errs[worst])
    if selective:   # unrefined instances keep an untouched history (no residual evaluated)
        for i, h in enumerate(Hs):
            if h.shape[0] > 2 * h.shape[1]:
                assert out["hist"][i][0] == -1.0, i
            else:
                assert out["hist"][i][0] > 0.0, i
