"""GPU parity of the direct RZF (Appendix: Cholesky factorisation, forward
and back substitution), the comparator of the paper's operation counts, run
as the JACPCG_DIRECT variant of the batched path: W against the oracle's
Cholesky precoder (the exact RZF of Eq. 7), through the C ABI.  Marked gpu."""
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


@pytest.mark.parametrize("precision", ["fp32", "tf32x3"])
def test_direct_matches_the_exact_rzf(precision):
    """Every K class (8 ... 256, shared-memory and in-workspace factorisation)
    in one ragged batch, K not a power of two included: W, X and beta within
    1e-5 of the oracle's Cholesky RZF; iters and resid report 0."""
    insts = C.generate_ragged(12, 6, k_set=(8, 16, 32, 64, 128, 256), m_set=(512, 1024, 2048))
    Hs = [C.round_complex64(i.H) for i in insts] + [
        C.round_complex64(C.generate_instance(C.ChannelSpec(M=M, S=1, K=K, r=(0.5, 0.5), n_vis=(1, 1),
                                                            snr_db=(10.0,)), 8, K).H)
        for K, M in ((3, 40), (100, 700), (200, 900))]
    xis = [i.xi for i in insts] + [0.3, 0.5, 0.8]
    out = run(Hs, xis, variant="direct", T=0, want_X=True, precision=precision)
    for i, (H, xi) in enumerate(zip(Hs, xis)):
        Wd, Xd, st = O.rzf_direct(H, xi)
        assert st == O.OK and out["status"][i] == 0
        assert rel_fro(out["W"][i], Wd) <= TOL_W, (i, H.shape, rel_fro(out["W"][i], Wd))
        assert rel_fro(out["X"][i], Xd) <= TOL_W, (i, H.shape)
        assert abs(out["beta"][i] - O.power_factor(Wd)) <= TOL_W * O.power_factor(Wd)
        assert out["iters"][i] == 0


def test_direct_solves_symbol_blocks():
    """With symbol vectors B (Eq. 16), X = P^{-1} B by the two substitutions."""
    import torch
    from paper_2305_13925_gb300 import binding
    rng = np.random.default_rng(12)
    cases = []
    for K, M, n in ((16, 256, 5), (64, 1024, 14), (256, 2048, 3)):
        inst = C.generate_instance(C.ChannelSpec(M=M, S=8, K=K, r=(0.3, 0.9), n_vis=(2, 6),
                                                 snr_db=(10.0,)), 9, K)
        B = (rng.standard_normal((K, n)) + 1j * rng.standard_normal((K, n))) / np.sqrt(2)
        cases.append((C.round_complex64(inst.H), inst.xi, B.astype(np.complex64).astype(np.complex128)))
    with binding.Precoder(max_instances=3, max_M=2048, max_K=256, variant="direct",
                          precision="tf32x3") as prec:
        Hd = [torch.from_numpy(np.ascontiguousarray(H.T).astype(np.complex64)).cuda() for H, _, _ in cases]
        Bd = [torch.from_numpy(np.ascontiguousarray(B.T).astype(np.complex64)).cuda() for _, _, B in cases]
        Wd = [torch.zeros((B.shape[1], H.shape[0]), dtype=torch.complex64, device="cuda") for H, _, B in cases]
        Xd = [torch.zeros((B.shape[1], B.shape[0]), dtype=torch.complex64, device="cuda") for _, _, B in cases]
        insts = [binding.instance(Hd[i], Wd[i], cases[i][1], 0, X=Xd[i], B=Bd[i]) for i in range(3)]
        status = torch.full((3,), -1, dtype=torch.int32, device="cuda")
        prec.precode(insts, status)
        torch.cuda.synchronize()
    assert (status.cpu().numpy() == 0).all()
    for i, (H, xi, B) in enumerate(cases):
        A = O.gram(H, xi)
        Xr, st = O.cholesky_solve(A, B)
        assert rel_fro(Xd[i].T.cpu().numpy().astype(np.complex128), Xr) <= TOL_W, i
        assert rel_fro(Wd[i].T.cpu().numpy().astype(np.complex128), O.matmul(H, Xr)) <= TOL_W, i


def test_direct_rejects_refinement():
    from paper_2305_13925_gb300 import binding
    with pytest.raises(binding.JacpcgError) as e:
        binding.Precoder(max_instances=1, max_M=64, max_K=8, variant="direct", refine_sweeps=1)
    assert e.value.status == binding.JACPCG_EINVAL
