"""The sliced tensor-core refinement residual of the K = 128 and 256 classes
(8-bit integer slices of the balanced A's rows and X's columns, exact slice
products and class sums on the FP16 tensor cores), through the C ABI: the residual norm it
reports after the last sweep against I - A X evaluated in FP64 on the host
from the library's own A and X, the refined W against the FP64-residual
refinement and against the direct RZF of Eq. 7, in one plan with instances
that keep the Dot2 residual (K = 64) and with per-symbol right-hand sides.
Marked gpu."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2305_13925_gb300 import channels as C

from gpu_util import rel_fro, run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_13925_gb300 import build
    build.build()


def _inst(K, M, seed, S=4):
    spec = C.ChannelSpec(M=M, S=S, K=K, r=(0.3, 0.9), n_vis=(2, S), snr_db=(10.0,))
    i = C.generate_instance(spec, seed, K * 11 + M)
    return i.H, i.xi


def _batch():
    # sliced: M > 2 K in the 128 and 256 classes; Dot2: the 64 class and M <= 2 K
    shapes = [(256, 4096), (256, 1024), (200, 900), (129, 512), (128, 2048), (64, 1024), (100, 400), (256, 480)]
    pairs = [_inst(K, M, 70 + n) for n, (K, M) in enumerate(shapes)]
    Hs = [C.round_complex_bf16(h) if h.shape[1] == 256 else C.round_complex64(h) for h, _ in pairs]
    return Hs, [x for _, x in pairs], [h.shape[1] == 256 for h in Hs]


@pytest.mark.parametrize("bf16", [False, True])
def test_sliced_residual_matches_fp64_host_residual(bf16):
    """Fixed T = 6 and one sweep, so the final residual stays near 1e-4 and its
    norm is a sharp check: hist[1] (the residual of the final X) against
    ||I - A X||_F / sqrt(K) in FP64 from the library's A and X; the refined W
    against the same refinement with the FP64 residual."""
    Hs, xis, _ = _batch()
    if bf16:
        Hs = [C.round_complex_bf16(h) for h in Hs]
    kw = dict(T=6, precision="tf32x3", bf16=bf16, refine_sweeps=1, want_hist=True, want_A=True, want_X=True)
    sl = run(Hs, xis, refine_residual="sliced", **kw)
    f64 = run(Hs, xis, refine_residual="fp64", **kw)
    assert (sl["status"] == 0).all() and (f64["status"] == 0).all()
    for i, H in enumerate(Hs):
        K = H.shape[1]
        A, X = sl["A"][i], sl["X"][i]
        r_host = np.linalg.norm(np.eye(K) - A @ X) / np.sqrt(K)
        r_gpu = float(sl["hist"][i][1])
        assert abs(r_gpu - r_host) <= 1e-3 * r_host, (i, H.shape, r_gpu, r_host)
        assert rel_fro(sl["W"][i], f64["W"][i]) <= 1e-6, (i, H.shape)


def test_sliced_residual_refinement_reaches_the_direct_rzf():
    """Tolerance 1e-5 and two sweeps, the XL headline's kind of run: every W
    within 1e-5 of the direct RZF and within 1e-6 of the FP64-residual run."""
    Hs, xis, _ = _batch()
    kw = dict(T=100, tol=1e-5, precision="tf32x3", refine_sweeps=2)
    sl = run(Hs, xis, refine_residual="sliced", **kw)
    f64 = run(Hs, xis, refine_residual="fp64", **kw)
    assert (sl["status"] == 0).all()
    for i, H in enumerate(Hs):
        assert rel_fro(sl["W"][i], f64["W"][i]) <= 1e-6, (i, H.shape)
        assert rel_fro(sl["W"][i], O.rzf_direct(H, xis[i])[0]) <= 1e-5, (i, H.shape)


def test_sliced_residual_symbol_blocks():
    """Per-symbol right-hand sides with refinement: R = B - A X with the
    caller's B in the sliced kernel; W against the oracle's direct solve."""
    import torch
    from paper_2305_13925_gb300 import binding
    K, M, n_rhs = 256, 1500, 40
    H, xi = _inst(K, M, 91)
    H = C.round_complex64(H)
    rng = np.random.default_rng(5)
    B = ((rng.standard_normal((K, n_rhs)) + 1j * rng.standard_normal((K, n_rhs))) / np.sqrt(2))
    B = B.astype(np.complex64).astype(np.complex128)
    A = O.gram(H, xi)
    S_ref = H @ np.linalg.solve(A, B)
    Hd = torch.from_numpy(np.ascontiguousarray(H.T).astype(np.complex64)).cuda()
    Bd = torch.from_numpy(np.ascontiguousarray(B.T).astype(np.complex64)).cuda()
    Wd = torch.zeros((n_rhs, M), dtype=torch.complex64, device="cuda")
    st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    with binding.Precoder(max_instances=1, max_M=M, max_K=K, precision="tf32x3", refine_sweeps=2,
                          refine_residual="sliced") as prec:
        prec.precode([binding.instance(Hd, Wd, xi, 100, 1e-5, B=Bd)], st)
        torch.cuda.synchronize()
    assert int(st.item()) == 0
    assert rel_fro(Wd.T.cpu().numpy().astype(np.complex128), S_ref) <= 1e-5
