"""Mixed precision on the GPU: H stored as bfloat16 (values used exactly),
and iterative refinement with the true residual I - A X evaluated in FP64.
The oracle always runs on the bfloat16-rounded channel (upcast exactly)."""
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


@pytest.mark.parametrize("precision", ["fp32", "tf32x3"])
def test_bf16_storage_fixed_T_parity(precision):
    """bfloat16 H, T = 6: W matches the oracle on the same rounded channel
    within 1e-5 (K = 64 exercises the tensor path, K = 17 and 128 the SIMT one)."""
    H, xi = C.generate_batch("batched_1024x64", 6, 1, dtype="bf16")
    insts = list(zip(H, xi))
    for spec_k, spec_m in ((17, 256), (128, 512)):
        spec = C.ChannelSpec(M=spec_m, S=4, K=spec_k, r=(0.5, 0.5), n_vis=(2, 3), snr_db=(10.0,))
        i = C.generate_instance(spec, 3, spec_k, dtype="bf16")
        insts.append((i.H, i.xi))
    out = run([h for h, _ in insts], [x for _, x in insts], T=6, precision=precision, bf16=True)
    for k, (h, x) in enumerate(insts):
        ref = O.precode(h, x, "standard", max_iter=6)
        assert out["status"][k] == 0
        assert rel_fro(out["W"][k], ref["W"]) <= 1e-5, (k, rel_fro(out["W"][k], ref["W"]))


@pytest.mark.parametrize("fp64", [False, True])
@pytest.mark.parametrize("shape", [("xl_4096x256", 2), ("batched_1024x64", 4)])
def test_refinement_reaches_direct_rzf(shape, fp64):
    """A loose first solve (tol 1e-3) then three refinement sweeps: the FP64
    residual history decreases, and W ends within 1e-5 of the direct RZF of
    the bfloat16 channel; without refinement it does not."""
    preset, n = shape
    H, xi = C.generate_batch(preset, n, 2, dtype="bf16")
    before = run(list(H), list(xi), T=60, tol=1e-3, bf16=True, precision="tf32x3")
    after = run(list(H), list(xi), T=60, tol=1e-3, bf16=True, precision="tf32x3", refine_sweeps=3,
                want_hist=True, refine_fp64=fp64)
    for k in range(n):
        Wd, _, st = O.rzf_direct(H[k], xi[k])
        e0 = rel_fro(before["W"][k], Wd)
        e1 = rel_fro(after["W"][k], Wd)
        hist = after["hist"][k]
        assert e0 > 1e-5 and e1 <= 1e-5, (k, e0, e1, hist)
        # the first sweep removes most of the residual; later ones reach the FP32 floor of X
        assert hist[1] < hist[0] / 10 and hist[-1] <= hist[1] * 1.5, hist
        assert after["status"][k] == 0


def _mixed_batch():
    """Two K = 256 channels (SIMT iteration) and two K = 64 channels (tensor
    iteration) in one batch, bfloat16 storage."""
    H1, x1 = C.generate_batch("xl_4096x256", 2, 5, dtype="bf16")
    H2, x2 = C.generate_batch("batched_1024x64", 2, 5, dtype="bf16")
    return list(H1) + list(H2), list(x1) + list(x2)


def test_refinement_tol_stops_at_once():
    """refine_tol = 1 stops every instance at the first residual evaluation:
    no correction runs, the history repeats its first value and W equals the
    unrefined W."""
    Hs, xis = _mixed_batch()
    plain = run(Hs, xis, T=60, tol=1e-3, bf16=True, precision="tf32x3")
    out = run(Hs, xis, T=60, tol=1e-3, bf16=True, precision="tf32x3", refine_sweeps=3,
              want_hist=True, refine_tol=1.0)
    for k in range(len(Hs)):
        h = out["hist"][k]
        assert h[0] > 0 and np.all(h == h[0]), h
        assert rel_fro(out["W"][k], plain["W"][k]) == 0.0
        assert out["status"][k] == 0


@pytest.mark.parametrize("solve_tol", [0.0, 1e-2])
def test_refinement_tol_stops_early_and_reaches_direct_rzf(solve_tol):
    """refine_tol = 1e-7 with a loose first solve: each instance refines until
    its relative residual is below the target or stops falling; the history
    is constant from the stop on and W ends within 1e-5 of the direct RZF,
    also when each correction solve stops at 1e-2 of its residual."""
    Hs, xis = _mixed_batch()
    out = run(Hs, xis, T=60, tol=1e-3, bf16=True, precision="tf32x3", refine_sweeps=3,
              want_hist=True, refine_tol=1e-7, refine_solve_tol=solve_tol)
    for k in range(len(Hs)):
        h = out["hist"][k]
        Wd, _, _ = O.rzf_direct(Hs[k], xis[k])
        assert rel_fro(out["W"][k], Wd) <= 1e-5, (k, h)
        assert h[1] < h[0] / 10, h
        rep = [s for s in range(1, len(h)) if h[s] == h[s - 1]]
        if rep:   # stopped: nothing changes afterwards
            assert np.all(h[rep[0]:] == h[rep[0]]), h
        assert out["status"][k] == 0


@pytest.mark.parametrize("fp64", [False, True])
def test_refinement_residual_matches_fp64(fp64):
    """The true residual the refinement evaluates (Dot2 or FP64), checked
    through its history entry ||I - A X||_F / sqrt(K) against the same
    quantity recomputed in FP64 from the GPU's own A and X; K = 17, 100 and
    256 leave ragged 16-column blocks and rows beyond K in the K classes."""
    Hs, xis = [], []
    for K, M, seed in ((17, 256, 1), (100, 512, 2), (256, 1024, 3)):
        spec = C.ChannelSpec(M=M, S=4, K=K, r=(0.5, 0.5), n_vis=(2, 3), snr_db=(10.0,))
        inst = C.generate_instance(spec, seed, K)
        Hs.append(inst.H)
        xis.append(inst.xi)
    out = run(Hs, xis, T=60, tol=1e-3, precision="tf32x3", refine_sweeps=1, want_hist=True,
              refine_tol=1.0, want_X=True, want_A=True, refine_fp64=fp64)
    for k, H in enumerate(Hs):
        K = H.shape[1]
        R = np.eye(K) - out["A"][k] @ out["X"][k]
        ref = np.linalg.norm(R) / np.sqrt(K)
        h = out["hist"][k]
        assert ref > 0 and abs(h[0] - ref) <= 1e-4 * ref, (K, h[0], ref)
