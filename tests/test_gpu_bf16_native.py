"""The bfloat16 channels of the K = 128 and 256 classes on the kind::f16
tensor-core Gram and W = H X (H read by tiled tensor copies, X as three
exact bfloat16 terms), through the C ABI, against the FP64 oracle on the
bfloat16-rounded channel: A within a few FP32 roundings and exactly
Hermitian, W within the FP32 form's 1e-5 bar at fixed T, ragged M (not a
multiple of the 32-antenna stage, padded leading dimension), K at and around
the 128-user tile edge, per-symbol right-hand sides, many jobs per CTA.
Marked gpu."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2305_13925_gb300 import channels as C

from gpu_util import rel_fro, run, to_dev_bf16

pytestmark = pytest.mark.gpu

TOL_W = 1e-5
TOL_A = 1e-6   # relative Frobenius error of the Gram: exact products, FP32 sums of short chains


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_13925_gb300 import build
    build.build()


def _inst(K, M, seed):
    spec = C.ChannelSpec(M=M, S=1, K=K, r=(0.3, 0.9), n_vis=(1, 1), snr_db=(10.0,))
    i = C.generate_instance(spec, seed, K * 7 + M)
    return C.round_complex_bf16(i.H), i.xi


SHAPES = [(256, 4096), (200, 1000), (129, 333), (128, 1024), (100, 290), (256, 301)]


@pytest.mark.parametrize("K,M", SHAPES)
def test_bf16_gram_and_w_match_the_oracle(K, M):
    H, xi = _inst(K, M, 5)
    out = run([H], [xi], T=6, want_A=True, want_X=True, precision="tf32x3", bf16=True)
    A = out["A"][0]
    A_ref = O.gram(H, xi)
    assert out["status"][0] == 0
    assert rel_fro(A, A_ref) <= TOL_A, rel_fro(A, A_ref)
    assert np.array_equal(A, A.conj().T)                    # exactly Hermitian
    assert np.all(np.diag(A).imag == 0.0)
    ref = O.precode(H, xi, "standard", max_iter=6)
    assert rel_fro(out["X"][0], ref["X"]) <= TOL_W
    assert rel_fro(out["W"][0], ref["W"]) <= TOL_W, rel_fro(out["W"][0], ref["W"])
    assert abs(out["beta"][0] - ref["beta"]) <= TOL_W * ref["beta"]


def test_bf16_native_agrees_with_the_complex64_path():
    """The same bfloat16-exact channels stored as complex64 run the 3xTF32
    kernels; both forms land on the same W well inside the bar."""
    pairs = [_inst(256, 2048, 11), _inst(160, 777, 12)]
    Hs = [h for h, _ in pairs]
    xis = [x for _, x in pairs]
    a = run(Hs, xis, T=8, precision="tf32x3", bf16=True)
    b = run(Hs, xis, T=8, precision="tf32x3", bf16=False)
    for i in range(len(Hs)):
        assert rel_fro(a["W"][i], b["W"][i]) <= 2e-6, i


def test_bf16_many_jobs_per_cta():
    """More jobs than SMs on both kernels: 40 channels of K = 256 (3 Gram jobs,
    8 W = H X jobs each) and 60 of K = 128, every instance against the oracle."""
    insts = [_inst(256, 640, 100 + i) for i in range(40)] + [_inst(128, 384, 200 + i) for i in range(60)]
    Hs = [h for h, _ in insts]
    xis = [x for _, x in insts]
    out = run(Hs, xis, T=4, precision="tf32x3", bf16=True)
    W, _, _, _, _ = O.precode_batch(Hs, xis, "standard", max_iter=4)
    assert (out["status"] == 0).all()
    errs = [rel_fro(out["W"][i], W[i]) for i in range(len(Hs))]
    assert max(errs) <= TOL_W, (int(np.argmax(errs)), max(errs))


@pytest.mark.parametrize("n_rhs", [1, 33, 256])
def test_bf16_symbol_blocks(n_rhs):
    """Per-symbol right-hand sides (Eq. 16): W = H X with fewer output columns
    than users (one partial 32-column group, a ragged second group, all 256)."""
    import torch
    from paper_2305_13925_gb300 import binding
    K, M = 256, 1100
    H, xi = _inst(K, M, 41)
    rng = np.random.default_rng(n_rhs)
    B = ((rng.standard_normal((K, n_rhs)) + 1j * rng.standard_normal((K, n_rhs))) / np.sqrt(2))
    B = B.astype(np.complex64).astype(np.complex128)
    ref = O.precode_symbols(H, xi, B, "standard", max_iter=6)
    Hd = to_dev_bf16(H, torch)
    Bd = torch.from_numpy(np.ascontiguousarray(B.T).astype(np.complex64)).cuda()
    Wd = torch.zeros((n_rhs, M), dtype=torch.complex64, device="cuda")
    st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    with binding.Precoder(max_instances=1, max_M=M, max_K=256, precision="tf32x3") as prec:
        prec.precode([binding.instance(Hd, Wd, xi, 6, B=Bd)], st)
        torch.cuda.synchronize()
    assert int(st.item()) == 0
    assert rel_fro(Wd.T.cpu().numpy().astype(np.complex128), ref["S"]) <= TOL_W
