"""GPU parity of the tensor-core (tcgen05, 3xTF32) path against the FP64
oracle, through the C ABI.  Same bar as the FP32 SIMT path: relative
Frobenius error of W at most 1e-5 per instance."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2305_13925_gb300 import channels as C

from gpu_util import rel_fro, run

pytestmark = pytest.mark.gpu

TOL_W = 1e-5
TOL_A = 4e-6      # FP32 accumulation of 2M terms inside the tensor core


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_13925_gb300 import build
    build.build()


def check(Hs, xis, T=6, variant="standard", simt_iteration=False):
    Hs = [C.round_complex64(h) for h in Hs]
    out = run(Hs, xis, variant=variant, T=T, want_X=True, want_A=True, precision="tf32x3",
              simt_iteration=simt_iteration)
    errs = []
    for i, (H, xi) in enumerate(zip(Hs, xis)):
        ref = O.precode(H, xi, variant, max_iter=T)
        e = rel_fro(out["W"][i], ref["W"])
        errs.append(e)
        assert out["status"][i] == 0, (i, out["status"][i])
        assert rel_fro(out["A"][i], ref["A"]) <= TOL_A, (i, rel_fro(out["A"][i], ref["A"]))
        assert np.array_equal(out["A"][i], out["A"][i].conj().T)
        assert e <= TOL_W, (i, H.shape, e)
        assert abs(out["beta"][i] - ref["beta"]) <= 1e-5 * ref["beta"]
    return out, errs


@pytest.mark.parametrize("simt_iteration", [False, True])
def test_tensor_batched_1024x64_subset(simt_iteration):
    H, xi = C.generate_batch("batched_1024x64", 24, 1)
    check(list(H), list(xi), T=6, simt_iteration=simt_iteration)


@pytest.mark.parametrize("K,M", [(64, 1024), (64, 257), (40, 1000), (33, 96), (64, 4096)])
def test_tensor_gram_shapes(K, M):
    spec = C.ChannelSpec(M=M, S=1, K=K, r=(0.5, 0.5), n_vis=(1, 1), snr_db=(10.0,))
    inst = C.generate_instance(spec, 9, K * 7 + M)
    check([inst.H], [inst.xi], T=5)


def test_tensor_ragged_mix_with_simt_classes():
    insts = C.generate_ragged(12, 8, k_set=(16, 64, 128), m_set=(256, 1024))
    check([i.H for i in insts], [i.xi for i in insts], T=4)


@pytest.mark.parametrize("simt_iteration", [False, True])
def test_tensor_tolerance_mode_reaches_direct_rzf(simt_iteration):
    """tf32x3 with tol 1e-6: each column stops at its tolerance and W lands
    within 1e-5 of the direct RZF; iteration counts near the oracle's."""
    H, xi = C.generate_batch("batched_1024x64", 8, 11)
    out = run(list(H), list(xi), T=200, tol=1e-6, precision="tf32x3", simt_iteration=simt_iteration)
    for i in range(8):
        Wd, _, _ = O.rzf_direct(H[i], xi[i])
        assert rel_fro(out["W"][i], Wd) < 1e-5
        ref = O.precode(H[i], xi[i], "standard", max_iter=200, tol=1e-6)
        assert abs(int(out["iters"][i]) - ref["iters"]) <= 2
        assert out["status"][i] == 0


@pytest.mark.parametrize("simt_iteration", [False, True])
def test_tensor_plain_cg_variant(simt_iteration):
    """Plain CG on the tensor path, against the oracle with the FP32-drift bar."""
    from test_gpu_parity import tol_for
    H, xi = C.generate_batch("batched_1024x64", 8, 1)
    Hs = [C.round_complex64(h) for h in H]
    out = run(Hs, list(xi), variant="cg", T=6, precision="tf32x3", simt_iteration=simt_iteration)
    for i in range(8):
        ref = O.precode(Hs[i], xi[i], "cg", max_iter=6)
        assert rel_fro(out["W"][i], ref["W"]) <= tol_for(Hs[i], xi[i], "cg", 6)


@pytest.mark.parametrize("bf16", [False, True])
def test_tensor_many_instances_per_cta(bf16):
    """456 instances of the K = 64 class (three per persistent CTA), M not a
    multiple of the 128-row tile and K < 64 mixed in: the copy streams, split
    stages, B rewrites and TMEM buffers that cross instance boundaries inside
    one CTA, every instance against the oracle."""
    rng = np.random.default_rng(3)
    Hs, xis = [], []
    for n in range(456):
        M = int(rng.choice([96, 257, 1000, 1024]))
        K = int(rng.choice([33, 48, 64]))
        spec = C.ChannelSpec(M=M, S=1, K=K, r=(0.5, 0.5), n_vis=(1, 1), snr_db=(10.0,))
        inst = C.generate_instance(spec, 21, n)
        Hs.append(C.round_complex_bf16(inst.H) if bf16 else C.round_complex64(inst.H))
        xis.append(inst.xi)
    out = run(Hs, xis, T=6, precision="tf32x3", bf16=bf16)
    refs = O.precode_batch(Hs, xis, "standard", max_iter=6)[0]
    assert (out["status"] == 0).all()
    errs = [rel_fro(out["W"][i], refs[i]) for i in range(len(Hs))]
    worst = int(np.argmax(errs))
    assert errs[worst] <= TOL_W, (worst, Hs[worst].shape, errs[worst])


@pytest.mark.parametrize("K,M", [(65, 300), (100, 512), (128, 1024), (129, 700), (200, 1024),
                                 (256, 2048), (256, 300)])
def test_tensor_gram_multiblock_classes(K, M):
    """K = 128 and 256 classes: the Gram as 64 x 64 user-group blocks on the
    tensor cores (diagonal jobs + off-diagonal jobs with their conjugate
    mirrors), K not a multiple of 64 included; A exactly Hermitian and within
    the tensor accumulation bar, W through the SIMT iteration within 1e-5."""
    spec = C.ChannelSpec(M=M, S=1, K=K, r=(0.5, 0.5), n_vis=(1, 1), snr_db=(10.0,))
    inst = C.generate_instance(spec, 13, K * 3 + M)
    check([inst.H], [inst.xi], T=5)


@pytest.mark.parametrize("bf16", [False, True])
def test_tensor_gram_multiblock_many_instances(bf16):
    """Many K = 128 / 256 instances in one call (the off-diagonal jobs of one
    instance run on different SMs and report into shared accumulators)."""
    rng = np.random.default_rng(14)
    Hs, xis = [], []
    for n in range(40):
        K = int(rng.choice([100, 128, 200, 256]))
        M = int(rng.choice([300, 600]))
        spec = C.ChannelSpec(M=M, S=1, K=K, r=(0.5, 0.5), n_vis=(1, 1), snr_db=(10.0,))
        inst = C.generate_instance(spec, 15, n)
        Hs.append(C.round_complex_bf16(inst.H) if bf16 else C.round_complex64(inst.H))
        xis.append(inst.xi)
    out = run(Hs, xis, T=4, precision="tf32x3", bf16=bf16, want_A=True)
    refs = O.precode_batch(Hs, xis, "standard", max_iter=4)[0]
    assert (out["status"] == 0).all()
    for i, H in enumerate(Hs):
        A = O.gram(H, xis[i])
        assert np.array_equal(out["A"][i], out["A"][i].conj().T)
        assert rel_fro(out["A"][i], A) <= TOL_A, i
        assert rel_fro(out["W"][i], refs[i]) <= TOL_W, (i, H.shape)
