"""GPU SINR / SE pipeline (Eq. 9 per user, Eq. 10's sum SE) computed from
the GPU's own W and beta (instance field `sinr`), through the C ABI:
  - the kernel's arithmetic: per-user SINR against the oracle's Eq. 9 applied
    to the same GPU precoder (relative 1e-5; FP32 products, Dot2 sums);
  - the pipeline: sum SE from the GPU's converged Jac-PCG and direct
    precoders against the sum SE of the oracle's direct RZF (relative 1e-6;
    SE is second order in W near the RZF, so a W error of a few 1e-6 moves
    it by about 1e-8), and fixed-T SE against the oracle's fixed-T SE.
Marked gpu."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2305_13925_gb300 import channels as C

from gpu_util import to_dev, to_dev_bf16

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_13925_gb300 import build
    build.build()


def _channels():
    H, xi = C.generate_batch("batched_1024x64", 4, 1)
    insts = C.generate_ragged(8, 13, k_set=(8, 16, 32, 128, 256), m_set=(512, 1024))
    Hs = [C.round_complex64(h) for h in H] + [C.round_complex64(i.H) for i in insts]
    return Hs, list(xi) + [i.xi for i in insts]


def _run(Hs, xis, variant, T, tol=0.0, precision="tf32x3", noise=1.0, bf16=False):
    import torch
    from paper_2305_13925_gb300 import binding
    n = len(Hs)
    Hd = [to_dev_bf16(h, torch) if bf16 else to_dev(h, torch) for h in Hs]
    Wd = [to_dev(np.zeros(h.shape), torch) for h in Hs]
    Sd = [torch.full((h.shape[1],), -1.0, device="cuda") for h in Hs]
    insts = [binding.instance(Hd[i], Wd[i], xis[i], T, tol, sinr=Sd[i], noise=noise) for i in range(n)]
    status = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    beta = torch.zeros(n, dtype=torch.float32, device="cuda")
    with binding.Precoder(max_instances=n, max_M=max(h.shape[0] for h in Hs),
                          max_K=max(h.shape[1] for h in Hs), variant=variant, precision=precision) as prec:
        prec.precode(insts, status, None, None, beta)
        torch.cuda.synchronize()
    assert (status.cpu().numpy() == 0).all()
    return ([w.T.cpu().numpy().astype(np.complex128) for w in Wd], beta.cpu().numpy().astype(np.float64),
            [s.cpu().numpy().astype(np.float64) for s in Sd])


@pytest.mark.parametrize("bf16", [False, True])
def test_sinr_kernel_against_eq9_on_the_same_precoder(bf16):
    """Per-user SINR from the GPU equals Eq. 9 evaluated by the oracle on the
    GPU's own beta W (every K class, both storage types of H, noise 0.5)."""
    Hs, xis = _channels()
    if bf16:
        Hs = [C.round_complex_bf16(h) for h in Hs]
    W, beta, g = _run(Hs, xis, "standard", 6, noise=0.5, bf16=bf16)
    for i, H in enumerate(Hs):
        ref = O.sinr(H, beta[i] * W[i], 0.5)
        assert np.max(np.abs(g[i] - ref) / ref) <= 1e-5, (i, H.shape)


@pytest.mark.parametrize("variant,T,tol", [("standard", 2000, 1e-6), ("direct", 0, 0.0)])
def test_sum_se_matches_the_direct_rzf(variant, T, tol):
    """Sum SE (Eq. 10's argument) from the GPU's converged Jac-PCG precoder and
    from its direct precoder equals the oracle's direct-RZF SE within 1e-6."""
    Hs, xis = _channels()
    W, beta, g = _run(Hs, xis, variant, T, tol)
    for i, (H, xi) in enumerate(zip(Hs, xis)):
        Wd = O.rzf_direct(H, xi)[0]
        se_ref = O.sum_se(H, O.power_factor(Wd) * Wd)
        se = float(np.sum(np.log2(1.0 + g[i])))
        assert abs(se - se_ref) <= 1e-6 * se_ref, (i, H.shape, se, se_ref)


def test_fixed_T_sum_se_matches_the_oracle():
    """At a fixed T = 3 (far from converged) the GPU's SE equals the SE of the
    oracle's own T = 3 precoder within 1e-6."""
    Hs, xis = _channels()
    W, beta, g = _run(Hs, xis, "standard", 3)
    for i, (H, xi) in enumerate(zip(Hs, xis)):
        ref = O.precode(H, xi, "standard", max_iter=3)
        se_ref = O.sum_se(H, ref["beta"] * ref["W"])
        se = float(np.sum(np.log2(1.0 + g[i])))
        assert abs(se - se_ref) <= 1e-6 * se_ref, (i, H.shape, se, se_ref)


def test_sinr_needs_the_identity_right_hand_side():
    import torch
    from paper_2305_13925_gb300 import binding
    H = torch.zeros((8, 64), dtype=torch.complex64, device="cuda")
    W = torch.zeros((2, 64), dtype=torch.complex64, device="cuda")
    B = torch.zeros((2, 8), dtype=torch.complex64, device="cuda")
    S = torch.zeros(8, device="cuda")
    with binding.Precoder(max_instances=1, max_M=64, max_K=8) as prec:
        with pytest.raises(binding.JacpcgError) as e:
            prec.precode([binding.instance(H, W, 1.0, 4, B=B, sinr=S)])
        assert e.value.status == binding.JACPCG_EINVAL
