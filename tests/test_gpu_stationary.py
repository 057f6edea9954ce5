"""GPU parity of the JOR iteration (Sec. III-A, the paper's parallel
stationary method) against the FP64 oracle, through the C ABI.  The paper
gives no relaxation factor; each channel takes omega = 2 / (lambda_min +
lambda_max) of D^{-1} P, computed here on the host (the caller's choice), at
which JOR always converges.  Gauss-Seidel is sequential by the paper's own
account and lives in the oracle only.  Marked gpu."""
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


def omega_opt(H, xi):
    A = O.gram(H, xi)
    d = np.real(np.diag(A))
    lam = np.linalg.eigvalsh(A / np.sqrt(np.outer(d, d)))
    return 2.0 / (lam[0] + lam[-1])


def _mixed_instances():
    insts = C.generate_ragged(12, 5, k_set=(8, 16, 32, 64, 128, 256), m_set=(512, 1024, 2048))
    return [C.round_complex64(i.H) for i in insts], [i.xi for i in insts]


@pytest.mark.parametrize("precision", ["fp32", "tf32x3"])
@pytest.mark.parametrize("T", [1, 6])
def test_jor_fixed_T_parity(precision, T):
    """Every K class (8 ... 256) in one ragged batch, T sweeps of JOR, W, X
    and beta element by element against the oracle's JOR."""
    Hs, xis = _mixed_instances()
    om = [omega_opt(h, x) for h, x in zip(Hs, xis)]
    out = run(Hs, xis, variant="jor", T=T, want_X=True, precision=precision, omegas=om)
    for i, (H, xi) in enumerate(zip(Hs, xis)):
        ref = O.precode(H, xi, "jor", max_iter=T, omega=om[i])
        assert out["status"][i] == 0
        assert rel_fro(out["W"][i], ref["W"]) <= TOL_W, (i, H.shape)
        assert rel_fro(out["X"][i], ref["X"]) <= TOL_W, (i, H.shape)
        assert abs(out["beta"][i] - ref["beta"]) <= TOL_W * ref["beta"]
        assert out["iters"][i] == T


def test_jor_tolerance_reaches_the_direct_rzf():
    """Under a tolerance JOR runs to the RZF of Eq. 7: each W within 1e-5 of
    the direct (Cholesky) precoder, iteration counts within one of the
    oracle's (the stopping residual is a recurrence in FP32 there)."""
    Hs, xis = _mixed_instances()
    om = [omega_opt(h, x) for h, x in zip(Hs, xis)]
    out = run(Hs, xis, variant="jor", T=4000, tol=1e-7, precision="tf32x3", omegas=om)
    for i, (H, xi) in enumerate(zip(Hs, xis)):
        Wd = O.rzf_direct(H, xi)[0]
        ref = O.precode(H, xi, "jor", max_iter=4000, tol=1e-7, omega=om[i])
        assert out["status"][i] == 0
        assert rel_fro(out["W"][i], Wd) <= TOL_W, (i, H.shape, rel_fro(out["W"][i], Wd))
        assert abs(int(out["iters"][i]) - ref["iters"]) <= max(2, ref["iters"] // 20), (i, out["iters"][i], ref["iters"])


def test_jor_omega_zero_is_the_jacobi_iteration():
    """omega = 0 in the instance means 1 (Jacobi): bit-identical to omega = 1."""
    inst = C.generate_instance(C.PRESETS["single_256x16"], 0, 2)
    H = C.round_complex64(inst.H)
    a = run([H], [inst.xi], variant="jor", T=5, omegas=[0.0])
    b = run([H], [inst.xi], variant="jor", T=5, omegas=[1.0])
    assert np.array_equal(a["W"][0], b["W"][0])
    ref = O.precode(H, inst.xi, "jor", max_iter=5, omega=1.0)
    assert rel_fro(a["W"][0], ref["W"]) <= TOL_W


def test_jor_rejects_invalid_omega():
    import torch
    from paper_2305_13925_gb300 import binding
    inst = C.generate_instance(C.PRESETS["single_256x16"], 0, 2)
    with binding.Precoder(max_instances=1, max_M=256, max_K=16, variant="jor") as prec:
        Hd = torch.from_numpy(np.ascontiguousarray(inst.H.T).astype(np.complex64)).cuda()
        Wd = torch.empty_like(Hd)
        for bad in (2.0, -0.5, float("nan")):
            with pytest.raises(binding.JacpcgError) as e:
                prec.precode([binding.instance(Hd, Wd, inst.xi, 4, omega=bad)])
            assert e.value.status == binding.JACPCG_EINVAL
