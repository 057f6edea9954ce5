"""GPU parity of the tensor-core iteration of the K = 128 and 256 classes
(A streamed in TF32 stages, P resident as the MMA's B operand, 32 columns
per CTA) against the FP64 oracle, through the C ABI.  Bar: relative
Frobenius error of W (and X) at most 1e-5 per instance, the FP32 form's bar;
plain CG with the FP32-drift bar of its fixed-T trajectory."""
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


def _inst(K, M, seed, S=1, n_vis=(1, 1), snr=(10.0,)):
    spec = C.ChannelSpec(M=M, S=S, K=K, r=(0.3, 0.9), n_vis=n_vis, snr_db=snr)
    return C.generate_instance(spec, seed, K * 13 + M)


def _check(Hs, xis, T, variant="standard", bf16=False, tol_w=TOL_W):
    Hs = [C.round_complex_bf16(h) if bf16 else C.round_complex64(h) for h in Hs]
    out = run(Hs, xis, variant=variant, T=T, want_X=True, precision="tf32x3", bf16=bf16)
    errs = []
    for i, (H, xi) in enumerate(zip(Hs, xis)):
        ref = O.precode(H, xi, variant, max_iter=T)
        e = rel_fro(out["W"][i], ref["W"])
        errs.append(e)
        assert out["status"][i] == 0, (i, H.shape, out["status"][i])
        assert e <= tol_w, (i, H.shape, e)
        assert rel_fro(out["X"][i], ref["X"]) <= tol_w, (i, H.shape)
        assert abs(out["beta"][i] - ref["beta"]) <= tol_w * ref["beta"]
        assert out["iters"][i] == ref["iters"]
    return out, errs


@pytest.mark.parametrize("K,M", [(128, 1024), (100, 700), (129, 512), (200, 900), (256, 2048)])
def test_wide_fixed_T_parity(K, M):
    """One instance per shape, K below, at and above a class edge, T = 6."""
    inst = _inst(K, M, 21, S=4 if M % 4 == 0 else 1, n_vis=(2, 4) if M % 4 == 0 else (1, 1))
    _check([inst.H], [inst.xi], T=6)


def test_wide_xl_bf16_batch():
    """Channels of the XL shape (M = 4096, K = 256), H stored as bfloat16,
    T = 8, the oracle on the bfloat16-rounded channel."""
    H, xi = C.generate_batch("xl_4096x256", 3, 2)
    _check(list(H), list(xi), T=8, bf16=True)


def test_wide_plain_cg():
    """Plain CG (C = I) on the wide tensor path, with the FP32-drift bar."""
    from test_gpu_parity import tol_for
    insts = [_inst(K, M, 23) for K, M in ((128, 1024), (256, 1024))]
    Hs = [C.round_complex64(i.H) for i in insts]
    xis = [i.xi for i in insts]
    out = run(Hs, xis, variant="cg", T=6, precision="tf32x3")
    for i, (H, xi) in enumerate(zip(Hs, xis)):
        ref = O.precode(H, xi, "cg", max_iter=6)
        assert rel_fro(out["W"][i], ref["W"]) <= tol_for(H, xi, "cg", 6), i


def test_wide_many_jobs_per_cta():
    """More (instance, 32-column) jobs than SMs: 96 instances of K = 128 (4 jobs
    each) and 8 of K = 256 (8 jobs each), so each persistent CTA walks several
    jobs of different instances; every instance against the oracle."""
    a = [_inst(128, 512, 31 + i) for i in range(96)]
    b = [_inst(256, 768, 131 + i) for i in range(8)]
    Hs = [C.round_complex64(i.H) for i in a + b]
    xis = [i.xi for i in a + b]
    out = run(Hs, xis, T=4, precision="tf32x3")
    W, _, _, _, st = O.precode_batch(Hs, xis, "standard", max_iter=4)
    assert (out["status"] == 0).all()
    errs = [rel_fro(out["W"][i], W[i]) for i in range(len(Hs))]
    assert max(errs) <= TOL_W, (int(np.argmax(errs)), max(errs))


@pytest.mark.parametrize("n_rhs", [1, 5, 33, 64])
def test_wide_symbol_blocks(n_rhs):
    """Per-symbol right-hand sides (Eq. 16) on the 256 class: n_rhs below one
    CTA's 32 columns, a ragged second block, two full blocks; T = 6."""
    import torch
    from paper_2305_13925_gb300 import binding
    inst = _inst(200, 1024, 41, S=4, n_vis=(2, 4))
    H = C.round_complex64(inst.H)
    K, M = 200, 1024
    rng = np.random.default_rng(n_rhs)
    B = ((rng.standard_normal((K, n_rhs)) + 1j * rng.standard_normal((K, n_rhs))) / np.sqrt(2))
    B = B.astype(np.complex64).astype(np.complex128)
    ref = O.precode_symbols(H, inst.xi, B, "standard", max_iter=6)
    Hd = torch.from_numpy(np.ascontiguousarray(H.T).astype(np.complex64)).cuda()
    Bd = torch.from_numpy(np.ascontiguousarray(B.T).astype(np.complex64)).cuda()
    Wd = torch.zeros((n_rhs, M), dtype=torch.complex64, device="cuda")
    Xd = torch.zeros((n_rhs, K), dtype=torch.complex64, device="cuda")
    st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    with binding.Precoder(max_instances=1, max_M=M, max_K=256, precision="tf32x3") as prec:
        prec.precode([binding.instance(Hd, Wd, inst.xi, 6, X=Xd, B=Bd)], st)
        torch.cuda.synchronize()
    assert int(st.item()) == 0
    assert rel_fro(Xd.T.cpu().numpy().astype(np.complex128), ref["X"]) <= TOL_W
    assert rel_fro(Wd.T.cpu().numpy().astype(np.complex128), ref["S"]) <= TOL_W


def test_wide_warm_start_fixed_T():
    """Warm start from X0 (one extra product A X0 before the first update):
    equals the oracle started from the same X0, T = 4."""
    import torch
    from paper_2305_13925_gb300 import binding
    inst = _inst(256, 1024, 43, S=4, n_vis=(2, 4))
    H = C.round_complex64(inst.H)
    K, M = 256, 1024
    X0 = O.precode(H, inst.xi, "standard", max_iter=2)["X"].astype(np.complex64).astype(np.complex128)
    A = O.gram(H, inst.xi)
    Xr, _, _, _ = O.pcg(A, None, "standard", max_iter=4, X0=X0)
    Hd = torch.from_numpy(np.ascontiguousarray(H.T).astype(np.complex64)).cuda()
    X0d = torch.from_numpy(np.ascontiguousarray(X0.T).astype(np.complex64)).cuda()
    Wd = torch.zeros((K, M), dtype=torch.complex64, device="cuda")
    Xd = torch.zeros((K, K), dtype=torch.complex64, device="cuda")
    st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    with binding.Precoder(max_instances=1, max_M=M, max_K=K, precision="tf32x3") as prec:
        prec.precode([binding.instance(Hd, Wd, inst.xi, 4, X=Xd, X0=X0d)], st)
        torch.cuda.synchronize()
    assert int(st.item()) == 0
    assert rel_fro(Xd.T.cpu().numpy().astype(np.complex128), Xr) <= TOL_W


def test_wide_tolerance_and_refinement_reach_the_direct_rzf():
    """Tolerance 1e-5 with Dot2 refinement (stop at relative residual 1e-7):
    each W within 1e-5 of the direct RZF, on K = 128 and 256 channels,
    including a near-square one (M = 2K at 20 dB)."""
    insts = [_inst(128, 1024, 51), _inst(256, 2048, 52), _inst(256, 512, 53, snr=(20.0,))]
    Hs = [C.round_complex64(i.H) for i in insts]
    xis = [i.xi for i in insts]
    out = run(Hs, xis, T=1000, tol=1e-5, precision="tf32x3", refine_sweeps=3, refine_tol=1e-7,
              refine_solve_tol=1e-2)
    for i, (H, xi) in enumerate(zip(Hs, xis)):
        Wd = O.rzf_direct(H, xi)[0]
        assert out["status"][i] == 0, (i, out["status"][i])
        assert rel_fro(out["W"][i], Wd) <= TOL_W, (i, H.shape, rel_fro(out["W"][i], Wd))


def test_autotune_chooses_between_tensor_and_simt_paths():
    """With TF32X3 every class from 64 up has the tensor path as candidate -1
    next to the SIMT launch shapes: each choice stays within 1e-5 of the
    oracle, and the autotuner's table times every candidate and records the
    path it kept."""
    from paper_2305_13925_gb300 import binding
    insts = C.generate_ragged(9, 61, k_set=(64, 128, 256), m_set=(512, 1024))
    Hs = [C.round_complex64(i.H) for i in insts]
    xis = [i.xi for i in insts]
    refs = [O.precode(h, x, "standard", max_iter=5)["W"] for h, x in zip(Hs, xis)]
    prec = binding.Precoder(max_instances=9, max_M=1024, max_K=256, precision="tf32x3")
    try:
        for KC in (64, 128, 256):
            assert binding.jacpcg_get_shape(prec.ctx, KC)[0] == -1     # tensor path by default
        for sh in (-1, 0, 1):
            for KC in (64, 128, 256):
                binding.jacpcg_set_shape(prec.ctx, KC, sh)
            out = run(Hs, xis, T=5, prec=prec, precision="tf32x3")
            for k in range(len(Hs)):
                assert rel_fro(out["W"][k], refs[k]) <= TOL_W, (sh, k)
        import torch
        from gpu_util import to_dev
        Hd = [to_dev(h, torch) for h in Hs]
        Wd = [to_dev(np.zeros(h.shape), torch) for h in Hs]
        table = binding.jacpcg_autotune(prec.ctx, [binding.instance(Hd[k], Wd[k], xis[k], 5)
                                                   for k in range(len(Hs))])
        for KC in (64, 128, 256):
            e = table[str(KC)]
            n_simt = binding.jacpcg_get_shape(prec.ctx, KC)[1]
            assert len(e["ms_per_candidate"]) == n_simt + 1
            assert e["path"] == ("tensor" if e["shape"] == -1 else "simt")
        out = run(Hs, xis, T=5, prec=prec, precision="tf32x3")
        for k in range(len(Hs)):
            assert rel_fro(out["W"][k], refs[k]) <= TOL_W, k
    finally:
        prec.close()
