"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs, element by element.  Bar: relative Frobenius error
of W at most 1e-5 per instance (FP32 arithmetic); A, X and beta are checked
alongside.  Marked gpu."""
import math

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


def fp32_deviation(H, xi, variant, T):
    """Relative distance between the FP64 oracle's W and an independent
    complex64 (numpy) evaluation of the same fixed-T iteration: how far any
    FP32 evaluation of this iteration drifts from exact arithmetic on this
    channel (for plain CG and the literal Algorithm 1 the finite-precision
    loss of conjugacy makes this far larger than rounding of the inputs)."""
    c = np.complex64
    Hc = H.astype(c)
    A = Hc.conj().T @ Hc + c(xi) * np.eye(H.shape[1], dtype=c)
    d = np.real(np.diag(A)).astype(np.float32)
    dinv = (np.float32(1) / d) if variant != "cg" else np.ones_like(d)
    K = H.shape[1]
    X = np.zeros((K, K), dtype=c)
    for j in range(K):
        b = np.zeros(K, dtype=c)
        b[j] = 1
        x = np.zeros(K, dtype=c)
        if variant == "alg1":
            r = dinv * b
            m = r.copy()
            rr = np.vdot(r, r).real
            for _ in range(T):
                u = dinv * (A @ m)
                den = np.vdot(m, u)
                al = c(rr / den) if den != 0 else c(0)
                x = x + al * m
                r = r - al * u
                rn = np.vdot(r, r).real
                m = r + np.float32(rn / rr if rr != 0 else 0) * m
                rr = rn
        else:
            r = b.copy()
            z = dinv * r
            p = z.copy()
            rz = np.vdot(r, z).real
            for _ in range(T):
                q = A @ p
                pq = np.vdot(p, q).real
                lam = np.float32(rz / pq) if pq > 0 else np.float32(0)
                x = x + lam * p
                r = r - lam * q
                z = dinv * r
                rzn = np.vdot(r, z).real
                p = z + np.float32(rzn / rz if rz != 0 else 0) * p
                rz = rzn
        X[:, j] = x
    W32 = Hc @ X
    ref = O.precode(H, xi, variant, max_iter=T)["W"]
    return rel_fro(W32.astype(np.complex128), ref)


def tol_for(H, xi, variant, T):
    """Parity bar for W: 1e-5 for Jacobi-PCG (the method); for plain CG and
    the literal Algorithm 1 the larger of 1e-5 and 30 x the drift of an
    independent FP32 evaluation of the same iteration from the oracle."""
    if variant == "standard":
        return TOL_W
    return max(TOL_W, 30.0 * fp32_deviation(H, xi, variant, T))


def check_batch(Hs, xis, variant="standard", T=6, tol_w=None, **kw):
    Hs = [C.round_complex64(h) for h in Hs]      # the oracle sees exactly what the GPU reads
    out = run(Hs, xis, variant=variant, T=T, want_X=True, want_A=True, **kw)
    errs = []
    for i, (H, xi) in enumerate(zip(Hs, xis)):
        ref = O.precode(H, xi, variant, max_iter=T)
        e = rel_fro(out["W"][i], ref["W"])
        errs.append(e)
        bar = tol_w if tol_w is not None else tol_for(H, xi, variant, T)
        assert e <= bar, (i, H.shape, e, bar)
        assert rel_fro(out["A"][i], ref["A"]) <= 1e-6
        assert rel_fro(out["X"][i], ref["X"]) <= bar
        # beta = sqrt(P) / ||W||_F: its relative error is at most W's
        assert abs(out["beta"][i] - ref["beta"]) <= max(1e-5, bar) * ref["beta"]
        assert out["iters"][i] == ref["iters"]
        assert out["status"][i] == 0
    return out, errs


def test_single_256x16_T8():
    """Single instance: M = 256 (4 subarrays of 64), K = 16, r = 0.5, 2 of 4
    subarrays visible, SNR 10 dB, xi = K / SNR, 8 iterations."""
    inst = C.generate_instance(C.PRESETS["single_256x16"], 0, 0)
    out, errs = check_batch([inst.H], [inst.xi], T=8)
    # and close to the direct RZF
    Wd, _, _ = O.rzf_direct(inst.H, inst.xi)
    assert rel_fro(out["W"][0], Wd) < 1e-3


@pytest.mark.parametrize("variant", ["standard", "cg"])
def test_batched_1024x64_T6_subset(variant):
    """Uniform batch shape M = 1024 (8 subarrays of 128), K = 64, T = 6, on 24 instances."""
    H, xi = C.generate_batch("batched_1024x64", 24, 1)
    out, errs = check_batch(list(H), list(xi), variant=variant, T=6)
    if variant == "standard":
        assert max(errs) <= TOL_W


@pytest.mark.parametrize("precision", ["fp32", "tf32x3"])
def test_batched_1024x64_full_batch(precision):
    """The bench's launch configuration: all 2048 instances of the batched
    shape in one call (each persistent CTA walks 13-14 of them), T = 6; every
    instance checked against the oracle (run on all host threads), so that an
    error confined to some positions of a CTA's walk cannot hide."""
    import torch
    from paper_2305_13925_gb300 import binding
    Hst, xi = C.generate_batch_device_layout("batched_1024x64", 2048, 1)
    Hd = torch.from_numpy(Hst).cuda()
    Wd = torch.empty_like(Hd)
    status = torch.empty(2048, dtype=torch.int32, device="cuda")
    with binding.Precoder(max_instances=2048, max_M=1024, max_K=64, precision=precision) as prec:
        insts = [binding.instance(Hd[i], Wd[i], float(xi[i]), 6) for i in range(2048)]
        prec.precode(insts, status)
        torch.cuda.synchronize()
    assert (status.cpu().numpy() == 0).all()
    Hs = [Hst[i].T for i in range(2048)]
    refs = O.precode_batch(Hs, xi, "standard", max_iter=6)[0]
    W = Wd.cpu().numpy()
    errs = [rel_fro(W[i].T.astype(np.complex128), refs[i]) for i in range(2048)]
    worst = int(np.argmax(errs))
    assert errs[worst] <= TOL_W, (worst, errs[worst])


def test_alg1_variant_parity():
    """Algorithm 1 as printed, on channels with a mild diagonal spread
    (equal column norms make D = cI, where it is well behaved)."""
    H, xi = C.generate_batch("single_256x16", 6, 5)
    Hn = [h / np.maximum(np.linalg.norm(h, axis=0), 1e-30)[None, :] for h in H]
    check_batch(Hn, list(xi), variant="alg1", T=8)


@pytest.mark.parametrize("preset,n,seed,Ts,precision", [
    ("single_256x16", 6, 5, (2, 3), "fp32"),
    ("batched_1024x64", 4, 1, (2, 4), "tf32x3"),
])
def test_alg1_variant_parity_complex_step(preset, n, seed, Ts, precision):
    """Algorithm 1 on the channels as generated: shadowing spreads the diagonal
    of P over one to three decades, so C^{-1} P is not Hermitian and every step
    alpha is complex.  Element by element against the oracle at T = 2..4, before
    the printed iteration drifts; the bar (at most 2e-3 here) is far below the
    distance (>= 1.7e-2 on these channels) of an evaluation whose step
    denominator is conjugated."""
    H, xi = C.generate_batch(preset, n, seed)
    for h, x in zip(H, xi):
        d = np.real(np.diag(O.gram(C.round_complex64(h), x)))
        assert d.max() > 20 * d.min()
    for T in Ts:
        bars = [tol_for(C.round_complex64(h), x, "alg1", T) for h, x in zip(H, xi)]
        assert max(bars) <= 2e-3, bars
        check_batch(list(H), list(xi), variant="alg1", T=T, precision=precision)


@pytest.mark.parametrize("K,M", [(1, 64), (2, 9), (3, 130), (8, 256), (17, 1000), (33, 96),
                                 (64, 257), (100, 512), (128, 640), (200, 700), (256, 1024)])
def test_ragged_shapes_and_tails(K, M):
    """K classes 8..256 with K not a power of two, M not a multiple of the
    64-row tile, and tiny K; standard variant, T = 5."""
    spec = C.ChannelSpec(M=M, S=1, K=K, r=(0.5, 0.5), n_vis=(1, 1), snr_db=(10.0,))
    inst = C.generate_instance(spec, 7, K + M)
    check_batch([inst.H], [inst.xi], T=5)


def test_ragged_batch_one_launch_sequence():
    """A ragged batch (every K class, several M) in one call matches each
    instance's oracle."""
    insts = C.generate_ragged(12, 3, k_set=(8, 16, 32, 64, 128, 256), m_set=(256, 512, 1024))
    check_batch([i.H for i in insts], [i.xi for i in insts], T=4)


def test_more_users_than_antennas_with_regulariser():
    """K > M is admissible when xi > 0 (A = H^H H + xi I stays HPD, Eq. 18)."""
    rng = np.random.default_rng(3)
    H = (rng.standard_normal((24, 40)) + 1j * rng.standard_normal((24, 40))) / math.sqrt(2)
    H = C.round_complex64(H)
    check_batch([H], [2.0], T=6)


def test_diagonal_gram_exact_in_one_step():
    """Orthogonal columns of unequal norm: A is diagonal and one Jac-PCG step
    gives X = D^{-1} exactly (up to FP32 rounding)."""
    M, K = 64, 8
    m = np.arange(M)[:, None]
    k = np.arange(K)[None, :]
    H = np.exp(-2j * np.pi * m * k / M) / math.sqrt(M) * np.geomspace(0.5, 4.0, K)[None, :]
    H = C.round_complex64(H)
    out = run([H], [0.3], T=3, want_X=True)
    ref = O.precode(H, 0.3, "standard", max_iter=1)
    assert rel_fro(out["X"][0], ref["X"]) < 1e-6
    assert out["iters"][0] == 3 and out["status"][0] == 0


def test_tolerance_mode_reaches_direct_rzf():
    """tol > 0: columns stop at ||r|| <= tol; the result is close to the
    direct RZF, iteration counts are near the oracle's and status is OK."""
    H, xi = C.generate_batch("batched_1024x64", 8, 11)
    out = run(list(H), list(xi), T=200, tol=1e-6)
    for i in range(8):
        Wd, _, _ = O.rzf_direct(H[i], xi[i])
        assert rel_fro(out["W"][i], Wd) < 1e-5
        ref = O.precode(H[i], xi[i], "standard", max_iter=200, tol=1e-6)
        assert abs(int(out["iters"][i]) - ref["iters"]) <= 2
        assert out["status"][i] == 0 and out["resid"][i] <= 1e-6


def test_not_converged_status():
    """A tolerance that cannot be met in max_iter reports ENOTCONV, and the
    result is still the max_iter iterate."""
    H, xi = C.generate_batch("batched_1024x64", 2, 12)
    out = run(list(H), list(xi), T=2, tol=1e-9)
    assert list(out["status"]) == [4, 4]
    for i in range(2):
        ref = O.precode(H[i], xi[i], "standard", max_iter=2)
        assert rel_fro(out["W"][i], ref["W"]) <= TOL_W


def test_nonfinite_input_reported():
    H, xi = C.generate_batch("single_256x16", 2, 13)
    H = H.copy()
    H[1][5, 3] = np.nan
    out = run(list(H), list(xi), T=4)
    assert out["status"][0] == 0 and out["status"][1] == 6


def test_zero_user_channel():
    """A user with no visible subarray (zero column): A_kk = xi, and that
    user's column of X is e_k / xi."""
    inst = C.generate_instance(C.PRESETS["single_256x16"], 0, 4)
    H = inst.H.copy()
    H[:, 5] = 0
    out = run([H], [inst.xi], T=8, want_X=True)
    ref = O.precode(H, inst.xi, "standard", max_iter=8)
    assert rel_fro(out["W"][0], ref["W"]) <= TOL_W
    assert abs(out["X"][0][5, 5] - 1.0 / inst.xi) < 1e-6 / inst.xi


def test_plan_and_graph_replay_bitwise_equal():
    """A plan executed directly, replayed from a CUDA graph, and a one-shot
    precode call give bit-identical W."""
    H, xi = C.generate_batch("batched_1024x64", 16, 21)
    a = run(list(H), list(xi), T=6)
    b = run(list(H), list(xi), T=6, plan=True, graph=False, repeats=2)
    c = run(list(H), list(xi), T=6, plan=True, graph=True, repeats=3)
    for i in range(16):
        assert np.array_equal(a["W"][i], b["W"][i]) and np.array_equal(a["W"][i], c["W"][i])


def test_result_alone_equals_result_in_mix():
    """Batch composition does not change any instance's bits (fixed reduction
    order per instance, no cross-instance arithmetic)."""
    insts = C.generate_ragged(10, 31, k_set=(16, 64, 128), m_set=(256, 1024))
    mix = run([i.H for i in insts], [i.xi for i in insts], T=5)
    for j in (0, 3, 7):
        alone = run([insts[j].H], [insts[j].xi], T=5)
        assert np.array_equal(alone["W"][0], mix["W"][j])
        assert alone["beta"][0] == mix["beta"][j]


def test_invalid_arguments_rejected():
    import torch
    from paper_2305_13925_gb300 import binding
    with pytest.raises(binding.JacpcgError):
        binding.Precoder(max_instances=1, max_M=64, max_K=300)
    prec = binding.Precoder(max_instances=2, max_M=128, max_K=16)
    try:
        H = torch.zeros((16, 128), dtype=torch.complex64, device="cuda")
        W = torch.zeros_like(H)
        good = binding.instance(H, W, 1.0, 4)
        for field, val in (("K", 0), ("K", 17), ("M", 129), ("ldh", 64), ("xi", -1.0),
                           ("max_iter", -1), ("ldw", 127)):
            bad = binding.instance(H, W, 1.0, 4)
            setattr(bad, field, val)
            with pytest.raises(binding.JacpcgError) as e:
                prec.precode([bad])
            assert e.value.status == binding.JACPCG_EINVAL
        bad = binding.instance(H, W, 1.0, 4)
        bad.H = H.data_ptr() + 8
        with pytest.raises(binding.JacpcgError):
            prec.precode([bad])
        with pytest.raises(binding.JacpcgError):
            prec.precode([good, good, good])       # more than max_instances
        prec.precode([good])                        # the context is still usable
        torch.cuda.synchronize()
    finally:
        prec.close()


def test_every_launch_shape_bit_identical_and_autotune():
    """Each candidate launch shape of the iteration kernel gives the same bits
    (the per-column arithmetic does not depend on the shape); the autotuned
    context keeps parity with the oracle."""
    import torch
    from paper_2305_13925_gb300 import binding
    insts = C.generate_ragged(12, 91, k_set=(8, 16, 32, 64, 128, 256), m_set=(256, 512))
    Hs = [C.round_complex64(i.H) for i in insts]
    xis = [i.xi for i in insts]
    base = run(Hs, xis, T=5)
    prec = binding.Precoder(max_instances=12, max_M=512, max_K=256)
    try:
        for KC in (8, 16, 32, 64, 128, 256):
            n_shapes = binding.jacpcg_get_shape(prec.ctx, KC)[1]
            for sh in range(1, n_shapes):
                binding.jacpcg_set_shape(prec.ctx, KC, sh)
                out = run(Hs, xis, T=5, prec=prec)
                for k in range(len(Hs)):
                    assert np.array_equal(out["W"][k], base["W"][k]), (KC, sh, k)
            binding.jacpcg_set_shape(prec.ctx, KC, 0)
    except Exception:
        prec.close()
        raise
    from gpu_util import to_dev
    Hd = [to_dev(h, torch) for h in Hs]
    Wd = [to_dev(np.zeros(h.shape), torch) for h in Hs]
    table = binding.jacpcg_autotune(prec.ctx, [binding.instance(Hd[k], Wd[k], xis[k], 5)
                                               for k in range(len(Hs))])
    present = {str(1 << max(3, (int(h.shape[1]) - 1).bit_length())) for h in Hs}
    assert set(table) == present
    tuned = run(Hs, xis, T=5, prec=prec)
    prec.close()
    for k in range(len(Hs)):
        assert np.array_equal(tuned["W"][k], base["W"][k])


def test_empty_batch_is_a_no_op():
    """n_inst = 0: JACPCG_OK, nothing enqueued (the output arrays keep their
    contents); the context stays usable."""
    import torch
    from paper_2305_13925_gb300 import binding
    prec = binding.Precoder(max_instances=4, max_M=64, max_K=8)
    try:
        st = torch.full((4,), 77, dtype=torch.int32, device="cuda")
        prec.precode([], st)
        torch.cuda.synchronize()
        assert (st == 77).all()
    finally:
        prec.close()


@pytest.mark.parametrize("precision", ["fp32", "tf32x3"])
def test_zero_iterations(precision):
    """T = 0 (the degenerate schedule): X stays 0, so W = H X is exactly zero,
    iters 0, status OK, and beta (undefined for W = 0) is reported as 0;
    K = 64 (tensor classes) and K = 17 (SIMT) in one batch."""
    H1, x1 = C.generate_batch("batched_1024x64", 1, 3)
    spec = C.ChannelSpec(M=256, S=4, K=17, r=(0.5, 0.5), n_vis=(2, 3), snr_db=(10.0,))
    i2 = C.generate_instance(spec, 3, 17)
    out = run([H1[0], i2.H], [x1[0], i2.xi], T=0, precision=precision)
    for k in range(2):
        assert not np.any(out["W"][k]), k
        assert out["status"][k] == 0 and out["iters"][k] == 0 and out["beta"][k] == 0.0
        ref = O.precode(C.round_complex64([H1[0], i2.H][k]), [x1[0], i2.xi][k], "standard", max_iter=0)
        assert not np.any(ref["W"])



@pytest.mark.parametrize("precision", ["fp32", "tf32x3"])
def test_output_guards_untouched(precision):
    """Canary padding: W (ldw > M), X and A sit inside buffers filled with a
    sentinel; after the call every byte outside the outputs' M x K (K x K)
    regions -- guards before and after, rows M .. ldw - 1 of each W column --
    still holds the sentinel, and the outputs match the oracle.  K = 17
    (SIMT), 64 and 100 (tensor classes), M = 300 (not a tile multiple)."""
    import torch
    from paper_2305_13925_gb300 import binding
    from gpu_util import to_dev
    sent = complex(1234.5, -6789.25)
    G = 64                                          # guard entries (512 bytes) on each side
    M = 300
    cases = []
    for K, seed in ((17, 31), (64, 32), (100, 33)):
        spec = C.ChannelSpec(M=M, S=4, K=K, r=(0.5, 0.5), n_vis=(2, 3), snr_db=(10.0,))
        inst = C.generate_instance(spec, seed, K)
        ldw = M + 6
        Wb = torch.full((2 * G + K * ldw,), sent, dtype=torch.complex64, device="cuda")
        Xb = torch.full((2 * G + K * K,), sent, dtype=torch.complex64, device="cuda")
        Ab = torch.full((2 * G + K * K,), sent, dtype=torch.complex64, device="cuda")
        W = Wb[G:G + K * ldw].view(K, ldw)[:, :M]
        X = Xb[G:G + K * K].view(K, K)
        A = Ab[G:G + K * K].view(K, K)
        cases.append((inst, to_dev(inst.H, torch), W, X, A, Wb, Xb, Ab, ldw))
    prec = binding.Precoder(max_instances=3, max_M=M, max_K=100, precision=precision)
    try:
        descs = [binding.instance(c[1], c[2], c[0].xi, 6, X=c[3], A=c[4]) for c in cases]
        st = torch.full((3,), -1, dtype=torch.int32, device="cuda")
        prec.precode(descs, st)
        torch.cuda.synchronize()
    finally:
        prec.close()
    assert (st == 0).all()
    for inst, _, W, X, A, Wb, Xb, Ab, ldw in cases:
        K = inst.H.shape[1]
        wb = Wb.cpu().numpy()
        assert np.all(wb[:G] == sent) and np.all(wb[G + K * ldw:] == sent)
        assert np.all(wb[G:G + K * ldw].reshape(K, ldw)[:, M:] == sent)
        for b, n in ((Xb.cpu().numpy(), K * K), (Ab.cpu().numpy(), K * K)):
            assert np.all(b[:G] == sent) and np.all(b[G + n:] == sent)
        ref = O.precode(C.round_complex64(inst.H), inst.xi, "standard", max_iter=6)
        assert rel_fro(W.T.cpu().numpy().astype(np.complex128), ref["W"]) <= 1e-5, K


@pytest.mark.parametrize("K", [17, 64])
def test_extreme_column_norms(K):
    """User channels scaled by amplitudes from 1e-3 to 1e3 (a dynamic range of
    1e12 on the diagonal of A): the Jacobi scaling keeps the iteration
    well-posed and W matches the oracle at fixed T within 1e-5 on both
    precisions."""
    spec = C.ChannelSpec(M=512, S=4, K=K, r=(0.5, 0.5), n_vis=(2, 3), snr_db=(10.0,))
    inst = C.generate_instance(spec, 41, K)
    scale = 10.0 ** np.linspace(-3.0, 3.0, K)
    H = (inst.H * scale[None, :]).astype(np.complex64).astype(np.complex128)
    xi = inst.xi * 1e-6
    ref = O.precode(H, xi, "standard", max_iter=6)
    for precision in ("fp32", "tf32x3"):
        out = run([H], [xi], T=6, precision=precision)
        assert out["status"][0] == 0
        e = rel_fro(out["W"][0], ref["W"])
        assert e <= 1e-5, (precision, e)
