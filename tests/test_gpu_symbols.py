"""GPU parity of the per-symbol right-hand-side form (Eqs. 15-16) and of the
warm start (initial point w^0, Sec. III-B Step 1) against the FP64 oracle,
through the C ABI: W = H X for a block B of symbol vectors, X = P^{-1} B by
the iteration, beta normalising the block's mean transmit power."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2305_13925_gb300 import channels as C

from gpu_util import rel_fro, to_dev

pytestmark = pytest.mark.gpu

TOL_W = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_13925_gb300 import build
    build.build()


def _channel(M, K, seed):
    spec = C.ChannelSpec(M=M, S=1, K=K, r=(0.5, 0.5), n_vis=(1, 1), snr_db=(10.0,))
    inst = C.generate_instance(spec, seed, K + M)
    return C.round_complex64(inst.H), inst.xi


def _symbols(K, n, seed):
    rng = np.random.default_rng(seed)
    qpsk = (rng.integers(0, 2, (K, n)) * 2 - 1 + 1j * (rng.integers(0, 2, (K, n)) * 2 - 1)) / np.sqrt(2)
    return qpsk.astype(np.complex64).astype(np.complex128)


def run_symbols(Hs, xis, Bs, X0s=None, T=6, tol=0.0, precision="fp32", variant="standard",
                refine_sweeps=0, power=1.0):
    """Bs[i]: K x n_i symbol block or None (B = I); X0s[i]: K x n_i start or None."""
    import torch
    from paper_2305_13925_gb300 import binding
    n = len(Hs)
    X0s = X0s or [None] * n
    Hd = [to_dev(h, torch) for h in Hs]
    ncol = [h.shape[1] if b is None else b.shape[1] for h, b in zip(Hs, Bs)]
    Wd = [to_dev(np.full((h.shape[0], c), np.nan, dtype=np.complex128), torch) for h, c in zip(Hs, ncol)]
    Xd = [torch.zeros((c, h.shape[1]), dtype=torch.complex64, device="cuda") for h, c in zip(Hs, ncol)]
    Bd = [None if b is None else torch.from_numpy(np.ascontiguousarray(b.T).astype(np.complex64)).cuda()
          for b in Bs]
    X0d = [None if x is None else torch.from_numpy(np.ascontiguousarray(x.T).astype(np.complex64)).cuda()
           for x in X0s]
    insts = [binding.instance(Hd[i], Wd[i], xis[i], T, tol, power, X=Xd[i], B=Bd[i], X0=X0d[i])
             for i in range(n)]
    status = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    iters = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    resid = torch.full((n,), -1.0, dtype=torch.float32, device="cuda")
    beta = torch.full((n,), -1.0, dtype=torch.float32, device="cuda")
    with binding.Precoder(max_instances=n, max_M=max(h.shape[0] for h in Hs),
                          max_K=max(h.shape[1] for h in Hs), variant=variant, precision=precision,
                          refine_sweeps=refine_sweeps) as prec:
        prec.precode(insts, status, iters, resid, beta)
        torch.cuda.synchronize()
    return dict(W=[w.T.cpu().numpy().astype(np.complex128) for w in Wd],
                X=[x.T.cpu().numpy().astype(np.complex128) for x in Xd],
                status=status.cpu().numpy(), iters=iters.cpu().numpy(),
                resid=resid.cpu().numpy(), beta=beta.cpu().numpy())


@pytest.mark.parametrize("precision", ["fp32", "tf32x3"])
@pytest.mark.parametrize("K,M,n", [(5, 40, 1), (16, 256, 3), (64, 1024, 14), (64, 1024, 64),
                                   (48, 300, 7), (100, 512, 20), (200, 700, 256)])
def test_symbol_blocks_fixed_T(precision, K, M, n):
    H, xi = _channel(M, K, 31)
    B = _symbols(K, n, 32)
    out = run_symbols([H], [xi], [B], T=6, precision=precision, power=2.0)
    ref = O.precode_symbols(H, xi, B, "standard", max_iter=6, power=2.0)
    assert out["status"][0] == 0
    assert rel_fro(out["W"][0], ref["S"]) <= TOL_W
    assert rel_fro(out["X"][0], ref["X"]) <= TOL_W
    assert abs(out["beta"][0] - ref["beta"]) <= 1e-5 * ref["beta"]
    assert out["iters"][0] == 6


@pytest.mark.parametrize("precision", ["fp32", "tf32x3"])
@pytest.mark.parametrize("K,M", [(16, 256), (64, 1024), (128, 640)])
def test_warm_start_tolerance(precision, K, M):
    """Slot-to-slot: start from the solution for a perturbed channel; the
    warm solve stops sooner than the cold one and both reach the direct
    solution; the iteration count matches the oracle's."""
    H, xi = _channel(M, K, 33)
    rng = np.random.default_rng(34)
    Hp = C.round_complex64(H + 0.02 * (rng.standard_normal(H.shape) + 1j * rng.standard_normal(H.shape)))
    B = _symbols(K, 12, 35)
    X0 = O.precode_symbols(Hp, xi, B, "standard", max_iter=400, tol=1e-10)["X"]
    X0 = X0.astype(np.complex64).astype(np.complex128)
    cold = run_symbols([H], [xi], [B], T=300, tol=1e-6, precision=precision)
    warm = run_symbols([H], [xi], [B], [X0], T=300, tol=1e-6, precision=precision)
    S_direct = H @ np.linalg.solve(H.conj().T @ H + xi * np.eye(K), B)
    for out in (cold, warm):
        assert out["status"][0] == 0
        assert rel_fro(out["W"][0], S_direct) <= 1e-5
        assert out["resid"][0] <= 1e-6
    assert warm["iters"][0] < cold["iters"][0]
    ref = O.precode_symbols(H, xi, B, "standard", max_iter=300, tol=1e-6, X0=X0)
    assert abs(int(warm["iters"][0]) - ref["iters"]) <= 2


@pytest.mark.parametrize("precision", ["fp32", "tf32x3"])
def test_warm_start_fixed_T_matches_oracle(precision):
    """Fixed T from a start at the solution's scale (the solution with 30 %
    random perturbations, as a previous slot's X would be), B = I and
    B = symbols, against the oracle started from the same point.  (A start
    far larger than the solution makes X = X0 + E cancel in FP32; that is a
    property of the start, not of the kernels.)"""
    H, xi = _channel(1024, 64, 36)
    rng = np.random.default_rng(37)
    Bs = [None, _symbols(64, 9, 38)]
    A = H.conj().T @ H + xi * np.eye(64)
    X0s = []
    for b in Bs:
        Bm = np.eye(64) if b is None else b
        Xs = np.linalg.solve(A, Bm)
        noise = rng.standard_normal(Xs.shape) + 1j * rng.standard_normal(Xs.shape)
        X0s.append((Xs * (1 + 0.3 * noise)).astype(np.complex64).astype(np.complex128))
    out = run_symbols([H, H], [xi, xi], Bs, X0s, T=5, precision=precision)
    for i, b in enumerate(Bs):
        Bm = np.eye(64) if b is None else b
        ref = O.precode_symbols(H, xi, Bm, "standard", max_iter=5, X0=X0s[i])
        assert out["status"][i] == 0
        assert rel_fro(out["W"][i], ref["S"]) <= TOL_W, i


def test_mixed_batch_and_refinement():
    """One call mixing B = I, symbol blocks and warm starts over several K
    classes, with two Dot2 refinement sweeps: every W within 1e-6 of the
    direct solution."""
    specs = [(16, 200), (64, 1024), (40, 512), (128, 600), (8, 100)]
    Hs, xis, Bs, X0s = [], [], [], []
    for t, (K, M) in enumerate(specs):
        H, xi = _channel(M, K, 40 + t)
        Hs.append(H)
        xis.append(xi)
        Bs.append(None if t % 2 == 0 else _symbols(K, 3 + t, 50 + t))
        n = K if Bs[-1] is None else Bs[-1].shape[1]
        X0s.append(None if t % 3 else np.zeros((K, n)))
    out = run_symbols(Hs, xis, Bs, X0s, T=8, tol=1e-6, refine_sweeps=2)
    for i, H in enumerate(Hs):
        K = H.shape[1]
        Bm = np.eye(K) if Bs[i] is None else Bs[i]
        S_direct = H @ np.linalg.solve(H.conj().T @ H + xis[i] * np.eye(K), Bm)
        assert rel_fro(out["W"][i], S_direct) <= 1e-6, i


def test_invalid_right_hand_sides_rejected():
    """n_rhs outside 1 .. K class, ldb < K, or a misaligned B: EINVAL, and
    nothing runs."""
    import torch
    from paper_2305_13925_gb300 import binding
    H, xi = _channel(64, 16, 60)
    Hd = to_dev(H, torch)
    Wd = torch.empty((17, 64), dtype=torch.complex64, device="cuda")
    B = torch.zeros((3, 16), dtype=torch.complex64, device="cuda")
    Bbig = torch.zeros((17, 16), dtype=torch.complex64, device="cuda")   # n_rhs > K class 16
    bad = [binding.instance(Hd, Wd, xi, 4, B=Bbig)]
    q = binding.instance(Hd, Wd, xi, 4, B=B)
    q.n_rhs = 0
    bad.append(q)
    q = binding.instance(Hd, Wd, xi, 4, B=B)
    q.ldb = 15
    bad.append(q)
    q = binding.instance(Hd, Wd, xi, 4, B=B)
    q.B = q.B + 8
    bad.append(q)
    q = binding.instance(Hd, Wd, xi, 4, B=B)
    q.X0 = B.data_ptr() + 8
    bad.append(q)
    with binding.Precoder(max_instances=1, max_M=64, max_K=16) as prec:
        for q in bad:
            with pytest.raises(binding.JacpcgError) as e:
                prec.precode([q])
            assert e.value.status == binding.JACPCG_EINVAL
