"""Python face of the FP64 CPU oracle (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline and
reference legs of ``bench.py`` may import this module.  The product package
never imports it, and it imports nothing from the product package.

The arithmetic lives in ``jacpcg_oracle.c`` (plain loops, FP64, one
function per passage of arXiv 2305.13925); this file only marshals numpy
arrays through ctypes and adds the paper's operation counts (Appendix),
which are closed-form formulas.

Array conventions: matrices are numpy complex128 in math shape (rows, cols);
they are converted to column-major (Fortran) order before every call.
"""
from __future__ import annotations

import ctypes
import os
import pathlib
import subprocess
import threading

import numpy as np

HERE = pathlib.Path(__file__).resolve().parent
SRC = HERE / "jacpcg_oracle.c"
LIB = HERE / "_build" / "libjacpcg_oracle.so"

STANDARD, ALG1, CG, JOR, GS = 0, 1, 2, 3, 4
VARIANTS = {"standard": STANDARD, "alg1": ALG1, "cg": CG, "jor": JOR, "gs": GS}
STATIONARY = (JOR, GS)
OK, BREAKDOWN, NOMEM, NOTHPD = 0, 1, 2, 3

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> pathlib.Path:
    """Compile the oracle with gcc (plain C99, no contraction of a*b+c)."""
    LIB.parent.mkdir(exist_ok=True)
    if force or not LIB.exists() or LIB.stat().st_mtime < SRC.stat().st_mtime:
        tmp = LIB.with_suffix(f".{os.getpid()}.tmp")
        subprocess.check_call(["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                               "-pthread", "-o", str(tmp), str(SRC), "-lm"])
        os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(str(LIB))
            P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
            L.orc_gram.argtypes = [I, I, P, I, D, P]
            L.orc_gram.restype = None
            L.orc_pcg.argtypes = [I, P, P, I, I, I, I, D, P, I, P, I, P, P]
            L.orc_pcg.restype = I
            L.orc_stationary.argtypes = [I, P, P, I, I, I, D, I, D, P, I, P, I, P, P]
            L.orc_stationary.restype = I
            L.orc_matmul.argtypes = [I, I, I, P, I, P, I, P, I]
            L.orc_matmul.restype = None
            L.orc_power_factor.argtypes = [I, I, P, I, D]
            L.orc_power_factor.restype = D
            L.orc_cholesky_solve.argtypes = [I, P, P, I, I, P, I]
            L.orc_cholesky_solve.restype = I
            L.orc_sinr.argtypes = [I, I, P, I, P, I, D, P]
            L.orc_sinr.restype = None
            L.orc_precode.argtypes = [I, I, P, I, D, I, I, D, D, P, I, P, P, P, P, P]
            L.orc_precode.restype = I
            L.orc_precode_batch.argtypes = [I, P, P, P, P, P, I, I, D, D, P, P, P, P, P, P, I]
            L.orc_precode_batch.restype = I
            _lib = L
    return _lib


def _f(a) -> np.ndarray:
    return np.asfortranarray(np.asarray(a, dtype=np.complex128))


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _variant(v) -> int:
    return VARIANTS[v] if isinstance(v, str) else int(v)


def gram(H: np.ndarray, xi: float) -> np.ndarray:
    """A = H^H H + xi I (Sec. II after Eq. 7)."""
    Hf = _f(H)
    M, K = Hf.shape
    A = np.zeros((K, K), dtype=np.complex128, order="F")
    lib().orc_gram(M, K, _p(Hf), M, float(xi), _p(A))
    return np.ascontiguousarray(A)


def pcg(A: np.ndarray, B: np.ndarray | None = None, variant="standard", max_iter: int = 8,
        tol: float = 0.0, X0: np.ndarray | None = None, omega: float = 1.0):
    """Solve A X = B (B = None for the identity) with the chosen iteration,
    starting from X0 (None: zero) in every column.  The Krylov forms
    ("standard", "alg1", "cg") are Sec. III-B's; "jor" and "gs" are the
    stationary iterations of Sec. III-A (omega: JOR's relaxation factor).

    Returns (X, iters per column, relative residual per column, status): the
    recurrence residual for the Krylov forms, the true residual for JOR / GS.
    """
    Af = _f(A)
    K = Af.shape[0]
    if B is None:
        nrhs, Bp, ldb = K, None, K
        Bf = None
    else:
        Bf = _f(B.reshape(K, -1))
        nrhs, ldb = Bf.shape[1], K
        Bp = _p(Bf)
    X0f = None if X0 is None else _f(np.asarray(X0).reshape(K, nrhs))
    X = np.zeros((K, nrhs), dtype=np.complex128, order="F")
    it = np.zeros(nrhs, dtype=np.int32)
    rr = np.zeros(nrhs, dtype=np.float64)
    v = _variant(variant)
    x0p = None if X0f is None else _p(X0f)
    if v in STATIONARY:
        st = lib().orc_stationary(K, _p(Af), Bp, ldb, nrhs, v, float(omega), int(max_iter),
                                  float(tol), x0p, K, _p(X), K, _p(it), _p(rr))
    else:
        st = lib().orc_pcg(K, _p(Af), Bp, ldb, nrhs, v, int(max_iter), float(tol), x0p, K, _p(X),
                           K, _p(it), _p(rr))
    return np.ascontiguousarray(X), it, rr, st


def matmul(H: np.ndarray, X: np.ndarray) -> np.ndarray:
    """W = H X (Eq. 15 / Eq. 7 without the power factor)."""
    Hf, Xf = _f(H), _f(X)
    M, K = Hf.shape
    N = Xf.shape[1]
    W = np.zeros((M, N), dtype=np.complex128, order="F")
    lib().orc_matmul(M, K, N, _p(Hf), M, _p(Xf), K, _p(W), M)
    return np.ascontiguousarray(W)


def power_factor(W: np.ndarray, power: float = 1.0) -> float:
    """beta = sqrt(P / tr(W^H W)) (Sec. II after Eq. 7)."""
    Wf = _f(W)
    return lib().orc_power_factor(Wf.shape[0], Wf.shape[1], _p(Wf), Wf.shape[0], float(power))


def cholesky_solve(A: np.ndarray, B: np.ndarray | None = None):
    """Direct inversion of the Appendix: X = A^{-1} B via A = L L^H."""
    Af = _f(A)
    K = Af.shape[0]
    if B is None:
        nrhs, Bp = K, None
    else:
        Bf = _f(B.reshape(K, -1))
        nrhs, Bp = Bf.shape[1], _p(Bf)
    X = np.zeros((K, nrhs), dtype=np.complex128, order="F")
    st = lib().orc_cholesky_solve(K, _p(Af), Bp, K, nrhs, _p(X), K)
    return np.ascontiguousarray(X), st


def rzf_direct(H: np.ndarray, xi: float):
    """Exact RZF by direct inversion: returns (W_chol, X_chol, status)."""
    A = gram(H, xi)
    X, st = cholesky_solve(A)
    return matmul(H, X), X, st


def sinr(H: np.ndarray, G: np.ndarray, sigma2: float = 1.0) -> np.ndarray:
    """Per-user SINR of Eq. 9 (centralised form) for precoder G."""
    Hf, Gf = _f(H), _f(G)
    M, K = Hf.shape
    g = np.zeros(K, dtype=np.float64)
    lib().orc_sinr(M, K, _p(Hf), M, _p(Gf), M, float(sigma2), _p(g))
    return g


def sum_se(H: np.ndarray, G: np.ndarray, sigma2: float = 1.0) -> float:
    """Instantaneous sum SE, sum_k log2(1 + gamma_k) (the argument of Eq. 10)."""
    return float(np.sum(np.log2(1.0 + sinr(H, G, sigma2))))


def precode(H: np.ndarray, xi: float, variant="standard", max_iter: int = 8, tol: float = 0.0,
            power: float = 1.0, omega: float = 1.0):
    """Full precoder for one channel: dict with W, X, A, beta, iters, relres, status.
    JOR and GS (Sec. III-A) take the same steps: Gram, the iteration, W = H X, beta."""
    if _variant(variant) in STATIONARY:
        A = gram(H, xi)
        X, it, rr, st = pcg(A, None, variant, max_iter, tol, omega=omega)
        W = matmul(H, X)
        return dict(W=W, A=A, X=X, beta=power_factor(W, power), iters=int(it.max()),
                    relres=float(rr.max()), status=st)
    Hf = _f(H)
    M, K = Hf.shape
    W = np.zeros((M, K), dtype=np.complex128, order="F")
    A = np.zeros((K, K), dtype=np.complex128, order="F")
    X = np.zeros((K, K), dtype=np.complex128, order="F")
    beta = ctypes.c_double()
    iters = ctypes.c_int()
    relres = ctypes.c_double()
    st = lib().orc_precode(M, K, _p(Hf), M, float(xi), _variant(variant), int(max_iter), float(tol),
                           float(power), _p(W), M, _p(A), _p(X), ctypes.byref(beta),
                           ctypes.byref(iters), ctypes.byref(relres))
    return dict(W=np.ascontiguousarray(W), A=np.ascontiguousarray(A), X=np.ascontiguousarray(X),
                beta=beta.value, iters=iters.value, relres=relres.value, status=st)


def precode_symbols(H: np.ndarray, xi: float, B: np.ndarray, variant="standard",
                    max_iter: int = 8, tol: float = 0.0, power: float = 1.0,
                    X0: np.ndarray | None = None):
    """Per-symbol form (Eqs. 15-16): solve P W = B for the K x n block B of
    symbol vectors (from X0, None: zero), then the unnormalised transmit
    block H W.  beta normalises the block's average transmit power to P:
    beta = sqrt(P n / ||H W||_F^2), which equals the beta of Eq. 7 in
    expectation for unit-power symbols.  Dict with X (= W of Eq. 16), S (=
    H W), A, beta, iters (max over columns), relres (max), status."""
    Hf = _f(H)
    M, K = Hf.shape
    n = np.asarray(B).reshape(K, -1).shape[1]
    A = gram(Hf, xi)
    X, it, rr, st = pcg(A, np.asarray(B).reshape(K, n), variant, max_iter, tol, X0)
    S = matmul(Hf, X)
    beta = power_factor(S, power * n)
    return dict(X=X, S=S, A=A, beta=beta, iters=int(it.max()), relres=float(rr.max()), status=st)


def precode_blocks(H: np.ndarray, xi: float, blocks, variant="standard", max_iter: int = 8,
                   tol: float = 0.0, power: float = 1.0):
    """Per-subarray block precoder (Eq. 7 with the block structure of Eq. 6):
    each block (row0, rows, col0, cols) is the RZF of its sub-channel
    H[row0:row0+rows, col0:col0+cols] with its own beta_i.  Returns (G, betas)
    where G is M x K holding the unnormalised blocks W_i = H_i P_i^{-1} and
    zeros elsewhere (as the paper's G before the beta_i are applied)."""
    Hm = np.asarray(H)
    G = np.zeros(Hm.shape, dtype=np.complex128)
    betas = []
    for (r0, nr, c0, nc) in blocks:
        ref = precode(Hm[r0:r0 + nr, c0:c0 + nc], xi, variant, max_iter, tol, power)
        G[r0:r0 + nr, c0:c0 + nc] = ref["W"]
        betas.append(ref["beta"])
    return G, betas


def precode_batch(Hs, xis, variant="standard", max_iter: int = 8, tol: float = 0.0,
                  power: float = 1.0, nthreads: int | None = None):
    """Many precoders on host threads.  ``Hs``: sequence of (M_i, K_i) arrays
    or an (n, M, K) array.  Returns (list of W, beta, iters, relres, status)."""
    n = len(Hs)
    nthreads = nthreads or os.cpu_count() or 1
    Hf = [_f(h) for h in Hs]
    Ws = [np.zeros(h.shape, dtype=np.complex128, order="F") for h in Hf]
    Ms = np.array([h.shape[0] for h in Hf], dtype=np.int32)
    Ks = np.array([h.shape[1] for h in Hf], dtype=np.int32)
    Hp = (ctypes.c_void_p * n)(*[h.ctypes.data for h in Hf])
    Wp = (ctypes.c_void_p * n)(*[w.ctypes.data for w in Ws])
    xi = np.ascontiguousarray(np.asarray(xis, dtype=np.float64))
    beta = np.zeros(n)
    iters = np.zeros(n, dtype=np.int32)
    relres = np.zeros(n)
    status = np.zeros(n, dtype=np.int32)
    lib().orc_precode_batch(n, _p(Ms), _p(Ks), ctypes.cast(Hp, ctypes.c_void_p), _p(Ms), _p(xi),
                            _variant(variant), int(max_iter), float(tol), float(power),
                            ctypes.cast(Wp, ctypes.c_void_p), _p(Ms), _p(beta), _p(iters),
                            _p(relres), _p(status), int(nthreads))
    return [np.ascontiguousarray(w) for w in Ws], beta, iters, relres, status


# ---------------------------------------------------------------------------
# Operation counts of the Appendix (closed forms; complex arithmetic counted
# in real flops as the paper does).

def flops_rzf_direct(K: int) -> int:
    """Direct inversion via Cholesky: 4K^3 + K - 1 (the O(K) term dropped)."""
    return 4 * K ** 3 + K - 1


def flops_cg_iteration(K: int) -> int:
    """One CG iteration: 8K^2 + 46K - 6."""
    return 8 * K ** 2 + 46 * K - 6


def flops_jacobi_preprocessing(K: int) -> int:
    """The extra C^{-1} P preprocessing of Jac-PCG: 4K^2 + 2K."""
    return 4 * K ** 2 + 2 * K


def flops_cg(K: int, T: int) -> int:
    return T * flops_cg_iteration(K)


def flops_jacpcg(K: int, T: int, preprocess_every_iteration: bool = False) -> int:
    pre = flops_jacobi_preprocessing(K) * (T if preprocess_every_iteration else 1)
    return T * flops_cg_iteration(K) + pre


def flops_gs_iteration(K: int) -> int:
    return 8 * K ** 2 - 8 * K


def flops_gs_init(K: int) -> int:
    return 4 * K ** 3 - 3 * K ** 2 + K


def flops_jor_init(K: int) -> int:
    return 2 * K ** 2 + K + 1
