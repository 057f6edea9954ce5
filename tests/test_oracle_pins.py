"""Pins for the FP64 oracle: facts fixed by the paper or by mathematics, not
by the oracle itself.  Each test names the passage or theorem it relies on
and the plausible mistakes it would catch.  CPU only."""
import json
import math
import pathlib

import numpy as np
import pytest

from oracle import oracle as O
from paper_2305_13925_gb300 import channels as C

GOLDEN = pathlib.Path(__file__).parent / "golden"


def rand_h(M, K, seed, scales=None):
    rng = np.random.default_rng(seed)
    H = (rng.standard_normal((M, K)) + 1j * rng.standard_normal((M, K))) / math.sqrt(2)
    if scales is not None:
        H = H * np.asarray(scales)[None, :]
    return H


def dft_columns(M, K):
    m = np.arange(M)[:, None]
    k = np.arange(K)[None, :]
    return np.exp(-2j * np.pi * m * k / M) / math.sqrt(M)


# --------------------------------------------------------------------------
# Gram matrix P = H^H H + xi I (Sec. II after Eq. 7)

@pytest.mark.parametrize("M,K", [(7, 3), (64, 16), (100, 32)])
def test_gram_quadratic_form_eq18(M, K):
    """Eq. 18: q^H P q = ||H q||^2 + xi ||q||^2 for every q.  Catches a
    conjugated/transposed operand (gives conj(P)), a dropped xi, a wrong index."""
    H = rand_h(M, K, 1, scales=np.linspace(0.3, 3.0, K))
    xi = 0.7
    A = O.gram(H, xi)
    rng = np.random.default_rng(2)
    for _ in range(5):
        q = rng.standard_normal(K) + 1j * rng.standard_normal(K)
        lhs = np.vdot(q, A @ q)
        rhs = np.linalg.norm(H @ q) ** 2 + xi * np.linalg.norm(q) ** 2
        assert abs(lhs - rhs) <= 1e-12 * rhs


def test_gram_hermitian_exact_and_hpd():
    """P is Hermitian (entry by entry, exactly) and lambda_min(P) >= xi (Eq. 18)."""
    inst = C.generate_instance(C.PRESETS["single_256x16"], 0, 0)
    A = O.gram(inst.H, inst.xi)
    assert np.array_equal(A, A.conj().T)
    assert np.all(np.imag(np.diag(A)) == 0)
    lam = np.linalg.eigvalsh(A)
    assert lam.min() >= inst.xi * (1 - 1e-12)


def test_gram_orthonormal_columns():
    """Orthonormal columns (unitary DFT) give P = (1 + xi) I."""
    H = dft_columns(64, 16)
    A = O.gram(H, 0.25)
    assert np.abs(A - 1.25 * np.eye(16)).max() < 1e-14


def test_gram_single_user_and_trace():
    """K = 1: P = ||h||^2 + xi.  Any K: tr P = ||H||_F^2 + K xi."""
    h = rand_h(33, 1, 3)
    A = O.gram(h, 0.5)
    assert abs(A[0, 0] - (np.linalg.norm(h) ** 2 + 0.5)) < 1e-13
    H = rand_h(50, 9, 4)
    A = O.gram(H, 0.1)
    assert abs(np.trace(A) - (np.linalg.norm(H) ** 2 + 0.9)) < 1e-11


def test_gram_visibility_blocks_are_zero():
    """Users that share no visible subarray have P[k, j] = 0 exactly (the
    sparsity remark of Sec. III-B): disjoint supports give exact zeros."""
    H = np.zeros((8, 2), dtype=complex)
    H[:4, 0] = [1, 2j, 3, -1]
    H[4:, 1] = [2, 1j, -1, 1]
    A = O.gram(H, 0.1)
    assert A[0, 1] == 0 and A[1, 0] == 0


# --------------------------------------------------------------------------
# Direct inversion (Appendix, Cholesky)

def test_cholesky_matches_library_solve_and_rzf_identity():
    """Direct RZF: numpy.linalg.solve agrees; and H^H W = I - xi X, which follows
    from H^H H P^{-1} = I - xi P^{-1} (definition of P)."""
    inst = C.generate_instance(C.PRESETS["single_256x16"], 0, 3)
    W, X, st = O.rzf_direct(inst.H, inst.xi)
    assert st == O.OK
    A = inst.H.conj().T @ inst.H + inst.xi * np.eye(16)
    Xn = np.linalg.solve(A, np.eye(16))
    assert np.linalg.norm(X - Xn) / np.linalg.norm(Xn) < 1e-12
    lhs = inst.H.conj().T @ W
    assert np.abs(lhs - (np.eye(16) - inst.xi * X)).max() < 1e-12


def test_cholesky_rejects_indefinite():
    A = np.diag([1.0, -1.0, 2.0]).astype(complex)
    _, st = O.cholesky_solve(A)
    assert st == O.NOTHPD


# --------------------------------------------------------------------------
# (Preconditioned) conjugate gradients, Sec. III-B Steps 1-4, Eqs. 19-21

def small_system(K=8, M=24, seed=5, spread=(0.5, 4.0), xi=0.3):
    H = rand_h(M, K, seed, scales=np.geomspace(*spread, K))
    return H, O.gram(H, xi)


@pytest.mark.parametrize("K", [1, 2, 3, 5, 8])
@pytest.mark.parametrize("variant", ["standard", "cg"])
def test_exact_in_at_most_K_steps(K, variant):
    """CG and PCG (Hermitian preconditioner) terminate in at most K steps in
    exact arithmetic (finite termination theorem)."""
    H, A = small_system(K=K, M=3 * K + 2, seed=10 + K)
    X, it, rr, st = O.pcg(A, None, variant, max_iter=K)
    Xs = np.linalg.solve(A, np.eye(K))
    assert st == O.OK
    assert np.linalg.norm(X - Xs) / np.linalg.norm(Xs) < 1e-9


def krylov_minimiser(A, b, Minv, t):
    """argmin over x in span{v, Minv A v, ..., (Minv A)^{t-1} v}, v = Minv b, of
    ||x - A^{-1} b||_A: the Galerkin solution (Q^H A Q) y = Q^H b."""
    v = Minv @ b
    V = [v]
    for _ in range(t - 1):
        V.append(Minv @ (A @ V[-1]))
    Q, _ = np.linalg.qr(np.stack(V, axis=1))
    y = np.linalg.solve(Q.conj().T @ A @ Q, Q.conj().T @ b)
    return Q @ y


@pytest.mark.parametrize("variant", ["standard", "cg"])
@pytest.mark.parametrize("T", [1, 2, 3, 4, 6])
def test_fixed_T_iterate_is_krylov_minimiser(variant, T):
    """The t-th (P)CG iterate minimises the energy-norm error over the t-th
    Krylov space of the preconditioned operator (optimality of CG).  This
    pins the fixed-T iterate itself; a wrong sign, a dropped preconditioner,
    a wrong step or direction formula each break it."""
    H, A = small_system(K=12, M=40, seed=21)
    d = np.real(np.diag(A))
    Minv = np.diag(1.0 / d) if variant == "standard" else np.eye(12)
    rng = np.random.default_rng(7)
    B = rng.standard_normal((12, 3)) + 1j * rng.standard_normal((12, 3))
    X, it, rr, st = O.pcg(A, B, variant, max_iter=T)
    for j in range(3):
        xk = krylov_minimiser(A, B[:, j], Minv, T)
        assert np.linalg.norm(X[:, j] - xk) / np.linalg.norm(xk) < 1e-9
    assert np.all(it == T)


@pytest.mark.parametrize("variant", ["standard", "alg1", "cg"])
def test_recurrence_residual_equals_true_residual(variant):
    """The updated residual equals s - P w (Eq. 13; for Algorithm 1, D r = s - P w).
    Catches a mismatch between the solution and residual updates."""
    H, A = small_system(K=10, M=30, seed=31, spread=(0.8, 1.5))
    rng = np.random.default_rng(8)
    B = rng.standard_normal((10, 2)) + 1j * rng.standard_normal((10, 2))
    for T in (1, 3, 5):
        X, it, rr, st = O.pcg(A, B, variant, max_iter=T)
        true = np.linalg.norm(B - A @ X, axis=0) / np.linalg.norm(B, axis=0)
        assert np.allclose(rr, true, rtol=1e-8, atol=1e-13)


def test_jacobi_exact_in_one_step_for_diagonal_P():
    """Orthogonal channels of unequal norms make P diagonal: with C = D both
    Jac-PCG forms return D^{-1} s after one step; plain CG does not."""
    H = dft_columns(32, 8) * np.geomspace(0.5, 5.0, 8)[None, :]
    A = O.gram(H, 0.2)
    assert np.abs(A - np.diag(np.diag(A))).max() < 1e-13
    A = np.diag(np.diag(A))
    exact = np.diag(1.0 / np.diag(A))
    for v in ("standard", "alg1"):
        X, it, rr, st = O.pcg(A, None, v, max_iter=1)
        assert np.abs(X - exact).max() <= 1e-15 * np.abs(exact).max()
        X3, _, _, st3 = O.pcg(A, None, v, max_iter=3)       # iterating further changes nothing
        assert st3 == O.OK and np.array_equal(X3, X)
    Xcg, _, _, _ = O.pcg(A, None, "cg", max_iter=1)
    Bones = np.ones((8, 1), dtype=complex)
    xcg, _, _, _ = O.pcg(A, Bones, "cg", max_iter=1)
    assert np.linalg.norm(xcg[:, 0] - exact @ Bones[:, 0]) > 1e-3


def test_equal_diagonal_all_forms_coincide():
    """With D = cI the Jacobi preconditioner is a scalar: Jac-PCG (both forms)
    and plain CG produce the same iterates."""
    H = rand_h(30, 8, 41)
    H = H / np.linalg.norm(H, axis=0)[None, :]          # equal column norms
    A = O.gram(H, 0.4)
    assert np.ptp(np.real(np.diag(A))) < 1e-14
    for T in (1, 2, 4, 6):
        Xs = [O.pcg(A, None, v, max_iter=T)[0] for v in ("standard", "alg1", "cg")]
        assert np.linalg.norm(Xs[0] - Xs[2]) / np.linalg.norm(Xs[2]) < 1e-12
        assert np.linalg.norm(Xs[1] - Xs[2]) / np.linalg.norm(Xs[2]) < 1e-12


def test_brute_force_K1_K2():
    """K = 1: x = s / (||h||^2 + xi) after one step.  K = 2: two steps of CG or
    Jac-PCG give the closed-form 2 x 2 inverse."""
    h = rand_h(9, 1, 51)
    A = O.gram(h, 0.3)
    for v in ("standard", "alg1", "cg"):
        X, _, _, _ = O.pcg(A, None, v, max_iter=1)
        assert abs(X[0, 0] - 1.0 / (np.linalg.norm(h) ** 2 + 0.3)) < 1e-15
    H = rand_h(9, 2, 52)
    A = O.gram(H, 0.3)
    a, b, c, d = A[0, 0], A[0, 1], A[1, 0], A[1, 1]
    inv = np.array([[d, -b], [-c, a]]) / (a * d - b * c)
    for v in ("standard", "cg"):
        X, _, _, _ = O.pcg(A, None, v, max_iter=2)
        assert np.abs(X - inv).max() < 1e-13 * np.abs(inv).max()


def test_tolerance_stops_at_first_small_residual():
    """Step 2: a column stops at the first iterate with ||r|| <= tol ||s||;
    one iteration fewer leaves it above the tolerance."""
    inst = C.generate_instance(C.PRESETS["batched_1024x64"], 1, 0)
    A = O.gram(inst.H, inst.xi)
    tol = 1e-6
    X, it, rr, st = O.pcg(A, None, "standard", max_iter=200, tol=tol)
    assert np.all(rr <= tol) and np.all(it > 0)
    for j in (0, 17, 63):
        _, it2, rr2, _ = O.pcg(A, np.eye(64)[:, j], "standard", max_iter=int(it[j]) - 1)
        assert rr2[0] > tol


def test_converged_forms_reach_rzf():
    """At tolerance, standard Jac-PCG and CG converge to the direct RZF solution."""
    inst = C.generate_instance(C.PRESETS["single_256x16"], 0, 0)
    A = O.gram(inst.H, inst.xi)
    Xc, _ = O.cholesky_solve(A)
    for v in ("standard", "cg"):
        X, it, rr, st = O.pcg(A, None, v, max_iter=500, tol=1e-13)
        assert np.linalg.norm(X - Xc) / np.linalg.norm(Xc) < 1e-10


def test_alg1_converges_when_preconditioned_operator_is_mild():
    """Algorithm 1 (Euclidean products on D^{-1} P) converges to P^{-1} s when
    the diagonal is nearly constant."""
    H, A = small_system(K=8, M=40, seed=61, spread=(0.95, 1.05), xi=0.5)
    X, it, rr, st = O.pcg(A, None, "alg1", max_iter=400, tol=1e-12)
    Xs = np.linalg.solve(A, np.eye(8))
    assert np.linalg.norm(X - Xs) / np.linalg.norm(Xs) < 1e-9


def _gfrac(pair):
    from fractions import Fraction
    return complex(float(Fraction(pair[0])), float(Fraction(pair[1])))


def test_alg1_hand_worked_complex_step_k2():
    """Algorithm 1 on a 2 x 2 system with unequal diagonal, where C^{-1} P is
    not Hermitian and alpha is complex: the first two iterates equal the values
    derived by hand from the printed steps (tests/golden/alg1_k2_worked.json).
    Catches a conjugated or transposed step denominator, a step taken on
    r instead of m, a missing D^{-1} in the residual update, a wrong b."""
    g = json.loads((GOLDEN / "alg1_k2_worked.json").read_text())
    P = np.array([[_gfrac(e) for e in row] for row in g["P"]])
    s = np.array([_gfrac(e) for e in g["s"]]).reshape(2, 1)
    for T, key in ((1, "w1"), (2, "w2")):
        w, it, rr, st = O.pcg(P, s, "alg1", max_iter=T)
        want = np.array([_gfrac(e) for e in g[key]])
        assert st == O.OK and it[0] == T
        assert np.abs(w[:, 0] - want).max() <= 1e-15, (key, w[:, 0], want)
        # the recurrence residual D r equals s - P w (last printed r)
        r_want = np.array([_gfrac(e) for e in g["r" + key[1]]])
        d = np.real(np.diag(P))
        assert abs(rr[0] - np.linalg.norm(d * r_want) / np.linalg.norm(s)) <= 1e-15
    exact = np.array([_gfrac(e) for e in g["exact_solution"]])
    assert np.abs(w[:, 0] - exact).max() > 1e-2       # not exact in K steps


@pytest.mark.parametrize("seed", [81, 82])
def test_alg1_direction_orthogonal_to_next_residual(seed):
    """Algorithm 1's alpha = r^H r / (m^H C^{-1} P m) makes every new scaled
    residual orthogonal to the direction just taken: m_t^H r_{t+1} = 0 (from
    m_t^H r_t = r_t^H r_t, which the b-update keeps).  With m_t proportional
    to w_{t+1} - w_t and D r_{t+1} = s - P w_{t+1}, this reads
    (w_{t+1} - w_t)^H D^{-1} (s - P w_{t+1}) = 0.  On a random channel with a
    spread diagonal alpha is complex, so a conjugated denominator fails."""
    H, A = small_system(K=12, M=40, seed=seed, spread=(0.3, 3.0), xi=0.4)
    rng = np.random.default_rng(seed)
    s = (rng.standard_normal(12) + 1j * rng.standard_normal(12)).reshape(12, 1)
    dinv = 1.0 / np.real(np.diag(A))
    prev = np.zeros(12, dtype=complex)
    imag_steps = 0
    for T in range(1, 6):
        w = O.pcg(A, s, "alg1", max_iter=T)[0][:, 0]
        step = w - prev
        r = dinv * (s[:, 0] - A @ w)
        assert abs(np.vdot(step, r)) <= 1e-11 * np.linalg.norm(step) * np.linalg.norm(r)
        # alpha = r^H r / den is complex iff den = m^H D^{-1} P m is, and den has
        # the phase of step^H D^{-1} P step (step = alpha m)
        z = np.vdot(step, dinv * (A @ step))
        imag_steps += abs(z.imag) > 1e-3 * abs(z)
        prev = w
    assert imag_steps >= 3


def test_column_independence():
    """Each column of X depends only on its own column of B (Eq. 16 per column)."""
    H, A = small_system(K=6, M=20, seed=71)
    rng = np.random.default_rng(9)
    B = rng.standard_normal((6, 4)) + 1j * rng.standard_normal((6, 4))
    for v in ("standard", "alg1", "cg"):
        X, _, _, _ = O.pcg(A, B, v, max_iter=3)
        for j in range(4):
            xj, _, _, _ = O.pcg(A, B[:, j], v, max_iter=3)
            assert np.array_equal(X[:, j], xj[:, 0])


# --------------------------------------------------------------------------
# Precoder, power factor, SINR (Eqs. 7, 9, 15)

def test_precoder_identity_and_power():
    """Converged W satisfies H^H W = I - xi X, and ||beta W||_F^2 = P."""
    inst = C.generate_instance(C.PRESETS["single_256x16"], 0, 1)
    out = O.precode(inst.H, inst.xi, "standard", max_iter=300, tol=1e-14, power=3.0)
    lhs = inst.H.conj().T @ out["W"]
    assert np.abs(lhs - (np.eye(16) - inst.xi * out["X"])).max() < 1e-10
    assert abs(np.linalg.norm(out["beta"] * out["W"]) ** 2 - 3.0) < 1e-12
    W2 = inst.H @ out["X"]
    assert np.abs(out["W"] - W2).max() < 1e-12 * np.abs(W2).max()


def test_sinr_closed_form_orthogonal_channels():
    """Orthogonal channels: RZF columns are h_k / (||h_k||^2 + xi), there is no
    interference, and SINR_k = beta^2 (||h_k||^2 / (||h_k||^2 + xi))^2 / sigma^2
    with beta^2 = P / sum_k ||h_k||^2 / (||h_k||^2 + xi)^2."""
    norms = np.array([0.5, 1.0, 2.0, 3.5])
    H = dft_columns(16, 4) * norms[None, :]
    xi, P, s2 = 0.3, 2.0, 0.7
    W, X, st = O.rzf_direct(H, xi)
    beta = O.power_factor(W, P)
    g = O.sinr(H, beta * W, s2)
    n2 = norms ** 2
    beta2 = P / np.sum(n2 / (n2 + xi) ** 2)
    expect = beta2 * (n2 / (n2 + xi)) ** 2 / s2
    assert np.allclose(g, expect, rtol=1e-12)


def test_se_of_converged_pcg_matches_direct_rzf():
    """Sum SE (argument of Eq. 10) from converged Jac-PCG equals direct RZF's."""
    inst = C.generate_instance(C.PRESETS["single_256x16"], 0, 2)
    Wd, _, _ = O.rzf_direct(inst.H, inst.xi)
    out = O.precode(inst.H, inst.xi, "standard", max_iter=300, tol=1e-13)
    se_d = O.sum_se(inst.H, O.power_factor(Wd, 10.0) * Wd)
    se_p = O.sum_se(inst.H, out["beta"] * out["W"] * math.sqrt(10.0))
    assert abs(se_d - se_p) < 1e-9 * se_d


# --------------------------------------------------------------------------
# Operation counts of the Appendix and the printed complexity claim

def test_flop_formulas_and_54_percent_claim():
    g = json.loads((GOLDEN / "paper_printed.json").read_text())
    K = 30
    T = g["iterations_to_convergence"]["value"]
    # the CG iteration total is the sum of its listed parts (Appendix)
    parts = (8 * K - 2) + (8 * K ** 2 - 2 * K) + (8 * K - 2) + 8 * K + 8 * K + (8 * K - 2) + 8 * K
    assert parts == O.flops_cg_iteration(K)
    red = 1 - O.flops_jacpcg(K, T) / O.flops_rzf_direct(K)
    assert abs(red - 0.5693) < 5e-4
    claim = g["complexity_reduction_jacpcg_vs_rzf"]
    assert claim["K"] == K and abs(red - claim["value"]) < 0.04     # "about 54%"
    # Fig. 6 discussion: CG and Jac-PCG fall below direct RZF as K grows; with
    # the Appendix formulas at T = 5 the crossover is K = 15
    for K in range(15, 129):
        assert O.flops_cg(K, T) < O.flops_jacpcg(K, T) < O.flops_rzf_direct(K)
    assert O.flops_jacpcg(14, T) > O.flops_rzf_direct(14)


def test_table1_geometry():
    """Table I: N = 23.0610 m at spacing 2 lambda and 2.6 GHz gives M = 100."""
    g = json.loads((GOLDEN / "paper_printed.json").read_text())["table1"]
    lam = 299792458.0 / g["carrier_hz"]
    assert round(g["N_m"] / (g["antenna_spacing_lambda"] * lam)) == 100
    inst = C.paper_table1(0, 0)
    assert inst.H.shape == (100, 32)
    A = O.gram(inst.H, inst.xi)
    assert np.linalg.eigvalsh(A).min() >= inst.xi * (1 - 1e-9)


def test_batch_equals_single_instances():
    """The threaded batch entry computes each instance exactly as the single one."""
    insts = C.generate_ragged(6, 3, k_set=(8, 16, 32), m_set=(256, 512))
    Ws, beta, iters, relres, status = O.precode_batch([i.H for i in insts], [i.xi for i in insts],
                                                      "standard", max_iter=6, nthreads=3)
    for i, inst in enumerate(insts):
        one = O.precode(inst.H, inst.xi, "standard", max_iter=6)
        assert np.array_equal(Ws[i], one["W"]) and beta[i] == one["beta"]
        assert iters[i] == 6 and status[i] == O.OK


# ---------------------------------------------------------------------------
# Warm start (initial point w^0 of Sec. III-B Step 1) and the per-symbol
# right-hand-side form (Eqs. 15-16)

def _hpd_system(K, seed, n=None):
    rng = np.random.default_rng(seed)
    H = (rng.standard_normal((3 * K, K)) + 1j * rng.standard_normal((3 * K, K))) / np.sqrt(2)
    A = O.gram(H, 0.3)
    n = K if n is None else n
    B = rng.standard_normal((K, n)) + 1j * rng.standard_normal((K, n))
    return H, A, B


@pytest.mark.parametrize("variant", ["standard", "cg", "alg1"])
def test_warm_start_from_the_solution_stays_there(variant):
    """Starting at X* = A^{-1} B: the tolerance test stops before the first
    update (0 iterations, X = X0 exactly), and fixed-T runs stay at X*."""
    _, A, B = _hpd_system(12, 41, 5)
    Xs = np.linalg.solve(A, B)
    X, it, rr, st = O.pcg(A, B, variant, max_iter=20, tol=1e-10, X0=Xs)
    assert (it == 0).all() and np.array_equal(X, Xs)
    X, it, rr, st = O.pcg(A, B, variant, max_iter=6, X0=Xs)
    assert np.linalg.norm(X - Xs) <= 1e-10 * np.linalg.norm(Xs)


@pytest.mark.parametrize("variant", ["standard", "cg", "alg1"])
def test_warm_start_is_the_shifted_cold_solve(variant):
    """PCG from w^0 on P w = s runs the same Krylov recurrences as PCG from 0
    on P e = s - P w^0: every fixed-T iterate is w^0 + e_T.  A dropped or
    mis-signed P w^0 term, or an output without w^0, fails this."""
    _, A, B = _hpd_system(16, 42, 6)
    rng = np.random.default_rng(43)
    X0 = rng.standard_normal(B.shape) + 1j * rng.standard_normal(B.shape)
    for T in (1, 3, 7):
        Xw = O.pcg(A, B, variant, max_iter=T, X0=X0)[0]
        E = O.pcg(A, B - A @ X0, variant, max_iter=T)[0]
        assert np.linalg.norm(Xw - (X0 + E)) <= 1e-11 * np.linalg.norm(Xw), (variant, T)


def test_warm_start_near_the_solution_converges_sooner():
    """The slot-to-slot use: a start close to the solution reaches the
    tolerance in fewer iterations, and at tolerance both reach A^{-1} B."""
    _, A, B = _hpd_system(24, 44, 8)
    Xs = np.linalg.solve(A, B)
    rng = np.random.default_rng(45)
    X0 = Xs * (1 + 1e-3 * rng.standard_normal(Xs.shape))
    Xc, itc, _, _ = O.pcg(A, B, "standard", max_iter=200, tol=1e-9)
    Xw, itw, _, _ = O.pcg(A, B, "standard", max_iter=200, tol=1e-9, X0=X0)
    assert itw.max() < itc.max()
    for X in (Xc, Xw):
        assert np.linalg.norm(X - Xs) <= 1e-7 * np.linalg.norm(Xs)


def test_per_symbol_form_eq15_16():
    """Eqs. 15-16: for B = I the per-symbol form is the RZF precoder (S = W
    of Eq. 7, and the block power factor is sqrt(K) times Eq. 7's beta for
    the K unit symbol vectors); at tolerance S = H (H^H H + xi I)^{-1} B
    (direct solve); the block power factor normalises the mean power of the
    transmitted vectors to P."""
    H, _, B = _hpd_system(10, 46, 4)
    xi = 0.3
    ref = O.precode(H, xi, "standard", max_iter=6, power=2.0)
    s = O.precode_symbols(H, xi, np.eye(10), "standard", max_iter=6, power=2.0)
    assert np.allclose(s["S"], ref["W"], rtol=0, atol=1e-13 * np.abs(ref["W"]).max())
    assert math.isclose(s["beta"], math.sqrt(10) * ref["beta"], rel_tol=1e-12)
    s = O.precode_symbols(H, xi, B, "standard", max_iter=100, tol=1e-12, power=2.0)
    S_direct = H @ np.linalg.solve(H.conj().T @ H + xi * np.eye(10), B)
    assert np.linalg.norm(s["S"] - S_direct) <= 1e-9 * np.linalg.norm(S_direct)
    mean_power = np.linalg.norm(s["beta"] * s["S"]) ** 2 / B.shape[1]
    assert math.isclose(mean_power, 2.0, rel_tol=1e-12)


# ---------------------------------------------------------------------------
# Per-subarray block precoder (Eq. 7, block structure of Eq. 6)

def test_block_precoder_equals_full_rzf_on_block_diagonal_channel():
    """When the channel is block diagonal (each user group sees only its own
    antennas), P is block diagonal and every column of the iteration stays
    inside its block: the full fixed-T precoder equals the assembled block
    precoders, at any T.  A block placed at the wrong rows or columns, or a
    transposed extraction, fails this."""
    rng = np.random.default_rng(61)
    M, K = 40, 12
    blocks = [(0, 14, 0, 5), (14, 10, 5, 3), (24, 16, 8, 4)]
    H = np.zeros((M, K), dtype=np.complex128)
    for (r0, nr, c0, nc) in blocks:
        H[r0:r0 + nr, c0:c0 + nc] = rng.standard_normal((nr, nc)) + 1j * rng.standard_normal((nr, nc))
    for T in (1, 3, 6):
        G, betas = O.precode_blocks(H, 0.4, blocks, "standard", max_iter=T)
        W = O.precode(H, 0.4, "standard", max_iter=T)["W"]
        assert np.linalg.norm(G - W) <= 1e-12 * np.linalg.norm(W), T
        for (r0, nr, c0, nc), b in zip(blocks, betas):
            Wi = W[r0:r0 + nr, c0:c0 + nc]
            assert math.isclose(b, 1.0 / np.linalg.norm(Wi), rel_tol=1e-12)


def test_block_precoder_paper_structure_blocks_are_independent_rzf():
    """The paper's three blocks (group-1 antennas, common antennas, group-2
    antennas): each block at tolerance is the direct RZF of its sub-channel,
    the zero blocks of G stay zero, and the common block serves every user."""
    H = rand_h(48, 10, 62)
    blocks = [(0, 16, 0, 4), (16, 16, 0, 10), (32, 16, 4, 6)]
    G, betas = O.precode_blocks(H, 0.2, blocks, "standard", max_iter=200, tol=1e-13)
    assert np.count_nonzero(G[0:16, 4:]) == 0 and np.count_nonzero(G[32:48, :4]) == 0
    for (r0, nr, c0, nc) in blocks:
        Hi = H[r0:r0 + nr, c0:c0 + nc]
        Wd = Hi @ np.linalg.inv(Hi.conj().T @ Hi + 0.2 * np.eye(nc))
        assert np.linalg.norm(G[r0:r0 + nr, c0:c0 + nc] - Wd) <= 1e-9 * np.linalg.norm(Wd)


# --------------------------------------------------------------------------
# Stationary iterations of Sec. III-A: Gauss-Seidel and JOR

def _omega_opt(A):
    """2 / (lambda_min + lambda_max) of D^{-1} P (its eigenvalues are those of
    the Hermitian D^{-1/2} P D^{-1/2}); returns (omega, kappa)."""
    d = np.real(np.diag(A))
    lam = np.linalg.eigvalsh(A / np.sqrt(np.outer(d, d)))
    return 2.0 / (lam[0] + lam[-1]), lam[-1] / lam[0]


def test_stationary_hand_worked_k2():
    """GS and JOR (omega = 1 and 1/2) on the 2 x 2 system with unequal
    diagonal: the first two sweeps equal the values derived by hand from the
    printed splittings (tests/golden/stationary_k2_worked.json).  Catches GS
    using old values for the lower part (that is Jacobi), a transposed
    splitting (U for L), a missing omega or D^{-1}."""
    g = json.loads((GOLDEN / "stationary_k2_worked.json").read_text())
    P = np.array([[_gfrac(e) for e in row] for row in g["P"]])
    s = np.array([_gfrac(e) for e in g["s"]]).reshape(2, 1)
    from fractions import Fraction
    cases = [("gs", 1.0, g["gs"])] + [("jor", float(Fraction(c["omega"])), c) for c in g["jor"]]
    for method, omega, c in cases:
        for T, key in ((1, "w1"), (2, "w2")):
            w, it, rr, st = O.pcg(P, s, method, max_iter=T, omega=omega)
            want = np.array([_gfrac(e) for e in c[key]])
            assert st == O.OK and it[0] == T
            assert np.abs(w[:, 0] - want).max() <= 1e-15, (method, omega, key, w[:, 0], want)
            assert abs(rr[0] - np.linalg.norm(s[:, 0] - P @ want) / np.linalg.norm(s)) <= 1e-14


def test_stationary_exact_for_diagonal_P_and_K1():
    """Diagonal P (orthogonal channels): L = U = 0, so one GS sweep and one JOR
    sweep with omega = 1 give D^{-1} s, and further sweeps keep it.  K = 1:
    one sweep gives s / p (GS; JOR with omega = 1), omega s / p for JOR."""
    H = dft_columns(32, 8) * np.geomspace(0.5, 5.0, 8)[None, :]
    A = np.diag(np.diag(O.gram(H, 0.2)))
    exact = np.diag(1.0 / np.diag(A))
    for m in ("gs", "jor"):
        X1 = O.pcg(A, None, m, max_iter=1)[0]
        assert np.abs(X1 - exact).max() <= 1e-15 * np.abs(exact).max()
        assert np.abs(O.pcg(A, None, m, max_iter=4)[0] - exact).max() <= 1e-15 * np.abs(exact).max()
    p = np.array([[3.0 + 0j]])
    s = np.array([[1.5 - 2j]])
    assert O.pcg(p, s, "gs", max_iter=1)[0][0, 0] == s[0, 0] / 3.0
    assert abs(O.pcg(p, s, "jor", max_iter=1, omega=0.25)[0][0, 0] - 0.25 * s[0, 0] / 3.0) < 1e-16


def test_gs_sweep_is_a_lower_triangular_solve():
    """One GS sweep from any w^t is the solution of (D + L) w^{t+1} = s - U w^t
    (scipy's triangular solver as the independent routine)."""
    sl = pytest.importorskip("scipy.linalg")
    H, A = small_system(K=9, M=30, seed=91)
    rng = np.random.default_rng(91)
    s = rng.standard_normal(9) + 1j * rng.standard_normal(9)
    w0 = rng.standard_normal(9) + 1j * rng.standard_normal(9)
    w1 = O.pcg(A, s.reshape(9, 1), "gs", max_iter=1, X0=w0.reshape(9, 1))[0][:, 0]
    want = sl.solve_triangular(np.tril(A), s - np.triu(A, 1) @ w0, lower=True)
    assert np.linalg.norm(w1 - want) <= 1e-13 * np.linalg.norm(want)


def test_gs_energy_error_decreases_monotonically():
    """GS updates one coordinate at a time to the minimiser of the quadratic
    w^H P w - 2 Re(w^H s) along it, so for Hermitian positive definite P the
    energy-norm error ||w^t - P^{-1} s||_P never grows, and GS converges
    (theorem for HPD matrices).  A sweep that used the old values of the
    lower part (Jacobi) breaks the monotone decrease on this system."""
    H, A = small_system(K=12, M=20, seed=93, spread=(0.3, 3.0), xi=0.2)
    rng = np.random.default_rng(93)
    s = rng.standard_normal(12) + 1j * rng.standard_normal(12)
    ws = np.linalg.solve(A, s)
    errs = []
    for T in range(0, 12):
        e = O.pcg(A, s.reshape(12, 1), "gs", max_iter=T)[0][:, 0] - ws
        errs.append(np.sqrt(np.real(np.vdot(e, A @ e))))
    assert all(b < a for a, b in zip(errs, errs[1:]))
    w = O.pcg(A, s.reshape(12, 1), "gs", max_iter=5000, tol=1e-14)[0][:, 0]
    assert np.linalg.norm(w - ws) <= 1e-10 * np.linalg.norm(ws)


def test_jor_contracts_at_the_spectral_rate():
    """JOR at omega = 2 / (lambda_min + lambda_max) of D^{-1} P: in the
    D^{1/2}-weighted norm the error map I - omega D^{-1/2} P D^{-1/2} is
    Hermitian with spectral radius (kappa - 1) / (kappa + 1), so every sweep
    shrinks that norm by at least this factor, and JOR converges to P^{-1} s.
    A missing D^{-1} or omega, or a wrong sign, breaks the bound."""
    H, A = small_system(K=10, M=40, seed=95, spread=(0.4, 2.5), xi=0.3)
    omega, kappa = _omega_opt(A)
    rho = (kappa - 1.0) / (kappa + 1.0)
    dh = np.sqrt(np.real(np.diag(A)))
    rng = np.random.default_rng(95)
    s = rng.standard_normal(10) + 1j * rng.standard_normal(10)
    ws = np.linalg.solve(A, s)
    prev = np.linalg.norm(dh * ws)            # w^0 = 0
    for T in range(1, 9):
        e = O.pcg(A, s.reshape(10, 1), "jor", max_iter=T, omega=omega)[0][:, 0] - ws
        cur = np.linalg.norm(dh * e)
        assert cur <= rho * prev * (1 + 1e-9)
        prev = cur
    w = O.pcg(A, s.reshape(10, 1), "jor", max_iter=5000, tol=1e-14, omega=omega)[0][:, 0]
    assert np.linalg.norm(w - ws) <= 1e-10 * np.linalg.norm(ws)


def test_stationary_tolerance_semantics():
    """tol > 0 stops before the first sweep whose true residual is at most
    tol ||s||; the reported residual is that true residual."""
    H, A = small_system(K=8, M=30, seed=97, spread=(0.8, 1.5), xi=0.3)
    omega, _ = _omega_opt(A)
    s = np.ones((8, 1), dtype=complex)
    for m in ("gs", "jor"):
        w, it, rr, st = O.pcg(A, s, m, max_iter=500, tol=1e-6, omega=omega)
        true = np.linalg.norm(s[:, 0] - A @ w[:, 0]) / np.linalg.norm(s)
        assert rr[0] <= 1e-6 and abs(rr[0] - true) <= 1e-12
        wp = O.pcg(A, s, m, max_iter=int(it[0]) - 1, omega=omega)[0]
        assert np.linalg.norm(s[:, 0] - A @ wp[:, 0]) / np.linalg.norm(s) > 1e-6


def test_paper_convergence_ordering_on_table1_geometry():
    """Sec. IV on Fig. 3 and the summary table: Jac-PCG converges faster than
    CG, and GS faster than JOR.  The least-square error of W against the
    direct-inversion RZF, averaged over ten channels of the Table I geometry
    (M = 100, K = 32), keeps that order at every T from 2 to 8 (JOR at its
    convergent omega = 2 / (lambda_min + lambda_max) of D^{-1} P)."""
    insts = [C.paper_table1(0, i) for i in range(10)]
    lse = {m: np.zeros(9) for m in ("standard", "cg", "gs", "jor")}
    for inst in insts:
        H = C.round_complex64(inst.H)
        A = O.gram(H, inst.xi)
        omega, _ = _omega_opt(A)
        Wd = O.rzf_direct(H, inst.xi)[0]
        for m in lse:
            for T in range(2, 9):
                W = O.precode(H, inst.xi, m, max_iter=T, omega=omega)["W"]
                lse[m][T] += np.linalg.norm(W - Wd) ** 2 / np.linalg.norm(Wd) ** 2 / len(insts)
    for T in range(2, 9):
        assert lse["standard"][T] < lse["cg"][T], T
        assert lse["gs"][T] < lse["jor"][T], T
