/*
 * jacpcg_oracle.c -- plain FP64 CPU oracle for the Jac-PCG RZF precoder of
 * "Jac-PCG Based Low-Complexity Precoding for Extremely Large-Scale MIMO
 * Systems" (Xu, Zhang, Li, Xiao, Ai; arXiv 2305.13925).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline / reference legs of the benchmark load this library; the
 * product path never does.  It shares no code, header or constant with the
 * CUDA path.  Every function follows one passage of the paper, cited above
 * it, in the paper's order and with no blocking, fusion or reordering.
 *
 * Conventions
 *   - complex values are C99 `double complex`;
 *   - every matrix is column-major: element (i, j) of a matrix with leading
 *     dimension ld sits at [i + j * ld];
 *   - built with -ffp-contract=off: each product and each sum is one IEEE
 *     round-to-nearest operation, and every sum runs in index order.
 *
 * Parity status of each function is stated in its comment ("pinned by ..."
 * names the independent facts the tests check it against).
 */
#include <complex.h>
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

enum { ORC_STANDARD = 0, ORC_ALG1 = 1, ORC_CG = 2 };
enum { ORC_OK = 0, ORC_BREAKDOWN = 1, ORC_NOMEM = 2, ORC_NOTHPD = 3 };

/* ------------------------------------------------------------------------ */
/* Sec. II, after Eq. 7: P = H^H H + xi I (the matrix to invert in RZF).
 * H is M x K with leading dimension ldh; A receives the K x K result.
 * Every entry is its own sum over m; the (j, i) entry is therefore the
 * exact conjugate of the (i, j) entry.
 * Pinned by: the quadratic form of Eq. 18, orthonormal columns, K = 1,
 * trace, Hermitian symmetry, lambda_min >= xi.                            */
void orc_gram(int M, int K, const cplx *H, int ldh, double xi, cplx *A)
{
    for (int j = 0; j < K; ++j) {
        for (int i = 0; i < K; ++i) {
            cplx s = 0.0;
            for (int m = 0; m < M; ++m)
                s += conj(H[m + (size_t)i * ldh]) * H[m + (size_t)j * ldh];
            if (i == j)
                s += xi;
            A[i + (size_t)j * K] = s;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Helpers: plain loops over vectors of length K.                           */
static void matvec(int K, const cplx *A, const cplx *v, cplx *out)
{
    for (int i = 0; i < K; ++i) {
        cplx s = 0.0;
        for (int k = 0; k < K; ++k)
            s += A[i + (size_t)k * K] * v[k];
        out[i] = s;
    }
}

static cplx dotc(int K, const cplx *a, const cplx *b) /* a^H b */
{
    cplx s = 0.0;
    for (int i = 0; i < K; ++i)
        s += conj(a[i]) * b[i];
    return s;
}

static double norm2(int K, const cplx *a)
{
    double s = 0.0;
    for (int i = 0; i < K; ++i)
        s += creal(a[i]) * creal(a[i]) + cimag(a[i]) * cimag(a[i]);
    return sqrt(s);
}

/* ------------------------------------------------------------------------ */
/* Sec. III-B, Steps 1-4 (Eqs. 12-14 and 19-20) with the Jacobi choice C = D
 * of Eq. 21, for one right-hand side b.  Written in residual form
 * r = s - P w, i.e. r = -g where g is the gradient of Step 2 (a reading
 * of the sign convention); the search direction is d = z + beta d with
 * z = C^{-1} r, lambda = r^H z / d^H P d, and beta = r_new^H z_new / r^H z
 * (the ratio of Eq. 20 as printed is garbled; this is the standard PCG
 * ratio, the same form Algorithm 1 uses).  dinv = NULL gives C = I, plain CG.
 * The initial point w^0 is x0, or 0 when x0 is NULL (Step 1 leaves w^0 open;
 * the residual form starts from r^0 = s - P w^0, which for a warm start from
 * a previous slot's solution is small).  Step 2's test runs before each
 * update, always relative to ||s||: when tol > 0 the
 * column stops once ||r|| <= tol ||b||; tol <= 0 runs exactly max_iter
 * updates.  An exactly converged column (d^H P d == 0 with r == 0) keeps
 * its iterate.
 * Pinned by: exactness in <= K steps, the Krylov-subspace minimisation
 * property of (preconditioned) CG, one-step exactness for diagonal P, the
 * recurrence residual agreeing with s - P w, and for w^0 != 0: a start at
 * the solution stays there, and every iterate equals w^0 plus the cold
 * iterate for the right-hand side s - P w^0.                              */
static int pcg_standard(int K, const cplx *A, const double *dinv, const cplx *b,
                        const cplx *x0, int max_iter, double tol, cplx *x, int *iters,
                        double *relres, cplx *r, cplx *z, cplx *d, cplx *q)
{
    int status = ORC_OK;
    double bnorm = norm2(K, b);
    for (int i = 0; i < K; ++i)
        x[i] = x0 ? x0[i] : 0.0;
    matvec(K, A, x, q);                           /* P w^0 */
    for (int i = 0; i < K; ++i) {
        r[i] = b[i] - q[i];
        z[i] = dinv ? dinv[i] * r[i] : r[i];
        d[i] = z[i];
    }
    double rz = creal(dotc(K, r, z));
    int t = 0;
    for (; t < max_iter; ++t) {
        if (tol > 0.0 && norm2(K, r) <= tol * bnorm)
            break;
        matvec(K, A, d, q);                       /* P d */
        double dPd = creal(dotc(K, d, q));
        double lambda;
        if (dPd > 0.0) {
            lambda = rz / dPd;
        } else {
            if (norm2(K, r) != 0.0)
                status = ORC_NOTHPD;
            lambda = 0.0;
        }
        for (int i = 0; i < K; ++i) {
            x[i] += lambda * d[i];                /* Eq. 19 / Eq. 12 */
            r[i] -= lambda * q[i];                /* Eq. 13 */
            z[i] = dinv ? dinv[i] * r[i] : r[i];  /* z = C^{-1} r */
        }
        double rz_new = creal(dotc(K, r, z));
        double beta = (rz != 0.0) ? rz_new / rz : 0.0;
        for (int i = 0; i < K; ++i)
            d[i] = z[i] + beta * d[i];            /* Eq. 20, residual form */
        rz = rz_new;
    }
    *iters = t;
    *relres = (bnorm > 0.0) ? norm2(K, r) / bnorm : 0.0;
    return status;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1 (Jac-PCG), literally, for one right-hand side s:
 *   init  w = 0, r = C^{-1} s, m = r;
 *   loop  alpha = r^H r / (m^H C^{-1} P m); w += alpha m;
 *         r -= alpha C^{-1} P m; b = r_new^H r_new / r^H r; m = r_new + b m.
 * C = D, the diagonal of P (Eq. 21).  C^{-1} P is not Hermitian, so alpha
 * is complex in general.  With an initial point w^0 = x0 (NULL: 0) the
 * scaled residual starts as r = C^{-1} (s - P w^0).  The tolerance test (tol > 0) is applied before
 * each update to the unscaled residual D r = s - P w: ||D r|| <= tol ||s||.
 * Pinned by: one-step exactness for diagonal P, equality with plain CG when
 * D = cI, convergence to P^{-1} s, and D r agreeing with s - P w.         */
static int pcg_alg1(int K, const cplx *A, const double *dinv, const double *dvec,
                    const cplx *s, const cplx *x0, int max_iter, double tol, cplx *w,
                    int *iters, double *relres, cplx *r, cplx *m, cplx *u, cplx *tmp)
{
    int status = ORC_OK;
    double snorm = norm2(K, s);
    for (int i = 0; i < K; ++i)
        w[i] = x0 ? x0[i] : 0.0;
    matvec(K, A, w, tmp);                         /* P w^0 */
    for (int i = 0; i < K; ++i) {
        r[i] = dinv[i] * (s[i] - tmp[i]);
        m[i] = r[i];
    }
    double rr = creal(dotc(K, r, r));
    int t = 0;
    for (; t < max_iter; ++t) {
        if (tol > 0.0) {
            for (int i = 0; i < K; ++i)
                tmp[i] = dvec[i] * r[i];
            if (norm2(K, tmp) <= tol * snorm)
                break;
        }
        matvec(K, A, m, tmp);                     /* P m */
        for (int i = 0; i < K; ++i)
            u[i] = dinv[i] * tmp[i];              /* C^{-1} P m */
        cplx den = dotc(K, m, u);
        cplx alpha;
        if (den != 0.0) {
            alpha = rr / den;
        } else {
            if (rr != 0.0)
                status = ORC_BREAKDOWN;
            alpha = 0.0;
        }
        for (int i = 0; i < K; ++i) {
            w[i] += alpha * m[i];
            r[i] -= alpha * u[i];
        }
        double rr_new = creal(dotc(K, r, r));
        double bt = (rr != 0.0) ? rr_new / rr : 0.0;
        for (int i = 0; i < K; ++i)
            m[i] = r[i] + bt * m[i];
        rr = rr_new;
    }
    *iters = t;
    for (int i = 0; i < K; ++i)
        tmp[i] = dvec[i] * r[i];
    *relres = (snorm > 0.0) ? norm2(K, tmp) / snorm : 0.0;
    return status;
}

/* ------------------------------------------------------------------------ */
/* Solve P X = B column by column with the chosen iteration (Eq. 16 for each
 * column of B; B = I gives X = P^{-1} as used by the RZF precoder, Eq. 7).
 * B may be NULL for the identity.  X0 (K x nrhs, ld ldx0) is the initial
 * point of every column, NULL for zero.  iters / relres receive per-column
 * values (may be NULL).  Returns the worst column status.                 */
int orc_pcg(int K, const cplx *A, const cplx *B, int ldb, int nrhs, int variant,
            int max_iter, double tol, const cplx *X0, int ldx0, cplx *X, int ldx, int *iters,
            double *relres)
{
    double *dvec = malloc(sizeof(double) * K);
    double *dinv = malloc(sizeof(double) * K);
    cplx *work = malloc(sizeof(cplx) * (size_t)K * 5);
    if (!dvec || !dinv || !work) {
        free(dvec); free(dinv); free(work);
        return ORC_NOMEM;
    }
    for (int i = 0; i < K; ++i) {                 /* D = diag(P), Eq. 21 */
        dvec[i] = creal(A[i + (size_t)i * K]);
        dinv[i] = 1.0 / dvec[i];
    }
    cplx *b = work, *r = work + K, *z = work + 2 * K, *d = work + 3 * K, *q = work + 4 * K;
    int worst = ORC_OK;
    for (int j = 0; j < nrhs; ++j) {
        for (int i = 0; i < K; ++i)
            b[i] = B ? B[i + (size_t)j * ldb] : (i == j ? 1.0 : 0.0);
        int it = 0;
        double rel = 0.0;
        int st;
        cplx *x = X + (size_t)j * ldx;
        const cplx *x0 = X0 ? X0 + (size_t)j * ldx0 : NULL;
        if (variant == ORC_ALG1)
            st = pcg_alg1(K, A, dinv, dvec, b, x0, max_iter, tol, x, &it, &rel, r, z, d, q);
        else
            st = pcg_standard(K, A, variant == ORC_CG ? NULL : dinv, b, x0, max_iter, tol, x,
                              &it, &rel, r, z, d, q);
        if (iters) iters[j] = it;
        if (relres) relres[j] = rel;
        if (st > worst) worst = st;
    }
    free(dvec); free(dinv); free(work);
    return worst;
}

/* ------------------------------------------------------------------------ */
/* Sec. III-A, the two stationary iterations the paper compares, for P w = s
 * in the fixed-point form of Eq. 11, w^{t+1} = A_i w^t + b_i (the printed
 * "w^t = A_i w^t + b_i" read as one step from t to t + 1), with D, L, U the
 * diagonal, strictly lower and strictly upper parts of P:
 *   GS:  A_i = -(D + L)^{-1} U, b_i = (D + L)^{-1} s: each sweep forms
 *        v = s - U w^t and solves (D + L) w^{t+1} = v by forward substitution;
 *   JOR: A_i = I - omega D^{-1} P, b_i = omega D^{-1} s: each sweep forms
 *        w^{t+1} = w^t - omega D^{-1} (P w^t) + omega D^{-1} s.
 * The paper does not give omega; it is an input.  The start is w^0 = x0
 * (NULL: 0).  Stopping (tol > 0): before each sweep, stop once
 * ||s - P w|| <= tol ||s|| (these methods carry no recurrence residual, so
 * the true residual is formed every sweep).  iters = sweeps done; relres =
 * ||s - P w|| / ||s|| of the returned w.
 * Pinned by: a hand-worked K = 2 example of both, exactness after one sweep
 * for diagonal P (omega = 1), one GS sweep against a library triangular
 * solve, the monotone decrease of GS's P-norm error (P HPD), JOR's
 * contraction by (kappa - 1) / (kappa + 1) per sweep in the D^{1/2}-weighted
 * norm at omega = 2 / (lambda_min + lambda_max) of D^{-1} P, and
 * convergence to P^{-1} s.                                                */
enum { ORC_JOR = 3, ORC_GS = 4 };

static void stationary_column(int K, const cplx *A, const double *dvec, int method,
                              double omega, const cplx *s, const cplx *x0, int max_iter,
                              double tol, cplx *w, int *iters, double *relres, cplx *y,
                              cplx *v)
{
    double snorm = norm2(K, s);
    for (int i = 0; i < K; ++i)
        w[i] = x0 ? x0[i] : 0.0;
    int t = 0;
    double rn;
    for (;;) {
        matvec(K, A, w, y);                           /* P w^t */
        double acc = 0.0;
        for (int i = 0; i < K; ++i) {
            cplx e = s[i] - y[i];
            acc += creal(e) * creal(e) + cimag(e) * cimag(e);
        }
        rn = sqrt(acc);
        if (t >= max_iter || (tol > 0.0 && rn <= tol * snorm))
            break;
        if (method == ORC_JOR) {
            for (int i = 0; i < K; ++i)
                w[i] = w[i] - (omega / dvec[i]) * y[i] + (omega / dvec[i]) * s[i];
        } else {
            for (int i = 0; i < K; ++i) {             /* v = s - U w^t */
                cplx acc_u = s[i];
                for (int j = i + 1; j < K; ++j)
                    acc_u -= A[i + (size_t)j * K] * w[j];
                v[i] = acc_u;
            }
            for (int i = 0; i < K; ++i) {             /* (D + L) w^{t+1} = v */
                cplx acc_l = v[i];
                for (int j = 0; j < i; ++j)
                    acc_l -= A[i + (size_t)j * K] * w[j];
                w[i] = acc_l / dvec[i];
            }
        }
        ++t;
    }
    *iters = t;
    *relres = (snorm > 0.0) ? rn / snorm : 0.0;
}

int orc_stationary(int K, const cplx *A, const cplx *B, int ldb, int nrhs, int method,
                   double omega, int max_iter, double tol, const cplx *X0, int ldx0, cplx *X,
                   int ldx, int *iters, double *relres)
{
    double *dvec = malloc(sizeof(double) * K);
    cplx *work = malloc(sizeof(cplx) * (size_t)K * 3);
    if (!dvec || !work) {
        free(dvec); free(work);
        return ORC_NOMEM;
    }
    for (int i = 0; i < K; ++i)
        dvec[i] = creal(A[i + (size_t)i * K]);
    cplx *b = work, *y = work + K, *v = work + 2 * K;
    for (int j = 0; j < nrhs; ++j) {
        for (int i = 0; i < K; ++i)
            b[i] = B ? B[i + (size_t)j * ldb] : (i == j ? 1.0 : 0.0);
        int it = 0;
        double rel = 0.0;
        stationary_column(K, A, dvec, method, omega, b, X0 ? X0 + (size_t)j * ldx0 : NULL,
                          max_iter, tol, X + (size_t)j * ldx, &it, &rel, y, v);
        if (iters) iters[j] = it;
        if (relres) relres[j] = rel;
    }
    free(dvec); free(work);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Eq. 15: the precoded signal is beta H w; for the full precoder W = H X
 * (Eq. 7 without the power factor).  H is M x K (ldh), X is K x N (ldx).  */
void orc_matmul(int M, int K, int N, const cplx *H, int ldh, const cplx *X, int ldx,
                cplx *W, int ldw)
{
    for (int j = 0; j < N; ++j) {
        for (int m = 0; m < M; ++m) {
            cplx s = 0.0;
            for (int k = 0; k < K; ++k)
                s += H[m + (size_t)k * ldh] * X[k + (size_t)j * ldx];
            W[m + (size_t)j * ldw] = s;
        }
    }
}

/* Sec. II after Eq. 7: beta = sqrt(P / tr(F^H F)) with F = W; tr(W^H W) is
 * the squared Frobenius norm.                                              */
double orc_power_factor(int M, int N, const cplx *W, int ldw, double power)
{
    double s = 0.0;
    for (int j = 0; j < N; ++j)
        for (int m = 0; m < M; ++m) {
            cplx v = W[m + (size_t)j * ldw];
            s += creal(v) * creal(v) + cimag(v) * cimag(v);
        }
    return sqrt(power / s);
}

/* ------------------------------------------------------------------------ */
/* Appendix, direct inversion via Cholesky: (a) P = L L^H, (b) L^{-1} by
 * forward substitution, (c) P^{-1} = L^{-H} L^{-1}; then X = P^{-1} B.
 * B may be NULL for the identity.  Returns ORC_NOTHPD when a pivot is not
 * positive.  Pinned by: numpy's solve and the identity H^H W = I - xi X.  */
int orc_cholesky_solve(int K, const cplx *A, const cplx *B, int ldb, int nrhs, cplx *X,
                       int ldx)
{
    cplx *L = calloc((size_t)K * K, sizeof(cplx));
    cplx *Li = calloc((size_t)K * K, sizeof(cplx));
    cplx *Pi = calloc((size_t)K * K, sizeof(cplx));
    if (!L || !Li || !Pi) {
        free(L); free(Li); free(Pi);
        return ORC_NOMEM;
    }
    int status = ORC_OK;
    /* (a) L lower triangular with real positive diagonal, P = L L^H */
    for (int j = 0; j < K && status == ORC_OK; ++j) {
        double djj = creal(A[j + (size_t)j * K]);
        for (int k = 0; k < j; ++k)
            djj -= creal(L[j + (size_t)k * K]) * creal(L[j + (size_t)k * K]) +
                   cimag(L[j + (size_t)k * K]) * cimag(L[j + (size_t)k * K]);
        if (!(djj > 0.0)) {
            status = ORC_NOTHPD;
            break;
        }
        double ljj = sqrt(djj);
        L[j + (size_t)j * K] = ljj;
        for (int i = j + 1; i < K; ++i) {
            cplx s = A[i + (size_t)j * K];
            for (int k = 0; k < j; ++k)
                s -= L[i + (size_t)k * K] * conj(L[j + (size_t)k * K]);
            L[i + (size_t)j * K] = s / ljj;
        }
    }
    if (status == ORC_OK) {
        /* (b) L^{-1}: forward substitution on L Y = I, column by column */
        for (int j = 0; j < K; ++j) {
            for (int i = 0; i < K; ++i) {
                cplx s = (i == j) ? 1.0 : 0.0;
                for (int k = 0; k < i; ++k)
                    s -= L[i + (size_t)k * K] * Li[k + (size_t)j * K];
                Li[i + (size_t)j * K] = s / L[i + (size_t)i * K];
            }
        }
        /* (c) P^{-1} = (L^{-1})^H L^{-1} */
        for (int j = 0; j < K; ++j)
            for (int i = 0; i < K; ++i) {
                cplx s = 0.0;
                for (int k = 0; k < K; ++k)
                    s += conj(Li[k + (size_t)i * K]) * Li[k + (size_t)j * K];
                Pi[i + (size_t)j * K] = s;
            }
        /* X = P^{-1} B */
        for (int j = 0; j < nrhs; ++j)
            for (int i = 0; i < K; ++i) {
                cplx s = 0.0;
                for (int k = 0; k < K; ++k)
                    s += Pi[i + (size_t)k * K] * (B ? B[k + (size_t)j * ldb] : (k == j ? 1.0 : 0.0));
                X[i + (size_t)j * ldx] = s;
            }
    }
    free(L); free(Li); free(Pi);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Eq. 9 in its centralised form for single-antenna users and precoder G:
 * gamma_k = |h_k^H g_k|^2 / (sum_{j != k} |h_k^H g_j|^2 + sigma^2).
 * Pinned by: the interference-free closed form for orthogonal channels.   */
void orc_sinr(int M, int K, const cplx *H, int ldh, const cplx *G, int ldg, double sigma2,
              double *gamma)
{
    for (int k = 0; k < K; ++k) {
        double sig = 0.0, intf = 0.0;
        for (int j = 0; j < K; ++j) {
            cplx s = 0.0;
            for (int m = 0; m < M; ++m)
                s += conj(H[m + (size_t)k * ldh]) * G[m + (size_t)j * ldg];
            double p = creal(s) * creal(s) + cimag(s) * cimag(s);
            if (j == k) sig = p; else intf += p;
        }
        gamma[k] = sig / (intf + sigma2);
    }
}

/* ------------------------------------------------------------------------ */
/* One full precoder, Eq. 7 with B = I: A = H^H H + xi I, X by the chosen
 * iteration, W = H X, beta = sqrt(power / ||W||_F^2).  Outputs A, X may be
 * NULL.  iters receives the largest per-column iteration count, relres the
 * largest per-column recurrence residual.                                 */
int orc_precode(int M, int K, const cplx *H, int ldh, double xi, int variant, int max_iter,
                double tol, double power, cplx *W, int ldw, cplx *A_out, cplx *X_out,
                double *beta, int *iters, double *relres)
{
    cplx *A = malloc(sizeof(cplx) * (size_t)K * K);
    cplx *X = malloc(sizeof(cplx) * (size_t)K * K);
    int *it = malloc(sizeof(int) * K);
    double *rr = malloc(sizeof(double) * K);
    if (!A || !X || !it || !rr) {
        free(A); free(X); free(it); free(rr);
        return ORC_NOMEM;
    }
    orc_gram(M, K, H, ldh, xi, A);
    int st = orc_pcg(K, A, NULL, K, K, variant, max_iter, tol, NULL, K, X, K, it, rr);
    orc_matmul(M, K, K, H, ldh, X, K, W, ldw);
    if (beta) *beta = orc_power_factor(M, K, W, ldw, power);
    int imax = 0;
    double rmax = 0.0;
    for (int j = 0; j < K; ++j) {
        if (it[j] > imax) imax = it[j];
        if (rr[j] > rmax) rmax = rr[j];
    }
    if (iters) *iters = imax;
    if (relres) *relres = rmax;
    if (A_out) memcpy(A_out, A, sizeof(cplx) * (size_t)K * K);
    if (X_out) memcpy(X_out, X, sizeof(cplx) * (size_t)K * K);
    free(A); free(X); free(it); free(rr);
    return st;
}

/* ------------------------------------------------------------------------ */
/* Many independent precoders on host threads (instance i on thread
 * i % nthreads).  Each instance is computed exactly as orc_precode does,
 * so results do not depend on the thread count.                           */
typedef struct {
    int n, nthreads, tid, variant, max_iter;
    const int *M, *K, *ldh, *ldw;
    const cplx *const *H;
    cplx *const *W;
    const double *xi;
    double tol, power;
    double *beta;
    int *iters, *status;
    double *relres;
} batch_job;

static void *batch_worker(void *arg)
{
    batch_job *j = arg;
    for (int i = j->tid; i < j->n; i += j->nthreads) {
        j->status[i] = orc_precode(j->M[i], j->K[i], j->H[i], j->ldh[i], j->xi[i], j->variant,
                                   j->max_iter, j->tol, j->power, j->W[i], j->ldw[i], NULL, NULL,
                                   j->beta ? &j->beta[i] : NULL, &j->iters[i], &j->relres[i]);
    }
    return NULL;
}

int orc_precode_batch(int n, const int *M, const int *K, const cplx *const *H, const int *ldh,
                      const double *xi, int variant, int max_iter, double tol, double power,
                      cplx *const *W, const int *ldw, double *beta, int *iters, double *relres,
                      int *status, int nthreads)
{
    if (nthreads < 1) nthreads = 1;
    if (nthreads > n) nthreads = n > 0 ? n : 1;
    pthread_t *th = malloc(sizeof(pthread_t) * nthreads);
    batch_job *jobs = malloc(sizeof(batch_job) * nthreads);
    if (!th || !jobs) {
        free(th); free(jobs);
        return ORC_NOMEM;
    }
    for (int t = 0; t < nthreads; ++t) {
        jobs[t] = (batch_job){n, nthreads, t, variant, max_iter, M, K, ldh, ldw, H, W, xi, tol,
                              power, beta, iters, status, relres};
        pthread_create(&th[t], NULL, batch_worker, &jobs[t]);
    }
    for (int t = 0; t < nthreads; ++t)
        pthread_join(th[t], NULL);
    free(th); free(jobs);
    return ORC_OK;
}
