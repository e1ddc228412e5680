/*
 * Oracle: setup operators of the v-eta channel DNS, built in IEEE binary128.
 *
 * TEST INFRASTRUCTURE ONLY.  This file belongs to the CPU oracle that checks the
 * GPU path.  Only tests, the smoke check and the benchmark's CPU-baseline leg may
 * load it; the product library never links or calls it.
 *
 * Everything here is plain, unblocked linear algebra in quad precision
 * (__float128 on x86-64, long double on aarch64 -- both IEEE binary128, so the
 * results are bit-identical on both machines), rounded once to double on output.
 *
 * What is built (paper, Sec. 2 and Sec. 3):
 *   - Chebyshev-Gauss-Lobatto nodes, flipped to ascending y, and the collocation
 *     derivative D1 on them; D2 = D1*D1                (Listing 1, Sec. 2)
 *   - the clamped fourth derivative D4c on the interior nodes, i.e. the fourth
 *     derivative of the interpolant (1-y^2)^2 q(y) that satisfies v = v' = 0 at
 *     both walls (the cheb4bc construction cited in Sec. 2, Weideman & Reddy 2000)
 *   - per wavenumber pair and per RK3 sub-step length h in {1/2, 1}: the CN
 *     update operators for v (Eq. CN1, multiplied through by Delta) and eta
 *     (Eq. CN2, Listing 3):  M = A^{-1} B and P = -h dt A^{-1}
 *   - the mean-flow operators of Eq. CN3/CN4 with the wall columns moved to the
 *     right-hand side (Sec. 3.2), and the unit pressure-gradient response
 *   - Clenshaw-Curtis quadrature weights on the same nodes (for the bulk flux).
 */
#include <stdlib.h>
#include <string.h>
#include <float.h>

#if defined(__x86_64__)
#include <quadmath.h>
typedef __float128 qreal;
#define Q_COS(x) cosq(x)
#define Q_PI M_PIq
#else
#if LDBL_MANT_DIG != 113
#error "oracle needs IEEE binary128 long double on this platform"
#endif
#include <math.h>
typedef long double qreal;
#define Q_COS(x) cosl(x)
#define Q_PI 3.141592653589793238462643383279502884L
#endif

/* ------------------------------------------------------------------ nodes */

/* y_j = -cos(pi j/(My-1)), j = 0..My-1: the Gauss-Lobatto points of cheb,
 * flipped so that y ascends from the bottom wall (-1) to the top wall (+1). */
static void nodes_q(int My, qreal* y) {
    int N = My - 1;
    for (int j = 0; j < My; ++j) y[j] = -Q_COS(Q_PI * (qreal)j / (qreal)N);
    /* exact symmetry and exact walls */
    y[0] = -1; y[N] = 1;
    if (N % 2 == 0) y[N / 2] = 0;
}

/* First-derivative collocation matrix on arbitrary distinct nodes x[0..n-1]:
 * the derivative of the Lagrange interpolant, in barycentric form
 *   D[j][k] = (c_j / c_k) / (x_j - x_k),  c_j = prod_{i != j} (x_j - x_i),
 *   D[j][j] = -sum_{k != j} D[j][k]   (derivative of a constant is zero). */
static void diff1_q(int n, const qreal* x, qreal* D) {
    qreal* c = (qreal*)malloc(sizeof(qreal) * n);
    for (int j = 0; j < n; ++j) {
        qreal p = 1;
        for (int i = 0; i < n; ++i) if (i != j) p *= (x[j] - x[i]);
        c[j] = p;
    }
    for (int j = 0; j < n; ++j) {
        qreal s = 0;
        for (int k = 0; k < n; ++k) {
            if (k == j) continue;
            qreal d = (c[j] / c[k]) / (x[j] - x[k]);
            D[j * n + k] = d;
            s += d;
        }
        D[j * n + j] = -s;
    }
    free(c);
}

/* C = A * B, all n x n row-major */
static void matmul_q(int n, const qreal* A, const qreal* B, qreal* C) {
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            qreal s = 0;
            for (int k = 0; k < n; ++k) s += A[i * n + k] * B[k * n + j];
            C[i * n + j] = s;
        }
}

/* D1 and D2 = D1*D1 on the full My-point grid (Listing 1: D2F = DYF*DYF). */
static void cheb_full_q(int My, qreal* y, qreal* D1, qreal* D2) {
    nodes_q(My, y);
    diff1_q(My, y, D1);
    matmul_q(My, D1, D1, D2);
}

/* Clamped fourth derivative on the Ny = My-2 interior nodes.
 * p(y) = w(y) q(y), w = (1-y^2)^2, q = interpolant of v_k / w(y_k) on the interior
 * nodes.  p'''' = w q'''' + 4 w' q''' + 6 w'' q'' + 4 w''' q' + w'''' q, with
 * w' = 4y^3 - 4y, w'' = 12y^2 - 4, w''' = 24y, w'''' = 24.  The interior
 * derivative matrices of q are powers of the interior first-derivative matrix
 * (exact for the degree Ny-1 interpolant). */
static void d4_clamped_q(int My, const qreal* y, qreal* D4c) {
    int n = My - 2;
    qreal* xi = (qreal*)malloc(sizeof(qreal) * n);
    for (int j = 0; j < n; ++j) xi[j] = y[j + 1];
    size_t nn = (size_t)n * n;
    qreal* T1 = (qreal*)malloc(sizeof(qreal) * nn);
    qreal* T2 = (qreal*)malloc(sizeof(qreal) * nn);
    qreal* T3 = (qreal*)malloc(sizeof(qreal) * nn);
    qreal* T4 = (qreal*)malloc(sizeof(qreal) * nn);
    diff1_q(n, xi, T1);
    matmul_q(n, T1, T1, T2);
    matmul_q(n, T2, T1, T3);
    matmul_q(n, T3, T1, T4);
    for (int j = 0; j < n; ++j) {
        qreal t = xi[j];
        qreal w0 = (1 - t * t) * (1 - t * t);
        qreal w1 = 4 * t * t * t - 4 * t;
        qreal w2 = 12 * t * t - 4;
        qreal w3 = 24 * t;
        qreal w4 = 24;
        for (int k = 0; k < n; ++k) {
            qreal tk = xi[k];
            qreal wk = (1 - tk * tk) * (1 - tk * tk);
            size_t o = (size_t)j * n + k;
            qreal v = w0 * T4[o] + 4 * w1 * T3[o] + 6 * w2 * T2[o] + 4 * w3 * T1[o];
            if (j == k) v += w4;
            D4c[o] = v / wk;
        }
    }
    free(xi); free(T1); free(T2); free(T3); free(T4);
}

/* Gauss-Jordan elimination with partial pivoting on the augmented matrix
 * [A | R] (n rows, A n x n, R n x m): on return R holds A^{-1} R.
 * Returns 0 on success, -1 on a zero pivot. */
static int gauss_jordan_q(int n, qreal* A, int m, qreal* R) {
    for (int col = 0; col < n; ++col) {
        int piv = col;
        qreal best = A[col * n + col] < 0 ? -A[col * n + col] : A[col * n + col];
        for (int r = col + 1; r < n; ++r) {
            qreal a = A[r * n + col] < 0 ? -A[r * n + col] : A[r * n + col];
            if (a > best) { best = a; piv = r; }
        }
        if (best == 0) return -1;
        if (piv != col) {
            for (int k = 0; k < n; ++k) { qreal t = A[col * n + k]; A[col * n + k] = A[piv * n + k]; A[piv * n + k] = t; }
            for (int k = 0; k < m; ++k) { qreal t = R[col * m + k]; R[col * m + k] = R[piv * m + k]; R[piv * m + k] = t; }
        }
        qreal inv = 1 / A[col * n + col];
        for (int k = 0; k < n; ++k) A[col * n + k] *= inv;
        for (int k = 0; k < m; ++k) R[col * m + k] *= inv;
        for (int r = 0; r < n; ++r) {
            if (r == col) continue;
            qreal f = A[r * n + col];
            if (f == 0) continue;
            for (int k = 0; k < n; ++k) A[r * n + k] -= f * A[col * n + k];
            for (int k = 0; k < m; ++k) R[r * m + k] -= f * R[col * m + k];
        }
    }
    return 0;
}

static void to_double(size_t cnt, const qreal* a, double* out) {
    for (size_t i = 0; i < cnt; ++i) out[i] = (double)a[i];
}

/* ------------------------------------------------------------- exported */

/* Grid: y[My], D1[My*My], D2[My*My], D4c[(My-2)^2], all row-major doubles. */
int orc_grid(int My, double* y, double* D1, double* D2, double* D4c) {
    if (My < 5) return -1;
    size_t m2 = (size_t)My * My, n2 = (size_t)(My - 2) * (My - 2);
    qreal* yq = (qreal*)malloc(sizeof(qreal) * My);
    qreal* a = (qreal*)malloc(sizeof(qreal) * m2);
    qreal* b = (qreal*)malloc(sizeof(qreal) * m2);
    qreal* c = (qreal*)malloc(sizeof(qreal) * n2);
    cheb_full_q(My, yq, a, b);
    d4_clamped_q(My, yq, c);
    if (y) to_double(My, yq, y);
    if (D1) to_double(m2, a, D1);
    if (D2) to_double(m2, b, D2);
    if (D4c) to_double(n2, c, D4c);
    free(yq); free(a); free(b); free(c);
    return 0;
}

/* Clenshaw-Curtis weights on the flipped CGL nodes, from the moment equations
 * sum_j w_j T_p(y_j) = int_{-1}^{1} T_p(y) dy  (= 2/(1-p^2) for even p, 0 for odd),
 * p = 0..My-1, solved directly. */
int orc_cc_weights(int My, double* w) {
    int n = My;
    qreal* yq = (qreal*)malloc(sizeof(qreal) * n);
    nodes_q(My, yq);
    qreal* A = (qreal*)malloc(sizeof(qreal) * n * n);
    qreal* R = (qreal*)malloc(sizeof(qreal) * n);
    int N = My - 1;
    for (int p = 0; p < n; ++p) {
        for (int j = 0; j < n; ++j) {
            /* T_p(y_j) with y_j = cos(pi (N-j)/N) */
            A[p * n + j] = Q_COS(Q_PI * (qreal)p * (qreal)(N - j) / (qreal)N);
        }
        R[p] = (p % 2 == 0) ? (qreal)2 / (1 - (qreal)p * p) : 0;
    }
    int rc = gauss_jordan_q(n, A, 1, R);
    to_double(n, R, w);
    free(yq); free(A); free(R);
    return rc;
}

/* Per-wavenumber CN operators for one sub-step length h (Eqs. CN1, CN2, Listing 3).
 *   g = h dt / (2 Re),  Delta = D2_int - k2 I,  DD = D4c - 2 k2 D2_int + k2^2 I
 *   v  : A = Delta - g DD,  B = Delta + g DD   (CN1 multiplied through by Delta)
 *   eta: A = I - g Delta,   B = I + g Delta
 *   M = A^{-1} B,  P = -h dt A^{-1}
 * Outputs are nk2 consecutive (My-2)^2 row-major blocks; any output may be NULL. */
int orc_cn_ops(int My, int nk2, const double* k2, double dt, double re, double h,
               double* Mv, double* Pv, double* Me, double* Pe) {
    int n = My - 2;
    size_t nn = (size_t)n * n;
    qreal* yq = (qreal*)malloc(sizeof(qreal) * My);
    qreal* D1 = (qreal*)malloc(sizeof(qreal) * My * My);
    qreal* D2 = (qreal*)malloc(sizeof(qreal) * My * My);
    qreal* D4 = (qreal*)malloc(sizeof(qreal) * nn);
    cheb_full_q(My, yq, D1, D2);
    d4_clamped_q(My, yq, D4);
    qreal* D2i = (qreal*)malloc(sizeof(qreal) * nn);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) D2i[i * n + j] = D2[(i + 1) * My + (j + 1)];
    qreal g = (qreal)h * (qreal)dt / (2 * (qreal)re);
    qreal hdt = (qreal)h * (qreal)dt;
    int status = 0;
#pragma omp parallel for schedule(dynamic) reduction(| : status)
    for (int q = 0; q < nk2; ++q) {
        qreal kk = (qreal)k2[q];
        qreal* A = (qreal*)malloc(sizeof(qreal) * nn);
        qreal* R = (qreal*)malloc(sizeof(qreal) * nn * 2);
        double* tmp = (double*)malloc(sizeof(double) * nn);
        /* v operator */
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                qreal del = D2i[i * n + j] - (i == j ? kk : 0);
                qreal dd = D4[i * n + j] - 2 * kk * D2i[i * n + j] + (i == j ? kk * kk : 0);
                A[i * n + j] = del - g * dd;
                R[i * 2 * n + j] = del + g * dd;            /* B */
                R[i * 2 * n + n + j] = (i == j) ? -hdt : 0; /* -h dt I */
            }
        if (gauss_jordan_q(n, A, 2 * n, R) != 0) status |= 1;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                if (Mv) Mv[q * nn + i * n + j] = (double)R[i * 2 * n + j];
                if (Pv) Pv[q * nn + i * n + j] = (double)R[i * 2 * n + n + j];
            }
        /* eta operator */
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                qreal del = D2i[i * n + j] - (i == j ? kk : 0);
                A[i * n + j] = (i == j ? 1 : 0) - g * del;
                R[i * 2 * n + j] = (i == j ? 1 : 0) + g * del;
                R[i * 2 * n + n + j] = (i == j) ? -hdt : 0;
            }
        if (gauss_jordan_q(n, A, 2 * n, R) != 0) status |= 1;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                if (Me) Me[q * nn + i * n + j] = (double)R[i * 2 * n + j];
                if (Pe) Pe[q * nn + i * n + j] = (double)R[i * 2 * n + n + j];
            }
        free(A); free(R); free(tmp);
    }
    free(yq); free(D1); free(D2); free(D4); free(D2i);
    return status ? -1 : 0;
}

/* Mean-flow operators of Eqs. CN3/CN4 for one h (Sec. 3.2): with
 * A = I - g D2_int, the wall columns of [I - g D2] are moved to the right-hand
 * side, so that  U_int(t+h dt) = MU U_int(t) + bU [U(-1), U(+1)] + PU f + gamma Ug:
 *   MU = A^{-1} (I + g D2_int),   bU = A^{-1} (2 g D2[int, {0, My-1}])  (n x 2),
 *   PU = -h dt A^{-1},            Ug = h dt A^{-1} 1.                          */
int orc_mean_ops(int My, double dt, double re, double h,
                 double* MU, double* PU, double* bU, double* Ug) {
    int n = My - 2;
    size_t nn = (size_t)n * n;
    qreal* yq = (qreal*)malloc(sizeof(qreal) * My);
    qreal* D1 = (qreal*)malloc(sizeof(qreal) * My * My);
    qreal* D2 = (qreal*)malloc(sizeof(qreal) * My * My);
    cheb_full_q(My, yq, D1, D2);
    qreal g = (qreal)h * (qreal)dt / (2 * (qreal)re);
    qreal hdt = (qreal)h * (qreal)dt;
    int m = 2 * n + 3;
    qreal* A = (qreal*)malloc(sizeof(qreal) * nn);
    qreal* R = (qreal*)malloc(sizeof(qreal) * n * m);
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j < n; ++j) {
            qreal d2 = D2[(i + 1) * My + (j + 1)];
            A[i * n + j] = (i == j ? 1 : 0) - g * d2;
            R[i * m + j] = (i == j ? 1 : 0) + g * d2;
            R[i * m + n + j] = (i == j) ? -hdt : 0;
        }
        R[i * m + 2 * n + 0] = 2 * g * D2[(i + 1) * My + 0];
        R[i * m + 2 * n + 1] = 2 * g * D2[(i + 1) * My + (My - 1)];
        R[i * m + 2 * n + 2] = hdt;
    }
    int rc = gauss_jordan_q(n, A, m, R);
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j < n; ++j) {
            if (MU) MU[i * n + j] = (double)R[i * m + j];
            if (PU) PU[i * n + j] = (double)R[i * m + n + j];
        }
        if (bU) { bU[i * 2 + 0] = (double)R[i * m + 2 * n]; bU[i * 2 + 1] = (double)R[i * m + 2 * n + 1]; }
        if (Ug) Ug[i] = (double)R[i * m + 2 * n + 2];
    }
    free(yq); free(D1); free(D2); free(A); free(R);
    return rc;
}

/* Dense solve in quad for tests: X = A^{-1} B (A n x n, B n x m, doubles in/out). */
int orc_solve(int n, const double* A, int m, const double* B, double* X) {
    qreal* a = (qreal*)malloc(sizeof(qreal) * n * n);
    qreal* r = (qreal*)malloc(sizeof(qreal) * n * m);
    for (int i = 0; i < n * n; ++i) a[i] = A[i];
    for (int i = 0; i < n * m; ++i) r[i] = B[i];
    int rc = gauss_jordan_q(n, a, m, r);
    to_double((size_t)n * m, r, X);
    free(a); free(r);
    return rc;
}

/* 2 pi / L rounded once to double: the fundamental wavenumber of a period L. */
double orc_fundamental(double L) { return (double)(2 * Q_PI / (qreal)L); }
