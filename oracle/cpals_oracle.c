/*
 * cpals_oracle.c -- plain, slow, FP64 CPU reference for CP-ALS-QR and CP-ALS.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg load this file's library.  It shares no code, header, table
 * or helper with the CUDA path.
 *
 * Source: Minster, Viviano, Liu, Ballard, "CP Decomposition for Tensors via
 * Alternating Least Squares with QR Decomposition" (arXiv 2112.10855).  Each
 * function names the passage it follows.  Everything is written out with plain
 * loops in the paper's order and notation.  There is no blocking and no
 * reordering beyond what the definition states.
 *
 * Conventions (paper Sec. 2.2, Kronecker index rule: the right operand's index
 * runs fastest):
 *  - matrices are column-major and 0-based: M(i,j) = M[i + rows*j];
 *  - a tensor of dims I_1..I_N stores element (i_1..i_N) at
 *    sum_m i_m prod_{k<m} I_k (mode 1 fastest);
 *  - the mode-n unfolding X_(n) is I_n x prod_{m!=n} I_m; column index
 *    sum_{m!=n} i_m prod_{k<m,k!=n} I_k.  This column order is the one that
 *    makes the Multi-TTM and the Khatri-Rao forms (Eq. multittm, Eq. cp_mat)
 *    consistent.
 *
 * Readings where the paper is silent (also listed in the design notes):
 *  - QR sign: Householder QR with diag(R) >= 0 (rows of R and columns of Q
 *    are flipped together);
 *  - column normalisation uses the 2-norm; a zero column keeps lambda = 0;
 *  - QR-solve singularity: |R0(k,k)| <= R * eps * max_j |R0(j,j)|;
 *  - SVD truncation keeps sigma_i > rtol * sigma_1;
 *  - the single TTMs run in decreasing-dimension order, ties by higher mode;
 *  - fit = 1 - sqrt(max(res^2, 0)) / ||X||.
 *
 * Parity-pinned by tests/test_oracle_pins.py.  That file checks each function
 * against numpy/LAPACK, brute-force explicit Kronecker forms, identities
 * and invariants.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAXN 16

/* ------------------------------------------------------------------ */
/* Small dense helpers                                                  */
/* ------------------------------------------------------------------ */

/* C (m x n) = A (m x k) * B (k x n), plain triple loop. */
void orc_matmul(int64_t m, int64_t k, int64_t n, const double* A, const double* B, double* C)
{
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < m; ++i) {
            double s = 0.0;
            for (int64_t p = 0; p < k; ++p) s += A[i + m * p] * B[p + k * j];
            C[i + m * j] = s;
        }
}

/* C (m x n) = A^T (A is k x m) * B (k x n). */
void orc_matmul_tn(int64_t m, int64_t k, int64_t n, const double* A, const double* B, double* C)
{
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < m; ++i) {
            double s = 0.0;
            for (int64_t p = 0; p < k; ++p) s += A[p + k * i] * B[p + k * j];
            C[i + m * j] = s;
        }
}

/* ------------------------------------------------------------------ */
/* Householder QR (Sec. 2.1: compact/thin QR A = QR, Q with the shape of */
/* A, R square), explicit Q, diag(R) >= 0.                              */
/* ------------------------------------------------------------------ */
/* Multiply-adds of the two O(m n^2) loop nests of orc_qr (the reflector
 * applications to W and to Q), summed over calls: the flop-count pin of
 * Eq. QRcost reads it.  The oracle is single-threaded. */
static int64_t g_qr_madds = 0;

int64_t orc_qr_madds(int reset)
{
    int64_t v = g_qr_madds;
    if (reset) g_qr_madds = 0;
    return v;
}

void orc_qr(int64_t m, int64_t n, const double* A, double* Q, double* R)
{
    double* W = (double*)malloc(sizeof(double) * (size_t)(m * n));
    double* V = (double*)calloc((size_t)(m * n), sizeof(double));   /* reflector j in column j */
    double* beta = (double*)calloc((size_t)n, sizeof(double));
    memcpy(W, A, sizeof(double) * (size_t)(m * n));

    for (int64_t j = 0; j < n; ++j) {
        double sigma = 0.0;
        for (int64_t i = j; i < m; ++i) sigma += W[i + m * j] * W[i + m * j];
        double norm = sqrt(sigma);
        if (norm == 0.0) { beta[j] = 0.0; continue; }        /* H_j = I */
        double alpha = (W[j + m * j] >= 0.0) ? -norm : norm;  /* new diagonal entry */
        double vnorm2 = 0.0;
        for (int64_t i = j; i < m; ++i) {
            double v = W[i + m * j];
            if (i == j) v -= alpha;
            V[i + m * j] = v;
            vnorm2 += v * v;
        }
        beta[j] = (vnorm2 > 0.0) ? 2.0 / vnorm2 : 0.0;
        /* apply H_j = I - beta v v^T to the remaining columns */
        for (int64_t k = j + 1; k < n; ++k) {
            double s = 0.0;
            for (int64_t i = j; i < m; ++i) s += V[i + m * j] * W[i + m * k];
            s *= beta[j];
            for (int64_t i = j; i < m; ++i) W[i + m * k] -= s * V[i + m * j];
            g_qr_madds += 2 * (m - j);
        }
        W[j + m * j] = alpha;
        for (int64_t i = j + 1; i < m; ++i) W[i + m * j] = 0.0;
    }
    /* R = upper triangle of W */
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < n; ++i) R[i + n * j] = (i <= j) ? W[i + m * j] : 0.0;
    /* Q = H_0 H_1 ... H_{n-1} [I_n; 0], accumulated backwards.  When H_j is
     * applied, columns k < j are still e_k, zero in rows j..m-1 where v_j
     * lives, so H_j leaves them as they are and only columns j..n-1 change.
     * With the loop above this is the 4 m n^2 - (4/3) n^3 flops of a
     * Householder QR with explicit Q (Sec. 3.2, Eq. QRcost). */
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < m; ++i) Q[i + m * j] = (i == j) ? 1.0 : 0.0;
    for (int64_t j = n - 1; j >= 0; --j) {
        if (beta[j] == 0.0) continue;
        for (int64_t k = j; k < n; ++k) {
            double s = 0.0;
            for (int64_t i = j; i < m; ++i) s += V[i + m * j] * Q[i + m * k];
            s *= beta[j];
            for (int64_t i = j; i < m; ++i) Q[i + m * k] -= s * V[i + m * j];
            g_qr_madds += 2 * (m - j);
        }
    }
    /* sign convention: diag(R) >= 0 */
    for (int64_t j = 0; j < n; ++j) {
        if (R[j + n * j] < 0.0) {
            for (int64_t k = 0; k < n; ++k) R[j + n * k] = -R[j + n * k];
            for (int64_t i = 0; i < m; ++i) Q[i + m * j] = -Q[i + m * j];
        }
    }
    free(W); free(V); free(beta);
}

/* ------------------------------------------------------------------ */
/* Khatri-Rao product (Sec. 2.2): column r of M_0 (.) M_1 (.) ... is     */
/* M_0(:,r) (x) M_1(:,r) (x) ..., the last matrix's row index fastest.  */
/* ------------------------------------------------------------------ */
void orc_krp(int nmat, const int64_t* rows, const double* const* mats, int64_t R, double* out)
{
    int64_t total = 1;
    for (int k = 0; k < nmat; ++k) total *= rows[k];
    double* cur = (double*)malloc(sizeof(double) * (size_t)total);
    double* nxt = (double*)malloc(sizeof(double) * (size_t)total);
    for (int64_t r = 0; r < R; ++r) {
        int64_t len = 1;
        cur[0] = 1.0;
        for (int k = 0; k < nmat; ++k) {
            /* Kronecker rule: [a (x) b](K*i + k) = a(i) b(k) */
            int64_t K = rows[k];
            for (int64_t i = 0; i < len; ++i)
                for (int64_t kk = 0; kk < K; ++kk)
                    nxt[K * i + kk] = cur[i] * mats[k][kk + K * r];
            len *= K;
            double* t = cur; cur = nxt; nxt = t;
        }
        memcpy(out + total * r, cur, sizeof(double) * (size_t)total);
    }
    free(cur); free(nxt);
}

/* ------------------------------------------------------------------ */
/* Unfolding X_(n) (Sec. 2.2) and TTM Y = X x_mode U (Sec. 2.2)          */
/* ------------------------------------------------------------------ */
void orc_unfold(int N, const int64_t* dims, const double* X, int n, double* Xn)
{
    int64_t P = 1, stride[ORC_MAXN], idx[ORC_MAXN];
    for (int m = 0; m < N; ++m) P *= dims[m];
    int64_t s = 1;
    for (int m = 0; m < N; ++m) {
        if (m == n) { stride[m] = 0; continue; }
        stride[m] = s; s *= dims[m];
    }
    for (int m = 0; m < N; ++m) idx[m] = 0;
    for (int64_t lin = 0; lin < P; ++lin) {
        int64_t col = 0;
        for (int m = 0; m < N; ++m) col += idx[m] * stride[m];
        Xn[idx[n] + dims[n] * col] = X[lin];
        for (int m = 0; m < N; ++m) {            /* advance the multi-index, mode 1 fastest */
            if (++idx[m] < dims[m]) break;
            idx[m] = 0;
        }
    }
}

/* Y(i_1..j..i_N) = sum_{i_mode} X(i_1..i_mode..i_N) U(j, i_mode); U is J x I_mode. */
void orc_ttm(int N, const int64_t* dims, const double* X, int mode, int64_t J, const double* U,
             double* Y)
{
    int64_t L = 1, T = 1, K = dims[mode];
    for (int m = 0; m < mode; ++m) L *= dims[m];
    for (int m = mode + 1; m < N; ++m) T *= dims[m];
    for (int64_t t = 0; t < T; ++t)
        for (int64_t j = 0; j < J; ++j)
            for (int64_t l = 0; l < L; ++l) {
                double s = 0.0;
                for (int64_t k = 0; k < K; ++k) s += X[l + L * (k + K * t)] * U[j + J * k];
                Y[l + L * (j + J * t)] = s;
            }
}

/* Default TTM order of Sec. 3.2: decreasing dimension, ties by higher mode. */
static void default_order(int N, const int64_t* dims, int n, int* order)
{
    int cnt = 0;
    for (int m = 0; m < N; ++m) if (m != n) order[cnt++] = m;
    for (int a = 0; a < cnt; ++a)
        for (int b = a + 1; b < cnt; ++b) {
            int x = order[a], y = order[b];
            if (dims[y] > dims[x] || (dims[y] == dims[x] && y > x)) { order[a] = y; order[b] = x; }
        }
}

void orc_ttm_order(int N, const int64_t* dims, int n, int* order) { default_order(N, dims, n, order); }

/*
 * Multi-TTM of Eq. multittm / Alg. cp-als-qr (the Multi-TTM step):
 * Y = X x_1 Q_1^T ... (all modes but n), as a sequence of single TTMs in
 * `order` (N-1 modes; NULL = decreasing dimension).  The result is written
 * as the unfolding Y_(n), I_n x R^{N-1}.
 * Returns the number of multiply-adds performed (for the flop-count pin).
 */
int64_t orc_multi_ttm(int N, const int64_t* dims, const double* X, int n, int64_t R,
                      const double* const* Q, const int* order, double* Yn)
{
    int ord[ORC_MAXN];
    if (order) for (int k = 0; k < N - 1; ++k) ord[k] = order[k];
    else default_order(N, dims, n, ord);

    int64_t cur_dims[ORC_MAXN];
    for (int m = 0; m < N; ++m) cur_dims[m] = dims[m];
    int64_t P = 1;
    for (int m = 0; m < N; ++m) P *= dims[m];
    double* cur = (double*)malloc(sizeof(double) * (size_t)P);
    memcpy(cur, X, sizeof(double) * (size_t)P);
    int64_t madds = 0;
    for (int k = 0; k < N - 1; ++k) {
        int m = ord[k];
        /* U = Q_m^T (R x I_m) */
        double* U = (double*)malloc(sizeof(double) * (size_t)(R * dims[m]));
        for (int64_t i = 0; i < dims[m]; ++i)
            for (int64_t r = 0; r < R; ++r) U[r + R * i] = Q[m][i + dims[m] * r];
        int64_t newP = P / cur_dims[m] * R;
        double* nxt = (double*)malloc(sizeof(double) * (size_t)newP);
        orc_ttm(N, cur_dims, cur, m, R, U, nxt);
        madds += P * R;
        cur_dims[m] = R;
        P = newP;
        free(U); free(cur);
        cur = nxt;
    }
    orc_unfold(N, cur_dims, cur, n, Yn);
    free(cur);
    return madds;
}

/* ------------------------------------------------------------------ */
/* Solves                                                               */
/* ------------------------------------------------------------------ */

/* Eq. ls-qr-q0-step solved by substitution: Ahat R0^T = W, i.e.
 * R0 Ahat(i,:)^T = W(i,:)^T for each row i (R0 upper triangular).
 * Returns 1 (and leaves Ahat untouched) if R0 is numerically singular. */
int orc_trsm_qr(int64_t I, int64_t R, const double* W, const double* R0, double* Ahat)
{
    double dmax = 0.0;
    for (int64_t k = 0; k < R; ++k) dmax = fmax(dmax, fabs(R0[k + R * k]));
    for (int64_t k = 0; k < R; ++k)
        if (!(fabs(R0[k + R * k]) > (double)R * 2.220446049250313e-16 * dmax)) return 1;
    double* x = (double*)malloc(sizeof(double) * (size_t)R);
    for (int64_t i = 0; i < I; ++i) {
        for (int64_t k = R - 1; k >= 0; --k) {
            double s = W[i + I * k];
            for (int64_t j = k + 1; j < R; ++j) s -= R0[k + R * j] * x[j];
            x[k] = s / R0[k + R * k];
        }
        for (int64_t k = 0; k < R; ++k) Ahat[i + I * k] = x[k];
    }
    free(x);
    return 0;
}

/* One-sided Jacobi SVD (Hestenes): rotate column pairs of B = A until
 * they are orthogonal; then A V = B = U Sigma.  Singular values sorted
 * descending.  A is n x n; U, V n x n; S length n. */
void orc_jacobi_svd(int64_t n, const double* A, double* U, double* S, double* V)
{
    double* B = (double*)malloc(sizeof(double) * (size_t)(n * n));
    double* Vt = (double*)malloc(sizeof(double) * (size_t)(n * n));
    memcpy(B, A, sizeof(double) * (size_t)(n * n));
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < n; ++i) Vt[i + n * j] = (i == j) ? 1.0 : 0.0;
    const double eps = 2.220446049250313e-16;
    for (int sweep = 0; sweep < 80; ++sweep) {
        int rotated = 0;
        for (int64_t p = 0; p < n - 1; ++p)
            for (int64_t q = p + 1; q < n; ++q) {
                double a = 0.0, b = 0.0, g = 0.0;
                for (int64_t i = 0; i < n; ++i) {
                    a += B[i + n * p] * B[i + n * p];
                    b += B[i + n * q] * B[i + n * q];
                    g += B[i + n * p] * B[i + n * q];
                }
                if (g == 0.0 || fabs(g) <= eps * sqrt(a * b)) continue;
                rotated = 1;
                double zeta = (b - a) / (2.0 * g);
                double t = ((zeta >= 0.0) ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
                for (int64_t i = 0; i < n; ++i) {
                    double bp = B[i + n * p], bq = B[i + n * q];
                    B[i + n * p] = c * bp - s * bq;
                    B[i + n * q] = s * bp + c * bq;
                    double vp = Vt[i + n * p], vq = Vt[i + n * q];
                    Vt[i + n * p] = c * vp - s * vq;
                    Vt[i + n * q] = s * vp + c * vq;
                }
            }
        if (!rotated) break;
    }
    /* column norms and sort descending (selection sort keeps it plain) */
    int64_t* perm = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    double* sig = (double*)malloc(sizeof(double) * (size_t)n);
    for (int64_t j = 0; j < n; ++j) {
        double s = 0.0;
        for (int64_t i = 0; i < n; ++i) s += B[i + n * j] * B[i + n * j];
        sig[j] = sqrt(s);
        perm[j] = j;
    }
    for (int64_t a = 0; a < n; ++a)
        for (int64_t b = a + 1; b < n; ++b)
            if (sig[perm[b]] > sig[perm[a]]) { int64_t t = perm[a]; perm[a] = perm[b]; perm[b] = t; }
    for (int64_t j = 0; j < n; ++j) {
        int64_t src = perm[j];
        S[j] = sig[src];
        for (int64_t i = 0; i < n; ++i) {
            U[i + n * j] = (sig[src] > 0.0) ? B[i + n * src] / sig[src] : 0.0;
            V[i + n * j] = Vt[i + n * src];
        }
    }
    free(B); free(Vt); free(perm); free(sig);
}

/* CP-ALS-QR-SVD solve (Sec. 3.1): R0 = U Sigma V^T, Ahat = W U Sigma^+ V^T,
 * keeping sigma_i > rtol * sigma_1.  Returns the number of kept values. */
int orc_svd_solve(int64_t I, int64_t R, const double* W, const double* R0, double rtol,
                  double* Ahat)
{
    double* U = (double*)malloc(sizeof(double) * (size_t)(R * R));
    double* V = (double*)malloc(sizeof(double) * (size_t)(R * R));
    double* S = (double*)malloc(sizeof(double) * (size_t)R);
    double* WU = (double*)malloc(sizeof(double) * (size_t)(I * R));
    orc_jacobi_svd(R, R0, U, S, V);
    orc_matmul(I, R, R, W, U, WU);                          /* W U */
    int kept = 0;
    for (int64_t j = 0; j < R; ++j) {                       /* (W U) Sigma^+ */
        int keep = S[j] > rtol * S[0] && S[j] > 0.0;
        kept += keep;
        for (int64_t i = 0; i < I; ++i) WU[i + I * j] = keep ? WU[i + I * j] / S[j] : 0.0;
    }
    for (int64_t i = 0; i < I; ++i)                          /* ... V^T */
        for (int64_t k = 0; k < R; ++k) {
            double s = 0.0;
            for (int64_t j = 0; j < R; ++j) s += WU[i + I * j] * V[k + R * j];
            Ahat[i + I * k] = s;
        }
    free(U); free(V); free(S); free(WU);
    return kept;
}

/* Normalise columns (Alg. cp-als-qr, normalisation step): lambda_r = ||Ahat(:,r)||_2. */
void orc_normalize(int64_t I, int64_t R, const double* Ahat, double* A, double* lambda)
{
    for (int64_t r = 0; r < R; ++r) {
        double s = 0.0;
        for (int64_t i = 0; i < I; ++i) s += Ahat[i + I * r] * Ahat[i + I * r];
        double l = sqrt(s);
        lambda[r] = l;
        for (int64_t i = 0; i < I; ++i) A[i + I * r] = (l > 0.0) ? Ahat[i + I * r] / l : Ahat[i + I * r];
    }
}

/* MTTKRP M_n = X_(n) Z_n (Alg. cp-als, MTTKRP step), element by element:
 * M(i_n, r) = sum over all X entries of X(i) prod_{m != n} A_m(i_m, r). */
void orc_mttkrp(int N, const int64_t* dims, const double* X, int n, int64_t R,
                const double* const* A, double* M)
{
    int64_t P = 1, idx[ORC_MAXN];
    for (int m = 0; m < N; ++m) { P *= dims[m]; idx[m] = 0; }
    for (int64_t k = 0; k < dims[n] * R; ++k) M[k] = 0.0;
    for (int64_t lin = 0; lin < P; ++lin) {
        double x = X[lin];
        for (int64_t r = 0; r < R; ++r) {
            double p = x;
            for (int m = 0; m < N; ++m)
                if (m != n) p *= A[m][idx[m] + dims[m] * r];
            M[idx[n] + dims[n] * r] += p;
        }
        for (int m = 0; m < N; ++m) {
            if (++idx[m] < dims[m]) break;
            idx[m] = 0;
        }
    }
}

/* Normal-equations solve of Alg. cp-als: Ahat S = M with S symmetric positive
 * definite, by Cholesky S = L L^T (MATLAB backslash in the paper).  Returns 1
 * if S is not positive definite. */
int orc_cholesky_solve(int64_t I, int64_t R, const double* M, const double* S, double* Ahat)
{
    double* L = (double*)calloc((size_t)(R * R), sizeof(double));
    for (int64_t j = 0; j < R; ++j) {
        double d = S[j + R * j];
        for (int64_t k = 0; k < j; ++k) d -= L[j + R * k] * L[j + R * k];
        if (!(d > 0.0)) { free(L); return 1; }
        L[j + R * j] = sqrt(d);
        for (int64_t i = j + 1; i < R; ++i) {
            double s = S[i + R * j];
            for (int64_t k = 0; k < j; ++k) s -= L[i + R * k] * L[j + R * k];
            L[i + R * j] = s / L[j + R * j];
        }
    }
    double* y = (double*)malloc(sizeof(double) * (size_t)R);
    for (int64_t i = 0; i < I; ++i) {
        /* S x = m: L y = m, L^T x = y */
        for (int64_t k = 0; k < R; ++k) {
            double s = M[i + I * k];
            for (int64_t j = 0; j < k; ++j) s -= L[k + R * j] * y[j];
            y[k] = s / L[k + R * k];
        }
        for (int64_t k = R - 1; k >= 0; --k) {
            double s = y[k];
            for (int64_t j = k + 1; j < R; ++j) s -= L[j + R * k] * Ahat[i + I * j];
            Ahat[i + I * k] = s / L[k + R * k];
        }
    }
    free(L); free(y);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Errors (Sec. 3.3.1)                                                  */
/* ------------------------------------------------------------------ */

/* ||X - Xhat||_F with Xhat = sum_r lambda_r a_r^(1) o ... o a_r^(N) formed entry by entry. */
double orc_residual_direct(int N, const int64_t* dims, const double* X, int64_t R,
                           const double* lambda, const double* const* A)
{
    int64_t P = 1, idx[ORC_MAXN];
    for (int m = 0; m < N; ++m) { P *= dims[m]; idx[m] = 0; }
    double s = 0.0;
    for (int64_t lin = 0; lin < P; ++lin) {
        double xh = 0.0;
        for (int64_t r = 0; r < R; ++r) {
            double p = lambda[r];
            for (int m = 0; m < N; ++m) p *= A[m][idx[m] + dims[m] * r];
            xh += p;
        }
        double d = X[lin] - xh;
        s += d * d;
        for (int m = 0; m < N; ++m) {
            if (++idx[m] < dims[m]) break;
            idx[m] = 0;
        }
    }
    return sqrt(s);
}

double orc_norm2(int64_t P, const double* X)
{
    double s = 0.0;
    for (int64_t i = 0; i < P; ++i) s += X[i] * X[i];
    return s;
}

/* Efficient CP-ALS-QR error of Sec. 3.3.1:
 * res^2 = ||X||^2 - 2 <W_N, Ahat_N R0^T> + <R0^T R0, diag(l) R_N^T R_N diag(l)>. */
double orc_fit_efficient_qr(double normX2, int64_t IN, int64_t R, const double* WN,
                            const double* AhatN, const double* R0, const double* RN,
                            const double* lambda)
{
    double inner = 0.0;
    for (int64_t i = 0; i < IN; ++i)
        for (int64_t k = 0; k < R; ++k) {
            double s = 0.0;                       /* (Ahat_N R0^T)(i,k) */
            for (int64_t j = 0; j < R; ++j) s += AhatN[i + IN * j] * R0[k + R * j];
            inner += WN[i + IN * k] * s;
        }
    double nrm = 0.0;
    for (int64_t a = 0; a < R; ++a)
        for (int64_t b = 0; b < R; ++b) {
            double g0 = 0.0, gN = 0.0;           /* (R0^T R0)(a,b), (R_N^T R_N)(a,b) */
            for (int64_t k = 0; k < R; ++k) {
                g0 += R0[k + R * a] * R0[k + R * b];
                gN += RN[k + R * a] * RN[k + R * b];
            }
            nrm += g0 * lambda[a] * gN * lambda[b];
        }
    double res2 = normX2 - 2.0 * inner + nrm;
    if (res2 < 0.0) res2 = 0.0;
    return 1.0 - sqrt(res2) / sqrt(normX2);
}

/* Efficient CP-ALS error of Sec. 3.3.1: <X, Xhat> = <M_N, Ahat_N>,
 * ||Xhat||^2 = <S_N, diag(l) G_N diag(l)>. */
double orc_fit_efficient_normal(double normX2, int64_t IN, int64_t R, const double* MN,
                                const double* AhatN, const double* SN, const double* GN,
                                const double* lambda)
{
    double inner = 0.0;
    for (int64_t k = 0; k < IN * R; ++k) inner += MN[k] * AhatN[k];
    double nrm = 0.0;
    for (int64_t a = 0; a < R; ++a)
        for (int64_t b = 0; b < R; ++b) nrm += SN[a + R * b] * lambda[a] * GN[a + R * b] * lambda[b];
    double res2 = normX2 - 2.0 * inner + nrm;
    if (res2 < 0.0) res2 = 0.0;
    return 1.0 - sqrt(res2) / sqrt(normX2);
}

/* ------------------------------------------------------------------ */
/* Driver state: Alg. cp-als-qr and Alg. cp-als                        */
/* ------------------------------------------------------------------ */
enum { ORC_QR = 0, ORC_SVD = 1, ORC_NORMAL = 2, ORC_NORMAL_PINV = 3 };

typedef struct {
    int N;
    int64_t dims[ORC_MAXN];
    int64_t R;
    const double* X;          /* borrowed */
    double normX2;
    double* A[ORC_MAXN];      /* normalised factors, I_m x R */
    double* Q[ORC_MAXN];      /* A_m = Q_m R_m */
    double* Rf[ORC_MAXN];
    double* G[ORC_MAXN];      /* Gram A_m^T A_m */
    double* lambda;
    /* last mode update, for the error and for parity checks */
    int last_mode;
    double* V; double* Q0; double* R0;      /* R^{N-1} x R, R x R */
    double* Y; double* W; double* Ahat; double* M; double* S;
    double last_fit;
    int last_status;
} orc_state;

orc_state* orc_create(int N, const int64_t* dims, int64_t R, const double* X)
{
    if (N < 2 || N > ORC_MAXN || R < 1) return NULL;
    orc_state* st = (orc_state*)calloc(1, sizeof(orc_state));
    st->N = N; st->R = R; st->X = X;
    int64_t P = 1, Imax = 0, RN1 = 1;
    for (int m = 0; m < N; ++m) {
        st->dims[m] = dims[m]; P *= dims[m];
        if (dims[m] > Imax) Imax = dims[m];
        st->A[m] = (double*)calloc((size_t)(dims[m] * R), sizeof(double));
        st->Q[m] = (double*)calloc((size_t)(dims[m] * R), sizeof(double));
        st->Rf[m] = (double*)calloc((size_t)(R * R), sizeof(double));
        st->G[m] = (double*)calloc((size_t)(R * R), sizeof(double));
    }
    for (int m = 0; m < N - 1; ++m) RN1 *= R;
    st->lambda = (double*)calloc((size_t)R, sizeof(double));
    st->V = (double*)calloc((size_t)(RN1 * R), sizeof(double));
    st->Q0 = (double*)calloc((size_t)(RN1 * R), sizeof(double));
    st->R0 = (double*)calloc((size_t)(R * R), sizeof(double));
    st->Y = (double*)calloc((size_t)(Imax * RN1), sizeof(double));
    st->W = (double*)calloc((size_t)(Imax * R), sizeof(double));
    st->Ahat = (double*)calloc((size_t)(Imax * R), sizeof(double));
    st->M = (double*)calloc((size_t)(Imax * R), sizeof(double));
    st->S = (double*)calloc((size_t)(R * R), sizeof(double));
    st->normX2 = orc_norm2(P, X);
    st->last_mode = -1;
    return st;
}

void orc_destroy(orc_state* st)
{
    if (!st) return;
    for (int m = 0; m < st->N; ++m) { free(st->A[m]); free(st->Q[m]); free(st->Rf[m]); free(st->G[m]); }
    free(st->lambda); free(st->V); free(st->Q0); free(st->R0); free(st->Y); free(st->W);
    free(st->Ahat); free(st->M); free(st->S); free(st);
}

/* Initialisation (Alg. cp-als-qr: initial factors, then their compact QR;
 * Alg. cp-als: initial Grams).  lambda = NULL means ones. */
void orc_set_factors(orc_state* st, const double* const* A, const double* lambda)
{
    for (int m = 0; m < st->N; ++m) {
        memcpy(st->A[m], A[m], sizeof(double) * (size_t)(st->dims[m] * st->R));
        orc_qr(st->dims[m], st->R, st->A[m], st->Q[m], st->Rf[m]);
        orc_matmul_tn(st->R, st->dims[m], st->R, st->A[m], st->A[m], st->G[m]);
    }
    for (int64_t r = 0; r < st->R; ++r) st->lambda[r] = lambda ? lambda[r] : 1.0;
}

/* KRP of the triangular factors and its QR (Alg. cp-als-qr, first two steps of
 * the mode loop): V_n = R_N (.) ... (.) R_{n+1} (.) R_{n-1} (.) ... (.) R_1 = Q0 R0. */
void orc_krp_qr(orc_state* st, int n)
{
    const double* mats[ORC_MAXN];
    int64_t rows[ORC_MAXN];
    int cnt = 0;
    for (int m = st->N - 1; m >= 0; --m)
        if (m != n) { mats[cnt] = st->Rf[m]; rows[cnt] = st->R; ++cnt; }
    orc_krp(cnt, rows, mats, st->R, st->V);
    int64_t RN1 = 1;
    for (int k = 0; k < st->N - 1; ++k) RN1 *= st->R;
    orc_qr(RN1, st->R, st->V, st->Q0, st->R0);
}

/* One CP-ALS-QR mode update (Alg. cp-als-qr mode loop) or one CP-ALS mode update
 * (Alg. cp-als mode loop, Cholesky or pseudo-inverse solve).  Returns 0 on success, 1 if the solve was singular
 * (factor left unchanged). */
int orc_update_mode(orc_state* st, int n, int solve, double rtol)
{
    const int N = st->N;
    const int64_t R = st->R, In = st->dims[n];
    int64_t RN1 = 1;
    for (int k = 0; k < N - 1; ++k) RN1 *= R;
    st->last_mode = n;
    if (solve == ORC_NORMAL || solve == ORC_NORMAL_PINV) {
        /* S_n = Hadamard product of the other Grams */
        for (int64_t k = 0; k < R * R; ++k) st->S[k] = 1.0;
        for (int m = 0; m < N; ++m)
            if (m != n)
                for (int64_t k = 0; k < R * R; ++k) st->S[k] *= st->G[m][k];
        orc_mttkrp(N, st->dims, st->X, n, R, (const double* const*)st->A, st->M);
        if (solve == ORC_NORMAL) {
            if (orc_cholesky_solve(In, R, st->M, st->S, st->Ahat)) { st->last_status = 1; return 1; }
        } else {
            /* CP-ALS-PINV (Sec. 2.3): Ahat = M pinv(S); S symmetric, so pinv(S^T) = pinv(S)
               and the SVD solve of Sec. 2.1 applies with S in place of R0 */
            orc_svd_solve(In, R, st->M, st->S, rtol, st->Ahat);
        }
    } else {
        orc_krp_qr(st, n);
        orc_multi_ttm(N, st->dims, st->X, n, R, (const double* const*)st->Q, NULL, st->Y);
        orc_matmul(In, RN1, R, st->Y, st->Q0, st->W);                 /* W_n = Y_(n) Q0 */
        if (solve == ORC_QR) {
            if (orc_trsm_qr(In, R, st->W, st->R0, st->Ahat)) { st->last_status = 1; return 1; }
        } else {
            orc_svd_solve(In, R, st->W, st->R0, rtol, st->Ahat);
        }
    }
    orc_normalize(In, R, st->Ahat, st->A[n], st->lambda);
    orc_qr(In, R, st->A[n], st->Q[n], st->Rf[n]);                       /* A_n = Q_n R_n */
    orc_matmul_tn(R, In, R, st->A[n], st->A[n], st->G[n]);               /* G_n */
    st->last_status = 0;
    return 0;
}

/* Efficient fit after the update of the last mode (Sec. 3.3.1). */
double orc_fit_last(orc_state* st, int solve)
{
    const int n = st->N - 1;
    if (solve == ORC_NORMAL || solve == ORC_NORMAL_PINV)
        return orc_fit_efficient_normal(st->normX2, st->dims[n], st->R, st->M, st->Ahat, st->S,
                                        st->G[n], st->lambda);
    return orc_fit_efficient_qr(st->normX2, st->dims[n], st->R, st->W, st->Ahat, st->R0,
                                st->Rf[n], st->lambda);
}

/* Outer loop (Alg. cp-als-qr / cp-als): `iters` sweeps over the modes; stop
 * early when |fit change| < tol (tol > 0).  fits[it] receives the efficient fit
 * after each sweep.  Returns the number of sweeps run, or -(it+1) if a solve
 * was singular in sweep it. */
int orc_iterate(orc_state* st, int iters, double tol, int solve, double rtol, double* fits)
{
    double prev = 0.0;
    for (int it = 0; it < iters; ++it) {
        for (int n = 0; n < st->N; ++n)
            if (orc_update_mode(st, n, solve, rtol)) return -(it + 1);
        double f = orc_fit_last(st, solve);
        if (fits) fits[it] = f;
        st->last_fit = f;
        if (tol > 0.0 && it > 0 && fabs(f - prev) < tol) return it + 1;
        prev = f;
    }
    return iters;
}

double orc_fit_direct(orc_state* st)
{
    double res = orc_residual_direct(st->N, st->dims, st->X, st->R, st->lambda,
                                     (const double* const*)st->A);
    return 1.0 - res / sqrt(st->normX2);
}

/* Accessors (copy out). */
double orc_get_normX2(const orc_state* st) { return st->normX2; }
void orc_get_factor(const orc_state* st, int m, double* A) { memcpy(A, st->A[m], sizeof(double) * (size_t)(st->dims[m] * st->R)); }
void orc_get_qr_factor(const orc_state* st, int m, double* Q, double* Rm)
{
    memcpy(Q, st->Q[m], sizeof(double) * (size_t)(st->dims[m] * st->R));
    memcpy(Rm, st->Rf[m], sizeof(double) * (size_t)(st->R * st->R));
}
void orc_get_lambda(const orc_state* st, double* l) { memcpy(l, st->lambda, sizeof(double) * (size_t)st->R); }
void orc_get_last(const orc_state* st, double* Q0, double* R0, double* Y, double* W, double* Ahat)
{
    int64_t RN1 = 1;
    for (int k = 0; k < st->N - 1; ++k) RN1 *= st->R;
    int64_t In = st->dims[st->last_mode < 0 ? 0 : st->last_mode];
    if (Q0) memcpy(Q0, st->Q0, sizeof(double) * (size_t)(RN1 * st->R));
    if (R0) memcpy(R0, st->R0, sizeof(double) * (size_t)(st->R * st->R));
    if (Y) memcpy(Y, st->Y, sizeof(double) * (size_t)(In * RN1));
    if (W) memcpy(W, st->W, sizeof(double) * (size_t)(In * st->R));
    if (Ahat) memcpy(Ahat, st->Ahat, sizeof(double) * (size_t)(In * st->R));
}
void orc_get_mttkrp(const orc_state* st, double* M, double* S)
{
    int64_t In = st->dims[st->last_mode < 0 ? 0 : st->last_mode];
    if (M) memcpy(M, st->M, sizeof(double) * (size_t)(In * st->R));
    if (S) memcpy(S, st->S, sizeof(double) * (size_t)(st->R * st->R));
}

/* ------------------------------------------------------------------ */
/* Factor match score (Sec. 4.2 metric; formula not printed in the paper):
 * unit-normalised columns, score = max over permutations pi of
 * (1/R) sum_r (1 - |l_r - m_pi(r)| / max(l_r, m_pi(r))) prod_n |a_r^(n)T b_pi(r)^(n)|.
 * Brute force over permutations (R <= 9); returns -1 for larger R. */
/* ------------------------------------------------------------------ */
static double score_perm(int N, const int64_t* dims, int64_t R, const double* l1,
                         const double* const* A1, const double* l2, const double* const* A2,
                         const int64_t* pi)
{
    double total = 0.0;
    for (int64_t r = 0; r < R; ++r) {
        int64_t q = pi[r];
        double lm = fmax(l1[r], l2[q]);
        double term = (lm > 0.0) ? 1.0 - fabs(l1[r] - l2[q]) / lm : 1.0;
        for (int m = 0; m < N; ++m) {
            double d = 0.0, n1 = 0.0, n2 = 0.0;
            for (int64_t i = 0; i < dims[m]; ++i) {
                double a = A1[m][i + dims[m] * r], b = A2[m][i + dims[m] * q];
                d += a * b; n1 += a * a; n2 += b * b;
            }
            term *= (n1 > 0.0 && n2 > 0.0) ? fabs(d) / sqrt(n1 * n2) : 0.0;
        }
        total += term;
    }
    return total / (double)R;
}

double orc_score(int N, const int64_t* dims, int64_t R, const double* l1, const double* const* A1,
                 const double* l2, const double* const* A2)
{
    if (R > 9) return -1.0;
    int64_t pi[9], c[9];
    for (int64_t i = 0; i < R; ++i) { pi[i] = i; c[i] = 0; }
    double best = score_perm(N, dims, R, l1, A1, l2, A2, pi);
    int64_t i = 1;
    while (i < R) {                     /* Heap's algorithm over all permutations */
        if (c[i] < i) {
            int64_t a = (i % 2 == 0) ? 0 : c[i];
            int64_t t = pi[a]; pi[a] = pi[i]; pi[i] = t;
            double s = score_perm(N, dims, R, l1, A1, l2, A2, pi);
            if (s > best) best = s;
            ++c[i]; i = 1;
        } else { c[i] = 0; ++i; }
    }
    return best;
}
