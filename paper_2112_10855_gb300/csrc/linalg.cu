// linalg.cu -- the small FP64 linear algebra of a CP-ALS-QR mode update
// (Alg. cp-als-qr): Householder QR of the factors and of the Khatri-Rao
// product V_n (Sec. 3.1, Eq. Z_qr), W_n = Y_(n) Q0, the R0 substitution or the
// truncated SVD solve, column normalisation, Grams and Cholesky for the
// normal-equations baseline (Alg. cp-als), and the efficient fit (Sec. 3.3.1).
//
// FP64 on this part runs at 2 DFMA/clk/SM, so every step that is not O(R^3)
// is spread over many CTAs: tall QRs go through a recursive TSQR whose leaves
// are Householder QRs in shared memory, and the GEMM and fit reductions are
// split over row blocks and then reduced in a fixed order (deterministic).
#include <algorithm>

#include "dev_common.cuh"
#include "internal.cuh"

namespace cpals {

namespace {

constexpr int kQrThreads = 512;

// dlarfg for a column with leading entry alpha and tail sum of squares s:
// H = I - tau v v^T with v = [1; scale * tail] maps the column to beta e_1
// (|beta| = its norm, sign opposite to alpha; tau = 0 when the tail is zero).
// tau = d / beta and scale = -1 / d with d = beta - alpha take one division.
__device__ __forceinline__ void hh_reflector(double alpha, double s, double* tau_j, double* scale, double* diag)
{
    double t = 0.0, sc = 0.0, beta = alpha;
    if (s > 0.0) {
        const double nrm = sqrt(fma(alpha, alpha, s));
        beta = (alpha >= 0.0) ? -nrm : nrm;
        const double d = beta - alpha;
        const double r = 1.0 / (beta * d);
        t = d * d * r;
        sc = -beta * r;
    }
    *tau_j = t;
    *scale = sc;
    *diag = beta;
}

// ---------------------------------------------------------------- Householder
// CTA b factors rows [off_b, off_{b+1}) of the m x n matrix A (lda), with
// off_b = b*m/nb, into an explicit Q_b (written to the same rows of Qout, ldq)
// and R_b (written to rows [b*n, (b+1)*n) of Rout, ldr).  Reflectors follow
// LAPACK's dlarfg form H = I - tau v v^T with v(0) = 1; the diagonal of R is
// made non-negative by flipping the matching row of R and column of Q.
__global__ void __launch_bounds__(kQrThreads) hh_qr_blocks_kernel(
    const double* __restrict__ A, int64_t lda, int64_t m, int n, int nb, double* __restrict__ Qout,
    int64_t ldq, double* __restrict__ Rout, int64_t ldr, const int* __restrict__ status, const int* __restrict__ gate)
{
    if (*status != kStatusOk || (gate && *gate == 0)) return;
    extern __shared__ double sm[];
    const int b = blockIdx.x;
    const int64_t off = (int64_t)b * m / nb, end = (int64_t)(b + 1) * m / nb;
    const int mb = (int)(end - off);
    double* W = sm;                       // mb x n (reflectors below the diagonal, R above)
    double* Qs = sm + (size_t)mb * n;     // mb x n
    double* tau = Qs + (size_t)mb * n;    // n
    double* red = tau + n;                // 32 scratch
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = kQrThreads / 32;

    for (int64_t e = tid; e < (int64_t)mb * n; e += kQrThreads) {
        const int j = (int)(e / mb), i = (int)(e - (int64_t)j * mb);
        W[e] = A[(off + i) + lda * j];
    }
    __syncthreads();

    const int kmax = min(mb, n);
    // Look-ahead: in step j warp 0 applies H_j to column j+1 first, sums the
    // squares of its new tail and forms reflector j+1 while the other warps
    // apply H_j to columns j+2..n-1, so a step needs one block barrier and the
    // reflector's serial chain (norm, square root, one division) overlaps the
    // updates.  Reflector tails stay unscaled during the loop (the dlarfg
    // scale of column j, scl[j], enters each dot product and update once) and
    // are scaled afterwards.
    double* scl = red + 32;               // n dlarfg scales
    if (warp == 0 && kmax > 0) {
        double s = 0.0;
        for (int i = 1 + lane; i < mb; i += 32) s = fma(W[i], W[i], s);
        s = warp_sum(s);
        if (lane == 0) hh_reflector(W[0], s, &tau[0], &scl[0], &W[0]);
    }
    __syncthreads();
    for (int j = 0; j < kmax; ++j) {
        const double tj = tau[j], sc = scl[j];
        const double* wj = W + (size_t)mb * j;
        double s2 = 0.0;                  // warp 0: squares of the tail of column j+1
        if (tj != 0.0) {
            for (int k = j + 1 + warp; k < n; k += nwarps) {
                double* wk = W + (size_t)mb * k;
                double s = 0.0;
                for (int i = j + 1 + lane; i < mb; i += 32) s = fma(wj[i], wk[i], s);
                s = fma(warp_sum(s), sc, wk[j]) * tj;
                const double ss = s * sc;
                const bool next = (k == j + 1);
                for (int i = j + 1 + lane; i < mb; i += 32) {
                    const double w = fma(-ss, wj[i], wk[i]);
                    wk[i] = w;
                    if (next && i > k) s2 = fma(w, w, s2);
                }
                if (lane == 0) wk[j] -= s;
            }
        } else if (warp == 0 && j + 1 < n) {
            const double* wk = W + (size_t)mb * (j + 1);
            for (int i = j + 2 + lane; i < mb; i += 32) s2 = fma(wk[i], wk[i], s2);
        }
        if (warp == 0 && j + 1 < kmax) {
            s2 = warp_sum(s2);
            double* wn = W + (size_t)mb * (j + 1);
            if (lane == 0) hh_reflector(wn[j + 1], s2, &tau[j + 1], &scl[j + 1], &wn[j + 1]);
        }
        __syncthreads();
    }
    for (int64_t e = tid; e < (int64_t)mb * kmax; e += kQrThreads) {
        const int j = (int)(e / mb), i = (int)(e - (int64_t)j * mb);
        if (i > j && tau[j] != 0.0) W[e] *= scl[j];
    }
    __syncthreads();
    for (int j = kmax; j < n; ++j) if (tid == 0) tau[j] = 0.0;
    // explicit Q = H_0 ... H_{k-1} [I; 0], backward accumulation
    for (int64_t e = tid; e < (int64_t)mb * n; e += kQrThreads) {
        const int j = (int)(e / mb), i = (int)(e - (int64_t)j * mb);
        Qs[e] = (i == j) ? 1.0 : 0.0;
    }
    __syncthreads();
    for (int j = kmax - 1; j >= 0; --j) {
        const double tj = tau[j];
        if (tj != 0.0) {
            for (int k = j + warp; k < n; k += nwarps) {
                double s = 0.0;
                for (int i = j + lane; i < mb; i += 32) {
                    const double v = (i == j) ? 1.0 : W[i + mb * j];
                    s = fma(v, Qs[i + mb * k], s);
                }
                s = warp_sum(s) * tj;
                for (int i = j + lane; i < mb; i += 32) {
                    const double v = (i == j) ? 1.0 : W[i + mb * j];
                    Qs[i + mb * k] = fma(-s, v, Qs[i + mb * k]);
                }
            }
        }
        __syncthreads();
    }
    // sign convention diag(R) >= 0, write out
    for (int64_t e = tid; e < (int64_t)mb * n; e += kQrThreads) {
        const int j = (int)(e / mb), i = (int)(e - (int64_t)j * mb);
        const double sgn = (j < kmax && W[j + mb * j] < 0.0) ? -1.0 : 1.0;
        Qout[(off + i) + ldq * j] = sgn * Qs[e];
    }
    for (int e = tid; e < n * n; e += kQrThreads) {
        const int j = e / n, i = e - j * n;     // R(i, j)
        double v = 0.0;
        if (i <= j && i < kmax) {
            const double sgn = (W[i + mb * i] < 0.0) ? -1.0 : 1.0;
            v = sgn * W[i + mb * j];
        }
        Rout[((int64_t)b * n + i) + ldr * j] = v;
    }
}

// Householder QR of dense row blocks with 32 < n <= 64 columns (the TSQR
// leaves of a rank-33..64 factor).  Same block split, reflector form, sign
// convention and outputs as hh_qr_blocks_kernel, but thread (c, g) = (tid %
// 64, tid / 64) of the eight compute warps owns column c and the rows i = g
// mod 4, as in the triangle-pair kernel: a warp-wide FP64 instruction then
// serves 32 columns, where a warp per column spends five shuffle-adds per
// column and step on a block only ~n rows tall.  A ninth warp forms the next
// reflector beside the compute warps' dot products; tails stay unscaled in
// the loop; two block barriers per step.
constexpr int kColsThreads = 256, kColsBlock = kColsThreads + 32;

inline size_t cols_smem_bytes(int64_t mb, int n)
{
    const int64_t ldw = mb | 1;
    return sizeof(double) * ((size_t)2 * ldw * n + 2 * (size_t)n + 256 + 4);
}

__global__ void __launch_bounds__(kColsBlock) hh_qr_cols_kernel(
    const double* __restrict__ A, int64_t lda, int64_t m, int n, int nb, double* __restrict__ Qout, int64_t ldq,
    double* __restrict__ Rout, int64_t ldr, const int* __restrict__ status, const int* __restrict__ gate)
{
    if (*status != kStatusOk || (gate && *gate == 0)) return;
    extern __shared__ double sm[];
    const int b = blockIdx.x;
    const int64_t off = (int64_t)b * m / nb, end = (int64_t)(b + 1) * m / nb;
    const int mb = (int)(end - off);          // >= n (the caller's split keeps it so)
    const int ldw = mb | 1;                   // odd: lanes on consecutive columns hit distinct banks
    double* W = sm;                           // mb x n: reflectors below the diagonal, R on and above
    double* Qs = W + (size_t)ldw * n;         // mb x n explicit Q
    double* tau = Qs + (size_t)ldw * n;
    double* scl = tau + n;
    double* part = scl + n;                   // 4 x 64
    double* part2 = part + 256;               // 4
    const int tid = threadIdx.x;
    const bool comp = tid < kColsThreads;
    const int c = tid & 63, g = tid >> 6;
    for (int e = tid; e < mb * n; e += kColsBlock) {
        const int j = e / mb, i = e - j * mb;
        W[i + ldw * j] = A[(off + i) + lda * j];
    }
    __syncthreads();
    if (comp && c == 0) {
        double q = 0.0;
        for (int i = 1 + g; i < mb; i += 4) q = fma(W[i], W[i], q);
        part2[g] = q;
    }
    __syncthreads();
    if (tid == kColsThreads) {
        const double s2 = ((part2[0] + part2[1]) + part2[2]) + part2[3];
        hh_reflector(W[0], s2, &tau[0], &scl[0], &W[0]);
    }
    __syncthreads();
    // W(j, c) -= s waits in the thread that owns row j of column c and is
    // written before that thread's next dot product (rows j+2.. of the next
    // step do not include row j, and nobody else reads it meanwhile)
    double pend = 0.0;
    int jp = -1;
    for (int j = 0; j < n; ++j) {
        const bool col = comp && c > j && c < n;
        if (jp >= 0) { W[jp + ldw * c] -= pend; jp = -1; }
        if (col) {
            double p = 0.0;
            for (int i = j + 1 + ((g - (j + 1)) & 3); i < mb; i += 4) p = fma(W[i + ldw * j], W[i + ldw * c], p);
            part[g * 64 + c] = p;
        }
        __syncthreads();
        const double tj = tau[j], sc = scl[j];
        double q = 0.0;
        if (col && tj != 0.0) {
            const double sd = ((part[c] + part[64 + c]) + part[128 + c]) + part[192 + c];
            const double sj = fma(sd, sc, W[j + ldw * c]) * tj;
            const double ss = sj * sc;
            for (int i = j + 1 + ((g - (j + 1)) & 3); i < mb; i += 4) {
                const double w = fma(-ss, W[i + ldw * j], W[i + ldw * c]);
                W[i + ldw * c] = w;
                if (c == j + 1 && i > j + 1) q = fma(w, w, q);
            }
            if (g == (j & 3)) { pend = sj; jp = j; }
        } else if (col && c == j + 1) {
            for (int i = j + 2 + ((g - (j + 2)) & 3); i < mb; i += 4) q = fma(W[i + ldw * c], W[i + ldw * c], q);
        }
        if (comp && c == j + 1 && c < n) part2[g] = q;
        __syncthreads();
        if (tid == kColsThreads && j + 1 < n) {
            const double s2 = ((part2[0] + part2[1]) + part2[2]) + part2[3];
            double* d = W + (j + 1) + ldw * (j + 1);
            hh_reflector(*d, s2, &tau[j + 1], &scl[j + 1], d);
        }
    }
    if (jp >= 0) W[jp + ldw * c] -= pend;
    __syncthreads();
    for (int e = tid; e < mb * n; e += kColsBlock) {
        const int j = e / mb, i = e - j * mb;
        if (i > j && tau[j] != 0.0) W[i + ldw * j] *= scl[j];
        Qs[i + ldw * j] = (i == j) ? 1.0 : 0.0;
    }
    __syncthreads();
    // explicit Q = H_0 ... H_{n-1} [I; 0], backward.  Q(j, c) -= s waits in
    // the thread that owns row j of column c, which writes it before its next
    // dot product reads the row (step j-1 reads rows j.. of column c)
    jp = -1;
    for (int j = n - 1; j >= 0; --j) {
        const double tj = tau[j];
        const bool col = comp && c >= j && c < n;
        if (jp >= 0) { Qs[jp + ldw * c] -= pend; jp = -1; }
        if (col) {
            double p = 0.0;
            for (int i = j + 1 + ((g - (j + 1)) & 3); i < mb; i += 4) p = fma(W[i + ldw * j], Qs[i + ldw * c], p);
            part[g * 64 + c] = p;
        }
        __syncthreads();
        if (col && tj != 0.0) {
            const double sc = (((part[c] + part[64 + c]) + part[128 + c]) + part[192 + c] + Qs[j + ldw * c]) * tj;
            for (int i = j + 1 + ((g - (j + 1)) & 3); i < mb; i += 4)
                Qs[i + ldw * c] = fma(-sc, W[i + ldw * j], Qs[i + ldw * c]);
            if (g == (j & 3)) { pend = sc; jp = j; }
        }
        __syncthreads();
    }
    if (jp >= 0) Qs[jp + ldw * c] -= pend;
    __syncthreads();
    for (int e = tid; e < mb * n; e += kColsBlock) {
        const int j = e / mb, i = e - j * mb;
        const double sgn = (W[j + ldw * j] < 0.0) ? -1.0 : 1.0;
        Qout[(off + i) + ldq * j] = sgn * Qs[i + ldw * j];
    }
    for (int e = tid; e < n * n; e += kColsBlock) {
        const int j = e / n, i = e - j * n;       // R(i, j)
        double v = 0.0;
        if (i <= j) v = ((W[i + ldw * i] < 0.0) ? -1.0 : 1.0) * W[i + ldw * j];
        Rout[((int64_t)b * n + i) + ldr * j] = v;
    }
}

// Qout(block rows of b) = Qi(block rows of b) * Qtop(b*n:(b+1)*n, :)  (TSQR combine)
__global__ void tsqr_combine_kernel(const double* __restrict__ Qi, int64_t m, int n, int nb,
                                    const double* __restrict__ Qtop, int64_t ldt, double* __restrict__ Qout,
                                    const int* __restrict__ status, const int* __restrict__ gate)
{
    if (*status != kStatusOk || (gate && *gate == 0)) return;
    const int64_t total = m * n;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e / m, row = e - c * m;
        // block of this row: largest b with b*m/nb <= row
        int64_t b = (row * nb) / m;
        while (b + 1 < nb && (b + 1) * m / nb <= row) ++b;
        while (b > 0 && b * m / nb > row) --b;
        const double* t = Qtop + b * n + ldt * c;
        double s = 0.0;
        for (int k = 0; k < n; ++k) s = fma(Qi[row + m * k], t[k], s);
        Qout[e] = s;
    }
}

// QR of pairs of stacked upper-triangular n x n blocks (the TSQR tree above
// the leaves).  CTA b takes triangles 2b and 2b+1 of the K stacked in A (rows
// [2bn, 2bn+2n)); when K is odd the last CTA's second triangle is zero.  The
// Householder reflector of column j has its unit entry in row j of the upper
// block and its other non-zeros in rows 0..j of the lower block (the rest of
// the column is already zero), and applying it keeps both blocks upper
// triangular, so a pair costs about (2/3) n^3 flops for R and as much for the
// explicit Q, against 8 n^3 each for a dense 2n x n Householder QR.  Same
// reflector form and sign convention as hh_qr_blocks_kernel.  Output: Q of
// the pair (2n x n) in rows [2bn, 2bn+2n) of Qout, R in rows [bn, bn+n) of Rout.
//
// Thread (c, g) = (tid % 64, tid / 64) of the eight compute warps owns column
// c and the rows i = g mod 4 of every update, so each FP64 instruction works
// on 32 columns at once; the four partial dot products of a column are added
// in a fixed order by every thread that needs the sum.  A ninth warp forms
// the reflectors: step j ends with the threads of column j+1 leaving the
// partial sums of squares of its updated tail, and while the compute warps
// form step j+1's partial dot products (which use the unscaled tail) the
// reflector warp turns those sums into tau, the dlarfg scale and beta.  The
// tails are scaled once after the loop.  Two block barriers per step.
constexpr int kTriThreads = 256;                 // compute threads
constexpr int kTriBlock = kTriThreads + 32;      // + the reflector warp

__global__ void __launch_bounds__(kTriBlock) hh_qr_tri_kernel(
    const double* __restrict__ A, int64_t lda, int K, int n, double* __restrict__ Qout, int64_t ldq,
    double* __restrict__ Rout, int64_t ldr, const int* __restrict__ status, const int* __restrict__ gate)
{
    if (*status != kStatusOk || (gate && *gate == 0)) return;
    extern __shared__ double sm[];
    const int ld = n + 1;             // odd leading dimension: lanes on consecutive columns hit distinct banks
    double* U = sm;                   // upper block
    double* Lo = U + n * ld;          // lower block; rows 0..j of column j: reflector j (unscaled in the loop)
    double* Qt = Lo + n * ld;         // explicit Q, upper half
    double* Qb = Qt + n * ld;         // explicit Q, lower half
    double* tau = Qb + n * ld;        // n
    double* scl = tau + n;            // n dlarfg scales
    double* part = scl + n;           // 4 x 64 partial sums
    double* part2 = part + 256;       // 4 partial sums of squares (next column)
    const int b = blockIdx.x;
    const bool second = 2 * b + 1 < K;
    const int tid = threadIdx.x;
    const bool comp = tid < kTriThreads;
    const int c = tid & 63, g = tid >> 6;
    const double* A1 = A + (int64_t)2 * b * n;
    const double* A2 = A1 + n;
    for (int e = tid; e < n * n; e += kTriBlock) {
        const int j = e / n, i = e - j * n;
        U[i + ld * j] = (i <= j) ? A1[i + lda * j] : 0.0;
        Lo[i + ld * j] = (second && i <= j) ? A2[i + lda * j] : 0.0;
    }
    __syncthreads();
    if (tid == kTriThreads) {          // reflector 0: the tail of column 0 is Lo(0, 0)
        const double v = Lo[0];
        hh_reflector(U[0], v * v, &tau[0], &scl[0], &U[0]);
    }
    __syncthreads();
    // U(j, c) -= s is held in a register of the group-0 thread of column c and
    // written during the next step's dot products, which do not read U
    double upend = 0.0;
    int ujp = -1;
    for (int j = 0; j < n; ++j) {
        const bool col = comp && c > j && c < n;
        // partial dot products of the unscaled tail of column j with column c
        if (col) {
            double p = 0.0;
            for (int i = g; i <= j; i += 4) p = fma(Lo[i + ld * j], Lo[i + ld * c], p);
            part[g * 64 + c] = p;
        }
        if (ujp >= 0) { U[ujp + ld * c] -= upend; ujp = -1; }
        __syncthreads();
        const double tj = tau[j], sc = scl[j];
        double q = 0.0;
        if (col && tj != 0.0) {
            const double sd = ((part[c] + part[64 + c]) + part[128 + c]) + part[192 + c];
            const double sj = fma(sd, sc, U[j + ld * c]) * tj;
            const double ss = sj * sc;
            for (int i = g; i <= j; i += 4) {
                const double w = fma(-ss, Lo[i + ld * j], Lo[i + ld * c]);
                Lo[i + ld * c] = w;
                if (c == j + 1) q = fma(w, w, q);
            }
            if (g == 0) { upend = sj; ujp = j; }
        } else if (col && c == j + 1) {
            for (int i = g; i <= j; i += 4) q = fma(Lo[i + ld * c], Lo[i + ld * c], q);
        }
        if (comp && c == j + 1 && c < n) {
            // row j+1 of the lower block joins the tail of column j+1 (untouched so far)
            if (((j + 1) & 3) == g) q = fma(Lo[(j + 1) + ld * c], Lo[(j + 1) + ld * c], q);
            part2[g] = q;
        }
        __syncthreads();
        if (tid == kTriThreads && j + 1 < n) {
            const double s2 = ((part2[0] + part2[1]) + part2[2]) + part2[3];
            hh_reflector(U[(j + 1) + ld * (j + 1)], s2, &tau[j + 1], &scl[j + 1], &U[(j + 1) + ld * (j + 1)]);
        }
        // the next step's partial dots read neither tau, scl nor U: the
        // reflector warp runs beside them, and the barrier after the dots
        // orders its writes before their use
    }
    if (ujp >= 0) U[ujp + ld * c] -= upend;
    __syncthreads();
    for (int e = tid; e < n * n; e += kTriBlock) {
        const int j = e / n, i = e - j * n;
        if (i <= j && tau[j] != 0.0) Lo[i + ld * j] *= scl[j];
    }
    // explicit Q = H_0 ... H_{n-1} [I; 0], backward accumulation (H_j touches columns >= j)
    for (int e = tid; e < n * n; e += kTriBlock) {
        const int j = e / n, i = e - j * n;
        Qt[i + ld * j] = (i == j) ? 1.0 : 0.0;
        Qb[i + ld * j] = 0.0;
    }
    __syncthreads();
    // Qt(j, c) -= sc likewise waits in the group-0 thread for the next step's
    // dot products, which read only Qb and the reflectors
    double qpend = 0.0;
    int qjp = -1;
    for (int j = n - 1; j >= 0; --j) {
        const double tj = tau[j];
        const bool col = comp && c >= j && c < n;
        if (col) {
            double p = 0.0;
            for (int i = g; i <= j; i += 4) p = fma(Lo[i + ld * j], Qb[i + ld * c], p);
            part[g * 64 + c] = p;
        }
        if (qjp >= 0) { Qt[qjp + ld * c] -= qpend; qjp = -1; }
        __syncthreads();
        if (col && tj != 0.0) {
            const double sc = (((part[c] + part[64 + c]) + part[128 + c]) + part[192 + c] + Qt[j + ld * c]) * tj;
            for (int i = g; i <= j; i += 4) Qb[i + ld * c] = fma(-sc, Lo[i + ld * j], Qb[i + ld * c]);
            if (g == 0) { qpend = sc; qjp = j; }
        }
        __syncthreads();
    }
    if (qjp >= 0) Qt[qjp + ld * c] -= qpend;
    __syncthreads();
    double* Q1 = Qout + (int64_t)2 * b * n;
    for (int e = tid; e < n * n; e += kTriBlock) {
        const int j = e / n, i = e - j * n;
        const double sgn = (U[j + ld * j] < 0.0) ? -1.0 : 1.0;
        Q1[i + ldq * j] = sgn * Qt[i + ld * j];
        Q1[n + i + ldq * j] = sgn * Qb[i + ld * j];
        double v = 0.0;
        if (i <= j) v = ((U[i + ld * i] < 0.0) ? -1.0 : 1.0) * U[i + ld * j];
        Rout[((int64_t)b * n + i) + ldr * j] = v;
    }
}

// Qout(r, :) = Qi(r, :) * Qt(p n : p n + n, :) for the rows r < rows of pair
// p = r / (2n) (the TSQR tree's combine of a level with the level above).
__global__ void tri_combine_kernel(const double* __restrict__ Qi, int64_t ldqi, int64_t rows, int n,
                                   const double* __restrict__ Qt, int64_t ldt, double* __restrict__ Qout,
                                   int64_t ldo, const int* __restrict__ status, const int* __restrict__ gate)
{
    if (*status != kStatusOk || (gate && *gate == 0)) return;
    const int64_t total = rows * n;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e / rows, r = e - c * rows;
        const int64_t p = r / (2 * n);
        const double* t = Qt + p * n + ldt * c;
        double s = 0.0;
        for (int k = 0; k < n; ++k) s = fma(Qi[r + ldqi * k], t[k], s);
        Qout[r + ldo * c] = s;
    }
}

inline size_t tri_smem_bytes(int n) { return sizeof(double) * ((size_t)4 * n * (n + 1) + 2 * (size_t)n + 256 + 4); }

// W and Q (mb x n each), tau (n), 32 scratch values and the n reflector scales
inline size_t qr_smem_bytes(int64_t mb, int n)
{
    return sizeof(double) * ((size_t)2 * (size_t)mb * n + 2 * (size_t)n + 32);
}

constexpr size_t kQrSmemMaxBytes = 200 * 1024;   // one leaf CTA's shared memory
inline bool qr_leaf_fits(int64_t mb, int n) { return qr_smem_bytes(mb, n) <= kQrSmemMaxBytes; }

// ---------------------------------------------------------------- staircase QR of F (.) G
// (stair_qr_block in dev_common.cuh) as a kernel of its own: one CTA.
constexpr int kStairMaxN = 32;
// Fold steps go through the cluster kernel's CholeskyQR2 from this rank up.
// Below it the one-CTA staircase kernel is about as fast (38 us at R = 10)
// and, needing a single SM, runs on the side stream beside a pass over X,
// while a 16-CTA cluster waits for that pass to free the SMs.
constexpr int kFoldCqrMinR = 16;

__global__ void __launch_bounds__(kQrThreads) krp_stair_qr_kernel(
    const double* __restrict__ F, const double* __restrict__ G, int n, double* __restrict__ Qout,
    double* __restrict__ Rout, const int* __restrict__ status, const int* __restrict__ gate)
{
    if (*status != kStatusOk || (gate && *gate == 0)) return;
    extern __shared__ double sm[];
    const int tot = stair_off(n);
    double* W = sm;
    double* Qs = W + tot;
    double* tau = Qs + tot;
    double* red = tau + n;
    __shared__ int rowi[kStairMaxN * kStairMaxN], rowj[kStairMaxN * kStairMaxN];
    stair_qr_block(F, G, n, W, Qs, tau, red, rowi, rowj, Qout, Rout);
}

inline size_t stair_smem_bytes(int n)
{
    const size_t tot = (size_t)n * (n + 1) * (2 * n + 1) / 6;
    return sizeof(double) * (2 * tot + n + 32);
}

// ---------------------------------------------------------------- Khatri-Rao
// M(i*R + j, c) = F(i, c) * G(j, c): the Khatri-Rao product F (.) G of two
// R x R factors, the right factor's row index fastest (Sec. 2.2).
__global__ void krp2_kernel(const double* __restrict__ F, const double* __restrict__ G, int R,
                            double* __restrict__ M, const int* __restrict__ status)
{
    if (*status != kStatusOk) return;
    const int64_t rows = (int64_t)R * R, total = rows * R;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e / rows, row = e - c * rows;
        const int64_t i = row / R, j = row - i * R;
        M[e] = F[i + (int64_t)R * c] * G[j + (int64_t)R * c];
    }
}

// out = (I_outer (x) Qb) Qp: out(i*S + j, c) = sum_c' Qb(j, c') Qp(i*R + c', c),
// with Qb of size S x R and Qp of size (outer R) x R (Kronecker index rule,
// Sec. 2.2).
__global__ void kron_left_apply_kernel(const double* __restrict__ Qb, int64_t S, const double* __restrict__ Qp,
                                       int R, int64_t outer, double* __restrict__ out, const int* __restrict__ status)
{
    if (*status != kStatusOk) return;
    const int64_t rows = outer * S, total = rows * R;
    const int64_t ldp = outer * R;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e / rows, row = e - c * rows;
        const int64_t i = row / S, j = row - i * S;
        const double* qp = Qp + i * R + ldp * c;
        double acc = 0.0;
        for (int cp = 0; cp < R; ++cp) acc = fma(Qb[j + S * cp], qp[cp], acc);
        out[e] = acc;
    }
}

// out = (Qa (x) I_S) Qp: out(a*S + j, c) = sum_c' Qa(a, c') Qp(c'*S + j, c),
// with Qa of size Sa x R and Qp of size (R S) x R.
__global__ void kron_right_apply_kernel(const double* __restrict__ Qa, int64_t Sa, const double* __restrict__ Qp,
                                        int R, int64_t S, double* __restrict__ out, const int* __restrict__ status)
{
    if (*status != kStatusOk) return;
    const int64_t rows = Sa * S, total = rows * R;
    const int64_t ldp = (int64_t)R * S;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e / rows, row = e - c * rows;
        const int64_t a = row / S, j = row - a * S;
        const double* qp = Qp + j + ldp * c;
        double acc = 0.0;
        for (int cp = 0; cp < R; ++cp) acc = fma(Qa[a + Sa * cp], qp[(int64_t)cp * S], acc);
        out[e] = acc;
    }
}

// ---------------------------------------------------------------- solves
// Triangular solves of the I_n rows of W (Alg. cp-als-qr's substitution, and
// the Cholesky solves of Alg. cp-als) run one warp per row, the row's R <= 64
// entries spread over the lanes (entry e in lane e % 32, slot e / 32).  A
// dependent FP64 operation costs 64 cycles on this part whatever the number
// of active lanes, so the column-oriented form -- x_k = w_k / d_k, then every
// lane updates its entries with x_k -- keeps the chain at R steps of one
// multiply and one FMA, against ~R^2/2 dependent FMAs for one thread per row.
constexpr int kSolveWarps = 8;

// Ahat R0^T = W, i.e. R0 x = w for each row w of W (back substitution).
// Singularity test: |R0(k,k)| <= R * eps * max_j |R0(j,j)| sets the status
// word and writes nothing.
__global__ void __launch_bounds__(kSolveWarps * 32) trsm_qr_kernel(
    const double* __restrict__ W, const double* __restrict__ R0, int64_t I, int R, double* __restrict__ Ahat,
    int* __restrict__ status)
{
    if (*status != kStatusOk) return;
    __shared__ double r0[kMaxRank * kMaxRank];
    __shared__ int singular;
    for (int e = threadIdx.x; e < R * R; e += blockDim.x) r0[e] = R0[e];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int e0 = lane, e1 = lane + 32;
    const double a0 = e0 < R ? fabs(r0[e0 + R * e0]) : 0.0;
    const double a1 = e1 < R ? fabs(r0[e1 + R * e1]) : 0.0;
    if (warp == 0) {
        double dmax = fmax(a0, a1);
        for (int o = 16; o > 0; o >>= 1) dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
        const double tol = (double)R * kEps * dmax;
        const bool bad = (e0 < R && !(a0 > tol)) || (e1 < R && !(a1 > tol));
        const int s = __any_sync(0xffffffffu, bad) ? 1 : 0;
        if (lane == 0) {
            singular = s;
            if (s && blockIdx.x == 0) atomicCAS(status, kStatusOk, (int)CPALS_ERR_SINGULAR);
        }
    }
    __syncthreads();
    if (singular) return;
    const double d0 = e0 < R ? 1.0 / r0[e0 + R * e0] : 0.0;
    const double d1 = e1 < R ? 1.0 / r0[e1 + R * e1] : 0.0;
    const int64_t gw = (int64_t)blockIdx.x * kSolveWarps + warp, nw = (int64_t)gridDim.x * kSolveWarps;
    for (int64_t i = gw; i < I; i += nw) {
        double w0 = e0 < R ? W[i + I * e0] : 0.0;
        double w1 = e1 < R ? W[i + I * e1] : 0.0;
        warp_subst(w0, w1, r0, R, d0, d1, true, false);
        if (e0 < R) Ahat[i + I * e0] = w0;
        if (e1 < R) Ahat[i + I * e1] = w1;
    }
}

// One-sided Jacobi SVD of R0 (Hestenes), then T = U pinv(Sigma) V^T keeping
// sigma_j > rtol * sigma_max.  Pairs are visited in round-robin order so that
// the R/2 rotations of a round are independent.  Lane l of every warp works
// on pair l, warp w on rows [w RW, (w+1) RW): the three dot products of a
// pair are summed over the warps in a fixed order, warp 0 forms all rotations
// of the round at once, and every warp rotates its rows of B and V.  A pair is
// rotated while the cosine of the angle between its columns exceeds R times
// the unit roundoff of the arithmetic (the rounding level of their length-R
// dot product); a sweep with no rotation ends the iteration.
//
// At R >= 32 the sweeps start from an FP32 preconditioner: one-sided Jacobi
// of R0 in FP32 (whose pipe issues 64 times faster than FP64 here) gives an
// orthogonal-to-FP32 V32 (sweeps stop below 8 R u_32 or after 20); one
// Newton-Schulz step V <- V (3 I - V^T V) / 2 in FP64 squares its distance
// from orthogonality (about 1e-6 -> 1e-12); then the
// FP64 sweeps run on B = R0 V, which is already nearly column-orthogonal, and
// converge in a few sweeps instead of about twelve.  The result is the SVD of
// R0 to FP64 accuracy either way.
// Truncation test ahead of the SVD solve.  The truncated operator
// T = U pinv(Sigma) V^T of R0 = U Sigma V^T keeps sigma_i > rtol sigma_max
// (Sec. 3.1).  Since sigma_min >= 1 / ||R0^-1||_F and sigma_max <= ||R0||_F,
// ||R0||_F ||R0^-1||_F < 1 / rtol proves that nothing is truncated, and then
// T = U Sigma^-1 V^T = R0^-T exactly.  The kernel forms X = R0^-1 by back
// substitution, one warp per column over ceil(R / 8) CTAs (lanes over the
// rows), writes T = X^T and, per column j, ||X(:, j)||^2 and ||R0(:, j)||^2
// to parts[2 j], parts[2 j + 1].  The Jacobi kernel that follows sums them
// in column order and, when ||R0||_F ||X||_F rtol <= 1/4 (the margin covers
// the rounding of X), keeps T and returns; otherwise it forms T by the SVD.
// A zero or non-finite diagonal entry writes infinite parts, which sends R0
// to the SVD.
constexpr int kInvWarps = 8;
__global__ void __launch_bounds__(kInvWarps * 32) svd_shortcut_kernel(const double* __restrict__ R0, int R,
                                                                      double* __restrict__ T,
                                                                      double* __restrict__ parts,
                                                                      const int* __restrict__ status)
{
    if (*status != kStatusOk) return;
    __shared__ double r0[kMaxRank * kMaxRank];
    __shared__ double dinv[kMaxRank];
    __shared__ int bad;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) bad = 0;
    for (int e = tid; e < R * R; e += kInvWarps * 32) r0[e] = R0[e];
    __syncthreads();
    if (tid < R) {
        const double d = r0[tid + R * tid];
        if (!(fabs(d) > 0.0) || !(fabs(d) < INFINITY)) bad = 1;
        dinv[tid] = 1.0 / d;
    }
    __syncthreads();
    const int j = blockIdx.x * kInvWarps + warp;
    if (j >= R) return;
    if (bad) {
        if (lane == 0) { parts[2 * j] = INFINITY; parts[2 * j + 1] = INFINITY; }
        return;
    }
    double sx = 0.0, sr = 0.0;
    const int e0 = lane, e1 = lane + 32;
    // X(:, j): R0 x = e_j, from k = j down
    double w0 = (e0 == j) ? 1.0 : 0.0, w1 = (e1 == j) ? 1.0 : 0.0;
    for (int k = j; k >= 0; --k) {
        double xk;
        if (k < 32) {
            if (lane == k) w0 *= dinv[k];
            xk = __shfl_sync(0xffffffffu, w0, k);
        } else {
            if (lane == k - 32) w1 *= dinv[k];
            xk = __shfl_sync(0xffffffffu, w1, k - 32);
        }
        if (e0 < k) w0 = fma(-r0[e0 + R * k], xk, w0);
        if (e1 < k) w1 = fma(-r0[e1 + R * k], xk, w1);
    }
    // T = X^T: T(j, i) = X(i, j)
    if (e0 <= j) { T[j + R * e0] = w0; sx = fma(w0, w0, sx); }
    if (e1 <= j && e1 < R) { T[j + R * e1] = w1; sx = fma(w1, w1, sx); }
    if (e0 > j && e0 < R) T[j + R * e0] = 0.0;
    if (e1 > j && e1 < R) T[j + R * e1] = 0.0;
    if (e0 <= j) sr = fma(r0[e0 + R * j], r0[e0 + R * j], sr);
    if (e1 <= j && e1 < R) sr = fma(r0[e1 + R * j], r0[e1 + R * j], sr);
    for (int o = 16; o > 0; o >>= 1) {
        sx += __shfl_xor_sync(0xffffffffu, sx, o);
        sr += __shfl_xor_sync(0xffffffffu, sr, o);
    }
    if (lane == 0) { parts[2 * j] = sx; parts[2 * j + 1] = sr; }
}

constexpr int kJacobiWarps = 8;
constexpr int kJacobiThreads = 32 * kJacobiWarps;
constexpr int kJacobiMixedMinR = 32;

__host__ __device__ constexpr size_t jacobi_smem_doubles()
{
    // B, V (FP64), B32, V32 (FP32, half the space), G (FP64 R x R), partial sums, rotations, sigma, 1/sigma^2
    return (size_t)2 * kMaxRank * (kMaxRank + 1) + (size_t)kMaxRank * (kMaxRank + 1) +
           (size_t)kMaxRank * kMaxRank + (size_t)kJacobiWarps * 32 * 3 + 32 * 3 + 2 * kMaxRank;
}

// Sweeps of one-sided Jacobi on the columns of B (R x Rp, leading dimension
// ld), accumulating the rotations into V.  Block-wide; returns the sweep count.
template <typename T>
__device__ int jacobi_sweeps(T* B, T* V, int ld, int R, T tol, int max_sweeps, T* part, T* rot, int* rotated)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int Rp = (R + 1) & ~1;   // padded to even; column R (if any) is a zero dummy
    const int np = Rp / 2;
    const int RW = (R + kJacobiWarps - 1) / kJacobiWarps;
    const int i0 = warp * RW, i1 = min(R, i0 + RW);
    int sweep = 0;
    for (; sweep < max_sweeps; ++sweep) {
        if (tid == 0) *rotated = 0;
        for (int round = 0; round < Rp - 1; ++round) {
            // round-robin pairing: position 0 fixed, others rotate
            const int pi = lane;
            int p = 0, q = 0;
            if (pi < np) {
                const int a = (pi == 0) ? 0 : 1 + (pi - 1 + round) % (Rp - 1);
                const int b = 1 + (Rp - 2 - pi + round) % (Rp - 1);
                p = min(a, b);
                q = max(a, b);
            }
            const bool live = pi < np && q < R;   // q == R: the dummy column
            if (live) {
                T sa = 0, sb = 0, sg = 0;
                for (int i = i0; i < i1; ++i) {
                    const T bp = B[i + ld * p], bq = B[i + ld * q];
                    sa = fma(bp, bp, sa);
                    sb = fma(bq, bq, sb);
                    sg = fma(bp, bq, sg);
                }
                T* pp = part + (warp * 32 + pi) * 3;
                pp[0] = sa; pp[1] = sb; pp[2] = sg;
            }
            __syncthreads();
            if (warp == 0) {
                T c = 1, sn = 0, flag = 0;
                if (live) {
                    T sa = 0, sb = 0, sg = 0;
                    for (int w = 0; w < kJacobiWarps; ++w) {
                        const T* pp = part + (w * 32 + pi) * 3;
                        if (w * RW < R) { sa += pp[0]; sb += pp[1]; sg += pp[2]; }
                    }
                    if (sg != T(0) && fabs(sg) > tol * sqrt(sa * sb)) {
                        const T zeta = (sb - sa) / (T(2) * sg);
                        const T t = ((zeta >= T(0)) ? T(1) : T(-1)) / (fabs(zeta) + sqrt(T(1) + zeta * zeta));
                        c = T(1) / sqrt(T(1) + t * t);
                        sn = c * t;
                        flag = 1;
                    }
                }
                if (pi < 32) { rot[3 * pi] = c; rot[3 * pi + 1] = sn; rot[3 * pi + 2] = flag; }
                if (__any_sync(0xffffffffu, flag != T(0)) && lane == 0) *rotated = 1;
            }
            __syncthreads();
            if (live && rot[3 * pi + 2] != T(0)) {
                const T c = rot[3 * pi], sn = rot[3 * pi + 1];
                for (int i = i0; i < i1; ++i) {
                    const T bp = B[i + ld * p], bq = B[i + ld * q];
                    B[i + ld * p] = c * bp - sn * bq;
                    B[i + ld * q] = sn * bp + c * bq;
                    const T vp = V[i + ld * p], vq = V[i + ld * q];
                    V[i + ld * p] = c * vp - sn * vq;
                    V[i + ld * q] = sn * vp + c * vq;
                }
            }
            __syncthreads();
        }
        if (!*rotated) break;   // uniform: read after the round's last barrier
        __syncthreads();        // nobody clears the flag before everyone has read it
    }
    return sweep;
}

// sc_parts (may be NULL): the truncation test's per-column norms (see
// svd_shortcut_kernel); when they prove that nothing is truncated, T is
// already R0^-T and the kernel returns.
__global__ void __launch_bounds__(kJacobiThreads) jacobi_pinv_kernel(const double* __restrict__ R0, int R,
                                                                    double rtol, double* __restrict__ T,
                                                                    const int* __restrict__ status,
                                                                    const double* __restrict__ sc_parts)
{
    if (*status != kStatusOk) return;
    if (sc_parts != nullptr) {
        __shared__ int keep;
        if (threadIdx.x == 0) {
            double a = 0.0, b = 0.0;
            for (int j = 0; j < R; ++j) { a += sc_parts[2 * j]; b += sc_parts[2 * j + 1]; }
            const double bound = sqrt(a) * sqrt(b);
            keep = (bound < INFINITY && bound * rtol <= 0.25) ? 1 : 0;
        }
        __syncthreads();
        if (keep) return;
    }
    extern __shared__ double jsm[];
    const int ld = R + 1;                     // odd: lanes on different columns hit different banks
    const int Rp = (R + 1) & ~1;
    double* B = jsm;                          // R x Rp
    double* V = B + (size_t)kMaxRank * (kMaxRank + 1);
    float* B32 = reinterpret_cast<float*>(V + (size_t)kMaxRank * (kMaxRank + 1));
    float* V32 = B32 + (size_t)kMaxRank * (kMaxRank + 1);
    double* G = reinterpret_cast<double*>(V32 + (size_t)kMaxRank * (kMaxRank + 1));   // R x R
    double* part = G + (size_t)kMaxRank * kMaxRank;          // [warp][pair][3]
    double* rot = part + kJacobiWarps * 32 * 3;             // [pair][c, s, flag]
    double* sig = rot + 32 * 3;                             // R
    double* isq = sig + kMaxRank;                           // R: 1 / sigma_j^2 or 0 (truncated)
    __shared__ int rotated;
    const int tid = threadIdx.x;
    if (R >= kJacobiMixedMinR) {
        // FP32 preconditioner
        for (int e = tid; e < Rp * R; e += kJacobiThreads) {
            const int j = e / R, i = e - j * R;
            B32[i + ld * j] = (j < R) ? (float)R0[i + R * j] : 0.0f;
            V32[i + ld * j] = (i == j) ? 1.0f : 0.0f;
        }
        __syncthreads();
        // stop at 8 R u_32 (clear of the FP32 rounding level of the dot products);
        // the FP64 sweeps converge quadratically from there
        jacobi_sweeps<float>(B32, V32, ld, R, 8.0f * (float)R * 5.9604645e-8f, 20, reinterpret_cast<float*>(part),
                             reinterpret_cast<float*>(rot), &rotated);
        // G = V32^T V32 in FP64; V = V32 (3 I - G) / 2
        for (int e = tid; e < R * R; e += kJacobiThreads) {
            const int b = e / R, a = e - b * R;
            double s = 0.0;
            for (int i = 0; i < R; ++i) s = fma((double)V32[i + ld * a], (double)V32[i + ld * b], s);
            G[a + R * b] = s;
        }
        __syncthreads();
        for (int e = tid; e < Rp * R; e += kJacobiThreads) {
            const int j = e / R, i = e - j * R;
            double s = 0.0;
            if (j < R) {
                for (int k = 0; k < R; ++k) s = fma((double)V32[i + ld * k], (k == j ? 3.0 : 0.0) - G[k + R * j], s);
                s *= 0.5;
            }
            V[i + ld * j] = s;
        }
        __syncthreads();
        // B = R0 V (the input is a full matrix: R0, or S for the pseudo-inverse solve)
        for (int e = tid; e < Rp * R; e += kJacobiThreads) {
            const int j = e / R, i = e - j * R;
            double s = 0.0;
            if (j < R)
                for (int k = 0; k < R; ++k) s = fma(R0[i + R * k], V[k + ld * j], s);
            B[i + ld * j] = s;
        }
        __syncthreads();
    } else {
        for (int e = tid; e < Rp * R; e += kJacobiThreads) {
            const int j = e / R, i = e - j * R;
            B[i + ld * j] = (j < R) ? R0[i + R * j] : 0.0;
            V[i + ld * j] = (i == j) ? 1.0 : 0.0;
        }
        __syncthreads();
    }
    jacobi_sweeps<double>(B, V, ld, R, (double)R * kEps, 80, part, rot, &rotated);
    for (int j = tid; j < R; j += kJacobiThreads) {
        double s = 0.0;
        for (int i = 0; i < R; ++i) s = fma(B[i + ld * j], B[i + ld * j], s);
        sig[j] = sqrt(s);
    }
    __syncthreads();
    double smax = 0.0;
    for (int j = 0; j < R; ++j) smax = fmax(smax, sig[j]);
    for (int j = tid; j < R; j += kJacobiThreads)
        isq[j] = (sig[j] > rtol * smax && sig[j] > 0.0) ? 1.0 / (sig[j] * sig[j]) : 0.0;
    __syncthreads();
    for (int e = tid; e < R * R; e += kJacobiThreads) {
        const int bcol = e / R, a = e - bcol * R;   // T(a, bcol) = sum_j B(a,j) V(bcol,j) / sig_j^2
        double s = 0.0;
        for (int j = 0; j < R; ++j) s = fma(B[a + ld * j] * isq[j], V[bcol + ld * j], s);
        T[a + R * bcol] = s;
    }
}

// S = Hadamard product of the Grams G_m, m != n; then its Cholesky factor L
// (lower) into Lout.  Not SPD sets the status word.
struct GPtrs {
    const double* G[kMaxN];
};

__global__ void hadamard_cholesky_kernel(GPtrs gp, int N, int n, int R, double* __restrict__ S,
                                         double* __restrict__ Lout, int* __restrict__ status, int chol)
{
    if (*status != kStatusOk) return;
    __shared__ double L[kMaxRank * kMaxRank];
    __shared__ int bad;
    const int tid = threadIdx.x;
    for (int e = tid; e < R * R; e += blockDim.x) {
        double s = 1.0;
        for (int m = 0; m < N; ++m)
            if (m != n) s *= gp.G[m][e];
        S[e] = s;
        L[e] = s;
    }
    if (tid == 0) bad = 0;
    __syncthreads();
    if (!chol) return;
    for (int j = 0; j < R; ++j) {
        if (tid == 0) {
            double d = L[j + R * j];
            for (int k = 0; k < j; ++k) d -= L[j + R * k] * L[j + R * k];
            if (!(d > 0.0)) bad = 1;
            L[j + R * j] = (d > 0.0) ? sqrt(d) : 1.0;
        }
        __syncthreads();
        for (int i = j + 1 + tid; i < R; i += blockDim.x) {
            double s = L[i + R * j];
            for (int k = 0; k < j; ++k) s -= L[i + R * k] * L[j + R * k];
            L[i + R * j] = s / L[j + R * j];
        }
        __syncthreads();
    }
    if (bad) {
        if (tid == 0) atomicCAS(status, kStatusOk, (int)CPALS_ERR_SINGULAR);
        return;
    }
    for (int e = tid; e < R * R; e += blockDim.x) {
        const int j = e / R, i = e - j * R;
        Lout[e] = (i >= j) ? L[e] : 0.0;
    }
}

// Ahat S = M with S = L L^T: per row, L y = m, L^T x = y.
__global__ void __launch_bounds__(kSolveWarps * 32) chol_rows_kernel(
    const double* __restrict__ Mm, const double* __restrict__ Lg, int64_t I, int R, double* __restrict__ Ahat,
    const int* __restrict__ status)
{
    if (*status != kStatusOk) return;
    __shared__ double L[kMaxRank * kMaxRank];
    for (int e = threadIdx.x; e < R * R; e += blockDim.x) L[e] = Lg[e];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int e0 = lane, e1 = lane + 32;
    const double d0 = e0 < R ? 1.0 / L[e0 + R * e0] : 0.0;
    const double d1 = e1 < R ? 1.0 / L[e1 + R * e1] : 0.0;
    const int64_t gw = (int64_t)blockIdx.x * kSolveWarps + warp, nw = (int64_t)gridDim.x * kSolveWarps;
    for (int64_t i = gw; i < I; i += nw) {
        double w0 = e0 < R ? Mm[i + I * e0] : 0.0;
        double w1 = e1 < R ? Mm[i + I * e1] : 0.0;
        warp_subst(w0, w1, L, R, d0, d1, false, false);   // L y = m
        warp_subst(w0, w1, L, R, d0, d1, true, true);     // L^T x = y
        if (e0 < R) Ahat[i + I * e0] = w0;
        if (e1 < R) Ahat[i + I * e1] = w1;
    }
}

// lambda_r = ||Ahat(:, r)||_2, A(:, r) = Ahat(:, r) / lambda_r (one CTA per column).
__global__ void normalize_kernel(const double* __restrict__ Ahat, int64_t I, double* __restrict__ A,
                                 double* __restrict__ lambda, const int* __restrict__ status)
{
    if (*status != kStatusOk) return;
    __shared__ double sh[32];
    __shared__ double lam;
    const int r = blockIdx.x;
    const double* col = Ahat + I * r;
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < I; i += blockDim.x) s = fma(col[i], col[i], s);
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
        v = warp_sum(v);
        if (threadIdx.x == 0) { lam = sqrt(v); lambda[r] = lam; }
    }
    __syncthreads();
    const double l = lam;
    for (int64_t i = threadIdx.x; i < I; i += blockDim.x) A[i + I * r] = (l > 0.0) ? col[i] / l : col[i];
}

// G = A^T A (R x R), one thread per entry, summing over the I rows in order.
__global__ void gram_kernel(const double* __restrict__ A, int64_t I, int R, double* __restrict__ G,
                            const int* __restrict__ status)
{
    if (*status != kStatusOk) return;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= R * R) return;
    const int b = e / R, a = e - b * R;
    double s = 0.0;
    for (int64_t i = 0; i < I; ++i) s = fma(A[i + I * a], A[i + I * b], s);
    G[e] = s;
}

// ---------------------------------------------------------------- fit (Sec. 3.3.1)
// Partial inner products over row blocks of 32:
//  QR:     sum_{i,k} W(i,k) (Ahat R0^T)(i,k)
//  NORMAL: sum_{i,k} M(i,k) Ahat(i,k)
__global__ void fit_inner_kernel(const double* __restrict__ Wm, const double* __restrict__ Ahat,
                                 const double* __restrict__ R0, int64_t I, int R, int qr, int kchunk,
                                 double* __restrict__ part, const int* __restrict__ status)
{
    if (*status != kStatusOk) return;
    __shared__ double sh[32];
    double s = 0.0;
    const int64_t i = (int64_t)blockIdx.x * 32 + (threadIdx.x & 31);
    const int kb = blockIdx.y * kchunk, ke = min(R, kb + kchunk);
    if (i < I) {
        for (int k = kb + (threadIdx.x >> 5); k < ke; k += (blockDim.x >> 5)) {
            double v;
            if (qr) {
                v = 0.0;
                for (int j = 0; j < R; ++j) v = fma(Ahat[i + I * j], R0[k + R * j], v);
            } else {
                v = Ahat[i + I * k];
            }
            s = fma(Wm[i + I * k], v, s);
        }
    }
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
        part[blockIdx.x + (int64_t)gridDim.x * blockIdx.y] = t;
    }
}

// Block-wide sum (fixed order: strided per thread, then warps, then thread 0).
__device__ double block_sum(double v, double* sh)
{
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    __syncthreads();
    return t;   // valid in thread 0
}

// Model norm, row i of the R x R sum per block (thread j: entry (i, j)):
//  QR:     <R0^T R0, diag(l) R_N^T R_N diag(l)> = ||R0 diag(l) R_N^T||_F^2
//          (R0 and R_N upper triangular: entry (i, j) sums k >= max(i, j))
//  NORMAL: <S_N, diag(l) G_N diag(l)>
// written to part[i].
__global__ void fit_norm_kernel(const double* __restrict__ R0orS, const double* __restrict__ RNorG,
                                const double* __restrict__ lambda, int R, int qr, double* __restrict__ part,
                                const int* __restrict__ status)
{
    if (*status != kStatusOk) return;
    __shared__ double sh[32];
    const int i = blockIdx.x;
    double nrm = 0.0;
    for (int j = threadIdx.x; j < R; j += blockDim.x) {
        if (qr) {
            double v = 0.0;
            for (int k = max(i, j); k < R; ++k) v = fma(R0orS[i + R * k] * lambda[k], RNorG[j + R * k], v);
            nrm = fma(v, v, nrm);
        } else {
            const int e = i + R * j;
            nrm = fma(R0orS[e] * lambda[i], RNorG[e] * lambda[j], nrm);
        }
    }
    const double t = block_sum(nrm, sh);
    if (threadIdx.x == 0) part[i] = t;
}

// Final: inner = the sum of the nparts inner partials, the model norm = the
// sum of the R row partials after them (fixed orders);
// fit = 1 - sqrt(max(||X||^2 - 2 inner + nrm, 0)) / ||X||, appended to the ring.
__global__ void fit_final_kernel(const double* __restrict__ part, int nparts, int R,
                                 const double* __restrict__ normX2, double* __restrict__ ring, int cap,
                                 int* __restrict__ count, double* __restrict__ last, const int* __restrict__ status)
{
    if (*status != kStatusOk) return;
    __shared__ double sh[32];
    double nrm = 0.0;
    for (int p = threadIdx.x; p < R; p += blockDim.x) nrm += part[nparts + p];
    double in = 0.0;
    for (int p = threadIdx.x; p < nparts; p += blockDim.x) in += part[p];
    const double tot = block_sum(nrm, sh);
    const double inner = block_sum(in, sh);
    if (threadIdx.x == 0) {
        double res2 = *normX2 - 2.0 * inner + tot;
        if (res2 < 0.0) res2 = 0.0;
        const double f = 1.0 - sqrt(res2) / sqrt(*normX2);
        const int c = *count;
        ring[c % cap] = f;
        *count = c + 1;
        *last = f;
    }
}

inline unsigned grid_for(int64_t n, int threads, int num_sms)
{
    int64_t g = (n + threads - 1) / threads;
    const int64_t cap = (int64_t)num_sms * 8;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (unsigned)g;
}

// Recursive TSQR.  ws must hold 3*m*n doubles for the top call (geometric sum).
// A leaf QR is latency-bound (n sequential reflector steps), so a matrix that
// fits one CTA's shared memory is factored by a single leaf; taller ones are
// split into blocks of max(2n, 32, m / #SMs) rows.
// Q (K n x n) and R (n x n) of K >= 2 stacked upper-triangular blocks, by a
// binary tree of pair QRs.
cudaError_t tsqr_tri(Handle* h, const double* Rs, int K, int n, double* Q, double* R, double* ws, int64_t ws_elems,
                     const int* gate)
{
    const int P = (K + 1) / 2;
    const size_t smem = tri_smem_bytes(n);
    if (P == 1) {   // K == 2: the pair's Q is the result
        hh_qr_tri_kernel<<<1, kTriBlock, smem, h->stream>>>(Rs, (int64_t)K * n, K, n, Q, (int64_t)K * n, R, n,
                                                            h->d_status, gate);
        h->launches++;
        return cudaGetLastError();
    }
    const int64_t nn = (int64_t)n * n;
    double* Qi = ws;                        // 2P n x n
    double* Rs2 = Qi + 2 * P * nn;          // P n x n
    double* Qt = Rs2 + P * nn;              // P n x n
    const int64_t used = 4 * P * nn;
    if (used > ws_elems) return cudaErrorInvalidValue;
    hh_qr_tri_kernel<<<P, kTriBlock, smem, h->stream>>>(Rs, (int64_t)K * n, K, n, Qi, 2 * (int64_t)P * n, Rs2,
                                                         (int64_t)P * n, h->d_status, gate);
    h->launches++;
    CPALS_CUDA_TRY(cudaGetLastError());
    CPALS_CUDA_TRY(tsqr_tri(h, Rs2, P, n, Qt, R, ws + used, ws_elems - used, gate));
    const int64_t rows = (int64_t)K * n;
    tri_combine_kernel<<<grid_for(rows * n, 256, h->num_sms), 256, 0, h->stream>>>(
        Qi, 2 * (int64_t)P * n, rows, n, Qt, (int64_t)P * n, Q, rows, h->d_status, gate);
    h->launches++;
    return cudaGetLastError();
}

// Tall-skinny QR: one CTA when the matrix is small (about 1 MFLOP or less),
// else dense Householder leaves of at least n rows spread over the SMs, the
// tree of triangle pairs, and one combine back to the leaves.
// Dense leaves with 32 < n <= 64 columns (and at least n rows) go through the
// column-per-thread kernel; structured ones (the Khatri-Rao steps, whose
// reflectors are mostly empty) keep the warp-per-column kernel, which skips
// a column's update when its reflector is the identity.
inline bool use_cols_leaf(bool dense, int64_t mb, int n)
{
    return dense && n > 32 && n <= 64 && mb >= n && cols_smem_bytes(mb, n) <= kQrSmemMaxBytes;
}

void launch_leaves(Handle* h, bool cols, unsigned nb, int64_t mbmax, const double* A, int64_t m, int n, double* Q,
                   double* R, int64_t ldr, const int* gate)
{
    if (cols)
        hh_qr_cols_kernel<<<nb, kColsBlock, cols_smem_bytes(mbmax, n), h->stream>>>(A, m, m, n, (int)nb, Q, m, R, ldr,
                                                                                  h->d_status, gate);
    else
        hh_qr_blocks_kernel<<<nb, kQrThreads, qr_smem_bytes((int)mbmax, n), h->stream>>>(A, m, m, n, (int)nb, Q, m,
                                                                                          R, ldr, h->d_status, gate);
    h->launches++;
}

cudaError_t tsqr(Handle* h, const double* A, int64_t m, int n, double* Q, double* R, double* ws, int64_t ws_elems,
                 bool dense, const int* gate)
{
    if (qr_leaf_fits(m, n) && m * n * n <= ((int64_t)1 << 18)) {
        launch_leaves(h, use_cols_leaf(dense, m, n), 1, m, A, m, n, Q, R, n, gate);
        return cudaGetLastError();
    }
    const int64_t leaf_rows = std::max<int64_t>({(int64_t)n, 32, (m + h->num_sms - 1) / h->num_sms});
    int64_t nb = (m + leaf_rows - 1) / leaf_rows;
    // each block must keep >= n rows: balanced blocks have floor(m/nb) rows
    while (nb > 1 && m / nb < n) --nb;
    const int64_t mbmax = (m + nb - 1) / nb;
    if (!qr_leaf_fits(mbmax, n)) return cudaErrorInvalidValue;
    if (nb == 1) {
        launch_leaves(h, use_cols_leaf(dense, m, n), 1, m, A, m, n, Q, R, n, gate);
        return cudaGetLastError();
    }
    double* Qi = ws;                        // m x n
    double* Rs = Qi + m * n;                // (nb*n) x n
    double* Qt = Rs + nb * n * n;           // (nb*n) x n
    double* rest = Qt + nb * n * n;
    const int64_t used = m * n + 2 * nb * n * n;
    if (used > ws_elems) return cudaErrorInvalidValue;
    launch_leaves(h, use_cols_leaf(dense, mbmax, n), (unsigned)nb, mbmax, A, m, n, Qi, Rs, nb * n, gate);
    CPALS_CUDA_TRY(cudaGetLastError());
    CPALS_CUDA_TRY(tsqr_tri(h, Rs, (int)nb, n, Qt, R, rest, ws_elems - used, gate));
    tsqr_combine_kernel<<<grid_for(m * n, 256, h->num_sms), 256, 0, h->stream>>>(Qi, m, n, (int)nb, Qt, nb * n, Q,
                                                                                  h->d_status, gate);
    h->launches++;
    return cudaGetLastError();
}

}  // namespace

// Shared-memory limits of the QR kernels, set once per process.
cudaError_t qr_kernel_attrs()
{
    static cudaError_t err = [] {
        cudaError_t e = cudaFuncSetAttribute(hh_qr_blocks_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kQrSmemMaxBytes);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(hh_qr_tri_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)tri_smem_bytes(kMaxRank));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(krp_stair_qr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)stair_smem_bytes(kStairMaxN));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(hh_qr_cols_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kQrSmemMaxBytes);
        return e;
    }();
    return err;
}

cudaError_t householder_qr(Handle* h, const double* A, int64_t m, int n, double* Q, double* R, bool dense,
                           const int* gate)
{
    CPALS_CUDA_TRY(qr_kernel_attrs());
    return tsqr(h, A, m, n, Q, R, h->qr_ws, h->qr_ws_elems, dense, gate);
}

// QR of the Khatri-Rao product Rl[cnt-1] (.) ... (.) Rl[0] of upper-triangular
// R x R factors (Rl[0] rightmost: its row index runs fastest), cnt >= 2, by
// the Kronecker fold: if B = Q_B R_B then F (.) B = (I (x) Q_B)(F (.) R_B)
// (Eq. kr-id), so each step is the QR of a Khatri-Rao product of two
// triangular factors.  Writes the explicit Q (R^cnt x R) to Qout and R to
// Rout; with implicit = true the Q factor of every step goes to h->KP instead
// (the Kruskal-input path applies Q0 in that factored form).
cudaError_t fold_qr(Handle* h, const double* const* Rl, int cnt, double* Qout, double* Rout, bool implicit)
{
    if (cnt < 2) return cudaErrorInvalidValue;
    CPALS_CUDA_TRY(qr_kernel_attrs());
    const int R = h->R;
    const size_t R3 = (size_t)R * R * R;
    const double* curR = Rl[0];
    int64_t S = 0;                       // rows of the current Q_B (0: Q_B = I)
    for (int k = 1; k < cnt; ++k) {
        const bool last = (k == cnt - 1);
        double* Ro = last ? Rout : h->KR[k & 1];
        // QR of F (.) R_B, F = Rl[k]: both factors are upper triangular
        auto step_qr = [&](double* Qo) -> cudaError_t {
            if (R <= kStairMaxN) {
                const int* gate = nullptr;
                if (tail_fused(h) && R >= kFoldCqrMinR && mode_tail_ok((int64_t)R * R, R, 4)) {
                    // CholeskyQR2 of the explicit F (.) R_B in the cluster kernel; the
                    // staircase Householder QR runs only if that was refused
                    krp2_kernel<<<grid_for((int64_t)R * R * R, 256, h->num_sms), 256, 0, h->stream>>>(
                        Rl[k], curR, R, h->KM, h->d_status);
                    h->launches++;
                    CPALS_CUDA_TRY(cudaGetLastError());
                    CPALS_CUDA_TRY(cqr2_rows(h, h->KM, (int64_t)R * R, Qo, Ro, h->VG, h->d_vgate));
                    gate = h->d_vgate;
                }
                krp_stair_qr_kernel<<<1, kQrThreads, stair_smem_bytes(R), h->stream>>>(Rl[k], curR, R, Qo, Ro,
                                                                                       h->d_status, gate);
                h->launches++;
                return cudaGetLastError();
            }
            krp2_kernel<<<grid_for((int64_t)R * R * R, 256, h->num_sms), 256, 0, h->stream>>>(Rl[k], curR, R, h->KM,
                                                                                              h->d_status);
            h->launches++;
            CPALS_CUDA_TRY(cudaGetLastError());
            const int* gate = nullptr;
            if (tail_fused(h) && (wide_tail_on(h) || mode_tail_ok((int64_t)R * R, R, 4))) {
                // CholeskyQR2 (GPU-wide above rank 32, its first Gram from F and R_B); the
                // TSQR runs only if that was refused
                CPALS_CUDA_TRY(cqr2_rows(h, h->KM, (int64_t)R * R, Qo, Ro, h->VG, h->d_vgate, Rl[k], curR));
                gate = h->d_vgate;
            }
            return householder_qr(h, h->KM, (int64_t)R * R, R, Qo, Ro, false, gate);
        };
        if (implicit) {
            CPALS_CUDA_TRY(step_qr(h->KP + (size_t)(k - 1) * R3));
        } else if (S == 0) {
            // Q_B = I: the QR of F (.) R_B is already the result (or the next Q_B)
            CPALS_CUDA_TRY(step_qr(last ? Qout : h->KQb[k & 1]));
            S = (int64_t)R * R;
        } else {
            CPALS_CUDA_TRY(step_qr(h->KQ));
            const double* Qb = h->KQb[(k - 1) & 1];
            double* Qo = last ? Qout : h->KQb[k & 1];
            kron_left_apply_kernel<<<grid_for((int64_t)R * S * R, 256, h->num_sms), 256, 0, h->stream>>>(
                Qb, S, h->KQ, R, (int64_t)R, Qo, h->d_status);
            h->launches++;
            CPALS_CUDA_TRY(cudaGetLastError());
            S *= R;
        }
        curR = Ro;
    }
    return cudaSuccess;
}

// QR of V_n = F_1 (.) F_2 (.) ... (.) F_{N-1} (the R_m of every mode m != n, highest
// mode first; Sec. 3.1) without forming V_n.  If B = Q_B R_B is the thin QR
// of the trailing Khatri-Rao product, then by Eq. kr-id
//     F (.) B = (I_R (x) Q_B) (F (.) R_B),
// and I_R (x) Q_B has orthonormal columns, so QR(F (.) B) needs only the QR of
// the R^2 x R matrix F (.) R_B.  Folding from the lowest mode upward, the QR of V_n
// takes N-2 QRs of R^2 x R matrices and one Kronecker-structured product per
// step to build the explicit Q0 (R^{N-1} x R).  The thin QR with diag(R0) >= 0
// is unique, so this equals the Householder QR of the explicit V_n up to
// rounding.
cudaError_t krp_qr(Handle* h, int n, bool implicit)
{
    CPALS_CUDA_TRY(qr_kernel_attrs());
    const int R = h->R;
    const double* Rl[kMaxN];
    int cnt = 0;
    for (int m = 0; m < h->N; ++m)
        if (m != n) Rl[cnt++] = h->Rf[m];   // ascending: Rl[0] is the fastest (rightmost) factor
    if (cnt == 1) return householder_qr(h, Rl[0], R, R, implicit ? h->KP : h->Q0, h->R0, false);
    return fold_qr(h, Rl, cnt, implicit ? nullptr : h->Q0, h->R0, implicit);
}

cudaError_t krp_qr_half(Handle* h, const int* modes, int cnt, int slot)
{
    h->hq_single[slot] = (cnt == 1);
    if (cnt == 1) {                       // one factor: its own R, Q = I
        h->hr_ptr[slot] = h->Rf[modes[0]];
        h->hq_rows[slot] = h->R;
        return cudaSuccess;
    }
    const double* Rl[kMaxN];
    int64_t rows = 1;
    for (int k = 0; k < cnt; ++k) {
        Rl[k] = h->Rf[modes[k]];
        rows *= h->R;
    }
    h->hr_ptr[slot] = h->HR[slot];
    h->hq_rows[slot] = rows;
    return fold_qr(h, Rl, cnt, h->HQ[slot], h->HR[slot], false);
}

cudaError_t krp_qr_tree(Handle* h, int n, int slot, bool other_left, const int* own, int nown)
{
    const int R = h->R;
    const double* Rl[kMaxN];
    int cnt = 0;
    int64_t S = 1;                        // rows of the Khatri-Rao product of the own factors
    for (int k = 0; k < nown; ++k) S *= R;
    (void)n;
    if (other_left) {
        // V_n = L (.) Own = (Q_L (x) I_S)(R_L (.) Own)
        for (int k = 0; k < nown; ++k) Rl[cnt++] = h->Rf[own[k]];
        Rl[cnt++] = h->hr_ptr[slot];
        if (h->hq_single[slot]) return fold_qr(h, Rl, cnt, h->Q0, h->R0, false);
        CPALS_CUDA_TRY(fold_qr(h, Rl, cnt, h->Qin, h->R0, false));
        const int64_t Sa = h->hq_rows[slot];
        kron_right_apply_kernel<<<grid_for(Sa * S * R, 256, h->num_sms), 256, 0, h->stream>>>(
            h->HQ[slot], Sa, h->Qin, R, S, h->Q0, h->d_status);
        h->launches++;
        return cudaGetLastError();
    }
    // V_n = Own (.) M = (I_S (x) Q_M)(Own (.) R_M)
    if (nown == 0) {
        const int64_t rows = h->hq_rows[slot];
        if (h->hq_single[slot]) return householder_qr(h, h->hr_ptr[slot], R, R, h->Q0, h->R0, false);
        CPALS_CUDA_TRY(cudaMemcpyAsync(h->Q0, h->HQ[slot], sizeof(double) * rows * R, cudaMemcpyDeviceToDevice,
                                       h->stream));
        return cudaMemcpyAsync(h->R0, h->hr_ptr[slot], sizeof(double) * R * R, cudaMemcpyDeviceToDevice, h->stream);
    }
    Rl[cnt++] = h->hr_ptr[slot];
    for (int k = 0; k < nown; ++k) Rl[cnt++] = h->Rf[own[k]];
    if (h->hq_single[slot]) return fold_qr(h, Rl, cnt, h->Q0, h->R0, false);
    CPALS_CUDA_TRY(fold_qr(h, Rl, cnt, h->Qin, h->R0, false));
    const int64_t Sm = h->hq_rows[slot];
    kron_left_apply_kernel<<<grid_for(S * Sm * R, 256, h->num_sms), 256, 0, h->stream>>>(
        h->HQ[slot], Sm, h->Qin, R, S, h->Q0, h->d_status);
    h->launches++;
    return cudaGetLastError();
}

// CTAs of kSolveWarps row-warps for the I rows of a solve (grid-stride above
// four CTAs per SM)
inline unsigned solve_grid(int64_t I, int num_sms)
{
    const int64_t g = (I + kSolveWarps - 1) / kSolveWarps;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(g, 4LL * num_sms));
}

cudaError_t solve_qr(Handle* h, int64_t In)
{
    trsm_qr_kernel<<<solve_grid(In, h->num_sms), kSolveWarps * 32, 0, h->stream>>>(h->W, h->R0, In, h->R, h->Ahat,
                                                                                    h->d_status);
    h->launches++;
    return cudaGetLastError();
}

cudaError_t svd_operator(Handle* h, double rtol)
{
    if (!(rtol > 0.0)) rtol = (double)h->R * kEps;
    constexpr size_t smem = sizeof(double) * jacobi_smem_doubles();
    static bool attr_set = false;
    if (!attr_set) {
        CPALS_CUDA_TRY(cudaFuncSetAttribute(jacobi_pinv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)smem));
        attr_set = true;
    }
    const double* parts = nullptr;
    if (h->svd_shortcut) {
        svd_shortcut_kernel<<<(h->R + kInvWarps - 1) / kInvWarps, kInvWarps * 32, 0, h->stream>>>(
            h->R0, h->R, h->T, h->svd_parts, h->d_status);
        h->launches++;
        CPALS_CUDA_TRY(cudaGetLastError());
        parts = h->svd_parts;
    }
    jacobi_pinv_kernel<<<1, kJacobiThreads, smem, h->stream>>>(h->R0, h->R, rtol, h->T, h->d_status, parts);
    h->launches++;
    return cudaGetLastError();
}

cudaError_t solve_svd(Handle* h, int64_t In, double rtol, bool have_operator)
{
    if (!have_operator) CPALS_CUDA_TRY(svd_operator(h, rtol));
    return gemm_rows(h, h->W, In, h->R, h->T, h->R, h->Ahat);
}

cudaError_t normal_operator(Handle* h, int n, bool pinv, double rtol)
{
    GPtrs gp;
    for (int m = 0; m < h->N; ++m) gp.G[m] = h->G[m];
    hadamard_cholesky_kernel<<<1, 256, 0, h->stream>>>(gp, h->N, n, h->R, h->S, h->T, h->d_status, pinv ? 0 : 1);
    h->launches++;
    CPALS_CUDA_TRY(cudaGetLastError());
    if (!pinv) return cudaSuccess;
    // S is symmetric, so pinv(S) = pinv(S^T): the same operator as the SVD solve with R0 -> S
    if (!(rtol > 0.0)) rtol = (double)h->R * kEps;
    constexpr size_t smem = sizeof(double) * jacobi_smem_doubles();
    static bool attr_set = false;
    if (!attr_set) {
        CPALS_CUDA_TRY(cudaFuncSetAttribute(jacobi_pinv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)smem));
        attr_set = true;
    }
    jacobi_pinv_kernel<<<1, kJacobiThreads, smem, h->stream>>>(h->S, h->R, rtol, h->T, h->d_status, nullptr);
    h->launches++;
    return cudaGetLastError();
}

cudaError_t solve_normal(Handle* h, int n, bool have_operator)
{
    if (!have_operator) CPALS_CUDA_TRY(normal_operator(h, n, false, 0.0));
    chol_rows_kernel<<<solve_grid(h->dims[n], h->num_sms), kSolveWarps * 32, 0, h->stream>>>(
        h->M, h->T, h->dims[n], h->R, h->Ahat, h->d_status);
    h->launches++;
    return cudaGetLastError();
}

cudaError_t solve_normal_pinv(Handle* h, int n, double rtol, bool have_operator)
{
    if (!have_operator) CPALS_CUDA_TRY(normal_operator(h, n, true, rtol));
    return gemm_rows(h, h->M, h->dims[n], h->R, h->T, h->R, h->Ahat);
}

cudaError_t gram(Handle* h, const double* A, int64_t I, double* G)
{
    const int RR = h->R * h->R;
    gram_kernel<<<(RR + 127) / 128, 128, 0, h->stream>>>(A, I, h->R, G, h->d_status);
    h->launches++;
    return cudaGetLastError();
}

cudaError_t normalize_and_refactor(Handle* h, int n)
{
    normalize_kernel<<<h->R, 256, 0, h->stream>>>(h->Ahat, h->dims[n], h->A[n], h->lambda, h->d_status);
    h->launches++;
    return cudaGetLastError();
}

cudaError_t fit_efficient(Handle* h, int solve)
{
    const int n = h->N - 1;
    const int64_t I = h->dims[n];
    const int qr = (solve != CPALS_SOLVE_NORMAL && solve != CPALS_SOLVE_NORMAL_PINV);
    const unsigned nb = (unsigned)((I + 31) / 32);
    // split the R columns over CTAs too, so that short modes still fill the SMs
    const int ks = (int)std::max<int64_t>(1, std::min<int64_t>(h->R, (2LL * h->num_sms + nb - 1) / nb));
    const int kchunk = (h->R + ks - 1) / ks;
    const int kgrid = (h->R + kchunk - 1) / kchunk;
    fit_inner_kernel<<<dim3(nb, (unsigned)kgrid), 256, 0, h->stream>>>(qr ? h->W : h->M, h->Ahat, h->R0, I, h->R, qr,
                                                                      kchunk, h->scratch, h->d_status);
    const int nparts = (int)nb * kgrid;
    fit_norm_kernel<<<h->R, 64, 0, h->stream>>>(qr ? h->R0 : h->S, qr ? h->Rf[n] : h->G[n], h->lambda, h->R, qr,
                                                h->scratch + nparts, h->d_status);
    fit_final_kernel<<<1, 256, 0, h->stream>>>(h->scratch, nparts, h->R, h->d_normX2, h->d_fit, h->fit_cap,
                                               h->d_fit_count, h->d_fit + h->fit_cap, h->d_status);
    h->launches += 3;
    return cudaGetLastError();
}

}  // namespace cpals
