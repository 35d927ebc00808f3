// batch.cu -- many independent 3-way CP-ALS-QR problems of uneven dims and
// ranks advancing together.  A sweep follows the dimension tree of Sec. 3.3.3
// for every problem at once (modes {0, 1} | {2}), so X is read twice:
//   pass 1:  P = X x_2 Q_2^T                       (all problems, one launch)
//   mode 0:  Y_(0) from P x_1 Q_1^T, W_0, update
//   mode 1:  Y_(1) from P x_0 Q_0^T (new Q_0), W_1, update
//   pass 2:  T = X x_1 Q_1^T (new Q_1)
//   mode 2:  Y_(2) from T x_0 Q_0^T, W_2, update, efficient fit (Sec. 3.3.1).
// Every contraction -- the two passes, the last TTM of each Multi-TTM
// (Eq. multittm) and W_n = Y_(n) Q0 (Eq. ls-qr-q0-step) -- is one launch over
// all problems whose CTAs take (problem, row tile) work items from a device
// queue (an atomic counter: no CTA waits on another, so nothing needs a time
// limit); whatever the mix of sizes, every SM works on every contraction.
// These run in FP32, W accumulating in FP32 like the Multi-TTM it extends.
// What is left of a mode update is the FP64 factorisation chain of each
// problem, one CTA per problem (largest first):
//   - the substitution Ahat R0^T = W (a singular R0 sets the problem's status
//     and keeps its factor),
//   - column normalisation (2-norm) into A_n and lambda,
//   - the QR A_n = Q_n R_n (CholeskyQR2 with its check, Householder when refused),
//   - and, for the next mode, the QR V_{n+1} = Q0 R0 of the Khatri-Rao
//     product of its two other R factors (Sec. 3.1), by the staircase
//     Householder QR of a product of two triangular factors (Sec. 3.3.3: no
//     fill-in).  The QR of V_0 needs only the previous sweep's R_1, R_2, so it
//     runs on a graph branch beside pass 1.
// The sweep is captured once into a CUDA graph (twelve kernels).  The first
// iterate picks the row tile of the grouped contractions and the CTA size
// and count of the factorisation kernels by timing one sweep per candidate.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "dev_common.cuh"
#include "internal.cuh"

namespace cpals {

namespace {

constexpr double kEpsB = 2.220446049250313e-16;
constexpr int kBMaxR = 16;

struct BProb {
    int I[3];
    int R;
    int64_t x;        // FP32 X (floats)
    int64_t a[3];     // A_m (I_m x R), doubles
    int64_t q[3];     // Q_m (I_m x R)
    int64_t rf[3];    // R_m (R x R)
    int64_t lam;      // lambda (R)
    int64_t q0f, r0;  // Q0 of the current mode's V_n as FP32 [col][r] (floats), R0 (R x R, doubles)
    int64_t qf[3];    // Q_m as FP32 [k][r] (floats): what the contractions read
    int64_t w;        // W_n (up to max_n I_n x R)
    int64_t p1;       // X x_2 Q_2^T: I0 x I1 x R (floats)
    int64_t t2;       // X x_1 Q_1^T: I0 x R x I2 (floats)
    int64_t y;        // Y_(n): up to max_n I_n R^2 (floats)
    double normX2;
};

__device__ __forceinline__ double warp_sum_b(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Householder QR of the m x n matrix W (shared memory, leading dimension m,
// overwritten by the reflectors and R) with explicit Q (m x n, shared memory)
// and R (n x n, leading dimension n) with diag(R) >= 0.  Same arithmetic as the
// single-problem leaf kernel: one warp per column, dlarfg reflectors.
__device__ void cta_householder(double* W, int m, int n, double* Q, double* Rout, double* tau, double* red)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    const int kmax = min(m, n);
    for (int j = 0; j < kmax; ++j) {
        if (warp == 0) {
            double s = 0.0;
            for (int i = j + 1 + lane; i < m; i += 32) s = fma(W[i + m * j], W[i + m * j], s);
            s = warp_sum_b(s);
            if (lane == 0) {
                const double alpha = W[j + m * j];
                double t = 0.0, scale = 0.0, beta = alpha;
                if (s > 0.0) {
                    const double nrm = sqrt(fma(alpha, alpha, s));
                    beta = (alpha >= 0.0) ? -nrm : nrm;
                    const double d = beta - alpha;
                    const double r = 1.0 / (beta * d);
                    t = d * d * r;
                    scale = -beta * r;
                }
                tau[j] = t;
                red[0] = scale;
                W[j + m * j] = beta;
            }
        }
        __syncthreads();
        const double scale = red[0], tj = tau[j];
        if (tj != 0.0)
            for (int i = j + 1 + tid; i < m; i += blockDim.x) W[i + m * j] *= scale;
        __syncthreads();
        if (tj != 0.0) {
            for (int k = j + 1 + warp; k < n; k += nwarps) {
                double s = 0.0;
                for (int i = j + lane; i < m; i += 32) s = fma((i == j) ? 1.0 : W[i + m * j], W[i + m * k], s);
                s = warp_sum_b(s) * tj;
                for (int i = j + lane; i < m; i += 32) W[i + m * k] = fma(-s, (i == j) ? 1.0 : W[i + m * j], W[i + m * k]);
            }
        }
        __syncthreads();
    }
    for (int e = tid; e < m * n; e += blockDim.x) {
        const int j = e / m, i = e - j * m;
        Q[e] = (i == j) ? 1.0 : 0.0;
    }
    __syncthreads();
    for (int j = kmax - 1; j >= 0; --j) {
        const double tj = tau[j];
        if (tj != 0.0) {
            for (int k = j + warp; k < n; k += nwarps) {
                double s = 0.0;
                for (int i = j + lane; i < m; i += 32) s = fma((i == j) ? 1.0 : W[i + m * j], Q[i + m * k], s);
                s = warp_sum_b(s) * tj;
                for (int i = j + lane; i < m; i += 32) Q[i + m * k] = fma(-s, (i == j) ? 1.0 : W[i + m * j], Q[i + m * k]);
            }
        }
        __syncthreads();
    }
    // diag(R) >= 0: flip row i of R and column i of Q together
    for (int e = tid; e < m * n; e += blockDim.x) {
        const int j = e / m;
        if (j < kmax && W[j + m * j] < 0.0) Q[e] = -Q[e];
    }
    for (int e = tid; e < n * n; e += blockDim.x) {
        const int j = e / n, i = e - j * n;
        double v = 0.0;
        if (i <= j && i < kmax) v = ((W[i + m * i] < 0.0) ? -1.0 : 1.0) * W[i + m * j];
        Rout[e] = v;
    }
    __syncthreads();
}

// ---------------------------------------------------------------- CholeskyQR2 in one CTA
// The factor QR A_n = Q_n R_n by CholeskyQR2 (Fukaya, Nakatsukasa,
// Yanagisawa, Yamamoto 2014): R1 = chol(A^T A), Q1 = A R1^-1,
// R2 = chol(Q1^T Q1), Q = Q1 R2^-1, R = R2 R1.  It is accepted when the first
// Cholesky has no breakdown and every entry of Q1^T Q1 lies within 1e-2 of
// the identity (which bounds cond(A) near 7e6, where CholeskyQR2 is as
// accurate as Householder); otherwise the caller runs its Householder QR.
// The triangular inverses are formed one warp per column, so the products
// with them are independent FMAs; every sum runs in a fixed order.  (The QR
// of V stays the staircase Householder QR: CholeskyQR2 would treat the
// R^2 x R product as dense, about six times the FP64 work, and the batch's
// factorisation kernels are bound by FP64 throughput.)
constexpr double kCqrCheckB = 1e-2;
constexpr int kCqMaxE = kBMaxR * (kBMaxR + 1) / 2;
constexpr int kCqMaxWarps = 8;                 // factorisation CTAs have at most 256 threads
constexpr int kCqDoubles = kCqMaxWarps * kCqMaxE + 3 * kBMaxR * kBMaxR + kBMaxR;

struct CqWs {
    double* part;   // kCqMaxWarps x kCqMaxE Gram partials
    double* G;      // n x n Gram, then the Cholesky factor
    double* U1;     // n x n, R1
    double* X;      // n x n row-major triangular inverse
    double* d;      // n reciprocals of the diagonal
};

__device__ CqWs cq_ws(double* base)
{
    CqWs w;
    w.part = base;
    w.G = w.part + kCqMaxWarps * kCqMaxE;
    w.U1 = w.G + kBMaxR * kBMaxR;
    w.X = w.U1 + kBMaxR * kBMaxR;
    w.d = w.X + kBMaxR * kBMaxR;
    return w;
}

// G (n x n, both triangles) = S^T S for the row-major m x n matrix S: warps
// over contiguous row blocks, lanes over the packed upper-triangle entries,
// the warps' partials then added in warp order.
__device__ void cq_gram(const double* S, int m, int n, double* part, double* G)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int nE = n * (n + 1) / 2;
    constexpr int EJ = (kCqMaxE + 31) / 32;
    int ea[EJ], eb[EJ];
    double acc[EJ];
#pragma unroll
    for (int j = 0; j < EJ; ++j) {
        acc[j] = 0.0;
        ea[j] = eb[j] = 0;
        if (lane + 32 * j < nE) tri_index(lane + 32 * j, ea[j], eb[j]);
    }
    for (int i = warp * m / nw; i < (warp + 1) * m / nw; ++i) {
        const double* row = S + (size_t)i * n;
#pragma unroll
        for (int j = 0; j < EJ; ++j)
            if (lane + 32 * j < nE) acc[j] = fma(row[ea[j]], row[eb[j]], acc[j]);
    }
#pragma unroll
    for (int j = 0; j < EJ; ++j)
        if (lane + 32 * j < nE) part[warp * nE + lane + 32 * j] = acc[j];
    __syncthreads();
    for (int e = threadIdx.x; e < nE; e += blockDim.x) {
        double t = 0.0;
        for (int w = 0; w < nw; ++w) t += part[w * nE + e];
        int a, b;
        tri_index(e, a, b);
        G[a + n * b] = t;
        G[b + n * a] = t;
    }
    __syncthreads();
}

// In-place upper Cholesky of G (n x n, n <= 32) on warp 0, square roots
// deferred to the end: step j subtracts M(j, a) M(j, b) / d_j from the
// trailing triangle.  Then U(j, k) = M(j, k) / sqrt(d_j), zero below, and
// d[j] = 1 / U(j, j).  Returns false (in every thread) on a pivot that is not
// positive and finite.
__device__ bool cq_cholesky(double* G, int n, double* d, int* flag)
{
    if ((threadIdx.x >> 5) == 0) {
        const int lane = threadIdx.x & 31;
        bool bad = false;
        for (int j = 0; j < n; ++j) {
            const double piv = G[j + n * j];
            const bool ok = piv > 0.0 && piv < INFINITY;
            bad = bad || !ok;
            const double inv = ok ? rcp_nr(piv) : 0.0;
            for (int a = j + 1 + lane; a < n; a += 32) G[a + n * j] = G[j + n * a] * inv;
            __syncwarp();
            const int m = n - 1 - j;
            for (int p = lane; p < m * (m + 1) / 2; p += 32) {
                int a, b;
                tri_index(p, a, b);
                a += j + 1;
                b += j + 1;
                G[a + n * b] = fma(-G[a + n * j], G[j + n * b], G[a + n * b]);
            }
            __syncwarp();
        }
        for (int j = lane; j < n; j += 32) {
            const double piv = G[j + n * j];
            d[j] = (piv > 0.0 && piv < INFINITY) ? rsqrt_nr(piv) : 1.0;
        }
        __syncwarp();
        for (int p = lane; p < n * n; p += 32) {
            const int a = p % n, b = p / n;
            if (a > b) G[p] = 0.0;
            else if (a == b) G[p] = (G[p] > 0.0 && G[p] < INFINITY) ? G[p] * d[a] : 1.0;
            else G[p] *= d[a];
        }
        if (lane == 0) *flag = bad ? 1 : 0;
    }
    __syncthreads();
    return *flag == 0;
}

// X = U^-1 (U upper, n x n column-major; d[k] = 1 / U(k, k)) into X row-major
// (X(k, c) at X[k n + c]), one warp per column, lanes over the rows: from the
// bottom row up, X(i, c) = delta_ic / U(i, i) - (sum_{k > i} U(i, k) X(k, c))
// / U(i, i), each known value broadcast and added to the rows above.
__device__ void cq_inverse(const double* U, const double* d, int n, double* X)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int c = warp; c < n; c += nw) {
        double acc = 0.0, x = 0.0;
        for (int i = c; i >= 0; --i) {
            double xi = 0.0;
            if (lane == i) {
                xi = fma(-acc, d[i], (i == c) ? d[i] : 0.0);
                x = xi;
            }
            xi = __shfl_sync(0xffffffffu, xi, i);
            if (lane < i) acc = fma(U[lane + n * i], xi, acc);
        }
        if (lane < n) X[lane * n + c] = (lane <= c) ? x : 0.0;
    }
    __syncthreads();
}

// out(i, c) = sum_{k <= c} val(i, k) X(k, c) for the m rows (X row-major,
// upper), written through store(i, c, value).
template <typename Val, typename Store>
__device__ void cq_apply(int m, int n, const double* X, Val val, Store store)
{
    for (int p = threadIdx.x; p < m * n; p += blockDim.x) {
        const int i = p / n, c = p - i * n;
        double s = 0.0;
        for (int k = 0; k <= c; ++k) s = fma(val(i, k), X[k * n + c], s);
        store(i, c, s);
    }
    __syncthreads();
}

// The check on Q1^T Q1 (in G) and the second pass: R2 = chol(Q1^T Q1) in
// w.G, its inverse in w.X.  False when refused.
__device__ bool cq_second(CqWs w, int n, int* flag)
{
    if (threadIdx.x == 0) *flag = 0;
    __syncthreads();
    for (int p = threadIdx.x; p < n * n; p += blockDim.x) {
        const int a = p % n, b = p / n;
        if (!(fabs(w.G[p] - (a == b ? 1.0 : 0.0)) <= kCqrCheckB)) *flag = 1;
    }
    __syncthreads();
    if (*flag) return false;
    if (!cq_cholesky(w.G, n, w.d, flag)) return false;
    cq_inverse(w.G, w.d, n, w.X);
    return true;
}

// R = R2 R1 (upper; R2 in w.G, R1 in w.U1) into Rout (n x n column-major).
__device__ void cq_rprod(CqWs w, int n, double* Rout)
{
    for (int p = threadIdx.x; p < n * n; p += blockDim.x) {
        const int a = p % n, b = p / n;
        double s = 0.0;
        for (int k = a; k <= b; ++k) s = fma(w.G[a + n * k], w.U1[k + n * b], s);
        Rout[p] = (a <= b) ? s : 0.0;
    }
    __syncthreads();
}

// Factor QR of A (m x n column-major, ld m; left as it is).  S, S2: m x n
// row-major scratch.  On success Q (m x n column-major) is in S and R in Rout.
__device__ bool cta_cqr2(const double* A, int m, int n, double* S, double* S2, double* Rout, CqWs w, int* flag)
{
    for (int p = threadIdx.x; p < m * n; p += blockDim.x) {
        const int i = p / n, c = p - i * n;
        S[p] = A[i + m * c];
    }
    __syncthreads();
    cq_gram(S, m, n, w.part, w.G);
    if (!cq_cholesky(w.G, n, w.d, flag)) return false;
    for (int p = threadIdx.x; p < n * n; p += blockDim.x) w.U1[p] = w.G[p];
    cq_inverse(w.G, w.d, n, w.X);
    cq_apply(m, n, w.X, [&](int i, int k) { return S[i * n + k]; }, [&](int i, int c, double v) { S2[i * n + c] = v; });
    cq_gram(S2, m, n, w.part, w.G);
    if (!cq_second(w, n, flag)) return false;
    cq_apply(m, n, w.X, [&](int i, int k) { return S2[i * n + k]; }, [&](int i, int c, double v) { S[i + m * c] = v; });
    cq_rprod(w, n, Rout);
    return true;
}

// ---------------------------------------------------------------- grouped contractions
// One TTM of every problem, viewed as [L, K, T] (Sec. 2.2):
//   which 0: X  x_2 Q_2^T -> P   [L = I0 I1, K = I2, T = 1]   (pass 1)
//   which 1: X  x_1 Q_1^T -> T   [L = I0,    K = I1, T = I2]  (pass 2)
//   which 2: P  x_1 Q_1^T -> Y   [L = I0,    K = I1, T = R]   (mode 0)
//   which 3: P  x_0 Q_0^T -> Y   [L = 1,     K = I0, T = I1 R] (mode 1)
//   which 4: T  x_0 Q_0^T -> Y   [L = 1,     K = I0, T = R I2] (mode 2)
struct BView {
    int64_t in, out;     // offsets into the input and output arrays
    int m;               // the contracted mode (its Q_m)
    int64_t L, T;
    int K;
};

__host__ __device__ inline BView view_of(const BProb& pr, int which)
{
    BView v;
    const int64_t R = pr.R;
    switch (which) {
        case 0: v = {pr.x, pr.p1, 2, (int64_t)pr.I[0] * pr.I[1], 1, pr.I[2]}; break;
        case 1: v = {pr.x, pr.t2, 1, pr.I[0], pr.I[2], pr.I[1]}; break;
        case 2: v = {pr.p1, pr.y, 1, pr.I[0], R, pr.I[1]}; break;
        case 3: v = {pr.p1, pr.y, 0, 1, (int64_t)pr.I[1] * R, pr.I[0]}; break;
        default: v = {pr.t2, pr.y, 0, 1, R * pr.I[2], pr.I[0]}; break;
    }
    return v;
}

// One thread per flattened row f = l + L t of the view, its R FP32
// accumulators summed in order of k; loads along l are coalesced when L > 1.
template <int R>
__device__ __forceinline__ void ttm_row(const float* __restrict__ X, int64_t L, int K, int64_t T, const float* qs,
                                        int64_t f, float* __restrict__ out)
{
    if (f >= L * T) return;
    const int64_t t = f / L, l = f - t * L;
    const float* x = X + l + L * (int64_t)K * t;
    float acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = 0.0f;
    // sixteen loads in flight per thread: the passes stream X, so the bytes
    // in flight per SM (not the FMAs) set the rate
    int k = 0;
    for (; k + 16 <= K; k += 16) {
        float v[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) v[u] = __ldg(x + L * (int64_t)(k + u));
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int r = 0; r < R; ++r) acc[r] = fmaf(v[u], qs[(k + u) * R + r], acc[r]);
    }
    for (; k < K; ++k) {
        const float v = __ldg(x + L * (int64_t)k);
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] = fmaf(v, qs[k * R + r], acc[r]);
    }
    float* o = out + l + L * (int64_t)R * t;
#pragma unroll
    for (int r = 0; r < R; ++r) o[L * r] = acc[r];
}

struct BItem {
    int p;
    int f0;
};

// The next work item of a grouped launch (thread 0 takes it from the queue).
__device__ __forceinline__ int next_item(int* counter, int* s_item)
{
    __syncthreads();
    if (threadIdx.x == 0) *s_item = atomicAdd(counter, 1);
    __syncthreads();
    return *s_item;
}

__global__ void batch_ttm_kernel(const BProb* __restrict__ probs, const BItem* __restrict__ items, int n_items,
                                 int* __restrict__ counter, int which, const float* __restrict__ Xall,
                                 float* __restrict__ P1all, float* __restrict__ T2all, float* __restrict__ Yall,
                                 const float* __restrict__ Qf, const int* __restrict__ pstatus)
{
    __shared__ float qs[128 * kBMaxR];   // Q_m as FP32 [k][r] for K <= 128
    __shared__ int s_item;
    int cached = -1;
    for (;;) {
        const int it = next_item(counter, &s_item);
        if (it >= n_items) break;
        const BItem item = items[it];
        if (pstatus[item.p] != kStatusOk) continue;
        const BProb& pr = probs[item.p];
        const BView v = view_of(pr, which);
        const int R = pr.R;
        const float* in = (which <= 1 ? Xall : (which == 4 ? T2all : P1all)) + v.in;
        float* out = (which == 0 ? P1all : (which == 1 ? T2all : Yall)) + v.out;
        const float* Q = Qf + pr.qf[v.m];              // [k][r]
        const int64_t f = item.f0 + threadIdx.x;
        if (v.K <= 128) {
            if (cached != item.p) {
                for (int e = threadIdx.x; e < v.K * R; e += blockDim.x) qs[e] = __ldg(Q + e);
                cached = item.p;
                __syncthreads();
            }
            switch (R) {
#define CPALS_BT(RV) case RV: ttm_row<RV>(in, v.L, v.K, v.T, qs, f, out); break;
                CPALS_BT(1) CPALS_BT(2) CPALS_BT(3) CPALS_BT(4) CPALS_BT(5) CPALS_BT(6) CPALS_BT(7) CPALS_BT(8)
                CPALS_BT(9) CPALS_BT(10) CPALS_BT(11) CPALS_BT(12) CPALS_BT(13) CPALS_BT(14) CPALS_BT(15) CPALS_BT(16)
#undef CPALS_BT
                default: break;
            }
        } else if (f < v.L * v.T) {
            // long modes: Q read through L1, the same sums in order of k
            const int64_t t = f / v.L, l = f - t * v.L;
            const float* x = in + l + v.L * (int64_t)v.K * t;
            float acc[kBMaxR];
#pragma unroll
            for (int r = 0; r < kBMaxR; ++r) acc[r] = 0.0f;
            for (int k = 0; k < v.K; ++k) {
                const float xv = __ldg(x + v.L * (int64_t)k);
#pragma unroll
                for (int r = 0; r < kBMaxR; ++r)
                    if (r < R) acc[r] = fmaf(xv, __ldg(Q + (int64_t)k * R + r), acc[r]);
            }
            float* o = out + l + v.L * (int64_t)R * t;
#pragma unroll
            for (int r = 0; r < kBMaxR; ++r)
                if (r < R) o[v.L * r] = acc[r];
            cached = -1;
        }
    }
}

// W_n = Y_(n) Q0 for every problem: one thread per row i of a tile, its R
// FP32 accumulators summed over the R^2 columns in order.  Y element (i, col),
// col = a + Rn c, sits at a + Rn (i + In c) with Rn = 1, R, R^2 for n = 0, 1, 2.
// Q0 is staged once per problem from its FP32 [col][r] copy.
template <int R>
__device__ __forceinline__ void w_row(const float* __restrict__ Y, int In, int n, const float* q0f, int i,
                                      double* __restrict__ W)
{
    if (i >= In) return;
    constexpr int RR = R * R;
    float acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = 0.0f;
    // eight columns at a time, loads first; col = a + Rn c sits at a + Rn (i + In c)
    for (int col0 = 0; col0 < RR; col0 += 8) {
        float y[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int col = col0 + u;
            int64_t addr;
            if (n == 0) addr = i + (int64_t)In * col;                                   // Rn = 1
            else if (n == 1) addr = col % R + (int64_t)R * (i + (int64_t)In * (col / R));  // Rn = R
            else addr = col + (int64_t)RR * i;                                          // Rn = R^2
            y[u] = (col < RR) ? __ldg(Y + addr) : 0.0f;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int col = (col0 + u < RR) ? col0 + u : RR - 1;   // y is zero past the end
#pragma unroll
            for (int r = 0; r < R; ++r) acc[r] = fmaf(y[u], q0f[col * R + r], acc[r]);
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) W[i + (int64_t)In * r] = (double)acc[r];
}

__global__ void batch_w_kernel(const BProb* __restrict__ probs, const BItem* __restrict__ items, int n_items,
                               int* __restrict__ counter, int n, const float* __restrict__ Yall,
                               const float* __restrict__ Qf, double* __restrict__ F, const int* __restrict__ pstatus)
{
    __shared__ float q0f[kBMaxR * kBMaxR * kBMaxR];
    __shared__ int s_item;
    int cached = -1;
    for (;;) {
        const int it = next_item(counter, &s_item);
        if (it >= n_items) break;
        const BItem item = items[it];
        if (pstatus[item.p] != kStatusOk) continue;
        const BProb& pr = probs[item.p];
        const int R = pr.R, RR = R * R, In = pr.I[n];
        if (cached != item.p) {
            const float* Q0 = Qf + pr.q0f;                 // [col][r]
            for (int e = threadIdx.x; e < RR * R; e += blockDim.x) q0f[e] = __ldg(Q0 + e);
            cached = item.p;
            __syncthreads();
        }
        const int i = item.f0 + threadIdx.x;
        const float* Y = Yall + pr.y;
        double* W = F + pr.w;
        switch (R) {
#define CPALS_BW(RV) case RV: w_row<RV>(Y, In, n, q0f, i, W); break;
            CPALS_BW(1) CPALS_BW(2) CPALS_BW(3) CPALS_BW(4) CPALS_BW(5) CPALS_BW(6) CPALS_BW(7) CPALS_BW(8)
            CPALS_BW(9) CPALS_BW(10) CPALS_BW(11) CPALS_BW(12) CPALS_BW(13) CPALS_BW(14) CPALS_BW(15) CPALS_BW(16)
#undef CPALS_BW
            default: break;
        }
    }
}

// ---------------------------------------------------------------- factorisation chain
struct BSmem {
    int64_t regA, regB, r0, rn, w, cq;   // offsets in doubles
    int64_t total;
};

__host__ __device__ inline BSmem bsmem_layout(int maxR, int maxI)
{
    BSmem s;
    // the staircase QR of V_n needs two compact copies (R(R+1)(2R+1)/6 each) and
    // the 2 R^2 row indices; the factor QR needs I R
    const int64_t stair = (int64_t)maxR * (maxR + 1) * (2 * maxR + 1) / 3 + (int64_t)maxR * maxR + 8;
    const int64_t ir = (int64_t)maxI * maxR;
    const int64_t sa = ir > stair ? ir : stair;
    const int64_t sb = ir > (int64_t)maxR * maxR * maxR ? ir : (int64_t)maxR * maxR * maxR;
    s.regA = 0;
    s.regB = s.regA + sa;
    s.r0 = s.regB + sb;
    s.rn = s.r0 + (int64_t)maxR * maxR;
    s.w = s.rn + (int64_t)maxR * maxR;
    s.cq = s.w + ir;
    s.total = s.cq + kCqDoubles + 128;    // + tau / red
    return s;
}

// V = R_hi (.) R_lo of the mode `next` and its staircase QR into the
// problem's Q0, R0 (global).  rhi / rlo may point to shared or global memory.
__device__ void v_qr(const BProb& pr, const double* rhi, const double* rlo, double* F, float* Qf, double* regA,
                     double* qtmp, double* tau, double* red)
{
    const int R = pr.R, RR = R * R, tot = stair_off(R);
    int* rows_i = reinterpret_cast<int*>(regA + 2 * tot);
    stair_qr_block(rhi, rlo, R, regA, regA + tot, tau, red, rows_i, rows_i + RR, qtmp, F + pr.r0);
    for (int e = threadIdx.x; e < RR * R; e += blockDim.x) {
        const int col = e / R, r = e - col * R;
        Qf[pr.q0f + e] = (float)qtmp[col + RR * r];
    }
    __syncthreads();
}

// Q_m (FP64, I x R column-major, shared or global) as the FP32 [k][r] copy.
__device__ void write_qf(const BProb& pr, int m, const double* Q, float* Qf)
{
    const int I = pr.I[m], R = pr.R;
    for (int e = threadIdx.x; e < I * R; e += blockDim.x) {
        const int k = e / R, r = e - k * R;
        Qf[pr.qf[m] + e] = (float)Q[k + I * r];
    }
}

// The QR of V_0 = R_2 (.) R_1 of every problem (the start of a sweep).
__global__ void batch_vqr_kernel(const BProb* __restrict__ probs, const int* __restrict__ order, int count,
                                 int maxR, int maxI, double* __restrict__ F, float* __restrict__ Qf,
                                 const int* __restrict__ pstatus)
{
    extern __shared__ double bsm[];
    const BSmem L = bsmem_layout(maxR, maxI);
    double* tau = bsm + L.total - 128;
    double* red = tau + 64;
    for (int idx = blockIdx.x; idx < count; idx += gridDim.x) {
        const int p = order[idx];
        if (pstatus[p] != kStatusOk) continue;
        const BProb pr = probs[p];
        v_qr(pr, F + pr.rf[2], F + pr.rf[1], F, Qf, bsm + L.regA, bsm + L.regB, tau, red);
    }
}

// The FP64 end of mode n's update for every problem: substitution,
// normalisation, factor QR, then the QR of the next mode's V (n < 2) or the
// efficient fit (n = 2).
__global__ void batch_tail_kernel(const BProb* __restrict__ probs, const int* __restrict__ order, int count, int n,
                                  int maxR, int maxI, double* __restrict__ F, float* __restrict__ Qf,
                                  int* __restrict__ pstatus, double* __restrict__ fit_last)
{
    extern __shared__ double bsm[];
    const BSmem L = bsmem_layout(maxR, maxI);
    double* regA = bsm + L.regA;
    double* regB = bsm + L.regB;
    double* R0s = bsm + L.r0;
    double* Rns = bsm + L.rn;
    double* Ws = bsm + L.w;
    double* tau = bsm + L.total - 128;
    double* red = tau + 64;
    const CqWs cw = cq_ws(bsm + L.cq);
    __shared__ int singular, cq_flag;
    __shared__ double inner_sh;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;

    for (int idx = blockIdx.x; idx < count; idx += gridDim.x) {
        const int p = order[idx];
        if (pstatus[p] != kStatusOk) continue;       // a failed problem stays as it was
        const BProb pr = probs[p];
        const int R = pr.R, In = pr.I[n], RR = R * R;
        for (int e = tid; e < RR; e += blockDim.x) R0s[e] = F[pr.r0 + e];
        for (int e = tid; e < In * R; e += blockDim.x) Ws[e] = F[pr.w + e];
        __syncthreads();
        if (tid == 0) {
            double dmax = 0.0;
            for (int k = 0; k < R; ++k) dmax = fmax(dmax, fabs(R0s[k + R * k]));
            int s = 0;
            for (int k = 0; k < R; ++k)
                if (!(fabs(R0s[k + R * k]) > (double)R * kEpsB * dmax)) s = 1;
            singular = s;
            if (s) pstatus[p] = CPALS_ERR_SINGULAR;
        }
        __syncthreads();
        if (singular) continue;
        // Ahat R0^T = W by substitution, one row per thread (Ahat into regA);
        // loops unrolled over the largest rank so that x stays in registers
        if (tid < R) red[16 + tid] = 1.0 / R0s[tid + R * tid];
        __syncthreads();
        for (int i = tid; i < In; i += blockDim.x) {
            double x[kBMaxR];
#pragma unroll
            for (int k = kBMaxR - 1; k >= 0; --k) {
                if (k < R) {
                    double s = Ws[i + In * k];
#pragma unroll
                    for (int j = k + 1; j < kBMaxR; ++j)
                        if (j < R) s = fma(-R0s[k + R * j], x[j], s);
                    x[k] = s * red[16 + k];
                } else {
                    x[k] = 0.0;
                }
            }
#pragma unroll
            for (int k = 0; k < kBMaxR; ++k)
                if (k < R) regA[i + In * k] = x[k];
        }
        __syncthreads();
        // efficient-fit inner product <W, Ahat R0^T> (last mode only)
        if (n == 2) {
            double s = 0.0;
            for (int e = tid; e < In * R; e += blockDim.x) {
                const int k = e / In, i = e - k * In;
                double v = 0.0;
                for (int j = 0; j < R; ++j) v = fma(regA[i + In * j], R0s[k + R * j], v);
                s = fma(Ws[e], v, s);
            }
            s = warp_sum_b(s);
            if (lane == 0) red[8 + warp] = s;
            __syncthreads();
            if (tid == 0) {
                double t = 0.0;
                for (int w = 0; w < nwarps; ++w) t += red[8 + w];
                inner_sh = t;
            }
            __syncthreads();
        }
        // normalise columns (2-norm): A_n and lambda
        double* lam = F + pr.lam;
        for (int r = warp; r < R; r += nwarps) {
            double s = 0.0;
            for (int i = lane; i < In; i += 32) s = fma(regA[i + In * r], regA[i + In * r], s);
            s = warp_sum_b(s);
            if (lane == 0) red[32 + r] = sqrt(s);
        }
        __syncthreads();
        double* An = F + pr.a[n];
        for (int e = tid; e < In * R; e += blockDim.x) {
            const int r = e / In;
            const double l = red[32 + r];
            const double v = (l > 0.0) ? regA[e] / l : regA[e];
            regA[e] = v;
            An[e] = v;
        }
        if (tid < R) lam[tid] = red[32 + tid];
        __syncthreads();
        // A_n = Q_n R_n (FP64, shared memory): CholeskyQR2 (Q into Ws, the
        // W stash, which is spent), Householder when it is refused
        const double* Qs = Ws;
        if (!cta_cqr2(regA, In, R, Ws, regB, Rns, cw, &cq_flag)) {
            cta_householder(regA, In, R, regB, Rns, tau, red);
            Qs = regB;
        }
        double* Qn = F + pr.q[n];
        double* Rn_g = F + pr.rf[n];
        for (int e = tid; e < In * R; e += blockDim.x) Qn[e] = Qs[e];
        for (int e = tid; e < RR; e += blockDim.x) Rn_g[e] = Rns[e];
        write_qf(pr, n, Qs, Qf);
        if (n == 2) {
            // efficient fit after the last mode (Sec. 3.3.1)
            double s = 0.0;
            for (int e = tid; e < RR; e += blockDim.x) {
                const int b = e / R, a = e - b * R;
                double g0 = 0.0, gN = 0.0;
                for (int k = 0; k < R; ++k) {
                    g0 = fma(R0s[k + R * a], R0s[k + R * b], g0);
                    gN = fma(Rns[k + R * a], Rns[k + R * b], gN);
                }
                s = fma(g0 * red[32 + a], gN * red[32 + b], s);
            }
            s = warp_sum_b(s);
            __syncthreads();
            if (lane == 0) red[8 + warp] = s;
            __syncthreads();
            if (tid == 0) {
                double nrm = 0.0;
                for (int w = 0; w < nwarps; ++w) nrm += red[8 + w];
                double res2 = pr.normX2 - 2.0 * inner_sh + nrm;
                if (res2 < 0.0) res2 = 0.0;
                fit_last[p] = 1.0 - sqrt(res2) / sqrt(pr.normX2);
            }
        } else {
            // the next mode's V = R_hi (.) R_lo: mode 1 takes R_2 (.) R_0, mode 2 R_1 (.) R_0
            __syncthreads();
            const double* rhi = (n == 0) ? F + pr.rf[2] : F + pr.rf[1];
            v_qr(pr, (n == 1) ? Rns : rhi, (n == 0) ? Rns : F + pr.rf[0], F, Qf, regA, regB, tau, red);
        }
        __syncthreads();
    }
}

// QR of every initial factor: one CTA per (problem, mode).
__global__ void batch_factor_qr_kernel(BProb* __restrict__ probs, int count, int maxR, int maxI,
                                       double* __restrict__ F, float* __restrict__ Qf)
{
    extern __shared__ double bsm[];
    const BSmem L = bsmem_layout(maxR, maxI);
    const int p = blockIdx.x / 3, m = blockIdx.x % 3;
    if (p >= count) return;
    const BProb pr = probs[p];
    const int I = pr.I[m], R = pr.R;
    double* regA = bsm + L.regA;
    double* regB = bsm + L.regB;
    double* Rs = bsm + L.r0;
    double* tau = bsm + L.total - 128;
    double* red = tau + 64;
    const double* A = F + pr.a[m];
    for (int e = threadIdx.x; e < I * R; e += blockDim.x) regA[e] = A[e];
    __syncthreads();
    cta_householder(regA, I, R, regB, Rs, tau, red);
    for (int e = threadIdx.x; e < I * R; e += blockDim.x) F[pr.q[m] + e] = regB[e];
    for (int e = threadIdx.x; e < R * R; e += blockDim.x) F[pr.rf[m] + e] = Rs[e];
    write_qf(pr, m, regB, Qf);
}

// ||X_p||^2 in FP64, one CTA per problem.
__global__ void batch_norm_kernel(BProb* __restrict__ probs, int count, const float* __restrict__ Xall)
{
    const int p = blockIdx.x;
    if (p >= count) return;
    const BProb pr = probs[p];
    const int64_t P = (int64_t)pr.I[0] * pr.I[1] * pr.I[2];
    double s = 0.0;
    for (int64_t e = threadIdx.x; e < P; e += blockDim.x) {
        const double v = Xall[pr.x + e];
        s = fma(v, v, s);
    }
    __shared__ double sh[32];
    s = warp_sum_b(s);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
        probs[p].normX2 = t;
    }
}

}  // namespace

// ---------------------------------------------------------------- host side
constexpr int kTiles[2] = {128, 256};
constexpr int kTtmWhich = 5;       // grouped TTMs: two passes, three last TTMs
constexpr int kSweepKernels = 12;  // V_0 QR, five TTMs, three W, three factorisation kernels

struct Batch {
    int count = 0, maxR = 0, maxI = 0;
    std::vector<BProb> probs;
    std::vector<int> order;
    BProb* d_probs = nullptr;
    int* d_order = nullptr;
    float* Xall = nullptr;
    double* F = nullptr;
    float* Qf = nullptr;                 // FP32 copies of Q_m ([k][r]) and Q0 ([col][r])
    float* P1all = nullptr;
    float* T2all = nullptr;
    float* Yall = nullptr;
    int* d_pstatus = nullptr;
    double* d_fit = nullptr;
    // work items of the grouped launches per candidate row tile: the five TTMs, then W for modes 0..2
    BItem* d_items[2][kTtmWhich + 3] = {};
    int n_items[2][kTtmWhich + 3] = {};
    int* d_counter = nullptr;            // one queue counter per grouped launch of a sweep
    int64_t x_elems = 0, f_elems = 0, qf_elems = 0, p1_elems = 0, t2_elems = 0, y_elems = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t side = nullptr;         // the QR of V_0 beside pass 1
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    int num_sms = 0;
    // tuned shape: the grouped launches' tile (threads) and grid; the factorisation kernels' threads and grid
    int tile = 0, group_grid = 0, w_grid = 0, grid = 0, threads = 0;
    cudaGraphExec_t graph = nullptr;
    int64_t launches = 0;
    size_t smem = 0;
    bool have_X = false, have_factors = false;
    char err[512] = {0};
};

static int64_t align4(int64_t v) { return (v + 3) & ~(int64_t)3; }

cudaError_t batch_build(Batch* b, int count, const int64_t* dims, const int* ranks)
{
    b->count = count;
    b->probs.resize(count);
    int64_t xo = 0, fo = 0, qfo = 0, p1o = 0, t2o = 0, yo = 0;
    std::vector<double> work(count);
    for (int p = 0; p < count; ++p) {
        BProb& pr = b->probs[p];
        for (int m = 0; m < 3; ++m) pr.I[m] = (int)dims[3 * p + m];
        pr.R = ranks[p];
        b->maxR = std::max(b->maxR, pr.R);
        for (int m = 0; m < 3; ++m) b->maxI = std::max(b->maxI, pr.I[m]);
        const int64_t P = (int64_t)pr.I[0] * pr.I[1] * pr.I[2];
        const int64_t R = pr.R;
        pr.x = xo;
        xo += align4(P);
        for (int m = 0; m < 3; ++m) { pr.a[m] = fo; fo += pr.I[m] * R; }
        for (int m = 0; m < 3; ++m) { pr.q[m] = fo; fo += pr.I[m] * R; }
        for (int m = 0; m < 3; ++m) { pr.rf[m] = fo; fo += R * R; }
        pr.lam = fo;
        fo += R;
        for (int m = 0; m < 3; ++m) { pr.qf[m] = qfo; qfo += align4(pr.I[m] * R); }
        pr.q0f = qfo;
        qfo += align4(R * R * R);
        pr.r0 = fo;
        fo += R * R;
        pr.w = fo;
        fo += (int64_t)std::max({pr.I[0], pr.I[1], pr.I[2]}) * R;
        pr.p1 = p1o;
        p1o += align4((int64_t)pr.I[0] * pr.I[1] * R);
        pr.t2 = t2o;
        t2o += align4((int64_t)pr.I[0] * R * pr.I[2]);
        int64_t ymax = 0;
        for (int n = 0; n < 3; ++n) ymax = std::max(ymax, (int64_t)pr.I[n] * R * R);
        pr.y = yo;
        yo += align4(ymax);
        pr.normX2 = 0.0;
        // the factorisation chain: Householder steps over I_n x R and the staircase of R^2 x R
        work[p] = (double)R * R * (pr.I[0] + pr.I[1] + pr.I[2]) + 3.0 * R * R * R * R;
    }
    b->order.resize(count);
    std::iota(b->order.begin(), b->order.end(), 0);
    std::stable_sort(b->order.begin(), b->order.end(), [&](int a, int c) { return work[a] > work[c]; });
    b->x_elems = xo; b->f_elems = fo; b->qf_elems = qfo; b->p1_elems = p1o; b->t2_elems = t2o; b->y_elems = yo;
    CPALS_CUDA_TRY(cudaMalloc(&b->d_probs, sizeof(BProb) * count));
    CPALS_CUDA_TRY(cudaMalloc(&b->d_order, sizeof(int) * count));
    CPALS_CUDA_TRY(cudaMalloc(&b->Xall, sizeof(float) * std::max<int64_t>(xo, 1)));
    CPALS_CUDA_TRY(cudaMalloc(&b->F, sizeof(double) * std::max<int64_t>(fo, 1)));
    CPALS_CUDA_TRY(cudaMalloc(&b->Qf, sizeof(float) * std::max<int64_t>(qfo, 1)));
    CPALS_CUDA_TRY(cudaMalloc(&b->P1all, sizeof(float) * std::max<int64_t>(p1o, 1)));
    CPALS_CUDA_TRY(cudaMalloc(&b->T2all, sizeof(float) * std::max<int64_t>(t2o, 1)));
    CPALS_CUDA_TRY(cudaMalloc(&b->Yall, sizeof(float) * std::max<int64_t>(yo, 1)));
    CPALS_CUDA_TRY(cudaMalloc(&b->d_pstatus, sizeof(int) * count));
    CPALS_CUDA_TRY(cudaMalloc(&b->d_fit, sizeof(double) * count));
    CPALS_CUDA_TRY(cudaMalloc(&b->d_counter, sizeof(int) * (kTtmWhich + 3)));
    CPALS_CUDA_TRY(cudaMemset(b->F, 0, sizeof(double) * std::max<int64_t>(fo, 1)));
    CPALS_CUDA_TRY(cudaMemset(b->d_pstatus, 0, sizeof(int) * count));
    CPALS_CUDA_TRY(cudaMemset(b->d_fit, 0, sizeof(double) * count));
    CPALS_CUDA_TRY(cudaMemcpy(b->d_probs, b->probs.data(), sizeof(BProb) * count, cudaMemcpyHostToDevice));
    CPALS_CUDA_TRY(cudaMemcpy(b->d_order, b->order.data(), sizeof(int) * count, cudaMemcpyHostToDevice));
    // work items: the tiles of each problem's rows, problems with the most
    // rows first, for each candidate tile
    for (int ti = 0; ti < 2; ++ti)
        for (int g = 0; g < kTtmWhich + 3; ++g) {
            auto rows_of = [&](int p) -> int64_t {
                const BProb& pr = b->probs[p];
                if (g < kTtmWhich) {
                    const BView v = view_of(pr, g);
                    return v.L * v.T;
                }
                return pr.I[g - kTtmWhich];
            };
            std::vector<int> by(count);
            std::iota(by.begin(), by.end(), 0);
            std::stable_sort(by.begin(), by.end(), [&](int a, int c) {
                return rows_of(a) * b->probs[a].R > rows_of(c) * b->probs[c].R;
            });
            std::vector<BItem> items;
            for (int p : by) {
                const int64_t rows = rows_of(p);
                for (int64_t f0 = 0; f0 < rows; f0 += kTiles[ti]) items.push_back(BItem{p, (int)f0});
            }
            b->n_items[ti][g] = (int)items.size();
            CPALS_CUDA_TRY(cudaMalloc(&b->d_items[ti][g], sizeof(BItem) * std::max<size_t>(items.size(), 1)));
            CPALS_CUDA_TRY(cudaMemcpy(b->d_items[ti][g], items.data(), sizeof(BItem) * items.size(),
                                      cudaMemcpyHostToDevice));
        }
    int dev = 0;
    CPALS_CUDA_TRY(cudaGetDevice(&dev));
    CPALS_CUDA_TRY(cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, dev));
    int lo = 0, hi = 0;
    CPALS_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    CPALS_CUDA_TRY(cudaStreamCreateWithPriority(&b->side, cudaStreamNonBlocking, hi));
    CPALS_CUDA_TRY(cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming));
    CPALS_CUDA_TRY(cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming));
    b->smem = sizeof(double) * (size_t)bsmem_layout(b->maxR, b->maxI).total;
    CPALS_CUDA_TRY(cudaFuncSetAttribute(batch_tail_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem));
    CPALS_CUDA_TRY(cudaFuncSetAttribute(batch_vqr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem));
    CPALS_CUDA_TRY(cudaFuncSetAttribute(batch_factor_qr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)b->smem));
    return cudaSuccess;
}

void batch_free(Batch* b)
{
    auto f = [](void* p) { if (p) cudaFree(p); };
    f(b->d_probs); f(b->d_order); f(b->Xall); f(b->F); f(b->Qf); f(b->P1all); f(b->T2all); f(b->Yall); f(b->d_pstatus);
    f(b->d_fit); f(b->d_counter);
    for (int ti = 0; ti < 2; ++ti)
        for (int g = 0; g < kTtmWhich + 3; ++g) f(b->d_items[ti][g]);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->side) cudaStreamDestroy(b->side);
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    if (b->ev_join) cudaEventDestroy(b->ev_join);
}

cudaError_t batch_norms(Batch* b)
{
    batch_norm_kernel<<<b->count, 256, 0, b->stream>>>(b->d_probs, b->count, b->Xall);
    b->launches++;
    return cudaGetLastError();
}

cudaError_t batch_factor_qr(Batch* b)
{
    batch_factor_qr_kernel<<<3 * b->count, 256, b->smem, b->stream>>>(b->d_probs, b->count, b->maxR, b->maxI, b->F,
                                                                       b->Qf);
    b->launches++;
    return cudaGetLastError();
}

static cudaError_t grouped_ttm(Batch* b, int ti, int which, int grid)
{
    CPALS_CUDA_TRY(cudaMemsetAsync(b->d_counter + which, 0, sizeof(int), b->stream));
    batch_ttm_kernel<<<grid, kTiles[ti], 0, b->stream>>>(b->d_probs, b->d_items[ti][which], b->n_items[ti][which],
                                                         b->d_counter + which, which, b->Xall, b->P1all, b->T2all,
                                                         b->Yall, b->Qf, b->d_pstatus);
    b->launches++;
    return cudaGetLastError();
}

static cudaError_t grouped_w(Batch* b, int ti, int n, int grid)
{
    const int g = kTtmWhich + n;
    CPALS_CUDA_TRY(cudaMemsetAsync(b->d_counter + g, 0, sizeof(int), b->stream));
    batch_w_kernel<<<grid, kTiles[ti], 0, b->stream>>>(b->d_probs, b->d_items[ti][g], b->n_items[ti][g],
                                                       b->d_counter + g, n, b->Yall, b->Qf, b->F, b->d_pstatus);
    b->launches++;
    return cudaGetLastError();
}

static cudaError_t chain(Batch* b, int n, int grid, int threads)
{
    batch_tail_kernel<<<grid, threads, b->smem, b->stream>>>(b->d_probs, b->d_order, b->count, n, b->maxR, b->maxI,
                                                             b->F, b->Qf, b->d_pstatus, b->d_fit);
    b->launches++;
    return cudaGetLastError();
}

// One sweep along the dimension tree.  The QR of V_0 runs on the side stream
// beside pass 1 (two branches of the captured graph).
static cudaError_t batch_sweep(Batch* b, int ti, int group_grid, int w_grid, int grid, int threads)
{
    CPALS_CUDA_TRY(cudaEventRecord(b->ev_fork, b->stream));
    CPALS_CUDA_TRY(cudaStreamWaitEvent(b->side, b->ev_fork, 0));
    batch_vqr_kernel<<<grid, threads, b->smem, b->side>>>(b->d_probs, b->d_order, b->count, b->maxR, b->maxI, b->F,
                                                          b->Qf, b->d_pstatus);
    b->launches++;
    CPALS_CUDA_TRY(cudaGetLastError());
    CPALS_CUDA_TRY(cudaEventRecord(b->ev_join, b->side));
    CPALS_CUDA_TRY(grouped_ttm(b, ti, 0, group_grid));           // pass 1
    CPALS_CUDA_TRY(cudaStreamWaitEvent(b->stream, b->ev_join, 0));
    for (int n = 0; n < 3; ++n) {
        if (n == 2) CPALS_CUDA_TRY(grouped_ttm(b, ti, 1, group_grid));   // pass 2
        CPALS_CUDA_TRY(grouped_ttm(b, ti, 2 + n, group_grid));            // the last TTM of mode n
        CPALS_CUDA_TRY(grouped_w(b, ti, n, w_grid));
        CPALS_CUDA_TRY(chain(b, n, grid, threads));
    }
    return cudaSuccess;
}

// Pick the launch shapes by timing one sweep per candidate on a copy of the
// factors (restored afterwards): the grouped launches' row tile (128 or 256
// rows per work item, as many resident CTAs as fit), and the factorisation
// kernels' CTA size (128 or 256) and CTAs per SM.  Then capture the sweep as
// a CUDA graph.
cudaError_t batch_prepare(Batch* b)
{
    if (b->graph) return cudaSuccess;
    double* saved = nullptr;
    float* saved_qf = nullptr;
    CPALS_CUDA_TRY(cudaMalloc(&saved, sizeof(double) * std::max<int64_t>(b->f_elems, 1)));
    CPALS_CUDA_TRY(cudaMalloc(&saved_qf, sizeof(float) * std::max<int64_t>(b->qf_elems, 1)));
    CPALS_CUDA_TRY(cudaMemcpyAsync(saved, b->F, sizeof(double) * b->f_elems, cudaMemcpyDeviceToDevice, b->stream));
    CPALS_CUDA_TRY(cudaMemcpyAsync(saved_qf, b->Qf, sizeof(float) * b->qf_elems, cudaMemcpyDeviceToDevice,
                                   b->stream));
    cudaEvent_t e0, e1;
    CPALS_CUDA_TRY(cudaEventCreate(&e0));
    CPALS_CUDA_TRY(cudaEventCreate(&e1));
    float best = 1e30f;
    int ggrid[2] = {0, 0}, wgrid[2] = {0, 0};
    for (int ti = 0; ti < 2; ++ti) {
        int o1 = 0, o2 = 0;
        CPALS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o1, batch_ttm_kernel, kTiles[ti], 0));
        CPALS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o2, batch_w_kernel, kTiles[ti], 0));
        ggrid[ti] = std::max(1, o1) * b->num_sms;
        wgrid[ti] = std::max(1, o2) * b->num_sms;
    }
    const int threads_c[2] = {128, 256};
    for (int ti = 0; ti < 2; ++ti)
        for (int mi = 0; mi < 2; ++mi) {
            int occ = 0;
            CPALS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, batch_tail_kernel, threads_c[mi],
                                                                         b->smem));
            if (occ < 1) continue;
            for (int per = 1; per <= occ; ++per) {
                const int grid = std::min(b->count, b->num_sms * per);
                CPALS_CUDA_TRY(cudaMemcpyAsync(b->F, saved, sizeof(double) * b->f_elems, cudaMemcpyDeviceToDevice,
                                               b->stream));
                CPALS_CUDA_TRY(cudaMemcpyAsync(b->Qf, saved_qf, sizeof(float) * b->qf_elems,
                                               cudaMemcpyDeviceToDevice, b->stream));
                CPALS_CUDA_TRY(cudaEventRecord(e0, b->stream));
                CPALS_CUDA_TRY(batch_sweep(b, ti, ggrid[ti], wgrid[ti], grid, threads_c[mi]));
                CPALS_CUDA_TRY(cudaEventRecord(e1, b->stream));
                CPALS_CUDA_TRY(cudaEventSynchronize(e1));
                float ms = 0.f;
                CPALS_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
                if (ms < best) {
                    best = ms;
                    b->tile = kTiles[ti];
                    b->group_grid = ggrid[ti];
                    b->w_grid = wgrid[ti];
                    b->grid = grid;
                    b->threads = threads_c[mi];
                }
                if (grid == b->count) break;
            }
        }
    CPALS_CUDA_TRY(cudaMemcpyAsync(b->F, saved, sizeof(double) * b->f_elems, cudaMemcpyDeviceToDevice, b->stream));
    CPALS_CUDA_TRY(cudaMemcpyAsync(b->Qf, saved_qf, sizeof(float) * b->qf_elems, cudaMemcpyDeviceToDevice,
                                   b->stream));
    CPALS_CUDA_TRY(cudaMemsetAsync(b->d_pstatus, 0, sizeof(int) * b->count, b->stream));
    CPALS_CUDA_TRY(cudaStreamSynchronize(b->stream));
    cudaFree(saved);
    cudaFree(saved_qf);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (b->grid == 0) return cudaErrorInvalidConfiguration;
    // capture one sweep
    cudaStream_t cap = b->stream;
    bool own = false;
    if (cap == nullptr) {
        CPALS_CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        own = true;
    }
    cudaStream_t saved_stream = b->stream;
    b->stream = cap;
    const int64_t l0 = b->launches;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    cudaError_t e2 = cudaSuccess;
    if (e == cudaSuccess) {
        e2 = batch_sweep(b, b->tile == kTiles[0] ? 0 : 1, b->group_grid, b->w_grid, b->grid, b->threads);
        e = cudaStreamEndCapture(cap, &g);
    }
    b->stream = saved_stream;
    b->launches = l0;
    if (own) cudaStreamDestroy(cap);
    CPALS_CUDA_TRY(e2);
    CPALS_CUDA_TRY(e);
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    return e;
}

cudaError_t batch_run(Batch* b, int iters);

size_t batch_smem_bytes(int maxR, int maxI) { return sizeof(double) * (size_t)bsmem_layout(maxR, maxI).total; }

Batch* batch_new() { return new (std::nothrow) Batch(); }

void batch_delete(Batch* b)
{
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    else cudaDeviceSynchronize();
    batch_free(b);
    delete b;
}

cudaError_t batch_set_stream(Batch* b, cudaStream_t s)
{
    b->stream = s;
    if (b->graph) {                       // the graph was captured on another stream: recapture
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    return cudaSuccess;
}

cudaError_t batch_set_tensors(Batch* b, const float* const* X, bool host)
{
    const cudaMemcpyKind kind = host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    for (int p = 0; p < b->count; ++p) {
        const BProb& pr = b->probs[p];
        const int64_t P = (int64_t)pr.I[0] * pr.I[1] * pr.I[2];
        CPALS_CUDA_TRY(cudaMemcpyAsync(b->Xall + pr.x, X[p], sizeof(float) * P, kind, b->stream));
    }
    CPALS_CUDA_TRY(batch_norms(b));
    CPALS_CUDA_TRY(cudaStreamSynchronize(b->stream));
    b->have_X = true;
    return cudaSuccess;
}

cudaError_t batch_set_factors(Batch* b, const double* const* A, bool host)
{
    const cudaMemcpyKind kind = host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    std::vector<double> ones(kBMaxR, 1.0);
    for (int p = 0; p < b->count; ++p) {
        const BProb& pr = b->probs[p];
        for (int m = 0; m < 3; ++m)
            CPALS_CUDA_TRY(cudaMemcpyAsync(b->F + pr.a[m], A[3 * p + m], sizeof(double) * pr.I[m] * pr.R, kind,
                                           b->stream));
        CPALS_CUDA_TRY(cudaMemcpyAsync(b->F + pr.lam, ones.data(), sizeof(double) * pr.R, cudaMemcpyHostToDevice,
                                       b->stream));
    }
    CPALS_CUDA_TRY(batch_factor_qr(b));
    CPALS_CUDA_TRY(cudaMemsetAsync(b->d_pstatus, 0, sizeof(int) * b->count, b->stream));
    CPALS_CUDA_TRY(cudaStreamSynchronize(b->stream));
    b->have_factors = true;
    return cudaSuccess;
}

cudaError_t batch_get_factors(Batch* b, double* const* A, double* const* lambda, bool host)
{
    const cudaMemcpyKind kind = host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    for (int p = 0; p < b->count; ++p) {
        const BProb& pr = b->probs[p];
        if (A)
            for (int m = 0; m < 3; ++m)
                if (A[3 * p + m])
                    CPALS_CUDA_TRY(cudaMemcpyAsync(A[3 * p + m], b->F + pr.a[m], sizeof(double) * pr.I[m] * pr.R,
                                                   kind, b->stream));
        if (lambda && lambda[p])
            CPALS_CUDA_TRY(cudaMemcpyAsync(lambda[p], b->F + pr.lam, sizeof(double) * pr.R, kind, b->stream));
    }
    return cudaStreamSynchronize(b->stream);
}

cudaError_t batch_iterate(Batch* b, int iters, double* fits_host, int* status_host)
{
    CPALS_CUDA_TRY(batch_run(b, iters));
    if (fits_host)
        CPALS_CUDA_TRY(cudaMemcpyAsync(fits_host, b->d_fit, sizeof(double) * b->count, cudaMemcpyDeviceToHost,
                                       b->stream));
    if (status_host)
        CPALS_CUDA_TRY(cudaMemcpyAsync(status_host, b->d_pstatus, sizeof(int) * b->count, cudaMemcpyDeviceToHost,
                                       b->stream));
    return cudaStreamSynchronize(b->stream);
}

int64_t batch_launches(const Batch* b) { return b->launches; }
bool batch_ready(const Batch* b) { return b->have_X && b->have_factors; }
int batch_tuned_grid(const Batch* b) { return b->grid; }
int batch_tuned_threads(const Batch* b) { return b->threads; }
char* batch_err(Batch* b) { return b->err; }

cudaError_t batch_run(Batch* b, int iters)
{
    CPALS_CUDA_TRY(batch_prepare(b));
    for (int it = 0; it < iters; ++it) {
        CPALS_CUDA_TRY(cudaGraphLaunch(b->graph, b->stream));
        b->launches += kSweepKernels;
    }
    return cudaSuccess;
}

}  // namespace cpals
