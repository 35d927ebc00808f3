// tail.cu -- the end of a mode update in one thread-block cluster: everything
// of Alg. cp-als-qr's mode-loop body after W_n = Y_(n) Q0 (and of Alg.
// cp-als's after the MTTKRP), i.e.
//   1. the solve: Ahat R0^T = W by substitution (Eq. ls-qr-q0-step; a
//      numerically singular R0 sets CPALS_ERR_SINGULAR and nothing is written),
//      Ahat = W T with the truncated SVD or pseudo-inverse operator T (Sec. 3.1,
//      Sec. 2.3), or Ahat S = M with S = L L^T (Alg. cp-als).  Above rank 32
//      the R^2 work per row is better spread over every SM, so the host runs
//      the solve with the GPU-wide kernels first and the cluster starts from
//      Ahat (kind 3);
//   2. lambda_r = ||Ahat(:, r)||_2 and A_n = Ahat diag(lambda)^-1 (a zero
//      column keeps lambda_r = 0 and stays as it is);
//   3. G_n = A_n^T A_n (the Gram that the normal equations use);
//   4. the factor QR A_n = Q_n R_n with diag(R_n) > 0 (Alg. cp-als-qr's re-QR)
//      by CholeskyQR2 (Fukaya, Nakatsukasa, Yanagisawa, Yamamoto 2014):
//      R1 = chol(G_n), Q1 = A_n R1^-1, R2 = chol(Q1^T Q1), Q_n = Q1 R2^-1,
//      R_n = R2 R1.  The thin QR with a positive diagonal is unique, so this is
//      the factorisation Householder QR gives, up to rounding, as long as A_n
//      is well conditioned.  The check after the first pass (Cholesky without
//      breakdown, and every entry of Q1^T Q1 within 1e-2 of the identity,
//      which bounds cond(A_n) near 7e6) decides; when it fails the kernel
//      writes no Q_n, R_n and sets a gate word, and the Householder QR that
//      the host enqueues behind it runs (it is a no-op while the gate is 0).
// Kind 4 takes a factor as it is (no solve, no normalisation) and gives its
// Gram and QR only.  Every factor QR of a handle goes through this kernel
// (the initial ones and those a later QR solve needs after normal-equations
// sweeps), and the Gram is always taken over the same rows split the same way,
// so a run resumed from saved factors repeats the uninterrupted run bit for
// bit.
//
// Why one cluster: FP64 on this part issues 2 DFMA/clk/SM and a dependent
// FP64 operation takes 64 cycles, so the separate kernels of this tail (the
// substitution, the normalisation, a Householder QR on one SM) were bound by
// latency and launch gaps.  Here the rows of the factor are split over the C
// CTAs of one cluster; the column sums and the Grams are reduced across the
// cluster through distributed shared memory, in a fixed order (every CTA adds
// the C partials itself, so all of them hold the same sums and no broadcast
// step is needed); the R x R Cholesky factorisations run in every CTA.  All
// CTAs pass the same four cluster barriers whatever the data, so the kernel
// cannot deadlock on a data-dependent branch.
//
// FP64 issues one warp instruction per 64 cycles per scheduler here, however
// many lanes are active, so the substitutions give each row T lanes (T from a
// cost model: the fewest FP64 instructions on the busiest scheduler), the
// Cholesky keeps only one reciprocal per step on its sequential chain (square
// roots at the end), and those reciprocals come from an FP32 seed refined by
// Newton-Raphson steps.
#include <cooperative_groups.h>

#include <algorithm>
#include <mutex>

#include "dev_common.cuh"
#include "internal.cuh"

namespace cg = cooperative_groups;

namespace cpals {

namespace {

constexpr int kTailThreads = 512;
constexpr int kTailWarps = kTailThreads / 32;
constexpr int kTailMaxCluster = 16;
constexpr size_t kTailSmemMax = 210 * 1024;
// Q1^T Q1 within this of the identity (entrywise) after the first pass
constexpr double kCqrCheck = 1e-2;

struct TailArgs {
    const double* W;     // I x R: W_n (QR, SVD), M_n (normal equations), Ahat (kind 3) or A_n (kind 4)
    const double* Op;    // R x R: R0 (kind 0), T (kind 1), the Cholesky factor L of S_n (kind 2); else unused
    int64_t I;
    int R;
    int kind;
    int want_qr;
    int lanes;           // lanes per row in the substitutions (a power of two, at most 32)
    double* Ahat;        // I x R
    double* A;           // I x R, the normalised factor
    double* lambda;      // R
    double* G;           // R x R, A^T A
    double* Q;           // I x R
    double* Rf;          // R x R, upper
    int* gate;           // 1: the Householder QR must run (written by CTA 0 when want_qr)
    int* status;
};

// Shared-memory layout (doubles): operator / R1, Cholesky work matrix, two
// partial-sum buffers read by the other CTAs, per-group partials, the pivots
// (and lambda), two row stashes of rl x (R+1) (the second only for kind 1).
struct TailSmem {
    int R, nE, rl;
    size_t op, gw, pa, pb, gp, piv, rows, rows2, total;
    __host__ __device__ TailSmem(int R_, int rl_, int kind) : R(R_), rl(rl_)
    {
        nE = R * (R + 1) / 2;
        const size_t RR = (size_t)R * R;
        // the solve operator (kinds 0..2) also holds R1 later; kinds 3 and 4
        // have no operator and park R1 in the output R instead
        op = 0;
        gw = op + (kind <= 2 ? RR : 0);
        pa = gw + RR;
        pb = pa + (size_t)nE;
        gp = pb + (size_t)nE;
        piv = gp + (size_t)kTailThreads;   // kTailThreads >= (kTailThreads / R) * R for the column sums
        rows = piv + (size_t)2 * R;
        // the stash also stages R2 R1 (R x R) at the end for kinds 3 and 4
        const size_t stash = (size_t)rl * (R + 1) > RR ? (size_t)rl * (R + 1) : RR;
        rows2 = rows + stash;
        total = rows2 + (kind == 1 ? (size_t)rl * (R + 1) : 0);
    }
};

// 1/d and 1/sqrt(d) to about one ulp: the FP32 hardware approximation
// (rcp.approx / rsqrt.approx, about 2^-23 relative) refined by two
// Newton-Raphson steps in FP64 -- y <- y + y (1 - d y) for the reciprocal,
// y <- y + y (1/2 - (d/2) y^2) for the reciprocal square root -- each of
// which squares the relative error.  A dependent FP64 operation costs 64
// cycles on this part, and these are a few of them against the much longer
// exact division and square root.  Outside the FP32 normal range the exact
// FP64 operations are used.
__device__ __forceinline__ double rcp_nr(double d)
{
    const double a = fabs(d);
    if (!(a > 1e-36 && a < 1e36)) return 1.0 / d;
    float f;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(f) : "f"((float)d));
    double y = (double)f;
    double e = fma(-d, y, 1.0);
    y = fma(y, e, y);
    e = fma(-d, y, 1.0);
    return fma(y, e, y);
}

__device__ __forceinline__ double rsqrt_nr(double d)
{
    if (!(d > 1e-36 && d < 1e36)) return 1.0 / sqrt(d);
    float f;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(f) : "f"((float)d));
    double y = (double)f;
    const double h = 0.5 * d;
    double e = fma(-h * y, y, 0.5);
    y = fma(y, e, y);
    e = fma(-h * y, y, 0.5);
    return fma(y, e, y);
}

// Upper-triangle index e -> (a, b) with a <= b, e = b (b + 1) / 2 + a.
__device__ __forceinline__ void tri_index(int e, int& a, int& b)
{
    int q = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
    while (q * (q + 1) / 2 > e) --q;
    while ((q + 1) * (q + 2) / 2 <= e) ++q;
    b = q;
    a = e - q * (q + 1) / 2;
}

// part[e] = sum over the stashed rows of row[a] * row[b] (upper triangle of
// the local Gram), rows summed in a fixed order per group and the groups in
// order.
__device__ void local_gram(const double* rows, int rl, int R, double* gp, double* part)
{
    const int nE = R * (R + 1) / 2, ld = R + 1, tid = threadIdx.x;
    if (2 * nE <= kTailThreads) {
        const int groups = kTailThreads / nE;
        if (tid < groups * nE) {
            const int e = tid % nE, g = tid / nE;
            int a, b;
            tri_index(e, a, b);
            double s = 0.0;
            for (int li = g; li < rl; li += groups) s = fma(rows[li * ld + a], rows[li * ld + b], s);
            gp[g * nE + e] = s;
        }
        __syncthreads();
        if (tid < nE) {
            double s = gp[tid];
            for (int g = 1; g < groups; ++g) s += gp[g * nE + tid];
            part[tid] = s;
        }
    } else {
        for (int e = tid; e < nE; e += kTailThreads) {
            int a, b;
            tri_index(e, a, b);
            double s = 0.0;
            for (int li = 0; li < rl; ++li) s = fma(rows[li * ld + a], rows[li * ld + b], s);
            part[e] = s;
        }
    }
}

// M (R x R, full symmetric) = sum over the cluster's CTAs, in rank order, of
// their partial upper triangles.
__device__ void cluster_gram(cg::cluster_group& cluster, double* part, int R, double* M)
{
    const int nE = R * (R + 1) / 2, C = (int)cluster.num_blocks();
    for (int e = threadIdx.x; e < nE; e += kTailThreads) {
        double s = 0.0;
        for (int c = 0; c < C; ++c) s += cluster.map_shared_rank(part, c)[e];
        int a, b;
        tri_index(e, a, b);
        M[a + R * b] = s;
        M[b + R * a] = s;
    }
}

// In-place upper Cholesky M = U^T U, block-parallel and right-looking, with
// the square roots taken at the end: step j subtracts M(j,a) M(j,b) / d_j
// from the trailing block (d_j the pivot, M's row j not yet scaled), so the
// sequential chain holds one reciprocal per step.  Then U(j,j) = sqrt(d_j),
// U(j,k) = M(j,k) / sqrt(d_j), and dinv[j] = 1 / U(j,j).  The strict lower
// triangle is set to zero.  Returns false (in every thread) on a pivot that
// is not positive and finite.
__device__ bool block_cholesky(double* M, int R, double* piv, double* dinv, int* bad)
{
    const int tid = threadIdx.x;
    if (tid == 0) *bad = 0;
    __syncthreads();
    for (int j = 0; j < R; ++j) {
        if (tid == 0) {
            const double d = M[j + R * j];
            if (!(d > 0.0) || !(d < INFINITY)) *bad = 1;
            piv[j] = (d > 0.0 && d < INFINITY) ? rcp_nr(d) : 0.0;
        }
        __syncthreads();
        const double inv = piv[j];
        const int m = R - 1 - j;
        for (int p = tid; p < m * m; p += kTailThreads) {
            const int a = j + 1 + p % m, b = j + 1 + p / m;
            if (a <= b) M[a + R * b] = fma(-M[j + R * a] * inv, M[j + R * b], M[a + R * b]);
        }
        __syncthreads();
    }
    if (tid < R) {
        const double d = M[tid + R * tid];
        const double r = (d > 0.0 && d < INFINITY) ? rsqrt_nr(d) : 1.0;
        dinv[tid] = r;
        piv[tid] = r;
    }
    __syncthreads();
    for (int p = tid; p < R * R; p += kTailThreads) {
        const int a = p % R, b = p / R;
        if (a > b) M[p] = 0.0;
        else if (a == b) M[p] = (M[p] > 0.0 && M[p] < INFINITY) ? M[p] * piv[a] : 1.0;
        else M[p] *= piv[a];
    }
    __syncthreads();
    return *bad == 0;
}

// One triangular substitution on each stashed row (a row vector w of R
// entries), T lanes per row (lane g of the group owns entries g, g + T, ...),
// in place:
//   back = true:  U x = w, U(e, k) = A[e + R k] upper (or A[k + R e] when trans),
//                 from k = R-1 down;
//   back = false: L y = w, L(e, k) = A[e + R k] lower (or A[k + R e] when trans),
//                 from k = 0 up.
// dinv holds the reciprocals of the diagonal.  Every lane of the warp passes
// the same shuffles, whatever its row.
__device__ void subst_rows(double* rows, int ld, int rl, const double* A, const double* dinv, int R, int T,
                           bool back, bool trans)
{
    const int tid = threadIdx.x, lane = tid & 31;
    const int gi = lane & (T - 1), gbase = lane - gi;
    const int per_pass = kTailThreads / T;
    for (int li0 = 0; li0 < rl; li0 += per_pass) {
        const int li = li0 + tid / T;
        const bool ok = li < rl;
        double* w = rows + (size_t)(ok ? li : 0) * ld;
        for (int t = 0; t < R; ++t) {
            const int k = back ? R - 1 - t : t;
            const int owner = k & (T - 1);
            double xk = 0.0;
            if (ok && gi == owner) {
                xk = w[k] * dinv[k];
                w[k] = xk;
            }
            xk = __shfl_sync(0xffffffffu, xk, gbase + owner);
            if (ok) {
                if (back) {
                    for (int e = gi; e < k; e += T) w[e] = fma(-(trans ? A[k + R * e] : A[e + R * k]), xk, w[e]);
                } else {
                    for (int e = k + 1 + ((gi - (k + 1)) & (T - 1)); e < R; e += T)
                        w[e] = fma(-(trans ? A[k + R * e] : A[e + R * k]), xk, w[e]);
                }
            }
        }
    }
}

// part[e] = sum over the stashed rows of row[e]^2 for e < R, in a fixed
// order (rows in groups, then the groups in order).
__device__ void local_colsq(const double* rows, int rl, int R, double* gp, double* part)
{
    const int ld = R + 1, tid = threadIdx.x;
    const int groups = kTailThreads / R;
    if (tid < groups * R) {
        const int e = tid % R, g = tid / R;
        double s = 0.0;
        for (int li = g; li < rl; li += groups) s = fma(rows[li * ld + e], rows[li * ld + e], s);
        gp[g * R + e] = s;
    }
    __syncthreads();
    if (tid < R) {
        double s = gp[tid];
        for (int g = 1; g < groups; ++g) s += gp[g * R + tid];
        part[tid] = s;
    }
}

__global__ void __launch_bounds__(kTailThreads, 1) mode_tail_kernel(TailArgs g)
{
    cg::cluster_group cluster = cg::this_cluster();
    extern __shared__ double sm[];
    __shared__ int flag_bad, flag_skip, flag_check;
    __shared__ double dinv[kMaxRank];
    const int R = g.R, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int C = (int)cluster.num_blocks(), c = (int)cluster.block_rank();
    const int64_t r0 = (int64_t)c * g.I / C, r1 = (int64_t)(c + 1) * g.I / C;
    const int rl = (int)(r1 - r0);
    const TailSmem L(R, rl, g.kind);
    double* Mo = sm + L.op;
    double* Gw = sm + L.gw;
    double* pa = sm + L.pa;
    double* pb = sm + L.pb;
    double* gp = sm + L.gp;
    double* piv = sm + L.piv;
    double* rows = sm + L.rows;
    const int ld = R + 1;
    const int T = g.lanes;
    const bool solve = g.kind <= 2, normalise = g.kind <= 3;

    if (tid == 0) flag_skip = (*(volatile int*)g.status != kStatusOk) ? 1 : 0;
    if (solve)
        for (int e = tid; e < R * R; e += kTailThreads) Mo[e] = g.Op[e];
    // the rows of W (or of Ahat, or of A_n) into the stash
    for (int p = tid; p < rl * R; p += kTailThreads) {
        const int li = p % rl, e = p / rl;
        rows[li * ld + e] = g.W[(r0 + li) + g.I * e];
    }
    __syncthreads();
    if (!flag_skip && g.kind == 0 && warp == 0) {
        // singular R0: |R0(k,k)| <= R eps max_j |R0(j,j)| (every CTA decides alike)
        const int e0 = lane, e1 = lane + 32;
        const double a0 = e0 < R ? fabs(Mo[e0 + R * e0]) : 0.0;
        const double a1 = e1 < R ? fabs(Mo[e1 + R * e1]) : 0.0;
        double dmax = fmax(a0, a1);
        for (int o = 16; o > 0; o >>= 1) dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
        const double tol = (double)R * kEps * dmax;
        const bool bad = (e0 < R && !(a0 > tol)) || (e1 < R && !(a1 > tol));
        if (__any_sync(0xffffffffu, bad) && lane == 0) {
            flag_skip = 1;
            if (c == 0) atomicCAS(g.status, kStatusOk, (int)CPALS_ERR_SINGULAR);
        }
    }
    __syncthreads();
    const bool skip = flag_skip != 0;

    // 1. the solve, in place on the stash (kind 1: into the second stash),
    // and the column sums of squares of Ahat
    if (!skip && normalise) {
        if ((g.kind == 0 || g.kind == 2) && tid < R) dinv[tid] = 1.0 / Mo[tid + R * tid];
        __syncthreads();
        if (g.kind == 0) {
            subst_rows(rows, ld, rl, Mo, dinv, R, T, true, false);
        } else if (g.kind == 2) {
            subst_rows(rows, ld, rl, Mo, dinv, R, T, false, false);    // L y = m
            subst_rows(rows, ld, rl, Mo, dinv, R, T, true, true);      // L^T x = y
        } else if (g.kind == 1) {
            double* out = sm + L.rows2;                               // W T, summed in order of k
            for (int p = tid; p < rl * R; p += kTailThreads) {
                const int li = p / R, e = p - li * R;
                double x = 0.0;
                for (int k = 0; k < R; ++k) x = fma(rows[li * ld + k], Mo[k + R * e], x);
                out[li * ld + e] = x;
            }
            rows = out;
        }
        __syncthreads();
        if (solve)
            for (int p = tid; p < rl * R; p += kTailThreads) {
                const int li = p % rl, e = p / rl;
                g.Ahat[(r0 + li) + g.I * e] = rows[li * ld + e];
            }
        local_colsq(rows, rl, R, gp, pa);
    }
    cluster.sync();                                               // (1) column sums of squares

    // 2. lambda and A_n = Ahat diag(lambda)^-1; the local Gram of A_n
    if (!skip) {
        if (normalise) {
            if (tid < R) {
                double s = 0.0;
                for (int q = 0; q < C; ++q) s += cluster.map_shared_rank(pa, q)[tid];
                const double l = sqrt(s);
                piv[tid] = l;
                if (c == 0) g.lambda[tid] = l;
            }
            __syncthreads();
            for (int p = tid; p < rl * R; p += kTailThreads) {
                const int li = p % rl, e = p / rl;
                const double l = piv[e];
                const double v = rows[li * ld + e];
                const double a = (l > 0.0) ? v / l : v;
                rows[li * ld + e] = a;
                g.A[(r0 + li) + g.I * e] = a;
            }
            __syncthreads();
        }
        local_gram(rows, rl, R, gp, pb);
    }
    cluster.sync();                                               // (2) Gram partials of A_n

    bool qr_ok = false;
    if (!skip) {
        cluster_gram(cluster, pb, R, Gw);
        __syncthreads();
        if (c == 0)
            for (int e = tid; e < R * R; e += kTailThreads) g.G[e] = Gw[e];
        if (g.want_qr) {
            // 3. the first CholeskyQR pass: R1 = chol(G_n), Q1 = A_n R1^-1
            qr_ok = block_cholesky(Gw, R, piv, dinv, &flag_bad);
            // keep R1: in Mo (the solve operator is spent), or in the output R
            // (CTA 0) when there is no operator buffer
            if (solve) {
                for (int e = tid; e < R * R; e += kTailThreads) Mo[e] = Gw[e];
            } else if (c == 0) {
                for (int e = tid; e < R * R; e += kTailThreads) g.Rf[e] = Gw[e];
            }
            __syncthreads();
            if (qr_ok) {
                subst_rows(rows, ld, rl, solve ? Mo : Gw, dinv, R, T, false, true);   // R1^T q^T = a^T
                __syncthreads();
                local_gram(rows, rl, R, gp, pa);
            }
        }
    }
    cluster.sync();                                               // (3) Gram partials of Q1

    if (!skip && g.want_qr) {
        // every CTA took the same first pass (identical sums), so qr_ok agrees
        if (qr_ok) {
            cluster_gram(cluster, pa, R, Gw);
            if (tid == 0) flag_check = 0;
            __syncthreads();
            for (int e = tid; e < R * R; e += kTailThreads) {
                const int a = e % R, b = e / R;
                const double dev = Gw[e] - (a == b ? 1.0 : 0.0);
                if (!(fabs(dev) <= kCqrCheck)) flag_check = 1;
            }
            __syncthreads();
            qr_ok = flag_check == 0;
            if (qr_ok) qr_ok = block_cholesky(Gw, R, piv, dinv, &flag_bad);
        }
        if (qr_ok) {
            // 4. Q_n = Q1 R2^-1 by rows; R_n = R2 R1
            subst_rows(rows, ld, rl, Gw, dinv, R, T, false, true);
            __syncthreads();
            for (int p = tid; p < rl * R; p += kTailThreads) {
                const int li = p % rl, e = p / rl;
                g.Q[(r0 + li) + g.I * e] = rows[li * ld + e];
            }
            if (c == 0) {
                if (solve) {
                    for (int e = tid; e < R * R; e += kTailThreads) {
                        const int a = e % R, b = e / R;
                        double s = 0.0;
                        for (int k = a; k <= b; ++k) s = fma(Gw[a + R * k], Mo[k + R * b], s);
                        g.Rf[e] = (a <= b) ? s : 0.0;
                    }
                } else {
                    // R1 from the output R, R2 R1 through the row stash (the
                    // rows are written out above), then back to the output
                    __syncthreads();
                    for (int e = tid; e < R * R; e += kTailThreads) {
                        const int a = e % R, b = e / R;
                        double s = 0.0;
                        for (int k = a; k <= b; ++k) s = fma(Gw[a + R * k], g.Rf[k + R * b], s);
                        rows[e] = (a <= b) ? s : 0.0;
                    }
                    __syncthreads();
                    for (int e = tid; e < R * R; e += kTailThreads) g.Rf[e] = rows[e];
                }
            }
        }
        if (c == 0 && tid == 0) *g.gate = qr_ok ? 0 : 1;
    }
    cluster.sync();                                               // (4) no CTA leaves while its shared memory is read
}

// Cluster size: up to 16 CTAs with at least 8 rows each.
int tail_cluster(int64_t I)
{
    return (int)std::max<int64_t>(1, std::min<int64_t>(kTailMaxCluster, I / 8));
}

// Lanes per row for the substitutions: the count with the fewest FP64 warp
// instructions on the busiest of the SM's four schedulers (rows of a CTA
// spread over T-lane groups; a step costs one multiply and ceil(R/T) FMAs).
int tail_lanes(int rl, int R)
{
    int best = 1;
    int64_t best_cost = -1;
    for (int T = 1; T <= 32; T *= 2) {
        if (T > 1 && T / 2 >= R) break;
        const int64_t lanes = (int64_t)rl * T;
        const int64_t warps = std::min<int64_t>((lanes + 31) / 32, kTailWarps);
        const int64_t passes = (lanes + kTailThreads - 1) / kTailThreads;
        const int64_t per_sched = (warps + 3) / 4;
        const int64_t cost = passes * per_sched * R * (1 + (R + T - 1) / T);
        if (best_cost < 0 || cost < best_cost) { best_cost = cost; best = T; }
    }
    return best;
}

__global__ void recip_check_kernel(const double* __restrict__ x, int64_t n, double* __restrict__ rcp,
                                   double* __restrict__ rsq)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        rcp[i] = rcp_nr(x[i]);
        rsq[i] = x[i] > 0.0 ? rsqrt_nr(x[i]) : 0.0;
    }
}

}  // namespace

cudaError_t recip_check(const double* x, int64_t n, double* rcp, double* rsq, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 4096);
    recip_check_kernel<<<(unsigned)blocks, 256, 0, st>>>(x, n, rcp, rsq);
    return cudaGetLastError();
}

bool mode_tail_ok(int64_t I, int R, int kind)
{
    if (R < 1 || R > kMaxRank || I < 1) return false;
    const int C = tail_cluster(I);
    const int rl = (int)((I + C - 1) / C);
    return TailSmem(R, rl, kind).total * sizeof(double) <= kTailSmemMax;
}

namespace {

// Launch the cluster kernel for I rows with the arguments of a.
cudaError_t launch_tail(Handle* h, int64_t I, TailArgs a)
{
    const int R = a.R;
    if (!mode_tail_ok(I, R, a.kind)) return cudaErrorInvalidValue;
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [] {
        attr_err = cudaFuncSetAttribute(mode_tail_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)kTailSmemMax);
        if (attr_err == cudaSuccess)
            attr_err = cudaFuncSetAttribute(mode_tail_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    });
    CPALS_CUDA_TRY(attr_err);
    int C = tail_cluster(I);
    a.I = I;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(kTailThreads);
    cfg.stream = h->stream;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    // a cluster of more than 8 CTAs is not portable: take the largest size
    // the device can place
    for (;;) {
        const int rl = (int)((I + C - 1) / C);
        cfg.gridDim = dim3((unsigned)C);
        cfg.dynamicSmemBytes = TailSmem(R, rl, a.kind).total * sizeof(double);
        attr[0].val.clusterDim.x = (unsigned)C;
        int nclusters = 0;
        if (C <= 8 || (cudaOccupancyMaxActiveClusters(&nclusters, mode_tail_kernel, &cfg) == cudaSuccess &&
                       nclusters > 0))
            break;
        cudaGetLastError();
        C = 8;
    }
    a.lanes = tail_lanes((int)((I + C - 1) / C), R);
    CPALS_CUDA_TRY(cudaLaunchKernelEx(&cfg, mode_tail_kernel, a));
    h->launches++;
    return cudaSuccess;
}

}  // namespace

cudaError_t mode_tail(Handle* h, int n, int kind, const double* W, const double* Op, bool want_qr)
{
    TailArgs a;
    a.W = W;
    a.Op = Op;
    a.R = h->R;
    a.kind = kind;
    a.want_qr = want_qr ? 1 : 0;
    a.Ahat = h->Ahat;
    a.A = h->A[n];
    a.lambda = h->lambda;
    a.G = h->G[n];
    a.Q = h->Q[n];
    a.Rf = h->Rf[n];
    a.gate = h->d_gate;
    a.status = h->d_status;
    return launch_tail(h, h->dims[n], a);
}

cudaError_t cqr2_rows(Handle* h, const double* V, int64_t rows, double* Q, double* Rout, double* G, int* gate)
{
    TailArgs a;
    a.W = V;
    a.Op = nullptr;
    a.R = h->R;
    a.kind = 4;
    a.want_qr = 1;
    a.Ahat = nullptr;
    a.A = nullptr;
    a.lambda = nullptr;
    a.G = G;
    a.Q = Q;
    a.Rf = Rout;
    a.gate = gate;
    a.status = h->d_status;
    return launch_tail(h, rows, a);
}

}  // namespace cpals
