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
// roots at the end), and those reciprocals come from a hardware approximation
// refined by one third-order Newton step.
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
__device__ __forceinline__ void cholesky_pivot(const double* M, int R, int j, double* piv, int* bad)
{
    const double d = M[j + R * j];
    if (!(d > 0.0) || !(d < INFINITY)) *bad = 1;
    piv[j] = (d > 0.0 && d < INFINITY) ? rcp_nr(d) : 0.0;
}

__device__ bool block_cholesky(double* M, int R, double* piv, double* dinv, int* bad)
{
    // (a, b) of the packed upper-triangle index p (p = b (b + 1) / 2 + a),
    // a | b << 8, for the trailing triangles of every step
    __shared__ uint16_t tri_ab[(kMaxRank - 1) * kMaxRank / 2];
    const int tid = threadIdx.x;
    for (int p = tid; p < (R - 1) * R / 2; p += kTailThreads) {
        int a, b;
        tri_index(p, a, b);
        tri_ab[p] = (uint16_t)(a | (b << 8));
    }
    if (tid == 0) {
        *bad = 0;
        cholesky_pivot(M, R, 0, piv, bad);
    }
    __syncthreads();
    for (int j = 0; j < R; ++j) {
        const double inv = piv[j];
        const int m = R - 1 - j;
        // the pivot row scaled once (M(j, a) / d_j into the strict lower
        // triangle's column j, which no later step reads), then one FMA per
        // entry of the trailing upper triangle, packed so that no lane of an
        // FP64 warp instruction idles.  The thread that updates entry
        // (j+1, j+1) -- the next pivot, final after this step -- takes its
        // reciprocal at once, while the other warps are still updating.
        for (int a = j + 1 + tid; a < R; a += kTailThreads) M[a + R * j] = M[j + R * a] * inv;
        __syncthreads();
        for (int p = tid; p < m * (m + 1) / 2; p += kTailThreads) {
            const int ab = tri_ab[p];
            const int a = (ab & 0xff) + j + 1, b = (ab >> 8) + j + 1;
            M[a + R * b] = fma(-M[a + R * j], M[j + R * b], M[a + R * b]);
            if (p == 0) cholesky_pivot(M, R, j + 1, piv, bad);
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

// ------------------------------------------------------------------------
// GPU-wide CholeskyQR2 (rank above 32): the normalisation and factor QR
// A_n = Q_n R_n that close a mode update of Alg. cp-als-qr, and the QR of each
// Kronecker fold step of V_n (Eq. kr-id, Sec. 3.3.3), by the CholeskyQR2 of
// Fukaya, Nakatsukasa, Yanagisawa and Yamamoto (2014) with the cluster
// kernel's acceptance check.  There the tail's FP64 work per row is R^2, and the cluster's 16 SMs hold a tenth of the GPU's FP64 rate, so the
// kinds that start from Ahat or A (3, 4) and the fold-step QRs run as a chain
// of kernels over every SM instead:
//   colsq   column sums of squares of Ahat per row block            (kind 3)
//   lambda  lambda_r = sqrt of their sum, in block order             (kind 3)
//   rows    A_n = Ahat diag(lambda)^-1, and the Gram partial of A_n per row
//           block (kind 4: of the A_n given)
//   reduce  the partials summed in 8 fixed groups of blocks
//   chol    G_n = the sum of the groups; R1 = chol(G_n) and R1^-1 (one CTA)
//   rows    Q1 = A_n R1^-1 and the Gram partial of Q1 per row block
//   reduce
//   chol2   the check on Q1^T Q1, R2 = chol(Q1^T Q1), R2^-1, R_n = R2 R1
//   rows    Q_n = Q1 R2^-1 (in place)
// For a fold step V = F (.) B the first Gram is (F^T F) * (B^T B) entrywise
// (the Gram of a Khatri-Rao product is the Hadamard product of the Grams),
// O(R^3) work in the chol kernel instead of a pass over V.  Every sum runs in
// a fixed order over a split of the rows that depends only on the row count,
// so kind 4 on the A_n that kind 3 wrote repeats its Gram and QR bit for bit.
// The substitutions use explicit triangular inverses, so each row's products
// are independent FMAs over the whole GPU; the a-posteriori check and the
// second pass are those of the cluster kernel.  The gate word is set by the
// chol kernel (0 accepted so far, 1 refused) and the later kernels return at
// once when it is 1.
constexpr int kWideThreads = 256;
constexpr int kWideChunk = 32;     // rows staged in shared memory at a time
constexpr int kWideGroups = 8;     // fixed groups of row blocks in the reduction
constexpr int kWideMaxE = (kMaxRank * (kMaxRank + 1) / 2 + kWideThreads - 1) / kWideThreads;

// Row blocks of the split: about 8 rows each, at most two per SM.
int wide_blocks(int64_t rows, int num_sms)
{
    return (int)std::max<int64_t>(1, std::min<int64_t>((rows + 7) / 8, 2LL * num_sms));
}

__device__ __forceinline__ bool wide_skip(const int* status, const int* gate)
{
    if (*(volatile const int*)status != kStatusOk) return true;
    return gate != nullptr && *(volatile const int*)gate != 0;
}

// cparts[b][e] = sum over block b's rows of X(r, e)^2 (a warp per column,
// lanes over rows, a fixed shuffle tree).
__global__ void __launch_bounds__(kWideThreads) wide_colsq_kernel(const double* __restrict__ X, int64_t I, int R,
                                                                  int nblk, double* __restrict__ cparts,
                                                                  const int* __restrict__ status)
{
    if (wide_skip(status, nullptr)) return;
    const int b = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t r0 = (int64_t)b * I / nblk, r1 = (int64_t)(b + 1) * I / nblk;
    for (int e = warp; e < R; e += kWideThreads / 32) {
        double s = 0.0;
        for (int64_t r = r0 + lane; r < r1; r += 32) {
            const double v = X[r + I * e];
            s = fma(v, v, s);
        }
        s = warp_sum(s);
        if (lane == 0) cparts[(size_t)b * R + e] = s;
    }
}

// lambda_r = sqrt(sum over the blocks of cparts[b][r]): the blocks in
// kWideThreads / R contiguous groups, then the groups in order.
__global__ void __launch_bounds__(kWideThreads) wide_lambda_kernel(const double* __restrict__ cparts, int nblk, int R,
                                                                   double* __restrict__ lambda_out,
                                                                   double* __restrict__ lam,
                                                                   const int* __restrict__ status)
{
    if (wide_skip(status, nullptr)) return;
    __shared__ double red[kWideThreads];
    const int tid = threadIdx.x, groups = kWideThreads / R, q = tid / R, e = tid - q * R;
    double s = 0.0;
    if (q < groups)
        for (int b = q * nblk / groups; b < (q + 1) * nblk / groups; ++b) s += cparts[(size_t)b * R + e];
    red[tid] = s;
    __syncthreads();
    if (tid < R) {
        double t = red[tid];
        for (int g = 1; g < groups; ++g) t += red[g * R + tid];
        const double l = sqrt(t);
        lam[tid] = l;
        if (lambda_out) lambda_out[tid] = l;
    }
}

// The row-block kernel.  Block b takes rows [b I / nblk, (b+1) I / nblk) in
// chunks of kWideChunk rows staged in shared memory (row-major, ld R + 1):
//   NORM:  a = x / lambda (lambda > 0; else a = x), written to out;
//   APPLY: a = x X for the upper-triangular X (R x R), written to out (out
//          may alias src: a block reads a chunk whole before writing it);
//   GRAM:  parts[b][e] = sum over the rows of a(r, i) a(r, j) for the upper
//          triangle entry e = (i, j), accumulated in registers over the chunks.
//   RPROD: besides, R_n = R2 R1 (both upper triangular): a warp per entry
//          (a, c), a <= c, lanes over k = a..c and a fixed shuffle tree, the
//          entries spread over the blocks' warps; the strict lower triangle
//          of Rout set to zero.
template <bool NORM, bool APPLY, bool GRAM, bool RPROD>
__global__ void __launch_bounds__(kWideThreads) wide_rows_kernel(const double* src, int64_t I, int R, int nblk,
                                                                 const double* __restrict__ lam,
                                                                 const double* __restrict__ Xg, double* out,
                                                                 double* __restrict__ parts,
                                                                 const double* __restrict__ R2g,
                                                                 const double* __restrict__ R1g,
                                                                 double* __restrict__ Rout,
                                                                 const int* __restrict__ gate,
                                                                 const int* __restrict__ status)
{
    if (wide_skip(status, gate)) return;
    if (RPROD) {
        const int lane = threadIdx.x & 31, wpb = kWideThreads / 32;
        for (int e = blockIdx.x * wpb + (threadIdx.x >> 5); e < R * (R + 1) / 2; e += nblk * wpb) {
            int a, c;
            tri_index(e, a, c);
            double s = 0.0;
            for (int k = a + lane; k <= c; k += 32) s = fma(R2g[a + R * k], R1g[k + R * c], s);
            s = warp_sum(s);
            if (lane == 0) Rout[a + R * c] = s;
        }
        for (int p = blockIdx.x * kWideThreads + threadIdx.x; p < R * R; p += nblk * kWideThreads)
            if (p % R > p / R) Rout[p] = 0.0;
    }
    extern __shared__ double wsm[];
    const int ld = R + 1, tid = threadIdx.x, nE = R * (R + 1) / 2;
    double* Xs = wsm;                                   // APPLY: X row-major, X(k, c) at Xs[k R + c]
    double* st = wsm + (APPLY ? R * R : 0);             // the staged input rows
    double* ot = st + kWideChunk * ld;                  // APPLY: the product rows
    const int b = blockIdx.x;
    const int64_t r0 = (int64_t)b * I / nblk, r1 = (int64_t)(b + 1) * I / nblk;
    if (APPLY)
        for (int p = tid; p < R * R; p += kWideThreads) {
            const int k = p / R, c = p - k * R;
            Xs[p] = Xg[k + R * c];
        }
    double acc[kWideMaxE];
    int ea[kWideMaxE], eb[kWideMaxE];
    if (GRAM) {
#pragma unroll
        for (int j = 0; j < kWideMaxE; ++j) {
            acc[j] = 0.0;
            ea[j] = eb[j] = 0;
            const int e = tid + j * kWideThreads;
            if (e < nE) tri_index(e, ea[j], eb[j]);
        }
    }
    for (int64_t c0 = r0; c0 < r1; c0 += kWideChunk) {
        const int rl = (int)(r1 - c0 < kWideChunk ? r1 - c0 : kWideChunk);
        __syncthreads();                                // the previous chunk is read
        for (int p = tid; p < rl * R; p += kWideThreads) {
            const int e = p / rl, li = p - e * rl;
            double v = src[(c0 + li) + I * e];
            if (NORM) {
                const double l = lam[e];
                v = (l > 0.0) ? v / l : v;
                out[(c0 + li) + I * e] = v;
            }
            st[li * ld + e] = v;
        }
        __syncthreads();
        const double* gs = st;
        if (APPLY) {
            for (int p = tid; p < rl * R; p += kWideThreads) {
                const int c = p / rl, li = p - c * rl;
                const double* a = st + li * ld;
                double s = 0.0;
                for (int k = 0; k <= c; ++k) s = fma(a[k], Xs[k * R + c], s);
                ot[li * ld + c] = s;
                out[(c0 + li) + I * c] = s;
            }
            __syncthreads();
            gs = ot;
        }
        if (GRAM) {
#pragma unroll
            for (int j = 0; j < kWideMaxE; ++j) {
                if (tid + j * kWideThreads < nE) {
                    const int ia = ea[j], ib = eb[j];
                    double s = acc[j];
                    for (int li = 0; li < rl; ++li) s = fma(gs[li * ld + ia], gs[li * ld + ib], s);
                    acc[j] = s;
                }
            }
        }
    }
    if (GRAM) {
#pragma unroll
        for (int j = 0; j < kWideMaxE; ++j) {
            const int e = tid + j * kWideThreads;
            if (e < nE) parts[(size_t)b * nE + e] = acc[j];
        }
    }
}

// gparts[g][e] = sum of parts[b][e] over the g-th of kWideGroups contiguous
// ranges of blocks, in block order.
__global__ void __launch_bounds__(kWideThreads) wide_reduce_kernel(const double* __restrict__ parts, int nblk, int nE,
                                                                   double* __restrict__ gparts,
                                                                   const int* __restrict__ gate,
                                                                   const int* __restrict__ status)
{
    if (wide_skip(status, gate)) return;
    const int e = blockIdx.x * kWideThreads + threadIdx.x, g = blockIdx.y;
    if (e >= nE) return;
    double s = 0.0;
    for (int b = g * nblk / kWideGroups; b < (g + 1) * nblk / kWideGroups; ++b) s += parts[(size_t)b * nE + e];
    gparts[(size_t)g * nE + e] = s;
}

// M (R x R, full symmetric) = the sum of the kWideGroups group partials, in order.
__device__ void wide_group_sum(const double* gparts, int R, double* M)
{
    const int nE = R * (R + 1) / 2;
    for (int e = threadIdx.x; e < nE; e += kTailThreads) {
        double s = 0.0;
        for (int g = 0; g < kWideGroups; ++g) s += gparts[(size_t)g * nE + e];
        int a, b;
        tri_index(e, a, b);
        M[a + R * b] = s;
        M[b + R * a] = s;
    }
}

// X = U^-1 for the upper-triangular U (U(a, b) = U[a + R b]) given dinv[k] =
// 1 / U(k, k) (the Cholesky's), one warp per column c of X, the rows split
// over the lanes (k = lane, lane + 32).  U X = I gives, from the bottom row up,
//   X(i, c) = delta_ic / U(i, i) - (sum_{k > i} U(i, k) X(k, c)) / U(i, i)
// (one FMA),
// and once X(i, c) is known (its lane broadcasts it) every lane adds
// U(k, i) X(i, c) to its rows k < i: a fixed order, no block barrier.  U goes
// through shared memory; the strict lower triangle of X is zero.
constexpr int kInvWarps = 4;

__global__ void __launch_bounds__(kInvWarps * 32) wide_inv_kernel(const double* __restrict__ U,
                                                                  const double* __restrict__ dinv, int R,
                                                                  double* __restrict__ X,
                                                                  const int* __restrict__ gate,
                                                                  const int* __restrict__ status)
{
    if (wide_skip(status, gate)) return;
    __shared__ double Us[kMaxRank * kMaxRank];
    __shared__ double ds[kMaxRank];
    for (int p = threadIdx.x; p < R * R; p += kInvWarps * 32) Us[p] = U[p];
    for (int p = threadIdx.x; p < R; p += kInvWarps * 32) ds[p] = dinv[p];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int c = blockIdx.x * kInvWarps + (threadIdx.x >> 5);
    if (c >= R) return;
    const int k0 = lane, k1 = lane + 32;
    double acc0 = 0.0, acc1 = 0.0, x0 = 0.0, x1 = 0.0;
    for (int i = c; i >= 0; --i) {
        double xi = 0.0;
        const double dd = (i == c) ? ds[i] : 0.0;     // delta_ic / U(i, i)
        if (i == k0) { xi = fma(-acc0, ds[i], dd); x0 = xi; }
        if (i == k1) { xi = fma(-acc1, ds[i], dd); x1 = xi; }
        xi = __shfl_sync(0xffffffffu, xi, i & 31);
        if (k0 < i) acc0 = fma(Us[k0 + R * i], xi, acc0);
        if (k1 < i) acc1 = fma(Us[k1 + R * i], xi, acc1);
    }
    if (k0 < R) X[k0 + R * c] = (k0 <= c) ? x0 : 0.0;
    if (k1 < R) X[k1 + R * c] = (k1 <= c) ? x1 : 0.0;
}

// The Gram of a fold step V = F (.) B with F, B upper triangular: G = (F^T F)
// * (B^T B) entrywise, (F^T F)(a, b) = sum_{p <= a} F(p, a) F(p, b) for a <= b.
// A warp per upper-triangle entry (lanes over p, a fixed shuffle tree), G
// written whole (R x R).
__global__ void __launch_bounds__(kWideThreads) wide_hadamard_kernel(const double* __restrict__ F,
                                                                     const double* __restrict__ B, int R,
                                                                     double* __restrict__ G,
                                                                     const int* __restrict__ status)
{
    if (wide_skip(status, nullptr)) return;
    const int lane = threadIdx.x & 31;
    const int e = blockIdx.x * (kWideThreads / 32) + (threadIdx.x >> 5);
    if (e >= R * (R + 1) / 2) return;
    int a, b;
    tri_index(e, a, b);
    double sf = 0.0, sb = 0.0;
    for (int p = lane; p <= a; p += 32) {
        sf = fma(F[p + R * a], F[p + R * b], sf);
        sb = fma(B[p + R * a], B[p + R * b], sb);
    }
    sf = warp_sum(sf);
    sb = warp_sum(sb);
    if (lane == 0) {
        const double v = sf * sb;
        G[a + R * b] = v;
        G[b + R * a] = v;
    }
}

// One CTA: the first Gram (the group sums, or Gin given whole), written to
// Gout; with want_qr R1 = chol(Gram) to R1g, the reciprocals of its diagonal
// to D1g, and the gate word (1 when the Cholesky breaks down).
__global__ void __launch_bounds__(kTailThreads, 1) wide_chol_kernel(const double* __restrict__ gparts,
                                                                    const double* __restrict__ Gin, int R,
                                                                    double* __restrict__ Gout, int want_qr,
                                                                    double* __restrict__ R1g,
                                                                    double* __restrict__ D1g, int* __restrict__ gate,
                                                                    const int* __restrict__ status)
{
    if (wide_skip(status, nullptr)) return;
    extern __shared__ double wsm[];
    __shared__ double piv[2 * kMaxRank], dinv[kMaxRank];
    __shared__ int flag_bad;
    double* M = wsm;
    const int tid = threadIdx.x;
    if (Gin != nullptr) {
        for (int p = tid; p < R * R; p += kTailThreads) M[p] = Gin[p];
    } else {
        wide_group_sum(gparts, R, M);
    }
    __syncthreads();
    if (Gout)
        for (int p = tid; p < R * R; p += kTailThreads) Gout[p] = M[p];
    if (!want_qr) return;
    const bool ok = block_cholesky(M, R, piv, dinv, &flag_bad);
    for (int p = tid; p < R * R; p += kTailThreads) R1g[p] = M[p];
    if (tid < R) D1g[tid] = dinv[tid];
    if (tid == 0) *gate = ok ? 0 : 1;
}

// One CTA: Q1^T Q1 from the group sums; if every entry is within kCqrCheck of
// the identity and its Cholesky succeeds, R2 to R2g and the reciprocals of
// its diagonal to D2g; else the gate word goes to 1.
__global__ void __launch_bounds__(kTailThreads, 1) wide_chol2_kernel(const double* __restrict__ gparts, int R,
                                                                     double* __restrict__ R2g,
                                                                     double* __restrict__ D2g,
                                                                     int* __restrict__ gate,
                                                                     const int* __restrict__ status)
{
    if (wide_skip(status, gate)) return;
    extern __shared__ double wsm[];
    __shared__ double piv[2 * kMaxRank], dinv[kMaxRank];
    __shared__ int flag_bad, flag_check;
    double* M = wsm;
    const int tid = threadIdx.x;
    wide_group_sum(gparts, R, M);
    if (tid == 0) flag_check = 0;
    __syncthreads();
    for (int p = tid; p < R * R; p += kTailThreads) {
        const int a = p % R, b = p / R;
        if (!(fabs(M[p] - (a == b ? 1.0 : 0.0)) <= kCqrCheck)) flag_check = 1;
    }
    __syncthreads();
    bool ok = flag_check == 0;
    if (ok) ok = block_cholesky(M, R, piv, dinv, &flag_bad);
    if (!ok) {
        if (tid == 0) *gate = 1;
        return;
    }
    for (int p = tid; p < R * R; p += kTailThreads) R2g[p] = M[p];
    if (tid < R) D2g[tid] = dinv[tid];
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

bool wide_tail_on(const Handle* h) { return h->wide_tail && h->R > 32 && h->wide[0].base != nullptr; }

int64_t wide_ws_elems(int R, int num_sms)
{
    const int64_t nE = (int64_t)R * (R + 1) / 2, nb = 2LL * num_sms;
    return nb * nE + kWideGroups * nE + nb * R + 3LL * R + 5LL * R * R;
}

void wide_ws_carve(WideWs& ws, int R, int num_sms)
{
    const int64_t nE = (int64_t)R * (R + 1) / 2, nb = 2LL * num_sms;
    double* p = ws.base;
    ws.parts = p; p += nb * nE;
    ws.gparts = p; p += kWideGroups * nE;
    ws.cparts = p; p += nb * R;
    ws.lam = p; p += R;
    ws.R1 = p; p += (int64_t)R * R;
    ws.X1 = p; p += (int64_t)R * R;
    ws.X2 = p; p += (int64_t)R * R;
    ws.R2 = p; p += (int64_t)R * R;
    ws.Gh = p; p += (int64_t)R * R;
    ws.D1 = p; p += R;
    ws.D2 = p;
}

namespace {

// The GPU-wide chain on h->stream (see the kernels above).  src: I x R;
// norm: kind 3 (lambda to lambda_out, A_n to Aout); F, B: a fold step's
// triangular factors (first Gram from them, src = F (.) B).
cudaError_t wide_cqr2(Handle* h, WideWs& ws, const double* src, int64_t I, bool norm, double* lambda_out,
                      double* Aout, double* G, bool want_qr, double* Q, double* Rout, int* gate, const double* F,
                      const double* B)
{
    const int R = h->R, nE = R * (R + 1) / 2;
    if (R > kMaxRank || I < 1) return cudaErrorInvalidValue;
    const int nblk = wide_blocks(I, h->num_sms);
    const size_t st_bytes = (size_t)kWideChunk * (R + 1) * sizeof(double);
    const size_t apply_bytes = (size_t)R * R * sizeof(double) + 2 * st_bytes;
    const size_t chol_bytes = (size_t)R * R * sizeof(double);
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [] {
        const int mx = (int)(kMaxRank * kMaxRank * sizeof(double) + 2 * kWideChunk * (kMaxRank + 1) * sizeof(double));
        attr_err = cudaFuncSetAttribute(wide_rows_kernel<false, true, true, false>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
        if (attr_err == cudaSuccess)
            attr_err = cudaFuncSetAttribute(wide_rows_kernel<false, true, false, true>,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    });
    CPALS_CUDA_TRY(attr_err);
    cudaStream_t st = h->stream;
    const dim3 rgrid((unsigned)((nE + kWideThreads - 1) / kWideThreads), kWideGroups);
    const double* qsrc = src;
    const double* Gin = nullptr;
    if (F != nullptr) {
        const int wpb = kWideThreads / 32;
        wide_hadamard_kernel<<<(nE + wpb - 1) / wpb, kWideThreads, 0, st>>>(F, B, R, ws.Gh, h->d_status);
        h->launches++;
        Gin = ws.Gh;
    } else {
        if (norm) {
            wide_colsq_kernel<<<nblk, kWideThreads, 0, st>>>(src, I, R, nblk, ws.cparts, h->d_status);
            wide_lambda_kernel<<<1, kWideThreads, 0, st>>>(ws.cparts, nblk, R, lambda_out, ws.lam, h->d_status);
            wide_rows_kernel<true, false, true, false><<<nblk, kWideThreads, st_bytes, st>>>(
                src, I, R, nblk, ws.lam, nullptr, Aout, ws.parts, nullptr, nullptr, nullptr, nullptr, h->d_status);
            h->launches += 3;
            qsrc = Aout;
        } else {
            wide_rows_kernel<false, false, true, false><<<nblk, kWideThreads, st_bytes, st>>>(
                src, I, R, nblk, nullptr, nullptr, nullptr, ws.parts, nullptr, nullptr, nullptr, nullptr,
                h->d_status);
            h->launches++;
        }
        wide_reduce_kernel<<<rgrid, kWideThreads, 0, st>>>(ws.parts, nblk, nE, ws.gparts, nullptr, h->d_status);
        h->launches++;
    }
    const unsigned igrid = (unsigned)((R + kInvWarps - 1) / kInvWarps);
    wide_chol_kernel<<<1, kTailThreads, chol_bytes, st>>>(ws.gparts, Gin, R, G, want_qr ? 1 : 0, ws.R1, ws.D1, gate,
                                                          h->d_status);
    h->launches++;
    if (!want_qr) return cudaGetLastError();
    wide_inv_kernel<<<igrid, kInvWarps * 32, 0, st>>>(ws.R1, ws.D1, R, ws.X1, gate, h->d_status);
    wide_rows_kernel<false, true, true, false><<<nblk, kWideThreads, apply_bytes, st>>>(
        qsrc, I, R, nblk, nullptr, ws.X1, Q, ws.parts, nullptr, nullptr, nullptr, gate, h->d_status);
    wide_reduce_kernel<<<rgrid, kWideThreads, 0, st>>>(ws.parts, nblk, nE, ws.gparts, gate, h->d_status);
    wide_chol2_kernel<<<1, kTailThreads, chol_bytes, st>>>(ws.gparts, R, ws.R2, ws.D2, gate, h->d_status);
    wide_inv_kernel<<<igrid, kInvWarps * 32, 0, st>>>(ws.R2, ws.D2, R, ws.X2, gate, h->d_status);
    wide_rows_kernel<false, true, false, true><<<nblk, kWideThreads, apply_bytes, st>>>(
        Q, I, R, nblk, nullptr, ws.X2, Q, nullptr, ws.R2, ws.R1, Rout, gate, h->d_status);
    h->launches += 6;
    return cudaGetLastError();
}

}  // namespace

cudaError_t mode_tail(Handle* h, int n, int kind, const double* W, const double* Op, bool want_qr)
{
    if (kind >= 3 && wide_tail_on(h))
        return wide_cqr2(h, h->wide[0], W, h->dims[n], kind == 3, h->lambda, h->A[n], h->G[n], want_qr, h->Q[n],
                         h->Rf[n], h->d_gate, nullptr, nullptr);
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

cudaError_t cqr2_rows(Handle* h, const double* V, int64_t rows, double* Q, double* Rout, double* G, int* gate,
                      const double* F, const double* B)
{
    if (wide_tail_on(h))
        return wide_cqr2(h, h->wide[1], V, rows, false, nullptr, nullptr, G, true, Q, Rout, gate, F, B);
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
