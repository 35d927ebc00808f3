// dev_common.cuh -- device helpers shared by the FP64 linear-algebra
// translation units (linalg.cu, tail.cu, batch.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace cpals {
namespace {

constexpr double kEps = 2.220446049250313e-16;   // FP64 machine epsilon, 2^-52

// 1/d and 1/sqrt(d) to about one ulp from the hardware approximations.  The
// reciprocal starts from rcp.approx.ftz.f64 and takes one third-order step of
// the Newton iteration for 1/d: with e = 1 - d y, y (1 + e + e^2) =
// (1 - e^3) / d, so the relative error goes from e to e^3 in three dependent
// FMAs (the accuracy test checks the result within 2 ulp over 40 decades).
// The reciprocal square root starts from the FP32 rsqrt.approx (about 2^-23)
// and takes two Newton-Raphson steps, y <- y + y (1/2 - (d/2) y^2), each
// squaring the error.  A dependent FP64 operation costs 64 cycles on this part, and these
// are a few of them against the much longer exact division and square root.
// Outside the FP32 normal range the exact FP64 operations are used.
__device__ __forceinline__ double rcp_nr(double d)
{
    const double a = fabs(d);
    if (!(a > 1e-36 && a < 1e36)) return 1.0 / d;
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(d));
    const double e = fma(-d, y, 1.0);
    return fma(y, fma(e, e, e), y);
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

__device__ __forceinline__ double warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// One substitution on the warp-distributed row w (slots w0, w1):
//   back = false: L y = w with L(e, k) = A[e + R k] (lower), from k = 0 up;
//   back = true:  U x = w with U(e, k) = A[e + R k] (upper), from k = R-1 down;
//   trans:        the matrix is read transposed (A[k + R e]), so an upper
//                 triangle serves as L (back = false) and a lower one as U.
// d0, d1 are the lanes' reciprocals of the diagonal.
__device__ __forceinline__ void warp_subst(double& w0, double& w1, const double* A, int R, double d0, double d1,
                                           bool back, bool trans)
{
    const int lane = threadIdx.x & 31;
    for (int t = 0; t < R; ++t) {
        const int k = back ? R - 1 - t : t;
        double xk;
        if (k < 32) {
            if (lane == k) w0 *= d0;
            xk = __shfl_sync(0xffffffffu, w0, k);
        } else {
            if (lane == k - 32) w1 *= d1;
            xk = __shfl_sync(0xffffffffu, w1, k - 32);
        }
        const int e0 = lane, e1 = lane + 32;
        if (e0 < R && (back ? e0 < k : e0 > k)) w0 = fma(-(trans ? A[k + R * e0] : A[e0 + R * k]), xk, w0);
        if (R > 32 && e1 < R && (back ? e1 < k : e1 > k))
            w1 = fma(-(trans ? A[k + R * e1] : A[e1 + R * k]), xk, w1);
    }
}

// ---------------------------------------------------------------- staircase QR of F (.) G
// Thin QR of the Khatri-Rao product F (.) G of two upper-triangular n x n
// factors (one step of the QR of V_n, Sec. 3.1 and Eq. kr-id), without
// forming the n^2 x n product densely.  Row (i, j) (index i n + j, the right
// factor's row fastest) is zero left of column max(i, j) (Sec. 3.3.3: the
// columns of a Khatri-Rao product of triangular factors are sparse).  Ordered
// by that level c = max(i, j) -- level c holds the 2c + 1 rows (c, 0..c),
// (0..c-1, c) at positions c^2 .. (c+1)^2 - 1 -- the matrix is a staircase:
// the Householder reflector of column j spans only positions j .. (j+1)^2 - 1,
// and neither the reflectors nor the explicit Q fill in outside positions
// < (k+1)^2 of column k.  Column k is stored compactly ((k+1)^2 values), and
// the QR costs about n^4 / 3 flops instead of 4 n^4.  Householder reflectors
// in LAPACK's dlarfg form with diag(R) >= 0 (row of R and column of Q
// flipped together); the thin QR with a positive diagonal is unique, so this
// is the factorisation a dense Householder QR gives, up to rounding.
__device__ __forceinline__ int stair_pos(int i, int j)
{
    const int c = i > j ? i : j;
    return c * c + (i == c ? j : c + 1 + i);
}

__device__ __forceinline__ int stair_off(int k) { return k * (k + 1) * (2 * k + 1) / 6; }

// Block-wide (any block size that is a multiple of 32).  Work space: W and Qs
// of stair_off(n) doubles each, tau (n), red (32), rowi and rowj (n^2 ints).
// Writes the explicit Q (n^2 x n, column-major, rows in the Khatri-Rao order
// i n + j) to Qout and R (n x n) to Rout; both may be shared or global memory.
__device__ void stair_qr_block(const double* __restrict__ F, const double* __restrict__ G, int n, double* W,
                               double* Qs, double* tau, double* red, int* rowi, int* rowj, double* Qout,
                               double* Rout)
{
    const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarps = nthr >> 5;
    for (int p = tid; p < n * n; p += nthr) {
        const int c = (int)sqrtf((float)p + 0.5f);   // level: c^2 <= p < (c+1)^2
        const int cc = (c * c > p) ? c - 1 : ((c + 1) * (c + 1) <= p ? c + 1 : c);
        const int q = p - cc * cc;
        rowi[p] = (q <= cc) ? cc : q - cc - 1;
        rowj[p] = (q <= cc) ? q : cc;
    }
    __syncthreads();
    for (int k = 0; k < n; ++k)
        for (int p = tid; p < (k + 1) * (k + 1); p += nthr)
            W[stair_off(k) + p] = F[rowi[p] + n * k] * G[rowj[p] + n * k];
    __syncthreads();
    for (int j = 0; j < n; ++j) {
        const int end = (j + 1) * (j + 1);
        double* wj = W + stair_off(j);
        if (warp == 0) {
            double s = 0.0;
            for (int p = j + 1 + lane; p < end; p += 32) s = fma(wj[p], wj[p], s);
            s = warp_sum(s);
            if (lane == 0) {
                const double alpha = wj[j];
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
                wj[j] = beta;
            }
        }
        __syncthreads();
        const double tj = tau[j];
        if (tj != 0.0) {
            const double scale = red[0];
            for (int p = j + 1 + tid; p < end; p += nthr) wj[p] *= scale;
        }
        __syncthreads();
        if (tj != 0.0) {
            for (int k = j + 1 + warp; k < n; k += nwarps) {
                double* wk = W + stair_off(k);
                double s = 0.0;
                for (int p = j + lane; p < end; p += 32) s = fma(p == j ? 1.0 : wj[p], wk[p], s);
                s = warp_sum(s) * tj;
                for (int p = j + lane; p < end; p += 32) wk[p] = fma(-s, p == j ? 1.0 : wj[p], wk[p]);
            }
        }
        __syncthreads();
    }
    // explicit Q = H_0 ... H_{n-1} [I; 0] (sorted rows), backward accumulation
    for (int k = 0; k < n; ++k)
        for (int p = tid; p < (k + 1) * (k + 1); p += nthr) Qs[stair_off(k) + p] = (p == k) ? 1.0 : 0.0;
    __syncthreads();
    for (int j = n - 1; j >= 0; --j) {
        const double tj = tau[j];
        if (tj != 0.0) {
            const int end = (j + 1) * (j + 1);
            const double* wj = W + stair_off(j);
            for (int k = j + warp; k < n; k += nwarps) {
                double* qk = Qs + stair_off(k);
                double s = 0.0;
                for (int p = j + lane; p < end; p += 32) s = fma(p == j ? 1.0 : wj[p], qk[p], s);
                s = warp_sum(s) * tj;
                for (int p = j + lane; p < end; p += 32) qk[p] = fma(-s, p == j ? 1.0 : wj[p], qk[p]);
            }
        }
        __syncthreads();
    }
    // sign convention diag(R) >= 0; rows back to the Khatri-Rao order i n + j
    for (int e = tid; e < n * n * n; e += nthr) {
        const int k = e / (n * n), rho = e - k * n * n;
        const int i = rho / n, jj = rho - i * n;
        const int p = stair_pos(i, jj);
        const double sgn = (W[stair_off(k) + k] < 0.0) ? -1.0 : 1.0;
        Qout[rho + (int64_t)n * n * k] = (p < (k + 1) * (k + 1)) ? sgn * Qs[stair_off(k) + p] : 0.0;
    }
    for (int e = tid; e < n * n; e += nthr) {
        const int k = e / n, i = e - k * n;       // R(i, k)
        double v = 0.0;
        if (i <= k) v = ((W[stair_off(i) + i] < 0.0) ? -1.0 : 1.0) * W[stair_off(k) + i];
        Rout[i + n * k] = v;
    }
    __syncthreads();
}

}  // namespace
}  // namespace cpals
