// dev_common.cuh -- device helpers shared by the FP64 linear-algebra
// translation units (linalg.cu, tail.cu).
#pragma once

#include <cuda_runtime.h>

namespace cpals {
namespace {

constexpr double kEps = 2.220446049250313e-16;   // FP64 machine epsilon, 2^-52

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

}  // namespace
}  // namespace cpals
