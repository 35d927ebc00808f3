// batch.cu -- many independent 3-way CP-ALS-QR problems of uneven dims and
// ranks advancing together: one persistent kernel per mode update (the body of
// the mode loop of Alg. cp-als-qr) in which each CTA takes whole problems from
// a largest-first list and runs, on chip:
//   1. V_n = R_hi (.) R_lo (the two other R factors, Sec. 3.1) and its Householder
//      QR V_n = Q0 R0 (FP64, shared memory);
//   2. the Multi-TTM Y = X x_{m != n} Q_m^T (Eq. multittm) as two single TTMs,
//      larger dim first (Sec. 3.2), in FP32 through an L2-resident per-problem
//      scratch;
//   3. W_n = Y_(n) Q0 (Eq. ls-qr-q0-step), FP64;
//   4. the substitution Ahat R0^T = W (singular R0 -> per-problem status, factor
//      kept);
//   5. column normalisation (2-norm) into A_n and lambda;
//   6. the Householder QR A_n = Q_n R_n (FP64, shared memory);
//   7. after the last mode, the efficient fit of Sec. 3.3.1.
// The sweep (three launches) is captured once into a CUDA graph.  The CTA
// count (per SM) and the CTA size are picked by timing the first sweep.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

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
    int64_t t1;       // first-TTM intermediate (floats)
    int64_t y;        // Multi-TTM result (floats)
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

// One CTA: Out(l, r, t) = sum_k In(l, k, t) * qs[k*R + r] over the [L, K, T] view.
// Loads are issued eight k at a time so that each thread keeps eight in flight.
__device__ void cta_ttm_f32(const float* __restrict__ in, int64_t L, int K, int64_t T, const float* qs, int R,
                            float* __restrict__ out)
{
    const int64_t rows = L * T;
    for (int64_t f = threadIdx.x; f < rows; f += blockDim.x) {
        const int64_t t = f / L, l = f - t * L;
        const float* p = in + l + L * K * t;
        float acc[kBMaxR];
#pragma unroll
        for (int r = 0; r < kBMaxR; ++r) acc[r] = 0.0f;
        int k = 0;
        for (; k + 8 <= K; k += 8) {
            float x[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) x[u] = __ldg(p + L * (k + u));
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const float* q = qs + (k + u) * R;
#pragma unroll
                for (int r = 0; r < kBMaxR; ++r)
                    if (r < R) acc[r] = fmaf(x[u], q[r], acc[r]);
            }
        }
        for (; k < K; ++k) {
            const float x = __ldg(p + L * k);
            const float* q = qs + k * R;
#pragma unroll
            for (int r = 0; r < kBMaxR; ++r)
                if (r < R) acc[r] = fmaf(x, q[r], acc[r]);
        }
        float* o = out + l + L * (int64_t)R * t;
#pragma unroll
        for (int r = 0; r < kBMaxR; ++r)
            if (r < R) o[L * r] = acc[r];
    }
}

// stage Q_m (FP64, I x R column-major) as FP32 [k][r]
__device__ void stage_q(const double* __restrict__ Qm, int I, int R, float* qs)
{
    for (int e = threadIdx.x; e < I * R; e += blockDim.x) {
        const int k = e / R, r = e - k * R;
        qs[e] = (float)Qm[k + I * r];
    }
    __syncthreads();
}

struct BSmem {
    int64_t regA, regB, r0, rn, w, qst;   // offsets in doubles
    int64_t total;
};

__host__ __device__ inline BSmem bsmem_layout(int maxR, int maxI)
{
    BSmem s;
    const int64_t sa = std::max<int64_t>((int64_t)maxR * maxR * maxR, (int64_t)maxI * maxR);
    s.regA = 0;
    s.regB = s.regA + sa;
    s.r0 = s.regB + sa;
    s.rn = s.r0 + (int64_t)maxR * maxR;
    s.w = s.rn + (int64_t)maxR * maxR;
    s.qst = s.w + (int64_t)maxI * maxR;
    s.total = s.qst + ((int64_t)maxI * maxR + 1) / 2 + 128;   // FP32 staging, tau/red
    return s;
}

__global__ void batch_mode_kernel(BProb* __restrict__ probs, const int* __restrict__ order, int count, int n,
                                  int maxR, int maxI, const float* __restrict__ Xall, double* __restrict__ F,
                                  float* __restrict__ T1all, float* __restrict__ Yall, int* __restrict__ pstatus,
                                  double* __restrict__ fit_last)
{
    extern __shared__ double bsm[];
    const BSmem L = bsmem_layout(maxR, maxI);
    double* regA = bsm + L.regA;
    double* regB = bsm + L.regB;
    double* R0s = bsm + L.r0;
    double* Rns = bsm + L.rn;
    double* Ws = bsm + L.w;
    float* qst = reinterpret_cast<float*>(bsm + L.qst);
    double* tau = bsm + L.total - 128;
    double* red = tau + 64;
    __shared__ int singular;
    __shared__ double inner_sh;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;

    for (int idx = blockIdx.x; idx < count; idx += gridDim.x) {
        const int p = order[idx];
        BProb pr = probs[p];
        if (pstatus[p] != kStatusOk) continue;       // a failed problem stays as it was
        const int R = pr.R, In = pr.I[n];
        int mo[2], cnt = 0;
        for (int m = 0; m < 3; ++m)
            if (m != n) mo[cnt++] = m;
        const int lo = mo[0], hi = mo[1];            // V_n = R_hi (.) R_lo
        // ---- 1. V_n and its QR (FP64, shared memory)
        const double* Rhi = F + pr.rf[hi];
        const double* Rlo = F + pr.rf[lo];
        const int RR = R * R;
        for (int e = tid; e < RR * R; e += blockDim.x) {
            const int c = e / RR, row = e - c * RR;
            const int i = row / R, j = row - i * R;
            regA[e] = Rhi[i + R * c] * Rlo[j + R * c];
        }
        __syncthreads();
        cta_householder(regA, RR, R, regB, R0s, tau, red);   // Q0 in regB (R^2 x R), R0 in R0s
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
        // ---- 2. Multi-TTM: larger contracted dim first (ties: higher mode)
        int c1 = (pr.I[hi] >= pr.I[lo]) ? hi : lo;
        int c2 = (c1 == hi) ? lo : hi;
        int64_t d[3] = {pr.I[0], pr.I[1], pr.I[2]};
        {
            stage_q(F + pr.q[c1], pr.I[c1], R, qst);
            int64_t Lw = 1, Tw = 1;
            for (int m = 0; m < c1; ++m) Lw *= d[m];
            for (int m = c1 + 1; m < 3; ++m) Tw *= d[m];
            cta_ttm_f32(Xall + pr.x, Lw, (int)d[c1], Tw, qst, R, T1all + pr.t1);
            d[c1] = R;
            __syncthreads();
        }
        {
            stage_q(F + pr.q[c2], pr.I[c2], R, qst);
            int64_t Lw = 1, Tw = 1;
            for (int m = 0; m < c2; ++m) Lw *= d[m];
            for (int m = c2 + 1; m < 3; ++m) Tw *= d[m];
            cta_ttm_f32(T1all + pr.t1, Lw, (int)d[c2], Tw, qst, R, Yall + pr.y);
            d[c2] = R;
            __syncthreads();
        }
        // ---- 3. W = Y_(n) Q0 (FP64); Y element (col, i) at a + Rn*(i + In*c), col = a + Rn*c
        // one thread per row i with all R accumulators; Q0 rows are shared-memory broadcasts
        const float* Y = Yall + pr.y;
        const int Rn = (n == 0) ? 1 : (n == 1 ? R : RR);
        for (int i = tid; i < In; i += blockDim.x) {
            double acc[kBMaxR];
#pragma unroll
            for (int r = 0; r < kBMaxR; ++r) acc[r] = 0.0;
            for (int c0 = 0; c0 < RR; c0 += 8) {
                float y[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int col = c0 + u;
                    const int a = col % Rn, c = col / Rn;
                    y[u] = (col < RR) ? __ldg(Y + a + (int64_t)Rn * (i + (int64_t)In * c)) : 0.0f;
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int col = c0 + u;
                    if (col < RR) {
#pragma unroll
                        for (int r = 0; r < kBMaxR; ++r)
                            if (r < R) acc[r] = fma((double)y[u], regB[col + RR * r], acc[r]);
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < kBMaxR; ++r)
                if (r < R) Ws[i + In * r] = acc[r];
        }
        __syncthreads();
        // ---- 4. Ahat R0^T = W by substitution, one row per thread (Ahat into regA)
        for (int i = tid; i < In; i += blockDim.x) {
            double x[kBMaxR];
            for (int k = R - 1; k >= 0; --k) {
                double s = Ws[i + In * k];
                for (int j = k + 1; j < R; ++j) s = fma(-R0s[k + R * j], x[j], s);
                x[k] = s / R0s[k + R * k];
            }
            for (int k = 0; k < R; ++k) regA[i + In * k] = x[k];
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
        // ---- 5. normalise columns (2-norm): A_n and lambda
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
        // ---- 6. A_n = Q_n R_n (FP64, shared memory)
        cta_householder(regA, In, R, regB, Rns, tau, red);
        double* Qn = F + pr.q[n];
        double* Rn_g = F + pr.rf[n];
        for (int e = tid; e < In * R; e += blockDim.x) Qn[e] = regB[e];
        for (int e = tid; e < RR; e += blockDim.x) Rn_g[e] = Rns[e];
        // ---- 7. efficient fit after the last mode (Sec. 3.3.1)
        if (n == 2) {
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
        }
        __syncthreads();
    }
}

// QR of every initial factor: one CTA per (problem, mode).
__global__ void batch_factor_qr_kernel(BProb* __restrict__ probs, int count, int maxR, int maxI,
                                       double* __restrict__ F)
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
struct Batch {
    int count = 0, maxR = 0, maxI = 0;
    std::vector<BProb> probs;
    std::vector<int> order;
    BProb* d_probs = nullptr;
    int* d_order = nullptr;
    float* Xall = nullptr;
    double* F = nullptr;
    float* T1all = nullptr;
    float* Yall = nullptr;
    int* d_pstatus = nullptr;
    double* d_fit = nullptr;
    int64_t x_elems = 0, f_elems = 0, t1_elems = 0, y_elems = 0;
    cudaStream_t stream = nullptr;
    int num_sms = 0;
    int grid = 0, threads = 0;           // autotuned launch shape (0 = not tuned yet)
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
    int64_t xo = 0, fo = 0, t1o = 0, yo = 0;
    std::vector<double> work(count);
    for (int p = 0; p < count; ++p) {
        BProb& pr = b->probs[p];
        for (int m = 0; m < 3; ++m) pr.I[m] = (int)dims[3 * p + m];
        pr.R = ranks[p];
        b->maxR = std::max(b->maxR, pr.R);
        for (int m = 0; m < 3; ++m) b->maxI = std::max(b->maxI, pr.I[m]);
        const int64_t P = (int64_t)pr.I[0] * pr.I[1] * pr.I[2];
        pr.x = xo;
        xo += align4(P);
        for (int m = 0; m < 3; ++m) { pr.a[m] = fo; fo += (int64_t)pr.I[m] * pr.R; }
        for (int m = 0; m < 3; ++m) { pr.q[m] = fo; fo += (int64_t)pr.I[m] * pr.R; }
        for (int m = 0; m < 3; ++m) { pr.rf[m] = fo; fo += (int64_t)pr.R * pr.R; }
        pr.lam = fo;
        fo += pr.R;
        int64_t t1max = 0, ymax = 0;
        for (int n = 0; n < 3; ++n) {
            int o[2], c = 0;
            for (int m = 0; m < 3; ++m)
                if (m != n) o[c++] = m;
            const int c1 = (pr.I[o[1]] >= pr.I[o[0]]) ? o[1] : o[0];
            t1max = std::max(t1max, P / pr.I[c1] * pr.R);
            ymax = std::max(ymax, (int64_t)pr.I[n] * pr.R * pr.R);
        }
        pr.t1 = t1o;
        t1o += align4(t1max);
        pr.y = yo;
        yo += align4(ymax);
        pr.normX2 = 0.0;
        work[p] = (double)P * pr.R;
    }
    b->order.resize(count);
    std::iota(b->order.begin(), b->order.end(), 0);
    std::stable_sort(b->order.begin(), b->order.end(), [&](int a, int c) { return work[a] > work[c]; });
    b->x_elems = xo; b->f_elems = fo; b->t1_elems = t1o; b->y_elems = yo;
    CPALS_CUDA_TRY(cudaMalloc(&b->d_probs, sizeof(BProb) * count));
    CPALS_CUDA_TRY(cudaMalloc(&b->d_order, sizeof(int) * count));
    CPALS_CUDA_TRY(cudaMalloc(&b->Xall, sizeof(float) * std::max<int64_t>(xo, 1)));
    CPALS_CUDA_TRY(cudaMalloc(&b->F, sizeof(double) * std::max<int64_t>(fo, 1)));
    CPALS_CUDA_TRY(cudaMalloc(&b->T1all, sizeof(float) * std::max<int64_t>(t1o, 1)));
    CPALS_CUDA_TRY(cudaMalloc(&b->Yall, sizeof(float) * std::max<int64_t>(yo, 1)));
    CPALS_CUDA_TRY(cudaMalloc(&b->d_pstatus, sizeof(int) * count));
    CPALS_CUDA_TRY(cudaMalloc(&b->d_fit, sizeof(double) * count));
    CPALS_CUDA_TRY(cudaMemset(b->d_pstatus, 0, sizeof(int) * count));
    CPALS_CUDA_TRY(cudaMemset(b->d_fit, 0, sizeof(double) * count));
    CPALS_CUDA_TRY(cudaMemcpy(b->d_probs, b->probs.data(), sizeof(BProb) * count, cudaMemcpyHostToDevice));
    CPALS_CUDA_TRY(cudaMemcpy(b->d_order, b->order.data(), sizeof(int) * count, cudaMemcpyHostToDevice));
    int dev = 0;
    CPALS_CUDA_TRY(cudaGetDevice(&dev));
    CPALS_CUDA_TRY(cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, dev));
    b->smem = sizeof(double) * (size_t)bsmem_layout(b->maxR, b->maxI).total;
    CPALS_CUDA_TRY(cudaFuncSetAttribute(batch_mode_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem));
    CPALS_CUDA_TRY(cudaFuncSetAttribute(batch_factor_qr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)b->smem));
    return cudaSuccess;
}

void batch_free(Batch* b)
{
    auto f = [](void* p) { if (p) cudaFree(p); };
    f(b->d_probs); f(b->d_order); f(b->Xall); f(b->F); f(b->T1all); f(b->Yall); f(b->d_pstatus); f(b->d_fit);
    if (b->graph) cudaGraphExecDestroy(b->graph);
}

cudaError_t batch_norms(Batch* b)
{
    batch_norm_kernel<<<b->count, 256, 0, b->stream>>>(b->d_probs, b->count, b->Xall);
    b->launches++;
    return cudaGetLastError();
}

cudaError_t batch_factor_qr(Batch* b)
{
    batch_factor_qr_kernel<<<3 * b->count, 256, b->smem, b->stream>>>(b->d_probs, b->count, b->maxR, b->maxI, b->F);
    b->launches++;
    return cudaGetLastError();
}

static cudaError_t batch_sweep(Batch* b, int grid, int threads)
{
    for (int n = 0; n < 3; ++n) {
        batch_mode_kernel<<<grid, threads, b->smem, b->stream>>>(b->d_probs, b->d_order, b->count, n, b->maxR,
                                                                 b->maxI, b->Xall, b->F, b->T1all, b->Yall,
                                                                 b->d_pstatus, b->d_fit);
        b->launches++;
        CPALS_CUDA_TRY(cudaGetLastError());
    }
    return cudaSuccess;
}

// Pick the launch shape by timing one sweep per candidate on a copy of the
// factors (restored afterwards), then capture the sweep as a CUDA graph.
cudaError_t batch_prepare(Batch* b)
{
    if (b->graph) return cudaSuccess;
    double* saved = nullptr;
    CPALS_CUDA_TRY(cudaMalloc(&saved, sizeof(double) * std::max<int64_t>(b->f_elems, 1)));
    CPALS_CUDA_TRY(cudaMemcpyAsync(saved, b->F, sizeof(double) * b->f_elems, cudaMemcpyDeviceToDevice, b->stream));
    cudaEvent_t e0, e1;
    CPALS_CUDA_TRY(cudaEventCreate(&e0));
    CPALS_CUDA_TRY(cudaEventCreate(&e1));
    float best = 1e30f;
    const int threads_c[2] = {128, 256};
    for (int ti = 0; ti < 2; ++ti) {
        int occ = 0;
        CPALS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, batch_mode_kernel, threads_c[ti], b->smem));
        if (occ < 1) continue;
        for (int per = 1; per <= occ; ++per) {
            const int grid = std::min(b->count, b->num_sms * per);
            CPALS_CUDA_TRY(cudaMemcpyAsync(b->F, saved, sizeof(double) * b->f_elems, cudaMemcpyDeviceToDevice,
                                           b->stream));
            CPALS_CUDA_TRY(cudaEventRecord(e0, b->stream));
            CPALS_CUDA_TRY(batch_sweep(b, grid, threads_c[ti]));
            CPALS_CUDA_TRY(cudaEventRecord(e1, b->stream));
            CPALS_CUDA_TRY(cudaEventSynchronize(e1));
            float ms = 0.f;
            CPALS_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
            if (ms < best) { best = ms; b->grid = grid; b->threads = threads_c[ti]; }
            if (grid == b->count) break;
        }
    }
    CPALS_CUDA_TRY(cudaMemcpyAsync(b->F, saved, sizeof(double) * b->f_elems, cudaMemcpyDeviceToDevice, b->stream));
    CPALS_CUDA_TRY(cudaMemsetAsync(b->d_pstatus, 0, sizeof(int) * b->count, b->stream));
    CPALS_CUDA_TRY(cudaStreamSynchronize(b->stream));
    cudaFree(saved);
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
        e2 = batch_sweep(b, b->grid, b->threads);
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
        b->launches += 3;
    }
    return cudaSuccess;
}

}  // namespace cpals
