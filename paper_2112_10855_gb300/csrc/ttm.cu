// ttm.cu -- passes over the data tensor X: Multi-TTM (Eq. multittm, Alg.
// cp-als-qr Multi-TTM step), MTTKRP (Alg. cp-als), ||X||^2 and the direct
// residual (Sec. 3.3.1).
//
// A single TTM over mode m views the current tensor as [L, K, T] (L = prod of
// the dims before m, K = I_m, T = prod of the dims after m) and computes
//     Out(l, r, t) = sum_k In(l, k, t) * Q(k, r),     Q = Q_m (K x R)
// i.e. Y = X x_m Q_m^T.  The Multi-TTM applies the N-1 TTMs in
// decreasing-dimension order (Sec. 3.2), ping-ponging between two workspace
// buffers; the first one streams X from HBM, the later ones read the shrunken
// intermediate (R/I of the previous size), which usually stays in L2.
//
// Kernel per TTM: FP64 -> ttm_rows_kernel (CTA size chosen per launch);
// FP32 -> the TMA-ring pipeline of tc_split.cu when 9 <= R <= 64 and
// L % 4 == 0, else ttm_fiber4_kernel for L == 1, ttm_rows4_kernel for
// L % 4 == 0, ttm_rows_kernel otherwise; 3xBF16 / 3xTF32 run the pass over X
// on the tensor cores (tc_split.cu) and their later TTMs like FP32.  Small
// row counts split K over grid.z with a fixed-order reduction.
#include <algorithm>
#include <mutex>

#include "internal.cuh"

namespace cpals {

namespace {

constexpr int kKC = 32;   // k-chunk of Q staged in shared memory

template <typename T>
__device__ __forceinline__ T fma_t(T a, T b, T c);
template <>
__device__ __forceinline__ double fma_t<double>(double a, double b, double c) { return fma(a, b, c); }
template <>
__device__ __forceinline__ float fma_t<float>(float a, float b, float c) { return fmaf(a, b, c); }

// One thread per flattened output row f = l + L*t and RC output columns
// (RC = R rounded up to an instantiated width; grid.y covers wider R in
// chunks).  Q(k, r) for a k-chunk is staged in shared memory as qs[k][r] and
// read as a broadcast.  Loads of In along k are coalesced across the warp
// whenever L >= 32; for small L each thread walks its own fiber and the lines
// are reused from L1.  grid.z splits K: with gridDim.z > 1 each split writes
// its partial sums to part + z * (L*R*T) in the output layout, and
// reduce_splits_kernel adds them in split order (deterministic).
template <typename T, int RC, int TPB>
__global__ void __launch_bounds__(TPB) ttm_rows_kernel(
    const T* __restrict__ in, const double* __restrict__ Q, int64_t ldq, T* __restrict__ out,
    int64_t L, int64_t K, int64_t Tn, int R, int64_t kchunk, const int* __restrict__ status)
{
    if (*status != kStatusOk) return;
    __shared__ T qs[kKC][RC];
    const int64_t rows = L * Tn;
    const int64_t f = (int64_t)blockIdx.x * TPB + threadIdx.x;
    const int r0 = blockIdx.y * RC;
    const int rc = min(RC, R - r0);
    const bool active = f < rows;
    const int64_t kb = (int64_t)blockIdx.z * kchunk;
    const int64_t ke = (kb + kchunk < K) ? kb + kchunk : K;
    int64_t t = 0, l = 0;
    if (active) { t = f / L; l = f - t * L; }
    const T* p = in + l + L * K * t;

    T acc[RC];
#pragma unroll
    for (int r = 0; r < RC; ++r) acc[r] = T(0);

    for (int64_t k0 = kb; k0 < ke; k0 += kKC) {
        const int kc = (int)((ke - k0) < (int64_t)kKC ? (ke - k0) : (int64_t)kKC);
        __syncthreads();
        for (int i = threadIdx.x; i < kKC * RC; i += TPB) {
            const int kk = i / RC, rr = i - kk * RC;
            qs[kk][rr] = (kk < kc && rr < rc) ? (T)Q[(k0 + kk) + ldq * (int64_t)(r0 + rr)] : T(0);
        }
        __syncthreads();
        if (!active) continue;
        const T* pk = p + L * k0;
        int kk = 0;
        for (; kk + 8 <= kc; kk += 8) {
            T x[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) x[u] = __ldg(pk + L * (kk + u));
#pragma unroll
            for (int u = 0; u < 8; ++u)
#pragma unroll
                for (int r = 0; r < RC; ++r) acc[r] = fma_t(x[u], qs[kk + u][r], acc[r]);
        }
        for (; kk < kc; ++kk) {
            const T x = __ldg(pk + L * kk);
#pragma unroll
            for (int r = 0; r < RC; ++r) acc[r] = fma_t(x, qs[kk][r], acc[r]);
        }
    }
    if (active) {
        T* o = out + (int64_t)blockIdx.z * (L * (int64_t)R * Tn) + l + L * (int64_t)R * t;
#pragma unroll
        for (int r = 0; r < RC; ++r)
            if (r < rc) o[L * (int64_t)(r0 + r)] = acc[r];
    }
}

// FP32 variant with four rows per thread (L % 4 == 0, so the four rows share
// t and are contiguous): one 128-bit load and RC broadcast reads of Q per k
// feed 4*RC FMAs.  This makes the kernel FMA-bound instead of bound by the
// shared-memory broadcasts.
template <int RC, int TPB>
__global__ void __launch_bounds__(TPB) ttm_rows4_kernel(
    const float* __restrict__ in, const double* __restrict__ Q, int64_t ldq, float* __restrict__ out,
    int64_t L, int64_t K, int64_t Tn, int R, int64_t kchunk, const int* __restrict__ status)
{
    if (*status != kStatusOk) return;
    __shared__ float qs[kKC][RC];
    const int64_t rows = L * Tn;
    const int64_t f = 4 * ((int64_t)blockIdx.x * TPB + threadIdx.x);
    const int r0 = blockIdx.y * RC;
    const int rc = min(RC, R - r0);
    const bool active = f < rows;          // rows % 4 == 0, so all four rows exist
    const int64_t kb = (int64_t)blockIdx.z * kchunk;
    const int64_t ke = (kb + kchunk < K) ? kb + kchunk : K;
    int64_t t = 0, l = 0;
    if (active) { t = f / L; l = f - t * L; }
    const float* p = in + l + L * K * t;

    float acc[4][RC];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int r = 0; r < RC; ++r) acc[i][r] = 0.0f;

    for (int64_t k0 = kb; k0 < ke; k0 += kKC) {
        const int kc = (int)((ke - k0) < (int64_t)kKC ? (ke - k0) : (int64_t)kKC);
        __syncthreads();
        for (int i = threadIdx.x; i < kKC * RC; i += TPB) {
            const int kk = i / RC, rr = i - kk * RC;
            qs[kk][rr] = (kk < kc && rr < rc) ? (float)Q[(k0 + kk) + ldq * (int64_t)(r0 + rr)] : 0.0f;
        }
        __syncthreads();
        if (!active) continue;
        const float* pk = p + L * k0;
        int kk = 0;
        for (; kk + 4 <= kc; kk += 4) {
            float4 x[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) x[u] = __ldg(reinterpret_cast<const float4*>(pk + L * (kk + u)));
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int r = 0; r < RC; ++r) {
                    const float q = qs[kk + u][r];
                    acc[0][r] = fmaf(x[u].x, q, acc[0][r]);
                    acc[1][r] = fmaf(x[u].y, q, acc[1][r]);
                    acc[2][r] = fmaf(x[u].z, q, acc[2][r]);
                    acc[3][r] = fmaf(x[u].w, q, acc[3][r]);
                }
        }
        for (; kk < kc; ++kk) {
            const float4 x = __ldg(reinterpret_cast<const float4*>(pk + L * kk));
#pragma unroll
            for (int r = 0; r < RC; ++r) {
                const float q = qs[kk][r];
                acc[0][r] = fmaf(x.x, q, acc[0][r]);
                acc[1][r] = fmaf(x.y, q, acc[1][r]);
                acc[2][r] = fmaf(x.z, q, acc[2][r]);
                acc[3][r] = fmaf(x.w, q, acc[3][r]);
            }
        }
    }
    if (active) {
        float* o = out + (int64_t)blockIdx.z * (L * (int64_t)R * Tn) + l + L * (int64_t)R * t;
#pragma unroll
        for (int r = 0; r < RC; ++r)
            if (r < rc)
                *reinterpret_cast<float4*>(o + L * (int64_t)(r0 + r)) =
                    make_float4(acc[0][r], acc[1][r], acc[2][r], acc[3][r]);
    }
}

// FP32 TTM over the fastest mode (L = 1): row t of the output contracts the
// contiguous fiber In(:, t).  One thread per fiber reads it four indices at
// a time (16-byte loads; K % 4 == 0 and a 16-byte aligned tensor), and Q's
// chunk sits in shared memory as qs[k][r] with r padded to RC4 (a multiple of
// 4), so four columns of one k come in one broadcast 16-byte read.  With one
// scalar load per k the row kernel's warp touches 32 lines per instruction
// and its L1 becomes the bottleneck; here that count falls fourfold.
template <int RC4>
__global__ void __launch_bounds__(128) ttm_fiber4_kernel(
    const float* __restrict__ in, const double* __restrict__ Q, int64_t ldq, float* __restrict__ out, int64_t K,
    int64_t Tn, int R, int64_t kchunk, const int* __restrict__ status)
{
    if (*status != kStatusOk) return;
    __shared__ __align__(16) float qs[kKC][RC4];
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int r0 = blockIdx.y * RC4;
    const int rc = min(RC4, R - r0);
    const bool active = t < Tn;
    const int64_t kb = (int64_t)blockIdx.z * kchunk;
    const int64_t ke = (kb + kchunk < K) ? kb + kchunk : K;
    const float* p = in + K * (active ? t : 0);
    float acc[RC4];
#pragma unroll
    for (int r = 0; r < RC4; ++r) acc[r] = 0.0f;
    for (int64_t k0 = kb; k0 < ke; k0 += kKC) {
        const int kc = (int)((ke - k0) < (int64_t)kKC ? (ke - k0) : (int64_t)kKC);
        __syncthreads();
        for (int i = threadIdx.x; i < kKC * RC4; i += blockDim.x) {
            const int kk = i / RC4, rr = i - kk * RC4;
            qs[kk][rr] = (kk < kc && rr < rc) ? (float)Q[(k0 + kk) + ldq * (int64_t)(r0 + rr)] : 0.0f;
        }
        __syncthreads();
        if (!active) continue;
        for (int kk = 0; kk < kc; kk += 4) {          // kc % 4 == 0: K and kchunk are multiples of 4
            const float4 x = __ldg(reinterpret_cast<const float4*>(p + k0 + kk));
            const float xv[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int r = 0; r < RC4; r += 4) {
                    const float4 q = *reinterpret_cast<const float4*>(&qs[kk + u][r]);
                    acc[r] = fmaf(xv[u], q.x, acc[r]);
                    acc[r + 1] = fmaf(xv[u], q.y, acc[r + 1]);
                    acc[r + 2] = fmaf(xv[u], q.z, acc[r + 2]);
                    acc[r + 3] = fmaf(xv[u], q.w, acc[r + 3]);
                }
        }
    }
    if (active) {
        float* o = out + (int64_t)blockIdx.z * ((int64_t)R * Tn) + (int64_t)R * t;
#pragma unroll
        for (int r = 0; r < RC4; ++r)
            if (r < rc) o[r0 + r] = acc[r];
    }
}

// FP32 TTM over the fastest mode (L = 1) as a tiled GEMM: one single TTM of
// the Multi-TTM (Eq. multittm, Sec. 3.2) when the contracted mode is mode 0,
// out(t, r) = sum_k In(k, t) Q(k, r) with every fiber In(:, t) contiguous.  A CTA of 256
// threads owns 128 fibers and BN columns (BN = 32 or 64, Q zero-padded to
// BN) and walks its K range in chunks of 32.  The [128 fibers x 32] block is
// read as 128-byte fiber rows (eight threads per row, 16-byte loads, K % 4
// == 0) and stored k-major in shared memory; Q's FP32 chunk [32 x BN] sits
// beside it.  Each thread accumulates BN/8 fibers x 4 columns from two
// 16-byte reads per k, and the next chunk is loaded into registers while the
// current one is multiplied.  With a K split (blockIdx.z) each split writes
// its partial at out + z R T.  The k order per output is ascending within a
// split, as in the one-thread-per-fiber kernel above.
constexpr int kFgRows = 128;
constexpr int kFgK = 32;
constexpr int kFgThreads = 256;
constexpr int kFgLd = kFgRows + 4;     // k-major rows of the fiber block, 16-byte aligned

template <int BN>
__global__ void __launch_bounds__(kFgThreads) ttm_fiber_gemm_kernel(const float* __restrict__ in,
                                                                    const float* __restrict__ qf,
                                                                    float* __restrict__ out, int64_t K, int64_t Tn,
                                                                    int R, int64_t kchunk,
                                                                    const int* __restrict__ status)
{
    if (*status != kStatusOk) return;
    constexpr int TM = BN / 8;                 // fibers per thread
    constexpr int CG = BN / 4;                 // column groups of 4
    constexpr int A4 = kFgRows * kFgK / 4 / kFgThreads;   // float4 of the fiber block per thread (4)
    constexpr int B4 = kFgK * BN / 4 / kFgThreads;        // float4 of the Q chunk per thread (1 or 2)
    __shared__ __align__(16) float As[kFgK][kFgLd];
    __shared__ __align__(16) float Bs[kFgK][BN];
    const int tid = threadIdx.x;
    const int cg = tid % CG, tg = tid / CG;
    const int64_t t0 = (int64_t)blockIdx.x * kFgRows;
    const int64_t kb = (int64_t)blockIdx.z * kchunk;
    const int64_t ke = (kb + kchunk < K) ? kb + kchunk : K;
    float acc[TM][4];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;
    float4 ra[A4], rb[B4];
    auto load = [&](int64_t k0) {
#pragma unroll
        for (int u = 0; u < A4; ++u) {
            const int idx = tid + u * kFgThreads;
            const int row = idx >> 3, k4 = idx & 7;
            const int64_t t = t0 + row, k = k0 + 4 * k4;
            ra[u] = (t < Tn && k < ke) ? __ldg(reinterpret_cast<const float4*>(in + t * K + k))
                                       : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < B4; ++u) {
            const int idx = tid + u * kFgThreads;
            const int kk = idx / CG, c4 = idx - kk * CG;
            rb[u] = *reinterpret_cast<const float4*>(qf + (k0 + kk) * BN + 4 * c4);
        }
    };
    auto store = [&]() {
#pragma unroll
        for (int u = 0; u < A4; ++u) {
            const int idx = tid + u * kFgThreads;
            const int row = idx >> 3, k4 = idx & 7;
            As[4 * k4 + 0][row] = ra[u].x;
            As[4 * k4 + 1][row] = ra[u].y;
            As[4 * k4 + 2][row] = ra[u].z;
            As[4 * k4 + 3][row] = ra[u].w;
        }
#pragma unroll
        for (int u = 0; u < B4; ++u) {
            const int idx = tid + u * kFgThreads;
            const int kk = idx / CG, c4 = idx - kk * CG;
            *reinterpret_cast<float4*>(&Bs[kk][4 * c4]) = rb[u];
        }
    };
    if (kb < ke) load(kb);
    for (int64_t k0 = kb; k0 < ke; k0 += kFgK) {
        __syncthreads();                       // the previous chunk is read
        store();
        __syncthreads();
        if (k0 + kFgK < ke) load(k0 + kFgK);
#pragma unroll 8
        for (int k = 0; k < kFgK; ++k) {
            float a[TM];
#pragma unroll
            for (int i = 0; i < TM; i += 4) {
                const float4 v = *reinterpret_cast<const float4*>(&As[k][tg * TM + i]);
                a[i] = v.x; a[i + 1] = v.y; a[i + 2] = v.z; a[i + 3] = v.w;
            }
            const float4 b = *reinterpret_cast<const float4*>(&Bs[k][4 * cg]);
#pragma unroll
            for (int i = 0; i < TM; ++i) {
                acc[i][0] = fmaf(a[i], b.x, acc[i][0]);
                acc[i][1] = fmaf(a[i], b.y, acc[i][1]);
                acc[i][2] = fmaf(a[i], b.z, acc[i][2]);
                acc[i][3] = fmaf(a[i], b.w, acc[i][3]);
            }
        }
    }
    float* o = out + (int64_t)blockIdx.z * ((int64_t)R * Tn);
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const int64_t t = t0 + tg * TM + i;
        if (t >= Tn) break;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = 4 * cg + j;
            if (c < R) o[t * R + c] = acc[i][j];
        }
    }
}

// Q (K x R, FP64, ldq) to the FP32 [Kp x BN] copy of the fiber GEMM (zero
// beyond K and R).
__global__ void fiber_q_kernel(const double* __restrict__ Q, int64_t ldq, int64_t K, int R, int64_t Kp, int BN,
                               float* __restrict__ qf, const int* __restrict__ status)
{
    if (*status != kStatusOk) return;
    const int64_t total = Kp * BN;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = e / BN;
        const int c = (int)(e - k * BN);
        qf[e] = (k < K && c < R) ? (float)Q[k + ldq * (int64_t)c] : 0.0f;
    }
}

// out[g*n + e] = sum of part[q*n + e] over the splits q of group g (groups of
// `group` consecutive splits, added in split order).  With one group this is
// the final sum; with several, a second call adds the group sums in order.
template <typename T>
__global__ void reduce_splits_kernel(const T* __restrict__ part, int ks, int group, int64_t n, T* __restrict__ out,
                                     const int* __restrict__ status)
{
    if (*status != kStatusOk) return;
    const int ng = (ks + group - 1) / group;
    const int64_t total = n * ng;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < total; w += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = w / n, e = w - g * n;
        const int q0 = (int)g * group, q1 = min(ks, q0 + group);
        T s = part[(int64_t)q0 * n + e];
        for (int q = q0 + 1; q < q1; ++q) s += part[(int64_t)q * n + e];
        out[g * n + e] = s;
    }
}

// CTA size: FP32 is bound by HBM and uses 256-row CTAs; FP64 takes the CTA
// size of plan_rows_f64 (ttm_plan.h), picked per launch.
constexpr int kRowsMaxTpb = 256;
// FP32 row-quad kernel: 4 rows per thread; its CTA size (64, 96 or 128
// threads) is picked per launch from the resident CTAs per SM, so that a pass
// does not end in a ragged second wave (at 135 registers a thread, 128-thread
// CTAs fit three to an SM).
constexpr int kQuadTpb[] = {128, 96, 64};

template <int W, int C>
int quad_occupancy()
{
    static const int occ = [] {
        int v = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, ttm_rows4_kernel<W, C>, C, 0) != cudaSuccess) v = 1;
        return v > 0 ? v : 1;
    }();
    return occ;
}

template <int W>
int quad_occupancy(int tpb)
{
    return tpb == 64 ? quad_occupancy<W, 64>() : tpb == 96 ? quad_occupancy<W, 96>() : quad_occupancy<W, 128>();
}

template <int W>
void launch_rows4(dim3 grid, int tpb, cudaStream_t st, const float* in, const double* Q, int64_t ldq, float* out,
                  TtmShape s, int R, int64_t kchunk, const int* status)
{
    if (tpb == 64) ttm_rows4_kernel<W, 64><<<grid, 64, 0, st>>>(in, Q, ldq, out, s.L, s.K, s.T, R, kchunk, status);
    else if (tpb == 96) ttm_rows4_kernel<W, 96><<<grid, 96, 0, st>>>(in, Q, ldq, out, s.L, s.K, s.T, R, kchunk, status);
    else ttm_rows4_kernel<W, 128><<<grid, 128, 0, st>>>(in, Q, ldq, out, s.L, s.K, s.T, R, kchunk, status);
}

template <typename T, int RC>
void launch_rows(dim3 grid, int tpb, cudaStream_t st, const T* in, const double* Q, int64_t ldq, T* out,
                 TtmShape s, int R, int64_t kchunk, const int* status)
{
#define CPALS_TPB(C)                                                                                           \
    case C: ttm_rows_kernel<T, RC, C><<<grid, C, 0, st>>>(in, Q, ldq, out, s.L, s.K, s.T, R, kchunk, status); break;
    if constexpr (sizeof(T) == 8) {
        switch (tpb) {
            CPALS_TPB(96) CPALS_TPB(128)
            default: ttm_rows_kernel<T, RC, 64><<<grid, 64, 0, st>>>(in, Q, ldq, out, s.L, s.K, s.T, R, kchunk, status);
        }
    } else {
        (void)tpb;
        ttm_rows_kernel<T, RC, kRowsMaxTpb><<<grid, kRowsMaxTpb, 0, st>>>(in, Q, ldq, out, s.L, s.K, s.T, R, kchunk,
                                                                          status);
    }
#undef CPALS_TPB
}

// Sum the ks K-split partials (part, ks x outn) into out in split order: one
// pass for up to 16 splits, else groups of 16 and then the group sums.
template <typename T>
cudaError_t reduce_ksplit(Handle* h, T* part, int64_t ks, int64_t outn, T* out)
{
    if (ks <= 1) return cudaSuccess;
    constexpr int kGroup = (int)kSplitGroup;
    const int64_t ng = (ks + kGroup - 1) / kGroup;
    auto grid_of = [&](int64_t work) {
        int64_t g = (work + 255) / 256;
        return (unsigned)std::max<int64_t>(1, std::min<int64_t>(g, 16LL * h->num_sms));
    };
    if (ng == 1) {
        reduce_splits_kernel<T><<<grid_of(outn), 256, 0, h->stream>>>(part, (int)ks, kGroup, outn, out, h->d_status);
        h->launches++;
    } else {
        T* gsum = part + ks * outn;     // group sums after the partials
        reduce_splits_kernel<T><<<grid_of(outn * ng), 256, 0, h->stream>>>(part, (int)ks, kGroup, outn, gsum,
                                                                           h->d_status);
        reduce_splits_kernel<T><<<grid_of(outn), 256, 0, h->stream>>>(gsum, (int)ng, (int)ng, outn, out,
                                                                      h->d_status);
        h->launches += 2;
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_ttm_split(Handle* h, const T* in, const double* Q, int64_t ldq, T* out, TtmShape s, int R,
                             T* part, int64_t part_elems)
{
    const int64_t rows = s.L * s.T;
    if (rows == 0) return cudaSuccess;
    const int rc = ttm_width(R);
    // FP32 with four rows per thread when the rows come in aligned quads
    const bool quad = sizeof(T) == 4 && (s.L % 4) == 0 && rc <= 24 &&
                      (((uintptr_t)in) & 15) == 0 && (((uintptr_t)out) & 15) == 0 && (((uintptr_t)part) & 15) == 0;
    const int64_t gy = (R + rc - 1) / rc;
    const int64_t outn = rows * R;
    // FP32 contraction of the fastest mode: a tiled GEMM above rank 16 (its
    // FP32 copy of Q is carved from the end of the partials' space), else one
    // thread per contiguous fiber
    const bool fiber = sizeof(T) == 4 && s.L == 1 && (s.K % 4) == 0 && (((uintptr_t)in) & 15) == 0;
    if (fiber && R > 16 && R <= 64 && part != nullptr) {
        const int BN = R > 32 ? 64 : 32;
        const int64_t Kp = (s.K + kFgK - 1) / kFgK * kFgK;
        const int64_t qelems = (Kp * BN + 3) / 4 * 4;       // floats, 16-byte multiple
        const int64_t qe_T = (qelems * 4 + (int64_t)sizeof(T) - 1) / (int64_t)sizeof(T);
        if (part_elems >= qe_T + outn) {
            float* qf = reinterpret_cast<float*>(part + (part_elems - qe_T));
            if ((((uintptr_t)qf) & 15) == 0) {
                const int64_t pe = part_elems - qe_T;
                const int64_t gx = (s.T + kFgRows - 1) / kFgRows;
                int64_t ks = ttm_ksplit(gx, kFgThreads, s.K / kFgK, h->num_sms, outn, pe, true);
                int64_t kc = ((s.K + ks - 1) / ks + kFgK - 1) / kFgK * kFgK;      // whole 32-chunks
                ks = (s.K + kc - 1) / kc;
                const unsigned qgrid = (unsigned)std::max<int64_t>(
                    1, std::min<int64_t>((Kp * BN + 255) / 256, 8LL * h->num_sms));
                fiber_q_kernel<<<qgrid, 256, 0, h->stream>>>(Q, ldq, s.K, R, Kp, BN, qf, h->d_status);
                h->launches++;
                CPALS_CUDA_TRY(cudaGetLastError());
                const dim3 grid((unsigned)gx, 1, (unsigned)ks);
                float* dst = reinterpret_cast<float*>(ks > 1 ? part : out);
                const float* fin = reinterpret_cast<const float*>(in);
                if (BN == 64)
                    ttm_fiber_gemm_kernel<64><<<grid, kFgThreads, 0, h->stream>>>(fin, qf, dst, s.K, s.T, R, kc,
                                                                                  h->d_status);
                else
                    ttm_fiber_gemm_kernel<32><<<grid, kFgThreads, 0, h->stream>>>(fin, qf, dst, s.K, s.T, R, kc,
                                                                                  h->d_status);
                h->launches++;
                CPALS_CUDA_TRY(cudaGetLastError());
                return reduce_ksplit<T>(h, part, ks, outn, out);
            }
        }
    }
    if (fiber) {
        const int rc4 = R > 24 ? 32 : (R + 3) / 4 * 4;
        constexpr int tpbf = 128;
        const int64_t fgx = (s.T + tpbf - 1) / tpbf, fgy = (R + rc4 - 1) / rc4;
        int64_t fks = ttm_ksplit(fgx * fgy, tpbf, s.K / 4, h->num_sms, outn, part_elems, part != nullptr);
        int64_t fkc = ((s.K / 4 + fks - 1) / fks) * 4;    // chunks of whole quads
        fks = (s.K + fkc - 1) / fkc;
        const dim3 fgrid((unsigned)fgx, (unsigned)fgy, (unsigned)fks);
        float* fdst = reinterpret_cast<float*>(fks > 1 ? part : out);
        const float* fin = reinterpret_cast<const float*>(in);
        switch (rc4) {
#define CPALS_RF(W)                                                                                            \
    case W:                                                                                                    \
        ttm_fiber4_kernel<W><<<fgrid, tpbf, 0, h->stream>>>(fin, Q, ldq, fdst, s.K, s.T, R, fkc, h->d_status); \
        break;
            CPALS_RF(4) CPALS_RF(8) CPALS_RF(12) CPALS_RF(16) CPALS_RF(20) CPALS_RF(24) CPALS_RF(32)
#undef CPALS_RF
            default: return cudaErrorInvalidValue;
        }
        h->launches++;
        CPALS_CUDA_TRY(cudaGetLastError());
        return reduce_ksplit<T>(h, part, fks, outn, out);
    }
    int tpb = quad ? 128 : kRowsMaxTpb;
    int64_t rows_per_cta = quad ? 4 * tpb : tpb;
    int64_t gx = (rows + rows_per_cta - 1) / rows_per_cta;
    int64_t ks = ttm_ksplit(gx * gy, tpb, s.K, h->num_sms, outn, part_elems, part != nullptr);
    if (quad) {
        // the CTA size with the smallest per-SM share of rows, a ragged
        // second wave counted as a quarter more
        int64_t best = -1;
        for (int c : kQuadTpb) {
            int occ = 1;
            switch (rc) {
#define CPALS_RO(W) case W: occ = quad_occupancy<W>(c); break;
                CPALS_RO(1) CPALS_RO(2) CPALS_RO(3) CPALS_RO(4) CPALS_RO(5) CPALS_RO(6) CPALS_RO(7) CPALS_RO(8)
                CPALS_RO(9) CPALS_RO(10) CPALS_RO(11) CPALS_RO(12) CPALS_RO(13) CPALS_RO(14) CPALS_RO(15) CPALS_RO(16)
                CPALS_RO(20) CPALS_RO(24)
#undef CPALS_RO
                default: break;
            }
            const int64_t cx = (rows + 4 * c - 1) / (4 * c);
            const int64_t cks = ttm_ksplit(cx * gy, c, s.K, h->num_sms, outn, part_elems, part != nullptr);
            const int64_t ckc = (s.K + cks - 1) / cks;
            const int64_t per_sm = (cx * gy * cks + h->num_sms - 1) / h->num_sms;
            int64_t cost = per_sm * 4 * c * ckc;
            if (per_sm > occ) cost += cost / 4;
            if (best < 0 || cost < best) { best = cost; tpb = c; gx = cx; ks = cks; }
        }
    }
    if (sizeof(T) == 8) {
        // FP64: the CTA size with the smallest per-SM share of rows x indices
        const RowsPlan p = plan_rows_f64(h->num_sms, s, R, part_elems, part != nullptr);
        tpb = p.tpb; gx = p.gx; ks = p.ks;
    }
    const int64_t kchunk = (s.K + ks - 1) / ks;
    dim3 grid((unsigned)gx, (unsigned)gy, (unsigned)ks);
    T* dst = (ks > 1) ? part : out;
    if (quad) {
        const float* fin = reinterpret_cast<const float*>(in);
        float* fdst = reinterpret_cast<float*>(dst);
        switch (rc) {
#define CPALS_RQ(W) \
    case W: launch_rows4<W>(grid, tpb, h->stream, fin, Q, ldq, fdst, s, R, kchunk, h->d_status); break;
            CPALS_RQ(1) CPALS_RQ(2) CPALS_RQ(3) CPALS_RQ(4) CPALS_RQ(5) CPALS_RQ(6) CPALS_RQ(7) CPALS_RQ(8)
            CPALS_RQ(9) CPALS_RQ(10) CPALS_RQ(11) CPALS_RQ(12) CPALS_RQ(13) CPALS_RQ(14) CPALS_RQ(15) CPALS_RQ(16)
            CPALS_RQ(20) CPALS_RQ(24)
#undef CPALS_RQ
            default: return cudaErrorInvalidValue;
        }
    } else switch (rc) {
#define CPALS_RC(W) case W: launch_rows<T, W>(grid, tpb, h->stream, in, Q, ldq, dst, s, R, kchunk, h->d_status); break;
        CPALS_RC(1) CPALS_RC(2) CPALS_RC(3) CPALS_RC(4) CPALS_RC(5) CPALS_RC(6) CPALS_RC(7) CPALS_RC(8)
        CPALS_RC(9) CPALS_RC(10) CPALS_RC(11) CPALS_RC(12) CPALS_RC(13) CPALS_RC(14) CPALS_RC(15) CPALS_RC(16)
        CPALS_RC(20) CPALS_RC(24) CPALS_RC(32)
#undef CPALS_RC
        default: return cudaErrorInvalidValue;
    }
    h->launches++;
    CPALS_CUDA_TRY(cudaGetLastError());
    return reduce_ksplit<T>(h, part, ks, outn, out);
}

// One TTM: FP32 through the TMA-fed pipeline where the shape allows it, else
// the row kernels.
template <typename T>
cudaError_t launch_ttm(Handle* h, const T* in, const double* Q, int64_t ldq, T* out, TtmShape s, int R)
{
    if constexpr (sizeof(T) == 4) {
        if (h->f32_pipe && f32_pipe_ok(in, out, s, R)) return ttm_f32_pipe(h, in, Q, ldq, out, s, R);
    }
    return launch_ttm_split<T>(h, in, Q, ldq, out, s, R, (T*)h->scratch,
                               h->scratch_elems * (int64_t)(sizeof(double) / sizeof(T)));
}

// Final Multi-TTM tensor (dims R for m != n, I_n at n; mode 0 fastest) to the
// FP64 unfolding Y_(n): element e = a + Rn*(i + In*c) with a < Rn = R^n maps to
// column a + Rn*c.
template <typename T>
__global__ void unfold_kernel(const T* __restrict__ in, double* __restrict__ Yn, int64_t Rn, int64_t In,
                              int64_t total, const int* __restrict__ status)
{
    if (*status != kStatusOk) return;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = e % Rn;
        const int64_t q = e / Rn;
        const int64_t i = q % In;
        const int64_t c = q / In;
        Yn[i + In * (a + Rn * c)] = (double)in[e];
    }
}

// The same unfolding in FP32 (no conversion).
__global__ void unfold32_kernel(const float* __restrict__ in, float* __restrict__ Yn, int64_t Rn, int64_t In,
                                int64_t total, const int* __restrict__ status)
{
    if (*status != kStatusOk) return;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = e % Rn;
        const int64_t q = e / Rn;
        const int64_t i = q % In;
        const int64_t c = q / In;
        Yn[i + In * (a + Rn * c)] = in[e];
    }
}

__global__ void widen_kernel(const float* __restrict__ in, double* __restrict__ out, int64_t n,
                             const int* __restrict__ status)
{
    if (*status != kStatusOk) return;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        out[e] = (double)in[e];
}

// Diagonal contraction of the MTTKRP: after the first TTM one mode (position
// cpos) holds the rank index r; contracting mode m with A_m(:, r) keeps r:
//   Out(l, t) = sum_k In(l, k, t) * A(k, r(l, t)).
template <typename T>
__global__ void diag_contract_kernel(const T* __restrict__ in, const double* __restrict__ A, int64_t lda,
                                     T* __restrict__ out, int64_t L, int64_t K, int64_t Tn, int r_in_l,
                                     int64_t r_div, int R, const int* __restrict__ status)
{
    if (*status != kStatusOk) return;
    const int64_t rows = L * Tn;
    for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < rows;
         f += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = f / L, l = f - t * L;
        const int r = (int)(((r_in_l ? l : t) / r_div) % R);
        const T* p = in + l + L * K * t;
        const double* a = A + lda * r;
        T acc = T(0);
        for (int64_t k = 0; k < K; ++k) acc = fma_t(p[L * k], (T)a[k], acc);
        out[f] = acc;
    }
}

// out(i, r) = in[i*si + r*sr] as FP64 (I x R, column-major).
template <typename T>
__global__ void gather2d_kernel(const T* __restrict__ in, double* __restrict__ out, int64_t I, int R,
                                int64_t si, int64_t sr, const int* __restrict__ status)
{
    if (*status != kStatusOk) return;
    const int64_t total = I * R;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / I, i = e - r * I;
        out[e] = (double)in[i * si + r * sr];
    }
}

inline unsigned grid_for(int64_t n, int threads, int num_sms) {
    int64_t g = (n + threads - 1) / threads;
    const int64_t cap = (int64_t)num_sms * 16;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (unsigned)g;
}

template <typename T>
const T* x_ptr(Handle* h);
template <>
const double* x_ptr<double>(Handle* h) { return h->X64; }
template <>
const float* x_ptr<float>(Handle* h) { return h->X32; }

// The BF16X3 and TF32X3 precisions run the first TTM (the pass over X) on the
// tensor cores when the rank fills an MMA tile (R >= 16); otherwise FP32 FMA.
template <typename T>
bool first_on_tensor_cores(const Handle* h)
{
    return sizeof(T) == 4 && (h->prec == CPALS_BF16X3 || h->prec == CPALS_TF32X3) && tc_supported(h->R);
}

// Contract the listed modes of `in` (current dims d, updated in place) with
// Q_m^T, largest original dim first (ties: higher mode), ping-ponging through
// the two TTM buffers.  The last TTM writes to final_out when given.  With
// from_x the first TTM reads X and may run on the tensor cores.  *result
// receives the tensor that holds the contraction (in itself if nm == 0).
template <typename T>
cudaError_t ttm_chain(Handle* h, const T* in, int64_t* d, const int* modes_in, int nm, const double* const* Q,
                      bool from_x, T* final_out, const T** result)
{
    const int N = h->N, R = h->R;
    int modes[kMaxN];
    for (int k = 0; k < nm; ++k) modes[k] = modes_in[k];
    for (int a = 0; a < nm; ++a)
        for (int b = a + 1; b < nm; ++b) {
            const int x = modes[a], y = modes[b];
            if (h->dims[y] > h->dims[x] || (h->dims[y] == h->dims[x] && y > x)) { modes[a] = y; modes[b] = x; }
        }
    int cur = 0;
    for (int k = 0; k < nm; ++k) {
        const int m = modes[k];
        const TtmShape s = ttm_shape(N, d, m);
        T* out = (k == nm - 1 && final_out) ? final_out : (T*)h->tbuf[cur];
        if (k == 0 && from_x && first_on_tensor_cores<T>(h))
            CPALS_CUDA_TRY(ttm_split_tc(h, (const float*)in, Q[m], h->dims[m], (float*)out, s, R,
                                        h->prec == CPALS_TF32X3));
        else
            CPALS_CUDA_TRY(launch_ttm<T>(h, in, Q[m], h->dims[m], out, s, R));
        d[m] = R;
        in = out;
        cur ^= 1;
    }
    *result = in;
    return cudaSuccess;
}

// Final Multi-TTM tensor of mode n (R in every other mode) to the unfolding
// Y_(n): FP64 into h->Yn, or -- for an FP32 Multi-TTM inside a mode update
// with h->yn32_mode -- FP32 into the TTM buffer that does not hold `in`
// (h->yn32), for W = Y_(n) Q0 in FP32.
template <typename T>
cudaError_t unfold_yn(Handle* h, const T* in, int n)
{
    int64_t Rn = 1;
    for (int m = 0; m < n; ++m) Rn *= h->R;
    const int64_t total = h->dims[n] * h->RN1;
    if constexpr (sizeof(T) == 4) {
        if (h->yn32_mode) {
            float* out = (in == (const T*)h->tbuf[0]) ? (float*)h->tbuf[1] : (float*)h->tbuf[0];
            unfold32_kernel<<<grid_for(total, 256, h->num_sms), 256, 0, h->stream>>>(in, out, Rn, h->dims[n], total,
                                                                                    h->d_status);
            h->launches++;
            h->yn32 = out;
            return cudaGetLastError();
        }
    }
    h->yn32 = nullptr;
    unfold_kernel<T><<<grid_for(total, 256, h->num_sms), 256, 0, h->stream>>>(in, h->Yn, Rn, h->dims[n], total,
                                                                               h->d_status);
    h->launches++;
    return cudaGetLastError();
}

template <typename T>
cudaError_t multi_ttm_impl(Handle* h, int n, const double* const* Q)
{
    int modes[kMaxN], nm = 0;
    for (int m = 0; m < h->N; ++m)
        if (m != n) modes[nm++] = m;
    int64_t d[kMaxN];
    for (int m = 0; m < h->N; ++m) d[m] = h->dims[m];
    const T* res = nullptr;
    CPALS_CUDA_TRY(ttm_chain<T>(h, x_ptr<T>(h), d, modes, nm, Q, true, nullptr, &res));
    return unfold_yn<T>(h, res, n);
}

// Dimension tree (Sec. 3.3.3): X contracted over `modes` into h->tA.
template <typename T>
cudaError_t dimtree_pass_impl(Handle* h, const int* modes, int nm)
{
    for (int m = 0; m < h->N; ++m) h->tA_dims[m] = h->dims[m];
    const T* res = nullptr;
    return ttm_chain<T>(h, x_ptr<T>(h), h->tA_dims, modes, nm, h->Q, true, (T*)h->tA, &res);
}

// Y_(n) from the shared partial h->tA: contract the modes that the pass left
// uncontracted, other than n, with their current Q_m.
template <typename T>
cudaError_t multi_ttm_from_partial_impl(Handle* h, int n)
{
    int modes[kMaxN], nm = 0;
    int64_t d[kMaxN];
    for (int m = 0; m < h->N; ++m) {
        d[m] = h->tA_dims[m];
        if (m != n && !h->tA_contracted[m]) modes[nm++] = m;
    }
    const T* res = nullptr;
    CPALS_CUDA_TRY(ttm_chain<T>(h, (const T*)h->tA, d, modes, nm, h->Q, false, nullptr, &res));
    return unfold_yn<T>(h, res, n);
}

// MTTKRP contractions (Alg. cp-als): the first contraction of X over a mode c
// is a full TTM with A_c (cost 2 P R), after which the rank index r sits in
// the place of mode c; every later mode m is contracted diagonally with
// A_m(:, r) and leaves a dimension of 1.  `rank_pos` is -1 before the first
// contraction.  The modes go largest first (ties: higher mode), like the
// TTMs of the Multi-TTM.  The last contraction writes to final_out when given.
template <typename T>
cudaError_t mttkrp_chain(Handle* h, const T* in, int64_t* d, const int* modes_in, int nm, int* rank_pos, bool from_x,
                         T* final_out, const T** result)
{
    const int N = h->N, R = h->R;
    int modes[kMaxN];
    for (int k = 0; k < nm; ++k) modes[k] = modes_in[k];
    for (int a = 0; a < nm; ++a)
        for (int b = a + 1; b < nm; ++b) {
            const int x = modes[a], y = modes[b];
            if (h->dims[y] > h->dims[x] || (h->dims[y] == h->dims[x] && y > x)) { modes[a] = y; modes[b] = x; }
        }
    int cur = 0;
    for (int k = 0; k < nm; ++k) {
        const int m = modes[k];
        const TtmShape s = ttm_shape(N, d, m);
        T* out = (k == nm - 1 && final_out) ? final_out : (T*)h->tbuf[cur];
        if (*rank_pos < 0) {
            if (from_x && first_on_tensor_cores<T>(h))
                CPALS_CUDA_TRY(ttm_split_tc(h, (const float*)in, h->A[m], h->dims[m], (float*)out, s, R,
                                            h->prec == CPALS_TF32X3));
            else
                CPALS_CUDA_TRY(launch_ttm<T>(h, in, h->A[m], h->dims[m], out, s, R));
            d[m] = R;
            *rank_pos = m;
        } else {
            const int c = *rank_pos;
            int64_t div = 1;
            int r_in_l;
            if (c < m) { r_in_l = 1; for (int q = 0; q < c; ++q) div *= d[q]; }
            else { r_in_l = 0; for (int q = m + 1; q < c; ++q) div *= d[q]; }
            const int64_t rows = s.L * s.T;
            diag_contract_kernel<T><<<grid_for(rows, 256, h->num_sms), 256, 0, h->stream>>>(
                in, h->A[m], h->dims[m], out, s.L, s.K, s.T, r_in_l, div, R, h->d_status);
            h->launches++;
            CPALS_CUDA_TRY(cudaGetLastError());
            d[m] = 1;
        }
        in = out;
        cur ^= 1;
    }
    *result = in;
    return cudaSuccess;
}

// M_n(i, r) from a tensor whose dims are I_n at n, R at the rank position c
// and 1 elsewhere.
template <typename T>
cudaError_t mttkrp_gather(Handle* h, const T* in, const int64_t* d, int n, int c)
{
    int64_t sn = 1, sc = 1;
    for (int q = 0; q < n; ++q) sn *= d[q];
    for (int q = 0; q < c; ++q) sc *= d[q];
    gather2d_kernel<T><<<grid_for(h->dims[n] * h->R, 256, h->num_sms), 256, 0, h->stream>>>(
        in, h->M, h->dims[n], h->R, sn, sc, h->d_status);
    h->launches++;
    return cudaGetLastError();
}

template <typename T>
cudaError_t mttkrp_impl(Handle* h, int n)
{
    int modes[kMaxN], nm = 0;
    int64_t d[kMaxN];
    for (int m = 0; m < h->N; ++m) {
        d[m] = h->dims[m];
        if (m != n) modes[nm++] = m;
    }
    int c = -1;
    const T* res = nullptr;
    CPALS_CUDA_TRY(mttkrp_chain<T>(h, x_ptr<T>(h), d, modes, nm, &c, true, nullptr, &res));
    return mttkrp_gather<T>(h, res, d, n, c);
}

// Dimension tree for the normal equations: X contracted over `modes` (one
// half) into h->tA, the rank index at h->tA_rank.
template <typename T>
cudaError_t mttkrp_tree_pass_impl(Handle* h, const int* modes, int nm)
{
    for (int m = 0; m < h->N; ++m) h->tA_dims[m] = h->dims[m];
    int c = -1;
    const T* res = nullptr;
    CPALS_CUDA_TRY(mttkrp_chain<T>(h, x_ptr<T>(h), h->tA_dims, modes, nm, &c, true, (T*)h->tA, &res));
    h->tA_rank = c;
    return cudaSuccess;
}

// M_n from the partial: the uncontracted modes other than n, with their current A_m.
template <typename T>
cudaError_t mttkrp_from_partial_impl(Handle* h, int n)
{
    int modes[kMaxN], nm = 0;
    int64_t d[kMaxN];
    for (int m = 0; m < h->N; ++m) {
        d[m] = h->tA_dims[m];
        if (m != n && !h->tA_contracted[m]) modes[nm++] = m;
    }
    int c = h->tA_rank;
    const T* res = (const T*)h->tA;
    CPALS_CUDA_TRY(mttkrp_chain<T>(h, (const T*)h->tA, d, modes, nm, &c, false, nullptr, &res));
    return mttkrp_gather<T>(h, res, d, n, c);
}

// ---------------------------------------------------------------- reductions
// Deterministic two-phase sum: fixed grid, per-block tree, then one block.
constexpr int kRedBlocks = 1024;

__device__ __forceinline__ double block_sum(double v, double* sh)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) sh[w] = v;
    __syncthreads();
    if (w == 0) {
        v = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    }
    return v;
}

template <typename T>
__global__ void sumsq_partial_kernel(const T* __restrict__ x, int64_t n, double* __restrict__ part)
{
    __shared__ double sh[32];
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = (double)x[i];
        s = fma(v, v, s);
    }
    s = block_sum(s, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void sum_final_kernel(const double* __restrict__ part, int n, double* __restrict__ out)
{
    __shared__ double sh[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += part[i];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) *out = s;
}

// (X - Xhat)^2 summed, Xhat(i) = sum_r lambda_r prod_m A_m(i_m, r).
struct FactorPtrs {
    const double* A[kMaxN];
    int64_t dims[kMaxN];
};

template <typename T>
__global__ void residual_partial_kernel(const T* __restrict__ x, int64_t P, int N, int R, FactorPtrs f,
                                        const double* __restrict__ lambda, double* __restrict__ part)
{
    __shared__ double sh[32];
    double s = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < P; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t idx[kMaxN];
        int64_t rem = e;
        for (int m = 0; m < N; ++m) { idx[m] = rem % f.dims[m]; rem /= f.dims[m]; }
        double xh = 0.0;
        for (int r = 0; r < R; ++r) {
            double p = lambda[r];
            for (int m = 0; m < N; ++m) p *= f.A[m][idx[m] + f.dims[m] * r];
            xh += p;
        }
        const double dlt = (double)x[e] - xh;
        s = fma(dlt, dlt, s);
    }
    s = block_sum(s, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void cast_kernel(const double* __restrict__ src, float* __restrict__ dst, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = __double2float_rn(src[i]);
}

}  // namespace

cudaError_t dimtree_pass(Handle* h, const int* modes, int nm)
{
    for (int m = 0; m < h->N; ++m) h->tA_contracted[m] = 0;
    for (int k = 0; k < nm; ++k) h->tA_contracted[modes[k]] = 1;
    if (h->prec == CPALS_F64) return dimtree_pass_impl<double>(h, modes, nm);
    return dimtree_pass_impl<float>(h, modes, nm);
}

cudaError_t multi_ttm_from_partial(Handle* h, int n)
{
    if (h->prec == CPALS_F64) return multi_ttm_from_partial_impl<double>(h, n);
    return multi_ttm_from_partial_impl<float>(h, n);
}

cudaError_t multi_ttm(Handle* h, int n, const double* const* Q)
{
    if (h->prec == CPALS_F64) return multi_ttm_impl<double>(h, n, Q);
    return multi_ttm_impl<float>(h, n, Q);
}

// W_n = Y_(n) Q0 (Eq. ls-qr-q0-step).  After an FP32 Multi-TTM with the
// FP32 unfolding (h->yn32), the product runs in FP32 like the contractions
// before it (one more TTM, K = R^{N-1}) and W is widened to FP64 for the
// solve; otherwise FP64 from h->Yn.
cudaError_t apply_q0(Handle* h, int n)
{
    const int64_t In = h->dims[n];
    if (h->yn32) {
        // few rows and a long K: the row kernels with K split over the SMs
        // (the TMA-ring kernel keeps one CTA per row tile)
        const TtmShape s{In, h->RN1, 1};
        CPALS_CUDA_TRY(launch_ttm_split<float>(h, h->yn32, h->Q0, h->RN1, h->W32, s, h->R, (float*)h->scratch,
                                               h->scratch_elems * 2));
        const int64_t total = In * h->R;
        widen_kernel<<<grid_for(total, 256, h->num_sms), 256, 0, h->stream>>>(h->W32, h->W, total, h->d_status);
        h->launches++;
        h->yn32 = nullptr;
        return cudaGetLastError();
    }
    return gemm_rows(h, h->Yn, In, h->RN1, h->Q0, h->R, h->W);
}

// C (m x n) = A (m x k) B (k x n), column-major FP64: a TTM with L = m,
// K = k, T = 1 (rows of A are the output rows), with the same split-K.
cudaError_t gemm_rows(Handle* h, const double* A, int64_t m, int64_t k, const double* B, int n, double* C)
{
    TtmShape s{m, k, 1};
    return launch_ttm<double>(h, A, B, k, C, s, n);
}

cudaError_t ttm_first(Handle* h, int n)
{
    int order[kMaxN];
    ttm_order(h->N, h->dims, n, order);
    const TtmShape s = ttm_shape(h->N, h->dims, order[0]);
    if (h->prec == CPALS_F64)
        return launch_ttm<double>(h, h->X64, h->Q[order[0]], h->dims[order[0]], (double*)h->tbuf[0], s, h->R);
    if (first_on_tensor_cores<float>(h))
        return ttm_split_tc(h, h->X32, h->Q[order[0]], h->dims[order[0]], (float*)h->tbuf[0], s, h->R,
                            h->prec == CPALS_TF32X3);
    return launch_ttm<float>(h, h->X32, h->Q[order[0]], h->dims[order[0]], (float*)h->tbuf[0], s, h->R);
}

cudaError_t mttkrp(Handle* h, int n)
{
    if (h->prec == CPALS_F64) return mttkrp_impl<double>(h, n);
    return mttkrp_impl<float>(h, n);
}

cudaError_t mttkrp_tree_pass(Handle* h, const int* modes, int nm)
{
    for (int m = 0; m < h->N; ++m) h->tA_contracted[m] = 0;
    for (int k = 0; k < nm; ++k) h->tA_contracted[modes[k]] = 1;
    if (h->prec == CPALS_F64) return mttkrp_tree_pass_impl<double>(h, modes, nm);
    return mttkrp_tree_pass_impl<float>(h, modes, nm);
}

cudaError_t mttkrp_from_partial(Handle* h, int n)
{
    if (h->prec == CPALS_F64) return mttkrp_from_partial_impl<double>(h, n);
    return mttkrp_from_partial_impl<float>(h, n);
}

cudaError_t norm2(Handle* h)
{
    if (h->X64) sumsq_partial_kernel<double><<<kRedBlocks, 256, 0, h->stream>>>(h->X64, h->P, h->scratch);
    else sumsq_partial_kernel<float><<<kRedBlocks, 256, 0, h->stream>>>(h->X32, h->P, h->scratch);
    sum_final_kernel<<<1, 1024, 0, h->stream>>>(h->scratch, kRedBlocks, h->d_normX2);
    h->launches += 2;
    return cudaGetLastError();
}

cudaError_t residual_direct(Handle* h, double* d_out)
{
    FactorPtrs f;
    for (int m = 0; m < h->N; ++m) { f.A[m] = h->A[m]; f.dims[m] = h->dims[m]; }
    if (h->X64)
        residual_partial_kernel<double><<<kRedBlocks, 256, 0, h->stream>>>(h->X64, h->P, h->N, h->R, f, h->lambda,
                                                                           h->scratch);
    else
        residual_partial_kernel<float><<<kRedBlocks, 256, 0, h->stream>>>(h->X32, h->P, h->N, h->R, f, h->lambda,
                                                                          h->scratch);
    sum_final_kernel<<<1, 1024, 0, h->stream>>>(h->scratch, kRedBlocks, d_out);
    h->launches += 2;
    return cudaGetLastError();
}

cudaError_t cast_f64_f32(Handle* h, const double* src, float* dst, int64_t n)
{
    cast_kernel<<<grid_for(n, 256, h->num_sms), 256, 0, h->stream>>>(src, dst, n);
    h->launches++;
    return cudaGetLastError();
}


// ---------------------------------------------------------------- no-allocation Multi-TTM
// Scratch for cpals_multi_ttm_static: the TTM intermediates and split-K
// partials live in this fixed array, so that entry point never allocates.
// Every GPU that loads the library holds it (16 MiB) until the process exits.
constexpr int64_t kStaticScratchDoubles = int64_t(1) << 21;
static __device__ __align__(256) double g_static_scratch[kStaticScratchDoubles];
static __device__ __align__(256) int g_static_status[1];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_static_mutex;
double* g_static_scratch_ptr[kMaxDevices] = {nullptr};
int* g_static_status_ptr[kMaxDevices] = {nullptr};

// Device addresses of the static arrays for the current device (set up once
// per device, with that device current).
cudaError_t static_scratch(int device, double** scratch, int** status)
{
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_static_mutex);
    if (!g_static_scratch_ptr[device]) {
        void* p = nullptr;
        void* q = nullptr;
        CPALS_CUDA_TRY(cudaGetSymbolAddress(&p, g_static_scratch));
        CPALS_CUDA_TRY(cudaGetSymbolAddress(&q, g_static_status));
        g_static_scratch_ptr[device] = static_cast<double*>(p);
        g_static_status_ptr[device] = static_cast<int*>(q);
    }
    *scratch = g_static_scratch_ptr[device];
    *status = g_static_status_ptr[device];
    return cudaSuccess;
}

}  // namespace

int64_t multi_ttm_static_capacity() { return kStaticScratchDoubles; }

cudaError_t multi_ttm_static(int N, const int64_t* dims, int R, int n, const double* X, const double* const* Q,
                             double* Y, cudaStream_t stream)
{
    int device = 0;
    CPALS_CUDA_TRY(cudaGetDevice(&device));
    double* scratch = nullptr;
    int* status = nullptr;
    CPALS_CUDA_TRY(static_scratch(device, &scratch, &status));
    Handle h;                       // launch context only: no buffers are allocated
    h.N = N;
    h.R = R;
    h.stream = stream;
    for (int m = 0; m < N; ++m) h.dims[m] = dims[m];
    CPALS_CUDA_TRY(cudaDeviceGetAttribute(&h.num_sms, cudaDevAttrMultiProcessorCount, device));
    h.d_status = status;
    // the scratch layout, with every TTM's split-K partials and group sums
    // inside the array (the caller has checked sp.ok on the same dims)
    const StaticPlan sp = plan_multi_ttm_static(N, dims, R, n, h.num_sms, kStaticScratchDoubles);
    if (!sp.ok) return cudaErrorInvalidValue;
    // the kernels skip their work unless the status word is zero
    CPALS_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int), stream));

    int order[kMaxN];
    ttm_order(N, dims, n, order);
    int64_t d[kMaxN];
    for (int m = 0; m < N; ++m) d[m] = dims[m];
    double* buf[2] = {scratch, scratch + sp.s0};
    double* part = scratch + sp.s0 + sp.s1;
    const double* in = X;
    int cur = 0;
    for (int k = 0; k < N - 1; ++k) {
        const int m = order[k];
        const TtmShape s = ttm_shape(N, d, m);
        CPALS_CUDA_TRY(launch_ttm_split<double>(&h, in, Q[m], dims[m], buf[cur], s, R, part, sp.part_elems));
        d[m] = R;
        in = buf[cur];
        cur ^= 1;
    }
    int64_t Rn = 1;
    for (int m = 0; m < n; ++m) Rn *= R;
    int64_t RN1 = 1;
    for (int m = 0; m < N - 1; ++m) RN1 *= R;
    const int64_t total = dims[n] * RN1;
    unfold_kernel<double><<<grid_for(total, 256, h.num_sms), 256, 0, stream>>>(in, Y, Rn, dims[n], total, status);
    return cudaGetLastError();
}

// The static Multi-TTM's plan on the current device (for the size check of
// the C-ABI entry point).
cudaError_t multi_ttm_static_plan(int N, const int64_t* dims, int R, int n, StaticPlan* out)
{
    int device = 0, sms = 0;
    CPALS_CUDA_TRY(cudaGetDevice(&device));
    CPALS_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    *out = plan_multi_ttm_static(N, dims, R, n, sms, kStaticScratchDoubles);
    return cudaSuccess;
}

}  // namespace cpals
