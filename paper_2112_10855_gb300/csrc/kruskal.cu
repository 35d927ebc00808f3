// kruskal.cu -- CP-ALS-QR / CP-ALS on a tensor given in Kruskal form
// (Sec. 3.3.2): X = sum_s mu_s v_s^(1) o ... o v_s^(N), with V_m (I_m x S).
// The dense tensor is never formed.
//
// Multi-TTM: Y = X x_{m != n} Q_m^T is again a Kruskal tensor, with factors
// C_m = Q_m^T V_m (R x S) for m != n and V_n, so
//     W_n = Y_(n) Q0 = V_n diag(mu) [ (C_{m_last} (.) ... (.) C_{m_0})^T Q0 ],
// an MTTKRP of Q0 (viewed as an R x ... x R x R tensor) followed by a small
// product (Sec. 3.3.2).  Q0 is never formed either: the QR of V_n is built by
// the Kronecker fold (Eq. kr-id), Q0 = (I (x) Q_{k-1}) P_k recursively, and
// (c_i (x) c')^T (I (x) Q) = c_i (x) (c'^T Q) column by column, so the
// bracket is obtained by the recursion
//     M_0(s, j) = C_{m_0}(j, s),
//     M_k(s, c) = sum_{i, j} C_{m_k}(i, s) M_{k-1}(s, j) P_k(i R + j, c),
// at O(N S R^3) instead of O(R^N S).  The MTTKRP of the normal-equations
// baseline is V_n diag(mu) (*_{m != n} V_m^T A_m) (Hadamard product).
// ||X||^2 = mu^T (*_m V_m^T V_m) mu.
//
// All arithmetic is FP64; every sum runs in a fixed order.
#include <algorithm>

#include "internal.cuh"

namespace cpals {

namespace {

__device__ __forceinline__ double warp_sum_d(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// out(a, b) = sum_i A(i, a) B(i, b) for a < na, b < nb (A: I x na, B: I x nb,
// column-major with leading dimension I); one warp per output element.
__global__ void atb_kernel(const double* __restrict__ A, const double* __restrict__ B, int64_t I, int na, int nb,
                           double* __restrict__ out, const int* __restrict__ status)
{
    if (*status != kStatusOk) return;
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= (int64_t)na * nb) return;
    const int b = (int)(w / na), a = (int)(w - (int64_t)b * na);
    const double* pa = A + I * a;
    const double* pb = B + I * b;
    double s = 0.0;
    for (int64_t i = lane; i < I; i += 32) s = fma(pa[i], pb[i], s);
    s = warp_sum_d(s);
    if (lane == 0) out[a + (int64_t)na * b] = s;
}

struct KPtrs {
    const double* p[kMaxN];
};

// ||X||^2 = sum_{s,t} mu_s mu_t prod_m GV_m(s, t); one CTA, fixed order.
__global__ void kr_norm2_kernel(KPtrs gv, int N, const double* __restrict__ mu, int S, double* __restrict__ out,
                                const int* __restrict__ status)
{
    if (*status != kStatusOk) return;
    __shared__ double part[256];
    double acc = 0.0;
    for (int e = threadIdx.x; e < S * S; e += blockDim.x) {
        const int t = e / S, s = e - t * S;
        double v = mu[s] * mu[t];
        for (int m = 0; m < N; ++m) v *= gv.p[m][s + S * t];
        acc += v;
    }
    part[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < (int)blockDim.x; ++i) s += part[i];
        *out = s;
    }
}

// One step of the fold contraction: out(s, c) = sum_{i,j} Ck(i, s) prev(s, j) P(i R + j, c),
// with prev(s, j) = C0(j, s) when first (M_0 = C_{m_0}^T).
__global__ void kr_contract_kernel(const double* __restrict__ Ck, const double* __restrict__ prev, int first,
                                   const double* __restrict__ P, int R, int S, double* __restrict__ out,
                                   const int* __restrict__ status)
{
    if (*status != kStatusOk) return;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)S * R) return;
    const int c = (int)(e / S), s = (int)(e - (int64_t)c * S);
    double acc = 0.0;
    for (int i = 0; i < R; ++i) {
        const double ci = Ck[i + (int64_t)R * s];
        const double* pcol = P + (int64_t)R * R * c + (int64_t)i * R;
        double t = 0.0;
        for (int j = 0; j < R; ++j) {
            const double pj = first ? prev[j + (int64_t)R * s] : prev[s + (int64_t)S * j];
            t = fma(pj, pcol[j], t);
        }
        acc = fma(ci, t, acc);
    }
    out[s + (int64_t)S * c] = acc;
}

// H(s, c) = prod_{m != n} E_m(s, c)  (S x R)
__global__ void kr_hadamard_kernel(KPtrs E, int N, int n, int S, int R, double* __restrict__ H,
                                   const int* __restrict__ status)
{
    if (*status != kStatusOk) return;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= S * R) return;
    double v = 1.0;
    for (int m = 0; m < N; ++m)
        if (m != n) v *= E.p[m][e];
    H[e] = v;
}

// out(i, c) = sum_s V(i, s) mu_s M(s, c)  (I x R)
__global__ void kr_apply_kernel(const double* __restrict__ V, const double* __restrict__ mu,
                                const double* __restrict__ M, int64_t I, int S, int R, double* __restrict__ out,
                                const int* __restrict__ status)
{
    if (*status != kStatusOk) return;
    const int64_t total = I * R;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e / I, i = e - c * I;
        double acc = 0.0;
        for (int s = 0; s < S; ++s) acc = fma(V[i + I * s] * mu[s], M[s + (int64_t)S * c], acc);
        out[e] = acc;
    }
}

// Y_(n)(i, col) = sum_s V_n(i, s) mu_s prod_{m != n} C_m(r_m, s), with col =
// sum of r_m R^{pos(m)} over the modes m != n in ascending order (the lowest
// fastest).
__global__ void kr_unfold_kernel(const double* __restrict__ Vn, const double* __restrict__ mu, KPtrs C, int N,
                                 int n, int64_t In, int R, int S, int64_t RN1, double* __restrict__ Y,
                                 const int* __restrict__ status)
{
    if (*status != kStatusOk) return;
    const int64_t total = In * RN1;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t col = e / In, i = e - col * In;
        int r[kMaxN];
        int64_t q = col;
        for (int m = 0; m < N; ++m) {
            if (m == n) continue;
            r[m] = (int)(q % R);
            q /= R;
        }
        double acc = 0.0;
        for (int s = 0; s < S; ++s) {
            double v = Vn[i + In * s] * mu[s];
            for (int m = 0; m < N; ++m)
                if (m != n) v *= C.p[m][r[m] + (int64_t)R * s];
            acc += v;
        }
        Y[e] = acc;
    }
}

struct KrResidualArgs {
    const double* V[kMaxN];
    const double* A[kMaxN];
    int64_t dims[kMaxN];
};

// Partial sums of (x - xhat)^2 over contiguous ranges of the P entries, with
// x = sum_s mu_s prod_m V_m(i_m, s) and xhat = sum_r lambda_r prod_m A_m(i_m, r):
// the direct residual of Sec. 3.3.1 without forming either tensor.
__global__ void kr_residual_partial_kernel(KrResidualArgs a, int N, const double* __restrict__ mu, int S,
                                           const double* __restrict__ lambda, int R, int64_t P,
                                           double* __restrict__ part, const int* __restrict__ status)
{
    if (*status != kStatusOk) return;
    __shared__ double red[256];
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t chunk = (P + nthreads - 1) / nthreads;
    const int64_t b = t * chunk, e = std::min<int64_t>(P, b + chunk);
    double acc = 0.0;
    for (int64_t lin = b; lin < e; ++lin) {
        int64_t idx[kMaxN];
        int64_t q = lin;
        for (int m = 0; m < N; ++m) {
            idx[m] = q % a.dims[m];
            q /= a.dims[m];
        }
        double x = 0.0, xh = 0.0;
        for (int s = 0; s < S; ++s) {
            double v = mu[s];
            for (int m = 0; m < N; ++m) v *= a.V[m][idx[m] + a.dims[m] * s];
            x += v;
        }
        for (int r = 0; r < R; ++r) {
            double v = lambda[r];
            for (int m = 0; m < N; ++m) v *= a.A[m][idx[m] + a.dims[m] * r];
            xh += v;
        }
        const double d = x - xh;
        acc = fma(d, d, acc);
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void kr_sum_kernel(const double* __restrict__ part, int n, double* __restrict__ out,
                              const int* __restrict__ status)
{
    if (*status != kStatusOk) return;
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += part[i];
        *out = s;
    }
}

inline unsigned warps_grid(int64_t warps) { return (unsigned)std::max<int64_t>(1, (warps * 32 + 255) / 256); }

}  // namespace

cudaError_t kr_atb(Handle* h, const double* A, const double* B, int64_t I, int na, int nb, double* out)
{
    atb_kernel<<<warps_grid((int64_t)na * nb), 256, 0, h->stream>>>(A, B, I, na, nb, out, h->d_status);
    h->launches++;
    return cudaGetLastError();
}

cudaError_t kr_norm2(Handle* h)
{
    const int S = h->KS;
    KPtrs gv;
    for (int m = 0; m < h->N; ++m) {
        double* g = h->KGV + (size_t)m * S * S;
        CPALS_CUDA_TRY(kr_atb(h, h->KV[m], h->KV[m], h->dims[m], S, S, g));
        gv.p[m] = g;
    }
    kr_norm2_kernel<<<1, 256, 0, h->stream>>>(gv, h->N, h->Kmu, S, h->d_normX2, h->d_status);
    h->launches++;
    return cudaGetLastError();
}

cudaError_t kr_refresh_c(Handle* h, int m)
{
    return kr_atb(h, h->Q[m], h->KV[m], h->dims[m], h->R, h->KS, h->KC[m]);
}

cudaError_t kr_refresh_e(Handle* h, int m)
{
    return kr_atb(h, h->KV[m], h->A[m], h->dims[m], h->KS, h->R, h->KE[m]);
}

// W_n = V_n diag(mu) (C_{m_last} (.) ... (.) C_{m_0})^T Q0 from the fold factors
// of the QR of V_n (h->KP, written by krp_qr in implicit mode).
cudaError_t kr_apply_q0(Handle* h, int n)
{
    const int R = h->R, S = h->KS;
    int modes[kMaxN], cnt = 0;
    for (int m = 0; m < h->N; ++m)
        if (m != n) modes[cnt++] = m;
    const double* Mcur = nullptr;
    if (cnt == 1) {
        // V_n = R_{m_0}: Q0 is the R x R factor in KP
        CPALS_CUDA_TRY(kr_atb(h, h->KC[modes[0]], h->KP, R, S, R, h->KMw[0]));
        Mcur = h->KMw[0];
    } else {
        const double* prev = h->KC[modes[0]];
        int first = 1;
        for (int k = 1; k < cnt; ++k) {
            double* out = h->KMw[k & 1];
            kr_contract_kernel<<<(unsigned)((S * R + 127) / 128), 128, 0, h->stream>>>(
                h->KC[modes[k]], prev, first, h->KP + (size_t)(k - 1) * R * R * R, R, S, out, h->d_status);
            h->launches++;
            CPALS_CUDA_TRY(cudaGetLastError());
            prev = out;
            first = 0;
        }
        Mcur = prev;
    }
    const int64_t In = h->dims[n];
    const int64_t total = In * R;
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 16LL * h->num_sms));
    kr_apply_kernel<<<grid, 256, 0, h->stream>>>(h->KV[n], h->Kmu, Mcur, In, S, R, h->W, h->d_status);
    h->launches++;
    return cudaGetLastError();
}

// MTTKRP of the normal equations: M = V_n diag(mu) (*_{m != n} V_m^T A_m).
cudaError_t kr_mttkrp(Handle* h, int n)
{
    const int R = h->R, S = h->KS;
    KPtrs E;
    for (int m = 0; m < h->N; ++m) E.p[m] = h->KE[m];
    kr_hadamard_kernel<<<(unsigned)((S * R + 127) / 128), 128, 0, h->stream>>>(E, h->N, n, S, R, h->KMw[0],
                                                                                h->d_status);
    h->launches++;
    CPALS_CUDA_TRY(cudaGetLastError());
    const int64_t In = h->dims[n];
    const int64_t total = In * R;
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 16LL * h->num_sms));
    kr_apply_kernel<<<grid, 256, 0, h->stream>>>(h->KV[n], h->Kmu, h->KMw[0], In, S, R, h->M, h->d_status);
    h->launches++;
    return cudaGetLastError();
}

cudaError_t kr_unfold(Handle* h, int n, double* Y)
{
    KPtrs C;
    for (int m = 0; m < h->N; ++m) C.p[m] = h->KC[m];
    const int64_t total = h->dims[n] * h->RN1;
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 16LL * h->num_sms));
    kr_unfold_kernel<<<grid, 256, 0, h->stream>>>(h->KV[n], h->Kmu, C, h->N, n, h->dims[n], h->R, h->KS, h->RN1, Y,
                                                  h->d_status);
    h->launches++;
    return cudaGetLastError();
}

cudaError_t kr_residual(Handle* h, double* out)
{
    KrResidualArgs a;
    int64_t P = 1;
    for (int m = 0; m < h->N; ++m) {
        a.V[m] = h->KV[m];
        a.A[m] = h->A[m];
        a.dims[m] = h->dims[m];
        P *= h->dims[m];
    }
    const int blocks = std::max(1, std::min<int>(4 * h->num_sms, (int)((P + 255) / 256)));
    kr_residual_partial_kernel<<<blocks, 256, 0, h->stream>>>(a, h->N, h->Kmu, h->KS, h->lambda, h->R, P,
                                                              h->scratch, h->d_status);
    kr_sum_kernel<<<1, 32, 0, h->stream>>>(h->scratch, blocks, out, h->d_status);
    h->launches += 2;
    return cudaGetLastError();
}

}  // namespace cpals
