// tc_bf16x3.cu -- the first TTM of the Multi-TTM (the pass that streams X) on
// the tcgen05 tensor cores, for the BF16X3 precision:
//     Out(l, r, t) = sum_k X(l, k, t) * Q(k, r)            (Y = X x_m Q_m^T)
// X is the FP32 copy of the tensor.  Each x and each q are split into bf16
// parts, x = x_hi + x_lo (x_hi = bf16(x), x_lo = bf16(x - x_hi)), and
// x*q ~ x_hi*q_hi + x_hi*q_lo + x_lo*q_hi.  Three MMAs per K step accumulate the
// products (exact in FP32) into one FP32 accumulator in tensor memory.  The
// dropped x_lo*q_lo term and the rounding of the lo parts leave a relative error
// of about 2^-16 per product.
//
// Tiling: a CTA of 128 threads owns 128 consecutive flattened rows f = l + L*t
// (M = 128) and all R outputs (N = R rounded up to a multiple of 16).  It walks
// K in chunks of 64.  Per chunk every thread loads the 64 FP32 values of its
// row (coalesced across the warp for each k), splits them, and writes the hi and
// lo parts into shared memory in the K-major no-swizzle canonical layout:
// 8-row x 16-byte core matrices, K-adjacent cores 128 B apart (LBO), 8-row
// groups 1024 B apart (SBO).  Q's chunk is split the same way.  One thread
// then issues 4 K-steps x 3 tcgen05.mma (kind::f16, bf16 x bf16 -> f32,
// M=128) and commits them to an mbarrier.  The next chunk waits on it before it
// overwrites the operands.  Several CTAs per SM overlap their loads with each
// other's MMAs.  The epilogue reads the accumulator with tcgen05.ld (one warp
// per 32 TMEM lanes) and stores the R valid columns.
//
// Every wait is bounded.  On timeout the kernel records CPALS_ERR_TIMEOUT in
// the status word, frees its tensor memory and returns.
#include <cuda_bf16.h>

#include <algorithm>

#include "internal.cuh"

namespace cpals {

namespace {

constexpr int kTcRows = 128;     // M
constexpr int kTcKChunk = 64;    // K per shared-memory stage
constexpr int kTcThreads = 128;
constexpr uint32_t kSbo = 1024;  // bytes between 8-row core groups (K chunk of 64 bf16 = 8 cores x 128 B)
constexpr uint32_t kLbo = 128;   // bytes between K-adjacent core matrices

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor: start address, LBO and SBO in 16-byte
// units, descriptor version 1 (bit 46), no swizzle (bits 61-63 = 0).
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((kLbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((kSbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor, kind::f16: D f32 (bits 4-5 = 1), A bf16 (bits 7-9 = 1),
// B bf16 (bits 10-12 = 1), A and B K-major (bits 15, 16 = 0), N>>3 at bits
// 17-22, M>>4 at bits 24-28.
__host__ __device__ constexpr uint32_t make_idesc(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
        :
        : "r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :
                 : "r"(smem_u32(mbar))
                 : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* mbar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" : : "r"(smem_u32(mbar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* mbar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(mbar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait on an mbarrier phase: false after ~2^24 failed polls.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* mbar, uint32_t parity)
{
    for (uint32_t it = 0; it < (1u << 24); ++it) {
        if (mbar_try_wait(mbar, parity)) return true;
        if (it > 64) __nanosleep(64);
    }
    return false;
}

template <int NCOLS>
__device__ __forceinline__ void tmem_alloc(uint32_t* dst)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :
                 : "r"(smem_u32(dst)), "r"((uint32_t)NCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

template <int NCOLS>
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" : : "r"(taddr), "r"((uint32_t)NCOLS)
                 : "memory");
}

__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// 16 consecutive f32 accumulator columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v)
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 a, __nv_bfloat16 b)
{
    return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

// Byte offset of element (row, k) of a [rows x 64] K-major no-swizzle tile.
__device__ __forceinline__ uint32_t tile_off(int row, int k)
{
    return (uint32_t)(row >> 3) * kSbo + (uint32_t)(k >> 3) * kLbo + (uint32_t)(row & 7) * 16u + (uint32_t)(k & 7) * 2u;
}

template <int N>
struct TcCfg {
    static constexpr int kNcols = (N <= 32) ? 32 : (N <= 64 ? 64 : 128);   // TMEM columns (power of 2 >= 32)
    static constexpr uint32_t kABytes = kTcRows * kTcKChunk * 2;          // one bf16 A tile (16 KB)
    static constexpr uint32_t kBBytes = N * kTcKChunk * 2;                // one bf16 B tile
    static constexpr uint32_t kSmem = 2 * kABytes + 2 * kBBytes + 64 + 1024;  // + barrier/tmem slot + alignment
};

template <int N>
__global__ void __launch_bounds__(kTcThreads) ttm_bf16x3_kernel(
    const float* __restrict__ in, const double* __restrict__ Q, int64_t ldq, float* __restrict__ out, int64_t L,
    int64_t K, int64_t Tn, int R, int* __restrict__ status)
{
    using Cfg = TcCfg<N>;
    if (*status != kStatusOk) return;
    extern __shared__ uint8_t smem_raw[];
    // 1024-byte aligned operand tiles
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* a_hi = smem;
    uint8_t* a_lo = a_hi + Cfg::kABytes;
    uint8_t* b_hi = a_lo + Cfg::kABytes;
    uint8_t* b_lo = b_hi + Cfg::kBBytes;
    uint64_t* mbar = (uint64_t*)(b_lo + Cfg::kBBytes);
    uint32_t* tmem_slot = (uint32_t*)(mbar + 1);
    __shared__ int timed_out;

    const int tid = threadIdx.x, warp = tid >> 5;
    const int64_t rows = L * Tn;
    const int64_t f = (int64_t)blockIdx.x * kTcRows + tid;
    const bool active = f < rows;
    int64_t t = 0, l = 0;
    if (active) { t = f / L; l = f - t * L; }
    const float* p = in + l + L * K * t;

    if (warp == 0) tmem_alloc<Cfg::kNcols>(tmem_slot);
    if (tid == 0) {
        mbar_init(mbar, 1);
        fence_mbar_init();
        timed_out = 0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    constexpr uint32_t idesc = make_idesc(kTcRows, N);

    uint32_t phase = 0;
    bool first = true;
    for (int64_t k0 = 0; k0 < K; k0 += kTcKChunk) {
        const int kc = (int)std::min<int64_t>(kTcKChunk, K - k0);
        // --- A: this thread's row, 64 k values, split into hi/lo, K-major canonical layout
#pragma unroll
        for (int g = 0; g < kTcKChunk / 8; ++g) {
            float x[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int k = g * 8 + e;
                x[e] = (active && k < kc) ? __ldg(p + L * (k0 + k)) : 0.0f;
            }
            uint32_t hi[4], lo[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const __nv_bfloat16 h0 = __float2bfloat16_rn(x[2 * e]);
                const __nv_bfloat16 h1 = __float2bfloat16_rn(x[2 * e + 1]);
                const __nv_bfloat16 l0 = __float2bfloat16_rn(x[2 * e] - __bfloat162float(h0));
                const __nv_bfloat16 l1 = __float2bfloat16_rn(x[2 * e + 1] - __bfloat162float(h1));
                hi[e] = pack2(h0, h1);
                lo[e] = pack2(l0, l1);
            }
            const uint32_t off = tile_off(tid, g * 8);
            *reinterpret_cast<uint4*>(a_hi + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
            *reinterpret_cast<uint4*>(a_lo + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
        }
        // --- B: Q(k0 + k, n) for n < N (zero past R and past kc), split the same way
        for (int u = tid; u < N * (kTcKChunk / 8); u += kTcThreads) {
            const int n = u / (kTcKChunk / 8), g = u - n * (kTcKChunk / 8);
            uint32_t hi[4], lo[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                __nv_bfloat16 hv[2], lv[2];
#pragma unroll
                for (int s = 0; s < 2; ++s) {
                    const int k = g * 8 + 2 * e + s;
                    const double q = (n < R && k < kc) ? Q[(k0 + k) + ldq * (int64_t)n] : 0.0;
                    hv[s] = __double2bfloat16(q);
                    lv[s] = __double2bfloat16(q - (double)__bfloat162float(hv[s]));
                }
                hi[e] = pack2(hv[0], hv[1]);
                lo[e] = pack2(lv[0], lv[1]);
            }
            const uint32_t off = tile_off(n, g * 8);
            *reinterpret_cast<uint4*>(b_hi + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
            *reinterpret_cast<uint4*>(b_lo + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
        }
        fence_proxy_async();          // generic-proxy smem writes -> visible to the tensor core
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            const uint32_t ah = smem_u32(a_hi), al = smem_u32(a_lo), bh = smem_u32(b_hi), bl = smem_u32(b_lo);
#pragma unroll
            for (int ks = 0; ks < kTcKChunk / 16; ++ks) {
                const uint32_t step = (uint32_t)ks * 2u * kLbo;     // 16 K elements = 2 core matrices
                mma_bf16(tmem, make_desc(ah + step), make_desc(bh + step), idesc, first ? 0u : 1u);
                mma_bf16(tmem, make_desc(ah + step), make_desc(bl + step), idesc, 1u);
                mma_bf16(tmem, make_desc(al + step), make_desc(bh + step), idesc, 1u);
                first = false;
            }
            mma_commit(mbar);
        }
        first = false;
        // the next chunk overwrites the operands: wait for these MMAs (bounded)
        if (!mbar_wait_bounded(mbar, phase)) {
            timed_out = 1;
            mbar_wait_bounded(mbar, phase);   // once more (bounded) for MMAs still in flight
        }
        phase ^= 1u;
        __syncthreads();
        if (timed_out) break;
    }
    tc_fence_after();
    if (!timed_out) {
        // epilogue: warp w reads TMEM lanes 32w..32w+31 (its rows), N columns
#pragma unroll
        for (int c0 = 0; c0 < N; c0 += 16) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            if (active) {
                float* o = out + l + L * (int64_t)R * t;
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    if (c0 + j < R) o[L * (int64_t)(c0 + j)] = v[j];
            }
        }
    } else if (tid == 0) {
        atomicCAS(status, kStatusOk, (int)CPALS_ERR_TIMEOUT);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc<Cfg::kNcols>(tmem);
}

template <int N>
cudaError_t launch_tc(Handle* h, const float* in, const double* Q, int64_t ldq, float* out, TtmShape s, int R)
{
    using Cfg = TcCfg<N>;
    static bool attr = false;
    if (!attr) {
        CPALS_CUDA_TRY(cudaFuncSetAttribute(ttm_bf16x3_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)Cfg::kSmem));
        attr = true;
    }
    const int64_t rows = s.L * s.T;
    const int64_t grid = (rows + kTcRows - 1) / kTcRows;
    ttm_bf16x3_kernel<N><<<(unsigned)grid, kTcThreads, Cfg::kSmem, h->stream>>>(in, Q, ldq, out, s.L, s.K, s.T, R,
                                                                                h->d_status);
    h->launches++;
    return cudaGetLastError();
}

}  // namespace

bool tc_supported(int R) { return R >= 16 && R <= 64; }

cudaError_t ttm_bf16x3(Handle* h, const float* in, const double* Q, int64_t ldq, float* out, TtmShape s, int R)
{
    if (s.L * s.T == 0) return cudaSuccess;
    if (R <= 16) return launch_tc<16>(h, in, Q, ldq, out, s, R);
    if (R <= 32) return launch_tc<32>(h, in, Q, ldq, out, s, R);
    if (R <= 48) return launch_tc<48>(h, in, Q, ldq, out, s, R);
    return launch_tc<64>(h, in, Q, ldq, out, s, R);
}

}  // namespace cpals
