// tc_split.cu -- the first TTM of the Multi-TTM (Eq. multittm; the pass that
// streams X, which dominates a mode update at small rank, Sec. 3.2) on the
// tcgen05 tensor cores with split-precision products:
//     Out(l, r, t) = sum_k X(l, k, t) * Q(k, r)            (Y = X x_m Q_m^T)
// X is the FP32 copy of the tensor.  Each x and each q are split into two
// parts of the operand type, x = x_hi + x_lo (x_hi = round(x),
// x_lo = round(x - x_hi)), and x*q ~ x_hi*q_hi + x_hi*q_lo + x_lo*q_hi.  Three
// MMAs per K step accumulate the products (exact in FP32) into one FP32
// accumulator in tensor memory.
//   BF16X3 (kind::f16, bf16 parts of 8 significant bits): the dropped
//     x_lo*q_lo and the rounding of the lo parts leave ~2^-16 per product.
//   TF32X3 (kind::tf32, tf32 parts of 11 bits): ~2^-21 per product, the level
//     of FP32 arithmetic.
//
// Tiling: a CTA of 128 threads owns 128 consecutive flattened rows f = l + L*t
// (M = 128) and all R outputs (N = R rounded up to a multiple of 16).  It walks
// K in chunks of 128 bytes per row (64 bf16 or 32 tf32 values).  Operands live
// in shared memory in the K-major no-swizzle canonical layout: 8-row x 16-byte
// core matrices, K-adjacent cores 128 B apart (LBO), 8-row groups 1024 B apart
// (SBO).  Q_m is split once per launch into tiles already in that layout.
// Every thread splits two (4-row, 16-byte K group) units of X per chunk, loading
// four rows at once with 128-bit loads when L % 4 == 0.  Two stages are in
// flight: the loads of chunk c+1 are issued before the CTA waits on the MMAs
// of chunk c-1.  One thread issues the 3 tcgen05.mma per K step (M=128) and
// commits each chunk to that stage's mbarrier.  The epilogue reads the
// accumulator with tcgen05.ld (one warp per 32 TMEM lanes) and stores the R
// valid columns.
//
// Every wait is bounded.  On timeout the kernel records CPALS_ERR_TIMEOUT in
// the status word, frees its tensor memory and returns.
//
// A second, persistent kernel (ttm_split_tc_pipe_kernel, below) serves the
// shapes whose row stride L is a multiple of 4 floats: one CTA per SM walks a
// list of row tiles.  A producer warp streams X in [rows x K-chunk] boxes with
// the Tensor Memory Accelerator (cp.async.bulk.tensor) into a deep ring of
// shared-memory stages; eight split warps turn each box into hi/lo A operands
// written straight to tensor memory (tcgen05.st) and free the box at once; a
// second producer warp brings the pre-split Q tiles of each item
// (cp.async.bulk) into a short ring of operand slots; one thread issues the
// MMAs with A read from tensor memory; four epilogue warps drain a
// double-buffered accumulator while the next tile accumulates.
//
// The same TMA ring also feeds FP32 FMAs on the CUDA cores
// (ttm_f32_pipe_kernel, at the end): the FP32 precision's passes over X and
// the FP32 contractions of intermediates in the mixed precisions.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "internal.cuh"

namespace cpals {

namespace {

constexpr int kTcRows = 128;     // M
constexpr int kTcThreads = 128;
constexpr uint32_t kSbo = 1024;  // bytes between 8-row core groups (a 128-byte K chunk = 8 cores x 128 B)
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

// Operand element type of the split: bf16 (kind::f16) or tf32 (kind::tf32).
// A K-chunk is 128 bytes of one row (64 bf16 or 32 tf32), so both share one
// byte layout: 8 core matrices of 16 bytes per 8-row group.
template <bool TF32>
struct Elem {
    static constexpr int kBytes = TF32 ? 4 : 2;
    static constexpr int kPerGroup = 16 / kBytes;          // elements per 16-byte core row
    static constexpr int kChunk = 128 / kBytes;            // K elements per stage
    static constexpr int kStep = 32 / kBytes;              // K per MMA (two core matrices)
};

// Byte offset of element (row, k) of a [rows x chunk] K-major no-swizzle tile.
template <bool TF32>
__host__ __device__ __forceinline__ uint32_t tile_off_e(int row, int k)
{
    using E = Elem<TF32>;
    return (uint32_t)(row >> 3) * kSbo + (uint32_t)(k / E::kPerGroup) * kLbo + (uint32_t)(row & 7) * 16u +
           (uint32_t)(k % E::kPerGroup) * (uint32_t)E::kBytes;
}

// hi = round(x), lo = round(x - hi) in the operand type, packed for a 16-byte
// core row (4 values for tf32: one uint4 each for hi and lo; 8 for bf16).
__device__ __forceinline__ uint32_t to_tf32(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// The same rounding on the bit pattern: add half a unit in the last tf32 place
// to the magnitude bits and clear the 13 dropped bits (round to nearest, ties
// away from zero; a carry into the exponent is the correct rounding up).
// Equal to cvt.rna.tf32.f32 for finite inputs below the largest finite float.
__device__ __forceinline__ uint32_t tf32_rna_bits(uint32_t xb) { return (xb + 0x1000u) & 0xFFFFE000u; }

template <bool TF32>
__device__ __forceinline__ void split_group(const float* x, uint4& hi, uint4& lo)
{
    if constexpr (TF32) {
        uint32_t h[4], l[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            h[e] = to_tf32(x[e]);
            l[e] = to_tf32(x[e] - __uint_as_float(h[e]));
        }
        hi = make_uint4(h[0], h[1], h[2], h[3]);
        lo = make_uint4(l[0], l[1], l[2], l[3]);
    } else {
        uint32_t h[4], l[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const __nv_bfloat16 h0 = __float2bfloat16_rn(x[2 * e]);
            const __nv_bfloat16 h1 = __float2bfloat16_rn(x[2 * e + 1]);
            h[e] = pack2(h0, h1);
            l[e] = pack2(__float2bfloat16_rn(x[2 * e] - __bfloat162float(h0)),
                         __float2bfloat16_rn(x[2 * e + 1] - __bfloat162float(h1)));
        }
        hi = make_uint4(h[0], h[1], h[2], h[3]);
        lo = make_uint4(l[0], l[1], l[2], l[3]);
    }
}

// Instruction descriptor: D f32; A and B bf16 (format 1, kind::f16) or tf32
// (format 2, kind::tf32); both K-major; N>>3 at bits 17-22, M>>4 at 24-28.
template <bool TF32>
__host__ __device__ constexpr uint32_t make_idesc_e(int M, int N)
{
    return (1u << 4) | ((TF32 ? 2u : 1u) << 7) | ((TF32 ? 2u : 1u) << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

template <bool TF32>
__device__ __forceinline__ void mma_split(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate)
{
    if constexpr (TF32) {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n"
            :
            : "r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
    } else {
        mma_bf16(d_tmem, adesc, bdesc, idesc, accumulate);
    }
}

template <int N>
struct TcCfg {
    static constexpr int kNcols = (N <= 32) ? 32 : (N <= 64 ? 64 : 128);   // TMEM columns (power of 2 >= 32)
    static constexpr uint32_t kABytes = kTcRows * 128;                    // one A tile: 128 rows x 128 B (16 KB)
    static constexpr uint32_t kBBytes = N * 128;                          // one B tile
    static constexpr uint32_t kStage = 2 * kABytes + 2 * kBBytes;         // hi + lo of A and B
    static constexpr uint32_t kSmem = 2 * kStage + 64 + 1024;             // two stages + barriers + alignment
};

// Q_m split into hi/lo B tiles once per launch, already in the shared-memory
// layout: tiles[c][0|1] is the hi|lo tile of K-chunk c (N x chunk, zero past R
// and past K).
template <int N, bool TF32>
__global__ void split_q_kernel(const double* __restrict__ Q, int64_t ldq, int64_t K, int R,
                               uint8_t* __restrict__ tiles, int nchunks, const int* __restrict__ status)
{
    using E = Elem<TF32>;
    using Cfg = TcCfg<N>;
    if (*status != kStatusOk) return;
    const int64_t groups = (int64_t)nchunks * N * (E::kChunk / E::kPerGroup);
    for (int64_t gidx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; gidx < groups;
         gidx += (int64_t)gridDim.x * blockDim.x) {
        const int perc = N * (E::kChunk / E::kPerGroup);
        const int c = (int)(gidx / perc);
        const int rem = (int)(gidx - (int64_t)c * perc);
        const int n = rem / (E::kChunk / E::kPerGroup), g = rem - n * (E::kChunk / E::kPerGroup);
        float xv[8];
        for (int e = 0; e < E::kPerGroup; ++e) {
            const int64_t k = (int64_t)c * E::kChunk + g * E::kPerGroup + e;
            xv[e] = (n < R && k < K) ? (float)Q[k + ldq * (int64_t)n] : 0.0f;
        }
        uint4 hi, lo;
        split_group<TF32>(xv, hi, lo);
        uint8_t* base = tiles + (size_t)c * 2 * Cfg::kBBytes;
        const uint32_t off = tile_off_e<TF32>(n, g * E::kPerGroup);
        *reinterpret_cast<uint4*>(base + off) = hi;
        *reinterpret_cast<uint4*>(base + Cfg::kBBytes + off) = lo;
    }
}

// Main kernel.  Work unit for the A operand: (row quad q, 16-byte K group g);
// 32 quads x 8 groups per stage, two units per thread.  With L % 4 == 0 the
// four rows of a quad are contiguous and 16-byte aligned, so each k needs one
// 128-bit load; otherwise four scalar loads.  Stages are double-buffered: the
// loads of chunk c+1 are issued before the CTA waits on the MMAs of chunk c-1.
template <int N, bool TF32>
__global__ void __launch_bounds__(kTcThreads) ttm_split_tc_kernel(
    const float* __restrict__ in, const uint8_t* __restrict__ btiles, float* __restrict__ out, int64_t L,
    int64_t K, int64_t Tn, int R, int nchunks, int* __restrict__ status)
{
    using E = Elem<TF32>;
    using Cfg = TcCfg<N>;
    __shared__ int skip;   // one read of the status word, so every thread takes the same branch
    if (threadIdx.x == 0) skip = *(volatile int*)status != kStatusOk;
    __syncthreads();
    if (skip) return;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* mbar = (uint64_t*)(smem + 2 * Cfg::kStage);
    uint32_t* tmem_slot = (uint32_t*)(mbar + 2);
    __shared__ int timed_out;

    const int tid = threadIdx.x, warp = tid >> 5;
    const int64_t rows = L * Tn;
    const int64_t f_base = (int64_t)blockIdx.x * kTcRows;
    const bool vec = (L % 4) == 0 && (((uintptr_t)in) & 15) == 0;

    // this thread's two units: unit u = tid + 128*j, quad = u & 31, group = u >> 5
    int64_t rowoff[2][4];
    bool rowok[2][4];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const int u = tid + kTcThreads * j;
        const int q = u & 31;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int64_t f = f_base + 4 * q + i;
            rowok[j][i] = f < rows;
            const int64_t t = rowok[j][i] ? f / L : 0;
            const int64_t l = rowok[j][i] ? f - t * L : 0;
            rowoff[j][i] = l + L * K * t;
        }
    }

    if (warp == 0) tmem_alloc<Cfg::kNcols>(tmem_slot);
    if (tid == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        fence_mbar_init();
        timed_out = 0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    constexpr uint32_t idesc = make_idesc_e<TF32>(kTcRows, N);

    float xr[2][E::kPerGroup][4];   // [unit][k in group][row in quad]
    auto load_chunk = [&](int c) {
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int g = (tid + kTcThreads * j) >> 5;
#pragma unroll
            for (int e = 0; e < E::kPerGroup; ++e) {
                const int64_t k = (int64_t)c * E::kChunk + g * E::kPerGroup + e;
                const bool kok = k < K;
                if (vec && rowok[j][0] && rowok[j][3] && rowoff[j][3] == rowoff[j][0] + 3) {
                    float4 v = kok ? __ldg(reinterpret_cast<const float4*>(in + rowoff[j][0] + L * k))
                                   : make_float4(0.f, 0.f, 0.f, 0.f);
                    xr[j][e][0] = v.x; xr[j][e][1] = v.y; xr[j][e][2] = v.z; xr[j][e][3] = v.w;
                } else {
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        xr[j][e][i] = (kok && rowok[j][i]) ? __ldg(in + rowoff[j][i] + L * k) : 0.0f;
                }
            }
        }
    };

    load_chunk(0);
    for (int c = 0; c < nchunks; ++c) {
        const int b = c & 1;
        uint8_t* stage = smem + (size_t)b * Cfg::kStage;
        uint8_t* a_hi = stage;
        uint8_t* a_lo = a_hi + Cfg::kABytes;
        uint8_t* b_hi = a_lo + Cfg::kABytes;
        uint8_t* b_lo = b_hi + Cfg::kBBytes;
        if (c >= 2) {                       // MMAs of chunk c-2 read this stage
            if (!mbar_wait_bounded(&mbar[b], (uint32_t)((c - 2) >> 1) & 1u)) timed_out = 1;
        }
        // A: split the registers of chunk c into this stage
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int u = tid + kTcThreads * j;
            const int q = u & 31, g = u >> 5;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                float xv[8];
#pragma unroll
                for (int e = 0; e < E::kPerGroup; ++e) xv[e] = xr[j][e][i];
                uint4 hi, lo;
                split_group<TF32>(xv, hi, lo);
                const uint32_t off = tile_off_e<TF32>(4 * q + i, g * E::kPerGroup);
                *reinterpret_cast<uint4*>(a_hi + off) = hi;
                *reinterpret_cast<uint4*>(a_lo + off) = lo;
            }
        }
        // B: copy the pre-split tiles of chunk c
        {
            const uint4* src = reinterpret_cast<const uint4*>(btiles + (size_t)c * 2 * Cfg::kBBytes);
            uint4* dst = reinterpret_cast<uint4*>(b_hi);
            for (int i = tid; i < (int)(2 * Cfg::kBBytes / 16); i += kTcThreads) dst[i] = __ldg(src + i);
        }
        if (c + 1 < nchunks) load_chunk(c + 1);   // in flight while the MMAs run
        fence_proxy_async();
        __syncthreads();
        if (timed_out) break;
        if (tid == 0) {
            tc_fence_after();
            const uint32_t ah = smem_u32(a_hi), al = smem_u32(a_lo), bh = smem_u32(b_hi), bl = smem_u32(b_lo);
#pragma unroll
            for (int ks = 0; ks < E::kChunk / E::kStep; ++ks) {
                const uint32_t step = (uint32_t)ks * 2u * kLbo;
                mma_split<TF32>(tmem, make_desc(ah + step), make_desc(bh + step), idesc, (c | ks) ? 1u : 0u);
                mma_split<TF32>(tmem, make_desc(ah + step), make_desc(bl + step), idesc, 1u);
                mma_split<TF32>(tmem, make_desc(al + step), make_desc(bh + step), idesc, 1u);
            }
            mma_commit(&mbar[b]);
        }
    }
    // the last commit covers every MMA of this thread
    if (!timed_out && nchunks > 0) {
        const int c = nchunks - 1;
        if (!mbar_wait_bounded(&mbar[c & 1], (uint32_t)(c >> 1) & 1u)) timed_out = 1;
    }
    __syncthreads();
    tc_fence_after();
    if (!timed_out) {
#pragma unroll
        for (int c0 = 0; c0 < N; c0 += 16) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            const int64_t f = f_base + tid;
            if (f < rows) {
                const int64_t t = f / L, l = f - t * L;
                float* o = out + l + L * (int64_t)R * t;
#pragma unroll
                for (int jj = 0; jj < 16; ++jj)
                    if (c0 + jj < R) o[L * (int64_t)(c0 + jj)] = v[jj];
            }
        }
    } else {
        if (tid == 0) atomicCAS(status, kStatusOk, (int)CPALS_ERR_TIMEOUT);
        // once more (bounded) for MMAs still in flight before the memory is freed
        if (nchunks > 0) mbar_wait_bounded(&mbar[(nchunks - 1) & 1], (uint32_t)((nchunks - 1) >> 1) & 1u);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc<Cfg::kNcols>(tmem);
}

// ---------------------------------------------------------------- persistent pipeline

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// try_wait with a suspend-time hint: the thread sleeps until the phase
// completes or about `ns` nanoseconds pass, without issuing instructions.
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t* mbar, uint32_t parity, uint32_t ns)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(mbar)), "r"(parity), "r"(ns)
        : "memory");
    return ok != 0;
}

// Wait for the phase of `parity` on mbar; false when the CTA's abort flag is
// raised or after limit_ns (default ~1 s), which raises the flag.
constexpr uint64_t kPipeWaitNs = 1000000000ull;
__device__ __forceinline__ bool pipe_wait(uint64_t* mbar, uint32_t parity, volatile int* abort_flag,
                                          uint64_t limit_ns = kPipeWaitNs)
{
    if (mbar_try_wait(mbar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (;;) {
        if (mbar_try_wait_sleep(mbar, parity, 100000u)) return true;
        if (*abort_flag) return false;
        if (global_ns() - t0 > limit_ns) { *abort_flag = 1; return false; }
    }
}

// Drain wait used on the way out: ignores the abort flag, gives up after ~1 s.
__device__ __forceinline__ void pipe_drain(uint64_t* mbar, uint32_t parity)
{
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait_sleep(mbar, parity, 100000u))
        if (global_ns() - t0 > 1000000000ull) return;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* mbar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" : : "r"(smem_u32(mbar)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* mbar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" : : "r"(smem_u32(mbar)), "r"(bytes)
                 : "memory");
}

// TMA: a 3-D box of the tensor map at (x, y, z) into shared memory.
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* mbar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];"
        :
        : "r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(mbar))
        : "memory");
}

// Untiled bulk copy global -> shared (16-byte aligned addresses, size a multiple of 16).
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* mbar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        :
        : "r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(mbar))
        : "memory");
}

// 16 consecutive 32-bit tensor-memory columns of this thread's lane.
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t* v)
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
        "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16};"
        :
        : "r"(taddr), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]),
          "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
        : "memory");
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// D (tensor memory) += A (tensor memory) x B (shared memory descriptor).
template <bool TF32>
__device__ __forceinline__ void mma_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate)
{
    if constexpr (TF32) {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}\n"
            :
            : "r"(d_tmem), "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}\n"
            :
            : "r"(d_tmem), "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
    }
}

// Persistent pipeline configuration.  Two rings:
//  - X ring (SX stages, sized at launch): one fp32 box of X per item (128 rows
//    x one 128-byte operand K-chunk), filled by the TMA producer warp and
//    released as soon as the split warps have read it;
//  - A/B slots (kASlots): the hi|lo A operands of an item in tensor memory (64
//    columns: hi in the first 32, lo in the next 32; bf16 packs two K values
//    per column, tf32 one) and the hi|lo Q tiles of its chunk in shared memory
//    (2N rows), filled by the split warps and the Q producer warp and released
//    by the MMA commit.  When the Q tiles of all K-chunks fit in kBResident
//    bytes they are loaded once and stay resident (every row tile uses the
//    same Q_m), and the slots hold only the A operands.
// Tensor memory (512 columns) also holds two accumulators of 2N columns
// (A_hi*B_hi + A_lo*B_hi in the first N, A_hi*B_lo in the second N).
template <int N, bool TF32>
struct PipeCfg {
    using E = Elem<TF32>;
    // an item is IC operand chunks of 128 bytes per row: 64 K values for bf16
    // (one chunk) and for tf32 (two), i.e. a 32 KB box of X either way
    static constexpr int IC = TF32 ? 2 : 1;
    static constexpr int kc = E::kChunk * IC;                         // K per item
    static constexpr int kSteps = kc / E::kStep;                      // MMA K steps per item
    static constexpr uint32_t kXBytes = kTcRows * kc * 4;             // fp32 box
    static constexpr uint32_t kChunkB = 2u * N * 128u;                // hi + lo Q tiles of one chunk
    static constexpr uint32_t kBBytes = IC * kChunkB;                 // Q tiles of one item
    static constexpr int kAccCols = 2 * N;
    static constexpr int kHalfCols = 32 * IC;                         // TMEM columns of A_hi (or A_lo) per item
    static constexpr int kACols = 2 * kHalfCols;
    static constexpr int kASlotsFit = (512 - 2 * kAccCols) / kACols;
    static constexpr int kASlots = kASlotsFit < 4 ? kASlotsFit : 4;
    static constexpr uint32_t kBResident = 64u * 1024u;
    static constexpr uint32_t kRingBudget = 220u * 1024u;           // X ring + Q tiles
    static constexpr int kMaxX = 16;
    static constexpr int kEpiWarps = 4, kSplitWarps = 8;
    static constexpr int kXProducerWarp = kEpiWarps + kSplitWarps, kMmaWarp = kXProducerWarp + 1,
                         kBProducerWarp = kMmaWarp + 1;
    static constexpr int kThreads = (kBProducerWarp + 1) * 32;
    static constexpr uint32_t kSmemMax = kRingBudget + 1024 + 512;   // + alignment + barriers
    static_assert(2 * kAccCols + kASlots * kACols <= 512, "tensor memory budget");
    static_assert(kASlots >= 2, "two operand slots at least");
    static_assert(kASlots * kBBytes <= kBResident, "the Q region holds the ring slots");
    static_assert((kRingBudget - kBResident) / kXBytes * kXBytes > 114 * 1024,
                  "one CTA per SM owns all 512 TMEM columns");
    static_assert(kSmemMax + 16 <= 232448, "shared memory per CTA");
    // X stages and Q-region bytes for a launch
    static int x_stages(uint32_t bregion)
    {
        const int n = (int)((kRingBudget - bregion) / kXBytes);
        return n < kMaxX ? n : kMaxX;
    }
};

// Out(l, r, t) = sum_k X(l, k, t) Q(k, r) for the tiles blockIdx.x, +gridDim.x, ...
// A tile is BL consecutive l times BT consecutive t (BL*BT <= 128 rows) and
// nitems items of K.  Every split warp waits on every item and every ring
// has a single in-order consumer per barrier, so each parity wait refers to
// an unambiguous phase.
template <int N, bool TF32>
__global__ void __launch_bounds__(PipeCfg<N, TF32>::kThreads, 1) ttm_split_tc_pipe_kernel(
    const __grid_constant__ CUtensorMap xmap, const uint8_t* __restrict__ btiles, float* __restrict__ out,
    int64_t L, int64_t Tn, int R, int BL, int BT, int64_t ntl, int64_t ntiles, int nitems, int SX, int bres,
    int* __restrict__ status, uint64_t wait_ns, int withhold)
{
    using Cfg = PipeCfg<N, TF32>;
    using E = Elem<TF32>;
    constexpr int SA = Cfg::kASlots;
    __shared__ int skip;   // one read of the status word, so every thread takes the same branch
    if (threadIdx.x == 0) skip = *(volatile int*)status != kStatusOk;
    __syncthreads();
    if (skip) return;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* xring = smem;
    uint8_t* bslots = smem + (size_t)SX * Cfg::kXBytes;
    const uint32_t bregion = bres ? (uint32_t)nitems * Cfg::kBBytes : (uint32_t)SA * Cfg::kBBytes;
    uint64_t* xfull = (uint64_t*)(bslots + bregion);
    uint64_t* xempty = xfull + Cfg::kMaxX;
    uint64_t* bfull = xempty + Cfg::kMaxX;
    uint64_t* ready = bfull + SA;
    uint64_t* aempty = ready + SA;
    uint64_t* accfull = aempty + SA;
    uint64_t* accempty = accfull + 2;
    uint32_t* tmem_slot = (uint32_t*)(accempty + 2);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == Cfg::kMmaWarp) tmem_alloc<512>(tmem_slot);
    if (tid == 0) {
        for (int s = 0; s < SX; ++s) {
            mbar_init(&xfull[s], 1);
            mbar_init(&xempty[s], Cfg::kSplitWarps);
        }
        for (int j = 0; j < SA; ++j) {
            mbar_init(&bfull[j], 1);
            mbar_init(&ready[j], Cfg::kSplitWarps);
            mbar_init(&aempty[j], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&accfull[a], 1);
            mbar_init(&accempty[a], Cfg::kEpiWarps);
        }
        *abort_flag = 0;
        fence_mbar_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    const int64_t my_tiles = (ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x;
    const int64_t items = my_tiles * nitems;
    const int rows_used = BL * BT;
    auto acol = [&](int j) { return (uint32_t)(2 * Cfg::kAccCols + j * Cfg::kACols); };
    (void)sizeof(E);
    // last item issued on slot `s` of a ring of `n` slots when `it` items were issued
    auto last_on = [](int64_t it, int s, int n) { return it - 1 - ((it - 1 - s) % n + n) % n; };

    if (warp == Cfg::kXProducerWarp) {
        if (lane == 0) {
            const uint32_t tx = (uint32_t)rows_used * Cfg::kc * 4u;
            int64_t it = 0;
            // (the test hook withholds every copy: the consumers' waits run out)
            for (; it < items && !withhold; ++it) {
                const int s = (int)(it % SX);
                if (!pipe_wait(&xempty[s], (uint32_t)((it / SX) & 1) ^ 1u, abort_flag, wait_ns)) break;
                const int64_t tile = blockIdx.x + (it / nitems) * (int64_t)gridDim.x;
                const int c = (int)(it % nitems);
                const int64_t tt = tile / ntl, tl = tile - tt * ntl;
                mbar_expect_tx(&xfull[s], tx);
                tma_load_3d(xring + (size_t)s * Cfg::kXBytes, &xmap, (int)(tl * BL), c * Cfg::kc, (int)(tt * BT),
                            &xfull[s]);
            }
            for (int s = 0; s < SX; ++s) {   // every issued copy lands before the CTA may exit
                const int64_t last = last_on(it, s, SX);
                if (last >= 0) pipe_drain(&xfull[s], (uint32_t)((last / SX) & 1));
            }
        }
        __syncwarp();
    } else if (warp == Cfg::kBProducerWarp) {
        if (lane == 0 && bres) {
            // Q tiles of every chunk, once
            mbar_expect_tx(&bfull[0], bregion);
            bulk_load(bslots, btiles, bregion, &bfull[0]);
            pipe_drain(&bfull[0], 0u);
        } else if (lane == 0) {
            int64_t it = 0;
            for (; it < items; ++it) {
                const int j = (int)(it % SA);
                if (!pipe_wait(&aempty[j], (uint32_t)((it / SA) & 1) ^ 1u, abort_flag, wait_ns)) break;
                const int c = (int)(it % nitems);
                mbar_expect_tx(&bfull[j], Cfg::kBBytes);
                bulk_load(bslots + (size_t)j * Cfg::kBBytes, btiles + (size_t)c * Cfg::kBBytes, Cfg::kBBytes,
                          &bfull[j]);
            }
            for (int j = 0; j < SA; ++j) {
                const int64_t last = last_on(it, j, SA);
                if (last >= 0) pipe_drain(&bfull[j], (uint32_t)((last / SA) & 1));
            }
        }
        __syncwarp();
    } else if (warp == Cfg::kMmaWarp) {
        if (lane == 0) {
            constexpr uint32_t idesc2 = make_idesc_e<TF32>(kTcRows, 2 * N);
            constexpr uint32_t idesc1 = make_idesc_e<TF32>(kTcRows, N);
            int64_t it = 0;
            bool ok = !bres || pipe_wait(&bfull[0], 0u, abort_flag, wait_ns);
            for (int64_t t = 0; t < my_tiles && ok; ++t) {
                const int a = (int)(t & 1);
                if (!pipe_wait(&accempty[a], (uint32_t)((t >> 1) & 1) ^ 1u, abort_flag, wait_ns)) break;
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(a * Cfg::kAccCols);
                for (int c = 0; c < nitems; ++c, ++it) {
                    const int j = (int)(it % SA);
                    const uint32_t ph = (uint32_t)((it / SA) & 1);
                    if ((!bres && !pipe_wait(&bfull[j], ph, abort_flag, wait_ns)) || !pipe_wait(&ready[j], ph, abort_flag, wait_ns)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t ahi = tmem + acol(j), alo = ahi + (uint32_t)Cfg::kHalfCols;
                    const uint32_t bh = smem_u32(bslots + (size_t)(bres ? c : j) * Cfg::kBBytes);
#pragma unroll
                    for (int ks = 0; ks < Cfg::kSteps; ++ks) {
                        // K step ks sits in 128-byte chunk ks / 4 of the item, 32 bytes per step
                        const uint64_t bd =
                            make_desc(bh + (uint32_t)(ks >> 2) * Cfg::kChunkB + (uint32_t)(ks & 3) * 2u * kLbo);
                        mma_ts<TF32>(d, ahi + 8u * ks, bd, idesc2, (c | ks) ? 1u : 0u);   // [hi*hi | hi*lo]
                        mma_ts<TF32>(d, alo + 8u * ks, bd, idesc1, 1u);                    // += lo*hi
                    }
                    mma_commit(&aempty[j]);
                }
                if (ok) mma_commit(&accfull[a]);
            }
            // the MMAs read tensor memory and shared memory: drain before exit
            if (it > 0) {
                const int64_t last = it - 1;
                pipe_drain(&aempty[last % SA], (uint32_t)((last / SA) & 1));
            }
        }
        __syncwarp();
    } else if (warp >= Cfg::kEpiWarps) {
        // split warps: lane quadrant q = warp % 4, K half h
        const int q = warp & 3, h = (warp - Cfg::kEpiWarps) >> 2;
        const int m = 32 * q + lane;
        const bool mok = m < rows_used;
        const int bt = mok ? m / BL : 0, bl = mok ? m - bt * BL : 0;
        const int xoff = bt * Cfg::kc * BL + bl;
        const uint32_t lane_base = (uint32_t)(32 * q) << 16;
        constexpr int kHalf = Cfg::kc / 2;                      // K values per split thread per item
        constexpr int kCols = TF32 ? kHalf : kHalf / 2;        // TMEM columns of them (hi, and again lo)
        for (int64_t it = 0; it < items; ++it) {
            const int s = (int)(it % SX), j = (int)(it % SA);
            // warp-uniform outcome: tcgen05.st below is warp-collective
            const bool got = pipe_wait(&xfull[s], (uint32_t)((it / SX) & 1), abort_flag, wait_ns) &&
                             pipe_wait(&aempty[j], (uint32_t)((it / SA) & 1) ^ 1u, abort_flag, wait_ns);
            if (!__all_sync(0xffffffffu, got)) break;
            // rows past the tile's last valid row split row 0's values: their
            // accumulator rows are never stored
            const float* xk = reinterpret_cast<const float*>(xring + (size_t)s * Cfg::kXBytes) + xoff + h * kHalf * BL;
            const uint32_t col = tmem + acol(j) + (uint32_t)(h * kCols);
#pragma unroll
            for (int g = 0; g < kCols / 16; ++g) {
                uint32_t hi[16], lo[16];
                if constexpr (TF32) {
#pragma unroll
                    for (int p = 0; p < 16; ++p) {
                        const uint32_t xb = __float_as_uint(xk[(16 * g + p) * BL]);
                        hi[p] = tf32_rna_bits(xb);
                        lo[p] = tf32_rna_bits(__float_as_uint(__uint_as_float(xb) - __uint_as_float(hi[p])));
                    }
                } else {
#pragma unroll
                    for (int p = 0; p < 16; ++p) {
                        const float x0 = xk[(32 * g + 2 * p) * BL], x1 = xk[(32 * g + 2 * p + 1) * BL];
                        const __nv_bfloat162 hh = __floats2bfloat162_rn(x0, x1);
                        const float2 hf = __bfloat1622float2(hh);
                        const __nv_bfloat162 ll = __floats2bfloat162_rn(x0 - hf.x, x1 - hf.y);
                        hi[p] = *reinterpret_cast<const uint32_t*>(&hh);
                        lo[p] = *reinterpret_cast<const uint32_t*>(&ll);
                    }
                }
                tmem_st16(lane_base + col + (uint32_t)(16 * g), hi);
                tmem_st16(lane_base + col + (uint32_t)(Cfg::kHalfCols + 16 * g), lo);
            }
            // the box has been read (its values went through registers above)
            __syncwarp();
            if (lane == 0) mbar_arrive(&xempty[s]);
            tmem_wait_st();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&ready[j]);
        }
    } else {
        // epilogue warps 0..3: lane quadrant = warp
        const int m = 32 * warp + lane;
        const bool mok = m < rows_used;
        const int bt = mok ? m / BL : 0, bl = mok ? m - bt * BL : 0;
        const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
        for (int64_t t = 0; t < my_tiles; ++t) {
            const int a = (int)(t & 1);
            // warp-uniform outcome: tcgen05.ld below is warp-collective
            if (!__all_sync(0xffffffffu, pipe_wait(&accfull[a], (uint32_t)((t >> 1) & 1), abort_flag, wait_ns))) break;
            tc_fence_after();
            const int64_t tile = blockIdx.x + t * (int64_t)gridDim.x;
            const int64_t tt = tile / ntl, tl = tile - tt * ntl;
            const int64_t l = tl * BL + bl, tq = tt * BT + bt;
            const bool ok = mok && l < L && tq < Tn;
            float* o = out + l + L * (int64_t)R * tq;
#pragma unroll
            for (int c0 = 0; c0 < N; c0 += 16) {
                float v[16], w[16];
                tmem_ld16(tmem + lane_base + (uint32_t)(a * Cfg::kAccCols + c0), v);
                tmem_ld16(tmem + lane_base + (uint32_t)(a * Cfg::kAccCols + N + c0), w);
                if (ok) {
#pragma unroll
                    for (int jj = 0; jj < 16; ++jj)
                        if (c0 + jj < R) o[L * (int64_t)(c0 + jj)] = v[jj] + w[jj];
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&accempty[a]);
        }
    }

    __syncthreads();
    if (*abort_flag && tid == 0) atomicCAS(status, kStatusOk, (int)CPALS_ERR_TIMEOUT);
    tc_fence_after();
    if (warp == Cfg::kMmaWarp) tmem_dealloc<512>(tmem);
}

// ---------------------------------------------------------------- FP32 pipeline (CUDA cores)
// The same TMA ring feeds FP32 FMAs on the CUDA cores: the FP32 precision's
// passes over X and the FP32 contractions of intermediates (Eq. multittm).
// One producer warp streams [rows x 64 K] boxes of In (tensor map [L, K, T])
// and, unless Q fits whole in shared memory, the matching 64-row chunk of Q
// into a ring of stages.  Four compute warps own a tile of 128 rows: lane q
// takes rows 4q..4q+3 (one 16-byte read per k; BL % 4 == 0 keeps the four in
// one t) and warp g takes columns g TN .. g TN + TN - 1 (TN = RC / 4), whose Q
// values sit together in the stage ([g][k][TNP], TNP = TN rounded up to 4) so
// a k costs TNP / 4 broadcast 16-byte reads.  The FMAs run in order of k, and
// a tile's outputs are written with 16-byte stores along l.  Up to four CTAs
// share an SM (as registers allow), each with a short ring: with only four
// compute warps a CTA leaves the FMA pipe idle while its warps wait on shared
// memory, and more CTAs per SM cover that better than a longer ring.
constexpr int kF32Kc = 64;              // K per item
constexpr int kF32ComputeWarps = 4;
constexpr int kF32Threads = (kF32ComputeWarps + 1) * 32;
constexpr uint32_t kF32XBytes = kTcRows * kF32Kc * 4;     // 32 KB box at 128 rows
constexpr uint32_t kF32SmemBudget = 54u * 1024u;          // four CTAs per SM
constexpr uint32_t kF32SmemBudgetWide = 110u * 1024u;     // RC >= 48: registers allow two
constexpr int kF32MaxStages = 6;
constexpr uint32_t kF32QResident = 20u * 1024u;

template <int RC>
struct F32Cfg {
    static constexpr int TN = RC / 4;
    static constexpr int TNP = (TN + 3) / 4 * 4;
    static constexpr uint32_t kQItemBytes = 4u * kF32Kc * TNP * 4u;      // one item's Q chunk, all groups
    static constexpr uint32_t kBudget = RC >= 48 ? kF32SmemBudgetWide : kF32SmemBudget;
};

// Q (K x R, FP64, ldq) to the FP32 item chunks [c][g][k][TNP] (zero padded).
template <int RC>
__global__ void f32_q_kernel(const double* __restrict__ Q, int64_t ldq, int64_t K, int R, float* __restrict__ qf,
                             int nitems, const int* __restrict__ status)
{
    if (*status != kStatusOk) return;
    using C = F32Cfg<RC>;
    const int64_t total = (int64_t)nitems * 4 * kF32Kc * C::TNP;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(e % C::TNP);
        const int64_t r1 = e / C::TNP;
        const int k = (int)(r1 % kF32Kc);
        const int64_t r2 = r1 / kF32Kc;
        const int g = (int)(r2 % 4);
        const int64_t c = r2 / 4;
        const int64_t kk = c * kF32Kc + k;
        const int col = g * C::TN + j;
        qf[e] = (j < C::TN && kk < K && col < R) ? (float)Q[kk + ldq * (int64_t)col] : 0.0f;
    }
}

template <int RC>
__global__ void __launch_bounds__(kF32Threads) ttm_f32_pipe_kernel(
    const __grid_constant__ CUtensorMap xmap, const float* __restrict__ qf, float* __restrict__ out, int64_t L,
    int64_t Tn, int R, int BL, int BT, int64_t ntl, int64_t ntiles, int nitems, int SX, int qres,
    int* __restrict__ status)
{
    using C = F32Cfg<RC>;
    __shared__ int skip;
    if (threadIdx.x == 0) skip = *(volatile int*)status != kStatusOk;
    __syncthreads();
    if (skip) return;
    extern __shared__ uint8_t smem_raw[];
    // 128-byte aligned ring: an offset from the shared array itself, so the
    // compiler still knows every X and Q read below is a shared-memory load
    uint8_t* smem = smem_raw + ((128u - ((uint32_t)__cvta_generic_to_shared(smem_raw) & 127u)) & 127u);
    const uint32_t qbytes = qres ? (uint32_t)nitems * C::kQItemBytes : 0u;
    const uint32_t stage = kF32XBytes + (qres ? 0u : C::kQItemBytes);
    uint8_t* qregion = smem;
    uint8_t* ring = smem + qbytes;
    uint64_t* full = (uint64_t*)(ring + (size_t)SX * stage);
    uint64_t* empty = full + kF32MaxStages;
    uint64_t* qfull = empty + kF32MaxStages;
    volatile int* abort_flag = (volatile int*)(qfull + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int s = 0; s < SX; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kF32ComputeWarps);
        }
        mbar_init(qfull, 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    __syncthreads();

    const int64_t my_tiles = (ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x;
    const int64_t items = my_tiles * nitems;
    const int rows_used = BL * BT;
    auto last_on = [](int64_t it, int s, int n) { return it - 1 - ((it - 1 - s) % n + n) % n; };

    if (warp == kF32ComputeWarps) {
        if (lane == 0) {
            if (qres) {
                mbar_expect_tx(qfull, qbytes);
                bulk_load(qregion, qf, qbytes, qfull);
            }
            const uint32_t tx = (uint32_t)rows_used * kF32Kc * 4u + (qres ? 0u : C::kQItemBytes);
            int64_t it = 0;
            for (; it < items; ++it) {
                const int s = (int)(it % SX);
                if (!pipe_wait(&empty[s], (uint32_t)((it / SX) & 1) ^ 1u, abort_flag)) break;
                const int64_t tile = blockIdx.x + (it / nitems) * (int64_t)gridDim.x;
                const int c = (int)(it % nitems);
                const int64_t tt = tile / ntl, tl = tile - tt * ntl;
                uint8_t* st = ring + (size_t)s * stage;
                mbar_expect_tx(&full[s], tx);
                tma_load_3d(st, &xmap, (int)(tl * BL), c * kF32Kc, (int)(tt * BT), &full[s]);
                if (!qres)
                    bulk_load(st + kF32XBytes, qf + (size_t)c * (C::kQItemBytes / 4), C::kQItemBytes, &full[s]);
            }
            for (int s = 0; s < SX; ++s) {   // every issued copy lands before the CTA may exit
                const int64_t last = last_on(it, s, SX);
                if (last >= 0) pipe_drain(&full[s], (uint32_t)((last / SX) & 1));
            }
            if (qres) pipe_drain(qfull, 0u);
        }
        __syncwarp();
    } else {
        const int g = warp, q = lane;
        const int m0 = 4 * q;                      // first of this thread's four rows in the tile
        const bool mok = m0 < rows_used;
        const int bt = mok ? m0 / BL : 0, bl = mok ? m0 - bt * BL : 0;
        const int xoff = bt * kF32Kc * BL + bl;    // box layout [bt][k][bl]
        bool ok = !qres || pipe_wait(qfull, 0u, abort_flag);
        int64_t it = 0;
        for (int64_t t = 0; t < my_tiles && ok; ++t) {
            float acc[4][C::TN];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < C::TN; ++j) acc[i][j] = 0.0f;
            for (int c = 0; c < nitems; ++c, ++it) {
                const int s = (int)(it % SX);
                if (!pipe_wait(&full[s], (uint32_t)((it / SX) & 1), abort_flag)) { ok = false; break; }
                const uint8_t* st = ring + (size_t)s * stage;
                const float* xs = reinterpret_cast<const float*>(st) + xoff;
                const float* qs = qres ? reinterpret_cast<const float*>(qregion) + (size_t)c * (C::kQItemBytes / 4)
                                       : reinterpret_cast<const float*>(st + kF32XBytes);
                qs += (size_t)g * kF32Kc * C::TNP;
#pragma unroll 4
                for (int k = 0; k < kF32Kc; ++k) {
                    const float4 x = *reinterpret_cast<const float4*>(xs + k * BL);
                    float qv[C::TNP];
#pragma unroll
                    for (int j = 0; j < C::TNP; j += 4) {
                        const float4 v = *reinterpret_cast<const float4*>(qs + k * C::TNP + j);
                        qv[j] = v.x; qv[j + 1] = v.y; qv[j + 2] = v.z; qv[j + 3] = v.w;
                    }
#pragma unroll
                    for (int j = 0; j < C::TN; ++j) {
                        acc[0][j] = fmaf(x.x, qv[j], acc[0][j]);
                        acc[1][j] = fmaf(x.y, qv[j], acc[1][j]);
                        acc[2][j] = fmaf(x.z, qv[j], acc[2][j]);
                        acc[3][j] = fmaf(x.w, qv[j], acc[3][j]);
                    }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[s]);
            }
            if (!ok) break;
            const int64_t tile = blockIdx.x + t * (int64_t)gridDim.x;
            const int64_t tt = tile / ntl, tl = tile - tt * ntl;
            const int64_t l = tl * BL + bl, tq = tt * BT + bt;
            if (mok && l < L && tq < Tn) {         // L % 4 == 0: the four rows are valid together
                float* o = out + l + L * (int64_t)R * tq;
#pragma unroll
                for (int j = 0; j < C::TN; ++j) {
                    const int col = g * C::TN + j;
                    if (col < R)
                        *reinterpret_cast<float4*>(o + L * (int64_t)col) =
                            make_float4(acc[0][j], acc[1][j], acc[2][j], acc[3][j]);
                }
            }
        }
    }
    __syncthreads();
    if (*abort_flag && tid == 0) atomicCAS(status, kStatusOk, (int)CPALS_ERR_TIMEOUT);
}

using EncodeTiledFn = PFN_cuTensorMapEncodeTiled_v12000;

EncodeTiledFn encode_tiled_fn()
{
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

// The pipeline serves a shape when the TMA strides are 16-byte multiples
// (L % 4 == 0, 16-byte aligned X) and every coordinate fits in int32.
bool pipe_shape_ok(const float* in, TtmShape s)
{
    const int64_t lim = (int64_t)1 << 30;
    return s.L % 4 == 0 && (((uintptr_t)in) & 15) == 0 && s.L < lim && s.K < lim && s.T < lim &&
           encode_tiled_fn() != nullptr;
}

template <int N, bool TF32>
cudaError_t launch_pipe(Handle* h, const float* in, const uint8_t* tiles, float* out, TtmShape s, int R,
                        int nitems)
{
    using Cfg = PipeCfg<N, TF32>;
    static std::once_flag attr_once;
    cudaError_t attr_err = cudaSuccess;
    std::call_once(attr_once, [&] {
        attr_err = cudaFuncSetAttribute(ttm_split_tc_pipe_kernel<N, TF32>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::kSmemMax);
    });
    CPALS_CUDA_TRY(attr_err);
    const int BL = s.L >= kTcRows ? kTcRows : (int)s.L;
    const int BT = kTcRows / BL;
    CUtensorMap map;
    const cuuint64_t gdim[3] = {(cuuint64_t)s.L, (cuuint64_t)s.K, (cuuint64_t)s.T};
    const cuuint64_t gstride[2] = {(cuuint64_t)s.L * 4u, (cuuint64_t)s.L * (cuuint64_t)s.K * 4u};
    const cuuint32_t box[3] = {(cuuint32_t)BL, (cuuint32_t)Cfg::kc, (cuuint32_t)BT};
    const cuuint32_t estride[3] = {1, 1, 1};
    const CUresult cr = encode_tiled_fn()(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(in), gdim,
                                          gstride, box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (cr != CUDA_SUCCESS) return cudaErrorInvalidValue;
    const int64_t ntl = (s.L + BL - 1) / BL;
    const int64_t ntiles = ntl * ((s.T + BT - 1) / BT);
    const int grid = (int)std::min<int64_t>(ntiles, (int64_t)h->num_sms);
    const bool bres = (uint64_t)nitems * Cfg::kBBytes <= Cfg::kBResident;
    const uint32_t bregion = bres ? (uint32_t)nitems * Cfg::kBBytes : (uint32_t)Cfg::kASlots * Cfg::kBBytes;
    const int SX = Cfg::x_stages(bregion);
    const uint32_t smem = (uint32_t)SX * Cfg::kXBytes + bregion + 1024 + 512;
    ttm_split_tc_pipe_kernel<N, TF32><<<grid, Cfg::kThreads, smem, h->stream>>>(
        map, tiles, out, s.L, s.T, R, BL, BT, ntl, ntiles, nitems, SX, bres ? 1 : 0, h->d_status,
        h->test_withhold ? 1000000ull : kPipeWaitNs, h->test_withhold ? 1 : 0);
    h->launches++;
    return cudaGetLastError();
}

template <int N, bool TF32>
cudaError_t launch_tc(Handle* h, const float* in, const double* Q, int64_t ldq, float* out, TtmShape s, int R)
{
    using Cfg = TcCfg<N>;
    using E = Elem<TF32>;
    static bool attr = false;
    if (!attr) {
        CPALS_CUDA_TRY(cudaFuncSetAttribute(ttm_split_tc_kernel<N, TF32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)Cfg::kSmem));
        attr = true;
    }
    const bool pipe = h->tc_pipe && pipe_shape_ok(in, s);
    // 128-byte K chunks of the pre-split Q tiles: whole items for the pipeline
    constexpr int IC = PipeCfg<N, TF32>::IC;
    int nchunks = (int)((s.K + E::kChunk - 1) / E::kChunk);
    const int nitems = (nchunks + IC - 1) / IC;
    if (pipe) nchunks = nitems * IC;
    const size_t tile_bytes = (size_t)nchunks * 2 * Cfg::kBBytes;
    if (tile_bytes > (size_t)h->scratch_elems * sizeof(double)) return cudaErrorInvalidValue;
    uint8_t* tiles = reinterpret_cast<uint8_t*>(h->scratch);
    const int64_t groups = (int64_t)nchunks * N * (E::kChunk / E::kPerGroup);
    split_q_kernel<N, TF32><<<(unsigned)std::min<int64_t>((groups + 255) / 256, 4096), 256, 0, h->stream>>>(
        Q, ldq, s.K, R, tiles, nchunks, h->d_status);
    h->launches++;
    CPALS_CUDA_TRY(cudaGetLastError());
    if (pipe) return launch_pipe<N, TF32>(h, in, tiles, out, s, R, nitems);
    const int64_t rows = s.L * s.T;
    const int64_t grid = (rows + kTcRows - 1) / kTcRows;
    ttm_split_tc_kernel<N, TF32><<<(unsigned)grid, kTcThreads, Cfg::kSmem, h->stream>>>(
        in, tiles, out, s.L, s.K, s.T, R, nchunks, h->d_status);
    h->launches++;
    return cudaGetLastError();
}

template <int RC>
cudaError_t launch_f32_pipe(Handle* h, const float* in, const double* Q, int64_t ldq, float* out, TtmShape s, int R)
{
    using C = F32Cfg<RC>;
    static std::once_flag attr_once;
    cudaError_t attr_err = cudaSuccess;
    std::call_once(attr_once, [&] {
        attr_err = cudaFuncSetAttribute(ttm_f32_pipe_kernel<RC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)(C::kBudget + 256));
    });
    CPALS_CUDA_TRY(attr_err);
    const int nitems = (int)((s.K + kF32Kc - 1) / kF32Kc);
    const size_t qfloats = (size_t)nitems * (C::kQItemBytes / 4);
    if (qfloats * sizeof(float) > (size_t)h->scratch_elems * sizeof(double)) return cudaErrorInvalidValue;
    float* qf = reinterpret_cast<float*>(h->scratch);
    f32_q_kernel<RC><<<(unsigned)std::min<size_t>((qfloats + 255) / 256, 4096), 256, 0, h->stream>>>(
        Q, ldq, s.K, R, qf, nitems, h->d_status);
    h->launches++;
    CPALS_CUDA_TRY(cudaGetLastError());
    const int BL = s.L >= kTcRows ? kTcRows : (int)s.L;
    const int BT = kTcRows / BL;
    CUtensorMap map;
    const cuuint64_t gdim[3] = {(cuuint64_t)s.L, (cuuint64_t)s.K, (cuuint64_t)s.T};
    const cuuint64_t gstride[2] = {(cuuint64_t)s.L * 4u, (cuuint64_t)s.L * (cuuint64_t)s.K * 4u};
    const cuuint32_t box[3] = {(cuuint32_t)BL, (cuuint32_t)kF32Kc, (cuuint32_t)BT};
    const cuuint32_t estride[3] = {1, 1, 1};
    const CUresult cr = encode_tiled_fn()(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(in), gdim,
                                          gstride, box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (cr != CUDA_SUCCESS) return cudaErrorInvalidValue;
    const int64_t ntl = (s.L + BL - 1) / BL;
    const int64_t ntiles = ntl * ((s.T + BT - 1) / BT);
    const bool qres = (uint64_t)nitems * C::kQItemBytes <= kF32QResident;
    const uint32_t qbytes = qres ? (uint32_t)nitems * C::kQItemBytes : 0u;
    const uint32_t stage = kF32XBytes + (qres ? 0u : C::kQItemBytes);
    const int SX = (int)std::min<uint32_t>(kF32MaxStages, (C::kBudget - qbytes) / stage);
    if (SX < 1) return cudaErrorInvalidValue;
    const uint32_t smem = qbytes + (uint32_t)SX * stage + 128 + 8 * (2 * kF32MaxStages + 1) + 16;
    int per_sm = 1;
    CPALS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ttm_f32_pipe_kernel<RC>, kF32Threads, smem));
    if (per_sm < 1) per_sm = 1;
    const int grid = (int)std::min<int64_t>(ntiles, (int64_t)per_sm * h->num_sms);
    ttm_f32_pipe_kernel<RC><<<grid, kF32Threads, smem, h->stream>>>(map, qf, out, s.L, s.T, R, BL, BT, ntl, ntiles,
                                                                    nitems, SX, qres ? 1 : 0, h->d_status);
    h->launches++;
    return cudaGetLastError();
}

}  // namespace

// Below R = 9 the row-quad kernel streams X faster (at R = 8 the pipeline
// holds 3.0 TB/s against 4.5 TB/s): the pipeline takes R = 9..64.
bool f32_pipe_ok(const float* in, const float* out, TtmShape s, int R)
{
    return R > 8 && R <= 64 && pipe_shape_ok(in, s) && (((uintptr_t)out) & 15) == 0;
}

cudaError_t ttm_f32_pipe(Handle* h, const float* in, const double* Q, int64_t ldq, float* out, TtmShape s, int R)
{
    if (s.L * s.T == 0) return cudaSuccess;
    if (R <= 8) return cudaErrorInvalidValue;   // f32_pipe_ok excludes it
    if (R <= 12) return launch_f32_pipe<12>(h, in, Q, ldq, out, s, R);
    if (R <= 16) return launch_f32_pipe<16>(h, in, Q, ldq, out, s, R);
    if (R <= 20) return launch_f32_pipe<20>(h, in, Q, ldq, out, s, R);
    if (R <= 24) return launch_f32_pipe<24>(h, in, Q, ldq, out, s, R);
    if (R <= 32) return launch_f32_pipe<32>(h, in, Q, ldq, out, s, R);
    if (R <= 48) return launch_f32_pipe<48>(h, in, Q, ldq, out, s, R);
    return launch_f32_pipe<64>(h, in, Q, ldq, out, s, R);
}

bool tc_supported(int R) { return R >= 16 && R <= 64; }

cudaError_t ttm_split_tc(Handle* h, const float* in, const double* Q, int64_t ldq, float* out, TtmShape s, int R,
                         bool tf32)
{
    if (s.L * s.T == 0) return cudaSuccess;
    if (tf32) {
        if (R <= 16) return launch_tc<16, true>(h, in, Q, ldq, out, s, R);
        if (R <= 32) return launch_tc<32, true>(h, in, Q, ldq, out, s, R);
        if (R <= 48) return launch_tc<48, true>(h, in, Q, ldq, out, s, R);
        return launch_tc<64, true>(h, in, Q, ldq, out, s, R);
    }
    if (R <= 16) return launch_tc<16, false>(h, in, Q, ldq, out, s, R);
    if (R <= 32) return launch_tc<32, false>(h, in, Q, ldq, out, s, R);
    if (R <= 48) return launch_tc<48, false>(h, in, Q, ldq, out, s, R);
    return launch_tc<64, false>(h, in, Q, ldq, out, s, R);
}

}  // namespace cpals
