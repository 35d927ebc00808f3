// ttm_plan.h -- host-side launch planning of the row-per-thread TTM kernels
// (plain C++, no CUDA): the TTM order of Sec. 3.2, the [L, K, T] view of a
// single TTM (Sec. 2.2), the split of the contracted index over grid.z and the
// scratch that split needs.  ttm.cu launches from these plans; a CPU test
// compiles this header alone and sweeps shapes against the scratch bound.
#pragma once

#include <stdint.h>

#include <algorithm>

namespace cpals {

constexpr int kMaxN = 12;
constexpr int kMaxRank = 64;

// A TTM over mode m of a tensor with (current) dims d views it as
// [L, K, T] with L = prod_{k<m} d_k, K = d_m, T = prod_{k>m} d_k (Sec. 2.2).
struct TtmShape {
    int64_t L, K, T;
};

inline TtmShape ttm_shape(int N, const int64_t* d, int m) {
    TtmShape s{1, d[m], 1};
    for (int k = 0; k < m; ++k) s.L *= d[k];
    for (int k = m + 1; k < N; ++k) s.T *= d[k];
    return s;
}

// Decreasing-dimension TTM order of Sec. 3.2 (ties: higher mode first).
inline void ttm_order(int N, const int64_t* dims, int n, int* order) {
    int cnt = 0;
    for (int m = 0; m < N; ++m)
        if (m != n) order[cnt++] = m;
    for (int a = 0; a < cnt; ++a)
        for (int b = a + 1; b < cnt; ++b) {
            int x = order[a], y = order[b];
            if (dims[y] > dims[x] || (dims[y] == dims[x] && y > x)) { order[a] = y; order[b] = x; }
        }
}

// prod(dims) with an overflow check: false when the product does not fit in
// int64 (every dim must be positive).
inline bool checked_prod(int N, const int64_t* dims, int64_t* out) {
    int64_t p = 1;
    for (int m = 0; m < N; ++m) {
        if (dims[m] <= 0) return false;
        if (p > INT64_MAX / dims[m]) return false;
        p *= dims[m];
    }
    *out = p;
    return true;
}

// Split-K reduction: up to kSplitGroup partials are added in one pass; more
// are added in groups of kSplitGroup whose sums follow the partials in the
// scratch buffer, then the group sums.
constexpr int64_t kSplitGroup = 16;

// Scratch elements a split into ks parts of an output of outn elements uses:
// ks partials, plus the group sums when the reduction takes two passes.
inline int64_t ksplit_scratch_elems(int64_t ks, int64_t outn) {
    if (ks <= 1) return 0;
    const int64_t groups = ks > kSplitGroup ? (ks + kSplitGroup - 1) / kSplitGroup : 0;
    return (ks + groups) * outn;
}

// Number of K splits for a row kernel with ctas_xy row blocks of tpb threads:
// split K when the row blocks alone cannot fill the SMs with about 2048
// threads each, keeping >= 8 indices per split.  The result is the split
// count after K is cut into equal chunks of ceil(K / ks), and its partials and
// group sums fit in part_elems (ksplit_scratch_elems(result, outn) <=
// part_elems whenever have_part).
inline int64_t ttm_ksplit(int64_t ctas_xy, int tpb, int64_t K, int num_sms, int64_t outn, int64_t part_elems,
                          bool have_part)
{
    constexpr int64_t kMinSplitK = 8;
    const int64_t want = (int64_t)num_sms * (2048 / tpb);
    int64_t ks = 1;
    if (ctas_xy < want && K >= 2 * kMinSplitK && have_part) {
        ks = (want + ctas_xy - 1) / ctas_xy;
        ks = std::min<int64_t>(ks, K / kMinSplitK);
        ks = std::min<int64_t>(ks, part_elems / std::max<int64_t>(outn, 1));
        if (ks < 2) ks = 1;
    }
    // up to 16 splits take one reduction pass instead of two: stay there when
    // the grid still gives every SM four CTAs
    if (ks > kSplitGroup && ctas_xy * kSplitGroup >= 4LL * num_sms) ks = kSplitGroup;
    // equal chunks can only lower the count; then drop splits until the
    // partials and the group sums fit (the scratch need grows with ks)
    for (;;) {
        const int64_t kchunk = (K + ks - 1) / ks;
        const int64_t eff = (K + kchunk - 1) / kchunk;
        if (eff <= 1 || ksplit_scratch_elems(eff, outn) <= part_elems) return eff <= 1 ? 1 : eff;
        ks = eff - 1;
    }
}

// Register width per thread: R itself up to 16, then 20, 24, 32.  Wider R is
// cut into ceil(R / 32) equal column blocks, each rounded up to one of those
// widths (R = 40: 2 x 20, R = 48: 2 x 24, R = 64: 2 x 32), so that no block
// computes many columns that are not there.
inline int ttm_width(int R) {
    if (R <= 16) return R;
    if (R <= 20) return 20;
    if (R <= 24) return 24;
    if (R <= 32) return 32;
    const int gy = (R + 31) / 32;
    const int w = (R + gy - 1) / gy;
    return w <= 20 ? 20 : (w <= 24 ? 24 : 32);
}

// CTA sizes of the FP64 row kernel.  FP64 is bound by the FP64 pipe of each
// SM, so what counts is the largest number of rows any SM holds: the CTA size
// minimises ceil(CTAs / SMs) x rows per CTA x indices per split, which keeps
// every SM within a fraction of a percent of the mean at the large passes.
constexpr int kF64Tpb[] = {64, 96, 128};

struct RowsPlan {
    int tpb;
    int64_t gx, gy, ks, kchunk;
};

// Launch plan of the FP64 row kernel for one TTM of shape s and rank R with
// part_elems doubles of scratch for split-K partials (have_part = false: no
// split).
inline RowsPlan plan_rows_f64(int num_sms, TtmShape s, int R, int64_t part_elems, bool have_part)
{
    const int64_t rows = s.L * s.T;
    const int rc = ttm_width(R);
    const int64_t gy = (R + rc - 1) / rc;
    const int64_t outn = rows * R;
    RowsPlan p{kF64Tpb[0], 0, gy, 1, s.K};
    int64_t best = -1;
    for (int c : kF64Tpb) {
        const int64_t cx = (rows + c - 1) / c;
        const int64_t cks = ttm_ksplit(cx * gy, c, s.K, num_sms, outn, part_elems, have_part);
        const int64_t ckc = (s.K + cks - 1) / cks;
        const int64_t ctas = cx * gy * cks;
        const int64_t cost = ((ctas + num_sms - 1) / num_sms) * c * ckc;
        if (best < 0 || cost < best) { best = cost; p.tpb = c; p.gx = cx; p.ks = cks; p.kchunk = ckc; }
    }
    return p;
}

// Scratch layout of the Multi-TTM that runs from a fixed array of `capacity`
// doubles (cpals_multi_ttm_static): the first intermediate at 0 (s0 doubles),
// the second after it (s1 doubles), later intermediates ping-pong between the
// two, and the split-K partials of every TTM after both.
struct StaticPlan {
    bool ok;              // false: overflow in the sizes, or the intermediates do not fit
    int64_t s0, s1;       // the two ping-pong intermediates
    int64_t part_elems;   // scratch left for split-K partials
    int64_t peak;         // the highest scratch element any TTM of the Multi-TTM touches, plus one
    int64_t max_splits;   // the largest split count of the TTMs
};

inline StaticPlan plan_multi_ttm_static(int N, const int64_t* dims, int R, int n, int num_sms, int64_t capacity)
{
    StaticPlan sp{false, 0, 0, 0, 0, 1};
    int64_t P = 0;
    if (N < 2 || N > kMaxN || R < 1 || n < 0 || n >= N || !checked_prod(N, dims, &P)) return sp;
    int order[kMaxN];
    ttm_order(N, dims, n, order);
    // the sizes only shrink (R <= every dim), so the first two are the largest
    sp.s0 = P / dims[order[0]] * R;
    sp.s1 = (N > 2) ? sp.s0 / dims[order[1]] * R : 0;
    if (sp.s0 + sp.s1 > capacity) return sp;
    sp.part_elems = capacity - sp.s0 - sp.s1;
    int64_t d[kMaxN];
    for (int m = 0; m < N; ++m) d[m] = dims[m];
    int64_t cur = sp.s0 + sp.s1;
    for (int k = 0; k < N - 1; ++k) {
        const int m = order[k];
        const TtmShape s = ttm_shape(N, d, m);
        const RowsPlan p = plan_rows_f64(num_sms, s, R, sp.part_elems, true);
        const int64_t use = sp.s0 + sp.s1 + ksplit_scratch_elems(p.ks, s.L * s.T * R);
        cur = std::max(cur, use);
        sp.max_splits = std::max(sp.max_splits, p.ks);
        d[m] = R;
    }
    sp.peak = cur;
    sp.ok = cur <= capacity;
    return sp;
}

}  // namespace cpals
