// capi.cu -- the extern "C" entry points of include/cpals.h: handle lifecycle,
// data movement, the per-mode update of Alg. cp-als-qr / Alg. cp-als, and
// the sweep loop replayed as one CUDA graph per solve kind.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <vector>

#include "internal.cuh"

using cpals::Handle;

namespace {

thread_local char g_create_err[512] = "";

int fail(Handle* h, int code, const char* fmt, const char* detail = "")
{
    char* dst = h ? h->err : g_create_err;
    snprintf(dst, 512, fmt, detail);
    return code;
}

int cuda_fail(Handle* h, cudaError_t e, const char* where)
{
    char* dst = h ? h->err : g_create_err;
    snprintf(dst, 512, "%s: %s", where, cudaGetErrorString(e));
    return CPALS_ERR_CUDA;
}

#define CUDA_OR_FAIL(h, expr, where)                 \
    do {                                             \
        cudaError_t _e = (expr);                     \
        if (_e != cudaSuccess) return cuda_fail((h), _e, (where)); \
    } while (0)

// A device allocation: out of memory is CPALS_ERR_NOMEM, anything else CPALS_ERR_CUDA.
#define ALLOC_OR_FAIL(h, expr, where)                                                              \
    do {                                                                                           \
        cudaError_t _e = (expr);                                                                   \
        if (_e == cudaErrorMemoryAllocation) {                                                     \
            cudaGetLastError();                                                                    \
            return fail((h), CPALS_ERR_NOMEM, "%s: device allocation failed", (where));            \
        }                                                                                          \
        if (_e != cudaSuccess) return cuda_fail((h), _e, (where));                                 \
    } while (0)

// Test hook (cpals_test_fail_allocation): the n-th device allocation of a
// handle from now on fails as if the device were out of memory.
std::atomic<int> g_fail_alloc_in{0};

cudaError_t device_alloc(void** p, size_t bytes)
{
    int n = g_fail_alloc_in.load();
    while (n > 0 && !g_fail_alloc_in.compare_exchange_weak(n, n - 1)) {}
    if (n == 1) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

template <typename T>
cudaError_t dalloc(Handle* h, T** p, size_t elems)
{
    const size_t bytes = std::max<size_t>(elems, 1) * sizeof(T);
    cudaError_t e = device_alloc((void**)p, bytes);
    if (e == cudaSuccess) h->owned_bytes += bytes;
    return e;
}

void free_all(Handle* h)
{
    auto f = [](void* p) { if (p) cudaFree(p); };
    for (int m = 0; m < cpals::kMaxN; ++m) { f(h->A[m]); f(h->Q[m]); f(h->Rf[m]); f(h->G[m]); }
    f(h->lambda); f(h->Q0); f(h->R0); f(h->Yn); f(h->W); f(h->W32); f(h->Ahat); f(h->M); f(h->S); f(h->T);
    f(h->KM); f(h->KQ); f(h->KR[0]); f(h->KR[1]); f(h->KQb[0]); f(h->KQb[1]);
    f(h->HQ[0]); f(h->HQ[1]); f(h->HR[0]); f(h->HR[1]); f(h->Qin);
    f(h->tbuf[0]); f(h->tbuf[1]); f(h->tA); f(h->scratch); f(h->d_status); f(h->d_gate); f(h->svd_parts); f(h->d_vgate); f(h->VG); f(h->d_normX2); f(h->d_fit);
    f(h->wide[0].base); f(h->wide[1].base);
    f(h->d_fit_count); f(h->X64_owned); f(h->X32_owned); f(h->qr_ws);
    for (int m = 0; m < cpals::kMaxN; ++m) { f(h->KV[m]); f(h->KC[m]); f(h->KE[m]); }
    f(h->Kmu); f(h->KGV); f(h->KP); f(h->KMw[0]); f(h->KMw[1]);
    for (int i = 0; i < cpals::kProfMax; ++i) {
        if (h->prof_a[i]) cudaEventDestroy(h->prof_a[i]);
        if (h->prof_b[i]) cudaEventDestroy(h->prof_b[i]);
    }
    if (h->side) cudaStreamDestroy(h->side);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    for (int s = 0; s < 4; ++s) if (h->graph[s]) cudaGraphExecDestroy(h->graph[s]);
}

// The two workspaces of the GPU-wide CholeskyQR2 (rank above 32 only).
bool alloc_wide(Handle* h)
{
    if (h->R <= 32) return true;
    for (auto& ws : h->wide) {
        if (dalloc(h, &ws.base, cpals::wide_ws_elems(h->R, h->num_sms)) != cudaSuccess) return false;
        cpals::wide_ws_carve(ws, h->R, h->num_sms);
    }
    return true;
}

// Largest TTM intermediate over all modes and steps of the Multi-TTM (and MTTKRP).
int64_t max_intermediate(const Handle* h)
{
    int64_t best = 1;
    for (int n = 0; n < h->N; ++n) {
        int order[cpals::kMaxN];
        cpals::ttm_order(h->N, h->dims, n, order);
        int64_t d[cpals::kMaxN];
        for (int m = 0; m < h->N; ++m) d[m] = h->dims[m];
        int64_t P = h->P;
        for (int k = 0; k < h->N - 1; ++k) {
            const int m = order[k];
            P = P / d[m] * h->R;
            d[m] = h->R;
            best = std::max(best, P);
        }
    }
    return best;
}

bool mem_ok(int mem) { return mem == CPALS_MEM_DEVICE || mem == CPALS_MEM_HOST; }

cudaMemcpyKind kind_in(int mem) { return mem == CPALS_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice; }
cudaMemcpyKind kind_out(int mem) { return mem == CPALS_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice; }

// Reads and clears the device status word (synchronises).
int take_status(Handle* h)
{
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "stream synchronize");
    int st = 0;
    e = cudaMemcpy(&st, h->d_status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(h, e, "status read");
    if (st != cpals::kStatusOk) {
        const int zero = 0;
        cudaMemcpy(h->d_status, &zero, sizeof(int), cudaMemcpyHostToDevice);
        if (st == CPALS_ERR_SINGULAR)
            return fail(h, CPALS_ERR_SINGULAR, "%s", "singular least-squares system (R0 or S); factor left unchanged");
        if (st == CPALS_ERR_TIMEOUT) return fail(h, CPALS_ERR_TIMEOUT, "%s", "a bounded device wait gave up");
        return fail(h, st, "%s", "device error");
    }
    return CPALS_OK;
}

// Events around one phase of a profiled sweep (no-op unless h->prof).
struct ProfScope {
    Handle* h;
    int i = -1;
    ProfScope(Handle* hh, int bucket) : h(hh)
    {
        if (h->prof && h->prof_n < cpals::kProfMax) {
            i = h->prof_n++;
            h->prof_bucket[i] = bucket;
            cudaEventRecord(h->prof_a[i], h->stream);
        }
    }
    ~ProfScope()
    {
        if (i >= 0) cudaEventRecord(h->prof_b[i], h->stream);
    }
};

inline bool is_normal(int solve) { return solve == CPALS_SOLVE_NORMAL || solve == CPALS_SOLVE_NORMAL_PINV; }

// The Gram of the current factor A_m and, with want_qr, its QR (diag(R_m) >= 0).
// With CPALS_OPT_FUSED_TAIL they come from the same cluster kernel as the
// mode updates' (kind 4: the factor as it is), so that factors set from a
// checkpoint give the same Q_m, R_m and G_m as the run that saved them.
cudaError_t factor_qr_gram(Handle* h, int m, bool want_qr)
{
    const int64_t I = h->dims[m];
    if (cpals::tail_fused(h) && (cpals::wide_tail_on(h) || cpals::mode_tail_ok(I, h->R, 1))) {
        CPALS_CUDA_TRY(cpals::mode_tail(h, m, 4, h->A[m], nullptr, want_qr));
        if (want_qr) CPALS_CUDA_TRY(cpals::householder_qr(h, h->A[m], I, h->R, h->Q[m], h->Rf[m], true, h->d_gate));
        return cudaSuccess;
    }
    if (want_qr) CPALS_CUDA_TRY(cpals::householder_qr(h, h->A[m], I, h->R, h->Q[m], h->Rf[m]));
    return cpals::gram(h, h->A[m], I, h->G[m]);
}

// Make the derived data (Q_m, R_m for QR/SVD; G_m for NORMAL) of every mode
// other than `skip` current.
cudaError_t refresh_derived(Handle* h, int solve, int skip)
{
    for (int m = 0; m < h->N; ++m) {
        if (m == skip) continue;
        if (is_normal(solve)) {
            if (!h->gram_valid[m]) {
                ProfScope ps(h, cpals::kProfFactor);
                CPALS_CUDA_TRY(factor_qr_gram(h, m, false));
                h->gram_valid[m] = true;
            }
            if (h->kruskal && h->have_X && !h->ke_valid[m]) {
                CPALS_CUDA_TRY(cpals::kr_refresh_e(h, m));
                h->ke_valid[m] = true;
            }
        } else {
            if (!h->qr_valid[m]) {
                ProfScope ps(h, cpals::kProfFactor);
                CPALS_CUDA_TRY(factor_qr_gram(h, m, true));
                h->qr_valid[m] = true;
                h->gram_valid[m] = true;
                h->kc_valid[m] = false;
            }
            if (h->kruskal && h->have_X && !h->kc_valid[m]) {
                CPALS_CUDA_TRY(cpals::kr_refresh_c(h, m));
                h->kc_valid[m] = true;
            }
        }
    }
    return cudaSuccess;
}

// Invalidate everything derived from the factors (after new factors or Q/R).
void factors_changed(Handle* h)
{
    for (int m = 0; m < h->N; ++m) { h->kc_valid[m] = false; h->ke_valid[m] = false; }
}

// Where the QR of V_n comes from in a dimension-tree sweep: the QR of the
// other half's Khatri-Rao product (slot) and the own half's other modes.
// ready = true: the sweep has already enqueued this mode's QR on the side
// stream (followed by ev_join), so the mode update only waits for it.
struct TreeQR {
    int slot;
    bool other_left;
    const int* own;
    int nown;
    bool ready;
};

// The end of a mode update once W_n (or M_n) and the solve operator are ready:
// the solve, lambda and the normalised A_n, and its QR (QR/SVD solves) or Gram
// (normal equations).  With CPALS_OPT_FUSED_TAIL the whole tail runs in one
// thread-block cluster (tail.cu; above rank 32 after the GPU-wide solve
// kernels), followed by the Householder QR, which runs only if the cluster's
// CholeskyQR2 was refused; otherwise the separate kernels run.
cudaError_t finish_update(Handle* h, int n, int solve, double rtol, bool have_operator)
{
    const int64_t In = h->dims[n];
    const bool normal = is_normal(solve);
    if (cpals::tail_fused(h) && (cpals::wide_tail_on(h) || cpals::mode_tail_ok(In, h->R))) {
        int kind = 0;
        const double* Win = normal ? h->M : h->W;
        const double* Op = h->R0;
        if (solve == CPALS_SOLVE_SVD || solve == CPALS_SOLVE_NORMAL_PINV) {
            if (!have_operator) {
                ProfScope ps(h, cpals::kProfOther);
                if (solve == CPALS_SOLVE_SVD) CPALS_CUDA_TRY(cpals::svd_operator(h, rtol));
                else CPALS_CUDA_TRY(cpals::normal_operator(h, n, true, rtol));
            }
            kind = 1;
            Op = h->T;
        } else if (solve == CPALS_SOLVE_NORMAL) {
            if (!have_operator) {
                ProfScope ps(h, cpals::kProfOther);
                CPALS_CUDA_TRY(cpals::normal_operator(h, n, false, 0.0));
            }
            kind = 2;
            Op = h->T;
        }
        if (h->R > 32) {
            // the R^2 work per row of the solve on every SM, then the cluster from Ahat
            ProfScope ps(h, cpals::kProfOther);
            switch (solve) {
                case CPALS_SOLVE_QR: CPALS_CUDA_TRY(cpals::solve_qr(h, In)); break;
                case CPALS_SOLVE_SVD: CPALS_CUDA_TRY(cpals::solve_svd(h, In, rtol, true)); break;
                case CPALS_SOLVE_NORMAL: CPALS_CUDA_TRY(cpals::solve_normal(h, n, true)); break;
                default: CPALS_CUDA_TRY(cpals::solve_normal_pinv(h, n, rtol, true)); break;
            }
            kind = 3;
            Win = h->Ahat;
        }
        {
            // the fused tail holds the solve and the normalisation too
            ProfScope ps(h, cpals::kProfFactor);
            CPALS_CUDA_TRY(cpals::mode_tail(h, n, kind, Win, Op, !normal));
            if (!normal)
                CPALS_CUDA_TRY(cpals::householder_qr(h, h->A[n], In, h->R, h->Q[n], h->Rf[n], true, h->d_gate));
        }
        h->gram_valid[n] = true;
        h->qr_valid[n] = !normal;
        return cudaSuccess;
    }
    {
        ProfScope ps(h, cpals::kProfOther);
        switch (solve) {
            case CPALS_SOLVE_QR: CPALS_CUDA_TRY(cpals::solve_qr(h, In)); break;
            case CPALS_SOLVE_SVD: CPALS_CUDA_TRY(cpals::solve_svd(h, In, rtol, have_operator)); break;
            case CPALS_SOLVE_NORMAL: CPALS_CUDA_TRY(cpals::solve_normal(h, n, have_operator)); break;
            default: CPALS_CUDA_TRY(cpals::solve_normal_pinv(h, n, rtol, have_operator)); break;
        }
        CPALS_CUDA_TRY(cpals::normalize_and_refactor(h, n));
    }
    ProfScope ps(h, cpals::kProfFactor);
    if (normal) {
        CPALS_CUDA_TRY(cpals::gram(h, h->A[n], In, h->G[n]));
        h->gram_valid[n] = true;
        h->qr_valid[n] = false;
    } else {
        CPALS_CUDA_TRY(cpals::householder_qr(h, h->A[n], In, h->R, h->Q[n], h->Rf[n]));
        h->qr_valid[n] = true;
        h->gram_valid[n] = false;
    }
    return cudaSuccess;
}

// One mode update (Alg. cp-als-qr mode-loop body, or Alg. cp-als for NORMAL).
cudaError_t mode_update(Handle* h, int n, int solve, double rtol, bool from_partial = false,
                        const TreeQR* tq = nullptr)
{
    CPALS_CUDA_TRY(refresh_derived(h, solve, n));
    if (h->kruskal) {
        // Kruskal input (Sec. 3.3.2): no pass over a dense tensor
        if (is_normal(solve)) {
            ProfScope ps(h, cpals::kProfTTM);
            CPALS_CUDA_TRY(cpals::kr_mttkrp(h, n));
        } else {
            {
                ProfScope ps(h, cpals::kProfQ0);
                CPALS_CUDA_TRY(cpals::krp_qr(h, n, true));
            }
            h->krp_mode = n;
            ProfScope ps(h, cpals::kProfApplyQ0);
            CPALS_CUDA_TRY(cpals::kr_apply_q0(h, n));
        }
        CPALS_CUDA_TRY(finish_update(h, n, solve, rtol, false));
        if (is_normal(solve)) {
            CPALS_CUDA_TRY(cpals::kr_refresh_e(h, n));
            h->ke_valid[n] = true;
            h->kc_valid[n] = false;
        } else {
            CPALS_CUDA_TRY(cpals::kr_refresh_c(h, n));
            h->kc_valid[n] = true;
            h->ke_valid[n] = false;
        }
        return cudaSuccess;
    }
    if (is_normal(solve)) {
        // S_n and its Cholesky factor or pseudo-inverse need only the Grams:
        // the side stream forms them while the MTTKRP runs (tq->ready: the
        // sweep has enqueued them already)
        if (!(tq && tq->ready)) {
            CPALS_CUDA_TRY(cudaEventRecord(h->ev_fork, h->stream));
            CPALS_CUDA_TRY(cudaStreamWaitEvent(h->side, h->ev_fork, 0));
            cudaStream_t main = h->stream;
            h->stream = h->side;
            cudaError_t e;
            {
                ProfScope ps(h, cpals::kProfOther);
                e = cpals::normal_operator(h, n, solve == CPALS_SOLVE_NORMAL_PINV, rtol);
            }
            h->stream = main;
            CPALS_CUDA_TRY(e);
            CPALS_CUDA_TRY(cudaEventRecord(h->ev_join, h->side));
        }
        {
            ProfScope ps(h, cpals::kProfTTM);
            if (from_partial) CPALS_CUDA_TRY(cpals::mttkrp_from_partial(h, n));
            else CPALS_CUDA_TRY(cpals::mttkrp(h, n));
        }
        CPALS_CUDA_TRY(cudaStreamWaitEvent(h->stream, h->ev_join, 0));
    } else {
        // The QR of V_n needs only the R_m and the Multi-TTM only the Q_m: run the
        // QR on the side stream meanwhile and join before W = Y_(n) Q0.
        if (!(tq && tq->ready)) {
            CPALS_CUDA_TRY(cudaEventRecord(h->ev_fork, h->stream));
            CPALS_CUDA_TRY(cudaStreamWaitEvent(h->side, h->ev_fork, 0));
            cudaStream_t main = h->stream;
            h->stream = h->side;
            cudaError_t e;
            {
                ProfScope ps(h, cpals::kProfQ0);
                e = tq ? cpals::krp_qr_tree(h, n, tq->slot, tq->other_left, tq->own, tq->nown) : cpals::krp_qr(h, n);
            }
            // the SVD operator of R0 needs nothing else: it follows on the side stream
            if (e == cudaSuccess && solve == CPALS_SOLVE_SVD) {
                ProfScope ps(h, cpals::kProfOther);
                e = cpals::svd_operator(h, rtol);
            }
            h->stream = main;
            CPALS_CUDA_TRY(e);
            CPALS_CUDA_TRY(cudaEventRecord(h->ev_join, h->side));
        }
        h->krp_mode = n;
        {
            ProfScope ps(h, cpals::kProfTTM);
            // mixed precisions: the unfolding stays FP32 for W in FP32
            h->yn32_mode = h->prec != CPALS_F64 && h->q0_fp32;
            cudaError_t e = from_partial ? cpals::multi_ttm_from_partial(h, n) : cpals::multi_ttm(h, n, h->Q);
            h->yn32_mode = false;
            CPALS_CUDA_TRY(e);
        }
        CPALS_CUDA_TRY(cudaStreamWaitEvent(h->stream, h->ev_join, 0));
        ProfScope ps(h, cpals::kProfApplyQ0);
        CPALS_CUDA_TRY(cpals::apply_q0(h, n));
    }
    return finish_update(h, n, solve, rtol, true);
}

cudaError_t fit_scoped(Handle* h, int solve)
{
    ProfScope ps(h, cpals::kProfOther);
    return cpals::fit_efficient(h, solve);
}

// One sweep over the modes.  For an N >= 3 dense tensor the Multi-TTMs
// follow a dimension tree (Sec. 3.3.3): the modes split into halves
// H1 = {0..h-1} and H2 = {h..N-1}.  X is contracted once over H2 (whose Q_m do
// not change while H1 is updated), and each H1 mode contracts the rest of H1
// from that partial with the current Q_m.  Then X is contracted once over H1
// with the updated Q_m for the H2 modes.  That makes two passes over X per
// sweep instead of N.  The TTMs of a Multi-TTM can run in any order
// (Sec. 2.2), so only rounding differs from the per-mode Multi-TTM.  The
// normal equations share the same tree for their MTTKRPs (A_m instead of
// Q_m, diagonal contractions after the first).
cudaError_t sweep(Handle* h, int solve, double rtol)
{
    if (h->N < 3 || !h->dimtree || !h->tA || h->kruskal) {
        for (int n = 0; n < h->N; ++n) CPALS_CUDA_TRY(mode_update(h, n, solve, rtol));
        return fit_scoped(h, solve);
    }
    const int N = h->N, h1 = (N + 1) / 2;
    int H1[cpals::kMaxN], H2[cpals::kMaxN], n1 = 0, n2 = 0;
    for (int m = 0; m < N; ++m) {
        if (m < h1) H1[n1++] = m;
        else H2[n2++] = m;
    }
    // the normal equations use the same halves with the MTTKRP's contractions
    auto pass = [&](const int* modes, int nm) {
        ProfScope ps(h, cpals::kProfTTM);
        return is_normal(solve) ? cpals::mttkrp_tree_pass(h, modes, nm) : cpals::dimtree_pass(h, modes, nm);
    };
    if (is_normal(solve)) {
        // the first mode of each half needs only Grams that the pass does not
        // change: its S_n operator is formed on the side stream under the pass
        auto early_op = [&](int n) -> cudaError_t {
            CPALS_CUDA_TRY(cudaEventRecord(h->ev_fork, h->stream));
            CPALS_CUDA_TRY(cudaStreamWaitEvent(h->side, h->ev_fork, 0));
            cudaStream_t main = h->stream;
            h->stream = h->side;
            cudaError_t e;
            {
                ProfScope ps(h, cpals::kProfOther);
                e = cpals::normal_operator(h, n, solve == CPALS_SOLVE_NORMAL_PINV, rtol);
            }
            h->stream = main;
            CPALS_CUDA_TRY(e);
            return cudaEventRecord(h->ev_join, h->side);
        };
        const TreeQR ready{0, false, nullptr, 0, true};
        CPALS_CUDA_TRY(early_op(H1[0]));
        CPALS_CUDA_TRY(pass(H2, n2));
        for (int k = 0; k < n1; ++k)
            CPALS_CUDA_TRY(mode_update(h, H1[k], solve, rtol, true, k == 0 ? &ready : nullptr));
        CPALS_CUDA_TRY(early_op(H2[0]));
        CPALS_CUDA_TRY(pass(H1, n1));
        for (int k = 0; k < n2; ++k)
            CPALS_CUDA_TRY(mode_update(h, H2[k], solve, rtol, true, k == 0 ? &ready : nullptr));
        return fit_scoped(h, solve);
    }
    if (!h->krp_tree) {
        CPALS_CUDA_TRY(pass(H2, n2));
        for (int k = 0; k < n1; ++k) CPALS_CUDA_TRY(mode_update(h, H1[k], solve, rtol, true));
        CPALS_CUDA_TRY(pass(H1, n1));
        for (int k = 0; k < n2; ++k) CPALS_CUDA_TRY(mode_update(h, H2[k], solve, rtol, true));
        return fit_scoped(h, solve);
    }
    // The QR of V_n follows the same tree: V_n of an H1 mode is (Khatri-Rao of
    // H2) (.) (the other H1 modes), and the H2 factors do not change while H1
    // is updated, so the QR of the H2 half is taken once, on the side stream
    // under the pass over X for H1's partial; the QR of the H1 half likewise
    // under the second pass.  Each mode then folds only its own half's other
    // R_m onto that half's R and applies the half's Q as a Kronecker factor
    // (Eq. kr-id), which leaves the same Q0, R0 up to rounding.
    auto half_qr = [&](const int* modes, int nm, int slot) -> cudaError_t {
        CPALS_CUDA_TRY(cudaEventRecord(h->ev_fork, h->stream));
        CPALS_CUDA_TRY(cudaStreamWaitEvent(h->side, h->ev_fork, 0));
        cudaStream_t main = h->stream;
        h->stream = h->side;
        cudaError_t e;
        {
            ProfScope ps(h, cpals::kProfQ0);
            e = cpals::krp_qr_half(h, modes, nm, slot);
        }
        h->stream = main;
        return e;
    };
    int own[cpals::kMaxN];
    auto own_of = [&](const int* modes, int nm, int n) {
        int c = 0;
        for (int k = 0; k < nm; ++k)
            if (modes[k] != n) own[c++] = modes[k];
        return c;
    };
    // The first mode of each half needs no factor updated in that half, so its
    // Q0, R0 follow the half's QR on the side stream, also under the pass.
    auto early_qr = [&](int n, const TreeQR& tq) -> cudaError_t {
        cudaStream_t main = h->stream;
        h->stream = h->side;
        cudaError_t e;
        {
            ProfScope ps(h, cpals::kProfQ0);
            e = cpals::krp_qr_tree(h, n, tq.slot, tq.other_left, tq.own, tq.nown);
        }
        if (e == cudaSuccess && solve == CPALS_SOLVE_SVD) {
            ProfScope ps(h, cpals::kProfOther);
            e = cpals::svd_operator(h, rtol);
        }
        h->stream = main;
        CPALS_CUDA_TRY(e);
        return cudaEventRecord(h->ev_join, h->side);
    };
    CPALS_CUDA_TRY(half_qr(H2, n2, 1));
    const TreeQR first1{1, true, own, own_of(H1, n1, H1[0]), true};
    CPALS_CUDA_TRY(early_qr(H1[0], first1));
    CPALS_CUDA_TRY(pass(H2, n2));
    for (int k = 0; k < n1; ++k) {
        const TreeQR tq = (k == 0) ? first1 : TreeQR{1, true, own, own_of(H1, n1, H1[k]), false};
        CPALS_CUDA_TRY(mode_update(h, H1[k], solve, rtol, true, &tq));
    }
    CPALS_CUDA_TRY(half_qr(H1, n1, 0));
    const TreeQR first2{0, false, own, own_of(H2, n2, H2[0]), true};
    CPALS_CUDA_TRY(early_qr(H2[0], first2));
    CPALS_CUDA_TRY(pass(H1, n1));
    for (int k = 0; k < n2; ++k) {
        const TreeQR tq = (k == 0) ? first2 : TreeQR{0, false, own, own_of(H2, n2, H2[k]), false};
        CPALS_CUDA_TRY(mode_update(h, H2[k], solve, rtol, true, &tq));
    }
    return fit_scoped(h, solve);
}

// FMA throughput probe kernels (dependent chains, 8 independent accumulators).
template <typename T>
__global__ void fma_probe_kernel(T* out, int iters, T a, T b)
{
    T acc[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) acc[i] = (T)(threadIdx.x + i);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) acc[i] = acc[i] * a + b;
    }
    T s = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += acc[i];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" {

int cpals_create(const int64_t* dims, int N, int rank, int precision, cpals_handle** out)
{
    if (!out) return fail(nullptr, CPALS_ERR_ARG, "%s", "out is NULL");
    *out = nullptr;
    if (!dims) return fail(nullptr, CPALS_ERR_ARG, "%s", "dims is NULL");
    if (N < 2 || N > cpals::kMaxN) return fail(nullptr, CPALS_ERR_ARG, "%s", "N must be in [2, 12]");
    if (rank < 1 || rank > cpals::kMaxRank) return fail(nullptr, CPALS_ERR_ARG, "%s", "rank must be in [1, 64]");
    {
        // the dense path holds Q0 (R^{N-1} x R) and Y_(n) (I_n x R^{N-1})
        double rn1 = 1.0;
        for (int m = 0; m < N - 1; ++m) rn1 *= rank;
        if (rn1 * rank > (double)(1LL << 36))
            return fail(nullptr, CPALS_ERR_ARG, "%s", "R^N too large for a dense tensor handle (use Kruskal input)");
    }
    if (precision != CPALS_F64 && precision != CPALS_F32 && precision != CPALS_BF16X3 && precision != CPALS_TF32X3)
        return fail(nullptr, CPALS_ERR_ARG, "%s", "unknown precision");
    for (int m = 0; m < N; ++m)
        if (dims[m] < 1) return fail(nullptr, CPALS_ERR_ARG, "%s", "dims must be >= 1");
    {
        int64_t P = 0;
        if (!cpals::checked_prod(N, dims, &P))
            return fail(nullptr, CPALS_ERR_ARG, "%s", "prod(dims) does not fit in 64 bits");
    }
    for (int m = 0; m < N; ++m)
        if (dims[m] < rank)
            return fail(nullptr, CPALS_ERR_ARG, "%s",
                        "rank must not exceed any dim (the compact QR of each I_m x R factor needs I_m >= R)");
    Handle* h = new (std::nothrow) Handle();
    if (!h) return fail(nullptr, CPALS_ERR_NOMEM, "%s", "host allocation failed");
    h->N = N; h->R = rank; h->prec = precision;
    h->P = 1; h->RN1 = 1; h->Imax = 0;
    for (int m = 0; m < N; ++m) {
        h->dims[m] = dims[m];
        h->P *= dims[m];
        h->Imax = std::max(h->Imax, dims[m]);
    }
    for (int m = 0; m < N - 1; ++m) h->RN1 *= rank;
    cudaError_t e = cudaGetDevice(&h->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
    if (e != cudaSuccess) { int rc = cuda_fail(nullptr, e, "device query"); delete h; return rc; }

    const int R = rank;
    const int64_t big = std::max(h->Imax, h->RN1);
    h->tbuf_elems = max_intermediate(h);
    const size_t tsz = (precision == CPALS_F64) ? sizeof(double) : sizeof(float);
    h->scratch_elems = std::max<int64_t>({4 * big * R + 64 * R * R, 4096, (int64_t)h->num_sms * 2 * h->Imax * R});
    h->fit_cap = 4096;
    bool ok = true;
    for (int m = 0; m < N && ok; ++m) {
        ok = dalloc(h, &h->A[m], dims[m] * R) == cudaSuccess && dalloc(h, &h->Q[m], dims[m] * R) == cudaSuccess &&
             dalloc(h, &h->Rf[m], (size_t)R * R) == cudaSuccess && dalloc(h, &h->G[m], (size_t)R * R) == cudaSuccess;
    }
    ok = ok && dalloc(h, &h->lambda, R) == cudaSuccess &&
         dalloc(h, &h->Q0, h->RN1 * R) == cudaSuccess && dalloc(h, &h->R0, (size_t)R * R) == cudaSuccess &&
         dalloc(h, &h->Yn, h->Imax * h->RN1) == cudaSuccess && dalloc(h, &h->W, h->Imax * R) == cudaSuccess &&
         dalloc(h, &h->W32, h->Imax * R) == cudaSuccess &&
         dalloc(h, &h->Ahat, h->Imax * R) == cudaSuccess && dalloc(h, &h->M, h->Imax * R) == cudaSuccess &&
         dalloc(h, &h->S, (size_t)R * R) == cudaSuccess && dalloc(h, &h->T, (size_t)R * R) == cudaSuccess &&
         dalloc(h, &h->KM, (size_t)R * R * R) == cudaSuccess && dalloc(h, &h->KQ, (size_t)R * R * R) == cudaSuccess &&
         dalloc(h, &h->KR[0], (size_t)R * R) == cudaSuccess && dalloc(h, &h->KR[1], (size_t)R * R) == cudaSuccess &&
         dalloc(h, &h->KQb[0], h->RN1 * R) == cudaSuccess && dalloc(h, &h->KQb[1], h->RN1 * R) == cudaSuccess &&
         dalloc(h, &h->scratch, h->scratch_elems) == cudaSuccess && dalloc(h, &h->d_status, 1) == cudaSuccess &&
         dalloc(h, &h->d_gate, 1) == cudaSuccess && dalloc(h, &h->svd_parts, 2 * (size_t)R) == cudaSuccess &&
         dalloc(h, &h->d_vgate, 1) == cudaSuccess && dalloc(h, &h->VG, (size_t)R * R) == cudaSuccess &&
         dalloc(h, &h->d_normX2, 1) == cudaSuccess && dalloc(h, &h->d_fit, h->fit_cap + 1) == cudaSuccess &&
         dalloc(h, &h->d_fit_count, 1) == cudaSuccess;
    // TSQR: leaf Q (m x R), stacked leaf R factors and their Q (2 m x R at most), the
    // tree levels above (4 m x R at most in total)
    h->qr_ws_elems = std::max<int64_t>(8 * big * R + 64 * R * R, 4096);
    ok = ok && dalloc(h, &h->qr_ws, h->qr_ws_elems) == cudaSuccess;
    ok = ok && alloc_wide(h);
    if (ok) {
        int lo = 0, hi = 0;
        ok = cudaDeviceGetStreamPriorityRange(&lo, &hi) == cudaSuccess &&
             cudaStreamCreateWithPriority(&h->side, cudaStreamNonBlocking, hi) == cudaSuccess &&
             cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming) == cudaSuccess;
    }
    if (ok && N >= 3) {
        const int h1 = (N + 1) / 2;
        int64_t a = 1, b = 1;
        for (int m = 0; m < N; ++m) {
            a *= (m < h1) ? dims[m] : (int64_t)rank;
            b *= (m < h1) ? (int64_t)rank : dims[m];
        }
        h->tA_elems = std::max(a, b);
        void* pa = nullptr;
        ok = device_alloc(&pa, tsz * h->tA_elems) == cudaSuccess;
        h->tA = pa;
        if (ok) h->owned_bytes += tsz * h->tA_elems;
        // per-half QR of the Khatri-Rao products: R^|H1| and R^|H2| rows; the
        // inner fold of a mode has R^|H1| rows at most (|H1| >= |H2|)
        int64_t r1 = 1, r2 = 1;
        for (int m = 0; m < N; ++m) (m < h1 ? r1 : r2) *= rank;
        ok = ok && dalloc(h, &h->HQ[0], r1 * R) == cudaSuccess && dalloc(h, &h->HQ[1], r2 * R) == cudaSuccess &&
             dalloc(h, &h->HR[0], (size_t)R * R) == cudaSuccess && dalloc(h, &h->HR[1], (size_t)R * R) == cudaSuccess &&
             dalloc(h, &h->Qin, r1 * R) == cudaSuccess;
    }
    if (ok) {
        void* p0 = nullptr; void* p1 = nullptr;
        ok = device_alloc(&p0, tsz * h->tbuf_elems) == cudaSuccess &&
             device_alloc(&p1, tsz * h->tbuf_elems) == cudaSuccess;
        h->tbuf[0] = p0; h->tbuf[1] = p1;
        if (ok) h->owned_bytes += 2 * tsz * h->tbuf_elems;
    }
    if (!ok) {
        free_all(h);
        delete h;
        cudaGetLastError();
        return fail(nullptr, CPALS_ERR_NOMEM, "%s", "device allocation failed");
    }
    e = cudaMemset(h->d_status, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(h->d_fit_count, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(h->lambda, 0, sizeof(double) * R);
    if (e != cudaSuccess) { int rc = cuda_fail(nullptr, e, "memset"); free_all(h); delete h; return rc; }
    *out = reinterpret_cast<cpals_handle*>(h);
    return CPALS_OK;
}

int cpals_destroy(cpals_handle* hh)
{
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h) return CPALS_OK;
    cudaStreamSynchronize(h->stream);
    if (h->side) cudaStreamSynchronize(h->side);
    free_all(h);
    delete h;
    return CPALS_OK;
}

int cpals_create_kruskal(const int64_t* dims, int N, int rank, int S, cpals_handle** out)
{
    if (!out) return fail(nullptr, CPALS_ERR_ARG, "%s", "out is NULL");
    *out = nullptr;
    if (!dims) return fail(nullptr, CPALS_ERR_ARG, "%s", "dims is NULL");
    if (N < 2 || N > cpals::kMaxN) return fail(nullptr, CPALS_ERR_ARG, "%s", "N must be in [2, 12]");
    if (rank < 1 || rank > cpals::kMaxRank) return fail(nullptr, CPALS_ERR_ARG, "%s", "rank must be in [1, 64]");
    if (S < 1 || S > 4096) return fail(nullptr, CPALS_ERR_ARG, "%s", "the Kruskal rank S must be in [1, 4096]");
    for (int m = 0; m < N; ++m)
        if (dims[m] < rank)
            return fail(nullptr, CPALS_ERR_ARG, "%s",
                        "rank must not exceed any dim (the compact QR of each I_m x R factor needs I_m >= R)");
    Handle* h = new (std::nothrow) Handle();
    if (!h) return fail(nullptr, CPALS_ERR_NOMEM, "%s", "host allocation failed");
    h->N = N; h->R = rank; h->prec = CPALS_F64; h->kruskal = true; h->KS = S;
    h->P = 1; h->RN1 = 1; h->Imax = 0;
    double pd = 1.0, rd = 1.0;
    for (int m = 0; m < N; ++m) {
        h->dims[m] = dims[m];
        pd *= (double)dims[m];
        h->Imax = std::max(h->Imax, dims[m]);
    }
    for (int m = 0; m < N - 1; ++m) rd *= rank;
    // P and R^{N-1} are only used when they fit (direct fit, Y_(n) for small cases)
    h->P = pd < 9.0e18 ? (int64_t)pd : -1;
    h->RN1 = rd < 9.0e18 ? (int64_t)rd : -1;
    cudaError_t e = cudaGetDevice(&h->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
    if (e != cudaSuccess) { int rc = cuda_fail(nullptr, e, "device query"); delete h; return rc; }
    const int R = rank;
    const int64_t big = std::max<int64_t>(h->Imax, (int64_t)R * R);
    const size_t R2 = (size_t)R * R, R3 = R2 * R;
    h->scratch_elems = std::max<int64_t>({4 * big * R + 64 * R * R, 4096, (int64_t)h->num_sms * 2 * h->Imax * R});
    h->fit_cap = 4096;
    bool ok = true;
    for (int m = 0; m < N && ok; ++m) {
        ok = dalloc(h, &h->A[m], dims[m] * R) == cudaSuccess && dalloc(h, &h->Q[m], dims[m] * R) == cudaSuccess &&
             dalloc(h, &h->Rf[m], R2) == cudaSuccess && dalloc(h, &h->G[m], R2) == cudaSuccess &&
             dalloc(h, &h->KV[m], dims[m] * S) == cudaSuccess && dalloc(h, &h->KC[m], (size_t)R * S) == cudaSuccess &&
             dalloc(h, &h->KE[m], (size_t)S * R) == cudaSuccess;
    }
    ok = ok && dalloc(h, &h->lambda, R) == cudaSuccess && dalloc(h, &h->R0, R2) == cudaSuccess &&
         dalloc(h, &h->W, h->Imax * R) == cudaSuccess && dalloc(h, &h->Ahat, h->Imax * R) == cudaSuccess &&
         dalloc(h, &h->M, h->Imax * R) == cudaSuccess && dalloc(h, &h->S, R2) == cudaSuccess &&
         dalloc(h, &h->T, R2) == cudaSuccess && dalloc(h, &h->KM, R3) == cudaSuccess &&
         dalloc(h, &h->KQ, R3) == cudaSuccess && dalloc(h, &h->KR[0], R2) == cudaSuccess &&
         dalloc(h, &h->KR[1], R2) == cudaSuccess && dalloc(h, &h->KP, std::max(1, N - 2) * R3) == cudaSuccess &&
         dalloc(h, &h->Kmu, S) == cudaSuccess && dalloc(h, &h->KGV, (size_t)N * S * S) == cudaSuccess &&
         dalloc(h, &h->KMw[0], (size_t)S * R) == cudaSuccess && dalloc(h, &h->KMw[1], (size_t)S * R) == cudaSuccess &&
         dalloc(h, &h->scratch, h->scratch_elems) == cudaSuccess && dalloc(h, &h->d_status, 1) == cudaSuccess &&
         dalloc(h, &h->d_gate, 1) == cudaSuccess && dalloc(h, &h->svd_parts, 2 * (size_t)R) == cudaSuccess &&
         dalloc(h, &h->d_vgate, 1) == cudaSuccess && dalloc(h, &h->VG, (size_t)R * R) == cudaSuccess &&
         dalloc(h, &h->d_normX2, 1) == cudaSuccess && dalloc(h, &h->d_fit, h->fit_cap + 1) == cudaSuccess &&
         dalloc(h, &h->d_fit_count, 1) == cudaSuccess;
    // Y_(n) is formed (for cpals_multi_ttm) only when it is small
    if (ok && h->RN1 > 0 && (double)h->Imax * (double)h->RN1 <= (double)(1 << 24))
        ok = dalloc(h, &h->Yn, h->Imax * h->RN1) == cudaSuccess;
    h->qr_ws_elems = std::max<int64_t>(8 * big * R + 64 * R * R, 4096);
    ok = ok && dalloc(h, &h->qr_ws, h->qr_ws_elems) == cudaSuccess;
    ok = ok && alloc_wide(h);
    if (ok) {
        int lo = 0, hi = 0;
        ok = cudaDeviceGetStreamPriorityRange(&lo, &hi) == cudaSuccess &&
             cudaStreamCreateWithPriority(&h->side, cudaStreamNonBlocking, hi) == cudaSuccess &&
             cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming) == cudaSuccess;
    }
    if (!ok) {
        free_all(h);
        delete h;
        cudaGetLastError();
        return fail(nullptr, CPALS_ERR_NOMEM, "%s", "device allocation failed");
    }
    h->dimtree = false;
    e = cudaMemset(h->d_status, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(h->d_fit_count, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(h->lambda, 0, sizeof(double) * R);
    if (e != cudaSuccess) { int rc = cuda_fail(nullptr, e, "memset"); free_all(h); delete h; return rc; }
    *out = reinterpret_cast<cpals_handle*>(h);
    return CPALS_OK;
}

int cpals_set_tensor_kruskal(cpals_handle* hh, const double* mu, const double* const* V, int mem)
{
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h) return fail(nullptr, CPALS_ERR_ARG, "%s", "null handle");
    if (!h->kruskal) return fail(h, CPALS_ERR_STATE, "%s", "the handle was not made by cpals_create_kruskal");
    if (!V || !mem_ok(mem)) return fail(h, CPALS_ERR_ARG, "%s", "bad factor pointers or mem flag");
    for (int m = 0; m < h->N; ++m)
        if (!V[m]) return fail(h, CPALS_ERR_ARG, "%s", "a factor pointer is NULL");
    const int S = h->KS;
    for (int m = 0; m < h->N; ++m)
        CUDA_OR_FAIL(h, cudaMemcpyAsync(h->KV[m], V[m], sizeof(double) * h->dims[m] * S, kind_in(mem), h->stream),
                     "copy Kruskal factor");
    std::vector<double> ones(S, 1.0);   // lives until the synchronisation below
    if (mu) {
        CUDA_OR_FAIL(h, cudaMemcpyAsync(h->Kmu, mu, sizeof(double) * S, kind_in(mem), h->stream), "copy weights");
    } else {
        CUDA_OR_FAIL(h, cudaMemcpyAsync(h->Kmu, ones.data(), sizeof(double) * S, cudaMemcpyHostToDevice, h->stream),
                     "copy weights");
    }
    CUDA_OR_FAIL(h, cpals::kr_norm2(h), "norm of X");
    CUDA_OR_FAIL(h, cudaMemcpyAsync(&h->normX2_host, h->d_normX2, sizeof(double), cudaMemcpyDeviceToHost, h->stream),
                 "norm read");
    CUDA_OR_FAIL(h, cudaStreamSynchronize(h->stream), "set_tensor sync");
    if (!isfinite(h->normX2_host))
        return fail(h, CPALS_ERR_ARG, "%s", "X contains NaN or Inf (or values whose squares overflow FP64)");
    h->have_X = true;
    h->last_sweep_solve = -1;
    factors_changed(h);
    return take_status(h);
}

const char* cpals_last_error(const cpals_handle* hh)
{
    const Handle* h = reinterpret_cast<const Handle*>(hh);
    return h ? h->err : g_create_err;
}

int cpals_set_stream(cpals_handle* hh, void* stream)
{
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h) return fail(nullptr, CPALS_ERR_ARG, "%s", "null handle");
    h->stream = reinterpret_cast<cudaStream_t>(stream);
    return CPALS_OK;
}

int cpals_workspace_bytes(const cpals_handle* hh, size_t* bytes)
{
    const Handle* h = reinterpret_cast<const Handle*>(hh);
    if (!h || !bytes) return CPALS_ERR_ARG;
    *bytes = h->owned_bytes;
    return CPALS_OK;
}

int cpals_set_tensor(cpals_handle* hh, const void* X, int elem, int mem)
{
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h) return fail(nullptr, CPALS_ERR_ARG, "%s", "null handle");
    if (!X) return fail(h, CPALS_ERR_ARG, "%s", "X is NULL");
    if (!mem_ok(mem) || (elem != CPALS_ELEM_F64 && elem != CPALS_ELEM_F32))
        return fail(h, CPALS_ERR_ARG, "%s", "bad elem or mem flag");
    if (elem == CPALS_ELEM_F32 && h->prec == CPALS_F64)
        return fail(h, CPALS_ERR_ARG, "%s", "an FP32 tensor needs precision F32, BF16X3 or TF32X3");
    if (h->kruskal) return fail(h, CPALS_ERR_STATE, "%s", "a Kruskal-input handle takes cpals_set_tensor_kruskal");
    h->X64 = nullptr; h->X32 = nullptr; h->have_X = false;
    if (h->prec == CPALS_F64) {
        if (mem == CPALS_MEM_DEVICE) {
            h->X64 = static_cast<const double*>(X);
        } else {
            if (!h->X64_owned) ALLOC_OR_FAIL(h, dalloc(h, &h->X64_owned, h->P), "allocate X");
            CUDA_OR_FAIL(h, cudaMemcpyAsync(h->X64_owned, X, sizeof(double) * h->P, cudaMemcpyHostToDevice, h->stream),
                         "copy X");
            h->X64 = h->X64_owned;
        }
    } else {
        if (!h->X32_owned && !(elem == CPALS_ELEM_F32 && mem == CPALS_MEM_DEVICE))
            ALLOC_OR_FAIL(h, dalloc(h, &h->X32_owned, h->P), "allocate FP32 X");
        if (elem == CPALS_ELEM_F32) {
            if (mem == CPALS_MEM_DEVICE) {
                h->X32 = static_cast<const float*>(X);
            } else {
                CUDA_OR_FAIL(h, cudaMemcpyAsync(h->X32_owned, X, sizeof(float) * h->P, cudaMemcpyHostToDevice,
                                                h->stream), "copy X");
                h->X32 = h->X32_owned;
            }
        } else {
            const double* src = static_cast<const double*>(X);
            if (mem == CPALS_MEM_HOST) {
                // stage through the owned FP64 buffer
                if (!h->X64_owned) ALLOC_OR_FAIL(h, dalloc(h, &h->X64_owned, h->P), "allocate X staging");
                CUDA_OR_FAIL(h, cudaMemcpyAsync(h->X64_owned, X, sizeof(double) * h->P, cudaMemcpyHostToDevice,
                                                h->stream), "copy X");
                src = h->X64_owned;
            }
            CUDA_OR_FAIL(h, cpals::cast_f64_f32(h, src, h->X32_owned, h->P), "cast X");
            h->X32 = h->X32_owned;
            h->X64 = src;   // the norm uses the FP64 values
        }
    }
    // ||X||^2 and the direct fit use the FP64 values when the caller gave them;
    // the passes over X (Multi-TTM, MTTKRP) read the FP32 copy only
    CUDA_OR_FAIL(h, cpals::norm2(h), "norm of X");
    CUDA_OR_FAIL(h, cudaMemcpyAsync(&h->normX2_host, h->d_normX2, sizeof(double), cudaMemcpyDeviceToHost, h->stream),
                 "norm read");
    CUDA_OR_FAIL(h, cudaStreamSynchronize(h->stream), "set_tensor sync");
    if (!isfinite(h->normX2_host))
        return fail(h, CPALS_ERR_ARG, "%s", "X contains NaN or Inf (or values whose squares overflow FP64)");
    h->have_X = true;
    h->last_sweep_solve = -1;
    return CPALS_OK;
}

int cpals_set_factors(cpals_handle* hh, const double* const* A, const double* lambda, int mem)
{
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h) return fail(nullptr, CPALS_ERR_ARG, "%s", "null handle");
    if (!A || !mem_ok(mem)) return fail(h, CPALS_ERR_ARG, "%s", "bad factor pointers or mem flag");
    for (int m = 0; m < h->N; ++m)
        if (!A[m]) return fail(h, CPALS_ERR_ARG, "%s", "a factor pointer is NULL");
    const int R = h->R;
    for (int m = 0; m < h->N; ++m)
        CUDA_OR_FAIL(h, cudaMemcpyAsync(h->A[m], A[m], sizeof(double) * h->dims[m] * R, kind_in(mem), h->stream),
                     "copy factor");
    if (lambda) {
        CUDA_OR_FAIL(h, cudaMemcpyAsync(h->lambda, lambda, sizeof(double) * R, kind_in(mem), h->stream), "copy lambda");
    } else {
        std::vector<double> ones(R, 1.0);
        CUDA_OR_FAIL(h, cudaMemcpyAsync(h->lambda, ones.data(), sizeof(double) * R, cudaMemcpyHostToDevice, h->stream),
                     "copy lambda");
        CUDA_OR_FAIL(h, cudaStreamSynchronize(h->stream), "sync");
    }
    for (int m = 0; m < h->N; ++m) {
        CUDA_OR_FAIL(h, factor_qr_gram(h, m, true), "factor QR and Gram");
        h->qr_valid[m] = true;
        h->gram_valid[m] = true;
    }
    if (mem == CPALS_MEM_HOST) CUDA_OR_FAIL(h, cudaStreamSynchronize(h->stream), "sync");
    h->have_factors = true;
    h->krp_mode = -1;
    h->last_sweep_solve = -1;
    factors_changed(h);
    return CPALS_OK;
}

int cpals_get_factors(cpals_handle* hh, double* const* A, double* lambda, int mem)
{
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h) return fail(nullptr, CPALS_ERR_ARG, "%s", "null handle");
    if (!mem_ok(mem)) return fail(h, CPALS_ERR_ARG, "%s", "bad mem flag");
    for (int m = 0; m < h->N && A; ++m)
        if (A[m])
            CUDA_OR_FAIL(h, cudaMemcpyAsync(A[m], h->A[m], sizeof(double) * h->dims[m] * h->R, kind_out(mem),
                                            h->stream), "copy factor out");
    if (lambda)
        CUDA_OR_FAIL(h, cudaMemcpyAsync(lambda, h->lambda, sizeof(double) * h->R, kind_out(mem), h->stream),
                     "copy lambda out");
    if (mem == CPALS_MEM_HOST) return take_status(h);
    return CPALS_OK;
}

int cpals_get_factor_qr(cpals_handle* hh, int mode, double* Q, double* R, int mem)
{
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h) return fail(nullptr, CPALS_ERR_ARG, "%s", "null handle");
    if (mode < 0 || mode >= h->N || !mem_ok(mem)) return fail(h, CPALS_ERR_ARG, "%s", "bad mode or mem flag");
    if (!h->have_factors) return fail(h, CPALS_ERR_STATE, "%s", "no factors set");
    CUDA_OR_FAIL(h, refresh_derived(h, CPALS_SOLVE_QR, -1), "refresh QR");
    if (Q) CUDA_OR_FAIL(h, cudaMemcpyAsync(Q, h->Q[mode], sizeof(double) * h->dims[mode] * h->R, kind_out(mem),
                                           h->stream), "copy Q");
    if (R) CUDA_OR_FAIL(h, cudaMemcpyAsync(R, h->Rf[mode], sizeof(double) * h->R * h->R, kind_out(mem), h->stream),
                        "copy R");
    if (mem == CPALS_MEM_HOST) return take_status(h);
    return CPALS_OK;
}

int cpals_set_factor_qr(cpals_handle* hh, const double* const* Q, const double* const* R, int mem)
{
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h) return fail(nullptr, CPALS_ERR_ARG, "%s", "null handle");
    if (!Q || !R || !mem_ok(mem)) return fail(h, CPALS_ERR_ARG, "%s", "bad pointers or mem flag");
    for (int m = 0; m < h->N; ++m) {
        if (!Q[m] || !R[m]) return fail(h, CPALS_ERR_ARG, "%s", "a Q or R pointer is NULL");
        CUDA_OR_FAIL(h, cudaMemcpyAsync(h->Q[m], Q[m], sizeof(double) * h->dims[m] * h->R, kind_in(mem), h->stream),
                     "copy Q");
        CUDA_OR_FAIL(h, cudaMemcpyAsync(h->Rf[m], R[m], sizeof(double) * h->R * h->R, kind_in(mem), h->stream),
                     "copy R");
        h->qr_valid[m] = true;
    }
    if (mem == CPALS_MEM_HOST) CUDA_OR_FAIL(h, cudaStreamSynchronize(h->stream), "sync");
    h->have_factors = true;
    h->krp_mode = -1;
    factors_changed(h);
    return CPALS_OK;
}

int cpals_krp_qr(cpals_handle* hh, int mode, double* Q0, double* R0, int mem)
{
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h) return fail(nullptr, CPALS_ERR_ARG, "%s", "null handle");
    if (mode < 0 || mode >= h->N || !mem_ok(mem)) return fail(h, CPALS_ERR_ARG, "%s", "bad mode or mem flag");
    if (!h->have_factors) return fail(h, CPALS_ERR_STATE, "%s", "no factors set");
    if (Q0 && h->kruskal) return fail(h, CPALS_ERR_ARG, "%s", "a Kruskal-input handle keeps Q0 in factored form");
    CUDA_OR_FAIL(h, refresh_derived(h, CPALS_SOLVE_QR, mode), "refresh QR");
    CUDA_OR_FAIL(h, cpals::krp_qr(h, mode, h->kruskal), "KRP QR");
    h->krp_mode = mode;
    if (Q0) CUDA_OR_FAIL(h, cudaMemcpyAsync(Q0, h->Q0, sizeof(double) * h->RN1 * h->R, kind_out(mem), h->stream),
                         "copy Q0");
    if (R0) CUDA_OR_FAIL(h, cudaMemcpyAsync(R0, h->R0, sizeof(double) * h->R * h->R, kind_out(mem), h->stream),
                         "copy R0");
    if (mem == CPALS_MEM_HOST) return take_status(h);
    return CPALS_OK;
}

int cpals_multi_ttm(cpals_handle* hh, int mode, double* Y, double* W, int mem)
{
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h) return fail(nullptr, CPALS_ERR_ARG, "%s", "null handle");
    if (mode < 0 || mode >= h->N || !mem_ok(mem)) return fail(h, CPALS_ERR_ARG, "%s", "bad mode or mem flag");
    if (!h->have_X) return fail(h, CPALS_ERR_STATE, "%s", "no tensor set");
    if (!h->have_factors) return fail(h, CPALS_ERR_STATE, "%s", "no factors set");
    if (W && h->krp_mode != mode) return fail(h, CPALS_ERR_STATE, "%s", "W needs cpals_krp_qr on this mode first");
    CUDA_OR_FAIL(h, refresh_derived(h, CPALS_SOLVE_QR, mode), "refresh QR");
    const int64_t In = h->dims[mode];
    if (h->kruskal) {
        if (Y && !h->Yn) return fail(h, CPALS_ERR_ARG, "%s", "Y_(n) of this size is not formed for Kruskal input");
        if (Y) CUDA_OR_FAIL(h, cpals::kr_unfold(h, mode, h->Yn), "Kruskal Y");
        if (W) CUDA_OR_FAIL(h, cpals::kr_apply_q0(h, mode), "Kruskal W");
        if (Y) CUDA_OR_FAIL(h, cudaMemcpyAsync(Y, h->Yn, sizeof(double) * In * h->RN1, kind_out(mem), h->stream),
                            "copy Y");
        if (W) CUDA_OR_FAIL(h, cudaMemcpyAsync(W, h->W, sizeof(double) * In * h->R, kind_out(mem), h->stream),
                            "copy W");
        if (mem == CPALS_MEM_HOST) return take_status(h);
        return CPALS_OK;
    }
    CUDA_OR_FAIL(h, cpals::multi_ttm(h, mode, h->Q), "Multi-TTM");
    if (W) CUDA_OR_FAIL(h, cpals::gemm_rows(h, h->Yn, In, h->RN1, h->Q0, h->R, h->W), "apply Q0");
    if (Y) CUDA_OR_FAIL(h, cudaMemcpyAsync(Y, h->Yn, sizeof(double) * In * h->RN1, kind_out(mem), h->stream), "copy Y");
    if (W) CUDA_OR_FAIL(h, cudaMemcpyAsync(W, h->W, sizeof(double) * In * h->R, kind_out(mem), h->stream), "copy W");
    if (mem == CPALS_MEM_HOST) return take_status(h);
    return CPALS_OK;
}

int cpals_ttm_first(cpals_handle* hh, int mode)
{
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h) return fail(nullptr, CPALS_ERR_ARG, "%s", "null handle");
    if (mode < 0 || mode >= h->N) return fail(h, CPALS_ERR_ARG, "%s", "bad mode");
    if (!h->have_X || !h->have_factors) return fail(h, CPALS_ERR_STATE, "%s", "tensor and factors must be set");
    if (h->kruskal) return fail(h, CPALS_ERR_STATE, "%s", "no pass over a dense tensor with Kruskal input");
    CUDA_OR_FAIL(h, refresh_derived(h, CPALS_SOLVE_QR, mode), "refresh QR");
    CUDA_OR_FAIL(h, cpals::ttm_first(h, mode), "first TTM");
    return CPALS_OK;
}

int cpals_mttkrp(cpals_handle* hh, int mode, double* M, int mem)
{
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h) return fail(nullptr, CPALS_ERR_ARG, "%s", "null handle");
    if (mode < 0 || mode >= h->N || !mem_ok(mem)) return fail(h, CPALS_ERR_ARG, "%s", "bad mode or mem flag");
    if (!h->have_X || !h->have_factors) return fail(h, CPALS_ERR_STATE, "%s", "tensor and factors must be set");
    if (h->kruskal) {
        for (int m = 0; m < h->N; ++m)
            if (m != mode && !h->ke_valid[m]) {
                CUDA_OR_FAIL(h, cpals::kr_refresh_e(h, m), "V^T A");
                h->ke_valid[m] = true;
            }
        CUDA_OR_FAIL(h, cpals::kr_mttkrp(h, mode), "Kruskal MTTKRP");
    } else {
        CUDA_OR_FAIL(h, cpals::mttkrp(h, mode), "MTTKRP");
    }
    if (M) CUDA_OR_FAIL(h, cudaMemcpyAsync(M, h->M, sizeof(double) * h->dims[mode] * h->R, kind_out(mem), h->stream),
                        "copy M");
    if (mem == CPALS_MEM_HOST) return take_status(h);
    return CPALS_OK;
}

int cpals_solve_mode(cpals_handle* hh, int mode, int solve, double svd_rtol)
{
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h) return fail(nullptr, CPALS_ERR_ARG, "%s", "null handle");
    if (mode < 0 || mode >= h->N) return fail(h, CPALS_ERR_ARG, "%s", "bad mode");
    if (solve < CPALS_SOLVE_QR || solve > CPALS_SOLVE_NORMAL_PINV) return fail(h, CPALS_ERR_ARG, "%s", "bad solve kind");
    if (!h->have_X || !h->have_factors) return fail(h, CPALS_ERR_STATE, "%s", "tensor and factors must be set");
    CUDA_OR_FAIL(h, mode_update(h, mode, solve, svd_rtol), "mode update");
    h->last_sweep_solve = -1;
    return CPALS_OK;
}

int cpals_iterate(cpals_handle* hh, int iters, double tol, int solve, double svd_rtol, int* done, double* fits_host)
{
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h) return fail(nullptr, CPALS_ERR_ARG, "%s", "null handle");
    if (done) *done = 0;
    if (iters < 0 || tol < 0.0) return fail(h, CPALS_ERR_ARG, "%s", "iters and tol must be >= 0");
    if (solve < CPALS_SOLVE_QR || solve > CPALS_SOLVE_NORMAL_PINV) return fail(h, CPALS_ERR_ARG, "%s", "bad solve kind");
    if (!h->have_X || !h->have_factors) return fail(h, CPALS_ERR_STATE, "%s", "tensor and factors must be set");
    if (iters == 0) return CPALS_OK;
    // derived data valid for every mode, so that one captured sweep fits all
    CUDA_OR_FAIL(h, refresh_derived(h, solve, -1), "refresh derived factors");
    CUDA_OR_FAIL(h, cudaMemsetAsync(h->d_fit_count, 0, sizeof(int), h->stream), "reset fit count");
    if (h->graph[solve] && h->graph_rtol[solve] != svd_rtol) {
        cudaGraphExecDestroy(h->graph[solve]);
        h->graph[solve] = nullptr;
    }
    if (!h->graph[solve]) {
        // capture one sweep
        cudaStream_t cap = h->stream;
        bool own = false;
        if (cap == nullptr) {
            CUDA_OR_FAIL(h, cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "capture stream");
            own = true;
            CUDA_OR_FAIL(h, cudaDeviceSynchronize(), "sync before capture");
        }
        cudaStream_t saved = h->stream;
        h->stream = cap;
        const int64_t l0 = h->launches;
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        cudaError_t e2 = cudaSuccess;
        if (e == cudaSuccess) {
            e2 = sweep(h, solve, svd_rtol);
            e = cudaStreamEndCapture(cap, &g);
        }
        h->stream = saved;
        if (own) cudaStreamDestroy(cap);
        if (e2 != cudaSuccess) { if (g) cudaGraphDestroy(g); return cuda_fail(h, e2, "capture sweep"); }
        CUDA_OR_FAIL(h, e, "end capture");
        cudaGraphExec_t ge = nullptr;
        e = cudaGraphInstantiate(&ge, g, 0);
        cudaGraphDestroy(g);
        CUDA_OR_FAIL(h, e, "instantiate sweep graph");
        h->graph[solve] = ge;
        h->graph_rtol[solve] = svd_rtol;
        h->graph_nodes[solve] = h->launches - l0;
        h->launches = l0;
    }
    int ran = 0;
    double prev = 0.0;
    for (int it = 0; it < iters; ++it) {
        CUDA_OR_FAIL(h, cudaGraphLaunch(h->graph[solve], h->stream), "launch sweep graph");
        h->launches += h->graph_nodes[solve];
        ++ran;
        if (tol > 0.0) {
            double f = 0.0;
            CUDA_OR_FAIL(h, cudaMemcpyAsync(&f, h->d_fit + h->fit_cap, sizeof(double), cudaMemcpyDeviceToHost,
                                            h->stream), "fit read");
            int st = take_status(h);
            if (st != CPALS_OK) { if (done) *done = ran; return st; }
            if (it > 0 && fabs(f - prev) < tol) break;
            prev = f;
        }
    }
    h->last_sweep_solve = solve;
    if (done) *done = ran;
    if (fits_host) {
        const int n = std::min(ran, h->fit_cap);
        CUDA_OR_FAIL(h, cudaMemcpyAsync(fits_host, h->d_fit, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream),
                     "fit history read");
    }
    return take_status(h);
}

int cpals_profile_sweeps(cpals_handle* hh, int sweeps, int solve, double svd_rtol, double* bucket_ms)
{
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h) return fail(nullptr, CPALS_ERR_ARG, "%s", "null handle");
    if (sweeps < 1 || sweeps > 16 || !bucket_ms) return fail(h, CPALS_ERR_ARG, "%s", "sweeps in [1, 16], bucket_ms");
    if (solve < CPALS_SOLVE_QR || solve > CPALS_SOLVE_NORMAL_PINV) return fail(h, CPALS_ERR_ARG, "%s", "bad solve kind");
    if (!h->have_X || !h->have_factors) return fail(h, CPALS_ERR_STATE, "%s", "tensor and factors must be set");
    for (int i = 0; i < cpals::kProfMax; ++i) {
        if (!h->prof_a[i]) CUDA_OR_FAIL(h, cudaEventCreate(&h->prof_a[i]), "profile events");
        if (!h->prof_b[i]) CUDA_OR_FAIL(h, cudaEventCreate(&h->prof_b[i]), "profile events");
    }
    CUDA_OR_FAIL(h, refresh_derived(h, solve, -1), "refresh derived factors");
    CUDA_OR_FAIL(h, cudaMemsetAsync(h->d_fit_count, 0, sizeof(int), h->stream), "reset fit count");
    // every phase on the handle's stream, one after the other
    cudaStream_t side = h->side;
    h->side = h->stream;
    h->prof = true;
    h->prof_n = 0;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < sweeps && e == cudaSuccess; ++k) e = sweep(h, solve, svd_rtol);
    h->prof = false;
    h->side = side;
    CUDA_OR_FAIL(h, e, "profiled sweep");
    CUDA_OR_FAIL(h, cudaStreamSynchronize(h->stream), "profile sync");
    for (int b = 0; b < cpals::kProfBuckets; ++b) bucket_ms[b] = 0.0;
    for (int i = 0; i < h->prof_n; ++i) {
        float ms = 0.f;
        CUDA_OR_FAIL(h, cudaEventElapsedTime(&ms, h->prof_a[i], h->prof_b[i]), "profile event time");
        bucket_ms[h->prof_bucket[i]] += ms / sweeps;
    }
    if (h->prof_n >= cpals::kProfMax) return fail(h, CPALS_ERR_ARG, "%s", "too many phases: profile fewer sweeps");
    h->last_sweep_solve = solve;
    return take_status(h);
}

int cpals_fit(cpals_handle* hh, int direct, double* fit_host)
{
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h) return fail(nullptr, CPALS_ERR_ARG, "%s", "null handle");
    if (!fit_host) return fail(h, CPALS_ERR_ARG, "%s", "fit_host is NULL");
    if (!h->have_X || !h->have_factors) return fail(h, CPALS_ERR_STATE, "%s", "tensor and factors must be set");
    if (direct) {
        double* d_res = h->d_fit + h->fit_cap;   // reuse the "last fit" slot for the residual
        double res2 = 0.0;
        if (h->kruskal) CUDA_OR_FAIL(h, cpals::kr_residual(h, d_res), "direct residual");
        else CUDA_OR_FAIL(h, cpals::residual_direct(h, d_res), "direct residual");
        CUDA_OR_FAIL(h, cudaMemcpyAsync(&res2, d_res, sizeof(double), cudaMemcpyDeviceToHost, h->stream), "read");
        int st = take_status(h);
        if (st != CPALS_OK) return st;
        *fit_host = 1.0 - sqrt(std::max(res2, 0.0)) / sqrt(h->normX2_host);
        return CPALS_OK;
    }
    if (h->last_sweep_solve < 0) return fail(h, CPALS_ERR_STATE, "%s", "the efficient fit needs a finished sweep");
    CUDA_OR_FAIL(h, cudaMemcpyAsync(fit_host, h->d_fit + h->fit_cap, sizeof(double), cudaMemcpyDeviceToHost, h->stream),
                 "fit read");
    return take_status(h);
}

int cpals_sync(cpals_handle* hh)
{
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h) return fail(nullptr, CPALS_ERR_ARG, "%s", "null handle");
    return take_status(h);
}

int cpals_set_option(cpals_handle* hh, int option, int64_t value)
{
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h) return fail(nullptr, CPALS_ERR_ARG, "%s", "null handle");
    if (option == CPALS_OPT_FUSED_TAIL) {
        if (value < 0 || value > 2) return fail(h, CPALS_ERR_ARG, "%s", "unknown option or value");
        const bool a = value == 2, f = value == 1;
        if (a != h->fused_tail_auto || (!a && f != h->fused_tail)) {
            h->fused_tail_auto = a;
            if (!a) h->fused_tail = f;
            for (int s = 0; s < 4; ++s)         // captured sweeps hold the old kernels and schedule
                if (h->graph[s]) { cudaGraphExecDestroy(h->graph[s]); h->graph[s] = nullptr; }
        }
        return CPALS_OK;
    }
    bool* field = nullptr;
    switch (option) {
        case CPALS_OPT_DIMTREE: field = &h->dimtree; break;
        case CPALS_OPT_TC_PIPELINE: field = &h->tc_pipe; break;
        case CPALS_OPT_KRP_TREE: field = &h->krp_tree; break;
        case CPALS_OPT_F32_PIPELINE: field = &h->f32_pipe; break;
        case CPALS_OPT_TEST_WITHHOLD_COPIES: field = &h->test_withhold; break;
        case CPALS_OPT_SVD_SHORTCUT: field = &h->svd_shortcut; break;
        case CPALS_OPT_APPLY_Q0_FP32: field = &h->q0_fp32; break;
        case CPALS_OPT_WIDE_TAIL: field = &h->wide_tail; break;
        default: break;
    }
    if (!field || (value != 0 && value != 1)) return fail(h, CPALS_ERR_ARG, "%s", "unknown option or value");
    const bool v = value != 0;
    if (v != *field) {
        *field = v;
        for (int s = 0; s < 4; ++s)             // captured sweeps hold the old kernels and schedule
            if (h->graph[s]) { cudaGraphExecDestroy(h->graph[s]); h->graph[s] = nullptr; }
    }
    return CPALS_OK;
}

int cpals_test_newton_recip(const double* x, int64_t n, double* rcp, double* rsqrt)
{
    if (n < 0 || (n > 0 && (!x || !rcp || !rsqrt))) return fail(nullptr, CPALS_ERR_ARG, "%s", "bad arguments");
    cudaError_t e = cpals::recip_check(x, n, rcp, rsqrt, nullptr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "reciprocal check");
    return CPALS_OK;
}

int cpals_test_fail_allocation(int nth)
{
    if (nth < 0) return fail(nullptr, CPALS_ERR_ARG, "%s", "nth must be >= 0");
    g_fail_alloc_in.store(nth);
    return CPALS_OK;
}

int64_t cpals_launch_count(const cpals_handle* hh)
{
    const Handle* h = reinterpret_cast<const Handle*>(hh);
    return h ? h->launches : -1;
}

int cpals_multi_ttm_static(const int64_t* dims, int N, int rank, int mode, const double* X,
                           const double* const* Q, double* Y, void* stream)
{
    if (!dims || !X || !Q || !Y) return fail(nullptr, CPALS_ERR_ARG, "%s", "a pointer argument is NULL");
    if (N < 2 || N > cpals::kMaxN) {
        snprintf(g_create_err, sizeof(g_create_err), "N must be in [2, %d]", cpals::kMaxN);
        return CPALS_ERR_ARG;
    }
    if (rank < 1 || rank > cpals::kMaxRank) {
        snprintf(g_create_err, sizeof(g_create_err), "rank must be in [1, %d]", cpals::kMaxRank);
        return CPALS_ERR_ARG;
    }
    if (mode < 0 || mode >= N) return fail(nullptr, CPALS_ERR_ARG, "%s", "bad mode");
    for (int m = 0; m < N; ++m) {
        if (dims[m] < rank) return fail(nullptr, CPALS_ERR_ARG, "%s", "rank must not exceed any dim");
        if (m != mode && !Q[m]) return fail(nullptr, CPALS_ERR_ARG, "%s", "a Q pointer is NULL");
    }
    int64_t P = 0;
    if (!cpals::checked_prod(N, dims, &P))
        return fail(nullptr, CPALS_ERR_ARG, "%s", "prod(dims) does not fit in 64 bits");
    cpals::StaticPlan sp{};
    cudaError_t e = cpals::multi_ttm_static_plan(N, dims, rank, mode, &sp);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "device query");
    if (!sp.ok) {
        snprintf(g_create_err, sizeof(g_create_err),
                 "problem too large for the static scratch: the two largest TTM intermediates need %lld doubles, "
                 "the fixed array holds %lld",
                 (long long)(sp.s0 + sp.s1), (long long)cpals::multi_ttm_static_capacity());
        return CPALS_ERR_ARG;
    }
    e = cpals::multi_ttm_static(N, dims, rank, mode, X, Q, Y, reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "static Multi-TTM");
    return CPALS_OK;
}

// ---------------------------------------------------------------- batched problems
int cpals_batch_create(int count, const int64_t* dims, const int* ranks, cpals_batch** out)
{
    if (!out) return fail(nullptr, CPALS_ERR_ARG, "%s", "out is NULL");
    *out = nullptr;
    if (count < 1 || !dims || !ranks) return fail(nullptr, CPALS_ERR_ARG, "%s", "count >= 1 with dims and ranks");
    int maxR = 0, maxI = 0;
    for (int p = 0; p < count; ++p) {
        const int R = ranks[p];
        if (R < 1 || R > 16) return fail(nullptr, CPALS_ERR_ARG, "%s", "batched ranks must be in [1, 16]");
        for (int m = 0; m < 3; ++m) {
            const int64_t d = dims[3 * p + m];
            if (d < R || d > 4096)
                return fail(nullptr, CPALS_ERR_ARG, "%s", "batched dims must be in [rank, 4096]");
            maxI = std::max<int>(maxI, (int)d);
        }
        maxR = std::max(maxR, R);
    }
    if (cpals::batch_smem_bytes(maxR, maxI) > 220 * 1024)
        return fail(nullptr, CPALS_ERR_ARG, "%s", "batched problem too large for one CTA's shared memory");
    cpals::Batch* b = cpals::batch_new();
    if (!b) return fail(nullptr, CPALS_ERR_NOMEM, "%s", "host allocation failed");
    cudaError_t e = cpals::batch_build(b, count, dims, ranks);
    if (e != cudaSuccess) {
        cpals::batch_delete(b);
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? fail(nullptr, CPALS_ERR_NOMEM, "%s", "device allocation failed")
                                              : cuda_fail(nullptr, e, "batch create");
    }
    *out = reinterpret_cast<cpals_batch*>(b);
    return CPALS_OK;
}

int cpals_batch_destroy(cpals_batch* bb)
{
    cpals::batch_delete(reinterpret_cast<cpals::Batch*>(bb));
    return CPALS_OK;
}

int cpals_batch_set_stream(cpals_batch* bb, void* stream)
{
    auto* b = reinterpret_cast<cpals::Batch*>(bb);
    if (!b) return fail(nullptr, CPALS_ERR_ARG, "%s", "null batch");
    cpals::batch_set_stream(b, reinterpret_cast<cudaStream_t>(stream));
    return CPALS_OK;
}

int cpals_batch_set_tensors(cpals_batch* bb, const float* const* X, int mem)
{
    auto* b = reinterpret_cast<cpals::Batch*>(bb);
    if (!b || !X || !mem_ok(mem)) return fail(nullptr, CPALS_ERR_ARG, "%s", "bad batch, tensors or mem flag");
    cudaError_t e = cpals::batch_set_tensors(b, X, mem == CPALS_MEM_HOST);
    return e == cudaSuccess ? CPALS_OK : cuda_fail(nullptr, e, "batch set tensors");
}

int cpals_batch_set_factors(cpals_batch* bb, const double* const* A, int mem)
{
    auto* b = reinterpret_cast<cpals::Batch*>(bb);
    if (!b || !A || !mem_ok(mem)) return fail(nullptr, CPALS_ERR_ARG, "%s", "bad batch, factors or mem flag");
    cudaError_t e = cpals::batch_set_factors(b, A, mem == CPALS_MEM_HOST);
    return e == cudaSuccess ? CPALS_OK : cuda_fail(nullptr, e, "batch set factors");
}

int cpals_batch_get_factors(cpals_batch* bb, double* const* A, double* const* lambda, int mem)
{
    auto* b = reinterpret_cast<cpals::Batch*>(bb);
    if (!b || !mem_ok(mem)) return fail(nullptr, CPALS_ERR_ARG, "%s", "bad batch or mem flag");
    cudaError_t e = cpals::batch_get_factors(b, A, lambda, mem == CPALS_MEM_HOST);
    return e == cudaSuccess ? CPALS_OK : cuda_fail(nullptr, e, "batch get factors");
}

int cpals_batch_iterate(cpals_batch* bb, int iters, double* fits_host, int* status_host)
{
    auto* b = reinterpret_cast<cpals::Batch*>(bb);
    if (!b || iters < 0) return fail(nullptr, CPALS_ERR_ARG, "%s", "bad batch or iteration count");
    if (!cpals::batch_ready(b)) return fail(nullptr, CPALS_ERR_STATE, "%s", "tensors and factors must be set");
    cudaError_t e = cpals::batch_iterate(b, iters, fits_host, status_host);
    return e == cudaSuccess ? CPALS_OK : cuda_fail(nullptr, e, "batch iterate");
}

int64_t cpals_batch_launch_count(const cpals_batch* bb)
{
    const auto* b = reinterpret_cast<const cpals::Batch*>(bb);
    return b ? cpals::batch_launches(b) : -1;
}

int cpals_batch_launch_shape(const cpals_batch* bb, int* grid, int* threads)
{
    const auto* b = reinterpret_cast<const cpals::Batch*>(bb);
    if (!b) return CPALS_ERR_ARG;
    if (grid) *grid = cpals::batch_tuned_grid(b);
    if (threads) *threads = cpals::batch_tuned_threads(b);
    return CPALS_OK;
}

int cpals_probe_fma_peak(double ms_target, double* fp64_tflops, double* fp32_tflops)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CPALS_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return CPALS_ERR_CUDA;
    const int blocks = sms * 4, threads = 256;
    void* out = nullptr;
    if (cudaMalloc(&out, sizeof(double) * blocks * threads) != cudaSuccess) return CPALS_ERR_NOMEM;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double res[2] = {0, 0};
    for (int which = 0; which < 2; ++which) {
        int iters = which == 0 ? 2000 : 100000;
        float ms = 0.f;
        for (int rep = 0; rep < 8; ++rep) {
            cudaEventRecord(e0);
            if (which == 0) fma_probe_kernel<double><<<blocks, threads>>>((double*)out, iters, 0.999999, 1e-7);
            else fma_probe_kernel<float><<<blocks, threads>>>((float*)out, iters, 0.999999f, 1e-7f);
            cudaEventRecord(e1);
            cudaEventSynchronize(e1);
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < 0.5 * ms_target && iters < (1 << 28)) { iters *= 2; continue; }
            const double flops = 2.0 * 8 * (double)iters * blocks * threads;
            res[which] = std::max(res[which], flops / (ms * 1e-3) / 1e12);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (cudaGetLastError() != cudaSuccess) return CPALS_ERR_CUDA;
    if (fp64_tflops) *fp64_tflops = res[0];
    if (fp32_tflops) *fp32_tflops = res[1];
    return CPALS_OK;
}

}  // extern "C"
