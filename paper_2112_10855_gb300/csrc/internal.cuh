// internal.cuh -- handle layout and kernel launchers shared by the CUDA
// translation units of libcpals.  Not part of the public C-ABI (include/cpals.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include "../../include/cpals.h"
#include "ttm_plan.h"

namespace cpals {

// Device status word values (a subset of cpals_status).
constexpr int kStatusOk = 0;

// kMaxN, kMaxRank, TtmShape, ttm_shape and ttm_order come from ttm_plan.h.

// Phase buckets of cpals_profile_sweeps (the component breakdown of the
// paper's Table its_parts): the pass over X (Multi-TTM, or MTTKRP), the
// factor QR (or Gram), computing Q0 (QR of V_n), applying Q0 (W = Y_(n) Q0),
// and the rest (solve operators, fit).
enum { kProfTTM = 0, kProfFactor = 1, kProfQ0 = 2, kProfApplyQ0 = 3, kProfOther = 4, kProfBuckets = 5 };
constexpr int kProfMax = 1024;

// ------------------------------------------------------------------ handle
// Workspace of the GPU-wide CholeskyQR2 (one allocation, carved up): the
// Gram partials of the row blocks, their group sums, the column sums of
// squares of the row blocks, lambda, R1, R1^-1, R2^-1, R2, a fold step's
// first Gram and the reciprocals of the diagonals of R1 and R2.
struct WideWs {
    double* base = nullptr;
    double* parts = nullptr;
    double* gparts = nullptr;
    double* cparts = nullptr;
    double* lam = nullptr;
    double* R1 = nullptr;
    double* X1 = nullptr;
    double* X2 = nullptr;
    double* R2 = nullptr;
    double* Gh = nullptr;
    double* D1 = nullptr;
    double* D2 = nullptr;
};

struct Handle {
    int N = 0, R = 0, prec = CPALS_F64;
    int64_t dims[kMaxN] = {0};
    int64_t P = 0;        // prod dims
    int64_t RN1 = 0;      // R^{N-1}
    int64_t Imax = 0;
    cudaStream_t stream = nullptr;
    int device = 0, num_sms = 0;

    // data tensor
    const double* X64 = nullptr;
    const float* X32 = nullptr;
    double* X64_owned = nullptr;
    float* X32_owned = nullptr;
    bool have_X = false, have_factors = false;
    double normX2_host = 0.0;

    // factors and their QR / Gram (device, FP64)
    double* A[kMaxN] = {nullptr};
    double* Q[kMaxN] = {nullptr};
    double* Rf[kMaxN] = {nullptr};
    double* G[kMaxN] = {nullptr};
    double* lambda = nullptr;
    // host-side validity of the derived data of each factor (the QR for the
    // QR/SVD solves, the Gram for the normal equations)
    bool qr_valid[kMaxN] = {false};
    bool gram_valid[kMaxN] = {false};

    // per-mode-update buffers
    double* Q0 = nullptr;    // R^{N-1} x R
    double* R0 = nullptr;    // R x R
    double* Yn = nullptr;    // Imax x R^{N-1} (unfolding, FP64)
    double* W = nullptr;     // Imax x R
    float* W32 = nullptr;    // Imax x R: W in FP32 before widening (mixed precisions)
    // mixed precisions inside a mode update: the Multi-TTM leaves an FP32
    // unfolding (yn32, in a TTM buffer) for W = Y_(n) Q0 in FP32
    bool yn32_mode = false;
    bool q0_fp32 = true;     // CPALS_OPT_APPLY_Q0_FP32
    const float* yn32 = nullptr;
    double* Ahat = nullptr;  // Imax x R
    double* M = nullptr;     // Imax x R (MTTKRP)
    double* S = nullptr;     // R x R (Hadamard of Grams)
    double* T = nullptr;     // R x R solve operator (SVD path)
    // structured QR of V_n: Khatri-Rao of two R x R factors, its Q, the two
    // ping-pong R factors, and the ping-pong partial Q0 (up to R^{N-1} x R)
    double* KM = nullptr;    // R^2 x R
    double* KQ = nullptr;    // R^2 x R
    double* KR[2] = {nullptr, nullptr};
    double* KQb[2] = {nullptr, nullptr};
    int krp_mode = -1;       // mode whose Q0/R0 are current
    // tree-structured QR of V_n in a dimension-tree sweep: the QR of the
    // Khatri-Rao product of each half's R_m (HQ[s] rows x R, HR[s]), computed
    // once per sweep; a half of one mode keeps Q = I and R = its own R_m.
    // Qin holds the inner fold (R x own factors) before the Kronecker apply.
    bool krp_tree = true;
    bool f32_pipe = true;    // FP32 TTMs through the TMA-fed CUDA-core pipeline where the shape allows
    double* HQ[2] = {nullptr, nullptr};
    double* HR[2] = {nullptr, nullptr};
    const double* hr_ptr[2] = {nullptr, nullptr};
    bool hq_single[2] = {false, false};
    int64_t hq_rows[2] = {0, 0};
    double* Qin = nullptr;

    // TTM intermediates (ping-pong), in the Multi-TTM's arithmetic type
    void* tbuf[2] = {nullptr, nullptr};
    int64_t tbuf_elems = 0;
    // dimension tree (Sec. 3.3.3): X contracted over one half of the modes,
    // shared by the Multi-TTMs of the other half within a sweep
    void* tA = nullptr;
    int64_t tA_elems = 0;
    int64_t tA_dims[kMaxN] = {0};
    int tA_contracted[kMaxN] = {0};
    int tA_rank = -1;        // normal-equations partial: position of the rank index
    bool dimtree = true;
    // first TTM on the tensor cores through the persistent TMA pipeline when
    // the shape allows it (else one CTA per 128-row tile)
    bool tc_pipe = true;
    // test hook: the persistent tensor-core pipeline issues no copies of X and
    // its waits give up after 1 ms (CPALS_OPT_TEST_WITHHOLD_COPIES)
    bool test_withhold = false;
    // FP64 scratch for split-K partials, reductions and pre-split tensor-core
    // tiles (main stream), and a separate workspace for the TSQR levels, so a QR
    // on the side stream never shares memory with the Multi-TTM
    double* scratch = nullptr;
    int64_t scratch_elems = 0;
    double* qr_ws = nullptr;
    int64_t qr_ws_elems = 0;
    // side stream (higher priority) for the QR of V_n, which overlaps the
    // Multi-TTM; fork/join events
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;

    // device scalars
    int* d_status = nullptr;
    int* d_gate = nullptr;          // fused tail: 1 when the factor QR falls back to Householder
    double* svd_parts = nullptr;    // SVD solve: per-column norms of R0^-1 and R0 (the truncation test)
    int* d_vgate = nullptr;         // QR of a Khatri-Rao fold step: 1 when the staircase Householder must run
    double* VG = nullptr;           // R x R: the Gram of a fold step (written by its CholeskyQR2)
    bool svd_shortcut = true;       // CPALS_OPT_SVD_SHORTCUT
    bool fused_tail = true;         // CPALS_OPT_FUSED_TAIL = 1 / 0
    bool fused_tail_auto = true;    // CPALS_OPT_FUSED_TAIL = 2 (the default)
    bool wide_tail = true;          // CPALS_OPT_WIDE_TAIL
    // GPU-wide CholeskyQR2 above rank 32 (tail.cu): [0] serves the mode tails
    // and factor QRs (main stream), [1] the fold steps of the QR of V_n (side
    // stream), so the two never share memory
    WideWs wide[2];
    double* d_normX2 = nullptr;
    double* d_fit = nullptr;        // fit history ring
    int* d_fit_count = nullptr;
    int fit_cap = 0;
    int last_sweep_solve = -1;      // solve kind of the last finished sweep

    // graphs, one per solve kind
    cudaGraphExec_t graph[4] = {nullptr, nullptr, nullptr, nullptr};
    double graph_rtol[4] = {0, 0, 0, 0};
    int64_t graph_nodes[4] = {0, 0, 0, 0};

    int64_t launches = 0;
    // phase timing: while prof is set, an eagerly run sweep records a pair of
    // events on the handle's stream around each phase (prof_n pairs so far)
    bool prof = false;
    int prof_n = 0;
    int prof_bucket[kProfMax] = {0};
    cudaEvent_t prof_a[kProfMax] = {nullptr};
    cudaEvent_t prof_b[kProfMax] = {nullptr};
    // Kruskal-tensor input (Sec. 3.3.2): X = sum_s mu_s v_s^(1) o ... o v_s^(N),
    // V_m = KV[m] (I_m x S); C_m = Q_m^T V_m (R x S) for the QR solves, E_m =
    // V_m^T A_m (S x R) for the normal equations; the Gram V_m^T V_m of each
    // mode (S x S, for ||X||^2); the fold factors of the QR of V_n (KP: up to
    // N-2 matrices of R^2 x R) and two S x R work matrices.
    bool kruskal = false;
    int KS = 0;
    double* KV[kMaxN] = {nullptr};
    double* KC[kMaxN] = {nullptr};
    double* KE[kMaxN] = {nullptr};
    bool kc_valid[kMaxN] = {false};
    bool ke_valid[kMaxN] = {false};
    double* Kmu = nullptr;
    double* KGV = nullptr;
    double* KP = nullptr;
    double* KMw[2] = {nullptr, nullptr};

    size_t owned_bytes = 0;
    char err[512] = {0};
};

// Whether the end of the mode updates and the factor QRs run in the fused
// kernels (tail.cu): CPALS_OPT_FUSED_TAIL = 1 always, 0 never, 2 (the
// default) from rank kFusedTailMinR up.  Below it the separate kernels
// measured faster (a 4-way 128^4 rank-4 sweep: 3935 against 3260 per second),
// since a Householder QR of four or five columns is short; from rank 10 the
// fused kernels win.  The choice depends on the handle's rank only, so every
// factor QR of a handle takes the same path.
constexpr int kFusedTailMinR = 8;
inline bool tail_fused(const Handle* h) { return h->fused_tail_auto ? h->R >= kFusedTailMinR : h->fused_tail; }

// ------------------------------------------------------------------ launchers
// All launchers enqueue on h->stream, count their launches in h->launches
// and return cudaGetLastError().

// Multi-TTM (Alg. cp-als-qr Multi-TTM step): writes the FP64 unfolding Y_(n)
// into h->Yn using Q_m = h->Q[m] (or the given override array).
cudaError_t multi_ttm(Handle* h, int n, const double* const* Q);
// Dimension tree: X contracted over `modes` into h->tA; then Y_(n) for a mode of
// the other half from h->tA (the remaining modes other than n).
cudaError_t dimtree_pass(Handle* h, const int* modes, int nm);
cudaError_t multi_ttm_from_partial(Handle* h, int n);
// Only the first TTM of the Multi-TTM of mode n (the pass over X).
cudaError_t ttm_first(Handle* h, int n);
// Multi-TTM with all scratch in a fixed file-scope device array (no allocation).
cudaError_t multi_ttm_static(int N, const int64_t* dims, int R, int n, const double* X, const double* const* Q,
                             double* Y, cudaStream_t stream);
int64_t multi_ttm_static_capacity();
cudaError_t multi_ttm_static_plan(int N, const int64_t* dims, int R, int n, StaticPlan* out);
// First TTM on the tcgen05 tensor cores with split products (FP32 X):
// 3 x bf16 (kind::f16) or, with tf32 = true, 3 x tf32 (kind::tf32).
bool tc_supported(int R);
// FP32 TTM on the CUDA cores fed by the TMA ring of the tensor-core pipeline
// (L % 4 == 0, 16-byte aligned tensors, R <= 64; f32_pipe_ok says when).
bool f32_pipe_ok(const float* in, const float* out, TtmShape s, int R);
cudaError_t ttm_f32_pipe(Handle* h, const float* in, const double* Q, int64_t ldq, float* out, TtmShape s, int R);
cudaError_t ttm_split_tc(Handle* h, const float* in, const double* Q, int64_t ldq, float* out, TtmShape s, int R,
                         bool tf32);
// MTTKRP M_n = X_(n) Z_n (Alg. cp-als) into h->M.
cudaError_t mttkrp(Handle* h, int n);
// Dimension tree for the MTTKRP: X contracted over `modes` (full TTM with the
// first A_m, then diagonal contractions) into h->tA; then M_n from h->tA.
cudaError_t mttkrp_tree_pass(Handle* h, const int* modes, int nm);
cudaError_t mttkrp_from_partial(Handle* h, int n);
// Squared Frobenius norm of X into h->d_normX2.
cudaError_t norm2(Handle* h);
// FP64 -> FP32 copy with round-to-nearest-even.
cudaError_t cast_f64_f32(Handle* h, const double* src, float* dst, int64_t n);
// Direct residual ||X - Xhat||^2 into *d_out.
cudaError_t residual_direct(Handle* h, double* d_out);

// Householder QR with explicit Q and diag(R) >= 0 (Sec. 2.1).  A is m x n
// (lda = m), Q is m x n, R is n x n.  A may alias Q.
// dense = false for structured inputs (Khatri-Rao steps, triangular factors),
// whose leaves keep the kernel that skips identity reflectors.
// gate (device int, may be NULL): the kernels return at once while *gate == 0
// (the fused mode tail writes it: 1 when its CholeskyQR2 was refused).
cudaError_t householder_qr(Handle* h, const double* A, int64_t m, int n, double* Q, double* R, bool dense = true,
                           const int* gate = nullptr);
// The end of a mode update in one thread-block cluster (tail.cu): the solve
// (kind 0: Ahat R0^T = W; 1: Ahat = W T; 2: Ahat S = M with S = L L^T; 3: Ahat
// given in h->Ahat), lambda, A_n, G_n and, with want_qr, Q_n R_n by
// CholeskyQR2 (h->d_gate = 1 when the Householder QR has to take over).
// kind: 0..2 solve from W (an R x R operator), 3 from Ahat, 4 the QR of a
// given matrix; the default asks about every kind.
bool mode_tail_ok(int64_t I, int R, int kind = 1);
// The tail's Newton-Raphson 1/x and 1/sqrt(x) on n values (for their accuracy test).
cudaError_t recip_check(const double* x, int64_t n, double* rcp, double* rsq, cudaStream_t st);
cudaError_t mode_tail(Handle* h, int n, int kind, const double* W, const double* Op, bool want_qr);
// The same kernel's QR alone (CholeskyQR2 with its check) of an explicit
// rows x R matrix V: Q (rows x R), R (R x R), the Gram V^T V into G (R x R);
// *gate = 1 when CholeskyQR2 was refused and a Householder QR has to follow.
// V = F (.) B for upper-triangular R x R factors F, B (a Khatri-Rao fold step,
// B's row index fastest) may pass them: above rank 32 the first Gram is then
// (F^T F) * (B^T B) instead of a pass over V.
cudaError_t cqr2_rows(Handle* h, const double* V, int64_t rows, double* Q, double* Rout, double* G, int* gate,
                      const double* F = nullptr, const double* B = nullptr);
// True when the tail of kind 3 or 4 (and cqr2_rows) runs the GPU-wide
// CholeskyQR2 kernels instead of the cluster kernel (rank above 32); those
// take any number of rows.
bool wide_tail_on(const Handle* h);
// Elements of one GPU-wide CholeskyQR2 workspace for rank R, and carving it up.
int64_t wide_ws_elems(int R, int num_sms);
void wide_ws_carve(WideWs& ws, int R, int num_sms);
// QR of V_n (Khatri-Rao of the R_m, Sec. 3.1) into h->Q0, h->R0 (structured, V_n not formed).
// With implicit = true Q0 is not formed either: the Q factors of the fold steps
// go to h->KP (for the Kruskal-input path) and only R0 is written.
cudaError_t krp_qr(Handle* h, int n, bool implicit = false);
// QR of the Khatri-Rao product of the upper-triangular factors Rl[cnt-1] (.)
// ... (.) Rl[0] (Rl[0] fastest), cnt >= 2, by the Kronecker fold; explicit Q
// to Qout (R^cnt x R) and R to Rout, or the step Q's to h->KP (implicit).
cudaError_t fold_qr(Handle* h, const double* const* Rl, int cnt, double* Qout, double* Rout, bool implicit);
// QR of the Khatri-Rao product of the R_m of one half of the modes (ascending
// list) into h->HQ[slot], h->HR[slot] (a single mode: Q = I, R = its R_m).
cudaError_t krp_qr_half(Handle* h, const int* modes, int cnt, int slot);
// Q0, R0 of V_n from the QR of the other half (slot) and the R_m of the own
// half's other modes (ascending list own[0..nown)): other_left = true when the
// other half holds the higher (slower) modes.
cudaError_t krp_qr_tree(Handle* h, int n, int slot, bool other_left, const int* own, int nown);
// C (m x n) = A (m x k) B (k x n), FP64, column-major, on the TTM kernel (one thread per output row, R-wide
// register tile, split-K): used for W = Y_(n) Q0 and W T.
cudaError_t gemm_rows(Handle* h, const double* A, int64_t m, int64_t k, const double* B, int n, double* C);
// W_n = Y_(n) Q0 into h->W: FP32 from h->yn32 when the Multi-TTM left it, else FP64 from h->Yn.
cudaError_t apply_q0(Handle* h, int n);
// Solve Ahat R0^T = W (QR) or Ahat = W U pinv(S) V^T (SVD) into h->Ahat.
cudaError_t solve_qr(Handle* h, int64_t In);
// T = U pinv(Sigma) V^T of R0 (truncated one-sided Jacobi SVD) into h->T; it
// needs only R0, so a sweep runs it beside the Multi-TTM.
cudaError_t svd_operator(Handle* h, double rtol);
// Ahat = W T; the operator T is formed first unless have_operator.
cudaError_t solve_svd(Handle* h, int64_t In, double rtol, bool have_operator = false);
// S_n = Hadamard product of the other Grams (Alg. cp-als) into h->S, and into
// h->T its Cholesky factor (pinv = false) or its truncated pseudo-inverse
// (pinv = true, CP-ALS-PINV).  It needs only the Grams, so a sweep runs it
// beside the MTTKRP.
cudaError_t normal_operator(Handle* h, int n, bool pinv, double rtol);
// Ahat S_n = M by the Cholesky factor, or Ahat = M pinv(S_n); the operator is
// formed first unless have_operator.
cudaError_t solve_normal(Handle* h, int n, bool have_operator = false);
cudaError_t solve_normal_pinv(Handle* h, int n, double rtol, bool have_operator = false);
// Normalise columns of h->Ahat into A_n and lambda; then QR and Gram of A_n.
cudaError_t normalize_and_refactor(Handle* h, int n);
// Gram G = A^T A for an I x R factor.
cudaError_t gram(Handle* h, const double* A, int64_t I, double* G);
// Efficient fit after the last mode of a sweep; appends to the fit ring.
cudaError_t fit_efficient(Handle* h, int solve);

// ---------------------------------------------------------------- Kruskal-tensor input (kruskal.cu)
// out (na x nb) = A^T B for column-major A (I x na), B (I x nb).
cudaError_t kr_atb(Handle* h, const double* A, const double* B, int64_t I, int na, int nb, double* out);
// ||X||^2 of the Kruskal tensor into h->d_normX2.
cudaError_t kr_norm2(Handle* h);
// C_m = Q_m^T V_m and E_m = V_m^T A_m.
cudaError_t kr_refresh_c(Handle* h, int m);
cudaError_t kr_refresh_e(Handle* h, int m);
// W_n = Y_(n) Q0 into h->W from the fold factors in h->KP (krp_qr implicit).
cudaError_t kr_apply_q0(Handle* h, int n);
// MTTKRP of the normal equations into h->M.
cudaError_t kr_mttkrp(Handle* h, int n);
// The unfolding Y_(n) (I_n x R^{N-1}) into Y (device).
cudaError_t kr_unfold(Handle* h, int n, double* Y);
// Direct residual ||X - Xhat||^2 into *out (device), entry by entry.
cudaError_t kr_residual(Handle* h, double* out);

// ---------------------------------------------------------------- batched problems
struct Batch;
Batch* batch_new();
void batch_delete(Batch* b);
cudaError_t batch_build(Batch* b, int count, const int64_t* dims, const int* ranks);
size_t batch_smem_bytes(int maxR, int maxI);
cudaError_t batch_set_stream(Batch* b, cudaStream_t s);
cudaError_t batch_set_tensors(Batch* b, const float* const* X, bool host);
cudaError_t batch_set_factors(Batch* b, const double* const* A, bool host);
cudaError_t batch_get_factors(Batch* b, double* const* A, double* const* lambda, bool host);
cudaError_t batch_iterate(Batch* b, int iters, double* fits_host, int* status_host);
int64_t batch_launches(const Batch* b);
bool batch_ready(const Batch* b);
int batch_tuned_grid(const Batch* b);
int batch_tuned_threads(const Batch* b);
char* batch_err(Batch* b);

}  // namespace cpals

#define CPALS_CUDA_TRY(expr)                                  \
    do {                                                      \
        cudaError_t _e = (expr);                              \
        if (_e != cudaSuccess) return _e;                     \
    } while (0)
