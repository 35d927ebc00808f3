/*
 * cpals.h -- C-ABI of the GB300 (sm_103a) CP-ALS-QR hot path.
 *
 * Method: Minster, Viviano, Liu, Ballard, "CP Decomposition for Tensors via
 * Alternating Least Squares with QR Decomposition" (arXiv 2112.10855).
 * For mode n, Alg. cp-als-qr solves the least-squares problem of Eq. ls_n,
 *     min || X_(n) - Ahat_n Z_n^T ||_F,  Z_n = A_N (.) ... (.) A_{n+1} (.) A_{n-1} (.) ... (.) A_1,
 * through the structured QR Z_n = [(Q_N (x) ... (x) Q_1) Q0] R0 of Eq. Z_qr.
 * Alg. cp-als gives the normal-equations baseline (MTTKRP + Cholesky).
 *
 * Conventions
 *  - Modes are 0-based: `mode` = n - 1 in the paper's numbering.
 *  - X has dims I_0..I_{N-1} and is stored with mode 0 fastest: element
 *    (i_0..i_{N-1}) sits at sum_m i_m prod_{k<m} I_k.
 *  - Matrices are column-major (element (i,j) of an m x n matrix at i + m*j).
 *    Factor A_m and Q_m are I_m x R.  R_m, R0 and S are R x R.  Q0 is R^{N-1} x R.
 *  - The unfolding Y_(n) is I_n x R^{N-1}.  Its column index is
 *    sum_{m != n} r_m R^{pos(m)}, where pos counts the modes below m other
 *    than n (mode 0 fastest, as in Eq. multittm with the Kronecker rule of
 *    Sec. 2.2).  The rows of V_n and Q0 use the same order.
 *  - Every call returns a cpals_status.  cpals_last_error() gives a message.
 *  - Work is enqueued on the stream set with cpals_set_stream (default: the
 *    legacy default stream) and is asynchronous, except where a call says it
 *    synchronises.  Inside a mode update or a sweep the handle also runs work
 *    on a private high-priority stream (the QR of V_n, the solve operators of
 *    R0 or S_n): it forks from the caller's stream with an event and joins
 *    back before the call's last kernel, so every call stays ordered on the
 *    caller's stream.  Distinct handles may be driven from distinct host
 *    threads; one handle must not be used by two threads at once.
 *  - Pointer arguments carry a `mem` flag: CPALS_MEM_DEVICE means device
 *    memory that the caller owns; CPALS_MEM_HOST means host memory.  Host
 *    transfers are synchronous with respect to the host.
 *  - Errors found on the device (a singular R0, an S that is not positive
 *    definite, a device wait that ran out) are recorded in a device status
 *    word.  After one is recorded, every later kernel of the handle becomes
 *    a no-op, so the factors stay as they were when the failure happened.
 *    The word is reported, and then cleared, by the next synchronising call:
 *    cpals_sync, cpals_fit, cpals_iterate, or a get call with host memory.
 *  - A handle is not thread-safe.  Use one handle per host thread.
 *  - Errors of a call that lists none of its own: CPALS_ERR_ARG for a NULL
 *    handle, a mode outside [0, N), a bad mem flag or a NULL pointer that the
 *    call needs; CPALS_ERR_STATE when the call needs a tensor or factors that
 *    were not set; CPALS_ERR_NOMEM or CPALS_ERR_CUDA when an allocation or a
 *    CUDA call fails.  A call with mem = CPALS_MEM_HOST synchronises, so it
 *    also reports a device error recorded by earlier work (CPALS_ERR_SINGULAR,
 *    CPALS_ERR_TIMEOUT).
 *  - A process drives one GPU.  Kernel attributes (opt-in dynamic shared
 *    memory, non-portable cluster sizes) are set once per process, on the
 *    device current at the first call that needs them.  Handles created on a
 *    second device of the same process are not supported: launches that need
 *    those attributes fail there with CPALS_ERR_CUDA.  Run one process per GPU.
 */
#ifndef CPALS_H
#define CPALS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cpals_handle cpals_handle;

typedef enum {
    CPALS_OK = 0,
    CPALS_ERR_ARG = 1,       /* invalid argument (dims, rank, mode, null pointer, sizes) */
    CPALS_ERR_NOMEM = 2,     /* device or host allocation failed */
    CPALS_ERR_CUDA = 3,      /* a CUDA runtime call failed */
    CPALS_ERR_SINGULAR = 4,  /* R0 numerically singular (QR solve) or S not SPD (normal equations) */
    CPALS_ERR_TIMEOUT = 5,   /* a bounded device wait gave up */
    CPALS_ERR_STATE = 6      /* call order violated (e.g. no tensor, no factors) */
} cpals_status;

/* Arithmetic of the passes over X (Multi-TTM and MTTKRP).  The small
 * factors (QR of A_m and of V_n, the R0 solve or SVD, normalisation, fit)
 * always run in FP64. */
typedef enum {
    CPALS_F64 = 0,     /* X read as FP64, FP64 FMA */
    CPALS_F32 = 1,     /* X read as an FP32 copy (round to nearest even), FP32 FMA; Y promoted to FP64 */
    CPALS_BF16X3 = 2,  /* FP32 copy split into bf16 hi/lo parts; hi*hi+hi*lo+lo*hi on tcgen05 tensor cores
                          (kind::f16), FP32 accumulate; ~2^-16 relative per product.  Tensor cores for
                          the first TTM when rank >= 16, FP32 FMA otherwise */
    CPALS_TF32X3 = 3   /* the same with tf32 hi/lo parts (kind::tf32): ~2^-21 relative per product */
} cpals_precision;

typedef enum {
    CPALS_SOLVE_QR = 0,     /* CP-ALS-QR: substitution with R0 (Eq. ls-qr-q0-step) */
    CPALS_SOLVE_SVD = 1,    /* CP-ALS-QR-SVD: Ahat = W U pinv(Sigma) V^T with R0 = U Sigma V^T (Sec. 3.1) */
    CPALS_SOLVE_NORMAL = 2, /* CP-ALS: MTTKRP and Cholesky of the Hadamard product of Grams (Alg. cp-als) */
    CPALS_SOLVE_NORMAL_PINV = 3 /* CP-ALS-PINV: the same normal equations solved with the pseudo-inverse of S
                                   (Sec. 2.3), Ahat = M pinv(S) keeping sigma_i > svd_rtol * sigma_1 */
} cpals_solve;

typedef enum { CPALS_MEM_DEVICE = 0, CPALS_MEM_HOST = 1 } cpals_mem;
typedef enum { CPALS_ELEM_F64 = 0, CPALS_ELEM_F32 = 1 } cpals_elem;

/* Create a rank-`rank` CP-ALS problem for an N-way tensor of the given dims
 * (Sec. 3.1).  Requires 2 <= N <= 12, 1 <= rank <= 64, rank <= dims[m]
 * for every m, and rank^N <= 2^36 (Q0 and Y_(n) are held densely).  The compact QR A_m = Q_m R_m with Q_m of size I_m x R
 * (Sec. 3.1) needs I_m >= R, and that also keeps every Z_n from being wide.
 * Allocates every device workspace buffer now (cudaMalloc), on the current
 * device.  On success, *out receives the handle.
 * Errors: CPALS_ERR_ARG, CPALS_ERR_NOMEM, CPALS_ERR_CUDA. */
int cpals_create(const int64_t* dims, int N, int rank, int precision, cpals_handle** out);

/* Free the handle and every buffer it owns.  Synchronises its stream.  NULL is a no-op. */
int cpals_destroy(cpals_handle* h);

/* Static message for the last failing call on h (or on creation when h is NULL). */
const char* cpals_last_error(const cpals_handle* h);

/* Enqueue all later work on `stream` (a cudaStream_t; NULL = legacy default stream). */
int cpals_set_stream(cpals_handle* h, void* stream);

/* Bytes of device memory the handle owns (workspace plus any owned copy of X). */
int cpals_workspace_bytes(const cpals_handle* h, size_t* bytes);

/* Attach the data tensor X (prod(dims) elements, mode 0 fastest).
 *  elem = CPALS_ELEM_F64: with precision F64 and mem DEVICE, the pointer is
 *    borrowed and must stay valid until the handle is destroyed or another
 *    tensor is set; with mem HOST, X is copied into a device buffer that the
 *    handle owns.  With precision F32/BF16X3/TF32X3, X is rounded (round to
 *    nearest even) into an FP32 copy that the handle owns.  The passes over X
 *    read only that copy.  ||X||^2 and the direct fit use the FP64 values, so
 *    a device FP64 pointer stays borrowed in that case too.
 *  elem = CPALS_ELEM_F32: allowed only with precision F32/BF16X3/TF32X3;
 *    borrowed (DEVICE) or copied (HOST).
 * Also computes ||X||_F^2 in FP64 (Sec. 3.3.1: it is pre-computed once).
 * Synchronises.  A tensor with a NaN or an Inf (||X||^2 not finite) is
 * refused with CPALS_ERR_ARG, and the handle then holds no tensor
 * (CPALS_ERR_STATE for the calls that need one) until a valid one is set. */
int cpals_set_tensor(cpals_handle* h, const void* X, int elem, int mem);

/* Kruskal-tensor input (Sec. 3.3.2).  The data tensor is given in Kruskal
 * form X = sum_{s<S} mu_s v_s^(1) o ... o v_s^(N) and is never formed: the
 * Multi-TTM Y = X x_{m != n} Q_m^T is again a Kruskal tensor with factors
 * Q_m^T V_m (m != n) and V_n, so W_n = Y_(n) Q0 is an MTTKRP of Q0 followed
 * by a small product (Sec. 3.3.2).  Q0 itself stays in the factored form of
 * its structured QR (Eq. kr-id), which makes a mode update O(N S R^3 +
 * sum_m I_m R S) and allows orders and ranks whose R^{N-1} x R matrix Q0
 * could not be stored.  The MTTKRP of the normal equations is
 * V_n diag(mu) (*_{m != n} V_m^T A_m); ||X||^2 = mu^T (*_m V_m^T V_m) mu.
 *
 * cpals_create_kruskal: dims, N, rank as for cpals_create (2 <= N <= 12,
 *   1 <= rank <= 64, rank <= dims[m]; no bound on rank^N); S = the Kruskal
 *   rank of X, 1 <= S <= 4096.  FP64 throughout.  Allocates every buffer now.
 *   Errors: CPALS_ERR_ARG, CPALS_ERR_NOMEM, CPALS_ERR_CUDA.
 * The handle accepts every call below except cpals_set_tensor and
 * cpals_ttm_first (CPALS_ERR_STATE: there is no dense tensor), with these
 * differences: cpals_krp_qr returns R0 only (Q0 != NULL -> CPALS_ERR_ARG);
 * cpals_multi_ttm returns Y_(n) only while I_max * R^{N-1} <= 2^24
 * (CPALS_ERR_ARG otherwise); cpals_fit(direct = 1) evaluates both tensors
 * entry by entry (prod(dims) entries, (S + R) N products each);
 * CPALS_OPT_DIMTREE has no effect. */
int cpals_create_kruskal(const int64_t* dims, int N, int rank, int S, cpals_handle** out);

/* Set the Kruskal tensor of a handle from cpals_create_kruskal: N pointers
 * V[m] (I_m x S, column-major, FP64) and the S weights mu (NULL for ones).
 * The data is copied; ||X||^2 is computed.  Synchronises.
 * Errors: CPALS_ERR_ARG (NULL pointers, bad mem flag), CPALS_ERR_STATE (a
 * dense-tensor handle), CPALS_ERR_CUDA. */
int cpals_set_tensor_kruskal(cpals_handle* h, const double* mu, const double* const* V, int mem);

/* Set the factors A_m (N pointers, I_m x R, FP64) and weights lambda (R values,
 * or NULL for ones).  Alg. cp-als-qr initialisation: the compact QR
 * A_m = Q_m R_m (diag(R_m) >= 0) is computed for every m, and so is the Gram
 * A_m^T A_m (Alg. cp-als initialisation).  The data is copied. */
int cpals_set_factors(cpals_handle* h, const double* const* A, const double* lambda, int mem);

/* Copy out the current factors A_m (entries of A may be NULL to skip a mode)
 * and lambda (may be NULL). */
int cpals_get_factors(cpals_handle* h, double* const* A, double* lambda, int mem);

/* Copy out Q_m (I_m x R) and R_m (R x R) of the current factor of `mode`
 * (Alg. cp-als-qr factor-QR step).  Either output may be NULL. */
int cpals_get_factor_qr(cpals_handle* h, int mode, double* Q, double* R, int mem);

/* Override Q_m and R_m of every mode (N pointers each, FP64, mem as given),
 * without touching A_m.  This feeds externally computed orthonormal factors
 * to the Multi-TTM and KRP steps, for checking them one at a time. */
int cpals_set_factor_qr(cpals_handle* h, const double* const* Q, const double* const* R, int mem);

/* Alg. cp-als-qr, KRP and Q0 steps: V_n = R_{N-1} (.) ... (.) R_0 without
 * `mode`, then its compact QR V_n = Q0 R0 with diag(R0) >= 0 (Eq. Z_qr).
 * Q0 (R^{N-1} x R) and R0 (R x R) may be NULL.  The result is kept in the
 * handle for the W step of cpals_multi_ttm on the same mode. */
int cpals_krp_qr(cpals_handle* h, int mode, double* Q0, double* R0, int mem);

/* Alg. cp-als-qr, Multi-TTM step (Eq. multittm): Y = X x_m Q_m^T for every m != mode,
 * as single TTMs in decreasing-dimension order (Sec. 3.2).
 *  Y (may be NULL): I_n x R^{N-1} unfolding Y_(n), FP64.
 *  W (may be NULL): W_n = Y_(n) Q0 (Eq. ls-qr-q0-step), I_n x R, FP64.  It
 *    needs a cpals_krp_qr on the same mode first (CPALS_ERR_STATE otherwise). */
int cpals_multi_ttm(cpals_handle* h, int mode, double* Y, double* W, int mem);

/* Measurement entry point: the first single TTM of the Multi-TTM of `mode`
 * alone.  It is the pass that streams X from HBM (2 P R flops, Eq. TTMcost
 * leading term).  Its output goes to the handle's workspace.  The benchmark
 * times this kernel with events for the roofline figure. */
int cpals_ttm_first(cpals_handle* h, int mode);

/* Alg. cp-als, MTTKRP step: M_n = X_(n) Z_n (I_n x R, FP64) with the current
 * factors; the arithmetic follows the handle's precision. */
int cpals_mttkrp(cpals_handle* h, int mode, double* M, int mem);

/* One mode update.
 *  QR/SVD: the mode-loop body of Alg. cp-als-qr (KRP, QR of V_n, Multi-TTM,
 *    apply Q0, solve by substitution or by the truncated SVD of R0 keeping
 *    sigma_i > svd_rtol * sigma_1, normalise columns with the 2-norm into A_n
 *    and lambda, re-QR A_n = Q_n R_n).
 *  NORMAL / NORMAL_PINV: the mode-loop body of Alg. cp-als (Hadamard product
 *    of Grams S_n, MTTKRP, Cholesky or pseudo-inverse solve, normalise,
 *    re-Gram).  The QR of a factor is refreshed only when a later QR/SVD solve
 *    needs it.
 * svd_rtol <= 0 selects R * eps.  Asynchronous; a singular solve is recorded
 * in the device status word and leaves the factor unchanged. */
int cpals_solve_mode(cpals_handle* h, int mode, int solve, double svd_rtol);

/* Run sweeps over all modes (the outer loop of Alg. cp-als-qr / cp-als).
 * Each sweep ends with the efficient fit of Sec. 3.3.1.
 *  tol > 0: stop once |fit - previous fit| < tol.  This reads the fit on the
 *    host after every sweep.
 *  tol == 0: run exactly `iters` sweeps, with no host synchronisation until
 *    the end.
 * The sweep is captured once per solve kind into a CUDA graph and replayed.
 * fits_host (may be NULL) receives one fit per sweep that ran.
 * *done (may be NULL) receives the number of sweeps run.  Synchronises at the end. */
int cpals_iterate(cpals_handle* h, int iters, double tol, int solve, double svd_rtol, int* done,
                  double* fits_host);

/* The per-iteration component breakdown of Table its_parts (Sec. 4.1):
 * runs `sweeps` sweeps (1..16) like cpals_iterate with tol = 0, but eagerly
 * and with every phase on the handle's stream one after the other (no side
 * stream, no graph), records CUDA events around each phase, and writes the
 * mean milliseconds per sweep of five buckets to bucket_ms[0..4]:
 *   0: the passes over X -- Multi-TTM (QR, SVD) or MTTKRP (normal equations);
 *   1: the QR of the factor matrices (QR, SVD) or their Grams (normal
 *      equations); with CPALS_OPT_FUSED_TAIL the fused tail also holds the
 *      solve and the normalisation;
 *   2: computing Q0 (the QR of V_n);
 *   3: applying Q0 (W = Y_(n) Q0);
 *   4: other (solve operators of R0 or S_n, the solve when not fused, the fit).
 * The factors advance as in cpals_iterate.  The sum of the buckets exceeds a
 * graph sweep's time by the overlap and the launch gaps the graph removes.
 * Synchronises.  Errors: CPALS_ERR_ARG, CPALS_ERR_STATE, CPALS_ERR_CUDA, and
 * the device errors of a sweep. */
int cpals_profile_sweeps(cpals_handle* h, int sweeps, int solve, double svd_rtol, double* bucket_ms);

/* fit = 1 - ||X - Xhat|| / ||X||.  direct = 0: the efficient form of
 * Sec. 3.3.1 from the last sweep's W_N, Ahat_N, R0 and R_N (or, after a
 * NORMAL sweep, from M_N and S_N).  It is accurate to about sqrt(eps) and
 * needs a finished sweep (CPALS_ERR_STATE otherwise).  direct = 1: one pass
 * over X that forms Xhat entry by entry.  Synchronises. */
int cpals_fit(cpals_handle* h, int direct, double* fit_host);

/* Synchronise the handle's stream and report (then clear) the device status word. */
int cpals_sync(cpals_handle* h);

/* Options of a handle.
 *  CPALS_OPT_DIMTREE (default 1): sweeps of cpals_iterate on an N >= 3
 *    dense tensor share Multi-TTM work (and, for the NORMAL / NORMAL_PINV
 *    solves, MTTKRP work) across modes by a dimension tree (Sec. 3.3.3).  X is contracted once over the modes of the
 *    second half for the Multi-TTMs of the first half, and once over the first
 *    half (with its updated Q_m) for the second half.  That is two passes over
 *    X per sweep instead of N.  0 runs a full Multi-TTM from X per mode.  The
 *    results differ only by rounding (Sec. 2.2: TTMs commute).
 *  CPALS_OPT_TC_PIPELINE (default 1): with CPALS_BF16X3 / CPALS_TF32X3, the
 *    first TTM of a Multi-TTM (the pass over X, Eq. multittm) runs in one
 *    persistent tensor-core kernel per launch that streams X through the
 *    Tensor Memory Accelerator, whenever the product of the dims before the
 *    contracted mode is a multiple of 4.  0 always uses one CTA per 128-row
 *    tile.  Both compute the same split products; the sums differ only in the
 *    order of two FP32 additions per output.
 *  CPALS_OPT_KRP_TREE (default 1): in a dimension-tree sweep with the QR or
 *    SVD solve, the QR of V_n follows the same halves.  The QR of the
 *    Khatri-Rao product of each half's R_m is taken once per sweep, on a side
 *    stream while X is contracted, and each mode folds only the R_m of its own
 *    half onto the other half's R and applies that half's Q as a Kronecker
 *    factor (Eq. kr-id).  0 folds all N-1 factors for every mode.  The Q0, R0
 *    differ only by rounding.
 *  CPALS_OPT_F32_PIPELINE (default 1): FP32 TTMs (the CPALS_F32 passes over
 *    X and the FP32 contractions of intermediates in every precision but
 *    F64) run on the CUDA cores fed by a ring of TMA boxes, whenever the
 *    product of the dims before the contracted mode is a multiple of 4 and
 *    9 <= R <= 64.  0 uses the row-per-thread kernels.  Both sum each output in
 *    order of the contracted index (the row kernels within each K split,
 *    whose sums they add in a fixed order), so only rounding differs.
 *  CPALS_OPT_TEST_WITHHOLD_COPIES (default 0): a test hook for the failure
 *    path of the bounded device waits (the paper has no counterpart).  With 1,
 *    the persistent tensor-core pass over X (BF16X3 / TF32X3, rank >= 16)
 *    issues no copies of X and its waits give up after 1 ms instead of 1 s,
 *    with nothing left in flight.  The pass records CPALS_ERR_TIMEOUT in the
 *    device status word; the rest of the update is skipped and the factors
 *    stay as they were, and the next synchronising call reports the error.
 *    Set it back to 0 and the handle works as before.
 *  CPALS_OPT_FUSED_TAIL (0, 1 or 2; default 2): the end of each mode update -- the
 *    solve (substitution with R0, the SVD or pseudo-inverse operator, or the
 *    Cholesky factor of S_n), the column normalisation into lambda and A_n,
 *    and the QR A_n = Q_n R_n (QR/SVD solves) or the Gram A_n^T A_n (normal
 *    equations) -- runs in one thread-block cluster whose CTAs split the
 *    rows of A_n.  The factor QR there is CholeskyQR2 (two passes of Gram,
 *    Cholesky and substitution); it is accepted only when the first pass
 *    leaves Q1^T Q1 within 1e-2 of the identity (cond(A_n) below about 7e6),
 *    and otherwise the Householder QR runs as with 0.  Both give the thin QR
 *    with a positive diagonal of R_n, so only rounding differs.  0 runs the
 *    separate solve, normalisation and Householder QR kernels.  2 (the
 *    default) takes 1 from rank 8 up and 0 below it, where the separate
 *    kernels measured faster; the choice depends on the rank only, so every
 *    factor QR of a handle takes the same path.  Values other than 0, 1 and
 *    2 are CPALS_ERR_ARG.
 *  CPALS_OPT_SVD_SHORTCUT (default 1): before the Jacobi SVD of R0 (the SVD
 *    solve), X = R0^-1 is formed by substitution; when
 *    ||R0||_F ||X||_F svd_rtol <= 1/4, no singular value can fall below
 *    svd_rtol * sigma_max (sigma_min >= 1/||X||_F, sigma_max <= ||R0||_F), so
 *    the truncated solve is W R0^-T exactly and the operator R0^-T is used
 *    without the SVD.  Otherwise the Jacobi SVD runs as with 0.  The two
 *    differ only by rounding.
 *  CPALS_OPT_APPLY_Q0_FP32 (default 1): with CPALS_F32 / BF16X3 / TF32X3,
 *    the mode updates keep the Multi-TTM's unfolding Y_(n) in FP32 and form
 *    W_n = Y_(n) Q0 (Eq. ls-qr-q0-step) in FP32, one more contraction of the
 *    FP32 chain, before the FP64 solve.  0 widens Y_(n) to FP64 and forms W
 *    in FP64.  The explicit cpals_multi_ttm keeps FP64 either way.
 *  CPALS_OPT_WIDE_TAIL (default 1; ranks above 32 with CPALS_OPT_FUSED_TAIL):
 *    the CholeskyQR2 of the factor QRs (after the GPU-wide solve) and of the
 *    Khatri-Rao fold steps of the QR of V_n runs as a chain of kernels over
 *    every SM: Gram partials of row blocks summed in a fixed order, the
 *    Cholesky factors and their triangular inverses in one CTA, and the row
 *    products Q1 = A R1^-1, Q = Q1 R2^-1 over all rows.  The first Gram of a
 *    fold step F (.) R_B is (F^T F) * (R_B^T R_B).  The acceptance check and
 *    the Householder fallback are those of the cluster kernel.  0 keeps the
 *    one-cluster kernel (16 SMs).  Results differ only by rounding. */
typedef enum {
    CPALS_OPT_DIMTREE = 0,
    CPALS_OPT_TC_PIPELINE = 1,
    CPALS_OPT_KRP_TREE = 2,
    CPALS_OPT_F32_PIPELINE = 3,
    CPALS_OPT_TEST_WITHHOLD_COPIES = 4,
    CPALS_OPT_FUSED_TAIL = 5,
    CPALS_OPT_SVD_SHORTCUT = 6,
    CPALS_OPT_APPLY_Q0_FP32 = 7,
    CPALS_OPT_WIDE_TAIL = 8
} cpals_option;
int cpals_set_option(cpals_handle* h, int option, int64_t value);

/* Test hook (the paper has no counterpart): the reciprocal and reciprocal
 * square root that the factor QR of the fused mode tail uses on its
 * sequential chain (hardware approximations refined in FP64: one
 * third-order Newton step for the reciprocal, two Newton-Raphson steps for
 * the reciprocal square root), applied to n device values x (rsqrt gets 0 where
 * x <= 0).  x, rcp, rsqrt: device arrays of n doubles.  Synchronises the
 * device.  Errors: CPALS_ERR_ARG, CPALS_ERR_CUDA. */
int cpals_test_newton_recip(const double* x, int64_t n, double* rcp, double* rsqrt);

/* Test hook for the allocation-failure path (the paper has no counterpart):
 * the nth device allocation that a handle makes from now on (counted over
 * the process, 1 = the next one) fails as if the device were out of memory,
 * without calling cudaMalloc.  cpals_create then frees what it holds and
 * returns CPALS_ERR_NOMEM; cpals_set_tensor, whose first call with host
 * memory or a mixed precision allocates the owned copy of X, returns the same.
 * 0 disables the hook.  Errors: CPALS_ERR_ARG for nth < 0. */
int cpals_test_fail_allocation(int nth);

/* Number of kernel launches the handle has issued so far (graph replays count
 * each kernel node once per replay). */
int64_t cpals_launch_count(const cpals_handle* h);

/* Multi-TTM Y_(n) = X_(n) (Q_{N-1} (x) ... (x) Q_0, without `mode`) of
 * Eq. multittm (Alg. cp-als-qr, Multi-TTM step) for callers that cannot
 * allocate device memory.  The paper has no counterpart
 * to this entry point.  Such callers include a host framework that hands all
 * device memory to its own pool allocator, a process that runs under a hard
 * device-memory budget, and a latency-critical loop where the implicit
 * device synchronisation of cudaMalloc/cudaFree is not acceptable.
 *
 * It computes what cpals_multi_ttm computes (FP64, the same kernels, the
 * single TTMs in decreasing-dimension order) without a handle.  It calls
 * no cudaMalloc, cudaFree or allocating library routine.  Its scratch (the
 * TTM intermediates and split-K partial sums) is one fixed file-scope device
 * array of 2^21 doubles (16 MiB).  Every GPU that loads the library holds
 * that array until the process exits.
 *
 *  dims, N, rank: as for cpals_create (2 <= N <= 12, 1 <= rank <= 64,
 *    rank <= every dim).
 *  mode: the kept mode n (0-based).
 *  X: device pointer to prod(dims) FP64 values (mode 0 fastest), read only.
 *  Q: host array of N device pointers to the I_m x R column-major FP64
 *    matrices Q_m; Q[mode] is not read and may be NULL.
 *  Y: device pointer to I_n x R^{N-1} FP64 values (the unfolding Y_(n)),
 *    written.
 *  stream: cudaStream_t to enqueue on (NULL = legacy default stream).
 *    Asynchronous.
 * The caller owns X, Q and Y.  Sizes whose two largest TTM intermediates need
 * more than 2^21 doubles are rejected with CPALS_ERR_ARG and a message from
 * cpals_last_error(NULL), before any work is enqueued.
 * On the first call on each device, with that device current, the call looks
 * up the array's device address (cudaGetSymbolAddress).  That first call
 * should therefore come before any stream capture.
 * Every call shares the one array, and the array keeps the last call's
 * contents.  Each call writes every scratch element before reading it and
 * clears the status word it needs, so stale contents do no harm.  Calls
 * that overlap on the GPU (other streams, other host threads, the same
 * device) race on the array and give wrong results. */
int cpals_multi_ttm_static(const int64_t* dims, int N, int rank, int mode, const double* X,
                           const double* const* Q, double* Y, void* stream);

/* ---------------------------------------------------------------------
 * Batched problems: many independent 3-way CP-ALS-QR problems of uneven dims
 * and ranks advance together.  A sweep follows the dimension tree of
 * Sec. 3.3.3 for every problem at once: one pass over all tensors contracts
 * mode 2 (X x_2 Q_2^T), the updates of modes 0 and 1 finish their
 * Multi-TTMs from that partial, a second pass contracts mode 1 with the new
 * Q_1, and the update of mode 2 finishes from it -- two reads of X per sweep.
 * Every contraction (the passes, the last TTM of each Multi-TTM and
 * W = Y_(n) Q0) is one launch over all problems whose CTAs take
 * (problem, row tile) work items from a device queue, in FP32.  The rest of
 * each mode update of Alg. cp-als-qr -- the R0 substitution, normalisation,
 * the factor QR and the QR of the next mode's V = R_hi (.) R_lo -- is one
 * FP64 kernel with a CTA per problem; the efficient fit of Sec. 3.3.1
 * follows the last mode.
 * --------------------------------------------------------------------- */
typedef struct cpals_batch cpals_batch;

/* count problems; dims is count x 3 (row p = I_0, I_1, I_2 of problem p),
 * ranks has count entries.  Requires 1 <= rank <= 16 and rank <= every dim
 * <= 4096, and the largest problem's working set (Q0, R0, W and the factor QR in
 * FP64) within one CTA's shared memory.  Allocates all device buffers. */
int cpals_batch_create(int count, const int64_t* dims, const int* ranks, cpals_batch** out);
int cpals_batch_destroy(cpals_batch* b);
int cpals_batch_set_stream(cpals_batch* b, void* stream);

/* X: count pointers to FP32 tensors (prod(dims_p) values, mode 0 fastest),
 * copied into the batch; ||X_p||^2 is computed in FP64. */
int cpals_batch_set_tensors(cpals_batch* b, const float* const* X, int mem);

/* A: 3*count pointers (A[3p+m] = factor m of problem p, I_m x R_p column-major
 * FP64), copied; lambda = 1; the QR of every factor is taken (Alg. cp-als-qr
 * initialisation); per-problem status words are cleared. */
int cpals_batch_set_factors(cpals_batch* b, const double* const* A, int mem);

/* Copy out factors (A as for set; entries may be NULL) and lambda (count
 * pointers of R_p values; entries may be NULL). */
int cpals_batch_get_factors(cpals_batch* b, double* const* A, double* const* lambda, int mem);

/* `iters` sweeps over the three modes for every problem.  The sweep is a
 * captured CUDA graph of twelve kernel launches (the QR of V_0, five grouped
 * TTMs, three grouped W products, three factorisation kernels).  The first
 * call picks the grouped launches' row tile and the factorisation kernels'
 * CTA size and count by timing one sweep per candidate on a saved copy of
 * the factors.
 * fits_host (count values, may be NULL) receives each problem's efficient fit
 * after the last sweep; status_host (count values, may be NULL) receives each
 * problem's status: CPALS_ERR_SINGULAR for a problem whose R0 became
 * numerically singular (its factors stay as they were, and it is skipped
 * after that).  Synchronises. */
int cpals_batch_iterate(cpals_batch* b, int iters, double* fits_host, int* status_host);

/* Kernel launches issued so far (a graph replay counts its twelve kernels). */
int64_t cpals_batch_launch_count(const cpals_batch* b);

/* The factorisation kernels' launch shape the first iterate picked (0 before it). */
int cpals_batch_launch_shape(const cpals_batch* b, int* grid, int* threads);

/* Measured FMA throughput probe (not part of the method): runs dependent
 * FMA chains on every SM for `ms_target` ms and writes the achieved
 * TFLOP/s for FP64 and FP32.  Used to state the ALU roofline.  Synchronises. */
int cpals_probe_fma_peak(double ms_target, double* fp64_tflops, double* fp32_tflops);

#ifdef __cplusplus
}
#endif
#endif /* CPALS_H */
