/*
 * bks.h — C-ABI of a GB300 (sm_103a) library for randomized Block Krylov Iteration
 * and Simultaneous Iteration (Musco & Musco, arXiv 1504.05477).
 *
 * Conventions shared by every entry point
 *  - All matrix pointers are DEVICE pointers on the context's device unless a name
 *    ends in `_host`.  The caller owns them; the library never frees or keeps them
 *    past the call.
 *  - Dense matrices are row-major with a leading dimension in elements (>= columns).
 *    "n x k row-major" below means element (i, j) sits at ptr[i * ld + j].
 *  - Every call is asynchronous on the context's stream except where it says it
 *    synchronises.  Solves synchronise once, at the end, to read the device status
 *    word; nothing else blocks the host.
 *  - Errors are returned as bks_status codes; nothing is thrown across the ABI and
 *    no kernel traps.  Argument errors are detected on the host before any launch.
 *    Device-detected problems (non-finite values, Cholesky breakdown that the
 *    shifted retry could not repair, a Jacobi sweep cap) are reported through the
 *    status word.  bks_last_error() gives a one-line explanation.
 *  - A context is not thread-safe; use one per host thread.
 */
#ifndef BKS_H
#define BKS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BKS_OK = 0,
    BKS_ERR_INVALID_ARG = 1,    /* bad size, null pointer, bad dtype: nothing launched */
    BKS_ERR_CUDA = 2,           /* a CUDA runtime call failed (message in bks_last_error) */
    BKS_ERR_NOMEM = 3,          /* workspace allocation failed */
    BKS_ERR_NONFINITE = 4,      /* a NaN/Inf reached a Gram matrix or M */
    BKS_ERR_BREAKDOWN = 5,      /* Cholesky of a Gram matrix failed even after shifting */
    BKS_ERR_NOT_CONVERGED = 6,  /* Jacobi eigen-solver hit its sweep cap */
    BKS_ERR_TIMEOUT = 7,        /* a bounded device-side wait gave up */
    BKS_ERR_UNSUPPORTED = 8,    /* valid request the library does not implement */
    BKS_WARN_DEFLATED = 100     /* results valid; q was capped or Krylov columns were dependent */
} bks_status;

typedef enum { BKS_F64 = 0, BKS_F32 = 1, BKS_BF16 = 2 } bks_dtype;
typedef enum { BKS_DENSE = 0, BKS_CSR = 1 } bks_kind;

/* Precision of a solve.  AUTO: FP64 for FP64 input, else FP32.  F32: products with
 * FP32-accurate arithmetic, Krylov blocks in FP32, Gram matrices accumulated in FP64.
 * BF16: products in BF16 with FP32 accumulation (A must be BF16); with `refine` a
 * final FP32-accurate B = A^T Q recomputes M before the eigen-solve. */
typedef enum { BKS_PREC_AUTO = 0, BKS_PREC_F64 = 1, BKS_PREC_F32 = 2, BKS_PREC_BF16 = 3 } bks_precision;

/* The matrix A (n x d).  Paper, Sec. 1: A in R^{n x d}; the methods touch it only
 * through products with A and A^T (Sec. 4).  Dense: row-major, `vals` holds n*ld
 * elements of `dtype`.  CSR: `row_ptr` (n+1, int64, non-decreasing from 0 to nnz),
 * `col_idx` (nnz, int32, in [0, d) and strictly increasing within a row), `vals` (nnz,
 * FP32); the structure is checked on the device before anything is indexed through it
 * and a malformed CSR returns BKS_ERR_INVALID_ARG.  The optional CSR of A^T (`t_*`, d+1 / nnz /
 * nnz) lets the A^T products run row-parallel; when absent bks_csr_transpose builds
 * it.  `col_mean` (d floats, device) makes every product use A - 1 mu^T instead of A
 * (footnote 1 of Sec. 1: principal components after mean centring), applied
 * implicitly. */
typedef struct {
    int32_t kind;
    int32_t dtype;
    int64_t n, d;
    int64_t ld;
    const void* vals;
    const int64_t* row_ptr;
    const int32_t* col_idx;
    int64_t nnz;
    const int64_t* t_row_ptr;
    const int32_t* t_col_idx;
    const void* t_vals;
    const float* col_mean;
} bks_matrix;

typedef struct {
    int32_t precision;          /* bks_precision */
    int32_t refine;             /* BF16 only: final FP32 Rayleigh-Ritz pass (default 1) */
    int32_t basis_only;         /* 1: skip steps 4-5 and return Z = first k columns of Q
                                   (Sec. 4.1: enough for low-rank approximation) */
    int32_t sign_fix;           /* 1 (default): flip each z_i so its largest |entry| is > 0 */
    int32_t jacobi_max_sweeps;  /* default 40 */
    double jacobi_tol;          /* rotation threshold |x_p.x_q| <= tol |x_p||x_q|; 0 = default */
    int32_t profile;            /* 1: record per-kernel-class CUDA-event times into bks_stats */
    int32_t product_path;       /* products with a dense A: 0 auto (tensor cores when the
                                   operands meet the TMA alignment rules, else CUDA cores),
                                   1 CUDA cores (SIMT) only */
    int32_t rr_mode;            /* input of the eigen-solve of M (step 5): 0 auto (M = B^T B
                                   for the tridiagonal solver and for the Jacobi at w <= 512,
                                   else 1), 1 the triangular factor R of a block QR of B in
                                   d-space (M = R^T R, one-sided Jacobi on R^T), 2 M = B^T B */
    int32_t eig_mode;           /* eigen-solve of M (step 6): 0 auto (when only the k leading
                                   vectors are returned and w > k: Householder tridiagonal form
                                   of M = B^T B, multisection and inverse iteration, if w fits
                                   its kernels; otherwise the one-sided Jacobi), 1 always the
                                   one-sided Jacobi */
    int32_t block_p;            /* columns p of Pi and width of every Krylov block (Sec. 8,
                                   "Improved Convergence With Spectral Decay": any p >= k, with
                                   q iterations depending on sigma_k / sigma_{p+1}); 0 = k.  The
                                   call still returns the k leading Ritz vectors; w = p (q + 1)
                                   (BKI) or p (SI), q capped so that w <= min(n, d); a caller-
                                   supplied Pi is d x p.  Must be 0 or in [k, min(n, d)], at
                                   most 128; Ritz triplets take p = k */
    int32_t eig_f64;            /* FP32 and BF16 precisions: 1 solves the eigen-problem of M in FP64
                                   (M formed as usual, then the one-sided Jacobi in FP64 and the
                                   eigenvectors rounded to FP32); 0 (default) in FP32.  Widths up to
                                   512 (BKS_ERR_UNSUPPORTED beyond).  Ignored on the FP64 path */
    int32_t max_sms;            /* SMs the call's kernels spread over (grid sizes of the products,
                                   orthonormalisations and reductions); 0 = all.  Results depend on
                                   it in the last bits (summation orders follow the grid).  Batched
                                   calls: 0 lets the call choose per shape class (see
                                   bks_block_krylov_batched); a value > 0 applies to every matrix */
    int32_t reserved[1];
} bks_opts;

typedef struct {
    int32_t q_eff;              /* iterations actually run (q capped so k(q+1) <= min(n,d)) */
    int32_t width;              /* columns of Q: k(q_eff+1) for BKI, k for SI */
    int32_t jacobi_sweeps;
    int32_t chol_shifts;        /* Cholesky factorisations that needed a diagonal shift */
    int32_t launches;           /* kernels launched by the call */
    int32_t product_launches;   /* of which products with A or A^T */
    float ms_product;           /* with opts.profile: summed event time of A / A^T products */
    float ms_orth;              /* ... of block orthonormalisation */
    float ms_rr;                /* ... of M, eigen-solve and Ritz vectors */
    float ms_total;             /* ... of the whole call */
    double product_bytes;       /* algorithmic bytes moved by the A / A^T products */
    double product_flops;       /* algorithmic flops of the A / A^T products */
    float ms_product_kernel;    /* with opts.profile: summed event time of the launches of the
                                   dominant product kernel alone (dense FP32: the tensor-core
                                   kernel; BF16: its BF16-rounded products; CSR: the SpMM) */
    int32_t product_kernel_launches;
    int32_t eig_path;           /* eigen-solve that ran: 0 one-sided Jacobi, 1 tridiagonal, 2 the
                                   one-sided Jacobi in FP64 (opts.eig_f64) */
    int32_t reserved[5];
} bks_stats;

typedef struct bks_ctx bks_ctx;

/* ---- context -------------------------------------------------------------------- */

/* Create a context on `device`.  Allocates nothing on the device yet. */
bks_status bks_create(bks_ctx** ctx, int device);
/* Free the context's workspace (if the library allocated it) and the context. */
bks_status bks_destroy(bks_ctx* ctx);
/* Stream (a cudaStream_t, NULL = legacy default) on which every later call runs. */
bks_status bks_set_stream(bks_ctx* ctx, void* stream);
/* Hand the context a caller-owned device workspace of `bytes` (256-byte aligned).
 * Later calls use it and allocate nothing while it is large enough; NULL reverts to
 * library-owned workspace.  Size it with bks_workspace_size. */
bks_status bks_set_workspace(bks_ctx* ctx, void* ptr, size_t bytes);
/* Workspace bytes a solve of A at rank k, q iterations needs. method: 0 BKI (and Block
 * Lanczos), 1 SI. */
bks_status bks_workspace_size(const bks_matrix* A, int k, int q, int method,
                              const bks_opts* opts, size_t* bytes);
/* Fill *opts with the defaults described in bks_opts. */
void bks_opts_default(bks_opts* opts);
const char* bks_status_string(bks_status s);
const char* bks_last_error(const bks_ctx* ctx);
/* Library version (major * 100 + minor). */
int bks_version(void);

/* ---- solves (Algorithms 1 and 2) ------------------------------------------------- */

/* Block Krylov Iteration, Algorithm 2 (Sec. 2.1), with per-block reorthonormalisation
 * (Sec. 4.2) and Rayleigh-Ritz post-processing (Lemma 4.1).
 *   K = [A Pi, (AA^T) A Pi, ..., (AA^T)^q A Pi]  (q+1 blocks of k columns),
 *   Q = orthonormal basis of span(K), M = Q^T A A^T Q, Z = Q Ubar_k, Sigma_k = sqrt(lambda_1..k(M)).
 * k      target rank, 1 <= k <= min(n, d).
 * q      iterations, >= 0; capped to q_eff = min(q, floor(min(n,d)/k) - 1) with
 *        BKS_WARN_DEFLATED returned when the cap applies.
 * seed   start block Pi ~ N(0,1)^{d x k} from the SplitMix64 -> Box-Muller generator
 *        (see bks_gen_pi), used when `pi` is NULL.
 * pi     optional caller start block, d x k row-major (ld = k), dtype FP64 on the FP64
 *        path else FP32.
 * Z      out, n x k row-major (ld = k): FP64 on the FP64 path, else FP32.
 * sigma  out, k Ritz values, descending, same dtype as Z.
 * V      optional out, d x k row-major: right Ritz vectors A^T z_i / sigma_i.
 * opts   NULL = defaults.  stats: optional out. */
bks_status bks_block_krylov(bks_ctx* ctx, const bks_matrix* A, int k, int q, uint64_t seed,
                            const void* pi, void* Z, void* sigma, void* V,
                            const bks_opts* opts, bks_stats* stats);

/* Simultaneous Iteration, Algorithm 1 (Sec. 2.1), orthonormalised after every
 * iteration (Sec. 4.1): Q <- orth(A (A^T Q)) from Q = orth(A Pi), then the same
 * Rayleigh-Ritz step with a k x k matrix M.  Arguments as bks_block_krylov. */
bks_status bks_simul_iter(bks_ctx* ctx, const bks_matrix* A, int k, int q, uint64_t seed,
                          const void* pi, void* Z, void* sigma, void* V,
                          const bks_opts* opts, bks_stats* stats);

/* Block Krylov Iteration with the iteration count chosen on the fly (extends the q of
 * Algorithm 2; Sec. 8 bounds q through sigma_k / sigma_{p+1}, which a caller rarely
 * knows).  After B_{i-1} = A^T Q_{i-1} (which the next block needs anyway) the k leading
 * Ritz values of the i-block space are computed (M_i = B^T B over those blocks,
 * tridiagonal form and bisection, no vectors); the iteration stops at the first i >= 2
 * where every one of them moved by at most `tol` (relative) since i - 1 blocks, and the
 * Rayleigh-Ritz step runs on those i blocks.  Otherwise it runs q_max iterations
 * (capped as in bks_block_krylov).  stats->q_eff reports the iterations run.  The test
 * reads k values back to the host once per iteration (a stream synchronisation).
 * tol in (0, 1); other arguments as bks_block_krylov (opts.block_p applies).  With
 * widths beyond the tridiagonal kernels the test is skipped and q_max iterations run. */
bks_status bks_block_krylov_adaptive(bks_ctx* ctx, const bks_matrix* A, int k, int q_max, double tol,
                                     uint64_t seed, const void* pi, void* Z, void* sigma, void* V,
                                     const bks_opts* opts, bks_stats* stats);

/* Block Lanczos (Sec. 4, "computing Q"): the classic method the paper relates Algorithm 2
 * to.  Same Krylov space of A A^T from Q_0 = orth(A Pi), built by the three-term block
 * recurrence
 *   W_j = A A^T Q_j - Q_j D_j - Q_{j-1} R_{j-1}^T = Q_{j+1} R_j,   D_j = B_j^T B_j,
 *   R_{j-1} = B_j^T B_{j-1},  B_j = A^T Q_j,
 * so that the Rayleigh quotient T = Q^T A A^T Q is block tridiagonal (k x k blocks D_j on
 * the diagonal, R_j below it, zero elsewhere).  Only that band is formed: no w x w product
 * B^T B as in bks_block_krylov.  Rayleigh-Ritz then takes the k leading eigenvectors of T:
 * Z = Q Ubar_k, sigma_i = |A^T z_i|, V as in bks_block_krylov.  The paper notes that the
 * recurrence may need extra steps to stay numerically orthogonal; `reorth` chooses them:
 *   BKS_REORTH_FULL   W_j is projected twice against every earlier block before its QR
 *                     (Q is then the basis of bks_block_krylov, up to rounding);
 *   BKS_REORTH_LOCAL  twice against Q_{j-1} and Q_j only (the blocks the recurrence uses);
 *   BKS_REORTH_NONE   the recurrence alone (Q drifts from orthogonality once Ritz values
 *                     converge; for study, not for results).
 * The QR of W_j is CholeskyQR2 in every mode.  Other arguments, precisions, opts (except
 * rr_mode, which does not apply) and errors as bks_block_krylov; q is capped the same
 * way. */
typedef enum { BKS_REORTH_FULL = 0, BKS_REORTH_LOCAL = 1, BKS_REORTH_NONE = 2 } bks_reorth;
bks_status bks_block_lanczos(bks_ctx* ctx, const bks_matrix* A, int k, int q, int reorth, uint64_t seed,
                             const void* pi, void* Z, void* sigma, void* V, const bks_opts* opts,
                             bks_stats* stats);

/* ---- building blocks (each one step of the path, exposed for tests and timing) ------ */

/* Start block Pi (Alg. 1/2 step 1), d x k row-major, generated on the device:
 * element e = j*k + c uses SplitMix64 outputs 2(e/2) and 2(e/2)+1 of the stream
 * seeded with `seed` (Steele, Lea & Flood 2014), Box-Muller in FP64 (cosine for even
 * e, sine for odd e), rounded once to `dtype` (BKS_F32 or BKS_F64). */
bks_status bks_gen_pi(bks_ctx* ctx, uint64_t seed, int64_t d, int k, int dtype, void* out);
/* Same generator on the host (FP32 out), for cross-checks without a GPU. */
bks_status bks_gen_pi_host(uint64_t seed, int64_t d, int k, float* out_host);

/* One product with A (Sec. 4: the only access to A): trans = 0 gives Y = A X
 * (X d x c, Y n x c), trans = 1 gives Y = A^T X (X n x c, Y d x c).  X and Y are
 * stored COLUMN-major with leading dimension ldx / ldy (column j of X starts at
 * X + j*ldx), FP32 (FP64 for an FP64 matrix).  flags: BKS_MATMUL_EXACT (BF16 A only)
 * splits X into three BF16 parts so the product is FP32-accurate instead of rounding X
 * to BF16; BKS_MATMUL_SIMT forces the CUDA-core kernel instead of the tensor cores.
 * Honours A->col_mean.  Synchronises the stream once at the end to read the device
 * status word (BKS_ERR_TIMEOUT if a bounded pipeline wait gave up). */
#define BKS_MATMUL_EXACT 1
#define BKS_MATMUL_SIMT 2
bks_status bks_matmul(bks_ctx* ctx, const bks_matrix* A, int trans, int c,
                      const void* X, int64_t ldx, void* Y, int64_t ldy, int flags);

/* CSR of A^T for a CSR matrix A (setup, once per matrix): t_row_ptr (d+1), t_col_idx
 * (nnz, row indices of A) and t_vals (nnz), caller-allocated on the device.  Within a row
 * of A^T the entries keep the ascending row order of A, so products through it are
 * deterministic.  Pass the three arrays in bks_matrix.t_* to every later call on A; a
 * CSR matrix given without them has its transpose rebuilt in the workspace on each
 * call.  Synchronises the stream. */
bks_status bks_csr_transpose(bks_ctx* ctx, const bks_matrix* A, int64_t* t_row_ptr,
                             int32_t* t_col_idx, float* t_vals);

/* Block orthonormalisation (Sec. 4.1/4.2 reorthonormalisation): W (len x c,
 * column-major, ldw) is projected twice against the m orthonormal columns of Qb
 * (len x m, column-major, ldq; m may be 0) and then orthonormalised by CholeskyQR2,
 * in place.  FP32 or FP64 (dtype).  Returns BKS_ERR_BREAKDOWN when W has no
 * numerically independent part left. */
bks_status bks_orthonormalize(bks_ctx* ctx, int dtype, int64_t len, int m, int c,
                              const void* Qb, int64_t ldq, void* W, int64_t ldw);

/* Eigen-decomposition of a symmetric positive semi-definite w x w matrix M (row-major,
 * ldm) by one-sided Jacobi (Alg. 2 step 5: the top singular vectors of M are its top
 * eigenvectors).  lam: out, w eigenvalues, descending.  U: out, w x w row-major,
 * column i the eigenvector of lam[i].  FP32 or FP64 (dtype).  Non-finite entries of M
 * are not detected: the results are then undefined (or BKS_ERR_NOT_CONVERGED). */
bks_status bks_sym_eig(bks_ctx* ctx, int dtype, int w, const void* M, int64_t ldm,
                       void* lam, void* U, int64_t ldu);

/* ---- batches and differentiation ------------------------------------------------- */

/* Block Krylov on a batch of independent matrices (As[0..batch), each dense or CSR, of
 * any shapes), the same k, q and opts for all: Zs[i] (n_i x k), sigmas[i] (k) and, if Vs
 * is non-NULL, Vs[i] (d_i x k), device buffers as for bks_block_krylov.  seeds[i] (NULL:
 * seed i) or pis[i] (NULL array, or NULL entries: generate from the seed) give the start
 * blocks.  The solves run on up to 16 streams of the context (created on first use),
 * launched from up to 8 host threads, so several are in flight at once; each result is
 * that of the single call made with the batch's opts.max_sms (below).  The batch is
 * ordered after the work already on the
 * context's stream, and later work on that stream after the batch.  Each solve's kernels
 * spread over opts.max_sms SMs; with max_sms = 0 the budget cached by bks_batched_autotune
 * for this batch's signature, else an eighth of the SMs, so that several latency-bound
 * solves share the GPU.  statuses[i] (host,
 * may be NULL) receives each solve's status; the return value is the first error, else
 * BKS_WARN_DEFLATED if any solve was capped, else BKS_OK.  stats (may be NULL) sums
 * launches, product bytes and flops over the batch.  Synchronises the streams. */
bks_status bks_block_krylov_batched(bks_ctx* ctx, int batch, const bks_matrix* As, int k, int q,
                                    const uint64_t* seeds, const void* const* pis, void* const* Zs,
                                    void* const* sigmas, void* const* Vs, const bks_opts* opts,
                                    bks_stats* stats, bks_status* statuses);

/* Chooses the SM budget (bks_opts.max_sms) of bks_block_krylov_batched for this batch: runs
 * the batch once per candidate (1/16, 1/8, 1/4, 1/2 and all of the GPU's SMs per solve, after
 * a warm-up pass), keeps the fastest, caches it in the context under the batch's signature
 * (k, q, and the multiset of the matrices' shape classes: kind, dtype, ceil log2 of n and d)
 * and leaves in Zs / sigmas / Vs the results computed with it.  Later batched calls with
 * opts.max_sms = 0 and the same signature use the cached budget; batches never tuned use an
 * eighth of the SMs.  *best_max_sms (may be NULL) receives the budget, *best_ms (may be NULL)
 * its time for the whole batch.  Arguments otherwise as bks_block_krylov_batched. */
bks_status bks_batched_autotune(bks_ctx* ctx, int batch, const bks_matrix* As, int k, int q,
                                const uint64_t* seeds, const void* const* pis, void* const* Zs,
                                void* const* sigmas, void* const* Vs, const bks_opts* opts,
                                int* best_max_sms, float* best_ms);

/* The SM budget a batched solve (method 0 BKI, 1 SI) with opts.max_sms = 0 would use for
 * this batch: the one cached by bks_batched_autotune for its signature, else an eighth of
 * the SMs.  A single call with opts.max_sms set to it reproduces a batch member bit for bit.
 * 0 for bad arguments. */
int bks_batch_budget(const bks_ctx* ctx, int batch, const bks_matrix* As, int k, int q, int method);

/* Krylov width w of a solve: k(q_eff + 1) for Block Krylov (method 0; q capped so that
 * w <= min(n, d), Sec. 4), k for Simultaneous Iteration (method 1).  0 for bad sizes. */
int bks_krylov_width(int64_t n, int64_t d, int k, int q, int method);

/* All w Ritz triplets of a solve (method 0: Algorithm 2, 1: Algorithm 1) instead of the
 * top k: U (n x w, row-major; column j = Q ubar_j, Sec. 4), sigma (w, descending) and V
 * (d x w, row-major; v_j = A^T u_j / sigma_j).  The first k columns are bks_block_krylov's
 * Z and V.  w = bks_krylov_width(n, d, k, q, method).  Dense or CSR A, FP32 or FP64;
 * errors as for bks_block_krylov.  This is the forward state that bks_backward needs. */
bks_status bks_ritz_triplets(bks_ctx* ctx, const bks_matrix* A, int k, int q, uint64_t seed,
                             const void* pi, int method, void* U, void* sigma, void* V,
                             const bks_opts* opts, bks_stats* stats);

/* The Ritz triplets of a batch of independent matrices (the forward state of a batched
 * forward and backward): for each i, as bks_ritz_triplets on As[i], Us[i] (n_i x w_i),
 * sigmas[i] (w_i) and Vs[i] (d_i x w_i), w_i = bks_krylov_width(n_i, d_i, k, q, method).
 * Streams, host threads, seeds, pis, statuses and the return value as for
 * bks_block_krylov_batched (the SM budget included); every result is that of the single
 * call made with the same opts.max_sms.  Synchronises the streams. */
bks_status bks_ritz_triplets_batched(bks_ctx* ctx, int batch, const bks_matrix* As, int k, int q,
                                     const uint64_t* seeds, const void* const* pis, int method,
                                     void* const* Us, void* const* sigmas, void* const* Vs,
                                     const bks_opts* opts, bks_status* statuses);

/* Gradient of a loss through Sigma_k and A_k = Z Z^T A with respect to A, from the w Ritz
 * triplets (U n x w, sigma w, V d x w, row-major, as written by bks_ritz_triplets).  No
 * counterpart in the paper, which does not differentiate its outputs.  g_sigma (k,
 * device, may be NULL) is dL/dSigma_k, G (n x d row-major, device, may be NULL) is
 * dL/dA_k; dA (n x d row-major) receives
 *   U_k diag(g_sigma) V_k^T + U_k U_k^T G + sum_{i<=k<j<=w} c_ij (s_i u_j v_i^T + s_j u_i v_j^T)
 *   + (I - U_w U_w^T) G V_k V_k^T,   c_ij = (s_i u_j^T G v_i + s_j u_i^T G v_j) / (s_i^2 - s_j^2),
 * with c_ij = 0 where s_i^2 - s_j^2 <= gap_tau s_1^2 (gap_tau <= 0: 1e-10 for FP64, 1e-6
 * for FP32).  Exact when the Krylov space contains range(A).  dtype BKS_F32 or BKS_F64
 * for every array.  BKS_ERR_INVALID_ARG when both upstream gradients are NULL.
 * Synchronises the context's stream. */
bks_status bks_backward(bks_ctx* ctx, int dtype, int64_t n, int64_t d, int k, int w,
                        const void* U, const void* sigma, const void* V, const void* g_sigma,
                        const void* G, void* dA, double gap_tau);

/* bks_backward for a batch of independent solves: matrix i is ns[i] x ds[i] with Krylov
 * width ws[i], triplets Us[i], sigmas[i], Vs[i] (as written by bks_ritz_triplets_batched),
 * upstream gradients g_sigmas[i] (k) and Gs[i] (ns[i] x ds[i]) -- either array may be NULL,
 * and so may its entries, but not both for one matrix -- and output dAs[i].  The calls run
 * on the context's batch streams from several host threads; each result is that of
 * bks_backward.  statuses (host, may be NULL) receives each status; the return value is
 * the first error, else BKS_OK.  Synchronises the streams. */
bks_status bks_backward_batched(bks_ctx* ctx, int dtype, int batch, const int64_t* ns, const int64_t* ds,
                                int k, const int* ws, const void* const* Us, const void* const* sigmas,
                                const void* const* Vs, const void* const* g_sigmas, const void* const* Gs,
                                void* const* dAs, double gap_tau, bks_status* statuses);

/* out (n x d row-major) = U_r diag(sigma_r) V_r^T with the first r columns of U (n x ldu)
 * and V (d x ldv), row-major, dtype BKS_F32 or BKS_F64: the rank-r approximation
 * A_r = Z Z^T A of a solve (Z = U_r, A^T Z = V_r diag(sigma_r)).  Synchronises the
 * context's stream. */
bks_status bks_low_rank(bks_ctx* ctx, int dtype, int64_t n, int64_t d, int r, const void* U,
                        int64_t ldu, const void* sigma, const void* V, int64_t ldv, void* out);

/* ---- failure-path self-test ------------------------------------------------------- */

/* Runs one of the library's bounded device-side waits on a condition that nothing
 * satisfies, so that the failure path can be tested without a GPU fault: which = 0 waits
 * on an mbarrier phase that no thread or copy completes (the wait of the tensor-core
 * pipelines), which = 1 on a grid barrier that expects one more CTA than is launched (the
 * barrier of the cooperative orthonormalisation kernels).  The wait gives up after its
 * limit (1 s), the kernel returns normally and the call returns BKS_ERR_TIMEOUT; the
 * context and the stream remain usable.  No counterpart in the paper.  Synchronises the
 * context's stream. */
bks_status bks_selftest_wait(bks_ctx* ctx, int which);

/* ---- allocation-free variant ------------------------------------------------------ */

/* bks_sym_eig without any device allocation.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory when they call, for
 * example code running where cudaMalloc's implicit device synchronisation is not
 * allowed, applications whose device memory is owned by another runtime or a fixed
 * arena, or deployments that must not grow their footprint after start-up.
 *
 * Same computation and arguments as bks_sym_eig (one-sided Jacobi on a symmetric PSD
 * w x w matrix M; lam descending, U's columns the eigenvectors), with no context: it
 * runs on the caller's current device and on `stream` (a cudaStream_t, NULL = legacy
 * default stream), and synchronises that stream once at the end to read its status.
 * M, lam and U are caller-owned device buffers.
 *
 * All scratch lives in one statically sized device array of 5 MiB that is part of the
 * library image: every GPU that loads the library holds it until the process exits.
 * The limit is w <= BKS_NOALLOC_EIG_MAX_W (FP32 or FP64); larger w returns
 * BKS_ERR_INVALID_ARG.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  Every call shares the one array, which keeps the
 * previous call's contents (the status words are cleared at the start of each call):
 * calls whose work overlaps on the GPU (other streams, other host threads) race on it
 * and must be serialised by the caller.  The address looked up on the first call is
 * kept for the life of the process: it assumes the device's primary context (the one
 * the CUDA runtime uses) and no cudaDeviceReset in between.  As for bks_sym_eig,
 * non-finite entries of M are not detected.  Errors are returned as status codes only
 * (there is no context for bks_last_error). */
#define BKS_NOALLOC_EIG_MAX_W 512
bks_status bks_sym_eig_noalloc(void* stream, int dtype, int w, const void* M, int64_t ldm,
                               void* lam, void* U, int64_t ldu);

#ifdef __cplusplus
}
#endif
#endif /* BKS_H */
