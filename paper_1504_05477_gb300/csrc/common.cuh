// Internal declarations shared by the kernels and the host orchestration.
// Layout conventions inside the library:
//   * "thin blocks" (Pi, Krylov blocks Q_i, B_i = A^T Q_i, Ritz vectors) are stored
//     column by column: a block of c columns of length L is a c x ld row-major array
//     whose row j is column j (ld >= L, padded to a multiple of 32 elements, pad = 0).
//   * A is the caller's row-major n x d matrix (ld >= d).
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace bks {

// Device status word bits (OR-ed by kernels, read once by the host at the end).
enum : int {
    ST_NONFINITE = 1,
    ST_BREAKDOWN = 2,
    ST_NOT_CONVERGED = 4,
    ST_TIMEOUT = 8,
    ST_SHIFTED = 16,
    ST_BADINPUT = 32,     // a CSR structure check failed (nothing indexed through it)
};

inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// Element conversions used by templated loads.
template <typename T> __device__ __forceinline__ T cvt(float x) { return static_cast<T>(x); }
template <typename T> __device__ __forceinline__ T cvt(double x) { return static_cast<T>(x); }
template <typename T> __device__ __forceinline__ T cvt(__nv_bfloat16 x) {
    return static_cast<T>(__bfloat162float(x));
}

template <typename T> __device__ __forceinline__ bool finite_val(T x) { return isfinite(x); }

// Events bracketing every launch of the dominant product kernel (profiling only).
struct KernelLog {
    static constexpr int CAP = 512;
    cudaEvent_t ev[CAP];
    int created = 0;
    int n = 0;
    void record(cudaStream_t s) {
        if (n >= CAP) return;
        if (n >= created) {
            cudaEventCreate(&ev[n]);
            created = n + 1;
        }
        cudaEventRecord(ev[n++], s);
    }
};

// Raise a kernel's dynamic shared-memory limit to the device's opt-in maximum, once per
// kernel and device (thread-safe); fails when `need` exceeds it.  A per-launch limit set to
// each launch's own size would race between host threads that launch the same kernel
// with different sizes (the limit is per function, not per launch).
cudaError_t allow_dynamic_smem(const void* fn, size_t need);

// Per-call launch bookkeeping.
struct Exec {
    cudaStream_t stream = nullptr;
    int* status = nullptr;       // device status word
    int num_sms = 148;
    int launches = 0;
    int product_launches = 0;
    KernelLog* klog = nullptr;   // non-null: time each product-kernel launch
};

// ------------------------------------------------------------------ SIMT GEMM
// Out[m][n] = alpha * sum_k X[m][k] * Yop[k][n] (+ beta * Out), where X is row-major
// M x K and Yop[k][n] = Y[n][k] (y_kmajor) or Y[k][n] (!y_kmajor).
struct GemmDesc {
    int64_t M, N, K;
    const void* X; int64_t ldx;
    const void* Y; int64_t ldy;
    bool y_kmajor;
    int y_dtype;               // 0 f64, 1 f32, 2 bf16 (bks_dtype)
    // output
    void* out; int64_t ldo;
    bool out_transposed;       // store Out[m][n] at out[n * ldo + m]
    bool out_f64 = false;      // output is FP64 whatever T is (Gram matrices)
    double alpha, beta;
    // centring correction for the dense-A products: Out[m][n] -= alpha * corr
    //   y_kmajor (A X):    corr = (mu . X[m,:])            (same for every n)
    //   !y_kmajor (A^T X): corr = mu[n] * sum_k X[m][k]
    const float* col_mean = nullptr;
};

// Launch the SIMT tile GEMM in precision T (float or double).  Split-K is chosen
// internally; partial sums go through `partials` (FP64, caller workspace, at least
// gemm_partial_elems(...) doubles) and are reduced in a fixed order.
template <typename T>
void gemm_simt(Exec& ex, const GemmDesc& g, double* partials, int64_t partial_cap);
int64_t gemm_partial_elems(int64_t M, int64_t N, int64_t K, int num_sms);

// Tensor-core (tcgen05, 3xTF32) product with an FP32 dense A: Y = (A X)^T (trans false)
// or (A^T X)^T (trans true), thin blocks column-major.  xh/xl: c x ldx scratch each;
// part: tc_partial_floats(...) floats.  Returns false, launching nothing, when the
// operands do not meet the TMA alignment rules.
// subtract: Y -= the product (Y is read) instead of Y = the product.
bool tc_product_f32(Exec& ex, const float* A, int64_t n, int64_t d, int64_t lda, bool trans, int c,
                    const float* X, int64_t ldx, float* Y, int64_t ldy, float* xh, float* xl,
                    float* part, int64_t part_cap, bool subtract = false);
int64_t tc_partial_floats(int64_t n, int64_t d, int c, int num_sms);
// Tensor-core product with a BF16 A (kind::f16): X (FP32) is split into np = 1 (X
// rounded to BF16) or np = 3 (FP32-accurate) BF16 pieces in xb (np * min(c, 128) * ldx
// elements at least, xb_cap).  Returns false, launching nothing, when the operands do
// not meet the TMA alignment rules.
bool tc_product_bf16(Exec& ex, const __nv_bfloat16* A, int64_t n, int64_t d, int64_t lda, bool trans,
                     int c, int np, const float* X, int64_t ldx, float* Y, int64_t ldy, __nv_bfloat16* xb,
                     int64_t xb_cap, float* part, int64_t part_cap);
int64_t tc_bf16_partial_floats(int64_t n, int64_t d, int c, int num_sms);

// ------------------------------------------------------------------ sparse A (CSR)
size_t csr_transpose_scratch(int64_t n, int64_t d);
// Structure check of a CSR (rows x cols): row_ptr[0] = 0, non-decreasing, row_ptr[rows] =
// nnz, column indices in [0, cols) and strictly increasing within each row.  A failure
// ORs ST_BADINPUT into *status; every later CSR kernel of the call reads *status and
// then indexes nothing through the arrays.
void csr_check(Exec& ex, const int64_t* row_ptr, const int32_t* col, int64_t rows, int64_t cols,
               int64_t nnz, int* status);
// CSR of A^T (rows of A^T in ascending row order of A: deterministic).
void csr_transpose(Exec& ex, const int64_t* row_ptr, const int32_t* col, const float* val, int64_t n,
                   int64_t d, int64_t nnz, int64_t* t_row_ptr, int32_t* t_col, float* t_val,
                   void* scratch);
int64_t seg_upper_bound(int64_t rows, int64_t nnz);
void csr_segments(Exec& ex, const int64_t* row_ptr, int64_t rows, int64_t* nseg_tmp, int64_t* seg_off,
                  int64_t* seg_row, int64_t* sums);
// Row pitch (floats) of the row-major staging of X and Y, and the doubles the centring
// sums need, for c columns.
int csr_row_pitch(int c);
int64_t csr_cvec_doubles(int c);
// Yt (c x ldy thin) = op(A) Xt with op(A) given by its CSR (rows x cols); corr_kind 0: none,
// 1: subtract mu^T X from every row, 2: subtract mu[row] (1^T X).
void csr_product(Exec& ex, const int64_t* row_ptr, const int32_t* col, const float* val, int64_t rows,
                 int64_t cols, int64_t nnz, const int64_t* seg_off, const int64_t* seg_row,
                 int64_t nseg_bound, const float* Xt, int64_t ldx, int c, float* Yt, int64_t ldy,
                 float* x_rm, float* y_rm, float* part, int corr_kind, const float* mu, double* cvec);

// ------------------------------------------------------------------ building blocks
template <typename T>
void gen_pi_device(Exec& ex, uint64_t seed, int64_t d, int k, T* out, int64_t ld_row,
                   bool transposed);
void gen_pi_host(uint64_t seed, int64_t d, int k, float* out);

// Copy a row-major rows x cols matrix (src dtype -> T) into column-major thin storage.
template <typename T>
void transpose_in(Exec& ex, const void* src, int src_dtype, int64_t rows, int64_t cols,
                  int64_t lds, T* dst, int64_t ldd);

// Scratch of the block orthonormalisation (pointers into the caller's workspace).
struct OrthWs {
    double* partials = nullptr;   // SIMT split-K partials (cap doubles)
    int64_t cap = 0;
    void* g = nullptr;            // c x ldp Gram matrix (T)
    void* rfac = nullptr;         // c x ldp, P = R^{-T} (T)
    int ldp = 0;
    void* ct = nullptr;           // c x ldc projection coefficients (T)
    int64_t ldc = 0;
    float* xh = nullptr;          // tensor-core path (FP32 only; nullptr disables it):
    float* xl = nullptr;          //   c x ld_max hi / lo split of the X operand
    float* tpart = nullptr;       //   stream-K partial tiles
    int64_t tpart_cap = 0;
    int* shifted_flag = nullptr;  // device int: a Cholesky needed a diagonal shift
    float* fpart = nullptr;       // fused kernel (FP32; nullptr disables it): per-CTA partial
    int64_t fpart_cap = 0;        //   Grams (floats), the reduced Gram and the barrier words
    float* fgram = nullptr;
    unsigned* fbar = nullptr;
    // tensor-core kernel (FP32; otc_part == nullptr disables it): partial Grams, the
    // coefficient tiles (128 x otc_ldct), the reduced c x c Gram and the barrier words
    float* otc_part = nullptr;
    int64_t otc_cap = 0;
    float* otc_cts = nullptr;
    int64_t otc_ldct = 0;
    float* otc_h = nullptr;
    unsigned* otc_bar = nullptr;
    // row-major copy of the m earlier columns (len x ldr); the call appends its output
    // block at columns [m, m + c).  nullptr: only m = 0 runs on the tensor-core kernel
    float* qr = nullptr;
    int64_t ldr = 0;
    bool qr_append = false;       // write the output block into qr at columns [m, m + c)
    bool* tc_used = nullptr;      // host flag: set to whether the tensor-core kernel ran
};
// Byte sizes of those buffers for blocks of c columns, at most mmax earlier columns and
// lengths up to len_max (pitch up to ld_max).
struct OrthSizes {
    size_t partials, g, rfac, ct, xh, tpart, fpart, fgram, fbar, otc_part, otc_cts, otc_h, otc_bar;
    int ldp;
    int64_t ldc, cap, tcap, fcap, otc_cap, otc_ldct;
};
OrthSizes orth_sizes(int64_t len_max, int64_t ld_max, int mmax, int c, int elem_bytes, bool tc, int num_sms);

// Tensor-core block orthonormalisation (orth_tc.cu): W (c x ld) against Qc (m x ld) and its
// row-major copy Qr (len x ldr; may be nullptr when m = 0), result in Qout and, when Qr_out
// is non-null, row-major at Qr_out (pitch ldr).  False, launching nothing, when the
// shapes do not fit.
bool orth_tc_fits(int64_t len, int m, int c, int num_sms);
// Failure-path self-test: one bounded wait (0: mbarrier, 1: grid barrier) on a condition
// nothing satisfies; it gives up after its limit and ORs ST_TIMEOUT into *ex.status.
// bar: two zeroed words of device scratch.  False for an unknown `which`.
bool wait_selftest(Exec& ex, int which, unsigned* bar);
size_t orth_tc_part_floats(int64_t len, int mmax, int c, int num_sms);
bool orth_tc(Exec& ex, int64_t len, int64_t ld, const float* Qc, int m, const float* W, int c, float* Qout,
             const float* Qr, float* Qr_out, int64_t ldr, float* part, int64_t part_cap, float* cts, int64_t ldct,
             float* hbuf, unsigned* bar, int* shifted_flag);

// Block orthonormalisation: W (c x ld thin) against Qb (m x ld thin), BCGS2 then
// CholeskyQR2, result in Qout (may equal W); Wtmp: c x ld scratch.
template <typename T>
void orth_block(Exec& ex, int64_t len, int64_t ld, const T* Qb, int m, T* W, int c, T* Wtmp, T* Qout,
                const OrthWs& ws);
// Jacobi launch plan (cluster size C, block width b, register tile E, shared bytes).
bool jacobi_plan(int w, int elem_bytes, int& C, int& b, int& E, size_t& smem);

// One-sided Jacobi on X (w x w, column j = row j of Xin; X is a w x ldw scratch copy).
// On return lam[0..w) = column norms of the converged X (descending), nrm[j] the norm
// of column j, Vt (w x ldv) row i = normalised column of lam[i].
template <typename T>
void sym_eig(Exec& ex, int w, const T* Xin, int64_t ldx, T* X, int64_t ldw, T* lam, T* nrm,
             T* Vt, int64_t ldv, int* order, int max_sweeps, double tol, int* sweeps_dev);

// Eigenvectors of the m largest eigenvalues of the symmetric w x w M (row pitch w) by
// Householder tridiagonalisation, multisection, inverse iteration and one CholeskyQR2
// (orth_block with `ows`, sized for blocks of m columns at least w long): row i of Vt
// (pitch ldv) = eigenvector of the i-th largest eigenvalue.  `scratch`:
// tridiag_scratch_elems elements of T.  False (nothing launched) when the sizes do not
// fit its kernels.
template <typename T>
bool tridiag_fits(int w, int m);
size_t tridiag_scratch_elems(int w, int m);
struct OrthWs;
template <typename T>
bool topk_tridiag(Exec& ex, int w, const T* M, int m, T* Vt, int64_t ldv, T* scratch, const OrthWs& ows);
// The m largest eigenvalues alone (tridiagonal form and multisection): on return *lam
// points at m device values, descending, to be multiplied by the device scalar at
// *scale; both live in `scratch`.
template <typename T>
bool topk_values(Exec& ex, int w, const T* M, int m, T* scratch, const T** lam, const T** scale);

// Column-wise argmax |.| sign normalisation of a row-major n x k matrix (and the
// matching rows of Ut, k x ldu).
template <typename T>
void sign_fix(Exec& ex, T* Z, int64_t n, int k, int64_t ldz, T* Ut, int64_t w, int64_t ldu);
// The same on a column-major Zt (column i at Zt + i ldz): coalesced column scans.
template <typename T>
void sign_fix_cm(Exec& ex, T* Zt, int64_t n, int k, int64_t ldz, T* Ut, int64_t w, int64_t ldu);

// sigma_i = |row i of Vt| (FP64 accumulation); optionally scale row i by 1/sigma_i.
template <typename T>
void row_norms(Exec& ex, T* Vt, int k, int64_t len, int64_t ldv, T* sigma, bool normalise);

// dst (rows x cols, row pitch ldd) = src (row pitch lds), converted element by element.
template <typename TS, typename TD>
void cast_2d(Exec& ex, const TS* src, int64_t rows, int64_t cols, int64_t lds, TD* dst, int64_t ldd);

// Scan `n` values for non-finite entries, OR-ing ST_NONFINITE into the status word.
template <typename T>
void check_finite(Exec& ex, const T* x, int64_t n);

// Block Lanczos (Sec. 4): complete the block-tridiagonal T (w x w, row-major, ld w) whose
// row blocks hold [R_{j-1} D_j] (k x k Gram products of the B blocks, lower band and
// diagonal): the diagonal blocks are symmetrised, R_{j-1}^T is mirrored above the
// diagonal and every block off the band is set to zero.
template <typename T>
void lanczos_band(Exec& ex, T* t, int w, int k);

}  // namespace bks
