// Block orthonormalisation of a new Krylov block (Sec. 4.1 and 4.2: orthonormalise
// each block as it is computed; the span is unchanged in exact arithmetic).
//   1. Block classical Gram-Schmidt, twice (BCGS2):  W <- W - Q (Q^T W)
//   2. CholeskyQR, twice (CholeskyQR2):  G = W^T W,  G = R^T R,  W <- W R^{-1}
// Gram matrices are accumulated in FP64 across CTAs; the Cholesky factorisation runs
// in FP64 in one CTA; W R^{-1} is a row-parallel forward substitution.  A Gram
// matrix whose Cholesky factorisation meets a non-positive pivot is retried with a
// growing diagonal shift (shifted CholeskyQR, Fukaya et al. 2020) and a third
// CholeskyQR pass then restores orthogonality.
#include "common.cuh"

namespace bks {

namespace {

// G (c x c, FP64, row-major) -> R (c x c upper triangular, row-major, type T).
// One CTA.  Right-looking factorisation on the upper triangle held in shared memory.
template <typename T>
__global__ void chol_kernel(const double* __restrict__ G, int c, T* __restrict__ R,
                            int* status, int* shifted_flag) {
    extern __shared__ double S[];   // c*c
    __shared__ int ok_s;
    __shared__ double trace_s;
    const int tid = threadIdx.x, nt = blockDim.x;
    bool bad = false;
    for (int e = tid; e < c * c; e += nt) bad |= !isfinite(G[e]);
    if (__syncthreads_or(bad)) {
        if (tid == 0) atomicOr(status, ST_NONFINITE);
        for (int e = tid; e < c * c; e += nt) R[e] = T((e / c == e % c) ? 1.0 : 0.0);
        return;
    }
    if (tid == 0) {
        double t = 0.0;
        for (int j = 0; j < c; ++j) t += G[j * c + j];
        trace_s = t;
    }
    __syncthreads();
    double shift = 0.0;
    for (int attempt = 0; attempt < 6; ++attempt) {
        for (int e = tid; e < c * c; e += nt) {
            const int a = e / c, b = e % c;
            // use the upper triangle only (symmetric input)
            S[e] = (a <= b) ? G[a * c + b] : 0.0;
            if (a == b) S[e] += shift;
        }
        if (tid == 0) ok_s = 1;
        __syncthreads();
        for (int j = 0; j < c; ++j) {
            const double piv = S[j * c + j];
            if (!(piv > 0.0) || !isfinite(piv)) {   // uniform: every thread sees the same value
                if (tid == 0) ok_s = 0;
                break;
            }
            const double rjj = sqrt(piv);
            const double inv = 1.0 / rjj;
            __syncthreads();
            for (int l = j + 1 + tid; l < c; l += nt) S[j * c + l] *= inv;
            if (tid == 0) S[j * c + j] = rjj;
            __syncthreads();
            const int m = c - j - 1;
            // trailing update of the upper triangle: S[a][b] -= R[j][a] R[j][b], j < a <= b
            for (int e = tid; e < m * m; e += nt) {
                const int a = j + 1 + e / m, b = j + 1 + e % m;
                if (a <= b) S[a * c + b] -= S[j * c + a] * S[j * c + b];
            }
            __syncthreads();
        }
        __syncthreads();
        if (ok_s) break;
        // shifted CholeskyQR: grow the diagonal shift relative to the trace
        shift = (shift == 0.0) ? 1e-12 * trace_s / c : shift * 1e3;
        if (tid == 0) atomicOr(shifted_flag, 1);
        __syncthreads();
    }
    if (!ok_s) {
        if (tid == 0) atomicOr(status, ST_BREAKDOWN);
        for (int e = tid; e < c * c; e += nt) R[e] = T((e / c == e % c) ? 1.0 : 0.0);
        return;
    }
    if (shift > 0.0 && tid == 0) atomicOr(status, ST_SHIFTED);
    for (int e = tid; e < c * c; e += nt) {
        const int a = e / c, b = e % c;
        R[e] = T(a <= b ? S[e] : 0.0);
    }
}

// Q = W R^{-1} row by row: for position r, q_j = (w_j - sum_{i<j} q_i R[i][j]) / R[j][j].
// W and Q are column-major thin blocks (row j of the array = column j).  W == Q allowed.
template <typename T>
__global__ void trsm_rows_kernel(const T* W, int64_t ldw, const T* __restrict__ R, int c, T* Q,
                                 int64_t ldq, int64_t len) {
    extern __shared__ unsigned char smem_raw[];
    T* Rs = reinterpret_cast<T*>(smem_raw);          // c*c
    T* Ws = Rs + c * c;                              // c * blockDim.x
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int e = tid; e < c * c; e += nt) Rs[e] = R[e];
    const int64_t r = int64_t(blockIdx.x) * nt + tid;
    const bool live = r < len;
    for (int j = 0; j < c; ++j) Ws[j * nt + tid] = live ? W[j * ldw + r] : T(0);
    __syncthreads();
    for (int j = 0; j < c; ++j) {
        T acc = Ws[j * nt + tid];
        for (int i = 0; i < j; ++i) acc = fma(-Ws[i * nt + tid], Rs[i * c + j], acc);
        Ws[j * nt + tid] = acc / Rs[j * c + j];
    }
    if (live)
        for (int j = 0; j < c; ++j) Q[j * ldq + r] = Ws[j * nt + tid];
}

template <typename T>
void cholqr_pass(Exec& ex, int64_t len, int64_t ld, const T* src, int c, T* dst, double* partials,
                 int64_t cap, double* gram, T* rfac, int* shifted_flag) {
    GemmDesc g{};
    g.M = c; g.N = c; g.K = len;
    g.X = src; g.ldx = ld; g.Y = src; g.ldy = ld;
    g.y_kmajor = true; g.y_dtype = sizeof(T) == 8 ? 0 : 1;
    g.out = gram; g.ldo = c; g.out_transposed = false; g.out_f64 = true;
    g.alpha = 1.0; g.beta = 0.0;
    gemm_simt<T>(ex, g, partials, cap);
    const size_t smem = size_t(c) * c * sizeof(double);
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(chol_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    chol_kernel<T><<<1, 256, smem, ex.stream>>>(gram, c, rfac, ex.status, shifted_flag);
    ex.launches++;
    int nt = 128;
    size_t smem2 = size_t(c) * c * sizeof(T) + size_t(c) * nt * sizeof(T);
    while (smem2 > 200 * 1024 && nt > 32) {
        nt /= 2;
        smem2 = size_t(c) * c * sizeof(T) + size_t(c) * nt * sizeof(T);
    }
    if (smem2 > 48 * 1024)
        cudaFuncSetAttribute(trsm_rows_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             int(smem2));
    trsm_rows_kernel<T><<<unsigned((len + nt - 1) / nt), nt, smem2, ex.stream>>>(src, ld, rfac, c,
                                                                                  dst, ld, len);
    ex.launches++;
}

}  // namespace

// W (c x ld) against Qb (m x ld): BCGS2 then CholeskyQR2, result in Qout.  Wtmp holds
// the first CholeskyQR iterate; `ct` (c x m, type T) the projection coefficients.
template <typename T>
void orth_block(Exec& ex, int64_t len, int64_t ld, const T* Qb, int m, T* W, int c, T* Wtmp,
                T* Qout, double* partials, int64_t cap, double* gram, T* rfac, T* ct,
                int* shifted_flag) {
    const int ydt = sizeof(T) == 8 ? 0 : 1;
    if (m > 0) {
        for (int pass = 0; pass < 2; ++pass) {
            GemmDesc g1{};   // ct = (Qb W^T)^T : c x m
            g1.M = m; g1.N = c; g1.K = len;
            g1.X = Qb; g1.ldx = ld; g1.Y = W; g1.ldy = ld;
            g1.y_kmajor = true; g1.y_dtype = ydt;
            g1.out = ct; g1.ldo = m; g1.out_transposed = true;
            g1.alpha = 1.0; g1.beta = 0.0;
            gemm_simt<T>(ex, g1, partials, cap);
            GemmDesc g2{};   // W -= ct Qb
            g2.M = c; g2.N = len; g2.K = m;
            g2.X = ct; g2.ldx = m; g2.Y = Qb; g2.ldy = ld;
            g2.y_kmajor = false; g2.y_dtype = ydt;
            g2.out = W; g2.ldo = ld; g2.out_transposed = false;
            g2.alpha = -1.0; g2.beta = 1.0;
            gemm_simt<T>(ex, g2, partials, cap);
        }
    }
    cholqr_pass<T>(ex, len, ld, W, c, Wtmp, partials, cap, gram, rfac, shifted_flag);
    cholqr_pass<T>(ex, len, ld, Wtmp, c, Qout, partials, cap, gram, rfac, shifted_flag);
}

// A third CholeskyQR pass in place (after a shifted factorisation).
template <typename T>
void cholqr_extra(Exec& ex, int64_t len, int64_t ld, T* Q, int c, double* partials, int64_t cap,
                  double* gram, T* rfac, int* shifted_flag) {
    cholqr_pass<T>(ex, len, ld, Q, c, Q, partials, cap, gram, rfac, shifted_flag);
}

#define BKS_INST(T)                                                                          \
    template void orth_block<T>(Exec&, int64_t, int64_t, const T*, int, T*, int, T*, T*,     \
                                double*, int64_t, double*, T*, T*, int*);                    \
    template void cholqr_extra<T>(Exec&, int64_t, int64_t, T*, int, double*, int64_t,        \
                                  double*, T*, int*);
BKS_INST(float)
BKS_INST(double)
#undef BKS_INST

}  // namespace bks
