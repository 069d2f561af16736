// Block orthonormalisation of a new Krylov block (Sec. 4.1 and 4.2: orthonormalise
// each block as it is computed; the span is unchanged in exact arithmetic).
//   1. Block classical Gram-Schmidt, twice (BCGS2):  W <- W - Q (Q^T W)
//   2. CholeskyQR, twice (CholeskyQR2):  G = W^T W,  G = R^T R,  W <- W R^{-1}
// Gram matrices are accumulated in FP64 across CTAs.  The c x c Cholesky factor and
// its inverse are formed by one CTA in the path's precision (FP32 on the FP32 path:
// the second CholeskyQR pass removes the orthogonality lost to the first pass's
// rounding as long as cond(W) stays below about 1e3, which the two projections
// ensure), and W R^{-1} runs as a parallel GEMM.  A factorisation that meets a
// non-positive pivot is retried with a growing diagonal shift (shifted CholeskyQR,
// Fukaya et al. 2020); the status word records the shift.
#include "common.cuh"

namespace bks {

namespace {

// G (c x c, FP64, row-major, symmetric) -> P = R^{-T} (c x c row-major, type T), where
// G = R^T R with R upper triangular; Q = W R^{-1} is then Q^T = P W^T.  One CTA.
template <typename T>
__global__ void chol_inv_kernel(const double* __restrict__ G, int c, T* __restrict__ P,
                                int* status, int* shifted_flag, bool gauss_jordan) {
    extern __shared__ unsigned char smem_raw[];
    T* S = reinterpret_cast<T*>(smem_raw);   // c*c: R (upper triangle)
    __shared__ int ok_s;
    __shared__ double trace_s;
    const int tid = threadIdx.x, nt = blockDim.x;
    __shared__ double red[32];
    // one coalesced pass over G: finiteness, the trace, and the upper triangle into S
    bool bad = false;
    double tr = 0.0;
    for (int e = tid; e < c * c; e += nt) {
        const double g = G[e];
        bad |= !isfinite(g);
        const int a = e / c, b = e - a * c;
        if (a == b) tr += g;
        S[e] = (a <= b) ? T(g) : T(0);
    }
    if (__syncthreads_or(bad)) {
        if (tid == 0) atomicOr(status, ST_NONFINITE);
        for (int e = tid; e < c * c; e += nt) P[e] = T((e / c == e % c) ? 1.0 : 0.0);
        return;
    }
    for (int o = 16; o > 0; o >>= 1) tr += __shfl_xor_sync(0xffffffffu, tr, o);
    if ((tid & 31) == 0) red[tid >> 5] = tr;
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < (nt >> 5); ++w) t += red[w];
        trace_s = t;
    }
    __syncthreads();
    double shift = 0.0;
    for (int attempt = 0; attempt < 6; ++attempt) {
        if (attempt > 0)   // rebuild S with a diagonal shift (rare path)
            for (int e = tid; e < c * c; e += nt) {
                const int a = e / c, b = e - a * c;
                S[e] = (a <= b) ? T(G[e] + (a == b ? shift : 0.0)) : T(0);
            }
        if (tid == 0) ok_s = 1;
        __syncthreads();
        for (int j = 0; j < c; ++j) {
            const T piv = S[j * c + j];
            if (!(piv > T(0)) || !isfinite(piv)) {   // uniform: every thread sees the same value
                if (tid == 0) ok_s = 0;
                break;
            }
            const T rjj = sqrt(piv);
            const T inv = T(1) / rjj;
            __syncthreads();
            for (int l = j + 1 + tid; l < c; l += nt) S[j * c + l] *= inv;
            if (tid == 0) S[j * c + j] = rjj;
            __syncthreads();
            // trailing update of the upper triangle: S[a][b] -= R[j][a] R[j][b], j < a <= b
            // (16 x 16 thread grid over the trailing square)
            const int ty = tid >> 4, tx = tid & 15;
            for (int a = j + 1 + ty; a < c; a += 16) {
                const T rja = S[j * c + a];
                for (int b = j + 1 + tx; b < c; b += 16)
                    if (a <= b) S[a * c + b] -= rja * S[j * c + b];
            }
            __syncthreads();
        }
        __syncthreads();
        if (ok_s) break;
        shift = (shift == 0.0) ? (sizeof(T) == 8 ? 1e-12 : 1e-6) * trace_s / c : shift * 1e3;
        if (tid == 0) atomicOr(shifted_flag, 1);
        __syncthreads();
    }
    if (!ok_s) {
        if (tid == 0) atomicOr(status, ST_BREAKDOWN);
        for (int e = tid; e < c * c; e += nt) P[e] = T((e / c == e % c) ? 1.0 : 0.0);
        return;
    }
    if (shift > 0.0 && tid == 0) atomicOr(status, ST_SHIFTED);
    if (gauss_jordan) {
        // R^{-1} by Gauss-Jordan elimination on [R | I], pivots from the last row up: row i
        // is scaled by 1/R[i][i], then column i is eliminated from the rows above.  Row i
        // of the inverse is non-zero only in columns >= i, so each step touches i x (c-i)
        // entries, all in parallel.
        T* Ri = S + c * c;
        for (int e = tid; e < c * c; e += nt) Ri[e] = T((e / c == e % c) ? 1.0 : 0.0);
        __syncthreads();
        const int ty = tid >> 4, tx = tid & 15;
        for (int i = c - 1; i >= 0; --i) {
            const T inv = T(1) / S[i * c + i];
            for (int j = i + tid; j < c; j += nt) Ri[i * c + j] *= inv;
            __syncthreads();
            for (int r = ty; r < i; r += 16) {
                const T f = S[r * c + i];
                for (int j = i + tx; j < c; j += 16) Ri[r * c + j] -= f * Ri[i * c + j];
            }
            __syncthreads();
        }
        for (int e = tid; e < c * c; e += nt) {
            const int a = e / c, b = e % c;
            P[e] = Ri[b * c + a];   // P = R^{-T}
        }
        return;
    }
    // (wide FP64 blocks) R^{-1} column by column: thread j solves R x = e_j by back
    // substitution and keeps x in row j of P = R^{-T} (only thread j touches that row)
    for (int j = tid; j < c; j += nt) {
        T* x = P + int64_t(j) * c;
        for (int i = j + 1; i < c; ++i) x[i] = T(0);
        x[j] = T(1) / S[j * c + j];
        for (int i = j - 1; i >= 0; --i) {
            T acc = T(0);
            for (int l = i + 1; l <= j; ++l) acc = fma(S[i * c + l], x[l], acc);
            x[i] = -acc / S[i * c + i];
        }
    }
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
    const bool gj = size_t(2) * c * c * sizeof(T) <= 200 * 1024;
    const size_t smem = size_t(gj ? 2 : 1) * c * c * sizeof(T);
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(chol_inv_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    chol_inv_kernel<T><<<1, 256, smem, ex.stream>>>(gram, c, rfac, ex.status, shifted_flag, gj);
    ex.launches++;
    GemmDesc ga{};   // dst^T = P src^T: row a of dst = sum_b P[a][b] row b of src
    ga.M = c; ga.N = len; ga.K = c;
    ga.X = rfac; ga.ldx = c; ga.Y = src; ga.ldy = ld;
    ga.y_kmajor = false; ga.y_dtype = sizeof(T) == 8 ? 0 : 1;
    ga.out = dst; ga.ldo = ld; ga.out_transposed = false;
    ga.alpha = 1.0; ga.beta = 0.0;
    gemm_simt<T>(ex, ga, partials, cap);
}

}  // namespace

// W (c x ld) against Qb (m x ld): BCGS2 then CholeskyQR2, result in Qout (Qout != W).
// Wtmp holds the first CholeskyQR iterate; `ct` (c x m, type T) the projection
// coefficients; `rfac` (c x c) the inverse Cholesky factor.
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

template <typename T>
void cholqr_extra(Exec& ex, int64_t len, int64_t ld, T* Q, int c, double* partials, int64_t cap,
                  double* gram, T* rfac, int* shifted_flag, T* tmp) {
    cholqr_pass<T>(ex, len, ld, Q, c, tmp, partials, cap, gram, rfac, shifted_flag);
    cudaMemcpyAsync(Q, tmp, size_t(c) * ld * sizeof(T), cudaMemcpyDeviceToDevice, ex.stream);
}

#define BKS_INST(T)                                                                          \
    template void orth_block<T>(Exec&, int64_t, int64_t, const T*, int, T*, int, T*, T*,     \
                                double*, int64_t, double*, T*, T*, int*);                    \
    template void cholqr_extra<T>(Exec&, int64_t, int64_t, T*, int, double*, int64_t,        \
                                  double*, T*, int*, T*);
BKS_INST(float)
BKS_INST(double)
#undef BKS_INST

}  // namespace bks
