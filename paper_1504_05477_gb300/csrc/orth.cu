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

// G (c x c, row pitch ldg, symmetric) -> P = R^{-T} (c x c, row pitch ldp), where
// G = R^T R with R upper triangular; Q = W R^{-1} is then Q^T = P W^T.  One CTA.
template <typename T>
__global__ void chol_inv_kernel(const T* __restrict__ G, int64_t ldg, int c, T* __restrict__ P,
                                int64_t ldp, int* status, int* shifted_flag, bool gauss_jordan) {
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
        const int a = e / c, b = e - a * c;
        const double g = double(G[a * ldg + b]);
        bad |= !isfinite(g);
        if (a == b) tr += g;
        S[e] = (a <= b) ? T(g) : T(0);
    }
    if (__syncthreads_or(bad)) {
        if (tid == 0) atomicOr(status, ST_NONFINITE);
        for (int e = tid; e < c * c; e += nt) P[(e / c) * ldp + e % c] = T((e / c == e % c) ? 1.0 : 0.0);
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
                S[e] = (a <= b) ? T(double(G[a * ldg + b]) + (a == b ? shift : 0.0)) : T(0);
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
        for (int e = tid; e < c * c; e += nt) P[(e / c) * ldp + e % c] = T((e / c == e % c) ? 1.0 : 0.0);
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
            P[a * ldp + b] = Ri[b * c + a];   // P = R^{-T}
        }
        return;
    }
    // (wide FP64 blocks) R^{-1} column by column: thread j solves R x = e_j by back
    // substitution and keeps x in row j of P = R^{-T} (only thread j touches that row)
    for (int j = tid; j < c; j += nt) {
        T* x = P + int64_t(j) * ldp;
        for (int i = j + 1; i < c; ++i) x[i] = T(0);
        x[j] = T(1) / S[j * c + j];
        for (int i = j - 1; i >= 0; --i) {
            T acc = T(0);
            for (int l = i + 1; l <= j; ++l) acc = fma(S[i * c + l], x[l], acc);
            x[i] = -acc / S[i * c + i];
        }
    }
}

// P = L^{-1} = R^{-T} for G = L L^T (c <= 128) by symmetric elimination on [G | I]
// with the elimination rows kept in registers: each thread owns a 4 x 4 tile of the
// trailing matrix S and of the lower-triangular E.  Step j publishes row j of S and E
// (double-buffered, one barrier per step) and every thread updates its tiles:
//   S[i][l] -= (S[i][j] / d_j) S[j][l],  E[i][l] -= (S[i][j] / d_j) E[j][l]   (i > j)
// with the pivot d_j = S[j][j].  At the end E = L_unit^{-1} for G = L_unit D L_unit^T,
// so L^{-1} = D^{-1/2} E.  Same breakdown handling as chol_inv_kernel.
constexpr int TR = 4, TC = 8;   // register tile: rows x columns per thread (c <= 128: 512 threads)
__global__ void __launch_bounds__(512) chol_inv_tiled_kernel(const float* __restrict__ G, int64_t ldg, int c,
                                                             float* __restrict__ P, int64_t ldp, int* status,
                                                             int* shifted_flag) {
    __shared__ float rowS[2][128], rowE[2][128];
    __shared__ double trace_s;
    const int ntc = (c + TC - 1) / TC, ntr = (c + TR - 1) / TR;
    const int tid = threadIdx.x;
    const bool active = tid < ntr * ntc;
    const int ti = active ? tid / ntc : 0, tj = active ? tid % ntc : 0;
    const int r0 = ti * TR, c0 = tj * TC;
    if (tid == 0) trace_s = 0.0;
    __syncthreads();
    bool nonfin = false;
    for (int a = 0; a < TR; ++a)
        for (int b = 0; b < TC; ++b) {
            const int i = r0 + a, l = c0 + b;
            if (!active || i >= c || l >= c) continue;
            const float g = G[int64_t(i) * ldg + l];
            nonfin |= !isfinite(g);
            if (i == l) atomicAdd(&trace_s, double(g));
        }
    if (__syncthreads_or(nonfin)) {
        if (tid == 0) atomicOr(status, ST_NONFINITE);
        for (int q = tid; q < c * c; q += blockDim.x) P[(q / c) * ldp + q % c] = (q / c == q % c) ? 1.f : 0.f;
        return;
    }
    double shift = 0.0;
    float s[TR][TC], e[TR][TC], dpiv[TR];
    bool ok = false;
    for (int attempt = 0; attempt < 6 && !ok; ++attempt) {
#pragma unroll
        for (int a = 0; a < TR; ++a) {
            dpiv[a] = 1.f;
#pragma unroll
            for (int b = 0; b < TC; ++b) {
                const int i = r0 + a, l = c0 + b;
                const float g = (active && i < c && l < c) ? G[int64_t(i) * ldg + l] : 0.f;
                s[a][b] = g + ((i == l) ? float(shift) : 0.f);
                e[a][b] = (i == l) ? 1.f : 0.f;
            }
        }
        ok = true;
        for (int j = 0; j < c; ++j) {
            const int par = j & 1;
            if (active && ti == j / TR) {
                const int a = j % TR;
#pragma unroll
                for (int aa = 0; aa < TR; ++aa)
                    if (aa == a) {
#pragma unroll
                        for (int b = 0; b < TC; ++b) {
                            rowS[par][c0 + b] = s[aa][b];
                            rowE[par][c0 + b] = e[aa][b];
                        }
                    }
            }
            __syncthreads();
            const float d = rowS[par][j];
            if (!(d > 0.f) || !isfinite(d)) {   // uniform: every thread reads the same value
                ok = false;
                break;
            }
            if (!active || r0 + TR - 1 < j) continue;   // rows of this tile are all done
            const float inv = 1.f / d;
#pragma unroll
            for (int a = 0; a < TR; ++a) {
                const int i = r0 + a;
                if (i == j) dpiv[a] = d;
                if (i <= j) continue;
                const float f = rowS[par][i] * inv;   // S[i][j] = S[j][i]
#pragma unroll
                for (int b = 0; b < TC; ++b) {
                    const int l = c0 + b;
                    if (l > j) s[a][b] = fmaf(-f, rowS[par][l], s[a][b]);
                    else e[a][b] = fmaf(-f, rowE[par][l], e[a][b]);
                }
            }
        }
        __syncthreads();
        if (!ok) {
            shift = (shift == 0.0) ? 1e-6 * trace_s / c : shift * 1e3;
            if (tid == 0) atomicOr(shifted_flag, 1);
        }
    }
    if (!ok) {
        if (tid == 0) atomicOr(status, ST_BREAKDOWN);
        for (int q = tid; q < c * c; q += blockDim.x) P[(q / c) * ldp + q % c] = (q / c == q % c) ? 1.f : 0.f;
        return;
    }
    if (shift > 0.0 && tid == 0) atomicOr(status, ST_SHIFTED);
    if (!active) return;
#pragma unroll
    for (int a = 0; a < TR; ++a) {
        const int i = r0 + a;
        if (i >= c) continue;
        const float sc = 1.f / sqrtf(dpiv[a]);
#pragma unroll
        for (int b = 0; b < TC; ++b) {
            const int l = c0 + b;
            if (l < c) P[int64_t(i) * ldp + l] = (l <= i) ? e[a][b] * sc : 0.f;
        }
    }
}

// Thin-block product through the tensor cores when T = float and the operands meet the
// TMA rules, else the SIMT kernel.  A: rows x len thin (pitch lda); X: c x (len or rows).
//   trans = false: Y (c x rows)  = (A X^T)^T,  Y[j][r] = sum_l A[r][l] X[j][l]
//   trans = true:  Y (c x len) (-)= (A^T X^T)^T, Y[j][l] = sum_r A[r][l] X[j][r]
template <typename T>
void thin_mm(Exec& ex, const T* A, int64_t rows, int64_t len, int64_t lda, bool trans, int c, const T* X,
             int64_t ldx, T* Y, int64_t ldy, bool subtract, const OrthWs& ws) {
    if (sizeof(T) == 4 && ws.xh != nullptr) {
        KernelLog* log = ex.klog;   // the kernel log times products with A only
        ex.klog = nullptr;
        const bool done = tc_product_f32(ex, reinterpret_cast<const float*>(A), rows, len, lda, trans, c,
                                         reinterpret_cast<const float*>(X), ldx, reinterpret_cast<float*>(Y),
                                         ldy, ws.xh, ws.xl, ws.tpart, ws.tpart_cap, subtract);
        ex.klog = log;
        if (done) return;
    }
    GemmDesc g{};
    g.M = c;
    g.N = trans ? len : rows;
    g.K = trans ? rows : len;
    g.X = X; g.ldx = ldx;
    g.Y = A; g.ldy = lda;
    g.y_kmajor = !trans;
    g.y_dtype = sizeof(T) == 8 ? 0 : 1;
    g.out = Y; g.ldo = ldy; g.out_transposed = false;
    g.alpha = subtract ? -1.0 : 1.0;
    g.beta = subtract ? 1.0 : 0.0;
    gemm_simt<T>(ex, g, ws.partials, ws.cap);
}

template <typename T>
void cholqr_pass(Exec& ex, int64_t len, int64_t ld, const T* src, int c, T* dst, const OrthWs& ws) {
    T* G = static_cast<T*>(ws.g);
    T* P = static_cast<T*>(ws.rfac);
    thin_mm<T>(ex, src, c, len, ld, false, c, src, ld, G, ws.ldp, false, ws);   // G = W^T W
    if (sizeof(T) == 4 && c <= 128) {
        const int nthreads = ((c + TR - 1) / TR) * ((c + TC - 1) / TC);
        chol_inv_tiled_kernel<<<1, (nthreads + 31) / 32 * 32, 0, ex.stream>>>(
            reinterpret_cast<const float*>(G), ws.ldp, c, reinterpret_cast<float*>(P), ws.ldp, ex.status,
            ws.shifted_flag);
    } else {
        const bool gj = size_t(2) * c * c * sizeof(T) <= 200 * 1024;
        const size_t smem = size_t(gj ? 2 : 1) * c * c * sizeof(T);
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(chol_inv_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        chol_inv_kernel<T><<<1, 256, smem, ex.stream>>>(G, ws.ldp, c, P, ws.ldp, ex.status, ws.shifted_flag, gj);
    }
    ex.launches++;
    thin_mm<T>(ex, src, c, len, ld, true, c, P, ws.ldp, dst, ld, false, ws);    // dst = (W R^{-1})^T
}

}  // namespace

// W (c x ld) against Qb (m x ld): BCGS2 then CholeskyQR2, result in Qout (Qout may be W).
template <typename T>
void orth_block(Exec& ex, int64_t len, int64_t ld, const T* Qb, int m, T* W, int c, T* Wtmp, T* Qout,
                const OrthWs& ws) {
    if (m > 0) {
        T* ct = static_cast<T*>(ws.ct);
        for (int pass = 0; pass < 2; ++pass) {
            thin_mm<T>(ex, Qb, m, len, ld, false, c, W, ld, ct, ws.ldc, false, ws);   // ct = (Q^T W)^T
            thin_mm<T>(ex, Qb, m, len, ld, true, c, ct, ws.ldc, W, ld, true, ws);     // W -= Q ct^T
        }
    }
    cholqr_pass<T>(ex, len, ld, W, c, Wtmp, ws);
    cholqr_pass<T>(ex, len, ld, Wtmp, c, Qout, ws);
}

OrthSizes orth_sizes(int64_t len_max, int64_t ld_max, int mmax, int c, int elem_bytes, bool tc,
                     int num_sms) {
    OrthSizes z{};
    const int64_t mm = mmax > 0 ? mmax : 1;
    z.ldp = int(round_up(c, 32));
    z.ldc = round_up(mm, 32);
    z.cap = int64_t(c) * c;
    for (int64_t e : {gemm_partial_elems(c, mm, len_max, num_sms), gemm_partial_elems(c, len_max, mm, num_sms),
                      gemm_partial_elems(c, c, len_max, num_sms), gemm_partial_elems(c, len_max, c, num_sms)})
        if (e > z.cap) z.cap = e;
    z.partials = size_t(z.cap) * sizeof(double);
    z.g = size_t(c) * z.ldp * elem_bytes;
    z.rfac = z.g;
    z.ct = size_t(c) * z.ldc * elem_bytes;
    if (tc) {
        const int64_t cp = round_up(c < 128 ? c : 128, 32);
        const int64_t big = len_max > mm ? len_max : mm;
        const int64_t tiles = (big + 127) / 128;
        z.tcap = int64_t(num_sms) * ((tiles + num_sms - 1) / num_sms + 3) * cp * 128;
        z.xh = size_t(c) * ld_max * 4;
        z.tpart = size_t(z.tcap) * 4;
    }
    return z;
}

#define BKS_INST(T)                                                                                 \
    template void orth_block<T>(Exec&, int64_t, int64_t, const T*, int, T*, int, T*, T*, const OrthWs&);
BKS_INST(float)
BKS_INST(double)
#undef BKS_INST

}  // namespace bks
