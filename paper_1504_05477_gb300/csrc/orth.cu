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
#include <mutex>

#include "common.cuh"
#include "chol_small.cuh"

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

__global__ void __launch_bounds__(512) chol_inv_tiled_kernel(const float* __restrict__ G, int64_t ldg, int c,
                                                             float* __restrict__ P, int64_t ldp, int* status,
                                                             int* shifted_flag) {
    chol_inv_block(G, ldg, c, P, ldp, status, shifted_flag);
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
        const int n4 = (c + TR - 1) / TR;   // 4 x 4 tiles when they fit in 512 threads, else 4 x 8
        const int nthreads = n4 * n4 <= 512 ? n4 * n4 : n4 * ((c + 7) / 8);
        chol_inv_tiled_kernel<<<1, (nthreads + 31) / 32 * 32, 0, ex.stream>>>(
            reinterpret_cast<const float*>(G), ws.ldp, c, reinterpret_cast<float*>(P), ws.ldp, ex.status,
            ws.shifted_flag);
    } else {
        const bool gj = size_t(2) * c * c * sizeof(T) <= 200 * 1024;
        const size_t smem = size_t(gj ? 2 : 1) * c * c * sizeof(T);
        if (smem > 48 * 1024) allow_dynamic_smem(reinterpret_cast<const void*>(chol_inv_kernel<T>), smem);
        chol_inv_kernel<T><<<1, 256, smem, ex.stream>>>(G, ws.ldp, c, P, ws.ldp, ex.status, ws.shifted_flag, gj);
    }
    ex.launches++;
    thin_mm<T>(ex, src, c, len, ld, true, c, P, ws.ldp, dst, ld, false, ws);    // dst = (W R^{-1})^T
}


// ------------------------------------------------------------------ fused orthonormalisation
// The whole of orth_block for one block in one cooperative launch (FP32; c <= 64,
// m + c <= 512).  CTA g owns rows [l0, l1) of the tall matrices and streams them through
// shared memory in chunks of LC; Grams are reduced across CTAs in a fixed order between
// grid barriers, and the small c x c factorisations are repeated by every CTA.
//   P1  C1 = Q^T W                                    (projection coefficients)
//   P2  W' = W - Q C1,  [C2; H] = [Q W']^T W'          (second projection, fused Gram)
//   P3  R1 = chol(H - C2^T C2)  (Pythagorean: the Gram of W' - Q C2),
//       W1 = (W' - Q C2) R1^{-1} = [Q W'] [-C2 R1^{-1}; R1^{-1}],  H3 = W1^T W1
//   P4  Qout = W1 chol(H3)^{-1}
// i.e. BCGS2 followed by CholeskyQR2, with the second projection and the first
// Cholesky sharing one Gram pass.
namespace of {

constexpr int NT = 256;
constexpr int LC = 32;           // rows of the tall matrices per chunk (= lanes of the apply)
constexpr int LCP = LC + 1;      // padded shared row
constexpr int NB = 2;            // chunk stages (cp.async double buffering)
constexpr int RMAX = 512;
constexpr int CMAX = 64;
constexpr int SLOTS = 8;
constexpr int MAXG = 160;
constexpr uint64_t WAIT_NS = 1000000000ull;
constexpr int MAX_DYN_FLOATS = 56 * 1024;   // 224 KB of dynamic shared memory at most

struct Args {
    const float* Q;
    float* W;
    float* Wtmp;
    float* Qout;
    int m, c;
    int64_t len, ld;
    float* part;      // grid x round_up((m + c) c, 4)
    float* gram;      // (m + c) x c
    unsigned* bar;    // [0] arrivals, [1] abort
    int* status;
    int* shifted_flag;
};

__host__ __device__ inline int r4(int x) { return (x + 3) & ~3; }

// Shared layout (floats).  The small factorisation buffers and the reduction scratch
// alias the chunk stages: they are used only outside the chunk loops.
// Column tile of the Gram (compile-time): 32 for c > 32, else c rounded up to 8.
__host__ __device__ inline int tile_j(int c) { return c > 32 ? 32 : (c + 7) / 8 * 8; }
// Zero rows after the real ones, so the column tiles and the 4-row groups run unguarded.
__host__ __device__ inline int pad_rows(int c) {
    const int tj = tile_j(c), nj = (c + tj - 1) / tj, p = nj * tj - c;
    return p > 4 ? p : 4;
}
struct Layout {
    int coef, ach, wout, hbuf, pbuf, red, total, stage, pad;
    __host__ __device__ Layout(int m, int c) {
        const int R = m + c;
        pad = pad_rows(c);
        stage = r4((R + pad) * LCP);
        coef = 0;
        ach = r4(R * r4(c));
        // scratch used outside the chunk loops, aliasing the stages
        hbuf = ach;
        pbuf = hbuf + r4(c * c);
        red = ach;                 // SLOTS x 32 x 4 doubles = 2048 floats
        int scratch_end = pbuf + r4(c * c);
        if (red + 2 * SLOTS * 32 * 4 > scratch_end) scratch_end = red + 2 * SLOTS * 32 * 4;
        wout = ach + NB * stage;
        if (scratch_end > wout) wout = scratch_end;
        total = wout + r4((c + pad) * LCP);
    }
};

__device__ __forceinline__ uint64_t gtime() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier (all CTAs are co-resident: cooperative launch).  Bounded: after 1 s
// the CTA flags ST_TIMEOUT and raises the abort word, which releases the others.
__device__ bool grid_sync(unsigned* bar, unsigned target, int* status) {
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(&bar[0], 1u);
        const uint64_t t0 = gtime();
        int ok = 1;
        while (*reinterpret_cast<volatile unsigned*>(&bar[0]) < target) {
            if (*reinterpret_cast<volatile unsigned*>(&bar[1])) { ok = 0; break; }
            if (gtime() - t0 > WAIT_NS) {
                atomicOr(status, ST_TIMEOUT);
                atomicExch(&bar[1], 1u);
                ok = 0;
                break;
            }
        }
        __threadfence();
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Stage rows [0, n1) of src1 and [0, n2) of src2 (pitch ld), columns [lb, lb + LC) clipped
// to l1, into dst rows 0.. and n1.. (zeros past l1).
__device__ __forceinline__ void issue_rows(float* dst, const float* src1, int n1, const float* src2, int n2,
                                           int64_t ld, int64_t lb, int64_t l1) {
    const int n = n1 + n2;
    for (int e = threadIdx.x; e < n * LC; e += NT) {
        const int r = e / LC, l = e % LC;
        float* d = dst + r * LCP + l;
        if (lb + l < l1) {
            const float* src = r < n1 ? src1 + int64_t(r) * ld : src2 + int64_t(r - n1) * ld;
            cp_async4(d, src + lb + l);
        } else {
            *d = 0.f;
        }
    }
    cp_commit();
}

// for every chunk of [l0, l1): stage it, then body(stage pointer, lb) (double-buffered)
template <class Body>
__device__ __forceinline__ void stream_chunks(float* stages, int stage, const float* src1, int n1,
                                              const float* src2, int n2, int64_t ld, int64_t l0, int64_t l1,
                                              Body body) {
    if (l0 >= l1) return;
    issue_rows(stages, src1, n1, src2, n2, ld, l0, l1);
    int k = 0;
    for (int64_t lb = l0; lb < l1; lb += LC, ++k) {
        if (lb + LC < l1) {
            issue_rows(stages + ((k + 1) % NB) * stage, src1, n1, src2, n2, ld, lb + LC, l1);
            cp_wait<1>();
        } else {
            cp_wait<0>();
        }
        __syncthreads();
        body(stages + (k % NB) * stage, lb);
        __syncthreads();
    }
}

__device__ __forceinline__ void store_rows(float* dst, const float* src, int nrows, int64_t ld, int64_t lb,
                                           int64_t l1) {
    for (int e = threadIdx.x; e < nrows * LC; e += NT) {
        const int r = e / LC, l = e % LC;
        if (lb + l < l1) dst[int64_t(r) * ld + lb + l] = src[r * LCP + l];
    }
}

// Gram of Ra rows of A against c rows of B over a chunk.  Thread t: tile t / LS (rows
// rg, rg + RS, rg + 2 RS, rg + 3 RS; columns j0 .. j0 + TJ - 1), chunk rows l = lsub,
// lsub + LS, ...; the LS partial tiles are combined by shuffles at the end.  Rows past
// Ra and columns past c read zero padding or rows whose results are discarded.
// Consecutive tiles take consecutive rg with the same j0, so a warp's loads of B are one
// broadcast address and its loads of A hit distinct banks.
template <int TJ>
struct GramMap {
    int RS, LS, rg, j0, lsub;
    bool on;
    __device__ GramMap(int Ra, int c) {
        const int nj = (c + TJ - 1) / TJ;
        RS = (Ra + 3) / 4;
        const int tiles = RS * nj;
        LS = 1;
        while (LS < 32 && tiles * LS * 2 <= NT) LS *= 2;
        const int t = threadIdx.x / LS;
        lsub = threadIdx.x % LS;
        on = t < tiles;
        rg = t % RS;
        j0 = (t / RS) * TJ;
    }
};

template <int TJ>
__device__ __forceinline__ void gram_acc(float (&acc)[4][TJ], const GramMap<TJ>& g, const float* A,
                                         const float* B) {
    if (!g.on) return;
    const float* a0 = A + g.rg * LCP;
    const float* b0 = B + g.j0 * LCP;
    const int rs = g.RS * LCP;
    for (int l = g.lsub; l < LC; l += g.LS) {
        float a[4], b[TJ];
#pragma unroll
        for (int k = 0; k < 4; ++k) a[k] = a0[k * rs + l];
#pragma unroll
        for (int jj = 0; jj < TJ; ++jj) b[jj] = b0[jj * LCP + l];
#pragma unroll
        for (int jj = 0; jj < TJ; ++jj)
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[k][jj] = fmaf(a[k], b[jj], acc[k][jj]);
    }
}

template <int TJ>
__device__ __forceinline__ void gram_write(float (&acc)[4][TJ], const GramMap<TJ>& g, float* dst, int Ra,
                                           int c) {
    for (int off = g.LS / 2; off > 0; off >>= 1) {   // lanes of one tile are adjacent
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
            for (int jj = 0; jj < TJ; ++jj) acc[k][jj] += __shfl_xor_sync(0xffffffffu, acc[k][jj], off);
    }
    if (!g.on || g.lsub != 0) return;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int r = g.rg + k * g.RS;
        if (r >= Ra) continue;
#pragma unroll
        for (int jj = 0; jj < TJ; ++jj)
            if (g.j0 + jj < c) dst[r * c + g.j0 + jj] = acc[k][jj];
    }
}

// out[e] = sum over CTAs g (in order) of part[g * ep + e], e < n: this CTA's stripe.
__device__ void reduce_stripe(const float* part, int G, int n, float* out, double* red) {
    const int ep = r4(n), nq = ep / 4;
    const int q0 = int(int64_t(blockIdx.x) * nq / G), q1 = int(int64_t(blockIdx.x + 1) * nq / G);
    const int lane = threadIdx.x & 31, slot = threadIdx.x >> 5;
    for (int qb = q0; qb < q1; qb += 32) {
        const int q = qb + lane;
        double s0 = 0, s1 = 0, s2 = 0, s3 = 0;
        if (q < q1) {
            float4 v[MAXG / SLOTS];
#pragma unroll
            for (int i = 0; i < MAXG / SLOTS; ++i) {
                const int g = slot + i * SLOTS;
                v[i] = g < G ? __ldcg(reinterpret_cast<const float4*>(part + int64_t(g) * ep) + q)
                             : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int i = 0; i < MAXG / SLOTS; ++i) {
                s0 += v[i].x; s1 += v[i].y; s2 += v[i].z; s3 += v[i].w;
            }
        }
        double* rr = red + (slot * 32 + lane) * 4;
        rr[0] = s0; rr[1] = s1; rr[2] = s2; rr[3] = s3;
        __syncthreads();
        if (slot == 0 && q < q1) {
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                double v = red[lane * 4 + t];
                for (int k = 1; k < SLOTS; ++k) v += red[(k * 32 + lane) * 4 + t];
                if (4 * q + t < n) out[4 * q + t] = float(v);
            }
        }
        __syncthreads();
    }
}

// wout[j][l] = (subtract ? base[j][l] : 0) -+ sum_{r < Ra} coef[r][j] A[r][l]
// (warp w: columns w JW .. w JW + JW - 1, lane = l).
__device__ __forceinline__ void apply_chunk(float* wout, const float* coef, int cs, const float* A, int Ra,
                                            const float* base, int c, bool subtract) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int JW = r4((c + 7) / 8);
    const int j0 = w * JW;
    if (j0 >= c) return;
    float acc[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) acc[t] = 0.f;
#pragma unroll 4
    for (int r = 0; r < Ra; ++r) {
        const float a = A[r * LCP + lane];
        const float4 c0 = *reinterpret_cast<const float4*>(coef + r * cs + j0);
        acc[0] = fmaf(c0.x, a, acc[0]);
        acc[1] = fmaf(c0.y, a, acc[1]);
        acc[2] = fmaf(c0.z, a, acc[2]);
        acc[3] = fmaf(c0.w, a, acc[3]);
        if (JW == 8) {
            const float4 c1 = *reinterpret_cast<const float4*>(coef + r * cs + j0 + 4);
            acc[4] = fmaf(c1.x, a, acc[4]);
            acc[5] = fmaf(c1.y, a, acc[5]);
            acc[6] = fmaf(c1.z, a, acc[6]);
            acc[7] = fmaf(c1.w, a, acc[7]);
        }
    }
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        const int j = j0 + t;
        if (t < JW && j < c)
            wout[j * LCP + lane] = subtract ? base[j * LCP + lane] - acc[t] : acc[t];
    }
}

template <int TJ>
__global__ void __launch_bounds__(NT, 1) orth_fused_kernel(Args a) {
    extern __shared__ float4 sm4[];
    float* sm = reinterpret_cast<float*>(sm4);
    const int m = a.m, c = a.c, R = m + c, cs = r4(c);
    const Layout L(m, c);
    float* coef = sm + L.coef;
    float* ach = sm + L.ach;
    float* wout = sm + L.wout;
    float* hbuf = sm + L.hbuf;
    float* pbuf = sm + L.pbuf;
    double* red = reinterpret_cast<double*>(sm + L.red);
    const int G = gridDim.x, cta = blockIdx.x, tid = threadIdx.x;
    const int64_t l0 = int64_t(cta) * a.len / G, l1 = int64_t(cta + 1) * a.len / G;
    unsigned phase = 0;
    float acc[4][TJ];
    auto zero = [&]() {
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
            for (int jj = 0; jj < TJ; ++jj) acc[k][jj] = 0.f;
    };
    // zero padding rows of the chunk stages and of wout (never written afterwards)
    for (int s2 = 0; s2 < NB; ++s2)
        for (int e = tid; e < L.pad * LCP; e += NT) ach[s2 * L.stage + R * LCP + e] = 0.f;
    for (int e = tid; e < L.pad * LCP; e += NT) wout[c * LCP + e] = 0.f;
    // partial Gram -> ordered cross-CTA sum in a.gram (two grid barriers)
    auto reduce = [&](const GramMap<TJ>& gm, int Ra) -> bool {
        gram_write(acc, gm, a.part + int64_t(cta) * r4(Ra * c), Ra, c);
        if (!grid_sync(a.bar, ++phase * G, a.status)) return false;
        reduce_stripe(a.part, G, Ra * c, a.gram, red);
        return grid_sync(a.bar, ++phase * G, a.status);
    };

    // ---- P1: C1 = Q^T W
    if (m > 0) {
        const GramMap<TJ> gm(m, c);
        zero();
        stream_chunks(ach, L.stage, a.Q, m, a.W, c, a.ld, l0, l1, [&](float* st, int64_t) {
            gram_acc<TJ>(acc, gm, st, st + m * LCP);
        });
        if (!reduce(gm, m)) return;
        for (int e = tid; e < m * c; e += NT) coef[(e / c) * cs + e % c] = __ldcg(a.gram + e);
        __syncthreads();
    }
    // ---- P2: W' = W - Q C1 (written back to W), Gram [Q W']^T W'
    {
        const GramMap<TJ> gm(R, c);
        zero();
        stream_chunks(ach, L.stage, a.Q, m, a.W, c, a.ld, l0, l1, [&](float* st, int64_t lb) {
            if (m > 0) {
                apply_chunk(wout, coef, cs, st, m, st + m * LCP, c, true);
                __syncthreads();
                for (int e = tid; e < c * LC; e += NT)
                    st[(m + e / LC) * LCP + e % LC] = wout[(e / LC) * LCP + e % LC];
                store_rows(a.W, wout, c, a.ld, lb, l1);
                __syncthreads();
            }
            gram_acc<TJ>(acc, gm, st, st + m * LCP);
        });
        if (!reduce(gm, R)) return;
    }
    // ---- P3: R1 from H - C2^T C2, P1 = R1^{-T}; W1 = (W' - Q C2) P1^T with its Gram
    for (int e = tid; e < R * c; e += NT) coef[(e / c) * cs + e % c] = __ldcg(a.gram + e);
    __syncthreads();
    {   // H - C2^T C2: 4 x 4 register tiles of the upper triangle (mirrored), each tile's
        // rows r of C2 split between S adjacent lanes and combined by shuffles
        const int nt4 = (c + 3) / 4, ntri = nt4 * (nt4 + 1) / 2;
        int S = 1;
        while (S < 8 && ntri * S * 2 <= NT) S *= 2;
        const int t = tid / S, sr = tid % S;
        int ti = 0, rem = t;
        while (ti < nt4 && rem >= nt4 - ti) {
            rem -= nt4 - ti;
            ++ti;
        }
        const bool on = t < ntri;
        const int i0 = ti * 4, j0 = (ti + rem) * 4;
        float h[4][4];
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
            for (int y = 0; y < 4; ++y) h[x][y] = 0.f;
        if (on) {
#pragma unroll 4
            for (int r = sr; r < m; r += S) {
                const float4 u = *reinterpret_cast<const float4*>(coef + r * cs + i0);
                const float4 v = *reinterpret_cast<const float4*>(coef + r * cs + j0);
                const float uu[4] = {u.x, u.y, u.z, u.w}, vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int x = 0; x < 4; ++x)
#pragma unroll
                    for (int y = 0; y < 4; ++y) h[x][y] = fmaf(uu[x], vv[y], h[x][y]);
            }
        }
        for (int off = 1; off < S; off <<= 1)   // the S lanes of a tile are adjacent
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y) h[x][y] += __shfl_xor_sync(0xffffffffu, h[x][y], off);
        if (on && sr == 0) {
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y) {
                    const int i = i0 + x, j = j0 + y;
                    if (i < c && j < c && i <= j) {
                        const float v = coef[(m + i) * cs + j] - h[x][y];
                        hbuf[i * c + j] = v;
                        hbuf[j * c + i] = v;
                    }
                }
        }
    }
    __syncthreads();
    chol_inv_block_t<4>(hbuf, c, c, pbuf, c, a.status, a.shifted_flag);   // c <= 64 on 256 threads
    __syncthreads();
    // rows m .. m + c - 1 of coef (H, no longer needed) take P1^T; rows 0 .. m - 1 keep C2
    for (int e = tid; e < c * c; e += NT) {
        const int b = e / c, j = e % c;
        coef[(m + b) * cs + j] = pbuf[j * c + b];
    }
    __syncthreads();
    {
        const GramMap<TJ> gm(c, c);
        zero();
        stream_chunks(ach, L.stage, a.Q, m, a.W, c, a.ld, l0, l1, [&](float* st, int64_t lb) {
            float* wrows = st + m * LCP;
            if (m > 0) {   // W' - Q C2, written over the chunk's W' rows
                apply_chunk(wout, coef, cs, st, m, wrows, c, true);
                __syncthreads();
                for (int e = tid; e < c * LC; e += NT)
                    wrows[(e / LC) * LCP + e % LC] = wout[(e / LC) * LCP + e % LC];
                __syncthreads();
            }
            apply_chunk(wout, coef + m * cs, cs, wrows, c, nullptr, c, false);
            __syncthreads();
            store_rows(a.Wtmp, wout, c, a.ld, lb, l1);
            gram_acc<TJ>(acc, gm, wout, wout);
        });
        if (!reduce(gm, c)) return;
    }
    // ---- P4: Qout = P2 W1, P2 = chol(H3)^{-T}
    for (int e = tid; e < c * c; e += NT) hbuf[e] = __ldcg(a.gram + e);
    __syncthreads();
    chol_inv_block_t<4>(hbuf, c, c, pbuf, c, a.status, a.shifted_flag);   // c <= 64 on 256 threads
    __syncthreads();
    for (int e = tid; e < c * c; e += NT) {
        const int b = e / c, j = e % c;
        coef[b * cs + j] = pbuf[j * c + b];
    }
    __syncthreads();
    stream_chunks(ach, L.stage, a.Wtmp, c, a.Wtmp, 0, a.ld, l0, l1, [&](float* st, int64_t lb) {
        apply_chunk(wout, coef, cs, st, c, nullptr, c, false);
        __syncthreads();
        store_rows(a.Qout, wout, c, a.ld, lb, l1);
    });
}

}  // namespace of

bool orth_fused_fits(int m, int c) {
    return c >= 1 && c <= of::CMAX && m + c <= of::RMAX && of::Layout(m, c).total <= of::MAX_DYN_FLOATS;
}

// One cooperative launch; false (nothing launched) when it cannot run.
bool orth_fused(Exec& ex, int64_t len, int64_t ld, const float* Qb, int m, float* W, int c, float* Wtmp,
                float* Qout, const OrthWs& ws) {
    if (ws.fpart == nullptr || !orth_fused_fits(m, c)) return false;
    const of::Layout L(m, c);
    const size_t smem = size_t(L.total) * sizeof(float);
    if (L.total > of::MAX_DYN_FLOATS) return false;
    const int tj = of::tile_j(c);
    void* fn = tj == 8    ? reinterpret_cast<void*>(of::orth_fused_kernel<8>)
               : tj == 16 ? reinterpret_cast<void*>(of::orth_fused_kernel<16>)
               : tj == 24 ? reinterpret_cast<void*>(of::orth_fused_kernel<24>)
                          : reinterpret_cast<void*>(of::orth_fused_kernel<32>);
    static std::mutex mu;   // host threads of a batch may get here together
    static int configured_device[4] = {-1, -1, -1, -1};
    static int per_sm[4] = {0, 0, 0, 0};
    const int ti = tj / 8 - 1;
    int dev = 0;
    cudaGetDevice(&dev);
    int resident = 0;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (configured_device[ti] != dev) {
            if (allow_dynamic_smem(fn, of::MAX_DYN_FLOATS * sizeof(float)) != cudaSuccess ||
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[ti], fn, of::NT,
                                                              of::MAX_DYN_FLOATS * sizeof(float)) != cudaSuccess) {
                cudaGetLastError();
                return false;
            }
            configured_device[ti] = dev;
        }
        resident = per_sm[ti];
    }
    // about 64 rows per CTA: a short block takes only a few SMs (other streams keep the rest)
    int G = ex.num_sms < of::MAXG ? ex.num_sms : of::MAXG;
    const int64_t want = (len + 63) / 64;
    if (want < G) G = int(want < 1 ? 1 : want);
    if (resident < 1 || int64_t(G) * of::r4((m + c) * c) > ws.fpart_cap) return false;
    of::Args a;
    a.Q = Qb; a.W = W; a.Wtmp = Wtmp; a.Qout = Qout;
    a.m = m; a.c = c; a.len = len; a.ld = ld;
    a.part = ws.fpart; a.gram = ws.fgram; a.bar = ws.fbar;
    a.status = ex.status; a.shifted_flag = ws.shifted_flag;
    cudaMemsetAsync(ws.fbar, 0, 2 * sizeof(unsigned), ex.stream);
    void* args[] = {&a};
    if (cudaLaunchCooperativeKernel(fn, dim3(G), dim3(of::NT), args, smem, ex.stream) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    ex.launches++;
    return true;
}

}  // namespace

// W (c x ld) against Qb (m x ld): BCGS2 then CholeskyQR2, result in Qout (Qout may be W).
template <typename T>
void orth_block(Exec& ex, int64_t len, int64_t ld, const T* Qb, int m, T* W, int c, T* Wtmp, T* Qout,
                const OrthWs& ws) {
    if (ws.tc_used) *ws.tc_used = false;
    if (sizeof(T) == 4 && ws.otc_part != nullptr && (m == 0 || ws.qr != nullptr) &&
        orth_tc(ex, len, ld, reinterpret_cast<const float*>(Qb), m, reinterpret_cast<const float*>(W), c,
                reinterpret_cast<float*>(Qout), ws.qr, ws.qr_append ? ws.qr + m : nullptr, ws.ldr, ws.otc_part,
                ws.otc_cap, ws.otc_cts, ws.otc_ldct,
                ws.otc_h, ws.otc_bar, ws.shifted_flag)) {
        if (ws.tc_used) *ws.tc_used = true;
        return;
    }
    if (sizeof(T) == 4 &&
        orth_fused(ex, len, ld, reinterpret_cast<const float*>(Qb), m, reinterpret_cast<float*>(W), c,
                   reinterpret_cast<float*>(Wtmp), reinterpret_cast<float*>(Qout), ws))
        return;
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
        const int R = int(mm + c < of::RMAX ? mm + c : of::RMAX);
        z.fcap = int64_t(of::MAXG) * of::r4(R * c);
        z.fpart = size_t(z.fcap) * 4;
        z.fgram = size_t(R) * c * 4;
        z.fbar = 16;
        if (orth_tc_fits(len_max, 0, c, num_sms)) {
            const int mt = int(mm < 448 ? mm : 448);
            z.otc_cap = int64_t(orth_tc_part_floats(len_max, mt, c, num_sms));
            z.otc_part = size_t(z.otc_cap) * 4;
            z.otc_ldct = round_up(mt, 32);
            z.otc_cts = size_t(128) * z.otc_ldct * 4;
            z.otc_h = 64 * 65 * 4;   // the c x c Gram and the c projection energies
            z.otc_bar = 16;
        }
    }
    return z;
}

#define BKS_INST(T)                                                                                 \
    template void orth_block<T>(Exec&, int64_t, int64_t, const T*, int, T*, int, T*, T*, const OrthWs&);
BKS_INST(float)
BKS_INST(double)
#undef BKS_INST

}  // namespace bks
