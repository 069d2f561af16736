// Top-k eigenvectors of the Rayleigh-Ritz matrix M = B^T B (Sec. 4.1, steps 5-6 of
// Algorithms 1 and 2) through a symmetric tridiagonal form.
//
// Steps 6-7 use only Ubar_k, the k leading eigenvectors of M.  This solver
//   1. reduces M to tridiagonal T = H^T M H by w - 2 Householder reflections in one
//      thread-block cluster: M is distributed column-cyclically over the CTAs' shared
//      memory and each column costs one cluster barrier;
//   2. finds the k largest eigenvalues of T by Sturm-count multisection (one warp per
//      eigenvalue, 31 shifts per round);
//   3. finds their eigenvectors by inverse iteration (Gaussian elimination with partial
//      pivoting of T - lambda I, two solves from a pseudo-random start), then makes the
//      k vectors orthonormal with one CholeskyQR2 (eigenvalues closer than the rounding
//      level give independent vectors of their common invariant subspace);
//   4. maps them back, u = H_0 ... H_{w-3} x, with the reflectors grouped 16 at a time in
//      compact WY form, I - V T V^T (one warp per vector).
// Its cost does not depend on the spectrum, unlike the sweep count of a Jacobi solve.
#include <cooperative_groups.h>

#include <cfloat>

#include "chol_small.cuh"
#include "common.cuh"
#include "tc_common.cuh"

namespace cg = cooperative_groups;

namespace bks {
namespace {

constexpr int TD_NT = 512;                   // threads per CTA of the reduction
constexpr int TD_NW = TD_NT / 32;
constexpr int TD_ROWS = 2;                   // rows of a gathered column per thread (w <= 1024)
constexpr int TD_PART = 8;                   // partial sums of p . v per lane (C TD_NW <= 256)
constexpr size_t SMEM_MAX = 200 * 1024;      // shared bytes per CTA the kernels may use
constexpr int WY_NB = 16;                    // reflectors per compact-WY block
constexpr int WY_WARPS = 4;                  // vectors per CTA of the back-transformation
constexpr int WY_MAXS = 4;                   // ring slots of reflector blocks (back-transformation)

// Row pitch of the reflector matrix V: a multiple of 16 bytes, so that a block of WY_NB
// rows is one contiguous bulk copy.  V has round_up(w, WY_NB) rows, zero outside the
// reflectors' supports.
__host__ __device__ constexpr int64_t v_pitch(int w) { return (int64_t(w) + 3) / 4 * 4; }

template <typename T> __device__ __forceinline__ T fast_div(T a, T b) { return a / b; }
template <> __device__ __forceinline__ float fast_div<float>(float a, float b) { return __fdividef(a, b); }
template <typename T> __device__ __forceinline__ T recip(T a) { return T(1) / a; }
template <> __device__ __forceinline__ float recip<float>(float a) { return __fdividef(1.f, a); }

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Shape of the reduction on a cluster of C CTAs: nl columns per CTA, tpc threads per
// column (nl tpc <= TD_NT), column pitch wp (wp = tpc mod 32 spreads the tpc-row groups
// of neighbouring columns over distinct banks).
struct TdShape {
    int C = 0, nl = 0, tpc = 0;
    int64_t wp = 0;
    size_t smem = 0;
};

template <typename T>
TdShape td_shape(int w, int C) {
    TdShape s;
    s.C = C;
    s.nl = (w + C - 1) / C;
    int p2 = 1;
    while (p2 < s.nl) p2 <<= 1;
    if (p2 > TD_NT) return TdShape{};
    s.tpc = TD_NT / p2 < 32 ? TD_NT / p2 : 32;
    s.wp = round_up(w, 32) + (s.tpc < 32 ? s.tpc : 0);
    const size_t nlp = size_t(round_up(s.nl, 4));
    s.smem = (size_t(s.nl + 3) * s.wp + 2 * nlp + 3 * TD_NW + 4) * sizeof(T);
    if (w > TD_ROWS * TD_NT || C * TD_NW > 32 * TD_PART) return TdShape{};
    return s;
}

// Smallest power-of-two cluster with at most 32 columns per CTA (else the widest that fits;
// measured on GB300: 32 columns per CTA beat 64 and 128 at w = 220 and 450).
template <typename T>
TdShape td_pick(int w) {
    TdShape best;
    for (int C = 1; C <= 16; C *= 2) {
        const TdShape s = td_shape<T>(w, C);
        if (s.C == 0 || s.smem > SMEM_MAX) continue;
        best = s;
        if (s.nl <= 32) break;
    }
    return best;
}

// Householder tridiagonalisation of the symmetric w x w M (row pitch w), scaled by
// 1 / max_i M_ii.  CTA r keeps columns c = l C + r (l < nl).  Step j: every CTA holds
// column j (rows j..w-1) in xa and derives the same reflector H_j = I - tau v v^T from it
// (v[j+1] = 1, v_i = s x_i below; all CTAs compute it in the same order, so bit for bit);
// tpc threads per own column c > j form p_c = tau A(j+1:, c) . v.  After the cluster
// barrier each CTA gathers p, K = (tau / 2) p . v and column j+1 (read in place from its
// owner: no step after j-1 writes it; all these remote loads are issued before any of
// them is used), forms w = p - K v, updates its columns, A -= v w^T + w v^T, and column
// j+1, which becomes the next step's xa (double-buffered).  Per step: one cluster barrier
// and two CTA barriers.  Outputs: dT (w), eT (w - 1), tau (w - 1), max_i M_ii in
// tau[w - 1] (the eigenvalues of M are those of T times it) and the reflectors: row j of
// V (pitch v_pitch(w)) holds v_j in columns j+1..w-1.
template <typename T>
__global__ void __launch_bounds__(TD_NT) tridiag_kernel(const T* __restrict__ M, int w, int tpc, int64_t wp,
                                                        T* __restrict__ dT, T* __restrict__ eT,
                                                        T* __restrict__ tau_out, T* __restrict__ V) {
    cg::cluster_group cl = cg::this_cluster();
    const int C = int(cl.num_blocks());
    const int lc = __ffs(C) - 1;
    const int r = int(cl.block_rank());
    const int nl = (w + C - 1) / C;
    const int nlp = (nl + 3) / 4 * 4;
    extern __shared__ __align__(16) unsigned char td_smem_raw[];
    T* A = reinterpret_cast<T*>(td_smem_raw);   // nl x wp
    T* xv = A + size_t(nl) * wp;                // 2 x wp: current column, next column
    T* pv = xv + 2 * wp;                        // gathered p (raw)
    T* pbuf = pv + wp;                          // 2 x nlp: p of the own columns
    T* red2 = pbuf + 2 * nlp;                   // 2 x TD_NW: warp partials of p . v
    T* red = red2 + 2 * TD_NW;                  // TD_NW: warp partials of |x|^2
    T* misc = red + TD_NW;                      // [K]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int lt = tid / tpc, sub = tid % tpc;
    const int ct = lt * C + r;                  // this thread's column
    const bool colv = lt < nl && ct < w;

    T mx = T(0);
    for (int i = tid; i < w; i += TD_NT) mx = fmax(mx, M[int64_t(i) * (w + 1)]);
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) red[warp] = mx;
    __syncthreads();
    mx = T(0);
    for (int q = 0; q < TD_NW; ++q) mx = fmax(mx, red[q]);
    const T sc = (mx > T(0) && isfinite(mx)) ? T(1) / mx : T(1);
    if (r == 0 && tid == 0) tau_out[w - 1] = T(1) / sc;   // eigenvalues of M = those of T times this
    for (int l0 = 0; l0 < nl; l0 += 8)
        for (int i = tid; i < w; i += TD_NT) {
            T rv[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int c = (l0 + u) * C + r;
                rv[u] = (l0 + u < nl && c < w) ? M[int64_t(c) * w + i] : T(0);
            }
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (l0 + u < nl) A[(l0 + u) * wp + i] = rv[u] * sc;
        }
    T ss0 = T(0);
    for (int i = tid; i < w; i += TD_NT) {
        const T x = M[i] * sc;
        xv[i] = x;
        if (i >= 2) ss0 += x * x;
    }
    ss0 = warp_sum(ss0);
    __syncthreads();   // everyone has read red (the maximum)
    if (lane == 0) red[warp] = ss0;
    __syncthreads();

    for (int j = 0;; ++j) {
        const int par = j & 1;
        const T* xa = xv + par * wp;            // column j
        T* xb = xv + (par ^ 1) * wp;            // column j+1 after this step
        if (r == 0 && tid == 0) dT[j] = xa[j];
        if (j == w - 1) break;
        // reflector from rows j+1.. of column j (beta = -sign(alpha) |x|), v_i = scal x_i
        T ss = T(0);
        for (int q = 0; q < TD_NW; ++q) ss += red[q];
        const T alpha = xa[j + 1];
        T tau = T(0), beta = alpha, scal = T(0);
        if (ss > T(0)) {
            beta = -copysign(sqrt(alpha * alpha + ss), alpha);
            tau = (beta - alpha) / beta;
            scal = T(1) / (alpha - beta);
        }
        const bool act = tau != T(0);
        if (r == 0) {
            if (tid == 0) {
                eT[j] = beta;
                tau_out[j] = tau;
            }
            for (int i = j + 1 + tid; i < w; i += TD_NT)
                V[int64_t(j) * v_pitch(w) + i] = act ? (i == j + 1 ? T(1) : xa[i] * scal) : T(0);
        }
        if (act) {
            // p_c = tau (A(j+1, c) + scal sum_{i >= j+2} A(i, c) x_i)
            // four rows per pass, all eight loads issued before the products
            T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
            const T* col = A + lt * wp;
            if (colv && ct > j) {
                int i = j + 2 + sub;
                for (; i + 3 * tpc < w; i += 4 * tpc) {
                    const T a0 = col[i], a1 = col[i + tpc], a2 = col[i + 2 * tpc], a3 = col[i + 3 * tpc];
                    const T x0 = xa[i], x1 = xa[i + tpc], x2 = xa[i + 2 * tpc], x3 = xa[i + 3 * tpc];
                    s0 += a0 * x0;
                    s1 += a1 * x1;
                    s2 += a2 * x2;
                    s3 += a3 * x3;
                }
                for (; i < w; i += tpc) s0 += col[i] * xa[i];
            }
            T s = (s0 + s1) + (s2 + s3);
            for (int o = tpc >> 1; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            T dp = T(0);
            if (colv && ct > j && sub == 0) {
                s = tau * (col[j + 1] + scal * s);
                pbuf[par * nlp + lt] = s;
                dp = s * (ct == j + 1 ? T(1) : xa[ct] * scal);
            }
            dp = warp_sum(dp);
            if (lane == 0) red2[par * TD_NW + warp] = dp;
        }
        // column j+1 of the owner's A: written last by step j-1, read-only from here on
        const int own1 = (j + 1) & (C - 1);
        cl.sync();
        const T* ycol = cl.map_shared_rank(A + ((j + 1) >> lc) * wp, own1);
        T yr[TD_ROWS];
#pragma unroll
        for (int u = 0; u < TD_ROWS; ++u) {
            const int i = j + 1 + tid + u * TD_NT;
            yr[u] = i < w ? ycol[i] : T(0);
        }
        T ssn = T(0);
        if (act) {
            for (int i = j + 1 + tid; i < w; i += TD_NT)
                pv[i] = cl.map_shared_rank(pbuf + par * nlp, i & (C - 1))[i >> lc];
            if (warp == 0) {
                T part[TD_PART];
#pragma unroll
                for (int u = 0; u < TD_PART; ++u) {
                    const int q = lane + 32 * u;
                    part[u] = q < C * TD_NW ? cl.map_shared_rank(red2 + par * TD_NW, q / TD_NW)[q % TD_NW] : T(0);
                }
                T dsum = T(0);
#pragma unroll
                for (int u = 0; u < TD_PART; ++u) dsum += part[u];
                dsum = warp_sum(dsum);
                if (lane == 0) misc[0] = T(0.5) * tau * dsum;
            }
            __syncthreads();   // pv, K
            const T K = misc[0];
            const T w1 = pv[j + 1] - K;   // v[j+1] = 1
#pragma unroll
            for (int u = 0; u < TD_ROWS; ++u) {
                const int i = j + 1 + tid + u * TD_NT;
                if (i >= w) break;
                const T vi = i == j + 1 ? T(1) : xa[i] * scal;
                const T x = yr[u] - (vi * w1 + (pv[i] - K * vi));
                xb[i] = x;
                if (i >= j + 3) ssn += x * x;
            }
            if (colv && ct > j + 1) {
                const T vc = xa[ct] * scal, wc = pv[ct] - K * vc;
                T* col = A + lt * wp;
                int i = j + 2 + sub;
                for (; i + 3 * tpc < w; i += 4 * tpc) {   // four rows per pass, loads first
                    T c4[4], x4[4], p4[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        c4[u] = col[i + u * tpc];
                        x4[u] = xa[i + u * tpc];
                        p4[u] = pv[i + u * tpc];
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const T vi = x4[u] * scal;
                        col[i + u * tpc] = c4[u] - (vi * wc + (p4[u] - K * vi) * vc);
                    }
                }
                for (; i < w; i += tpc) {
                    const T vi = xa[i] * scal;
                    col[i] -= vi * wc + (pv[i] - K * vi) * vc;
                }
            }
        } else {
#pragma unroll
            for (int u = 0; u < TD_ROWS; ++u) {
                const int i = j + 1 + tid + u * TD_NT;
                if (i >= w) break;
                const T x = yr[u];
                xb[i] = x;
                if (i >= j + 3) ssn += x * x;
            }
        }
        ssn = warp_sum(ssn);
        if (lane == 0) red[warp] = ssn;
        __syncthreads();
    }
    cl.sync();   // no CTA leaves while another may still read its shared memory
}

// Numbers of eigenvalues of T below x0 and below x1 (Sturm sequences of the LDL^T
// pivots), the two recurrences interleaved so that each hides the other's latency.
template <typename T>
__device__ void sturm_count2(const T* d, const T* e2, int w, T x0, T x1, T pivmin, int& c0, int& c1) {
    T q0 = d[0] - x0, q1 = d[0] - x1;
    if (fabs(q0) < pivmin) q0 = -pivmin;
    if (fabs(q1) < pivmin) q1 = -pivmin;
    c0 = q0 < T(0);
    c1 = q1 < T(0);
    for (int i = 1; i < w; ++i) {
        const T di = d[i], ei = e2[i - 1];
        q0 = (di - x0) - fast_div(ei, q0);
        q1 = (di - x1) - fast_div(ei, q1);
        if (fabs(q0) < pivmin) q0 = -pivmin;
        if (fabs(q1) < pivmin) q1 = -pivmin;
        c0 += q0 < T(0);
        c1 += q1 < T(0);
    }
}

// Eigenvalue i (descending, i < m) of T per warp: Gershgorin interval, then rounds of 63
// Sturm counts (two per lane) keeping the 1/64 of the interval that holds it, to an
// absolute width of 4 eps |T|.  lam[i] = midpoint; block 0 also stores |T| (largest
// Gershgorin bound).
template <typename T>
__global__ void bisect_kernel(const T* __restrict__ dT, const T* __restrict__ eT, int w, int m,
                              T* __restrict__ lam, T* __restrict__ tn) {
    extern __shared__ __align__(16) unsigned char bis_smem[];
    T* d = reinterpret_cast<T*>(bis_smem);
    T* e2 = d + w;
    __shared__ T s_lo[32], s_hi[32], s_e2[32];
    for (int i = threadIdx.x; i < w; i += blockDim.x) {
        d[i] = dT[i];
        if (i + 1 < w) e2[i] = eT[i] * eT[i];
    }
    T lo = T(INFINITY), hi = T(-INFINITY), me = T(0);
    for (int i = threadIdx.x; i < w; i += blockDim.x) {
        const T rad = (i > 0 ? fabs(eT[i - 1]) : T(0)) + (i + 1 < w ? fabs(eT[i]) : T(0));
        lo = fmin(lo, dT[i] - rad);
        hi = fmax(hi, dT[i] + rad);
        if (i + 1 < w) me = fmax(me, eT[i] * eT[i]);
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        me = fmax(me, __shfl_xor_sync(0xffffffffu, me, o));
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) { s_lo[warp] = lo; s_hi[warp] = hi; s_e2[warp] = me; }
    __syncthreads();
    lo = s_lo[0]; hi = s_hi[0]; me = s_e2[0];
    for (int q = 1; q < int(blockDim.x >> 5); ++q) {
        lo = fmin(lo, s_lo[q]);
        hi = fmax(hi, s_hi[q]);
        me = fmax(me, s_e2[q]);
    }
    const T eps = sizeof(T) == 8 ? T(DBL_EPSILON) : T(FLT_EPSILON);
    const T tiny = sizeof(T) == 8 ? T(DBL_MIN) : T(FLT_MIN);
    const T tnorm = fmax(fabs(lo), fabs(hi));
    if (blockIdx.x == 0 && threadIdx.x == 0) tn[0] = tnorm;
    const T pivmin = tiny * fmax(T(1), me);
    const T pad = T(2) * eps * tnorm + pivmin;   // both ends count correctly under rounding
    lo -= pad;
    hi += pad;
    const int i = blockIdx.x * int(blockDim.x >> 5) + warp;
    if (i >= m) return;
    const int t = w - 1 - i;   // ascending index
    const T tol = T(4) * eps * tnorm + pivmin;
    T a = lo, b = hi;
    // shift k < 64: a + (b - a) (k + 1) / 64 (k = 63: b, counted as w); lane l holds
    // k = 2l and 2l + 1, and the first shift with more than t eigenvalues below it is the
    // earlier of the first even and the first odd one the two ballots find.
    auto shift = [&](int k) -> T { return k == 63 ? b : a + (b - a) * (T(k + 1) / T(64)); };
    for (int it = 0; it < 16 && b - a > tol; ++it) {
        const T x0 = shift(2 * lane), x1 = shift(2 * lane + 1);
        int c0, c1;
        sturm_count2(d, e2, w, x0, x1, pivmin, c0, c1);
        if (lane == 31) c1 = w;
        const unsigned m0 = __ballot_sync(0xffffffffu, c0 >= t + 1);
        const unsigned m1 = __ballot_sync(0xffffffffu, c1 >= t + 1);
        const int l0 = m0 ? __ffs(m0) - 1 : 32, l1 = __ffs(m1) - 1;
        const int ks = min(2 * l0, 2 * l1 + 1);   // first shift with more than t below
        const T xa = shift(ks > 0 ? ks - 1 : 0), xb = shift(ks);
        if (ks > 0) a = xa;
        b = xb;
    }
    if (lane == 0) lam[i] = T(0.5) * (a + b);
}

// Pseudo-random start vector entry in [-1, 1) (32-bit integer hash of the position).
__device__ __forceinline__ float start_entry(int i, int t) {
    unsigned x = unsigned(i) * 0x9E3779B1u ^ unsigned(t + 1) * 0x85EBCA77u;
    x ^= x >> 15;
    x *= 0x2C1B3C6Du;
    x ^= x >> 12;
    x *= 0x297A2D39u;
    x ^= x >> 15;
    return float(x >> 8) * (1.f / 8388608.f) - 1.f;
}

// Inverse iteration, one thread per eigenvalue, vpc per CTA, everything in shared memory
// ([i][vector] layout).  The first round eliminates T - lam_t I with partial pivoting
// while applying the same steps to the right-hand side (a pseudo-random start), keeping
// U (reciprocal pivot and two super-diagonals) for the back substitution and each
// step's row swap and multiplier; the second round applies only those stored steps to
// its right-hand side (the first round's normalised solution) and substitutes back
// through the same U.  Tiny pivots are raised to eps |T|.
// Output: X (m x ldx, row t = unit vector t, zero pad).
template <typename T>
size_t invit_smem(int w, int vpc) {
    return (size_t(2) * w + size_t(6) * w * vpc) * sizeof(T);
}

template <typename T>
__global__ void invit_kernel(const T* __restrict__ dT, const T* __restrict__ eT, const T* __restrict__ lam,
                             const T* __restrict__ tn, int w, int m, T* __restrict__ X, int64_t ldx,
                             int* __restrict__ status) {
    extern __shared__ __align__(16) unsigned char iv_smem[];
    __shared__ T s_scale[32];
    const int vpc = blockDim.x;
    T* d = reinterpret_cast<T*>(iv_smem);
    T* e = d + w;
    T* R0 = e + w;                      // reciprocal pivots
    T* U1 = R0 + size_t(w) * vpc;
    T* U2 = U1 + size_t(w) * vpc;
    T* Z = U2 + size_t(w) * vpc;        // right-hand side, then solution
    T* MU = Z + size_t(w) * vpc;        // multipliers of the elimination
    T* SW = MU + size_t(w) * vpc;       // 1: rows i and i+1 swapped at step i
    for (int i = threadIdx.x; i < w; i += vpc) {
        d[i] = dT[i];
        e[i] = i + 1 < w ? eT[i] : T(0);
    }
    __syncthreads();
    const int tl = threadIdx.x;
    const int t = blockIdx.x * vpc + tl;
    const T eps = sizeof(T) == 8 ? T(DBL_EPSILON) : T(FLT_EPSILON);
    const T tnorm = tn[0];
    const T pert = eps * (tnorm > T(0) ? tnorm : T(1));
    T scale = T(0);
    if (t < m) {
        const T lt = lam[t];
        for (int round = 0; round < 2; ++round) {
            const T sprev = scale;
            T r0 = d[0] - lt, r1 = e[0];
            T ry = round == 0 ? T(start_entry(0, t)) : Z[tl] * sprev;
            if (round == 0) {
                for (int i = 0; i + 1 < w; ++i) {
                    const T ei = e[i];
                    const T an = d[i + 1] - lt;
                    const T en = e[i + 1];
                    const T yn = T(start_entry(i + 1, t));
                    const size_t o = size_t(i) * vpc + tl;
                    // pivot row: the active row (no swap) or row i+1 (swap), whichever has
                    // the larger entry in column i
                    const bool sw = fabs(ei) > fabs(r0);
                    if (!sw && fabs(r0) < pert) r0 = copysign(pert, r0);
                    const T piv = sw ? ei : r0;
                    const T oth = sw ? r0 : ei;
                    const T rc = recip(piv);
                    const T mu = oth * rc;
                    R0[o] = rc;
                    U1[o] = sw ? an : r1;
                    U2[o] = sw ? en : T(0);
                    MU[o] = mu;
                    SW[o] = sw ? T(1) : T(0);
                    Z[o] = sw ? yn : ry;
                    const T ry_n = sw ? ry - mu * yn : yn - mu * ry;
                    const T r0_n = sw ? r1 - mu * an : an - mu * r1;
                    r1 = sw ? -mu * en : en;
                    ry = ry_n;
                    r0 = r0_n;
                }
            } else {
                // the stored row operations on the new right-hand side (row i+1 is read
                // before step i+1 overwrites it)
                for (int i = 0; i + 1 < w; ++i) {
                    const size_t o = size_t(i) * vpc + tl;
                    const T yn = Z[o + vpc] * sprev;
                    const bool sw = SW[o] != T(0);
                    const T mu = MU[o];
                    Z[o] = sw ? yn : ry;
                    ry = sw ? ry - mu * yn : yn - mu * ry;
                }
            }
            const size_t ol = size_t(w - 1) * vpc + tl;
            if (round == 0) {
                if (fabs(r0) < pert) r0 = copysign(pert, r0);
                R0[ol] = recip(r0);
                U1[ol] = T(0);
                U2[ol] = T(0);
            }
            Z[ol] = ry;
            // back substitution; when the solution grows past BIG (many pivots at the
            // eps |T| floor, as for eigenvalues of a numerical null space), the whole
            // system is rescaled: only the direction is kept
            const T BIG = sizeof(T) == 8 ? T(1e150) : T(1e12f);
            T x1 = T(0), x2 = T(0), nn = T(0);
            for (int i = w - 1; i >= 0; --i) {
                const size_t o = size_t(i) * vpc + tl;
                T xi = (Z[o] - U1[o] * x1 - U2[o] * x2) * R0[o];
                if (!(fabs(xi) <= BIG) && isfinite(xi)) {
                    const T f = T(1) / fabs(xi);
                    for (int q = 0; q < w; ++q) Z[size_t(q) * vpc + tl] *= f;
                    xi *= f;
                    x1 *= f;
                    x2 *= f;
                    nn *= f * f;
                }
                Z[o] = xi;
                nn += xi * xi;
                x2 = x1;
                x1 = xi;
            }
            if (!isfinite(nn)) atomicOr(status, ST_NONFINITE);
            scale = nn > T(0) && isfinite(nn) ? T(1) / sqrt(nn) : T(0);
        }
    }
    s_scale[tl] = scale;
    __syncthreads();
    // store coalesced along i: row t of X = Z[:, tl] * scale
    const int nv = m - blockIdx.x * vpc < vpc ? m - blockIdx.x * vpc : vpc;
    for (int v = 0; v < nv; ++v)
        for (int i = tl; i < ldx; i += vpc)
            X[int64_t(blockIdx.x * vpc + v) * ldx + i] = i < w ? Z[size_t(i) * vpc + v] * s_scale[v] : T(0);
}

template <typename T>
int invit_vpc(int w) {
    for (int v = 32; v >= 4; v >>= 1)
        if (invit_smem<T>(w, v) <= SMEM_MAX) return v;
    return 0;
}

// Rows q0..q0+NB-1 of V into Vs (NB x wp), zero outside each reflector's support
// (v_q lives in columns q+1..w-1) and for rows past nb; all NB loads of a column index
// are issued before any store.
template <typename T>
__device__ void stage_block(const T* __restrict__ V, int w, int q0, int nb, T* Vs, int64_t wp) {
    for (int i = threadIdx.x; i < w; i += blockDim.x) {
        T r[WY_NB];
#pragma unroll
        for (int a = 0; a < WY_NB; ++a) r[a] = (a < nb && i > q0 + a) ? V[int64_t(q0 + a) * v_pitch(w) + i] : T(0);
#pragma unroll
        for (int a = 0; a < WY_NB; ++a) Vs[a * wp + i] = r[a];
    }
}

// Compact WY factor of reflector block b (reflectors q0 = b NB .. q0 + nb - 1):
// H_q0 ... H_{q0+nb-1} = I - Vb Tb Vb^T with Tb upper triangular (forward, columnwise:
// Tb[i][i] = tau_i, Tb[0:i, i] = -tau_i Tb[0:i, 0:i] (Vb[:, 0:i]^T v_i)).
template <typename T>
__global__ void wy_factor_kernel(const T* __restrict__ V, const T* __restrict__ tau, int w, int nref,
                                 T* __restrict__ Tw) {
    extern __shared__ __align__(16) unsigned char wy_smem[];
    const int64_t wp = (int64_t(w) + 3) / 4 * 4;
    T* Vs = reinterpret_cast<T*>(wy_smem);   // NB x wp
    __shared__ T G[WY_NB][WY_NB + 1];
    __shared__ T Tm[WY_NB][WY_NB + 1];
    const int q0 = blockIdx.x * WY_NB;
    const int nb = nref - q0 < WY_NB ? nref - q0 : WY_NB;
    stage_block(V, w, q0, nb, Vs, wp);
    for (int p = threadIdx.x; p < WY_NB * WY_NB; p += blockDim.x) {
        G[p / WY_NB][p % WY_NB] = T(0);
        Tm[p / WY_NB][p % WY_NB] = T(0);
    }
    __syncthreads();
    for (int p = threadIdx.x; p < WY_NB * WY_NB; p += blockDim.x) {
        const int a = p / WY_NB, c = p % WY_NB;
        if (a < c && c < nb) {
            T s = T(0);
            for (int i = q0 + c + 1; i < w; ++i) s += Vs[a * wp + i] * Vs[c * wp + i];
            G[a][c] = s;
        }
    }
    if (threadIdx.x < nb) Tm[threadIdx.x][threadIdx.x] = tau[q0 + threadIdx.x];
    __syncthreads();
    for (int c = 1; c < nb; ++c) {
        const int a = threadIdx.x;
        if (a < c) {
            T s = T(0);
            for (int e2 = a; e2 < c; ++e2) s += Tm[a][e2] * G[e2][c];
            Tm[a][c] = -tau[q0 + c] * s;
        }
        __syncthreads();
    }
    for (int p = threadIdx.x; p < WY_NB * WY_NB; p += blockDim.x)
        Tw[int64_t(blockIdx.x) * WY_NB * WY_NB + p] = Tm[p / WY_NB][p % WY_NB];
}

// Vt row t = H_0 ... H_{nref-1} x_t, the blocks applied last to first as
// x -= Vb (Tb (Vb^T x)); one warp per vector.  The reflector blocks (WY_NB rows of V,
// zero outside their supports, and their Tb) stream through a ring of ns slots in
// shared memory, each filled by two bulk copies that complete on the slot's mbarrier,
// so the next blocks' loads overlap the current block's arithmetic.  Every wait is
// bounded (ST_TIMEOUT).
template <typename T>
__global__ void __launch_bounds__(WY_WARPS * 32) wy_apply_kernel(const T* __restrict__ X, int64_t ldx, int w,
                                                                 int m, int nref, const T* __restrict__ V,
                                                                 const T* __restrict__ Tw, T* __restrict__ Vt,
                                                                 int64_t ldv, int ns, int* __restrict__ status) {
    extern __shared__ __align__(16) unsigned char wya_smem[];
    __shared__ uint64_t full[WY_MAXS];
    __shared__ int abort_flag;
    const int64_t vp = v_pitch(w);
    const int64_t slot = WY_NB * vp + WY_NB * WY_NB;          // elements per ring slot
    const uint32_t vbytes = uint32_t(WY_NB * vp * sizeof(T)), tbytes = uint32_t(WY_NB * WY_NB * sizeof(T));
    T* ring = reinterpret_cast<T*>(wya_smem);
    T* xs = ring + ns * slot;                                 // WY_WARPS x vp
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int t = blockIdx.x * WY_WARPS + warp;
    const int nblk = (nref + WY_NB - 1) / WY_NB;
    if (threadIdx.x == 0) {
        for (int q = 0; q < ns; ++q) tc::mbar_init(&full[q], 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // use u = 0, 1, ... takes block b = nblk - 1 - u in slot u % ns
    auto issue = [&](int u) {
        const int b = nblk - 1 - u;
        T* dst = ring + (u % ns) * slot;
        uint64_t* bar = &full[u % ns];
        tc::mbar_expect_tx(bar, vbytes + tbytes);
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                         tc::smem_u32(dst)),
                     "l"(V + int64_t(b) * WY_NB * vp), "r"(vbytes), "r"(tc::smem_u32(bar))
                     : "memory");
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                         tc::smem_u32(dst + WY_NB * vp)),
                     "l"(Tw + int64_t(b) * WY_NB * WY_NB), "r"(tbytes), "r"(tc::smem_u32(bar))
                     : "memory");
    };
    if (threadIdx.x == 0)
        for (int u = 0; u < ns && u < nblk; ++u) issue(u);
    T* x = xs + warp * vp;
    if (t < m)
        for (int i = lane; i < w; i += 32) x[i] = X[int64_t(t) * ldx + i];
    int issued = ns < nblk ? ns : nblk;
    for (int u = 0; u < nblk; ++u) {
        const int b = nblk - 1 - u, q0 = b * WY_NB;
        const T* Vs = ring + (u % ns) * slot;
        const T* Ts = Vs + WY_NB * vp;
        const bool ok = tc::wait_bar(&full[u % ns], uint32_t((u / ns) & 1), &abort_flag, status);
        if (ok && t < m) {
            T acc[WY_NB];
#pragma unroll
            for (int a = 0; a < WY_NB; ++a) acc[a] = T(0);
            for (int i = q0 + 1 + lane; i < w; i += 32) {
                const T xi = x[i];
#pragma unroll
                for (int a = 0; a < WY_NB; ++a) acc[a] += Vs[a * vp + i] * xi;
            }
#pragma unroll
            for (int a = 0; a < WY_NB; ++a) acc[a] = warp_sum(acc[a]);
            T mt = T(0);   // lane a < NB: (Tb s)_a
#pragma unroll
            for (int c = 0; c < WY_NB; ++c) mt += (lane < WY_NB ? Ts[lane * WY_NB + c] : T(0)) * acc[c];
            T tv[WY_NB];
#pragma unroll
            for (int a = 0; a < WY_NB; ++a) tv[a] = __shfl_sync(0xffffffffu, mt, a);
            for (int i = q0 + 1 + lane; i < w; i += 32) {
                T sm = T(0);
#pragma unroll
                for (int a = 0; a < WY_NB; ++a) sm += Vs[a * vp + i] * tv[a];
                x[i] -= sm;
            }
        }
        __syncthreads();   // slot u % ns is free
        if (threadIdx.x == 0 && issued < nblk && !abort_flag) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue(issued);
            ++issued;
        }
    }
    // every copy issued has landed before shared memory is released (bounded)
    if (threadIdx.x == 0)
        for (int u = issued > ns ? issued - ns : 0; u < issued; ++u) tc::drain_bar(&full[u % ns], (u / ns) & 1);
    __syncthreads();
    if (t < m && !abort_flag)
        for (int i = lane; i < w; i += 32) Vt[int64_t(t) * ldv + i] = x[i];
}

// ring slots of the back-transformation that fit next to the vectors (0: too wide)
template <typename T>
int wy_slots(int w) {
    const size_t vp = size_t(v_pitch(w));
    const size_t slot = (WY_NB * vp + WY_NB * WY_NB) * sizeof(T), xb = WY_WARPS * vp * sizeof(T);
    if (xb >= SMEM_MAX) return 0;
    const size_t n = (SMEM_MAX - xb) / slot;
    return n >= 2 ? int(n < WY_MAXS ? n : WY_MAXS) : 0;
}

template <typename T>
size_t wy_apply_smem(int w) {
    const size_t vp = size_t(v_pitch(w));
    return (size_t(wy_slots<T>(w)) * (WY_NB * vp + WY_NB * WY_NB) + WY_WARPS * vp) * sizeof(T);
}

// CholeskyQR2 of a small FP32 block held whole in one CTA's shared memory: X (c x ld,
// rows = vectors of length len), c <= 64, in place.  Each pass forms the Gram
// G = X X^T (4 x 4 tiles, one warp per tile with the lanes splitting the length, so
// every entry sums len / 32 products per lane and then a 32-way tree), factors
// G = L L^T into P = L^{-1} (chol_inv_block: shifted retries and breakdown flagged in
// status) and applies X <- P X, one thread per column of X.
constexpr int SQ_NT = 512;
constexpr int SQ_C = 64;
constexpr int SQ_GP = 65;   // row pitch of G
constexpr int SQ_PP = 68;   // row pitch of P (float4 rows)
inline int64_t sq_pitch(int len) { return (int64_t(len) + 3) / 4 * 4; }
inline size_t sq_smem(int c, int len) {
    return (size_t((c + 3) / 4 * 4) * size_t(sq_pitch(len)) + size_t(SQ_C) * (SQ_GP + SQ_PP)) * sizeof(float);
}

__global__ void __launch_bounds__(SQ_NT) small_cholqr2_kernel(float* __restrict__ X, int c, int len, int64_t ld,
                                                              int* __restrict__ status, int* __restrict__ shifted) {
    extern __shared__ __align__(16) unsigned char sq_smem_raw[];
    const int64_t xp = (int64_t(len) + 3) / 4 * 4;
    const int c4 = (c + 3) / 4 * 4;
    float* Xs = reinterpret_cast<float*>(sq_smem_raw);   // c4 x xp
    float* G = Xs + c4 * xp;                              // SQ_C x SQ_GP
    float* P = G + SQ_C * SQ_GP;                          // SQ_C x SQ_PP
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int e = tid; e < c4 * len; e += SQ_NT) {
        const int a = e / len, i = e - a * len;
        Xs[a * xp + i] = a < c ? X[int64_t(a) * ld + i] : 0.f;
    }
    __syncthreads();
    const int nt = c4 / 4, ntiles = nt * (nt + 1) / 2;
    for (int pass = 0; pass < 2; ++pass) {
        for (int e = warp; e < ntiles; e += SQ_NT / 32) {
            int ta = 0, rem = e;   // tile (ta, tb), ta <= tb, row-major over the upper triangle
            while (rem >= nt - ta) {
                rem -= nt - ta;
                ++ta;
            }
            const int tb = ta + rem;
            float acc[4][4] = {};
            for (int i = lane; i < len; i += 32) {
                float xa[4], xb[4];
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    xa[r] = Xs[(4 * ta + r) * xp + i];
                    xb[r] = Xs[(4 * tb + r) * xp + i];
                }
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc[r][q] = fmaf(xa[r], xb[q], acc[r][q]);
            }
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[r][q] = warp_sum(acc[r][q]);
            if (lane == 0)
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int a = 4 * ta + r, b = 4 * tb + q;
                        if (a < c && b < c) {
                            G[a * SQ_GP + b] = acc[r][q];
                            G[b * SQ_GP + a] = acc[r][q];
                        }
                    }
        }
        __syncthreads();
        chol_inv_block(G, SQ_GP, c, P, SQ_PP, status, shifted);
        __syncthreads();
        for (int i = tid; i < len; i += SQ_NT) {
            float x[SQ_C];
#pragma unroll
            for (int b = 0; b < SQ_C; ++b) x[b] = b < c ? Xs[b * xp + i] : 0.f;
#pragma unroll
            for (int a = 0; a < SQ_C; ++a) {
                if (a >= c) break;
                float y = 0.f;
#pragma unroll
                for (int b4 = 0; b4 <= a; b4 += 4) {   // P is lower triangular: P[a][b] = 0 for b > a
                    const float4 pr = *reinterpret_cast<const float4*>(P + a * SQ_PP + b4);
                    y = fmaf(pr.x, x[b4], y);
                    if (b4 + 1 <= a) y = fmaf(pr.y, x[b4 + 1], y);
                    if (b4 + 2 <= a) y = fmaf(pr.z, x[b4 + 2], y);
                    if (b4 + 3 <= a) y = fmaf(pr.w, x[b4 + 3], y);
                }
                Xs[a * xp + i] = y;
            }
        }
        __syncthreads();
    }
    for (int e = tid; e < c * len; e += SQ_NT) {
        const int a = e / len, i = e - a * len;
        X[int64_t(a) * ld + i] = Xs[a * xp + i];
    }
}

// The small-block CholeskyQR2 above when it applies (FP32, c <= 64, the block within the
// shared-memory budget); false: the caller orthonormalises through orth_block.
bool small_cholqr2(Exec& ex, float* X, int c, int len, int64_t ld, int* shifted_flag) {
    if (shifted_flag == nullptr || c < 1 || c > SQ_C || len < c || sq_smem(c, len) > SMEM_MAX) return false;
    const size_t smem = sq_smem(c, len);
    if (allow_dynamic_smem(reinterpret_cast<const void*>(small_cholqr2_kernel), smem) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    small_cholqr2_kernel<<<1, SQ_NT, smem, ex.stream>>>(X, c, len, ld, ex.status, shifted_flag);
    ex.launches += 1;
    return true;
}

}  // namespace

template <typename T>
bool tridiag_fits(int w, int m) {
    return w >= 3 && m >= 1 && m <= w && td_pick<T>(w).C > 0 && invit_vpc<T>(w) > 0 && wy_slots<T>(w) > 0;
}

// Scratch layout (element offsets, each buffer starting on a 64-element boundary): dT,
// eT, tau, |T| (w each), lam (m), V (round_up(w, NB) x v_pitch(w)), X and its
// orthonormalisation scratch (m x ldx each), WY factors (ceil(w / NB) NB^2).
struct TdScratch {
    size_t dT, eT, tau, tn, lam, V, X, Xtmp, Tw, total;
    TdScratch(int w, int m) {
        const size_t ldx = size_t(round_up(w, 32));
        const size_t nblk = size_t(w + WY_NB - 1) / WY_NB;
        size_t o = 0;
        auto take = [&](size_t n) { const size_t at = o; o += size_t(round_up(int64_t(n), 64)); return at; };
        dT = take(w); eT = take(w); tau = take(w); tn = take(w); lam = take(m);
        V = take(size_t(round_up(w, WY_NB)) * size_t(v_pitch(w)));
        X = take(size_t(m) * ldx); Xtmp = take(size_t(m) * ldx);
        Tw = take(nblk * WY_NB * WY_NB);
        total = o;
    }
};

size_t tridiag_scratch_elems(int w, int m) { return TdScratch(w, m).total; }

namespace {

// Tridiagonal reduction and multisection of the m largest eigenvalues (scaled by
// 1 / max_i M_ii, the inverse of the scale in tau[w - 1]).
template <typename T>
bool reduce_and_bisect(Exec& ex, int w, const T* M, int m, T* scratch, const TdScratch& L) {
    const TdShape sh = td_pick<T>(w);
    auto kern = tridiag_kernel<T>;
    if (allow_dynamic_smem(reinterpret_cast<const void*>(kern), sh.smem) != cudaSuccess ||
        (sh.C > 8 && cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)) {
        cudaGetLastError();
        return false;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(sh.C), 1, 1);
    cfg.blockDim = dim3(TD_NT, 1, 1);
    cfg.dynamicSmemBytes = sh.smem;
    cfg.stream = ex.stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = unsigned(sh.C);
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, kern, M, w, sh.tpc, sh.wp, scratch + L.dT, scratch + L.eT, scratch + L.tau,
                           scratch + L.V) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    const int wpb = 8;   // eigenvalues (warps) per CTA of the multisection
    bisect_kernel<T><<<(m + wpb - 1) / wpb, wpb * 32, size_t(2) * w * sizeof(T), ex.stream>>>(
        scratch + L.dT, scratch + L.eT, w, m, scratch + L.lam, scratch + L.tn);
    ex.launches += 2;
    return true;
}

}  // namespace

template <typename T>
bool topk_values(Exec& ex, int w, const T* M, int m, T* scratch, const T** lam, const T** inv_scale) {
    if (!tridiag_fits<T>(w, m)) return false;
    const TdScratch L(w, m);
    if (!reduce_and_bisect(ex, w, M, m, scratch, L)) return false;
    *lam = scratch + L.lam;
    *inv_scale = scratch + L.tau + (w - 1);
    return true;
}

template <typename T>
bool topk_tridiag(Exec& ex, int w, const T* M, int m, T* Vt, int64_t ldv, T* scratch, const OrthWs& ows) {
    if (!tridiag_fits<T>(w, m)) return false;
    const int64_t ldx = round_up(w, 32);
    const TdScratch L(w, m);
    T* dT = scratch + L.dT;
    T* eT = scratch + L.eT;
    T* tau = scratch + L.tau;
    T* tn = scratch + L.tn;
    T* lam = scratch + L.lam;
    T* V = scratch + L.V;
    T* X = scratch + L.X;
    T* Xtmp = scratch + L.Xtmp;
    T* Tw = scratch + L.Tw;
    // the reduction writes each reflector's support only: the rest of V stays zero
    cudaMemsetAsync(V, 0, size_t(round_up(w, WY_NB)) * size_t(v_pitch(w)) * sizeof(T), ex.stream);
    if (!reduce_and_bisect(ex, w, M, m, scratch, L)) return false;
    const int vpc = invit_vpc<T>(w);
    const size_t ismem = invit_smem<T>(w, vpc);
    if (ismem > 48 * 1024) allow_dynamic_smem(reinterpret_cast<const void*>(invit_kernel<T>), ismem);
    invit_kernel<T><<<(m + vpc - 1) / vpc, vpc, ismem, ex.stream>>>(dT, eT, lam, tn, w, m, X, ldx, ex.status);
    ex.launches += 1;
    // orthonormal eigenvector basis (CholeskyQR2 of the m x w block; thin blocks keep
    // their pad rows at zero, so the scratch block starts zeroed)
    if (!(sizeof(T) == 4 && small_cholqr2(ex, reinterpret_cast<float*>(X), m, w, ldx, ows.shifted_flag))) {
        cudaMemsetAsync(Xtmp, 0, size_t(m) * ldx * sizeof(T), ex.stream);
        orth_block<T>(ex, w, ldx, X, 0, X, m, Xtmp, X, ows);
    }
    const int nref = w - 2;
    const int nblk = (nref + WY_NB - 1) / WY_NB;
    const size_t fsmem = size_t(WY_NB) * v_pitch(w) * sizeof(T);
    if (fsmem > 48 * 1024) allow_dynamic_smem(reinterpret_cast<const void*>(wy_factor_kernel<T>), fsmem);
    wy_factor_kernel<T><<<nblk, 256, fsmem, ex.stream>>>(V, tau, w, nref, Tw);
    const size_t asmem = wy_apply_smem<T>(w);
    if (asmem > 48 * 1024) allow_dynamic_smem(reinterpret_cast<const void*>(wy_apply_kernel<T>), asmem);
    wy_apply_kernel<T><<<(m + WY_WARPS - 1) / WY_WARPS, WY_WARPS * 32, asmem, ex.stream>>>(
        X, ldx, w, m, nref, V, Tw, Vt, ldv, wy_slots<T>(w), ex.status);
    ex.launches += 2;
    return true;
}

template bool tridiag_fits<float>(int, int);
template bool tridiag_fits<double>(int, int);
template bool topk_tridiag<float>(Exec&, int, const float*, int, float*, int64_t, float*, const OrthWs&);
template bool topk_tridiag<double>(Exec&, int, const double*, int, double*, int64_t, double*, const OrthWs&);
template bool topk_values<float>(Exec&, int, const float*, int, float*, const float**, const float**);
template bool topk_values<double>(Exec&, int, const double*, int, double*, const double**, const double**);

}  // namespace bks
