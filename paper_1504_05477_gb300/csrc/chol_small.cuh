// The small Cholesky inverse shared by the orthonormalisation kernels: a block-wide
// device routine (every thread of the block calls it) for c <= 128.
#pragma once
#include "common.cuh"

namespace bks {

// P = L^{-1} = R^{-T} for G = L L^T (c <= 128) by symmetric elimination on [G | I]
// with the elimination rows kept in registers: each thread owns a 4 x TC tile of the
// trailing matrix S and of the lower-triangular E.  Step j publishes row j of S and E
// (double-buffered, one barrier per step) and every thread updates its tiles:
//   S[i][l] -= (S[i][j] / d_j) S[j][l],  E[i][l] -= (S[i][j] / d_j) E[j][l]   (i > j)
// with the pivot d_j = S[j][j].  At the end E = L_unit^{-1} for G = L_unit D L_unit^T,
// so L^{-1} = D^{-1/2} E.  A non-positive or non-finite pivot restarts the elimination
// with a diagonal shift (shifted CholeskyQR), up to six times, and sets *shifted_flag;
// a non-finite G sets ST_NONFINITE and a factorisation that still fails ST_BREAKDOWN,
// both with P = I.  Only P[i][l] for i, l < c is written.
constexpr int TR = 4;   // register tile rows per thread; columns TC = 4 when the block has
                        // (c/4)^2 threads (c <= 64 on 256 threads), else 8 (c <= 128: 512 threads)
template <int TC>
__device__ inline void chol_inv_block_t(const float* G, int64_t ldg, int c, float* P, int64_t ldp, int* status,
                                 int* shifted_flag) {
    __shared__ __align__(16) float rowS[2][128];
    __shared__ __align__(16) float rowE[2][128];
    __shared__ double trace_s;
    const int ntc = (c + TC - 1) / TC, ntr = (c + TR - 1) / TR;
    const int tid = threadIdx.x;
    const bool active = tid < ntr * ntc;
    const int ti = active ? tid / ntc : 0, tj = active ? tid % ntc : 0;
    const int r0 = ti * TR, c0 = tj * TC;
    bool nonfin = false;
    for (int a = 0; a < TR; ++a)
        for (int b = 0; b < TC; ++b) {
            const int i = r0 + a, l = c0 + b;
            if (!active || i >= c || l >= c) continue;
            nonfin |= !isfinite(G[int64_t(i) * ldg + l]);
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
            // branch-free update: row j of S and E read once (c0 is a multiple of 4), rows
            // at or above the pivot get a zero multiplier, columns pick S (l > j) or E
            const float inv = __frcp_rn(d);
            float rsv[TC], rev[TC];
#pragma unroll
            for (int b4 = 0; b4 < TC; b4 += 4) {
                const float4 sa = *reinterpret_cast<const float4*>(&rowS[par][c0 + b4]);
                const float4 ea = *reinterpret_cast<const float4*>(&rowE[par][c0 + b4]);
                rsv[b4] = sa.x; rsv[b4 + 1] = sa.y; rsv[b4 + 2] = sa.z; rsv[b4 + 3] = sa.w;
                rev[b4] = ea.x; rev[b4 + 1] = ea.y; rev[b4 + 2] = ea.z; rev[b4 + 3] = ea.w;
            }
            const float4 fr = *reinterpret_cast<const float4*>(&rowS[par][r0]);
            const float fv[TR] = {fr.x, fr.y, fr.z, fr.w};
#pragma unroll
            for (int a = 0; a < TR; ++a) {
                const int i = r0 + a;
                dpiv[a] = (i == j) ? d : dpiv[a];
                const float f = (i > j) ? fv[a] * inv : 0.f;   // S[i][j] = S[j][i]
#pragma unroll
                for (int b = 0; b < TC; ++b) {
                    const bool right = c0 + b > j;
                    const float us = fmaf(-f, rsv[b], s[a][b]);
                    const float ue = fmaf(-f, rev[b], e[a][b]);
                    s[a][b] = right ? us : s[a][b];
                    e[a][b] = right ? e[a][b] : ue;
                }
            }
        }
        __syncthreads();
        if (!ok) {
            if (shift == 0.0) {   // first retry: the shift is relative to the trace of G
                if (tid == 0) {
                    double t = 0.0;
                    for (int i = 0; i < c; ++i) t += double(G[int64_t(i) * ldg + i]);
                    trace_s = t;
                }
                __syncthreads();
                shift = 1e-6 * trace_s / c;
            } else {
                shift *= 1e3;
            }
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

// Block-wide device routine (all threads of the block call it; G and P may live in global
// or shared memory): the 4 x 4 register tiling when the block has enough threads for it.
__device__ inline void chol_inv_block(const float* G, int64_t ldg, int c, float* P, int64_t ldp, int* status,
                               int* shifted_flag) {
    const int n4 = (c + 3) / 4;
    if (n4 * n4 <= int(blockDim.x))
        chol_inv_block_t<4>(G, ldg, c, P, ldp, status, shifted_flag);
    else
        chol_inv_block_t<8>(G, ldg, c, P, ldp, status, shifted_flag);
}

}  // namespace bks
