// Eigen-decomposition of the small symmetric PSD matrix M = Q^T A A^T Q (Algorithms 1
// and 2, step 5: its top singular vectors are its top eigenvectors) by one-sided
// (Hestenes) Jacobi: X <- M, V <- I; for column pairs (p, q) with alpha = |x_p|^2,
// beta = |x_q|^2, gamma = x_p . x_q, the plane rotation with
// zeta = (beta - alpha) / (2 gamma), t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)),
// c = 1 / sqrt(1 + t^2), s = c t makes x_p, x_q orthogonal; the same rotation is
// applied to V.  At convergence X = M V has orthogonal columns, so
// lambda_j = |x_j| and v_j is the matching eigenvector.
//
// Parallel ordering: the w columns are cut into 2C blocks of b columns held in the
// shared memory of a thread-block cluster of C CTAs (two blocks per CTA).  Each round
// a CTA orthogonalises every column of its first block against every column of its
// second block; between rounds the blocks move round-robin (circle method) through
// distributed shared memory, so every block pair meets once per sweep.  Pairs inside
// a block are handled in the first round of each sweep.  The columns of a CTA's first
// block live in registers (one column per warp) during the cross-block rounds.
#include <cooperative_groups.h>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace bks {

namespace {

constexpr int JW = 16;   // warps per CTA

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Rotation coefficients; returns false when the pair is already orthogonal to tol.
template <typename T>
__device__ __forceinline__ bool rot_coeffs(T alpha, T beta, T gamma, T tol, T& c, T& s) {
    if (gamma == T(0) || !(fabs(gamma) > tol * sqrt(alpha * beta))) return false;
    const T zeta = (beta - alpha) / (T(2) * gamma);
    const T t = copysign(T(1), zeta) / (fabs(zeta) + sqrt(T(1) + zeta * zeta));
    c = T(1) / sqrt(T(1) + t * t);
    s = c * t;
    return true;
}

// Both columns in shared memory (intra-block pairs).
template <typename T, int E>
__device__ bool rotate_smem_pair(T* xp, T* xq, T tol, int lane) {
    T a = 0, b = 0, g = 0;
    T p[E], q[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        p[e] = xp[lane + 32 * e];
        q[e] = xq[lane + 32 * e];
        a = fma(p[e], p[e], a);
        b = fma(q[e], q[e], b);
        g = fma(p[e], q[e], g);
    }
    a = warp_sum(a); b = warp_sum(b); g = warp_sum(g);
    T c, s;
    if (!rot_coeffs(a, b, g, tol, c, s)) return false;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        xp[lane + 32 * e] = c * p[e] - s * q[e];
        xq[lane + 32 * e] = s * p[e] + c * q[e];
    }
    return true;
}

// Circle-method pairing of P (even) players, round s in [0, P-1), pair index i in [0, P/2).
__device__ __forceinline__ void circle_pair(int P, int s, int i, int& a, int& b) {
    if (i == 0) {
        a = P - 1;
        b = s;
    } else {
        a = (s + i) % (P - 1);
        b = (s - i + (P - 1)) % (P - 1);
    }
}

constexpr int MOVE_REGS = 16;   // registers per thread per slot used to move one chunk

// One-sided Jacobi on the columns of X (w x w; column j is row j of the input array).
// Shared-memory layout per CTA: [slot 0..1][col 0..b)[WP].
template <typename T, int E>
__global__ void __launch_bounds__(JW * 32) jacobi_cluster_kernel(
    const T* __restrict__ Xin, int64_t ldx, int w, int b, T* Xout, int64_t ldw, int max_sweeps,
    T tol, int* status, int* sweeps_out) {
    constexpr int WP = 32 * E;
    extern __shared__ unsigned char smem_raw[];
    T* buf = reinterpret_cast<T*>(smem_raw);
    __shared__ int blk_id[2];
    __shared__ int rotated_s;
    __shared__ int flags[2][16];

    cg::cluster_group cluster = cg::this_cluster();
    const int C = int(cluster.num_blocks());
    const int rank = int(cluster.block_rank());
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    auto col = [&](int slot, int j) -> T* { return buf + (size_t(slot) * b + j) * WP; };

    // initial placement: CTA r holds blocks 2r (slot 0) and 2r+1 (slot 1)
    if (tid == 0) {
        blk_id[0] = 2 * rank;
        blk_id[1] = 2 * rank + 1;
    }
    for (int slot = 0; slot < 2; ++slot) {
        const int blk = 2 * rank + slot;
        for (int j = 0; j < b; ++j) {
            const int gc = blk * b + j;
            T* x = col(slot, j);
            for (int l = tid; l < WP; l += blockDim.x)
                x[l] = (gc < w && l < w) ? Xin[int64_t(gc) * ldx + l] : T(0);
        }
    }
    if (tid < 32) flags[tid >> 4][tid & 15] = 0;
    __syncthreads();
    cluster.sync();

    const int P = 2 * C;               // players in the block round robin
    const int bp = b + (b & 1);        // intra-block players (even)
    const int per_slot = b * WP;
    const int chunk = JW * 32 * MOVE_REGS;
    int sweep = 0;
    bool converged = false;
    for (; sweep < max_sweeps && !converged; ++sweep) {
        if (tid == 0) rotated_s = 0;
        __syncthreads();
        bool any = false;
        for (int round = 0; round < P - 1; ++round) {
            if (round == 0) {
                // intra-block pairs of both slots, once per sweep
                for (int s = 0; s < bp - 1; ++s) {
                    for (int u = warp; u < bp; u += JW) {
                        const int slot = u / (bp / 2), i = u % (bp / 2);
                        int a, c2;
                        circle_pair(bp, s, i, a, c2);
                        if (a >= b || c2 >= b) continue;
                        any |= rotate_smem_pair<T, E>(col(slot, a), col(slot, c2), tol, lane);
                    }
                    __syncthreads();
                }
            }
            // cross pairs: warp keeps slot-0 column j in registers for b sub-rounds
            for (int j0 = 0; j0 < b; j0 += JW) {
                const int j = j0 + warp;
                const bool own = j < b;
                T xr[E];
                if (own) {
#pragma unroll
                    for (int e = 0; e < E; ++e) xr[e] = col(0, j)[lane + 32 * e];
                }
                for (int s = 0; s < b; ++s) {
                    if (own) {
                        T* xq = col(1, (j + s) % b);
                        T q[E];
                        T a = 0, bb = 0, g = 0;
#pragma unroll
                        for (int e = 0; e < E; ++e) {
                            q[e] = xq[lane + 32 * e];
                            a = fma(xr[e], xr[e], a);
                            bb = fma(q[e], q[e], bb);
                            g = fma(xr[e], q[e], g);
                        }
                        a = warp_sum(a); bb = warp_sum(bb); g = warp_sum(g);
                        T c, sn;
                        if (rot_coeffs(a, bb, g, tol, c, sn)) {
                            any = true;
#pragma unroll
                            for (int e = 0; e < E; ++e) {
                                const T p = xr[e];
                                xr[e] = c * p - sn * q[e];
                                xq[lane + 32 * e] = sn * p + c * q[e];
                            }
                        }
                    }
                    __syncthreads();
                }
                if (own) {
#pragma unroll
                    for (int e = 0; e < E; ++e) col(0, j)[lane + 32 * e] = xr[e];
                }
                __syncthreads();
            }
            if (C > 1) {
                // circle-method move of whole blocks: top row t_0 fixed; t_i -> top i+1
                // (t_{C-1} -> bottom C-1); b_0 -> top 1; b_i -> bottom i-1.  Incoming
                // blocks are pulled chunk by chunk through registers: read remote,
                // cluster barrier, write local.
                int src_rank[2] = {-1, -1}, src_slot[2] = {0, 0};
                if (rank == 1) { src_rank[0] = 0; src_slot[0] = 1; }
                else if (rank >= 2) { src_rank[0] = rank - 1; src_slot[0] = 0; }
                if (rank == C - 1) { src_rank[1] = C - 1; src_slot[1] = 0; }
                else { src_rank[1] = rank + 1; src_slot[1] = 1; }
                int ids[2] = {0, 0};
                cluster.sync();
                for (int base = 0; base < per_slot; base += chunk) {
                    T reg[2][MOVE_REGS];
                    for (int slot = 0; slot < 2; ++slot) {
                        if (src_rank[slot] < 0) continue;
                        const T* src = cluster.map_shared_rank(buf, src_rank[slot]) +
                                       size_t(src_slot[slot]) * per_slot;
#pragma unroll
                        for (int r = 0; r < MOVE_REGS; ++r) {
                            const int e = base + tid + r * (JW * 32);
                            if (e < per_slot) reg[slot][r] = src[e];
                        }
                        if (base == 0) ids[slot] = cluster.map_shared_rank(blk_id, src_rank[slot])[src_slot[slot]];
                    }
                    cluster.sync();
                    for (int slot = 0; slot < 2; ++slot) {
                        if (src_rank[slot] < 0) continue;
                        T* dst = buf + size_t(slot) * per_slot;
#pragma unroll
                        for (int r = 0; r < MOVE_REGS; ++r) {
                            const int e = base + tid + r * (JW * 32);
                            if (e < per_slot) dst[e] = reg[slot][r];
                        }
                    }
                }
                __syncthreads();
                if (tid == 0) {
                    if (src_rank[0] >= 0) blk_id[0] = ids[0];
                    if (src_rank[1] >= 0) blk_id[1] = ids[1];
                }
                __syncthreads();
            }
        }
        // cluster-wide "did anybody rotate" for this sweep
        if (any) rotated_s = 1;
        __syncthreads();
        const int par = sweep & 1;
        if (tid == 0) cluster.map_shared_rank(&flags[0][0], 0)[par * 16 + rank] = rotated_s;
        cluster.sync();
        int tot = 0;
        {
            const int* f0 = cluster.map_shared_rank(&flags[0][0], 0);
            for (int r = 0; r < C; ++r) tot |= f0[par * 16 + r];
        }
        cluster.sync();
        if (rank == 0 && tid < 16) flags[par][tid] = 0;
        converged = (tot == 0);
    }
    if (!converged && tid == 0 && rank == 0) atomicOr(status, ST_NOT_CONVERGED);
    if (tid == 0 && rank == 0) *sweeps_out = sweep;
    // write back in original column order
    for (int slot = 0; slot < 2; ++slot) {
        const int blk = blk_id[slot];
        for (int j = 0; j < b; ++j) {
            const int gc = blk * b + j;
            if (gc >= w) continue;
            const T* x = col(slot, j);
            for (int l = tid; l < w; l += blockDim.x) Xout[int64_t(gc) * ldw + l] = x[l];
        }
    }
    cluster.sync();   // keep shared memory alive until remote readers are done
}

// sv_j = |x_j| (FP64 accumulation) and a descending order (ties: lower index first).
template <typename T>
__global__ void eig_rank_kernel(const T* X, int64_t ldw, int w, T* lam, int* order, T* nrm) {
    extern __shared__ double lsh[];
    const int tid = threadIdx.x;
    for (int j = tid; j < w; j += blockDim.x) {
        double s = 0.0;
        for (int l = 0; l < w; ++l) {
            const double v = double(X[int64_t(j) * ldw + l]);
            s += v * v;
        }
        // NaN sorts last, so the ranks below always form a permutation of 0..w-1
        const double v = sqrt(s);
        lsh[j] = isnan(v) ? -1.0 : v;
        nrm[j] = T(v);
    }
    __syncthreads();
    for (int j = tid; j < w; j += blockDim.x) {
        const double lj = lsh[j];
        int r = 0;
        for (int i = 0; i < w; ++i) {
            const double li = lsh[i];
            r += (li > lj) || (li == lj && i < j);
        }
        lam[r] = T(lj);
        order[r] = j;
    }
}

// Vt row r = x_{order[r]} / |x_{order[r]}| (rows of X are its columns).
template <typename T>
__global__ void eig_gather_kernel(const T* X, int64_t ldw, int w, const int* order, const T* nrm,
                                  T* Vt, int64_t ldv) {
    const int r = blockIdx.x;
    int j = order[r];
    if (j < 0 || j >= w) j = r;   // defensive: order is a permutation of 0..w-1
    const T nj = nrm[j];
    const T inv = (nj > T(0) && isfinite(nj)) ? T(1) / nj : T(0);
    for (int l = threadIdx.x; l < w; l += blockDim.x)
        Vt[int64_t(r) * ldv + l] = X[int64_t(j) * ldw + l] * inv;
}

template <typename T, int E>
cudaError_t launch_cluster(cudaStream_t st, int C, size_t smem, const T* Xin, int64_t ldx, int w,
                           int b, T* X, int64_t ldw, int max_sweeps, T tol, int* status,
                           int* sweeps) {
    auto kern = jacobi_cluster_kernel<T, E>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    if (C > 8) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(C), 1, 1);
    cfg.blockDim = dim3(JW * 32, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = unsigned(C);
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, Xin, ldx, w, b, X, ldw, max_sweeps, tol, status, sweeps);
}

}  // namespace

// Plan: cluster size C (power of two <= 16), block width b = ceil(w / 2C) and register
// tile E (elements per lane per column, WP = 32 E >= w).  Returns false when w is too
// large for this solver (shared memory per CTA would exceed 200 KB).
bool jacobi_plan(int w, int elem_bytes, int& C, int& b, int& E, size_t& smem) {
    static const int Es[] = {1, 2, 4, 8, 12, 16, 24, 32};
    E = 0;
    for (int e : Es)
        if (32 * e >= w) { E = e; break; }
    if (E == 0) return false;
    C = 1;
    while (C < 16 && w / (2 * C) >= 16) C *= 2;   // about 16 columns per block
    for (;; C *= 2) {
        b = (w + 2 * C - 1) / (2 * C);
        smem = size_t(2) * b * 32 * E * elem_bytes;
        if (smem <= 200 * 1024) return true;
        if (C >= 16) return false;
    }
}

// One-sided Jacobi on X (w x w, column j given as row j of Xin).  The solver passes
// X = R^T with R^T R = M, so the converged columns are U Sigma with U the eigenvectors
// of M and Sigma its square-root eigenvalues; for a PSD X = M the column norms are the
// eigenvalues themselves.  On return lam[0..w) holds the column norms in descending
// order, nrm[j] the norm of column j, and Vt row i the matching normalised column.
template <typename T>
void sym_eig(Exec& ex, int w, const T* Xin, int64_t ldx, T* X, int64_t ldw, T* lam, T* nrm,
             T* Vt, int64_t ldv, int* order, int max_sweeps, double tol, int* sweeps_dev) {
    int C, b, E;
    size_t smem;
    if (!jacobi_plan(w, int(sizeof(T)), C, b, E, smem)) {
        cudaMemsetAsync(sweeps_dev, 0xff, sizeof(int), ex.stream);
        return;
    }
    const T ttol = T(tol > 0 ? tol : 4.0 * sqrt(double(w)) * (sizeof(T) == 8 ? 1.1102230246251565e-16
                                                                            : 5.960464477539063e-08));
    cudaError_t err = cudaErrorInvalidValue;
#define BKS_JAC(EE) \
    case EE: err = launch_cluster<T, EE>(ex.stream, C, smem, Xin, ldx, w, b, X, ldw, max_sweeps, ttol, ex.status, sweeps_dev); break;
    switch (E) {
        BKS_JAC(1) BKS_JAC(2) BKS_JAC(4) BKS_JAC(8) BKS_JAC(12) BKS_JAC(16) BKS_JAC(24) BKS_JAC(32)
    }
#undef BKS_JAC
    ex.launches++;
    if (err != cudaSuccess) {
        cudaGetLastError();
        cudaMemsetAsync(sweeps_dev, 0xff, sizeof(int), ex.stream);   // reported as -1 sweeps
        return;
    }
    const size_t lsmem = size_t(w) * sizeof(double);
    if (lsmem > 48 * 1024)
        cudaFuncSetAttribute(eig_rank_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(lsmem));
    eig_rank_kernel<T><<<1, 1024, lsmem, ex.stream>>>(X, ldw, w, lam, order, nrm);
    eig_gather_kernel<T><<<w, 128, 0, ex.stream>>>(X, ldw, w, order, nrm, Vt, ldv);
    ex.launches += 2;
}

template void sym_eig<float>(Exec&, int, const float*, int64_t, float*, int64_t, float*, float*,
                             float*, int64_t, int*, int, double, int*);
template void sym_eig<double>(Exec&, int, const double*, int64_t, double*, int64_t, double*,
                              double*, double*, int64_t, int*, int, double, int*);

}  // namespace bks
