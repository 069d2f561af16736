// Eigen-decomposition of the small symmetric PSD matrix M = Q^T A A^T Q (Algorithms 1
// and 2, step 5: its top singular vectors are its top eigenvectors) by one-sided
// (Hestenes) Jacobi on the columns of X: for a column pair (p, q) with
// alpha = |x_p|^2, beta = |x_q|^2, gamma = x_p . x_q, the plane rotation with
// zeta = (beta - alpha) / (2 gamma), t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)),
// c = 1 / sqrt(1 + t^2), s = c t makes x_p, x_q orthogonal, and afterwards
// |x_p|^2 = alpha - t gamma, |x_q|^2 = beta + t gamma.  The solver passes X = R^T with
// R^T R = M (preconditioned Jacobi: no V is accumulated; the converged columns are
// U Sigma with U the eigenvectors of M); for a PSD X = M the converged column norms
// are its eigenvalues.
//
// Parallel ordering: the w columns are cut into 2C blocks of b columns held in the
// shared memory of a thread-block cluster of C CTAs (two blocks per CTA).  Each round
// a CTA orthogonalises every column of its first block against every column of its
// second block; between rounds the blocks move round-robin (circle method) through
// distributed shared memory, so every block pair meets once per sweep.  Pairs inside
// a block are handled in the first round of each sweep.  During the cross-block
// rounds a warp keeps one first-block column in registers.
//
// Two pair engines share this structure: a generic one (FP64 path) that recomputes
// the three dot products per pair, and an FP32 one that uses paired FP32 arithmetic
// (two lanes of data per instruction) and carries the column norms, recomputed
// exactly at the start of every round, so each pair needs a single reduction.
#include <cooperative_groups.h>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace bks {

namespace {

constexpr int JW = 16;          // warps per CTA
constexpr int MOVE_REGS = 16;   // registers per thread per slot used to move one chunk

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Rotation coefficients; returns false when the pair is already orthogonal to tol.
// With x = beta - alpha, y = 2 gamma and r = sqrt(x^2 + y^2), the smaller root of
// t^2 + 2 (x / y) t - 1 = 0 is t = sign(x) y / (|x| + r) (no cancellation; x = 0 gives
// t = sign(y)), then
// c = 1 / sqrt(1 + t^2), s = c t.  The threshold |gamma| > tol sqrt(alpha beta) is
// tested squared.
template <typename T>
__device__ __forceinline__ bool rot_coeffs(T alpha, T beta, T gamma, T tol, T& c, T& s, T& t) {
    if (!(gamma * gamma > tol * tol * (alpha * beta)) || gamma == T(0)) return false;
    const T x = beta - alpha, y = T(2) * gamma;
    const T r = sqrt(fma(x, x, y * y));
    t = (x >= T(0) ? y : -y) / (fabs(x) + r);   // sign(x) y / (|x| + r)
    c = T(1) / sqrt(fma(t, t, T(1)));
    s = c * t;
    return true;
}
// FP32: the same formulas on the special-function unit (rsqrt and reciprocal
// approximations, within a few ulp: the rotation stays orthogonal to rounding level).
template <>
__device__ __forceinline__ bool rot_coeffs<float>(float alpha, float beta, float gamma, float tol, float& c,
                                                  float& s, float& t) {
    if (!(gamma * gamma > tol * tol * (alpha * beta)) || gamma == 0.f) return false;
    const float x = beta - alpha, y = 2.f * gamma;
    const float r2 = fmaf(x, x, y * y);
    const float r = r2 * rsqrtf(r2);
    t = (x >= 0.f ? y : -y) * __frcp_rn(fabsf(x) + r);   // sign(x) y / (|x| + r)
    c = rsqrtf(fmaf(t, t, 1.f));
    s = c * t;
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

// Per-CTA state in shared memory: two slots of b columns, WP values each (four when the
// block moves are double-buffered: parity par selects the pair in use).
template <typename T>
struct Blocks {
    T* buf;
    int b, WP;
    int par;
    __device__ T* col(int slot, int j) const { return buf + (size_t(par * 2 + slot) * b + j) * WP; }
};

// Circle-method move of whole blocks between CTAs: top row t_0 stays; t_i -> top i+1
// (t_{C-1} -> bottom C-1); b_0 -> top 1; b_i -> bottom i-1.  Incoming blocks are pulled
// chunk by chunk through registers: read remote, cluster barrier, write local.
template <typename T>
__device__ void move_blocks(cg::cluster_group& cluster, T* buf, int per_slot, int* blk_id,
                            int rank, int C, int tid) {
    int src_rank[2] = {-1, -1}, src_slot[2] = {0, 0};
    if (rank == 1) { src_rank[0] = 0; src_slot[0] = 1; }
    else if (rank >= 2) { src_rank[0] = rank - 1; src_slot[0] = 0; }
    if (rank == C - 1) { src_rank[1] = C - 1; src_slot[1] = 0; }
    else { src_rank[1] = rank + 1; src_slot[1] = 1; }
    int ids[2] = {0, 0};
    const int chunk = JW * 32 * MOVE_REGS;
    cluster.sync();
    for (int base = 0; base < per_slot; base += chunk) {
        T reg[2][MOVE_REGS];
        for (int slot = 0; slot < 2; ++slot) {
            if (src_rank[slot] < 0) continue;
            const T* src = cluster.map_shared_rank(buf, src_rank[slot]) + size_t(src_slot[slot]) * per_slot;
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

// The same circle-method move, pushed: each CTA writes its two blocks into the other
// parity of the receiving CTAs' shared memory (DSMEM stores), then one cluster barrier
// makes them visible and every CTA switches parity.  The receivers' other parity was
// last used in the previous round, which the previous barrier closed.
template <typename T>
__device__ void push_blocks(cg::cluster_group& cluster, Blocks<T>& B, int* blk_id, int rank, int C, int tid) {
    int dr[2], ds[2];
    if (rank == 0) { dr[0] = 0; ds[0] = 0; }
    else if (rank <= C - 2) { dr[0] = rank + 1; ds[0] = 0; }
    else { dr[0] = C - 1; ds[0] = 1; }
    if (rank == 0) { dr[1] = 1; ds[1] = 0; }
    else { dr[1] = rank - 1; ds[1] = 1; }
    __syncthreads();
    const int np = B.par ^ 1;
    const size_t per_slot = size_t(B.b) * B.WP;
    for (int slot = 0; slot < 2; ++slot) {
        const T* src = B.col(slot, 0);
        T* dst = cluster.map_shared_rank(B.buf, dr[slot]) + size_t(np * 2 + ds[slot]) * per_slot;
        if (sizeof(T) == 4) {
            const float4* s4 = reinterpret_cast<const float4*>(src);
            float4* d4 = reinterpret_cast<float4*>(dst);
            for (size_t e = tid; e < per_slot / 4; e += blockDim.x) d4[e] = s4[e];
        } else {
            const double2* s2 = reinterpret_cast<const double2*>(src);
            double2* d2 = reinterpret_cast<double2*>(dst);
            for (size_t e = tid; e < per_slot / 2; e += blockDim.x) d2[e] = s2[e];
        }
        if (tid == 0) cluster.map_shared_rank(blk_id, dr[slot])[np * 2 + ds[slot]] = blk_id[B.par * 2 + slot];
    }
    cluster.sync();
    B.par = np;
}

// Cluster-wide OR of "this CTA rotated during the sweep"; flags live in CTA 0 and
// alternate between two rows so a row is cleared two sweeps before its next use.
__device__ bool cluster_any(cg::cluster_group& cluster, int (*flags)[16], int par, int rank, int C,
                            int tid, int mine) {
    if (tid == 0) cluster.map_shared_rank(&flags[0][0], 0)[par * 16 + rank] = mine;
    cluster.sync();
    int tot = 0;
    const int* f0 = cluster.map_shared_rank(&flags[0][0], 0);
    for (int r = 0; r < C; ++r) tot |= f0[par * 16 + r];
    cluster.sync();
    if (rank == 0 && tid < 16) flags[par][tid] = 0;
    return tot != 0;
}

// ------------------------------------------------------------ generic pair engine
template <typename T, int E>
struct GenericEngine {
    static constexpr bool kNorms = false;
    // both columns in shared memory
    __device__ static bool pair_smem(T* xp, T* xq, T* np, T* nq, T tol, int lane) {
        (void)np; (void)nq;
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
        T c, s, t;
        if (!rot_coeffs(a, b, g, tol, c, s, t)) return false;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            xp[lane + 32 * e] = c * p[e] - s * q[e];
            xq[lane + 32 * e] = s * p[e] + c * q[e];
        }
        return true;
    }
    struct Reg { T x[E]; T a; };
    __device__ static void load(Reg& r, const T* xp, const T* np, int lane) {
        (void)np;
#pragma unroll
        for (int e = 0; e < E; ++e) r.x[e] = xp[lane + 32 * e];
    }
    __device__ static void store(const Reg& r, T* xp, T* np, int lane) {
        (void)np;
#pragma unroll
        for (int e = 0; e < E; ++e) xp[lane + 32 * e] = r.x[e];
    }
    // first column in registers, second in shared memory
    __device__ static bool pair_reg(Reg& r, T* xq, T* nq, T tol, int lane) {
        (void)nq;
        T q[E];
        T a = 0, bb = 0, g = 0;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            q[e] = xq[lane + 32 * e];
            a = fma(r.x[e], r.x[e], a);
            bb = fma(q[e], q[e], bb);
            g = fma(r.x[e], q[e], g);
        }
        a = warp_sum(a); bb = warp_sum(bb); g = warp_sum(g);
        T c, sn, t;
        if (!rot_coeffs(a, bb, g, tol, c, sn, t)) return false;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const T p = r.x[e];
            r.x[e] = c * p - sn * q[e];
            xq[lane + 32 * e] = sn * p + c * q[e];
        }
        return true;
    }
};

// -------------------------------------------------------- paired-FP32 pair engine
// Lane l holds the float2 elements l + 32 i (i < E/2) of a column, i.e. the value
// pairs (2l + 64 i, 2l + 64 i + 1): one 64-bit shared-memory access per pair.
template <int E>
struct F32x2Engine {
    static constexpr bool kNorms = true;
    static constexpr int H = E / 2;
    __device__ static float dot(const float2* p, const float2* q) {
        float2 g = make_float2(0.f, 0.f);
#pragma unroll
        for (int i = 0; i < H; ++i) g = __ffma2_rn(p[i], q[i], g);
        return warp_sum(g.x + g.y);
    }
    __device__ static void rotate(float2* p, float2* q, float c, float s) {
        const float2 c2 = make_float2(c, c), s2 = make_float2(s, s), ns2 = make_float2(-s, -s);
#pragma unroll
        for (int i = 0; i < H; ++i) {
            const float2 pi = p[i];
            p[i] = __ffma2_rn(ns2, q[i], __fmul2_rn(c2, pi));
            q[i] = __ffma2_rn(s2, pi, __fmul2_rn(c2, q[i]));
        }
    }
    __device__ static bool pair_smem(float* xp, float* xq, float* np, float* nq, float tol, int lane) {
        float2 p[H], q[H];
        const float2* p2 = reinterpret_cast<const float2*>(xp);
        const float2* q2 = reinterpret_cast<const float2*>(xq);
#pragma unroll
        for (int i = 0; i < H; ++i) { p[i] = p2[lane + 32 * i]; q[i] = q2[lane + 32 * i]; }
        const float g = dot(p, q);
        const float a = *np, b = *nq;
        float c, s, t;
        if (!rot_coeffs(a, b, g, tol, c, s, t)) return false;
        rotate(p, q, c, s);
        float2* pw = reinterpret_cast<float2*>(xp);
        float2* qw = reinterpret_cast<float2*>(xq);
#pragma unroll
        for (int i = 0; i < H; ++i) { pw[lane + 32 * i] = p[i]; qw[lane + 32 * i] = q[i]; }
        __syncwarp();
        if (lane == 0) { *np = a - t * g; *nq = b + t * g; }
        return true;
    }
    struct Reg { float2 x[H]; float a; };
    __device__ static void load(Reg& r, const float* xp, const float* np, int lane) {
        const float2* p2 = reinterpret_cast<const float2*>(xp);
#pragma unroll
        for (int i = 0; i < H; ++i) r.x[i] = p2[lane + 32 * i];
        r.a = *np;
    }
    __device__ static void store(const Reg& r, float* xp, float* np, int lane) {
        float2* p2 = reinterpret_cast<float2*>(xp);
#pragma unroll
        for (int i = 0; i < H; ++i) p2[lane + 32 * i] = r.x[i];
        if (lane == 0) *np = r.a;
    }
    __device__ static bool pair_reg(Reg& r, float* xq, float* nq, float tol, int lane) {
        float2 q[H];
        const float2* q2 = reinterpret_cast<const float2*>(xq);
#pragma unroll
        for (int i = 0; i < H; ++i) q[i] = q2[lane + 32 * i];
        const float g = dot(r.x, q);
        const float b = *nq;
        float c, s, t;
        if (!rot_coeffs(r.a, b, g, tol, c, s, t)) return false;
        rotate(r.x, q, c, s);
        float2* qw = reinterpret_cast<float2*>(xq);
#pragma unroll
        for (int i = 0; i < H; ++i) qw[lane + 32 * i] = q[i];
        r.a = r.a - t * g;
        __syncwarp();
        if (lane == 0) *nq = b + t * g;
        return true;
    }
};

// Exact squared norms of every column this CTA holds (one warp per column).
template <typename T>
__device__ void recompute_norms(const Blocks<T>& B, T* nrm2, int warp, int lane) {
    for (int u = warp; u < 2 * B.b; u += JW) {
        const T* x = B.col(u / B.b, u % B.b);
        T s = 0;
        for (int l = lane; l < B.WP; l += 32) s = fma(x[l], x[l], s);
        s = warp_sum(s);
        if (lane == 0) nrm2[u] = s;
    }
}

template <typename T, int E, class Eng, bool DB>
__global__ void __launch_bounds__(JW * 32) jacobi_cluster_kernel(
    const T* __restrict__ Xin, int64_t ldx, int w, int b, T* Xout, int64_t ldw, int max_sweeps,
    T tol, int* status, int* sweeps_out) {
    constexpr int WP = 32 * E;
    constexpr int SLOTS = DB ? 4 : 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Blocks<T> B{reinterpret_cast<T*>(smem_raw), b, WP, 0};
    T* nrm2 = B.buf + size_t(SLOTS) * b * WP;   // squared column norms [slot * b + j]
    __shared__ int blk_id[4];                   // [parity * 2 + slot]
    __shared__ int rotated_s;
    __shared__ int flags[2][16];


    cg::cluster_group cluster = cg::this_cluster();
    const int C = int(cluster.num_blocks());
    const int rank = int(cluster.block_rank());
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    // initial placement: CTA r holds blocks 2r (slot 0) and 2r+1 (slot 1)
    if (tid == 0) {
        blk_id[0] = 2 * rank;
        blk_id[1] = 2 * rank + 1;
    }
    for (int slot = 0; slot < 2; ++slot) {
        const int blk = 2 * rank + slot;
        for (int j = 0; j < b; ++j) {
            const int gc = blk * b + j;
            T* x = B.col(slot, j);
            for (int l = tid; l < WP; l += blockDim.x)
                x[l] = (gc < w && l < w) ? Xin[int64_t(gc) * ldx + l] : T(0);
        }
    }
    if (tid < 32) flags[tid >> 4][tid & 15] = 0;
    __syncthreads();
    cluster.sync();

    const int P = 2 * C;               // players in the block round robin
    const int bp = b + (b & 1);        // intra-block players (even)
    int sweep = 0;
    bool converged = false;
    for (; sweep < max_sweeps && !converged; ++sweep) {
        if (tid == 0) rotated_s = 0;
        __syncthreads();
        bool any = false;
        for (int round = 0; round < P - 1; ++round) {
            if (Eng::kNorms) {
                recompute_norms(B, nrm2, warp, lane);
                __syncthreads();
            }
            if (round == 0) {
                // intra-block pairs of both slots, once per sweep
                for (int s = 0; s < bp - 1; ++s) {
                    for (int u = warp; u < bp; u += JW) {
                        const int slot = u / (bp / 2), i = u % (bp / 2);
                        int a, c2;
                        circle_pair(bp, s, i, a, c2);
                        if (a >= b || c2 >= b) continue;
                        any |= Eng::pair_smem(B.col(slot, a), B.col(slot, c2), nrm2 + slot * b + a,
                                              nrm2 + slot * b + c2, tol, lane);
                    }
                    __syncthreads();
                }
            }
            // cross pairs: a warp keeps slot-0 column j in registers for b sub-rounds
            for (int j0 = 0; j0 < b; j0 += JW) {
                const int j = j0 + warp;
                const bool own = j < b;
                typename Eng::Reg r;
                if (own) Eng::load(r, B.col(0, j), nrm2 + j, lane);
                for (int s = 0; s < b; ++s) {
                    if (own) {
                        const int qj = (j + s) % b;
                        any |= Eng::pair_reg(r, B.col(1, qj), nrm2 + b + qj, tol, lane);
                    }
                    __syncthreads();
                }
                if (own) Eng::store(r, B.col(0, j), nrm2 + j, lane);
                __syncthreads();
            }
            if (C > 1) {
                if (DB) push_blocks(cluster, B, blk_id, rank, C, tid);
                else move_blocks(cluster, B.buf, b * WP, blk_id, rank, C, tid);
            }
        }
        if (any) rotated_s = 1;
        __syncthreads();
        converged = !cluster_any(cluster, flags, sweep & 1, rank, C, tid, rotated_s);
    }
    if (!converged && tid == 0 && rank == 0) atomicOr(status, ST_NOT_CONVERGED);
    if (tid == 0 && rank == 0) *sweeps_out = sweep;
    // write back in original column order
    for (int slot = 0; slot < 2; ++slot) {
        const int blk = blk_id[B.par * 2 + slot];
        for (int j = 0; j < b; ++j) {
            const int gc = blk * b + j;
            if (gc >= w) continue;
            const T* x = B.col(slot, j);
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
struct EngineFor { using type = GenericEngine<T, E>; };
template <int E>
struct EngineFor<float, E> { using type = F32x2Engine<E>; };

template <typename T, int E, bool DB>
cudaError_t launch_cluster(cudaStream_t st, int C, size_t smem, const T* Xin, int64_t ldx, int w,
                           int b, T* X, int64_t ldw, int max_sweeps, T tol, int* status,
                           int* sweeps) {
    auto kern = jacobi_cluster_kernel<T, E, typename EngineFor<T, E>::type, DB>;
    cudaError_t e = allow_dynamic_smem(reinterpret_cast<const void*>(kern), smem);
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
// tile E (even: elements per lane per column, WP = 32 E >= w).  Returns false when w is
// too large for this solver (shared memory per CTA would exceed 200 KB).
bool jacobi_plan(int w, int elem_bytes, int& C, int& b, int& E, size_t& smem) {
    static const int Es[] = {2, 4, 8, 12, 16, 24, 32};
    E = 0;
    for (int e : Es)
        if (32 * e >= w) { E = e; break; }
    if (E == 0) return false;
    C = 1;
    while (C < 16 && w / (2 * C) >= 16) C *= 2;   // about 16 columns per block
    for (;; C *= 2) {
        b = (w + 2 * C - 1) / (2 * C);
        smem = (size_t(2) * b * 32 * E + size_t(2) * b) * elem_bytes;
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
    // double-buffered (pushed) block moves when four slots fit in shared memory
    const size_t smem_db = (size_t(4) * b * 32 * E + size_t(2) * b) * sizeof(T);
    const bool db = C > 1 && smem_db <= 200 * 1024;
    if (db) smem = smem_db;
    cudaError_t err = cudaErrorInvalidValue;
#define BKS_JAC(EE)                                                                                          \
    case EE:                                                                                                 \
        err = db ? launch_cluster<T, EE, true>(ex.stream, C, smem, Xin, ldx, w, b, X, ldw, max_sweeps, ttol, \
                                               ex.status, sweeps_dev)                                        \
                 : launch_cluster<T, EE, false>(ex.stream, C, smem, Xin, ldx, w, b, X, ldw, max_sweeps, ttol, \
                                                ex.status, sweeps_dev);                                      \
        break;
    switch (E) {
        BKS_JAC(2) BKS_JAC(4) BKS_JAC(8) BKS_JAC(12) BKS_JAC(16) BKS_JAC(24) BKS_JAC(32)
    }
#undef BKS_JAC
    ex.launches++;
    if (err != cudaSuccess) {
        cudaGetLastError();
        cudaMemsetAsync(sweeps_dev, 0xff, sizeof(int), ex.stream);   // reported as -1 sweeps
        return;
    }
    const size_t lsmem = size_t(w) * sizeof(double);
    if (lsmem > 48 * 1024) allow_dynamic_smem(reinterpret_cast<const void*>(eig_rank_kernel<T>), lsmem);
    eig_rank_kernel<T><<<1, 1024, lsmem, ex.stream>>>(X, ldw, w, lam, order, nrm);
    eig_gather_kernel<T><<<w, 128, 0, ex.stream>>>(X, ldw, w, order, nrm, Vt, ldv);
    ex.launches += 2;
}

template void sym_eig<float>(Exec&, int, const float*, int64_t, float*, int64_t, float*, float*,
                             float*, int64_t, int*, int, double, int*);
template void sym_eig<double>(Exec&, int, const double*, int64_t, double*, int64_t, double*,
                              double*, double*, int64_t, int*, int, double, int*);

}  // namespace bks
