// SIMT tile GEMM used for every contraction whose one side is a thin block:
//   Out = X . Y^T  (y_kmajor: both operands run along the contraction index)
//   Out = X . Y    (!y_kmajor: Y's rows run along the contraction index)
// X is a thin block (M <= a few hundred rows), Y is either the matrix A or another
// thin block.  64 x 128 output tile per CTA, 16-deep K slices staged in shared
// memory, 4 x 8 register tile per thread.  When the output alone cannot fill the
// GPU the contraction is split across CTAs; partial sums are written in FP64 and
// added in a fixed order, so results are deterministic.
#include "common.cuh"

namespace bks {

namespace {
constexpr int BM = 64, BN = 128, BK = 16, NT = 256, TM = 4, TN = 8;

template <typename T, typename TY, bool YK>
__global__ void __launch_bounds__(NT) gemm_tile_kernel(GemmDesc g, int64_t kchunk,
                                                       double* part) {
    __shared__ T Xs[BK][BM + 4];
    __shared__ T Ys[BK][BN + 4];
    const T* X = static_cast<const T*>(g.X);
    const TY* Y = static_cast<const TY*>(g.Y);
    const int tid = threadIdx.x;
    const int tx = tid % 16, ty = tid / 16;
    const int64_t m0 = int64_t(blockIdx.y) * BM, n0 = int64_t(blockIdx.x) * BN;
    const int64_t kb = int64_t(blockIdx.z) * kchunk;
    const int64_t ke = min(g.K, kb + kchunk);

    T acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = T(0);

    for (int64_t k0 = kb; k0 < ke; k0 += BK) {
#pragma unroll
        for (int i = 0; i < (BM * BK) / NT; ++i) {
            const int e = tid + NT * i;
            const int r = e / BK, kk = e % BK;
            const int64_t gm = m0 + r, gk = k0 + kk;
            T v = T(0);
            if (gm < g.M && gk < ke) v = X[gm * g.ldx + gk];
            Xs[kk][r] = v;
        }
        if (YK) {
#pragma unroll
            for (int i = 0; i < (BN * BK) / NT; ++i) {
                const int e = tid + NT * i;
                const int r = e / BK, kk = e % BK;
                const int64_t gn = n0 + r, gk = k0 + kk;
                T v = T(0);
                if (gn < g.N && gk < ke) v = cvt<T>(Y[gn * g.ldy + gk]);
                Ys[kk][r] = v;
            }
        } else {
#pragma unroll
            for (int i = 0; i < (BN * BK) / NT; ++i) {
                const int e = tid + NT * i;
                const int kk = e / BN, c = e % BN;
                const int64_t gn = n0 + c, gk = k0 + kk;
                T v = T(0);
                if (gn < g.N && gk < ke) v = cvt<T>(Y[gk * g.ldy + gn]);
                Ys[kk][c] = v;
            }
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T a[TM], b[TN];
#pragma unroll
            for (int i = 0; i < TM; ++i) a[i] = Xs[kk][ty * TM + i];
#pragma unroll
            for (int j = 0; j < TN; ++j) b[j] = Ys[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }

    if (part != nullptr) {
        double* p = part + int64_t(blockIdx.z) * g.M * g.N;
#pragma unroll
        for (int i = 0; i < TM; ++i) {
            const int64_t m = m0 + ty * TM + i;
            if (m >= g.M) continue;
#pragma unroll
            for (int j = 0; j < TN; ++j) {
                const int64_t n = n0 + tx + 16 * j;
                if (n < g.N) p[m * g.N + n] = double(acc[i][j]);
            }
        }
        return;
    }
    T* out = static_cast<T*>(g.out);
    const T alpha = T(g.alpha), beta = T(g.beta);
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const int64_t m = m0 + ty * TM + i;
        if (m >= g.M) continue;
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            const int64_t n = n0 + tx + 16 * j;
            if (n >= g.N) continue;
            T* o = g.out_transposed ? out + n * g.ldo + m : out + m * g.ldo + n;
            T v = alpha * acc[i][j];
            if (g.beta != 0.0) v = fma(beta, *o, v);
            *o = v;
        }
    }
}

// out[m][n] = alpha * sum_z part[z][m][n] + beta * out[m][n]; sums in FP64, fixed order.
template <typename T>
__global__ void split_reduce_kernel(const double* __restrict__ part, int S, int64_t M, int64_t N,
                                    T* out, int64_t ldo, bool transposed, double alpha,
                                    double beta) {
    const int64_t total = M * N;
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < total;
         e += int64_t(gridDim.x) * blockDim.x) {
        double s = 0.0;
        for (int z = 0; z < S; ++z) s += part[int64_t(z) * total + e];
        const int64_t m = e / N, n = e % N;
        T* o = transposed ? out + n * ldo + m : out + m * ldo + n;
        double v = alpha * s;
        if (beta != 0.0) v += beta * double(*o);
        *o = T(v);
    }
}

int choose_splits(int64_t M, int64_t N, int64_t K, int num_sms) {
    const int64_t tiles = ((M + BM - 1) / BM) * ((N + BN - 1) / BN);
    const int64_t target = 4LL * num_sms;
    if (tiles >= target || K <= 512) return 1;
    int64_t s = (target + tiles - 1) / tiles;
    const int64_t smax = (K + 255) / 256;   // keep >= 256 contraction steps per split
    if (s > smax) s = smax;
    return int(s < 1 ? 1 : s);
}
}  // namespace

int64_t gemm_partial_elems(int64_t M, int64_t N, int64_t K, int num_sms) {
    const int s = choose_splits(M, N, K, num_sms);
    return s > 1 ? int64_t(s) * M * N : 0;
}

template <typename T>
void gemm_simt(Exec& ex, const GemmDesc& g, double* partials, int64_t partial_cap) {
    if (g.M <= 0 || g.N <= 0) return;
    const int64_t total = g.M * g.N;
    int rblocks = int((total + 255) / 256);
    if (rblocks > 8 * ex.num_sms) rblocks = 8 * ex.num_sms;
    auto reduce = [&](const double* part, int S) {
        if (g.out_f64)
            split_reduce_kernel<double><<<rblocks, 256, 0, ex.stream>>>(
                part, S, g.M, g.N, static_cast<double*>(g.out), g.ldo, g.out_transposed, g.alpha,
                g.beta);
        else
            split_reduce_kernel<T><<<rblocks, 256, 0, ex.stream>>>(
                part, S, g.M, g.N, static_cast<T*>(g.out), g.ldo, g.out_transposed, g.alpha, g.beta);
        ex.launches++;
    };
    if (g.K <= 0) {  // empty contraction: Out = beta * Out
        reduce(nullptr, 0);
        return;
    }
    const bool need_part = g.out_f64 && sizeof(T) != sizeof(double);
    int S = choose_splits(g.M, g.N, g.K, ex.num_sms);
    if (need_part && S < 1) S = 1;
    if (S > 1 && (partials == nullptr || int64_t(S) * total > partial_cap)) S = 1;
    int64_t kchunk = (g.K + S - 1) / S;
    kchunk = (kchunk + BK - 1) / BK * BK;
    S = int((g.K + kchunk - 1) / kchunk);
    double* part = (S > 1 || need_part) ? partials : nullptr;
    dim3 grid(unsigned((g.N + BN - 1) / BN), unsigned((g.M + BM - 1) / BM), unsigned(S));
#define BKS_LAUNCH(TY, YK)                                                              \
    gemm_tile_kernel<T, TY, YK><<<grid, NT, 0, ex.stream>>>(g, kchunk, part)
    if (g.y_dtype == 2) {
        if (g.y_kmajor) BKS_LAUNCH(__nv_bfloat16, true); else BKS_LAUNCH(__nv_bfloat16, false);
    } else if (g.y_dtype == 1) {
        if (g.y_kmajor) BKS_LAUNCH(float, true); else BKS_LAUNCH(float, false);
    } else {
        if (g.y_kmajor) BKS_LAUNCH(double, true); else BKS_LAUNCH(double, false);
    }
#undef BKS_LAUNCH
    ex.launches++;
    if (part != nullptr) reduce(part, S);
}

template void gemm_simt<float>(Exec&, const GemmDesc&, double*, int64_t);
template void gemm_simt<double>(Exec&, const GemmDesc&, double*, int64_t);

}  // namespace bks
