// Differentiating Sigma_k and A_k = Z Z^T A with respect to A from the Ritz triplets of a
// solve (the method itself is not differentiated, Secs. 1-4 define only the forward
// computation).  With the w Ritz triplets (u_a, s_a, v_a) of the Krylov space, upstream
// gradients g (k) for Sigma_k and G (n x d) for A_k, M[a][b] = u_a^T G v_b and
// lambda = s^2:
//   dA = U_k diag(g) V_k^T + U_k (U_k^T G)
//        + sum_{i <= k < j <= w} c_ij (s_i u_j v_i^T + s_j u_i v_j^T)
//        + (G V_k - U_w (U_w^T G V_k)) V_k^T,
//   c_ij = (s_i M[j][i] + s_j M[i][j]) / (lambda_i - lambda_j)   (0 when the gap is
//          below tau lambda_1).
// The terms are gathered as dA = U_w X V_w^T + (G V_k) V_k^T + U_k (U_w^T G)_{:k}: one w x w
// coefficient matrix X, two thin products with G and one GEMM that writes dA.  It is exact when the Krylov space holds
// range(A) (w >= rank A); otherwise the directions outside it are taken as singular
// values 0, which is what the complement term accounts for.
#include <cstring>
#include <string>

#include "../../include/bks.h"
#include "common.cuh"
#include "ctx.cuh"

namespace bks {
namespace {

template <typename T>
__global__ void backward_coef_kernel(const T* __restrict__ M, const T* __restrict__ s, const T* __restrict__ g,
                                     int k, int w, double tau, int has_G, T* __restrict__ X) {
    const double lam1 = double(s[0]) * double(s[0]);
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < w * w; e += gridDim.x * blockDim.x) {
        const int a = e / w, b = e % w;
        double x = 0.0;
        if (a == b && a < k && g != nullptr) x += double(g[a]);
        if (has_G) {
            int i = -1, j = -1;
            if (b < k && a >= k) { i = b; j = a; }   // X[j][i] += c_ij s_i
            if (a < k && b >= k) { i = a; j = b; }   // X[i][j] += c_ij s_j
            if (i >= 0) {
                const double si = double(s[i]), sj = double(s[j]);
                const double gap = si * si - sj * sj;
                if (gap > tau * lam1) {
                    const double c = (si * double(M[j * w + i]) + sj * double(M[i * w + j])) / gap;
                    x += (b < k) ? c * si : c * sj;
                }
            }
            if (b < k) x -= double(M[a * w + b]);   // complement: - U_w (U_w^T G V_k)
        }
        X[e] = T(x);
    }
}

// Vs[a][b] = s[a] V[b][a] (r x d)
template <typename T>
__global__ void scale_rows_kernel(const T* __restrict__ V, int64_t ldv, const T* __restrict__ s, int r, int64_t d,
                                  T* __restrict__ Vs) {
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < int64_t(r) * d;
         e += int64_t(gridDim.x) * blockDim.x) {
        const int64_t a = e / d, b = e % d;
        Vs[e] = s[a] * V[b * ldv + a];
    }
}

struct Arena2 {
    size_t off = 0;
    size_t take(size_t bytes) {
        const size_t o = off;
        off += (bytes + 255) / 256 * 256;
        return o;
    }
};

template <typename T>
GemmDesc desc(int64_t M, int64_t N, int64_t K, const T* X, int64_t ldx, const T* Y, int64_t ldy, bool y_kmajor,
              T* out, int64_t ldo, double beta) {
    GemmDesc g{};
    g.M = M; g.N = N; g.K = K;
    g.X = X; g.ldx = ldx; g.Y = Y; g.ldy = ldy;
    g.y_kmajor = y_kmajor;
    g.y_dtype = sizeof(T) == 8 ? BKS_F64 : BKS_F32;
    g.out = out; g.ldo = ldo;
    g.alpha = 1.0; g.beta = beta;
    return g;
}

// Workspace of backward_impl (byte offsets), laid out by backward_layout.
struct BwdLayout {
    int64_t ldn, ldd, Kt;
    size_t Vt, Ut, GVt, UtG, M, X, L, R, xh, xl, tpart, part, stat, total;
    int64_t tcap, cap;
};

BwdLayout backward_layout(int64_t n, int64_t d, int k, int w, size_t tb, int sms) {
    BwdLayout L{};
    L.ldn = round_up(n, 32);
    L.ldd = round_up(d, 32);
    L.Kt = w + 2 * int64_t(k);
    Arena2 a;
    L.Vt = a.take(size_t(w) * L.ldd * tb);
    L.Ut = a.take(size_t(w) * L.ldn * tb);
    L.GVt = a.take(size_t(w) * L.ldn * tb);
    L.UtG = a.take(size_t(w) * L.ldd * tb);
    L.M = a.take(size_t(w) * w * tb);
    L.X = a.take(size_t(w) * w * tb);
    L.L = a.take(size_t(n) * L.Kt * tb);
    L.R = a.take(size_t(L.Kt) * d * tb);
    const int64_t ldmax = L.ldn > L.ldd ? L.ldn : L.ldd;
    L.xh = a.take(tb == 4 ? size_t(w) * ldmax * 4 : 0);
    L.xl = a.take(tb == 4 ? size_t(w) * ldmax * 4 : 0);
    L.tcap = tb == 4 ? tc_partial_floats(n, d, w, sms) : 0;
    L.tpart = a.take(size_t(L.tcap) * 4);
    L.cap = 0;
    for (int64_t e : {gemm_partial_elems(w, n, d, sms), gemm_partial_elems(w, d, n, sms),
                      gemm_partial_elems(w, w, d, sms), gemm_partial_elems(w, d, w, sms),
                      gemm_partial_elems(n, d, L.Kt, sms)})
        if (e > L.cap) L.cap = e;
    L.part = a.take(size_t(L.cap) * 8);
    L.stat = a.take(16);
    L.total = a.off;
    return L;
}

// dA = [U_w | G V_k | U_k] [X V_w^T ; V_k^T ; (U_w^T G)_{:k}]: one GEMM writes dA once.  The
// two passes over G (G V_w and U_w^T G, the only products with an n x d operand besides
// the output) run on the tensor cores (3xTF32) on the FP32 path when the operands meet
// the TMA alignment rules, else on the CUDA cores.
template <typename T>
void backward_impl(Exec& ex, int64_t n, int64_t d, int k, int w, const T* U, const T* s, const T* V, const T* g,
                   const T* G, T* dA, double tau, char* base, const BwdLayout& Ly) {
    T* Vt = reinterpret_cast<T*>(base + Ly.Vt);
    T* Ut = reinterpret_cast<T*>(base + Ly.Ut);
    T* GVt = reinterpret_cast<T*>(base + Ly.GVt);
    T* UtG = reinterpret_cast<T*>(base + Ly.UtG);
    T* M = reinterpret_cast<T*>(base + Ly.M);
    T* X = reinterpret_cast<T*>(base + Ly.X);
    T* Lm = reinterpret_cast<T*>(base + Ly.L);
    T* Rm = reinterpret_cast<T*>(base + Ly.R);
    double* part = reinterpret_cast<double*>(base + Ly.part);
    const int64_t cap = Ly.cap, ldn = Ly.ldn, ldd = Ly.ldd, Kt = Ly.Kt;
    const int dt = sizeof(T) == 8 ? BKS_F64 : BKS_F32;
    transpose_in<T>(ex, V, dt, d, w, w, Vt, ldd);   // V_w^T (w x d)
    if (G != nullptr) {
        transpose_in<T>(ex, U, dt, n, w, w, Ut, ldn);   // U_w^T (w x n)
        bool tc = false;
        if (sizeof(T) == 4) {
            float* xh = reinterpret_cast<float*>(base + Ly.xh);
            float* xl = reinterpret_cast<float*>(base + Ly.xl);
            float* tp = reinterpret_cast<float*>(base + Ly.tpart);
            const float* Gf = reinterpret_cast<const float*>(G);
            tc = tc_product_f32(ex, Gf, n, d, d, false, w, reinterpret_cast<const float*>(Vt), ldd,
                                reinterpret_cast<float*>(GVt), ldn, xh, xl, tp, Ly.tcap) &&
                 tc_product_f32(ex, Gf, n, d, d, true, w, reinterpret_cast<const float*>(Ut), ldn,
                                reinterpret_cast<float*>(UtG), ldd, xh, xl, tp, Ly.tcap);
        }
        if (!tc) {
            gemm_simt<T>(ex, desc<T>(w, n, d, Vt, ldd, G, d, true, GVt, ldn, 0.0), part, cap);   // (G V_w)^T
            gemm_simt<T>(ex, desc<T>(w, d, n, Ut, ldn, G, d, false, UtG, ldd, 0.0), part, cap);  // U_w^T G
        }
        gemm_simt<T>(ex, desc<T>(w, w, d, UtG, ldd, Vt, ldd, true, M, w, 0.0), part, cap);      // U_w^T G V_w
    }
    backward_coef_kernel<T><<<(w * w + 255) / 256 < 1024 ? (w * w + 255) / 256 : 1024, 256, 0, ex.stream>>>(
        M, s, g, k, w, tau, G != nullptr ? 1 : 0, X);
    ex.launches++;
    const int64_t kt = G != nullptr ? Kt : w;   // columns of L in use
    // L = [U_w | (G V_k) | U_k] (n x Kt), R = [X V_w^T ; V_k^T ; (U_w^T G)_{:k}] (Kt x d)
    cudaMemcpy2DAsync(Lm, size_t(Kt) * sizeof(T), U, size_t(w) * sizeof(T), size_t(w) * sizeof(T), size_t(n),
                      cudaMemcpyDeviceToDevice, ex.stream);
    gemm_simt<T>(ex, desc<T>(w, d, w, X, w, Vt, ldd, false, Rm, d, 0.0), part, cap);   // X V_w^T
    if (G != nullptr) {
        transpose_in<T>(ex, GVt, dt, k, n, ldn, Lm + w, Kt);                       // G V_k
        cudaMemcpy2DAsync(Lm + w + k, size_t(Kt) * sizeof(T), U, size_t(w) * sizeof(T), size_t(k) * sizeof(T),
                          size_t(n), cudaMemcpyDeviceToDevice, ex.stream);          // U_k
        cudaMemcpy2DAsync(Rm + int64_t(w) * d, size_t(d) * sizeof(T), Vt, size_t(ldd) * sizeof(T),
                          size_t(d) * sizeof(T), size_t(k), cudaMemcpyDeviceToDevice, ex.stream);   // V_k^T
        cudaMemcpy2DAsync(Rm + int64_t(w + k) * d, size_t(d) * sizeof(T), UtG, size_t(ldd) * sizeof(T),
                          size_t(d) * sizeof(T), size_t(k), cudaMemcpyDeviceToDevice, ex.stream);   // (U^T G)_{:k}
    }
    gemm_simt<T>(ex, desc<T>(n, d, kt, Lm, Kt, Rm, d, false, dA, d, 0.0), part, cap);
}

}  // namespace
}  // namespace bks

using namespace bks;

extern "C" {

int bks_krylov_width(int64_t n, int64_t d, int k, int q, int method) {
    if (k < 1 || q < 0 || n < 1 || d < 1) return 0;
    if (method != 0) return k;
    const int64_t mn = n < d ? n : d;
    int64_t qe = q, cap = mn / k - 1;
    if (qe > cap) qe = cap;
    if (qe < 0) qe = 0;
    return int(int64_t(k) * (qe + 1));
}

bks_status bks_backward(bks_ctx* ctx, int dtype, int64_t n, int64_t d, int k, int w, const void* U,
                        const void* sigma, const void* V, const void* g_sigma, const void* G, void* dA,
                        double gap_tau) {
    if (ctx == nullptr) return BKS_ERR_INVALID_ARG;
    if ((dtype != BKS_F32 && dtype != BKS_F64) || n < 1 || d < 1 || k < 1 || w < k || U == nullptr ||
        sigma == nullptr || V == nullptr || dA == nullptr || (g_sigma == nullptr && G == nullptr))
        return ctx_fail(ctx, BKS_ERR_INVALID_ARG, "bad bks_backward arguments");
    const size_t tb = dtype == BKS_F64 ? 8 : 4;
    const int sms = ctx_num_sms(ctx);
    const BwdLayout Ly = backward_layout(n, d, k, w, tb, sms);
    CtxInfo ci;
    bks_status s = ctx_workspace(ctx, Ly.total, &ci);
    if (s != BKS_OK) return s;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(ci.device);
    char* base = static_cast<char*>(ci.ws);
    cudaStream_t stream = ci.stream;
    Exec ex;
    ex.stream = stream;
    ex.num_sms = sms;
    ex.status = reinterpret_cast<int*>(base + Ly.stat);
    cudaMemsetAsync(ex.status, 0, 16, stream);
    const double tau = gap_tau > 0 ? gap_tau : (dtype == BKS_F64 ? 1e-10 : 1e-6);
    if (dtype == BKS_F64)
        backward_impl<double>(ex, n, d, k, w, static_cast<const double*>(U), static_cast<const double*>(sigma),
                              static_cast<const double*>(V), static_cast<const double*>(g_sigma),
                              static_cast<const double*>(G), static_cast<double*>(dA), tau, base, Ly);
    else
        backward_impl<float>(ex, n, d, k, w, static_cast<const float*>(U), static_cast<const float*>(sigma),
                             static_cast<const float*>(V), static_cast<const float*>(g_sigma),
                             static_cast<const float*>(G), static_cast<float*>(dA), tau, base, Ly);
    cudaError_t e = cudaStreamSynchronize(stream);
    if (e == cudaSuccess) e = cudaGetLastError();
    int status = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&status, ex.status, sizeof(int), cudaMemcpyDeviceToHost);
    cudaSetDevice(prev);
    if (e != cudaSuccess) return ctx_fail(ctx, BKS_ERR_CUDA, cudaGetErrorString(e));
    if (status & ST_TIMEOUT) return ctx_fail(ctx, BKS_ERR_TIMEOUT, "a tensor-core pipeline wait timed out");
    return BKS_OK;
}

bks_status bks_low_rank(bks_ctx* ctx, int dtype, int64_t n, int64_t d, int r, const void* U, int64_t ldu,
                        const void* sigma, const void* V, int64_t ldv, void* out) {
    if (ctx == nullptr) return BKS_ERR_INVALID_ARG;
    if ((dtype != BKS_F32 && dtype != BKS_F64) || n < 1 || d < 1 || r < 1 || U == nullptr || sigma == nullptr ||
        V == nullptr || out == nullptr || ldu < r || ldv < r)
        return ctx_fail(ctx, BKS_ERR_INVALID_ARG, "bad bks_low_rank arguments");
    const size_t tb = dtype == BKS_F64 ? 8 : 4;
    const int sms = ctx_num_sms(ctx);
    const int64_t cap = gemm_partial_elems(n, d, r, sms);
    Arena2 a;
    const size_t o_vs = a.take(size_t(r) * d * tb), o_part = a.take(size_t(cap) * 8);
    CtxInfo ci;
    bks_status s = ctx_workspace(ctx, a.off, &ci);
    if (s != BKS_OK) return s;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(ci.device);
    char* base = static_cast<char*>(ci.ws);
    cudaStream_t stream = ci.stream;
    Exec ex;
    ex.stream = stream;
    ex.num_sms = sms;
    const int blocks = int((int64_t(r) * d + 255) / 256 < 4096 ? (int64_t(r) * d + 255) / 256 : 4096);
    if (dtype == BKS_F64) {
        double* vs = reinterpret_cast<double*>(base + o_vs);
        scale_rows_kernel<double><<<blocks, 256, 0, stream>>>(static_cast<const double*>(V), ldv,
                                                             static_cast<const double*>(sigma), r, d, vs);
        gemm_simt<double>(ex, desc<double>(n, d, r, static_cast<const double*>(U), ldu, vs, d, false,
                                           static_cast<double*>(out), d, 0.0),
                          reinterpret_cast<double*>(base + o_part), cap);
    } else {
        float* vs = reinterpret_cast<float*>(base + o_vs);
        scale_rows_kernel<float><<<blocks, 256, 0, stream>>>(static_cast<const float*>(V), ldv,
                                                            static_cast<const float*>(sigma), r, d, vs);
        gemm_simt<float>(ex, desc<float>(n, d, r, static_cast<const float*>(U), ldu, vs, d, false,
                                         static_cast<float*>(out), d, 0.0),
                         reinterpret_cast<double*>(base + o_part), cap);
    }
    cudaError_t e = cudaStreamSynchronize(stream);
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaSetDevice(prev);
    if (e != cudaSuccess) return ctx_fail(ctx, BKS_ERR_CUDA, cudaGetErrorString(e));
    return BKS_OK;
}

}  // extern "C"
