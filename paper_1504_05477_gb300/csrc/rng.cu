// Start block Pi ~ N(0,1)^{d x k} (Algorithms 1 and 2, step 1).  The paper names no
// generator; this is SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) feeding
// Box-Muller (1958), counter-based so every element is computed independently:
//   output i of the stream seeded with s = mix(s + (i + 1) * 0x9E3779B97F4A7C15),
//   element e = j*k + c of the row-major d x k block uses outputs 2(e/2), 2(e/2)+1,
//   u1 = ((x1 >> 11) + 1) 2^-53, u2 = (x2 >> 11) 2^-53, r = sqrt(-2 ln u1),
//   theta = 2 pi u2, value = r cos(theta) for even e, r sin(theta) for odd e,
//   computed in FP64 and rounded once to the output type.
#include <cmath>

#include "common.cuh"

namespace bks {

namespace {
__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// out[c * ld_row + j] (transposed, column-major thin block) or out[j * ld_row + c].
template <typename T>
__global__ void gen_pi_kernel(uint64_t seed, int64_t d, int k, T* out, int64_t ld_row,
                              bool transposed) {
    const int64_t total = d * int64_t(k);
    const int64_t pairs = (total + 1) / 2;
    for (int64_t p = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; p < pairs;
         p += int64_t(gridDim.x) * blockDim.x) {
        const uint64_t x1 = splitmix64(seed, 2 * uint64_t(p));
        const uint64_t x2 = splitmix64(seed, 2 * uint64_t(p) + 1);
        const double u1 = double((x1 >> 11) + 1) * 0x1.0p-53;
        const double u2 = double(x2 >> 11) * 0x1.0p-53;
        const double r = sqrt(-2.0 * log(u1));
        const double theta = 6.283185307179586 * u2;
        double s, c;
        sincos(theta, &s, &c);
        const double v[2] = {r * c, r * s};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int64_t e = 2 * p + h;
            if (e >= total) break;
            const int64_t j = e / k, col = e % k;
            const int64_t idx = transposed ? col * ld_row + j : j * ld_row + col;
            out[idx] = T(v[h]);
        }
    }
}

template <typename T, typename TS>
__global__ void transpose_in_kernel(const TS* __restrict__ src, int64_t rows, int64_t cols,
                                    int64_t lds, T* __restrict__ dst, int64_t ldd) {
    __shared__ T tile[32][33];
    const int64_t r0 = int64_t(blockIdx.y) * 32, c0 = int64_t(blockIdx.x) * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int64_t r = r0 + i, c = c0 + threadIdx.x;
        tile[i][threadIdx.x] = (r < rows && c < cols) ? cvt<T>(src[r * lds + c]) : T(0);
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int64_t c = c0 + i, r = r0 + threadIdx.x;
        if (c < cols && r < rows) dst[c * ldd + r] = tile[threadIdx.x][i];
    }
}

template <typename T>
__global__ void check_finite_kernel(const T* __restrict__ x, int64_t n, int* status) {
    bool bad = false;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n;
         i += int64_t(gridDim.x) * blockDim.x)
        bad |= !isfinite(x[i]);
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(status, ST_NONFINITE);
}

// One CTA per column: find the entry of largest magnitude (lowest row on ties) and
// flip the column (and row c of Ut) if it is negative.
template <typename T>
__global__ void sign_fix_kernel(T* Z, int64_t n, int64_t rs, int64_t cs, T* Ut, int64_t w, int64_t ldu) {
    const int c = blockIdx.x;
    T best = T(-1);
    int64_t bidx = INT64_MAX;
    for (int64_t r = threadIdx.x; r < n; r += blockDim.x) {
        const T v = fabs(Z[r * rs + c * cs]);
        if (v > best) { best = v; bidx = r; }
    }
    __shared__ T sb[1024];
    __shared__ int64_t si[1024];
    sb[threadIdx.x] = best;
    si[threadIdx.x] = bidx;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            const T ob = sb[threadIdx.x + s];
            const int64_t oi = si[threadIdx.x + s];
            if (ob > sb[threadIdx.x] || (ob == sb[threadIdx.x] && oi < si[threadIdx.x])) {
                sb[threadIdx.x] = ob;
                si[threadIdx.x] = oi;
            }
        }
        __syncthreads();
    }
    const int64_t imax = si[0];
    __syncthreads();
    if (imax == INT64_MAX) return;
    if (!(Z[imax * rs + c * cs] < T(0))) return;
    for (int64_t r = threadIdx.x; r < n; r += blockDim.x) Z[r * rs + c * cs] = -Z[r * rs + c * cs];
    if (Ut != nullptr)
        for (int64_t j = threadIdx.x; j < w; j += blockDim.x) Ut[c * ldu + j] = -Ut[c * ldu + j];
}

// sigma[i] = |Vt[i, :len]| accumulated in FP64; optionally Vt[i] /= sigma[i].
template <typename T>
__global__ void row_norms_kernel(T* Vt, int64_t len, int64_t ldv, T* sigma, bool normalise) {
    const int i = blockIdx.x;
    double s = 0.0;
    for (int64_t j = threadIdx.x; j < len; j += blockDim.x) {
        const double v = double(Vt[i * ldv + j]);
        s += v * v;
    }
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) red[0] = t;
    }
    __syncthreads();
    const double nrm = sqrt(red[0]);
    if (threadIdx.x == 0) sigma[i] = T(nrm);
    if (normalise && nrm > 0.0) {
        const T inv = T(1.0 / nrm);
        for (int64_t j = threadIdx.x; j < len; j += blockDim.x) Vt[i * ldv + j] *= inv;
    }
}
}  // namespace

template <typename T>
void gen_pi_device(Exec& ex, uint64_t seed, int64_t d, int k, T* out, int64_t ld_row,
                   bool transposed) {
    const int64_t pairs = (d * int64_t(k) + 1) / 2;
    int blocks = int((pairs + 255) / 256);
    if (blocks > 4 * ex.num_sms) blocks = 4 * ex.num_sms;
    if (blocks < 1) blocks = 1;
    gen_pi_kernel<T><<<blocks, 256, 0, ex.stream>>>(seed, d, k, out, ld_row, transposed);
    ex.launches++;
}

void gen_pi_host(uint64_t seed, int64_t d, int k, float* out) {
    const int64_t total = d * int64_t(k);
    for (int64_t p = 0; p < (total + 1) / 2; ++p) {
        const uint64_t x1 = splitmix64(seed, 2 * uint64_t(p));
        const uint64_t x2 = splitmix64(seed, 2 * uint64_t(p) + 1);
        const double u1 = double((x1 >> 11) + 1) * 0x1.0p-53;
        const double u2 = double(x2 >> 11) * 0x1.0p-53;
        const double r = std::sqrt(-2.0 * std::log(u1));
        const double theta = 6.283185307179586 * u2;
        const double c = r * std::cos(theta);
        const double s = r * std::sin(theta);
        out[2 * p] = float(c);
        if (2 * p + 1 < total) out[2 * p + 1] = float(s);
    }
}

template <typename T>
void transpose_in(Exec& ex, const void* src, int src_dtype, int64_t rows, int64_t cols,
                  int64_t lds, T* dst, int64_t ldd) {
    dim3 block(32, 8);
    dim3 grid(unsigned((cols + 31) / 32), unsigned((rows + 31) / 32));
    if (src_dtype == 0)
        transpose_in_kernel<T, double><<<grid, block, 0, ex.stream>>>(
            static_cast<const double*>(src), rows, cols, lds, dst, ldd);
    else if (src_dtype == 1)
        transpose_in_kernel<T, float><<<grid, block, 0, ex.stream>>>(
            static_cast<const float*>(src), rows, cols, lds, dst, ldd);
    else
        transpose_in_kernel<T, __nv_bfloat16><<<grid, block, 0, ex.stream>>>(
            static_cast<const __nv_bfloat16*>(src), rows, cols, lds, dst, ldd);
    ex.launches++;
}

template <typename TS, typename TD>
__global__ void cast_2d_kernel(const TS* __restrict__ src, int64_t rows, int64_t cols, int64_t lds,
                               TD* __restrict__ dst, int64_t ldd) {
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < rows * cols;
         e += int64_t(gridDim.x) * blockDim.x) {
        const int64_t r = e / cols, c = e % cols;
        dst[r * ldd + c] = TD(src[r * lds + c]);
    }
}

template <typename TS, typename TD>
void cast_2d(Exec& ex, const TS* src, int64_t rows, int64_t cols, int64_t lds, TD* dst, int64_t ldd) {
    int64_t blocks = (rows * cols + 255) / 256;
    if (blocks > 8 * int64_t(ex.num_sms)) blocks = 8 * int64_t(ex.num_sms);
    if (blocks < 1) blocks = 1;
    cast_2d_kernel<TS, TD><<<unsigned(blocks), 256, 0, ex.stream>>>(src, rows, cols, lds, dst, ldd);
    ex.launches++;
}
template void cast_2d<float, double>(Exec&, const float*, int64_t, int64_t, int64_t, double*, int64_t);
template void cast_2d<double, float>(Exec&, const double*, int64_t, int64_t, int64_t, float*, int64_t);

template <typename T>
void check_finite(Exec& ex, const T* x, int64_t n) {
    int blocks = int((n + 255) / 256);
    if (blocks > 2 * ex.num_sms) blocks = 2 * ex.num_sms;
    if (blocks < 1) blocks = 1;
    check_finite_kernel<T><<<blocks, 256, 0, ex.stream>>>(x, n, ex.status);
    ex.launches++;
}

template <typename T>
void sign_fix(Exec& ex, T* Z, int64_t n, int k, int64_t ldz, T* Ut, int64_t w, int64_t ldu) {
    sign_fix_kernel<T><<<k, 1024, 0, ex.stream>>>(Z, n, ldz, 1, Ut, w, ldu);
    ex.launches++;
}

template <typename T>
void sign_fix_cm(Exec& ex, T* Zt, int64_t n, int k, int64_t ldz, T* Ut, int64_t w, int64_t ldu) {
    sign_fix_kernel<T><<<k, 1024, 0, ex.stream>>>(Zt, n, 1, ldz, Ut, w, ldu);
    ex.launches++;
}

template <typename T>
void row_norms(Exec& ex, T* Vt, int k, int64_t len, int64_t ldv, T* sigma, bool normalise) {
    row_norms_kernel<T><<<k, 256, 0, ex.stream>>>(Vt, len, ldv, sigma, normalise);
    ex.launches++;
}

#define BKS_INST(T)                                                                        \
    template void gen_pi_device<T>(Exec&, uint64_t, int64_t, int, T*, int64_t, bool);      \
    template void transpose_in<T>(Exec&, const void*, int, int64_t, int64_t, int64_t, T*,  \
                                  int64_t);                                                \
    template void check_finite<T>(Exec&, const T*, int64_t);                               \
    template void sign_fix<T>(Exec&, T*, int64_t, int, int64_t, T*, int64_t, int64_t);     \
    template void sign_fix_cm<T>(Exec&, T*, int64_t, int, int64_t, T*, int64_t, int64_t);  \
    template void row_norms<T>(Exec&, T*, int, int64_t, int64_t, T*, bool);
BKS_INST(float)
BKS_INST(double)
#undef BKS_INST

}  // namespace bks
