// Block Lanczos (Sec. 4, "computing Q"): the Rayleigh quotient T = Q^T A A^T Q of the
// three-term recurrence is block tridiagonal with k x k blocks,
//   A A^T Q_j = Q_{j-1} R_{j-1}^T + Q_j D_j + Q_{j+1} R_j,
// so only D_j = B_j^T B_j and R_{j-1} = B_j^T B_{j-1} (B_j = A^T Q_j) are formed.  The
// solver writes the Gram products [B_{j-1}; B_j]^T B_j as row block j of T (the lower
// band: R_{j-1} and D_j); this kernel completes the band (symmetric D_j, R_{j-1}^T
// mirrored above the diagonal) and sets the blocks off it to zero, the three-term
// property.
#include "common.cuh"

namespace bks {

namespace {

// One thread per unordered pair {r, c} (r >= c): the two entries of a pair are written by
// that thread alone, so the completion runs in place without a race.
template <typename T>
__global__ void lanczos_band_kernel(T* __restrict__ t, int w, int k) {
    const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= int64_t(w) * w) return;
    const int r = int(idx / w), c = int(idx % w);
    if (r < c) return;
    const int rb = r / k, cb = c / k;
    T* lo = t + int64_t(r) * w + c;
    T* up = t + int64_t(c) * w + r;
    if (rb == cb) {
        const T s = (*lo + *up) * T(0.5);
        *lo = s;
        *up = s;
    } else if (rb == cb + 1) {
        *up = *lo;
    } else {
        *lo = T(0);
        *up = T(0);
    }
}

}  // namespace

template <typename T>
void lanczos_band(Exec& ex, T* t, int w, int k) {
    const int64_t total = int64_t(w) * w;
    const unsigned blocks = unsigned((total + 255) / 256);
    lanczos_band_kernel<T><<<blocks, 256, 0, ex.stream>>>(t, w, k);
    ex.launches++;
}

template void lanczos_band<float>(Exec&, float*, int, int);
template void lanczos_band<double>(Exec&, double*, int, int);

}  // namespace bks
