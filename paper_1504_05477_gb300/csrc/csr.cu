// Products with a sparse A in CSR form (Sec. 4: the methods touch A only through
// products with A and A^T, at O(nnz(A) k) cost per product, Theorems 7 and 8), with
// optional implicit mean centring (footnote 1 of Sec. 1):
//   (A - 1 mu^T) X   = A X   - 1 (mu^T X)
//   (A - 1 mu^T)^T Y = A^T Y - mu (1^T Y)
// A^T is applied through the CSR of A^T (built once by bks_csr_transpose), so both
// products are row-parallel gathers.  Rows are cut into segments of at most SEG
// non-zeros; one warp handles one segment, lanes run over the output columns and
// gather the matching rows of X (row-major copy, L2-resident).  Rows with several
// segments (the power-law columns of a term-document matrix) are summed afterwards in
// segment order, in FP64, so results are deterministic.
#include "common.cuh"

namespace bks {

namespace {

constexpr int SEG = 512;   // non-zeros per segment

// ------------------------------------------------------------------ scans
// Exclusive scan of n int64 values (in -> out, out[n] = total), three phases.
constexpr int SCAN_BLOCK = 1024;

__global__ void scan_block_sums(const int64_t* in, int64_t n, int64_t* sums) {
    __shared__ int64_t s[SCAN_BLOCK];
    const int64_t i = int64_t(blockIdx.x) * SCAN_BLOCK + threadIdx.x;
    s[threadIdx.x] = i < n ? in[i] : 0;
    __syncthreads();
    for (int o = SCAN_BLOCK / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) sums[blockIdx.x] = s[0];
}

// Serial exclusive scan of the block sums (few thousand at most), one thread.
__global__ void scan_sums_serial(int64_t* sums, int64_t nb) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int64_t acc = 0;
    for (int64_t b = 0; b < nb; ++b) {
        const int64_t v = sums[b];
        sums[b] = acc;
        acc += v;
    }
    sums[nb] = acc;
}

__global__ void scan_apply(const int64_t* in, int64_t n, const int64_t* sums, int64_t* out) {
    __shared__ int64_t s[SCAN_BLOCK];
    const int64_t i = int64_t(blockIdx.x) * SCAN_BLOCK + threadIdx.x;
    const int64_t v = i < n ? in[i] : 0;
    s[threadIdx.x] = v;
    __syncthreads();
    // Hillis-Steele inclusive scan within the block
    for (int o = 1; o < SCAN_BLOCK; o <<= 1) {
        const int64_t t = threadIdx.x >= o ? s[threadIdx.x - o] : 0;
        __syncthreads();
        s[threadIdx.x] += t;
        __syncthreads();
    }
    if (i < n) out[i] = sums[blockIdx.x] + s[threadIdx.x] - v;
    if (i == n - 1) out[n] = sums[blockIdx.x] + s[threadIdx.x];
}

// ------------------------------------------------------------------ structure check
__device__ __forceinline__ bool bad_input(const int* status) {
    return (*reinterpret_cast<const volatile int*>(status) & ST_BADINPUT) != 0;
}

__global__ void csr_check_ptr(const int64_t* row_ptr, int64_t rows, int64_t nnz, int* status) {
    for (int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; r <= rows;
         r += int64_t(gridDim.x) * blockDim.x) {
        const int64_t v = row_ptr[r];
        bool bad = v < 0 || v > nnz || (r == 0 && v != 0) || (r == rows && v != nnz);
        if (r < rows && row_ptr[r + 1] < v) bad = true;
        if (bad) atomicOr(status, ST_BADINPUT);
    }
}

// Row r holding entry p: the last r with row_ptr[r] <= p (empty rows share offsets).
__device__ __forceinline__ int64_t row_of(const int64_t* row_ptr, int64_t rows, int64_t p) {
    int64_t lo = 0, hi = rows;   // row_ptr[lo] <= p < row_ptr[hi] (row_ptr[rows] = nnz > p)
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (row_ptr[mid] <= p) lo = mid; else hi = mid;
    }
    return lo;
}

// Column indices in range and strictly increasing within rows; runs only when the row
// pointers passed.  One warp per run of 512 entries (coalesced), each lane locating its
// first entry's row by binary search and walking forward.
constexpr int CHECK_RUN = 512;
__global__ void csr_check_cols(const int64_t* row_ptr, const int32_t* col, int64_t rows, int64_t cols,
                               int64_t nnz, int* status) {
    if (bad_input(status)) return;
    const int lane = threadIdx.x & 31;
    bool bad = false;
    for (int64_t base = ((blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5) * CHECK_RUN; base < nnz;
         base += ((int64_t(gridDim.x) * blockDim.x) >> 5) * CHECK_RUN) {
        const int64_t end = base + CHECK_RUN < nnz ? base + CHECK_RUN : nnz;
        int64_t q = base + lane;
        if (q >= end) continue;
        int64_t r = row_of(row_ptr, rows, q);
        for (; q < end; q += 32) {
            while (row_ptr[r + 1] <= q) ++r;
            const int32_t c = col[q];
            if (c < 0 || c >= cols || (q > row_ptr[r] && col[q - 1] >= c)) bad = true;
        }
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(status, ST_BADINPUT);
}

// ------------------------------------------------------------------ transpose
__global__ void col_counts(const int32_t* col, int64_t nnz, int64_t* cnt, const int* status) {
    if (bad_input(status)) return;
    for (int64_t p = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; p < nnz;
         p += int64_t(gridDim.x) * blockDim.x)
        atomicAdd(reinterpret_cast<unsigned long long*>(&cnt[col[p]]), 1ull);
}

// Per row-block column counts: bc[b * d + c] (int32), rows [b*RB, (b+1)*RB).
__global__ void block_col_counts(const int64_t* row_ptr, const int32_t* col, int64_t n, int64_t d,
                                 int rb, int* bc, const int* status) {
    if (bad_input(status)) return;
    const int64_t b = blockIdx.x;
    const int64_t r0 = b * rb, r1 = min(n, r0 + rb);
    for (int64_t p = row_ptr[r0] + threadIdx.x; p < row_ptr[r1]; p += blockDim.x)
        atomicAdd(&bc[b * d + col[p]], 1);
}

// Turn block counts into block offsets: bc[b][c] <- t_row_ptr[c] + sum_{b' < b} count[b'][c].
__global__ void block_col_offsets(int* bc, const int64_t* t_row_ptr, int64_t d, int64_t nblocks,
                                  int64_t* boff) {
    for (int64_t c = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; c < d;
         c += int64_t(gridDim.x) * blockDim.x) {
        int64_t acc = t_row_ptr[c];
        for (int64_t b = 0; b < nblocks; ++b) {
            const int v = bc[b * d + c];
            boff[b * d + c] = acc;
            acc += v;
        }
    }
}

// One warp per row block, rows in order; the columns of one row are distinct, so the
// lanes of a step never share a counter: entries land in ascending row order.
__global__ void ordered_scatter(const int64_t* row_ptr, const int32_t* col, const float* val,
                                int64_t n, int64_t d, int rb, int64_t nblocks, int64_t* boff,
                                int32_t* t_col, float* t_val, const int* status) {
    if (bad_input(status)) return;
    const int64_t b = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (b >= nblocks) return;
    const int64_t r0 = b * rb, r1 = min(n, r0 + rb);
    int64_t* off = boff + b * d;
    for (int64_t r = r0; r < r1; ++r) {
        for (int64_t p = row_ptr[r] + lane; p < row_ptr[r + 1]; p += 32) {
            const int c = col[p];
            const int64_t dst = off[c];
            off[c] = dst + 1;
            t_col[dst] = int32_t(r);
            t_val[dst] = val[p];
        }
        __syncwarp();
    }
}

// ------------------------------------------------------------------ segments
// After a failed structure check every row gets one segment (a plan that stays in bounds).
__global__ void seg_counts(const int64_t* row_ptr, int64_t rows, int64_t* nseg, const int* status) {
    const bool bad = bad_input(status);
    for (int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; r < rows;
         r += int64_t(gridDim.x) * blockDim.x) {
        const int64_t len = bad ? 0 : row_ptr[r + 1] - row_ptr[r];
        nseg[r] = len <= SEG ? 1 : (len + SEG - 1) / SEG;
    }
}

__global__ void seg_fill(const int64_t* row_ptr, int64_t rows, const int64_t* seg_off,
                         int64_t* seg_row) {
    for (int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; r < rows;
         r += int64_t(gridDim.x) * blockDim.x)
        for (int64_t s = seg_off[r]; s < seg_off[r + 1]; ++s) seg_row[s] = r;
}

// ------------------------------------------------------------------ SpMM
// out (rows x xp, row-major) = M X - corr; M in CSR (rows), X (cols x xp, row-major,
// xp a multiple of 4).  One warp per segment; the columns are covered by q4 = ceil(cb/4)
// lanes with float4 loads, so a warp advances 32 / q4 non-zeros per step (6 at c = 20)
// and the per-group sums are added in group order at the end.  Columns are taken in
// blocks of 128.  corr: kind 0 none; kind 1 (A X centring): subtract cvec[j] from every
// row; kind 2 (A^T Y centring): subtract mu[row] * cvec[j].
__device__ __forceinline__ float4 corr4(float4 v, int corr_kind, const double* cvec, const float* mu, int64_t r,
                                        int j, int c) {
    if (corr_kind == 0) return v;
    const double m = corr_kind == 2 ? double(mu[r]) : 1.0;
    if (j + 0 < c) v.x -= float(m * cvec[j + 0]);
    if (j + 1 < c) v.y -= float(m * cvec[j + 1]);
    if (j + 2 < c) v.z -= float(m * cvec[j + 2]);
    if (j + 3 < c) v.w -= float(m * cvec[j + 3]);
    return v;
}

__global__ void spmm_seg_kernel(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                const float* __restrict__ val, const int64_t* __restrict__ seg_off,
                                const int64_t* __restrict__ seg_row, int64_t rows, const float* __restrict__ X,
                                int c, int xp, float* __restrict__ out, float* __restrict__ part, int corr_kind,
                                const double* __restrict__ cvec, const float* __restrict__ mu,
                                const int* status) {
    if (bad_input(status)) return;
    const int lane = threadIdx.x & 31;
    const int64_t nseg = seg_off[rows];   // segments actually planned
    for (int64_t s = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; s < nseg;
         s += (int64_t(gridDim.x) * blockDim.x) >> 5) {
        const int64_t r = seg_row[s];
        const int64_t first = seg_off[r];
        const bool single = seg_off[r + 1] - first == 1;
        const int64_t beg = row_ptr[r] + (s - first) * SEG;
        const int64_t end = min(row_ptr[r + 1], beg + SEG);
        for (int j0 = 0; j0 < c; j0 += 128) {
            const int cb = c - j0 < 128 ? c - j0 : 128;
            const int q4 = (cb + 3) >> 2, groups = 32 / q4;
            const int g = lane / q4, v = lane - g * q4;
            const bool active = g < groups;
            const int j = j0 + 4 * v;
            float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int64_t p0 = beg; p0 < end; p0 += 32) {
                const int cnt = int(min(int64_t(32), end - p0));
                int cc = 0;
                float vv = 0.f;
                if (lane < cnt) {
                    cc = col[p0 + lane];
                    vv = val[p0 + lane];
                }
                for (int t0 = 0; t0 < cnt; t0 += groups) {
                    const int t = t0 + g;
                    const int ct = __shfl_sync(0xffffffffu, cc, t & 31);
                    const float vt = __shfl_sync(0xffffffffu, vv, t & 31);
                    if (active && t < cnt) {
                        const float4 x = *reinterpret_cast<const float4*>(X + int64_t(ct) * xp + j);
                        acc.x = fmaf(vt, x.x, acc.x);
                        acc.y = fmaf(vt, x.y, acc.y);
                        acc.z = fmaf(vt, x.z, acc.z);
                        acc.w = fmaf(vt, x.w, acc.w);
                    }
                }
            }
            for (int gg = 1; gg < groups; ++gg) {   // group sums in group order
                const int src = (lane + gg * q4) & 31;
                const float ox = __shfl_sync(0xffffffffu, acc.x, src);
                const float oy = __shfl_sync(0xffffffffu, acc.y, src);
                const float oz = __shfl_sync(0xffffffffu, acc.z, src);
                const float ow = __shfl_sync(0xffffffffu, acc.w, src);
                if (g == 0) {
                    acc.x += ox; acc.y += oy; acc.z += oz; acc.w += ow;
                }
            }
            if (g == 0) {
                if (single)
                    *reinterpret_cast<float4*>(out + r * xp + j) = corr4(acc, corr_kind, cvec, mu, r, j, c);
                else
                    *reinterpret_cast<float4*>(part + s * xp + j) = acc;
            }
        }
    }
}

// Rows with several segments: sum the partials in segment order (FP64), then centre.
__global__ void spmm_fixup_kernel(const int64_t* __restrict__ seg_off, int64_t rows,
                                  const float* __restrict__ part, int c, int xp, float* __restrict__ out,
                                  int corr_kind, const double* __restrict__ cvec, const float* __restrict__ mu) {
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < rows * c;
         e += int64_t(gridDim.x) * blockDim.x) {
        const int64_t r = e / c;
        const int j = int(e % c);
        const int64_t s0 = seg_off[r], s1 = seg_off[r + 1];
        if (s1 - s0 <= 1) continue;
        double acc = 0.0;
        for (int64_t s = s0; s < s1; ++s) acc += double(part[s * xp + j]);
        if (corr_kind == 1) acc -= cvec[j];
        else if (corr_kind == 2) acc -= double(mu[r]) * cvec[j];
        out[r * xp + j] = float(acc);
    }
}

// cvec[j] = sum_l w[l] * Xt[j][l] (w = mu, or w = NULL for the plain sum 1^T x), FP64:
// block (j, slice) sums one of WS_SLICES slices, then the slices are added in order.
constexpr int WS_SLICES = 16;
__global__ void weighted_sums_part(const float* __restrict__ Xt, int64_t ld, int64_t len,
                                   const float* __restrict__ w, double* __restrict__ part) {
    const int j = blockIdx.x, sl = blockIdx.y;
    const int64_t per = (len + WS_SLICES - 1) / WS_SLICES;
    const int64_t l0 = sl * per, l1 = l0 + per < len ? l0 + per : len;
    double s = 0.0;
    for (int64_t l = l0 + threadIdx.x; l < l1; l += blockDim.x)
        s += double(Xt[j * ld + l]) * (w ? double(w[l]) : 1.0);
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) part[j * WS_SLICES + sl] = t;
    }
}

__global__ void weighted_sums_final(const double* __restrict__ part, int c, double* __restrict__ cvec) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= c) return;
    double s = 0.0;
    for (int sl = 0; sl < WS_SLICES; ++sl) s += part[j * WS_SLICES + sl];
    cvec[j] = s;
}

void exclusive_scan(Exec& ex, const int64_t* in, int64_t n, int64_t* out, int64_t* sums) {
    const int64_t nb = (n + SCAN_BLOCK - 1) / SCAN_BLOCK;
    scan_block_sums<<<unsigned(nb), SCAN_BLOCK, 0, ex.stream>>>(in, n, sums);
    scan_sums_serial<<<1, 32, 0, ex.stream>>>(sums, nb);
    scan_apply<<<unsigned(nb), SCAN_BLOCK, 0, ex.stream>>>(in, n, sums, out);
    ex.launches += 3;
}

int grid_for(int64_t work, int per_block, int num_sms) {
    int64_t g = (work + per_block - 1) / per_block;
    if (g > 64LL * num_sms) g = 64LL * num_sms;
    return int(g < 1 ? 1 : g);
}

}  // namespace

// ---------------------------------------------------------------------- public pieces
void csr_check(Exec& ex, const int64_t* row_ptr, const int32_t* col, int64_t rows, int64_t cols,
               int64_t nnz, int* status) {
    csr_check_ptr<<<grid_for(rows + 1, 256, ex.num_sms), 256, 0, ex.stream>>>(row_ptr, rows, nnz, status);
    csr_check_cols<<<grid_for((nnz + CHECK_RUN - 1) / CHECK_RUN, 8, ex.num_sms), 256, 0, ex.stream>>>(
        row_ptr, col, rows, cols, nnz, status);
    ex.launches += 2;
}

size_t csr_transpose_scratch(int64_t n, int64_t d) {
    const int rb = 512;
    const int64_t nb = (n + rb - 1) / rb;
    return size_t(d + 1) * 8 * 2 + size_t(nb) * d * (4 + 8) + size_t((d + SCAN_BLOCK) / SCAN_BLOCK + 2) * 8 + 4096;
}

void csr_transpose(Exec& ex, const int64_t* row_ptr, const int32_t* col, const float* val, int64_t n,
                   int64_t d, int64_t nnz, int64_t* t_row_ptr, int32_t* t_col, float* t_val,
                   void* scratch) {
    const int rb = 512;
    const int64_t nb = (n + rb - 1) / rb;
    char* s = static_cast<char*>(scratch);
    int64_t* cnt = reinterpret_cast<int64_t*>(s);
    int64_t* sums = cnt + (d + 1);
    int* bc = reinterpret_cast<int*>(sums + (d + SCAN_BLOCK) / SCAN_BLOCK + 2);
    int64_t* boff = reinterpret_cast<int64_t*>(bc + nb * d + 2);
    boff = reinterpret_cast<int64_t*>((reinterpret_cast<uintptr_t>(boff) + 7) & ~uintptr_t(7));
    cudaMemsetAsync(cnt, 0, size_t(d + 1) * 8, ex.stream);
    cudaMemsetAsync(bc, 0, size_t(nb) * d * 4, ex.stream);
    col_counts<<<grid_for(nnz, 256, ex.num_sms), 256, 0, ex.stream>>>(col, nnz, cnt, ex.status);
    exclusive_scan(ex, cnt, d, t_row_ptr, sums);
    block_col_counts<<<unsigned(nb), 256, 0, ex.stream>>>(row_ptr, col, n, d, rb, bc, ex.status);
    block_col_offsets<<<grid_for(d, 256, ex.num_sms), 256, 0, ex.stream>>>(bc, t_row_ptr, d, nb, boff);
    ordered_scatter<<<unsigned((nb * 32 + 255) / 256), 256, 0, ex.stream>>>(row_ptr, col, val, n, d, rb, nb,
                                                                            boff, t_col, t_val, ex.status);
    ex.launches += 4;
}

// Segment plan of a CSR (rows + 1 offsets): seg_off (rows + 1), seg_row (nseg).
// Returns nothing on the host: nseg = seg_off[rows] is read by the kernels themselves.
int64_t seg_upper_bound(int64_t rows, int64_t nnz) { return rows + nnz / SEG + 1; }

void csr_segments(Exec& ex, const int64_t* row_ptr, int64_t rows, int64_t* nseg_tmp, int64_t* seg_off,
                  int64_t* seg_row, int64_t* sums) {
    seg_counts<<<grid_for(rows, 256, ex.num_sms), 256, 0, ex.stream>>>(row_ptr, rows, nseg_tmp, ex.status);
    exclusive_scan(ex, nseg_tmp, rows, seg_off, sums);
    seg_fill<<<grid_for(rows, 256, ex.num_sms), 256, 0, ex.stream>>>(row_ptr, rows, seg_off, seg_row);
    ex.launches += 2;
}

int csr_row_pitch(int c) { return (c + 3) / 4 * 4; }
int64_t csr_cvec_doubles(int c) { return int64_t(c) * (WS_SLICES + 1); }

// Y_t (c x ldy, thin) = op(A) X_t with op(A) given by its CSR (rows x cols); centring per
// corr_kind (see spmm_seg_kernel).  x_rm: cols x xp scratch, y_rm: rows x xp scratch,
// part: seg_upper_bound x xp scratch, cvec: csr_cvec_doubles(c) doubles (xp =
// csr_row_pitch(c)).
void csr_product(Exec& ex, const int64_t* row_ptr, const int32_t* col, const float* val, int64_t rows,
                 int64_t cols, int64_t nnz, const int64_t* seg_off, const int64_t* seg_row,
                 int64_t nseg_bound, const float* Xt, int64_t ldx, int c, float* Yt, int64_t ldy,
                 float* x_rm, float* y_rm, float* part, int corr_kind, const float* mu, double* cvec) {
    (void)nnz;
    const int xp = csr_row_pitch(c);
    transpose_in<float>(ex, Xt, 1, c, cols, ldx, x_rm, xp);   // x_rm[l][j] = Xt[j][l]
    if (corr_kind != 0) {   // kind 1: mu^T X; kind 2: 1^T Y
        double* wpart = cvec + c;
        weighted_sums_part<<<dim3(unsigned(c), WS_SLICES), 256, 0, ex.stream>>>(
            Xt, ldx, cols, corr_kind == 1 ? mu : nullptr, wpart);
        weighted_sums_final<<<(c + 127) / 128, 128, 0, ex.stream>>>(wpart, c, cvec);
        ex.launches += 2;
    }
    const int warps_per_block = 8;
    if (ex.klog) ex.klog->record(ex.stream);
    spmm_seg_kernel<<<grid_for(nseg_bound, warps_per_block, ex.num_sms), 32 * warps_per_block, 0, ex.stream>>>(
        row_ptr, col, val, seg_off, seg_row, rows, x_rm, c, xp, y_rm, part, corr_kind, cvec, mu, ex.status);
    if (ex.klog) ex.klog->record(ex.stream);
    spmm_fixup_kernel<<<grid_for(rows * c, 256, ex.num_sms), 256, 0, ex.stream>>>(seg_off, rows, part, c, xp, y_rm,
                                                                                 corr_kind, cvec, mu);
    transpose_in<float>(ex, y_rm, 1, rows, c, xp, Yt, ldy);   // Yt[j][r] = y_rm[r][j]
    ex.launches += 2;
}

}  // namespace bks
