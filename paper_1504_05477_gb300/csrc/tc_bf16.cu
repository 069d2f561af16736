// Tensor-core products with a dense BF16 A (kind::f16, FP32 accumulation):
//   mode AX : Out (c x n, column-major thin block) = (A X)^T,   X a c x d thin block
//   mode ATX: Out (c x d)                          = (A^T X)^T, X a c x n thin block
// X is FP32.  It is split on the device into NP BF16 pieces x = x_1 + ... + x_NP with
// x_1 = bf16(x), x_2 = bf16(x - x_1), x_3 = bf16(x - x_1 - x_2):
//   NP = 1: the BF16 product of the mixed-precision mode (X rounded to BF16),
//   NP = 3: FP32-accurate (24 significant bits of x; A is exactly BF16, so every
//           product a * x_p is exact in FP32 and only the accumulation rounds).  This
//           is the refinement product B = A^T Q at the full Krylov width.
// A reaches the MMA straight from TMA: K-major tiles for A X (A's rows run along the
// contraction), MN-major tiles for A^T X (A's rows run along the output), so no pass
// over A in registers is needed.
//
// One persistent CTA per SM, stream-K over (tile, 64-deep chunk) units with a
// deterministic fix-up (as for the FP32 kernel).  Warp roles:
//   warp 0      TMA: A tile and the NP X pieces of a chunk into one ring stage
//   warp 1      tcgen05.mma issue (one thread); owns the TMEM allocation
//   warps 2-5   epilogue: tcgen05.ld the accumulator into round-to-nearest register sums
// The FP32 accumulation inside the tensor core truncates; every TMEM accumulator holds
// at most FL chunks before the epilogue adds it into the register sum, which keeps the
// long contraction unbiased.  Every wait is bounded (1 s); on timeout the CTA flags
// ST_TIMEOUT, drains what it issued, frees its TMEM and returns.
#include <cuda_bf16.h>

#include "tc_common.cuh"

namespace bks {
namespace tc {
namespace b16 {

constexpr int KC = 64;                          // contraction per chunk: 128 bytes of BF16
constexpr uint32_t A_BYTES = BM * KC * 2;       // 16 KB
constexpr int NWARP = 6;
constexpr int NTHREADS = NWARP * 32;
constexpr uint32_t RING_BUDGET = 196 * 1024;

template <int CP, int NP>
struct Cfg {
    static constexpr uint32_t B_BYTES = uint32_t(NP) * CP * 128;
    static constexpr uint32_t STAGE = A_BYTES + B_BYTES;
    static constexpr int STAGES = RING_BUDGET / STAGE > 8 ? 8 : int(RING_BUDGET / STAGE);
    static constexpr int FL = NP == 1 ? 8 : 2;  // chunks per TMEM accumulation window
    static constexpr uint32_t TMEM_COLS = 2 * CP <= 64 ? 64 : 2 * CP <= 128 ? 128 : 256;
    static constexpr uint32_t ACC_STRIDE = TMEM_COLS / 2;   // column offset of accumulator 1
};

struct Smem {
    uint64_t full[8], empty[8];
    uint64_t acc_full[2], acc_empty[2];
    uint64_t drain;
    uint32_t tmem_base;
    int abort_flag;
};

// Instruction descriptor of kind::f16: D = F32, A = B = BF16, B K-major, A K-major
// (a_mn = 0) or MN-major (a_mn = 1), M = 128.
__host__ __device__ constexpr uint32_t idesc_bf16(int n, int a_mn) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(a_mn) << 15) | (uint32_t(n >> 3) << 17) |
           (uint32_t(BM >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

template <int CP, int NP>
__global__ void __launch_bounds__(NTHREADS, 1)
    bf16_product_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmX,
                        Params p) {
    using C = Cfg<CP, NP>;
    extern __shared__ unsigned char smem_dyn[];
    unsigned char* ring = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_dyn) + 1023) & ~uintptr_t(1023));
    Smem* sm = reinterpret_cast<Smem*>(ring + C::STAGES * C::STAGE);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int G = gridDim.x, cta = blockIdx.x;
    const int64_t U = p.tiles * p.cpt;
    int64_t ustart, uend;
    unit_range(U, G, cta, ustart, uend);
    volatile int* abort_flag = &sm->abort_flag;

    if (tid == 0) {
        for (int i = 0; i < C::STAGES; ++i) { mbar_init(&sm->full[i], 1); mbar_init(&sm->empty[i], 1); }
        for (int i = 0; i < 2; ++i) { mbar_init(&sm->acc_full[i], 1); mbar_init(&sm->acc_empty[i], 4); }
        mbar_init(&sm->drain, 1);
        sm->abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_async_smem();
    }
    if (warp == 1) {   // TMEM: two accumulators of CP columns
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&sm->tmem_base)),
                     "r"(C::TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sm->tmem_base;

    if (warp == 0) {
        // ---------------------------------------------------------------- TMA producer
        if (lane == 0) {
            int last[8];
            for (int s = 0; s < 8; ++s) last[s] = -1;
            UnitWalk w(ustart, p.cpt);
            int s = 0, ph = 0;
            for (int64_t u = ustart; u < uend; ++u, w.next()) {
                if (!wait_bar(&sm->empty[s], uint32_t(ph ^ 1), abort_flag, p.status)) break;
                const int t = int(w.t), kc = w.kc;
                unsigned char* st = ring + s * C::STAGE;
                mbar_expect_tx(&sm->full[s], C::STAGE);
                if (p.mode == 0) {   // A X: box {64 (d), 128 (n)}, K-major
                    tma_load_2d(st, &tmA, kc * KC, t * BM, &sm->full[s]);
                } else {             // A^T X: two boxes {64 (d), 64 (n)}, MN-major halves
                    tma_load_2d(st, &tmA, t * BM, kc * KC, &sm->full[s]);
                    tma_load_2d(st + A_BYTES / 2, &tmA, t * BM + 64, kc * KC, &sm->full[s]);
                }
#pragma unroll
                for (int pc = 0; pc < NP; ++pc)
                    tma_load_2d(st + A_BYTES + pc * CP * 128, &tmX, kc * KC, pc * p.c, &sm->full[s]);
                last[s] = ph;
                if (++s == C::STAGES) { s = 0; ph ^= 1; }
            }
            for (int s = 0; s < C::STAGES; ++s) drain_bar(&sm->full[s], last[s]);
        }
    } else if (warp == 1) {
        // ---------------------------------------------------------------- MMA issuer
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16(CP, p.mode);
            int i = 0;
            int sub = -1;
            bool first = true;
            UnitWalk w(ustart, p.cpt);
            for (int64_t u = ustart; u < uend; ++u, ++i) {
                if (u == ustart || w.kc % C::FL == 0) {   // a new accumulation window
                    ++sub;
                    if (!wait_bar(&sm->acc_empty[sub & 1], uint32_t(((sub >> 1) & 1) ^ 1), abort_flag, p.status)) break;
                    tc_fence_after();
                    first = true;
                }
                const int s = i % C::STAGES;
                if (!wait_bar(&sm->full[s], uint32_t((i / C::STAGES) & 1), abort_flag, p.status)) break;
                tc_fence_after();
                const uint32_t d_tmem = tmem + uint32_t(sub & 1) * C::ACC_STRIDE;
                const uint32_t sa = smem_u32(ring + s * C::STAGE);
                const uint64_t db = desc_sw128(sa + A_BYTES);
#pragma unroll
                for (int kk = 0; kk < KC / 16; ++kk) {   // K = 16 per MMA = 32 bytes
                    const uint64_t da = p.mode == 0 ? desc_sw128(sa) + uint64_t(kk * 2)
                                                    : desc_sw128(sa + kk * 2048, A_BYTES / 2, 1024);
#pragma unroll
                    for (int pc = 0; pc < NP; ++pc)
                        mma_bf16(d_tmem, da, db + uint64_t((pc * CP * 128) >> 4) + uint64_t(kk * 2), idesc,
                                 (first && kk == 0 && pc == 0) ? 0u : 1u);
                }
                first = false;
                umma_commit(&sm->empty[s]);
                w.next();
                if (u + 1 == uend || w.kc % C::FL == 0)   // the next unit opens a window
                    umma_commit(&sm->acc_full[sub & 1]);
            }
            umma_commit(&sm->drain);
            wait_bar(&sm->drain, 0, abort_flag, p.status);
        }
    } else {
        // ---------------------------------------------------------------- epilogue
        const int grp = warp & 3;                 // TMEM lanes 32*grp .. 32*grp+31
        const int m = grp * 32 + lane;
        int seg = -1, sub = -1;
        int64_t u = ustart;
        bool ok = true;
        while (u < uend && ok) {
            const int64_t t = u / p.cpt;
            const int64_t seg_end = (t + 1) * p.cpt < uend ? (t + 1) * p.cpt : uend;
            const bool whole = (u == t * p.cpt) && (seg_end == (t + 1) * p.cpt);
            ++seg;
            float run[CP];
#pragma unroll
            for (int j = 0; j < CP; ++j) run[j] = 0.f;
            while (u < seg_end) {
                // the window ends at the next chunk that is a multiple of FL, or at seg_end
                const int kc = int(u - t * p.cpt);
                int64_t w_end = u + (C::FL - kc % C::FL);
                if (w_end > seg_end) w_end = seg_end;
                ++sub;
                if (!wait_bar(&sm->acc_full[sub & 1], uint32_t((sub >> 1) & 1), abort_flag, p.status)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t acc = tmem + uint32_t(sub & 1) * C::ACC_STRIDE + (uint32_t(grp * 32) << 16);
#pragma unroll
                for (int j0 = 0; j0 < CP; j0 += 32) {
                    float h[32];
                    tmem_ld32(acc + uint32_t(j0), h);
#pragma unroll
                    for (int j = 0; j < 32; ++j) run[j0 + j] += h[j];
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&sm->acc_empty[sub & 1]);
                u = w_end;
            }
            if (!ok) break;
            const int64_t row = t * BM + m;
            float* dst;
            int64_t stride;
            if (whole) {
                dst = p.out + row;
                stride = p.ldo;
            } else {
                const int64_t slot = int64_t(cta) * p.maxseg + seg;
                dst = p.part + slot * int64_t(CP) * BM + m;
                stride = BM;
            }
            if (!whole || row < p.rows_out) {
#pragma unroll
                for (int j = 0; j < CP; ++j)
                    if (j < p.c) dst[int64_t(j) * stride] = run[j];
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::TMEM_COLS));
    }
}

// x (rows x len thin, pitch ld) -> np BF16 pieces, piece p at rows [p*rows, (p+1)*rows).
// Row r = blockIdx.y; the x blocks stride along it.
__global__ void bf16_split_kernel(const float* __restrict__ x, int rows, int64_t len, int64_t ld, int np,
                                  __nv_bfloat16* __restrict__ xb) {
    const int64_t r = blockIdx.y;
    for (int64_t l = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; l < len;
         l += int64_t(gridDim.x) * blockDim.x) {
        float v = x[r * ld + l];
        for (int pc = 0; pc < np; ++pc) {
            const __nv_bfloat16 b = __float2bfloat16_rn(v);
            xb[(int64_t(pc) * rows + r) * ld + l] = b;
            v -= __bfloat162float(b);
        }
    }
}

template <int CP, int NP>
size_t smem_bytes() {
    return size_t(Cfg<CP, NP>::STAGES) * Cfg<CP, NP>::STAGE + sizeof(Smem) + 1024;
}

template <int CP, int NP>
cudaError_t launch(Exec& ex, const CUtensorMap& tmA, const CUtensorMap& tmX, const Params& p, int G) {
    const size_t smem = smem_bytes<CP, NP>();
    cudaError_t err = cudaFuncSetAttribute(bf16_product_kernel<CP, NP>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (err != cudaSuccess) return err;
    // the kernel log times the HBM-bound products (X rounded to BF16) only
    KernelLog* log = NP == 1 ? ex.klog : nullptr;
    if (log) log->record(ex.stream);
    bf16_product_kernel<CP, NP><<<G, NTHREADS, smem, ex.stream>>>(tmA, tmX, p);
    if (log) log->record(ex.stream);
    return cudaGetLastError();
}

}  // namespace b16
}  // namespace tc

bool tc_product_bf16(Exec& ex, const __nv_bfloat16* A, int64_t n, int64_t d, int64_t lda, bool trans,
                     int c, int np, const float* X, int64_t ldx, float* Y, int64_t ldy, __nv_bfloat16* xb,
                     int64_t xb_cap, float* part, int64_t part_cap) {
    using namespace tc;
    using namespace tc::b16;
    if (c < 1) return true;
    if (np != 1 && np != 3) return false;
    if ((reinterpret_cast<uintptr_t>(A) & 15) || ((lda * 2) & 15) || ((ldx * 2) & 15) ||
        (reinterpret_cast<uintptr_t>(xb) & 15))
        return false;
    const int64_t len = trans ? n : d, rows_out = trans ? d : n;
    if (len > INT32_MAX || rows_out > INT32_MAX) return false;
    CUtensorMap tmA;
    if (!encode_2d(&tmA, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, A, uint64_t(d), uint64_t(n), uint64_t(lda) * 2,
                   KC, trans ? 64 : BM, CU_TENSOR_MAP_SWIZZLE_128B))
        return false;
    const int G = ex.num_sms;
    for (int c0 = 0; c0 < c; c0 += 128) {
        const int cg = c - c0 < 128 ? c - c0 : 128;
        const int cp = (cg + 31) / 32 * 32;
        if (int64_t(np) * cg * ldx > xb_cap) return false;
        {
            int64_t bx = (len + 255) / 256;
            const int64_t cap = (4 * int64_t(G) + cg - 1) / cg;
            if (bx > cap) bx = cap;
            if (bx < 1) bx = 1;
            bf16_split_kernel<<<dim3(unsigned(bx), unsigned(cg)), 256, 0, ex.stream>>>(X + int64_t(c0) * ldx, cg, len,
                                                                                      ldx, np, xb);
            ex.launches++;
        }
        CUtensorMap tmX;
        if (!encode_2d(&tmX, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, xb, uint64_t(len), uint64_t(np) * cg,
                       uint64_t(ldx) * 2, KC, uint32_t(cp), CU_TENSOR_MAP_SWIZZLE_128B))
            return false;
        Params p{};
        p.mode = trans ? 1 : 0;
        p.c = cg;
        p.cp = cp;
        p.rows_out = rows_out;
        p.tiles = (rows_out + BM - 1) / BM;
        p.cpt = (len + KC - 1) / KC;
        p.out = Y + int64_t(c0) * ldy;
        p.ldo = ldy;
        const int64_t U = p.tiles * p.cpt;
        const int Gc = grid_for_units(U, G);
        const int64_t per = (U + Gc - 1) / Gc;
        p.maxseg = int(per / p.cpt + 2);
        if (int64_t(Gc) * p.maxseg * cp * BM > part_cap) return false;
        p.part = part;
        p.status = ex.status;
        cudaError_t err = cudaErrorInvalidValue;
        if (np == 1) {
            switch (cp) {
                case 32: err = launch<32, 1>(ex, tmA, tmX, p, Gc); break;
                case 64: err = launch<64, 1>(ex, tmA, tmX, p, Gc); break;
                case 96: err = launch<96, 1>(ex, tmA, tmX, p, Gc); break;
                case 128: err = launch<128, 1>(ex, tmA, tmX, p, Gc); break;
            }
        } else {
            switch (cp) {
                case 32: err = launch<32, 3>(ex, tmA, tmX, p, Gc); break;
                case 64: err = launch<64, 3>(ex, tmA, tmX, p, Gc); break;
                case 96: err = launch<96, 3>(ex, tmA, tmX, p, Gc); break;
                case 128: err = launch<128, 3>(ex, tmA, tmX, p, Gc); break;
            }
        }
        if (err != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        fixup(ex, p, Gc);
        ex.launches++;
    }
    return true;
}

int64_t tc_bf16_partial_floats(int64_t n, int64_t d, int c, int num_sms) {
    const int cp = ((c < 128 ? c : 128) + 31) / 32 * 32;
    const int64_t a = tc::partial_floats(n, d, tc::b16::KC, cp, num_sms);
    const int64_t b = tc::partial_floats(d, n, tc::b16::KC, cp, num_sms);
    return a > b ? a : b;
}

}  // namespace bks
