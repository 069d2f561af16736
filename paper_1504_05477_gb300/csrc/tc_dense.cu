// Tensor-core products with a dense FP32 A (the hot path of Algorithms 1 and 2: every
// iteration touches A only through A X and A^T X, Sec. 4):
//   mode AX : Out (c x n, column-major thin block) = (A X)^T,   X a c x d thin block
//   mode ATX: Out (c x d)                          = (A^T X)^T, X a c x n thin block
// FP32 accuracy from TF32 tensor cores by a three-term split: with
// hi(v) = v truncated to TF32 and lo(v) = v - hi(v) (exact in FP32),
//   A X ~ hi(A) hi(X) + hi(A) lo(X) + lo(A) hi(X),
// dropping only lo(A) lo(X) (relative 2^-22).  hi(X) and lo(X) are stacked as the two
// halves of one N = 2cp operand, so hi(A) [hi(X) | lo(X)] is one MMA and
// lo(A) hi(X) a second one accumulating into the first half.
//
// One persistent CTA per SM.  The (tile, 32-deep chunk) units of the whole product are
// dealt out in equal contiguous ranges (stream-K); a tile cut between CTAs is summed
// in CTA order (by the last of them to finish, or by a fix-up kernel), so results are
// deterministic.
//   warp 0      TMA: raw A tiles -> ring (6 deep; 8-10 when A comes from tensor memory)
//   warp 1      TMA: [hi(X) | lo(X)] tiles -> their own ring (2 or 4 deep)
//   warp 2      tcgen05.mma issue (one thread); owns the TMEM allocation
//   warps 3-6   converters: raw A -> hi(A), lo(A) in the UMMA K-major 128B-swizzled
//               layout (for A^T X this is also the transpose)
//   warps 7-10  epilogue: tcgen05.ld the accumulator, add the halves, store
// Every wait is bounded (1 s of globaltimer); on timeout the CTA records
// ST_TIMEOUT, drains what it issued (bounded again), frees its TMEM and returns.
#include "tc_common.cuh"

namespace bks {
namespace tc {

constexpr int KC = 32;             // contraction depth per chunk (128 bytes of FP32)
constexpr int RA = 6;              // raw A ring depth
constexpr int OP = 2;              // converted A (hi / lo) ring depth
// ring depth of the [hi(X) | lo(X)] tiles, streamed from L2 once per chunk.  A stage is
// refilled only after the MMAs of its chunk complete, so the ring must cover an L2 round
// trip plus the MMA time: 2 stages held a 64-column product to about one chunk per
// 0.7 us, 4 do not limit it.
__host__ __device__ constexpr int x_ring(int cp) { return cp <= 64 ? 4 : 2; }
constexpr int XR_MAX = 6;
// Tiles of up to 64 columns take A from tensor memory ("TS" form): the converter writes
// hi(A) and lo(A) into OPT TMEM stages next to the two accumulators instead of into shared
// memory, which frees shared memory for a deeper raw A ring.
__host__ __device__ constexpr bool ts_form(int cp) { return cp <= 64; }
// raw A ring depth (TS form): the rest of the shared memory after the X ring
__host__ __device__ constexpr int raw_ring_ts(int cp) { return cp <= 32 ? 10 : 8; }
constexpr int RAT = 10;            // deepest raw A ring (TS form)
constexpr int OPT = 4;             // converted A stages in TMEM (TS form)
constexpr int ACOL = 256;          // first TMEM column of the A stages (TS form)
constexpr int RA_MAX = RAT > RA ? RAT : RA;
constexpr int OP_MAX = OPT > OP ? OPT : OP;
static_assert(x_ring(32) == OPT && x_ring(64) == OPT && x_ring(96) == OP && x_ring(128) == OP,
              "the X ring and the converted-A ring share their release barriers");
constexpr int NWARP = 11;
constexpr int NTHREADS = NWARP * 32;
constexpr uint32_t TILE_BYTES = BM * KC * 4;   // 16 KB
constexpr int FLUSH = 4;           // chunks (32 tf32 MMA steps) per TMEM accumulation window

// Instruction descriptor of kind::tf32: D = F32, A = B = TF32, both K-major, M = 128.
__host__ __device__ constexpr uint32_t idesc_tf32(int n) {
    return (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t(n >> 3) << 17) | (uint32_t(BM >> 4) << 24);
}
// A from tensor memory (TS form): a_tmem is the TMEM address of the A tile's first column.
__device__ __forceinline__ void mma_tf32_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b, uint32_t idesc,
                                            uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b), "r"(idesc), "r"(accumulate));
}
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}
__device__ __forceinline__ float tf32_hi(float v) {
    return __uint_as_float(__float_as_uint(v) & 0xFFFFE000u);
}

struct Smem {
    uint64_t raw_full[RA_MAX], raw_empty[RA_MAX];
    uint64_t op_empty[OP_MAX], conv_full[OP_MAX];
    uint64_t x_full[XR_MAX];
    uint64_t acc_full[2], acc_empty[2];
    uint64_t drain;
    uint32_t tmem_base;
    int abort_flag;
};

template <int CP>
__global__ void __launch_bounds__(NTHREADS, 1)
    tc_product_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmXh,
                      const __grid_constant__ CUtensorMap tmXl, Params p) {
    extern __shared__ unsigned char smem_dyn[];
    __shared__ int fix_last;   // epilogue: this CTA completes the cut tile it just wrote
    // 1024-byte alignment for the swizzled tiles
    unsigned char* base = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_dyn) + 1023) & ~uintptr_t(1023));
    constexpr bool TS = ts_form(CP);
    constexpr int NRA = TS ? raw_ring_ts(CP) : RA;               // raw A ring depth
    constexpr int NOP = TS ? OPT : OP;                           // converted A stages
    constexpr uint32_t ACC_STRIDE = TS ? 2 * CP : 256;           // TMEM columns per accumulator
    const uint32_t b_bytes = uint32_t(2 * CP) * 128u;
    unsigned char* raw = base;                                   // NRA x 16 KB
    unsigned char* hi = raw + NRA * TILE_BYTES;                  // OP x 16 KB (shared-memory form)
    unsigned char* lo = hi + (TS ? 0 : OP) * TILE_BYTES;         // OP x 16 KB (shared-memory form)
    constexpr int XR = x_ring(CP);
    unsigned char* bop = lo + (TS ? 0 : OP) * TILE_BYTES;        // XR x b_bytes
    Smem* sm = reinterpret_cast<Smem*>(bop + XR * b_bytes);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int G = gridDim.x, cta = blockIdx.x;
    const int64_t U = p.tiles * p.cpt;
    int64_t ustart, uend;
    unit_range(U, G, cta, ustart, uend);
    volatile int* abort_flag = &sm->abort_flag;

    if (tid == 0) {
        for (int i = 0; i < NRA; ++i) { mbar_init(&sm->raw_full[i], 1); mbar_init(&sm->raw_empty[i], 4); }
        for (int i = 0; i < NOP; ++i) {
            mbar_init(&sm->op_empty[i], 1);
            mbar_init(&sm->conv_full[i], 4);
        }
        for (int i = 0; i < XR; ++i) mbar_init(&sm->x_full[i], 1);
        for (int i = 0; i < 2; ++i) { mbar_init(&sm->acc_full[i], 1); mbar_init(&sm->acc_empty[i], 4); }
        mbar_init(&sm->drain, 1);
        sm->abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_async_smem();
    }
    if (warp == 2) {   // TMEM: two accumulators of up to 256 columns
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&sm->tmem_base)),
                     "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sm->tmem_base;

    if (warp == 0) {
        // ---------------------------------------------------------------- A producer
        if (lane == 0) {
            int last[RA_MAX];   // phase of the last load issued into each stage (-1: none)
            for (int s = 0; s < RA_MAX; ++s) last[s] = -1;
            UnitWalk w(ustart, p.cpt);
            int s = 0, ph = 0;
            for (int64_t u = ustart; u < uend; ++u, w.next()) {
                if (!wait_bar(&sm->raw_empty[s], uint32_t(ph ^ 1), abort_flag, p.status)) break;
                mbar_expect_tx(&sm->raw_full[s], TILE_BYTES);
                if (p.mode == 0)   // AX: box {32 (d), 128 (n)}
                    tma_load_2d(raw + s * TILE_BYTES, &tmA, w.kc * KC, int(w.t * BM), &sm->raw_full[s]);
                else               // ATX: box {128 (d), 32 (n)}
                    tma_load_2d(raw + s * TILE_BYTES, &tmA, int(w.t * BM), w.kc * KC, &sm->raw_full[s]);
                last[s] = ph;
                if (++s == NRA) { s = 0; ph ^= 1; }
            }
            // every load issued has landed before shared memory is released (bounded)
            for (int s = 0; s < NRA; ++s) drain_bar(&sm->raw_full[s], last[s]);
        }
    } else if (warp == 1) {
        // ---------------------------------------------------------------- X producer
        if (lane == 0) {
            int last[XR_MAX];
            for (int o = 0; o < XR_MAX; ++o) last[o] = -1;
            UnitWalk w(ustart, p.cpt);
            int o = 0, ph = 0;
            for (int64_t u = ustart; u < uend; ++u, w.next()) {
                // X stage o and converted-A stage o are released together by one commit
                // (both rings are XR = NOP deep and advance with the unit index)
                if (!wait_bar(&sm->op_empty[o], uint32_t(ph ^ 1), abort_flag, p.status)) break;
                mbar_expect_tx(&sm->x_full[o], b_bytes);
                unsigned char* dst = bop + o * b_bytes;
                tma_load_2d(dst, &tmXh, w.kc * KC, 0, &sm->x_full[o]);
                tma_load_2d(dst + CP * 128, &tmXl, w.kc * KC, 0, &sm->x_full[o]);
                last[o] = ph;
                if (++o == XR) { o = 0; ph ^= 1; }
            }
            for (int o = 0; o < XR; ++o) drain_bar(&sm->x_full[o], last[o]);
        }
    } else if (warp == 2) {
        // ---------------------------------------------------------------- MMA issuer
        if (lane == 0) {
            const uint32_t id_full = idesc_tf32(2 * CP), id_half = idesc_tf32(CP);
            int i = 0;
            int sub = -1;   // accumulation window: at most FLUSH chunks per TMEM accumulator
            bool first = true;
            UnitWalk w(ustart, p.cpt);
            for (int64_t u = ustart; u < uend; ++u, ++i) {
                if (u == ustart || w.kc % FLUSH == 0) {   // a new accumulation window
                    ++sub;
                    if (!wait_bar(&sm->acc_empty[sub & 1], uint32_t(((sub >> 1) & 1) ^ 1), abort_flag, p.status)) break;
                    tc_fence_after();
                    first = true;
                }
                const int o = i % NOP, xs = i % XR;
                const uint32_t par = uint32_t((i / NOP) & 1);
                if (!wait_bar(&sm->conv_full[o], par, abort_flag, p.status)) break;
                if (!wait_bar(&sm->x_full[xs], uint32_t((i / XR) & 1), abort_flag, p.status)) break;
                tc_fence_after();
                const uint32_t d_tmem = tmem + uint32_t(sub & 1) * ACC_STRIDE;
                const uint64_t db = desc_sw128(smem_u32(bop + xs * b_bytes));
                if constexpr (TS) {
                    // A stage o: hi(A) in columns [0, 32), lo(A) in [32, 64), one column per K
                    const uint32_t a_hi = tmem + uint32_t(ACOL + o * 64), a_lo = a_hi + 32;
#pragma unroll
                    for (int kk = 0; kk < KC / 8; ++kk) {   // K = 8 per tf32 MMA
                        const uint64_t adv = uint64_t(kk * 2);
                        mma_tf32_ts(d_tmem, a_hi + uint32_t(kk * 8), db + adv, id_full, (first && kk == 0) ? 0u : 1u);
                        mma_tf32_ts(d_tmem, a_lo + uint32_t(kk * 8), db + adv, id_half, 1u);
                    }
                } else {
                    const uint64_t dh = desc_sw128(smem_u32(hi + o * TILE_BYTES));
                    const uint64_t dl = desc_sw128(smem_u32(lo + o * TILE_BYTES));
#pragma unroll
                    for (int kk = 0; kk < KC / 8; ++kk) {   // K = 8 per tf32 MMA = 32 bytes
                        const uint64_t adv = uint64_t(kk * 2);
                        mma_tf32(d_tmem, dh + adv, db + adv, id_full, (first && kk == 0) ? 0u : 1u);
                        mma_tf32(d_tmem, dl + adv, db + adv, id_half, 1u);
                    }
                }
                first = false;
                umma_commit(&sm->op_empty[o]);   // frees converted-A stage o and X stage xs (= o)
                w.next();
                if (u + 1 == uend || w.kc % FLUSH == 0)   // the next unit opens a window
                    umma_commit(&sm->acc_full[sub & 1]);
            }
            // drain: every MMA issued so far has completed before TMEM is released
            umma_commit(&sm->drain);
            wait_bar(&sm->drain, 0, abort_flag, p.status);
        }
    } else if (warp <= 6) {
        // ---------------------------------------------------------------- converters
        const int ct = tid - 96;   // 0..127
        int i = 0;
        if constexpr (TS) {
            // thread = TMEM lane = row m of the A tile (a warp reaches lanes 32 (warp % 4) ..).
            // Software-pipelined over tiles with two register buffers: the next tile is read
            // from shared memory while the current tile's stores to tensor memory are in
            // flight (a tcgen05.st's source registers are free only after tcgen05.wait::st).
            const int m = (warp & 3) * 32 + lane;
            const uint32_t lane_addr = uint32_t((warp & 3) * 32) << 16;
            // raw tile of unit i (stage i % NRA) -> hi / lo registers; releases the stage
            auto load = [&](int ii, uint32_t (&h)[32], uint32_t (&l)[32]) -> bool {
                const int s = ii % NRA;
                if (!wait_bar(&sm->raw_full[s], uint32_t((ii / NRA) & 1), abort_flag, p.status)) return false;
                const unsigned char* rs = raw + s * TILE_BYTES;
                if (p.mode == 0) {   // 128B-swizzled K-major raw tile: row m's eight 16-byte chunks
                    const int rowoff = (m >> 3) * 1024 + (m & 7) * 128;
#pragma unroll
                    for (int g = 0; g < 8; ++g) {
                        const float4 v = *reinterpret_cast<const float4*>(rs + rowoff + ((g ^ (m & 7)) << 4));
                        const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const float hv = tf32_hi(vv[e]);
                            h[4 * g + e] = __float_as_uint(hv);
                            l[4 * g + e] = __float_as_uint(vv[e] - hv);
                        }
                    }
                } else {             // raw tile: 32 contraction rows x 128 columns (row pitch 512 B)
                    const float* rf = reinterpret_cast<const float*>(rs);
#pragma unroll
                    for (int kk = 0; kk < 32; ++kk) {
                        const float v = rf[kk * BM + m];
                        const float hv = tf32_hi(v);
                        h[kk] = __float_as_uint(hv);
                        l[kk] = __float_as_uint(v - hv);
                    }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&sm->raw_empty[s]);   // the raw tile is in registers
                return true;
            };
            // registers of unit i -> converted-A stage i % NOP (after the stage is free)
            auto store = [&](int ii, const uint32_t (&h)[32], const uint32_t (&l)[32]) -> bool {
                const int o = ii % NOP;
                if (!wait_bar(&sm->op_empty[o], uint32_t(((ii / NOP) & 1) ^ 1), abort_flag, p.status)) return false;
                tc_fence_after();
                const uint32_t col = tmem + lane_addr + uint32_t(ACOL + o * 64);
                tmem_st32(col, h);
                tmem_st32(col + 32, l);
                return true;
            };
            auto publish = [&](int ii) {   // the stores of unit i have landed
                tmem_wait_st();
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&sm->conv_full[ii % NOP]);
            };
            const int nunits = int(uend - ustart);
            uint32_t h0[32], l0[32], h1[32], l1[32];
            bool ok = nunits > 0 && load(0, h0, l0);
            for (int ii = 0; ok && ii < nunits; ii += 2) {
                if (!store(ii, h0, l0)) break;
                if (ii + 1 < nunits && !load(ii + 1, h1, l1)) { tmem_wait_st(); break; }
                publish(ii);
                if (ii + 1 >= nunits) break;
                if (!store(ii + 1, h1, l1)) break;
                if (ii + 2 < nunits && !load(ii + 2, h0, l0)) { tmem_wait_st(); break; }
                publish(ii + 1);
            }
            tmem_wait_st();
        } else
        for (int64_t u = ustart; u < uend; ++u, ++i) {
            const int s = i % RA, o = i % OP;
            if (!wait_bar(&sm->raw_full[s], uint32_t((i / RA) & 1), abort_flag, p.status)) break;
            if (!wait_bar(&sm->op_empty[o], uint32_t(((i / OP) & 1) ^ 1), abort_flag, p.status)) break;
            const unsigned char* rs = raw + s * TILE_BYTES;
            unsigned char* hs = hi + o * TILE_BYTES;
            unsigned char* ls = lo + o * TILE_BYTES;
            if (p.mode == 0) {
                // same 128B-swizzled K-major layout in and out: elementwise on 16-byte chunks
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int off = (ct + 128 * q) * 16;
                    const float4 v = *reinterpret_cast<const float4*>(rs + off);
                    float4 h, l;
                    h.x = tf32_hi(v.x); h.y = tf32_hi(v.y); h.z = tf32_hi(v.z); h.w = tf32_hi(v.w);
                    l.x = v.x - h.x; l.y = v.y - h.y; l.z = v.z - h.z; l.w = v.w - h.w;
                    *reinterpret_cast<float4*>(hs + off) = h;
                    *reinterpret_cast<float4*>(ls + off) = l;
                }
            } else {
                // raw tile: 32 rows (contraction) x 128 columns (M), row pitch 512 B.
                // Thread ct owns M-row ct; it gathers 4 contraction values per 16-byte chunk.
                const float* rf = reinterpret_cast<const float*>(rs);
                const int rowoff = (ct >> 3) * 1024 + (ct & 7) * 128;
#pragma unroll
                for (int g = 0; g < 8; ++g) {
                    float4 v;
                    v.x = rf[(4 * g + 0) * BM + ct];
                    v.y = rf[(4 * g + 1) * BM + ct];
                    v.z = rf[(4 * g + 2) * BM + ct];
                    v.w = rf[(4 * g + 3) * BM + ct];
                    float4 h, l;
                    h.x = tf32_hi(v.x); h.y = tf32_hi(v.y); h.z = tf32_hi(v.z); h.w = tf32_hi(v.w);
                    l.x = v.x - h.x; l.y = v.y - h.y; l.z = v.z - h.z; l.w = v.w - h.w;
                    const int off = rowoff + ((g ^ (ct & 7)) << 4);
                    *reinterpret_cast<float4*>(hs + off) = h;
                    *reinterpret_cast<float4*>(ls + off) = l;
                }
            }
            fence_async_smem();
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&sm->raw_empty[s]);
                mbar_arrive(&sm->conv_full[o]);
            }
        }
    } else {
        // ---------------------------------------------------------------- epilogue
        const int grp = warp & 3;                 // TMEM lanes 32*grp .. 32*grp+31
        const int m = grp * 32 + lane;            // row of D owned by this thread
        // A failed wait (timeout or abort) clears `ok`; the warp then keeps walking the same
        // segments without touching TMEM or the output, so that the four warps always meet
        // at the same named barriers.
        int seg = -1, sub = -1;
        int64_t u = ustart;
        bool ok = true;
        while (u < uend) {
            const int64_t t = u / p.cpt;
            const int64_t seg_end = (t + 1) * p.cpt < uend ? (t + 1) * p.cpt : uend;
            const bool whole = (u == t * p.cpt) && (seg_end == (t + 1) * p.cpt);
            ++seg;
            // running sum of the tile segment in registers (round to nearest): every
            // TMEM accumulator holds at most FLUSH chunks, so its truncating FP32
            // accumulation never runs long enough to bias the result
            float run[CP];
#pragma unroll
            for (int j = 0; j < CP; ++j) run[j] = 0.f;
            while (u < seg_end) {
                // the window ends at the next chunk that is a multiple of FLUSH, or at seg_end
                const int kc = int(u - t * p.cpt);
                int64_t w_end = u + (FLUSH - kc % FLUSH);
                if (w_end > seg_end) w_end = seg_end;
                ++sub;
                if (ok && !wait_bar(&sm->acc_full[sub & 1], uint32_t((sub >> 1) & 1), abort_flag, p.status))
                    ok = false;
                if (!ok) {
                    u = w_end;
                    continue;
                }
                tc_fence_after();
                const uint32_t acc = tmem + uint32_t(sub & 1) * ACC_STRIDE + (uint32_t(grp * 32) << 16);
                if constexpr (CP <= 64) {   // hi.hi and hi.lo halves, one wait per 32 columns
#pragma unroll
                    for (int j0 = 0; j0 < CP; j0 += 32) {
                        uint32_t hh[32], hl[32];
                        tmem_ld32_async(acc + uint32_t(j0), hh);
                        tmem_ld32_async(acc + uint32_t(CP + j0), hl);
                        tmem_wait();
#pragma unroll
                        for (int j = 0; j < 32; ++j)
                            run[j0 + j] += __uint_as_float(hh[j]) + __uint_as_float(hl[j]);
                    }
                } else {   // wide tiles: the registers hold one load at a time
#pragma unroll
                    for (int j0 = 0; j0 < CP; j0 += 32) {
                        float h[32];
                        tmem_ld32(acc + uint32_t(j0), h);
#pragma unroll
                        for (int j = 0; j < 32; ++j) run[j0 + j] += h[j];
                        tmem_ld32(acc + uint32_t(CP + j0), h);
#pragma unroll
                        for (int j = 0; j < 32; ++j) run[j0 + j] += h[j];
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&sm->acc_empty[sub & 1]);
                u = w_end;
            }
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
            if (!ok || *abort_flag) {
                // nothing is written after a failed wait
            } else if (whole && p.accumulate) {
                if (row < p.rows_out) {
#pragma unroll
                    for (int j = 0; j < CP; ++j)
                        if (j < p.c) dst[int64_t(j) * stride] += run[j];
                }
            } else if (!whole || row < p.rows_out) {
#pragma unroll
                for (int j = 0; j < CP; ++j)
                    if (j < p.c) dst[int64_t(j) * stride] = run[j];
            }
            if (!whole && p.tile_cnt != nullptr) {
                // cut tile: the last of its CTAs to get here adds the partials in CTA order
                // (for up to 8 CTAs per tile the order of tc_fixup_kernel: the same bits)
                const int64_t G = gridDim.x, U = p.tiles * p.cpt;
                const int64_t c_first = ((t * p.cpt + 1) * G - 1) / U;
                const int64_t c_last = (((t + 1) * p.cpt) * G - 1) / U;
                int ncontrib = 0;
                for (int64_t cc = c_first; cc <= c_last; ++cc) ncontrib += ((cc + 1) * U) / G != (cc * U) / G;
                __threadfence();
                asm volatile("bar.sync 1, 128;" ::: "memory");   // the four epilogue warps
                if (m == 0) fix_last = ok && atomicAdd(&p.tile_cnt[t], 1u) == unsigned(ncontrib - 1);
                asm volatile("bar.sync 1, 128;" ::: "memory");
                if (fix_last && !*abort_flag) {
                    __threadfence();
                    float v[CP];
#pragma unroll
                    for (int j = 0; j < CP; ++j) v[j] = 0.f;
                    for (int64_t cc = c_first; cc <= c_last; ++cc) {
                        const int64_t start = (cc * U) / G;
                        if (((cc + 1) * U) / G == start) continue;
                        const float* src = p.part + ((cc * p.maxseg + (t - start / p.cpt)) * CP) * BM + m;
#pragma unroll
                        for (int j = 0; j < CP; ++j)
                            if (j < p.c) v[j] += __ldcg(src + int64_t(j) * BM);
                    }
                    if (row < p.rows_out) {
                        float* o = p.out + row;
#pragma unroll
                        for (int j = 0; j < CP; ++j)
                            if (j < p.c) o[int64_t(j) * p.ldo] = p.accumulate ? o[int64_t(j) * p.ldo] + v[j] : v[j];
                    }
                }
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 2) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
    }
}

// Tiles cut between CTAs: out[j][t*BM + m] = sum over the covering CTAs.  The CTA
// owning unit u is floor(((u + 1) G - 1) / U) for the ranges of unit_range.  Block
// (tile, 4 columns), 1024 threads: thread (slot s, row m) sums the CTAs s, s + 8, ...
// of the covering range, then the 8 slot sums are added in slot order (deterministic).
constexpr int FIX_SLOTS = 8;
__global__ void __launch_bounds__(FIX_SLOTS * BM) tc_fixup_kernel(Params p, int G) {
    __shared__ float red[FIX_SLOTS][4][BM];
    const int64_t t = blockIdx.x;
    const int64_t U = p.tiles * p.cpt;
    const int64_t u0 = t * p.cpt, u1 = (t + 1) * p.cpt - 1;
    const int64_t c_first = ((u0 + 1) * G - 1) / U, c_last = ((u1 + 1) * G - 1) / U;
    if (c_first == c_last) return;   // one CTA wrote the whole tile
    const int m = threadIdx.x % BM, slot = threadIdx.x / BM;
    const int j = int(blockIdx.y) * 4;
    const int64_t row = t * BM + m;
    float s[4] = {0.f, 0.f, 0.f, 0.f};
    for (int64_t cc = c_first + slot; cc <= c_last; cc += FIX_SLOTS) {
        const int64_t start = (cc * U) / G;
        if (((cc + 1) * U) / G == start) continue;   // a CTA with no units wrote nothing
        const float* src = p.part + ((cc * p.maxseg + (t - start / p.cpt)) * p.cp) * BM + m;
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (j + q < p.c) s[q] += src[int64_t(j + q) * BM];
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) red[slot][q][m] = s[q];
    __syncthreads();
    if (slot != 0 || row >= p.rows_out) return;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        if (j + q >= p.c) continue;
        float v = red[0][q][m];
        for (int k = 1; k < FIX_SLOTS; ++k) v += red[k][q][m];
        float* o = p.out + int64_t(j + q) * p.ldo + row;
        *o = p.accumulate ? *o + v : v;
    }
}

// hi/lo split of sign * x for a thin block (rows x len, row pitch ld; sign = +-1).
// Row r = blockIdx.y; the x blocks stride along it.
__global__ void tf32_split_kernel(const float* __restrict__ x, int rows, int64_t len, int64_t ld,
                                  float sign, float* __restrict__ xh, float* __restrict__ xl) {
    const int64_t r = blockIdx.y;
    for (int64_t l = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; l < len;
         l += int64_t(gridDim.x) * blockDim.x) {
        const float v = sign * x[r * ld + l];
        const float h = tf32_hi(v);
        xh[r * ld + l] = h;
        xl[r * ld + l] = v - h;
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
        else
            cudaGetLastError();
    }
    return fn;
}

bool encode_2d(CUtensorMap* map, CUtensorMapDataType type, const void* ptr, uint64_t inner,
               uint64_t outer, uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer,
               CUtensorMapSwizzle sw) {
    auto fn = encode_fn();
    if (fn == nullptr) return false;
    if ((reinterpret_cast<uintptr_t>(ptr) & 15) != 0 || (row_bytes & 15) != 0) return false;
    cuuint64_t dims[2] = {inner, outer};
    cuuint64_t strides[1] = {row_bytes};
    cuuint32_t box[2] = {box_inner, box_outer};
    cuuint32_t estr[2] = {1, 1};
    return fn(map, type, 2, const_cast<void*>(ptr), dims, strides, box,
              estr, CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int grid_for_units(int64_t U, int num_sms) {
    const int64_t g = U / MIN_UNITS_PER_CTA;
    return int(g < 1 ? 1 : (g < num_sms ? g : num_sms));
}

void fixup(Exec& ex, const Params& p, int G) {
    tc_fixup_kernel<<<dim3(unsigned(p.tiles), unsigned((p.c + 3) / 4)), FIX_SLOTS * BM, 0, ex.stream>>>(p, G);
    ex.launches++;
}

int64_t partial_floats(int64_t rows_out, int64_t len, int kc, int cp, int num_sms) {
    const int64_t tiles = (rows_out + BM - 1) / BM, cpt = (len + kc - 1) / kc;
    const int64_t U = tiles * cpt, G = grid_for_units(U, num_sms), per = (U + G - 1) / G;
    return G * (per / cpt + 2) * cp * BM + tiles + 32;   // partial tiles, then the tile counters
}

size_t smem_bytes(int cp) {
    if (ts_form(cp))
        return size_t(raw_ring_ts(cp)) * TILE_BYTES + size_t(x_ring(cp)) * 2 * cp * 128 + sizeof(Smem) + 1024;
    return size_t(RA) * TILE_BYTES + size_t(2 * OP) * TILE_BYTES + size_t(x_ring(cp)) * 2 * cp * 128 +
           sizeof(Smem) + 1024;
}

}  // namespace tc

// Product with an FP32 A on the tensor cores.  Returns false (nothing launched) when the
// operands do not meet the TMA alignment rules; the caller then uses the SIMT kernel.
bool tc_product_f32(Exec& ex, const float* A, int64_t n, int64_t d, int64_t lda, bool trans, int c,
                    const float* X, int64_t ldx, float* Y, int64_t ldy, float* xh, float* xl,
                    float* part, int64_t part_cap, bool subtract) {
    using namespace tc;
    if (c < 1) return true;
    if ((reinterpret_cast<uintptr_t>(A) & 15) || ((lda * 4) & 15) || (reinterpret_cast<uintptr_t>(X) & 15) ||
        ((ldx * 4) & 15) || (reinterpret_cast<uintptr_t>(xh) & 15) || (reinterpret_cast<uintptr_t>(xl) & 15))
        return false;
    const int64_t len = trans ? n : d;          // contraction length
    const int64_t rows_out = trans ? d : n;     // tiled output dimension
    if (len > INT32_MAX || rows_out > INT32_MAX) return false;
    CUtensorMap tmA;
    if (!trans) {
        if (!encode_2d(&tmA, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, A, uint64_t(d), uint64_t(n), uint64_t(lda) * 4, KC, BM, CU_TENSOR_MAP_SWIZZLE_128B))
            return false;
    } else {
        if (!encode_2d(&tmA, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, A, uint64_t(d), uint64_t(n), uint64_t(lda) * 4, BM, KC, CU_TENSOR_MAP_SWIZZLE_NONE))
            return false;
    }
    const int G = ex.num_sms;
    for (int c0 = 0; c0 < c; c0 += 128) {
        const int cg = c - c0 < 128 ? c - c0 : 128;
        const int cp = (cg + 31) / 32 * 32;
        const float* Xg = X + int64_t(c0) * ldx;
        float* xhg = xh + int64_t(c0) * ldx;
        float* xlg = xl + int64_t(c0) * ldx;
        {
            int64_t bx = (len + 255) / 256;
            const int64_t cap = (4 * int64_t(G) + cg - 1) / cg;
            if (bx > cap) bx = cap;
            if (bx < 1) bx = 1;
            tf32_split_kernel<<<dim3(unsigned(bx), unsigned(cg)), 256, 0, ex.stream>>>(
                Xg, cg, len, ldx, subtract ? -1.f : 1.f, xhg, xlg);
            ex.launches++;
        }
        CUtensorMap tmXh, tmXl;
        if (!encode_2d(&tmXh, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, xhg, uint64_t(len), uint64_t(cg), uint64_t(ldx) * 4, KC, uint32_t(cp),
                       CU_TENSOR_MAP_SWIZZLE_128B) ||
            !encode_2d(&tmXl, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, xlg, uint64_t(len), uint64_t(cg), uint64_t(ldx) * 4, KC, uint32_t(cp),
                       CU_TENSOR_MAP_SWIZZLE_128B))
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
        const int64_t slots = int64_t(Gc) * p.maxseg * cp * BM;
        if (slots > part_cap) return false;
        p.part = part;
        p.status = ex.status;
        p.accumulate = subtract ? 1 : 0;
        // cut tiles are completed inside the kernel when at most four CTAs share a tile (the
        // completing CTA then adds up to four partials) and the counters fit after the slots;
        // finer splits (short products such as M = B^T B) keep the parallel fix-up kernel
        const int64_t max_share = (p.cpt + per - 1) / per + 1;
        p.tile_cnt = max_share <= 4 && slots + p.tiles <= part_cap ? reinterpret_cast<unsigned*>(part + slots)
                                                                   : nullptr;
        if (p.tile_cnt) cudaMemsetAsync(p.tile_cnt, 0, size_t(p.tiles) * sizeof(unsigned), ex.stream);
        const size_t smem = smem_bytes(cp);
        cudaError_t err;
        switch (cp) {
#define BKS_TC(CPV)                                                                         \
    case CPV:                                                                               \
        err = cudaFuncSetAttribute(tc_product_kernel<CPV>,                                  \
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)); \
        if (err == cudaSuccess) {                                                           \
            if (ex.klog) ex.klog->record(ex.stream);                                        \
            tc_product_kernel<CPV><<<Gc, NTHREADS, smem, ex.stream>>>(tmA, tmXh, tmXl, p);  \
            if (ex.klog) ex.klog->record(ex.stream);                                        \
        }                                                                                   \
        break;
            BKS_TC(32) BKS_TC(64) BKS_TC(96) BKS_TC(128)
#undef BKS_TC
            default: err = cudaErrorInvalidValue;
        }
        if (err != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        if (!p.tile_cnt) fixup(ex, p, Gc);
        ex.launches++;
    }
    return true;
}

int64_t tc_partial_floats(int64_t n, int64_t d, int c, int num_sms) {
    const int cp = ((c < 128 ? c : 128) + 31) / 32 * 32;
    const int64_t a = tc::partial_floats(n, d, tc::KC, cp, num_sms);   // A X
    const int64_t b = tc::partial_floats(d, n, tc::KC, cp, num_sms);   // A^T X
    return a > b ? a : b;
}

}  // namespace bks
