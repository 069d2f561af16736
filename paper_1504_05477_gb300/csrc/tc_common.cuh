// Pieces shared by the tensor-core product kernels (FP32 A on kind::tf32, BF16 A on
// kind::f16): mbarrier and TMA wrappers, bounded waits, tcgen05 descriptors and TMEM
// loads, the stream-K unit split and the fix-up of tiles cut between CTAs.
#pragma once
#include <cuda.h>
#include <cudaTypedefs.h>

#include "common.cuh"

namespace bks {
namespace tc {

constexpr int BM = 128;                        // UMMA M: rows of D per tile
constexpr uint64_t WAIT_NS = 1000000000ull;    // 1 s bound on every wait

struct Params {
    int mode;          // 0: AX, 1: ATX
    int c;             // real output columns (<= 128)
    int cp;            // padded columns (32, 64, 96, 128)
    int64_t rows_out;  // extent of the tiled dimension (n for AX, d for ATX)
    int64_t tiles;     // ceil(rows_out / BM)
    int64_t cpt;       // chunks per tile (contraction length / chunk depth, rounded up)
    float* out;        // c x ldo
    int64_t ldo;
    float* part;       // partial tiles: [grid][maxseg][cp][BM]
    int maxseg;
    int* status;
    int accumulate;    // 1: out += result (out is read first), 0: out = result
    unsigned* tile_cnt;   // non-null: per-tile arrival counters (zeroed before the launch); the
                          // last CTA to finish a cut tile sums its partials (no fix-up launch)
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(
                     smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Bounded wait: false on timeout (status flagged, abort raised) or when another role
// already aborted.
__device__ __forceinline__ bool wait_bar(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                         int* status) {
    if (mbar_try(bar, parity)) return true;
    const uint64_t t0 = gtimer();
    while (true) {
        if (mbar_try(bar, parity)) return true;
        if (*abort_flag) return false;
        if (gtimer() - t0 > WAIT_NS) {
            atomicOr(status, ST_TIMEOUT);
            *abort_flag = 1;
            return false;
        }
    }
}
// Wait (bounded, no status) for the last transfer into a stage before shared memory is
// released.
__device__ __forceinline__ void drain_bar(uint64_t* bar, int last_parity) {
    if (last_parity < 0) return;
    const uint64_t t0 = gtimer();
    while (!mbar_try(bar, uint32_t(last_parity)) && gtimer() - t0 < WAIT_NS) {
    }
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, "
        "{%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}
// UMMA shared-memory descriptor, 128-byte swizzle.  K-major operand: 8-row atoms `sbo`
// bytes apart (lbo unused).  MN-major operand: 128-byte rows along M hold 64 16-bit
// elements; successive 64-element blocks of M lie `lbo` bytes apart and successive
// groups of 8 K rows `sbo` bytes apart.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr, uint32_t lbo = 16, uint32_t sbo = 1024) {
    uint64_t d = uint64_t((saddr & 0x3FFFF) >> 4);
    d |= uint64_t((lbo >> 4) & 0x3FFF) << 16;
    d |= uint64_t((sbo >> 4) & 0x3FFF) << 32;
    d |= uint64_t(1) << 46;            // descriptor version
    d |= uint64_t(2) << 61;            // 128-byte swizzle
    return d;
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// 32 consecutive columns of this warp's 32 TMEM lanes into registers; the caller waits
// (tmem_wait) before reading them, so several loads can be in flight.
__device__ __forceinline__ void tmem_ld32_async(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
        "%28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
// 32 consecutive columns of this warp's 32 TMEM lanes from registers (then tmem_wait_st).
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
        "%28, %29, %30, %31, %32};" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
        "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]),
        "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]),
        "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
        : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
        "%28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Units of CTA `cta`: [start, end) in the flattened (tile, chunk) order.
__device__ __forceinline__ void unit_range(int64_t U, int G, int cta, int64_t& s, int64_t& e) {
    s = (int64_t(cta) * U) / G;
    e = (int64_t(cta + 1) * U) / G;
}

// Position (tile t, chunk kc) of a CTA's current unit, advanced by one increment per unit:
// one 64-bit division at the start of the range instead of one per unit (a 64-bit
// division is a long software sequence, and one per unit capped a role's unit rate).
struct UnitWalk {
    int64_t t;
    int kc, cpt;
    __device__ UnitWalk(int64_t u, int64_t cpt_) : t(u / cpt_), kc(int(u % cpt_)), cpt(int(cpt_)) {}
    __device__ __forceinline__ void next() {
        if (++kc == cpt) {
            kc = 0;
            ++t;
        }
    }
};

// Driver-API tensor-map encoder, looked up once.
PFN_cuTensorMapEncodeTiled_v12000 encode_fn();
bool encode_2d(CUtensorMap* map, CUtensorMapDataType type, const void* ptr, uint64_t inner,
               uint64_t outer, uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer,
               CUtensorMapSwizzle sw);
// CTAs of a stream-K launch over U units: one per SM, but no fewer than
// MIN_UNITS_PER_CTA units each (a short contraction then spreads over fewer CTAs and
// leaves fewer partial tiles to sum).
constexpr int64_t MIN_UNITS_PER_CTA = 16;
int grid_for_units(int64_t U, int num_sms);
// Sum the tiles cut between the G CTAs of a launch into p.out (deterministic order).
void fixup(Exec& ex, const Params& p, int G);
// Partial-tile floats a stream-K launch over (rows_out / BM) x (len / kc) units needs.
int64_t partial_floats(int64_t rows_out, int64_t len, int kc, int cp, int num_sms);

}  // namespace tc
}  // namespace bks
