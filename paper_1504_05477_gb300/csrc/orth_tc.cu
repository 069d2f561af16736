// Block orthonormalisation of a new Krylov block on the tensor cores (Sec. 4.1/4.2: each
// block is orthonormalised against the earlier ones as it is computed): block classical
// Gram-Schmidt twice (BCGS2), then CholeskyQR twice, the second pass reduced to a
// symmetric correction when the first one left the block orthonormal to rounding level:
//   P1  C1 = Q^T W
//   P2  W' = W - Q C1;   C2 = Q^T W' and G' = W'^T W' (one cross-CTA reduction)
//   P3  W'' = W' - Q C2;   H2 = W''^T W'' = R1^T R1;   W1 = W'' R1^{-1}
//       (H2 = G' - C2^T C2 by Pythagoras with Q^T Q = I; taken as G' when C2 is only
//       the first projection's rounding error, else summed from W'' in a reduction of
//       its own)
//   P4  H3 = W1^T W1 = I + E;   Qout = W1 (I - E / 2) when ||E||_F^2 <= 1e-7 (then
//       Qout^T Qout = I - (3/4) E^2 + O(E^3)), else Qout = W1 chol(H3)^{-1}
// with every contraction on tcgen05 (kind::tf32) in three TF32 terms: for operands x, y
// split as x = hi(x) + lo(x) (hi = x with the low 13 mantissa bits cleared, lo exact in
// FP32),  x y ~ hi(x) hi(y) + hi(x) lo(y) + lo(x) hi(y),  dropping lo(x) lo(y) (2^-22).
// The tensor cores' FP32 accumulation truncates, so the two Grams the factorisations
// use (H2, H3) accumulate each 32-row K-block in its own accumulator, summed afterwards
// in round-to-nearest FP32; the final product adds only the small correction W1 (-E / 2)
// (or W1 (P - I)) to W1.
//
#include "chol_small.cuh"
#include "tc_common.cuh"

namespace bks {
namespace otc {

using namespace tc;

constexpr int NT = 256;
constexpr int NCONS = 224;              // consumer threads (warps 0-6)
constexpr int CMAX = 64;                // block width limit
constexpr int SMAX = 144;               // rows per CTA: N of the update products
constexpr int KB = 32;                  // FP32 elements per 128-byte K-major row
constexpr int NKB_W = (SMAX + KB - 1) / KB;
constexpr uint32_t TILE = 128 * 128;    // 128 rows x 128 bytes: one K-block of a small operand
constexpr uint32_t HALF = 64 * 128;     // rows 64-127 of a tile start 8 KB in
constexpr int GCH = 128;                // Gram chunk: rows of Qc per TMA box
constexpr uint32_t QR_BOX = SMAX * 128; // bytes of one update box of Qr (S16 rows at most)
// stage: Gram = Qc tile (16 KB) + its lo (16 KB); update = C tile (16 KB) + Qr box + lo
constexpr uint32_t STAGE = TILE + 2 * QR_BOX;
// Gram pass: three stages of a Qc tile and its lo (the same shared memory as the two
// update stages)
constexpr int GST = 3;
constexpr uint32_t GSTAGE = 2 * TILE;
static_assert(GST * GSTAGE <= 2 * STAGE, "the Gram stages must fit in the update stages");
constexpr int TMEM_COLS = 512;
constexpr int MMAX = 448;               // round16(m) + 64 <= 512 TMEM columns
constexpr uint64_t WAIT_NS = 1000000000ull;
constexpr int QS_PITCH = SMAX + 1;       // row pitch of the output staging buffer
constexpr int GP = 65;                   // row pitch of the 64 x 64 Cholesky buffers
constexpr uint32_t APPLY_WIN = 160;      // TMEM columns per accumulation window of an apply
// one more projection when the last one removed more than this many times the energy it
// left (the in-span error of a projection is then comparable to the out-of-span part)
constexpr float MORE_PROJ = 10.f;
// ||W1^T W1 - I||_F^2 up to which the second pass is the symmetric correction I - E / 2
// (its error (3/4) ||E||^2 then stays below 1e-7)
constexpr float NEWTON_E2 = 1e-7f;
// The second projection's coefficients C2 = Q^T W' and the Gram G' = W'^T W' are summed in
// one cross-CTA reduction, and H2 = W''^T W'' = G' - C2^T C2 is taken as G', when the first
// projection removed at most this many times the energy it left: C2 is then the first
// pass's rounding error, and C2^T C2 is far below G' (the second CholeskyQR pass corrects
// what is left)
constexpr float MERGE_RATIO = 1e4f;

__host__ __device__ constexpr int r16(int x) { return (x + 15) & ~15; }
__host__ __device__ constexpr int r4(int x) { return (x + 3) & ~3; }

// kind::tf32, D = F32, A and B K-major, M = 128
__host__ __device__ constexpr uint32_t idesc(int n) {
    return (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t(n >> 3) << 17) | (uint32_t(128 >> 4) << 24);
}
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(id), "r"(acc));
}
__device__ __forceinline__ float hi_of(float v) { return __uint_as_float(__float_as_uint(v) & 0xFFFFE000u); }
// byte offset of element (row, k) (k < 32) in a 128B-swizzled K-major tile
__device__ __forceinline__ uint32_t swz(int row, int k) {
    return uint32_t((row >> 3) * 1024 + (row & 7) * 128 + ((((k >> 2) ^ row) & 7) << 4) + ((k & 3) << 2));
}
__device__ __forceinline__ void named_sync(int id, int n) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }

struct Args {
    const float* W;       // c x ld, the new block
    float* Qout;          // c x ld (may be W)
    float* Qr_out;        // row l gets the c output values at Qr_out + l ldr (nullptr: none)
    int64_t ldr;
    int m, c;
    int64_t len, ld;
    int S;                // rows per CTA (multiple of 8)
    float* part;          // gridDim.x partial Grams of prow x cpad floats ([r][j])
    int prow, cpad;
    float* cts;           // 128 x ldct: rows j hi(C^T), 64 + j lo(C^T)
    int64_t ldct;
    float* hbuf;          // c x c reduced Gram
    unsigned* bar;        // [0] arrivals, [1] abort
    int* status;
    int* shifted_flag;
};

struct Ctl {
    uint64_t full[2], freeb[2], fin;   // update pass: two stages of STAGE bytes
    uint64_t gfull[GST], gfree[GST];   // Gram pass: GST stages of GSTAGE bytes
    uint32_t tmem;
    int abort;
    int ok;
    int bad;
};

// ------------------------------------------------------------------ grid barrier
__device__ bool grid_sync(Ctl* ctl, unsigned* bar, unsigned target, int* status) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(&bar[0], 1u);
        const uint64_t t0 = gtimer();
        int ok = 1;
        while (*reinterpret_cast<volatile unsigned*>(&bar[0]) < target) {
            if (*reinterpret_cast<volatile unsigned*>(&bar[1])) { ok = 0; break; }
            if (gtimer() - t0 > WAIT_NS) {
                atomicOr(status, ST_TIMEOUT);
                atomicExch(&bar[1], 1u);
                ok = 0;
                break;
            }
            __nanosleep(32);
        }
        __threadfence();
        ctl->ok = ok;
    }
    __syncthreads();
    return ctl->ok != 0;
}

// ------------------------------------------------------------------ per-thread pipeline state
struct Pipe {
    int fill[2] = {0, 0};      // producer: loads issued into each stage (update pass)
    int use[2] = {0, 0};       // consumers: loads consumed from each stage (update pass)
    int gfill[GST] = {0, 0, 0};   // the same for the Gram pass
    int guse[GST] = {0, 0, 0};
    int fin = 0;               // completions of the fin barrier
};

// hi / lo split of a TMA-loaded tile in place: the tile keeps hi(), `lo` gets lo()
__device__ __forceinline__ void split_tile(unsigned char* t, unsigned char* lo, uint32_t bytes) {
    float4* a = reinterpret_cast<float4*>(t);
    float4* b = reinterpret_cast<float4*>(lo);
    for (uint32_t i = threadIdx.x; i < bytes / 16; i += NCONS) {
        float4 v = a[i], h, l;
        h.x = hi_of(v.x); h.y = hi_of(v.y); h.z = hi_of(v.z); h.w = hi_of(v.w);
        l.x = v.x - h.x; l.y = v.y - h.y; l.z = v.z - h.z; l.w = v.w - h.w;
        a[i] = h;
        b[i] = l;
    }
}

// store x as (hi, lo) at row j of the small-operand tile set `ts` (K-block = l / 32)
__device__ __forceinline__ void put_small(unsigned char* ts, int j, int l, float x) {
    unsigned char* blk = ts + (l >> 5) * TILE;
    const float h = hi_of(x);
    *reinterpret_cast<float*>(blk + swz(j, l & 31)) = h;
    *reinterpret_cast<float*>(blk + swz(64 + j, l & 31)) = x - h;
}
__device__ __forceinline__ float get_small(const unsigned char* ts, int j, int l) {
    const unsigned char* blk = ts + (l >> 5) * TILE;
    return *reinterpret_cast<const float*>(blk + swz(j, l & 31)) +
           *reinterpret_cast<const float*>(blk + swz(64 + j, l & 31));
}
// store x as (hi, lo) at row l, column j of a transposed tile set (rows = the CTA's rows,
// K = the block's columns): K-block j / 32 is `rows16 * 128` bytes, lo at `lo_off`
__device__ __forceinline__ void put_rows(unsigned char* ts, uint32_t blk_bytes, uint32_t lo_off, int l, int j,
                                         float x) {
    unsigned char* blk = ts + (j >> 5) * blk_bytes;
    const float h = hi_of(x);
    *reinterpret_cast<float*>(blk + swz(l, j & 31)) = h;
    *reinterpret_cast<float*>(blk + lo_off + swz(l, j & 31)) = x - h;
}

// ------------------------------------------------------------------ reduction
// part[g][e] (g < G, partials `stride` floats apart, e < E, in float4 units) summed over g
// in order with compensated sums; this CTA reduces its stripe of [0, E) and routes each
// element (j, r) = (e % cpad, e / cpad) through out(j, r, value).  Thread t takes unit
// t % nu of a batch of nu float4 units and the partials g = t / nu (mod 256 / nu), so
// small stripes (a c x c Gram spreads over a handful of units per CTA) still keep every
// thread loading; the slice sums are then combined in slice order.
__device__ __forceinline__ void neumaier(float& S, float& C, float v) {
    const float t = S + v;
    C += fabsf(S) >= fabsf(v) ? (S - t) + v : (v - t) + S;
    S = t;
}
template <class Out>
__device__ void reduce_stripe(const float* part, int G, int64_t stride, int E, int cpad, float* red, Out out) {
    const int E4 = E / 4;
    const int q0 = int(int64_t(blockIdx.x) * E4 / G), q1 = int(int64_t(blockIdx.x + 1) * E4 / G);
    const int tid = threadIdx.x;
    for (int qb = q0; qb < q1; qb += NT) {
        const int nu = q1 - qb < NT ? q1 - qb : NT;
        const int nsl = NT / nu;
        const int u = tid % nu, sl = tid / nu;
        float S[4] = {0.f, 0.f, 0.f, 0.f}, C[4] = {0.f, 0.f, 0.f, 0.f};
        if (sl < nsl) {
            const float4* src = reinterpret_cast<const float4*>(part) + qb + u;
            for (int g0 = sl; g0 < G; g0 += 8 * nsl) {
                float4 v[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int g = g0 + i * nsl;
                    v[i] = g < G ? __ldcg(src + int64_t(g) * (stride / 4)) : make_float4(0.f, 0.f, 0.f, 0.f);
                }
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    neumaier(S[0], C[0], v[i].x);
                    neumaier(S[1], C[1], v[i].y);
                    neumaier(S[2], C[2], v[i].z);
                    neumaier(S[3], C[3], v[i].w);
                }
            }
            float* rr = red + (sl * nu + u) * 8;
#pragma unroll
            for (int t = 0; t < 4; ++t) { rr[t] = S[t]; rr[4 + t] = C[t]; }
        }
        __syncthreads();
        for (int x = tid; x < 4 * nu; x += NT) {   // (unit, component): the slices in order
            const int uu = x >> 2, t = x & 3;
            float SS = 0.f, CC = 0.f;
            for (int k = 0; k < nsl; ++k) {
                const float* r2 = red + (k * nu + uu) * 8;
                neumaier(SS, CC, r2[t]);
                neumaier(SS, CC, r2[4 + t]);
            }
            const int e = 4 * (qb + uu) + t;
            out(e % cpad, e / cpad, SS + CC);
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ the kernel
// Per-thread view of the CTA's state.  The phases below are separate, non-inlined
// functions called from several places: each phase runs once per launch, so one copy of
// its code keeps the instruction footprint (and the cold instruction fetches) small.
struct Kst {
    const CUtensorMap *tmQc, *tmQr, *tmC;
    const Args* a;
    unsigned char *ws, *stg, *ptile, *wr;
    float *gbuf, *pbuf, *qs, *red;
    Ctl* ctl;
    uint32_t tmem, lanes, wr_blk, wr_lo;
    int tid, warp, lane, G, cta, m, c, S, S16, rows, nkb, m16;
    int64_t l0;
    unsigned phase;
    Pipe pp;
};

// all threads: the MMAs committed to `fin` have completed
__device__ __forceinline__ bool finish(Kst& k) {
    wait_bar(&k.ctl->fin, uint32_t(k.pp.fin & 1), &k.ctl->abort, k.a->status);
    k.pp.fin++;
    tc_fence_after();
    __syncthreads();
    return k.ctl->abort == 0;
}

// Gram of the block with the m columns of Q: D[j][r] = sum_l W[j][l] Qc[r][l] over this
// CTA's rows (Qc chunks of 128 rows at TMEM columns r), pipelined through two stages.
__device__ __forceinline__ bool gram_q(Kst& k) {
    Ctl* ctl = k.ctl;
    volatile int* abort_flag = &ctl->abort;
    const int nch = (k.m + GCH - 1) / GCH, U = nch * k.nkb;
    if (k.warp == 7) {
        if (k.lane == 0) {
            for (int u = 0; u < U; ++u) {
                const int s = u % GST;
                if (k.pp.gfill[s] > 0 &&
                    !wait_bar(&ctl->gfree[s], uint32_t((k.pp.gfill[s] - 1) & 1), abort_flag, k.a->status))
                    break;
                mbar_expect_tx(&ctl->gfull[s], TILE);
                tma_load_2d(k.stg + s * GSTAGE, k.tmQc, int(k.l0) + (u / nch) * KB, (u % nch) * GCH, &ctl->gfull[s]);
                k.pp.gfill[s]++;
            }
        }
    } else {
        // every consumer thread runs every unit and every named barrier, also after an
        // abort (the waits then return at once and nothing is issued)
        for (int u = 0; u < U; ++u) {
            const int s = u % GST;
            unsigned char* st = k.stg + s * GSTAGE;
            if (!*abort_flag && wait_bar(&ctl->gfull[s], uint32_t(k.pp.guse[s] & 1), abort_flag, k.a->status))
                split_tile(st, st + TILE, TILE);
            fence_async_smem();
            named_sync(1, NCONS);
            if (k.tid == 0 && !*abort_flag) {
                tc_fence_after();
                const int kb = u / nch, ch = u % nch;
                const int nr = (k.m16 - ch * GCH) < GCH ? (k.m16 - ch * GCH) : GCH;
                const uint32_t id = idesc(nr);
                const uint64_t a0 = desc_sw128(smem_u32(k.ws + kb * TILE));
                const uint64_t a64 = desc_sw128(smem_u32(k.ws + kb * TILE + HALF));
                const uint64_t bh = desc_sw128(smem_u32(st)), bl = desc_sw128(smem_u32(st + TILE));
                const uint32_t d = k.tmem + uint32_t(ch * GCH);
#pragma unroll
                for (int kk = 0; kk < KB / 8; ++kk) {
                    const uint64_t adv = uint64_t(kk * 2);
                    mma(d, a0 + adv, bh + adv, id, (kb > 0 || kk > 0) ? 1u : 0u);
                    mma(d, a0 + adv, bl + adv, id, 1u);
                    mma(d, a64 + adv, bh + adv, id, 1u);
                }
                umma_commit(&ctl->gfree[s]);
            }
            k.pp.guse[s]++;
        }
        if (k.tid == 0) {
            tc_fence_after();
            umma_commit(&ctl->fin);
        }
    }
    return finish(k);
}

// Gram of the block with itself, D[j][j2] = sum_l W[j][l] W[j2][l]: the hi-hi products
// of K-block kb in their own accumulator (TMEM columns 64 kb), the correction terms in
// one more (columns 64 nkb).  An FP32 tensor-core accumulation truncates, so a long
// chain into one accumulator drifts; the short windows are summed in gram_w_out.
__device__ __forceinline__ bool gram_w(Kst& k) {
    if (k.tid == 0) {
        tc_fence_after();
        const uint32_t id = idesc(64), dc = k.tmem + uint32_t(64 * k.nkb);
        for (int kb = 0; kb < k.nkb; ++kb) {
            const uint64_t a0 = desc_sw128(smem_u32(k.ws + kb * TILE));
            const uint64_t a64 = desc_sw128(smem_u32(k.ws + kb * TILE + HALF));
            const uint32_t dh = k.tmem + uint32_t(64 * kb);
#pragma unroll
            for (int kk = 0; kk < KB / 8; ++kk) {
                const uint64_t adv = uint64_t(kk * 2);
                mma(dh, a0 + adv, a0 + adv, id, kk > 0 ? 1u : 0u);
                mma(dc, a0 + adv, a64 + adv, id, (kb > 0 || kk > 0) ? 1u : 0u);
                mma(dc, a64 + adv, a0 + adv, id, 1u);
            }
        }
        umma_commit(&k.ctl->fin);
    }
    return finish(k);
}

// Gram epilogues: lanes j < c of the accumulator -> this CTA's partial part[cta][r][j]
// (r < m: the Q Gram of gram_q; r < c: the windows of gram_w, summed in FP32)
__device__ __forceinline__ void gram_out(Kst& k, bool windowed, int roff = 0) {
    const int cols = windowed ? 64 : k.m16;
    const int R = windowed ? k.c : k.m;
    const int ngroups = (cols + 31) / 32;
    if (k.warp == 0 || k.warp == 1 || k.warp == 4 || k.warp == 5) {
        const int j = (k.warp & 1) * 32 + k.lane;
        float* dst = k.a->part + (int64_t(k.cta) * k.a->prow + roff) * k.a->cpad + j;
        for (int g = (k.warp >> 2); g < ngroups; g += 2) {
            float v[32];
            tmem_ld32(k.tmem + k.lanes + uint32_t(g * 32), v);
            if (windowed) {
                for (int w = 1; w <= k.nkb; ++w) {
                    float u[32];
                    tmem_ld32(k.tmem + k.lanes + uint32_t(64 * w + g * 32), u);
#pragma unroll
                    for (int t = 0; t < 32; ++t) v[t] += u[t];
                }
            }
            if (j < k.c) {
#pragma unroll
                for (int t = 0; t < 32; ++t) {
                    const int r = g * 32 + t;
                    if (r < R) dst[int64_t(r) * k.a->cpad] = v[t];
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
}

// Ordered cross-CTA sum of the partials (R rows): rows r < qrows are coefficients and go
// to the C tiles (global, hi / lo, read back by TMA); the next c rows are a c x c Gram and
// go to hbuf, the row after them (the projection energies) to hbuf row c
__device__ __forceinline__ bool reduce(Kst& k, int R, int qrows) {
    const bool with_q = qrows > 0;
    const Args& a = *k.a;
    __threadfence();
    if (!grid_sync(k.ctl, a.bar, ++k.phase * unsigned(k.G), a.status)) return false;
    const int c = k.c;
    reduce_stripe(a.part, k.G, int64_t(a.prow) * a.cpad, R * a.cpad, a.cpad, k.red, [&](int j, int r, float v) {
        if (j >= c) return;
        if (r < qrows) {
            const float h = hi_of(v);
            a.cts[int64_t(j) * a.ldct + r] = h;
            a.cts[int64_t(64 + j) * a.ldct + r] = v - h;
        } else {
            const int g = r - qrows;
            a.hbuf[g < c ? j * c + g : c * c + j] = v;   // row c: the energies ||C_j||^2
        }
    });
    if (with_q) asm volatile("fence.proxy.async.global;" ::: "memory");
    __threadfence();
    const bool ok = grid_sync(k.ctl, a.bar, ++k.phase * unsigned(k.G), a.status);
    if (with_q) asm volatile("fence.proxy.async.global;" ::: "memory");
    return ok;
}

// update pass: D[j][l] = sum_r C[r][j] Q[l][r] (TMEM columns l < S16), C tiles and Qr
// boxes of 32 columns of Q pipelined through two stages
__device__ __forceinline__ bool update_pass(Kst& k) {
    Ctl* ctl = k.ctl;
    volatile int* abort_flag = &ctl->abort;
    const int U = (k.m + KB - 1) / KB;
    const uint32_t qbytes = uint32_t(k.S16) * 128;
    if (k.warp == 7) {
        if (k.lane == 0) {
            for (int u = 0; u < U; ++u) {
                const int s = u & 1;
                if (k.pp.fill[s] > 0 &&
                    !wait_bar(&ctl->freeb[s], uint32_t((k.pp.fill[s] - 1) & 1), abort_flag, k.a->status))
                    break;
                unsigned char* st = k.stg + s * STAGE;
                mbar_expect_tx(&ctl->full[s], TILE + qbytes);
                tma_load_2d(st, k.tmC, u * KB, 0, &ctl->full[s]);
                tma_load_2d(st + TILE, k.tmQr, u * KB, int(k.l0), &ctl->full[s]);
                k.pp.fill[s]++;
            }
        }
    } else {
        for (int u = 0; u < U; ++u) {
            const int s = u & 1;
            unsigned char* st = k.stg + s * STAGE;
            if (!*abort_flag && wait_bar(&ctl->full[s], uint32_t(k.pp.use[s] & 1), abort_flag, k.a->status))
                split_tile(st + TILE, st + TILE + QR_BOX, qbytes);
            fence_async_smem();
            named_sync(1, NCONS);
            if (k.tid == 0 && !*abort_flag) {
                tc_fence_after();
                const uint32_t id = idesc(k.S16);
                const uint64_t a0 = desc_sw128(smem_u32(st)), a64 = desc_sw128(smem_u32(st + HALF));
                const uint64_t bh = desc_sw128(smem_u32(st + TILE)), bl = desc_sw128(smem_u32(st + TILE + QR_BOX));
#pragma unroll
                for (int kk = 0; kk < KB / 8; ++kk) {
                    const uint64_t adv = uint64_t(kk * 2);
                    mma(k.tmem, a0 + adv, bh + adv, id, (u > 0 || kk > 0) ? 1u : 0u);
                    mma(k.tmem, a0 + adv, bl + adv, id, 1u);
                    mma(k.tmem, a64 + adv, bh + adv, id, 1u);
                }
                umma_commit(&ctl->freeb[s]);
            }
            k.pp.use[s]++;
        }
        if (k.tid == 0) {
            tc_fence_after();
            umma_commit(&ctl->fin);
        }
    }
    return finish(k);
}

// epilogue of an update pass: W[j][l] -= D[j][l] in the W tiles.  This CTA's share of
// ||D_j||^2 (= ||Q C_j||^2 = ||C_j||^2, the energy the projection removed) goes to row c
// of its partial, which the next reduction of a c x c Gram sums with it.
__device__ __forceinline__ void update_out(Kst& k, int erow) {
    const int ngroups = (k.S16 + 31) / 32;
    if (k.warp == 0 || k.warp == 1 || k.warp == 4 || k.warp == 5) {
        const int j = (k.warp & 1) * 32 + k.lane;
        float e2 = 0.f;
        for (int g = (k.warp >> 2); g < ngroups; g += 2) {
            float v[32];
            tmem_ld32(k.tmem + k.lanes + uint32_t(g * 32), v);
            if (j < k.c) {
#pragma unroll
                for (int t = 0; t < 32; ++t) {
                    const int l = g * 32 + t;
                    if (l < k.S16) put_small(k.ws, j, l, l < k.rows ? get_small(k.ws, j, l) - v[t] : 0.f);
                    if (l < k.rows) e2 = fmaf(v[t], v[t], e2);
                }
            }
        }
        // the two warps of a lane quarter (column groups g even / odd) add their shares
        float* rr = k.red + 32 * 8 * 2;   // 128 floats past the other uses of the scratch
        if (k.warp >= 4) rr[j] = e2;
        named_sync(2, 128);
        if (k.warp < 4 && j < k.c)
            k.a->part[(int64_t(k.cta) * k.a->prow + erow) * k.a->cpad + j] = e2 + rr[j];
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
}

// gbuf = the reduced c x c Gram (row pitch GP)
__device__ __forceinline__ void load_h(Kst& k) {
    for (int e = k.tid; e < k.c * k.c; e += NT) k.gbuf[(e / k.c) * GP + e % k.c] = __ldcg(k.a->hbuf + e);
    __syncthreads();
}

// another projection pass?  ||C||_F^2 (row c of hbuf) against trace(H2) = ||W''||_F^2:
// the same reduced values in every CTA, so every CTA takes the same decision
__device__ __forceinline__ bool more_projection(Kst& k) {
    if (k.tid == 0) {
        float cn = 0.f, tr = 0.f;
        for (int j = 0; j < k.c; ++j) {
            cn += __ldcg(k.a->hbuf + k.c * k.c + j);
            tr += k.gbuf[j * GP + j];
        }
        k.ctl->bad = (cn > MORE_PROJ * tr) ? 1 : 0;
    }
    __syncthreads();
    return k.ctl->bad != 0;
}

// H2 = G' for the merged second projection?  The energy the first projection removed
// (row c of hbuf) against trace(G') = ||W'||_F^2; the same in every CTA
__device__ __forceinline__ bool merge_holds(Kst& k) {
    if (k.tid == 0) {
        float cn = 0.f, tr = 0.f;
        for (int j = 0; j < k.c; ++j) {
            cn += __ldcg(k.a->hbuf + k.c * k.c + j);
            tr += k.gbuf[j * GP + j];
        }
        k.ctl->bad = (cn <= MERGE_RATIO * tr) ? 0 : 1;   // NaN: not merged
    }
    __syncthreads();
    return k.ctl->bad == 0;
}

// pbuf = R^{-T} for gbuf = R^T R (shifted retries and breakdown as chol_inv_block_t)
__device__ __forceinline__ void chol(Kst& k) {
    chol_inv_block_t<4>(k.gbuf, GP, k.c, k.pbuf, GP, k.a->status, k.a->shifted_flag);
    __syncthreads();
}

// P (c x c, pitch GP) -> the A tiles of an apply (hi rows 0-63, lo rows 64-127, K = b);
// minus_i: P - I instead (the final apply forms W1 + W1 (P - I): there P is close to the
// identity, so the tensor cores only add a small correction to W1)
__device__ __forceinline__ void p_tiles(Kst& k, bool minus_i) {
    for (int e = k.tid; e < 64 * 64; e += NT) {
        const int i = e / 64, b = e % 64;
        const float pv = (i < k.c && b < k.c) ? k.pbuf[i * GP + b] : 0.f;
        put_small(k.ptile, i, b, pv - (minus_i && i == b && i < k.c ? 1.f : 0.f));
    }
    fence_async_smem();
    __syncthreads();
}

// the block from the W tiles into the row tiles (rows = this CTA's rows, K = the
// block's columns), the B operand of an apply
__device__ __forceinline__ void rows_from_w(Kst& k) {
    for (int e = k.tid; e < k.S16 * 64; e += NT) {
        const int l = e / 64, j = e % 64;
        put_rows(k.wr, k.wr_blk, k.wr_lo, l, j, (j < k.c && l < k.rows) ? get_small(k.ws, j, l) : 0.f);
    }
    fence_async_smem();
    __syncthreads();
}

// apply: D[i][l] = sum_b P[i][b] W[l][b] (K = the block's columns, 2 K-blocks): the hi-hi
// products of each K-block in their own accumulator (TMEM columns 0 and APPLY_WIN), the
// corrections in a third (2 APPLY_WIN), summed in apply_out
__device__ __forceinline__ bool apply_pass(Kst& k) {
    if (k.tid == 0) {
        tc_fence_after();
        const uint32_t id = idesc(k.S16), dc = k.tmem + 2 * APPLY_WIN;
        for (int kb = 0; kb < 2; ++kb) {
            const uint64_t a0 = desc_sw128(smem_u32(k.ptile + kb * TILE));
            const uint64_t a64 = desc_sw128(smem_u32(k.ptile + kb * TILE + HALF));
            const uint64_t bh = desc_sw128(smem_u32(k.wr + kb * k.wr_blk));
            const uint64_t bl = desc_sw128(smem_u32(k.wr + k.wr_lo + kb * k.wr_blk));
            const uint32_t dh = k.tmem + uint32_t(kb) * APPLY_WIN;
#pragma unroll
            for (int kk = 0; kk < KB / 8; ++kk) {
                const uint64_t adv = uint64_t(kk * 2);
                mma(dh, a0 + adv, bh + adv, id, kk > 0 ? 1u : 0u);
                mma(dc, a0 + adv, bl + adv, id, (kb > 0 || kk > 0) ? 1u : 0u);
                mma(dc, a64 + adv, bh + adv, id, 1u);
            }
        }
        umma_commit(&k.ctl->fin);
    }
    return finish(k);
}

// epilogue of an apply: final = false: the result is the new block (W tiles);
// final = true: the output block Qout = W1 + D (and its row-major copy)
__device__ __forceinline__ void apply_out(Kst& k, bool final) {
    const int ngroups = (k.S16 + 31) / 32;
    const Args& a = *k.a;
    if (k.warp == 0 || k.warp == 1 || k.warp == 4 || k.warp == 5) {
        const int i = (k.warp & 1) * 32 + k.lane;
        for (int g = (k.warp >> 2); g < ngroups; g += 2) {
            float v[32], u[32], w[32];
            tmem_ld32_async(k.tmem + k.lanes + uint32_t(g * 32), reinterpret_cast<uint32_t(&)[32]>(v));
            tmem_ld32_async(k.tmem + k.lanes + uint32_t(APPLY_WIN + g * 32), reinterpret_cast<uint32_t(&)[32]>(u));
            tmem_wait();
            tmem_ld32(k.tmem + k.lanes + uint32_t(2 * APPLY_WIN + g * 32), w);
            if (i < k.c) {
#pragma unroll
                for (int t = 0; t < 32; ++t) {
                    const int l = g * 32 + t;
                    const float d = (v[t] + u[t]) + w[t];
                    if (!final) {
                        if (l < k.S16) put_small(k.ws, i, l, l < k.rows ? d : 0.f);
                    } else if (l < k.rows) {
                        const float q = get_small(k.ws, i, l) + d;   // W1 + W1 (P - I)
                        k.qs[i * QS_PITCH + l] = q;
                        if (a.Qr_out) a.Qr_out[(k.l0 + l) * a.ldr + i] = q;
                    }
                }
            }
        }
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    if (final) {   // the output block, row by row (coalesced)
        for (int e = k.tid; e < k.c * k.rows; e += NT) {
            const int i = e / k.rows, l = e - i * k.rows;
            a.Qout[int64_t(i) * a.ld + k.l0 + l] = k.qs[i * QS_PITCH + l];
        }
    }
}

// second CholeskyQR pass.  W1 is orthonormal up to E = W1^T W1 - I from the first pass's
// rounding.  When E is small, Qout = W1 (I - E / 2) gives Qout^T Qout = I - (3/4) E^2 +
// O(E^3), with the span unchanged: no second factorisation.  Otherwise Qout =
// W1 chol(H3)^{-1}.  Every CTA sees the same H3, so all take the same branch.
__device__ __forceinline__ void second_factor(Kst& k) {
    Ctl* ctl = k.ctl;
    const int c = k.c;
    float e2 = 0.f;
    for (int e = k.tid; e < c * c; e += NT) {
        const int i = e / c, j = e % c;
        const float v = k.gbuf[i * GP + j] - (i == j ? 1.f : 0.f);
        e2 = fmaf(v, v, e2);
    }
    for (int o = 16; o > 0; o >>= 1) e2 += __shfl_xor_sync(0xffffffffu, e2, o);
    if (k.lane == 0) k.red[k.warp] = e2;
    __syncthreads();
    if (k.tid == 0) {
        float t = 0.f;
        for (int w = 0; w < NT / 32; ++w) t += k.red[w];
        ctl->bad = (t <= NEWTON_E2) ? 0 : 1;   // NaN goes to the factorisation (which flags it)
    }
    __syncthreads();
    if (ctl->bad == 0) {
        for (int e = k.tid; e < c * c; e += NT) {
            const int i = e / c, j = e % c;
            k.pbuf[i * GP + j] = (i == j ? 1.5f : 0.f) - 0.5f * k.gbuf[i * GP + j];   // I - E / 2
        }
        __syncthreads();
    } else {
        chol(k);
    }
}

__global__ void __launch_bounds__(NT, 1)
    orth_tc_kernel(const __grid_constant__ CUtensorMap tmQc, const __grid_constant__ CUtensorMap tmQr,
                   const __grid_constant__ CUtensorMap tmC, const __grid_constant__ Args a) {
    extern __shared__ unsigned char smem_dyn[];
    unsigned char* base = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_dyn) + 1023) & ~uintptr_t(1023));
    Kst k;
    k.tmQc = &tmQc; k.tmQr = &tmQr; k.tmC = &tmC; k.a = &a;
    k.ws = base;                                   // W: NKB_W tiles (+ 8 KB read by row-64 descriptors)
    k.stg = k.ws + NKB_W * TILE + HALF;            // 2 stages
    k.ctl = reinterpret_cast<Ctl*>(k.stg + 2 * STAGE);
    k.red = reinterpret_cast<float*>(k.ctl + 1);   // reduction scratch: 8 x 32 x 8 floats
    // between the pipelined passes the stages hold the inverse factor's tiles (2 K-blocks,
    // hi rows 0-63 / lo rows 64-127), then either the Cholesky buffers (64 x GP floats
    // each) or, once the factor is in its tiles, the block transposed (rows = this CTA's
    // rows, K = the block's columns: 2 K-blocks of hi, then 2 of lo)
    k.ptile = k.stg;
    k.gbuf = reinterpret_cast<float*>(k.stg + 2 * TILE);
    k.pbuf = k.gbuf + 64 * GP;
    k.wr = k.stg + 2 * TILE;
    k.qs = reinterpret_cast<float*>(k.stg);        // the output block (after the last apply)
    k.tid = threadIdx.x; k.warp = k.tid >> 5; k.lane = k.tid & 31;
    k.G = gridDim.x; k.cta = blockIdx.x;
    k.m = a.m; k.c = a.c; k.S = a.S; k.S16 = r16(a.S);
    k.l0 = int64_t(k.cta) * k.S;
    k.rows = int(a.len - k.l0 < k.S ? a.len - k.l0 : k.S);
    k.nkb = (k.S + KB - 1) / KB;
    k.m16 = r16(k.m);
    k.wr_blk = uint32_t(k.S16) * 128;
    k.wr_lo = 2 * k.wr_blk;
    k.phase = 0;
    Ctl* ctl = k.ctl;
    const int m = k.m, c = k.c;

    if (k.tid == 0) {
        for (int s = 0; s < 2; ++s) { mbar_init(&ctl->full[s], 1); mbar_init(&ctl->freeb[s], 1); }
        for (int s = 0; s < GST; ++s) { mbar_init(&ctl->gfull[s], 1); mbar_init(&ctl->gfree[s], 1); }
        mbar_init(&ctl->fin, 1);
        ctl->abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (k.warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&ctl->tmem)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    // W slice -> (hi, lo) tiles; zero beyond the block's columns and the CTA's rows
    for (int e = k.tid; e < 64 * k.nkb * KB; e += NT) {
        const int j = e / (k.nkb * KB), l = e % (k.nkb * KB);
        put_small(k.ws, j, l, (j < c && l < k.rows) ? a.W[int64_t(j) * a.ld + k.l0 + l] : 0.f);
    }
    for (int e = k.tid; e < int(HALF / 4); e += NT) reinterpret_cast<float*>(k.ws + NKB_W * TILE)[e] = 0.f;
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    k.tmem = ctl->tmem;
    k.lanes = uint32_t((k.warp & 3) * 32) << 16;   // this warp's TMEM lane quarter
    bool ok = true;

    // P1: C1 = Q^T W, W' = W - Q C1 (the energy it removed to partial row m + c)
    // P2: C2 = Q^T W' and G' = W'^T W' in one reduction, W'' = W' - Q C2; H2 = G' when
    //     merge_holds, else (P3) H2 = W''^T W'' in a reduction of its own
    bool merged = false;
    if (m > 0) {
        ok = gram_q(k);
        if (ok) gram_out(k, false);
        if (ok) ok = reduce(k, m, m);
        if (ok) ok = update_pass(k);
        if (ok) update_out(k, m + c);
        if (ok) ok = gram_q(k);
        if (ok) gram_out(k, false);
        if (ok) ok = gram_w(k);
        if (ok) gram_out(k, true, m);
        if (ok) ok = reduce(k, m + c + 1, m);
        if (ok) ok = update_pass(k);
        if (ok) update_out(k, c);
        if (ok) {   // after the update: its stages share shared memory with gbuf
            load_h(k);
            merged = merge_holds(k);
        }
    }
    // P3: H2 = W''^T W''; then R1^T R1 = H2, W1 = W'' R1^{-1}
    if (ok && !merged) {
        ok = gram_w(k);
        if (ok) gram_out(k, true);
        if (ok) ok = reduce(k, m > 0 ? c + 1 : c, 0);
        if (ok) load_h(k);
    }
    // The tensor cores' truncating accumulation makes the error of Q C roughly
    // proportional to Q C, i.e. it lies inside span(Q).  When the block was almost
    // entirely inside span(Q) (the second projection removed much more energy than it
    // left: a converged or rank-deficient Krylov direction), that error is not small
    // against what is left, and one more projection removes it (at most two more).
    for (int extra = 0; extra < 2 && ok && m > 0 && !merged && more_projection(k); ++extra) {
        ok = gram_q(k);
        if (ok) gram_out(k, false);
        if (ok) ok = reduce(k, m, m);
        if (ok) ok = update_pass(k);
        if (ok) update_out(k, c);
        if (ok) ok = gram_w(k);
        if (ok) gram_out(k, true);
        if (ok) ok = reduce(k, c + 1, 0);
        if (ok) load_h(k);
    }
    if (ok) {
        chol(k);
        p_tiles(k, false);
        rows_from_w(k);
        ok = apply_pass(k);
        if (ok) apply_out(k, false);
    }
    // P4: H3 = W1^T W1, Qout = W1 (I - E / 2) or W1 chol(H3)^{-1}
    if (ok) ok = gram_w(k);
    if (ok) gram_out(k, true);
    if (ok) ok = reduce(k, c, 0);
    if (ok) {
        load_h(k);
        second_factor(k);
        p_tiles(k, true);
        rows_from_w(k);
        ok = apply_pass(k);
        if (ok) apply_out(k, true);
    }
    if (!ok && k.tid == 0) atomicExch(&a.bar[1], 1u);   // releases the other CTAs' barriers

    // drain: every TMA load issued has landed before shared memory is released (bounded)
    if (k.warp == 7 && k.lane == 0) {
        for (int s = 0; s < 2; ++s)
            if (k.pp.fill[s] > 0) drain_bar(&ctl->full[s], (k.pp.fill[s] - 1) & 1);
        for (int s = 0; s < GST; ++s)
            if (k.pp.gfill[s] > 0) drain_bar(&ctl->gfull[s], (k.pp.gfill[s] - 1) & 1);
    }
    tc_fence_before();
    __syncthreads();
    if (k.warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(k.tmem), "r"(TMEM_COLS));
    }
}

size_t smem_bytes() { return size_t(NKB_W) * TILE + HALF + 2 * STAGE + sizeof(Ctl) + 8 * 32 * 8 * 4 + 1024; }

// Failure-path self-test of the two bounded waits every pipeline and cooperative kernel
// here relies on, each on a condition that nothing satisfies: which = 0 an mbarrier phase
// no thread or copy completes (tc::wait_bar, the TMA / MMA pipeline wait), which = 1 the
// grid barrier with one more arrival expected than there are CTAs (grid_sync).  Both give
// up after WAIT_NS and flag ST_TIMEOUT; the kernel then returns normally.
__global__ void wait_selftest_kernel(int which, unsigned* bar, int* status) {
    __shared__ Ctl ctl;
    __shared__ uint64_t never;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        tc::mbar_init(&never, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (which == 0) {
        if (threadIdx.x == 0) tc::wait_bar(&never, 0, &abort_flag, status);
    } else {
        grid_sync(&ctl, bar, gridDim.x + 1, status);
    }
}

}  // namespace otc

// Rows per CTA and CTAs of the tensor-core orthonormalisation for a block of length len.
static void otc_grid(int64_t len, int num_sms, int& S, int& G) {
    int64_t s = (len + num_sms - 1) / num_sms;
    s = (s + 7) / 8 * 8;
    if (s < 8) s = 8;
    S = int(s);
    G = int((len + s - 1) / s);
}

bool orth_tc_fits(int64_t len, int m, int c, int num_sms) {
    int S, G;
    otc_grid(len, num_sms, S, G);
    return c >= 1 && c <= otc::CMAX && m >= 0 && m <= otc::MMAX && S <= otc::SMAX && G <= num_sms;
}

size_t orth_tc_part_floats(int64_t len, int mmax, int c, int num_sms) {
    int S, G;
    otc_grid(len, num_sms, S, G);
    return size_t(G) * size_t(mmax + c + 1) * size_t(otc::r4(c));
}

// W (c x ld) against Qc (m x ld) with its row-major copy Qr (len x ldr, columns [0, m));
// result in Qout and, when Qr_out is non-null, in row-major form at Qr_out (pitch ldr).
// False (nothing launched) when the shapes or alignments do not fit.
bool orth_tc(Exec& ex, int64_t len, int64_t ld, const float* Qc, int m, const float* W, int c, float* Qout,
             const float* Qr, float* Qr_out, int64_t ldr, float* part, int64_t part_cap, float* cts, int64_t ldct,
             float* hbuf, unsigned* bar, int* shifted_flag) {
    using namespace otc;
    if (!orth_tc_fits(len, m, c, ex.num_sms) || part == nullptr || cts == nullptr || hbuf == nullptr ||
        bar == nullptr)
        return false;
    if (m > 0 && (Qc == nullptr || Qr == nullptr)) return false;
    if (((ld * 4) & 15) || ((ldr * 4) & 15) || ((ldct * 4) & 15) || (reinterpret_cast<uintptr_t>(Qc) & 15) ||
        (reinterpret_cast<uintptr_t>(Qr) & 15) || (reinterpret_cast<uintptr_t>(cts) & 15) || ldct < m)
        return false;
    int S, G;
    otc_grid(len, ex.num_sms, S, G);
    const int cpad = r4(c), prow = m + c + 1;
    if (int64_t(G) * prow * cpad > part_cap) return false;
    CUtensorMap tmQc, tmQr, tmC;
    memset(&tmQc, 0, sizeof(tmQc));
    memset(&tmQr, 0, sizeof(tmQr));
    memset(&tmC, 0, sizeof(tmC));
    if (m > 0) {
        if (!encode_2d(&tmQc, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, Qc, uint64_t(len), uint64_t(m), uint64_t(ld) * 4, KB,
                       GCH, CU_TENSOR_MAP_SWIZZLE_128B) ||
            !encode_2d(&tmQr, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, Qr, uint64_t(m), uint64_t(len), uint64_t(ldr) * 4, KB,
                       uint32_t(r16(S)), CU_TENSOR_MAP_SWIZZLE_128B) ||
            !encode_2d(&tmC, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, cts, uint64_t(m), 128, uint64_t(ldct) * 4, KB, 128,
                       CU_TENSOR_MAP_SWIZZLE_128B))
            return false;
    }
    const size_t smem = smem_bytes();
    if (allow_dynamic_smem(reinterpret_cast<const void*>(orth_tc_kernel), smem) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    Args a;
    a.W = W; a.Qout = Qout; a.Qr_out = Qr_out; a.ldr = ldr;
    a.m = m; a.c = c; a.len = len; a.ld = ld; a.S = S;
    a.part = part; a.prow = prow; a.cpad = cpad; a.cts = cts; a.ldct = ldct; a.hbuf = hbuf; a.bar = bar;
    a.status = ex.status; a.shifted_flag = shifted_flag;
    cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), ex.stream);
    void* args[] = {&tmQc, &tmQr, &tmC, &a};
    if (cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(orth_tc_kernel), dim3(G), dim3(NT), args, smem,
                                    ex.stream) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    ex.launches++;
    return true;
}

bool wait_selftest(Exec& ex, int which, unsigned* bar) {
    if (which != 0 && which != 1) return false;
    cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), ex.stream);
    // two CTAs for the grid barrier: both are resident, neither reaches the target
    otc::wait_selftest_kernel<<<which == 0 ? 1 : 2, 32, 0, ex.stream>>>(which, bar, ex.status);
    ex.launches++;
    return true;
}

}  // namespace bks
