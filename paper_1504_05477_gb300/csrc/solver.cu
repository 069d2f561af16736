// Host orchestration of Algorithms 1 and 2 and the C-ABI declared in include/bks.h.
//
// Block Krylov Iteration (Alg. 2) as run here:
//   Pi -> W_0 = A Pi -> Q_0 = orth(W_0)
//   for i = 1..q_eff:  B_{i-1} = A^T Q_{i-1};  W_i = A B_{i-1};
//                      Q_i = orth(W_i against Q_0..Q_{i-1})          (Sec. 4.2)
//   B_q = A^T Q_q;  M = B^T B (= Q^T A A^T Q, Lemma 4.1);  M = Ubar Lambda Ubar^T;
//   Z = Q Ubar_k;  sigma_i = |B ubar_i| (= |A^T z_i|, the Ritz values).
// Simultaneous Iteration (Alg. 1): Q <- orth(A (A^T Q)) q times, then the same
// Rayleigh-Ritz step with w = k (Sec. 4.1).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <cudaTypedefs.h>

#include "../../include/bks.h"
#include "common.cuh"
#include "ctx.cuh"

namespace bks {
namespace tc {
PFN_cuTensorMapEncodeTiled_v12000 encode_fn();   // tensor-core products: looked up on first use
}
}  // namespace bks


using namespace bks;

// A solve whose status has been queued for copy-back but not yet read (batched calls).
struct PendingSolve {
    bool active = false;
    int q_eff = 0, w = 0;
    bool deflated = false, basis_only = false;
    int launches = 0, product_launches = 0;
    int eig_path = 0;
    double product_bytes = 0, product_flops = 0;
};

struct bks_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;            // sub-contexts of batched calls own their stream
    std::vector<bks_ctx*> subs;         // batched calls: one sub-context per stream
    PendingSolve pending;
    int num_sms = 148;
    void* ws = nullptr;
    size_t ws_bytes = 0;
    bool ws_owned = false;
    int* host_status = nullptr;   // pinned: [status, sweeps, shifted]
    double* host_vals = nullptr;  // pinned, 256 doubles: Ritz values of the adaptive stopping test
    std::string last_error;
    std::vector<cudaEvent_t> events;
    KernelLog klog;
    std::map<std::string, int> batch_sms;   // SM budget per batch signature (bks_batched_autotune)
    ~bks_ctx() {
        for (int i = 0; i < klog.created; ++i) cudaEventDestroy(klog.ev[i]);
    }
};

namespace {

constexpr int BKS_VERSION = 100;
constexpr int BKS_BATCH_THREADS = 8;   // host threads issuing the solves of a batch
constexpr int BKS_BATCH_STREAMS = 16;  // solves of a batch in flight at once (two per thread)

struct Arena {
    size_t off = 0;
    size_t take(size_t bytes) {
        const size_t o = off;
        off += (bytes + 255) / 256 * 256;
        return o;
    }
};

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

bks_status fail(bks_ctx* ctx, bks_status s, const std::string& msg) {
    if (ctx) ctx->last_error = msg;
    return s;
}

bks_status cuda_fail(bks_ctx* ctx, cudaError_t e, const char* where) {
    return fail(ctx, BKS_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

bks_status ensure_ws(bks_ctx* ctx, size_t bytes) {
    if (bytes <= ctx->ws_bytes && ctx->ws != nullptr) return BKS_OK;
    if (ctx->ws != nullptr && !ctx->ws_owned)
        return fail(ctx, BKS_ERR_NOMEM, "caller workspace too small: need " + std::to_string(bytes) +
                                            " bytes, have " + std::to_string(ctx->ws_bytes));
    if (ctx->ws_owned && ctx->ws) {
        cudaStreamSynchronize(ctx->stream);
        cudaFree(ctx->ws);
        ctx->ws = nullptr;
        ctx->ws_bytes = 0;
    }
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, BKS_ERR_NOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
    }
    ctx->ws = p;
    ctx->ws_bytes = bytes;
    ctx->ws_owned = true;
    return BKS_OK;
}

bool dtype_ok(int dt) { return dt == BKS_F64 || dt == BKS_F32 || dt == BKS_BF16; }
size_t dtype_bytes(int dt) { return dt == BKS_F64 ? 8 : dt == BKS_F32 ? 4 : 2; }

bks_status check_matrix(bks_ctx* ctx, const bks_matrix* A) {
    if (A == nullptr) return fail(ctx, BKS_ERR_INVALID_ARG, "A is NULL");
    if (A->n < 1 || A->d < 1) return fail(ctx, BKS_ERR_INVALID_ARG, "A must be at least 1 x 1");
    if (!dtype_ok(A->dtype)) return fail(ctx, BKS_ERR_INVALID_ARG, "unknown A dtype");
    if (A->kind == BKS_DENSE) {
        if (A->vals == nullptr) return fail(ctx, BKS_ERR_INVALID_ARG, "A->vals is NULL");
        if (A->ld < A->d) return fail(ctx, BKS_ERR_INVALID_ARG, "A->ld < A->d");
        if (A->col_mean != nullptr)
            return fail(ctx, BKS_ERR_UNSUPPORTED, "implicit centring is implemented for CSR A only");
        return BKS_OK;
    }
    if (A->kind == BKS_CSR) {
        if (A->dtype != BKS_F32) return fail(ctx, BKS_ERR_UNSUPPORTED, "CSR values must be FP32");
        if (A->row_ptr == nullptr || A->col_idx == nullptr || A->vals == nullptr || A->nnz < 0)
            return fail(ctx, BKS_ERR_INVALID_ARG, "CSR arrays missing");
        const bool tr = A->t_row_ptr != nullptr, tc = A->t_col_idx != nullptr, tv = A->t_vals != nullptr;
        if (tr != tc || tc != tv)
            return fail(ctx, BKS_ERR_INVALID_ARG, "give all three arrays of the CSR of A^T or none");
        return BKS_OK;
    }
    return fail(ctx, BKS_ERR_INVALID_ARG, "unknown matrix kind");
}

// Scratch of the sparse products: segment plans of A and A^T (index 0 and 1), the CSR
// of A^T when the caller did not give it, row-major staging of X and Y, partial sums.
struct CsrWs {
    const int64_t* rp[2] = {nullptr, nullptr};
    const int32_t* ci[2] = {nullptr, nullptr};
    const float* cv[2] = {nullptr, nullptr};
    int64_t* seg_off[2] = {nullptr, nullptr};
    int64_t* seg_row[2] = {nullptr, nullptr};
    int64_t segb[2] = {0, 0};
    float* x_rm = nullptr;
    float* y_rm = nullptr;
    float* part = nullptr;
    double* cvec = nullptr;
};

// Scratch of the tensor-core product: hi/lo split of X and partial tiles.
struct ProductWs {
    float* xh = nullptr;
    float* xl = nullptr;
    float* tpart = nullptr;
    int64_t tpart_cap = 0;
    bool simt_only = false;
    __nv_bfloat16* xb = nullptr;   // BF16 pieces of X (BF16 A)
    int64_t xb_cap = 0;            // elements
    int bf16_pieces = 3;           // 1: X rounded to BF16; 3: FP32-accurate
    CsrWs csr;
};

// Workspace layout of the sparse machinery for c columns; `build` also lays out room
// for the CSR of A^T and the transpose scratch when the caller did not give it.
struct CsrLayout {
    size_t seg_off0, seg_row0, seg_off1, seg_row1, nseg_tmp, sums, x_rm, y_rm, part, cvec;
    size_t t_rp, t_ci, t_cv, tscratch;
    int64_t segb0, segb1;
    bool build;
    void take(Arena& a, const bks_matrix* A, int c) {
        const int64_t n = A->n, d = A->d, nnz = A->nnz, mx = n > d ? n : d;
        segb0 = seg_upper_bound(n, nnz);
        segb1 = seg_upper_bound(d, nnz);
        seg_off0 = a.take(size_t(n + 1) * 8);
        seg_row0 = a.take(size_t(segb0) * 8);
        seg_off1 = a.take(size_t(d + 1) * 8);
        seg_row1 = a.take(size_t(segb1) * 8);
        nseg_tmp = a.take(size_t(mx + 1) * 8);
        sums = a.take(size_t(mx / 1024 + 4) * 8);
        const int64_t xp = csr_row_pitch(c);
        x_rm = a.take(size_t(mx) * xp * 4);
        y_rm = a.take(size_t(mx) * xp * 4);
        part = a.take(size_t(segb0 > segb1 ? segb0 : segb1) * xp * 4);
        cvec = a.take(size_t(csr_cvec_doubles(c)) * 8);
        build = A->t_row_ptr == nullptr;
        if (build) {
            t_rp = a.take(size_t(d + 1) * 8);
            t_ci = a.take(size_t(nnz) * 4 + 16);
            t_cv = a.take(size_t(nnz) * 4 + 16);
            tscratch = a.take(csr_transpose_scratch(n, d));
        }
    }
    // Build the CSR of A^T if needed and both segment plans; fill ws.
    void prepare(Exec& ex, char* base, const bks_matrix* A, CsrWs& ws) const {
        ws.rp[0] = A->row_ptr;
        ws.ci[0] = A->col_idx;
        ws.cv[0] = static_cast<const float*>(A->vals);
        csr_check(ex, A->row_ptr, A->col_idx, A->n, A->d, A->nnz, ex.status);
        if (!build) csr_check(ex, A->t_row_ptr, A->t_col_idx, A->d, A->n, A->nnz, ex.status);
        if (build) {
            int64_t* trp = reinterpret_cast<int64_t*>(base + t_rp);
            int32_t* tci = reinterpret_cast<int32_t*>(base + t_ci);
            float* tcv = reinterpret_cast<float*>(base + t_cv);
            csr_transpose(ex, A->row_ptr, A->col_idx, static_cast<const float*>(A->vals), A->n, A->d,
                          A->nnz, trp, tci, tcv, base + tscratch);
            ws.rp[1] = trp;
            ws.ci[1] = tci;
            ws.cv[1] = tcv;
        } else {
            ws.rp[1] = A->t_row_ptr;
            ws.ci[1] = A->t_col_idx;
            ws.cv[1] = static_cast<const float*>(A->t_vals);
        }
        ws.seg_off[0] = reinterpret_cast<int64_t*>(base + seg_off0);
        ws.seg_row[0] = reinterpret_cast<int64_t*>(base + seg_row0);
        ws.seg_off[1] = reinterpret_cast<int64_t*>(base + seg_off1);
        ws.seg_row[1] = reinterpret_cast<int64_t*>(base + seg_row1);
        ws.segb[0] = segb0;
        ws.segb[1] = segb1;
        int64_t* tmp = reinterpret_cast<int64_t*>(base + nseg_tmp);
        int64_t* sm = reinterpret_cast<int64_t*>(base + sums);
        csr_segments(ex, ws.rp[0], A->n, tmp, ws.seg_off[0], ws.seg_row[0], sm);
        csr_segments(ex, ws.rp[1], A->d, tmp, ws.seg_off[1], ws.seg_row[1], sm);
        ws.x_rm = reinterpret_cast<float*>(base + x_rm);
        ws.y_rm = reinterpret_cast<float*>(base + y_rm);
        ws.part = reinterpret_cast<float*>(base + part);
        ws.cvec = reinterpret_cast<double*>(base + cvec);
    }
};

// Products with A, in precision T: the tcgen05 kernel for an FP32 dense A when the
// operands meet its alignment rules, else the SIMT tile kernel.
template <typename T>
void product(Exec& ex, const bks_matrix* A, bool trans, int c, const T* X, int64_t ldx, T* Y,
             int64_t ldy, double* part, int64_t cap, const ProductWs& pw) {
    if (A->kind == BKS_CSR) {   // FP32 only (checked on entry)
        const int s = trans ? 1 : 0;
        const int before = ex.launches;
        const CsrWs& w = pw.csr;
        csr_product(ex, w.rp[s], w.ci[s], w.cv[s], trans ? A->d : A->n, trans ? A->n : A->d, A->nnz,
                    w.seg_off[s], w.seg_row[s], w.segb[s], reinterpret_cast<const float*>(X), ldx, c,
                    reinterpret_cast<float*>(Y), ldy, w.x_rm, w.y_rm, w.part,
                    A->col_mean ? (trans ? 2 : 1) : 0, A->col_mean, w.cvec);
        ex.product_launches += ex.launches - before;
        return;
    }
    if (sizeof(T) == 4 && A->dtype == BKS_BF16 && !pw.simt_only && pw.xb != nullptr) {
        const int before = ex.launches;
        if (tc_product_bf16(ex, static_cast<const __nv_bfloat16*>(A->vals), A->n, A->d, A->ld, trans, c,
                            pw.bf16_pieces, reinterpret_cast<const float*>(X), ldx,
                            reinterpret_cast<float*>(Y), ldy, pw.xb, pw.xb_cap, pw.tpart, pw.tpart_cap)) {
            ex.product_launches += ex.launches - before;
            return;
        }
    }
    if (sizeof(T) == 4 && A->dtype == BKS_F32 && !pw.simt_only && pw.xh != nullptr) {
        const int before = ex.launches;
        if (tc_product_f32(ex, static_cast<const float*>(A->vals), A->n, A->d, A->ld, trans, c,
                           reinterpret_cast<const float*>(X), ldx, reinterpret_cast<float*>(Y), ldy,
                           pw.xh, pw.xl, pw.tpart, pw.tpart_cap)) {
            ex.product_launches += ex.launches - before;
            return;
        }
    }
    GemmDesc g{};
    g.M = c;
    g.N = trans ? A->d : A->n;
    g.K = trans ? A->n : A->d;
    g.X = X; g.ldx = ldx;
    g.Y = A->vals; g.ldy = A->ld;
    g.y_kmajor = !trans;
    g.y_dtype = A->dtype;
    g.out = Y; g.ldo = ldy; g.out_transposed = false;
    g.alpha = 1.0; g.beta = 0.0;
    const int before = ex.launches;
    gemm_simt<T>(ex, g, part, cap);
    ex.product_launches += ex.launches - before;
}

// ----------------------------------------------------------------- workspace plan
struct Plan {
    int64_t n, d, ldn, ldd;
    int k, q, w;
    size_t xh, xl, tpart, xb;
    int64_t tpart_cap, xb_cap;
    bool sparse;
    CsrLayout csr;
    size_t td, td_bytes;     // scratch of the tridiagonal eigen-solve (0 bytes when it cannot run)
    size_t Qt, Bt, QBt, Pit, W, Wtmp, Wb, Wbtmp, part, og, rfac, ct, Rm, JX, lam, nrm, Vt,
        order, Vk, stat, fpart, fgram, fbar, otc_part, otc_cts, otc_h, otc_bar, qr, vtp, zt, cf, Md, JXd, lamd,
        nrmd, Vtd;
    int64_t ldvt;         // row pitch of the padded copy of the Ritz coefficients (vtp)
    int64_t ldcf;         // row pitch of the Block Lanczos coefficients C_j (k x 2k)
    int64_t fcap, otc_cap, otc_ldct, ldr;
    int ldp;
    int64_t ldc;
    int64_t part_cap;
    size_t total;
};

int64_t max_partials(int64_t n, int64_t d, int k, int w, int sms) {
    int64_t p = 0;
    auto upd = [&](int64_t M, int64_t N, int64_t K) {
        const int64_t e = gemm_partial_elems(M, N, K, sms);
        if (e > p) p = e;
    };
    upd(k, n, d);        // A X
    upd(k, d, n);        // A^T X
    upd(k, n, w);        // Z = Q Ubar_k
    upd(k, d, w);        // B Ubar_k
    upd(w, w, d);        // R = Q_B^T B
    upd(k, 2 * k, d);    // Block Lanczos: [B_{j-1}; B_j]^T B_j
    upd(k, n, 2 * k);    // Block Lanczos: W -= [Q_{j-1} Q_j] C_j
    return p;
}

Plan make_plan(const bks_matrix* A, int k, int q_eff, int w, size_t tb, int sms, int kout, bool eig_f64) {
    const int64_t n = A->n, d = A->d;
    Plan p{};
    p.n = n; p.d = d; p.k = k; p.q = q_eff; p.w = w;
    p.ldn = round_up(n, 32);
    p.ldd = round_up(d, 32);
    Arena a;
    p.Qt = a.take(size_t(w) * p.ldn * tb);
    p.Bt = a.take(size_t(w) * p.ldd * tb);
    p.QBt = a.take(size_t(w) * p.ldd * tb);
    p.Pit = a.take(size_t(k) * p.ldd * tb);
    p.W = a.take(size_t(k) * p.ldn * tb);
    p.Wtmp = a.take(size_t(k) * p.ldn * tb);
    p.Wb = a.take(size_t(k) * p.ldd * tb);
    p.Wbtmp = a.take(size_t(k) * p.ldd * tb);
    const int64_t ldmax0 = p.ldn > p.ldd ? p.ldn : p.ldd;
    const OrthSizes on = orth_sizes(n, p.ldn, w, k, int(tb), tb == 4, sms);
    const OrthSizes od = orth_sizes(d, p.ldd, w, k, int(tb), tb == 4, sms);
    p.part_cap = max_partials(n, d, k, w, sms);
    if (on.cap > p.part_cap) p.part_cap = on.cap;
    if (od.cap > p.part_cap) p.part_cap = od.cap;
    p.part = a.take(size_t(p.part_cap) * sizeof(double));
    p.ldp = on.ldp;
    p.ldc = on.ldc;
    p.og = a.take(on.g);
    p.rfac = a.take(on.rfac);
    p.ct = a.take(on.ct);
    p.fcap = on.fcap > od.fcap ? on.fcap : od.fcap;
    p.fpart = a.take(size_t(p.fcap) * 4);
    p.fgram = a.take(on.fgram > od.fgram ? on.fgram : od.fgram);
    p.fbar = a.take(16);
    // tensor-core orthonormalisation of the n-space blocks (FP32): its scratch and the
    // row-major copy of Q it reads the updates from
    p.otc_cap = on.otc_cap;
    p.otc_ldct = on.otc_ldct;
    p.otc_part = a.take(on.otc_part);
    p.otc_cts = a.take(on.otc_cts);
    p.otc_h = a.take(on.otc_h);
    p.otc_bar = a.take(on.otc_bar);
    p.ldr = round_up(w, 32);
    p.qr = a.take(on.otc_part > 0 ? size_t(n) * p.ldr * 4 : 0);
    p.Rm = a.take(size_t(w) * w * tb);
    p.JX = a.take(size_t(w) * w * tb);
    p.lam = a.take(size_t(w) * tb);
    p.nrm = a.take(size_t(w) * tb);
    p.Vt = a.take(size_t(w) * w * tb);
    p.order = a.take(size_t(w) * sizeof(int));
    p.Vk = a.take(size_t(kout) * p.ldd * tb);
    p.ldcf = round_up(2 * k, 32);
    p.cf = a.take(size_t(k) * p.ldcf * tb);
    // FP64 eigen-solve of M on the FP32 path: M, the Jacobi scratch and U in FP64
    const size_t e64 = (tb == 4 && eig_f64) ? 8 : 0;
    p.Md = a.take(size_t(w) * w * e64);
    p.JXd = a.take(size_t(w) * w * e64);
    p.lamd = a.take(size_t(w) * e64);
    p.nrmd = a.take(size_t(w) * e64);
    p.Vtd = a.take(size_t(w) * w * e64);
    // FP32: Z = Q Ubar_k and B Ubar_k on the tensor cores, from a copy of the coefficients
    // with a 128-byte row pitch, through Z^T (kout x ldn)
    p.ldvt = round_up(w, 32);
    p.vtp = a.take(tb == 4 ? size_t(kout) * p.ldvt * 4 : 0);
    p.zt = a.take(tb == 4 ? size_t(kout) * p.ldn * 4 : 0);
    {
        const bool fits = tb == 4 ? tridiag_fits<float>(w, kout) : tridiag_fits<double>(w, kout);
        p.td_bytes = fits ? tridiag_scratch_elems(w, kout) * tb : 0;
        p.td = a.take(p.td_bytes);
    }
    const int64_t ldmax = p.ldn > p.ldd ? p.ldn : p.ldd;
    // hi/lo split of a thin operand: a k-wide block, or (FP32) all w rows of B for M = B^T B
    size_t xcap = size_t(k) * ldmax;
    if (tb == 4 && size_t(w) * p.ldd > xcap) xcap = size_t(w) * p.ldd;
    p.xh = a.take(xcap * 4);
    p.xl = a.take(xcap * 4);
    p.tpart_cap = tc_partial_floats(n, d, k, sms);
    if (tb == 4) {
        const int64_t b = tc_partial_floats(w, d, w, sms);   // M = B^T B on the tensor cores
        if (b > p.tpart_cap) p.tpart_cap = b;
        for (int64_t len : {n, d}) {                         // Q Ubar_k and B Ubar_k
            const int64_t z = tc_partial_floats(w, len, kout, sms);
            if (z > p.tpart_cap) p.tpart_cap = z;
            // Block Lanczos: the Gram [B_{j-1}; B_j]^T B_j and the update [Q_{j-1} Q_j] C_j
            const int64_t l = tc_partial_floats(2 * k, len, k, sms);
            if (l > p.tpart_cap) p.tpart_cap = l;
        }
    }
    if (on.tcap > p.tpart_cap) p.tpart_cap = on.tcap;
    if (od.tcap > p.tpart_cap) p.tpart_cap = od.tcap;
    (void)ldmax0;
    p.xb_cap = 0;
    if (A->kind == BKS_DENSE && A->dtype == BKS_BF16) {
        // the refinement product runs at width w in groups of up to 128 columns
        const int cmax = w > k ? (w < 128 ? w : 128) : k;
        const int64_t b = tc_bf16_partial_floats(n, d, cmax, sms);
        if (b > p.tpart_cap) p.tpart_cap = b;
        p.xb_cap = 3 * int64_t(cmax) * ldmax;
    }
    p.tpart = a.take(size_t(p.tpart_cap) * 4);
    p.xb = a.take(size_t(p.xb_cap) * 2 + 16);
    p.stat = a.take(4 * sizeof(int));
    p.sparse = A->kind == BKS_CSR;
    if (p.sparse) p.csr.take(a, A, k);
    p.total = a.off;
    return p;
}

// ----------------------------------------------------------------- profiling
struct Prof {
    bks_ctx* ctx;
    bool on;
    std::vector<std::pair<int, int>> spans[4];   // product, orth, rr, total
    int next = 0;
    Prof(bks_ctx* c, bool o) : ctx(c), on(o) {}
    int ev() {
        if (next >= int(ctx->events.size())) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            ctx->events.push_back(e);
        }
        return next++;
    }
    int begin() {
        if (!on) return -1;
        const int e = ev();
        cudaEventRecord(ctx->events[e], ctx->stream);
        return e;
    }
    void end(int cls, int b) {
        if (!on) return;
        const int e = ev();
        cudaEventRecord(ctx->events[e], ctx->stream);
        spans[cls].push_back({b, e});
    }
    float total(int cls) {
        float s = 0.f;
        for (auto& pr : spans[cls]) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ctx->events[pr.first], ctx->events[pr.second]);
            s += ms;
        }
        return s;
    }
};

// Wait for the queued solve of ctx, decode its status words and fill st.
bks_status finish_solve(bks_ctx* ctx, bks_stats* st) {
    PendingSolve ps = ctx->pending;
    ctx->pending.active = false;
    if (!ps.active) return BKS_OK;
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "solve");
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "kernel launch");
    const int status = ctx->host_status[0];
    if (st != nullptr) {
        std::memset(st, 0, sizeof(*st));
        st->q_eff = ps.q_eff;
        st->width = ps.w;
        st->jacobi_sweeps = ctx->host_status[1];
        st->chol_shifts = ctx->host_status[2];
        st->launches = ps.launches;
        st->product_launches = ps.product_launches;
        st->product_bytes = ps.product_bytes;
        st->product_flops = ps.product_flops;
        st->eig_path = ps.eig_path;
    }
    if (status & ST_TIMEOUT) return fail(ctx, BKS_ERR_TIMEOUT, "a bounded device-side wait gave up");
    if (status & ST_BADINPUT) return fail(ctx, BKS_ERR_INVALID_ARG, "CSR structure check failed");
    if (status & ST_NONFINITE) return fail(ctx, BKS_ERR_NONFINITE, "non-finite value in a Gram matrix or M");
    if (status & ST_BREAKDOWN) return fail(ctx, BKS_ERR_BREAKDOWN, "Cholesky breakdown after shifting");
    if (status & ST_NOT_CONVERGED) return fail(ctx, BKS_ERR_NOT_CONVERGED, "Jacobi sweep cap reached");
    if (!ps.basis_only && ctx->host_status[1] < 0)
        return fail(ctx, BKS_ERR_UNSUPPORTED, "Jacobi launch failed");
    ctx->last_error.clear();
    return ps.deflated ? BKS_WARN_DEFLATED : BKS_OK;
}

template <typename T>
bks_status solve(bks_ctx* ctx, const bks_matrix* A, int kz, int q, uint64_t seed, const void* pi,
                 void* Zv, void* sigv, void* Vv, const bks_opts& o, bks_stats* st, bool krylov,
                 bool triplets, bool defer, double adapt_tol, int lanczos) {
    const int64_t n = A->n, d = A->d;
    // block size: the p >= kz columns of Pi (Sec. 8, spectral decay); kz Ritz vectors returned
    const int k = o.block_p > 0 ? o.block_p : kz;
    const int64_t mn = n < d ? n : d;
    int q_eff = q;
    bool deflated = false;
    if (krylov) {
        const int64_t cap = mn / k - 1;
        if (q_eff > cap) { q_eff = int(cap); deflated = true; }
    }
    const int w = krylov ? k * (q_eff + 1) : k;
    {
        int C, b, E;
        size_t sm;
        if (!o.basis_only && !jacobi_plan(w, int(sizeof(T)), C, b, E, sm))
            return fail(ctx, BKS_ERR_UNSUPPORTED,
                        "Krylov width " + std::to_string(w) + " exceeds the Jacobi solver's limit");
        if (sizeof(T) == 4 && o.eig_f64 && !o.basis_only && !jacobi_plan(w, 8, C, b, E, sm))
            return fail(ctx, BKS_ERR_UNSUPPORTED,
                        "Krylov width " + std::to_string(w) + " exceeds the FP64 Jacobi solver's limit");
    }
    const int kout = triplets ? w : kz;   // Ritz vectors returned
    Plan p = make_plan(A, k, q_eff, w, sizeof(T), ctx->num_sms, kout, o.eig_f64 != 0);
    bks_status s = ensure_ws(ctx, p.total);
    if (s != BKS_OK) return s;
    char* base = static_cast<char*>(ctx->ws);
    T* Qt = reinterpret_cast<T*>(base + p.Qt);
    T* Bt = reinterpret_cast<T*>(base + p.Bt);
    T* QBt = reinterpret_cast<T*>(base + p.QBt);
    T* Pit = reinterpret_cast<T*>(base + p.Pit);
    T* W = reinterpret_cast<T*>(base + p.W);
    T* Wtmp = reinterpret_cast<T*>(base + p.Wtmp);
    T* Wb = reinterpret_cast<T*>(base + p.Wb);
    T* Wbtmp = reinterpret_cast<T*>(base + p.Wbtmp);
    double* part = reinterpret_cast<double*>(base + p.part);
    OrthWs ows;
    ows.partials = part;
    ows.cap = p.part_cap;
    ows.g = base + p.og;
    ows.rfac = base + p.rfac;
    ows.ldp = p.ldp;
    ows.ct = base + p.ct;
    ows.ldc = p.ldc;
    T* Rm = reinterpret_cast<T*>(base + p.Rm);
    T* JX = reinterpret_cast<T*>(base + p.JX);
    T* lam = reinterpret_cast<T*>(base + p.lam);
    T* nrm = reinterpret_cast<T*>(base + p.nrm);
    T* Vt = reinterpret_cast<T*>(base + p.Vt);
    int* order = reinterpret_cast<int*>(base + p.order);
    T* Vk = reinterpret_cast<T*>(base + p.Vk);
    ProductWs pw;
    pw.xh = reinterpret_cast<float*>(base + p.xh);
    pw.xl = reinterpret_cast<float*>(base + p.xl);
    pw.tpart = reinterpret_cast<float*>(base + p.tpart);
    pw.tpart_cap = p.tpart_cap;
    pw.simt_only = o.product_path == 1;
    pw.xb = p.xb_cap > 0 ? reinterpret_cast<__nv_bfloat16*>(base + p.xb) : nullptr;
    pw.xb_cap = p.xb_cap;
    // Mixed precision (BF16 A): the Krylov products take X rounded to BF16; with refine,
    // B = A^T Q is recomputed FP32-accurately at the full width before Rayleigh-Ritz.
    // eigen-solve input: R of a d-space block QR of B (rr_mode 1) or M = B^T B (2).  Auto:
    // the QR preconditioning saves Jacobi sweeps, which pays for its w / k extra block
    // orthonormalisations only at large widths (measured: M directly is faster at w = 220
    // and 450, slower at w = 700)
    // Eigen-solve: only Ubar_k is needed, so by default M = B^T B goes through the
    // tridiagonal top-k solver; the one-sided Jacobi covers Ritz triplets (all w vectors),
    // SI (w = k), widths beyond the tridiagonal kernels and eig_mode 1.
    // Block Lanczos (lanczos >= 0, the reorthogonalisation mode) forms T = Q^T A A^T Q from
    // its block-tridiagonal band during the iteration; rr_mode does not apply to it.
    const bool lz = krylov && lanczos >= 0;
    const bool use_td = !o.basis_only && !triplets && o.eig_mode != 1 && (lz || o.rr_mode != 1) && kz < w &&
                        tridiag_fits<T>(w, kz);
    const bool rr_qr = !lz && !use_td && (o.rr_mode == 1 || (o.rr_mode == 0 && w > 512));
    const bool bf16_mode = o.precision == BKS_PREC_BF16;
    const bool refine = bf16_mode && o.refine != 0;
    pw.bf16_pieces = bf16_mode ? 1 : 3;
    int* stat = reinterpret_cast<int*>(base + p.stat);   // [status, sweeps, shifted]
    T* Z = static_cast<T*>(Zv);
    T* sigma = static_cast<T*>(sigv);
    T* V = static_cast<T*>(Vv);

    Exec ex;
    ex.stream = ctx->stream;
    ex.status = stat;
    ex.num_sms = o.max_sms > 0 && o.max_sms < ctx->num_sms ? o.max_sms : ctx->num_sms;
    if (o.profile) {
        ctx->klog.n = 0;
        ex.klog = &ctx->klog;
    }
    Prof prof(ctx, o.profile != 0);
    const int t_all = prof.begin();
    cudaMemsetAsync(stat, 0, 4 * sizeof(int), ctx->stream);
    if (p.sparse) p.csr.prepare(ex, base, A, pw.csr);   // segment plans (+ CSR of A^T)

    // a0: start block, stored transposed (k x ldd)
    if (pi != nullptr)
        transpose_in<T>(ex, pi, sizeof(T) == 8 ? BKS_F64 : BKS_F32, d, k, k, Pit, p.ldd);
    else
        gen_pi_device<T>(ex, seed, d, k, Pit, p.ldd, true);

    auto prod = [&](bool trans, const T* X, int64_t ldx, T* Y, int64_t ldy, int c) {
        const int b = prof.begin();
        product<T>(ex, A, trans, c, X, ldx, Y, ldy, part, p.part_cap, pw);
        prof.end(0, b);
    };
    ows.shifted_flag = stat + 2;
    if (sizeof(T) == 4 && o.product_path != 1) {   // thin-block products on the tensor cores
        ows.xh = pw.xh;
        ows.xl = pw.xl;
        ows.tpart = pw.tpart;
        ows.tpart_cap = pw.tpart_cap;
        if (p.fcap > 0) {                            // fused one-launch orthonormalisation
            ows.fpart = reinterpret_cast<float*>(base + p.fpart);
            ows.fpart_cap = p.fcap;
            ows.fgram = reinterpret_cast<float*>(base + p.fgram);
            ows.fbar = reinterpret_cast<unsigned*>(base + p.fbar);
        }
        if (p.otc_cap > 0) {                         // tensor-core orthonormalisation
            ows.otc_part = reinterpret_cast<float*>(base + p.otc_part);
            ows.otc_cap = p.otc_cap;
            ows.otc_cts = reinterpret_cast<float*>(base + p.otc_cts);
            ows.otc_ldct = p.otc_ldct;
            ows.otc_h = reinterpret_cast<float*>(base + p.otc_h);
            ows.otc_bar = reinterpret_cast<unsigned*>(base + p.otc_bar);
        }
    }
    // Krylov blocks on the tensor-core kernel keep a row-major copy of Q (columns appended
    // block by block); once a block falls back to the CUDA-core kernel the copy is
    // incomplete and the later blocks stay on the CUDA cores.  Block Lanczos with local
    // reorthogonalisation reads a window of the copy starting at column (j-1)k, which the
    // TMA takes only at a 16-byte aligned address (k a multiple of 4); without
    // reorthogonalisation the copy is not read at all.
    bool qr_ok = krylov && p.otc_cap > 0 &&
                 (!lz || lanczos == BKS_REORTH_FULL || (lanczos == BKS_REORTH_LOCAL && k % 4 == 0));
    bool tc_ran = false;
    // W against the m orthonormal columns from Qb (column qcol of Q), result in Qout
    auto orth = [&](int m, const T* Qb, int64_t qcol, T* Qout) {
        const int b = prof.begin();
        if (qr_ok) {
            ows.qr = reinterpret_cast<float*>(base + p.qr) + qcol;
            ows.ldr = p.ldr;
            ows.qr_append = true;
            ows.tc_used = &tc_ran;
        }
        orth_block<T>(ex, n, p.ldn, Qb, m, W, k, Wtmp, Qout, ows);
        if (qr_ok && !tc_ran) qr_ok = false;
        ows.qr = nullptr;
        ows.ldr = 0;
        ows.qr_append = false;
        ows.tc_used = nullptr;
        prof.end(1, b);
    };
    // QR of the kept blocks B_i in d-space (R = Q_B^T B preconditions the eigen-solve)
    auto orth_b = [&](int m, const T* Bblk) {
        const int b = prof.begin();
        cudaMemcpyAsync(Wb, Bblk, size_t(k) * p.ldd * sizeof(T), cudaMemcpyDeviceToDevice,
                        ctx->stream);
        orth_block<T>(ex, d, p.ldd, QBt, m, Wb, k, Wbtmp, QBt + size_t(m) * p.ldd, ows);
        prof.end(1, b);
    };

    // Block Lanczos, row block j of T: C_j = [B_{j-1}; B_j]^T B_j = [R_{j-1}^T; D_j] (B_0^T B_0
    // alone at j = 0) into cf (k x ldcf, row i = column i of C_j), copied into rows jk..(j+1)k,
    // columns (j-1)k..(j+1)k of T.  Returns the rows of C_j.
    T* cf = reinterpret_cast<T*>(base + p.cf);
    auto lz_coef = [&](int j) {
        const int j0 = j > 0 ? j - 1 : 0;
        const int rows = (j - j0 + 1) * k;
        const T* Bw = Bt + size_t(j0) * k * p.ldd;
        const T* Bj = Bt + size_t(j) * k * p.ldd;
        KernelLog* klog = ex.klog;   // the kernel log times products with A only
        ex.klog = nullptr;
        const bool tc = sizeof(T) == 4 && o.product_path != 1 &&
                        tc_product_f32(ex, reinterpret_cast<const float*>(Bw), rows, d, p.ldd, false, k,
                                       reinterpret_cast<const float*>(Bj), p.ldd, reinterpret_cast<float*>(cf),
                                       p.ldcf, pw.xh, pw.xl, pw.tpart, pw.tpart_cap);
        ex.klog = klog;
        if (!tc) {
            GemmDesc g{};
            g.M = k; g.N = rows; g.K = d;
            g.X = Bj; g.ldx = p.ldd; g.Y = Bw; g.ldy = p.ldd;
            g.y_kmajor = true; g.y_dtype = sizeof(T) == 8 ? BKS_F64 : BKS_F32;
            g.out = cf; g.ldo = p.ldcf; g.alpha = 1.0; g.beta = 0.0;
            gemm_simt<T>(ex, g, part, p.part_cap);
        }
        cudaMemcpy2DAsync(Rm + size_t(j) * k * w + size_t(j0) * k, size_t(w) * sizeof(T), cf,
                          size_t(p.ldcf) * sizeof(T), size_t(rows) * sizeof(T), size_t(k),
                          cudaMemcpyDeviceToDevice, ex.stream);
    };
    // The three-term recurrence: W = A A^T Q_j - Q_j D_j - Q_{j-1} R_{j-1}^T, i.e.
    // W -= [Q_{j-1} Q_j] C_j with the C_j of lz_coef(j).
    auto lz_sub = [&](int j) {
        const int j0 = j > 0 ? j - 1 : 0;
        const int rows = (j - j0 + 1) * k;
        const T* Qw = Qt + size_t(j0) * k * p.ldn;
        KernelLog* klog = ex.klog;
        ex.klog = nullptr;
        const bool tc = sizeof(T) == 4 && o.product_path != 1 &&
                        tc_product_f32(ex, reinterpret_cast<const float*>(Qw), rows, n, p.ldn, true, k,
                                       reinterpret_cast<const float*>(cf), p.ldcf, reinterpret_cast<float*>(W),
                                       p.ldn, pw.xh, pw.xl, pw.tpart, pw.tpart_cap, true);
        ex.klog = klog;
        if (!tc) {
            GemmDesc g{};
            g.M = k; g.N = n; g.K = rows;
            g.X = cf; g.ldx = p.ldcf; g.Y = Qw; g.ldy = p.ldn;
            g.y_kmajor = false; g.y_dtype = sizeof(T) == 8 ? BKS_F64 : BKS_F32;
            g.out = W; g.ldo = p.ldn; g.alpha = -1.0; g.beta = 1.0;
            gemm_simt<T>(ex, g, part, p.part_cap);
        }
    };

    // Adaptive q: after B_{i-1} = A^T Q_{i-1}, the kz leading Ritz values of the i-block space
    // (M_i = B^T B over those blocks, tridiagonal form and multisection only); the
    // iteration stops at the first i >= 2 where none moved by more than adapt_tol
    // (relative) since i - 1 blocks.  B_{i-1} is then the last kept block: no product is
    // spent on the test.
    const bool adaptive = krylov && !lz && adapt_tol > 0 && !o.basis_only && p.td_bytes > 0;
    std::vector<double> prev_vals;
    auto stagnated = [&](int nb) -> bool {
        const int wc = nb * k;
        KernelLog* klog = ex.klog;
        ex.klog = nullptr;
        const bool tc = sizeof(T) == 4 && o.product_path != 1 &&
                        tc_product_f32(ex, reinterpret_cast<const float*>(Bt), wc, d, p.ldd, false, wc,
                                       reinterpret_cast<const float*>(Bt), p.ldd, reinterpret_cast<float*>(Rm),
                                       wc, pw.xh, pw.xl, pw.tpart, pw.tpart_cap);
        ex.klog = klog;
        if (!tc) {
            GemmDesc g{};
            g.M = wc; g.N = wc; g.K = d;
            g.X = Bt; g.ldx = p.ldd; g.Y = Bt; g.ldy = p.ldd;
            g.y_kmajor = true; g.y_dtype = sizeof(T) == 8 ? BKS_F64 : BKS_F32;
            g.out = Rm; g.ldo = wc; g.alpha = 1.0; g.beta = 0.0;
            gemm_simt<T>(ex, g, part, p.part_cap);
        }
        const int m = kz < wc ? kz : wc;
        const T* lam_d = nullptr;
        const T* scale_d = nullptr;
        if (!topk_values<T>(ex, wc, Rm, m, reinterpret_cast<T*>(base + p.td), &lam_d, &scale_d)) return false;
        if (ctx->host_vals == nullptr && cudaMallocHost(&ctx->host_vals, 256 * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            ctx->host_vals = nullptr;
            return false;
        }
        T* hv = reinterpret_cast<T*>(ctx->host_vals);
        cudaMemcpyAsync(hv, lam_d, size_t(m) * sizeof(T), cudaMemcpyDeviceToHost, ex.stream);
        cudaMemcpyAsync(hv + m, scale_d, sizeof(T), cudaMemcpyDeviceToHost, ex.stream);
        if (cudaStreamSynchronize(ex.stream) != cudaSuccess) return false;
        std::vector<double> cur(m);
        for (int j = 0; j < m; ++j) {
            const double l = double(hv[j]) * double(hv[m]);
            cur[j] = l > 0 ? std::sqrt(l) : 0.0;
        }
        bool done = false;
        if (prev_vals.size() == size_t(m)) {
            double delta = 0;
            const double floor = 1e-30 + 1e-12 * cur[0];
            for (int j = 0; j < m; ++j) {
                const double dj = std::fabs(cur[j] - prev_vals[j]) / (cur[j] > floor ? cur[j] : floor);
                if (!(dj <= delta)) delta = dj;   // NaN counts as not converged
            }
            done = delta <= adapt_tol;
        }
        prev_vals.swap(cur);
        return done;
    };

    // a1 + a4: W_0 = A Pi, Q_0 = orth(W_0)
    prod(false, Pit, p.ldd, W, p.ldn, k);
    orth(0, Qt, 0, Qt);
    int q_run = q_eff;   // iterations run (fewer when the adaptive test stops early)
    bool stopped = false;
    for (int i = 1; i <= q_eff; ++i) {
        T* Qprev = krylov ? Qt + size_t(i - 1) * k * p.ldn : Qt;
        T* Bprev = krylov ? Bt + size_t(i - 1) * k * p.ldd : Bt;
        prod(true, Qprev, p.ldn, Bprev, p.ldd, k);       // a2: B_{i-1} = A^T Q_{i-1}
        if (adaptive && stagnated(i) && i >= 2) {
            q_run = i - 1;
            stopped = true;
            break;
        }
        if (krylov && !o.basis_only && !refine && rr_qr) orth_b((i - 1) * k, Bprev);
        prod(false, Bprev, p.ldd, W, p.ldn, k);           // a3: W_i = A B_{i-1}
        if (lz) {
            // Block Lanczos: the three-term recurrence, then the reorthogonalisation against
            // every earlier block (full), against Q_{i-2} and Q_{i-1} (local) or none, and
            // CholeskyQR2 (W = Q_i R_{i-1})
            lz_coef(i - 1);
            lz_sub(i - 1);
            int m0 = 0, m = 0;
            if (lanczos == BKS_REORTH_FULL) {
                m = i * k;
            } else if (lanczos == BKS_REORTH_LOCAL) {
                m0 = i >= 2 ? i - 2 : 0;
                m = (i - m0) * k;
            }
            orth(m, Qt + size_t(m0) * k * p.ldn, int64_t(m0) * k, Qt + size_t(i) * k * p.ldn);
        } else if (krylov) {
            orth(i * k, Qt, 0, Qt + size_t(i) * k * p.ldn);   // a4: project + CholeskyQR2
        } else {
            orth(0, Qt, 0, Qt);                               // a9: SI re-orthonormalisation
        }
    }
    const int wr = krylov ? k * (q_run + 1) : k;   // width of the space Rayleigh-Ritz works on
    T* Blast = krylov ? Bt + size_t(q_run) * k * p.ldd : Bt;
    const T* Qlast = krylov ? Qt + size_t(q_run) * k * p.ldn : Qt;
    if (!refine) {
        if (!stopped) prod(true, Qlast, p.ldn, Blast, p.ldd, k);   // a5: B_q = A^T Q_q
    } else {
        // a8: B = A^T Q at the full width, FP32-accurate (three BF16 pieces of Q)
        pw.bf16_pieces = 3;
        prod(true, Qt, p.ldn, Bt, p.ldd, wr);
        if (krylov && !o.basis_only && rr_qr)
            for (int i = 0; i < q_run; ++i) orth_b(i * k, Bt + size_t(i) * k * p.ldd);
    }
    if (lz && !o.basis_only) {
        // the last row block of T (all of them again from the refined B), then the band
        if (refine)
            for (int j = 0; j < q_run; ++j) lz_coef(j);
        lz_coef(q_run);
        lanczos_band<T>(ex, Rm, wr, k);
    }

    const int t_rr = prof.begin();
    int eig_path = 0;
    if (o.basis_only) {
        // Z = first kz columns of Q (Sec. 4.1: enough for low-rank approximation)
        transpose_in<T>(ex, Qt, sizeof(T) == 8 ? BKS_F64 : BKS_F32, kz, n, p.ldn, Z, kz);
        row_norms<T>(ex, Bt, kz, d, p.ldd, sigma, false);
        if (V != nullptr) {
            row_norms<T>(ex, Bt, kz, d, p.ldd, sigma, true);
            transpose_in<T>(ex, Bt, sizeof(T) == 8 ? BKS_F64 : BKS_F32, kz, d, p.ldd, V, kz);
        }
    } else {
        // a5: M = B^T B.  For the Jacobi at w > 512 (or rr_mode 1) through a triangular
        // factor instead: with B = Q_B R (block QR of the kept blocks), M = R^T R, R = Q_B^T B,
        // and one-sided Jacobi on R^T converges to U Sigma with U the eigenvectors of M, in
        // fewer sweeps than on M itself and without accumulating V (Drmac & Veselic's
        // preconditioned Jacobi SVD).  Only the order of the column norms is used.
        if (rr_qr) orth_b(krylov ? q_run * k : 0, Blast);
        const int y_dtype = sizeof(T) == 8 ? BKS_F64 : BKS_F32;
        if (!lz) {
            GemmDesc gm{};
            gm.M = wr; gm.N = wr; gm.K = d;
            gm.X = rr_qr ? QBt : Bt; gm.ldx = p.ldd; gm.Y = Bt; gm.ldy = p.ldd;
            gm.y_kmajor = true; gm.y_dtype = sizeof(T) == 8 ? BKS_F64 : BKS_F32;
            gm.out = Rm; gm.ldo = wr; gm.alpha = 1.0; gm.beta = 0.0;
            // FP32: on the tensor cores (3xTF32): row j of Rm = row j of (A X)^T with A = B and
            // X = B (M, symmetric) or X = Q_B (row j of R = Q_B^T B)
            KernelLog* klog = ex.klog;   // the kernel log times products with A only
            ex.klog = nullptr;
            const bool tc_m = sizeof(T) == 4 && o.product_path != 1 &&
                              tc_product_f32(ex, reinterpret_cast<const float*>(Bt), wr, d, p.ldd, false, wr,
                                             reinterpret_cast<const float*>(rr_qr ? QBt : Bt), p.ldd,
                                             reinterpret_cast<float*>(Rm), wr, pw.xh, pw.xl, pw.tpart, pw.tpart_cap);
            ex.klog = klog;
            if (!tc_m) gemm_simt<T>(ex, gm, part, p.part_cap);
        }   // Block Lanczos: Rm holds T already
        check_finite<T>(ex, Rm, int64_t(wr) * wr);
        // a6: eigen-decomposition of M, descending (row j of Rm is column j of R^T)
        const int sweeps = o.jacobi_max_sweeps > 0 ? o.jacobi_max_sweeps : 40;
        if (sizeof(T) == 4 && o.eig_f64) {
            // FP64 eigen-solve of M (one-sided Jacobi), eigenvectors rounded to FP32
            double* Md = reinterpret_cast<double*>(base + p.Md);
            double* Vtd = reinterpret_cast<double*>(base + p.Vtd);
            cast_2d<float, double>(ex, reinterpret_cast<const float*>(Rm), wr, wr, wr, Md, wr);
            sym_eig<double>(ex, wr, Md, wr, reinterpret_cast<double*>(base + p.JXd), wr,
                            reinterpret_cast<double*>(base + p.lamd), reinterpret_cast<double*>(base + p.nrmd), Vtd,
                            wr, order, sweeps, o.jacobi_tol, stat + 1);
            cast_2d<double, float>(ex, Vtd, kout, wr, wr, reinterpret_cast<float*>(Vt), wr);
            eig_path = 2;
        } else {
            eig_path = use_td && tridiag_fits<T>(wr, kz) &&
                               topk_tridiag<T>(ex, wr, Rm, kz, Vt, wr, reinterpret_cast<T*>(base + p.td), ows)
                           ? 1
                           : 0;
            if (eig_path == 0)
                sym_eig<T>(ex, wr, Rm, wr, JX, wr, lam, nrm, Vt, wr, order, sweeps, o.jacobi_tol, stat + 1);
        }
        // a7: Z = Q Ubar_k (row-major n x k).  FP32: on the tensor cores as
        // Z^T = (Q_array^T X)^T with X = Ubar_k^T (rows of Vt, copied to a 128-byte pitch),
        // then transposed; otherwise the CUDA-core kernel writes Z directly
        KernelLog* klog_rr = ex.klog;   // the kernel log times products with A only
        ex.klog = nullptr;
        bool tc_ritz = false;
        if (sizeof(T) == 4 && o.product_path != 1) {
            float* vtp = reinterpret_cast<float*>(base + p.vtp);
            float* zt = reinterpret_cast<float*>(base + p.zt);
            cudaMemcpy2DAsync(vtp, size_t(p.ldvt) * 4, Vt, size_t(wr) * 4, size_t(wr) * 4, size_t(kout),
                              cudaMemcpyDeviceToDevice, ex.stream);
            tc_ritz = tc_product_f32(ex, reinterpret_cast<const float*>(Qt), wr, n, p.ldn, true, kout, vtp, p.ldvt,
                                     zt, p.ldn, pw.xh, pw.xl, pw.tpart, pw.tpart_cap);
            if (tc_ritz) {
                // the sign fix scans the column-major Z^T (contiguous columns), then Z is transposed
                if (o.sign_fix) sign_fix_cm<T>(ex, reinterpret_cast<T*>(zt), n, kout, p.ldn, Vt, wr, wr);
                transpose_in<T>(ex, zt, BKS_F32, kout, n, p.ldn, Z, kout);
            }
        }
        if (!tc_ritz) {
            GemmDesc gz{};
            gz.M = kout; gz.N = n; gz.K = wr;
            gz.X = Vt; gz.ldx = wr; gz.Y = Qt; gz.ldy = p.ldn;
            gz.y_kmajor = false; gz.y_dtype = y_dtype;
            gz.out = Z; gz.ldo = kout; gz.out_transposed = true; gz.alpha = 1.0; gz.beta = 0.0;
            gemm_simt<T>(ex, gz, part, p.part_cap);
        }
        if (o.sign_fix && !tc_ritz) sign_fix<T>(ex, Z, n, kout, kout, Vt, wr, wr);
        // sigma_i = |B ubar_i| = |A^T z_i|; V_k = B Ubar_k Sigma^{-1} (same two routes, after
        // the sign fix has flipped the rows of Vt)
        bool tc_v = false;
        if (tc_ritz) {
            float* vtp = reinterpret_cast<float*>(base + p.vtp);
            cudaMemcpy2DAsync(vtp, size_t(p.ldvt) * 4, Vt, size_t(wr) * 4, size_t(wr) * 4, size_t(kout),
                              cudaMemcpyDeviceToDevice, ex.stream);
            tc_v = tc_product_f32(ex, reinterpret_cast<const float*>(Bt), wr, d, p.ldd, true, kout, vtp, p.ldvt,
                                  reinterpret_cast<float*>(Vk), p.ldd, pw.xh, pw.xl, pw.tpart, pw.tpart_cap);
        }
        if (!tc_v) {
            GemmDesc gv{};
            gv.M = kout; gv.N = d; gv.K = wr;
            gv.X = Vt; gv.ldx = wr; gv.Y = Bt; gv.ldy = p.ldd;
            gv.y_kmajor = false; gv.y_dtype = y_dtype;
            gv.out = Vk; gv.ldo = p.ldd; gv.alpha = 1.0; gv.beta = 0.0;
            gemm_simt<T>(ex, gv, part, p.part_cap);
        }
        ex.klog = klog_rr;
        row_norms<T>(ex, Vk, kout, d, p.ldd, sigma, V != nullptr);
        if (V != nullptr)
            transpose_in<T>(ex, Vk, sizeof(T) == 8 ? BKS_F64 : BKS_F32, kout, d, p.ldd, V, kout);
    }
    prof.end(2, t_rr);
    prof.end(3, t_all);

    cudaError_t e = cudaMemcpyAsync(ctx->host_status, stat, 3 * sizeof(int), cudaMemcpyDeviceToHost,
                                    ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "solve");
    PendingSolve ps;
    ps.active = true;
    ps.q_eff = q_run;
    ps.w = wr;
    ps.deflated = deflated;
    ps.basis_only = o.basis_only != 0;
    ps.launches = ex.launches;
    ps.eig_path = eig_path;
    ps.product_launches = ex.product_launches;
    {
        const int nprod = 2 * q_run + 2;   // q+1 products with A, q+1 with A^T (both methods)
        // A once per product (CSR: values + column indices, and the row offsets of A or of
        // A^T, averaged), the thin input read once and the thin output written once.
        const double abytes = A->kind == BKS_CSR
                                  ? double(A->nnz) * 8.0 + double(n + d + 2) * 4.0
                                  : double(n) * double(A->ld) * double(dtype_bytes(A->dtype));
        const double nnz_like = A->kind == BKS_CSR ? double(A->nnz) : double(n) * double(d);
        ps.product_bytes = nprod * (abytes + double(k) * (n + d) * sizeof(T));
        ps.product_flops = nprod * 2.0 * k * nnz_like;
        if (refine) {   // the last A^T product runs at width w (groups of 128 columns)
            const double groups = double((wr + 127) / 128);
            ps.product_bytes += groups * abytes + double(wr - k) * (n + d) * sizeof(T);
            ps.product_flops += 2.0 * (wr - k) * nnz_like;
        }
    }
    ctx->pending = ps;
    if (defer) return BKS_OK;   // the caller reads the status later (finish_solve)
    const bks_status result = finish_solve(ctx, st);
    if (st != nullptr && o.profile) {
        st->ms_product = prof.total(0);
        st->ms_orth = prof.total(1);
        st->ms_rr = prof.total(2);
        st->ms_total = prof.total(3);
        float kms = 0.f;
        for (int i = 0; i + 1 < ctx->klog.n; i += 2) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ctx->klog.ev[i], ctx->klog.ev[i + 1]);
            kms += ms;
        }
        st->ms_product_kernel = kms;
        st->product_kernel_launches = ctx->klog.n / 2;
    }
    return result;
}

bks_status solve_entry(bks_ctx* ctx, const bks_matrix* A, int k, int q, uint64_t seed,
                       const void* pi, void* Z, void* sigma, void* V, const bks_opts* opts,
                       bks_stats* st, bool krylov, bool triplets = false, bool defer = false,
                       double adapt_tol = 0.0, int lanczos = -1) {
    if (ctx == nullptr) return BKS_ERR_INVALID_ARG;
    bks_status s = check_matrix(ctx, A);
    if (s != BKS_OK) return s;
    const int64_t mn = A->n < A->d ? A->n : A->d;
    if (k < 1 || int64_t(k) > mn) return fail(ctx, BKS_ERR_INVALID_ARG, "k must be in [1, min(n, d)]");
    if (k > 128)
        return fail(ctx, BKS_ERR_UNSUPPORTED, "k > 128: block Cholesky factors are held on one SM");
    if (q < 0) return fail(ctx, BKS_ERR_INVALID_ARG, "q must be >= 0");
    if (Z == nullptr || sigma == nullptr) return fail(ctx, BKS_ERR_INVALID_ARG, "Z and sigma are required");
    bks_opts o;
    if (opts) o = *opts; else bks_opts_default(&o);
    int prec = o.precision;
    if (prec == BKS_PREC_AUTO) prec = A->dtype == BKS_F64 ? BKS_PREC_F64 : BKS_PREC_F32;
    if (prec != BKS_PREC_F64 && prec != BKS_PREC_F32 && prec != BKS_PREC_BF16)
        return fail(ctx, BKS_ERR_INVALID_ARG, "bad precision");
    if (prec == BKS_PREC_BF16 && (A->kind != BKS_DENSE || A->dtype != BKS_BF16))
        return fail(ctx, BKS_ERR_UNSUPPORTED, "the BF16 mode needs a dense BF16 A");
    o.precision = prec;
    DeviceGuard g(ctx->device);
    if (A->kind == BKS_CSR && prec != BKS_PREC_F32)
        return fail(ctx, BKS_ERR_UNSUPPORTED, "a CSR matrix is solved on the FP32 path");
    if (triplets && o.basis_only)
        return fail(ctx, BKS_ERR_INVALID_ARG, "Ritz triplets need the Rayleigh-Ritz step (basis_only = 0)");
    if (o.block_p != 0) {
        if (o.block_p < k || int64_t(o.block_p) > mn)
            return fail(ctx, BKS_ERR_INVALID_ARG, "block_p must be 0 or in [k, min(n, d)]");
        if (o.block_p > 128)
            return fail(ctx, BKS_ERR_UNSUPPORTED, "block_p > 128: block Cholesky factors are held on one SM");
        if (triplets && o.block_p != k)
            return fail(ctx, BKS_ERR_INVALID_ARG, "Ritz triplets are computed with block_p = k");
    }
    if (o.max_sms < 0) return fail(ctx, BKS_ERR_INVALID_ARG, "max_sms must be >= 0");
    if (defer) o.profile = 0;
    if (prec == BKS_PREC_F64)
        return solve<double>(ctx, A, k, q, seed, pi, Z, sigma, V, o, st, krylov, triplets, defer, adapt_tol,
                             lanczos);
    // BF16 and F32 both run the FP32 pipeline (Krylov blocks, Z, sigma in FP32)
    return solve<float>(ctx, A, k, q, seed, pi, Z, sigma, V, o, st, krylov, triplets, defer, adapt_tol,
                        lanczos);
}


// ------------------------------------------------------------------- batches
int default_batch_sms(int num_sms) { return num_sms / 8 > 8 ? num_sms / 8 : 8; }

// Signature of a batch for the SM-budget cache: the solve (k, q, method, triplets) and the
// multiset of its matrices' shape classes (kind, dtype, ceil log2 of n and of d).
std::string batch_signature(int batch, const bks_matrix* As, int k, int q, bool krylov, bool triplets) {
    auto lg = [](int64_t x) {
        int l = 0;
        while ((int64_t(1) << l) < x) ++l;
        return l;
    };
    std::map<std::string, int> classes;
    for (int i = 0; i < batch; ++i)
        ++classes[std::to_string(As[i].kind) + "." + std::to_string(As[i].dtype) + "." + std::to_string(lg(As[i].n)) +
                  "." + std::to_string(lg(As[i].d))];
    std::string sig = std::to_string(k) + "/" + std::to_string(q) + "/" + (krylov ? "b" : "s") + (triplets ? "t" : "") + ":";
    for (const auto& c : classes) sig += c.first + "x" + std::to_string(c.second) + ";";
    return sig;
}

// Up to S stream contexts of ctx (created on first use, each with its own stream).
bks_status ensure_subs(bks_ctx* ctx, int S) {
    while (int(ctx->subs.size()) < S) {
        bks_ctx* sub = nullptr;
        bks_status cs = bks_create(&sub, ctx->device);
        if (cs != BKS_OK) return fail(ctx, cs, "could not create a stream context for the batch");
        if (cudaStreamCreateWithFlags(&sub->stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            bks_destroy(sub);
            return fail(ctx, BKS_ERR_CUDA, "could not create a stream for the batch");
        }
        sub->own_stream = true;
        ctx->subs.push_back(sub);
    }
    return BKS_OK;
}

// The batch starts after the work already queued on the caller's stream ...
cudaEvent_t batch_begin(bks_ctx* ctx, int S) {
    cudaEvent_t start;
    cudaEventCreateWithFlags(&start, cudaEventDisableTiming);
    cudaEventRecord(start, ctx->stream);
    for (int j = 0; j < S; ++j) cudaStreamWaitEvent(ctx->subs[j]->stream, start, 0);
    return start;
}

// ... and later work on the caller's stream is ordered after the batch.
void batch_end(bks_ctx* ctx, int S, cudaEvent_t ev) {
    for (int j = 0; j < S; ++j) {
        cudaEventRecord(ev, ctx->subs[j]->stream);
        cudaStreamWaitEvent(ctx->stream, ev, 0);
    }
    cudaEventDestroy(ev);
}

// worker(0) .. worker(T - 1): worker 0, and any that could not be given a thread, run here.
template <typename F>
void run_workers(int T, F&& worker) {
    tc::encode_fn();   // the tensor-map encoder's one-time lookup, before the threads start
    std::vector<std::thread> threads;
    int started = 0;   // threads 1 .. started run concurrently; the rest run here
    try {
        for (int t = 1; t < T; ++t, ++started) threads.emplace_back(worker, t);
    } catch (...) {
    }
    worker(0);
    for (int t = started + 1; t < T; ++t) worker(t);
    for (std::thread& th : threads) th.join();
}

// Independent solves (Algorithm 2 or 1, or their Ritz triplets) on the stream contexts.
bks_status batched_solve(bks_ctx* ctx, int batch, const bks_matrix* As, int k, int q, const uint64_t* seeds,
                         const void* const* pis, void* const* Zs, void* const* sigmas, void* const* Vs,
                         const bks_opts* opts, bks_stats* stats, bks_status* statuses, bool krylov, bool triplets,
                         const char* what) {
    if (ctx == nullptr) return BKS_ERR_INVALID_ARG;
    if (batch < 0 || (batch > 0 && (As == nullptr || Zs == nullptr || sigmas == nullptr)))
        return fail(ctx, BKS_ERR_INVALID_ARG, std::string("bad ") + what + " arguments");
    if (stats) std::memset(stats, 0, sizeof(*stats));
    if (batch == 0) return BKS_OK;
    DeviceGuard g(ctx->device);
    const int S = batch < BKS_BATCH_STREAMS ? batch : BKS_BATCH_STREAMS;
    bks_status cs = ensure_subs(ctx, S);
    if (cs != BKS_OK) return cs;
    {   // size every stream's workspace for the largest matrix once (no reallocation mid-batch)
        size_t need = 0;
        for (int i = 0; i < batch; ++i) {
            size_t b = 0;
            if (bks_workspace_size(&As[i], k, q, krylov ? 0 : 1, opts, &b) == BKS_OK && b > need) need = b;
        }
        for (int j = 0; j < S; ++j)
            if (need > 0 && ensure_ws(ctx->subs[j], need) != BKS_OK)
                return fail(ctx, BKS_ERR_NOMEM, "could not allocate the batch workspaces");
    }
    // SMs per solve: the caller's opts.max_sms, else the budget bks_batched_autotune cached
    // for this batch signature, else an eighth of the GPU (solves of a batch are short chains
    // of latency-bound launches: spread over every SM, the cooperative and tensor-core
    // kernels of one solve would leave no room for the others in flight)
    bks_opts ob;
    if (opts) ob = *opts; else bks_opts_default(&ob);
    if (ob.max_sms <= 0) {
        const auto it = ctx->batch_sms.find(batch_signature(batch, As, k, q, krylov, triplets));
        ob.max_sms = it != ctx->batch_sms.end() ? it->second : default_batch_sms(ctx->num_sms);
    }
    cudaEvent_t start = batch_begin(ctx, S);
    bks_status worst = BKS_OK;
    auto note = [&](int i, bks_status st_i, const bks_stats& one) {
        if (statuses) statuses[i] = st_i;
        if (st_i != BKS_OK && (worst == BKS_OK || (worst == BKS_WARN_DEFLATED && st_i != BKS_WARN_DEFLATED)))
            worst = st_i;
        if (stats) {
            stats->q_eff = one.q_eff;
            stats->width = one.width;
            stats->jacobi_sweeps = one.jacobi_sweeps > stats->jacobi_sweeps ? one.jacobi_sweeps : stats->jacobi_sweeps;
            stats->chol_shifts += one.chol_shifts;
            stats->launches += one.launches;
            stats->product_launches += one.product_launches;
            stats->product_bytes += one.product_bytes;
            stats->product_flops += one.product_flops;
        }
    };
    // T host threads issue the launches in parallel (a solve is a few dozen short kernels,
    // so one thread cannot keep the GPU busy): thread t takes matrices t, t + T, ... and
    // alternates between its stream contexts t and t + T, finishing the older solve on a
    // context before it reuses it.  Every solve is independent, so the results are those
    // of single solves, whatever the threads' timing.
    const int T = S < BKS_BATCH_THREADS ? S : BKS_BATCH_THREADS;
    std::vector<bks_status> st_all(size_t(batch), BKS_OK);
    std::vector<bks_stats> one_all(static_cast<size_t>(batch));
    auto worker = [&](int t) {
        DeviceGuard gd(ctx->device);
        int owner[2] = {-1, -1};
        bks_ctx* subs[2] = {ctx->subs[t], ctx->subs[t + T < S ? t + T : t]};
        int r = 0;
        for (int i = t; i < batch; i += T, ++r) {
            const int h = subs[1] == subs[0] ? 0 : (r & 1);   // one context: finish before reuse
            bks_ctx* sub = subs[h];
            if (owner[h] >= 0) st_all[owner[h]] = finish_solve(sub, &one_all[owner[h]]);
            owner[h] = -1;
            const bks_status st_i = solve_entry(sub, &As[i], k, q, seeds ? seeds[i] : uint64_t(i),
                                                pis ? pis[i] : nullptr, Zs[i], sigmas[i], Vs ? Vs[i] : nullptr,
                                                &ob, nullptr, krylov, triplets, true);
            if (sub->pending.active) owner[h] = i;
            else st_all[i] = st_i;
        }
        for (int h = 0; h < 2; ++h)
            if (owner[h] >= 0) st_all[owner[h]] = finish_solve(subs[h], &one_all[owner[h]]);
    };
    run_workers(T, worker);
    for (int i = 0; i < batch; ++i) note(i, st_all[i], one_all[i]);
    batch_end(ctx, S, start);
    if (worst != BKS_OK && worst != BKS_WARN_DEFLATED)
        return fail(ctx, worst, "at least one matrix of the batch failed (see statuses)");
    ctx->last_error.clear();
    return worst;
}

}  // namespace

namespace bks {

cudaError_t allow_dynamic_smem(const void* fn, size_t need) {
    struct Entry {
        const void* fn;
        int dev;
        int limit;
    };
    static std::mutex mu;
    static std::vector<Entry> done;
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    std::lock_guard<std::mutex> lock(mu);
    for (const Entry& e : done)
        if (e.fn == fn && e.dev == dev) return size_t(e.limit) >= need ? cudaSuccess : cudaErrorInvalidValue;
    cudaFuncAttributes fa;
    err = cudaFuncGetAttributes(&fa, fn);
    if (err != cudaSuccess) return err;
    int optin = 0;
    err = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (err != cudaSuccess) return err;
    const int limit = optin - int(fa.sharedSizeBytes);
    err = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, limit);
    if (err != cudaSuccess) return err;
    done.push_back(Entry{fn, dev, limit});
    return size_t(limit) >= need ? cudaSuccess : cudaErrorInvalidValue;
}

int ctx_num_sms(const bks_ctx* ctx) { return ctx->num_sms; }

bks_status ctx_workspace(bks_ctx* ctx, size_t bytes, CtxInfo* info) {
    DeviceGuard g(ctx->device);
    const bks_status s = ensure_ws(ctx, bytes);
    if (s != BKS_OK) return s;
    info->ws = ctx->ws;
    info->stream = ctx->stream;
    info->num_sms = ctx->num_sms;
    info->device = ctx->device;
    return BKS_OK;
}

bks_status ctx_fail(bks_ctx* ctx, bks_status s, const char* msg) { return fail(ctx, s, msg); }

}  // namespace bks

// ====================================================================== C-ABI

extern "C" {

void bks_opts_default(bks_opts* o) {
    if (o == nullptr) return;
    std::memset(o, 0, sizeof(*o));
    o->precision = BKS_PREC_AUTO;
    o->refine = 1;
    o->basis_only = 0;
    o->sign_fix = 1;
    o->jacobi_max_sweeps = 40;
    o->jacobi_tol = 0.0;
    o->profile = 0;
}

int bks_version(void) { return BKS_VERSION; }

const char* bks_status_string(bks_status s) {
    switch (s) {
        case BKS_OK: return "ok";
        case BKS_ERR_INVALID_ARG: return "invalid argument";
        case BKS_ERR_CUDA: return "CUDA error";
        case BKS_ERR_NOMEM: return "out of device memory";
        case BKS_ERR_NONFINITE: return "non-finite value";
        case BKS_ERR_BREAKDOWN: return "Cholesky breakdown";
        case BKS_ERR_NOT_CONVERGED: return "eigen-solver did not converge";
        case BKS_ERR_TIMEOUT: return "device wait timed out";
        case BKS_ERR_UNSUPPORTED: return "unsupported";
        case BKS_WARN_DEFLATED: return "ok (q capped or columns deflated)";
    }
    return "unknown status";
}

const char* bks_last_error(const bks_ctx* ctx) { return ctx ? ctx->last_error.c_str() : "no context"; }

bks_status bks_create(bks_ctx** out, int device) {
    if (out == nullptr) return BKS_ERR_INVALID_ARG;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
        cudaGetLastError();
        return BKS_ERR_INVALID_ARG;
    }
    bks_ctx* ctx = new bks_ctx();
    ctx->device = device;
    DeviceGuard g(device);
    cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (cudaMallocHost(&ctx->host_status, 4 * sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        delete ctx;
        return BKS_ERR_CUDA;
    }
    *out = ctx;
    return BKS_OK;
}

bks_status bks_destroy(bks_ctx* ctx) {
    if (ctx == nullptr) return BKS_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    for (bks_ctx* sub : ctx->subs) bks_destroy(sub);
    ctx->subs.clear();
    cudaStreamSynchronize(ctx->stream);
    if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    if (ctx->ws_owned && ctx->ws) cudaFree(ctx->ws);
    for (auto e : ctx->events) cudaEventDestroy(e);
    if (ctx->host_status) cudaFreeHost(ctx->host_status);
    if (ctx->host_vals) cudaFreeHost(ctx->host_vals);
    delete ctx;
    return BKS_OK;
}

bks_status bks_set_stream(bks_ctx* ctx, void* stream) {
    if (ctx == nullptr) return BKS_ERR_INVALID_ARG;
    ctx->stream = static_cast<cudaStream_t>(stream);
    return BKS_OK;
}

bks_status bks_set_workspace(bks_ctx* ctx, void* ptr, size_t bytes) {
    if (ctx == nullptr) return BKS_ERR_INVALID_ARG;
    if (ptr != nullptr && (reinterpret_cast<uintptr_t>(ptr) % 256) != 0)
        return fail(ctx, BKS_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    DeviceGuard g(ctx->device);
    if (ctx->ws_owned && ctx->ws) {
        cudaStreamSynchronize(ctx->stream);
        cudaFree(ctx->ws);
    }
    ctx->ws = ptr;
    ctx->ws_bytes = ptr ? bytes : 0;
    ctx->ws_owned = false;
    return BKS_OK;
}

bks_status bks_workspace_size(const bks_matrix* A, int k, int q, int method, const bks_opts* opts,
                              size_t* bytes) {
    if (A == nullptr || bytes == nullptr || k < 1 || q < 0) return BKS_ERR_INVALID_ARG;
    const int64_t mn = A->n < A->d ? A->n : A->d;
    if (int64_t(k) > mn) return BKS_ERR_INVALID_ARG;
    bks_opts o;
    if (opts) o = *opts; else bks_opts_default(&o);
    int prec = o.precision;
    if (prec == BKS_PREC_AUTO) prec = A->dtype == BKS_F64 ? BKS_PREC_F64 : BKS_PREC_F32;
    const size_t tb = prec == BKS_PREC_F64 ? 8 : 4;
    const int kz = k;
    if (o.block_p != 0 && (o.block_p < kz || int64_t(o.block_p) > mn)) return BKS_ERR_INVALID_ARG;
    k = o.block_p > 0 ? o.block_p : kz;   // block size
    int q_eff = q;
    if (method == 0) {
        const int64_t cap = mn / k - 1;
        if (q_eff > cap) q_eff = int(cap);
    }
    const int w = method == 0 ? k * (q_eff + 1) : k;
    int sms = 152;
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess)
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaGetLastError();
    *bytes = make_plan(A, k, q_eff, w, tb, sms, w, o.eig_f64 != 0).total;   // enough for the Ritz triplets too
    return BKS_OK;
}

bks_status bks_block_krylov(bks_ctx* ctx, const bks_matrix* A, int k, int q, uint64_t seed,
                            const void* pi, void* Z, void* sigma, void* V, const bks_opts* opts,
                            bks_stats* stats) {
    return solve_entry(ctx, A, k, q, seed, pi, Z, sigma, V, opts, stats, true);
}

bks_status bks_block_krylov_adaptive(bks_ctx* ctx, const bks_matrix* A, int k, int q_max, double tol,
                                     uint64_t seed, const void* pi, void* Z, void* sigma, void* V,
                                     const bks_opts* opts, bks_stats* stats) {
    if (ctx == nullptr) return BKS_ERR_INVALID_ARG;
    if (!(tol > 0.0) || !(tol < 1.0))
        return fail(ctx, BKS_ERR_INVALID_ARG, "tol must be in (0, 1)");
    return solve_entry(ctx, A, k, q_max, seed, pi, Z, sigma, V, opts, stats, true, false, false, tol);
}

bks_status bks_simul_iter(bks_ctx* ctx, const bks_matrix* A, int k, int q, uint64_t seed,
                          const void* pi, void* Z, void* sigma, void* V, const bks_opts* opts,
                          bks_stats* stats) {
    return solve_entry(ctx, A, k, q, seed, pi, Z, sigma, V, opts, stats, false);
}

bks_status bks_selftest_wait(bks_ctx* ctx, int which) {
    if (ctx == nullptr) return BKS_ERR_INVALID_ARG;
    if (which != 0 && which != 1) return fail(ctx, BKS_ERR_INVALID_ARG, "which must be 0 or 1");
    DeviceGuard g(ctx->device);
    bks_status s = ensure_ws(ctx, 256);
    if (s != BKS_OK) return s;
    Exec ex;
    ex.stream = ctx->stream;
    ex.num_sms = ctx->num_sms;
    ex.status = static_cast<int*>(ctx->ws);
    unsigned* bar = reinterpret_cast<unsigned*>(static_cast<char*>(ctx->ws) + 64);
    cudaMemsetAsync(ex.status, 0, 16, ctx->stream);
    wait_selftest(ex, which, bar);
    cudaError_t e = cudaMemcpyAsync(ctx->host_status, ex.status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "bks_selftest_wait");
    if (ctx->host_status[0] & ST_TIMEOUT)
        return fail(ctx, BKS_ERR_TIMEOUT, which == 0 ? "an mbarrier wait gave up (self-test)"
                                                    : "a grid-barrier wait gave up (self-test)");
    ctx->last_error.clear();
    return BKS_OK;
}

bks_status bks_block_lanczos(bks_ctx* ctx, const bks_matrix* A, int k, int q, int reorth, uint64_t seed,
                             const void* pi, void* Z, void* sigma, void* V, const bks_opts* opts,
                             bks_stats* stats) {
    if (ctx == nullptr) return BKS_ERR_INVALID_ARG;
    if (reorth != BKS_REORTH_FULL && reorth != BKS_REORTH_LOCAL && reorth != BKS_REORTH_NONE)
        return fail(ctx, BKS_ERR_INVALID_ARG, "reorth must be BKS_REORTH_FULL, _LOCAL or _NONE");
    return solve_entry(ctx, A, k, q, seed, pi, Z, sigma, V, opts, stats, true, false, false, 0.0, reorth);
}

bks_status bks_block_krylov_batched(bks_ctx* ctx, int batch, const bks_matrix* As, int k, int q,
                                    const uint64_t* seeds, const void* const* pis, void* const* Zs,
                                    void* const* sigmas, void* const* Vs, const bks_opts* opts,
                                    bks_stats* stats, bks_status* statuses) {
    return batched_solve(ctx, batch, As, k, q, seeds, pis, Zs, sigmas, Vs, opts, stats, statuses, true, false,
                         "bks_block_krylov_batched");
}

bks_status bks_batched_autotune(bks_ctx* ctx, int batch, const bks_matrix* As, int k, int q,
                                const uint64_t* seeds, const void* const* pis, void* const* Zs, void* const* sigmas,
                                void* const* Vs, const bks_opts* opts, int* best_max_sms, float* best_ms) {
    if (ctx == nullptr) return BKS_ERR_INVALID_ARG;
    if (batch < 1) return fail(ctx, BKS_ERR_INVALID_ARG, "bks_batched_autotune needs a non-empty batch");
    bks_opts ob;
    if (opts) ob = *opts; else bks_opts_default(&ob);
    DeviceGuard g(ctx->device);
    const int n_sm = ctx->num_sms;
    const int cands[] = {n_sm / 16, n_sm / 8, n_sm / 4, n_sm / 2, n_sm};
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int best = 0;
    float best_t = 0.f;
    bks_status worst = BKS_OK;
    for (int trial = 0; trial < 2; ++trial)   // a warm-up pass over the candidates, then the timed one
        for (int c : cands) {
            if (c < 1) continue;
            ob.max_sms = c;
            cudaEventRecord(e0, ctx->stream);
            const bks_status st = batched_solve(ctx, batch, As, k, q, seeds, pis, Zs, sigmas, Vs, &ob, nullptr,
                                                nullptr, true, false, "bks_batched_autotune");
            cudaEventRecord(e1, ctx->stream);
            if (st != BKS_OK && st != BKS_WARN_DEFLATED) {
                worst = st;
                break;
            }
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (trial == 1 && (best == 0 || ms < best_t)) {
                best = c;
                best_t = ms;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (worst != BKS_OK) return worst;
    ctx->batch_sms[batch_signature(batch, As, k, q, true, false)] = best;
    ob.max_sms = best;   // the outputs: those of the chosen budget
    const bks_status st = batched_solve(ctx, batch, As, k, q, seeds, pis, Zs, sigmas, Vs, &ob, nullptr, nullptr,
                                        true, false, "bks_batched_autotune");
    if (best_max_sms) *best_max_sms = best;
    if (best_ms) *best_ms = best_t;
    return st;
}

int bks_batch_budget(const bks_ctx* ctx, int batch, const bks_matrix* As, int k, int q, int method) {
    if (ctx == nullptr || batch < 1 || As == nullptr) return 0;
    const auto it = ctx->batch_sms.find(batch_signature(batch, As, k, q, method == 0, false));
    return it != ctx->batch_sms.end() ? it->second : default_batch_sms(ctx->num_sms);
}

bks_status bks_ritz_triplets_batched(bks_ctx* ctx, int batch, const bks_matrix* As, int k, int q,
                                     const uint64_t* seeds, const void* const* pis, int method, void* const* Us,
                                     void* const* sigmas, void* const* Vs, const bks_opts* opts,
                                     bks_status* statuses) {
    if (ctx == nullptr) return BKS_ERR_INVALID_ARG;
    if (method != 0 && method != 1) return fail(ctx, BKS_ERR_INVALID_ARG, "method must be 0 (BKI) or 1 (SI)");
    if (batch > 0 && Vs == nullptr) return fail(ctx, BKS_ERR_INVALID_ARG, "Vs is required for the Ritz triplets");
    for (int i = 0; i < batch && Vs != nullptr; ++i)
        if (Vs[i] == nullptr) return fail(ctx, BKS_ERR_INVALID_ARG, "Vs is required for the Ritz triplets");
    return batched_solve(ctx, batch, As, k, q, seeds, pis, Us, sigmas, Vs, opts, nullptr, statuses, method == 0,
                         true, "bks_ritz_triplets_batched");
}

bks_status bks_backward_batched(bks_ctx* ctx, int dtype, int batch, const int64_t* ns, const int64_t* ds, int k,
                                const int* ws, const void* const* Us, const void* const* sigmas,
                                const void* const* Vs, const void* const* g_sigmas, const void* const* Gs,
                                void* const* dAs, double gap_tau, bks_status* statuses) {
    if (ctx == nullptr) return BKS_ERR_INVALID_ARG;
    if (batch < 0 || (batch > 0 && (ns == nullptr || ds == nullptr || ws == nullptr || Us == nullptr ||
                                    sigmas == nullptr || Vs == nullptr || dAs == nullptr ||
                                    (g_sigmas == nullptr && Gs == nullptr))))
        return fail(ctx, BKS_ERR_INVALID_ARG, "bad bks_backward_batched arguments");
    if (batch == 0) return BKS_OK;
    DeviceGuard g(ctx->device);
    const int S = batch < BKS_BATCH_STREAMS ? batch : BKS_BATCH_STREAMS;
    bks_status cs = ensure_subs(ctx, S);
    if (cs != BKS_OK) return cs;
    cudaEvent_t start = batch_begin(ctx, S);
    // thread t takes matrices t, t + T, ... on its stream contexts t and t + T in turn (each
    // backward synchronises its own stream); every gradient is that of a single call
    const int T = S < BKS_BATCH_THREADS ? S : BKS_BATCH_THREADS;
    std::vector<bks_status> st_all(size_t(batch), BKS_OK);
    auto worker = [&](int t) {
        DeviceGuard gd(ctx->device);
        bks_ctx* subs[2] = {ctx->subs[t], ctx->subs[t + T < S ? t + T : t]};
        int r = 0;
        for (int i = t; i < batch; i += T, ++r)
            st_all[i] = bks_backward(subs[r & 1], dtype, ns[i], ds[i], k, ws[i], Us[i], sigmas[i], Vs[i],
                                     g_sigmas ? g_sigmas[i] : nullptr, Gs ? Gs[i] : nullptr, dAs[i], gap_tau);
    };
    run_workers(T, worker);
    batch_end(ctx, S, start);
    bks_status worst = BKS_OK;
    for (int i = 0; i < batch; ++i) {
        if (statuses) statuses[i] = st_all[i];
        if (st_all[i] != BKS_OK && worst == BKS_OK) worst = st_all[i];
    }
    if (worst != BKS_OK) return fail(ctx, worst, "at least one matrix of the batch failed (see statuses)");
    ctx->last_error.clear();
    return BKS_OK;
}

bks_status bks_ritz_triplets(bks_ctx* ctx, const bks_matrix* A, int k, int q, uint64_t seed, const void* pi,
                             int method, void* U, void* sigma, void* V, const bks_opts* opts, bks_stats* stats) {
    if (method != 0 && method != 1) return fail(ctx, BKS_ERR_INVALID_ARG, "method must be 0 (BKI) or 1 (SI)");
    if (V == nullptr) return fail(ctx, BKS_ERR_INVALID_ARG, "V is required for the Ritz triplets");
    return solve_entry(ctx, A, k, q, seed, pi, U, sigma, V, opts, stats, method == 0, true);
}

bks_status bks_gen_pi(bks_ctx* ctx, uint64_t seed, int64_t d, int k, int dtype, void* out) {
    if (ctx == nullptr) return BKS_ERR_INVALID_ARG;
    if (out == nullptr || d < 1 || k < 1 || (dtype != BKS_F32 && dtype != BKS_F64))
        return fail(ctx, BKS_ERR_INVALID_ARG, "bad bks_gen_pi arguments");
    DeviceGuard g(ctx->device);
    Exec ex;
    ex.stream = ctx->stream;
    ex.num_sms = ctx->num_sms;
    if (dtype == BKS_F32) gen_pi_device<float>(ex, seed, d, k, static_cast<float*>(out), k, false);
    else gen_pi_device<double>(ex, seed, d, k, static_cast<double*>(out), k, false);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? BKS_OK : cuda_fail(ctx, e, "bks_gen_pi");
}

bks_status bks_gen_pi_host(uint64_t seed, int64_t d, int k, float* out_host) {
    if (out_host == nullptr || d < 1 || k < 1) return BKS_ERR_INVALID_ARG;
    gen_pi_host(seed, d, k, out_host);
    return BKS_OK;
}

bks_status bks_csr_transpose(bks_ctx* ctx, const bks_matrix* A, int64_t* t_row_ptr,
                             int32_t* t_col_idx, float* t_vals) {
    if (ctx == nullptr) return BKS_ERR_INVALID_ARG;
    bks_status s = check_matrix(ctx, A);
    if (s != BKS_OK) return s;
    if (A->kind != BKS_CSR || t_row_ptr == nullptr || t_col_idx == nullptr || t_vals == nullptr)
        return fail(ctx, BKS_ERR_INVALID_ARG, "bks_csr_transpose needs a CSR matrix and three outputs");
    DeviceGuard g(ctx->device);
    const size_t o_stat = round_up(int64_t(csr_transpose_scratch(A->n, A->d)), 256);
    s = ensure_ws(ctx, o_stat + 256);
    if (s != BKS_OK) return s;
    Exec ex;
    ex.stream = ctx->stream;
    ex.num_sms = ctx->num_sms;
    ex.status = reinterpret_cast<int*>(static_cast<char*>(ctx->ws) + o_stat);
    cudaMemsetAsync(ex.status, 0, sizeof(int), ctx->stream);
    csr_check(ex, A->row_ptr, A->col_idx, A->n, A->d, A->nnz, ex.status);
    csr_transpose(ex, A->row_ptr, A->col_idx, static_cast<const float*>(A->vals), A->n, A->d, A->nnz,
                  t_row_ptr, t_col_idx, t_vals, ctx->ws);
    cudaError_t e = cudaMemcpyAsync(ctx->host_status, ex.status, sizeof(int), cudaMemcpyDeviceToHost,
                                    ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "bks_csr_transpose");
    if (ctx->host_status[0] & ST_BADINPUT)
        return fail(ctx, BKS_ERR_INVALID_ARG, "CSR structure check failed (row_ptr or col_idx)");
    return BKS_OK;
}

bks_status bks_matmul(bks_ctx* ctx, const bks_matrix* A, int trans, int c, const void* X,
                      int64_t ldx, void* Y, int64_t ldy, int flags) {
    if (ctx == nullptr) return BKS_ERR_INVALID_ARG;
    bks_status s = check_matrix(ctx, A);
    if (s != BKS_OK) return s;
    const int64_t rows_x = trans ? A->n : A->d, rows_y = trans ? A->d : A->n;
    if (c < 1 || X == nullptr || Y == nullptr || ldx < rows_x || ldy < rows_y)
        return fail(ctx, BKS_ERR_INVALID_ARG, "bad bks_matmul arguments");
    DeviceGuard g(ctx->device);
    const bool f64 = A->dtype == BKS_F64;
    const int64_t cap = gemm_partial_elems(c, rows_y, rows_x, ctx->num_sms);
    int64_t tcap = tc_partial_floats(A->n, A->d, c < 128 ? c : 128, ctx->num_sms);
    const bool bf16_a = A->kind == BKS_DENSE && A->dtype == BKS_BF16;
    const int64_t xb_cap = bf16_a ? 3 * int64_t(c < 128 ? c : 128) * ldx : 0;
    if (bf16_a) {
        const int64_t b = tc_bf16_partial_floats(A->n, A->d, c < 128 ? c : 128, ctx->num_sms);
        if (b > tcap) tcap = b;
    }
    Arena ar;
    const size_t o_part = ar.take(size_t(cap) * sizeof(double) + 8),
                 o_xh = ar.take(size_t(c) * ldx * 4), o_xl = ar.take(size_t(c) * ldx * 4),
                 o_tp = ar.take(size_t(tcap) * 4), o_stat = ar.take(16),
                 o_xb = ar.take(size_t(xb_cap) * 2 + 16);
    CsrLayout cl{};
    if (A->kind == BKS_CSR) cl.take(ar, A, c);
    s = ensure_ws(ctx, ar.off);
    if (s != BKS_OK) return s;
    Exec ex;
    ex.stream = ctx->stream;
    ex.num_sms = ctx->num_sms;
    char* wsb = static_cast<char*>(ctx->ws);
    double* part = reinterpret_cast<double*>(wsb + o_part);
    ProductWs pw;
    pw.xh = reinterpret_cast<float*>(wsb + o_xh);
    pw.xl = reinterpret_cast<float*>(wsb + o_xl);
    pw.tpart = reinterpret_cast<float*>(wsb + o_tp);
    pw.tpart_cap = tcap;
    pw.simt_only = (flags & BKS_MATMUL_SIMT) != 0;
    if (bf16_a) {
        pw.xb = reinterpret_cast<__nv_bfloat16*>(wsb + o_xb);
        pw.xb_cap = xb_cap;
        pw.bf16_pieces = (flags & BKS_MATMUL_EXACT) ? 3 : 1;
    }
    int* stat = reinterpret_cast<int*>(wsb + o_stat);
    ex.status = stat;
    cudaMemsetAsync(stat, 0, 16, ctx->stream);
    if (A->kind == BKS_CSR) cl.prepare(ex, wsb, A, pw.csr);
    if (f64)
        product<double>(ex, A, trans != 0, c, static_cast<const double*>(X), ldx,
                        static_cast<double*>(Y), ldy, part, cap, pw);
    else
        product<float>(ex, A, trans != 0, c, static_cast<const float*>(X), ldx,
                       static_cast<float*>(Y), ldy, part, cap, pw);
    cudaError_t e = cudaMemcpyAsync(ctx->host_status, stat, sizeof(int), cudaMemcpyDeviceToHost,
                                    ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "bks_matmul");
    if (ctx->host_status[0] & ST_BADINPUT) return fail(ctx, BKS_ERR_INVALID_ARG, "CSR structure check failed");
    if (ctx->host_status[0] & ST_TIMEOUT)
        return fail(ctx, BKS_ERR_TIMEOUT, "a tensor-core pipeline wait timed out");
    return BKS_OK;
}

bks_status bks_orthonormalize(bks_ctx* ctx, int dtype, int64_t len, int m, int c, const void* Qb,
                              int64_t ldq, void* W, int64_t ldw) {
    if (ctx == nullptr) return BKS_ERR_INVALID_ARG;
    if ((dtype != BKS_F32 && dtype != BKS_F64) || len < 1 || m < 0 || c < 1 || W == nullptr ||
        (m > 0 && Qb == nullptr) || ldw < len || (m > 0 && ldq != ldw) || int64_t(m) + c > len)
        return fail(ctx, BKS_ERR_INVALID_ARG, "bad bks_orthonormalize arguments (ldq must equal ldw)");
    DeviceGuard g(ctx->device);
    const size_t tb = dtype == BKS_F64 ? 8 : 4;
    const bool tc = dtype == BKS_F32;
    const OrthSizes z = orth_sizes(len, ldw, m, c, int(tb), tc, ctx->num_sms);
    Arena a;
    const size_t o_part = a.take(z.partials), o_g = a.take(z.g), o_rfac = a.take(z.rfac),
                 o_ct = a.take(z.ct), o_xh = a.take(z.xh), o_xl = a.take(z.xh), o_tp = a.take(z.tpart),
                 o_fp = a.take(z.fpart), o_fg = a.take(z.fgram), o_fb = a.take(z.fbar),
                 o_wtmp = a.take(size_t(c) * ldw * tb), o_stat = a.take(16),
                 o_op = a.take(z.otc_part), o_oc = a.take(z.otc_cts), o_oh = a.take(z.otc_h),
                 o_ob = a.take(z.otc_bar);
    // the tensor-core kernel reads the updates from a row-major copy of Qb
    const int64_t ldr = round_up(m > 0 ? m : 1, 32);
    const bool otc = tc && z.otc_cap > 0 && orth_tc_fits(len, m, c, ctx->num_sms);
    const size_t o_qr = a.take(otc && m > 0 ? size_t(len) * ldr * 4 : 0);
    bks_status s = ensure_ws(ctx, a.off);
    if (s != BKS_OK) return s;
    char* base = static_cast<char*>(ctx->ws);
    Exec ex;
    ex.stream = ctx->stream;
    ex.num_sms = ctx->num_sms;
    int* stat = reinterpret_cast<int*>(base + o_stat);
    ex.status = stat;
    cudaMemsetAsync(stat, 0, 16, ctx->stream);
    OrthWs ws;
    ws.partials = reinterpret_cast<double*>(base + o_part);
    ws.cap = z.cap;
    ws.g = base + o_g;
    ws.rfac = base + o_rfac;
    ws.ldp = z.ldp;
    ws.ct = base + o_ct;
    ws.ldc = z.ldc;
    ws.shifted_flag = stat + 2;
    if (tc) {
        ws.xh = reinterpret_cast<float*>(base + o_xh);
        ws.xl = reinterpret_cast<float*>(base + o_xl);
        ws.tpart = reinterpret_cast<float*>(base + o_tp);
        ws.tpart_cap = z.tcap;
        ws.fpart = reinterpret_cast<float*>(base + o_fp);
        ws.fpart_cap = z.fcap;
        ws.fgram = reinterpret_cast<float*>(base + o_fg);
        ws.fbar = reinterpret_cast<unsigned*>(base + o_fb);
    }
    if (otc) {
        ws.otc_part = reinterpret_cast<float*>(base + o_op);
        ws.otc_cap = z.otc_cap;
        ws.otc_cts = reinterpret_cast<float*>(base + o_oc);
        ws.otc_ldct = z.otc_ldct;
        ws.otc_h = reinterpret_cast<float*>(base + o_oh);
        ws.otc_bar = reinterpret_cast<unsigned*>(base + o_ob);
        if (m > 0) {
            ws.qr = reinterpret_cast<float*>(base + o_qr);
            ws.ldr = ldr;
            transpose_in<float>(ex, Qb, BKS_F32, m, len, ldq, ws.qr, ldr);   // qr[l][r] = Qb[r][l]
        }
    }
    if (dtype == BKS_F64)
        orth_block<double>(ex, len, ldw, static_cast<const double*>(Qb), m, static_cast<double*>(W), c,
                           reinterpret_cast<double*>(base + o_wtmp), static_cast<double*>(W), ws);
    else
        orth_block<float>(ex, len, ldw, static_cast<const float*>(Qb), m, static_cast<float*>(W), c,
                          reinterpret_cast<float*>(base + o_wtmp), static_cast<float*>(W), ws);
    cudaError_t e = cudaMemcpyAsync(ctx->host_status, stat, 3 * sizeof(int), cudaMemcpyDeviceToHost,
                                    ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "bks_orthonormalize");
    if (ctx->host_status[0] & ST_NONFINITE) return fail(ctx, BKS_ERR_NONFINITE, "non-finite Gram matrix");
    if (ctx->host_status[0] & ST_BREAKDOWN) return fail(ctx, BKS_ERR_BREAKDOWN, "Cholesky breakdown");
    return BKS_OK;
}

bks_status bks_sym_eig(bks_ctx* ctx, int dtype, int w, const void* M, int64_t ldm, void* lam,
                       void* U, int64_t ldu) {
    if (ctx == nullptr) return BKS_ERR_INVALID_ARG;
    if ((dtype != BKS_F32 && dtype != BKS_F64) || w < 1 || M == nullptr || lam == nullptr ||
        U == nullptr || ldm < w || ldu < w)
        return fail(ctx, BKS_ERR_INVALID_ARG, "bad bks_sym_eig arguments");
    const size_t tb = dtype == BKS_F64 ? 8 : 4;
    int C, b, E;
    size_t sm;
    if (!jacobi_plan(w, int(tb), C, b, E, sm))
        return fail(ctx, BKS_ERR_UNSUPPORTED, "w exceeds the Jacobi solver's limit");
    DeviceGuard g(ctx->device);
    Arena a;
    const size_t o_x = a.take(size_t(w) * w * tb), o_nrm = a.take(size_t(w) * tb),
                 o_vt = a.take(size_t(w) * w * tb), o_ord = a.take(size_t(w) * 4),
                 o_stat = a.take(16);
    bks_status s = ensure_ws(ctx, a.off);
    if (s != BKS_OK) return s;
    char* base = static_cast<char*>(ctx->ws);
    Exec ex;
    ex.stream = ctx->stream;
    ex.num_sms = ctx->num_sms;
    int* stat = reinterpret_cast<int*>(base + o_stat);
    ex.status = stat;
    cudaMemsetAsync(stat, 0, 16, ctx->stream);
    if (dtype == BKS_F64) {
        sym_eig<double>(ex, w, static_cast<const double*>(M), ldm, reinterpret_cast<double*>(base + o_x),
                        w, static_cast<double*>(lam), reinterpret_cast<double*>(base + o_nrm),
                        reinterpret_cast<double*>(base + o_vt), w, reinterpret_cast<int*>(base + o_ord),
                        40, 0.0, stat + 1);
        transpose_in<double>(ex, base + o_vt, BKS_F64, w, w, w, static_cast<double*>(U), ldu);
    } else {
        sym_eig<float>(ex, w, static_cast<const float*>(M), ldm, reinterpret_cast<float*>(base + o_x),
                       w, static_cast<float*>(lam), reinterpret_cast<float*>(base + o_nrm),
                       reinterpret_cast<float*>(base + o_vt), w, reinterpret_cast<int*>(base + o_ord),
                       40, 0.0, stat + 1);
        transpose_in<float>(ex, base + o_vt, BKS_F32, w, w, w, static_cast<float*>(U), ldu);
    }
    cudaError_t e = cudaMemcpyAsync(ctx->host_status, stat, 3 * sizeof(int), cudaMemcpyDeviceToHost,
                                    ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "bks_sym_eig");
    if (ctx->host_status[0] & ST_NOT_CONVERGED) return fail(ctx, BKS_ERR_NOT_CONVERGED, "Jacobi sweep cap");
    if (ctx->host_status[1] < 0) return fail(ctx, BKS_ERR_UNSUPPORTED, "Jacobi launch failed");
    return BKS_OK;
}

}  // extern "C"
