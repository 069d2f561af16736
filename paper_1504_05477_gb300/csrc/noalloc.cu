// Eigen-solve entry point that allocates nothing.
//
// Some callers cannot allocate device memory at call time: code that runs inside a
// host callback or a real-time loop where cudaMalloc's implicit device
// synchronisation is not allowed, applications whose memory is owned by another
// runtime or a fixed arena, and embedded uses that must not grow their footprint
// after start-up.  For them bks_sym_eig_noalloc runs the same one-sided Jacobi
// kernels as bks_sym_eig, with every scratch buffer carved from one statically sized
// device array that the library image carries (each GPU that loads the library holds
// it until the process exits).
#include <cstring>

#include "../../include/bks.h"
#include "common.cuh"

namespace bks {
namespace {

// Scratch of the no-allocation eigen-solve: X (w x w), Vt (w x w), column norms,
// order and the status words, each 256-byte aligned.  5 MiB covers w <=
// BKS_NOALLOC_EIG_MAX_W in FP32 and FP64 (the static_assert below checks the FP64 case).
constexpr size_t align256(size_t x) { return (x + 255) / 256 * 256; }
struct ScratchLayout {
    size_t x, nrm, vt, ord, stat, total;
    constexpr ScratchLayout(int w, size_t tb)
        : x(0),
          nrm(align256(size_t(w) * w * tb)),
          vt(nrm + align256(size_t(w) * tb)),
          ord(vt + align256(size_t(w) * w * tb)),
          stat(ord + align256(size_t(w) * 4)),
          total(stat + 256) {}
};
constexpr size_t kScratchBytes = size_t(5) << 20;
static_assert(ScratchLayout(BKS_NOALLOC_EIG_MAX_W, 8).total <= kScratchBytes,
              "the static scratch must hold the FP64 layout at the largest supported width");
static __device__ __align__(256) unsigned char g_eig_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
void* g_scratch_ptr[kMaxDevices];   // device address of g_eig_scratch, per device

}  // namespace
}  // namespace bks

using namespace bks;

extern "C" bks_status bks_sym_eig_noalloc(void* stream, int dtype, int w, const void* M,
                                          int64_t ldm, void* lam, void* U, int64_t ldu) {
    if ((dtype != BKS_F32 && dtype != BKS_F64) || w < 1 || w > BKS_NOALLOC_EIG_MAX_W ||
        M == nullptr || lam == nullptr || U == nullptr || ldm < w || ldu < w)
        return BKS_ERR_INVALID_ARG;
    const size_t tb = dtype == BKS_F64 ? 8 : 4;
    int C, b, E;
    size_t smem;
    if (!jacobi_plan(w, int(tb), C, b, E, smem)) return BKS_ERR_UNSUPPORTED;
    const ScratchLayout lay(w, tb);
    const size_t o_x = lay.x, o_nrm = lay.nrm, o_vt = lay.vt, o_ord = lay.ord, o_stat = lay.stat;
    if (lay.total > kScratchBytes) return BKS_ERR_INVALID_ARG;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return BKS_ERR_CUDA;
    }
    if (g_scratch_ptr[dev] == nullptr) {
        // once per device, with that device current: the array's device address (the
        // host-side symbol is only a stand-in and must never reach a kernel)
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_eig_scratch);
        if (e != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return BKS_ERR_CUDA;
        }
        g_scratch_ptr[dev] = p;
    }
    char* base = static_cast<char*>(g_scratch_ptr[dev]);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Exec ex;
    ex.stream = st;
    cudaDeviceGetAttribute(&ex.num_sms, cudaDevAttrMultiProcessorCount, dev);
    int* stat = reinterpret_cast<int*>(base + o_stat);   // [status, sweeps]
    ex.status = stat;
    cudaMemsetAsync(stat, 0, 2 * sizeof(int), st);       // the array keeps the last call's words
    if (dtype == BKS_F64) {
        sym_eig<double>(ex, w, static_cast<const double*>(M), ldm, reinterpret_cast<double*>(base + o_x), w,
                        static_cast<double*>(lam), reinterpret_cast<double*>(base + o_nrm),
                        reinterpret_cast<double*>(base + o_vt), w, reinterpret_cast<int*>(base + o_ord),
                        40, 0.0, stat + 1);
        transpose_in<double>(ex, base + o_vt, BKS_F64, w, w, w, static_cast<double*>(U), ldu);
    } else {
        sym_eig<float>(ex, w, static_cast<const float*>(M), ldm, reinterpret_cast<float*>(base + o_x), w,
                       static_cast<float*>(lam), reinterpret_cast<float*>(base + o_nrm),
                       reinterpret_cast<float*>(base + o_vt), w, reinterpret_cast<int*>(base + o_ord),
                       40, 0.0, stat + 1);
        transpose_in<float>(ex, base + o_vt, BKS_F32, w, w, w, static_cast<float*>(U), ldu);
    }
    int words[2] = {0, 0};
    cudaError_t e = cudaMemcpyAsync(words, stat, sizeof(words), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return BKS_ERR_CUDA;
    if (words[0] & ST_NOT_CONVERGED) return BKS_ERR_NOT_CONVERGED;
    if (words[1] < 0) return BKS_ERR_UNSUPPORTED;
    return BKS_OK;
}
