// Context services shared by the translation units that implement C-ABI entry points
// outside solver.cu (the context itself is defined there).
#pragma once
#include <cuda_runtime.h>

#include "../../include/bks.h"

namespace bks {

struct CtxInfo {
    void* ws;              // device workspace, at least the requested bytes
    cudaStream_t stream;   // the context's stream
    int num_sms;
    int device;
};

int ctx_num_sms(const bks_ctx* ctx);
// Grow the context workspace to `bytes` (synchronising the stream if it is reallocated).
bks_status ctx_workspace(bks_ctx* ctx, size_t bytes, CtxInfo* info);
// Record `msg` as the context's last error and return s.
bks_status ctx_fail(bks_ctx* ctx, bks_status s, const char* msg);

}  // namespace bks
