// Fused single-kernel path for small windows.  Not enabled yet: every geometry takes the generic path.
#include "runtime.hpp"

namespace dh {

bool use_fused(const dhk::Plan&) { return false; }

cudaError_t fused_init() { return cudaSuccess; }

int launch_fused_path(Handle*, const void*, int, int, void*, void*, cudaStream_t) {
    return fail(DH_ERROR_ERROR, "fused path unavailable");
}

}  // namespace dh
