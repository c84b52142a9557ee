// Which kernel path a call runs: the fused single-kernel paths (128 x 128 windows: k_fused.cu and its pruned and
// group-transform variants; 256 x 256 windows with 96 x 96 fields: k_fused256.cu) or the generic three-kernel
// path (k_split.cu), by the geometry, the frames' layout and the handle's variant setting.
#include <cuda_runtime.h>
#include <stdint.h>

#include "runtime.hpp"

namespace dh {

int resolve_variant(const Handle* H, const dhk::Plan& P, bool aligned) {
    // 256 x 256 windows: one fused kernel, which every variant but the generic one selects
    const bool big = aligned && use_fused256(P);
    const bool fused = aligned && use_fused(P);
    const bool pruned = fused && use_fused_pr(P);
    const bool groups = fused && use_fused_g(P);
    // without a tuner's choice, the fused kernel that transforms every column (measured fastest on the batching
    // workload; the pruned and group-transform kernels are tuner candidates)
    const int v = H->variant != kVariantAuto ? H->variant : (H->tuned ? H->tuned : kVariantFusedLegacy);
    if (v == kVariantGeneric) return kVariantGeneric;
    if (big) return kVariantFusedLegacy;
    if (v == kVariantFusedLegacy) return fused ? kVariantFusedLegacy : kVariantGeneric;
    if (v == kVariantFusedGroups) return groups ? kVariantFusedGroups : fused ? kVariantFusedLegacy : kVariantGeneric;
    return pruned ? kVariantFusedPruned : fused ? kVariantFusedLegacy : kVariantGeneric;
}

bool fused_allowed(const Handle* H, const dhk::Plan& P) { return resolve_variant(H, P, true) != kVariantGeneric; }

bool fused_layout_ok(const dhk::Plan& P, int dtype) {
    const int esz = dtype == DH_DTYPE_U16 ? 2 : 4;
    // tensor-copy rule: a 16-byte row pitch; the 256 x 256 kernel stages uint16 frames only
    if (use_fused256(P) && dtype != DH_DTYPE_U16) return false;
    return ((size_t)P.width * esz) % 16 == 0;
}

bool fused_frames_ok(const dhk::Plan& P, const void* frames, int dtype) {
    // tensor-copy rule: a 16-byte aligned base
    return ((uintptr_t)frames % 16 == 0) && fused_layout_ok(P, dtype);
}

int launch_fused_path(Handle* H, const dhk::Plan& P, const void* frames, int dtype, int batch, void* fields,
                      void* coefs, cudaStream_t st, dhk::StageTimer* tm) {
    if (use_fused256(P)) return launch_fused256(H, P, frames, dtype, batch, fields, coefs, st, tm);
    const int v = resolve_variant(H, P, true);
    if (v == kVariantFusedPruned) return launch_fused_pr(H, P, frames, dtype, batch, fields, coefs, st, tm);
    if (v == kVariantFusedGroups) return launch_fused_g(H, P, frames, dtype, batch, fields, coefs, st, tm);
    return launch_fused(H, P, frames, dtype, batch, 0, batch, dhk::kModeFull, nullptr, nullptr, fields, coefs, st, tm);
}

}  // namespace dh
