// vof_curvature_bwd.cu -- vector-Jacobian product of the curvature step with
// respect to the fill field (placeholder until the adjoint kernel lands).
#include "host_common.h"

extern "C" size_t plic_curv_bwd_workspace_bytes(int64_t cells, int64_t n_iface) {
    if (cells < 0 || n_iface < 0) return 0;
    const size_t a = ((size_t)cells * sizeof(int32_t) + 255) / 256 * 256;
    const size_t b = ((size_t)n_iface * 27 * sizeof(float) + 255) / 256 * 256;
    return a + b;
}

extern "C" plic_status vof_curvature_backward(const float*, int, int, int, const int32_t*, int64_t,
                                              const int64_t*, const float*, float*, plic_method,
                                              uint32_t, void*, size_t, void*) {
    return PLIC_ERR_UNSUPPORTED;
}
