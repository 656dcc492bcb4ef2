// vjp.cu -- backward pass (placeholder).
#include "mesh.cuh"

namespace fem {
fem_status launch_vjp(fem_mesh m, bool mixed, const void *X, fem_dtype xd, const void *c, fem_dtype cd,
                      const void *G, void *dX, void *dc, cudaStream_t s) {
    set_error("fem_vjp is not built yet");
    return FEM_ERR_UNSUPPORTED;
}
}  // namespace fem
