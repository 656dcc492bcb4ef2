// batched.cu -- builds of many meshes (placeholder: one launch per mesh).
#include "mesh.cuh"
#include "numeric.cuh"

namespace fem {
fem_status launch_batched(const fem_mesh *ms, int n, bool mixed, const void *const *X, fem_dtype xd,
                          const void *const *c, fem_dtype cd, void *const *vals, cudaStream_t s) {
    for (int i = 0; i < n; ++i) {
        fem_status st = fem_build_K(ms[i], mixed ? FEM_MIXED : FEM_FP64, X[i], xd, c[i], cd, vals[i], s);
        if (st != FEM_OK) return st;
    }
    return FEM_OK;
}
}  // namespace fem
