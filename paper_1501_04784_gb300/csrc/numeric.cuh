// numeric.cuh -- launch interfaces of the numeric kernels.
#pragma once

#include "mesh.cuh"

namespace fem {

static constexpr int PATCH_MAX_THREADS = 512;

// byte offsets of the patch kernel's shared-memory arrays
struct PatchSmem {
    size_t acc, hv, xs, cown, roff, hvf, rps, gid, eid, cvs, total;
};

struct IntegrateArgs {
    int npe;
    bool mixed;
    fem_dtype xd, cd;
    const int32_t *E;
    int64_t nel;
    const void *X, *c;
    void *ke;
    float thr;
    unsigned long long *nflag;
};

struct PatchArgs {
    const Plan *plan;
    int npe;
    bool mixed, fused;
    fem_dtype xd, cd;
    const void *X, *c, *ke;
    void *vals;
    float thr;
    int64_t p0, p1;
    int threads, blocks_per_sm;
    bool fp64_sums;  // high-valence sums with FP64 adds instead of FP32 TwoSum pairs
};

fem_status launch_integrate(const IntegrateArgs &a, cudaStream_t s);
fem_status launch_patch(const PatchArgs &a, cudaStream_t s);
PatchSmem patch_smem_layout(const Plan &P, bool fused, bool mixed, size_t xsize, size_t csize);

}  // namespace fem
