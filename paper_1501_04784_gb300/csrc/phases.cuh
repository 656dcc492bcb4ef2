// phases.cuh -- device helpers shared by the patch kernels (scalar and vector
// operators): closure-local node loads, the bounds checks of the debug build,
// and the colour phases on a ring of mbarriers.
#pragma once

#include "numeric.cuh"

namespace fem {

template <int NPE>
__device__ __forceinline__ void load_lnodes(const uint16_t *__restrict__ L, int64_t i, uint16_t (&ln)[NPE]) {
    if constexpr (NPE == 8) {
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(L + i * 8));
        ln[0] = v.x & 0xffff; ln[1] = v.x >> 16; ln[2] = v.y & 0xffff; ln[3] = v.y >> 16;
        ln[4] = v.z & 0xffff; ln[5] = v.z >> 16; ln[6] = v.w & 0xffff; ln[7] = v.w >> 16;
    } else {
        const uint2 v = __ldg(reinterpret_cast<const uint2 *>(L + i * 4));
        ln[0] = v.x & 0xffff; ln[1] = v.x >> 16; ln[2] = v.y & 0xffff; ln[3] = v.y >> 16;
    }
}

// Bounds-check build (-DFEM_DEBUG_BOUNDS, a stand-in for a memory checker): every
// index that comes from plan data is tested against its array before the access;
// a bad one sets STATUS_BOUNDS in the status word (fem_sync: FEM_ERR_INDEX) and
// the access is skipped.  In the normal build the tests compile away.
#ifdef FEM_DEBUG_BOUNDS
#define FEM_IN_BOUNDS(cond, status) ((cond) ? true : (atomicOr((status), STATUS_BOUNDS), false))
#else
#define FEM_IN_BOUNDS(cond, status) true
#endif

// ------------------------------------------------------------ colour phases
// The colour phases of a block are ordered by a ring of PHASE_RING mbarriers
// instead of block-wide barriers.  Phases are numbered g = 0, 1, ... over the
// block's whole run; every warp arrives once at each phase (barrier g mod
// PHASE_RING, count = warps).  A warp with elements in phase g first waits for
// phase g - 1 to complete; as every warp arrives at g - 1 only after its own
// scatters of that phase and its arrival at g - 2, completion of g - 1 means all
// scatters of phases < g are done, so each accumulator still receives its
// contributions in colour order.  A warp with nothing to add in a phase only
// arrives and may run ahead to integrate its next element, at most PHASE_RING - 1
// phases ahead (before arriving at g it waits for g - PHASE_RING, the previous
// use of that barrier).  The warp at the lowest phase waits only on phases every
// warp has passed, so the waits always end; they are bounded all the same.
static constexpr int PHASE_RING = 8;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void phase_init(uint64_t *mb) {
    if (threadIdx.x == 0)
        for (int k = 0; k < PHASE_RING; ++k)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mb + k)), "r"((int)(blockDim.x >> 5))
                         : "memory");
    __syncthreads();
}

// Waits until phase p has completed; after wc.spins polls it records the
// failure and returns (the kernel then finishes with undefined values).
__device__ __forceinline__ void phase_wait(uint64_t *mb, uint32_t p, const WaitCtl &wc) {
    const uint32_t a = smem_u32(mb + (p % PHASE_RING)), parity = (p / PHASE_RING) & 1u;
    for (int it = 0; it < wc.spins; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred P;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, P;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return;
    }
    if ((threadIdx.x & 31) == 0) atomicOr(wc.status, STATUS_TIMEOUT);
}

__device__ __forceinline__ void phase_arrive(uint64_t *mb, uint32_t p) {
    asm volatile(
        "{\n\t.reg .b64 st;\n\t"
        "mbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(mb + (p % PHASE_RING)))
        : "memory");
}

}  // namespace fem
