// elem_ops.cuh -- device helpers shared by the numeric kernels (patch and tile
// assembly): packed-entry counts, connectivity loads, the element matrix in the
// arithmetic of the precision mode, and the error-free pair accumulation of
// FP64-accurate sums.
#pragma once

#include "element.cuh"
#include "numeric.cuh"

namespace fem {

template <int NPE>
struct ElemTraits;
template <>
struct ElemTraits<8> {
    static constexpr int NP = 36;
};
template <>
struct ElemTraits<4> {
    static constexpr int NP = 10;
};

template <int NPE>
__device__ __forceinline__ void load_ids(const int32_t *__restrict__ E, int64_t e, int32_t (&g)[NPE]) {
    if constexpr (NPE == 8) {
        const int4 *p = reinterpret_cast<const int4 *>(E + e * 8);
        const int4 a = __ldg(p), b = __ldg(p + 1);
        g[0] = a.x; g[1] = a.y; g[2] = a.z; g[3] = a.w;
        g[4] = b.x; g[5] = b.y; g[6] = b.z; g[7] = b.w;
    } else {
        const int4 a = __ldg(reinterpret_cast<const int4 *>(E + e * 4));
        g[0] = a.x; g[1] = a.y; g[2] = a.z; g[3] = a.w;
    }
}

// Element matrix in the arithmetic of the precision mode.  FP64: everything in
// double.  MIXED: float, FP64 Jacobians for distorted elements.
template <int NPE, typename AccT, typename S, bool MIXED, typename CT>
__device__ __forceinline__ bool element_matrix(const S (*xc)[3], CT ce, float thr, unsigned mode,
                                               AccT (&k)[ElemTraits<NPE>::NP]) {
    const bool fp64_det = (mode & FP64_DETS) != 0;
    if (mode & OP_MASS) {
        if constexpr (MIXED) {
            if constexpr (NPE == 8) return brick_me_mixed<S>(xc, static_cast<float>(ce), thr, k);
            else return tet_me_mixed<S>(xc, static_cast<float>(ce), thr, fp64_det, k);
        } else {
            if constexpr (NPE == 8) brick_me<double, S>(xc, static_cast<double>(ce), k);
            else tet_me<double, S>(xc, static_cast<double>(ce), k);
            return false;
        }
    }
    if constexpr (MIXED) {
        if constexpr (NPE == 8) return brick_ke_mixed<S>(xc, static_cast<float>(ce), thr, k);
        else return tet_ke_mixed<S>(xc, static_cast<float>(ce), thr, fp64_det, k);
    } else {
        if constexpr (NPE == 8) brick_ke<double, S>(xc, static_cast<double>(ce), k);
        else tet_ke<double, S>(xc, static_cast<double>(ce), k);
        return false;
    }
}

// Knuth's TwoSum: s + err == a + b exactly (round-to-nearest, no reassociation).
__device__ __forceinline__ void two_sum_acc(float2 &acc, float x) {
    const float s = acc.x + x;
    const float bp = s - acc.x;
    const float err = (acc.x - (s - bp)) + (x - bp);
    acc.x = s;
    acc.y += err;
}

// Row a of packed entry q = a(a+1)/2 + b.
__host__ __device__ constexpr int tri_row(int q) {
    int a = 0;
    while ((a + 1) * (a + 2) / 2 <= q) ++a;
    return a;
}

}  // namespace fem
