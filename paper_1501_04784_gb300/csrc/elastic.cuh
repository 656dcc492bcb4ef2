// elastic.cuh -- element arithmetic of linear isotropic elasticity, the vector
// problem with three degrees of freedom per node (Algorithm 1's DOFxn = 3; the
// operator itself is the textbook one, the paper builds only the scalar case).
//
// Formulation.  With G_a = grad_x N_a at a quadrature point and Lame parameters
// (lambda, mu) of the element, the 3x3 block of nodes (a, b) of k_e is
//     K_ab = sum_q w_q |det J_q| [lambda G_a G_b^T + mu G_b G_a^T + mu (G_a.G_b) I],
// the Hessian of the strain energy lambda/2 (tr eps)^2 + mu eps:eps; entry (i, j)
// couples DOF 3a + i with DOF 3b + j.  Writing G_a = v_a / d with v_a built from
// the cofactor rows of the Jacobian (see below) and d its determinant, the
// per-point factor is s = w |det J| / d^2, so that with
//     P_ab = sum_q s_q v_a v_b^T
// the block is K_ab = lambda P_ab + mu P_ab^T + mu tr(P_ab) I.
//
// Work split.  NPE threads per element, thread a owning node a; the blocks each
// computes are listed below (elastic_nblk, blk_node), kept in registers as P_ab.
//   Brick: 8 threads per element, the circulant block set; shuffles share the
//   Gauss-point geometry and the nodes' gradient vectors.
//   Tetrahedron: 4 threads per element, the lower block row; the integrand is
//   constant and every thread forms the (cheap) geometry itself.
#pragma once

#include "element.cuh"

namespace fem {

// Bilinear interpolation of an edge family at Gauss indices (u, v) given at run
// time: sum_ij phi_i(u) phi_j(v) e[i][j] (phi_i(u) = GP if i == u else GQ).
template <typename T>
__device__ __forceinline__ Vec3<T> bilerp_rt(const Vec3<T> (&e)[2][2], int u, int v) {
    const T P = T(FEM_GP), Q = T(FEM_GQ);
    const T u0 = u ? Q : P, u1 = u ? P : Q, v0 = v ? Q : P, v1 = v ? P : Q;
    const Vec3<T> m0 = lerp2(v0, e[0][0], v1, e[0][1]);
    const Vec3<T> m1 = lerp2(v0, e[1][0], v1, e[1][1]);
    return lerp2(u0, m0, u1, m1);
}

// Hat products of node a's gradient at Gauss point q = 4 q1 + 2 q2 + q3 (compile
// time): component i of d N_a / d xi (times 2) is sigma_i h_i, h_i the product of
// the hats of the two other axes.
__host__ __device__ constexpr double hat1(int bit, int qb) { return bit == qb ? FEM_GP : FEM_GQ; }
__host__ __device__ constexpr double hgrad(int a, int q, int axis) {
    return axis == 0   ? hsig(hb1(a)) * hat1(hb2(a), (q >> 1) & 1) * hat1(hb3(a), q & 1)
           : axis == 1 ? hsig(hb2(a)) * hat1(hb1(a), q >> 2) * hat1(hb3(a), q & 1)
                       : hsig(hb3(a)) * hat1(hb1(a), q >> 2) * hat1(hb2(a), (q >> 1) & 1);
}

// Select of v[a] by a run-time index (selects, no dynamic register indexing).
template <typename T>
__device__ __forceinline__ Vec3<T> select4(const Vec3<T> (&v)[4], int a) {
    const bool s0 = a & 1, s1 = a & 2;
    auto sel = [](bool f, const Vec3<T> &x, const Vec3<T> &y) {
        return Vec3<T>{f ? y.x : x.x, f ? y.y : x.y, f ? y.z : x.z};
    };
    return sel(s1, sel(s0, v[0], v[1]), sel(s0, v[2], v[3]));
}

// K_ab from P_ab (in place): lambda P + mu P^T + mu tr(P) I.
template <typename T>
__device__ __forceinline__ void lame_block(T lam, T mu, T (&p)[9]) {
    const T tr = mu * (p[0] + p[4] + p[8]);
    T k[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) k[3 * i + j] = lam * p[3 * i + j] + mu * p[3 * j + i] + (i == j ? tr : T(0));
#pragma unroll
    for (int m = 0; m < 9; ++m) p[m] = k[m];
}

// Blocks a thread computes.  A brick thread (node a of its element, 8 threads per
// element) takes the circulant set b = (a + k) mod 8, k = 0..4: its diagonal block
// and the off-diagonal pairs at circular distance 1 to 3 from a, plus distance 4
// for a < 4.  Over the 8 threads that covers each of the 36 node pairs exactly
// once.  Every thread holds 5 blocks (the fifth idle for a >= 4), where a split
// by block rows would give thread a its a + 1 blocks (up to 8), and every
// register index stays compile-time.  A tetrahedron thread (4 per element) takes
// its lower block row b = 0..a.
template <int NPE>
__host__ __device__ constexpr int elastic_nblk() { return NPE == 8 ? 5 : 4; }
template <int NPE>
__device__ __forceinline__ int blk_node(int a, int k) { return NPE == 8 ? ((a + k) & 7) : k; }
template <int NPE>
__device__ __forceinline__ bool blk_valid(int a, int k) { return NPE == 8 ? (k < 4 || a < 4) : (k <= a); }

// Brick, thread a = lane & 7 of the 8-lane group that holds the element (all 32
// lanes of the warp must call it: it shuffles).  xc = the element's node
// coordinates (any values for an idle lane).  k[m][3i + j] = entry (3a + i, 3b + j)
// of k_e for b = blk_node(a, m).
//   Gauss point q = a: the thread forms the cofactor rows of 2 J_q and the point's
//   factor and hands them to the element's other threads by shuffles, so each
//   point's geometry is computed once per element.
//   At every point each thread forms its own node's gradient vector v_a and
//   takes its block partners' v_b from their lanes (shuffles again).
// Returns det(2 J) at the thread's own point (for the caller's degeneracy check).
template <typename T, typename S>
__device__ __forceinline__ T elastic_brick_blocks(const S (*xc)[3], T lam, T mu, T (&k)[5][9]) {
    const int lane = threadIdx.x & 31, a = lane & 7, base = lane & ~7;
    // this lane's Gauss point q = a: rows of 2 J (edge interpolations), cofactor
    // rows C_i = cross products of the other two rows, d = det(2 J)
    Vec3<T> C0, C1, C2;
    T s;
    T d;
    {
        Vec3<T> e[3][2][2];
        brick_edges<T, S>(xc, e);
        const int q1 = a >> 2, q2 = (a >> 1) & 1, q3 = a & 1;
        const Vec3<T> R = bilerp_rt(e[0], q2, q3), Sr = bilerp_rt(e[1], q1, q3), U = bilerp_rt(e[2], q1, q2);
        C0 = cross3(Sr, U);
        C1 = cross3(U, R);
        C2 = cross3(R, Sr);
        d = dot3(R, C0);
        // grad_x N = v / d with v = sum_i sigma_i h_i C_i; |det J| = |d| / 8, so
        // s = |det J| / d^2 = 1 / (8 |d|) (Gauss weights 1)
        s = rcp_rn(T(8) * (d < T(0) ? -d : d));
    }
    // node a's axis bits, its signs sigma_i and its hats at the two Gauss indices
    const int b1 = (a ^ (a >> 1)) & 1, b2 = (a >> 1) & 1, b3 = a >> 2;
    const T P = T(FEM_GP), Q = T(FEM_GQ);
    const T f1[2] = {b1 ? Q : P, b1 ? P : Q}, f2[2] = {b2 ? Q : P, b2 ? P : Q}, f3[2] = {b3 ? Q : P, b3 ? P : Q};
    const T g1 = b1 ? T(1) : T(-1), g2 = b2 ? T(1) : T(-1), g3 = b3 ? T(1) : T(-1);
    int src_b[5];
#pragma unroll
    for (int m = 0; m < 5; ++m) src_b[m] = base + ((a + m) & 7);
#pragma unroll
    for (int m = 0; m < 5; ++m)
#pragma unroll
        for (int n = 0; n < 9; ++n) k[m][n] = T(0);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int src = base + q;
        const Vec3<T> c0 = {__shfl_sync(0xffffffffu, C0.x, src), __shfl_sync(0xffffffffu, C0.y, src),
                            __shfl_sync(0xffffffffu, C0.z, src)};
        const Vec3<T> c1 = {__shfl_sync(0xffffffffu, C1.x, src), __shfl_sync(0xffffffffu, C1.y, src),
                            __shfl_sync(0xffffffffu, C1.z, src)};
        const Vec3<T> c2 = {__shfl_sync(0xffffffffu, C2.x, src), __shfl_sync(0xffffffffu, C2.y, src),
                            __shfl_sync(0xffffffffu, C2.z, src)};
        const T sq = __shfl_sync(0xffffffffu, s, src);
        const int q1 = q >> 2, q2 = (q >> 1) & 1, q3 = q & 1;  // folded by the unrolling
        const T h0 = g1 * f2[q2] * f3[q3], h1 = g2 * f1[q1] * f3[q3], h2 = g3 * f1[q1] * f2[q2];
        const Vec3<T> va = {h0 * c0.x + h1 * c1.x + h2 * c2.x, h0 * c0.y + h1 * c1.y + h2 * c2.y,
                            h0 * c0.z + h1 * c1.z + h2 * c2.z};
        const Vec3<T> w = {sq * va.x, sq * va.y, sq * va.z};
#pragma unroll
        for (int m = 0; m < 5; ++m) {
            Vec3<T> vb = va;
            if (m > 0)
                vb = {__shfl_sync(0xffffffffu, va.x, src_b[m]), __shfl_sync(0xffffffffu, va.y, src_b[m]),
                      __shfl_sync(0xffffffffu, va.z, src_b[m])};
            k[m][0] += w.x * vb.x; k[m][1] += w.x * vb.y; k[m][2] += w.x * vb.z;
            k[m][3] += w.y * vb.x; k[m][4] += w.y * vb.y; k[m][5] += w.y * vb.z;
            k[m][6] += w.z * vb.x; k[m][7] += w.z * vb.y; k[m][8] += w.z * vb.z;
        }
    }
#pragma unroll
    for (int m = 0; m < 5; ++m) lame_block(lam, mu, k[m]);
    return d;
}

// Tetrahedron, block row a (0..3).  grad lambda_b = F_b / det J (face vectors, see
// element.cuh), |T| = |det J| / 6: s = 1 / (6 |det J|).  Mixed precision takes the
// scalar operator's accurate geometry for distorted elements.  Returns det J.
template <typename T, typename S, bool MIXED>
__device__ __forceinline__ T elastic_tet_row(const S (*xc)[3], T lam, T mu, int a, float thr, bool fp64_det,
                                             T (&k)[4][9]) {
    Vec3<T> F[4];
    T det;
    if constexpr (MIXED) {
        tet_geometry_mixed<S>(xc, thr, fp64_det, F, det);
    } else {
        TetGeom<T> g;
        tet_geom<T, S>(xc, g);
        tet_faces(g, F, det);
    }
    const T s = rcp_rn(T(6) * (det < T(0) ? -det : det));
    const Vec3<T> fa = select4(F, a);
    const Vec3<T> w = {s * fa.x, s * fa.y, s * fa.z};
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        k[b][0] = w.x * F[b].x; k[b][1] = w.x * F[b].y; k[b][2] = w.x * F[b].z;
        k[b][3] = w.y * F[b].x; k[b][4] = w.y * F[b].y; k[b][5] = w.y * F[b].z;
        k[b][6] = w.z * F[b].x; k[b][7] = w.z * F[b].y; k[b][8] = w.z * F[b].z;
        lame_block(lam, mu, k[b]);
    }
    return det;
}

// Packed lower k_e over local DOFs (p = A(A+1)/2 + B, A = 3a + i, B = 3b + j,
// B <= A): the entries of block row a are the DOF rows 3a .. 3a + 2, one
// contiguous range of the packed array.
__host__ __device__ constexpr int elastic_np(int npe) { return 3 * npe * (3 * npe + 1) / 2; }

// Block (a, b) of a thread to or from the packed lower k_e: it lives in the
// packed rows of max(a, b) (as stored, transposed when a < b); a diagonal block
// keeps its lower half.
template <int NPE, typename T>
__device__ __forceinline__ void store_packed_blocks(T *out, int a, const T (&k)[elastic_nblk<NPE>()][9]) {
#pragma unroll
    for (int m = 0; m < elastic_nblk<NPE>(); ++m) {
        if (!blk_valid<NPE>(a, m)) continue;
        const int b = blk_node<NPE>(a, m), A = a > b ? a : b, B = a > b ? b : a;
        const bool tr = a < b;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const int R = 3 * A + i;
            T *row = out + R * (R + 1) / 2 + 3 * B;
#pragma unroll
            for (int j = 0; j < 3; ++j)
                if (A != B || j <= i) row[j] = tr ? k[m][3 * j + i] : k[m][3 * i + j];
        }
    }
}

template <int NPE, typename T>
__device__ __forceinline__ void load_packed_blocks(const T *in, int a, T (&k)[elastic_nblk<NPE>()][9]) {
#pragma unroll
    for (int m = 0; m < elastic_nblk<NPE>(); ++m) {
        const int b = blk_node<NPE>(a, m), A = a > b ? a : b, B = a > b ? b : a;
        const bool tr = a < b, ok = blk_valid<NPE>(a, m);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const int R = 3 * A + i;
            const T *row = in + R * (R + 1) / 2 + 3 * B;
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const T v = (ok && (A != B || j <= i)) ? __ldg(row + j) : T(0);
                if (tr) k[m][3 * j + i] = v; else k[m][3 * i + j] = v;
            }
        }
    }
}

}  // namespace fem
