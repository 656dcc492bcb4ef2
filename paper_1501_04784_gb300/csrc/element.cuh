// element.cuh -- per-element arithmetic of the integration step (Eqs. 7-9) for
// the 8-node trilinear brick (2x2x2 Gauss) and the 4-node linear tetrahedron
// (exact 1-point rule), in FP32 or FP64.
//
// Formulation.  With J_q the Jacobian at Gauss point q (rows d x / d xi_i) and
// B_q = J_q^{-1} dN_q (Section 3), the element matrix of Eq. 9 is
//     k_ab = c * sum_q  dN_q,a^T  M_q  dN_q,b,
//     M_q  = w_q |det J_q| J_q^{-T} J_q^{-1} = w_q cof(J_q) cof(J_q)^T / |det J_q|,
// where the rows of cof(J) are cross products of the rows of J.  Nothing is
// dropped or approximated: this is Eq. 9 with the inverse written as
// adj(J) / det J.  For the brick the natural derivatives are tensor products of
// the 1D hat functions, so the map from the 8 x 6 values of M_q to the 36
// packed entries factorises along the three axes (sum factorisation): about
// 1.2 kflop per element instead of about 3.8 kflop for forming B and B^T B
// point by point.  J_q itself is a bilinear interpolation of the 4 element edges
// along each axis, formed from coordinate differences so that FP32 keeps its
// accuracy relative to the element size.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fem {

// ----------------------------------------------------------------- brick layout
// Node a of the brick has axis bits (a1, a2, a3) in {0,1}^3 (xi = 2*bit - 1):
// nodes 0-3 on t = -1 counter-clockwise from (-1,-1,-1), nodes 4-7 on t = +1.
__host__ __device__ constexpr int hb1(int a) { return (a == 1 || a == 2 || a == 5 || a == 6) ? 1 : 0; }
__host__ __device__ constexpr int hb2(int a) { return (a == 2 || a == 3 || a == 6 || a == 7) ? 1 : 0; }
__host__ __device__ constexpr int hb3(int a) { return a >= 4 ? 1 : 0; }
__host__ __device__ constexpr int hnode(int b1, int b2, int b3) {
    return b3 * 4 + (b2 ? (b1 ? 2 : 3) : (b1 ? 1 : 0));
}
// class of a pair of bits: 0 = (0,0), 1 = (1,1), 2 = mixed
__host__ __device__ constexpr int hcls(int x, int y) { return x == y ? x : 2; }
__host__ __device__ constexpr int hsig(int x) { return x ? 1 : -1; }

// 1D two-point Gauss rule on [-1, 1]: points -g, +g (g = 1/sqrt(3)), weights 1.
// phi_i(x_j) of the linear hats phi_0 = (1 - x)/2, phi_1 = (1 + x)/2 is GP if
// i == j else GQ.  Products: GP^2 = 1/3 + g/2, GQ^2 = 1/3 - g/2, GP GQ = 1/6.
#define FEM_GP 0.78867513459481288225
#define FEM_GQ 0.21132486540518711775
#define FEM_GPP 0.62200846792814621559
#define FEM_GQQ 0.04465819873852045108
#define FEM_GPQ 0.16666666666666666667

template <typename T>
struct Vec3 {
    T x, y, z;
};
template <typename T>
__device__ __forceinline__ Vec3<T> cross3(const Vec3<T> &a, const Vec3<T> &b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
template <typename T>
__device__ __forceinline__ T dot3(const Vec3<T> &a, const Vec3<T> &b) {
    return a.x * b.x + a.y * b.y + a.z * b.z;
}
// Reciprocals.  FP32: the hardware approximation (rcp.approx) refined by one
// Newton-Raphson step r' = r + r (1 - x r), about 1 ulp, FP32 pipe only.  (The
// correctly rounded FP32 reciprocal and any conversion to double use the FP64
// pipe, which on this part runs at 1/64 of the FP32 rate.)  FP64: the correctly
// rounded double reciprocal.
__device__ __forceinline__ float rcp_rn(float x) {
    float r;
    asm("rcp.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    const float e = fmaf(-x, r, 1.0f);
    return fmaf(r, e, r);
}
__device__ __forceinline__ double rcp_rn(double x) { return __drcp_rn(x); }

// a*b - c*d with a single rounding error (Kahan's FMA-based 2x2 determinant):
// w = c*d is rounded, its rounding error is recovered exactly by an FMA.
__device__ __forceinline__ float det2(float a, float b, float c, float d) {
    const float w = __fmul_rn(c, d);
    const float err = __fmaf_rn(-c, d, w);
    const float f = __fmaf_rn(a, b, -w);
    return __fadd_rn(f, err);
}
__device__ __forceinline__ Vec3<float> cross3_accurate(const Vec3<float> &a, const Vec3<float> &b) {
    return {det2(a.y, b.z, a.z, b.y), det2(a.z, b.x, a.x, b.z), det2(a.x, b.y, a.y, b.x)};
}

// Error-free transformations: Knuth's TwoSum (a + b = s + e exactly) and the FMA
// form of Dekker's product (a * b = p + e exactly).  Written with the _rn
// intrinsics, which the compiler never contracts into FMAs: a contraction of
// p = a * b into a later sum would break the exactness, and could differ between
// kernels that inline the same code.
__device__ __forceinline__ void two_sum_f(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void two_prod_f(float a, float b, float &p, float &e) {
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

// x - y split into a float pair (h, l) with h + l == x - y: exactly for float
// inputs (TwoSum), to ~2^-48 relative for double inputs.
__device__ __forceinline__ void diff_ds(float x, float y, float &h, float &l) { two_sum_f(x, -y, h, l); }
__device__ __forceinline__ void diff_ds(double x, double y, float &h, float &l) {
    const double d = x - y;
    h = (float)d;
    l = (float)(d - (double)h);
}

// Jacobian determinant of a tetrahedron, det [x1 - x0; x2 - x0; x3 - x0], in
// double-single arithmetic: the edge vectors are formed exactly as float pairs,
// each product of pairs is split exactly (the FMA form of Dekker's product) with
// its cross terms added, each 2x2 minor and the final dot product are summed with
// TwoSum.  The result, rounded once to float, is accurate to a few units of
// 2^-46 times the sum of the magnitudes of the determinant's terms: what an FP64
// evaluation from the same coordinates gives a float result, in FP32 arithmetic.
template <typename S>
__device__ __forceinline__ float det3_ds(const S (*xc)[3]) {
    float h[3][3], l[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k) diff_ds(xc[i + 1][k], xc[0][k], h[i][k], l[i][k]);
    // product of pairs (ah + al)(bh + bl) as (p, e), dropping al * bl
    auto mul = [](float ah, float al, float bh, float bl, float &p, float &e) {
        two_prod_f(ah, bh, p, e);
        e = fmaf(ah, bl, fmaf(al, bh, e));
    };
    // minors of rows 1, 2 (the cofactors of row 0) as unevaluated pairs (s, t)
    float s[3], t[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int u = (k + 1) % 3, v = (k + 2) % 3;
        float p, ep, q, eq, es;
        mul(h[1][u], l[1][u], h[2][v], l[2][v], p, ep);
        mul(h[1][v], l[1][v], h[2][u], l[2][u], q, eq);
        two_sum_f(p, -q, s[k], es);
        t[k] = es + (ep - eq);
    }
    float P[3], E[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        two_prod_f(h[0][k], s[k], P[k], E[k]);
        E[k] = fmaf(h[0][k], t[k], fmaf(l[0][k], s[k], E[k]));
    }
    float a, e1, b, e2;
    two_sum_f(P[0], P[1], a, e1);
    two_sum_f(a, P[2], b, e2);
    return b + ((e1 + e2) + (E[0] + E[1] + E[2]));
}

template <typename T>
__device__ __forceinline__ Vec3<T> lerp2(T wa, const Vec3<T> &a, T wb, const Vec3<T> &b) {
    return {wa * a.x + wb * b.x, wa * a.y + wb * b.y, wa * a.z + wb * b.z};
}

// The two Gauss-point values (P a + Q b, Q a + P b) of the linear hats through
// a and b.  P + Q = 1, so they are b + P (a - b) and a - P (a - b): one
// subtraction and two explicit FMAs instead of two products and two FMAs.
template <typename T>
__device__ __forceinline__ void hat_pair(T a, T b, T &o0, T &o1) {
    const T d = a - b;
    o0 = fma(T(FEM_GP), d, b);
    o1 = fma(-T(FEM_GP), d, a);
}
template <typename T>
__device__ __forceinline__ void hat_pair(const Vec3<T> &a, const Vec3<T> &b, Vec3<T> &o0, Vec3<T> &o1) {
    hat_pair(a.x, b.x, o0.x, o1.x);
    hat_pair(a.y, b.y, o0.y, o1.y);
    hat_pair(a.z, b.z, o0.z, o1.z);
}

// Edge vectors of a brick along each axis, e[axis][i][j], the two other axes'
// bits (i, j) in increasing axis order.  xc[a] = coordinates of node a (input
// precision S); the differences are formed in S and rounded once to T.
template <typename T, typename S>
__device__ __forceinline__ void brick_edges(const S (*xc)[3], Vec3<T> (&e)[3][2][2]) {
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int r0 = hnode(0, i, j), r1 = hnode(1, i, j);
            const int s0 = hnode(i, 0, j), s1 = hnode(i, 1, j);
            const int t0 = hnode(i, j, 0), t1 = hnode(i, j, 1);
            e[0][i][j] = {T(xc[r1][0] - xc[r0][0]), T(xc[r1][1] - xc[r0][1]), T(xc[r1][2] - xc[r0][2])};
            e[1][i][j] = {T(xc[s1][0] - xc[s0][0]), T(xc[s1][1] - xc[s0][1]), T(xc[s1][2] - xc[s0][2])};
            e[2][i][j] = {T(xc[t1][0] - xc[t0][0]), T(xc[t1][1] - xc[t0][1]), T(xc[t1][2] - xc[t0][2])};
        }
}

// Jacobian rows (times 2) at the Gauss points: row[axis][u][v] with (u, v) the
// Gauss indices of the two other axes.  row = sum_ij phi_i(u) phi_j(v) e[i][j].
template <typename T>
__device__ __forceinline__ void brick_jrows(const Vec3<T> (&e)[3][2][2], Vec3<T> (&row)[3][2][2]) {
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        Vec3<T> m[2][2];  // m[i][v] = interpolation along the last axis
#pragma unroll
        for (int i = 0; i < 2; ++i) hat_pair(e[ax][i][0], e[ax][i][1], m[i][0], m[i][1]);
#pragma unroll
        for (int v = 0; v < 2; ++v) hat_pair(m[0][v], m[1][v], row[ax][0][v], row[ax][1][v]);
    }
}

// M_q (times 2, see brick_ke) for the 8 Gauss points q = 4 q1 + 2 q2 + q3, as
// (rr, ss, tt, rs, rt, st), times the factor s (the element's c / 8, applied
// once per point instead of once per packed entry); det[q] = det(2 J_q).
template <typename T>
__device__ __forceinline__ void brick_M(const Vec3<T> (&row)[3][2][2], T s, T (&M)[8][6], T (&det)[8]) {
#pragma unroll
    for (int q1 = 0; q1 < 2; ++q1)
#pragma unroll
        for (int q2 = 0; q2 < 2; ++q2)
#pragma unroll
            for (int q3 = 0; q3 < 2; ++q3) {
                const int q = 4 * q1 + 2 * q2 + q3;
                const Vec3<T> &R = row[0][q2][q3];
                const Vec3<T> &S = row[1][q1][q3];
                const Vec3<T> &U = row[2][q1][q2];
                const Vec3<T> C0 = cross3(S, U), C1 = cross3(U, R), C2 = cross3(R, S);
                const T d = dot3(R, C0);
                det[q] = d;
                const T inv = rcp_rn(d < T(0) ? -d : d) * s;
                M[q][0] = dot3(C0, C0) * inv;
                M[q][1] = dot3(C1, C1) * inv;
                M[q][2] = dot3(C2, C2) * inv;
                M[q][3] = dot3(C0, C1) * inv;
                M[q][4] = dot3(C0, C2) * inv;
                M[q][5] = dot3(C1, C2) * inv;
            }
}

// T[c][d] = sum_{u,v} A[u][v] F_c(u) F_d(v), F_0 = (PP, QQ), F_1 = (QQ, PP), F_2 = (PQ, PQ).
template <typename T>
__device__ __forceinline__ void contract_FF(const T (&A)[2][2], T (&out)[3][3]) {
    const T PP = T(FEM_GPP), QQ = T(FEM_GQQ), PQ = T(FEM_GPQ);
    T U[2][3];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        U[u][0] = PP * A[u][0] + QQ * A[u][1];
        U[u][1] = QQ * A[u][0] + PP * A[u][1];
        U[u][2] = PQ * (A[u][0] + A[u][1]);
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        out[0][d] = PP * U[0][d] + QQ * U[1][d];
        out[1][d] = QQ * U[0][d] + PP * U[1][d];
        out[2][d] = PQ * (U[0][d] + U[1][d]);
    }
}

// Contract one Gauss axis of m[8] (index 4 q1 + 2 q2 + q3) with the hats
// (kind 0: phi_x, 2 outputs) or the hat products (kind 1: F_c, 3 outputs).
// The cross terms need V[x or c][y or c][z or c] over the three axes in turn.
template <typename T, int K1, int K2, int K3>
__device__ __forceinline__ void contract_cross(const T (&m)[2][2][2], T (&V)[3][3][3]) {
    const T PP = T(FEM_GPP), QQ = T(FEM_GQQ), PQ = T(FEM_GPQ);
    constexpr int N1 = K1 ? 3 : 2, N2 = K2 ? 3 : 2, N3 = K3 ? 3 : 2;
    T W[2][2][3];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const T m0 = m[a][b][0], m1 = m[a][b][1];
            if (K3) {
                W[a][b][0] = PP * m0 + QQ * m1;
                W[a][b][1] = QQ * m0 + PP * m1;
                W[a][b][2] = PQ * (m0 + m1);
            } else {
                hat_pair(m0, m1, W[a][b][0], W[a][b][1]);
            }
        }
    T Y[2][3][3];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int k = 0; k < N3; ++k) {
            const T w0 = W[a][0][k], w1 = W[a][1][k];
            if (K2) {
                Y[a][0][k] = PP * w0 + QQ * w1;
                Y[a][1][k] = QQ * w0 + PP * w1;
                Y[a][2][k] = PQ * (w0 + w1);
            } else {
                hat_pair(w0, w1, Y[a][0][k], Y[a][1][k]);
            }
        }
#pragma unroll
    for (int j = 0; j < N2; ++j)
#pragma unroll
        for (int k = 0; k < N3; ++k) {
            const T y0 = Y[0][j][k], y1 = Y[1][j][k];
            if (K1) {
                V[0][j][k] = PP * y0 + QQ * y1;
                V[1][j][k] = QQ * y0 + PP * y1;
                V[2][j][k] = PQ * (y0 + y1);
            } else {
                hat_pair(y0, y1, V[0][j][k], V[1][j][k]);
            }
        }
    (void)N1;
}

// Packed lower k_e (36 entries, p = a(a+1)/2 + b) from the M_q of brick_M.
// With J~ = 2J and dN~ = 2 dN (signs instead of +-1/2), M = M~/2 and
// k_ab = (c / 8) sum_q dN~_a^T M~_q dN~_b; the factor c / 8 comes in M (brick_M).
template <typename T>
__device__ __forceinline__ void brick_contract(const T (&M)[8][6], T (&k)[36]) {
    T Arr[2][2], Ass[2][2], Att[2][2];
    T mrs[2][2][2], mrt[2][2][2], mst[2][2][2];
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int v = 0; v < 2; ++v) {
            Arr[u][v] = M[0 + 2 * u + v][0] + M[4 + 2 * u + v][0];      // sum over q1
            Ass[u][v] = M[4 * u + 0 + v][1] + M[4 * u + 2 + v][1];      // sum over q2
            Att[u][v] = M[4 * u + 2 * v + 0][2] + M[4 * u + 2 * v + 1][2];  // sum over q3
        }
#pragma unroll
    for (int q1 = 0; q1 < 2; ++q1)
#pragma unroll
        for (int q2 = 0; q2 < 2; ++q2)
#pragma unroll
            for (int q3 = 0; q3 < 2; ++q3) {
                const int q = 4 * q1 + 2 * q2 + q3;
                mrs[q1][q2][q3] = M[q][3];
                mrt[q1][q2][q3] = M[q][4];
                mst[q1][q2][q3] = M[q][5];
            }
    T Trr[3][3], Tss[3][3], Ttt[3][3];
    contract_FF(Arr, Trr);  // [c2][c3]
    contract_FF(Ass, Tss);  // [c1][c3]
    contract_FF(Att, Ttt);  // [c1][c2]
    T Vrs[3][3][3], Vrt[3][3][3], Vst[3][3][3];
    contract_cross<T, 0, 0, 1>(mrs, Vrs);  // [x][y][c3]
    contract_cross<T, 0, 1, 0>(mrt, Vrt);  // [x][c2][z]
    contract_cross<T, 1, 0, 0>(mst, Vst);  // [c1][y][z]
#pragma unroll
    for (int a = 0; a < 8; ++a) {
#pragma unroll
        for (int b = 0; b <= a; ++b) {
            const int a1 = hb1(a), a2 = hb2(a), a3 = hb3(a);
            const int b1 = hb1(b), b2 = hb2(b), b3 = hb3(b);
            const int c1 = hcls(a1, b1), c2 = hcls(a2, b2), c3 = hcls(a3, b3);
            T v = T(hsig(a1) * hsig(b1)) * Trr[c2][c3];
            v += T(hsig(a2) * hsig(b2)) * Tss[c1][c3];
            v += T(hsig(a3) * hsig(b3)) * Ttt[c1][c2];
            v += T(hsig(a1) * hsig(b2)) * Vrs[b1][a2][c3];
            v += T(hsig(a2) * hsig(b1)) * Vrs[a1][b2][c3];
            v += T(hsig(a1) * hsig(b3)) * Vrt[b1][c2][a3];
            v += T(hsig(a3) * hsig(b1)) * Vrt[a1][c2][b3];
            v += T(hsig(a2) * hsig(b3)) * Vst[c1][b2][a3];
            v += T(hsig(a3) * hsig(b2)) * Vst[c1][a2][b3];
            k[a * (a + 1) / 2 + b] = v;
        }
    }
}

// Full brick element: packed k_e in precision T from node coordinates in S.
template <typename T, typename S>
__device__ __forceinline__ void brick_ke(const S (*xc)[3], T c, T (&k)[36]) {
    Vec3<T> e[3][2][2];
    brick_edges<T, S>(xc, e);
    Vec3<T> row[3][2][2];
    brick_jrows(e, row);
    T M[8][6], det[8];
    brick_M(row, c * T(0.125), M, det);
    brick_contract(M, k);
}

// Mixed precision brick: FP32 throughout, except that an element whose ratio
// max_q det J / min_q det J exceeds `thr` (or with a det J <= 0) recomputes its
// Jacobians, determinants and M_q in FP64 from the coordinate differences.
// Returns true when the FP64 path was taken.
template <typename S>
__device__ __forceinline__ bool brick_ke_mixed(const S (*xc)[3], float c, float thr, float (&k)[36]) {
    Vec3<float> e[3][2][2];
    brick_edges<float, S>(xc, e);
    Vec3<float> row[3][2][2];
    brick_jrows(e, row);
    float M[8][6], det[8];
    brick_M(row, c * 0.125f, M, det);
    float dmin = det[0], dmax = det[0];
#pragma unroll
    for (int q = 1; q < 8; ++q) {
        dmin = fminf(dmin, det[q]);
        dmax = fmaxf(dmax, det[q]);
    }
    const bool flagged = !(dmin > 0.f) || dmax > thr * dmin;
    if (flagged) {
        Vec3<double> ed[3][2][2];
        brick_edges<double, S>(xc, ed);
        Vec3<double> rowd[3][2][2];
        brick_jrows(ed, rowd);
        double Md[8][6], detd[8];
        brick_M(rowd, (double)c * 0.125, Md, detd);
#pragma unroll
        for (int q = 0; q < 8; ++q)
#pragma unroll
            for (int i = 0; i < 6; ++i) M[q][i] = (float)Md[q][i];
    }
    brick_contract(M, k);
    return flagged;
}

// ----------------------------------------------------------- brick mass matrix
// M_ab = c integral N_a N_b (the mass operator of Section 5's generalisation) by
// the same 2x2x2 rule: M_ab = c sum_q |det J_q| N_a(q) N_b(q).  N_a(q) is a product
// of 1D hats, so the sum factorises like the stiffness matrix: with
// D[q1][q2][q3] = |det J_q| and V = D contracted with the hat products F_c on every
// axis, M_ab = c V[cls(a1,b1)][cls(a2,b2)][cls(a3,b3)].  det(2 J_q) = 8 det J_q.
template <typename T>
__device__ __forceinline__ void brick_dets(const Vec3<T> (&row)[3][2][2], T (&det)[8]) {
#pragma unroll
    for (int q1 = 0; q1 < 2; ++q1)
#pragma unroll
        for (int q2 = 0; q2 < 2; ++q2)
#pragma unroll
            for (int q3 = 0; q3 < 2; ++q3)
                det[4 * q1 + 2 * q2 + q3] = dot3(row[0][q2][q3], cross3(row[1][q1][q3], row[2][q1][q2]));
}

template <typename T>
__device__ __forceinline__ void brick_mass_from_dets(const T (&det)[8], T c, T (&m)[36]) {
    T D[2][2][2];
#pragma unroll
    for (int q = 0; q < 8; ++q) D[q >> 2][(q >> 1) & 1][q & 1] = det[q] < T(0) ? -det[q] : det[q];
    T V[3][3][3];
    contract_cross<T, 1, 1, 1>(D, V);
    const T s = c * T(0.125);
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b <= a; ++b)
            m[a * (a + 1) / 2 + b] = s * V[hcls(hb1(a), hb1(b))][hcls(hb2(a), hb2(b))][hcls(hb3(a), hb3(b))];
}

template <typename T, typename S>
__device__ __forceinline__ void brick_me(const S (*xc)[3], T c, T (&m)[36]) {
    Vec3<T> e[3][2][2];
    brick_edges<T, S>(xc, e);
    Vec3<T> row[3][2][2];
    brick_jrows(e, row);
    T det[8];
    brick_dets(row, det);
    brick_mass_from_dets(det, c, m);
}

// Brick determinants |det(2 J_q)| at the 8 Gauss points in precision T; with
// `mixed`, FP32 unless max_q det J / min_q det J exceeds thr (or some det J <= 0),
// then from FP64.  Returns true when FP64 was used.
template <typename T, typename S>
__device__ __forceinline__ bool brick_gauss_dets(const S (*xc)[3], float thr, bool mixed, T (&det)[8]) {
    Vec3<T> e[3][2][2];
    brick_edges<T, S>(xc, e);
    Vec3<T> row[3][2][2];
    brick_jrows(e, row);
    brick_dets(row, det);
    if (!mixed) return false;
    T dmin = det[0], dmax = det[0];
#pragma unroll
    for (int q = 1; q < 8; ++q) {
        dmin = det[q] < dmin ? det[q] : dmin;
        dmax = det[q] > dmax ? det[q] : dmax;
    }
    const bool flagged = !(dmin > T(0)) || dmax > T(thr) * dmin;
    if (flagged) {
        Vec3<double> ed[3][2][2];
        brick_edges<double, S>(xc, ed);
        Vec3<double> rowd[3][2][2];
        brick_jrows(ed, rowd);
        double detd[8];
        brick_dets(rowd, detd);
#pragma unroll
        for (int q = 0; q < 8; ++q) det[q] = (T)detd[q];
    }
    return flagged;
}

// Brick load vector f_a = s integral N_a = (s / 8) sum_q |det(2 J_q)| N_a(q): the
// determinants contracted with the single hats on every axis.
template <typename T>
__device__ __forceinline__ void brick_load_from_dets(const T (&det)[8], T s, T (&f)[8]) {
    T D[2][2][2];
#pragma unroll
    for (int q = 0; q < 8; ++q) D[q >> 2][(q >> 1) & 1][q & 1] = det[q] < T(0) ? -det[q] : det[q];
    T V[3][3][3];
    contract_cross<T, 0, 0, 0>(D, V);
#pragma unroll
    for (int a = 0; a < 8; ++a) f[a] = s * T(0.125) * V[hb1(a)][hb2(a)][hb3(a)];
}

// Mixed precision: FP32, except that an element whose max_q det J / min_q det J
// exceeds `thr` (or with a det J <= 0) takes its determinants from FP64.
template <typename S>
__device__ __forceinline__ bool brick_me_mixed(const S (*xc)[3], float c, float thr, float (&m)[36]) {
    Vec3<float> e[3][2][2];
    brick_edges<float, S>(xc, e);
    Vec3<float> row[3][2][2];
    brick_jrows(e, row);
    float det[8];
    brick_dets(row, det);
    float dmin = det[0], dmax = det[0];
#pragma unroll
    for (int q = 1; q < 8; ++q) {
        dmin = fminf(dmin, det[q]);
        dmax = fmaxf(dmax, det[q]);
    }
    const bool flagged = !(dmin > 0.f) || dmax > thr * dmin;
    if (flagged) {
        Vec3<double> ed[3][2][2];
        brick_edges<double, S>(xc, ed);
        Vec3<double> rowd[3][2][2];
        brick_jrows(ed, rowd);
        double detd[8];
        brick_dets(rowd, detd);
#pragma unroll
        for (int q = 0; q < 8; ++q) det[q] = (float)detd[q];
    }
    brick_mass_from_dets(det, c, m);
    return flagged;
}

// ---------------------------------------------------------------- tetrahedron
// Rows of J are the edge vectors x_i - x_0 (i = 1..3).  The gradient of the
// barycentric function lambda_a is F_a / det J, where F_a is twice the area
// vector of the face opposite node a: F_1, F_2, F_3 are the cofactor rows
// (R1 x R2, R2 x R0, R0 x R1) and F_0 = (x3 - x1) x (x2 - x1) = -(F_1 + F_2 + F_3).
// Hence k_ab = c |det J|/6 grad(lambda_a).grad(lambda_b) = c F_a.F_b / (6 |det J|).
// F_0 is formed from its own coordinate differences rather than as -(F_1+F_2+F_3),
// so no entry is a cancelling sum (the FP32 error stays relative to the element).
template <typename T>
struct TetGeom {
    Vec3<T> R0, R1, R2, D1, D2;  // x1-x0, x2-x0, x3-x0, x2-x1, x3-x1
};

template <typename T, typename S>
__device__ __forceinline__ void tet_geom(const S (*xc)[3], TetGeom<T> &g) {
    auto d = [&](int i, int j) {
        return Vec3<T>{T(xc[i][0] - xc[j][0]), T(xc[i][1] - xc[j][1]), T(xc[i][2] - xc[j][2])};
    };
    g.R0 = d(1, 0);
    g.R1 = d(2, 0);
    g.R2 = d(3, 0);
    g.D1 = d(2, 1);
    g.D2 = d(3, 1);
}

template <typename T>
__device__ __forceinline__ void tet_faces(const TetGeom<T> &g, Vec3<T> (&F)[4], T &det) {
    F[1] = cross3(g.R1, g.R2);
    F[2] = cross3(g.R2, g.R0);
    F[3] = cross3(g.R0, g.R1);
    F[0] = cross3(g.D2, g.D1);
    det = dot3(g.R0, F[1]);
}

template <typename T>
__device__ __forceinline__ void tet_from_faces(const Vec3<T> (&F)[4], T det, T c, T (&k)[10]) {
    const T s = c * rcp_rn(T(6) * (det < T(0) ? -det : det));
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b <= a; ++b) k[a * (a + 1) / 2 + b] = dot3(F[a], F[b]) * s;
}

template <typename T, typename S>
__device__ __forceinline__ void tet_ke(const S (*xc)[3], T c, T (&k)[10]) {
    TetGeom<T> g;
    tet_geom<T, S>(xc, g);
    Vec3<T> F[4];
    T det;
    tet_faces(g, F, det);
    tet_from_faces(F, det, c, k);
}

// Mixed precision tetrahedron: the aspect ratio (longest edge over shortest
// altitude = L_max |F|_max / |det J|) is evaluated in FP32; above `thr` the
// face vectors are recomputed with one rounding each and the determinant to
// FP64 accuracy -- in double-single FP32 arithmetic (det3_ds) by default, or in
// FP64 arithmetic when fp64_det is set -- and rounded once.  Returns true when
// the accurate path was taken.
template <typename S>
__device__ __forceinline__ bool tet_geometry_mixed(const S (*xc)[3], float thr, bool fp64_det, Vec3<float> (&F)[4],
                                                   float &det) {
    TetGeom<float> g;
    tet_geom<float, S>(xc, g);
    tet_faces(g, F, det);
    const Vec3<float> E5 = {g.R2.x - g.R1.x, g.R2.y - g.R1.y, g.R2.z - g.R1.z};
    const float L2 = fmaxf(fmaxf(fmaxf(dot3(g.R0, g.R0), dot3(g.R1, g.R1)), fmaxf(dot3(g.R2, g.R2), dot3(g.D1, g.D1))),
                           fmaxf(dot3(g.D2, g.D2), dot3(E5, E5)));
    const float A2 = fmaxf(fmaxf(dot3(F[0], F[0]), dot3(F[1], F[1])), fmaxf(dot3(F[2], F[2]), dot3(F[3], F[3])));
    const bool flagged = !(L2 * A2 <= thr * thr * det * det);
    if (flagged) {
        // Distorted: cofactors (face vectors) with one rounding each, and the
        // Jacobian determinant to FP64 accuracy.  The double-single form keeps
        // the work off the FP64 pipe (1/64 of the FP32 rate on this part), where
        // a warp with one distorted lane would otherwise stall all 32.
        F[1] = cross3_accurate(g.R1, g.R2);
        F[2] = cross3_accurate(g.R2, g.R0);
        F[3] = cross3_accurate(g.R0, g.R1);
        F[0] = cross3_accurate(g.D2, g.D1);
        if (fp64_det) {
            // FP64 from the coordinates: the edge vectors are exact in double
            // (differences of floats), the products of two of them too
            double r[3][3];
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int k = 0; k < 3; ++k) r[i][k] = (double)xc[i + 1][k] - (double)xc[0][k];
            const double m0 = fma(r[1][1], r[2][2], -(r[1][2] * r[2][1]));
            const double m1 = fma(r[1][2], r[2][0], -(r[1][0] * r[2][2]));
            const double m2 = fma(r[1][0], r[2][1], -(r[1][1] * r[2][0]));
            det = (float)fma(r[0][0], m0, fma(r[0][1], m1, r[0][2] * m2));
        } else {
            det = det3_ds<S>(xc);
        }
    }
    return flagged;
}

template <typename S>
__device__ __forceinline__ bool tet_ke_mixed(const S (*xc)[3], float c, float thr, bool fp64_det, float (&k)[10]) {
    Vec3<float> F[4];
    float det;
    const bool flagged = tet_geometry_mixed<S>(xc, thr, fp64_det, F, det);
    tet_from_faces(F, det, c, k);
    return flagged;
}

// ------------------------------------------------------------ tet mass matrix
// M_ab = c integral lambda_a lambda_b = c |T| (1 + delta_ab) / 20, |T| = |det J| / 6.
template <typename T>
__device__ __forceinline__ void tet_mass_from_det(T det, T c, T (&m)[10]) {
    const T s = c * (det < T(0) ? -det : det) * T(1.0 / 120.0);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b <= a; ++b) m[a * (a + 1) / 2 + b] = a == b ? s + s : s;
}

template <typename T, typename S>
__device__ __forceinline__ void tet_me(const S (*xc)[3], T c, T (&m)[10]) {
    TetGeom<T> g;
    tet_geom<T, S>(xc, g);
    Vec3<T> F[4];
    T det;
    tet_faces(g, F, det);
    tet_mass_from_det(det, c, m);
}

// Mixed precision: the same indicator and FP64-accurate determinant as k_e.
template <typename S>
__device__ __forceinline__ bool tet_me_mixed(const S (*xc)[3], float c, float thr, bool fp64_det, float (&m)[10]) {
    Vec3<float> F[4];
    float det;
    const bool flagged = tet_geometry_mixed<S>(xc, thr, fp64_det, F, det);
    tet_mass_from_det(det, c, m);
    return flagged;
}

}  // namespace fem
