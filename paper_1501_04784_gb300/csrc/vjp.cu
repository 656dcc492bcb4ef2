// vjp.cu -- backward pass of the build: vector-Jacobian product of
// L = sum over stored entries G_ij K_ij with respect to the node coordinates X
// and the coefficients c_e.
//
// Per element e, with S_ab = G at the slot of packed pair (a, b) and the
// symmetric upstream Ssym (S_aa on the diagonal, S_ab / 2 off it; each packed
// pair is counted once), L_e = c_e sum_q <M_q, H_q> where
// H_q = dN_q Ssym dN_q^T and M_q = w_q |det J_q| J_q^{-T} J_q^{-1} (Eq. 9 as in
// element.cuh).  Hence dL/dc_e = sum_q <M_q, H_q> and, with A = J^{-1},
//     dL/dJ_q = c_e (<M_q, H_q> I - 2 M_q H_q) A^T,
// (from d|det J| = |det J| tr(A dJ) and dA = -A dJ A), and because
// J = dN X_e, dL/dX_e = sum_q dN_q^T dL/dJ_q.  J, det J, A and B are recomputed
// here from X; nothing is stored by the forward pass.  The brick computes this
// gradient by reverse mode through the forward's own factorised steps
// (brick_vjp below); the tetrahedron evaluates it directly.
//
// The mass operator (M_ab = c sum_q |det J_q| N_a(q) N_b(q)) has
// L_e = c sum_q |det J_q| phi_q with phi_q = N_q^T Ssym N_q, hence dL/dc_e =
// sum_q |det J_q| phi_q and dL/dJ_q = c phi_q |det J_q| A^T (the tetrahedron:
// phi = sum_ab Ssym_ab (1 + delta_ab) / 20 over the volume |det J| / 6).
//
// Accumulation is owner-computes as in the forward kernel: the block of a patch
// visits its closure elements colour by colour and adds each element's node
// gradients into shared-memory accumulators of its owned nodes, then writes
// dX of every owned node once; dc_e is written by the patch that owns the
// element's first node.  No atomics on values; bitwise reproducible.  By default
// the pass is staged (k_vjp_elem: every element once, node gradients to library
// memory; k_vjp_gather: the colour-ordered adds); the fused kernel k_vjp
// recomputes an element in every closure that holds it and needs no memory.
#include "element.cuh"
#include "mesh.cuh"
#include "phases.cuh"

namespace fem {

// Coefficient of the 1D operator along one axis of the brick contraction:
// kind 0 = the hats phi_i at the Gauss points (2 x 2), kind 1 = the hat
// products F_i (3 x 2: F_0 = (PP, QQ), F_1 = (QQ, PP), F_2 = (PQ, PQ)).
template <typename T, int K>
__device__ __forceinline__ T axis_coef(int i, int a) {
    if (K) return i == 2 ? T(FEM_GPQ) : (i == a ? T(FEM_GPP) : T(FEM_GQQ));
    return i == a ? T(FEM_GP) : T(FEM_GQ);
}

// Adjoint of contract_FF: Abar[u][v] = sum_cd F_c(u) F_d(v) Tbar[c][d].
template <typename T>
__device__ __forceinline__ void contract_FF_adj(const T (&Tb)[3][3], T (&Ab)[2][2]) {
    T Z[3][2];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int v = 0; v < 2; ++v)
            Z[c][v] = axis_coef<T, 1>(0, v) * Tb[c][0] + axis_coef<T, 1>(1, v) * Tb[c][1] +
                      axis_coef<T, 1>(2, v) * Tb[c][2];
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int v = 0; v < 2; ++v)
            Ab[u][v] = axis_coef<T, 1>(0, u) * Z[0][v] + axis_coef<T, 1>(1, u) * Z[1][v] +
                       axis_coef<T, 1>(2, u) * Z[2][v];
}

// Adjoint of contract_cross<K1, K2, K3>: the forward applies one 1D operator per
// axis to m[2][2][2]; the adjoint applies their transposes to Vbar.
template <typename T, int K1, int K2, int K3>
__device__ __forceinline__ void contract_cross_adj(const T (&Vb)[3][3][3], T (&mb)[2][2][2]) {
    constexpr int N1 = K1 ? 3 : 2, N2 = K2 ? 3 : 2, N3 = K3 ? 3 : 2;
    T Y[2][3][3];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int j = 0; j < N2; ++j)
#pragma unroll
            for (int k = 0; k < N3; ++k) {
                T v = T(0);
#pragma unroll
                for (int i = 0; i < N1; ++i) v += axis_coef<T, K1>(i, a) * Vb[i][j][k];
                Y[a][j][k] = v;
            }
    T W[2][2][3];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int k = 0; k < N3; ++k) {
                T v = T(0);
#pragma unroll
                for (int j = 0; j < N2; ++j) v += axis_coef<T, K2>(j, b) * Y[a][j][k];
                W[a][b][k] = v;
            }
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                T v = T(0);
#pragma unroll
                for (int k = 0; k < N3; ++k) v += axis_coef<T, K3>(k, c) * W[a][b][k];
                mb[a][b][c] = v;
            }
}

// Adjoint of brick_contract with s = 1/8 (c is applied by the caller):
// Mb[q][6] = dL/dM~_q for L = sum_p Sp[p] k_p / c.
template <typename T>
__device__ __forceinline__ void brick_contract_adj(const T (&Sp)[36], T (&Mb)[8][6]) {
    T Trr[3][3], Tss[3][3], Ttt[3][3], Vrs[3][3][3], Vrt[3][3][3], Vst[3][3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            Trr[i][j] = Tss[i][j] = Ttt[i][j] = T(0);
#pragma unroll
            for (int k = 0; k < 3; ++k) Vrs[i][j][k] = Vrt[i][j][k] = Vst[i][j][k] = T(0);
        }
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b <= a; ++b) {
            const int a1 = hb1(a), a2 = hb2(a), a3 = hb3(a);
            const int b1 = hb1(b), b2 = hb2(b), b3 = hb3(b);
            const int c1 = hcls(a1, b1), c2 = hcls(a2, b2), c3 = hcls(a3, b3);
            const T v = T(0.125) * Sp[a * (a + 1) / 2 + b];
            Trr[c2][c3] += T(hsig(a1) * hsig(b1)) * v;
            Tss[c1][c3] += T(hsig(a2) * hsig(b2)) * v;
            Ttt[c1][c2] += T(hsig(a3) * hsig(b3)) * v;
            Vrs[b1][a2][c3] += T(hsig(a1) * hsig(b2)) * v;
            Vrs[a1][b2][c3] += T(hsig(a2) * hsig(b1)) * v;
            Vrt[b1][c2][a3] += T(hsig(a1) * hsig(b3)) * v;
            Vrt[a1][c2][b3] += T(hsig(a3) * hsig(b1)) * v;
            Vst[c1][b2][a3] += T(hsig(a2) * hsig(b3)) * v;
            Vst[c1][a2][b3] += T(hsig(a3) * hsig(b2)) * v;
        }
    T Arr[2][2], Ass[2][2], Att[2][2], mrs[2][2][2], mrt[2][2][2], mst[2][2][2];
    contract_FF_adj(Trr, Arr);
    contract_FF_adj(Tss, Ass);
    contract_FF_adj(Ttt, Att);
    contract_cross_adj<T, 0, 0, 1>(Vrs, mrs);
    contract_cross_adj<T, 0, 1, 0>(Vrt, mrt);
    contract_cross_adj<T, 1, 0, 0>(Vst, mst);
#pragma unroll
    for (int q1 = 0; q1 < 2; ++q1)
#pragma unroll
        for (int q2 = 0; q2 < 2; ++q2)
#pragma unroll
            for (int q3 = 0; q3 < 2; ++q3) {
                const int q = 4 * q1 + 2 * q2 + q3;
                Mb[q][0] = Arr[q2][q3];  // M~_q,rr enters A_rr summed over q1
                Mb[q][1] = Ass[q1][q3];
                Mb[q][2] = Att[q1][q2];
                Mb[q][3] = mrs[q1][q2][q3];
                Mb[q][4] = mrt[q1][q2][q3];
                Mb[q][5] = mst[q1][q2][q3];
            }
}

// Brick: packed upstream Sp[36] -> node gradients dx[8][3] and dc, by reverse
// mode through the forward's own steps (brick_edges -> brick_jrows -> brick_M ->
// brick_contract).  With the rows R, S, U of 2J_q, cofactors C0 = S x U,
// C1 = U x R, C2 = R x S, d = R.C0 and M~_ij = C_i.C_j / |d|, the point's share
// L_q = phi / |d| with phi = sum_ij Mb_ij C_i.C_j gives, with Y_i = sum_j Mb_ij C_j
// (Mb symmetric, off-diagonal halves) and lambda = phi / (|d| d),
//     dL/dR = (2/|d|)(Y1 x U + S x Y2) - lambda C0,
//     dL/dS = (2/|d|)(U x Y0 + Y2 x R) - lambda C1,
//     dL/dU = (2/|d|)(Y0 x S + R x Y1) - lambda C2.
// The row interpolation's 1D operator is symmetric, so brick_jrows is its own
// adjoint; the edges are node differences.  k is linear in c: dc = L / c.
template <typename T, typename S>
__device__ __forceinline__ void brick_vjp(const S (*xc)[3], T c, const T (&Sp)[36], T (&dx)[8][3], T &dc) {
    T Mb[8][6];
    brick_contract_adj(Sp, Mb);
    Vec3<T> e[3][2][2];
    brick_edges<T, S>(xc, e);
    Vec3<T> row[3][2][2];
    brick_jrows(e, row);
    Vec3<T> rb[3][2][2];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax)
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
            for (int v = 0; v < 2; ++v) rb[ax][u][v] = {T(0), T(0), T(0)};
    dc = T(0);
    const T h = T(0.5);
#pragma unroll
    for (int q1 = 0; q1 < 2; ++q1)
#pragma unroll
        for (int q2 = 0; q2 < 2; ++q2)
#pragma unroll
            for (int q3 = 0; q3 < 2; ++q3) {
                const int q = 4 * q1 + 2 * q2 + q3;
                const Vec3<T> &R = row[0][q2][q3];
                const Vec3<T> &Sv = row[1][q1][q3];
                const Vec3<T> &U = row[2][q1][q2];
                const Vec3<T> C0 = cross3(Sv, U), C1 = cross3(U, R), C2 = cross3(R, Sv);
                const T d = dot3(R, C0);
                const T inv = rcp_rn(d < T(0) ? -d : d);
                const T m0 = Mb[q][0], m1 = Mb[q][1], m2 = Mb[q][2];
                const T m3 = h * Mb[q][3], m4 = h * Mb[q][4], m5 = h * Mb[q][5];
                const Vec3<T> Y0 = {m0 * C0.x + m3 * C1.x + m4 * C2.x, m0 * C0.y + m3 * C1.y + m4 * C2.y,
                                    m0 * C0.z + m3 * C1.z + m4 * C2.z};
                const Vec3<T> Y1 = {m3 * C0.x + m1 * C1.x + m5 * C2.x, m3 * C0.y + m1 * C1.y + m5 * C2.y,
                                    m3 * C0.z + m1 * C1.z + m5 * C2.z};
                const Vec3<T> Y2 = {m4 * C0.x + m5 * C1.x + m2 * C2.x, m4 * C0.y + m5 * C1.y + m2 * C2.y,
                                    m4 * C0.z + m5 * C1.z + m2 * C2.z};
                const T phi = dot3(C0, Y0) + dot3(C1, Y1) + dot3(C2, Y2);
                dc += phi * inv;
                // 1/d = sign(d) / |d|: one reciprocal per point, not two; phi is scaled by
                // 1/|d| before the second factor, so no 1/d^2 is ever formed (it would
                // overflow FP32 for |d| below ~1e-19 where phi/|d|^2 stays finite)
                const T lam = ((d < T(0) ? -phi : phi) * inv) * inv, t = T(2) * inv;
                const Vec3<T> a0 = cross3(Y1, U), b0 = cross3(Sv, Y2);
                const Vec3<T> a1 = cross3(U, Y0), b1 = cross3(Y2, R);
                const Vec3<T> a2 = cross3(Y0, Sv), b2 = cross3(R, Y1);
                Vec3<T> &r0 = rb[0][q2][q3], &r1 = rb[1][q1][q3], &r2 = rb[2][q1][q2];
                r0 = {r0.x + t * (a0.x + b0.x) - lam * C0.x, r0.y + t * (a0.y + b0.y) - lam * C0.y,
                      r0.z + t * (a0.z + b0.z) - lam * C0.z};
                r1 = {r1.x + t * (a1.x + b1.x) - lam * C1.x, r1.y + t * (a1.y + b1.y) - lam * C1.y,
                      r1.z + t * (a1.z + b1.z) - lam * C1.z};
                r2 = {r2.x + t * (a2.x + b2.x) - lam * C2.x, r2.y + t * (a2.y + b2.y) - lam * C2.y,
                      r2.z + t * (a2.z + b2.z) - lam * C2.z};
            }
    Vec3<T> eb[3][2][2];
    brick_jrows(rb, eb);
#pragma unroll
    for (int a = 0; a < 8; ++a) dx[a][0] = dx[a][1] = dx[a][2] = T(0);
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int n0[3] = {hnode(0, i, j), hnode(i, 0, j), hnode(i, j, 0)};
            const int n1[3] = {hnode(1, i, j), hnode(i, 1, j), hnode(i, j, 1)};
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) {
                const Vec3<T> &g = eb[ax][i][j];
                dx[n1[ax]][0] += c * g.x;
                dx[n1[ax]][1] += c * g.y;
                dx[n1[ax]][2] += c * g.z;
                dx[n0[ax]][0] -= c * g.x;
                dx[n0[ax]][1] -= c * g.y;
                dx[n0[ax]][2] -= c * g.z;
            }
        }
}

// Tetrahedron: one point, weight 1/6, D = reference barycentric gradients.
template <typename T, typename S>
__device__ __forceinline__ void tet_vjp(const S (*xc)[3], T c, const T (&Sp)[10], T (&dx)[4][3], T &dc) {
    TetGeom<T> tg;
    tet_geom<T, S>(xc, tg);
    const Vec3<T> R0 = tg.R0, R1 = tg.R1, R2 = tg.R2;
    const Vec3<T> C0 = cross3(R1, R2), C1 = cross3(R2, R0), C2 = cross3(R0, R1);
    const T d = dot3(R0, C0);
    const T ad = d < T(0) ? -d : d;
    const T id = rcp_rn(d);
    T A[3][3] = {{C0.x * id, C1.x * id, C2.x * id}, {C0.y * id, C1.y * id, C2.y * id},
                 {C0.z * id, C1.z * id, C2.z * id}};
    const T w = rcp_rn(T(6) * ad);
    T M[3][3];
    M[0][0] = dot3(C0, C0) * w; M[1][1] = dot3(C1, C1) * w; M[2][2] = dot3(C2, C2) * w;
    M[0][1] = M[1][0] = dot3(C0, C1) * w;
    M[0][2] = M[2][0] = dot3(C0, C2) * w;
    M[1][2] = M[2][1] = dot3(C1, C2) * w;
    T Ss[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b <= a; ++b) {
            const T v = Sp[a * (a + 1) / 2 + b];
            Ss[a][b] = a == b ? v : T(0.5) * v;
            Ss[b][a] = Ss[a][b];
        }
    // D[i][a]: lambda_0 = 1 - sum xi, lambda_a = xi_{a-1}
    const T D[3][4] = {{T(-1), T(1), T(0), T(0)}, {T(-1), T(0), T(1), T(0)}, {T(-1), T(0), T(0), T(1)}};
    T H[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            T s = T(0);
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) s += D[i][a] * Ss[a][b] * D[j][b];
            H[i][j] = s;
        }
    T f = T(0);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) f += M[i][j] * H[i][j];
    dc = f;
    T G[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            T s = T(0);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                T mh = T(0);
#pragma unroll
                for (int l = 0; l < 3; ++l) mh += M[i][l] * H[l][k];
                s += ((i == k ? f : T(0)) - T(2) * mh) * A[j][k];
            }
            G[i][j] = c * s;
        }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int j = 0; j < 3; ++j) dx[a][j] = D[0][a] * G[0][j] + D[1][a] * G[1][j] + D[2][a] * G[2][j];
}

// Symmetric element upstream from the packed one (each packed pair counted once).
template <int NPE, typename T>
__device__ __forceinline__ void sym_upstream(const T (&Sp)[NPE * (NPE + 1) / 2], T (&Ss)[NPE][NPE]) {
#pragma unroll
    for (int a = 0; a < NPE; ++a)
#pragma unroll
        for (int b = 0; b <= a; ++b) {
            const T v = Sp[a * (a + 1) / 2 + b];
            Ss[a][b] = a == b ? v : T(0.5) * v;
            Ss[b][a] = Ss[a][b];
        }
}

// Mass operator, brick: the same 2x2x2 rule; N_a(q) are products of 1D hats.
template <typename T, typename S>
__device__ __forceinline__ void brick_mass_vjp(const S (*xc)[3], T c, const T (&Sp)[36], T (&dx)[8][3], T &dc) {
    Vec3<T> e[3][2][2];
    brick_edges<T, S>(xc, e);
    Vec3<T> row[3][2][2];
    brick_jrows(e, row);
    T Ss[8][8];
    sym_upstream<8, T>(Sp, Ss);
#pragma unroll
    for (int a = 0; a < 8; ++a) dx[a][0] = dx[a][1] = dx[a][2] = T(0);
    dc = T(0);
    const T P = T(FEM_GP), Q = T(FEM_GQ);
#pragma unroll 1
    for (int q = 0; q < 8; ++q) {
        const int q1 = q >> 2, q2 = (q >> 1) & 1, q3 = q & 1;
        Vec3<T> R = row[0][q2][q3], Sv = row[1][q1][q3], U = row[2][q1][q2];
        R = {T(0.5) * R.x, T(0.5) * R.y, T(0.5) * R.z};
        Sv = {T(0.5) * Sv.x, T(0.5) * Sv.y, T(0.5) * Sv.z};
        U = {T(0.5) * U.x, T(0.5) * U.y, T(0.5) * U.z};
        const Vec3<T> C0 = cross3(Sv, U), C1 = cross3(U, R), C2 = cross3(R, Sv);
        const T d = dot3(R, C0);
        const T ad = d < T(0) ? -d : d;
        const T id = rcp_rn(d);
        // A = J^{-1}: A[i][j] = C_j[i] / d
        const T A[3][3] = {{C0.x * id, C1.x * id, C2.x * id}, {C0.y * id, C1.y * id, C2.y * id},
                           {C0.z * id, C1.z * id, C2.z * id}};
        T N[8], D[3][8];
#pragma unroll
        for (int a = 0; a < 8; ++a) {
            const int a1 = hb1(a), a2 = hb2(a), a3 = hb3(a);
            const T f1 = a1 == q1 ? P : Q, f2 = a2 == q2 ? P : Q, f3 = a3 == q3 ? P : Q;
            N[a] = f1 * f2 * f3;
            D[0][a] = T(0.5 * hsig(a1)) * f2 * f3;
            D[1][a] = T(0.5 * hsig(a2)) * f1 * f3;
            D[2][a] = T(0.5 * hsig(a3)) * f1 * f2;
        }
        T phi = T(0);
#pragma unroll
        for (int a = 0; a < 8; ++a) {
            T s = T(0);
#pragma unroll
            for (int b = 0; b < 8; ++b) s += Ss[a][b] * N[b];
            phi += N[a] * s;
        }
        dc += ad * phi;
        // dL/dJ = c phi |det J| A^T
        const T k = c * phi * ad;
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
            for (int j = 0; j < 3; ++j)
                dx[a][j] += k * (D[0][a] * A[j][0] + D[1][a] * A[j][1] + D[2][a] * A[j][2]);
    }
}

// Mass operator, tetrahedron: M = c |det J| / 120 (1 + delta_ab).
template <typename T, typename S>
__device__ __forceinline__ void tet_mass_vjp(const S (*xc)[3], T c, const T (&Sp)[10], T (&dx)[4][3], T &dc) {
    TetGeom<T> tg;
    tet_geom<T, S>(xc, tg);
    const Vec3<T> R0 = tg.R0, R1 = tg.R1, R2 = tg.R2;
    const Vec3<T> C0 = cross3(R1, R2), C1 = cross3(R2, R0), C2 = cross3(R0, R1);
    const T d = dot3(R0, C0);
    const T ad = d < T(0) ? -d : d;
    const T id = rcp_rn(d);
    const T A[3][3] = {{C0.x * id, C1.x * id, C2.x * id}, {C0.y * id, C1.y * id, C2.y * id},
                       {C0.z * id, C1.z * id, C2.z * id}};
    T Ss[4][4];
    sym_upstream<4, T>(Sp, Ss);
    T psi = T(0);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) psi += Ss[a][b] * (a == b ? T(2) : T(1));
    psi *= T(1.0 / 120.0);
    dc = ad * psi;
    const T D[3][4] = {{T(-1), T(1), T(0), T(0)}, {T(-1), T(0), T(1), T(0)}, {T(-1), T(0), T(0), T(1)}};
    const T k = c * psi * ad;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int j = 0; j < 3; ++j) dx[a][j] = k * (D[0][a] * A[j][0] + D[1][a] * A[j][1] + D[2][a] * A[j][2]);
}

struct VjpSmem {
    size_t xs, cown, gid, dxs, total;
};

template <int NPE, typename T, typename S, typename CT, bool MASS>
__global__ void __launch_bounds__(256) k_vjp(PlanView pv, const int64_t *__restrict__ rowptr,
                                             const S *__restrict__ X, const CT *__restrict__ c,
                                             const T *__restrict__ G, T *__restrict__ dX, T *__restrict__ dcout,
                                             VjpSmem L, int *status) {
    constexpr int NP = NPE * (NPE + 1) / 2;
    extern __shared__ __align__(16) unsigned char vjp_smem[];
    S(*xs)[3] = reinterpret_cast<S(*)[3]>(vjp_smem + L.xs);
    int32_t *cown = reinterpret_cast<int32_t *>(vjp_smem + L.cown);
    int32_t *gid = reinterpret_cast<int32_t *>(vjp_smem + L.gid);
    T(*dxs)[3] = reinterpret_cast<T(*)[3]>(vjp_smem + L.dxs);
    const int tid = threadIdx.x, nthr = blockDim.x;
    for (int64_t p = blockIdx.x; p < pv.n_patches; p += gridDim.x) {
        const int64_t nb = pv.patch_node_ptr[p];
        const int nown = (int)(pv.patch_node_ptr[p + 1] - nb);
        const int64_t cb = pv.patch_cnode_ptr[p];
        const int ncn = (int)(pv.patch_cnode_ptr[p + 1] - cb);
        const int64_t eb = pv.patch_elem_ptr[p];
        const int nel = (int)(pv.patch_elem_ptr[p + 1] - eb);
        for (int j = tid; j < ncn; j += nthr) {
            const int32_t g = pv.cnode_gid[cb + j];
            gid[j] = g;
            cown[j] = pv.cnode_own[cb + j];
            xs[j][0] = X[3 * (int64_t)g + 0];
            xs[j][1] = X[3 * (int64_t)g + 1];
            xs[j][2] = X[3 * (int64_t)g + 2];
        }
        for (int k = tid; k < nown; k += nthr) dxs[k][0] = dxs[k][1] = dxs[k][2] = T(0);
        __syncthreads();
        for (int base = 0; base < nel; base += nthr) {
            const int i = base + tid;
            const bool act = i < nel;
            const int64_t ci = eb + i;
            int mycol = -1;
            int ln[NPE];
            T dx[NPE][3];
            if (act) {
                mycol = pv.celem_color[ci];
                const int64_t e = pv.celem_id[ci];
#pragma unroll
                for (int a = 0; a < NPE; ++a) ln[a] = pv.celem_lnode[ci * NPE + a];
                S xc[NPE][3];
#pragma unroll
                for (int a = 0; a < NPE; ++a) {
                    xc[a][0] = xs[ln[a]][0];
                    xc[a][1] = xs[ln[a]][1];
                    xc[a][2] = xs[ln[a]][2];
                }
                T Sp[NP];
                const uint8_t *pp = pv.celem_pos + ci * ((NP + 3) / 4 * 4);
#pragma unroll
                for (int a = 0; a < NPE; ++a)
#pragma unroll
                    for (int b = 0; b <= a; ++b) {
                        const int q = a * (a + 1) / 2 + b;
                        const int32_t r = gid[ln[a] > ln[b] ? ln[a] : ln[b]];
                        Sp[q] = G[rowptr[r] + pp[q]];
                    }
                T dcv;
                if constexpr (MASS) {
                    if constexpr (NPE == 8) brick_mass_vjp<T, S>(xc, (T)c[e], Sp, dx, dcv);
                    else tet_mass_vjp<T, S>(xc, (T)c[e], Sp, dx, dcv);
                } else {
                    if constexpr (NPE == 8) brick_vjp<T, S>(xc, (T)c[e], Sp, dx, dcv);
                    else tet_vjp<T, S>(xc, (T)c[e], Sp, dx, dcv);
                }
                if (cown[ln[0]] >= 0) {
                    dcout[e] = dcv;
                    if (!isfinite(dcv)) atomicOr(status, STATUS_NONFINITE);  // e.g. zero det J
                }
            }
            const int last = min(base + nthr, nel) - 1;
            const int c0 = pv.celem_color[eb + base], c1 = pv.celem_color[eb + last];
            for (int cc = c0; cc <= c1; ++cc) {
                if (mycol == cc) {
#pragma unroll
                    for (int a = 0; a < NPE; ++a) {
                        const int o = cown[ln[a]];
                        if (o >= 0) {
                            dxs[o][0] += dx[a][0];
                            dxs[o][1] += dx[a][1];
                            dxs[o][2] += dx[a][2];
                        }
                    }
                }
                __syncthreads();
            }
        }
        for (int k = tid; k < nown; k += nthr) {
            const int64_t g = pv.own_row[nb + k];
            dX[3 * g + 0] = dxs[k][0];
            dX[3 * g + 1] = dxs[k][1];
            dX[3 * g + 2] = dxs[k][2];
        }
        __syncthreads();
    }
}

static size_t a16(size_t v) { return (v + 15) & ~(size_t)15; }

template <int NPE, typename T, typename S, typename CT>
static fem_status launch_vjp_t(fem_mesh m, const Closure &cl, const void *X, const void *c, const void *G, void *dX,
                               void *dc, cudaStream_t s) {
    const Plan &P = m->plan;
    VjpSmem L{};
    size_t o = 0;
    L.xs = o;
    o = a16(o + (size_t)P.max_cnodes * 3 * sizeof(S));
    L.cown = o;
    o = a16(o + (size_t)P.max_cnodes * 4);
    L.gid = o;
    o = a16(o + (size_t)P.max_cnodes * 4);
    L.dxs = o;
    o = a16(o + (size_t)P.max_own * 3 * sizeof(T));
    L.total = o;
    auto f = m->opt.operator_kind == 1 ? k_vjp<NPE, T, S, CT, true> : k_vjp<NPE, T, S, CT, false>;
    FEM_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total));
    int per_sm = 0;
    FEM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, 256, L.total));
    if (per_sm < 1) {
        set_error("backward kernel cannot be resident with %zu bytes of shared memory", L.total);
        return FEM_ERR_UNSUPPORTED;
    }
    const int64_t np = cl.p1 - cl.p0;
    if (np <= 0) return FEM_OK;
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(np, (int64_t)num_sms() * per_sm));
    f<<<grid, 256, L.total, s>>>(P.view(cl), m->rowptr.ptr, (const S *)X, (const CT *)c, (const T *)G, (T *)dX,
                                 (T *)dc, L, m->status.ptr);
    FEM_LAUNCHED("k_vjp");
    return FEM_OK;
}

// ------------------------------------------------------------ staged backward
// Pass 1 (k_vjp_elem) integrates every element once -- its instance in the
// closure of the patch that owns its first node -- and writes the element's node
// gradients to dxe [n_elems][NPE][3] (library memory) and dc_e.  Pass 2
// (k_vjp_gather) adds dxe into the owned nodes of each patch colour by colour,
// the order of the fused kernel above, and writes dX.  The element work is done
// once instead of once per patch whose closure holds the element.

struct ElemSmem {
    size_t xs, cown, rp, list, total;  // rp: rowptr of each closure node
};

template <typename T, int N>
__device__ __forceinline__ void store_row(T *__restrict__ o, const T (&v)[N]) {
    // o is 16-byte aligned (N * sizeof(T) is a multiple of 16 for every use)
    static_assert((N * sizeof(T)) % 16 == 0, "row of 16-byte chunks");
    if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int k = 0; k < N; k += 4) reinterpret_cast<float4 *>(o)[k / 4] = make_float4(v[k], v[k + 1], v[k + 2], v[k + 3]);
    } else {
#pragma unroll
        for (int k = 0; k < N; k += 2) reinterpret_cast<double2 *>(o)[k / 2] = make_double2(v[k], v[k + 1]);
    }
}

// Closure elements of patch p whose first node the patch owns, compacted into
// list[0 .. return) (in no particular order: each element's outputs are its own).
__device__ __forceinline__ int primary_elems(const PlanView &pv, int npe, int64_t eb, int nel, const int32_t *cown,
                                             int32_t *list, int *count) {
    if (threadIdx.x == 0) *count = 0;
    __syncthreads();
    // one counter update per warp (ballot), not per element: same-address shared
    // atomics serialise; the loop bound is warp-uniform
    const int lane = threadIdx.x & 31;
    for (int j0 = 0; j0 < nel; j0 += blockDim.x) {
        const int j = j0 + threadIdx.x;
        const bool f = j < nel && cown[pv.celem_lnode[(eb + j) * npe]] >= 0;
        const unsigned bal = __ballot_sync(0xffffffffu, f);
        int w0 = 0;
        if (lane == 0 && bal) w0 = atomicAdd(count, __popc(bal));
        w0 = __shfl_sync(0xffffffffu, w0, 0);
        if (f) list[w0 + __popc(bal & ((1u << lane) - 1u))] = j;
    }
    __syncthreads();
    return *count;
}

// FP64 element work holds ~220 registers a thread: 128-thread blocks leave a
// smaller idle tail per patch at the same 8 warps per SM (measured: 4.83 -> 4.45
// ms on 1M bricks); FP32 runs 256-thread blocks (measured faster there).
template <typename T>
constexpr int vjp_elem_threads() { return sizeof(T) == 8 ? 128 : 256; }

template <int NPE, typename T, typename S, typename CT, bool MASS>
__global__ void __launch_bounds__(256) k_vjp_elem(PlanView pv, const int64_t *__restrict__ rowptr,
                                                  const S *__restrict__ X, const CT *__restrict__ c,
                                                  const T *__restrict__ G, T *__restrict__ dxe,
                                                  T *__restrict__ dcout, ElemSmem L, int *status) {
    constexpr int NP = NPE * (NPE + 1) / 2;
    extern __shared__ __align__(16) unsigned char vel_smem[];
    __shared__ int n_prim;
    S(*xs)[3] = reinterpret_cast<S(*)[3]>(vel_smem + L.xs);
    int32_t *cown = reinterpret_cast<int32_t *>(vel_smem + L.cown);
    int64_t *rp = reinterpret_cast<int64_t *>(vel_smem + L.rp);
    int32_t *list = reinterpret_cast<int32_t *>(vel_smem + L.list);
    const int tid = threadIdx.x, nthr = blockDim.x;
    for (int64_t p = blockIdx.x; p < pv.n_patches; p += gridDim.x) {
        const int64_t cb = pv.patch_cnode_ptr[p];
        const int ncn = (int)(pv.patch_cnode_ptr[p + 1] - cb);
        const int64_t eb = pv.patch_elem_ptr[p];
        const int nel = (int)(pv.patch_elem_ptr[p + 1] - eb);
        // closure nodes: ids, then their row starts and coordinates, CH nodes in
        // flight per thread (the second loads depend on the first)
        constexpr int CH = 4;
        for (int j0 = 0; j0 < ncn; j0 += CH * nthr) {
            int32_t gv[CH], ov[CH];
#pragma unroll
            for (int u = 0; u < CH; ++u) {
                const int j = j0 + u * nthr + tid;
                gv[u] = j < ncn ? pv.cnode_gid[cb + j] : 0;
                ov[u] = j < ncn ? pv.cnode_own[cb + j] : -1;
            }
            int64_t rv[CH];
            S xv[CH][3];
#pragma unroll
            for (int u = 0; u < CH; ++u) {
                const int j = j0 + u * nthr + tid;
                const int64_t g = gv[u];
                rv[u] = j < ncn ? rowptr[g] : 0;
                xv[u][0] = j < ncn ? X[3 * g + 0] : S(0);
                xv[u][1] = j < ncn ? X[3 * g + 1] : S(0);
                xv[u][2] = j < ncn ? X[3 * g + 2] : S(0);
            }
#pragma unroll
            for (int u = 0; u < CH; ++u) {
                const int j = j0 + u * nthr + tid;
                if (j < ncn) {
                    rp[j] = rv[u];
                    cown[j] = ov[u];
                    xs[j][0] = xv[u][0];
                    xs[j][1] = xv[u][1];
                    xs[j][2] = xv[u][2];
                }
            }
        }
        const int np = primary_elems(pv, NPE, eb, nel, cown, list, &n_prim);
        for (int k = tid; k < np; k += nthr) {
            const int64_t ci = eb + list[k];
            const int64_t e = pv.celem_id[ci];
            uint16_t lv[NPE];
            load_lnodes<NPE>(pv.celem_lnode, ci, lv);
            int ln[NPE];
#pragma unroll
            for (int a = 0; a < NPE; ++a) ln[a] = lv[a];
            S xc[NPE][3];
#pragma unroll
            for (int a = 0; a < NPE; ++a) {
                xc[a][0] = xs[ln[a]][0];
                xc[a][1] = xs[ln[a]][1];
                xc[a][2] = xs[ln[a]][2];
            }
            // the pair's row is its node with the larger global id (closure-local
            // indices ascend with it); positions read as 32-bit words
            constexpr int NW = (NP + 3) / 4;
            uint32_t pw[NW];
            const uint32_t *pp = reinterpret_cast<const uint32_t *>(pv.celem_pos + ci * (NW * 4));
#pragma unroll
            for (int w = 0; w < NW; ++w) pw[w] = __ldg(pp + w);
            int64_t rb[NPE];
#pragma unroll
            for (int a = 0; a < NPE; ++a) rb[a] = rp[ln[a]];
            T Sp[NP];
#pragma unroll
            for (int a = 0; a < NPE; ++a)
#pragma unroll
                for (int b = 0; b <= a; ++b) {
                    const int q = a * (a + 1) / 2 + b;
                    const int64_t r0 = ln[a] > ln[b] ? rb[a] : rb[b];
                    Sp[q] = __ldg(G + r0 + ((pw[q >> 2] >> (8 * (q & 3))) & 0xff));
                }
            T dx[NPE][3], dcv;
            if constexpr (MASS) {
                if constexpr (NPE == 8) brick_mass_vjp<T, S>(xc, (T)c[e], Sp, dx, dcv);
                else tet_mass_vjp<T, S>(xc, (T)c[e], Sp, dx, dcv);
            } else {
                if constexpr (NPE == 8) brick_vjp<T, S>(xc, (T)c[e], Sp, dx, dcv);
                else tet_vjp<T, S>(xc, (T)c[e], Sp, dx, dcv);
            }
            T flat[NPE * 3];
#pragma unroll
            for (int a = 0; a < NPE; ++a)
#pragma unroll
                for (int j = 0; j < 3; ++j) flat[3 * a + j] = dx[a][j];
            store_row<T, NPE * 3>(dxe + e * (NPE * 3), flat);
            dcout[e] = dcv;
            if (!isfinite(dcv)) atomicOr(status, STATUS_NONFINITE);  // e.g. zero det J
        }
        __syncthreads();
    }
}

struct GatherSmem {
    size_t cown, dxs, total;
};

// The colour order is kept by the forward kernel's ring of mbarrier phases
// (phases.cuh) instead of block-wide barriers: a warp with nothing to add in a
// colour only arrives and moves on.
template <int NPE, typename T>
__global__ void __launch_bounds__(256) k_vjp_gather(PlanView pv, const T *__restrict__ dxe, T *__restrict__ dX,
                                                    GatherSmem L, WaitCtl wc) {
    extern __shared__ __align__(16) unsigned char vg_smem[];
    __shared__ __align__(8) uint64_t mb[PHASE_RING];
    int32_t *cown = reinterpret_cast<int32_t *>(vg_smem + L.cown);
    T(*dxs)[3] = reinterpret_cast<T(*)[3]>(vg_smem + L.dxs);
    const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31;
    phase_init(mb);
    uint32_t g = 0;  // the block's running phase number
    for (int64_t p = blockIdx.x; p < pv.n_patches; p += gridDim.x) {
        const int64_t nb = pv.patch_node_ptr[p];
        const int nown = (int)(pv.patch_node_ptr[p + 1] - nb);
        const int64_t cb = pv.patch_cnode_ptr[p];
        const int ncn = (int)(pv.patch_cnode_ptr[p + 1] - cb);
        const int64_t eb = pv.patch_elem_ptr[p];
        const int nel = (int)(pv.patch_elem_ptr[p + 1] - eb);
        for (int j = tid; j < ncn; j += nthr) cown[j] = pv.cnode_own[cb + j];
        for (int k = tid; k < nown; k += nthr) dxs[k][0] = dxs[k][1] = dxs[k][2] = T(0);
        __syncthreads();
        for (int base = 0; base < nel; base += nthr) {
            const int i = base + tid;
            int mycol = -1;
            int own[NPE];
            T v[NPE][3];
#pragma unroll
            for (int a = 0; a < NPE; ++a) own[a] = -1;
            if (i < nel) {
                const int64_t ci = eb + i;
                mycol = pv.celem_color[ci];
                const int64_t e = pv.celem_id[ci];
                const T *src = dxe + e * (NPE * 3);
                uint16_t ln[NPE];
                load_lnodes<NPE>(pv.celem_lnode, ci, ln);
                // the element's row of node gradients in 16-byte pieces (rows are
                // 16-byte aligned: NPE * 3 values of 4 or 8 bytes)
                T row[NPE * 3];
                if constexpr (sizeof(T) == 4) {
#pragma unroll
                    for (int k = 0; k < NPE * 3; k += 4) {
                        const float4 w = __ldg(reinterpret_cast<const float4 *>(src) + k / 4);
                        row[k] = w.x; row[k + 1] = w.y; row[k + 2] = w.z; row[k + 3] = w.w;
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < NPE * 3; k += 2) {
                        const double2 w = __ldg(reinterpret_cast<const double2 *>(src) + k / 2);
                        row[k] = w.x; row[k + 1] = w.y;
                    }
                }
#pragma unroll
                for (int a = 0; a < NPE; ++a) {
                    own[a] = cown[ln[a]];
#pragma unroll
                    for (int j = 0; j < 3; ++j) v[a][j] = row[3 * a + j];
                }
            }
            const int last = min(base + nthr, nel) - 1;
            const int c0 = pv.celem_color[eb + base], c1 = pv.celem_color[eb + last];
            for (int cc = c0; cc <= c1; ++cc, ++g) {
                const bool mine = mycol == cc;
                if (__any_sync(0xffffffffu, mine)) {
                    if (g > 0) phase_wait(mb, g - 1, wc);
                    if (mine) {
#pragma unroll
                        for (int a = 0; a < NPE; ++a) {
                            const int o = own[a];
                            if (o >= 0) {
                                dxs[o][0] += v[a][0];
                                dxs[o][1] += v[a][1];
                                dxs[o][2] += v[a][2];
                            }
                        }
                    }
                    __syncwarp();
                }
                if (g >= (uint32_t)PHASE_RING) phase_wait(mb, g - PHASE_RING, wc);
                if (lane == 0) phase_arrive(mb, g);
            }
        }
        __syncthreads();  // every phase of the patch done
        for (int k = tid; k < nown; k += nthr) {
            const int64_t gr = pv.own_row[nb + k];
            dX[3 * gr + 0] = dxs[k][0];
            dX[3 * gr + 1] = dxs[k][1];
            dX[3 * gr + 2] = dxs[k][2];
        }
        __syncthreads();
    }
}

static int grid_for(const void *f, int threads, size_t smem, int64_t np, const char *what, fem_status *st) {
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, threads, smem);
    if (e != cudaSuccess || per_sm < 1) {
        set_error("%s cannot be resident with %zu bytes of shared memory", what, smem);
        *st = e != cudaSuccess ? cuda_status(e, what) : FEM_ERR_UNSUPPORTED;
        return 0;
    }
    *st = FEM_OK;
    return (int)std::max<int64_t>(1, std::min<int64_t>(np, (int64_t)num_sms() * per_sm));
}

ElemSmem elem_smem(const Plan &P, const Closure &cl, size_t xsize) {
    ElemSmem L{};
    size_t o = 0;
    L.xs = o;
    o = a16(o + (size_t)P.max_cnodes * 3 * xsize);
    L.cown = o;
    o = a16(o + (size_t)P.max_cnodes * 4);
    L.rp = o;
    o = a16(o + (size_t)P.max_cnodes * 8);
    L.list = o;
    o = a16(o + (size_t)std::max<int64_t>(cl.max_celems, P.max_celems) * 4);
    L.total = o;
    return L;
}

template <int NPE, typename T, typename S, typename CT>
static fem_status launch_vjp_elem_t(fem_mesh m, const Closure &cl, const void *X, const void *c, const void *G,
                                    void *dxe, void *dc, cudaStream_t s) {
    const Plan &P = m->plan;
    const ElemSmem L = elem_smem(P, cl, sizeof(S));
    auto f = m->opt.operator_kind == 1 ? k_vjp_elem<NPE, T, S, CT, true> : k_vjp_elem<NPE, T, S, CT, false>;
    FEM_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total));
    if constexpr (NPE == 4) {
        // tets: shared memory for two blocks per SM, the rest of the unified L1/shared
        // array kept as L1 for the element's gathers
        const int pct = (int)std::min<size_t>(100, (2 * (L.total + 1024) * 100 + 228 * 1024 - 1) / (228 * 1024));
        FEM_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, pct));
    }
    const int64_t np = cl.p1 - cl.p0;
    if (np <= 0) return FEM_OK;
    fem_status st;
    constexpr int nt = vjp_elem_threads<T>();
    const int grid = grid_for((const void *)f, nt, L.total, np, "backward element kernel", &st);
    if (st != FEM_OK) return st;
    f<<<grid, nt, L.total, s>>>(P.view(cl), m->rowptr.ptr, (const S *)X, (const CT *)c, (const T *)G,
                                              (T *)dxe, (T *)dc, L, m->status.ptr);
    FEM_LAUNCHED("k_vjp_elem");
    return FEM_OK;
}

template <int NPE, typename T>
static fem_status launch_gather_t(fem_mesh m, const Closure &cl, const void *dxe, void *dX, cudaStream_t s) {
    const Plan &P = m->plan;
    GatherSmem L{};
    size_t o = 0;
    L.cown = o;
    o = a16(o + (size_t)P.max_cnodes * 4);
    L.dxs = o;
    o = a16(o + (size_t)P.max_own * 3 * sizeof(T));
    L.total = o;
    auto f = k_vjp_gather<NPE, T>;
    FEM_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total));
    const int64_t np = cl.p1 - cl.p0;
    if (np <= 0) return FEM_OK;
    fem_status st;
    const int grid = grid_for((const void *)f, 256, L.total, np, "backward gather kernel", &st);
    if (st != FEM_OK) return st;
    const WaitCtl wc{m->status.ptr, m->opt.wait_spins > 0 ? m->opt.wait_spins : WAIT_SPINS_DEFAULT, 0};
    f<<<grid, 256, L.total, s>>>(P.view(cl), (const T *)dxe, (T *)dX, L, wc);
    FEM_LAUNCHED("k_vjp_gather");
    return FEM_OK;
}

// Pass 2 for every operator (the elasticity kernel writes the same dxe layout).
fem_status launch_vjp_gather(fem_mesh m, bool fp64, const void *dxe, void *dX, cudaStream_t s) {
    return for_each_group(m, s, [&](const Closure &cl) -> fem_status {
        if (fp64) return m->npe == 8 ? launch_gather_t<8, double>(m, cl, dxe, dX, s)
                                     : launch_gather_t<4, double>(m, cl, dxe, dX, s);
        return m->npe == 8 ? launch_gather_t<8, float>(m, cl, dxe, dX, s) : launch_gather_t<4, float>(m, cl, dxe, dX, s);
    });
}

// Library memory for dxe, in the mesh's FP64 element-matrix buffer (grown if
// needed); FEM_ERR_BUDGET when the budget refuses it.  Only for a plan whose
// closures are resident (pass 2 needs every element's pass 1 first).
fem_status vjp_scratch(fem_mesh m, bool fp64, void **dxe) {
    *dxe = nullptr;
    if (m->plan.chunked || m->opt.vjp_fused != 0) return FEM_ERR_BUDGET;
    const size_t need = ((size_t)m->n_elems * m->npe * 3 * (fp64 ? 8 : 4) + 7) / 8;
    if (m->ke64.n < need) FEM_TRY(m->ke64.alloc(m->arena, need, "backward element gradients"));
    *dxe = m->ke64.ptr;
    return FEM_OK;
}

static fem_status launch_vjp_elem(fem_mesh m, const Closure &cl, bool mixed, const void *X, fem_dtype xd,
                                  const void *c, fem_dtype cd, const void *G, void *dxe, void *dc, cudaStream_t s) {
#define FEM_E(NPE, T, S, CT) return launch_vjp_elem_t<NPE, T, S, CT>(m, cl, X, c, G, dxe, dc, s)
    if (!mixed) {
        if (m->npe == 8) FEM_E(8, double, double, double);
        FEM_E(4, double, double, double);
    }
    if (m->npe == 8) {
        if (xd == FEM_F32 && cd == FEM_F32) FEM_E(8, float, float, float);
        if (xd == FEM_F32 && cd == FEM_F64) FEM_E(8, float, float, double);
        if (xd == FEM_F64 && cd == FEM_F32) FEM_E(8, float, double, float);
        FEM_E(8, float, double, double);
    }
    if (xd == FEM_F32 && cd == FEM_F32) FEM_E(4, float, float, float);
    if (xd == FEM_F32 && cd == FEM_F64) FEM_E(4, float, float, double);
    if (xd == FEM_F64 && cd == FEM_F32) FEM_E(4, float, double, float);
    FEM_E(4, float, double, double);
#undef FEM_E
}

static fem_status launch_vjp_group(fem_mesh m, const Closure &cl, bool mixed, const void *X, fem_dtype xd,
                                   const void *c, fem_dtype cd, const void *G, void *dX, void *dc, cudaStream_t s) {
#define FEM_V(NPE, T, S, CT) return launch_vjp_t<NPE, T, S, CT>(m, cl, X, c, G, dX, dc, s)
    if (!mixed) {
        if (m->npe == 8) FEM_V(8, double, double, double);
        FEM_V(4, double, double, double);
    }
    if (m->npe == 8) {
        if (xd == FEM_F32 && cd == FEM_F32) FEM_V(8, float, float, float);
        if (xd == FEM_F32 && cd == FEM_F64) FEM_V(8, float, float, double);
        if (xd == FEM_F64 && cd == FEM_F32) FEM_V(8, float, double, float);
        FEM_V(8, float, double, double);
    }
    if (xd == FEM_F32 && cd == FEM_F32) FEM_V(4, float, float, float);
    if (xd == FEM_F32 && cd == FEM_F64) FEM_V(4, float, float, double);
    if (xd == FEM_F64 && cd == FEM_F32) FEM_V(4, float, double, float);
    FEM_V(4, float, double, double);
#undef FEM_V
}

fem_status launch_vjp(fem_mesh m, bool mixed, const void *X, fem_dtype xd, const void *c, fem_dtype cd,
                      const void *G, void *dX, void *dc, cudaStream_t s) {
    void *dxe = nullptr;
    const fem_status st = vjp_scratch(m, !mixed, &dxe);
    if (st == FEM_OK) {
        FEM_TRY(for_each_group(m, s, [&](const Closure &cl) {
            return launch_vjp_elem(m, cl, mixed, X, xd, c, cd, G, dxe, dc, s);
        }));
        return launch_vjp_gather(m, !mixed, dxe, dX, s);
    }
    if (st != FEM_ERR_BUDGET) return st;
    return for_each_group(m, s, [&](const Closure &cl) {
        return launch_vjp_group(m, cl, mixed, X, xd, c, cd, G, dX, dc, s);
    });
}

}  // namespace fem
