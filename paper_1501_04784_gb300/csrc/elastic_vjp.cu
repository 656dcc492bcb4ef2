// elastic_vjp.cu -- backward pass of the elasticity operator: the vector-Jacobian
// product of L = sum over stored entries G_ij K_ij with respect to the node
// coordinates X and the Lame parameters (lambda_e, mu_e).
//
// Per element, with W the symmetric DOF upstream (the stored entry's G on the
// diagonal of k_e, half of it off the diagonal: each packed pair counted once)
// and W^ab its 3x3 block of nodes (a, b), L_e = sum_q w_q |det J_q| Phi(G_q) with
// G = J^{-1} dN the physical gradients and
//     Phi(G) = sum_ab [lambda G_a^T W^ab G_b + mu G_b^T W^ab G_a + mu tr(W^ab) G_a.G_b].
// Phi is linear in lambda and mu, so dL/dlambda_e and dL/dmu_e are its two parts.
// With Psi_a = dPhi/dG_a = 2 sum_b T^ab G_b, T^ab = lambda W^ab + mu W^ab^T +
// mu tr(W^ab) I, and A = J^{-1} (d|det J| = |det J| tr(A dJ), dA = -A dJ A):
//     dL/dJ_q = w_q |det J_q| (Phi A^T - A^T sum_a Psi_a G_a^T),
// and J = dN X_e gives dL/dx_a = sum_q dN_q,a^T dL/dJ_q.  Nothing is kept from
// the forward pass.
//
// Work split as in the forward kernel: NPE threads per element, thread a owning
// node a and the blocks blk_node(a, m) (elastic.cuh); each thread forms its
// blocks' share of Phi, of sum_a Psi_a G_a^T and of dL/dlambda, dL/dmu, the shares
// are summed over the element's lanes by shuffles, and thread a then forms
// dL/dx_a.  Accumulation is owner-computes on the plan with colour-ordered adds,
// as the scalar backward kernel (vjp.cu): no atomics, bitwise reproducible.
#include "elastic.cuh"
#include "mesh.cuh"
#include "numeric.cuh"

namespace fem {

// Sum over the element's NPE lanes (lanes base .. base + NPE - 1 of the warp).
template <int NPE, typename T>
__device__ __forceinline__ T group_sum(T v) {
#pragma unroll
    for (int o = NPE / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// One Gauss point's share of the thread's blocks: Phi, P = sum_a Psi_a G_a^T (the
// thread's part), dL/dlambda and dL/dmu (times the point's w |det J|: wd).
template <int NPE, typename T>
__device__ __forceinline__ void point_shares(const T (&W)[elastic_nblk<NPE>()][9], const Vec3<T> &ga,
                                             const Vec3<T> (&gb)[elastic_nblk<NPE>()], int a, T lam, T mu, T wd,
                                             T &phi, T (&P)[9], T &dlam, T &dmu) {
    phi = T(0);
#pragma unroll
    for (int n = 0; n < 9; ++n) P[n] = T(0);
    const T g_a[3] = {ga.x, ga.y, ga.z};
#pragma unroll
    for (int m = 0; m < elastic_nblk<NPE>(); ++m) {
        if (!blk_valid<NPE>(a, m)) continue;
        const bool diag = blk_node<NPE>(a, m) == a;
        const T mult = diag ? T(1) : T(2);
        const T g_b[3] = {gb[m].x, gb[m].y, gb[m].z};
        const T t = W[m][0] + W[m][4] + W[m][8];
        T Wgb[3], WTgb[3], Wga[3], WTga[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            Wgb[i] = W[m][3 * i] * g_b[0] + W[m][3 * i + 1] * g_b[1] + W[m][3 * i + 2] * g_b[2];
            WTgb[i] = W[m][i] * g_b[0] + W[m][3 + i] * g_b[1] + W[m][6 + i] * g_b[2];
            Wga[i] = W[m][3 * i] * g_a[0] + W[m][3 * i + 1] * g_a[1] + W[m][3 * i + 2] * g_a[2];
            WTga[i] = W[m][i] * g_a[0] + W[m][3 + i] * g_a[1] + W[m][6 + i] * g_a[2];
        }
        const T lt = g_a[0] * Wgb[0] + g_a[1] * Wgb[1] + g_a[2] * Wgb[2];    // G_a^T W G_b
        const T mt = g_b[0] * Wga[0] + g_b[1] * Wga[1] + g_b[2] * Wga[2];    // G_b^T W G_a
        const T gab = g_a[0] * g_b[0] + g_a[1] * g_b[1] + g_a[2] * g_b[2];
        phi += mult * (lam * lt + mu * (mt + t * gab));
        dlam += wd * mult * lt;
        dmu += wd * mult * (mt + t * gab);
        // 2 T^ab G_b G_a^T, and for b != a also 2 T^ba G_a G_b^T
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const T u1 = T(2) * (lam * Wgb[i] + mu * WTgb[i] + mu * t * g_b[i]);
            const T u2 = T(2) * (lam * WTga[i] + mu * Wga[i] + mu * t * g_a[i]);
#pragma unroll
            for (int j = 0; j < 3; ++j) P[3 * i + j] += u1 * g_a[j] + (diag ? T(0) : u2 * g_b[j]);
        }
    }
}

// dL/dJ = wd (phi A^T - A^T P), then dx_a += D_a^T dL/dJ.
template <typename T>
__device__ __forceinline__ void add_dx(const T (&A)[3][3], T phi, const T (&P)[9], T wd, const T (&Da)[3],
                                       T (&dx)[3]) {
    T dJ[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            T s = phi * A[j][i];
#pragma unroll
            for (int k = 0; k < 3; ++k) s -= A[k][i] * P[3 * k + j];
            dJ[i][j] = wd * s;
        }
#pragma unroll
    for (int j = 0; j < 3; ++j) dx[j] += Da[0] * dJ[0][j] + Da[1] * dJ[1][j] + Da[2] * dJ[2][j];
}

// Brick: node a = lane & 7; all 32 lanes call it (it shuffles).  W = the thread's
// blocks of the symmetric upstream.  Outputs dx_a and (summed over the element)
// dlam, dmu.  At each point the thread forms only its own node's gradient G_a and
// takes its block partners' from their lanes; Psi_a (= dPhi/dG_a) gathers its own
// blocks' shares and, by shuffles back, the shares of the blocks in which node a
// is the partner, so sum_a Psi_a G_a^T needs one outer product per thread.
template <typename T, typename S>
__device__ __forceinline__ void elastic_brick_vjp(const S (*xc)[3], T lam, T mu, const T (&W)[5][9], T (&dx)[3],
                                                  T &dlam, T &dmu) {
    const int lane = threadIdx.x & 31, a = lane & 7, base = lane & ~7;
    Vec3<T> e[3][2][2];
    brick_edges<T, S>(xc, e);
    Vec3<T> row[3][2][2];
    brick_jrows(e, row);
    dx[0] = dx[1] = dx[2] = T(0);
    dlam = dmu = T(0);
    const T P = T(FEM_GP), Q = T(FEM_GQ);
    const int a1 = (a ^ (a >> 1)) & 1, a2 = (a >> 1) & 1, a3 = a >> 2;  // node a's axis bits
    const T s1 = a1 ? T(0.5) : T(-0.5), s2 = a2 ? T(0.5) : T(-0.5), s3 = a3 ? T(0.5) : T(-0.5);
    int src_b[5], src_r[5];
#pragma unroll
    for (int m = 0; m < 5; ++m) {
        src_b[m] = base + ((a + m) & 7);  // the partner of block m
        src_r[m] = base + ((a - m) & 7);  // the lane whose block m has node a as partner
    }
    T tr[5];
#pragma unroll
    for (int m = 0; m < 5; ++m) tr[m] = W[m][0] + W[m][4] + W[m][8];
#pragma unroll 1
    for (int q = 0; q < 8; ++q) {
        const int q1 = q >> 2, q2 = (q >> 1) & 1, q3 = q & 1;
        // true Jacobian rows (the stored rows are 2J), cofactors, A = J^{-1}
        Vec3<T> R = row[0][q2][q3], Sv = row[1][q1][q3], U = row[2][q1][q2];
        R = {T(0.5) * R.x, T(0.5) * R.y, T(0.5) * R.z};
        Sv = {T(0.5) * Sv.x, T(0.5) * Sv.y, T(0.5) * Sv.z};
        U = {T(0.5) * U.x, T(0.5) * U.y, T(0.5) * U.z};
        const Vec3<T> C0 = cross3(Sv, U), C1 = cross3(U, R), C2 = cross3(R, Sv);
        const T d = dot3(R, C0);
        const T id = rcp_rn(d);
        const T A[3][3] = {{C0.x * id, C1.x * id, C2.x * id}, {C0.y * id, C1.y * id, C2.y * id},
                           {C0.z * id, C1.z * id, C2.z * id}};
        const T wd = d < T(0) ? -d : d;  // Gauss weights 1
        // node a's natural derivatives and physical gradient at q
        const T f1 = a1 == q1 ? P : Q, f2 = a2 == q2 ? P : Q, f3 = a3 == q3 ? P : Q;
        const T Da[3] = {s1 * f2 * f3, s2 * f1 * f3, s3 * f1 * f2};
        const T g_a[3] = {A[0][0] * Da[0] + A[0][1] * Da[1] + A[0][2] * Da[2],
                          A[1][0] * Da[0] + A[1][1] * Da[1] + A[1][2] * Da[2],
                          A[2][0] * Da[0] + A[2][1] * Da[1] + A[2][2] * Da[2]};
        T phi = T(0), psi[3] = {T(0), T(0), T(0)}, u2[5][3];
#pragma unroll
        for (int m = 0; m < 5; ++m) {
            T g_b[3] = {g_a[0], g_a[1], g_a[2]};
            if (m > 0) {
#pragma unroll
                for (int i = 0; i < 3; ++i) g_b[i] = __shfl_sync(0xffffffffu, g_a[i], src_b[m]);
            }
            u2[m][0] = u2[m][1] = u2[m][2] = T(0);
            if (!blk_valid<8>(a, m)) continue;
            const T mult = m == 0 ? T(1) : T(2);
            const T t = tr[m];
            T Wgb[3], WTgb[3], Wga[3], WTga[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                Wgb[i] = W[m][3 * i] * g_b[0] + W[m][3 * i + 1] * g_b[1] + W[m][3 * i + 2] * g_b[2];
                WTgb[i] = W[m][i] * g_b[0] + W[m][3 + i] * g_b[1] + W[m][6 + i] * g_b[2];
                Wga[i] = W[m][3 * i] * g_a[0] + W[m][3 * i + 1] * g_a[1] + W[m][3 * i + 2] * g_a[2];
                WTga[i] = W[m][i] * g_a[0] + W[m][3 + i] * g_a[1] + W[m][6 + i] * g_a[2];
            }
            const T lt = g_a[0] * Wgb[0] + g_a[1] * Wgb[1] + g_a[2] * Wgb[2];  // G_a^T W G_b
            const T mt = g_b[0] * Wga[0] + g_b[1] * Wga[1] + g_b[2] * Wga[2];  // G_b^T W G_a
            const T gab = g_a[0] * g_b[0] + g_a[1] * g_b[1] + g_a[2] * g_b[2];
            phi += mult * (lam * lt + mu * (mt + t * gab));
            dlam += wd * mult * lt;
            dmu += wd * mult * (mt + t * gab);
            // dPhi/dG_a from this block: 2 T^ab G_b; for b != a, dPhi/dG_b = 2 T^ba G_a
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                psi[i] += T(2) * (lam * Wgb[i] + mu * WTgb[i] + mu * t * g_b[i]);
                if (m > 0) u2[m][i] = T(2) * (lam * WTga[i] + mu * Wga[i] + mu * t * g_a[i]);
            }
        }
#pragma unroll
        for (int m = 1; m < 5; ++m)
#pragma unroll
            for (int i = 0; i < 3; ++i) psi[i] += __shfl_sync(0xffffffffu, u2[m][i], src_r[m]);
        T Pm[9];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) Pm[3 * i + j] = psi[i] * g_a[j];
        phi = group_sum<8, T>(phi);
#pragma unroll
        for (int n = 0; n < 9; ++n) Pm[n] = group_sum<8, T>(Pm[n]);
        add_dx(A, phi, Pm, wd, Da, dx);
    }
    dlam = group_sum<8, T>(dlam);
    dmu = group_sum<8, T>(dmu);
}

// Tetrahedron: node a = lane & 3, one point of weight 1/6.
template <typename T, typename S>
__device__ __forceinline__ void elastic_tet_vjp(const S (*xc)[3], T lam, T mu, const T (&W)[4][9], T (&dx)[3],
                                                T &dlam, T &dmu) {
    const int a = threadIdx.x & 3;
    TetGeom<T> tg;
    tet_geom<T, S>(xc, tg);
    const Vec3<T> R0 = tg.R0, R1 = tg.R1, R2 = tg.R2;
    const Vec3<T> C0 = cross3(R1, R2), C1 = cross3(R2, R0), C2 = cross3(R0, R1);
    const T d = dot3(R0, C0);
    const T id = rcp_rn(d);
    const T A[3][3] = {{C0.x * id, C1.x * id, C2.x * id}, {C0.y * id, C1.y * id, C2.y * id},
                       {C0.z * id, C1.z * id, C2.z * id}};
    const T wd = (d < T(0) ? -d : d) * T(1.0 / 6.0);
    // D[i][b]: lambda_0 = 1 - sum xi, lambda_b = xi_{b-1}
    const T Dm[3][4] = {{T(-1), T(1), T(0), T(0)}, {T(-1), T(0), T(1), T(0)}, {T(-1), T(0), T(0), T(1)}};
    Vec3<T> Gn[4];
#pragma unroll
    for (int b = 0; b < 4; ++b)
        Gn[b] = {A[0][0] * Dm[0][b] + A[0][1] * Dm[1][b] + A[0][2] * Dm[2][b],
                 A[1][0] * Dm[0][b] + A[1][1] * Dm[1][b] + A[1][2] * Dm[2][b],
                 A[2][0] * Dm[0][b] + A[2][1] * Dm[1][b] + A[2][2] * Dm[2][b]};
    const Vec3<T> ga = select4(Gn, a);
    // natural derivatives of node a: (-1, -1, -1) for node 0, the unit vector e_{a-1} otherwise
    T Da[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) Da[k] = a == 0 ? T(-1) : (a == k + 1 ? T(1) : T(0));
    dx[0] = dx[1] = dx[2] = T(0);
    dlam = dmu = T(0);
    T phi, Pm[9];
    point_shares<4, T>(W, ga, Gn, a, lam, mu, wd, phi, Pm, dlam, dmu);
    phi = group_sum<4, T>(phi);
#pragma unroll
    for (int n = 0; n < 9; ++n) Pm[n] = group_sum<4, T>(Pm[n]);
    add_dx(A, phi, Pm, wd, Da, dx);
    dlam = group_sum<4, T>(dlam);
    dmu = group_sum<4, T>(dmu);
}

// The thread's blocks of the symmetric DOF upstream, read from G at the CSR
// positions of its element's entries.  Node row R (the pair's node with the
// larger global id) of length L gives DOF row 3R + r at 9 rowptr[R] - 3R +
// r 3 (L - 1) + r (r + 1) / 2; node column C at in-row position p gives DOF
// columns 3p + j (C != R) or 3 (L - 1) + j (the diagonal block, j <= r).
// db[j] = 9 rowptr[g] - 3 g and rl[j] = the node row length of closure node j
// (closure-local indices ascend with the global id).
template <int NPE, typename T>
__device__ __forceinline__ void load_upstream(const T *__restrict__ G, const uint8_t *pos, const int64_t *db,
                                              const int32_t *rl, const uint16_t (&ln)[NPE], int a,
                                              T (&W)[elastic_nblk<NPE>()][9]) {
    int la = ln[0];
#pragma unroll
    for (int k = 1; k < NPE; ++k)
        if (a == k) la = ln[k];
#pragma unroll
    for (int m = 0; m < elastic_nblk<NPE>(); ++m) {
#pragma unroll
        for (int n = 0; n < 9; ++n) W[m][n] = T(0);
        if (!blk_valid<NPE>(a, m)) continue;
        const int b = blk_node<NPE>(a, m);
        int lb = ln[0];
#pragma unroll
        for (int k = 1; k < NPE; ++k)
            if (b == k) lb = ln[k];
        const int A = a > b ? a : b, B = a > b ? b : a;
        const int q = A * (A + 1) / 2 + B;
        const int lr = la > lb ? la : lb;
        const int64_t base = db[lr];
        const int L = rl[lr];
        if (a == b) {
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j <= i; ++j) {
                    const T v = __ldg(G + base + i * 3 * (L - 1) + i * (i + 1) / 2 + 3 * (L - 1) + j);
                    W[m][3 * i + j] = i == j ? v : T(0.5) * v;
                    W[m][3 * j + i] = W[m][3 * i + j];
                }
        } else {
            const int p = pos[q];
            const bool row_a = la > lb;  // else the block is stored transposed, in row b
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    const T v = T(0.5) * __ldg(G + base + r * 3 * (L - 1) + r * (r + 1) / 2 + 3 * p + j);
                    if (row_a) W[m][3 * r + j] = v; else W[m][3 * j + r] = v;
                }
        }
    }
}

struct ElVjpSmem {
    size_t xs, cown, db, rl, dxs, total;  // dxs: owned-node accumulators (fused) or the
                                          // compacted element list (staged)
};

// One element of a closure on its NPE lanes (all lanes of the warp call it: the
// brick shuffles): lane a gets dx_a, and dlam, dmu summed over the element.
template <int NPE, typename T, typename S, typename CT>
__device__ __forceinline__ void elastic_element_vjp(const PlanView &pv, const CT *__restrict__ c,
                                                    const T *__restrict__ G,
                                                    const S (*xs)[3], const int64_t *db, const int32_t *rl,
                                                    int pos_stride,
                                                    bool act, int64_t ci, int a, uint16_t (&ln)[NPE], int64_t &e,
                                                    T (&dx)[3], T &dlam, T &dmu) {
    S xc[NPE][3];
    T lam = T(0), mu = T(0);
    T W[elastic_nblk<NPE>()][9];
    e = 0;
    if (act) {
        e = pv.celem_id[ci];
#pragma unroll
        for (int k = 0; k < NPE; ++k) ln[k] = pv.celem_lnode[ci * NPE + k];
        lam = T(c[2 * e]);
        mu = T(c[2 * e + 1]);
        load_upstream<NPE, T>(G, pv.celem_pos + ci * pos_stride, db, rl, ln, a, W);
    } else {
#pragma unroll
        for (int k = 0; k < NPE; ++k) ln[k] = 0;
#pragma unroll
        for (int m = 0; m < elastic_nblk<NPE>(); ++m)
#pragma unroll
            for (int n = 0; n < 9; ++n) W[m][n] = T(0);
    }
#pragma unroll
    for (int k = 0; k < NPE; ++k) {
        xc[k][0] = xs[ln[k]][0];
        xc[k][1] = xs[ln[k]][1];
        xc[k][2] = xs[ln[k]][2];
    }
    if constexpr (NPE == 8) elastic_brick_vjp<T, S>(xc, lam, mu, W, dx, dlam, dmu);
    else elastic_tet_vjp<T, S>(xc, lam, mu, W, dx, dlam, dmu);
}

template <typename S>
__device__ __forceinline__ void load_cnodes(const PlanView &pv, const int64_t *__restrict__ rowptr, int64_t cb,
                                            int ncn, const S *__restrict__ X, S (*xs)[3], int32_t *cown, int64_t *db,
                                            int32_t *rl) {
    // ids first, then their rows and coordinates, CH nodes in flight per thread
    constexpr int CH = 4;
    const int tid = threadIdx.x, nthr = blockDim.x;
    for (int j0 = 0; j0 < ncn; j0 += CH * nthr) {
        int32_t gv[CH], ov[CH];
#pragma unroll
        for (int u = 0; u < CH; ++u) {
            const int j = j0 + u * nthr + tid;
            gv[u] = j < ncn ? pv.cnode_gid[cb + j] : 0;
            ov[u] = j < ncn ? pv.cnode_own[cb + j] : -1;
        }
        int64_t r0[CH], r1[CH];
        S xv[CH][3];
#pragma unroll
        for (int u = 0; u < CH; ++u) {
            const int j = j0 + u * nthr + tid;
            const int64_t g = gv[u];
            r0[u] = j < ncn ? rowptr[g] : 0;
            r1[u] = j < ncn ? rowptr[g + 1] : 0;
            xv[u][0] = j < ncn ? X[3 * g + 0] : S(0);
            xv[u][1] = j < ncn ? X[3 * g + 1] : S(0);
            xv[u][2] = j < ncn ? X[3 * g + 2] : S(0);
        }
#pragma unroll
        for (int u = 0; u < CH; ++u) {
            const int j = j0 + u * nthr + tid;
            if (j < ncn) {
                db[j] = 9 * r0[u] - 3 * (int64_t)gv[u];
                rl[j] = (int)(r1[u] - r0[u]);
                cown[j] = ov[u];
                xs[j][0] = xv[u][0];
                xs[j][1] = xv[u][1];
                xs[j][2] = xv[u][2];
            }
        }
    }
}

template <int NPE, typename T, typename S, typename CT>
__global__ void __launch_bounds__(256) k_elastic_vjp(PlanView pv, const int64_t *__restrict__ rowptr,
                                                     const S *__restrict__ X, const CT *__restrict__ c,
                                                     const T *__restrict__ G, T *__restrict__ dX,
                                                     T *__restrict__ dcout, int pos_stride, ElVjpSmem L,
                                                     int *status) {
    extern __shared__ __align__(16) unsigned char evjp_smem[];
    S(*xs)[3] = reinterpret_cast<S(*)[3]>(evjp_smem + L.xs);
    int32_t *cown = reinterpret_cast<int32_t *>(evjp_smem + L.cown);
    int64_t *db = reinterpret_cast<int64_t *>(evjp_smem + L.db);
    int32_t *rl = reinterpret_cast<int32_t *>(evjp_smem + L.rl);
    T(*dxs)[3] = reinterpret_cast<T(*)[3]>(evjp_smem + L.dxs);
    const int tid = threadIdx.x, nthr = blockDim.x, a = tid % NPE, epb = nthr / NPE;
    for (int64_t p = blockIdx.x; p < pv.n_patches; p += gridDim.x) {
        const int64_t nb = pv.patch_node_ptr[p];
        const int nown = (int)(pv.patch_node_ptr[p + 1] - nb);
        const int64_t cb = pv.patch_cnode_ptr[p];
        const int ncn = (int)(pv.patch_cnode_ptr[p + 1] - cb);
        const int64_t eb = pv.patch_elem_ptr[p];
        const int nel = (int)(pv.patch_elem_ptr[p + 1] - eb);
        load_cnodes<S>(pv, rowptr, cb, ncn, X, xs, cown, db, rl);
        for (int k = tid; k < nown; k += nthr) dxs[k][0] = dxs[k][1] = dxs[k][2] = T(0);
        __syncthreads();
        // the loop bound is uniform over the block: every lane takes part in the
        // element's shuffles on every pass
        for (int base = 0; base < nel; base += epb) {
            const int i = base + tid / NPE;
            const bool act = i < nel;
            const int64_t ci = eb + i;
            const int mycol = act ? (int)pv.celem_color[ci] : -1;
            uint16_t ln[NPE];
            int64_t e;
            T dx[3], dlam, dmu;
            elastic_element_vjp<NPE, T, S, CT>(pv, c, G, xs, db, rl, pos_stride, act, ci, a, ln, e, dx, dlam,
                                               dmu);
            uint16_t lna = ln[0];
#pragma unroll
            for (int k = 1; k < NPE; ++k)
                if (a == k) lna = ln[k];
            if (act && a == 0 && cown[ln[0]] >= 0) {
                dcout[2 * e] = dlam;
                dcout[2 * e + 1] = dmu;
                if (!isfinite(dlam) || !isfinite(dmu)) atomicOr(status, STATUS_NONFINITE);  // e.g. zero det J
            }
            const int last = min(base + epb, nel) - 1;
            const int c0 = pv.celem_color[eb + base], c1 = pv.celem_color[eb + last];
            for (int cc = c0; cc <= c1; ++cc) {
                if (mycol == cc) {
                    const int o = cown[lna];
                    if (o >= 0) {
                        dxs[o][0] += dx[0];
                        dxs[o][1] += dx[1];
                        dxs[o][2] += dx[2];
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

// Staged pass 1: every element once (its instance in the patch that owns its
// first node), node gradients to dxe [n_elems][NPE][3] -- lane a writes node a's
// three -- and (dL/dlambda_e, dL/dmu_e) to dc.  Pass 2 is the scalar operators'
// gather (vjp.cu).
template <int NPE, typename T, typename S, typename CT>
__global__ void __launch_bounds__(256) k_elastic_vjp_elem(PlanView pv, const int64_t *__restrict__ rowptr,
                                                          const S *__restrict__ X, const CT *__restrict__ c,
                                                          const T *__restrict__ G, T *__restrict__ dxe,
                                                          T *__restrict__ dcout, int pos_stride, ElVjpSmem L,
                                                     int *status) {
    extern __shared__ __align__(16) unsigned char evje_smem[];
    __shared__ int n_prim;
    S(*xs)[3] = reinterpret_cast<S(*)[3]>(evje_smem + L.xs);
    int32_t *cown = reinterpret_cast<int32_t *>(evje_smem + L.cown);
    int64_t *db = reinterpret_cast<int64_t *>(evje_smem + L.db);
    int32_t *rl = reinterpret_cast<int32_t *>(evje_smem + L.rl);
    int32_t *list = reinterpret_cast<int32_t *>(evje_smem + L.dxs);
    const int tid = threadIdx.x, nthr = blockDim.x, a = tid % NPE, epb = nthr / NPE;
    for (int64_t p = blockIdx.x; p < pv.n_patches; p += gridDim.x) {
        const int64_t cb = pv.patch_cnode_ptr[p];
        const int ncn = (int)(pv.patch_cnode_ptr[p + 1] - cb);
        const int64_t eb = pv.patch_elem_ptr[p];
        const int nel = (int)(pv.patch_elem_ptr[p + 1] - eb);
        load_cnodes<S>(pv, rowptr, cb, ncn, X, xs, cown, db, rl);
        if (tid == 0) n_prim = 0;
        __syncthreads();
        // compaction with one counter update per warp (see k_vjp_elem)
        for (int j0 = 0; j0 < nel; j0 += nthr) {
            const int j = j0 + tid, lane = tid & 31;
            const bool f = j < nel && cown[pv.celem_lnode[(eb + j) * NPE]] >= 0;
            const unsigned bal = __ballot_sync(0xffffffffu, f);
            int w0 = 0;
            if (lane == 0 && bal) w0 = atomicAdd(&n_prim, __popc(bal));
            w0 = __shfl_sync(0xffffffffu, w0, 0);
            if (f) list[w0 + __popc(bal & ((1u << lane) - 1u))] = j;
        }
        __syncthreads();
        const int np = n_prim;
        for (int base = 0; base < np; base += epb) {  // uniform bound: see k_elastic_vjp
            const int i = base + tid / NPE;
            const bool act = i < np;
            const int64_t ci = eb + (act ? list[i] : 0);
            uint16_t ln[NPE];
            int64_t e;
            T dx[3], dlam, dmu;
            elastic_element_vjp<NPE, T, S, CT>(pv, c, G, xs, db, rl, pos_stride, act, ci, a, ln, e, dx, dlam,
                                               dmu);
            if (act) {
                T *o = dxe + e * (NPE * 3) + 3 * a;
                o[0] = dx[0];
                o[1] = dx[1];
                o[2] = dx[2];
                if (a == 0) {
                    dcout[2 * e] = dlam;
                    dcout[2 * e + 1] = dmu;
                    if (!isfinite(dlam) || !isfinite(dmu)) atomicOr(status, STATUS_NONFINITE);  // e.g. zero det J
                }
            }
        }
        __syncthreads();
    }
}

fem_status vjp_scratch(fem_mesh m, bool fp64, void **dxe);
fem_status launch_vjp_gather(fem_mesh m, bool fp64, const void *dxe, void *dX, cudaStream_t s);

static size_t ev_a16(size_t v) { return (v + 15) & ~(size_t)15; }

template <int NPE, typename T, typename S, typename CT>
static fem_status launch_elastic_vjp_t(fem_mesh m, const Closure &cl, const void *X, const void *c, const void *G,
                                       void *dX, void *dc, void *dxe, cudaStream_t s) {
    const Plan &P = m->plan;
    const bool staged = dxe != nullptr;
    ElVjpSmem L{};
    size_t o = 0;
    L.xs = o;
    o = ev_a16(o + (size_t)P.max_cnodes * 3 * sizeof(S));
    L.cown = o;
    o = ev_a16(o + (size_t)P.max_cnodes * 4);
    L.db = o;
    o = ev_a16(o + (size_t)P.max_cnodes * 8);
    L.rl = o;
    o = ev_a16(o + (size_t)P.max_cnodes * 4);
    L.dxs = o;
    o = ev_a16(o + (staged ? (size_t)std::max<int64_t>(cl.max_celems, P.max_celems) * 4
                           : (size_t)P.max_own * 3 * sizeof(T)));
    L.total = o;
    auto f = staged ? k_elastic_vjp_elem<NPE, T, S, CT> : k_elastic_vjp<NPE, T, S, CT>;
    FEM_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total));
    int per_sm = 0;
    FEM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, 256, L.total));
    if (per_sm < 1) {
        set_error("elasticity backward kernel cannot be resident with %zu bytes of shared memory", L.total);
        return FEM_ERR_UNSUPPORTED;
    }
    const int64_t np = cl.p1 - cl.p0;
    if (np <= 0) return FEM_OK;
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(np, (int64_t)num_sms() * per_sm));
    f<<<grid, 256, L.total, s>>>(P.view(cl), m->rowptr.ptr, (const S *)X, (const CT *)c, (const T *)G,
                                 (T *)(staged ? dxe : dX), (T *)dc, P.pos_stride, L, m->status.ptr);
    FEM_LAUNCHED(staged ? "k_elastic_vjp_elem" : "k_elastic_vjp");
    return FEM_OK;
}

static fem_status launch_elastic_vjp_group(fem_mesh m, const Closure &cl, bool mixed, const void *X, fem_dtype xd,
                                           const void *c, fem_dtype cd, const void *G, void *dX, void *dc, void *dxe,
                                           cudaStream_t s) {
#define FEM_EV(NPE, T, S, CT) return launch_elastic_vjp_t<NPE, T, S, CT>(m, cl, X, c, G, dX, dc, dxe, s)
    if (!mixed) {
        if (m->npe == 8) FEM_EV(8, double, double, double);
        FEM_EV(4, double, double, double);
    }
    if (m->npe == 8) {
        if (xd == FEM_F32 && cd == FEM_F32) FEM_EV(8, float, float, float);
        if (xd == FEM_F32 && cd == FEM_F64) FEM_EV(8, float, float, double);
        if (xd == FEM_F64 && cd == FEM_F32) FEM_EV(8, float, double, float);
        FEM_EV(8, float, double, double);
    }
    if (xd == FEM_F32 && cd == FEM_F32) FEM_EV(4, float, float, float);
    if (xd == FEM_F32 && cd == FEM_F64) FEM_EV(4, float, float, double);
    if (xd == FEM_F64 && cd == FEM_F32) FEM_EV(4, float, double, float);
    FEM_EV(4, float, double, double);
#undef FEM_EV
}

// Staged (element pass, then the gather) when the library memory for the node
// gradients is granted, else the fused kernel.
fem_status launch_elastic_vjp(fem_mesh m, bool mixed, const void *X, fem_dtype xd, const void *c, fem_dtype cd,
                              const void *G, void *dX, void *dc, cudaStream_t s) {
    void *dxe = nullptr;
    const fem_status st = vjp_scratch(m, !mixed, &dxe);
    if (st != FEM_OK && st != FEM_ERR_BUDGET) return st;
    FEM_TRY(for_each_group(m, s, [&](const Closure &cl) {
        return launch_elastic_vjp_group(m, cl, mixed, X, xd, c, cd, G, dX, dc, dxe, s);
    }));
    return dxe ? launch_vjp_gather(m, !mixed, dxe, dX, s) : FEM_OK;
}

}  // namespace fem
