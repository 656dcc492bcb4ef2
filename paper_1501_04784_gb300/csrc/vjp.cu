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
// here from X; nothing is stored by the forward pass.
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
// element's first node.  No atomics; bitwise reproducible.
#include "element.cuh"
#include "mesh.cuh"

namespace fem {

// Brick: packed upstream Sp[36] -> node gradients dx[8][3] and dc.
template <typename T, typename S>
__device__ __forceinline__ void brick_vjp(const S (*xc)[3], T c, const T (&Sp)[36], T (&dx)[8][3], T &dc) {
    Vec3<T> e[3][2][2];
    brick_edges<T, S>(xc, e);
    Vec3<T> row[3][2][2];
    brick_jrows(e, row);
    T Ss[8][8];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b <= a; ++b) {
            const T v = Sp[a * (a + 1) / 2 + b];
            Ss[a][b] = a == b ? v : T(0.5) * v;
            Ss[b][a] = Ss[a][b];
        }
#pragma unroll
    for (int a = 0; a < 8; ++a) dx[a][0] = dx[a][1] = dx[a][2] = T(0);
    dc = T(0);
    const T P = T(FEM_GP), Q = T(FEM_GQ);
#pragma unroll 1
    for (int q = 0; q < 8; ++q) {
        const int q1 = q >> 2, q2 = (q >> 1) & 1, q3 = q & 1;
        // true Jacobian rows (the stored rows are 2J)
        Vec3<T> R = row[0][q2][q3], Sv = row[1][q1][q3], U = row[2][q1][q2];
        R = {T(0.5) * R.x, T(0.5) * R.y, T(0.5) * R.z};
        Sv = {T(0.5) * Sv.x, T(0.5) * Sv.y, T(0.5) * Sv.z};
        U = {T(0.5) * U.x, T(0.5) * U.y, T(0.5) * U.z};
        const Vec3<T> C0 = cross3(Sv, U), C1 = cross3(U, R), C2 = cross3(R, Sv);
        const T d = dot3(R, C0);
        const T ad = d < T(0) ? -d : d;
        // A = J^{-1}: A[i][j] = C_j[i] / d
        const T id = T(1) / d;
        T A[3][3] = {{C0.x * id, C1.x * id, C2.x * id}, {C0.y * id, C1.y * id, C2.y * id},
                     {C0.z * id, C1.z * id, C2.z * id}};
        const T iad = T(1) / ad;
        T M[3][3];
        M[0][0] = dot3(C0, C0) * iad; M[1][1] = dot3(C1, C1) * iad; M[2][2] = dot3(C2, C2) * iad;
        M[0][1] = M[1][0] = dot3(C0, C1) * iad;
        M[0][2] = M[2][0] = dot3(C0, C2) * iad;
        M[1][2] = M[2][1] = dot3(C1, C2) * iad;
        // natural derivatives at q: D[i][a]
        T D[3][8];
#pragma unroll
        for (int a = 0; a < 8; ++a) {
            const int a1 = hb1(a), a2 = hb2(a), a3 = hb3(a);
            const T f1 = a1 == q1 ? P : Q, f2 = a2 == q2 ? P : Q, f3 = a3 == q3 ? P : Q;
            D[0][a] = T(0.5 * hsig(a1)) * f2 * f3;
            D[1][a] = T(0.5 * hsig(a2)) * f1 * f3;
            D[2][a] = T(0.5 * hsig(a3)) * f1 * f2;
        }
        // H = D Ss D^T
        T V[3][8];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int b = 0; b < 8; ++b) {
                T s = T(0);
#pragma unroll
                for (int a = 0; a < 8; ++a) s += D[i][a] * Ss[a][b];
                V[i][b] = s;
            }
        T H[3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                T s = T(0);
#pragma unroll
                for (int b = 0; b < 8; ++b) s += V[i][b] * D[j][b];
                H[i][j] = s;
            }
        T f = T(0);
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) f += M[i][j] * H[i][j];
        dc += f;
        // G = c (f I - 2 M H) A^T
        T W[3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                T s = T(0);
#pragma unroll
                for (int l = 0; l < 3; ++l) s += M[i][l] * H[l][k];
                W[i][k] = (i == k ? f : T(0)) - T(2) * s;
            }
        T G[3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                T s = T(0);
#pragma unroll
                for (int k = 0; k < 3; ++k) s += W[i][k] * A[j][k];
                G[i][j] = c * s;
            }
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
            for (int j = 0; j < 3; ++j) dx[a][j] += D[0][a] * G[0][j] + D[1][a] * G[1][j] + D[2][a] * G[2][j];
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
    const T id = T(1) / d;
    T A[3][3] = {{C0.x * id, C1.x * id, C2.x * id}, {C0.y * id, C1.y * id, C2.y * id},
                 {C0.z * id, C1.z * id, C2.z * id}};
    const T w = T(1) / (T(6) * ad);
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
        const T id = T(1) / d;
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
    const T id = T(1) / d;
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

template <int NPE, typename T, typename S, typename CT>
__global__ void __launch_bounds__(256) k_vjp(PlanView pv, const int64_t *__restrict__ rowptr,
                                             const S *__restrict__ X, const CT *__restrict__ c,
                                             const T *__restrict__ G, T *__restrict__ dX, T *__restrict__ dcout,
                                             VjpSmem L, bool mass) {
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
                if (mass) {
                    if constexpr (NPE == 8) brick_mass_vjp<T, S>(xc, (T)c[e], Sp, dx, dcv);
                    else tet_mass_vjp<T, S>(xc, (T)c[e], Sp, dx, dcv);
                } else {
                    if constexpr (NPE == 8) brick_vjp<T, S>(xc, (T)c[e], Sp, dx, dcv);
                    else tet_vjp<T, S>(xc, (T)c[e], Sp, dx, dcv);
                }
                if (cown[ln[0]] >= 0) dcout[e] = dcv;
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
    auto f = k_vjp<NPE, T, S, CT>;
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
                                 (T *)dc, L, m->opt.operator_kind == 1);
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
    size_t xs, cown, gid, list, total;
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
    for (int j = threadIdx.x; j < nel; j += blockDim.x)
        if (cown[pv.celem_lnode[(eb + j) * npe]] >= 0) list[atomicAdd(count, 1)] = j;
    __syncthreads();
    return *count;
}

template <int NPE, typename T, typename S, typename CT>
__global__ void __launch_bounds__(256) k_vjp_elem(PlanView pv, const int64_t *__restrict__ rowptr,
                                                  const S *__restrict__ X, const CT *__restrict__ c,
                                                  const T *__restrict__ G, T *__restrict__ dxe,
                                                  T *__restrict__ dcout, ElemSmem L, bool mass) {
    constexpr int NP = NPE * (NPE + 1) / 2;
    extern __shared__ __align__(16) unsigned char vel_smem[];
    __shared__ int n_prim;
    S(*xs)[3] = reinterpret_cast<S(*)[3]>(vel_smem + L.xs);
    int32_t *cown = reinterpret_cast<int32_t *>(vel_smem + L.cown);
    int32_t *gid = reinterpret_cast<int32_t *>(vel_smem + L.gid);
    int32_t *list = reinterpret_cast<int32_t *>(vel_smem + L.list);
    const int tid = threadIdx.x, nthr = blockDim.x;
    for (int64_t p = blockIdx.x; p < pv.n_patches; p += gridDim.x) {
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
        const int np = primary_elems(pv, NPE, eb, nel, cown, list, &n_prim);
        for (int k = tid; k < np; k += nthr) {
            const int64_t ci = eb + list[k];
            const int64_t e = pv.celem_id[ci];
            int ln[NPE];
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
            T dx[NPE][3], dcv;
            if (mass) {
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
        }
        __syncthreads();
    }
}

struct GatherSmem {
    size_t cown, dxs, total;
};

template <int NPE, typename T>
__global__ void __launch_bounds__(256) k_vjp_gather(PlanView pv, const T *__restrict__ dxe, T *__restrict__ dX,
                                                    GatherSmem L) {
    extern __shared__ __align__(16) unsigned char vg_smem[];
    int32_t *cown = reinterpret_cast<int32_t *>(vg_smem + L.cown);
    T(*dxs)[3] = reinterpret_cast<T(*)[3]>(vg_smem + L.dxs);
    const int tid = threadIdx.x, nthr = blockDim.x;
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
            if (i < nel) {
                const int64_t ci = eb + i;
                mycol = pv.celem_color[ci];
                const int64_t e = pv.celem_id[ci];
                const T *src = dxe + e * (NPE * 3);
#pragma unroll
                for (int a = 0; a < NPE; ++a) {
                    own[a] = cown[pv.celem_lnode[ci * NPE + a]];
#pragma unroll
                    for (int j = 0; j < 3; ++j) v[a][j] = own[a] >= 0 ? src[3 * a + j] : T(0);
                }
            }
            const int last = min(base + nthr, nel) - 1;
            const int c0 = pv.celem_color[eb + base], c1 = pv.celem_color[eb + last];
            for (int cc = c0; cc <= c1; ++cc) {
                if (mycol == cc) {
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
    L.gid = o;
    o = a16(o + (size_t)P.max_cnodes * 4);
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
    auto f = k_vjp_elem<NPE, T, S, CT>;
    FEM_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total));
    const int64_t np = cl.p1 - cl.p0;
    if (np <= 0) return FEM_OK;
    fem_status st;
    const int grid = grid_for((const void *)f, 256, L.total, np, "backward element kernel", &st);
    if (st != FEM_OK) return st;
    f<<<grid, 256, L.total, s>>>(P.view(cl), m->rowptr.ptr, (const S *)X, (const CT *)c, (const T *)G, (T *)dxe,
                                 (T *)dc, L, m->opt.operator_kind == 1);
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
    f<<<grid, 256, L.total, s>>>(P.view(cl), (const T *)dxe, (T *)dX, L);
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
