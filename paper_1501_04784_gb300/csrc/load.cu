// load.cu -- global load vector of a per-element constant source s_e:
// F_n = sum over elements e containing node n of f_e,a, f_e,a = s_e * integral N_a
// (Section 1, steps (ii)-(iii) of the FEM procedure of Fig. 1: the local load vectors f_e and their assembly into F).
//
// Bricks use the same 2x2x2 Gauss rule and |det J| as the stiffness matrix, with the
// sum factorised over the axes; tetrahedra take |T| / 4 per node.  In mixed
// precision the element arithmetic is FP32 and distorted elements take FP64-accurate
// determinants, as for k_e.  Assembly is owner-computes on the patch plan: the block
// of a patch adds its closure elements' node values into shared-memory accumulators
// of its owned nodes colour by colour (a fixed order, no atomics) and writes each
// owned node's F once.
//
// With NC = 3 (the elasticity operator, three DOFs per node) the source is a
// per-element body force b_e (3 components) and F[3n + i] = sum_e b_e,i integral N_a:
// the same integrals of N_a, times each component.
#include "element.cuh"
#include "mesh.cuh"
#include "numeric.cuh"

namespace fem {

struct LoadSmem {
    size_t xs, cown, gid, fs, total;
};

template <int NPE, typename T, typename S, typename CT, bool MIXED, int NC>
__global__ void __launch_bounds__(256) k_load(PlanView pv, const S *__restrict__ X, const CT *__restrict__ src,
                                              T *__restrict__ F, float thr, bool fp64_det, LoadSmem L) {
    extern __shared__ __align__(16) unsigned char load_smem[];
    S(*xs)[3] = reinterpret_cast<S(*)[3]>(load_smem + L.xs);
    int32_t *cown = reinterpret_cast<int32_t *>(load_smem + L.cown);
    T *fs = reinterpret_cast<T *>(load_smem + L.fs);
    const int tid = threadIdx.x, nthr = blockDim.x;
    for (int64_t p = blockIdx.x; p < pv.n_patches; p += gridDim.x) {
        const int64_t nb = pv.patch_node_ptr[p];
        const int nown = (int)(pv.patch_node_ptr[p + 1] - nb);
        const int64_t cb = pv.patch_cnode_ptr[p];
        const int ncn = (int)(pv.patch_cnode_ptr[p + 1] - cb);
        const int64_t eb = pv.patch_elem_ptr[p];
        const int nel = (int)(pv.patch_elem_ptr[p + 1] - eb);
        for (int j = tid; j < ncn; j += nthr) {
            const int64_t g = pv.cnode_gid[cb + j];
            cown[j] = pv.cnode_own[cb + j];
            xs[j][0] = X[3 * g + 0];
            xs[j][1] = X[3 * g + 1];
            xs[j][2] = X[3 * g + 2];
        }
        for (int k = tid; k < NC * nown; k += nthr) fs[k] = T(0);
        __syncthreads();
        for (int base = 0; base < nel; base += nthr) {
            const int i = base + tid;
            const int64_t ci = eb + i;
            int mycol = -1;
            int ln[NPE];
            T fe[NPE];
            T b[NC];
            if (i < nel) {
                mycol = pv.celem_color[ci];
                const int64_t e = pv.celem_id[ci];
                // scalar: the source scales the integrals; vector: integrals of N_a
                // alone, each component applied at the scatter
#pragma unroll
                for (int k = 0; k < NC; ++k) b[k] = (T)src[NC * e + k];
                const T s = NC == 1 ? b[0] : T(1);
                S xc[NPE][3];
#pragma unroll
                for (int a = 0; a < NPE; ++a) {
                    ln[a] = pv.celem_lnode[ci * NPE + a];
                    xc[a][0] = xs[ln[a]][0];
                    xc[a][1] = xs[ln[a]][1];
                    xc[a][2] = xs[ln[a]][2];
                }
                if constexpr (NPE == 8) {
                    T det[8];
                    brick_gauss_dets<T, S>(xc, thr, MIXED, det);
                    brick_load_from_dets(det, s, fe);
                } else {
                    T det;
                    if constexpr (MIXED) {
                        Vec3<float> Fv[4];
                        float d;
                        tet_geometry_mixed<S>(xc, thr, fp64_det, Fv, d);
                        det = d;
                    } else {
                        TetGeom<T> g;
                        tet_geom<T, S>(xc, g);
                        Vec3<T> Fv[4];
                        tet_faces(g, Fv, det);
                    }
                    const T share = s * (det < T(0) ? -det : det) * T(1.0 / 24.0);
#pragma unroll
                    for (int a = 0; a < 4; ++a) fe[a] = share;
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
                            if constexpr (NC == 1) {
                                fs[o] += fe[a];
                            } else {
#pragma unroll
                                for (int k = 0; k < NC; ++k) fs[NC * o + k] += b[k] * fe[a];
                            }
                        }
                    }
                }
                __syncthreads();
            }
        }
        for (int k = tid; k < NC * nown; k += nthr) F[NC * (int64_t)pv.own_row[nb + k / NC] + k % NC] = fs[k];
        __syncthreads();
    }
}

static size_t al16(size_t v) { return (v + 15) & ~(size_t)15; }

template <int NPE, typename T, typename S, typename CT, bool MIXED, int NC>
static fem_status launch_load_t(fem_mesh m, const Closure &cl, const void *X, const void *src, void *F, float thr,
                                bool fp64_det, cudaStream_t s) {
    const Plan &P = m->plan;
    LoadSmem L{};
    size_t o = 0;
    L.xs = o;
    o = al16(o + (size_t)P.max_cnodes * 3 * sizeof(S));
    L.cown = o;
    o = al16(o + (size_t)P.max_cnodes * 4);
    L.gid = o;
    L.fs = o;
    o = al16(o + (size_t)NC * P.max_own * sizeof(T));
    L.total = o;
    auto f = k_load<NPE, T, S, CT, MIXED, NC>;
    FEM_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total));
    int per_sm = 0;
    FEM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, 256, L.total));
    if (per_sm < 1) {
        set_error("load-vector kernel cannot be resident with %zu bytes of shared memory", L.total);
        return FEM_ERR_UNSUPPORTED;
    }
    const int64_t np = cl.p1 - cl.p0;
    if (np <= 0) return FEM_OK;
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(np, (int64_t)num_sms() * per_sm));
    f<<<grid, 256, L.total, s>>>(P.view(cl), (const S *)X, (const CT *)src, (T *)F, thr, fp64_det, L);
    FEM_LAUNCHED("k_load");
    return FEM_OK;
}

static fem_status launch_load_group(fem_mesh m, const Closure &cl, bool mixed, const void *X, fem_dtype xd,
                                    const void *src, fem_dtype sd, void *F, float thr, bool fp64_det,
                                    cudaStream_t s) {
#define FEM_L(NPE, T, S, CT, MX)                                                                  \
    return m->opt.operator_kind == 2 ? launch_load_t<NPE, T, S, CT, MX, 3>(m, cl, X, src, F, thr, fp64_det, s) \
                                     : launch_load_t<NPE, T, S, CT, MX, 1>(m, cl, X, src, F, thr, fp64_det, s)
    if (!mixed) {
        if (m->npe == 8) FEM_L(8, double, double, double, false);
        FEM_L(4, double, double, double, false);
    }
    if (m->npe == 8) {
        if (xd == FEM_F32 && sd == FEM_F32) FEM_L(8, float, float, float, true);
        if (xd == FEM_F32 && sd == FEM_F64) FEM_L(8, float, float, double, true);
        if (xd == FEM_F64 && sd == FEM_F32) FEM_L(8, float, double, float, true);
        FEM_L(8, float, double, double, true);
    }
    if (xd == FEM_F32 && sd == FEM_F32) FEM_L(4, float, float, float, true);
    if (xd == FEM_F32 && sd == FEM_F64) FEM_L(4, float, float, double, true);
    if (xd == FEM_F64 && sd == FEM_F32) FEM_L(4, float, double, float, true);
    FEM_L(4, float, double, double, true);
#undef FEM_L
}

fem_status launch_load(fem_mesh m, bool mixed, const void *X, fem_dtype xd, const void *src, fem_dtype sd, void *F,
                       float thr, bool fp64_det, cudaStream_t s) {
    return for_each_group(m, s, [&](const Closure &cl) {
        return launch_load_group(m, cl, mixed, X, xd, src, sd, F, thr, fp64_det, s);
    });
}

}  // namespace fem
