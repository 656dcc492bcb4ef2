// elastic.cu -- the numeric kernels of the elasticity operator (three DOFs per
// node, Algorithm 1's DOFxn = 3; element arithmetic in elastic.cuh) and the
// expansion of the node pattern into the DOF pattern.
//
// The global matrix is the lower triangle of the 3N x 3N matrix, DOF 3g + i being
// component i of node g.  Its pattern follows from the node pattern: node row I
// with lower columns J_0 < ... < J_{L-1} = I gives DOF rows 3I + r (r = 0, 1, 2)
// with columns 3 J_s + j (s < L - 1, j = 0..2) and then 3I + j (j <= r).  So the
// plan of the scalar operator serves unchanged: one accumulator slot per node
// pair holds its 3x3 block, and a patch's owned node rows become 3 DOF rows each,
// consecutive in the output (row 3I starts at 9 rowptr[I] - 3I).
//
// k_elastic_patch: one block per patch as in k_patch (numeric.cu): closure node
//   coordinates staged in shared memory, each closure element integrated by
//   NPE threads (one block row each), blocks added into the owned slots colour
//   by colour on the same mbarrier phases, each owned node's 3 DOF rows written
//   once.  With FUSED false it assembles given packed element matrices instead.
// k_elastic_integrate: packed lower k_e (78 or 300 entries) per element.
#include "elastic.cuh"
#include "mesh.cuh"
#include "numeric.cuh"
#include "phases.cuh"

namespace fem {

static constexpr int EL_INT_THREADS = 128;

template <typename F>
static fem_status el_set_smem(F *f, size_t bytes) {
    FEM_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    return FEM_OK;
}

static size_t el_align16(size_t v) { return (v + 15) & ~(size_t)15; }

// The thread's blocks of its element (node a = threadIdx.x % NPE; see elastic.cuh).
template <int NPE, typename T, typename S, bool MIXED>
__device__ __forceinline__ void elastic_blocks(const S (*xc)[3], T lam, T mu, int a, float thr, bool fp64_det,
                                               T (&k)[elastic_nblk<NPE>()][9]) {
    if constexpr (NPE == 8) elastic_brick_blocks<T, S>(xc, lam, mu, k);
    else elastic_tet_row<T, S, MIXED>(xc, lam, mu, a, thr, fp64_det, k);
}

// --------------------------------------------------------- k_elastic_integrate
template <int NPE, typename T, typename S, typename CT, bool MIXED>
__global__ void __launch_bounds__(EL_INT_THREADS) k_elastic_integrate(const int32_t *__restrict__ E, int64_t nel,
                                                                      const S *__restrict__ X,
                                                                      const CT *__restrict__ c, T *__restrict__ ke_out,
                                                                      float thr, unsigned mode, int *status) {
    constexpr int NPK = elastic_np(NPE);
    constexpr int EPB = EL_INT_THREADS / NPE;
    const int a = threadIdx.x % NPE;
    const bool fp64_det = (mode & FP64_DETS) != 0;
    // the loop bound is uniform over the block, so every lane takes part in the
    // brick's shuffles on every pass
    for (int64_t e0 = (int64_t)blockIdx.x * EPB; e0 < nel; e0 += (int64_t)gridDim.x * EPB) {
        const int64_t e = e0 + threadIdx.x / NPE;
        const bool act = e < nel;
        S xc[NPE][3];
        T lam = T(0), mu = T(0);
        if (act) {
#pragma unroll
            for (int b = 0; b < NPE; ++b) {
                const int64_t g = E[e * NPE + b];
                xc[b][0] = __ldg(X + 3 * g + 0);
                xc[b][1] = __ldg(X + 3 * g + 1);
                xc[b][2] = __ldg(X + 3 * g + 2);
            }
            lam = T(__ldg(c + 2 * e));
            mu = T(__ldg(c + 2 * e + 1));
        } else {
#pragma unroll
            for (int b = 0; b < NPE; ++b) xc[b][0] = xc[b][1] = xc[b][2] = S(0);
        }
        T k[elastic_nblk<NPE>()][9];
        elastic_blocks<NPE, T, S, MIXED>(xc, lam, mu, a, thr, fp64_det, k);
        if (act) {
            if (status && !isfinite(k[0][0])) atomicOr(status, STATUS_NONFINITE);
            store_packed_blocks<NPE, T>(ke_out + e * NPK, a, k);
        }
    }
}

// ----------------------------------------------------------- k_elastic_patch
template <int NPE, typename AccT, typename S, typename CT, bool FUSED, bool MIXED, bool WIN>
__device__ __forceinline__ void elastic_patch_body(const PlanView &pv, const S *__restrict__ X,
                                                   const CT *__restrict__ c, const AccT *__restrict__ ke,
                                                   AccT *__restrict__ vals, float thr, int64_t p, const PatchSmem &L,
                                                   unsigned mode, uint64_t *mb, uint32_t &g, const WaitCtl &wc) {
    constexpr int NPK = elastic_np(NPE);
    extern __shared__ __align__(16) unsigned char el_smem[];
    AccT *acc = reinterpret_cast<AccT *>(el_smem + L.acc);
    S(*xs)[3] = reinterpret_cast<S(*)[3]>(el_smem + L.xs);
    int32_t *roff = reinterpret_cast<int32_t *>(el_smem + L.roff);
    int64_t *rps = reinterpret_cast<int64_t *>(el_smem + L.rps);
    int32_t *orow = reinterpret_cast<int32_t *>(el_smem + L.cown);
    int32_t *gid = reinterpret_cast<int32_t *>(el_smem + L.gid);
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nwarps = nthr >> 5;
    const int a = tid % NPE;        // the thread's block row
    const int epb = nthr / NPE;     // elements per batch
    const bool fp64_det = (mode & FP64_DETS) != 0;

    const int64_t nb = pv.patch_node_ptr[p];
    const int nown = (int)(pv.patch_node_ptr[p + 1] - nb);
    const int64_t cb = pv.patch_cnode_ptr[p];
    const int ncn = (int)(pv.patch_cnode_ptr[p + 1] - cb);
    const int64_t eb = pv.patch_elem_ptr[p];
    const int nel = (int)(pv.patch_elem_ptr[p + 1] - eb);
    const int nacc = pv.patch_acc[p];  // node-pair slots owned by the patch

    if constexpr (FUSED)
        for (int j = tid; j < ncn; j += nthr) gid[j] = pv.cnode_gid[cb + j];
    for (int k = tid; k < nown; k += nthr) {
        roff[k] = pv.own_acc[nb + k];
        rps[k] = pv.own_rowptr[nb + k];
        orow[k] = pv.own_row[nb + k];
    }
    if (tid == 0) roff[nown] = nacc;
    __syncthreads();
    if constexpr (FUSED) {
        for (int j = tid; j < ncn; j += nthr) {
            int64_t gn = gid[j];
            if (!FEM_IN_BOUNDS(gn >= 0 && gn < pv.n_nodes, wc.status)) gn = 0;
            xs[j][0] = __ldg(X + 3 * gn + 0);
            xs[j][1] = __ldg(X + 3 * gn + 1);
            xs[j][2] = __ldg(X + 3 * gn + 2);
        }
    }
    __syncthreads();

    const uint16_t *aidx16 = reinterpret_cast<const uint16_t *>(pv.celem_aidx);
    // Owned rows in windows [k0, k1) whose slots fit the accumulators (L.win): with
    // WIN false one window covers the patch; with WIN true (blocks that outgrow
    // shared memory: FP64, or patches planned larger than the limit) each window
    // takes one pass over the closure, and slots outside it are skipped.
    for (int k0 = 0; k0 < nown;) {
        int k1 = nown;
        if constexpr (WIN) {
            int hi = nown;
            k1 = k0 + 1;
            while (k1 < hi) {
                const int mid = (k1 + hi + 1) >> 1;
                if (roff[mid] - roff[k0] <= L.win) k1 = mid; else hi = mid - 1;
            }
        }
        const int s0 = WIN ? roff[k0] : 0, s1 = WIN ? roff[k1] : nacc;
        for (int i = tid; i < 9 * (s1 - s0); i += nthr) acc[i] = AccT(0);
        __syncthreads();
        for (int base = 0; base < nel; base += epb) {
            const int i = base + tid / NPE;
            const bool act = i < nel;
            const int64_t ci = eb + i;
            uint16_t ln[NPE];
            int mycol = -1;
            if (act) {
                load_lnodes<NPE>(pv.celem_lnode, ci, ln);
                mycol = pv.celem_color[ci];
            } else {
#pragma unroll
                for (int b = 0; b < NPE; ++b) ln[b] = 0;
            }
#pragma unroll
            for (int b = 0; b < NPE; ++b)
                if (!FEM_IN_BOUNDS(ln[b] < ncn || !act, wc.status)) ln[b] = 0;
            constexpr int NB = elastic_nblk<NPE>();
            AccT k[NB][9];
            if constexpr (FUSED) {
                S xc[NPE][3];
#pragma unroll
                for (int b = 0; b < NPE; ++b) {
                    xc[b][0] = xs[ln[b]][0];
                    xc[b][1] = xs[ln[b]][1];
                    xc[b][2] = xs[ln[b]][2];
                }
                AccT lam = AccT(0), mu = AccT(0);
                if (act) {
                    int64_t e = pv.celem_id[ci];
                    if (!FEM_IN_BOUNDS(e >= 0 && e < pv.n_elems, wc.status)) e = 0;
                    lam = AccT(__ldg(c + 2 * e));
                    mu = AccT(__ldg(c + 2 * e + 1));
                }
                elastic_blocks<NPE, AccT, S, MIXED>(xc, lam, mu, a, thr, fp64_det, k);
                if (act && !isfinite(k[0][0])) atomicOr(wc.status, STATUS_NONFINITE);
            } else {
                if (act) {
                    int64_t e = pv.celem_id[ci];
                    if (!FEM_IN_BOUNDS(e >= 0 && e < pv.n_elems, wc.status)) e = 0;
                    load_packed_blocks<NPE, AccT>(ke + e * NPK, a, k);
                } else {
#pragma unroll
                    for (int m = 0; m < NB; ++m)
#pragma unroll
                        for (int n = 0; n < 9; ++n) k[m][n] = AccT(0);
                }
            }
            // accumulator slots of the thread's pairs (a, b) (scratch for rows the
            // patch does not own), and whether the pair's row is node b's: closure
            // nodes are numbered in ascending global order, so g_a < g_b exactly when
            // ln[a] < ln[b], and then the block goes in transposed
            int slot[NB];
            bool trans[NB];
            const uint16_t lna = NPE == 8 ? (a & 4 ? (a & 2 ? (a & 1 ? ln[7] : ln[6]) : (a & 1 ? ln[5] : ln[4]))
                                                   : (a & 2 ? (a & 1 ? ln[3] : ln[2]) : (a & 1 ? ln[1] : ln[0])))
                                          : (a & 2 ? (a & 1 ? ln[3] : ln[2]) : (a & 1 ? ln[1] : ln[0]));
#pragma unroll
            for (int m = 0; m < NB; ++m) {
                const int b = blk_node<NPE>(a, m);
                // ln[b]: the partner's lane holds it as its own (bricks), or b is m
                uint16_t lnb;
                if constexpr (NPE == 8) lnb = (uint16_t)__shfl_sync(0xffffffffu, (int)lna, (lane & ~7) + b);
                else lnb = ln[m];
                trans[m] = lna < lnb;
                slot[m] = -1;
                if (act && blk_valid<NPE>(a, m)) {
                    const int A = a > b ? a : b, B = a > b ? b : a;
                    const int q = A * (A + 1) / 2 + B;
                    int t = aidx16[((int64_t)(q >> 1) * pv.aidx_n + ci) * 2 + (q & 1)];
                    // scratch targets (rows of other patches) to the window's scratch,
                    // owned slots outside the window skipped
                    if constexpr (WIN) t = t >= L.trash ? L.win + (t - L.trash) : (t >= s0 && t < s1 ? t - s0 : -1);
                    if (!FEM_IN_BOUNDS(t < L.acc_cap, wc.status)) t = -1;
                    slot[m] = t;
                }
            }
            const int last = min(base + epb, nel) - 1;
            const int c0 = pv.celem_color[eb + base], c1 = pv.celem_color[eb + last];
            if (wc.stall == 1 && base == 0 && warp == 0) phase_wait(mb, g, wc);
            for (int cc = c0; cc <= c1; ++cc, ++g) {
                const bool mine = mycol == cc;
                if (__any_sync(0xffffffffu, mine)) {
                    if (g > 0) phase_wait(mb, g - 1, wc);
                    if (mine) {
#pragma unroll
                        for (int m = 0; m < NB; ++m) {
                            if (slot[m] < 0) continue;
                            AccT *dst = acc + 9 * slot[m];
                            if (blk_node<NPE>(a, m) == a) {
                                // diagonal block: its lower half (i >= j) only
                                AccT o0 = dst[0], o3 = dst[3], o4 = dst[4], o6 = dst[6], o7 = dst[7], o8 = dst[8];
                                dst[0] = o0 + k[m][0];
                                dst[3] = o3 + k[m][3];
                                dst[4] = o4 + k[m][4];
                                dst[6] = o6 + k[m][6];
                                dst[7] = o7 + k[m][7];
                                dst[8] = o8 + k[m][8];
                            } else {
                                const bool tr = trans[m];
                                AccT old[9];
#pragma unroll
                                for (int n = 0; n < 9; ++n) old[n] = dst[n];
#pragma unroll
                                for (int i3 = 0; i3 < 3; ++i3)
#pragma unroll
                                    for (int j3 = 0; j3 < 3; ++j3)
                                        dst[3 * i3 + j3] = old[3 * i3 + j3] + (tr ? k[m][3 * j3 + i3] : k[m][3 * i3 + j3]);
                            }
                        }
                    }
                    __syncwarp();
                }
                if (g >= (uint32_t)PHASE_RING) phase_wait(mb, g - PHASE_RING, wc);
                if (lane == 0) phase_arrive(mb, g);
            }
        }
        __syncthreads();  // every phase of the window done

        // each owned node's 3 DOF rows, one contiguous range of vals, by one warp:
        // DOF row r holds the node row's off-diagonal blocks' row r, then the
        // diagonal block's entries (r, 0..r)
        for (int k = k0 + warp; k < k1; k += nwarps) {
            const int o0 = roff[k] - s0, len = roff[k + 1] - roff[k];
            const int off3 = 3 * (len - 1);
            const int64_t out0 = 9 * rps[k] - 3 * (int64_t)orow[k];
            int total = 9 * len - 3;
            if (!FEM_IN_BOUNDS(o0 >= 0 && len >= 1 && o0 + len <= L.acc_cap && out0 >= 0 && out0 + total <= pv.nnz,
                               wc.status))
                total = 0;
            for (int f = lane; f < total; f += 32) {
                const int r = f < off3 + 1 ? 0 : (f < 2 * off3 + 3 ? 1 : 2);
                const int s = f - (r == 0 ? 0 : (r == 1 ? off3 + 1 : 2 * off3 + 3));
                const int src = s < off3 ? 9 * (o0 + s / 3) + 3 * r + s % 3 : 9 * (o0 + len - 1) + 3 * r + (s - off3);
                vals[out0 + f] = acc[src];
            }
        }
        __syncthreads();
        k0 = k1;
    }
}

// Launch bounds: FP32 bricks up to 512 threads at 128 registers (2 blocks of 256
// or 1 of 512 per SM); FP32 tetrahedra 256 threads, 3 blocks per SM; FP64 256
// threads, one block (its 72 double accumulators need the registers).
template <int NPE, typename AccT>
__host__ __device__ constexpr int elastic_max_threads() {
    return (sizeof(AccT) == 4 && NPE == 8) ? 512 : 256;
}
template <int NPE, typename AccT>
__host__ __device__ constexpr int elastic_min_blocks() {
    return sizeof(AccT) == 8 ? 1 : (NPE == 8 ? 1 : 3);
}

template <int NPE, typename AccT, typename S, typename CT, bool FUSED, bool MIXED, bool WIN>
__global__ void __launch_bounds__(elastic_max_threads<NPE, AccT>(), elastic_min_blocks<NPE, AccT>())
    k_elastic_patch(PlanView pv, const S *__restrict__ X, const CT *__restrict__ c, const AccT *__restrict__ ke,
                    AccT *__restrict__ vals, float thr, int64_t p0, int64_t p1, PatchSmem L, unsigned mode,
                    WaitCtl wc) {
    __shared__ uint64_t mb[PHASE_RING];
    phase_init(mb);
    uint32_t g = 0;
    for (int64_t p = p0 + blockIdx.x; p < p1; p += gridDim.x)
        elastic_patch_body<NPE, AccT, S, CT, FUSED, MIXED, WIN>(pv, X, c, ke, vals, thr, p, L, mode, mb, g, wc);
}

// Persistent kernel over the patches of many meshes (as k_patch_batched): work
// item w is patch w - prefix[m] of mesh m.
template <int NPE, typename AccT, bool MIXED, bool WIN>
__global__ void __launch_bounds__(elastic_max_threads<NPE, AccT>(), elastic_min_blocks<NPE, AccT>())
    k_elastic_patch_batched(const BatchItem *__restrict__ items, const int64_t *__restrict__ prefix, int n,
                            PatchSmem L, unsigned mode, WaitCtl wc) {
    const int64_t total = prefix[n];
    __shared__ uint64_t mb[PHASE_RING];
    phase_init(mb);
    uint32_t g = 0;
    for (int64_t w = blockIdx.x; w < total; w += gridDim.x) {
        int lo = 0, hi = n;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (prefix[mid] <= w) lo = mid; else hi = mid;
        }
        const BatchItem &it = items[lo];
        elastic_patch_body<NPE, AccT, AccT, AccT, true, MIXED, WIN>(it.pv, (const AccT *)it.X, (const AccT *)it.c,
                                                                    nullptr, (AccT *)it.vals, it.thr, w - prefix[lo],
                                                                    L, mode, mb, g, wc);
    }
}

// ------------------------------------------------------------------- launch
PatchSmem elastic_smem_layout(const PlanMax &P, bool fused, bool mixed, size_t xsize, int win) {
    PatchSmem L{};
    const size_t accsz = mixed ? sizeof(float) : sizeof(double);
    size_t o = 0;
    L.acc = o;
    L.win = win;
    L.trash = (int)P.max_acc;
    L.acc_cap = win + ACC_SCRATCH;
    o = el_align16(o + (size_t)9 * (win + ACC_SCRATCH) * accsz);
    L.xs = o;
    if (fused) o = el_align16(o + (size_t)P.max_cnodes * 3 * xsize);
    L.roff = o;
    o = el_align16(o + (size_t)(P.max_own + 1) * sizeof(int32_t));
    L.rps = o;
    o = el_align16(o + (size_t)P.max_own * sizeof(int64_t));
    L.cown = o;  // global ids of the owned nodes
    o = el_align16(o + (size_t)P.max_own * sizeof(int32_t));
    L.gid = o;
    if (fused) o = el_align16(o + (size_t)P.max_cnodes * sizeof(int32_t));
    L.hv = L.hvf = L.eid = L.cvs = o;
    L.hv_on = 0;
    L.wg_shift = 5;
    L.total = o;
    return L;
}

// Threads per block: bricks default to 512 (one block per SM holding a 4096-pair
// patch), tetrahedra to 256 (three blocks per SM).
int elastic_window(const PlanMax &P, bool fused, bool mixed, size_t xsize, size_t limit) {
    // the layout with no owned slots (scratch and staging arrays), then whole slots
    const size_t rest = elastic_smem_layout(P, fused, mixed, xsize, 0).total;
    const size_t per_slot = 9 * (mixed ? sizeof(float) : sizeof(double));
    if (rest + 16 >= limit) return 0;
    const int64_t fit = (int64_t)((limit - rest - 16) / per_slot);
    const int win = (int)std::min<int64_t>(P.max_acc, fit);
    return win >= 256 || win == P.max_acc ? win : 0;  // a row has at most 255 entries
}

int elastic_threads(int npe, int requested) {
    const int t = requested > 0 ? requested : (npe == 8 ? 512 : 256);
    return std::min(npe == 8 ? 512 : 256, std::max(32, (t + 31) / 32 * 32));
}

int elastic_blocks_per_sm(int npe, int threads) {
    int n = 0;
    cudaError_t e = npe == 8
        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_elastic_patch<8, float, float, float, true, true, false>,
                                                        threads, 0)
        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_elastic_patch<4, float, float, float, true, true, false>,
                                                        threads, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 2;
    }
    return std::max(1, n);
}

template <int NPE, typename AccT, typename S, typename CT, bool FUSED, bool MIXED>
static fem_status launch_elastic_patch_t(const PatchArgs &a, cudaStream_t s) {
    const Plan &P = *a.plan;
    const Closure &cl = a.closure ? *a.closure : P.full;
    PlanMax pm;
    pm.add(P);
    int dev = 0, max_optin = 0;
    FEM_CUDA(cudaGetDevice(&dev));
    FEM_CUDA(cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    cudaFuncAttributes fa{};
    FEM_CUDA(cudaFuncGetAttributes(&fa, k_elastic_patch<NPE, AccT, S, CT, FUSED, MIXED, true>));
    // the dynamic part shares the opt-in limit with the static mbarrier ring
    const int win = elastic_window(pm, FUSED, MIXED, sizeof(S), (size_t)max_optin - fa.sharedSizeBytes);
    if (win <= 0) {
        set_error("the closure of a patch does not fit in shared memory (limit %d bytes); lower patch_entries",
                  max_optin);
        return FEM_ERR_UNSUPPORTED;
    }
    const PatchSmem L = elastic_smem_layout(pm, FUSED, MIXED, sizeof(S), win);
    auto f = win >= pm.max_acc ? k_elastic_patch<NPE, AccT, S, CT, FUSED, MIXED, false>
                               : k_elastic_patch<NPE, AccT, S, CT, FUSED, MIXED, true>;
    FEM_TRY(el_set_smem(f, L.total));
    const int threads = std::min(elastic_threads(NPE, a.threads), elastic_max_threads<NPE, AccT>());
    int per_sm = 0;
    FEM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, threads, L.total));
    if (per_sm < 1) {
        set_error("elastic patch kernel cannot be resident with %d threads and %zu bytes of shared memory", threads,
                  L.total);
        return FEM_ERR_UNSUPPORTED;
    }
    if (a.blocks_per_sm > 0 && a.blocks_per_sm < per_sm) per_sm = a.blocks_per_sm;
    const int64_t np = cl.p1 - cl.p0;
    if (np <= 0) return FEM_OK;
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(np, (int64_t)num_sms() * per_sm));
    PlanView pv = P.view(cl);
    pv.nnz = 9 * P.nnz - 3 * P.n_nodes;  // the DOF matrix's entries (bounds of the debug build)
    f<<<grid, threads, L.total, s>>>(pv, (const S *)a.X, (const CT *)a.c, (const AccT *)a.ke, (AccT *)a.vals, a.thr, 0,
                                     np, L, a.mode, a.wait);
    FEM_LAUNCHED("k_elastic_patch");
    return FEM_OK;
}

fem_status launch_elastic_patch(const PatchArgs &a, cudaStream_t s) {
#define FEM_E(NPE, ACC, S, CT, FU, MX) return launch_elastic_patch_t<NPE, ACC, S, CT, FU, MX>(a, s)
    if (!a.mixed) {
        if (a.fused) {
            if (a.npe == 8) FEM_E(8, double, double, double, true, false);
            FEM_E(4, double, double, double, true, false);
        }
        if (a.npe == 8) FEM_E(8, double, double, double, false, false);
        FEM_E(4, double, double, double, false, false);
    }
    if (!a.fused) {
        if (a.npe == 8) FEM_E(8, float, float, float, false, true);
        FEM_E(4, float, float, float, false, true);
    }
    if (a.npe == 8) {
        if (a.xd == FEM_F32 && a.cd == FEM_F32) FEM_E(8, float, float, float, true, true);
        if (a.xd == FEM_F32 && a.cd == FEM_F64) FEM_E(8, float, float, double, true, true);
        if (a.xd == FEM_F64 && a.cd == FEM_F32) FEM_E(8, float, double, float, true, true);
        FEM_E(8, float, double, double, true, true);
    }
    if (a.xd == FEM_F32 && a.cd == FEM_F32) FEM_E(4, float, float, float, true, true);
    if (a.xd == FEM_F32 && a.cd == FEM_F64) FEM_E(4, float, float, double, true, true);
    if (a.xd == FEM_F64 && a.cd == FEM_F32) FEM_E(4, float, double, float, true, true);
    FEM_E(4, float, double, double, true, true);
#undef FEM_E
}

template <int NPE, typename AccT, bool MIXED>
static fem_status elastic_batched_config_t(const PlanMax &pm, int threads, int blocks_per_sm, BatchLaunch *out) {
    int dev = 0, max_optin = 0;
    FEM_CUDA(cudaGetDevice(&dev));
    FEM_CUDA(cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    cudaFuncAttributes fa{};
    FEM_CUDA(cudaFuncGetAttributes(&fa, k_elastic_patch_batched<NPE, AccT, MIXED, true>));
    const int win = elastic_window(pm, true, MIXED, sizeof(AccT), (size_t)max_optin - fa.sharedSizeBytes);
    if (win <= 0) {
        set_error("a patch of the batch does not fit in shared memory (limit %d bytes)", max_optin);
        return FEM_ERR_UNSUPPORTED;
    }
    const PatchSmem L = elastic_smem_layout(pm, true, MIXED, sizeof(AccT), win);
    const bool use_win = win < pm.max_acc;
    auto f = use_win ? k_elastic_patch_batched<NPE, AccT, MIXED, true> : k_elastic_patch_batched<NPE, AccT, MIXED, false>;
    FEM_TRY(el_set_smem(f, L.total));
    threads = std::min(threads, elastic_max_threads<NPE, AccT>());
    int per_sm = 0;
    FEM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, threads, L.total));
    if (per_sm < 1) {
        set_error("batched elasticity kernel cannot be resident with %d threads", threads);
        return FEM_ERR_UNSUPPORTED;
    }
    if (blocks_per_sm > 0 && blocks_per_sm < per_sm) per_sm = blocks_per_sm;
    out->L = L;
    out->threads = threads;
    out->grid = num_sms() * per_sm;
    out->elastic = true;
    out->win = use_win;
    return FEM_OK;
}

fem_status elastic_batched_config(int npe, bool mixed, const PlanMax &pm, int threads, int blocks_per_sm,
                                  BatchLaunch *out) {
    out->npe = npe;
    out->mixed = mixed;
    if (mixed) return npe == 8 ? elastic_batched_config_t<8, float, true>(pm, threads, blocks_per_sm, out)
                               : elastic_batched_config_t<4, float, true>(pm, threads, blocks_per_sm, out);
    return npe == 8 ? elastic_batched_config_t<8, double, false>(pm, threads, blocks_per_sm, out)
                    : elastic_batched_config_t<4, double, false>(pm, threads, blocks_per_sm, out);
}

fem_status launch_elastic_batched_kernel(const BatchLaunch &bl, cudaStream_t s) {
#define FEM_EB(NPE, T, MX, W)                                                                                 \
    k_elastic_patch_batched<NPE, T, MX, W><<<bl.grid, bl.threads, bl.L.total, s>>>(bl.items, bl.prefix, bl.n, \
                                                                                    bl.L, bl.mode, bl.wait)
    if (bl.mixed) {
        if (bl.npe == 8) {
            if (bl.win) FEM_EB(8, float, true, true); else FEM_EB(8, float, true, false);
        } else {
            if (bl.win) FEM_EB(4, float, true, true); else FEM_EB(4, float, true, false);
        }
    } else {
        if (bl.npe == 8) {
            if (bl.win) FEM_EB(8, double, false, true); else FEM_EB(8, double, false, false);
        } else {
            if (bl.win) FEM_EB(4, double, false, true); else FEM_EB(4, double, false, false);
        }
    }
#undef FEM_EB
    FEM_LAUNCHED("k_elastic_patch_batched");
    return FEM_OK;
}

template <int NPE, typename T, typename S, typename CT, bool MIXED>
static fem_status launch_elastic_integrate_t(const IntegrateArgs &a, cudaStream_t s) {
    auto f = k_elastic_integrate<NPE, T, S, CT, MIXED>;
    int per_sm = 0;
    FEM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, EL_INT_THREADS, 0));
    if (per_sm < 1) per_sm = 1;
    const int64_t tiles = cdiv(a.nel, EL_INT_THREADS / NPE);
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)num_sms() * per_sm * 4));
    f<<<grid, EL_INT_THREADS, 0, s>>>(a.E, a.nel, (const S *)a.X, (const CT *)a.c, (T *)a.ke, a.thr, a.mode,
                                       a.status);
    FEM_LAUNCHED("k_elastic_integrate");
    return FEM_OK;
}

fem_status launch_elastic_integrate(const IntegrateArgs &a, cudaStream_t s) {
    if (a.nel <= 0) return FEM_OK;
#define FEM_EI(NPE, T, S, CT, MX) return launch_elastic_integrate_t<NPE, T, S, CT, MX>(a, s)
    if (!a.mixed) {
        if (a.npe == 8) FEM_EI(8, double, double, double, false);
        FEM_EI(4, double, double, double, false);
    }
    if (a.npe == 8) {
        if (a.xd == FEM_F32 && a.cd == FEM_F32) FEM_EI(8, float, float, float, true);
        if (a.xd == FEM_F32 && a.cd == FEM_F64) FEM_EI(8, float, float, double, true);
        if (a.xd == FEM_F64 && a.cd == FEM_F32) FEM_EI(8, float, double, float, true);
        FEM_EI(8, float, double, double, true);
    }
    if (a.xd == FEM_F32 && a.cd == FEM_F32) FEM_EI(4, float, float, float, true);
    if (a.xd == FEM_F32 && a.cd == FEM_F64) FEM_EI(4, float, float, double, true);
    if (a.xd == FEM_F64 && a.cd == FEM_F32) FEM_EI(4, float, double, float, true);
    FEM_EI(4, float, double, double, true);
#undef FEM_EI
}

// ------------------------------------------------------------- DOF pattern
// One thread per node row I: DOF row pointers 3I .. 3I + 2 and their columns.
__global__ void k_dof_pattern(const int64_t *__restrict__ rowptr, const int32_t *__restrict__ col, int64_t n,
                              int64_t *__restrict__ rowptr3, int32_t *__restrict__ col3) {
    for (int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; I < n; I += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = rowptr[I], len = rowptr[I + 1] - b;
        const int64_t o = 9 * b - 3 * I;
        int64_t pos = o;
        for (int r = 0; r < 3; ++r) {
            if (rowptr3) rowptr3[3 * I + r] = pos;
            if (col3) {
                for (int64_t s = 0; s + 1 < len; ++s)
                    for (int j = 0; j < 3; ++j) col3[pos + 3 * s + j] = (int32_t)(3 * col[b + s] + j);
                for (int j = 0; j <= r; ++j) col3[pos + 3 * (len - 1) + j] = (int32_t)(3 * I + j);
            }
            pos += 3 * (len - 1) + r + 1;
        }
        if (rowptr3 && I == n - 1) rowptr3[3 * n] = pos;
    }
}

fem_status launch_dof_pattern(const int64_t *rowptr, const int32_t *col, int64_t n, int64_t *rowptr3, int32_t *col3,
                              cudaStream_t s) {
    if (n <= 0) {
        if (rowptr3) FEM_CUDA(cudaMemsetAsync(rowptr3, 0, sizeof(int64_t), s));
        return FEM_OK;
    }
    const unsigned grid = (unsigned)std::min<int64_t>(cdiv(n, 256), (int64_t)num_sms() * 8);
    k_dof_pattern<<<grid, 256, 0, s>>>(rowptr, col, n, rowptr3, col3);
    FEM_LAUNCHED("k_dof_pattern");
    return FEM_OK;
}

}  // namespace fem
