// numeric.cu -- the numeric kernels.
//
// k_integrate: Algorithm 2's kernel re-designed for sm_103a -- one thread per
//   element forms the packed lower k_e (Eqs. 7-9); the block stages its
//   elements' k_e in shared memory and writes them to HBM in one coalesced
//   stream.
// k_patch: integration fused with assembly (Eq. 6).  One block per patch of
//   owned rows (see mesh.cuh): node coordinates of the patch's closure are
//   gathered once into shared memory, every closure element is integrated by one
//   thread, its entries that fall in owned rows are added into shared-memory
//   accumulators colour by colour, and each owned row is written to HBM once.
//   The same kernel assembles given element matrices when FUSED is false.
#include "elem_ops.cuh"
#include "mesh.cuh"
#include "numeric.cuh"
#include "phases.cuh"

namespace fem {

// One element's packed k_e from the staged element matrices, in the widest
// vector loads its alignment allows (a row of 36 floats or of 10 or 36 doubles is
// a whole number of 16-byte units; a row of 10 floats, of 8-byte units).
template <int NP, typename T>
__device__ __forceinline__ void load_packed(const T *__restrict__ src, T (&kv)[NP]) {
    if constexpr (sizeof(T) == 4 && (NP * 4) % 16 == 0) {
#pragma unroll
        for (int w = 0; w < NP / 4; ++w) {
            const float4 v = __ldg(reinterpret_cast<const float4 *>(src) + w);
            kv[4 * w] = v.x; kv[4 * w + 1] = v.y; kv[4 * w + 2] = v.z; kv[4 * w + 3] = v.w;
        }
    } else if constexpr (sizeof(T) == 4 && NP % 2 == 0) {
#pragma unroll
        for (int w = 0; w < NP / 2; ++w) {
            const float2 v = __ldg(reinterpret_cast<const float2 *>(src) + w);
            kv[2 * w] = v.x; kv[2 * w + 1] = v.y;
        }
    } else if constexpr (sizeof(T) == 8 && NP % 2 == 0) {
#pragma unroll
        for (int w = 0; w < NP / 2; ++w) {
            const double2 v = __ldg(reinterpret_cast<const double2 *>(src) + w);
            kv[2 * w] = v.x; kv[2 * w + 1] = v.y;
        }
    } else {
#pragma unroll
        for (int q = 0; q < NP; ++q) kv[q] = __ldg(src + q);
    }
}

// ------------------------------------------------------------- k_integrate
// One element per thread, grid-stride.  FP32 bricks: the thread stores its packed
// k_e as its own row with 16-byte vector stores (a row of 36 floats is nine of
// them), with no shared memory and no block-wide barrier, so one warp's
// coordinate gathers overlap the others' arithmetic (0.109 -> 0.099 ms on 1M
// bricks).  Other rows (10 floats, or doubles) go through shared memory and leave
// in one coalesced stream per block, which measured faster for them.
static constexpr int INT_THREADS = 128;

template <int NPE, typename T>
__host__ __device__ constexpr bool int_direct() { return NPE == 8 && sizeof(T) == 4; }
template <int NPE, typename T>
__host__ __device__ constexpr int int_min_blocks() { return int_direct<NPE, T>() ? 4 : 1; }

template <int NP>
__device__ __forceinline__ void store_row16(float *__restrict__ dst, const float (&kv)[NP]) {
#pragma unroll
    for (int w = 0; w < NP / 4; ++w)
        reinterpret_cast<float4 *>(dst)[w] = make_float4(kv[4 * w], kv[4 * w + 1], kv[4 * w + 2], kv[4 * w + 3]);
}

template <int NPE, typename T, typename S, typename CT, bool MIXED>
__global__ void __launch_bounds__(INT_THREADS, (int_min_blocks<NPE, T>())) k_integrate(
    const int32_t *__restrict__ E, int64_t nel, const S *__restrict__ X, const CT *__restrict__ c,
    T *__restrict__ ke_out, float thr, unsigned mode, unsigned long long *nflag, int *status) {
    constexpr int NP = ElemTraits<NPE>::NP;
    constexpr int LD = NP + 1;  // odd stride: conflict-free staging
    extern __shared__ __align__(16) unsigned char int_smem[];
    T *st = reinterpret_cast<T *>(int_smem);
    unsigned flagged = 0;
    for (int64_t e0 = (int64_t)blockIdx.x * INT_THREADS; e0 < nel; e0 += (int64_t)gridDim.x * INT_THREADS) {
        const int64_t e = e0 + threadIdx.x;
        if (e < nel) {
            int32_t g[NPE];
            load_ids<NPE>(E, e, g);
            S xc[NPE][3];
#pragma unroll
            for (int a = 0; a < NPE; ++a) {
                xc[a][0] = __ldg(X + 3 * (int64_t)g[a] + 0);
                xc[a][1] = __ldg(X + 3 * (int64_t)g[a] + 1);
                xc[a][2] = __ldg(X + 3 * (int64_t)g[a] + 2);
            }
            T k[NP];
            flagged += element_matrix<NPE, T, S, MIXED>(xc, __ldg(c + e), thr, mode, k) ? 1u : 0u;
            if (status && !isfinite(k[0])) atomicOr(status, STATUS_NONFINITE);
            if constexpr (int_direct<NPE, T>()) {
                store_row16<NP>(reinterpret_cast<float *>(ke_out + e * NP), k);
            } else {
#pragma unroll
                for (int p = 0; p < NP; ++p) st[threadIdx.x * LD + p] = k[p];
            }
        }
        if constexpr (!int_direct<NPE, T>()) {
            __syncthreads();
            const int nb = (int)min((int64_t)INT_THREADS, nel - e0);
            T *out = ke_out + e0 * NP;
            for (int idx = threadIdx.x; idx < nb * NP; idx += INT_THREADS) out[idx] = st[(idx / NP) * LD + idx % NP];
            __syncthreads();
        }
    }
    if (nflag) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) flagged += __shfl_down_sync(0xffffffffu, flagged, o);
        if ((threadIdx.x & 31) == 0 && flagged) atomicAdd(nflag, (unsigned long long)flagged);
    }
}

// Adds the owned entries of one element's packed k_e into the block's
// accumulators.  Each entry's target comes precomputed from the plan (two 16-bit
// targets per word, see PlanView::celem_aidx).  The accumulator reads of a group
// of entries are issued together before their writes, so a group costs one
// shared-memory round trip instead of one per entry; all entries of one element
// are distinct, so the reads of a group do not alias its writes.

template <int NPE, typename AccT, bool MIXED>
__device__ __forceinline__ void scatter_element(const uint32_t (&aw)[NPE * (NPE + 1) / 4], const int32_t *roff,
                                                void *hv, bool fp64_sums, AccT *acc,
                                                const AccT (&kv)[NPE * (NPE + 1) / 2], int acc_cap, int nown,
                                                int *status) {
    (void)acc_cap;
    (void)nown;
    (void)status;
    constexpr int NP = NPE * (NPE + 1) / 2;
    constexpr int G = 12;
#pragma unroll
    for (int g0 = 0; g0 < NP; g0 += G) {
        int idx[G];
#pragma unroll
        for (int j = 0; j < G; ++j) {
            const int q = g0 + j;
            idx[j] = -1;
            if (q < NP) {
                const uint32_t t = (aw[q >> 1] >> (16 * (q & 1))) & 0xffffu;
                const int a = tri_row(q);
                if (q == a * (a + 1) / 2 + a && t >= AIDX_HV) {
                    // a diagonal summed FP64-accurately
                    const int k = (int)(t & 0x7fffu);
                    if (!FEM_IN_BOUNDS(k < nown, status)) continue;
                    if constexpr (MIXED) {
                        if (fp64_sums) static_cast<double *>(hv)[k] += (double)kv[q];
                        else two_sum_acc(static_cast<float2 *>(hv)[k], (float)kv[q]);
                    } else {
                        idx[j] = roff[k + 1] - 1;  // the diagonal closes a lower row
                    }
                } else {
                    idx[j] = (int)t;  // owned entry, or the lane's scratch slot
                }
                if (idx[j] >= 0 && !FEM_IN_BOUNDS(idx[j] < acc_cap, status)) idx[j] = -1;
            }
        }
        AccT old[G];
#pragma unroll
        for (int j = 0; j < G; ++j)
            if (idx[j] >= 0) old[j] = acc[idx[j]];
#pragma unroll
        for (int j = 0; j < G; ++j)
            if (idx[j] >= 0) acc[idx[j]] = old[j] + kv[g0 + j < NP ? g0 + j : 0];
    }
}

// ------------------------------------------------------------------ k_patch
// One patch: owned rows' accumulators in shared memory, the closure integrated
// batch by batch and added colour by colour, each owned row written once.

// The closure's batches: every element integrated (FUSED) or loaded from the
// staged element matrices, its owned entries added colour by colour.  `after`
// runs once, after the first batch's elements are integrated and before its
// colour phases (the prefetching kernel issues its next copies there).
template <int NPE, typename AccT, typename S, typename CT, bool FUSED, bool MIXED, typename After>
__device__ __forceinline__ void patch_batches(const PlanView &pv, const S *__restrict__ X, const CT *__restrict__ c,
                                              const AccT *__restrict__ ke, float thr, int64_t eb, int nel, int ncn,
                                              int nown, const PatchSmem &L, unsigned mode, uint64_t *mb, uint32_t &g,
                                              const WaitCtl &wc, AccT *acc, double *hv, const S (*xs)[3],
                                              const int32_t *roff, After after) {
    constexpr int NP = ElemTraits<NPE>::NP;
    const bool fp64_sums = (mode & FP64_SUMS) != 0;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5;
    (void)X;
    (void)ncn;

    // Coefficients come through a two-stage register pipeline: element ids two
    // batches ahead, c one batch ahead, so the dependent loads overlap compute.
    int32_t eid_n2 = -1;
    CT c_n1 = CT(0);
    if constexpr (FUSED) {
        const int32_t e0 = tid < nel ? pv.celem_id[eb + tid] : -1;
        c_n1 = e0 >= 0 ? __ldg(c + e0) : CT(0);
        eid_n2 = tid + nthr < nel ? pv.celem_id[eb + tid + nthr] : -1;
    }
    // tets (short integration): closure-local node indices, colours and
    // accumulator targets of the next batch are loaded one batch ahead as well;
    // bricks load them in place
    uint16_t ln_n[NPE];
    uint32_t aw_n[NP / 2];
    int col_n = -1;
    if (NPE == 4 && tid < nel) {
        load_lnodes<NPE>(pv.celem_lnode, eb + tid, ln_n);
        col_n = pv.celem_color[eb + tid];
#pragma unroll
        for (int w = 0; w < NP / 2; ++w) aw_n[w] = __ldg(pv.celem_aidx + w * pv.aidx_n + eb + tid);
    }
    bool first = true;
    for (int base = 0; base < nel; base += nthr) {
        const int i = base + tid;
        const bool act = i < nel;
        const int64_t ci = eb + i;
        AccT kv[NP];
        uint16_t ln[NPE];
        uint32_t aw[NP / 2];
        int mycol = -1;
        if constexpr (NPE == 4) {
#pragma unroll
            for (int a = 0; a < NPE; ++a) ln[a] = ln_n[a];
#pragma unroll
            for (int w = 0; w < NP / 2; ++w) aw[w] = aw_n[w];
            if (act) mycol = col_n;
            if (i + nthr < nel) {
                load_lnodes<NPE>(pv.celem_lnode, ci + nthr, ln_n);
                col_n = pv.celem_color[ci + nthr];
#pragma unroll
                for (int w = 0; w < NP / 2; ++w) aw_n[w] = __ldg(pv.celem_aidx + w * pv.aidx_n + ci + nthr);
            }
        } else if (act) {
            load_lnodes<NPE>(pv.celem_lnode, ci, ln);
            mycol = pv.celem_color[ci];
        }
        CT ce = CT(0);
        if constexpr (FUSED) {
            ce = c_n1;
            if (!FEM_IN_BOUNDS(eid_n2 < pv.n_elems, wc.status)) eid_n2 = -1;
            c_n1 = eid_n2 >= 0 ? __ldg(c + eid_n2) : CT(0);
            const int i2 = i + 2 * nthr;
            eid_n2 = i2 < nel ? pv.celem_id[eb + i2] : -1;
        }
        if (act) {
            if constexpr (FUSED) {
                S xc[NPE][3];
#pragma unroll
                for (int a = 0; a < NPE; ++a) {
                    if (!FEM_IN_BOUNDS(ln[a] < ncn, wc.status)) ln[a] = 0;
                    xc[a][0] = xs[ln[a]][0];
                    xc[a][1] = xs[ln[a]][1];
                    xc[a][2] = xs[ln[a]][2];
                }
                element_matrix<NPE, AccT, S, MIXED>(xc, ce, thr, mode, kv);
                // k_00 (m_00) is positive and finite for any element of nonzero volume
                if (!isfinite(kv[0])) atomicOr(wc.status, STATUS_NONFINITE);
            } else {
                int64_t e = pv.celem_id[ci];
                if (!FEM_IN_BOUNDS(e >= 0 && e < pv.n_elems, wc.status)) e = 0;
                load_packed<NP>(ke + e * NP, kv);
            }
            // bricks: accumulator targets after the integration, before the colour
            // phases, so that no phase waits on its own load (tets take them a
            // batch ahead, above)
            if constexpr (NPE == 8) {
#pragma unroll
                for (int w = 0; w < NP / 2; ++w) aw[w] = __ldg(pv.celem_aidx + w * pv.aidx_n + ci);
            }
        }
        if (first) {
            after();
            first = false;
        }
        const int last = min(base + nthr, nel) - 1;
        const int c0 = pv.celem_color[eb + base], c1 = pv.celem_color[eb + last];
        // testing: phase g cannot complete while warp 0 waits before arriving at it
        if (wc.stall == 1 && base == 0 && warp == 0) phase_wait(mb, g, wc);
        for (int cc = c0; cc <= c1; ++cc, ++g) {
            const bool mine = mycol == cc;
            if (__any_sync(0xffffffffu, mine)) {
                if (g > 0) phase_wait(mb, g - 1, wc);
                if (mine) scatter_element<NPE, AccT, MIXED>(aw, roff, hv, fp64_sums, acc, kv, L.acc_cap, nown, wc.status);
                __syncwarp();
            }
            if (g >= (uint32_t)PHASE_RING) phase_wait(mb, g - PHASE_RING, wc);
            if (lane == 0) phase_arrive(mb, g);
        }
    }
    if (first) after();
}

// Each owned row to HBM once: a group of 2^wg_shift lanes (about one row
// length) stores one row, so a warp writes 32 >> wg_shift rows per step, each as
// one contiguous segment.  `hv_row(k)` tells whether row k's diagonal comes from
// its FP64-accurate sum.
template <typename AccT, bool MIXED, typename HvRow>
__device__ __forceinline__ void patch_writeout(const PlanView &pv, AccT *__restrict__ vals, int nown,
                                               const PatchSmem &L, unsigned mode, const WaitCtl &wc,
                                               const AccT *acc, const double *hv, const int32_t *roff,
                                               const int64_t *rps, int64_t rp_sub, HvRow hv_row) {
    const bool fp64_sums = (mode & FP64_SUMS) != 0;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nwarps = nthr >> 5;
    const int gsh = L.wg_shift, gsz = 1 << gsh;
    const int rows_step = nwarps << (5 - gsh);
    for (int k = (warp << (5 - gsh)) + (lane >> gsh); k < nown; k += rows_step) {
        int o0 = roff[k], len = roff[k + 1] - o0;
        const int64_t rp = rps[k] - rp_sub;
        if (!FEM_IN_BOUNDS(o0 >= 0 && len >= 0 && o0 + len <= L.acc_cap && rp >= 0 && rp + len <= pv.nnz, wc.status))
            len = 0;
        AccT *dst = vals + rp;
        const AccT *src = acc + o0;
        // the diagonal (last entry of a lower row) of a high-valence row comes
        // from its FP64-accurate sum instead
        int jd = -1;
        AccT vd = AccT(0);
        if (MIXED && hv_row(k)) {
            jd = len - 1;
            if (fp64_sums) vd = (AccT)hv[k];
            else {
                const float2 pr = reinterpret_cast<const float2 *>(hv)[k];
                vd = (AccT)(pr.x + pr.y);  // the pair rounded once
            }
        }
        for (int j = lane & (gsz - 1); j < len; j += gsz) dst[j] = j == jd ? vd : src[j];
    }
}

template <int NPE, typename AccT, typename S, typename CT, bool FUSED, bool MIXED>
__device__ __forceinline__ void patch_body(const PlanView &pv, const S *__restrict__ X, const CT *__restrict__ c,
                                           const AccT *__restrict__ ke, AccT *__restrict__ vals, float thr,
                                           int64_t p, const PatchSmem &L, unsigned mode, uint64_t *mb,
                                           uint32_t &g, const WaitCtl &wc) {
    extern __shared__ __align__(16) unsigned char patch_smem[];
    AccT *acc = reinterpret_cast<AccT *>(patch_smem + L.acc);
    double *hv = reinterpret_cast<double *>(patch_smem + L.hv);
    S(*xs)[3] = reinterpret_cast<S(*)[3]>(patch_smem + L.xs);
    int32_t *roff = reinterpret_cast<int32_t *>(patch_smem + L.roff);
    uint8_t *hvf = patch_smem + L.hvf;
    const int tid = threadIdx.x, nthr = blockDim.x;
    int64_t *rps = reinterpret_cast<int64_t *>(patch_smem + L.rps);
    int32_t *gid = reinterpret_cast<int32_t *>(patch_smem + L.gid);
    const int64_t nb = pv.patch_node_ptr[p];
    const int nown = (int)(pv.patch_node_ptr[p + 1] - nb);
    const int64_t cb = pv.patch_cnode_ptr[p];
    const int ncn = (int)(pv.patch_cnode_ptr[p + 1] - cb);
    const int64_t eb = pv.patch_elem_ptr[p];
    const int nel = (int)(pv.patch_elem_ptr[p + 1] - eb);
    const int nacc = pv.patch_acc[p];

    // Prologue, stage 1: the patch's contiguous plan arrays.  Loads go out in
    // chunks of CH per thread before their shared-memory stores, so each thread
    // has CH global loads in flight instead of one per round trip.
    constexpr int CH = 8;
    if constexpr (FUSED) {
        for (int j0 = 0; j0 < ncn; j0 += CH * nthr) {
            int32_t vg[CH];
#pragma unroll
            for (int k = 0; k < CH; ++k) {
                const int j = j0 + k * nthr + tid;
                vg[k] = j < ncn ? pv.cnode_gid[cb + j] : 0;
            }
#pragma unroll
            for (int k = 0; k < CH; ++k) {
                const int j = j0 + k * nthr + tid;
                if (j < ncn) gid[j] = vg[k];
            }
        }
    }
    for (int k0 = 0; k0 < nown; k0 += CH * nthr) {
        int32_t vr[CH];
        int64_t vp[CH];
        uint8_t vh[CH];
#pragma unroll
        for (int k = 0; k < CH; ++k) {
            const int kk = k0 + k * nthr + tid;
            vr[k] = kk < nown ? pv.own_acc[nb + kk] : 0;
            vp[k] = kk < nown ? pv.own_rowptr[nb + kk] - pv.val_off : 0;
            vh[k] = (MIXED && kk < nown) ? pv.own_hv[nb + kk] : 0;
        }
#pragma unroll
        for (int k = 0; k < CH; ++k) {
            const int kk = k0 + k * nthr + tid;
            if (kk < nown) {
                roff[kk] = vr[k];
                rps[kk] = vp[k];
                if constexpr (MIXED) {
                    if (L.hv_on) hv[kk] = 0.0;  // also clears the (hi, lo) float pair
                    hvf[kk] = vh[k];
                }
            }
        }
    }
    if (tid == 0) roff[nown] = nacc;
    {
        // accumulators cleared with 16-byte stores (acc starts the layout)
        constexpr int V = 16 / sizeof(AccT);
        float4 *a4 = reinterpret_cast<float4 *>(acc);
        for (int i = tid; i < nacc / V; i += nthr) a4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int i = nacc / V * V + tid; i < nacc; i += nthr) acc[i] = AccT(0);
    }
    __syncthreads();
    // Prologue, stage 2: node coordinates of the closure, gathered through the
    // staged ids, CH nodes (3 CH loads) in flight per thread.
    if constexpr (FUSED) {
        for (int j0 = 0; j0 < ncn; j0 += CH * nthr) {
            S v[CH][3];
#pragma unroll
            for (int k = 0; k < CH; ++k) {
                const int j = j0 + k * nthr + tid;
                int64_t g = j < ncn ? gid[j] : 0;
#ifdef FEM_DEBUG_BOUNDS
                // testing the checks: one planted out-of-range node id per block
                if (wc.stall == 2 && j == 0) g = pv.n_nodes;
#endif
                if (!FEM_IN_BOUNDS(g >= 0 && g < pv.n_nodes, wc.status)) g = 0;
                v[k][0] = j < ncn ? __ldg(X + 3 * g + 0) : S(0);
                v[k][1] = j < ncn ? __ldg(X + 3 * g + 1) : S(0);
                v[k][2] = j < ncn ? __ldg(X + 3 * g + 2) : S(0);
            }
#pragma unroll
            for (int k = 0; k < CH; ++k) {
                const int j = j0 + k * nthr + tid;
                if (j < ncn) {
                    xs[j][0] = v[k][0];
                    xs[j][1] = v[k][1];
                    xs[j][2] = v[k][2];
                }
            }
        }
    }
    __syncthreads();
    patch_batches<NPE, AccT, S, CT, FUSED, MIXED>(pv, X, c, ke, thr, eb, nel, ncn, nown, L, mode, mb, g, wc, acc, hv,
                                                  xs, roff, [] {});
    __syncthreads();  // every phase of the patch done
    patch_writeout<AccT, MIXED>(pv, vals, nown, L, mode, wc, acc, hv, roff, rps, 0,
                                [&](int k) { return hvf[k] != 0; });
    __syncthreads();
}

template <int NPE, typename AccT, typename S, typename CT, bool FUSED, bool MIXED>
__global__ void __launch_bounds__(patch_max_threads(NPE), patch_min_blocks(NPE)) k_patch(PlanView pv, const S *__restrict__ X,
                                                             const CT *__restrict__ c, const AccT *__restrict__ ke,
                                                             AccT *__restrict__ vals, float thr, int64_t p0,
                                                             int64_t p1, PatchSmem L, unsigned mode,
                                                             WaitCtl wc) {
    __shared__ uint64_t mb[PHASE_RING];
    phase_init(mb);
    uint32_t g = 0;
    for (int64_t p = p0 + blockIdx.x; p < p1; p += gridDim.x)
        patch_body<NPE, AccT, S, CT, FUSED, MIXED>(pv, X, c, ke, vals, thr, p, L, mode, mb, g, wc);
}

// ------------------------------------------------- k_patch with prefetch
// The fused kernel with the next patch's prologue overlapped: while a block
// works on patch p, asynchronous copies (cp.async, no registers held) bring the
// closure ids and owned-row tables of its next patch into a second set of
// shared-memory arrays, then, once those ids have arrived, the closure's
// coordinates.  Each thread gathers the coordinates of the ids it copied itself,
// so it only waits for its own copies; the block barrier that already precedes
// the write-out makes every thread's copies visible.  The patch then starts with
// its data in place (0.263 -> 0.248 ms on 1M bricks); the arithmetic and the
// order of every sum are those of k_patch.
__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

struct PrologueSet {
    int32_t *gid, *roff;
    int64_t *rps;
    unsigned char *xs;
};
__device__ __forceinline__ PrologueSet prologue_set(const PatchSmem &L, int k) {
    extern __shared__ __align__(16) unsigned char patch_smem[];
    return PrologueSet{reinterpret_cast<int32_t *>(patch_smem + (k ? L.gid2 : L.gid)),
                       reinterpret_cast<int32_t *>(patch_smem + (k ? L.roff2 : L.roff)),
                       reinterpret_cast<int64_t *>(patch_smem + (k ? L.rps2 : L.rps)), patch_smem + (k ? L.xs2 : L.xs)};
}

// First copies of patch p: its closure-node ids and owned-row tables.
__device__ __forceinline__ void prefetch_plan(const PlanView &pv, int64_t p, const PrologueSet &b) {
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int64_t nb = pv.patch_node_ptr[p];
    const int nown = (int)(pv.patch_node_ptr[p + 1] - nb);
    const int64_t cb = pv.patch_cnode_ptr[p];
    const int ncn = (int)(pv.patch_cnode_ptr[p + 1] - cb);
    for (int j = tid; j < ncn; j += nthr) cp_async4(b.gid + j, pv.cnode_gid + cb + j);
    for (int k = tid; k < nown; k += nthr) {
        cp_async4(b.roff + k, pv.own_acc + nb + k);
        cp_async8(b.rps + k, pv.own_rowptr + nb + k);
    }
    cp_async_commit();
}

// Second copies: the coordinates of the closure nodes whose ids this thread
// copied (it waits for its own earlier copies first).
template <typename S>
__device__ __forceinline__ void prefetch_coords(const PlanView &pv, int64_t p, const PrologueSet &b,
                                                const S *__restrict__ X, const WaitCtl &wc) {
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int64_t cb = pv.patch_cnode_ptr[p];
    const int ncn = (int)(pv.patch_cnode_ptr[p + 1] - cb);
    cp_async_wait_all();
    S(*xs)[3] = reinterpret_cast<S(*)[3]>(b.xs);
    for (int j = tid; j < ncn; j += nthr) {
        int64_t g = b.gid[j];
#ifdef FEM_DEBUG_BOUNDS
        // testing the checks: one planted out-of-range node id per block
        if (wc.stall == 2 && j == 0) g = pv.n_nodes;
#endif
        if (!FEM_IN_BOUNDS(g >= 0 && g < pv.n_nodes, wc.status)) g = 0;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            if constexpr (sizeof(S) == 4) cp_async4(&xs[j][k], X + 3 * g + k);
            else cp_async8(&xs[j][k], X + 3 * g + k);
        }
    }
    cp_async_commit();
}

template <int NPE, typename AccT, typename S, typename CT, bool MIXED>
__global__ void __launch_bounds__(patch_max_threads(NPE), patch_min_blocks(NPE)) k_patch_prefetch(
    PlanView pv, const S *__restrict__ X, const CT *__restrict__ c, AccT *__restrict__ vals, float thr, int64_t p0,
    int64_t p1, PatchSmem L, unsigned mode, WaitCtl wc) {
    extern __shared__ __align__(16) unsigned char patch_smem[];
    __shared__ uint64_t mb[PHASE_RING];
    phase_init(mb);
    AccT *acc = reinterpret_cast<AccT *>(patch_smem + L.acc);
    double *hv = reinterpret_cast<double *>(patch_smem + L.hv);
    const int tid = threadIdx.x, nthr = blockDim.x;
    uint32_t g = 0;
    int set = 0;
    int64_t p = p0 + blockIdx.x;
    if (p < p1) {
        const PrologueSet b = prologue_set(L, 0);
        prefetch_plan(pv, p, b);
        prefetch_coords<S>(pv, p, b, X, wc);
    }
    for (; p < p1; p += gridDim.x, set ^= 1) {
        const PrologueSet cur = prologue_set(L, set), nxt = prologue_set(L, set ^ 1);
        const int64_t pn = p + gridDim.x < p1 ? p + gridDim.x : -1;
        const int64_t nb = pv.patch_node_ptr[p];
        const int nown = (int)(pv.patch_node_ptr[p + 1] - nb);
        const int ncn = (int)(pv.patch_cnode_ptr[p + 1] - pv.patch_cnode_ptr[p]);
        const int64_t eb = pv.patch_elem_ptr[p];
        const int nel = (int)(pv.patch_elem_ptr[p + 1] - eb);
        const int nacc = pv.patch_acc[p];
        cp_async_wait_all();  // this thread's copies of the patch's data
        {
            constexpr int V = 16 / sizeof(AccT);
            float4 *a4 = reinterpret_cast<float4 *>(acc);
            for (int i = tid; i < nacc / V; i += nthr) a4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int i = nacc / V * V + tid; i < nacc; i += nthr) acc[i] = AccT(0);
            if (MIXED && L.hv_on)
                for (int k = tid; k < nown; k += nthr) hv[k] = 0.0;  // also clears the (hi, lo) float pair
            if (tid == 0) cur.roff[nown] = nacc;
        }
        __syncthreads();  // everyone's copies visible, accumulators clear
        if (pn >= 0) prefetch_plan(pv, pn, nxt);
        patch_batches<NPE, AccT, S, CT, true, MIXED>(
            pv, X, c, nullptr, thr, eb, nel, ncn, nown, L, mode, mb, g, wc, acc, hv,
            reinterpret_cast<const S(*)[3]>(cur.xs), cur.roff, [&] {
                if (pn >= 0) prefetch_coords<S>(pv, pn, nxt, X, wc);
            });
        __syncthreads();  // every phase of the patch done
        patch_writeout<AccT, MIXED>(pv, vals, nown, L, mode, wc, acc, hv, cur.roff, cur.rps, pv.val_off,
                                    [&](int k) { return L.hv_on && pv.own_hv[nb + k] != 0; });
        __syncthreads();  // the write-out has read the accumulators and this set
    }
}

// Persistent kernel over the patches of many meshes: work item w is patch
// w - prefix[m] of mesh m, prefix[m] <= w < prefix[m + 1].
template <int NPE, typename AccT, typename S, typename CT, bool MIXED>
__global__ void __launch_bounds__(patch_max_threads(NPE), patch_min_blocks(NPE)) k_patch_batched(const BatchItem *__restrict__ items,
                                                                     const int64_t *__restrict__ prefix, int n,
                                                                     PatchSmem L, unsigned mode,
                                                                     WaitCtl wc) {
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
        patch_body<NPE, AccT, S, CT, true, MIXED>(it.pv, (const S *)it.X, (const CT *)it.c, nullptr,
                                                   (AccT *)it.vals, it.thr, w - prefix[lo], L, mode, mb, g, wc);
    }
}

// ------------------------------------------------------------------ launchers
template <typename F>
static fem_status set_smem(F *f, size_t bytes) {
    FEM_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    return FEM_OK;
}

template <int NPE, typename T, typename S, typename CT, bool MIXED>
static fem_status launch_integrate_t(const int32_t *E, int64_t nel, const void *X, const void *c, void *ke, float thr,
                                     unsigned mode, unsigned long long *nflag, int *status, cudaStream_t s) {
    constexpr int NP = ElemTraits<NPE>::NP;
    const size_t smem = int_direct<NPE, T>() ? 0 : (size_t)INT_THREADS * (NP + 1) * sizeof(T);
    auto f = k_integrate<NPE, T, S, CT, MIXED>;
    if (smem) FEM_TRY(set_smem(f, smem));
    int per_sm = 0;
    FEM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, INT_THREADS, smem));
    if (per_sm < 1) per_sm = 1;
    const int64_t tiles = cdiv(nel, INT_THREADS);
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)num_sms() * per_sm));
    f<<<grid, INT_THREADS, smem, s>>>(E, nel, (const S *)X, (const CT *)c, (T *)ke, thr, mode, nflag, status);
    FEM_LAUNCHED("k_integrate");
    return FEM_OK;
}

fem_status launch_integrate(const IntegrateArgs &a, cudaStream_t s) {
    if (a.nel <= 0) return FEM_OK;
#define FEM_INT(NPE, T, S, CT, MX) \
    return launch_integrate_t<NPE, T, S, CT, MX>(a.E, a.nel, a.X, a.c, a.ke, a.thr, a.mode, a.nflag, a.status, s)
    if (!a.mixed) {
        if (a.npe == 8) FEM_INT(8, double, double, double, false);
        FEM_INT(4, double, double, double, false);
    }
    if (a.npe == 8) {
        if (a.xd == FEM_F32 && a.cd == FEM_F32) FEM_INT(8, float, float, float, true);
        if (a.xd == FEM_F32 && a.cd == FEM_F64) FEM_INT(8, float, float, double, true);
        if (a.xd == FEM_F64 && a.cd == FEM_F32) FEM_INT(8, float, double, float, true);
        FEM_INT(8, float, double, double, true);
    }
    if (a.xd == FEM_F32 && a.cd == FEM_F32) FEM_INT(4, float, float, float, true);
    if (a.xd == FEM_F32 && a.cd == FEM_F64) FEM_INT(4, float, float, double, true);
    if (a.xd == FEM_F64 && a.cd == FEM_F32) FEM_INT(4, float, double, float, true);
    FEM_INT(4, float, double, double, true);
#undef FEM_INT
}

static size_t align16(size_t v) { return (v + 15) & ~(size_t)15; }

PatchSmem patch_smem_layout(const PlanMax &P, bool fused, bool mixed, size_t xsize, size_t csize, bool prefetch) {
    PatchSmem L{};
    const size_t accsz = mixed ? sizeof(float) : sizeof(double);
    size_t o = 0;
    L.acc = o;
    L.acc_cap = (int)(P.max_acc + ACC_SCRATCH);
    o = align16(o + (size_t)(P.max_acc + ACC_SCRATCH) * accsz);
    L.hv = o;
    L.hv_on = mixed && P.any_hv;
    if (L.hv_on) o = align16(o + (size_t)P.max_own * sizeof(double));
    L.xs = o;
    if (fused) o = align16(o + (size_t)P.max_cnodes * 3 * xsize);
    L.cown = o;  // unused: accumulator targets come from the plan
    L.roff = o;
    o = align16(o + (size_t)(P.max_own + 1) * sizeof(int32_t));
    L.hvf = o;
    if (mixed) o = align16(o + (size_t)P.max_own);
    L.rps = o;
    o = align16(o + (size_t)P.max_own * sizeof(int64_t));
    L.gid = o;
    if (fused) o = align16(o + (size_t)P.max_cnodes * sizeof(int32_t));
    L.eid = L.cvs = o;
    L.xs2 = L.roff2 = L.rps2 = L.gid2 = o;
    L.prefetch = fused && prefetch;
    if (L.prefetch) {
        // the second set of the prologue arrays (the next patch's)
        L.xs2 = o;
        o = align16(o + (size_t)P.max_cnodes * 3 * xsize);
        L.roff2 = o;
        o = align16(o + (size_t)(P.max_own + 1) * sizeof(int32_t));
        L.rps2 = o;
        o = align16(o + (size_t)P.max_own * sizeof(int64_t));
        L.gid2 = o;
        o = align16(o + (size_t)P.max_cnodes * sizeof(int32_t));
    }
    (void)csize;
    // lanes per row in the write-out: 4, so that a warp's per-row bookkeeping
    // covers 8 rows at once (faster than one lane group per mean row length for
    // rows of 8 to 14 entries)
    L.wg_shift = 2;
    L.total = o;
    return L;
}

template <int NPE, typename AccT, typename S, typename CT, bool FUSED, bool MIXED>
static fem_status launch_patch_t(const PatchArgs &a, cudaStream_t s) {
    const Plan &P = *a.plan;
    const Closure &cl = a.closure ? *a.closure : P.full;
    PlanMax pm;
    pm.add(P);
    const PatchSmem L = patch_smem_layout(pm, FUSED, MIXED, sizeof(S), sizeof(CT));
    int dev = 0, max_optin = 0;
    FEM_CUDA(cudaGetDevice(&dev));
    FEM_CUDA(cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    auto f = k_patch<NPE, AccT, S, CT, FUSED, MIXED>;
    cudaFuncAttributes fa{};
    FEM_CUDA(cudaFuncGetAttributes(&fa, f));
    // the dynamic part shares the opt-in limit with the static mbarrier ring
    if (L.total + fa.sharedSizeBytes > (size_t)max_optin) {
        set_error("a patch needs %zu bytes of shared memory (limit %d); lower patch_entries", L.total, max_optin);
        return FEM_ERR_UNSUPPORTED;
    }
    FEM_TRY(set_smem(f, L.total));
    const int threads = a.threads;
    int per_sm = 0;
    FEM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, threads, L.total));
    if (per_sm < 1) {
        set_error("patch kernel cannot be resident with %d threads and %zu bytes of shared memory", threads, L.total);
        return FEM_ERR_UNSUPPORTED;
    }
    if (a.blocks_per_sm > 0 && a.blocks_per_sm < per_sm) per_sm = a.blocks_per_sm;
    // the patches of [a.p0, a.p1) that the closure holds, relative to its first
    const int64_t q0 = std::max(a.p0, cl.p0) - cl.p0, q1 = std::min(a.p1, cl.p1) - cl.p0;
    if (q1 <= q0) return FEM_OK;
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(q1 - q0, (int64_t)num_sms() * per_sm));
    PlanView pv = P.view(cl);
    pv.val_off = a.val_off;
    if constexpr (FUSED && MIXED && NPE == 8) {
        // bricks: the prefetching kernel, when its second set of prologue arrays
        // fits without costing a resident block (tetrahedra, whose blocks are
        // small and three to an SM, measured slower with it)
        const PatchSmem Lp = patch_smem_layout(pm, true, true, sizeof(S), sizeof(CT), true);
        auto fp = k_patch_prefetch<NPE, AccT, S, CT, MIXED>;
        cudaFuncAttributes fpa{};
        FEM_CUDA(cudaFuncGetAttributes(&fpa, fp));
        if (Lp.total + fpa.sharedSizeBytes <= (size_t)max_optin) {
            FEM_TRY(set_smem(fp, Lp.total));
            int per_pf = 0;
            FEM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_pf, fp, threads, Lp.total));
            if (a.blocks_per_sm > 0 && a.blocks_per_sm < per_pf) per_pf = a.blocks_per_sm;
            if (per_pf >= per_sm) {
                fp<<<grid, threads, Lp.total, s>>>(pv, (const S *)a.X, (const CT *)a.c, (AccT *)a.vals, a.thr, q0, q1,
                                                   Lp, a.mode, a.wait);
                FEM_LAUNCHED("k_patch_prefetch");
                return FEM_OK;
            }
        }
    }
    f<<<grid, threads, L.total, s>>>(pv, (const S *)a.X, (const CT *)a.c, (const AccT *)a.ke, (AccT *)a.vals, a.thr,
                                     q0, q1, L, a.mode, a.wait);
    FEM_LAUNCHED("k_patch");
    return FEM_OK;
}

int patch_blocks_per_sm(int npe, int threads) {
    int n = 0;
    cudaError_t e = npe == 8
        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_patch<8, float, float, float, true, true>, threads, 0)
        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_patch<4, float, float, float, true, true>, threads, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 2;
    }
    return std::max(1, n);
}

fem_status launch_patch(const PatchArgs &a, cudaStream_t s) {
#define FEM_P(NPE, ACC, S, CT, FU, MX) return launch_patch_t<NPE, ACC, S, CT, FU, MX>(a, s)
    if (!a.mixed) {
        if (a.fused) {
            if (a.npe == 8) FEM_P(8, double, double, double, true, false);
            FEM_P(4, double, double, double, true, false);
        }
        if (a.npe == 8) FEM_P(8, double, double, double, false, false);
        FEM_P(4, double, double, double, false, false);
    }
    if (!a.fused) {
        if (a.npe == 8) FEM_P(8, float, float, float, false, true);
        FEM_P(4, float, float, float, false, true);
    }
    if (a.npe == 8) {
        if (a.xd == FEM_F32 && a.cd == FEM_F32) FEM_P(8, float, float, float, true, true);
        if (a.xd == FEM_F32 && a.cd == FEM_F64) FEM_P(8, float, float, double, true, true);
        if (a.xd == FEM_F64 && a.cd == FEM_F32) FEM_P(8, float, double, float, true, true);
        FEM_P(8, float, double, double, true, true);
    }
    if (a.xd == FEM_F32 && a.cd == FEM_F32) FEM_P(4, float, float, float, true, true);
    if (a.xd == FEM_F32 && a.cd == FEM_F64) FEM_P(4, float, float, double, true, true);
    if (a.xd == FEM_F64 && a.cd == FEM_F32) FEM_P(4, float, double, float, true, true);
    FEM_P(4, float, double, double, true, true);
#undef FEM_P
}

template <int NPE, typename AccT, bool MIXED>
static fem_status batched_config_t(const PlanMax &pm, int threads, int blocks_per_sm, BatchLaunch *out) {
    using T = AccT;
    const PatchSmem L = patch_smem_layout(pm, true, MIXED, sizeof(T), sizeof(T));
    int dev = 0, max_optin = 0;
    FEM_CUDA(cudaGetDevice(&dev));
    FEM_CUDA(cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    auto f = k_patch_batched<NPE, AccT, T, T, MIXED>;
    cudaFuncAttributes fa{};
    FEM_CUDA(cudaFuncGetAttributes(&fa, f));
    if (L.total + fa.sharedSizeBytes > (size_t)max_optin) {
        set_error("a patch of the batch needs %zu bytes of shared memory (limit %d)", L.total, max_optin);
        return FEM_ERR_UNSUPPORTED;
    }
    FEM_TRY(set_smem(f, L.total));
    int per_sm = 0;
    FEM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, threads, L.total));
    if (per_sm < 1) {
        set_error("batched kernel cannot be resident with %d threads", threads);
        return FEM_ERR_UNSUPPORTED;
    }
    if (blocks_per_sm > 0 && blocks_per_sm < per_sm) per_sm = blocks_per_sm;
    out->L = L;
    out->threads = threads;
    out->grid = num_sms() * per_sm;
    return FEM_OK;
}

fem_status batched_config(int npe, bool mixed, const PlanMax &pm, int threads, int blocks_per_sm, BatchLaunch *out) {
    out->npe = npe;
    out->mixed = mixed;
    if (mixed) return npe == 8 ? batched_config_t<8, float, true>(pm, threads, blocks_per_sm, out)
                               : batched_config_t<4, float, true>(pm, threads, blocks_per_sm, out);
    return npe == 8 ? batched_config_t<8, double, false>(pm, threads, blocks_per_sm, out)
                    : batched_config_t<4, double, false>(pm, threads, blocks_per_sm, out);
}

fem_status launch_batched_kernel(const BatchLaunch &bl, cudaStream_t s) {
    if (bl.elastic) return launch_elastic_batched_kernel(bl, s);
    if (bl.tiles) return launch_tile_batched_kernel(bl, s);
#define FEM_B(NPE, T, MX)                                                                                   \
    k_patch_batched<NPE, T, T, T, MX><<<bl.grid, bl.threads, bl.L.total, s>>>(bl.items, bl.prefix, bl.n, bl.L, \
                                                                               bl.mode, bl.wait)
    if (bl.mixed) {
        if (bl.npe == 8) FEM_B(8, float, true); else FEM_B(4, float, true);
    } else {
        if (bl.npe == 8) FEM_B(8, double, false); else FEM_B(4, double, false);
    }
#undef FEM_B
    FEM_LAUNCHED("k_patch_batched");
    return FEM_OK;
}

}  // namespace fem
