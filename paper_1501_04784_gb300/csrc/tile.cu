// tile.cu -- the fused build over element tiles (tile.cuh): every element is
// integrated once (Eqs. 7-9), its packed entries are added colour by colour into
// the shared-memory rows of its tile, interior rows go to K's values and border
// rows to their partial slots; k_tile_combine then sums each border row's
// partials in slot order (Eq. 6).
#include "elem_ops.cuh"
#include "mesh.cuh"
#include "numeric.cuh"
#include "phases.cuh"
#include "tile.cuh"

namespace fem {

static size_t align16(size_t v) { return (v + 15) & ~(size_t)15; }

TileSmem tile_smem_layout(const TileMax &T, int npe, bool mixed, size_t xsize) {
    TileSmem L{};
    const size_t accsz = mixed ? sizeof(float) : sizeof(double);
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = align16(o + bytes);
        return at;
    };
    L.acc = take((size_t)T.max_acc * accsz);
    L.hv_on = T.any_hv ? 1 : 0;
    L.hv = take(L.hv_on ? (size_t)T.max_npad * sizeof(double) : 0);
    L.xs = take((size_t)T.max_npad * 4 * xsize);
    L.s_id = take((size_t)T.max_epad * sizeof(int32_t));
    L.s_col = take((size_t)T.max_epad);
    L.s_ln = take((size_t)T.max_epad * npe * sizeof(uint16_t));
    L.s_pos = take((size_t)T.max_epad * tile_posw(npe) * sizeof(uint32_t));
    L.s_gid = take((size_t)T.max_npad * sizeof(int32_t));
    L.s_info = take((size_t)T.max_npad * sizeof(uint32_t));
    L.s_dest = take((size_t)T.max_npad * sizeof(int64_t));
    L.total = o;
    L.wg_shift = 2;
    return L;
}

// ------------------------------------------------------ bulk copies (TMA)
// One-dimensional bulk copy global -> shared, completing on an mbarrier's
// transaction count (addresses 16-byte aligned, size a multiple of 16).
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *mbar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(mbar))
                 : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)), "r"(bytes)
                 : "memory");
}
// Shared memory last touched by ordinary loads and stores, about to be written by
// bulk copies: order the two.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Waits for the staging copies of the tile with the given parity; after
// wc.spins polls it records the failure and returns (the kernel then finishes
// with undefined values; the copies target this block's own shared memory).
__device__ __forceinline__ void stage_wait(uint64_t *mbar, uint32_t parity, const WaitCtl &wc) {
    const uint32_t a = smem_u32(mbar);
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

// Adds one element's packed entries into the tile's accumulators.  The entry of
// pair (a, b) lies in the row of the pair's node with the larger id (the larger
// tile-local index: rows ascend by id), at the pair's in-row position; a
// diagonal whose row is summed FP64-accurately goes to that row's pair (mixed:
// TwoSum, or a double) instead.  The loads of a group of entries are issued
// before their stores: the entries of one element are distinct, so a group's
// loads never alias its stores.
template <int NPE, typename AccT, bool MIXED>
__device__ __forceinline__ void scatter_tile(const uint16_t (&ln)[NPE], const uint32_t (&ra)[NPE],
                                             const uint32_t *__restrict__ pos, int pstride, double *hv,
                                             bool fp64_sums, AccT *acc, const AccT (&kv)[NPE * (NPE + 1) / 2],
                                             int nacc, int *status) {
    (void)nacc;
    (void)status;
    constexpr int NP = NPE * (NPE + 1) / 2;
    constexpr int G = 12;
    uint32_t pw[(NP + 3) / 4];
#pragma unroll
    for (int w = 0; w < (NP + 3) / 4; ++w) pw[w] = pos[w * pstride];
#pragma unroll
    for (int g0 = 0; g0 < NP; g0 += G) {
        int idx[G];
#pragma unroll
        for (int j = 0; j < G; ++j) {
            const int q = g0 + j;
            idx[j] = -1;
            if (q < NP) {
                const int a = tri_row(q), b = q - a * (a + 1) / 2;
                const int ps = (int)((pw[q >> 2] >> (8 * (q & 3))) & 0xffu);
                if (a == b) {
                    if (ra[a] & TILE_HV) {
                        if constexpr (MIXED) {
                            if (fp64_sums) hv[ln[a]] += (double)kv[q];
                            else two_sum_acc(reinterpret_cast<float2 *>(hv)[ln[a]], (float)kv[q]);
                        } else {
                            hv[ln[a]] += (double)kv[q];
                        }
                        continue;
                    }
                    idx[j] = (int)(ra[a] & 0xffffu) + ps;
                } else {
                    const uint32_t r = ln[a] > ln[b] ? ra[a] : ra[b];
                    idx[j] = (int)(r & 0xffffu) + ps;
                }
                if (!FEM_IN_BOUNDS(idx[j] < nacc, status)) idx[j] = -1;
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

// Local nodes of staged element i (shared memory).
template <int NPE>
__device__ __forceinline__ void lnodes_smem(const uint16_t *L, int i, uint16_t (&ln)[NPE]) {
    if constexpr (NPE == 8) {
        const uint4 v = *reinterpret_cast<const uint4 *>(L + i * 8);
        ln[0] = v.x & 0xffff; ln[1] = v.x >> 16; ln[2] = v.y & 0xffff; ln[3] = v.y >> 16;
        ln[4] = v.z & 0xffff; ln[5] = v.z >> 16; ln[6] = v.w & 0xffff; ln[7] = v.w >> 16;
    } else {
        const uint2 v = *reinterpret_cast<const uint2 *>(L + i * 4);
        ln[0] = v.x & 0xffff; ln[1] = v.x >> 16; ln[2] = v.y & 0xffff; ln[3] = v.y >> 16;
    }
}

template <int NPE, typename S>
__device__ __forceinline__ void load_xs(const S *xs4, int node, S (&x)[3]) {
    if constexpr (sizeof(S) == 4) {
        const float4 v = *reinterpret_cast<const float4 *>(xs4 + 4 * node);
        x[0] = v.x; x[1] = v.y; x[2] = v.z;
    } else {
        const double2 v0 = *reinterpret_cast<const double2 *>(xs4 + 4 * node);
        const double2 v1 = *reinterpret_cast<const double2 *>(xs4 + 4 * node + 2);
        x[0] = v0.x; x[1] = v0.y; x[2] = v1.x;
    }
}

template <int NPE, typename AccT, typename S, typename CT, bool MIXED>
__device__ __forceinline__ void tile_body(const TileView &tv, const S *__restrict__ X, const CT *__restrict__ c,
                                          AccT *__restrict__ vals, AccT *__restrict__ part, float thr, int64_t t,
                                          const TileSmem &L, unsigned mode, uint64_t *mb, uint32_t &g,
                                          uint64_t *smb, uint32_t &stile, const WaitCtl &wc) {
    constexpr int NP = ElemTraits<NPE>::NP;
    constexpr int POSW = tile_posw(NPE);
    const bool fp64_sums = (mode & FP64_SUMS) != 0;
    extern __shared__ __align__(16) unsigned char tile_smem[];
    AccT *acc = reinterpret_cast<AccT *>(tile_smem + L.acc);
    double *hv = reinterpret_cast<double *>(tile_smem + L.hv);
    S *xs4 = reinterpret_cast<S *>(tile_smem + L.xs);
    int32_t *s_id = reinterpret_cast<int32_t *>(tile_smem + L.s_id);
    uint8_t *s_col = tile_smem + L.s_col;
    uint16_t *s_ln = reinterpret_cast<uint16_t *>(tile_smem + L.s_ln);
    uint32_t *s_pos = reinterpret_cast<uint32_t *>(tile_smem + L.s_pos);
    int32_t *s_gid = reinterpret_cast<int32_t *>(tile_smem + L.s_gid);
    uint32_t *s_info = reinterpret_cast<uint32_t *>(tile_smem + L.s_info);
    int64_t *s_dest = reinterpret_cast<int64_t *>(tile_smem + L.s_dest);
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nwarps = nthr >> 5;
    const int64_t ebp = tv.tile_elem_ptr[t], nbp = tv.tile_node_ptr[t];
    const int nelp = (int)(tv.tile_elem_ptr[t + 1] - ebp), npd = (int)(tv.tile_node_ptr[t + 1] - nbp);
    const int nel = tv.tile_nel[t], ncn = tv.tile_ncn[t], nacc = tv.tile_acc[t];

    // Stage the tile's plan slices in shared memory: one thread issues the bulk
    // copies (element ids, colours, local nodes, in-row positions; row ids,
    // layouts, destinations), all complete on one mbarrier.  The previous tile's
    // ordinary accesses to these buffers ended at its final barrier.
    if (tid == 0) {
        fence_proxy_async();
        const uint32_t be = (uint32_t)nelp, bn = (uint32_t)npd;
        mbar_expect_tx(smb, be * (4u + 1u + 2u * NPE + 4u * POSW) + bn * (4u + 4u + 8u));
        bulk_g2s(s_id, tv.elem_id + ebp, be * 4u, smb);
        bulk_g2s(s_col, tv.elem_color + ebp, be, smb);
        bulk_g2s(s_ln, tv.elem_lnode + ebp * NPE, be * 2u * NPE, smb);
        bulk_g2s(s_pos, tv.elem_pos + ebp * POSW, be * 4u * POSW, smb);
        bulk_g2s(s_gid, tv.node_gid + nbp, bn * 4u, smb);
        bulk_g2s(s_info, tv.node_info + nbp, bn * 4u, smb);
        bulk_g2s(s_dest, tv.node_dest + nbp, bn * 8u, smb);
    }
    // meanwhile: accumulators cleared with 16-byte stores
    {
        constexpr int V = 16 / sizeof(AccT);
        float4 *a4 = reinterpret_cast<float4 *>(acc);
        for (int i = tid; i < nacc / V; i += nthr) a4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int i = nacc / V * V + tid; i < nacc; i += nthr) acc[i] = AccT(0);
        if (L.hv_on)
            for (int k = tid; k < ncn; k += nthr) hv[k] = 0.0;  // also clears the (hi, lo) float pair
    }
    stage_wait(smb, stile & 1u, wc);
    ++stile;

    // Coordinates of the tile's nodes, gathered through the staged ids (CH nodes
    // in flight per thread), one 16-byte row per node.
    constexpr int CH = 8;
    for (int j0 = 0; j0 < ncn; j0 += CH * nthr) {
        S v[CH][3];
#pragma unroll
        for (int k = 0; k < CH; ++k) {
            const int j = j0 + k * nthr + tid;
            int64_t gg = j < ncn ? s_gid[j] : 0;
#ifdef FEM_DEBUG_BOUNDS
            if (wc.stall == 2 && j == 0) gg = tv.n_nodes;  // testing the checks: one planted bad id per tile
#endif
            if (!FEM_IN_BOUNDS(gg >= 0 && gg < tv.n_nodes, wc.status)) gg = 0;
            v[k][0] = j < ncn ? __ldg(X + 3 * gg + 0) : S(0);
            v[k][1] = j < ncn ? __ldg(X + 3 * gg + 1) : S(0);
            v[k][2] = j < ncn ? __ldg(X + 3 * gg + 2) : S(0);
        }
#pragma unroll
        for (int k = 0; k < CH; ++k) {
            const int j = j0 + k * nthr + tid;
            if (j < ncn) {
                xs4[4 * j + 0] = v[k][0];
                xs4[4 * j + 1] = v[k][1];
                xs4[4 * j + 2] = v[k][2];
            }
        }
    }
    // coefficient of this thread's first element (later ones one batch ahead)
    CT c_next = CT(0);
    {
        int32_t e = tid < nel ? s_id[tid] : -1;
        if (!FEM_IN_BOUNDS(e < tv.n_elems, wc.status)) e = -1;
        if (e >= 0) c_next = __ldg(c + e);
    }
    __syncthreads();

    for (int base = 0; base < nel; base += nthr) {
        const int i = base + tid;
        const bool act = i < nel;
        const CT ce = c_next;
        {
            int32_t e = i + nthr < nel ? s_id[i + nthr] : -1;
            if (!FEM_IN_BOUNDS(e < tv.n_elems, wc.status)) e = -1;
            if (e >= 0) c_next = __ldg(c + e);
        }
        AccT kv[NP];
        uint16_t ln[NPE];
        int mycol = -1;
        if (act) {
            lnodes_smem<NPE>(s_ln, i, ln);
            mycol = s_col[i];
            S xc[NPE][3];
#pragma unroll
            for (int a = 0; a < NPE; ++a) {
                if (!FEM_IN_BOUNDS(ln[a] < ncn, wc.status)) ln[a] = 0;
                load_xs<NPE, S>(xs4, ln[a], xc[a]);
            }
            element_matrix<NPE, AccT, S, MIXED>(xc, ce, thr, mode, kv);
            // k_00 (m_00) is positive and finite for any element of nonzero volume
            if (!isfinite(kv[0])) atomicOr(wc.status, STATUS_NONFINITE);
        }
        const int last = min(base + nthr, nel) - 1;
        const int c0 = s_col[base], c1 = s_col[last];
        // testing: phase g cannot complete while warp 0 waits before arriving at it
        if (wc.stall == 1 && base == 0 && warp == 0) phase_wait(mb, g, wc);
        for (int cc = c0; cc <= c1; ++cc, ++g) {
            const bool mine = mycol == cc;
            if (__any_sync(0xffffffffu, mine)) {
                if (g > 0) phase_wait(mb, g - 1, wc);
                if (mine) {
                    uint32_t ra[NPE];
#pragma unroll
                    for (int a = 0; a < NPE; ++a) ra[a] = s_info[ln[a]];
                    scatter_tile<NPE, AccT, MIXED>(ln, ra, s_pos + i, nelp, hv, fp64_sums, acc, kv, nacc, wc.status);
                }
                __syncwarp();
            }
            if (g >= (uint32_t)PHASE_RING) phase_wait(mb, g - PHASE_RING, wc);
            if (lane == 0) phase_arrive(mb, g);
        }
    }
    __syncthreads();  // every phase of the tile done

    // Rows out: a group of 2^wg_shift lanes stores one row.  Interior rows into
    // K's values, border rows into their partial slots (the FP64-accurate
    // diagonal of a border row as its unrounded pair, one value past the row).
    const int gsh = L.wg_shift, gsz = 1 << gsh, sub = lane & (gsz - 1);
    const int rows_step = nwarps << (5 - gsh);
    for (int k = (warp << (5 - gsh)) + (lane >> gsh); k < ncn; k += rows_step) {
        const uint32_t info = s_info[k];
        const int64_t dest = s_dest[k];
        const int o0 = (int)(info & 0xffffu);
        int len = (int)((info >> 16) & 0xffu);
        const bool border = (info & TILE_BORDER) != 0, hvr = (info & TILE_HV) != 0;
        if (!FEM_IN_BOUNDS(o0 + len <= nacc && dest >= 0 &&
                               dest + len + (border && hvr ? 1 : 0) <= (border ? tv.partial_n : tv.nnz),
                           wc.status))
            len = 0;
        AccT *dst = (border ? part : vals) + dest;
        AccT vd = AccT(0), vlo = AccT(0);
        if (hvr && len > 0) {
            if (MIXED && !fp64_sums) {
                const float2 pr = reinterpret_cast<const float2 *>(hv)[k];
                if (border) {
                    vd = (AccT)pr.x;
                    vlo = (AccT)pr.y;
                } else {
                    vd = (AccT)(pr.x + pr.y);  // the pair rounded once
                }
            } else {
                const double d = hv[k];
                vd = (AccT)d;
                if (border) vlo = (AccT)(d - (double)vd);
            }
        }
        for (int j = sub; j < len; j += gsz) dst[j] = (hvr && j == len - 1) ? vd : acc[o0 + j];
        if (border && hvr && len > 0 && sub == 0) dst[len] = vlo;
    }
    __syncthreads();  // the staging buffers and accumulators are free for the next tile
}

// Border row b: the sum of its k partial rows in slot order, written into K's
// values; the FP64-accurate diagonal sums the k unrounded pairs and rounds once.
template <typename AccT, bool MIXED>
__device__ __forceinline__ void combine_row(const TileView &tv, const AccT *__restrict__ part, AccT *__restrict__ vals,
                                            int64_t b, int sub, int gsz, bool fp64_sums, int *status) {
    (void)status;
    const uint32_t info = __ldg(tv.brow_info + b);
    const int64_t pb = __ldg(tv.brow_base + b), vo = __ldg(tv.brow_vo + b);
    int len = (int)(info & 0xffu);
    const bool hvr = ((info >> 8) & 1u) != 0;
    const int kk = (int)(info >> 16), stride = len + (hvr ? 1 : 0);
    if (!FEM_IN_BOUNDS(pb >= 0 && pb + (int64_t)kk * stride <= tv.partial_n && vo >= 0 && vo + len <= tv.nnz, status))
        len = 0;
    const AccT *src = part + pb;
    AccT *dst = vals + vo;
    for (int j = sub; j < len; j += gsz) {
        AccT v;
        if (hvr && j == len - 1) {
            if (MIXED && !fp64_sums) {
                float2 pr = make_float2(0.f, 0.f);
                for (int r = 0; r < kk; ++r) {
                    two_sum_acc(pr, (float)src[(int64_t)r * stride + j]);
                    two_sum_acc(pr, (float)src[(int64_t)r * stride + len]);
                }
                v = (AccT)(pr.x + pr.y);
            } else {
                double d = 0.0;
                for (int r = 0; r < kk; ++r)
                    d += (double)src[(int64_t)r * stride + j] + (double)src[(int64_t)r * stride + len];
                v = (AccT)d;
            }
        } else {
            v = src[j];
#pragma unroll 4
            for (int r = 1; r < kk; ++r) v += src[(int64_t)r * stride + j];
        }
        dst[j] = v;
    }
}

static constexpr int COMBINE_THREADS = 256, COMBINE_LANES = 4;

template <typename AccT, bool MIXED>
__global__ void __launch_bounds__(COMBINE_THREADS) k_tile_combine(TileView tv, const AccT *__restrict__ part,
                                                                 AccT *__restrict__ vals, unsigned mode, int *status) {
    const bool fp64_sums = (mode & FP64_SUMS) != 0;
    const int sub = threadIdx.x & (COMBINE_LANES - 1);
    const int64_t step = ((int64_t)gridDim.x * blockDim.x) / COMBINE_LANES;
    for (int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / COMBINE_LANES; b < tv.n_brows; b += step)
        combine_row<AccT, MIXED>(tv, part, vals, b, sub, COMBINE_LANES, fp64_sums, status);
}

// The border rows of many meshes: row w of the batch is border row w - bprefix[m]
// of mesh m.
template <typename AccT, bool MIXED>
__global__ void __launch_bounds__(COMBINE_THREADS)
    k_tile_combine_batched(const TileBatchItem *__restrict__ items, const int64_t *__restrict__ bprefix, int n,
                           unsigned mode, int *status) {
    const bool fp64_sums = (mode & FP64_SUMS) != 0;
    const int sub = threadIdx.x & (COMBINE_LANES - 1);
    const int64_t total = bprefix[n];
    const int64_t step = ((int64_t)gridDim.x * blockDim.x) / COMBINE_LANES;
    for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / COMBINE_LANES; w < total; w += step) {
        int lo = 0, hi = n;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (bprefix[mid] <= w) lo = mid; else hi = mid;
        }
        const TileBatchItem &it = items[lo];
        combine_row<AccT, MIXED>(it.tv, (const AccT *)it.part, (AccT *)it.vals, w - bprefix[lo], sub, COMBINE_LANES,
                                 fp64_sums, status);
    }
}

static unsigned combine_grid(int64_t rows) {
    const int64_t per_block = COMBINE_THREADS / COMBINE_LANES;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(cdiv(rows, per_block), (int64_t)num_sms() * 8));
}

// The staging mbarrier: one arrival (the thread that issues the copies) plus
// the copies' transaction bytes per tile.
__device__ __forceinline__ void stage_init(uint64_t *smb) {
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(smb)) : "memory");
        fence_proxy_async();
    }
    __syncthreads();
}

template <int NPE, typename AccT, typename S, typename CT, bool MIXED>
__global__ void __launch_bounds__(tile_max_threads(NPE), tile_min_blocks(NPE))
    k_tile(TileView tv, const S *__restrict__ X, const CT *__restrict__ c, AccT *__restrict__ vals,
           AccT *__restrict__ part, float thr, TileSmem L, unsigned mode, WaitCtl wc) {
    __shared__ uint64_t mb[PHASE_RING];
    __shared__ uint64_t smb;
    phase_init(mb);
    stage_init(&smb);
    uint32_t g = 0, stile = 0;
    for (int64_t t = blockIdx.x; t < tv.n_tiles; t += gridDim.x)
        tile_body<NPE, AccT, S, CT, MIXED>(tv, X, c, vals, part, thr, t, L, mode, mb, g, &smb, stile, wc);
}

// Persistent kernel over the tiles of many meshes: work item w is tile
// w - prefix[m] of mesh m, prefix[m] <= w < prefix[m + 1].
template <int NPE, typename AccT, bool MIXED>
__global__ void __launch_bounds__(tile_max_threads(NPE), tile_min_blocks(NPE))
    k_tile_batched(const TileBatchItem *__restrict__ items, const int64_t *__restrict__ prefix, int n, TileSmem L,
                   unsigned mode, WaitCtl wc) {
    const int64_t total = prefix[n];
    __shared__ uint64_t mb[PHASE_RING];
    __shared__ uint64_t smb;
    phase_init(mb);
    stage_init(&smb);
    uint32_t g = 0, stile = 0;
    for (int64_t w = blockIdx.x; w < total; w += gridDim.x) {
        int lo = 0, hi = n;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (prefix[mid] <= w) lo = mid; else hi = mid;
        }
        const TileBatchItem &it = items[lo];
        tile_body<NPE, AccT, AccT, AccT, MIXED>(it.tv, (const AccT *)it.X, (const AccT *)it.c, (AccT *)it.vals,
                                                (AccT *)it.part, it.thr, w - prefix[lo], L, mode, mb, g, &smb, stile,
                                                wc);
    }
}

template <int NPE, typename AccT, bool MIXED>
static fem_status tile_batched_config_t(const TileMax &tm, int threads, int blocks_per_sm, BatchLaunch *out) {
    const TileSmem L = tile_smem_layout(tm, NPE, MIXED, sizeof(AccT));
    int dev = 0, max_optin = 0;
    FEM_CUDA(cudaGetDevice(&dev));
    FEM_CUDA(cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    auto f = k_tile_batched<NPE, AccT, MIXED>;
    cudaFuncAttributes fa{};
    FEM_CUDA(cudaFuncGetAttributes(&fa, f));
    if (L.total + fa.sharedSizeBytes > (size_t)max_optin) {
        set_error("a tile of the batch needs %zu bytes of shared memory (limit %d)", L.total, max_optin);
        return FEM_ERR_UNSUPPORTED;
    }
    FEM_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total));
    int per_sm = 0;
    FEM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, threads, L.total));
    if (per_sm < 1) {
        set_error("batched tile kernel cannot be resident with %d threads", threads);
        return FEM_ERR_UNSUPPORTED;
    }
    if (blocks_per_sm > 0 && blocks_per_sm < per_sm) per_sm = blocks_per_sm;
    out->tl = L;
    out->tiles = true;
    out->threads = threads;
    out->grid = num_sms() * per_sm;
    out->combine_grid = (int)combine_grid(1ll << 40);
    return FEM_OK;
}

fem_status tile_batched_config(int npe, bool mixed, const TileMax &tm, int threads, int blocks_per_sm,
                               BatchLaunch *out) {
    out->npe = npe;
    out->mixed = mixed;
    if (mixed) return npe == 8 ? tile_batched_config_t<8, float, true>(tm, threads, blocks_per_sm, out)
                               : tile_batched_config_t<4, float, true>(tm, threads, blocks_per_sm, out);
    return npe == 8 ? tile_batched_config_t<8, double, false>(tm, threads, blocks_per_sm, out)
                    : tile_batched_config_t<4, double, false>(tm, threads, blocks_per_sm, out);
}

fem_status launch_tile_batched_kernel(const BatchLaunch &bl, cudaStream_t s) {
#define FEM_B(NPE, T, MX) \
    k_tile_batched<NPE, T, MX><<<bl.grid, bl.threads, bl.tl.total, s>>>(bl.titems, bl.prefix, bl.n, bl.tl, bl.mode, bl.wait)
    if (bl.mixed) {
        if (bl.npe == 8) FEM_B(8, float, true); else FEM_B(4, float, true);
    } else {
        if (bl.npe == 8) FEM_B(8, double, false); else FEM_B(4, double, false);
    }
#undef FEM_B
    FEM_LAUNCHED("k_tile_batched");
    if (bl.mixed)
        k_tile_combine_batched<float, true><<<bl.combine_grid, COMBINE_THREADS, 0, s>>>(bl.titems, bl.bprefix, bl.n,
                                                                                        bl.mode, bl.wait.status);
    else
        k_tile_combine_batched<double, false><<<bl.combine_grid, COMBINE_THREADS, 0, s>>>(bl.titems, bl.bprefix, bl.n,
                                                                                          bl.mode, bl.wait.status);
    FEM_LAUNCHED("k_tile_combine_batched");
    return FEM_OK;
}

int tile_blocks_per_sm(int npe, int threads) {
    int n = 0;
    cudaError_t e = npe == 8
        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_tile<8, float, float, float, true>, threads, 0)
        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_tile<4, float, float, float, true>, threads, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 2;
    }
    return std::max(1, n);
}

template <int NPE, typename AccT, typename S, typename CT, bool MIXED>
static fem_status launch_tile_t(const TileArgs &a, cudaStream_t s) {
    const TilePlan &T = *a.plan;
    TileMax tm;
    tm.add(T);
    const TileSmem L = tile_smem_layout(tm, NPE, MIXED, sizeof(S));
    int dev = 0, max_optin = 0;
    FEM_CUDA(cudaGetDevice(&dev));
    FEM_CUDA(cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    auto f = k_tile<NPE, AccT, S, CT, MIXED>;
    cudaFuncAttributes fa{};
    FEM_CUDA(cudaFuncGetAttributes(&fa, f));
    if (L.total + fa.sharedSizeBytes > (size_t)max_optin) {
        set_error("an element tile needs %zu bytes of shared memory (limit %d); lower tile_elems", L.total, max_optin);
        return FEM_ERR_UNSUPPORTED;
    }
    FEM_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total));
    int per_sm = 0;
    FEM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, a.threads, L.total));
    if (per_sm < 1) {
        set_error("tile kernel cannot be resident with %d threads and %zu bytes of shared memory", a.threads, L.total);
        return FEM_ERR_UNSUPPORTED;
    }
    if (a.blocks_per_sm > 0 && a.blocks_per_sm < per_sm) per_sm = a.blocks_per_sm;
    if (T.n_tiles <= 0) return FEM_OK;
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(T.n_tiles, (int64_t)num_sms() * per_sm));
    f<<<grid, a.threads, L.total, s>>>(a.view, (const S *)a.X, (const CT *)a.c, (AccT *)a.vals, (AccT *)a.part,
                                       a.thr, L, a.mode, a.wait);
    FEM_LAUNCHED("k_tile");
    if (T.n_brows > 0) {
        k_tile_combine<AccT, MIXED><<<combine_grid(T.n_brows), COMBINE_THREADS, 0, s>>>(
            a.view, (const AccT *)a.part, (AccT *)a.vals, a.mode, a.wait.status);
        FEM_LAUNCHED("k_tile_combine");
    }
    return FEM_OK;
}

fem_status launch_tile(const TileArgs &a, cudaStream_t s) {
#define FEM_T(NPE, ACC, S, CT, MX) return launch_tile_t<NPE, ACC, S, CT, MX>(a, s)
    if (!a.mixed) {
        if (a.npe == 8) FEM_T(8, double, double, double, false);
        FEM_T(4, double, double, double, false);
    }
    if (a.npe == 8) {
        if (a.xd == FEM_F32 && a.cd == FEM_F32) FEM_T(8, float, float, float, true);
        if (a.xd == FEM_F32 && a.cd == FEM_F64) FEM_T(8, float, float, double, true);
        if (a.xd == FEM_F64 && a.cd == FEM_F32) FEM_T(8, float, double, float, true);
        FEM_T(8, float, double, double, true);
    }
    if (a.xd == FEM_F32 && a.cd == FEM_F32) FEM_T(4, float, float, float, true);
    if (a.xd == FEM_F32 && a.cd == FEM_F64) FEM_T(4, float, float, double, true);
    if (a.xd == FEM_F64 && a.cd == FEM_F32) FEM_T(4, float, double, float, true);
    FEM_T(4, float, double, double, true);
#undef FEM_T
}

}  // namespace fem
