// tile_plan.cu -- the symbolic phase of the element-tile assembly (tile.cuh):
// element order, tiles, each tile's nodes and rows, its colouring, every packed
// pair's accumulator target, and the slots of the border rows' partial sums.
//
// Steps, all on the GPU:
//   1. Elements are sorted (stably) by the locality rank of their lowest-ranked
//      node, so that consecutive elements are neighbours in space; tiles are
//      consecutive runs of that order.
//   2. One block per tile sorts the tile's node ids in shared memory (bitonic),
//      keeps the distinct ones (the tile's rows, ascending by id) and counts, for
//      each, the tile's elements that hold it: fewer than the node's degree
//      makes it a border row.
//   3. A second pass of the same blocks lays the rows out (each row's whole lower
//      CSR row, in node order), colours the tile greedily in sweep order (no two
//      elements of a colour share a node), sorts the elements by (colour, sweep
//      position) and writes each packed pair's position in its CSR row (found by
//      one scan of the row), from which the kernel forms the pair's accumulator
//      offset.  A tile's element and row slices are padded to 16-byte units.
//   4. The (row, tile) pairs of border rows are sorted; a row's k tiles get
//      consecutive partial slots in ascending tile order, and the row gets its
//      entry in the table of the kernel that sums the partials.
#include <algorithm>
#include <climits>
#include <vector>

#include "mesh.cuh"
#include "numeric.cuh"
#include "tile.cuh"
#include "block_prims.cuh"

namespace fem {

int tile_blocks_per_sm(int npe, int threads);  // tile.cu

namespace {

constexpr int TP_THREADS = 512;
constexpr int TP_MAX_KEYS = 8192;  // node slots (elements x npe) a tile may hold
constexpr uint32_t KEY_PAD = 0xffffffffu;

unsigned grid_for(int64_t n, int tpb = 256) {
    const int64_t b = cdiv(n, tpb), cap = (int64_t)num_sms() * 32;
    return (unsigned)(b < 1 ? 1 : (b > cap ? cap : b));
}

int bits_for(int64_t v) {
    int b = 1;
    while ((v >> b) != 0) ++b;
    return b;
}


// Lower bound of g in the ascending list v[0, n).
__device__ __forceinline__ int lower_bound_i32(const int32_t *v, int n, int32_t g) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (v[mid] < g) lo = mid + 1; else hi = mid;
    }
    return lo;
}

struct TileIn {
    const int32_t *E;
    const uint32_t *eorder;   // element ids in sweep order
    const int64_t *tep;       // [n_tiles + 1] tile element ranges
    const int64_t *rowptr;
    const int32_t *col;
    const int64_t *inc_ptr;
    int hv_thr;               // INT_MAX: no FP64-accurate diagonals
};

// The tile's node slots, sorted: keys[0, n) = node ids of its elements, padded
// with KEY_PAD to the power of two sz.
template <int NPE>
__device__ void load_sorted_nodes(const TileIn &in, int64_t eb, int ne, uint32_t *keys, int sz) {
    const int n = ne * NPE;
    for (int i = threadIdx.x; i < sz; i += blockDim.x)
        keys[i] = i < n ? (uint32_t)in.E[(int64_t)in.eorder[eb + i / NPE] * NPE + i % NPE] : KEY_PAD;
    __syncthreads();
    block_bitonic(keys, sz);
}

// Pass 1: per tile, the number of distinct nodes (rows), the accumulator entries
// (sum of their lower-row lengths) and the border rows.
template <int NPE>
__global__ void __launch_bounds__(TP_THREADS) k_tile_count(TileIn in, int64_t n_tiles, int64_t *ncn, int64_t *nacc,
                                                           int64_t *nbord) {
    extern __shared__ __align__(16) unsigned char tp_smem[];
    uint32_t *keys = reinterpret_cast<uint32_t *>(tp_smem);
    __shared__ int cnt[3];
    for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        const int64_t eb = in.tep[t];
        const int ne = (int)(in.tep[t + 1] - eb), n = ne * NPE, sz = pow2_at_least(n);
        if (threadIdx.x < 3) cnt[threadIdx.x] = 0;
        load_sorted_nodes<NPE>(in, eb, ne, keys, sz);
        int c0 = 0, c1 = 0, c2 = 0;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const uint32_t g = keys[i];
            if (i > 0 && keys[i - 1] == g) continue;
            int run = 1;
            while (i + run < n && keys[i + run] == g) ++run;
            const int64_t deg = in.inc_ptr[g + 1] - in.inc_ptr[g];
            ++c0;
            c1 += (int)(in.rowptr[g + 1] - in.rowptr[g]);
            c2 += run < deg ? 1 : 0;
        }
        atomicAdd(&cnt[0], c0);
        atomicAdd(&cnt[1], c1);
        atomicAdd(&cnt[2], c2);
        __syncthreads();
        if (threadIdx.x == 0) {
            ncn[t] = cnt[0];
            nacc[t] = cnt[1];
            nbord[t] = cnt[2];
        }
        __syncthreads();
    }
}


// Per tile, from pass 1: where its rows and border pairs go.
struct TileOut {
    const int64_t *tnp;   // [n_tiles + 1] padded tile row ranges
    const int64_t *tep;   // [n_tiles + 1] padded tile element ranges
    const int64_t *bofs;  // [n_tiles] first border pair of each tile
    int32_t *tile_acc;
    int32_t *elem_id;
    uint8_t *elem_color;
    uint16_t *elem_lnode;
    uint8_t *pos;         // in-row positions, see TileView::elem_pos
    int32_t *node_gid;
    uint32_t *node_info;
    int64_t *node_dest;
    uint64_t *bkeys;      // (row << tbits) | tile of every border pair
    uint32_t *bvals;      // the pair's tile-row index
    int tbits;
    int *max_color;
};

// Shared-memory layout of pass 2 (byte offsets).
struct FillSmem {
    size_t keys, sbuf, ug, uinfo, ln, mask, ecol, total;
};

FillSmem fill_layout(int npe, int64_t pmax, int64_t ncn_max) {
    auto al = [](size_t v) { return (v + 15) & ~(size_t)15; };
    const size_t sz = (size_t)pow2_at_least((int)(pmax * npe));
    FillSmem L{};
    size_t o = 0;
    L.keys = o; o = al(o + sz * 4);
    L.sbuf = o; o = al(o + sz * 4);
    L.ug = o; o = al(o + (size_t)ncn_max * 4);
    L.uinfo = o; o = al(o + (size_t)ncn_max * 4);
    L.mask = o; o = al(o + (size_t)ncn_max * 32);
    L.ln = o; o = al(o + (size_t)pmax * npe * 2);
    L.ecol = o; o = al(o + (size_t)pmax);
    L.total = o;
    return L;
}

// Pass 2: a tile's rows (ids, layout, border flags), its colouring and element
// order, and every packed pair's accumulator target.
template <int NPE>
__global__ void __launch_bounds__(TP_THREADS) k_tile_fill(TileIn in, int64_t n_tiles, TileOut out, FillSmem L) {
    constexpr int NP = NPE * (NPE + 1) / 2;
    extern __shared__ __align__(16) unsigned char tp_smem[];
    uint32_t *keys = reinterpret_cast<uint32_t *>(tp_smem + L.keys);
    int *sbuf = reinterpret_cast<int *>(tp_smem + L.sbuf);
    int32_t *ug = reinterpret_cast<int32_t *>(tp_smem + L.ug);
    uint32_t *uinfo = reinterpret_cast<uint32_t *>(tp_smem + L.uinfo);
    unsigned long long *mask = reinterpret_cast<unsigned long long *>(tp_smem + L.mask);
    uint16_t *ln = reinterpret_cast<uint16_t *>(tp_smem + L.ln);
    uint8_t *ecol = tp_smem + L.ecol;
    __shared__ int ws[32];
    const int tid = threadIdx.x, nthr = blockDim.x;
    for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        const int64_t eb = in.tep[t], nb = out.tnp[t], ebp = out.tep[t];
        const int64_t nelp = out.tep[t + 1] - ebp;
        const int ne = (int)(in.tep[t + 1] - eb), n = ne * NPE, sz = pow2_at_least(n);
        load_sorted_nodes<NPE>(in, eb, ne, keys, sz);
        for (int i = tid; i < sz; i += nthr) sbuf[i] = (i < n && (i == 0 || keys[i] != keys[i - 1])) ? 1 : 0;
        __syncthreads();
        const int ncn = block_scan(sbuf, sz, ws);
        // distinct ids (the tile's rows, ascending) and how many of the tile's
        // elements hold each
        for (int i = tid; i < n; i += nthr) {
            if (i > 0 && keys[i - 1] == keys[i]) continue;
            int run = 1;
            while (i + run < n && keys[i + run] == keys[i]) ++run;
            ug[sbuf[i]] = (int32_t)keys[i];
            uinfo[sbuf[i]] = (uint32_t)run;
        }
        __syncthreads();
        for (int u = tid; u < ncn; u += nthr) {
            const int32_t g = ug[u];
            const int64_t deg = in.inc_ptr[g + 1] - in.inc_ptr[g];
            const int len = (int)(in.rowptr[g + 1] - in.rowptr[g]);
            const bool border = (int64_t)uinfo[u] < deg, hv = deg > in.hv_thr;
            sbuf[u] = len;
            uinfo[u] = ((uint32_t)len << 16) | (border ? TILE_BORDER : 0u) | (hv ? TILE_HV : 0u);
        }
        __syncthreads();
        const int nacc = block_scan(sbuf, ncn, ws);
        for (int u = tid; u < ncn; u += nthr) {
            const uint32_t info = uinfo[u] | (uint32_t)sbuf[u];
            const int32_t g = ug[u];
            uinfo[u] = info;
            out.node_gid[nb + u] = g;
            out.node_info[nb + u] = info;
            out.node_dest[nb + u] = (info & TILE_BORDER) ? -1 : in.rowptr[g];
            sbuf[u] = (info & TILE_BORDER) ? 1 : 0;
        }
        __syncthreads();
        block_scan(sbuf, ncn, ws);
        for (int u = tid; u < ncn; u += nthr)
            if (uinfo[u] & TILE_BORDER) {
                const int64_t j = out.bofs[t] + sbuf[u];
                out.bkeys[j] = ((uint64_t)(uint32_t)ug[u] << out.tbits) | (uint64_t)t;
                out.bvals[j] = (uint32_t)(nb + u);
            }
        if (tid == 0) out.tile_acc[t] = nacc;
        // tile-local node index of every node slot of every element (sweep order)
        for (int i = tid; i < n; i += nthr) {
            const int32_t g = in.E[(int64_t)in.eorder[eb + i / NPE] * NPE + i % NPE];
            ln[i] = (uint16_t)lower_bound_i32(ug, ncn, g);
        }
        for (int i = tid; i < 4 * ncn; i += nthr) mask[i] = 0ull;
        __syncthreads();
        // greedy colouring in sweep order: the lowest colour no element sharing a
        // node has taken (colour sets are 256-bit masks per row; colours 0-254, 255
        // marks an element no colour was left for)
        if (tid == 0) {
            int cmax = 0;
            for (int e = 0; e < ne; ++e) {
                unsigned long long mw[4] = {0ull, 0ull, 0ull, 0ull};
#pragma unroll
                for (int a = 0; a < NPE; ++a) {
                    const int o = ln[e * NPE + a];
#pragma unroll
                    for (int w = 0; w < 4; ++w) mw[w] |= mask[4 * o + w];
                }
                int c = 255;
#pragma unroll
                for (int w = 3; w >= 0; --w)
                    if (~mw[w]) c = 64 * w + __ffsll((long long)~mw[w]) - 1;
                if (c > 254) c = 255;
                ecol[e] = (uint8_t)c;
                if (c < 255) {
#pragma unroll
                    for (int a = 0; a < NPE; ++a) mask[4 * ln[e * NPE + a] + (c >> 6)] |= 1ull << (c & 63);
                }
                cmax = max(cmax, c);
            }
            atomicMax(out.max_color, cmax);
        }
        __syncthreads();
        // elements by (colour, sweep position)
        const int sze = pow2_at_least(ne);
        for (int i = tid; i < sze; i += nthr) keys[i] = i < ne ? ((uint32_t)ecol[i] << 16) | (uint32_t)i : KEY_PAD;
        __syncthreads();
        block_bitonic(keys, sze);
        for (int j = tid; j < ne; j += nthr) {
            const int e = (int)(keys[j] & 0xffffu);
            const int64_t dst = ebp + j;
            out.elem_id[dst] = (int32_t)in.eorder[eb + e];
            out.elem_color[dst] = (uint8_t)(keys[j] >> 16);
            int li[NPE];
            int32_t g[NPE];
            uint32_t info[NPE];
#pragma unroll
            for (int a = 0; a < NPE; ++a) {
                li[a] = ln[e * NPE + a];
                g[a] = ug[li[a]];
                info[a] = uinfo[li[a]];
                out.elem_lnode[dst * NPE + a] = (uint16_t)li[a];
            }
            // positions of the element's lower partners in each of its rows: one
            // scan of the row (independent loads) instead of a search per pair
            uint8_t pxy[NPE][NPE];
#pragma unroll
            for (int x = 0; x < NPE; ++x) {
                const int64_t r0 = in.rowptr[g[x]];
                const int rl = (int)((info[x] >> 16) & 0xffu);
#pragma unroll
                for (int y = 0; y < NPE; ++y) pxy[x][y] = 0;
                for (int k = 0; k < rl; ++k) {
                    const int32_t cj = in.col[r0 + k];
#pragma unroll
                    for (int y = 0; y < NPE; ++y)
                        if (g[y] == cj) pxy[x][y] = (uint8_t)k;
                }
            }
            int q = 0;
            const int64_t wb = ebp * tile_posw(NPE);
#pragma unroll
            for (int a = 0; a < NPE; ++a)
#pragma unroll
                for (int b = 0; b <= a; ++b, ++q) {
                    // the diagonal closes its lower row; an off-diagonal pair sits in
                    // the row of its node with the larger id
                    uint32_t ps;
                    if (a == b) ps = ((info[a] >> 16) & 0xffu) - 1u;
                    else ps = g[a] > g[b] ? pxy[a][b] : pxy[b][a];
                    out.pos[(wb + (int64_t)(q >> 2) * nelp + j) * 4 + (q & 3)] = (uint8_t)ps;
                }
            (void)NP;
        }
        __syncthreads();
    }
}

__global__ void k_node_rank(const int32_t *order, int64_t N, int32_t *rank) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x)
        rank[order[k]] = (int32_t)k;
}

// Sweep key of an element: the locality rank of its lowest-ranked node.
template <int NPE>
__global__ void k_elem_keys(const int32_t *__restrict__ E, int64_t nel, const int32_t *rank, uint64_t *keys,
                            uint32_t *vals) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nel; e += (int64_t)gridDim.x * blockDim.x) {
        int32_t r = INT_MAX;
#pragma unroll
        for (int a = 0; a < NPE; ++a) r = min(r, rank[E[e * NPE + a]]);
        keys[e] = (uint64_t)(uint32_t)r;
        vals[e] = (uint32_t)e;
    }
}

// ------------------------------------------------------------- border rows
__device__ __forceinline__ bool brow_start(const uint64_t *bk, int64_t i, int tbits) {
    return i == 0 || (bk[i] >> tbits) != (bk[i - 1] >> tbits);
}

__global__ void k_brow_flags(const uint64_t *bk, int64_t n, int tbits, int64_t *flags) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        flags[i] = brow_start(bk, i, tbits) ? 1 : 0;
}

// start[b] = first pair of border row b (flags: exclusive scan of the start flags)
__global__ void k_brow_start(const uint64_t *bk, const int64_t *flags, int64_t n, int64_t nrows, int tbits,
                             int64_t *start) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= n; i += (int64_t)gridDim.x * blockDim.x) {
        if (i == n) start[nrows] = n;
        else if (brow_start(bk, i, tbits)) start[flags[i]] = i;
    }
}

__device__ __forceinline__ int64_t brow_stride(int32_t g, const int64_t *rowptr, const int64_t *inc_ptr, int hv_thr) {
    return (rowptr[g + 1] - rowptr[g]) + ((inc_ptr[g + 1] - inc_ptr[g]) > hv_thr ? 1 : 0);
}

__global__ void k_brow_amount(const uint64_t *bk, const int64_t *start, int64_t nrows, int tbits,
                              const int64_t *rowptr, const int64_t *inc_ptr, int hv_thr, int64_t *amt,
                              int64_t *brow_vo, uint32_t *brow_info) {
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nrows; b += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = start[b + 1] - start[b];
        const int32_t g = (int32_t)(bk[start[b]] >> tbits);
        const int64_t len = rowptr[g + 1] - rowptr[g];
        const bool hv = (inc_ptr[g + 1] - inc_ptr[g]) > hv_thr;
        amt[b] = k * brow_stride(g, rowptr, inc_ptr, hv_thr);
        brow_vo[b] = rowptr[g];
        brow_info[b] = (uint32_t)len | (hv ? 1u << 8 : 0u) | ((uint32_t)k << 16);
    }
}

__global__ void k_brow_dest(const uint64_t *bk, const uint32_t *bv, const int64_t *flags, const int64_t *start,
                            const int64_t *base, int64_t n, int tbits, const int64_t *rowptr, const int64_t *inc_ptr,
                            int hv_thr, int64_t *node_dest) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = brow_start(bk, i, tbits) ? flags[i] : flags[i] - 1;
        const int32_t g = (int32_t)(bk[i] >> tbits);
        node_dest[bv[i]] = base[b] + (i - start[b]) * brow_stride(g, rowptr, inc_ptr, hv_thr);
    }
}

template <typename T>
fem_status read_scalar(const T *dev, T *host, cudaStream_t s) {
    FEM_CUDA(cudaMemcpyAsync(host, dev, sizeof(T), cudaMemcpyDeviceToHost, s));
    FEM_CUDA(cudaStreamSynchronize(s));
    return FEM_OK;
}

}  // namespace

TileView TilePlan::view(const fem_mesh_s *m) const {
    TileView v{};
    v.tile_elem_ptr = tile_elem_ptr.ptr;
    v.tile_nel = tile_nel.ptr;
    v.tile_node_ptr = tile_node_ptr.ptr;
    v.tile_ncn = tile_ncn.ptr;
    v.tile_acc = tile_acc.ptr;
    v.elem_id = elem_id.ptr;
    v.elem_color = elem_color.ptr;
    v.elem_lnode = elem_lnode.ptr;
    v.elem_pos = elem_pos.ptr;
    v.node_gid = node_gid.ptr;
    v.node_dest = node_dest.ptr;
    v.node_info = node_info.ptr;
    v.brow_base = brow_base.ptr;
    v.brow_vo = brow_vo.ptr;
    v.brow_info = brow_info.ptr;
    v.n_tiles = n_tiles;
    v.n_elems = m->n_elems;
    v.n_nodes = m->n_nodes;
    v.nnz = m->nnz;
    v.n_brows = n_brows;
    v.partial_n = partial_n;
    return v;
}

// Element tiles of mesh m (after the pattern).  The tile size is
// fem_options.tile_elems (default 512 bricks or 2048 tetrahedra), lowered until a
// tile fits the 16-bit targets and the pass's shared memory, and the tile count
// is rounded up to whole waves of the tile kernel at its default block size.  The
// plan (and so every sum's order) does not depend on the launch shape a build
// then uses.
fem_status build_tiles(fem_mesh m, cudaStream_t s) {
    NvtxRange nvtx_range("fem_tile_plan");
    TilePlan &T = m->tiles;
    batch_forget(m);  // cached batched launches were sized for the old tiles
    T.reset();
    Arena &ar = m->arena;
    const int npe = m->npe;
    const int64_t nel = m->n_elems, N = m->n_nodes;
    const int hv_thr = m->opt.valence_threshold;
    int64_t P = m->opt.tile_elems > 0 ? m->opt.tile_elems : (npe == 8 ? 512 : 2048);
    P = std::max<int64_t>(1, std::min<int64_t>(P, TP_MAX_KEYS / npe));

    // ---- sweep order of the elements
    DevBuf<uint32_t> eorder;
    FEM_TRY(eorder.alloc(ar, nel, "element sweep order"));
    {
        DevBuf<int32_t> rank;
        DevBuf<uint64_t> keys, alt;
        DevBuf<uint32_t> altv;
        DevBuf<int64_t> hist;
        FEM_TRY(rank.alloc(ar, N, "node ranks"));
        k_node_rank<<<grid_for(N), 256, 0, s>>>(m->order.ptr, N, rank.ptr);
        FEM_LAUNCHED("k_node_rank");
        FEM_TRY(keys.alloc(ar, nel, "element keys"));
        if (npe == 8) k_elem_keys<8><<<grid_for(nel), 256, 0, s>>>(m->E, nel, rank.ptr, keys.ptr, eorder.ptr);
        else k_elem_keys<4><<<grid_for(nel), 256, 0, s>>>(m->E, nel, rank.ptr, keys.ptr, eorder.ptr);
        FEM_LAUNCHED("k_elem_keys");
        FEM_TRY(alt.alloc(ar, nel, "sort scratch"));
        FEM_TRY(altv.alloc(ar, nel, "sort scratch"));
        FEM_TRY(hist.alloc(ar, radix_hist_elems(nel), "sort histogram"));
        FEM_TRY(radix_sort_u64(keys.ptr, eorder.ptr, nel, bits_for(N), alt.ptr, altv.ptr, hist.ptr, s));
        FEM_CUDA(cudaStreamSynchronize(s));
    }

    // ---- tiles: cut, counted (pass 1), recut to whole waves of the tile kernel
    int dev = 0, max_optin = 0;
    FEM_CUDA(cudaGetDevice(&dev));
    FEM_CUDA(cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    const size_t count_smem = (size_t)TP_MAX_KEYS * 4;
    if (npe == 8) FEM_CUDA(cudaFuncSetAttribute(k_tile_count<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)count_smem));
    else FEM_CUDA(cudaFuncSetAttribute(k_tile_count<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)count_smem));
    DevBuf<int64_t> tep, ncn, nacc, nbord;
    std::vector<int64_t> h_tep, h_ncn, h_nacc, h_nbord;
    int64_t nt = 0, max_ncn = 0, max_acc = 0, pmax = 0;
    const int per_sm = std::max(1, tile_blocks_per_sm(npe, 256));
    const int64_t wave = (int64_t)num_sms() * per_sm;
    for (int attempt = 0;; ++attempt) {
        nt = cdiv(nel, P);
        if (nt * 2 > wave) nt = cdiv(nt, wave) * wave;
        nt = std::min(nt, nel);
        h_tep.assign(nt + 1, 0);
        for (int64_t t = 0; t <= nt; ++t) h_tep[t] = (int64_t)((__int128)t * nel / nt);
        pmax = cdiv(nel, nt);
        FEM_TRY(tep.alloc(ar, nt + 1, "tile element ranges"));
        FEM_TRY(ncn.alloc(ar, nt, "tile rows"));
        FEM_TRY(nacc.alloc(ar, nt, "tile entries"));
        FEM_TRY(nbord.alloc(ar, nt, "tile border rows"));
        FEM_CUDA(cudaMemcpyAsync(tep.ptr, h_tep.data(), (nt + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
        TileIn in{m->E, eorder.ptr, tep.ptr, m->rowptr.ptr, m->col.ptr, m->inc_ptr.ptr, hv_thr};
        const unsigned grid = (unsigned)std::min<int64_t>(nt, (int64_t)num_sms() * 4);
        if (npe == 8) k_tile_count<8><<<grid, TP_THREADS, count_smem, s>>>(in, nt, ncn.ptr, nacc.ptr, nbord.ptr);
        else k_tile_count<4><<<grid, TP_THREADS, count_smem, s>>>(in, nt, ncn.ptr, nacc.ptr, nbord.ptr);
        FEM_LAUNCHED("k_tile_count");
        h_ncn.resize(nt);
        h_nacc.resize(nt);
        h_nbord.resize(nt);
        FEM_CUDA(cudaMemcpyAsync(h_ncn.data(), ncn.ptr, nt * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        FEM_CUDA(cudaMemcpyAsync(h_nacc.data(), nacc.ptr, nt * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        FEM_CUDA(cudaMemcpyAsync(h_nbord.data(), nbord.ptr, nt * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        FEM_CUDA(cudaStreamSynchronize(s));
        max_ncn = *std::max_element(h_ncn.begin(), h_ncn.end());
        max_acc = *std::max_element(h_nacc.begin(), h_nacc.end());
        // (the pass's static shared memory stays well inside the 1 KB margin); the
        // tile kernel's own shared memory is checked for its largest form (FP64
        // accumulators and double coordinates), which the same plan serves
        TileMax tm;
        tm.max_acc = max_acc;
        tm.max_epad = cdiv(pmax, TILE_EPAD) * TILE_EPAD;
        tm.max_npad = cdiv(max_ncn, TILE_NPAD) * TILE_NPAD;
        tm.any_hv = m->max_deg > hv_thr;
        const size_t kernel_smem = tile_smem_layout(tm, npe, false, sizeof(double)).total;
        const bool fits = max_acc < 32768 && fill_layout(npe, pmax, max_ncn).total + 1024 <= (size_t)max_optin &&
                          kernel_smem + 1024 <= (size_t)max_optin;
        if (fits) break;
        if (P <= 1 || attempt > 16) {
            set_error("element tiles: one element's rows need %lld accumulator entries; at most 32767 fit",
                      (long long)max_acc);
            return FEM_ERR_UNSUPPORTED;
        }
        P = std::max<int64_t>(1, P / 2);
    }
    T.n_tiles = nt;
    T.tile_elems = (int)P;
    T.max_acc = max_acc;
    T.max_tnodes = max_ncn;
    T.max_elems = pmax;
    T.any_hv = m->max_deg > hv_thr;

    // ---- layout of the plan: each tile's element and row slices padded to 16 bytes
    std::vector<int64_t> h_tnp(nt + 1), h_bofs(nt + 1), h_tepp(nt + 1);
    std::vector<int32_t> h_nel(nt), h_ncn32(nt);
    h_tnp[0] = h_bofs[0] = h_tepp[0] = 0;
    int64_t max_epad = 0, max_npad = 0;
    for (int64_t t = 0; t < nt; ++t) {
        const int64_t ne = h_tep[t + 1] - h_tep[t];
        const int64_t ep = cdiv(ne, TILE_EPAD) * TILE_EPAD, npd = cdiv(h_ncn[t], TILE_NPAD) * TILE_NPAD;
        h_tepp[t + 1] = h_tepp[t] + ep;
        h_tnp[t + 1] = h_tnp[t] + npd;
        h_bofs[t + 1] = h_bofs[t] + h_nbord[t];
        h_nel[t] = (int32_t)ne;
        h_ncn32[t] = (int32_t)h_ncn[t];
        max_epad = std::max(max_epad, ep);
        max_npad = std::max(max_npad, npd);
    }
    const int64_t ntn = h_tnp[nt], nbp = h_bofs[nt], nep = h_tepp[nt];
    int64_t real_tn = 0;
    for (int64_t t = 0; t < nt; ++t) real_tn += h_ncn[t];
    T.n_tnodes = real_tn;
    T.max_epad = max_epad;
    T.max_npad = max_npad;
    if (ntn >= ((int64_t)1 << 32)) {
        set_error("element tiles: too many tile rows (%lld)", (long long)ntn);
        return FEM_ERR_UNSUPPORTED;
    }
    ncn.free();
    nacc.free();
    nbord.free();
    DevBuf<int64_t> bofs;
    FEM_TRY(T.tile_elem_ptr.alloc(ar, nt + 1, "tile element ranges"));
    FEM_TRY(T.tile_node_ptr.alloc(ar, nt + 1, "tile row ranges"));
    FEM_TRY(T.tile_nel.alloc(ar, nt, "tile elements"));
    FEM_TRY(T.tile_ncn.alloc(ar, nt, "tile rows"));
    FEM_TRY(bofs.alloc(ar, nt + 1, "tile border offsets"));
    FEM_CUDA(cudaMemcpyAsync(T.tile_elem_ptr.ptr, h_tepp.data(), (nt + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    FEM_CUDA(cudaMemcpyAsync(T.tile_node_ptr.ptr, h_tnp.data(), (nt + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    FEM_CUDA(cudaMemcpyAsync(T.tile_nel.ptr, h_nel.data(), nt * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    FEM_CUDA(cudaMemcpyAsync(T.tile_ncn.ptr, h_ncn32.data(), nt * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    FEM_CUDA(cudaMemcpyAsync(bofs.ptr, h_bofs.data(), (nt + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    FEM_TRY(T.tile_acc.alloc(ar, nt, "tile entries"));
    FEM_TRY(T.elem_id.alloc(ar, nep, "tile element ids"));
    FEM_TRY(T.elem_color.alloc(ar, nep, "tile element colours"));
    FEM_TRY(T.elem_lnode.alloc(ar, nep * npe, "tile local nodes"));
    FEM_TRY(T.elem_pos.alloc(ar, nep * tile_posw(npe), "tile in-row positions"));
    FEM_TRY(T.node_gid.alloc(ar, ntn, "tile row ids"));
    FEM_TRY(T.node_info.alloc(ar, ntn, "tile row layout"));
    FEM_TRY(T.node_dest.alloc(ar, ntn, "tile row destinations"));
    // padding slots: element id -1 (never integrated), rows of length 0
    FEM_CUDA(cudaMemsetAsync(T.elem_id.ptr, 0xff, nep * sizeof(int32_t), s));
    FEM_CUDA(cudaMemsetAsync(T.elem_color.ptr, 0, nep, s));
    FEM_CUDA(cudaMemsetAsync(T.elem_lnode.ptr, 0, nep * npe * sizeof(uint16_t), s));
    FEM_CUDA(cudaMemsetAsync(T.elem_pos.ptr, 0, nep * tile_posw(npe) * sizeof(uint32_t), s));
    FEM_CUDA(cudaMemsetAsync(T.node_gid.ptr, 0, ntn * sizeof(int32_t), s));
    FEM_CUDA(cudaMemsetAsync(T.node_info.ptr, 0, ntn * sizeof(uint32_t), s));
    FEM_CUDA(cudaMemsetAsync(T.node_dest.ptr, 0, ntn * sizeof(int64_t), s));
    DevBuf<uint64_t> bkeys;
    DevBuf<uint32_t> bvals;
    DevBuf<int> mxc;
    FEM_TRY(bkeys.alloc(ar, nbp, "border pairs"));
    FEM_TRY(bvals.alloc(ar, nbp, "border pair rows"));
    FEM_TRY(mxc.alloc(ar, 1, "max colour"));
    FEM_CUDA(cudaMemsetAsync(mxc.ptr, 0, sizeof(int), s));
    const int tbits = bits_for(nt);
    {
        TileIn in{m->E, eorder.ptr, tep.ptr, m->rowptr.ptr, m->col.ptr, m->inc_ptr.ptr, hv_thr};
        TileOut out{T.tile_node_ptr.ptr, T.tile_elem_ptr.ptr, bofs.ptr, T.tile_acc.ptr, T.elem_id.ptr,
                    T.elem_color.ptr, T.elem_lnode.ptr, reinterpret_cast<uint8_t *>(T.elem_pos.ptr), T.node_gid.ptr,
                    T.node_info.ptr, T.node_dest.ptr, bkeys.ptr, bvals.ptr, tbits, mxc.ptr};
        const FillSmem L = fill_layout(npe, pmax, max_ncn);
        const unsigned grid = (unsigned)std::min<int64_t>(nt, (int64_t)num_sms() * 4);
        if (npe == 8) {
            FEM_CUDA(cudaFuncSetAttribute(k_tile_fill<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total));
            k_tile_fill<8><<<grid, TP_THREADS, L.total, s>>>(in, nt, out, L);
        } else {
            FEM_CUDA(cudaFuncSetAttribute(k_tile_fill<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total));
            k_tile_fill<4><<<grid, TP_THREADS, L.total, s>>>(in, nt, out, L);
        }
        FEM_LAUNCHED("k_tile_fill");
        int h_mxc = 0;
        FEM_TRY(read_scalar(mxc.ptr, &h_mxc, s));
        if (h_mxc >= 255) {
            set_error("element tiles: the colouring of a tile needs more than 255 colours");
            return FEM_ERR_UNSUPPORTED;
        }
        T.n_colors = h_mxc + 1;
    }
    eorder.free();
    tep.free();
    bofs.free();

    // ---- border rows: a row's tiles in ascending order get consecutive partial slots
    int64_t nrows = 0;
    if (nbp > 0) {
        {
            DevBuf<uint64_t> alt;
            DevBuf<uint32_t> altv;
            DevBuf<int64_t> hist;
            FEM_TRY(alt.alloc(ar, nbp, "sort scratch"));
            FEM_TRY(altv.alloc(ar, nbp, "sort scratch"));
            FEM_TRY(hist.alloc(ar, radix_hist_elems(nbp), "sort histogram"));
            FEM_TRY(radix_sort_u64(bkeys.ptr, bvals.ptr, nbp, bits_for(N) + tbits, alt.ptr, altv.ptr, hist.ptr, s));
            FEM_CUDA(cudaStreamSynchronize(s));
        }
        DevBuf<int64_t> flags, start, amt, tmp;
        FEM_TRY(flags.alloc(ar, nbp + 1, "border flags"));
        FEM_TRY(tmp.alloc(ar, scan_tmp_elems(nbp + 1), "scan scratch"));
        k_brow_flags<<<grid_for(nbp), 256, 0, s>>>(bkeys.ptr, nbp, tbits, flags.ptr);
        FEM_LAUNCHED("k_brow_flags");
        FEM_TRY(scan_exclusive_i64(flags.ptr, flags.ptr, nbp, true, tmp.ptr, s));
        FEM_TRY(read_scalar(flags.ptr + nbp, &nrows, s));
        FEM_TRY(start.alloc(ar, nrows + 1, "border row starts"));
        k_brow_start<<<grid_for(nbp + 1), 256, 0, s>>>(bkeys.ptr, flags.ptr, nbp, nrows, tbits, start.ptr);
        FEM_LAUNCHED("k_brow_start");
        FEM_TRY(T.brow_vo.alloc(ar, nrows, "border row offsets"));
        FEM_TRY(T.brow_info.alloc(ar, nrows, "border row layout"));
        FEM_TRY(T.brow_base.alloc(ar, nrows + 1, "border row partials"));
        FEM_TRY(amt.alloc(ar, nrows + 1, "border row sizes"));
        k_brow_amount<<<grid_for(nrows), 256, 0, s>>>(bkeys.ptr, start.ptr, nrows, tbits, m->rowptr.ptr,
                                                      m->inc_ptr.ptr, hv_thr, amt.ptr, T.brow_vo.ptr,
                                                      T.brow_info.ptr);
        FEM_LAUNCHED("k_brow_amount");
        tmp.free();
        FEM_TRY(tmp.alloc(ar, scan_tmp_elems(nrows + 1), "scan scratch"));
        FEM_TRY(scan_exclusive_i64(amt.ptr, T.brow_base.ptr, nrows, true, tmp.ptr, s));
        FEM_TRY(read_scalar(T.brow_base.ptr + nrows, &T.partial_n, s));
        k_brow_dest<<<grid_for(nbp), 256, 0, s>>>(bkeys.ptr, bvals.ptr, flags.ptr, start.ptr, T.brow_base.ptr, nbp,
                                                  tbits, m->rowptr.ptr, m->inc_ptr.ptr, hv_thr, T.node_dest.ptr);
        FEM_LAUNCHED("k_brow_dest");
        FEM_CUDA(cudaStreamSynchronize(s));
    }
    T.n_brows = nrows;
    FEM_CUDA(cudaStreamSynchronize(s));
    T.ready = true;
    return FEM_OK;
}

}  // namespace fem
