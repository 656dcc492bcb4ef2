// symbolic.cu -- the symbolic phase: validation of E, the node -> element
// incidence, the lower-CSR pattern of K, the locality order of the nodes and the
// per-block plan of the numeric kernels.
//
// Pattern (Algorithm 1's Mapping and the structure of the sparse conversion,
// Section 3).  Row i of the lower CSR holds every node j <= i that shares an
// element with i (explicit zeros included: the pattern is structural, as the
// nonzero counts of Table 1 are).  It is built row by row, one warp per row, from
// the elements incident to node i -- the property the paper credits to MILAMIN's
// sparse_create (no global triplet index arrays) -- so its memory is O(npe * nel)
// integers instead of a global sort of npe(npe+1)/2 * nel (row, col) keys.
#include <climits>
#include <functional>
#include <vector>

#include "block_prims.cuh"
#include "mesh.cuh"
#include "numeric.cuh"

namespace fem {

static constexpr int TPB = 256;

static unsigned grid_for(int64_t n, int tpb = TPB) {
    int64_t b = cdiv(n, tpb);
    const int64_t cap = (int64_t)num_sms() * 32;
    return (unsigned)(b < 1 ? 1 : (b > cap ? cap : b));
}

// ------------------------------------------------------------------ validation
__global__ void k_validate(const int32_t *__restrict__ E, int64_t nel, int npe, int64_t N,
                           unsigned long long *bad_index, unsigned long long *bad_repeat) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nel; e += (int64_t)gridDim.x * blockDim.x) {
        int32_t id[8];
        for (int a = 0; a < npe; ++a) id[a] = E[e * npe + a];
        bool bi = false, br = false;
        for (int a = 0; a < npe; ++a) {
            if (id[a] < 0 || (int64_t)id[a] >= N) bi = true;
            for (int b = 0; b < a; ++b)
                if (id[a] == id[b]) br = true;
        }
        if (bi) atomicMin(bad_index, (unsigned long long)e);
        if (br) atomicMin(bad_repeat, (unsigned long long)e);
    }
}

fem_status validate_connectivity(fem_mesh m, cudaStream_t s) {
    DevBuf<unsigned long long> flags;
    FEM_TRY(flags.alloc(m->arena, 2, "validation flags"));
    FEM_CUDA(cudaMemsetAsync(flags.ptr, 0xff, 2 * sizeof(unsigned long long), s));
    k_validate<<<grid_for(m->n_elems), TPB, 0, s>>>(m->E, m->n_elems, m->npe, m->n_nodes, flags.ptr, flags.ptr + 1);
    FEM_LAUNCHED("k_validate");
    unsigned long long h[2];
    FEM_CUDA(cudaMemcpyAsync(h, flags.ptr, sizeof(h), cudaMemcpyDeviceToHost, s));
    FEM_CUDA(cudaStreamSynchronize(s));
    if (h[0] != ~0ull) {
        set_error("element %llu has a node id outside [0, %lld)", h[0], (long long)m->n_nodes);
        return FEM_ERR_INDEX;
    }
    if (h[1] != ~0ull) {
        set_error("element %llu repeats a node", h[1]);
        return FEM_ERR_DEGENERATE;
    }
    return FEM_OK;
}

// ------------------------------------------------------------- locality order
// Nodes sorted (stably) by the 30-bit Morton code of their coordinates in the
// mesh's bounding box.  This is a locality heuristic only: any order gives the
// same K.
__device__ __forceinline__ unsigned long long ord_key(double v) {
    unsigned long long b = (unsigned long long)__double_as_longlong(v);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double ord_val(unsigned long long k) {
    unsigned long long b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
    return __longlong_as_double((long long)b);
}

// The row range (fem_options.host_chunks) holding node g: the last k < nr with
// rows[k] <= g; range 0 when there are none (rows null).
__device__ __forceinline__ int range_of(const int64_t *rows, int nr, int64_t g) {
    int k = 0;
    if (rows)
        for (int lo = 0, hi = nr - 1; lo <= hi;) {
            const int mid = (lo + hi) >> 1;
            if (rows[mid] <= g) { k = mid; lo = mid + 1; } else hi = mid - 1;
        }
    return k;
}

// Bounding box of each row range's nodes (one box when rows is null):
// bb[6k .. 6k+5] = min xyz, max xyz.  A warp whose 32 nodes share a range
// reduces them before its atomics.
template <typename S>
__global__ void k_bbox(const S *__restrict__ X, int64_t N, const int64_t *rows, int nr, unsigned long long *bb) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (N + 31) / 32 * 32;  // every lane of a warp takes the same trips
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nw; i += (int64_t)gridDim.x * blockDim.x) {
        const bool valid = i < N;
        const int r = valid ? range_of(rows, nr, i) : -1;
        double lo[3], hi[3];
        for (int d = 0; d < 3; ++d) {
            const double v = valid ? (double)X[3 * i + d] : 0.0;
            lo[d] = valid ? v : 1e300;
            hi[d] = valid ? v : -1e300;
        }
        const int r0 = __shfl_sync(0xffffffffu, r, 0);
        if (__all_sync(0xffffffffu, r == r0 || r < 0)) {
            for (int d = 0; d < 3; ++d)
                for (int o = 16; o > 0; o >>= 1) {
                    lo[d] = fmin(lo[d], __shfl_down_sync(0xffffffffu, lo[d], o));
                    hi[d] = fmax(hi[d], __shfl_down_sync(0xffffffffu, hi[d], o));
                }
            if (lane == 0 && r0 >= 0)
                for (int d = 0; d < 3; ++d) {
                    atomicMin(&bb[6 * r0 + d], ord_key(lo[d]));
                    atomicMax(&bb[6 * r0 + 3 + d], ord_key(hi[d]));
                }
        } else if (valid) {
            for (int d = 0; d < 3; ++d) {
                atomicMin(&bb[6 * r + d], ord_key(lo[d]));
                atomicMax(&bb[6 * r + 3 + d], ord_key(hi[d]));
            }
        }
    }
}

__device__ __forceinline__ uint32_t spread10(uint32_t v) {
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

// Key of node i: its row range above the 30-bit Morton code of its coordinates
// in that range's bounding box, scaled alike on the three axes.
template <typename S>
__global__ void k_morton(const S *__restrict__ X, int64_t N, const unsigned long long *bb, const int64_t *rows,
                         int nr, uint64_t *keys, uint32_t *vals) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const int r = range_of(rows, nr, i);
        double lo[3], ext[3], w = 0.0, vol = 1.0;
        for (int d = 0; d < 3; ++d) {
            lo[d] = ord_val(bb[6 * r + d]);
            ext[d] = ord_val(bb[6 * r + 3 + d]) - lo[d];
            w = fmax(w, ext[d]);
            vol *= fmax(ext[d], 1e-300);
        }
        // one scale for the three axes (cubic cells, whatever the box's shape)
        const double sc = w > 0 ? 1023.0 / w : 0.0;
        // Ranges: coordinates within half a mean node spacing of the box's faces
        // are moved onto that inset, so a layer of nodes on a face (a plane of a
        // structured numbering cut by the range) keeps one code per axis there
        // instead of straddling a coarse cell boundary, whose far side would hold
        // only that layer's nodes, visited apart from their neighbours.
        const double h = rows ? cbrt(vol / (double)(rows[r + 1] - rows[r])) : 0.0;
        uint32_t q[3];
        for (int d = 0; d < 3; ++d) {
            const double in = fmin(0.5 * h, 0.25 * ext[d]);
            const double v = fmin(fmax((double)X[3 * i + d], lo[d] + in), lo[d] + ext[d] - in);
            double t = (v - lo[d]) * sc;
            t = t < 0 ? 0 : (t > 1023 ? 1023 : t);
            q[d] = (uint32_t)t;
        }
        keys[i] = ((uint64_t)r << 30) | (uint64_t)(spread10(q[0]) | (spread10(q[1]) << 1) | (spread10(q[2]) << 2));
        vals[i] = (uint32_t)i;
    }
}

__global__ void k_iota(int32_t *o, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        o[i] = (int32_t)i;
}

fem_status build_locality_order(fem_mesh m, const void *X, fem_dtype xd, cudaStream_t s) {
    const int64_t N = m->n_nodes;
    // Row ranges of the host pipeline (fem_options.host_chunks, scalar operators):
    // n_r ranges of about N / n_r rows each.  The order then runs range by range,
    // each range along the Morton curve of its own bounding box: a range cut
    // through a plane of a structured numbering would otherwise leave the cut
    // plane's nodes that the global curve visits with the next range's nodes as a
    // scattered tail of this range.
    const int nr = (m->opt.host_chunks > 1 && m->opt.operator_kind != 2 && N > 0)
                       ? (int)std::min<int64_t>(std::min(m->opt.host_chunks, 4096), N)
                       : 1;
    m->chunk_rows.assign(nr + 1, 0);
    for (int k = 0; k <= nr; ++k) m->chunk_rows[k] = (int64_t)k * N / nr;
    FEM_TRY(m->order.alloc(m->arena, N, "node order"));
    if (!X || !m->opt.locality_order) {
        k_iota<<<grid_for(N), TPB, 0, s>>>(m->order.ptr, N);  // ids: already grouped by range
        FEM_LAUNCHED("k_iota");
        return FEM_OK;
    }
    DevBuf<unsigned long long> bb;
    DevBuf<uint64_t> keys, alt;
    DevBuf<uint32_t> alt_vals;
    DevBuf<int64_t> hist, rows;
    FEM_TRY(bb.alloc(m->arena, 6 * (size_t)nr, "bbox"));
    FEM_TRY(keys.alloc(m->arena, N, "morton keys"));
    FEM_TRY(alt.alloc(m->arena, N, "morton keys'"));
    FEM_TRY(alt_vals.alloc(m->arena, N, "morton vals'"));
    FEM_TRY(hist.alloc(m->arena, radix_hist_elems(N), "radix histogram"));
    std::vector<unsigned long long> init(6 * (size_t)nr);
    for (int k = 0; k < nr; ++k)
        for (int d = 0; d < 3; ++d) init[6 * k + d] = ~0ull, init[6 * k + 3 + d] = 0ull;
    FEM_CUDA(cudaMemcpyAsync(bb.ptr, init.data(), init.size() * sizeof(init[0]), cudaMemcpyHostToDevice, s));
    const int64_t *rp = nullptr;
    if (nr > 1) {
        FEM_TRY(rows.alloc(m->arena, nr + 1, "row ranges"));
        FEM_CUDA(cudaMemcpyAsync(rows.ptr, m->chunk_rows.data(), (nr + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
        rp = rows.ptr;
    }
    uint32_t *vals = reinterpret_cast<uint32_t *>(m->order.ptr);
    if (xd == FEM_F64) {
        k_bbox<double><<<grid_for(N), TPB, 0, s>>>((const double *)X, N, rp, nr, bb.ptr);
        FEM_LAUNCHED("k_bbox");
        k_morton<double><<<grid_for(N), TPB, 0, s>>>((const double *)X, N, bb.ptr, rp, nr, keys.ptr, vals);
    } else {
        k_bbox<float><<<grid_for(N), TPB, 0, s>>>((const float *)X, N, rp, nr, bb.ptr);
        FEM_LAUNCHED("k_bbox");
        k_morton<float><<<grid_for(N), TPB, 0, s>>>((const float *)X, N, bb.ptr, rp, nr, keys.ptr, vals);
    }
    FEM_LAUNCHED("k_morton");
    int bits = 0;
    while ((1 << bits) < nr) ++bits;
    FEM_TRY(radix_sort_u64(keys.ptr, vals, N, 30 + bits, alt.ptr, alt_vals.ptr, hist.ptr, s));
    FEM_CUDA(cudaStreamSynchronize(s));  // temporaries are freed on return
    return FEM_OK;
}

// ------------------------------------------------------------------ incidence
__global__ void k_degree(const int32_t *__restrict__ E, int64_t n_ent, unsigned long long *deg) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n_ent; t += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&deg[E[t]], 1ull);
}

__global__ void k_inc_fill(const int32_t *__restrict__ E, int64_t n_ent, int npe, const int64_t *inc_ptr,
                           unsigned int *cursor, int32_t *inc_elem) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n_ent; t += (int64_t)gridDim.x * blockDim.x) {
        const int32_t g = E[t];
        const unsigned k = atomicAdd(&cursor[g], 1u);
        inc_elem[inc_ptr[g] + k] = (int32_t)(t / npe);
    }
}

// Insertion sort of each node's (short) list of incident elements, so that the
// incidence does not depend on the order in which the atomics were served.
__global__ void k_inc_sort(const int64_t *inc_ptr, int32_t *inc_elem, int64_t N) {
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < N; g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = inc_ptr[g], e = inc_ptr[g + 1];
        for (int64_t i = b + 1; i < e; ++i) {
            const int32_t v = inc_elem[i];
            int64_t j = i - 1;
            while (j >= b && inc_elem[j] > v) {
                inc_elem[j + 1] = inc_elem[j];
                --j;
            }
            inc_elem[j + 1] = v;
        }
    }
}

__global__ void k_max_deg(const int64_t *inc_ptr, int64_t N, unsigned long long *mx) {
    unsigned long long m = 0;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < N; g += (int64_t)gridDim.x * blockDim.x)
        m = max(m, (unsigned long long)(inc_ptr[g + 1] - inc_ptr[g]));
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(mx, m);
}

// ------------------------------------------------------------- row pattern
// One warp per row i.  The warp lists the nodes j <= i of every element incident
// to i (cap >= max degree * npe candidates, in shared memory), drops repeats, and
// ranks each distinct j among the others: that rank is its position in the row.
// count pass: cnt[i] = number of distinct j; fill pass: col[rowptr[i] + rank] = j.
template <int NPE>
__global__ void k_row_pattern(const int32_t *__restrict__ E, const int64_t *__restrict__ inc_ptr,
                              const int32_t *__restrict__ inc_elem, int64_t N, int cap, int64_t *cnt,
                              const int64_t *__restrict__ rowptr, int32_t *col) {
    extern __shared__ int32_t pat_buf[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    int32_t *buf = pat_buf + (size_t)wib * cap;
    for (int64_t i = (int64_t)blockIdx.x * wpb + wib; i < N; i += (int64_t)gridDim.x * wpb) {
        const int64_t b0 = inc_ptr[i];
        const int n = (int)(inc_ptr[i + 1] - b0) * NPE;
        // candidates gathered four per lane at a time: the incidence loads, then the
        // connectivity loads, each four-wide
        for (int t0 = lane; t0 < n; t0 += 128) {
            int32_t e[4], g[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int t = t0 + 32 * u;
                e[u] = t < n ? inc_elem[b0 + t / NPE] : 0;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int t = t0 + 32 * u;
                g[u] = t < n ? E[(int64_t)e[u] * NPE + t % NPE] : 0;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int t = t0 + 32 * u;
                if (t < n) buf[t] = (g[u] <= i) ? g[u] : INT_MAX;
            }
        }
        __syncwarp();
        // mark repeats (keep the first occurrence); items of this lane: t = lane + 32 k
        unsigned long long dup = 0;
        for (int t = lane, k = 0; t < n; t += 32, ++k) {
            const int32_t v = buf[t];
            bool d = (v == INT_MAX);
            for (int u = 0; u < t && !d; ++u) d = (buf[u] == v);
            if (d) dup |= 1ull << k;
        }
        __syncwarp();
        for (int t = lane, k = 0; t < n; t += 32, ++k)
            if (dup >> k & 1ull) buf[t] = INT_MAX;
        __syncwarp();
        int mine = 0;
        for (int t = lane; t < n; t += 32) {
            const int32_t v = buf[t];
            if (v == INT_MAX) continue;
            ++mine;
            if (col) {
                int rank = 0;
                for (int u = 0; u < n; ++u) rank += (buf[u] < v);
                col[rowptr[i] + rank] = v;
            }
        }
        if (cnt) {
            for (int o = 16; o > 0; o >>= 1) mine += __shfl_down_sync(0xffffffffu, mine, o);
            if (lane == 0) cnt[i] = mine;
        }
        __syncwarp();
    }
}

// Ascending bitonic sort of the 32 K values a warp holds, K per lane in blocked
// order (value t = lane K + k): pairs closer than K swap in registers, the others
// through shuffles.
template <int K>
__device__ __forceinline__ void warp_bitonic(int32_t (&v)[K], int lane) {
#pragma unroll
    for (int size = 2; size <= 32 * K; size <<= 1)
#pragma unroll
        for (int j = size >> 1; j > 0; j >>= 1) {
            if (j < K) {
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    const int kp = k ^ j;
                    if (kp > k) {
                        const bool up = ((lane * K + k) & size) == 0;
                        const int32_t a = v[k], b = v[kp];
                        if ((a > b) == up) {
                            v[k] = b;
                            v[kp] = a;
                        }
                    }
                }
            } else {
                const int pl = j / K;
                const bool lower = (lane & pl) == 0;
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    const int32_t o = __shfl_xor_sync(0xffffffffu, v[k], pl);
                    const bool up = ((lane * K + k) & size) == 0;
                    v[k] = (lower == up) ? min(v[k], o) : max(v[k], o);
                }
            }
        }
}

// k_row_pattern for rows of at most 32 K candidates: the warp sorts them in
// registers, so repeats are neighbours and a column's position in its row is the
// number of distinct smaller columns (a ballot count), not a scan over all
// candidates.  Same passes and outputs as k_row_pattern, and with tmp (S slots
// a row) the count pass also keeps each row's first S columns there, so that
// the fill pass copies the rows of at most S entries instead of rebuilding them.
template <int NPE, int K>
__global__ void k_row_pattern_reg(const int32_t *__restrict__ E, const int64_t *__restrict__ inc_ptr,
                                  const int32_t *__restrict__ inc_elem, int64_t N, int64_t *cnt,
                                  const int64_t *__restrict__ rowptr, int32_t *col, int32_t *tmp, int S) {
    const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    for (int64_t i = (int64_t)blockIdx.x * wpb + (threadIdx.x >> 5); i < N; i += (int64_t)gridDim.x * wpb) {
        if (col && tmp) {
            const int64_t r0 = rowptr[i], len = rowptr[i + 1] - r0;
            if (len <= S) {  // warp-uniform
                if (lane < len) col[r0 + lane] = tmp[i * S + lane];
                continue;
            }
        }
        const int64_t b0 = inc_ptr[i];
        const int n = (int)(inc_ptr[i + 1] - b0) * NPE;
        int32_t e[K], v[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int t = lane * K + k;
            e[k] = t < n ? inc_elem[b0 + t / NPE] : -1;
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int t = lane * K + k;
            const int32_t g = e[k] >= 0 ? E[(int64_t)e[k] * NPE + t % NPE] : INT_MAX;
            v[k] = g <= i ? g : INT_MAX;
        }
        warp_bitonic<K>(v, lane);
        // first occurrences: the predecessor of value t is v[k-1], or lane-1's last
        const int32_t prev_last = __shfl_up_sync(0xffffffffu, v[K - 1], 1);
        unsigned first = 0;
        int mine = 0;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int32_t pv = k > 0 ? v[k - 1] : (lane > 0 ? prev_last : INT_MIN);
            if (v[k] != INT_MAX && v[k] != pv) {
                first |= 1u << k;
                ++mine;
            }
        }
        int incl = mine;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (col) {
            int r = incl - mine;
            const int64_t base = rowptr[i];
#pragma unroll
            for (int k = 0; k < K; ++k)
                if (first >> k & 1u) col[base + r++] = v[k];
        } else if (tmp) {
            int r = incl - mine;
#pragma unroll
            for (int k = 0; k < K; ++k)
                if (first >> k & 1u) {
                    if (r < S) tmp[i * S + r] = v[k];
                    ++r;
                }
        }
        if (cnt && lane == 31) cnt[i] = incl;
    }
}

__global__ void k_row_len_max(const int64_t *rowptr, int64_t N, unsigned long long *mx) {
    unsigned long long m = 0;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < N; g += (int64_t)gridDim.x * blockDim.x)
        m = max(m, (unsigned long long)(rowptr[g + 1] - rowptr[g]));
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(mx, m);
}

// ------------------------------------------------------------------- patches
// len_in_order[k] = length of row order[k]
__global__ void k_len_in_order(const int32_t *order, const int64_t *rowptr, int64_t N, int64_t *len) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) {
        const int32_t g = order[k];
        len[k] = rowptr[g + 1] - rowptr[g];
    }
}

// first index with pre[k] >= p * cap (lower bound), p = 0..npatch-1; ptr[npatch] = N
// Patch bounds inside row ranges.  Range k covers positions [c_row[k], c_row[k+1])
// of the node order and patches [c_patch[k], c_patch[k+1]); its patch j starts at
// the first position whose row-length prefix reaches pre[c_row[k]] + j * c_cap[k].
// One range spanning every node is the plain cut into patches of `cap` entries.
__global__ void k_patch_bounds(const int64_t *pre, const int64_t *c_row, const int64_t *c_patch,
                               const int64_t *c_cap, int nc, int64_t npatch, int64_t *ptr) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p <= npatch; p += (int64_t)gridDim.x * blockDim.x) {
        if (p == npatch) {
            ptr[p] = c_row[nc];
            continue;
        }
        int k = 0;  // the range holding patch p: the last with c_patch[k] <= p
        for (int lo = 0, hi = nc - 1; lo <= hi;) {
            const int mid = (lo + hi) >> 1;
            if (c_patch[mid] <= p) { k = mid; lo = mid + 1; } else hi = mid - 1;
        }
        const int64_t j = p - c_patch[k], r0 = c_row[k];
        if (j == 0) {
            ptr[p] = r0;
            continue;
        }
        const int64_t target = pre[r0] + j * c_cap[k];
        int64_t lo = r0, hi = c_row[k + 1];
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (pre[mid] < target) lo = mid + 1; else hi = mid;
        }
        ptr[p] = lo;
    }
}

__global__ void k_patch_nodes(const int32_t *order, const int64_t *pre, const int64_t *pn_ptr, int64_t N,
                              int64_t npatch, const int64_t *rowptr, const int64_t *inc_ptr, int hv_thr,
                              int32_t *node_patch, int32_t *own_idx, int32_t *own_row, int64_t *own_rowptr,
                              int32_t *own_acc, uint8_t *own_hv) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) {
        // the patch holding position k: the last p < npatch with pn_ptr[p] <= k
        int64_t p = 0;
        for (int64_t lo = 0, hi = npatch - 1; lo <= hi;) {
            const int64_t mid = (lo + hi) >> 1;
            if (pn_ptr[mid] <= k) { p = mid; lo = mid + 1; } else hi = mid - 1;
        }
        const int32_t g = order[k];
        node_patch[g] = (int32_t)p;
        own_idx[g] = (int32_t)(k - pn_ptr[p]);
        own_row[k] = g;
        own_rowptr[k] = rowptr[g];
        own_acc[k] = (int32_t)(pre[k] - pre[pn_ptr[p]]);
        own_hv[k] = (inc_ptr[g + 1] - inc_ptr[g]) > hv_thr ? 1 : 0;
    }
}

__global__ void k_patch_acc(const int64_t *pre, const int64_t *pn_ptr, int64_t npatch, int32_t *acc) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npatch; p += (int64_t)gridDim.x * blockDim.x)
        acc[p] = (int32_t)(pre[pn_ptr[p + 1]] - pre[pn_ptr[p]]);
}

// CSR start of each row range: val[k] = rowptr[row[k]], k = 0 .. nr.
__global__ void k_range_vals(const int64_t *rowptr, const int64_t *row, int nr, int64_t *val) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k <= nr; k += gridDim.x * blockDim.x) val[k] = rowptr[row[k]];
}

// ------------------------------------------------------------- closure lists
__global__ void k_unique_flags(const uint64_t *keys, int64_t n, int64_t *flags) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        flags[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1 : 0;
}

__global__ void k_unique_compact(const uint64_t *keys, int64_t n, const int64_t *pos, uint64_t *out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (i == 0 || keys[i] != keys[i - 1]) out[pos[i]] = keys[i];
}

// ptr[p] = first index whose key >> shift >= p (keys sorted); ptr[np] = n
__global__ void k_segment_ptr(const uint64_t *keys, int64_t n, int shift, int64_t np, int64_t *ptr) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p <= np; p += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = n;
        while (lo < hi) {
            int64_t mid = (lo + hi) >> 1;
            if ((keys[mid] >> shift) < (uint64_t)p) lo = mid + 1; else hi = mid;
        }
        ptr[p] = lo;
    }
}

// Greedy colouring of a patch's closure (elements in ascending id): an element
// takes the lowest colour not yet used by an element sharing an owned node with
// it.  Owned-node colour sets are 256-bit masks in shared memory (colours 0-254;
// 255 marks an element no colour was left for); the element -> owned-node table is
// staged chunk by chunk so that the serial loop runs from shared memory.
static constexpr int COLOR_CHUNK = 256;
static constexpr int COLOR_WORDS = 4;

template <int NPE>
__global__ void k_color(const uint64_t *ckeys, const int64_t *pe_ptr, const int64_t *pn_ptr, const int32_t *E,
                        const int32_t *node_patch, const int32_t *own_idx, int64_t npatch, int64_t p0,
                        uint8_t *color_out, int *max_color) {
    extern __shared__ unsigned long long col_smem[];
    for (int64_t p = blockIdx.x; p < npatch; p += gridDim.x) {
        const int nown = (int)(pn_ptr[p + 1] - pn_ptr[p]);
        unsigned long long *mask = col_smem;                                            // [4 * nown]
        int16_t *tab = reinterpret_cast<int16_t *>(col_smem + COLOR_WORDS * nown);      // [COLOR_CHUNK * NPE]
        for (int i = threadIdx.x; i < COLOR_WORDS * nown; i += blockDim.x) mask[i] = 0;
        const int64_t b = pe_ptr[p], n = pe_ptr[p + 1] - b;
        int local_max = -1;
        for (int64_t c0 = 0; c0 < n; c0 += COLOR_CHUNK) {
            const int cn = (int)min((int64_t)COLOR_CHUNK, n - c0);
            __syncthreads();
            // the chunk's element -> owned-node table: U entries per thread at a time,
            // so that each of the three dependent loads goes out U-wide
            constexpr int U = 8;
            const int ntab = cn * NPE;
            for (int t0 = threadIdx.x; t0 < ntab; t0 += blockDim.x * U) {
                int64_t e[U];
                int32_t g[U], np_[U], oi[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int t = t0 + u * blockDim.x;
                    e[u] = t < ntab ? (int64_t)(uint32_t)ckeys[b + c0 + t / NPE] : 0;
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int t = t0 + u * blockDim.x;
                    g[u] = t < ntab ? E[e[u] * NPE + t % NPE] : 0;
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    np_[u] = node_patch[g[u]];
                    oi[u] = own_idx[g[u]];
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int t = t0 + u * blockDim.x;
                    if (t < ntab) tab[t] = np_[u] == (int32_t)(p0 + p) ? (int16_t)oi[u] : (int16_t)-1;
                }
            }
            __syncthreads();
            // the greedy pass, element after element, by warp 0: lane (a, w) holds
            // word w of node a's used-colour mask, the words of the element's owned
            // nodes are or-ed across lanes, and the lowest free colour is the first
            // zero bit of the lowest word that has one
            if (threadIdx.x < 32) {
                const int lane = threadIdx.x, a = lane >> 2, w = lane & (COLOR_WORDS - 1);
                for (int i = 0; i < cn; ++i) {
                    const int o = a < NPE ? tab[i * NPE + a] : -1;
                    unsigned long long mw = o >= 0 ? mask[COLOR_WORDS * o + w] : 0ull;
                    mw |= __shfl_xor_sync(0xffffffffu, mw, 4);
                    mw |= __shfl_xor_sync(0xffffffffu, mw, 8);
                    mw |= __shfl_xor_sync(0xffffffffu, mw, 16);
                    const unsigned freew = __ballot_sync(0xffffffffu, lane < COLOR_WORDS && ~mw != 0ull);
                    int c = 255;
                    if (freew) {  // warp-uniform
                        const int w0 = __ffs((int)freew) - 1;
                        const unsigned long long m0 = __shfl_sync(0xffffffffu, mw, w0);
                        c = 64 * w0 + __ffsll((long long)~m0) - 1;
                    }
                    if (c > 254) c = 255;
                    if (lane == 0) color_out[b + c0 + i] = (uint8_t)c;
                    if (c < 255 && o >= 0 && w == (c >> 6)) mask[COLOR_WORDS * o + w] |= 1ull << (c & 63);
                    __syncwarp();
                    local_max = max(local_max, c);
                }
            }
        }
        if (threadIdx.x == 0) atomicMax(max_color, local_max);
        __syncthreads();
    }
}

// Colouring order: closure elements grouped by patch, then by the smallest
// patch-local index of their owned nodes (owned nodes follow the Morton order),
// so the greedy colouring sweeps each patch in space; key = (patch << 15) | that
// index, payload = the entry's position.
template <int NPE>
__global__ void k_sweep_keys(const uint64_t *ckeys, int64_t nce, const int32_t *__restrict__ E,
                             const int32_t *node_patch, const int32_t *own_idx, int64_t p0, uint64_t *keys,
                             uint32_t *vals) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nce; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = ckeys[i];
        const int64_t pl = (int64_t)(k >> 32), e = (int64_t)(k & 0xffffffffull);
        int mo = 32767;
#pragma unroll
        for (int a = 0; a < NPE; ++a) {
            const int32_t g = E[e * NPE + a];
            if (node_patch[g] == (int32_t)(p0 + pl)) mo = min(mo, own_idx[g]);
        }
        keys[i] = ((uint64_t)pl << 15) | (uint64_t)mo;
        vals[i] = (uint32_t)i;
    }
}

__global__ void k_gather_u64(const uint64_t *in, const uint32_t *perm, int64_t n, uint64_t *out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = in[perm[i]];
}

__global__ void k_color_keys(const uint64_t *ckeys, const uint8_t *color, int64_t n, uint64_t *out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = ckeys[i];
        out[i] = ((k >> 32) << 40) | ((uint64_t)color[i] << 32) | (k & 0xffffffffull);
    }
}

__global__ void k_cnode_pairs(const uint64_t *ckeys, int64_t nce, int npe, const int32_t *E, uint64_t *keys) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nce * npe; t += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = ckeys[t / npe];
        const uint64_t p = k >> 40;
        const int64_t e = (int64_t)(k & 0xffffffffull);
        keys[t] = (p << 32) | (uint64_t)(uint32_t)E[e * npe + t % npe];
    }
}

__global__ void k_cnode_own(const uint64_t *cn_keys, int64_t ncn, int64_t p0, const int32_t *node_patch,
                            const int32_t *own_idx, int32_t *gid, int32_t *own) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < ncn; j += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = cn_keys[j];
        const int32_t g = (int32_t)(k & 0xffffffffull);
        const int32_t p = (int32_t)(p0 + (int64_t)(k >> 32));
        gid[j] = g;
        own[j] = node_patch[g] == p ? own_idx[g] : -1;
    }
}

// Per closure element: id, colour, closure-local node indices (binary search in
// the patch's sorted closure-node list) and, for every packed pair (a, b), the
// position of min(g_a, g_b) within row max(g_a, g_b) of the pattern, plus the
// pair's target in the patch's accumulators (celem_aidx, see PlanView).
struct OwnTables {
    const int32_t *node_patch, *own_idx, *own_acc;
    const int64_t *patch_node_ptr;  // global patch index
    const uint8_t *own_hv;
    const int64_t *pe_ptr;          // closure-element range of each patch of the closure
    int64_t p0;
    int32_t trash;                  // first of the 32 scratch accumulators (the plan's max_acc)
};

// Position of packed pair (a, b) of an element with node ids g in its lower-CSR
// row: the pair's row is its node with the larger global id; the diagonal closes
// its lower row; an off-diagonal pair's position is a binary search of the
// smaller id in that (ascending) row.  r0, rl: start and length of each node's row.
template <int NPE>
__device__ __forceinline__ int pair_position(const int32_t (&g)[NPE], const int64_t (&r0)[NPE], const int (&rl)[NPE],
                                             int a, int b, const int32_t *__restrict__ col) {
    if (a == b) return rl[a] - 1;
    const bool ra = g[a] > g[b];
    const int64_t rb = ra ? r0[a] : r0[b];
    const int32_t v = ra ? g[b] : g[a];
    int lo = 0, n = ra ? rl[a] : rl[b];
    while (n > 1) {
        const int half = n >> 1;
        if (col[rb + lo + half] <= v) lo += half;
        n -= half;
    }
    return lo;
}

template <int NPE>
// One block per patch: the patch's closure-node ids (ascending) are staged in
// shared memory, so that the closure-local index of each element node is a
// binary search there rather than a chain of dependent global loads.  The in-row
// positions (pos) are written only when the closures carry them (pos non-null).
__global__ void __launch_bounds__(256, 3) k_celem_fill(const uint64_t *ckeys, int64_t np_, const int32_t *__restrict__ E,
                             const uint64_t *cn_keys, const int64_t *pc_ptr, const int64_t *__restrict__ rowptr,
                             const int32_t *__restrict__ col, int pos_stride, OwnTables ot, int32_t *celem_id,
                             uint8_t *celem_color, uint16_t *lnode, uint8_t *pos, uint16_t *aidx) {
    extern __shared__ int32_t cn_gid[];
    const int64_t nce = ot.pe_ptr[np_];
  for (int64_t pb = blockIdx.x; pb < np_; pb += gridDim.x) {
    const int64_t cb = pc_ptr[pb];
    const int ncn = (int)(pc_ptr[pb + 1] - cb);
    for (int j = threadIdx.x; j < ncn; j += blockDim.x) cn_gid[j] = (int32_t)(uint32_t)cn_keys[cb + j];
    __syncthreads();
    for (int64_t i = ot.pe_ptr[pb] + threadIdx.x; i < ot.pe_ptr[pb + 1]; i += blockDim.x) {
        const uint64_t k = ckeys[i];
        const uint64_t p = k >> 40;
        const int64_t e = (int64_t)(k & 0xffffffffull);
        celem_id[i] = (int32_t)e;
        celem_color[i] = (uint8_t)((k >> 32) & 0xff);
        int32_t g[NPE];
        uint32_t lw[NPE / 2];  // the local indices, two to a word
#pragma unroll
        for (int a = 0; a < NPE; ++a) {
            g[a] = E[e * NPE + a];
            int lo = 0, hi = ncn;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (cn_gid[mid] < g[a]) lo = mid + 1; else hi = mid;
            }
            if (a & 1) lw[a >> 1] |= (uint32_t)lo << 16; else lw[a >> 1] = (uint32_t)lo;
        }
        if constexpr (NPE == 8) reinterpret_cast<uint4 *>(lnode)[i] = make_uint4(lw[0], lw[1], lw[2], lw[3]);
        else reinterpret_cast<uint2 *>(lnode)[i] = make_uint2(lw[0], lw[1]);
        const int64_t gp = ot.p0 + (int64_t)p;
        const int64_t nb = ot.patch_node_ptr[gp];
        // Each element node x as a row: its start and length, and the row's
        // owner data.
        int64_t r0[NPE];
        int rl[NPE], base[NPE], hvk[NPE];
        bool own[NPE];
#pragma unroll
        for (int x = 0; x < NPE; ++x) {
            r0[x] = rowptr[g[x]];
            rl[x] = (int)(rowptr[g[x] + 1] - r0[x]);
            own[x] = ot.node_patch[g[x]] == gp;
            base[x] = 0;
            hvk[x] = -1;
            if (own[x]) {
                const int32_t kr = ot.own_idx[g[x]];
                base[x] = ot.own_acc[nb + kr];
                if (ot.own_hv[nb + kr]) hvk[x] = kr;
            }
        }
        // positions four to a word, targets two to a word (word-major), each word
        // stored once complete; pos_stride is a multiple of 4, its padding bytes
        // written as zeros
        constexpr int NP = NPE * (NPE + 1) / 2;
        static_assert(NP % 2 == 0, "targets pair up into words");
        uint32_t *pos32 = reinterpret_cast<uint32_t *>(pos + i * pos_stride);
        uint32_t *aidx32 = reinterpret_cast<uint32_t *>(aidx);
        uint32_t pw = 0, alo = 0;
        int q = 0;
#pragma unroll
        for (int a = 0; a < NPE; ++a)
#pragma unroll
            for (int b = 0; b <= a; ++b, ++q) {
                // the searches of an element's pairs are independent of one another
                const bool ra = g[a] > g[b];
                const int ps = pair_position<NPE>(g, r0, rl, a, b, col);
                pw |= (uint32_t)(ps & 0xff) << (8 * (q & 3));
                if ((q & 3) == 3 || q == NP - 1) {
                    if (pos) pos32[q >> 2] = pw;
                    pw = 0;
                }
                // a pair whose row the patch does not own goes to a scratch slot of
                // the lane that will hold the element, never read
                uint32_t t = (uint32_t)(ot.trash + ((i - ot.pe_ptr[p]) & 31));
                if (ra ? own[a] : own[b]) {
                    if (a == b && hvk[a] >= 0) t = AIDX_HV | (uint32_t)hvk[a];
                    else t = (uint32_t)((ra ? base[a] : base[b]) + ps);
                }
                // word q/2 of element i, low half for even q
                if (q & 1) aidx32[(int64_t)(q >> 1) * nce + i] = alo | ((t & 0xffffu) << 16);
                else alo = t & 0xffffu;
            }
        if (pos)
            for (int w = (NP + 3) / 4; w < pos_stride / 4; ++w) pos32[w] = 0;
    }
    __syncthreads();
  }
}

// The in-row positions of every closure element of an existing closure (the
// backward pass reads them; closures built before the first backward call do not
// carry them): the same positions k_celem_fill writes, from the element's ids.
template <int NPE>
__global__ void k_celem_pos(const int32_t *__restrict__ celem_id, int64_t nce, const int32_t *__restrict__ E,
                            const int64_t *__restrict__ rowptr, const int32_t *__restrict__ col, int pos_stride,
                            uint8_t *pos) {
    constexpr int NP = NPE * (NPE + 1) / 2;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nce; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = celem_id[i];
        int32_t g[NPE];
        int64_t r0[NPE];
        int rl[NPE];
#pragma unroll
        for (int x = 0; x < NPE; ++x) {
            g[x] = E[e * NPE + x];
            r0[x] = rowptr[g[x]];
            rl[x] = (int)(rowptr[g[x] + 1] - r0[x]);
        }
        uint32_t *pos32 = reinterpret_cast<uint32_t *>(pos + i * pos_stride);
        uint32_t pw = 0;
        int q = 0;
#pragma unroll
        for (int a = 0; a < NPE; ++a)
#pragma unroll
            for (int b = 0; b <= a; ++b, ++q) {
                pw |= (uint32_t)(pair_position<NPE>(g, r0, rl, a, b, col) & 0xff) << (8 * (q & 3));
                if ((q & 3) == 3 || q == NP - 1) {
                    pos32[q >> 2] = pw;
                    pw = 0;
                }
            }
        for (int w = (NP + 3) / 4; w < pos_stride / 4; ++w) pos32[w] = 0;
    }
}

// One pass of the row pattern (cnt: counts; else the columns at rowptr) over
// rows of at most cap candidates: sorted in registers up to 256 candidates, else
// by the shared-memory kernel.  That kernel's shared memory above the 48 KB
// default (a node in up to 2048 / npe elements needs up to 64 KB for 8 warps)
// is opted in per launch.
static fem_status launch_row_pattern(const int32_t *E, int npe, int64_t N, const int64_t *inc_ptr,
                                     const int32_t *inc_elem, int cap, int64_t *cnt, const int64_t *rowptr,
                                     int32_t *col, cudaStream_t s, int32_t *tmp = nullptr, int S = 0) {
    const int wpb = 8;
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(cdiv(N, wpb), (int64_t)num_sms() * 64));
#define FEM_RP(K)                                                                                           \
    do {                                                                                                    \
        if (npe == 8) k_row_pattern_reg<8, K><<<grid, wpb * 32, 0, s>>>(E, inc_ptr, inc_elem, N, cnt, rowptr, col, tmp, S); \
        else k_row_pattern_reg<4, K><<<grid, wpb * 32, 0, s>>>(E, inc_ptr, inc_elem, N, cnt, rowptr, col, tmp, S);          \
        FEM_LAUNCHED("k_row_pattern_reg");                                                                  \
        return FEM_OK;                                                                                      \
    } while (0)
    if (cap <= 64) FEM_RP(2);
    if (cap <= 128) FEM_RP(4);
    if (cap <= 256) FEM_RP(8);
#undef FEM_RP
    const size_t smem = (size_t)wpb * (cap > 0 ? cap : 1) * sizeof(int32_t);
    if (smem > (48u << 10)) {
        if (npe == 8) FEM_CUDA(cudaFuncSetAttribute(k_row_pattern<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        else FEM_CUDA(cudaFuncSetAttribute(k_row_pattern<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    }
    if (npe == 8) k_row_pattern<8><<<grid, wpb * 32, smem, s>>>(E, inc_ptr, inc_elem, N, cap, cnt, rowptr, col);
    else k_row_pattern<4><<<grid, wpb * 32, smem, s>>>(E, inc_ptr, inc_elem, N, cap, cnt, rowptr, col);
    FEM_LAUNCHED("k_row_pattern");
    return FEM_OK;
}


// --------------------------------------------------------------- orchestration
static int bits_for(int64_t v) {
    int b = 1;
    while ((v >> b) != 0) ++b;
    return b;
}

template <typename T>
static fem_status read_scalar(const T *dev, T *host, cudaStream_t s) {
    FEM_CUDA(cudaMemcpyAsync(host, dev, sizeof(T), cudaMemcpyDeviceToHost, s));
    FEM_CUDA(cudaStreamSynchronize(s));
    return FEM_OK;
}

static fem_status sort_unique(Arena &ar, DevBuf<uint64_t> &keys, int64_t n, int key_bits, DevBuf<uint64_t> &out,
                              int64_t *n_out, cudaStream_t s) {
    DevBuf<uint64_t> alt;
    DevBuf<int64_t> hist, flags;
    FEM_TRY(alt.alloc(ar, n, "sort scratch"));
    FEM_TRY(hist.alloc(ar, radix_hist_elems(n), "sort histogram"));
    FEM_TRY(radix_sort_u64(keys.ptr, nullptr, n, key_bits, alt.ptr, nullptr, hist.ptr, s));
    hist.free();
    FEM_TRY(flags.alloc(ar, n + 1, "unique flags"));
    k_unique_flags<<<grid_for(n), TPB, 0, s>>>(keys.ptr, n, flags.ptr);
    FEM_LAUNCHED("k_unique_flags");
    DevBuf<int64_t> tmp;
    FEM_TRY(tmp.alloc(ar, scan_tmp_elems(n + 1), "scan scratch"));
    FEM_TRY(scan_exclusive_i64(flags.ptr, flags.ptr, n, true, tmp.ptr, s));
    FEM_TRY(read_scalar(flags.ptr + n, n_out, s));
    alt.free();
    FEM_TRY(out.alloc(ar, *n_out, "unique keys"));
    k_unique_compact<<<grid_for(n), TPB, 0, s>>>(keys.ptr, n, flags.ptr, out.ptr);
    FEM_LAUNCHED("k_unique_compact");
    return FEM_OK;
}

fem_status build_pattern(fem_mesh m, cudaStream_t s) {
    Arena &ar = m->arena;
    const int64_t N = m->n_nodes, npe = m->npe, n_ent = m->n_elems * npe;

    // ---- node -> element incidence
    FEM_TRY(m->inc_ptr.alloc(ar, N + 1, "incidence pointers"));
    FEM_TRY(m->inc_elem.alloc(ar, n_ent, "incidence lists"));
    {
        DevBuf<int64_t> deg, tmp;
        DevBuf<unsigned int> cursor;
        FEM_TRY(deg.alloc(ar, N + 1, "degrees"));
        FEM_CUDA(cudaMemsetAsync(deg.ptr, 0, (N + 1) * sizeof(int64_t), s));
        k_degree<<<grid_for(n_ent), TPB, 0, s>>>(m->E, n_ent, reinterpret_cast<unsigned long long *>(deg.ptr));
        FEM_LAUNCHED("k_degree");
        FEM_TRY(tmp.alloc(ar, scan_tmp_elems(N + 1), "scan scratch"));
        FEM_TRY(scan_exclusive_i64(deg.ptr, m->inc_ptr.ptr, N, true, tmp.ptr, s));
        deg.free();
        FEM_TRY(cursor.alloc(ar, N, "incidence cursors"));
        FEM_CUDA(cudaMemsetAsync(cursor.ptr, 0, N * sizeof(unsigned int), s));
        k_inc_fill<<<grid_for(n_ent), TPB, 0, s>>>(m->E, n_ent, (int)npe, m->inc_ptr.ptr, cursor.ptr, m->inc_elem.ptr);
        FEM_LAUNCHED("k_inc_fill");
        k_inc_sort<<<grid_for(N), TPB, 0, s>>>(m->inc_ptr.ptr, m->inc_elem.ptr, N);
        FEM_LAUNCHED("k_inc_sort");
    }
    unsigned long long max_deg = 0;
    {
        DevBuf<unsigned long long> mx;
        FEM_TRY(mx.alloc(ar, 1, "max"));
        FEM_CUDA(cudaMemsetAsync(mx.ptr, 0, sizeof(unsigned long long), s));
        k_max_deg<<<grid_for(N), TPB, 0, s>>>(m->inc_ptr.ptr, N, mx.ptr);
        FEM_LAUNCHED("k_max_deg");
        FEM_TRY(read_scalar(mx.ptr, &max_deg, s));
    }
    m->max_deg = (int64_t)max_deg;
    const int cap = (int)(max_deg * npe);
    if (cap > 64 * 32) {
        set_error("a node belongs to %llu elements; at most %d are supported", max_deg, (int)(64 * 32 / npe));
        return FEM_ERR_UNSUPPORTED;
    }

    // ---- lower-CSR pattern, one warp per row
    FEM_TRY(m->rowptr.alloc(ar, N + 1, "rowptr"));
    {
        DevBuf<int64_t> cnt, tmp;
        FEM_TRY(cnt.alloc(ar, N + 1, "row counts"));
        // the count pass keeps up to S columns a row (when the budget allows the
        // N S slots; the register-sorted kernel only), so that the fill pass copies
        const int S = npe == 8 ? 16 : 32;
        DevBuf<int32_t> rows;
        const size_t rows_bytes = (size_t)N * S * sizeof(int32_t);
        if (cap <= 256 && (!ar.budget || ar.live + ar.kept + rows_bytes <= ar.budget) &&
            rows.alloc(ar, (size_t)N * S, "row columns (first pass)") != FEM_OK) {
            cudaGetLastError();
            rows.free();
        }
        FEM_TRY(launch_row_pattern(m->E, (int)npe, N, m->inc_ptr.ptr, m->inc_elem.ptr, cap, cnt.ptr, nullptr, nullptr,
                                   s, rows.ptr, rows.ptr ? S : 0));
        FEM_TRY(tmp.alloc(ar, scan_tmp_elems(N + 1), "scan scratch"));
        FEM_TRY(scan_exclusive_i64(cnt.ptr, m->rowptr.ptr, N, true, tmp.ptr, s));
        FEM_TRY(read_scalar(m->rowptr.ptr + N, &m->nnz, s));
        FEM_TRY(m->col.alloc(ar, m->nnz, "col"));
        FEM_TRY(launch_row_pattern(m->E, (int)npe, N, m->inc_ptr.ptr, m->inc_elem.ptr, cap, nullptr, m->rowptr.ptr,
                                   m->col.ptr, s, rows.ptr, rows.ptr ? S : 0));
        FEM_CUDA(cudaStreamSynchronize(s));  // the first-pass columns are freed on leaving
        DevBuf<unsigned long long> mx;
        FEM_TRY(mx.alloc(ar, 1, "max"));
        FEM_CUDA(cudaMemsetAsync(mx.ptr, 0, sizeof(unsigned long long), s));
        k_row_len_max<<<grid_for(N), TPB, 0, s>>>(m->rowptr.ptr, N, mx.ptr);
        FEM_LAUNCHED("k_row_len_max");
        unsigned long long ml = 0;
        FEM_TRY(read_scalar(mx.ptr, &ml, s));
        m->max_row_len = (int)ml;
        if (ml > 255) {
            set_error("a row of K has %llu lower entries; at most 255 are supported", ml);
            return FEM_ERR_UNSUPPORTED;
        }
    }

    return FEM_OK;
}

// Closure pairs of patches [p0, p1) from the node -> element incidence: for every
// owned node of the range and every element incident to it, the key
// ((patch - p0) << 32) | element.
__global__ void k_range_degree(const int32_t *own_row, const int64_t *inc_ptr, int64_t k0, int64_t nk, int64_t *deg) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nk; k += (int64_t)gridDim.x * blockDim.x) {
        const int32_t g = own_row[k0 + k];
        deg[k] = inc_ptr[g + 1] - inc_ptr[g];
    }
}

__global__ void k_range_pairs(const int32_t *own_row, const int32_t *node_patch, const int64_t *inc_ptr,
                              const int32_t *inc_elem, int64_t k0, int64_t nk, int64_t p0, const int64_t *off,
                              uint64_t *keys) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nk; k += (int64_t)gridDim.x * blockDim.x) {
        const int32_t g = own_row[k0 + k];
        const uint64_t pl = (uint64_t)(node_patch[g] - p0);
        int64_t o = off[k];
        for (int64_t t = inc_ptr[g]; t < inc_ptr[g + 1]; ++t, ++o) keys[o] = (pl << 32) | (uint64_t)(uint32_t)inc_elem[t];
    }
}

// Per-patch set building in shared memory: an open-addressing hash set of 32-bit
// keys (empty = all ones; linear probing, so an insert ends within `size` probes
// while the set holds fewer keys than slots) whose new members are appended to
// list[*count] in arrival order.  A set that fills its table sets *full (the
// key is then dropped, and the caller discards the set).
__device__ __forceinline__ void set_insert(uint32_t *table, int size, uint32_t key, uint32_t *list, int *count,
                                           int *full) {
    int h = (int)((key * 2654435761u) & (uint32_t)(size - 1));
    for (int probe = 0; probe < size; ++probe) {
        const uint32_t old = atomicCAS(&table[h], 0xffffffffu, key);
        if (old == 0xffffffffu) {
            list[atomicAdd(count, 1)] = key;
            return;
        }
        if (old == key) return;
        h = (h + 1) & (size - 1);
    }
    *full = 1;
}

// Largest table of the per-patch sets (slots of 4 bytes; a block holds the table
// and a list of as many slots).
static constexpr int SET_MAX_SLOTS = 16384;

// Closure elements of each patch (one block per patch), in the order the
// colouring sweeps them: the elements incident to the patch's owned nodes, made
// unique in a shared-memory hash set, then sorted by the smallest owned index
// among their nodes, ties by element id.  Written to tmp from the patch's
// candidate offset (cand_off: the incident slots of the earlier patches), with
// their number in cnt; k_patch_compact moves them into place.  A patch whose
// sort does not fit in the table's memory sets *overflow.
template <int NPE>
__global__ void __launch_bounds__(256) k_patch_celems(const int64_t *pn_ptr, int64_t np_, int64_t p0,
                                                      const int32_t *__restrict__ own_row,
                                                      const int64_t *__restrict__ inc_ptr,
                                                      const int32_t *__restrict__ inc_elem,
                                                      const int32_t *__restrict__ E, const int32_t *node_patch,
                                                      const int32_t *own_idx, const int64_t *cand_off, int hsize,
                                                      uint32_t *tmp, int64_t *cnt, int *overflow) {
    extern __shared__ __align__(16) unsigned char ce_smem[];
    uint32_t *table = reinterpret_cast<uint32_t *>(ce_smem);  // [hsize], then hsize / 2 sort keys
    uint64_t *skeys = reinterpret_cast<uint64_t *>(ce_smem);
    uint32_t *list = reinterpret_cast<uint32_t *>(ce_smem + (size_t)hsize * sizeof(uint32_t));  // [hsize]
    __shared__ int n_set, s_full;
    for (int64_t p = blockIdx.x; p < np_; p += gridDim.x) {
        for (int i = threadIdx.x; i < hsize; i += blockDim.x) table[i] = 0xffffffffu;
        if (threadIdx.x == 0) n_set = s_full = 0;
        __syncthreads();
        const int64_t k0 = pn_ptr[p], nown = pn_ptr[p + 1] - k0;
        for (int64_t k = threadIdx.x; k < nown; k += blockDim.x) {
            const int32_t g = own_row[k0 + k];
            for (int64_t t = inc_ptr[g]; t < inc_ptr[g + 1]; ++t)
                set_insert(table, hsize, (uint32_t)inc_elem[t], list, &n_set, &s_full);
        }
        __syncthreads();
        const int u = n_set, su = pow2_at_least(u);
        if (s_full || 2 * su > hsize) {  // a full table, or sort keys that would not fit in its memory
            if (threadIdx.x == 0) {
                *overflow = 1;
                cnt[p] = 0;
            }
            __syncthreads();
            continue;
        }
        const int32_t pg = (int32_t)(p0 + p);
        for (int j = threadIdx.x; j < su; j += blockDim.x) {
            uint64_t key = ~0ull;
            if (j < u) {
                const uint32_t e = list[j];
                int mo = 32767;
#pragma unroll
                for (int a = 0; a < NPE; ++a) {
                    const int32_t g = E[(int64_t)e * NPE + a];
                    if (node_patch[g] == pg) mo = min(mo, own_idx[g]);
                }
                key = ((uint64_t)mo << 32) | e;
            }
            skeys[j] = key;
        }
        __syncthreads();
        block_bitonic64(skeys, su);
        for (int r = threadIdx.x; r < u; r += blockDim.x) tmp[cand_off[p] + r] = (uint32_t)skeys[r];
        if (threadIdx.x == 0) cnt[p] = u;
        __syncthreads();
    }
}

// Closure nodes of each patch (one block per patch): the nodes of the patch's
// closure elements, made unique in a shared-memory hash set and sorted
// ascending, written to tmp from the patch's offset (npe slots per closure
// element) with their number in cnt.
template <int NPE>
__global__ void __launch_bounds__(256) k_patch_cnodes(const uint64_t *ckeys, const int64_t *pe_ptr, int64_t np_,
                                                      const int32_t *__restrict__ E, int hsize, uint32_t *tmp,
                                                      int64_t *cnt, int *overflow) {
    extern __shared__ __align__(16) unsigned char cn_smem[];
    uint32_t *table = reinterpret_cast<uint32_t *>(cn_smem);  // [hsize], then the sort keys
    uint32_t *list = reinterpret_cast<uint32_t *>(cn_smem + (size_t)hsize * sizeof(uint32_t));  // [hsize]
    __shared__ int n_set, s_full;
    for (int64_t p = blockIdx.x; p < np_; p += gridDim.x) {
        for (int i = threadIdx.x; i < hsize; i += blockDim.x) table[i] = 0xffffffffu;
        if (threadIdx.x == 0) n_set = s_full = 0;
        __syncthreads();
        const int64_t b = pe_ptr[p];
        const int n = (int)(pe_ptr[p + 1] - b) * NPE;
        for (int i = threadIdx.x; i < n; i += blockDim.x)
            set_insert(table, hsize, (uint32_t)E[(int64_t)(uint32_t)ckeys[b + i / NPE] * NPE + i % NPE], list, &n_set,
                       &s_full);
        __syncthreads();
        if (s_full) {
            if (threadIdx.x == 0) {
                *overflow = 1;
                cnt[p] = 0;
            }
            __syncthreads();
            continue;
        }
        const int u = n_set, su = pow2_at_least(u);
        for (int j = threadIdx.x; j < su; j += blockDim.x) table[j] = j < u ? list[j] : 0xffffffffu;
        __syncthreads();
        block_bitonic(table, su);
        for (int r = threadIdx.x; r < u; r += blockDim.x) tmp[b * NPE + r] = table[r];
        if (threadIdx.x == 0) cnt[p] = u;
        __syncthreads();
    }
}

// out[off[p] + r] = (p << 32) | tmp[from[p] * scale + r] for r < off[p + 1] - off[p].
__global__ void k_patch_compact(const uint32_t *tmp, const int64_t *from, int scale, const int64_t *off, int64_t np_,
                                uint64_t *out) {
    for (int64_t p = blockIdx.x; p < np_; p += gridDim.x) {
        const int64_t src = from[p] * scale, dst = off[p], n = off[p + 1] - dst;
        for (int64_t r = threadIdx.x; r < n; r += blockDim.x) out[dst + r] = ((uint64_t)p << 32) | tmp[src + r];
    }
}

// Candidate offset of each patch: off[p] = pre[pn[p] - k0].
__global__ void k_take_offsets(const int64_t *pre, const int64_t *pn, int64_t k0, int64_t np_, int64_t *off) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p <= np_; p += (int64_t)gridDim.x * blockDim.x)
        off[p] = pre[pn[p] - k0];
}

// Closure elements of each patch reordered by (colour, element id), one block per
// patch: out[i] = (patch << 40) | (colour << 32) | element, the layout of the
// global sort's keys.  Patches of at most SET_MAX_SLOTS / 2 elements.
__global__ void __launch_bounds__(512) k_patch_color_order(const uint64_t *ckeys, const uint8_t *color,
                                                           const int64_t *pe_ptr, int64_t np_, uint64_t *out) {
    extern __shared__ __align__(16) uint64_t co_keys[];
    for (int64_t p = blockIdx.x; p < np_; p += gridDim.x) {
        const int64_t b = pe_ptr[p];
        const int n = (int)(pe_ptr[p + 1] - b), sz = pow2_at_least(n);
        for (int i = threadIdx.x; i < sz; i += blockDim.x)
            co_keys[i] = i < n ? ((uint64_t)color[b + i] << 32) | (ckeys[b + i] & 0xffffffffull) : ~0ull;
        __syncthreads();
        block_bitonic64(co_keys, sz);
        for (int i = threadIdx.x; i < n; i += blockDim.x) out[b + i] = ((uint64_t)p << 40) | co_keys[i];
        __syncthreads();
    }
}

fem_status build_closure(fem_mesh m, int64_t p0, int64_t p1, Closure &cl, cudaStream_t s, bool with_pos) {
    Arena &ar = m->arena;
    Plan &P = m->plan;
    const int64_t npe = m->npe;
    const int64_t np_ = p1 - p0;
    cl.reset();
    cl.p0 = p0;
    cl.p1 = p1;
    std::vector<int64_t> h_pn(np_ + 1);
    FEM_CUDA(cudaMemcpyAsync(h_pn.data(), P.patch_node_ptr.ptr + p0, (np_ + 1) * sizeof(int64_t),
                             cudaMemcpyDeviceToHost, s));
    FEM_CUDA(cudaStreamSynchronize(s));
    const int64_t k0 = h_pn[0], nk = h_pn[np_] - h_pn[0];
    const int pbits = bits_for(np_);

    // ---- closure elements of each patch, in the colouring's sweep order: per
    // patch in shared memory, or (a patch too large for it) by global sorts
    DevBuf<uint64_t> ckeys;
    int64_t nce = 0;
    std::vector<int64_t> h_pe(np_ + 1, 0), h_pc(np_ + 1);
    bool swept = false;
    FEM_TRY(cl.patch_elem_ptr.alloc(ar, np_ + 1, "patch elem ptr"));
    {
        DevBuf<int64_t> deg, stmp, coff, cnt;
        DevBuf<int> ovf;
        FEM_TRY(deg.alloc(ar, nk + 1, "closure degrees"));
        k_range_degree<<<grid_for(nk), TPB, 0, s>>>(P.own_row.ptr, m->inc_ptr.ptr, k0, nk, deg.ptr);
        FEM_LAUNCHED("k_range_degree");
        FEM_TRY(stmp.alloc(ar, scan_tmp_elems(nk + 1), "scan scratch"));
        FEM_TRY(scan_exclusive_i64(deg.ptr, deg.ptr, nk, true, stmp.ptr, s));
        FEM_TRY(coff.alloc(ar, np_ + 1, "candidate offsets"));
        k_take_offsets<<<grid_for(np_ + 1), TPB, 0, s>>>(deg.ptr, P.patch_node_ptr.ptr + p0, k0, np_, coff.ptr);
        FEM_LAUNCHED("k_take_offsets");
        std::vector<int64_t> h_coff(np_ + 1);
        FEM_CUDA(cudaMemcpyAsync(h_coff.data(), coff.ptr, (np_ + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        FEM_CUDA(cudaStreamSynchronize(s));
        int64_t max_cand = 1;
        for (int64_t p = 0; p < np_; ++p) max_cand = std::max(max_cand, h_coff[p + 1] - h_coff[p]);
        const int hsize = pow2_at_least((int)std::min<int64_t>(max_cand, SET_MAX_SLOTS));
        DevBuf<uint32_t> ctmp;
        FEM_TRY(ctmp.alloc(ar, std::max<int64_t>(h_coff[np_], 1), "closure elements (unordered)"));
        FEM_TRY(cnt.alloc(ar, np_, "closure element counts"));
        FEM_TRY(ovf.alloc(ar, 1, "overflow flag"));
        FEM_CUDA(cudaMemsetAsync(ovf.ptr, 0, sizeof(int), s));
        const size_t smem = 2 * (size_t)hsize * sizeof(uint32_t);
        auto f = npe == 8 ? k_patch_celems<8> : k_patch_celems<4>;
        FEM_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int per_sm = 1;
        FEM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, 256, smem));
        const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(np_, (int64_t)num_sms() * std::max(per_sm, 1)));
        f<<<grid, 256, smem, s>>>(P.patch_node_ptr.ptr + p0, np_, p0, P.own_row.ptr, m->inc_ptr.ptr, m->inc_elem.ptr,
                                  m->E, P.node_patch.ptr, P.own_idx.ptr, coff.ptr, hsize, ctmp.ptr, cnt.ptr, ovf.ptr);
        FEM_LAUNCHED("k_patch_celems");
        int h_ovf = 0;
        std::vector<int64_t> h_cnt(np_);
        FEM_CUDA(cudaMemcpyAsync(h_cnt.data(), cnt.ptr, np_ * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        FEM_CUDA(cudaMemcpyAsync(&h_ovf, ovf.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
        FEM_CUDA(cudaStreamSynchronize(s));
        if (!h_ovf) {
            for (int64_t p = 0; p < np_; ++p) h_pe[p + 1] = h_pe[p] + h_cnt[p];
            nce = h_pe[np_];
            FEM_CUDA(cudaMemcpyAsync(cl.patch_elem_ptr.ptr, h_pe.data(), (np_ + 1) * sizeof(int64_t),
                                     cudaMemcpyHostToDevice, s));
            FEM_TRY(ckeys.alloc(ar, std::max<int64_t>(nce, 1), "closure keys (sweep order)"));
            const unsigned cg = (unsigned)std::max<int64_t>(1, std::min<int64_t>(np_, (int64_t)num_sms() * 8));
            k_patch_compact<<<cg, 256, 0, s>>>(ctmp.ptr, coff.ptr, 1, cl.patch_elem_ptr.ptr, np_, ckeys.ptr);
            FEM_LAUNCHED("k_patch_compact(elems)");
            FEM_CUDA(cudaStreamSynchronize(s));  // h_pe is read by the copy above; temporaries freed on return
            swept = true;
        }
    }
    if (!swept) {
        // unique (patch, element) pairs
        DevBuf<int64_t> deg, tmp;
        FEM_TRY(deg.alloc(ar, nk + 1, "closure degrees"));
        k_range_degree<<<grid_for(nk), TPB, 0, s>>>(P.own_row.ptr, m->inc_ptr.ptr, k0, nk, deg.ptr);
        FEM_LAUNCHED("k_range_degree");
        FEM_TRY(tmp.alloc(ar, scan_tmp_elems(nk + 1), "scan scratch"));
        FEM_TRY(scan_exclusive_i64(deg.ptr, deg.ptr, nk, true, tmp.ptr, s));
        int64_t npairs = 0;
        FEM_TRY(read_scalar(deg.ptr + nk, &npairs, s));
        DevBuf<uint64_t> pairs;
        FEM_TRY(pairs.alloc(ar, npairs, "closure pairs"));
        k_range_pairs<<<grid_for(nk), TPB, 0, s>>>(P.own_row.ptr, P.node_patch.ptr, m->inc_ptr.ptr, m->inc_elem.ptr,
                                                   k0, nk, p0, deg.ptr, pairs.ptr);
        FEM_LAUNCHED("k_range_pairs");
        deg.free();
        tmp.free();
        FEM_TRY(sort_unique(ar, pairs, npairs, 32 + pbits, ckeys, &nce, s));
        k_segment_ptr<<<grid_for(np_ + 1), TPB, 0, s>>>(ckeys.ptr, nce, 32, np_, cl.patch_elem_ptr.ptr);
        FEM_LAUNCHED("k_segment_ptr(elems)");
        FEM_CUDA(cudaMemcpyAsync(h_pe.data(), cl.patch_elem_ptr.ptr, (np_ + 1) * sizeof(int64_t),
                                 cudaMemcpyDeviceToHost, s));
        FEM_CUDA(cudaStreamSynchronize(s));
    }
    cl.total_celems = nce;
    for (int64_t p = 0; p < np_; ++p) cl.max_celems = std::max(cl.max_celems, h_pe[p + 1] - h_pe[p]);

    // ---- colouring of each closure (in sweep order), then order each closure by (colour, element)
    if (!swept) {
        DevBuf<uint64_t> skeys, salt, swk;
        DevBuf<uint32_t> sperm, spalt;
        DevBuf<int64_t> shist;
        FEM_TRY(skeys.alloc(ar, nce, "sweep keys"));
        FEM_TRY(sperm.alloc(ar, nce, "sweep order"));
        if (npe == 8)
            k_sweep_keys<8><<<grid_for(nce), TPB, 0, s>>>(ckeys.ptr, nce, m->E, P.node_patch.ptr, P.own_idx.ptr, p0,
                                                          skeys.ptr, sperm.ptr);
        else
            k_sweep_keys<4><<<grid_for(nce), TPB, 0, s>>>(ckeys.ptr, nce, m->E, P.node_patch.ptr, P.own_idx.ptr, p0,
                                                          skeys.ptr, sperm.ptr);
        FEM_LAUNCHED("k_sweep_keys");
        FEM_TRY(salt.alloc(ar, nce, "sort scratch"));
        FEM_TRY(spalt.alloc(ar, nce, "sort scratch"));
        FEM_TRY(shist.alloc(ar, radix_hist_elems(nce), "sort histogram"));
        FEM_TRY(radix_sort_u64(skeys.ptr, sperm.ptr, nce, 15 + pbits, salt.ptr, spalt.ptr, shist.ptr, s));
        FEM_TRY(swk.alloc(ar, nce, "closure keys (sweep order)"));
        k_gather_u64<<<grid_for(nce), TPB, 0, s>>>(ckeys.ptr, sperm.ptr, nce, swk.ptr);
        FEM_LAUNCHED("k_gather_u64");
        FEM_CUDA(cudaStreamSynchronize(s));
        std::swap(ckeys.ptr, swk.ptr);
        std::swap(ckeys.n, swk.n);
        std::swap(ckeys.arena, swk.arena);
    }
    {
        DevBuf<uint8_t> color;
        DevBuf<int> mxc;
        FEM_TRY(color.alloc(ar, nce, "colours"));
        FEM_TRY(mxc.alloc(ar, 1, "max colour"));
        FEM_CUDA(cudaMemsetAsync(mxc.ptr, 0, sizeof(int), s));
        const size_t smem = (size_t)COLOR_WORDS * P.max_own * sizeof(unsigned long long) +
                            (size_t)COLOR_CHUNK * npe * sizeof(int16_t);
        // four warps per patch: they stage the element table (the greedy pass itself
        // is one thread's dependent chain of shared-memory updates, so the SM is kept
        // busy by many patches at once; small chunks of the table keep each block's
        // shared memory small)
        const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(np_, (int64_t)num_sms() * 16));
        if (npe == 8) {
            FEM_CUDA(cudaFuncSetAttribute(k_color<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            k_color<8><<<grid, 128, smem, s>>>(ckeys.ptr, cl.patch_elem_ptr.ptr, P.patch_node_ptr.ptr + p0, m->E,
                                               P.node_patch.ptr, P.own_idx.ptr, np_, p0, color.ptr, mxc.ptr);
        } else {
            FEM_CUDA(cudaFuncSetAttribute(k_color<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            k_color<4><<<grid, 128, smem, s>>>(ckeys.ptr, cl.patch_elem_ptr.ptr, P.patch_node_ptr.ptr + p0, m->E,
                                               P.node_patch.ptr, P.own_idx.ptr, np_, p0, color.ptr, mxc.ptr);
        }
        FEM_LAUNCHED("k_color");
        int h_mxc = 0;
        FEM_TRY(read_scalar(mxc.ptr, &h_mxc, s));
        if (h_mxc >= 255) {
            set_error("the closure colouring needs more than 255 colours (more than 255 elements share a node)");
            return FEM_ERR_UNSUPPORTED;
        }
        cl.n_colors = h_mxc + 1;
        DevBuf<uint64_t> ck2, alt;
        DevBuf<int64_t> hist;
        FEM_TRY(ck2.alloc(ar, std::max<int64_t>(nce, 1), "closure keys"));
        if (cl.max_celems <= SET_MAX_SLOTS / 2) {
            // per patch in shared memory
            const size_t csm = (size_t)pow2_at_least((int)std::max<int64_t>(cl.max_celems, 1)) * sizeof(uint64_t);
            FEM_CUDA(cudaFuncSetAttribute(k_patch_color_order, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)csm));
            const unsigned cgrid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(np_, (int64_t)num_sms() * 2));
            k_patch_color_order<<<cgrid, 512, csm, s>>>(ckeys.ptr, color.ptr, cl.patch_elem_ptr.ptr, np_, ck2.ptr);
            FEM_LAUNCHED("k_patch_color_order");
            FEM_CUDA(cudaStreamSynchronize(s));
            color.free();
            ckeys.free();
        } else {
            k_color_keys<<<grid_for(nce), TPB, 0, s>>>(ckeys.ptr, color.ptr, nce, ck2.ptr);
            FEM_LAUNCHED("k_color_keys");
            FEM_CUDA(cudaStreamSynchronize(s));
            color.free();
            ckeys.free();
            FEM_TRY(alt.alloc(ar, nce, "sort scratch"));
            FEM_TRY(hist.alloc(ar, radix_hist_elems(nce), "sort histogram"));
            FEM_TRY(radix_sort_u64(ck2.ptr, nullptr, nce, 40 + pbits, alt.ptr, nullptr, hist.ptr, s));
            FEM_CUDA(cudaStreamSynchronize(s));
        }
        std::swap(ckeys.ptr, ck2.ptr);
        std::swap(ckeys.n, ck2.n);
        std::swap(ckeys.arena, ck2.arena);
    }

    // ---- closure nodes of each patch
    DevBuf<uint64_t> cnkeys;
    int64_t ncn = 0;
    bool cn_done = false;
    {
        // per patch in shared memory; a patch whose set outgrows its table takes
        // the global sort instead
        const int hsize = pow2_at_least((int)std::min<int64_t>(std::max<int64_t>(cl.max_celems * npe, 1), 8192));
        DevBuf<uint32_t> ntmp;
        DevBuf<int64_t> cnt, pc;
        DevBuf<int> ovf;
        FEM_TRY(ntmp.alloc(ar, std::max<int64_t>(nce * npe, 1), "closure nodes (per patch)"));
        FEM_TRY(cnt.alloc(ar, np_, "closure node counts"));
        FEM_TRY(ovf.alloc(ar, 1, "overflow flag"));
        FEM_CUDA(cudaMemsetAsync(ovf.ptr, 0, sizeof(int), s));
        const size_t smem = 2 * (size_t)hsize * sizeof(uint32_t);
        auto f = npe == 8 ? k_patch_cnodes<8> : k_patch_cnodes<4>;
        FEM_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int per_sm = 1;
        FEM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, 256, smem));
        const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(np_, (int64_t)num_sms() * std::max(per_sm, 1)));
        f<<<grid, 256, smem, s>>>(ckeys.ptr, cl.patch_elem_ptr.ptr, np_, m->E, hsize, ntmp.ptr, cnt.ptr, ovf.ptr);
        FEM_LAUNCHED("k_patch_cnodes");
        int h_ovf = 0;
        std::vector<int64_t> h_cnt(np_), h_off(np_ + 1, 0);
        FEM_CUDA(cudaMemcpyAsync(h_cnt.data(), cnt.ptr, np_ * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        FEM_CUDA(cudaMemcpyAsync(&h_ovf, ovf.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
        FEM_CUDA(cudaStreamSynchronize(s));
        if (!h_ovf) {
            for (int64_t p = 0; p < np_; ++p) h_off[p + 1] = h_off[p] + h_cnt[p];
            ncn = h_off[np_];
            FEM_TRY(pc.alloc(ar, np_ + 1, "closure node offsets"));
            FEM_CUDA(cudaMemcpyAsync(pc.ptr, h_off.data(), (np_ + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
            FEM_TRY(cnkeys.alloc(ar, std::max<int64_t>(ncn, 1), "closure nodes"));
            const unsigned cg = (unsigned)std::max<int64_t>(1, std::min<int64_t>(np_, (int64_t)num_sms() * 8));
            k_patch_compact<<<cg, 256, 0, s>>>(ntmp.ptr, cl.patch_elem_ptr.ptr, (int)npe, pc.ptr, np_, cnkeys.ptr);
            FEM_LAUNCHED("k_patch_compact(nodes)");
            FEM_CUDA(cudaStreamSynchronize(s));  // h_off is read by the copy above; temporaries freed on return
            cn_done = true;
        }
    }
    if (!cn_done) {
        DevBuf<uint64_t> pairs;
        FEM_TRY(pairs.alloc(ar, nce * npe, "closure node pairs"));
        k_cnode_pairs<<<grid_for(nce * npe), TPB, 0, s>>>(ckeys.ptr, nce, (int)npe, m->E, pairs.ptr);
        FEM_LAUNCHED("k_cnode_pairs");
        FEM_TRY(sort_unique(ar, pairs, nce * npe, 32 + pbits, cnkeys, &ncn, s));
    }
    cl.total_cnodes = ncn;
    FEM_TRY(cl.patch_cnode_ptr.alloc(ar, np_ + 1, "patch cnode ptr"));
    k_segment_ptr<<<grid_for(np_ + 1), TPB, 0, s>>>(cnkeys.ptr, ncn, 32, np_, cl.patch_cnode_ptr.ptr);
    FEM_LAUNCHED("k_segment_ptr(cnodes)");
    FEM_TRY(cl.cnode_gid.alloc(ar, ncn, "cnode gid"));
    FEM_TRY(cl.cnode_own.alloc(ar, ncn, "cnode own"));
    k_cnode_own<<<grid_for(ncn), TPB, 0, s>>>(cnkeys.ptr, ncn, p0, P.node_patch.ptr, P.own_idx.ptr, cl.cnode_gid.ptr,
                                              cl.cnode_own.ptr);
    FEM_LAUNCHED("k_cnode_own");

    // ---- per closure element data
    FEM_TRY(cl.celem_id.alloc(ar, nce, "celem id"));
    FEM_TRY(cl.celem_color.alloc(ar, nce, "celem colour"));
    FEM_TRY(cl.celem_lnode.alloc(ar, nce * npe, "celem local nodes"));
    if (with_pos) FEM_TRY(cl.celem_pos.alloc(ar, nce * P.pos_stride, "celem positions"));
    FEM_TRY(cl.celem_aidx.alloc(ar, nce * (m->np / 2), "celem accumulator targets"));
    const OwnTables ot{P.node_patch.ptr,     P.own_idx.ptr, P.own_acc.ptr,          P.patch_node_ptr.ptr,
                       P.own_hv.ptr,         cl.patch_elem_ptr.ptr, p0, (int32_t)P.max_acc};
    uint16_t *aidx16 = reinterpret_cast<uint16_t *>(cl.celem_aidx.ptr);
    FEM_CUDA(cudaMemcpyAsync(h_pc.data(), cl.patch_cnode_ptr.ptr, (np_ + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    FEM_CUDA(cudaStreamSynchronize(s));
    for (int64_t p = 0; p < np_; ++p) cl.max_cnodes = std::max(cl.max_cnodes, h_pc[p + 1] - h_pc[p]);
    if (cl.max_cnodes > 32768) {
        set_error("a patch touches %lld nodes; at most 32768 are supported", (long long)cl.max_cnodes);
        return FEM_ERR_UNSUPPORTED;
    }
    {
        const size_t smem = (size_t)std::max<int64_t>(cl.max_cnodes, 1) * sizeof(int32_t);
        const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(np_, (int64_t)num_sms() * 8));
        if (npe == 8) {
            FEM_CUDA(cudaFuncSetAttribute(k_celem_fill<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            k_celem_fill<8><<<grid, TPB, smem, s>>>(ckeys.ptr, np_, m->E, cnkeys.ptr, cl.patch_cnode_ptr.ptr,
                                                    m->rowptr.ptr, m->col.ptr, P.pos_stride, ot, cl.celem_id.ptr,
                                                    cl.celem_color.ptr, cl.celem_lnode.ptr,
                                                    with_pos ? cl.celem_pos.ptr : nullptr, aidx16);
        } else {
            FEM_CUDA(cudaFuncSetAttribute(k_celem_fill<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            k_celem_fill<4><<<grid, TPB, smem, s>>>(ckeys.ptr, np_, m->E, cnkeys.ptr, cl.patch_cnode_ptr.ptr,
                                                    m->rowptr.ptr, m->col.ptr, P.pos_stride, ot, cl.celem_id.ptr,
                                                    cl.celem_color.ptr, cl.celem_lnode.ptr,
                                                    with_pos ? cl.celem_pos.ptr : nullptr, aidx16);
        }
        FEM_LAUNCHED("k_celem_fill");
    }
    return FEM_OK;
}

// The closures carry the in-row positions from now on (the backward pass reads
// them; forward builds do not, so a mesh that only builds K does not hold them).
// Closures built per patch group get them when they are built; the cached full
// closure gets them here.  If the budget cannot hold them beside the cached
// closures, the plan is built again (in patch groups if need be).
fem_status ensure_positions(fem_mesh m, cudaStream_t s) {
    if (m->want_pos) return FEM_OK;
    m->want_pos = true;
    if (!m->plan_built || m->plan.chunked) return FEM_OK;  // group closures: built, or copied, with them
    Plan &P = m->plan;
    Closure &cl = P.full;
    const int64_t nce = cl.total_celems;
    fem_status st = cl.celem_pos.alloc(m->arena, (size_t)nce * P.pos_stride, "celem positions");
    if (st == FEM_ERR_BUDGET) {
        cudaGetLastError();
        cl.celem_pos.free();
        batch_forget(m);
        m->plan_built = false;
        ArenaKeep keep(m->arena);
        FEM_TRY(build_plan(m, s));
        m->plan_built = true;
        return FEM_OK;
    }
    FEM_TRY(st);
    if (nce > 0) {
        const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(cdiv(nce, TPB), (int64_t)num_sms() * 8));
        if (m->npe == 8)
            k_celem_pos<8><<<grid, TPB, 0, s>>>(cl.celem_id.ptr, nce, m->E, m->rowptr.ptr, m->col.ptr, P.pos_stride,
                                                cl.celem_pos.ptr);
        else
            k_celem_pos<4><<<grid, TPB, 0, s>>>(cl.celem_id.ptr, nce, m->E, m->rowptr.ptr, m->col.ptr, P.pos_stride,
                                                cl.celem_pos.ptr);
        FEM_LAUNCHED("k_celem_pos");
    }
    return FEM_OK;
}

// Patch groups under the memory budget (Eq. 10: the work is split into
// GPU_g = ceil(required / available) groups run one after the other).  A group
// of G patches is tried, halved while its closure does not fit, and every group
// is built once here to record the sizes the kernels' shared memory needs (and,
// with fem_options.group_cache, the host copies the numeric calls run from;
// groups.cu).
static fem_status plan_groups(fem_mesh m, cudaStream_t s) {
    Plan &P = m->plan;
    int64_t G = std::max<int64_t>(1, P.n_patches / 2);
    for (;;) {
        Closure cl;
        // (with the host copies, the groups are recorded with their in-row positions)
        fem_status st = build_closure(m, 0, std::min(G, P.n_patches), cl, s, m->want_pos || m->opt.group_cache);
        if (st == FEM_OK) break;
        cl.reset();
        cudaGetLastError();
        if (st != FEM_ERR_BUDGET) return st;
        if (G == 1) {
            set_error("the memory budget cannot hold the closure of one patch; raise it or lower patch_entries");
            return FEM_ERR_BUDGET;
        }
        G = std::max<int64_t>(1, G / 2);
    }
    m->group_patches = G;
    P.total_cnodes = P.total_celems = P.max_cnodes = P.max_celems = 0;
    P.n_colors = 0;
    return for_each_group(m, s, [&](const Closure &cl) {
        P.total_cnodes += cl.total_cnodes;
        P.total_celems += cl.total_celems;
        P.max_cnodes = std::max(P.max_cnodes, cl.max_cnodes);
        P.max_celems = std::max(P.max_celems, cl.max_celems);
        P.n_colors = std::max(P.n_colors, cl.n_colors);
        return FEM_OK;
    });
}

// Global part of the plan (patches of consecutive nodes in locality order, the
// owned-row tables), then the closures of all patches at once if the memory
// budget holds them, else closures are built per patch group by each numeric call.
static fem_status build_plan_cap(fem_mesh m, cudaStream_t s, int64_t cap_in) {
    Arena &ar = m->arena;
    const int64_t N = m->n_nodes;
    Plan &P = m->plan;
    batch_forget(m);  // cached batched launches were sized for the old plan
    P.reset();
    drop_group_cache(m);
    // the elasticity operator holds a 3x3 block per node pair: fewer pairs fit
    const bool elastic = m->opt.operator_kind == 2;
    // (defaults measured on the 1M-brick and 3.07M-tet workloads)
    int64_t cap_entries = cap_in > 0 ? cap_in
                                     : m->opt.patch_entries > 0 ? m->opt.patch_entries
                                                                : (elastic ? (m->npe == 8 ? 4096 : 1536) : 8192);
    if (cap_entries < 2 * (int64_t)m->max_row_len) cap_entries = 2 * (int64_t)m->max_row_len;
    P.cap_entries = cap_entries;
    int64_t cap_eff = cap_entries - m->max_row_len;
    // Row ranges of the host pipeline (fixed with the node order, which runs
    // range by range): their CSR starts.
    const int nc = (!elastic && m->nnz > 0 && m->chunk_rows.size() > 2) ? (int)m->chunk_rows.size() - 1 : 1;
    std::vector<int64_t> c_row(nc + 1), c_val(nc + 1);
    c_row[0] = 0, c_row[nc] = N, c_val[0] = 0, c_val[nc] = m->nnz;
    if (nc > 1) {
        c_row = m->chunk_rows;
        DevBuf<int64_t> rv;
        FEM_TRY(rv.alloc(ar, 2 * (nc + 1), "row ranges"));
        FEM_CUDA(cudaMemcpyAsync(rv.ptr, c_row.data(), (nc + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
        k_range_vals<<<1, 256, 0, s>>>(m->rowptr.ptr, rv.ptr, nc, rv.ptr + nc + 1);
        FEM_LAUNCHED("k_range_vals");
        FEM_CUDA(cudaMemcpyAsync(c_val.data(), rv.ptr + nc + 1, (nc + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        FEM_CUDA(cudaStreamSynchronize(s));
    }
    DevBuf<int64_t> pre;
    {
        DevBuf<int64_t> len, tmp;
        FEM_TRY(len.alloc(ar, N + 1, "row lengths"));
        FEM_TRY(pre.alloc(ar, N + 1, "row length prefix"));
        k_len_in_order<<<grid_for(N), TPB, 0, s>>>(m->order.ptr, m->rowptr.ptr, N, len.ptr);
        FEM_LAUNCHED("k_len_in_order");
        FEM_TRY(tmp.alloc(ar, scan_tmp_elems(N + 1), "scan scratch"));
        FEM_TRY(scan_exclusive_i64(len.ptr, pre.ptr, N, true, tmp.ptr, s));
        FEM_CUDA(cudaStreamSynchronize(s));
    }
    // Whole waves: a range's patch count is rounded up to a multiple of the
    // resident blocks of the patch kernel (smaller patches, same cap), so that no
    // block slot idles in the last wave while others run a patch more.  Below
    // half a wave the range keeps its patches.
    int64_t wave = 0;
    if (m->nnz > 0) {
        int threads = m->opt.block_threads > 0 ? m->opt.block_threads : 256;
        threads = std::min((threads + 31) / 32 * 32, patch_max_threads(m->npe));
        int per_sm = 0;
        if (elastic) {
            // resident blocks as registers and (about) the accumulators allow
            threads = elastic_threads(m->npe, m->opt.block_threads);
            per_sm = elastic_blocks_per_sm(m->npe, threads);
            const int64_t smem = 36 * (cap_entries + 32) + 16384;
            per_sm = (int)std::max<int64_t>(1, std::min<int64_t>(per_sm, (228 * 1024) / (smem + 1024)));
        } else {
            per_sm = patch_blocks_per_sm(m->npe, threads);
        }
        wave = (int64_t)num_sms() * per_sm;
    }
    std::vector<int64_t> c_patch(nc + 1, 0), c_cap(nc, cap_eff);
    for (int k = 0; k < nc; ++k) {
        const int64_t e = c_val[k + 1] - c_val[k];
        int64_t cap = cap_eff;
        const int64_t n0 = cdiv(e, cap);
        if (e > 0 && n0 * 2 > wave) cap = std::max<int64_t>(1, cdiv(e, cdiv(n0, wave) * wave));
        c_cap[k] = cap;
        c_patch[k + 1] = c_patch[k] + (e > 0 ? cdiv(e, cap) : 0);
    }
    if (c_patch[nc] == 0) c_patch[nc] = 1;  // no entries: one empty patch
    P.n_patches = c_patch[nc];
    P.n_nodes = m->n_nodes;
    P.n_elems = m->n_elems;
    P.nnz = m->nnz;
    const int64_t npatch = P.n_patches;
    if (npatch >= (1ll << 23)) {
        set_error("too many patches (%lld)", (long long)npatch);
        return FEM_ERR_UNSUPPORTED;
    }
    P.chunk_row = c_row;
    P.chunk_val = c_val;
    P.chunk_patch = c_patch;
    for (int k = 0; k < nc; ++k) P.max_chunk_vals = std::max(P.max_chunk_vals, c_val[k + 1] - c_val[k]);
    P.pos_stride = (int)((m->np + 3) / 4 * 4);
    FEM_TRY(P.patch_node_ptr.alloc(ar, npatch + 1, "patch node ptr"));
    {
        DevBuf<int64_t> tab;
        FEM_TRY(tab.alloc(ar, 3 * (size_t)nc + 2, "range table"));
        FEM_CUDA(cudaMemcpyAsync(tab.ptr, c_row.data(), (nc + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
        FEM_CUDA(cudaMemcpyAsync(tab.ptr + nc + 1, c_patch.data(), (nc + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
        FEM_CUDA(cudaMemcpyAsync(tab.ptr + 2 * nc + 2, c_cap.data(), nc * sizeof(int64_t), cudaMemcpyHostToDevice, s));
        k_patch_bounds<<<grid_for(npatch + 1), TPB, 0, s>>>(pre.ptr, tab.ptr, tab.ptr + nc + 1, tab.ptr + 2 * nc + 2,
                                                            nc, npatch, P.patch_node_ptr.ptr);
        FEM_LAUNCHED("k_patch_bounds");
        FEM_CUDA(cudaStreamSynchronize(s));  // the table is freed on leaving
    }
    FEM_TRY(P.node_patch.alloc(ar, N, "node patch"));
    FEM_TRY(P.own_idx.alloc(ar, N, "own index"));
    FEM_TRY(P.own_row.alloc(ar, N, "own row"));
    FEM_TRY(P.own_rowptr.alloc(ar, N, "own rowptr"));
    FEM_TRY(P.own_acc.alloc(ar, N, "own acc"));
    FEM_TRY(P.own_hv.alloc(ar, N, "own hv"));
    FEM_TRY(P.patch_acc.alloc(ar, npatch, "patch acc"));
    // FP64-accurate diagonals of high-valence rows: scalar operators only
    const int hv_thr = elastic ? INT32_MAX : m->opt.valence_threshold;
    P.any_hv = m->max_deg > hv_thr;
    k_patch_nodes<<<grid_for(N), TPB, 0, s>>>(m->order.ptr, pre.ptr, P.patch_node_ptr.ptr, N, npatch,
                                              m->rowptr.ptr, m->inc_ptr.ptr, hv_thr, P.node_patch.ptr, P.own_idx.ptr,
                                              P.own_row.ptr, P.own_rowptr.ptr, P.own_acc.ptr, P.own_hv.ptr);
    FEM_LAUNCHED("k_patch_nodes");
    k_patch_acc<<<grid_for(npatch), TPB, 0, s>>>(pre.ptr, P.patch_node_ptr.ptr, npatch, P.patch_acc.ptr);
    FEM_LAUNCHED("k_patch_acc");
    std::vector<int64_t> h_pn(npatch + 1);
    std::vector<int32_t> h_acc(npatch);
    FEM_CUDA(cudaMemcpyAsync(h_pn.data(), P.patch_node_ptr.ptr, (npatch + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    FEM_CUDA(cudaMemcpyAsync(h_acc.data(), P.patch_acc.ptr, npatch * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    FEM_CUDA(cudaStreamSynchronize(s));
    pre.free();
    for (int64_t p = 0; p < npatch; ++p) {
        P.max_own = std::max(P.max_own, h_pn[p + 1] - h_pn[p]);
        P.max_acc = std::max(P.max_acc, (int64_t)h_acc[p]);
    }
    if (P.max_own > 32767 || P.max_acc > 32767 - 32) {
        set_error("a patch owns %lld rows and %lld entries; at most 32767 and 32735 are supported",
                  (long long)P.max_own, (long long)P.max_acc);
        return FEM_ERR_UNSUPPORTED;
    }

    // closures of all patches, unless the budget refuses them
    fem_status st = build_closure(m, 0, npatch, P.full, s, m->want_pos);
    if (st == FEM_ERR_BUDGET) {
        P.full.reset();
        cudaGetLastError();
        P.chunked = true;
        return plan_groups(m, s);
    }
    FEM_TRY(st);
    P.total_cnodes = P.full.total_cnodes;
    P.total_celems = P.full.total_celems;
    P.max_cnodes = P.full.max_cnodes;
    P.max_celems = P.full.max_celems;
    P.n_colors = P.full.n_colors;
    m->n_groups = 1;
    return FEM_OK;
}

// The plan, with its patches halved until the largest closure fits the fused
// scalar kernel's shared memory (mixed precision, FP64 coordinates: its largest
// layout).  Closures that outgrow it come from patches whose owned nodes are
// scattered, e.g. row ranges of the host pipeline cut from a numbering without
// locality; the elasticity operator accumulates large patches in row windows.
fem_status build_plan(fem_mesh m, cudaStream_t s) {
    int dev = 0, limit = 0;
    FEM_CUDA(cudaGetDevice(&dev));
    FEM_CUDA(cudaDeviceGetAttribute(&limit, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    int64_t cap = 0;
    for (;;) {
        FEM_TRY(build_plan_cap(m, s, cap));
        if (m->opt.operator_kind == 2) return FEM_OK;
        PlanMax pm;
        pm.add(m->plan);
        const size_t need = patch_smem_layout(pm, true, true, sizeof(double), sizeof(double)).total + 1024;
        const int64_t half = m->plan.cap_entries / 2;
        if (need <= (size_t)limit || half < 2 * (int64_t)m->max_row_len) return FEM_OK;
        cap = half;
    }
}


}  // namespace fem

// ------------------------------------------------ pattern over caller scratch
// The steps of the row-wise pattern above, run over scratch memory the caller
// provides (used by the allocation-free entry point; the mesh-handle path
// allocates its own).  Scratch layout and sizes: see noalloc.cu.
namespace fem {

fem_status pattern_steps_validate(const int32_t *E, int64_t nel, int npe, int64_t N, unsigned long long *flags,
                                  cudaStream_t s) {
    FEM_CUDA(cudaMemsetAsync(flags, 0xff, 2 * sizeof(unsigned long long), s));
    k_validate<<<grid_for(nel), TPB, 0, s>>>(E, nel, npe, N, flags, flags + 1);
    FEM_LAUNCHED("k_validate");
    return FEM_OK;
}

fem_status pattern_steps_incidence(const int32_t *E, int64_t nel, int npe, int64_t N, int64_t *deg, int64_t *inc_ptr,
                                   unsigned int *cursor, int32_t *inc_elem, int64_t *scan_tmp,
                                   unsigned long long *mx, cudaStream_t s) {
    const int64_t n_ent = nel * npe;
    FEM_CUDA(cudaMemsetAsync(deg, 0, (N + 1) * sizeof(int64_t), s));
    FEM_CUDA(cudaMemsetAsync(cursor, 0, N * sizeof(unsigned int), s));
    FEM_CUDA(cudaMemsetAsync(mx, 0, sizeof(unsigned long long), s));
    k_degree<<<grid_for(n_ent), TPB, 0, s>>>(E, n_ent, reinterpret_cast<unsigned long long *>(deg));
    FEM_LAUNCHED("k_degree");
    FEM_TRY(scan_exclusive_i64(deg, inc_ptr, N, true, scan_tmp, s));
    k_inc_fill<<<grid_for(n_ent), TPB, 0, s>>>(E, n_ent, npe, inc_ptr, cursor, inc_elem);
    FEM_LAUNCHED("k_inc_fill");
    k_inc_sort<<<grid_for(N), TPB, 0, s>>>(inc_ptr, inc_elem, N);
    FEM_LAUNCHED("k_inc_sort");
    k_max_deg<<<grid_for(N), TPB, 0, s>>>(inc_ptr, N, mx);
    FEM_LAUNCHED("k_max_deg");
    return FEM_OK;
}

fem_status pattern_steps_rows(const int32_t *E, int npe, int64_t N, const int64_t *inc_ptr, const int32_t *inc_elem,
                              int cap, int64_t *cnt, const int64_t *rowptr, int32_t *col, cudaStream_t s) {
    return launch_row_pattern(E, npe, N, inc_ptr, inc_elem, cap, cnt, rowptr, col, s);
}

}  // namespace fem
