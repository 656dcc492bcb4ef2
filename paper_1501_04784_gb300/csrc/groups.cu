// groups.cu -- plans built per patch group under the memory budget (Eq. 10):
// the numeric calls run the groups one after the other, each group's closure
// either built for the call (closure_range) or copied back from its page-locked
// host copy (fem_options.group_cache) into one of two reusable device slots,
// the next group's copy overlapping the current group's run.
//
// A host copy holds a closure's element ids, colours, closure-local node indices,
// in-row positions and closure nodes; the accumulator targets (twice the bytes
// of the positions) are derived from the positions on the device after the copy
// (k_expand_targets), exactly as the closure fill derives them.
#include <algorithm>
#include <functional>
#include <vector>

#include "mesh.cuh"
#include "numeric.cuh"

namespace fem {

// Accumulator targets of a closure's packed pairs from its in-row positions: the
// targets k_celem_fill writes (see PlanView::celem_aidx).  One block per patch of
// the closure.  The pair's row is its node with the larger global id, i.e. the
// larger closure-local index (closure nodes ascend with the id); an owned row's
// entry is its offset in the patch's accumulators plus the position; a pair whose
// row the patch does not own goes to the scratch slot of the lane that will hold
// the element; an FP64-accurate diagonal is AIDX_HV | owned-row index.
template <int NPE>
__global__ void __launch_bounds__(256) k_expand_targets(int64_t np_, const int64_t *__restrict__ pe_ptr,
                                                        const int64_t *__restrict__ pc_ptr,
                                                        const uint16_t *__restrict__ lnode,
                                                        const uint8_t *__restrict__ pos, int pos_stride,
                                                        const int32_t *__restrict__ cnode_own,
                                                        const int64_t *__restrict__ patch_node_ptr,
                                                        const int32_t *__restrict__ own_acc,
                                                        const uint8_t *__restrict__ own_hv, int trash,
                                                        int64_t nce, uint32_t *__restrict__ aidx) {
    constexpr int NP = NPE * (NPE + 1) / 2;
    for (int64_t pb = blockIdx.x; pb < np_; pb += gridDim.x) {
        const int64_t e0 = pe_ptr[pb], e1 = pe_ptr[pb + 1], cb = pc_ptr[pb];
        const int64_t nb = patch_node_ptr[pb];
        for (int64_t i = e0 + threadIdx.x; i < e1; i += blockDim.x) {
            int ln[NPE], own[NPE], base[NPE];
            bool hv[NPE];
#pragma unroll
            for (int a = 0; a < NPE; ++a) {
                ln[a] = lnode[i * NPE + a];
                own[a] = cnode_own[cb + ln[a]];
                base[a] = own[a] >= 0 ? own_acc[nb + own[a]] : 0;
                hv[a] = own[a] >= 0 && own_hv[nb + own[a]] != 0;
            }
            const uint8_t *pp = pos + i * pos_stride;
            const uint32_t scratch = (uint32_t)(trash + ((i - e0) & 31));
            uint32_t lo = 0;
            int q = 0;
#pragma unroll
            for (int a = 0; a < NPE; ++a)
#pragma unroll
                for (int b = 0; b <= a; ++b, ++q) {
                    const int r = ln[a] > ln[b] ? a : b;
                    uint32_t t = scratch;
                    if (own[r] >= 0) {
                        if (a == b && hv[a]) t = AIDX_HV | (uint32_t)own[a];
                        else t = (uint32_t)(base[r] + pp[q]);
                    }
                    if (q & 1) aidx[(int64_t)(q >> 1) * nce + i] = lo | ((t & 0xffffu) << 16);
                    else lo = t & 0xffffu;
                }
            static_assert(NP % 2 == 0, "targets pair up into words");
        }
    }
}

// The targets of a closure whose positions (and everything else) are in place.
static fem_status expand_targets(fem_mesh m, const Closure &cl, uint32_t *aidx, cudaStream_t s) {
    const Plan &P = m->plan;
    const int64_t np_ = cl.p1 - cl.p0;
    if (np_ <= 0 || cl.total_celems == 0) return FEM_OK;
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(np_, (int64_t)num_sms() * 8));
#define FEM_EXPAND(NPE)                                                                                            \
    k_expand_targets<NPE><<<grid, 256, 0, s>>>(np_, cl.patch_elem_ptr.ptr, cl.patch_cnode_ptr.ptr,                \
                                               cl.celem_lnode.ptr, cl.celem_pos.ptr, P.pos_stride, cl.cnode_own.ptr, \
                                               P.patch_node_ptr.ptr + cl.p0, P.own_acc.ptr, P.own_hv.ptr,          \
                                               (int)P.max_acc, cl.total_celems, aidx)
    if (m->npe == 8) FEM_EXPAND(8);
    else FEM_EXPAND(4);
#undef FEM_EXPAND
    FEM_LAUNCHED("k_expand_targets");
    return FEM_OK;
}

// A page-locked host copy of a built closure (which carries its positions).
// Returns false (and leaves `h` empty) if the host memory cannot be had.
static bool closure_to_host(const Closure &cl, HostClosure &h, cudaStream_t s) {
    const int64_t np_ = cl.p1 - cl.p0;
    h.p0 = cl.p0, h.p1 = cl.p1, h.total_cnodes = cl.total_cnodes, h.total_celems = cl.total_celems;
    h.max_cnodes = cl.max_cnodes, h.max_celems = cl.max_celems, h.n_colors = cl.n_colors;
    h.n_pep = h.n_pcp = (size_t)np_ + 1;
    h.n_gid = h.n_own = (size_t)cl.total_cnodes;
    h.n_id = h.n_col = (size_t)cl.total_celems;
    h.n_pos = cl.celem_pos.n;
    h.n_ln = cl.celem_lnode.n;
    h.n_aidx = cl.celem_aidx.n;  // derived on the device, not copied
    if (!cl.celem_pos.ptr) return false;
    size_t o = 0;
    auto take = [&](size_t &off, size_t bytes) { off = o; o += (bytes + 255) & ~(size_t)255; };
    take(h.o_pep, h.n_pep * 8);
    take(h.o_pcp, h.n_pcp * 8);
    take(h.o_gid, h.n_gid * 4);
    take(h.o_own, h.n_own * 4);
    take(h.o_id, h.n_id * 4);
    take(h.o_col, h.n_col);
    take(h.o_pos, h.n_pos);
    take(h.o_ln, h.n_ln * 2);
    void *p = nullptr;
    if (cudaHostAlloc(&p, o, cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    h.host = static_cast<unsigned char *>(p);
    h.bytes = o;
    auto down = [&](size_t off, const void *src, size_t bytes) {
        return bytes == 0 || cudaMemcpyAsync(h.host + off, src, bytes, cudaMemcpyDeviceToHost, s) == cudaSuccess;
    };
    bool ok = down(h.o_pep, cl.patch_elem_ptr.ptr, h.n_pep * 8) && down(h.o_pcp, cl.patch_cnode_ptr.ptr, h.n_pcp * 8) &&
              down(h.o_gid, cl.cnode_gid.ptr, h.n_gid * 4) && down(h.o_own, cl.cnode_own.ptr, h.n_own * 4) &&
              down(h.o_id, cl.celem_id.ptr, h.n_id * 4) && down(h.o_col, cl.celem_color.ptr, h.n_col) &&
              down(h.o_pos, cl.celem_pos.ptr, h.n_pos) && down(h.o_ln, cl.celem_lnode.ptr, h.n_ln * 2);
    ok = ok && cudaStreamSynchronize(s) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        h.release();
    }
    return ok;
}

// ClosureSlot (mesh.cuh): device buffers that hold one cached group's closure at a
// time, sized for the largest group, kept by the mesh between calls and reused
// from group to group without freeing in between.
static void group_sizes(const std::vector<HostClosure> &hs, size_t (&n)[9]) {
    for (size_t &v : n) v = 1;
    for (const HostClosure &h : hs) {
        const size_t v[9] = {h.n_pep, h.n_pcp, h.n_gid, h.n_own, h.n_id, h.n_col, h.n_pos, h.n_ln, h.n_aidx};
        for (int k = 0; k < 9; ++k) n[k] = std::max(n[k], v[k]);
    }
}

bool ClosureSlot::fits(const std::vector<HostClosure> &hs) const {
    size_t n[9];
    group_sizes(hs, n);
    return aidx.ptr && pep.n >= n[0] && pcp.n >= n[1] && gid.n >= n[2] && own.n >= n[3] && id.n >= n[4] &&
           col.n >= n[5] && pos.n >= n[6] && ln.n >= n[7] && aidx.n >= n[8];
}

fem_status ClosureSlot::alloc(Arena &ar, const std::vector<HostClosure> &hs) {
    release();
    size_t n[9];
    group_sizes(hs, n);
    FEM_TRY(pep.alloc(ar, n[0], "group slot"));
    FEM_TRY(pcp.alloc(ar, n[1], "group slot"));
    FEM_TRY(gid.alloc(ar, n[2], "group slot"));
    FEM_TRY(own.alloc(ar, n[3], "group slot"));
    FEM_TRY(id.alloc(ar, n[4], "group slot"));
    FEM_TRY(col.alloc(ar, n[5], "group slot"));
    FEM_TRY(pos.alloc(ar, n[6], "group slot"));
    FEM_TRY(ln.alloc(ar, n[7], "group slot"));
    FEM_TRY(aidx.alloc(ar, n[8], "group slot"));
    return FEM_OK;
}

void ClosureSlot::release() {
    pep.free(); pcp.free(); gid.free(); own.free(); id.free(); col.free(); pos.free(); ln.free(); aidx.free();
}

void ClosureSlot::view(const HostClosure &h, Closure &cl) const {
    cl.p0 = h.p0, cl.p1 = h.p1, cl.total_cnodes = h.total_cnodes, cl.total_celems = h.total_celems;
    cl.max_cnodes = h.max_cnodes, cl.max_celems = h.max_celems, cl.n_colors = h.n_colors;
    auto lend = [](auto &d, auto *ptr, size_t n) {
        d.ptr = ptr;
        d.n = n;
        d.arena = nullptr;
    };
    lend(cl.patch_elem_ptr, pep.ptr, h.n_pep);
    lend(cl.patch_cnode_ptr, pcp.ptr, h.n_pcp);
    lend(cl.cnode_gid, gid.ptr, h.n_gid);
    lend(cl.cnode_own, own.ptr, h.n_own);
    lend(cl.celem_id, id.ptr, h.n_id);
    lend(cl.celem_color, col.ptr, h.n_col);
    lend(cl.celem_pos, pos.ptr, h.n_pos);
    lend(cl.celem_lnode, ln.ptr, h.n_ln);
    lend(cl.celem_aidx, aidx.ptr, h.n_aidx);
}

fem_status ClosureSlot::upload(fem_mesh m, const HostClosure &h, cudaStream_t s) {
    auto up = [&](void *dst, size_t off, size_t bytes) -> fem_status {
        if (bytes) FEM_CUDA(cudaMemcpyAsync(dst, h.host + off, bytes, cudaMemcpyHostToDevice, s));
        return FEM_OK;
    };
    FEM_TRY(up(pep.ptr, h.o_pep, h.n_pep * 8));
    FEM_TRY(up(pcp.ptr, h.o_pcp, h.n_pcp * 8));
    FEM_TRY(up(gid.ptr, h.o_gid, h.n_gid * 4));
    FEM_TRY(up(own.ptr, h.o_own, h.n_own * 4));
    FEM_TRY(up(id.ptr, h.o_id, h.n_id * 4));
    FEM_TRY(up(col.ptr, h.o_col, h.n_col));
    FEM_TRY(up(pos.ptr, h.o_pos, h.n_pos));
    FEM_TRY(up(ln.ptr, h.o_ln, h.n_ln * 2));
    Closure cl;
    view(h, cl);
    return expand_targets(m, cl, aidx.ptr, s);
}

void drop_group_cache(fem_mesh m) {
    m->group_cache.clear();
    m->group_slot[0].release();
    m->group_slot[1].release();
}

// Builds the closure of patches [p0, p1) (halving the range while the budget
// refuses it), runs fn on it and frees it; with `rec`, the closures are built
// with their positions and a host copy of each is appended to rec (rec_ok is
// cleared if host memory runs out).
static fem_status closure_range(fem_mesh m, int64_t p0, int64_t p1, cudaStream_t s,
                                const std::function<fem_status(const Closure &)> &fn, int *groups,
                                std::vector<HostClosure> *rec = nullptr, bool *rec_ok = nullptr) {
    Closure cl;
    fem_status st = build_closure(m, p0, p1, cl, s, m->want_pos || rec != nullptr);
    if (st == FEM_ERR_BUDGET && p1 - p0 > 1) {
        cl.reset();
        cudaGetLastError();
        const int64_t mid = p0 + (p1 - p0) / 2;
        FEM_TRY(closure_range(m, p0, mid, s, fn, groups, rec, rec_ok));
        return closure_range(m, mid, p1, s, fn, groups, rec, rec_ok);
    }
    FEM_TRY(st);
    ++*groups;
    FEM_TRY(fn(cl));
    if (rec && *rec_ok) {
        HostClosure h;
        if (closure_to_host(cl, h, s)) rec->push_back(std::move(h));
        else *rec_ok = false;
    }
    FEM_CUDA(cudaStreamSynchronize(s));  // the closure's buffers are freed on return
    return FEM_OK;
}

// The cached groups, copied back one after the other into slots.  With two slots
// (when the budget holds them) group i + 1 is copied in (and its targets
// derived) on a second stream while group i runs; with one, copies and runs
// alternate on the caller's stream.  *done stays false if not even one slot fits.
static fem_status run_cached_groups(fem_mesh m, cudaStream_t s,
                                    const std::function<fem_status(const Closure &)> &fn, bool *done) {
    *done = false;
    const std::vector<HostClosure> &hs = m->group_cache;
    const int n = (int)hs.size();
    ClosureSlot *slot = m->group_slot;  // kept between calls (allocating them each call would cost more)
    if (!slot[0].fits(hs) && slot[0].alloc(m->arena, hs) != FEM_OK) {
        cudaGetLastError();
        slot[0].release();
        return FEM_OK;
    }
    int nslots = 2;
    if (n < 2 || (!slot[1].fits(hs) && slot[1].alloc(m->arena, hs) != FEM_OK)) {
        cudaGetLastError();
        slot[1].release();
        nslots = 1;
    }
    if (nslots == 2 && !m->copy_stream) FEM_CUDA(cudaStreamCreateWithFlags(&m->copy_stream, cudaStreamNonBlocking));
    cudaEvent_t up[2] = {}, fin[2] = {};
    fem_status st = FEM_OK;
    for (int k = 0; k < nslots && st == FEM_OK; ++k) {
        if (cudaEventCreateWithFlags(&up[k], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&fin[k], cudaEventDisableTiming) != cudaSuccess)
            st = cuda_status(cudaGetLastError(), "group slot events");
    }
    // copies into a slot wait for the slot's previous group to have run (at the
    // start: for whatever the caller's stream did with memory the slot reuses)
    for (int k = 0; k < nslots && st == FEM_OK && nslots == 2; ++k)
        if (cudaEventRecord(fin[k], s) != cudaSuccess) st = cuda_status(cudaGetLastError(), "group slot events");
    auto copy_in = [&](int i) -> fem_status {
        const int k = i % nslots;
        if (nslots == 1) return slot[0].upload(m, hs[i], s);
        FEM_CUDA(cudaStreamWaitEvent(m->copy_stream, fin[k], 0));
        FEM_TRY(slot[k].upload(m, hs[i], m->copy_stream));
        FEM_CUDA(cudaEventRecord(up[k], m->copy_stream));
        return FEM_OK;
    };
    if (st == FEM_OK) st = copy_in(0);
    for (int i = 0; i < n && st == FEM_OK; ++i) {
        const int k = i % nslots;
        if (nslots == 2 && i + 1 < n) st = copy_in(i + 1);
        if (st != FEM_OK) break;
        if (nslots == 2 && cudaStreamWaitEvent(s, up[k], 0) != cudaSuccess) {
            st = cuda_status(cudaGetLastError(), "group slot wait");
            break;
        }
        Closure cl;
        slot[k].view(hs[i], cl);
        st = fn(cl);
        if (st != FEM_OK) break;
        if (nslots == 2 && cudaEventRecord(fin[k], s) != cudaSuccess) st = cuda_status(cudaGetLastError(), "group slot");
        if (nslots == 1 && i + 1 < n && st == FEM_OK) st = copy_in(i + 1);
    }
    // the slots are reused by the next call: everything that reads them must be done
    const cudaError_t e = cudaStreamSynchronize(s);
    if (st == FEM_OK && e != cudaSuccess) st = cuda_status(e, "group slots");
    if (nslots == 2) cudaStreamSynchronize(m->copy_stream);
    for (int k = 0; k < 2; ++k) {
        if (up[k]) cudaEventDestroy(up[k]);
        if (fin[k]) cudaEventDestroy(fin[k]);
    }
    if (st == FEM_OK) {
        m->n_groups = n;
        *done = true;
    }
    return st;
}

fem_status for_each_group(fem_mesh m, cudaStream_t s, const std::function<fem_status(const Closure &)> &fn) {
    Plan &P = m->plan;
    if (!P.chunked) return fn(P.full);
    int groups = 0;
    const bool use_cache = m->opt.group_cache != 0;
    if (use_cache && !m->group_cache.empty()) {
        bool done = false;
        FEM_TRY(run_cached_groups(m, s, fn, &done));
        if (done) return FEM_OK;
        // no slot fits beside what the call holds now: each group's closure is
        // built again, in smaller parts where it does not fit
        for (const HostClosure &h : m->group_cache) FEM_TRY(closure_range(m, h.p0, h.p1, s, fn, &groups));
        m->n_groups = groups;
        return FEM_OK;
    }
    // Building the groups (and, with the cache, their host copies): with the cache,
    // groups of half the size, so that two of them fit where one did and the
    // copy of one can overlap the run of the other.
    std::vector<HostClosure> rec;
    bool rec_ok = use_cache;
    const int64_t G = use_cache ? std::max<int64_t>(1, m->group_patches / 2) : m->group_patches;
    for (int64_t p0 = 0; p0 < P.n_patches; p0 += G)
        FEM_TRY(closure_range(m, p0, std::min(P.n_patches, p0 + G), s, fn, &groups, use_cache ? &rec : nullptr,
                              &rec_ok));
    m->n_groups = groups;
    if (use_cache && rec_ok) m->group_cache = std::move(rec);
    return FEM_OK;
}

fem_status for_each_group_in(fem_mesh m, int64_t pa, int64_t pb, cudaStream_t s,
                             const std::function<fem_status(const Closure &)> &fn) {
    Plan &P = m->plan;
    if (!P.chunked) return fn(P.full);
    int groups = 0;
    for (int64_t p0 = pa; p0 < pb; p0 += m->group_patches)
        FEM_TRY(closure_range(m, p0, std::min(pb, p0 + m->group_patches), s, fn, &groups));
    return FEM_OK;
}

}  // namespace fem
