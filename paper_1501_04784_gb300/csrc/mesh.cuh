// mesh.cuh -- the mesh handle behind the opaque fem_mesh, and the plan of the
// numeric kernels.
//
// Plan ("owner computes").  Nodes are ordered along a space-filling curve and
// cut into patches of consecutive nodes holding at most `patch_entries` lower-CSR
// entries; one thread block owns one patch's rows.  It integrates every element
// that touches an owned node (the patch's closure), accumulates the entries of
// its owned rows in shared memory, and writes each owned row once.  Elements of a
// closure are coloured so that no two elements of one colour share an owned node;
// the block adds colour by colour, so each entry is a sum in a fixed order and
// the result is bitwise reproducible without atomics.
#pragma once

#include <cstring>
#include <functional>
#include <utility>
#include <vector>

#include "common.cuh"
#include "tile.cuh"

namespace fem {

struct PlanView {
    const int64_t *patch_node_ptr;   // [n_patches + 1] into own_* (node order)
    const int64_t *patch_elem_ptr;   // [n_patches + 1] into celem_*
    const int64_t *patch_cnode_ptr;  // [n_patches + 1] into cnode_*
    const int32_t *patch_acc;        // [n_patches] entries owned by the patch
    const int32_t *own_acc;          // [n_nodes] offset of the owned row in its patch's entries
    const int64_t *own_rowptr;       // [n_nodes] rowptr of the owned row
    const uint8_t *own_hv;           // [n_nodes] 1 if the row's diagonal is summed in FP64 (mixed)
    const int32_t *cnode_gid;        // [total cnodes] global node id, ascending within a patch
    const int32_t *cnode_own;        // [total cnodes] owned-row index within the patch, or -1
    const int32_t *celem_id;         // [total celems] element id, sorted by (colour, id) in a patch
    const uint8_t *celem_color;      // [total celems]
    const uint16_t *celem_lnode;     // [total celems * npe] closure-local node index
    const uint8_t *celem_pos;        // [total celems * pos_stride] position of the entry in its row
    const int32_t *own_row;          // [n_nodes] global id of each owned row, in patch order
    int64_t n_patches;
    // [NP/2 words][total celems] (word-major, so a warp's loads of one word are
    // contiguous): two 16-bit targets per word, entry q in the low half when q is
    // even.  A target is the entry's offset in the patch's accumulators; for a
    // pair whose row the patch does not own, one of 32 scratch accumulators past
    // the largest patch's (max_acc + the element's lane in its batch), added to
    // and never read; 0x8000 | k for the diagonal of owned row k when that row's
    // diagonal is summed FP64-accurately.
    const uint32_t *celem_aidx;
    int64_t aidx_n;                  // total celems (the word stride)
    int64_t val_off;                 // subtracted from own_rowptr: vals holds the values from
                                     // this CSR position on (a row range of the host pipeline)
    int64_t n_nodes, n_elems, nnz;   // sizes of X, c and vals (bounds checks of the debug build)
};

// Marker bit of celem_aidx's FP64-accurate diagonals; scratch accumulators per block.
static constexpr uint32_t AIDX_HV = 0x8000u;
static constexpr int ACC_SCRATCH = 32;

// Closure data of a range of patches [p0, p1): the elements each patch
// integrates and the nodes they touch.  Patch indices inside are relative to p0.
struct Closure {
    int64_t p0 = 0, p1 = 0, total_cnodes = 0, total_celems = 0;
    int64_t max_cnodes = 0, max_celems = 0;
    int n_colors = 0;
    DevBuf<int64_t> patch_elem_ptr, patch_cnode_ptr;
    DevBuf<int32_t> cnode_gid, cnode_own, celem_id;
    DevBuf<uint8_t> celem_color, celem_pos;
    DevBuf<uint16_t> celem_lnode;
    DevBuf<uint32_t> celem_aidx;
    void reset() {
        patch_elem_ptr.free(); patch_cnode_ptr.free(); cnode_gid.free(); cnode_own.free(); celem_id.free();
        celem_color.free(); celem_pos.free(); celem_lnode.free(); celem_aidx.free();
        p0 = p1 = total_cnodes = total_celems = max_cnodes = max_celems = 0;
        n_colors = 0;
    }
    size_t bytes() const {
        return patch_elem_ptr.bytes() + patch_cnode_ptr.bytes() + cnode_gid.bytes() + cnode_own.bytes() +
               celem_id.bytes() + celem_color.bytes() + celem_pos.bytes() + celem_lnode.bytes() + celem_aidx.bytes();
    }
};

struct Plan {
    int64_t n_patches = 0;
    int64_t max_acc = 0, max_own = 0;
    int64_t n_nodes = 0, n_elems = 0, nnz = 0;
    int pos_stride = 0;
    bool any_hv = false;  // some row's diagonal is summed FP64-accurately (mixed)
    DevBuf<int64_t> patch_node_ptr, own_rowptr;
    DevBuf<int32_t> patch_acc, own_acc, own_row, node_patch, own_idx;
    DevBuf<uint8_t> own_hv;
    Closure full;          // closure of every patch, when it fits the memory budget
    bool chunked = false;  // closures built per patch group at each numeric call
    // aggregate statistics (over all groups when chunked)
    int64_t total_cnodes = 0, total_celems = 0, max_cnodes = 0, max_celems = 0;
    int n_colors = 0;
    // Row ranges of the host pipeline (fem_options.host_chunks; one range when
    // off): range k owns rows [chunk_row[k], chunk_row[k+1]), whose values are
    // CSR positions [chunk_val[k], chunk_val[k+1]), and patches
    // [chunk_patch[k], chunk_patch[k+1]) (no patch owns rows of two ranges).
    std::vector<int64_t> chunk_row, chunk_val, chunk_patch;
    int64_t max_chunk_vals = 0;
    int64_t cap_entries = 0;  // entries a patch was cut to hold
    int n_chunks() const { return chunk_row.empty() ? 1 : (int)chunk_row.size() - 1; }
    PlanView view(const Closure &cl) const {
        PlanView v{};
        v.patch_node_ptr = patch_node_ptr.ptr + cl.p0;
        v.patch_elem_ptr = cl.patch_elem_ptr.ptr;
        v.patch_cnode_ptr = cl.patch_cnode_ptr.ptr;
        v.patch_acc = patch_acc.ptr + cl.p0;
        v.own_acc = own_acc.ptr;
        v.own_rowptr = own_rowptr.ptr;
        v.own_hv = own_hv.ptr;
        v.cnode_gid = cl.cnode_gid.ptr;
        v.cnode_own = cl.cnode_own.ptr;
        v.celem_id = cl.celem_id.ptr;
        v.celem_color = cl.celem_color.ptr;
        v.celem_lnode = cl.celem_lnode.ptr;
        v.celem_pos = cl.celem_pos.ptr;
        v.own_row = own_row.ptr;
        v.n_patches = cl.p1 - cl.p0;
        v.celem_aidx = cl.celem_aidx.ptr;
        v.aidx_n = cl.total_celems;
        v.val_off = 0;
        v.n_nodes = n_nodes;
        v.n_elems = n_elems;
        v.nnz = nnz;
        return v;
    }
    PlanView view() const { return view(full); }
    void reset() {
        patch_node_ptr.free(); own_rowptr.free(); patch_acc.free(); own_acc.free(); own_row.free();
        node_patch.free(); own_idx.free(); own_hv.free(); full.reset();
        n_patches = max_acc = max_own = total_cnodes = total_celems = max_cnodes = max_celems = 0;
        n_colors = 0;
        chunked = false;
        any_hv = false;
        chunk_row.clear();
        chunk_val.clear();
        chunk_patch.clear();
        max_chunk_vals = 0;
        cap_entries = 0;
    }
    size_t bytes() const {
        return patch_node_ptr.bytes() + own_rowptr.bytes() + patch_acc.bytes() + own_acc.bytes() + own_row.bytes() +
               node_patch.bytes() + own_idx.bytes() + own_hv.bytes() + full.bytes();
    }
};

// A copy, in page-locked host memory, of one patch group's closure (plans built
// per patch group under the memory budget): the numeric calls copy it back to the
// device instead of building the closure again (fem_options.group_cache).  The
// copy holds the in-row positions instead of the accumulator targets (half their
// bytes over the host link); the targets are derived from them on the device.
struct HostClosure {
    int64_t p0 = 0, p1 = 0, total_cnodes = 0, total_celems = 0, max_cnodes = 0, max_celems = 0;
    int n_colors = 0;
    unsigned char *host = nullptr;
    size_t bytes = 0;
    // byte offsets of the arrays in `host` and their element counts (n_aidx: the
    // target words the device derives, which the copy does not hold)
    size_t o_pep, o_pcp, o_gid, o_own, o_id, o_col, o_pos, o_ln;
    size_t n_pep, n_pcp, n_gid, n_own, n_id, n_col, n_pos, n_ln, n_aidx;
    HostClosure() = default;
    HostClosure(const HostClosure &) = delete;
    HostClosure &operator=(const HostClosure &) = delete;
    HostClosure(HostClosure &&o) noexcept { *this = std::move(o); }
    HostClosure &operator=(HostClosure &&o) noexcept {
        if (this != &o) {
            release();
            std::memcpy(static_cast<void *>(this), static_cast<const void *>(&o), sizeof(HostClosure));
            o.host = nullptr;
            o.bytes = 0;
        }
        return *this;
    }
    void release() {
        if (host) cudaFreeHost(host);
        host = nullptr;
        bytes = 0;
    }
    ~HostClosure() { release(); }
};

// Device buffers that hold one patch group's closure copied back from its host
// copy (groups.cu), sized for the largest group and reused from group to group.
struct ClosureSlot {
    DevBuf<int64_t> pep, pcp;
    DevBuf<int32_t> gid, own, id;
    DevBuf<uint8_t> col, pos;
    DevBuf<uint16_t> ln;
    DevBuf<uint32_t> aidx;
    bool fits(const std::vector<HostClosure> &hs) const;
    fem_status alloc(Arena &ar, const std::vector<HostClosure> &hs);
    void release();
    void view(const HostClosure &h, Closure &cl) const;  // borrows the buffers (frees nothing)
    fem_status upload(fem_mesh m, const HostClosure &h, cudaStream_t s);  // copy in, derive the targets
};

}  // namespace fem

struct fem_mesh_s {
    fem_elem type;
    int npe = 0, np = 0;  // nodes per element, packed entries per element
    int64_t n_nodes = 0, n_elems = 0;
    const int32_t *E = nullptr;  // caller-owned connectivity
    fem_options opt;
    fem::Arena arena;
    fem::DevBuf<int32_t> order;    // node order along the locality curve (range by range, see chunk_rows)
    std::vector<int64_t> chunk_rows;  // row ranges of the host pipeline: [chunk_rows[k], chunk_rows[k+1])
    bool has_pattern = false;
    int64_t nnz = 0;
    int max_row_len = 0;
    int64_t max_deg = 0;  // most elements incident to one node
    fem::DevBuf<int64_t> rowptr;
    fem::DevBuf<int32_t> col;
    fem::DevBuf<int64_t> inc_ptr;  // node -> incident elements (kept for the backward pass)
    fem::DevBuf<int32_t> inc_elem;
    fem::Plan plan;
    bool plan_built = false;  // the patch plan exists (it is built on first use when tiles serve the builds)
    bool want_pos = false;    // closures carry the in-row positions (set by the first backward pass)
    fem::TilePlan tiles;      // element tiles of the scalar operators (tile.cuh)
    // device status word: set by a bounded device-side wait that gave up
    fem::DevBuf<int> status;
    // staging of the host-buffer entry points: HOST_STAGES slots used in turn, so
    // that a call's input copy and build overlap the output copies of the calls
    // before it (with three, a call's input copy does not wait for the output
    // copy of the call two before it, and the output link stays busy);
    // stage_free[k] is recorded after slot k's output copy, `built` after each
    // call's build kernels (the next call's kernels wait for it: builds of one
    // mesh never run concurrently, they share library buffers)
    static constexpr int HOST_STAGES = 3;
    fem::DevBuf<unsigned char> host_stage[HOST_STAGES];
    cudaEvent_t stage_free[HOST_STAGES] = {};
    cudaEvent_t built = nullptr;
    int stage_next = 0;
    ~fem_mesh_s() {
        for (cudaEvent_t e : stage_free)
            if (e) cudaEventDestroy(e);
        if (built) cudaEventDestroy(built);
        for (int j = 0; j < 2; ++j) {
            if (chunk_built[j]) cudaEventDestroy(chunk_built[j]);
            if (slot_free[j]) cudaEventDestroy(slot_free[j]);
        }
        if (copy_stream) cudaStreamDestroy(copy_stream);
    }
    // FP64 element matrices staged between integration and assembly (the FP64
    // pipe is the bound there, so integrating each element once beats recomputing
    // it in every closure that contains it)
    fem::DevBuf<double> ke64;
    // host pipeline over row ranges: two device value slots used in turn, the
    // stream their copies to the host run on, chunk_built[j] recorded after the
    // build of the range in slot j, slot_free[j] after its copy out
    fem::DevBuf<unsigned char> chunk_slots;
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t chunk_built[2] = {}, slot_free[2] = {};
    int n_groups = 1;
    int64_t group_patches = 0;  // patches per group when the closures are built per group
    // host copies of the patch groups' closures, in patch order (fem_options.group_cache),
    // and the two device slots the groups are copied back into (kept between calls)
    std::vector<fem::HostClosure> group_cache;
    fem::ClosureSlot group_slot[2];
};

namespace fem {
fem_status build_locality_order(fem_mesh m, const void *X, fem_dtype xd, cudaStream_t s);
fem_status validate_connectivity(fem_mesh m, cudaStream_t s);
void batch_forget(fem_mesh m);  // drops cached batched launches that use m's plan
fem_status build_pattern(fem_mesh m, cudaStream_t s);
fem_status build_plan(fem_mesh m, cudaStream_t s);
// Frees the host copies of the patch groups and their device slots (the plan changed).
void drop_group_cache(fem_mesh m);
// with_pos: the closure carries the in-row positions (the backward pass, the host copies)
fem_status build_closure(fem_mesh m, int64_t p0, int64_t p1, Closure &cl, cudaStream_t s, bool with_pos);
// From now on the closures carry the in-row positions the backward pass reads.
fem_status ensure_positions(fem_mesh m, cudaStream_t s);
// Runs fn over the closure of every patch group (one group covering all patches
// unless the plan is chunked under the memory budget).
fem_status for_each_group(fem_mesh m, cudaStream_t s, const std::function<fem_status(const Closure &)> &fn);
// The same over patches [pa, pb) only: closures that hold them (the whole plan's
// when it is not chunked; the caller restricts the launch to [pa, pb)).
fem_status for_each_group_in(fem_mesh m, int64_t pa, int64_t pb, cudaStream_t s,
                             const std::function<fem_status(const Closure &)> &fn);
}  // namespace fem
