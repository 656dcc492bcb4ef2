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

#include "common.cuh"

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
};

struct Plan {
    int64_t n_patches = 0, total_cnodes = 0, total_celems = 0;
    int64_t max_acc = 0, max_cnodes = 0, max_own = 0, max_celems = 0;
    int n_colors = 0;
    int pos_stride = 0;
    DevBuf<int64_t> patch_node_ptr, patch_elem_ptr, patch_cnode_ptr, own_rowptr;
    DevBuf<int32_t> patch_acc, own_acc, cnode_gid, cnode_own, celem_id, own_row, node_patch, own_idx;
    DevBuf<uint8_t> own_hv, celem_color, celem_pos;
    DevBuf<uint16_t> celem_lnode;
    PlanView view() const {
        return PlanView{patch_node_ptr.ptr, patch_elem_ptr.ptr, patch_cnode_ptr.ptr, patch_acc.ptr,
                        own_acc.ptr,        own_rowptr.ptr,     own_hv.ptr,          cnode_gid.ptr,
                        cnode_own.ptr,      celem_id.ptr,       celem_color.ptr,     celem_lnode.ptr,
                        celem_pos.ptr,      own_row.ptr,        n_patches};
    }
    size_t bytes() const {
        return patch_node_ptr.bytes() + patch_elem_ptr.bytes() + patch_cnode_ptr.bytes() + own_rowptr.bytes() +
               patch_acc.bytes() + own_acc.bytes() + cnode_gid.bytes() + cnode_own.bytes() + celem_id.bytes() +
               own_row.bytes() + node_patch.bytes() + own_idx.bytes() + own_hv.bytes() + celem_color.bytes() +
               celem_pos.bytes() + celem_lnode.bytes();
    }
};

}  // namespace fem

struct fem_mesh_s {
    fem_elem type;
    int npe = 0, np = 0;  // nodes per element, packed entries per element
    int64_t n_nodes = 0, n_elems = 0;
    const int32_t *E = nullptr;  // caller-owned connectivity
    fem_options opt;
    fem::Arena arena;
    fem::DevBuf<int32_t> order;    // node order along the locality curve
    bool has_pattern = false;
    int64_t nnz = 0;
    int max_row_len = 0;
    fem::DevBuf<int64_t> rowptr;
    fem::DevBuf<int32_t> col;
    fem::DevBuf<int64_t> inc_ptr;  // node -> incident elements (kept for the backward pass)
    fem::DevBuf<int32_t> inc_elem;
    fem::Plan plan;
    // staging for the _host entry point
    fem::DevBuf<unsigned char> host_stage;
    int n_groups = 1;
};

namespace fem {
fem_status build_locality_order(fem_mesh m, const void *X, fem_dtype xd, cudaStream_t s);
fem_status validate_connectivity(fem_mesh m, cudaStream_t s);
fem_status build_pattern_and_plan(fem_mesh m, cudaStream_t s);
}  // namespace fem
