// tile.cuh -- element tiles: the assembly of the scalar operators (stiffness and
// mass) that integrates every element exactly once.
//
// Elements are ordered along the locality curve and cut into tiles of about
// `tile_elems` consecutive elements (Eq. 10's element groups, made small enough
// for one thread block).  A block integrates its tile's elements (Eqs. 7-9) and
// adds their packed entries into shared-memory accumulators that hold the whole
// lower row of every node its elements touch.  Elements of a tile are coloured so
// that no two elements of one colour share a node; the block adds colour by
// colour, so every accumulator is a sum in a fixed order.
//
// A row whose incident elements all lie in the tile (interior) is then complete
// and goes straight into K's values.  A row touched by k >= 2 tiles (border) is
// written by each of them as a partial row into library memory, at a slot fixed
// by the plan (the k partials of a row in ascending tile order); a second kernel
// then sums every border row's k partials in slot order and writes the row.  No
// block waits for or signals another, the summation order of every entry is
// fixed by the plan, and the values are bitwise reproducible whatever order the
// blocks run in.
#pragma once

#include "common.cuh"

namespace fem {

// node_info bits: accumulator offset of the row in its tile (bits 0-15), row
// length (16-23), border row (24), diagonal summed FP64-accurately (25).
static constexpr uint32_t TILE_BORDER = 1u << 24, TILE_HV = 1u << 25;
// Per-tile padding of the plan's element and node arrays, so that every tile's
// slice starts on a 16-byte boundary and is a whole number of 16-byte units: the
// tile kernel stages a tile's slices in shared memory with bulk copies.
static constexpr int TILE_EPAD = 16, TILE_NPAD = 4;
// Words of in-row positions per element: four 8-bit positions a word.
__host__ __device__ constexpr int tile_posw(int npe) { return (npe * (npe + 1) / 2 + 3) / 4; }

struct TileView {
    const int64_t *tile_elem_ptr;  // [n_tiles + 1] padded ranges of the element arrays
    const int32_t *tile_nel;       // [n_tiles] elements of the tile
    const int64_t *tile_node_ptr;  // [n_tiles + 1] padded ranges of the row arrays
    const int32_t *tile_ncn;       // [n_tiles] rows (nodes) of the tile
    const int32_t *tile_acc;       // [n_tiles] accumulator entries of the tile (sum of its row lengths)
    const int32_t *elem_id;        // element ids in tile order, by (colour, sweep) within a tile
    const uint8_t *elem_color;
    const uint16_t *elem_lnode;    // [. * npe] tile-local node index (rows ascend by node id in a tile)
    // in-row positions of the packed pairs: per tile, [tile_posw][padded elements]
    // words starting at word tile_elem_ptr[t] * tile_posw, byte q & 3 of word q >> 2
    // for pair q: the position of min(g_a, g_b) in row max(g_a, g_b)
    const uint32_t *elem_pos;
    const int32_t *node_gid;   // global node id of each row
    const int64_t *node_dest;  // offset of the row in vals (interior) or in the partials (border)
    const uint32_t *node_info; // see TILE_BORDER
    const int64_t *brow_base;  // [n_brows] partials offset of the border row's first tile
    const int64_t *brow_vo;    // [n_brows] offset of the border row in vals
    const uint32_t *brow_info; // [n_brows] length | hv << 8 | tiles (>= 2) << 16
    int64_t n_tiles, n_elems, n_nodes, nnz, n_brows, partial_n;
};

struct TilePlan {
    bool ready = false;
    int64_t n_tiles = 0, n_tnodes = 0, n_brows = 0, partial_n = 0;
    int64_t max_acc = 0, max_tnodes = 0, max_elems = 0;
    int64_t max_epad = 0, max_npad = 0;  // largest padded slices (the kernel's staging)
    int n_colors = 0;
    bool any_hv = false;
    int tile_elems = 0;  // elements per tile the plan was cut for
    DevBuf<int64_t> tile_elem_ptr, tile_node_ptr, node_dest, brow_base, brow_vo;
    DevBuf<int32_t> tile_nel, tile_ncn, tile_acc, elem_id, node_gid;
    DevBuf<uint8_t> elem_color;
    DevBuf<uint16_t> elem_lnode;
    DevBuf<uint32_t> elem_pos, node_info, brow_info;
    // border partial rows of the last build: partial_n values of the build's
    // precision (float or double), allocated on first use
    DevBuf<unsigned char> partial;
    TileView view(const fem_mesh_s *m) const;
    void reset() {
        tile_elem_ptr.free(); tile_node_ptr.free(); node_dest.free(); brow_base.free(); brow_vo.free();
        tile_nel.free(); tile_ncn.free(); tile_acc.free(); elem_id.free(); node_gid.free(); elem_color.free();
        elem_lnode.free(); elem_pos.free(); node_info.free(); brow_info.free(); partial.free();
        ready = false;
        n_tiles = n_tnodes = n_brows = partial_n = max_acc = max_tnodes = max_elems = max_epad = max_npad = 0;
        n_colors = 0;
        any_hv = false;
        tile_elems = 0;
    }
    size_t bytes() const {
        return tile_elem_ptr.bytes() + tile_node_ptr.bytes() + node_dest.bytes() + brow_base.bytes() +
               brow_vo.bytes() + tile_nel.bytes() + tile_ncn.bytes() + tile_acc.bytes() + elem_id.bytes() +
               node_gid.bytes() + elem_color.bytes() + elem_lnode.bytes() + elem_pos.bytes() + node_info.bytes() +
               brow_info.bytes() + partial.bytes();
    }
};

// Launch bounds of the tile kernel per element type (as the patch kernel's).
__host__ __device__ constexpr int tile_max_threads(int npe) { return npe == 4 ? 256 : 512; }
__host__ __device__ constexpr int tile_min_blocks(int npe) { return npe == 4 ? 3 : 1; }

}  // namespace fem
