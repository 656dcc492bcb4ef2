// numeric.cuh -- launch interfaces of the numeric kernels.
#pragma once

#include <algorithm>

#include "mesh.cuh"

namespace fem {

static constexpr int PATCH_MAX_THREADS = 512;

// Launch bounds of the patch kernels per element type.  Tetrahedra need few
// registers: capping them at 256 threads and 3 resident blocks per SM (at most
// 85 registers a thread) lets three blocks share an SM.
__host__ __device__ constexpr int patch_max_threads(int npe) { return npe == 4 ? 256 : PATCH_MAX_THREADS; }
__host__ __device__ constexpr int patch_min_blocks(int npe) { return npe == 4 ? 3 : 1; }

// Resident blocks per SM of the mixed patch kernel at `threads` threads as its
// registers allow (the wave size the plan aligns its patch count to).
int patch_blocks_per_sm(int npe, int threads);

// byte offsets of the patch kernel's shared-memory arrays
struct PatchSmem {
    size_t acc, hv, xs, cown, roff, hvf, rps, gid, eid, cvs, total;
    // the fused kernel with prefetch: a second set of the prologue arrays, which
    // receives the next patch's closure ids, coordinates and owned-row tables by
    // asynchronous copies while the block works on the current patch
    size_t xs2, roff2, rps2, gid2;
    int prefetch;
    int wg_shift;  // log2 of the lanes that store one owned row
    int acc_cap;   // accumulators a block holds (largest patch + scratch slots)
    int hv_on;     // the hv region exists (some owned row has an FP64-accurate diagonal)
    int win;       // vector operators: owned node-pair slots a pass accumulates (rows in windows)
    int trash;     // vector operators: the plan's first scratch target (its largest patch)
};

// Mode bits of the element kernels: FP64_SUMS, FP64_DETS (mixed kernels;
// fem_options.fp64_sums, fp64_dets) and OP_MASS (fem_options.operator_kind: the
// mass matrix instead of the stiffness matrix).
static constexpr unsigned FP64_SUMS = 1u, FP64_DETS = 2u, OP_MASS = 4u;

// Device-side waits of the patch kernels (colour phases on mbarriers): each wait
// polls at most `spins` times, then records the failure in *status (read by
// fem_sync as FEM_ERR_TIMEOUT) and lets the thread go on, so the kernel ends.
// `stall` (testing) = 1 makes warp 0 of every block wait once for a phase that
// cannot complete, to exercise that path; = 2 (bounds-check build only) plants
// one out-of-range node id per block, to exercise the bounds checks.
struct WaitCtl {
    int *status;
    int spins;
    int stall;
};
static constexpr int WAIT_SPINS_DEFAULT = 1 << 20;

// Bits of the mesh's device status word.
static constexpr int STATUS_TIMEOUT = 1;    // a bounded device-side wait gave up
static constexpr int STATUS_NONFINITE = 2;  // an element matrix was not finite (zero det J, non-finite input)
static constexpr int STATUS_BOUNDS = 4;     // bounds-check build: an out-of-range index, caught and skipped

struct IntegrateArgs {
    int npe;
    bool mixed;
    fem_dtype xd, cd;
    const int32_t *E;
    int64_t nel;
    const void *X, *c;
    void *ke;
    float thr;
    unsigned long long *nflag;
    unsigned mode = 0;     // FP64_DETS, OP_MASS
    int *status = nullptr;  // STATUS_NONFINITE is or-ed in here
};

struct PatchArgs {
    const Plan *plan;
    const Closure *closure;  // the patch group to run (its p0..p1)
    int npe;
    bool mixed, fused;
    fem_dtype xd, cd;
    const void *X, *c, *ke;
    void *vals;
    float thr;
    int64_t p0, p1;    // patches to run (absolute numbers; those the closure holds)
    int64_t val_off;   // vals holds the CSR values from this position on (scalar operators)
    int threads, blocks_per_sm;
    WaitCtl wait;
    unsigned mode;  // FP64_SUMS: high-valence sums with FP64 adds instead of FP32 TwoSum pairs;
                    // FP64_DETS: distorted tetrahedra's determinant in FP64 arithmetic; OP_MASS
};

// Largest per-patch sizes over the plans a launch covers (sizes shared memory).
struct PlanMax {
    int64_t max_acc = 0, max_own = 0, max_cnodes = 0;
    bool any_hv = false;
    void add(const Plan &P) {
        any_hv = any_hv || P.any_hv;
        max_acc = std::max(max_acc, P.max_acc);
        max_own = std::max(max_own, P.max_own);
        max_cnodes = std::max(max_cnodes, P.max_cnodes);
    }
};

// One mesh of a batched build.
struct BatchItem {
    PlanView pv;
    const void *X, *c;
    void *vals;
    float thr;
    int pad;
};

// Shared memory of the tile kernels (byte offsets) and the largest tile sizes
// over the plans a launch covers.
struct TileSmem {
    size_t acc, hv, xs;                          // accumulators, FP64-accurate diagonals, coordinates
    size_t s_id, s_col, s_ln, s_pos;             // staged element slices of the tile (bulk copies)
    size_t s_gid, s_info, s_dest;                // staged row slices of the tile (bulk copies)
    size_t total;
    int hv_on;     // the plans have FP64-accurate diagonals
    int wg_shift;  // log2 of the lanes that store one row
};
struct TileMax {
    int64_t max_acc = 0, max_epad = 0, max_npad = 0;
    bool any_hv = false;
    void add(const TilePlan &T) {
        any_hv = any_hv || T.any_hv;
        max_acc = std::max(max_acc, T.max_acc);
        max_epad = std::max(max_epad, T.max_epad);
        max_npad = std::max(max_npad, T.max_npad);
    }
};
TileSmem tile_smem_layout(const TileMax &T, int npe, bool mixed, size_t xsize);

// One mesh of a batched build on element tiles.
struct TileBatchItem {
    TileView tv;
    const void *X, *c;
    void *vals, *part;
    float thr;
    int pad;
};

struct BatchLaunch {
    int npe = 8;
    bool mixed = true;
    unsigned mode = 0;
    const BatchItem *items = nullptr;
    const int64_t *prefix = nullptr;
    int n = 0;
    PatchSmem L{};
    int threads = 256, grid = 1;
    WaitCtl wait{nullptr, WAIT_SPINS_DEFAULT, 0};
    bool elastic = false;  // the elasticity operator's kernel (elastic.cu)
    bool win = false;      // its row-window variant (the FP64 blocks outgrow shared memory)
    bool tiles = false;    // the element-tile kernel (tile.cu) over titems
    const TileBatchItem *titems = nullptr;
    const int64_t *bprefix = nullptr;  // tiles: prefix sums of the meshes' border rows (the combine's work)
    TileSmem tl{};
    int combine_grid = 1;
};

// Shared memory, residency and grid of the batched kernel for `threads` threads
// and at most `blocks_per_sm` blocks per SM (0 = as many as fit).
fem_status batched_config(int npe, bool mixed, const PlanMax &pm, int threads, int blocks_per_sm, BatchLaunch *out);
fem_status launch_batched_kernel(const BatchLaunch &bl, cudaStream_t s);

fem_status launch_integrate(const IntegrateArgs &a, cudaStream_t s);

WaitCtl wait_ctl(fem_mesh m);
fem_status check_status(fem_mesh m, cudaStream_t s);

inline unsigned kernel_mode(const fem_options &o) {
    return (o.fp64_sums ? FP64_SUMS : 0u) | (o.fp64_dets ? FP64_DETS : 0u) | (o.operator_kind == 1 ? OP_MASS : 0u);
}
fem_status launch_patch(const PatchArgs &a, cudaStream_t s);

// Element-tile build of the scalar operators (tile.cu, tile_plan.cu).
struct TileArgs {
    const TilePlan *plan;
    TileView view;
    int npe;
    bool mixed;
    fem_dtype xd, cd;
    const void *X, *c;
    void *vals;
    void *part;  // the plan's partials buffer, partial_n values of the build's precision
    float thr;
    int threads, blocks_per_sm;
    WaitCtl wait;
    unsigned mode;  // FP64_SUMS, FP64_DETS, OP_MASS
};
fem_status launch_tile(const TileArgs &a, cudaStream_t s);
fem_status tile_batched_config(int npe, bool mixed, const TileMax &tm, int threads, int blocks_per_sm,
                               BatchLaunch *out);
fem_status launch_tile_batched_kernel(const BatchLaunch &bl, cudaStream_t s);
int tile_blocks_per_sm(int npe, int threads);
// Element tiles of mesh m (after its pattern).
fem_status build_tiles(fem_mesh m, cudaStream_t s);
PatchSmem patch_smem_layout(const PlanMax &P, bool fused, bool mixed, size_t xsize, size_t csize,
                            bool prefetch = false);

// Elasticity operator (three DOFs per node, elastic.cu): the patch kernel over the
// scalar operator's plan (3x3 block per node-pair slot), the packed element
// matrices (elastic_np entries each) and the DOF pattern from the node pattern.
fem_status launch_elastic_patch(const PatchArgs &a, cudaStream_t s);
fem_status launch_elastic_integrate(const IntegrateArgs &a, cudaStream_t s);
fem_status launch_dof_pattern(const int64_t *rowptr, const int32_t *col, int64_t n, int64_t *rowptr3, int32_t *col3,
                              cudaStream_t s);
PatchSmem elastic_smem_layout(const PlanMax &P, bool fused, bool mixed, size_t xsize, int win);
// Slots per pass of the elasticity patch kernel under the shared-memory limit: all
// of the largest patch's when they fit, else as many as fit (0 if fewer than one
// longest row).
int elastic_window(const PlanMax &P, bool fused, bool mixed, size_t xsize, size_t limit);
int elastic_threads(int npe, int requested);
int elastic_blocks_per_sm(int npe, int threads);
fem_status elastic_batched_config(int npe, bool mixed, const PlanMax &pm, int threads, int blocks_per_sm,
                                  BatchLaunch *out);
fem_status launch_elastic_batched_kernel(const BatchLaunch &bl, cudaStream_t s);

}  // namespace fem
