/*
 * fem.h -- C ABI of libfem: global stiffness-matrix construction for the 3D
 * Poisson equation on one GB300 (sm_103a).
 *
 * The operation (Ramirez-Gil, Tsuzuki, Montealegre-Rubio, "Global finite element
 * matrix construction based on a CPU-GPU implementation"):
 *   given node coordinates C, element connectivity E and a per-element
 *   coefficient MP = c_e (Section 3), build K = sum_e k_e (Eq. 6) with
 *   k_e = c_e * integral B^T B dOmega (Eq. 7), evaluated on the reference element
 *   (Eq. 8) by Gauss quadrature (Eq. 9): 2x2x2 points for the 8-node brick, the
 *   exact 1-point rule for the 4-node tetrahedron.  Only the lower triangle is
 *   computed and stored (Section 3: 36 of the 64 entries of a brick's k_e), and
 *   the result is a lower-triangular CSR matrix (the paper's CSC of the upper
 *   triangle has the same arrays).
 *
 * Conventions shared by every call
 *   - Pointers named X, c, E, ke, vals, rowptr, col, G, dX, dc are DEVICE
 *     pointers unless the function name ends in _host.  The caller owns them.
 *   - X is [n_nodes][3] row-major; E is [n_elems][npe] int32 row-major
 *     (npe = 8 or 4); c is [n_elems].  Brick node order: nodes 0-3 on the face
 *     t = -1 counter-clockwise from (-1,-1,-1), nodes 4-7 the same on t = +1.
 *   - Packed lower k_e: [n_elems][npe(npe+1)/2], entry p = a(a+1)/2 + b, b <= a.
 *     The local pair (a, b) lands at global (max(E[a], E[b]), min(E[a], E[b])).
 *   - CSR: rowptr [n_nodes + 1] int64, col [nnz] int32 ascending within a row
 *     (the diagonal is the last entry of each row), vals [nnz].
 *   - Precision.  FEM_FP64: X, c, ke and vals are double; all arithmetic FP64.
 *     FEM_MIXED: X and c are float or double (x_dtype, c_dtype); ke and vals are
 *     float; element arithmetic FP32 with FP32 accumulation, except the
 *     Jacobian determinant and inverse of elements whose distortion indicator
 *     exceeds fem_options.distortion_threshold (FP64 determinant) and the
 *     summation of entries that receive more than fem_options.valence_threshold
 *     contributions (FP64-accurate, rounded once; see fem_options.fp64_sums).
 *   - Every call is ordered on `stream` (a cudaStream_t; NULL = legacy default
 *     stream) and returns without waiting, except where stated.  Asynchronous
 *     CUDA errors surface at the next call on the mesh or at fem_sync.
 *   - Calls on one mesh handle must not overlap on the GPU: they share the
 *     mesh's library buffers (plan, staged element matrices or gradients, tile
 *     partials, host staging).  Order them on one stream, or synchronise between
 *     the streams they use (fem_build_K_host_async orders its own calls on one
 *     mesh across streams).  Different meshes are independent.
 *   - Every call returns a status; nothing throws across this boundary.  A
 *     one-line detail of the last failure on the calling thread is available
 *     from fem_last_error().
 *   - Values are deterministic: the order in which contributions are summed
 *     into each entry is fixed by the mesh's cached plan, so repeated builds of
 *     the same inputs are bitwise identical.
 */
#ifndef FEM_H
#define FEM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fem_mesh_s *fem_mesh; /* opaque, library-owned */

typedef enum {
    FEM_OK = 0,
    FEM_ERR_ARG = 1,         /* null or misaligned pointer, bad size, bad enum value */
    FEM_ERR_INDEX = 2,       /* a node id in E outside [0, n_nodes); in the bounds-check build,
                                also an out-of-range index met inside a patch kernel */
    FEM_ERR_DEGENERATE = 3,  /* a node repeated within one element (fem_mesh_create), or an
                                element matrix (build) or element gradient (fem_vjp) that is
                                not finite: zero volume, non-finite input (reported by
                                fem_sync after the call) */
    FEM_ERR_OOM = 4,         /* a device allocation failed */
    FEM_ERR_BUDGET = 5,      /* the memory budget cannot hold the smallest unit of work */
    FEM_ERR_CUDA = 6,        /* a CUDA runtime call or kernel failed */
    FEM_ERR_TIMEOUT = 7,     /* a bounded device-side wait gave up */
    FEM_ERR_STATE = 8,       /* call out of order, e.g. values before the pattern */
    FEM_ERR_UNSUPPORTED = 9  /* mesh outside the supported range (see fem_last_error) */
} fem_status;

typedef enum { FEM_TET4 = 4, FEM_HEX8 = 8 } fem_elem;
typedef enum { FEM_FP64 = 0, FEM_MIXED = 1 } fem_prec;
typedef enum { FEM_F32 = 0, FEM_F64 = 1 } fem_dtype;

typedef struct {
    size_t mem_budget_bytes;     /* cap on library-owned device memory; 0 = no cap */
    double distortion_threshold; /* mixed mode; brick: max_q detJ / min_q detJ, tet:
                                    longest edge / shortest altitude.  0 = default
                                    (brick 4, tetrahedron 10). */
    int valence_threshold;       /* mixed mode: entries with more contributions than
                                    this are summed in FP64.  Default 8. */
    int patch_entries;           /* lower-CSR entries owned by one thread block (0 = default) */
    int block_threads;           /* threads per block of the patch kernels (0 = default) */
    int blocks_per_sm;           /* resident blocks per SM for the patch kernels (0 = default) */
    int locality_order;          /* 1 = order nodes along a Morton curve of X (default); 0 = by id */
    int fp64_sums;               /* mixed mode, high-valence entries: 0 (default) = error-free
                                    FP32 pair summation (TwoSum, accurate to ~2^-48 like an
                                    FP64 sum, rounded once); 1 = FP64 adds */
    int fp64_fused;              /* FEM_FP64 builds: 0 (default) = integrate each element once
                                    into library memory, then assemble; 1 = recompute element
                                    matrices inside the assembly (no staging memory) */
    int fp64_dets;               /* mixed mode, distorted tetrahedra: 0 (default) = Jacobian
                                    determinant in double-single FP32 arithmetic (accurate to
                                    ~2^-46 of its terms, FP64-grade for the float result);
                                    1 = FP64 arithmetic */
    int wait_spins;              /* polls of one device-side wait of the patch kernels before it
                                    gives up (0 = default 2^20); a wait that gives up is reported
                                    by fem_sync as FEM_ERR_TIMEOUT */
    int debug_stall;             /* testing only: 1 = warp 0 of every block waits once for a
                                    phase that cannot complete, so that the wait gives up;
                                    2 (library built with -DFEM_DEBUG_BOUNDS only, else
                                    FEM_ERR_ARG) = one out-of-range node id is planted per
                                    block, caught by the bounds checks of that build and
                                    reported by fem_sync as FEM_ERR_INDEX */
    int operator_kind;           /* 0 (default) = stiffness matrix k_e = c int B^T B (Eq. 9);
                                    1 = mass matrix m_e = c int N^T N (the other operator the
                                    paper's construction generalises to, Section 5): same
                                    quadrature, packing, pattern and assembly;
                                    2 = linear isotropic elasticity, three DOFs per node
                                    (Algorithm 1's Mapping with DOFxn = 3): see "Elasticity"
                                    below.  fem_vjp covers all three */
    int host_direct;             /* fem_build_K_host / _async: 0 (default) = K's values are
                                    built in device staging and copied out in one transfer,
                                    unless the memory budget refuses the staging; 1 = always
                                    write them straight into vals_host (page-locked, mapped
                                    through unified addressing), for K larger than device
                                    memory or the budget */
    int vjp_fused;               /* fem_vjp: 0 (default) = each element's node gradients are
                                    computed once into library memory (n_elems * npe * 3
                                    values), then gathered into the owned nodes of every
                                    patch; 1 = recomputed in every patch whose closure holds
                                    the element (no library memory; also used when the
                                    budget refuses it or the plan is built per patch group) */
    int assembly;                /* scalar operators (stiffness, mass), fem_build_K, the host-
                                    buffer builds and batched builds: 0 (default) = node
                                    patches: each patch integrates every element that touches
                                    the rows it owns; 1 = element tiles: every element is
                                    integrated once, and a row whose elements span several
                                    tiles is summed from the tiles' partial rows, in a fixed
                                    order, by a second kernel (falls back to patches when the
                                    memory budget cannot hold the tile plan).  Elasticity,
                                    fem_vjp, fem_load_vector and fem_assemble_csr use patches,
                                    planned on their first call when tiles serve the builds */
    int tile_elems;              /* elements per tile (0 = default: 512 bricks, 2048 tetrahedra) */
    int host_chunks;             /* scalar operators, fem_build_K_host / _async without
                                    host_direct: 0 (default) = K's values are built whole in
                                    device staging and copied out in one transfer; n > 1 =
                                    the rows are split into n contiguous ranges of about
                                    n_nodes / n rows (the node order runs range by range,
                                    each along its own Morton curve, and the node patches
                                    are planned inside the ranges; fixed at
                                    fem_mesh_create), and range k + 1 is built into one of two device
                                    slots while range k's values are copied to vals_host
                                    from the other (Section 4.3's overlap of one group's
                                    transfer with the next group's integration): device
                                    memory holds 2 ranges of values, not K */
    int group_cache;             /* plans built per patch group (Eq. 10: the memory budget
                                    cannot hold every patch's closure at once): 1 (default) =
                                    each group's closure is built once and a copy kept in
                                    page-locked host memory (about 57 bytes per closure
                                    element); later calls copy the groups back to the device
                                    in turn (the next group's copy overlapping the current
                                    group's build when two fit the budget; the two device
                                    slots stay allocated between calls, within the budget)
                                    instead of building them again; 0 = build every group's closure at
                                    every call (no host memory).  If not even one group's
                                    copy fits beside the call's other buffers, the groups are
                                    built instead. */
} fem_options;

/*
 * Elasticity (operator_kind = 2).  k_e = int Be^T D Be: Be the 6 x 3npe strain-
 * displacement matrix, D the isotropic material matrix of the element's Lame
 * parameters; the same quadrature and |det J| as Eq. 9.  Degree of freedom 3g + i
 * is displacement component i of node g.  With it, for every entry point:
 *   - c is [n_elems][2] = (lambda_e, mu_e), interleaved, in c_dtype;
 *   - the matrix is the lower triangle of the 3 n_nodes x 3 n_nodes matrix:
 *     fem_pattern's nnz and fem_get_pattern's rowptr [3 n_nodes + 1] and col [nnz]
 *     are those of the DOF matrix (node row I of length L gives DOF rows 3I..3I+2
 *     of 9L - 3 entries in all, row 3I starting at 9 rowptr_node[I] - 3I);
 *   - fem_integrate_local and fem_assemble_csr use [n_elems][300|78] packed
 *     entries, p = A(A+1)/2 + B over local DOFs A = 3a + i, B <= A;
 *   - fem_build_K fuses integration and assembly in FP32 (mixed); FEM_FP64 integrates
 *     each element once into library memory (n_elems * 300|78 doubles, within the
 *     budget; fused if it refuses or fp64_fused is set) and then assembles; patches
 *     whose 3x3 blocks outgrow shared memory are accumulated in row windows;
 *   - patch_entries counts node pairs (each a 3x3 block; default 4096 for bricks,
 *     1536 for tetrahedra) and block_threads defaults to 512 for bricks;
 *   - fem_load_vector takes a body force [n_elems][3] and writes F [3 n_nodes];
 *   - fem_build_K_batched takes batches of elasticity meshes only (no mixing with
 *     scalar operators), fused in both precisions;
 *   - fem_pattern_ptrs and fem_vjp answer FEM_ERR_UNSUPPORTED; fem_mesh_create
 *     refuses 3 n_nodes >= 2^31.
 */

typedef struct {
    int64_t n_nodes, n_elems, nnz;
    int64_t n_patches;           /* thread-block work units of the numeric kernels */
    int64_t closure_elems;       /* sum over patches of the elements each one integrates */
    int64_t max_patch_entries, max_patch_cnodes, max_patch_elems;
    int32_t n_colors;            /* colours of the in-block accumulation order */
    int32_t max_row_len;
    size_t plan_bytes;           /* device bytes held by the cached pattern and plan */
    size_t budget_bytes;         /* the budget in force (0 = none) */
    int32_t n_groups;            /* patch groups the numeric build runs in under the budget */
    int32_t assembly;            /* what fem_build_K runs on: 0 = node patches, 1 = element tiles
                                    (then n_patches ... n_colors describe the tiles: n_patches =
                                    tiles, closure_elems = n_elems, max_patch_entries = the
                                    largest tile's accumulator entries, max_patch_cnodes its
                                    rows) */
    size_t live_bytes;           /* device bytes the library holds for the mesh now */
    size_t peak_bytes;           /* the most it has held at once */
    int32_t n_chunks;            /* row ranges of the host pipeline (fem_options.host_chunks;
                                    1 = none) */
    int32_t reserved0;
    int64_t tile_rows;           /* rows summed in tiles (a row in k tiles counts k times) */
    int64_t border_rows;         /* rows whose elements span several tiles */
    int64_t partial_values;      /* values of the border rows' partial sums */
} fem_info;

/* Default options (see the field comments). */
void fem_options_default(fem_options *opt);

/* Human-readable name of a status code (static storage). */
const char *fem_status_str(fem_status s);

/* Detail of the last failure on the calling thread (static thread-local storage). */
const char *fem_last_error(void);

/*
 * Create a mesh handle: validates E (Section 3's connectivity array) and caches
 * nothing else yet.  E must stay valid and unchanged until fem_mesh_destroy.
 * X (optional, may be NULL) is read once to order nodes along a space-filling
 * curve, which only changes locality; it is not retained.
 * Blocks until validation is done.  Errors: FEM_ERR_ARG (null E, sizes <= 0,
 * n_nodes >= 2^31, bad type), FEM_ERR_INDEX, FEM_ERR_DEGENERATE, FEM_ERR_OOM.
 */
fem_status fem_mesh_create(fem_mesh *out, fem_elem type, int64_t n_nodes, int64_t n_elems,
                           const int32_t *E, const void *X, fem_dtype x_dtype,
                           const fem_options *opt, void *stream);

/* Release the handle and everything it owns.  NULL is ignored. */
void fem_mesh_destroy(fem_mesh m);

/*
 * Symbolic phase (Algorithm 1's Mapping plus the structure of the sparse
 * conversion): build and cache the lower-CSR pattern of K -- every node pair
 * that shares an element, explicit zeros included -- and the per-block plan of
 * the numeric kernels.  Writes nnz to *nnz_out.  Idempotent.  Blocks (reads nnz
 * back).  Errors: FEM_ERR_OOM, FEM_ERR_BUDGET, FEM_ERR_UNSUPPORTED (a row with
 * more than 255 entries, more than 255 colours), FEM_ERR_CUDA.
 */
fem_status fem_pattern(fem_mesh m, int64_t *nnz_out, void *stream);

/* Copy the cached pattern into caller arrays rowptr [n_nodes+1], col [nnz]
 * (device).  FEM_ERR_STATE before fem_pattern. */
fem_status fem_get_pattern(fem_mesh m, int64_t *rowptr, int32_t *col, void *stream);

/* Library-owned device pointers of the cached pattern (valid until destroy). */
fem_status fem_pattern_ptrs(fem_mesh m, const int64_t **rowptr, const int32_t **col);

/*
 * Numerical integration (Algorithm 2, Eqs. 7-9): packed lower k_e of every
 * element into ke_out [n_elems][36|10] (double for FEM_FP64, float for
 * FEM_MIXED; 16-byte aligned, each row stored with vector stores).  Needs no
 * pattern.  FEM_ERR_ARG for a null or misaligned ke_out.
 */
fem_status fem_integrate_local(fem_mesh m, fem_prec p, const void *X, fem_dtype x_dtype,
                               const void *c, fem_dtype c_dtype, void *ke_out, void *stream);

/*
 * Assembly (Section 3: triplet-to-compressed conversion, Eq. 6): sum the packed
 * element matrices ke [n_elems][36|10] (16-byte aligned, read as vectors) into
 * vals [nnz] of the cached pattern.  Every entry is written (no need to clear
 * vals).  FEM_ERR_STATE before fem_pattern; FEM_ERR_ARG for a misaligned ke.
 */
fem_status fem_assemble_csr(fem_mesh m, fem_prec p, const void *ke, void *vals, void *stream);

/*
 * Integration and assembly: vals [nnz] of K for coordinates X and
 * coefficients c, with the pattern cached.  FEM_MIXED fuses both (no element
 * matrix goes through device memory).  FEM_FP64 integrates each element once
 * into library memory (n_elems * 36|10 doubles, within the budget) and then
 * assembles, unless fem_options.fp64_fused is set or the budget refuses the
 * buffer, in which case it fuses too.
 * FEM_ERR_STATE before fem_pattern.
 */
fem_status fem_build_K(fem_mesh m, fem_prec p, const void *X, fem_dtype x_dtype, const void *c,
                       fem_dtype c_dtype, void *vals, void *stream);

/*
 * fem_build_K with HOST inputs and outputs (page-locked memory gives full
 * copy bandwidth; pageable memory works but is slower): copies X and c to
 * library-owned device buffers (one staging slot, kept for the next call),
 * builds, copies vals back.  Blocks until vals is on the host.  With
 * fem_options.host_chunks the values are built and copied out row range by row
 * range, the copy of one range overlapping the build of the next, and the
 * device holds two ranges of them.  Host-resident K: when the memory budget
 * cannot hold the values (or fem_options.host_direct is set) the kernel writes
 * them straight into vals_host, which must then be page-locked
 * (FEM_ERR_BUDGET otherwise); with the patch groups of the budget this builds
 * K for meshes whose matrix exceeds device memory.
 */
fem_status fem_build_K_host(fem_mesh m, fem_prec p, const void *X_host, fem_dtype x_dtype,
                            const void *c_host, fem_dtype c_dtype, void *vals_host, void *stream);

/*
 * Asynchronous fem_build_K_host: the same copies and build, ordered on `stream`,
 * returning without waiting.  X_host, c_host and vals_host must be page-locked
 * (FEM_ERR_ARG otherwise) and stay untouched until the stream is synchronised;
 * vals_host is complete then.  Consecutive calls on one mesh use three device
 * staging slots in turn, so with streams taken in turn a call's input copy and
 * build overlap the output copies of the calls before it; the builds themselves
 * run one after the other.  Errors of the build surface at fem_sync.
 */
fem_status fem_build_K_host_async(fem_mesh m, fem_prec p, const void *X_host, fem_dtype x_dtype,
                                  const void *c_host, fem_dtype c_dtype, void *vals_host, void *stream);

/*
 * Backward pass: for L = sum over stored entries of G_ij K_ij (each packed pair
 * (a, b) of an element counted once), write dX [n_nodes][3] = dL/dX and
 * dc [n_elems] = dL/dc, recomputing J and B (nothing is kept from the forward
 * pass).  FEM_FP64: G, X, c, dX, dc double.  FEM_MIXED: G float, X and c per
 * dtype, dX and dc float; arithmetic FP32.  Every output entry is written.  For
 * the stiffness matrix (operator_kind 0) and the mass matrix (1; K = M there).
 * Elasticity (2): G has the DOF pattern (fem_pattern's), each stored DOF entry
 * counted once, and dc is [n_elems][2] = (dL/dlambda_e, dL/dmu_e); K is linear
 * in (lambda, mu), so these are the two halves of the element's L.
 */
fem_status fem_vjp(fem_mesh m, fem_prec p, const void *X, fem_dtype x_dtype, const void *c,
                   fem_dtype c_dtype, const void *G, void *dX, void *dc, void *stream);

/*
 * Global load vector of a per-element constant source (Section 1, FEM steps (ii)-(iii):
 * local load vectors f_e assembled into F): F[n] = sum over elements e that contain
 * node n of src[e] * integral over e of N_a (a = n's local index in e).  Bricks use
 * the 2x2x2 Gauss rule and |det J| of the stiffness matrix, tetrahedra |T| / 4 per
 * node.  X as for fem_build_K; src [n_elems] (src_dtype); F [n_nodes] device,
 * double (FEM_FP64) or float (FEM_MIXED: FP32 element arithmetic, FP64-accurate
 * determinants of distorted elements).  Every entry of F is written.  Uses the
 * cached plan, so FEM_ERR_STATE before fem_pattern.  The same for operator_kind 0
 * and 1; for elasticity (2) src is a body force [n_elems][3] and F [3 n_nodes],
 * F[3n + i] = sum over elements of src[e][i] * integral N_a.
 */
fem_status fem_load_vector(fem_mesh m, fem_prec p, const void *X, fem_dtype x_dtype, const void *src,
                           fem_dtype src_dtype, void *F, void *stream);

/*
 * Batched build of n meshes (each with its pattern cached) in one persistent
 * launch, replayed from a CUDA graph when the same mesh set is built again.
 * X[i], c[i], vals[i] are host arrays of n device pointers; all meshes share
 * p, x_dtype and c_dtype.  The launch takes its options (thread count, FP64
 * modes, wait settings) from meshes[0]; a device-side wait that gives up is
 * reported by fem_sync(meshes[0]).
 */
fem_status fem_build_K_batched(const fem_mesh *meshes, int n, fem_prec p, const void *const *X,
                               fem_dtype x_dtype, const void *const *c, fem_dtype c_dtype,
                               void *const *vals, void *stream);

/* Launch shape the batched build of exactly these meshes was tuned to (after a
 * first fem_build_K_batched call on them).  FEM_ERR_STATE otherwise. */
fem_status fem_batched_config(const fem_mesh *meshes, int n, fem_prec p, int *block_threads, int *blocks_per_sm,
                              int *grid);

typedef struct {
    int patch_entries;  /* chosen work unit of one thread block: elements per tile when the
                           builds run on element tiles (assembly 1), lower-CSR entries per
                           patch otherwise */
    int block_threads;  /* chosen threads per block (elements integrated per batch) */
    float ms;           /* median time of one fem_build_K from a cold L2, chosen configuration */
    int tried;          /* candidate configurations timed */
    int assembly;       /* 0 = node patches, 1 = element tiles (see fem_info.assembly) */
    int reserved[3];
} fem_tuning;

/*
 * Tuner: rebuilds the mesh's plan for each candidate work unit (elements per tile
 * when the builds run on element tiles, lower-CSR entries per patch otherwise)
 * and times fem_build_K for each candidate block size on the given inputs
 * (vals is overwritten): the median of 5 builds, each after a 256 MB scratch
 * rewrite that clears the L2 (skipped when the memory budget has no room for
 * it); the mesh keeps the fastest configuration.  Gauss-point unrolling is not a
 * candidate: the sum-factorised brick couples all 8 points.  Blocks.
 * FEM_ERR_STATE before fem_pattern.
 */
fem_status fem_autotune(fem_mesh m, fem_prec p, const void *X, fem_dtype x_dtype, const void *c, fem_dtype c_dtype,
                        void *vals, void *stream, fem_tuning *out);

/*
 * Apply a tuning chosen earlier (fem_autotune's patch_entries and block_threads,
 * for example from a cache kept by the caller per GPU, element type, precision,
 * operator and assembly): sets fem_options.tile_elems (builds on element tiles)
 * or patch_entries (on patches) and block_threads, and rebuilds the plan if the
 * pattern exists (else fem_pattern plans with them).  0 restores a default.  Blocks.
 * Errors: FEM_ERR_ARG, and those of fem_pattern.
 */
fem_status fem_set_tuning(fem_mesh m, int patch_entries, int block_threads, void *stream);

/* Wait for the mesh's work on `stream` and report any asynchronous error:
 * FEM_ERR_CUDA for a CUDA error; FEM_ERR_DEGENERATE if a build or backward pass
 * since the last fem_sync met an element matrix or element gradient that is not
 * finite (an element of zero volume, or non-finite coordinates, coefficients or
 * upstream values); FEM_ERR_TIMEOUT if a bounded device-side wait gave up.  The
 * values of that call are undefined; the context stays usable and the status
 * is cleared. */
fem_status fem_sync(fem_mesh m, void *stream);

/* Sizes and plan statistics of the mesh (after fem_pattern for the plan fields). */
fem_status fem_mesh_info(fem_mesh m, fem_info *info);

/* Number of kernel launches the library issued since the last reset (for
 * benchmarks that count the work inside a timed region). */
int64_t fem_launch_count(int reset);

/*
 * Allocation-free variant of the symbolic phase (the paper has no counterpart:
 * it exists for callers that cannot allocate device memory -- code under an
 * external memory manager that owns the device heap, plugins that may only
 * touch the buffers they are handed, or callers that must keep allocation and
 * its implicit synchronisation out of their stream).
 *
 * Computes the same lower-CSR pattern as fem_pattern (bit-identical rowptr and
 * col) for E [n_elems][npe] (device, 16-byte aligned) into rowptr [n_nodes + 1]
 * (device) and col [col_capacity] (device), and writes nnz to *nnz_out (host).
 * It needs no mesh handle and calls no cudaMalloc, cudaFree or other
 * allocating routine.  Its working memory is one static device array of
 * FEM_NOALLOC_SCRATCH_BYTES (16 MiB) inside the library, which every GPU that
 * loads the library holds until the process exits; the scratch needed is about
 * 28 * n_nodes + 4 * npe * n_elems bytes (a 64^3 brick grid, 262,144 elements,
 * fits; 65^3 does not).
 *   - Every call looks up the array's device address on the current device
 *     (cudaGetSymbolAddress); the first call on a device may load the library's
 *     device code, so make it before any stream capture.
 *   - Every call shares the array and leaves its contents behind; each call
 *     clears what must start at zero.  Calls that overlap on the GPU (other
 *     streams, other host threads) race on the array: serialise them.
 *   - Blocks the calling thread (reads sizes back).
 * Errors: FEM_ERR_ARG (bad sizes or pointers; col_capacity < nnz, in which
 * case *nnz_out still receives nnz), FEM_ERR_BUDGET (mesh larger than the
 * scratch), FEM_ERR_INDEX, FEM_ERR_DEGENERATE, FEM_ERR_UNSUPPORTED, FEM_ERR_CUDA.
 */
#define FEM_NOALLOC_SCRATCH_BYTES ((size_t)16 << 20)
fem_status fem_pattern_noalloc(fem_elem type, int64_t n_nodes, int64_t n_elems, const int32_t *E,
                               int64_t *rowptr, int32_t *col, int64_t col_capacity, int64_t *nnz_out,
                               void *stream);

#ifdef __cplusplus
}
#endif
#endif /* FEM_H */
