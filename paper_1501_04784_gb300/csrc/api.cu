// api.cu -- the C ABI declared in include/fem.h: argument checks, the mesh
// handle's lifecycle, and dispatch to the symbolic and numeric kernels.
#include <algorithm>
#include <cstring>
#include <new>

#include "mesh.cuh"
#include "numeric.cuh"

namespace fem {
int64_t launch_count(int reset);
fem_status launch_load(fem_mesh m, bool mixed, const void *X, fem_dtype xd, const void *src, fem_dtype sd, void *F,
                       float thr, bool fp64_det, cudaStream_t s);
fem_status launch_vjp(fem_mesh m, bool mixed, const void *X, fem_dtype xd, const void *c, fem_dtype cd,
                      const void *G, void *dX, void *dc, cudaStream_t s);
fem_status launch_elastic_vjp(fem_mesh m, bool mixed, const void *X, fem_dtype xd, const void *c, fem_dtype cd,
                              const void *G, void *dX, void *dc, cudaStream_t s);
fem_status launch_batched(const fem_mesh *ms, int n, bool mixed, bool tiles, const void *const *X, fem_dtype xd,
                          const void *const *c, fem_dtype cd, void *const *vals, cudaStream_t s);
fem_status batched_query(const fem_mesh *ms, int n, bool mixed, int *threads, int *blocks_per_sm, int *grid);
void batch_forget(fem_mesh m);
}  // namespace fem

using namespace fem;

static cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

static bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

static size_t dsize(fem_dtype d) { return d == FEM_F64 ? 8 : 4; }

// The elasticity operator: three DOFs per node, (lambda, mu) per element.
static bool is_elastic(const fem_mesh m) { return m->opt.operator_kind == 2; }

// Entries of the global matrix the caller sees: the node pattern's, or those of
// the lower DOF matrix (a node row of L entries gives 9 L - 3).
static int64_t user_nnz(const fem_mesh m) { return is_elastic(m) ? 9 * m->nnz - 3 * m->n_nodes : m->nnz; }

static float default_threshold(const fem_mesh m) {
    if (m->opt.distortion_threshold > 0) return (float)m->opt.distortion_threshold;
    return m->npe == 8 ? 4.0f : 10.0f;
}

// Threads per block of the tile kernel (fem_options.block_threads, capped per element type).
static int tile_threads(const fem_mesh m) {
    int t = m->opt.block_threads > 0 ? m->opt.block_threads : 256;
    t = (t + 31) / 32 * 32;
    return std::min(t, tile_max_threads(m->npe));
}

// fem_build_K runs on element tiles: scalar operators with a tile plan.
static bool use_tiles(const fem_mesh m) { return !is_elastic(m) && m->opt.assembly == 1 && m->tiles.ready; }

namespace fem {
// The patch plan, built on first use when the builds run on tiles.
fem_status ensure_plan(fem_mesh m, cudaStream_t s) {
    if (m->plan_built) return FEM_OK;
    ArenaKeep keep(m->arena);
    FEM_TRY(build_plan(m, s));
    m->plan_built = true;
    return FEM_OK;
}
}  // namespace fem

static fem_status check_dtype(fem_dtype d, const char *what) {
    if (d != FEM_F32 && d != FEM_F64) {
        set_error("%s: dtype must be FEM_F32 or FEM_F64", what);
        return FEM_ERR_ARG;
    }
    return FEM_OK;
}

// Inputs of a numeric call: FP64 mode takes double X and c; mixed takes either.
static fem_status check_inputs(fem_mesh m, fem_prec p, const void *X, fem_dtype xd, const void *c, fem_dtype cd) {
    if (!m) {
        set_error("null mesh");
        return FEM_ERR_ARG;
    }
    if (p != FEM_FP64 && p != FEM_MIXED) {
        set_error("precision must be FEM_FP64 or FEM_MIXED");
        return FEM_ERR_ARG;
    }
    FEM_TRY(check_dtype(xd, "x_dtype"));
    FEM_TRY(check_dtype(cd, "c_dtype"));
    if (p == FEM_FP64 && (xd != FEM_F64 || cd != FEM_F64)) {
        set_error("FEM_FP64 needs double X and c");
        return FEM_ERR_ARG;
    }
    if (!X || !c) {
        set_error("null X or c");
        return FEM_ERR_ARG;
    }
    if (!aligned(X, dsize(xd)) || !aligned(c, dsize(cd))) {
        set_error("X or c is not aligned to its element size");
        return FEM_ERR_ARG;
    }
    return FEM_OK;
}

namespace fem {
// Wait settings of the patch kernels for mesh m.
WaitCtl wait_ctl(fem_mesh m) {
    return WaitCtl{m->status.ptr, m->opt.wait_spins > 0 ? m->opt.wait_spins : WAIT_SPINS_DEFAULT, m->opt.debug_stall};
}

// Reads and clears the mesh's device status word (after the stream is synchronised).
fem_status check_status(fem_mesh m, cudaStream_t s) {
    int h = 0;
    FEM_CUDA(cudaMemcpyAsync(&h, m->status.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
    FEM_CUDA(cudaStreamSynchronize(s));
    if (h == 0) return FEM_OK;
    FEM_CUDA(cudaMemsetAsync(m->status.ptr, 0, sizeof(int), s));
    FEM_CUDA(cudaStreamSynchronize(s));
    if (h & STATUS_BOUNDS) {
        set_error("bounds-check build: a patch kernel met an out-of-range index (caught, the access skipped); "
                  "the values of that build are undefined");
        return FEM_ERR_INDEX;
    }
    if (h & STATUS_NONFINITE) {
        set_error("an element matrix or element gradient was not finite (an element with a zero Jacobian "
                  "determinant, or non-finite coordinates, coefficients or upstream values); the values of that "
                  "call are undefined");
        return FEM_ERR_DEGENERATE;
    }
    set_error("a device-side wait of a patch kernel gave up after %d polls; the values of that build are undefined",
              m->opt.wait_spins > 0 ? m->opt.wait_spins : WAIT_SPINS_DEFAULT);
    return FEM_ERR_TIMEOUT;
}
}  // namespace fem

extern "C" {

void fem_options_default(fem_options *opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->mem_budget_bytes = 0;
    opt->distortion_threshold = 0.0;  // 0 = per element type: brick 4, tetrahedron 10
    opt->valence_threshold = 8;
    opt->patch_entries = 0;
    opt->block_threads = 0;
    opt->blocks_per_sm = 0;
    opt->locality_order = 1;
    opt->group_cache = 1;
}

const char *fem_status_str(fem_status s) {
    switch (s) {
        case FEM_OK: return "FEM_OK";
        case FEM_ERR_ARG: return "FEM_ERR_ARG";
        case FEM_ERR_INDEX: return "FEM_ERR_INDEX";
        case FEM_ERR_DEGENERATE: return "FEM_ERR_DEGENERATE";
        case FEM_ERR_OOM: return "FEM_ERR_OOM";
        case FEM_ERR_BUDGET: return "FEM_ERR_BUDGET";
        case FEM_ERR_CUDA: return "FEM_ERR_CUDA";
        case FEM_ERR_TIMEOUT: return "FEM_ERR_TIMEOUT";
        case FEM_ERR_STATE: return "FEM_ERR_STATE";
        case FEM_ERR_UNSUPPORTED: return "FEM_ERR_UNSUPPORTED";
    }
    return "FEM_ERR_UNKNOWN";
}

const char *fem_last_error(void);  // defined in primitives.cu

fem_status fem_mesh_create(fem_mesh *out, fem_elem type, int64_t n_nodes, int64_t n_elems, const int32_t *E,
                           const void *X, fem_dtype x_dtype, const fem_options *opt, void *stream) {
    if (!out) {
        set_error("null output handle");
        return FEM_ERR_ARG;
    }
    *out = nullptr;
    if (type != FEM_HEX8 && type != FEM_TET4) {
        set_error("element type must be FEM_HEX8 or FEM_TET4");
        return FEM_ERR_ARG;
    }
    if (n_nodes <= 0 || n_elems <= 0 || n_nodes >= (1ll << 31) || n_elems >= (1ll << 31)) {
        set_error("sizes must be in [1, 2^31)");
        return FEM_ERR_ARG;
    }
    if (!E || !aligned(E, 16)) {
        set_error("E must be a non-null device pointer aligned to 16 bytes");
        return FEM_ERR_ARG;
    }
    if (X) {
        FEM_TRY(check_dtype(x_dtype, "x_dtype"));
        if (!aligned(X, dsize(x_dtype))) {
            set_error("X is not aligned to its element size");
            return FEM_ERR_ARG;
        }
    }
    fem_mesh m = new (std::nothrow) fem_mesh_s();
    if (!m) {
        set_error("host allocation failed");
        return FEM_ERR_OOM;
    }
    m->type = type;
    m->npe = (int)type;
    m->np = m->npe * (m->npe + 1) / 2;
    m->n_nodes = n_nodes;
    m->n_elems = n_elems;
    m->E = E;
    if (opt) m->opt = *opt; else fem_options_default(&m->opt);
    if (m->opt.valence_threshold <= 0) m->opt.valence_threshold = 8;
    if (m->opt.operator_kind < 0 || m->opt.operator_kind > 2) {
        delete m;
        set_error("operator_kind must be 0 (stiffness), 1 (mass) or 2 (elasticity)");
        return FEM_ERR_ARG;
    }
    if (m->opt.operator_kind == 2 && 3 * n_nodes >= ((int64_t)1 << 31)) {
        delete m;
        set_error("elasticity: 3 n_nodes must stay below 2^31 (int32 DOF columns)");
        return FEM_ERR_UNSUPPORTED;
    }
#ifdef FEM_DEBUG_BOUNDS
    const int max_stall = 2;
#else
    const int max_stall = 1;
#endif
    if (m->opt.debug_stall < 0 || m->opt.debug_stall > max_stall) {
        delete m;
        set_error("debug_stall must be 0 or 1 (2 only in the bounds-check build)");
        return FEM_ERR_ARG;
    }
    m->arena.budget = m->opt.mem_budget_bytes;
    cudaStream_t s = as_stream(stream);
    fem_status st = m->status.alloc(m->arena, 1, "status word");
    {
        ArenaKeep keep(m->arena);  // ends (and frees the kept blocks) before m may be deleted
        if (st == FEM_OK) {
            cudaError_t e = cudaMemsetAsync(m->status.ptr, 0, sizeof(int), s);
            if (e != cudaSuccess) st = cuda_status(e, "fem_mesh_create");
        }
        if (st == FEM_OK) st = validate_connectivity(m, s);
        if (st == FEM_OK) st = build_locality_order(m, X, x_dtype, s);
        if (st == FEM_OK) {
            cudaError_t e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) st = cuda_status(e, "fem_mesh_create");
        }
    }
    if (st != FEM_OK) {
        delete m;
        return st;
    }
    *out = m;
    return FEM_OK;
}

void fem_mesh_destroy(fem_mesh m) {
    if (!m) return;
    cudaDeviceSynchronize();
    batch_forget(m);
    delete m;
}

fem_status fem_pattern(fem_mesh m, int64_t *nnz_out, void *stream) {
    NvtxRange nvtx_range("fem_pattern");
    if (!m) {
        set_error("null mesh");
        return FEM_ERR_ARG;
    }
    if (!m->has_pattern) {
        cudaStream_t s = as_stream(stream);
        ArenaKeep keep(m->arena);
        fem_status st = build_pattern(m, s);
        if (st == FEM_OK) {
            if (!is_elastic(m) && m->opt.assembly == 1) {
                st = build_tiles(m, s);
                if (st == FEM_ERR_BUDGET || st == FEM_ERR_UNSUPPORTED) {
                    // the budget cannot hold the tile plan (or a tile is out of
                    // range): the builds run on patches, in groups if need be
                    m->tiles.reset();
                    cudaGetLastError();
                    st = FEM_OK;
                }
            }
            if (st == FEM_OK && !use_tiles(m)) st = ensure_plan(m, s);
        }
        if (st == FEM_OK) {
            cudaError_t e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) st = cuda_status(e, "fem_pattern");
        }
        if (st != FEM_OK) {
            m->has_pattern = false;
            return st;
        }
        m->has_pattern = true;
    }
    if (nnz_out) *nnz_out = user_nnz(m);
    return FEM_OK;
}

fem_status fem_get_pattern(fem_mesh m, int64_t *rowptr, int32_t *col, void *stream) {
    if (!m) {
        set_error("null mesh");
        return FEM_ERR_ARG;
    }
    if (!m->has_pattern) {
        set_error("fem_get_pattern before fem_pattern");
        return FEM_ERR_STATE;
    }
    cudaStream_t s = as_stream(stream);
    if (is_elastic(m)) return launch_dof_pattern(m->rowptr.ptr, m->col.ptr, m->n_nodes, rowptr, col, s);
    if (rowptr)
        FEM_CUDA(cudaMemcpyAsync(rowptr, m->rowptr.ptr, (m->n_nodes + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
    if (col && m->nnz)
        FEM_CUDA(cudaMemcpyAsync(col, m->col.ptr, m->nnz * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    return FEM_OK;
}

fem_status fem_pattern_ptrs(fem_mesh m, const int64_t **rowptr, const int32_t **col) {
    if (!m) {
        set_error("null mesh");
        return FEM_ERR_ARG;
    }
    if (!m->has_pattern) {
        set_error("fem_pattern_ptrs before fem_pattern");
        return FEM_ERR_STATE;
    }
    if (is_elastic(m)) {
        set_error("elasticity: the library keeps the node pattern only; use fem_get_pattern for the DOF pattern");
        return FEM_ERR_UNSUPPORTED;
    }
    if (rowptr) *rowptr = m->rowptr.ptr;
    if (col) *col = m->col.ptr;
    return FEM_OK;
}

fem_status fem_integrate_local(fem_mesh m, fem_prec p, const void *X, fem_dtype x_dtype, const void *c,
                               fem_dtype c_dtype, void *ke_out, void *stream) {
    FEM_TRY(check_inputs(m, p, X, x_dtype, c, c_dtype));
    if (!ke_out || !aligned(ke_out, 16)) {
        set_error("ke_out must be a non-null device pointer aligned to 16 bytes");
        return FEM_ERR_ARG;
    }
    IntegrateArgs a{m->npe, p == FEM_MIXED, x_dtype, c_dtype, m->E, m->n_elems, X, c, ke_out,
                    default_threshold(m), nullptr, kernel_mode(m->opt), m->status.ptr};
    if (is_elastic(m)) return launch_elastic_integrate(a, as_stream(stream));
    return launch_integrate(a, as_stream(stream));
}

static PatchArgs patch_args(fem_mesh m, fem_prec p, bool fused) {
    PatchArgs a{};
    a.plan = &m->plan;
    a.closure = nullptr;
    a.npe = m->npe;
    a.mixed = p == FEM_MIXED;
    a.fused = fused;
    a.thr = default_threshold(m);
    a.p0 = 0;
    a.p1 = m->plan.n_patches;
    a.threads = m->opt.block_threads > 0 ? m->opt.block_threads : 256;
    if (a.threads > patch_max_threads(m->npe)) a.threads = patch_max_threads(m->npe);
    a.threads = (a.threads + 31) / 32 * 32;
    if (is_elastic(m)) a.threads = elastic_threads(m->npe, m->opt.block_threads);  // its own default and cap
    a.blocks_per_sm = m->opt.blocks_per_sm;
    a.mode = kernel_mode(m->opt);
    a.wait = wait_ctl(m);
    return a;
}

fem_status fem_assemble_csr(fem_mesh m, fem_prec p, const void *ke, void *vals, void *stream) {
    if (!m) {
        set_error("null mesh");
        return FEM_ERR_ARG;
    }
    if (!m->has_pattern) {
        set_error("fem_assemble_csr before fem_pattern");
        return FEM_ERR_STATE;
    }
    if (p != FEM_FP64 && p != FEM_MIXED) {
        set_error("precision must be FEM_FP64 or FEM_MIXED");
        return FEM_ERR_ARG;
    }
    const size_t w = p == FEM_FP64 ? 8 : 4;
    if (!ke || !vals || !aligned(ke, 16) || !aligned(vals, w)) {
        set_error("ke (16-byte aligned) and vals (aligned to its element size) must be non-null device pointers");
        return FEM_ERR_ARG;
    }
    cudaStream_t s = as_stream(stream);
    FEM_TRY(ensure_plan(m, s));
    PatchArgs a = patch_args(m, p, false);
    a.xd = FEM_F32;
    a.cd = FEM_F32;
    a.ke = ke;
    a.vals = vals;
    const bool el = is_elastic(m);
    return for_each_group(m, s, [&](const Closure &cl) {
        a.closure = &cl;
        return el ? launch_elastic_patch(a, s) : launch_patch(a, s);
    });
}

fem_status fem_build_K(fem_mesh m, fem_prec p, const void *X, fem_dtype x_dtype, const void *c, fem_dtype c_dtype,
                       void *vals, void *stream) {
    NvtxRange nvtx_range("fem_build_K");
    FEM_TRY(check_inputs(m, p, X, x_dtype, c, c_dtype));
    if (!m->has_pattern) {
        set_error("fem_build_K before fem_pattern");
        return FEM_ERR_STATE;
    }
    if (!vals || !aligned(vals, p == FEM_FP64 ? 8 : 4)) {
        set_error("vals must be a non-null aligned device pointer");
        return FEM_ERR_ARG;
    }
    cudaStream_t s = as_stream(stream);
    if (use_tiles(m)) {
        // element tiles: each element integrated once, in the build's precision
        TilePlan &T = m->tiles;
        const size_t w = p == FEM_FP64 ? sizeof(double) : sizeof(float);
        const size_t need = (size_t)std::max<int64_t>(T.partial_n, 1) * w;
        fem_status st = FEM_OK;
        if (T.partial.n < need) {
            batch_forget(m);  // cached batched launches hold the old buffer
            st = T.partial.alloc(m->arena, need, "tile partial rows");
        }
        if (st == FEM_OK) {
            TileArgs a{};
            a.plan = &T;
            a.view = T.view(m);
            a.npe = m->npe;
            a.mixed = p == FEM_MIXED;
            a.xd = x_dtype;
            a.cd = c_dtype;
            a.X = X;
            a.c = c;
            a.vals = vals;
            a.part = T.partial.ptr;
            a.thr = default_threshold(m);
            a.threads = tile_threads(m);
            a.blocks_per_sm = m->opt.blocks_per_sm;
            a.wait = wait_ctl(m);
            a.mode = kernel_mode(m->opt);
            return launch_tile(a, s);
        }
        if (st != FEM_ERR_BUDGET) return st;
        cudaGetLastError();  // no room for the partials: patches
    }
    FEM_TRY(ensure_plan(m, s));
    if (is_elastic(m)) {
        if (p == FEM_FP64 && m->opt.fp64_fused == 0) {
            // FP64 integrates each element once into library memory (300 or 78
            // doubles per element), then assembles: the FP64 pipe bounds the
            // integration, and patches whose FP64 blocks outgrow shared memory are
            // assembled in row windows, each of which would otherwise integrate its
            // closure again.  Falls back to the fused kernel if the budget refuses.
            const size_t nk = 3 * (size_t)m->npe, n = (size_t)m->n_elems * (nk * (nk + 1) / 2);
            fem_status st = m->ke64.n >= n ? FEM_OK : m->ke64.alloc(m->arena, n, "FP64 element matrices");
            if (st == FEM_OK) {
                IntegrateArgs ia{m->npe, false, x_dtype, c_dtype, m->E, m->n_elems, X, c, m->ke64.ptr,
                                 default_threshold(m), nullptr, kernel_mode(m->opt), m->status.ptr};
                FEM_TRY(launch_elastic_integrate(ia, s));
                PatchArgs a = patch_args(m, p, false);
                a.xd = FEM_F64;
                a.cd = FEM_F64;
                a.ke = m->ke64.ptr;
                a.vals = vals;
                return for_each_group(m, s, [&](const Closure &cl) {
                    a.closure = &cl;
                    return launch_elastic_patch(a, s);
                });
            }
            if (st != FEM_ERR_BUDGET) return st;
            cudaGetLastError();
        }
        PatchArgs a = patch_args(m, p, true);
        a.xd = x_dtype;
        a.cd = c_dtype;
        a.X = X;
        a.c = c;
        a.vals = vals;
        return for_each_group(m, s, [&](const Closure &cl) {
            a.closure = &cl;
            return launch_elastic_patch(a, s);
        });
    }
    if (p == FEM_FP64 && !m->plan.chunked && m->opt.fp64_fused == 0) {
        // integrate once into library memory, then assemble (falls back to the
        // fused kernel if the budget refuses the buffer)
        const size_t n = (size_t)m->n_elems * m->np;
        fem_status st = m->ke64.n >= n ? FEM_OK : m->ke64.alloc(m->arena, n, "FP64 element matrices");
        if (st == FEM_OK) {
            IntegrateArgs ia{m->npe, false, x_dtype, c_dtype, m->E, m->n_elems, X, c, m->ke64.ptr,
                             default_threshold(m), nullptr, kernel_mode(m->opt), m->status.ptr};
            FEM_TRY(launch_integrate(ia, s));
            PatchArgs a = patch_args(m, p, false);
            a.xd = FEM_F64;
            a.cd = FEM_F64;
            a.ke = m->ke64.ptr;
            a.vals = vals;
            return for_each_group(m, s, [&](const Closure &cl) {
                a.closure = &cl;
                return launch_patch(a, s);
            });
        }
        if (st != FEM_ERR_BUDGET) return st;
    }
    PatchArgs a = patch_args(m, p, true);
    a.xd = x_dtype;
    a.cd = c_dtype;
    a.X = X;
    a.c = c;
    a.vals = vals;
    return for_each_group(m, s, [&](const Closure &cl) {
        a.closure = &cl;
        return launch_patch(a, s);
    });
}

namespace fem {
// Device address of a page-locked host buffer (unified addressing), or null if
// the buffer is not page-locked.
static void *mapped(void *host) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, host) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// Host pipeline over the plan's row ranges (fem_options.host_chunks): range k is
// built into device slot k % 2 on s while the values of range k - 1 go from the
// other slot to vals_host on the mesh's copy stream (Section 4.3: one group's
// transfer overlapped with the next group's integration).  Device memory holds
// two ranges of values.  On return s is ordered after the last copy.
static fem_status chunk_pipeline(fem_mesh m, fem_prec p, const void *X, fem_dtype xd, const void *c, fem_dtype cd,
                                 void *vals_host, cudaStream_t s) {
    Plan &P = m->plan;
    const size_t w = p == FEM_FP64 ? sizeof(double) : sizeof(float);
    const size_t slot = ((size_t)P.max_chunk_vals * w + 255) / 256 * 256;
    if (!m->copy_stream) FEM_CUDA(cudaStreamCreateWithFlags(&m->copy_stream, cudaStreamNonBlocking));
    for (int j = 0; j < 2; ++j) {
        if (!m->chunk_built[j]) FEM_CUDA(cudaEventCreateWithFlags(&m->chunk_built[j], cudaEventDisableTiming));
        if (!m->slot_free[j]) FEM_CUDA(cudaEventCreateWithFlags(&m->slot_free[j], cudaEventDisableTiming));
    }
    if (m->chunk_slots.n < 2 * slot) {
        for (cudaEvent_t e : m->slot_free) FEM_CUDA(cudaEventSynchronize(e));  // no copy reads the old slots
        m->chunk_slots.free();
        fem_status st = m->chunk_slots.alloc(m->arena, 2 * slot, "host pipeline value slots");
        if (st == FEM_ERR_BUDGET)
            set_error("the memory budget cannot hold two row ranges of values (%zu bytes); raise host_chunks", 2 * slot);
        FEM_TRY(st);
    }
    // FP64 integrates every element once up front (the FP64 pipe bounds it) and
    // assembles the ranges from those matrices; falls back to the fused kernel
    // when the budget refuses them
    bool staged = false;
    if (p == FEM_FP64 && !P.chunked && m->opt.fp64_fused == 0) {
        const size_t n = (size_t)m->n_elems * m->np;
        fem_status st = m->ke64.n >= n ? FEM_OK : m->ke64.alloc(m->arena, n, "FP64 element matrices");
        if (st == FEM_OK) {
            IntegrateArgs ia{m->npe, false, xd, cd, m->E, m->n_elems, X, c, m->ke64.ptr,
                             default_threshold(m), nullptr, kernel_mode(m->opt), m->status.ptr};
            FEM_TRY(launch_integrate(ia, s));
            staged = true;
        } else if (st != FEM_ERR_BUDGET) {
            return st;
        }
    }
    PatchArgs a = patch_args(m, p, !staged);
    if (staged) {
        a.xd = a.cd = FEM_F64;
        a.ke = m->ke64.ptr;
    } else {
        a.xd = xd;
        a.cd = cd;
        a.X = X;
        a.c = c;
    }
    unsigned char *host = static_cast<unsigned char *>(vals_host);
    for (int k = 0; k < P.n_chunks(); ++k) {
        const int j = k & 1;
        const int64_t v0 = P.chunk_val[k], nv = P.chunk_val[k + 1] - v0;
        if (nv == 0) continue;
        unsigned char *dst = m->chunk_slots.ptr + j * slot;
        FEM_CUDA(cudaStreamWaitEvent(s, m->slot_free[j], 0));  // the slot's previous range has left
        a.vals = dst;
        a.val_off = v0;
        a.p0 = P.chunk_patch[k];
        a.p1 = P.chunk_patch[k + 1];
        FEM_TRY(for_each_group_in(m, a.p0, a.p1, s, [&](const Closure &cl) {
            a.closure = &cl;
            return launch_patch(a, s);
        }));
        FEM_CUDA(cudaEventRecord(m->chunk_built[j], s));
        FEM_CUDA(cudaStreamWaitEvent(m->copy_stream, m->chunk_built[j], 0));
        FEM_CUDA(cudaMemcpyAsync(host + v0 * w, dst, nv * w, cudaMemcpyDeviceToHost, m->copy_stream));
        FEM_CUDA(cudaEventRecord(m->slot_free[j], m->copy_stream));
    }
    for (cudaEvent_t e : m->slot_free) FEM_CUDA(cudaStreamWaitEvent(s, e, 0));
    return FEM_OK;
}

// Copy in, build, copy out, ordered on s through one of the mesh's staging
// slots (see fem_mesh_s::host_stage); returns without waiting.
static fem_status host_build(fem_mesh m, fem_prec p, const void *X_host, fem_dtype x_dtype, const void *c_host,
                             fem_dtype c_dtype, void *vals_host, cudaStream_t s, const char *who, bool rotate) {
    NvtxRange nvtx_range(who);
    FEM_TRY(check_inputs(m, p, X_host, x_dtype, c_host, c_dtype));
    if (!m->has_pattern) {
        set_error("%s before fem_pattern", who);
        return FEM_ERR_STATE;
    }
    if (!vals_host) {
        set_error("null vals");
        return FEM_ERR_ARG;
    }
    const size_t xb = (size_t)m->n_nodes * 3 * dsize(x_dtype);
    const size_t cb = (size_t)m->n_elems * (is_elastic(m) ? 2 : 1) * dsize(c_dtype);
    const size_t vb = (size_t)user_nnz(m) * (p == FEM_FP64 ? 8 : 4);
    const size_t xo = 0, co = (xb + 255) / 256 * 256, vo = co + (cb + 255) / 256 * 256;
    // Values in device staging and one copy out; or (host_direct, or when the
    // budget refuses the staging) written by the kernel straight into vals_host
    // through its device mapping.
    // Or (host_chunks) built and copied out row range by row range.
    void *direct = nullptr;
    // the asynchronous entry takes the slots in turn; the blocking one always
    // takes slot 0 (it is done with it on return), so it holds one slot
    const int k = rotate ? m->stage_next : 0;
    bool pipe = m->opt.host_chunks > 1 && !m->opt.host_direct && !is_elastic(m);
    if (pipe) {
        FEM_TRY(ensure_plan(m, s));
        pipe = m->plan.n_chunks() > 1;
    }
    const bool stage_fits = pipe || m->host_stage[k].n >= vo + vb || !m->arena.budget ||
                            m->arena.live - m->host_stage[k].n + vo + vb <= m->arena.budget;
    if (m->opt.host_direct || !stage_fits) {
        direct = mapped(vals_host);
        if (!direct) {
            set_error("%s: %s; page-lock vals_host to have the values written straight into it", who,
                      m->opt.host_direct ? "host_direct is set" : "the memory budget cannot stage the values");
            return m->opt.host_direct ? FEM_ERR_ARG : FEM_ERR_BUDGET;
        }
    }
    const size_t total = (direct || pipe) ? vo : vo + vb;
    for (cudaEvent_t &e : m->stage_free)
        if (!e) FEM_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    if (!m->built) FEM_CUDA(cudaEventCreateWithFlags(&m->built, cudaEventDisableTiming));
    if (m->host_stage[k].n < total) {
        FEM_CUDA(cudaEventSynchronize(m->stage_free[k]));  // the slot's last output copy is done
        m->host_stage[k].free();
        FEM_TRY(m->host_stage[k].alloc(m->arena, total, "host staging"));
    }
    if (rotate) m->stage_next = (k + 1) % fem_mesh_s::HOST_STAGES;
    unsigned char *base = m->host_stage[k].ptr;
    FEM_CUDA(cudaStreamWaitEvent(s, m->stage_free[k], 0));
    FEM_CUDA(cudaMemcpyAsync(base + xo, X_host, xb, cudaMemcpyHostToDevice, s));
    FEM_CUDA(cudaMemcpyAsync(base + co, c_host, cb, cudaMemcpyHostToDevice, s));
    FEM_CUDA(cudaStreamWaitEvent(s, m->built, 0));
    if (pipe)
        FEM_TRY(chunk_pipeline(m, p, base + xo, x_dtype, base + co, c_dtype, vals_host, s));
    else
        FEM_TRY(fem_build_K(m, p, base + xo, x_dtype, base + co, c_dtype, direct ? direct : base + vo, s));
    FEM_CUDA(cudaEventRecord(m->built, s));
    if (!direct && !pipe) FEM_CUDA(cudaMemcpyAsync(vals_host, base + vo, vb, cudaMemcpyDeviceToHost, s));
    FEM_CUDA(cudaEventRecord(m->stage_free[k], s));
    return FEM_OK;
}

static bool pinned(const void *p) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}
}  // namespace fem

fem_status fem_build_K_host(fem_mesh m, fem_prec p, const void *X_host, fem_dtype x_dtype, const void *c_host,
                            fem_dtype c_dtype, void *vals_host, void *stream) {
    cudaStream_t s = as_stream(stream);
    FEM_TRY(host_build(m, p, X_host, x_dtype, c_host, c_dtype, vals_host, s, "fem_build_K_host", false));
    FEM_CUDA(cudaStreamSynchronize(s));
    return check_status(m, s);
}

fem_status fem_build_K_host_async(fem_mesh m, fem_prec p, const void *X_host, fem_dtype x_dtype, const void *c_host,
                                  fem_dtype c_dtype, void *vals_host, void *stream) {
    if (!pinned(X_host) || !pinned(c_host) || !pinned(vals_host)) {
        set_error("fem_build_K_host_async needs page-locked host buffers (cudaHostAlloc or cudaHostRegister)");
        return FEM_ERR_ARG;
    }
    return host_build(m, p, X_host, x_dtype, c_host, c_dtype, vals_host, as_stream(stream), "fem_build_K_host_async",
                      true);
}

fem_status fem_vjp(fem_mesh m, fem_prec p, const void *X, fem_dtype x_dtype, const void *c, fem_dtype c_dtype,
                   const void *G, void *dX, void *dc, void *stream) {
    NvtxRange nvtx_range("fem_vjp");
    FEM_TRY(check_inputs(m, p, X, x_dtype, c, c_dtype));
    if (!m->has_pattern) {
        set_error("fem_vjp before fem_pattern");
        return FEM_ERR_STATE;
    }
    const size_t w = p == FEM_FP64 ? 8 : 4;
    if (!G || !dX || !dc || !aligned(G, w) || !aligned(dX, w) || !aligned(dc, w)) {
        set_error("G, dX and dc must be non-null aligned device pointers");
        return FEM_ERR_ARG;
    }
    FEM_TRY(ensure_plan(m, as_stream(stream)));
    FEM_TRY(ensure_positions(m, as_stream(stream)));
    if (is_elastic(m))
        return launch_elastic_vjp(m, p == FEM_MIXED, X, x_dtype, c, c_dtype, G, dX, dc, as_stream(stream));
    return launch_vjp(m, p == FEM_MIXED, X, x_dtype, c, c_dtype, G, dX, dc, as_stream(stream));
}

fem_status fem_load_vector(fem_mesh m, fem_prec p, const void *X, fem_dtype x_dtype, const void *src,
                           fem_dtype src_dtype, void *F, void *stream) {
    NvtxRange nvtx_range("fem_load_vector");
    FEM_TRY(check_inputs(m, p, X, x_dtype, src, src_dtype));
    if (!m->has_pattern) {
        set_error("fem_load_vector before fem_pattern");
        return FEM_ERR_STATE;
    }
    if (!F || !aligned(F, p == FEM_FP64 ? 8 : 4)) {
        set_error("F must be a non-null aligned device pointer");
        return FEM_ERR_ARG;
    }
    FEM_TRY(ensure_plan(m, as_stream(stream)));
    return launch_load(m, p == FEM_MIXED, X, x_dtype, src, src_dtype, F, default_threshold(m), m->opt.fp64_dets != 0,
                       as_stream(stream));
}

fem_status fem_build_K_batched(const fem_mesh *meshes, int n, fem_prec p, const void *const *X, fem_dtype x_dtype,
                               const void *const *c, fem_dtype c_dtype, void *const *vals, void *stream) {
    NvtxRange nvtx_range("fem_build_K_batched");
    if (!meshes || n < 0 || (n > 0 && (!X || !c || !vals))) {
        set_error("bad batch arguments");
        return FEM_ERR_ARG;
    }
    for (int i = 0; i < n; ++i) {
        FEM_TRY(check_inputs(meshes[i], p, X[i], x_dtype, c[i], c_dtype));
        if (!meshes[i]->has_pattern) {
            set_error("mesh %d of the batch has no pattern", i);
            return FEM_ERR_STATE;
        }
        if (!vals[i]) {
            set_error("null vals for mesh %d", i);
            return FEM_ERR_ARG;
        }
    }
    if (n == 0) return FEM_OK;
    cudaStream_t s = as_stream(stream);
    // element tiles when every mesh of the batch builds on them (each mesh's
    // partials buffer sized for the precision first), else patches
    bool tiles = true;
    for (int i = 0; i < n; ++i) tiles = tiles && use_tiles(meshes[i]);
    if (tiles) {
        const size_t w = p == FEM_FP64 ? sizeof(double) : sizeof(float);
        for (int i = 0; i < n; ++i) {
            TilePlan &T = meshes[i]->tiles;
            const size_t need = (size_t)std::max<int64_t>(T.partial_n, 1) * w;
            if (T.partial.n < need) {
                batch_forget(meshes[i]);  // cached launches hold the old buffer
                FEM_TRY(T.partial.alloc(meshes[i]->arena, need, "tile partial rows"));
            }
        }
    } else {
        for (int i = 0; i < n; ++i) FEM_TRY(ensure_plan(meshes[i], s));
        for (int i = 0; i < n; ++i)
            if (meshes[i]->plan.chunked) {
                set_error("mesh %d of the batch is planned in groups under its memory budget", i);
                return FEM_ERR_UNSUPPORTED;
            }
    }
    return launch_batched(meshes, n, p == FEM_MIXED, tiles, X, x_dtype, c, c_dtype, vals, s);
}

fem_status fem_batched_config(const fem_mesh *meshes, int n, fem_prec p, int *block_threads, int *blocks_per_sm,
                              int *grid) {
    if (!meshes || n <= 0) {
        set_error("bad batch arguments");
        return FEM_ERR_ARG;
    }
    for (int i = 0; i < n; ++i)
        if (!meshes[i] || !meshes[i]->has_pattern) {
            set_error("mesh %d of the batch has no pattern", i);
            return FEM_ERR_STATE;
        }
    return batched_query(meshes, n, p == FEM_MIXED, block_threads, blocks_per_sm, grid);
}

// Tuner of the assembly tile and of the threads per block: the plan is rebuilt
// for each candidate size (elements per tile when the builds run on tiles,
// lower-CSR entries per patch otherwise) and every candidate is timed on the
// caller's inputs; the mesh keeps the fastest.
fem_status fem_autotune(fem_mesh m, fem_prec p, const void *X, fem_dtype x_dtype, const void *c, fem_dtype c_dtype,
                        void *vals, void *stream, fem_tuning *out) {
    NvtxRange nvtx_range("fem_autotune");
    FEM_TRY(check_inputs(m, p, X, x_dtype, c, c_dtype));
    if (!m->has_pattern) {
        set_error("fem_autotune before fem_pattern");
        return FEM_ERR_STATE;
    }
    if (!vals) {
        set_error("null vals");
        return FEM_ERR_ARG;
    }
    cudaStream_t s = as_stream(stream);
    const bool tiles = use_tiles(m);
    const fem_options keep = m->opt;
    static const int entries_scalar[] = {4096, 6144, 8192, 12288, 16384};
    static const int entries_elastic[] = {1536, 2048, 3072, 4096, 5120};
    static const int tiles_brick[] = {256, 384, 512, 768, 1024};
    static const int tiles_tet[] = {512, 1024, 1536, 2048, 2048};
    static const int threads_scalar[] = {128, 256, 512};
    static const int threads_elastic[] = {256, 512, 512};
    const int *sizes = tiles ? (m->npe == 8 ? tiles_brick : tiles_tet)
                             : (is_elastic(m) ? entries_elastic : entries_scalar);
    const int *threads = is_elastic(m) ? threads_elastic : threads_scalar;
    auto replan = [&](cudaStream_t st) -> fem_status {
        if (tiles) return build_tiles(m, st);
        fem_status r = build_plan(m, st);
        if (r == FEM_OK) m->plan_built = true;
        return r;
    };
    float best = 1e30f;
    int best_e = 0, best_t = 0, tried = 0;
    cudaEvent_t e0, e1;
    FEM_CUDA(cudaEventCreate(&e0));
    FEM_CUDA(cudaEventCreate(&e1));
    // Candidates are timed from a cold L2, as a build that follows other work
    // sees it: a 256 MB scratch (twice the L2) is rewritten before every timed
    // build, when the memory budget has room for it.  Median of 5 builds.
    DevBuf<unsigned char> flush;
    const size_t flush_bytes = (size_t)256 << 20;
    if (flush.alloc(m->arena, flush_bytes, "tuner L2 flush") != FEM_OK) cudaGetLastError();
    for (int ie = 0; ie < 5; ++ie) {
        const int pe = sizes[ie];
        if (ie > 0 && pe == sizes[ie - 1]) continue;
        for (int it = 0; it < 3; ++it) {
            const int t = threads[it];
            if (it > 0 && t == threads[it - 1]) continue;
            if (tiles && t > tile_max_threads(m->npe)) continue;
            m->opt = keep;
            if (tiles) m->opt.tile_elems = pe; else m->opt.patch_entries = pe;
            m->opt.block_threads = t;
            m->opt.blocks_per_sm = 0;
            // the plan does not depend on the block size
            if (it == 0 && replan(s) != FEM_OK) {
                cudaGetLastError();
                if (tiles) continue;
                break;
            }
            if (fem_build_K(m, p, X, x_dtype, c, c_dtype, vals, stream) != FEM_OK) continue;
            float rep[5];
            for (int r = 0; r < 5; ++r) {
                if (flush.ptr) FEM_CUDA(cudaMemsetAsync(flush.ptr, r, flush_bytes, s));
                FEM_CUDA(cudaEventRecord(e0, s));
                FEM_TRY(fem_build_K(m, p, X, x_dtype, c, c_dtype, vals, stream));
                FEM_CUDA(cudaEventRecord(e1, s));
                FEM_CUDA(cudaEventSynchronize(e1));
                FEM_CUDA(cudaEventElapsedTime(&rep[r], e0, e1));
            }
            std::sort(rep, rep + 5);
            const float tot = rep[2];
            ++tried;
            if (tot < best) {
                best = tot;
                best_e = pe;
                best_t = t;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    m->opt = keep;
    if (!tried) {
        FEM_TRY(replan(s));
        set_error("no candidate configuration ran");
        return FEM_ERR_UNSUPPORTED;
    }
    if (tiles) m->opt.tile_elems = best_e; else m->opt.patch_entries = best_e;
    m->opt.block_threads = best_t;
    FEM_TRY(replan(s));
    if (out) {
        std::memset(out, 0, sizeof(*out));
        out->patch_entries = best_e;
        out->block_threads = best_t;
        out->ms = best;
        out->tried = tried;
        out->assembly = tiles ? 1 : 0;
    }
    return FEM_OK;
}

// A tuning chosen before (by fem_autotune, possibly in another process): the plan
// is rebuilt for it without timing anything.
fem_status fem_set_tuning(fem_mesh m, int patch_entries, int block_threads, void *stream) {
    if (!m || patch_entries < 0 || block_threads < 0 || block_threads > 1024) {
        set_error("bad tuning arguments");
        return FEM_ERR_ARG;
    }
    const bool tiles = use_tiles(m) || (!m->has_pattern && !is_elastic(m) && m->opt.assembly == 1);
    if (tiles) m->opt.tile_elems = patch_entries; else m->opt.patch_entries = patch_entries;
    m->opt.block_threads = block_threads;
    m->opt.blocks_per_sm = 0;
    if (!m->has_pattern) return FEM_OK;  // fem_pattern will plan with these settings
    cudaStream_t s = as_stream(stream);
    ArenaKeep keep(m->arena);
    fem_status st = FEM_OK;
    if (use_tiles(m)) {
        st = build_tiles(m, s);
    } else if (m->plan_built) {
        st = build_plan(m, s);
    }
    if (st == FEM_OK) {
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_status(e, "fem_set_tuning");
    }
    return st;
}

fem_status fem_sync(fem_mesh m, void *stream) {
    cudaError_t e = cudaStreamSynchronize(as_stream(stream));
    if (e != cudaSuccess) return cuda_status(e, "fem_sync");
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_status(e, "fem_sync");
    return m ? check_status(m, as_stream(stream)) : FEM_OK;
}

fem_status fem_mesh_info(fem_mesh m, fem_info *info) {
    if (!m || !info) {
        set_error("null argument");
        return FEM_ERR_ARG;
    }
    std::memset(info, 0, sizeof(*info));
    info->n_nodes = m->n_nodes;
    info->n_elems = m->n_elems;
    info->nnz = user_nnz(m);
    if (use_tiles(m)) {
        const TilePlan &T = m->tiles;
        info->assembly = 1;
        info->n_patches = T.n_tiles;
        info->closure_elems = m->n_elems;
        info->max_patch_entries = T.max_acc;
        info->max_patch_cnodes = T.max_tnodes;
        info->max_patch_elems = T.max_elems;
        info->n_colors = T.n_colors;
        info->tile_rows = T.n_tnodes;
        info->border_rows = T.n_brows;
        info->partial_values = T.partial_n;
    } else {
        info->assembly = 0;
        info->n_patches = m->plan.n_patches;
        info->closure_elems = m->plan.total_celems;
        info->max_patch_entries = m->plan.max_acc;
        info->max_patch_cnodes = m->plan.max_cnodes;
        info->max_patch_elems = m->plan.max_celems;
        info->n_colors = m->plan.n_colors;
    }
    info->max_row_len = m->max_row_len;
    info->plan_bytes = m->plan.bytes() + m->tiles.bytes() + m->rowptr.bytes() + m->col.bytes() + m->inc_ptr.bytes() +
                       m->inc_elem.bytes();
    info->budget_bytes = m->arena.budget;
    info->n_groups = m->n_groups;
    info->n_chunks = m->plan_built ? m->plan.n_chunks() : 1;
    info->live_bytes = m->arena.live;
    info->peak_bytes = m->arena.peak;
    return FEM_OK;
}

int64_t fem_launch_count(int reset) { return launch_count(reset); }

}  // extern "C"
