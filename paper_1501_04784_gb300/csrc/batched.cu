// batched.cu -- many meshes built in one persistent launch, replayed from a CUDA
// graph.
//
// A batch context is keyed by the exact list of mesh handles, the precision and
// the dtypes.  On first use it lays out a device table of per-mesh descriptors
// (plan view, input and output pointers) and the prefix sums of the meshes'
// work units -- element tiles, or patches where the meshes build on patches --
// (the work table of the persistent kernel), picks the kernel's
// threads per block and blocks per SM by timing the candidates on the real batch
// (the tuner), and captures the single launch into a CUDA graph.  Later calls
// with the same meshes only refresh the descriptor table (inputs and outputs may
// move) and replay the graph: one copy and one graph launch per build.
#include <algorithm>
#include <memory>
#include <mutex>
#include <vector>

#include "mesh.cuh"
#include "numeric.cuh"

namespace fem {

struct BatchCtx {
    std::vector<fem_mesh> meshes;
    bool mixed = true;
    fem_dtype xd = FEM_F32, cd = FEM_F32;
    int npe = 8;
    bool elastic = false;  // the elasticity operator (operator_kind 2)
    bool tiles = false;    // the meshes build on element tiles
    BatchItem *d_items = nullptr;
    TileBatchItem *d_titems = nullptr;
    std::vector<TileBatchItem> h_titems;
    int64_t *d_prefix = nullptr;
    int64_t *d_bprefix = nullptr;  // tiles: prefix sums of the border rows
    std::vector<BatchItem> h_items;
    BatchLaunch bl;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    float tuned_ms = 0.f;
    int tried = 0;
    ~BatchCtx() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (d_items) cudaFree(d_items);
        if (d_titems) cudaFree(d_titems);
        if (d_prefix) cudaFree(d_prefix);
        if (d_bprefix) cudaFree(d_bprefix);
    }
};

static std::mutex g_batch_mu;
static std::vector<std::unique_ptr<BatchCtx>> g_batch_ctx;  // most recent last
static constexpr size_t MAX_BATCH_CTX = 8;

// Drops every cached batch that contains mesh m (called on destroy).
void batch_forget(fem_mesh m) {
    std::lock_guard<std::mutex> lock(g_batch_mu);
    g_batch_ctx.erase(std::remove_if(g_batch_ctx.begin(), g_batch_ctx.end(),
                                     [m](const std::unique_ptr<BatchCtx> &c) {
                                         return std::find(c->meshes.begin(), c->meshes.end(), m) != c->meshes.end();
                                     }),
                      g_batch_ctx.end());
}

static float mesh_threshold(fem_mesh m) {
    if (m->opt.distortion_threshold > 0) return (float)m->opt.distortion_threshold;
    return m->npe == 8 ? 4.0f : 10.0f;
}

static void fill_items(BatchCtx &c, const void *const *X, const void *const *cc, void *const *vals) {
    if (c.tiles) {
        for (size_t i = 0; i < c.meshes.size(); ++i) {
            const fem_mesh m = c.meshes[i];
            c.h_titems[i] = TileBatchItem{m->tiles.view(m), X[i], cc[i], vals[i], m->tiles.partial.ptr,
                                          mesh_threshold(m), 0};
        }
        return;
    }
    for (size_t i = 0; i < c.meshes.size(); ++i) {
        c.h_items[i] = BatchItem{c.meshes[i]->plan.view(), X[i], cc[i], vals[i], mesh_threshold(c.meshes[i]), 0};
        // the elasticity operator's values: the DOF matrix (bounds of the debug build)
        if (c.elastic) c.h_items[i].pv.nnz = 9 * c.meshes[i]->nnz - 3 * c.meshes[i]->n_nodes;
    }
}

static fem_status upload_items(BatchCtx &c, cudaStream_t s) {
    // pageable source: the copy is staged before the call returns, so the host
    // table can be refilled by the next call at once
    if (c.tiles)
        FEM_CUDA(cudaMemcpyAsync(c.d_titems, c.h_titems.data(), c.h_titems.size() * sizeof(TileBatchItem),
                                 cudaMemcpyHostToDevice, s));
    else
        FEM_CUDA(cudaMemcpyAsync(c.d_items, c.h_items.data(), c.h_items.size() * sizeof(BatchItem),
                                 cudaMemcpyHostToDevice, s));
    return FEM_OK;
}

static fem_status create_ctx(BatchCtx &c, const void *const *X, const void *const *cc, void *const *vals,
                             cudaStream_t s) {
    const int n = (int)c.meshes.size();
    std::vector<int64_t> prefix(n + 1, 0), bprefix(n + 1, 0);
    PlanMax pm;
    TileMax tm;
    for (int i = 0; i < n; ++i) {
        if (c.tiles) {
            prefix[i + 1] = prefix[i] + c.meshes[i]->tiles.n_tiles;
            bprefix[i + 1] = bprefix[i] + c.meshes[i]->tiles.n_brows;
            tm.add(c.meshes[i]->tiles);
        } else {
            prefix[i + 1] = prefix[i] + c.meshes[i]->plan.n_patches;
            pm.add(c.meshes[i]->plan);
        }
    }
    if (c.tiles) FEM_CUDA(cudaMalloc(&c.d_titems, n * sizeof(TileBatchItem)));
    else FEM_CUDA(cudaMalloc(&c.d_items, n * sizeof(BatchItem)));
    FEM_CUDA(cudaMalloc(&c.d_prefix, (n + 1) * sizeof(int64_t)));
    FEM_CUDA(cudaMemcpyAsync(c.d_prefix, prefix.data(), (n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    if (c.tiles) {
        FEM_CUDA(cudaMalloc(&c.d_bprefix, (n + 1) * sizeof(int64_t)));
        FEM_CUDA(cudaMemcpyAsync(c.d_bprefix, bprefix.data(), (n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    }
    c.h_items.resize(n);
    c.h_titems.resize(n);
    fill_items(c, X, cc, vals);
    FEM_TRY(upload_items(c, s));

    // tuner: time every candidate launch shape on the real batch, keep the fastest
    const fem_options &o = c.meshes[0]->opt;
    std::vector<std::pair<int, int>> cands;
    if (c.elastic) {
        if (o.block_threads > 0) cands.push_back({elastic_threads(c.npe, o.block_threads), o.blocks_per_sm});
        else
            for (int t : {128, 256, 512})
                if (t <= elastic_threads(c.npe, 512)) cands.push_back({t, 0});
    } else if (o.block_threads > 0) {
        const int cap = c.tiles ? tile_max_threads(c.npe) : patch_max_threads(c.npe);
        cands.push_back({std::min((o.block_threads + 31) / 32 * 32, cap), o.blocks_per_sm});
    } else {
        const int cap = c.tiles ? tile_max_threads(c.npe) : patch_max_threads(c.npe);
        for (int t : {128, 256, 512})
            if (t <= cap)
                for (int b : {0, 1}) cands.push_back({t, b});
    }
    cudaEvent_t e0, e1;
    FEM_CUDA(cudaEventCreate(&e0));
    FEM_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    BatchLaunch best_bl;
    bool have = false;
    for (auto &cd : cands) {
        BatchLaunch bl;
        bl.items = c.d_items;
        bl.titems = c.d_titems;
        bl.bprefix = c.d_bprefix;
        bl.prefix = c.d_prefix;
        bl.n = n;
        bl.mode = kernel_mode(c.meshes[0]->opt);
        bl.wait = wait_ctl(c.meshes[0]);
        const fem_status cs = c.elastic ? elastic_batched_config(c.npe, c.mixed, pm, cd.first, cd.second, &bl)
                              : c.tiles ? tile_batched_config(c.npe, c.mixed, tm, cd.first, cd.second, &bl)
                                        : batched_config(c.npe, c.mixed, pm, cd.first, cd.second, &bl);
        if (cs != FEM_OK) continue;
        FEM_TRY(launch_batched_kernel(bl, s));  // warm-up
        float tot = 0.f;
        const int reps = cands.size() > 1 ? 3 : 0;
        for (int r = 0; r < reps; ++r) {
            FEM_CUDA(cudaEventRecord(e0, s));
            FEM_TRY(launch_batched_kernel(bl, s));
            FEM_CUDA(cudaEventRecord(e1, s));
            FEM_CUDA(cudaEventSynchronize(e1));
            float ms = 0.f;
            FEM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            tot += ms;
        }
        ++c.tried;
        if (!have || tot < best) {
            best = tot;
            best_bl = bl;
            have = true;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!have) {
        set_error("no launch shape of the batched kernel fits this batch");
        return FEM_ERR_UNSUPPORTED;
    }
    c.bl = best_bl;
    c.tuned_ms = best / 3.f;

    // capture the launch once
    cudaStream_t cs;
    FEM_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    fem_status st = FEM_OK;
    if (e == cudaSuccess) {
        st = launch_batched_kernel(c.bl, cs);
        e = cudaStreamEndCapture(cs, &c.graph);
    }
    cudaStreamDestroy(cs);
    if (st != FEM_OK) return st;
    if (e != cudaSuccess) return cuda_status(e, "batched graph capture");
    FEM_CUDA(cudaGraphInstantiate(&c.exec, c.graph, 0));
    return FEM_OK;
}

static BatchCtx *find_ctx(const fem_mesh *ms, int n, bool mixed, bool tiles, fem_dtype xd, fem_dtype cd) {
    for (auto it = g_batch_ctx.begin(); it != g_batch_ctx.end(); ++it) {
        BatchCtx &c = **it;
        if (c.mixed != mixed || c.tiles != tiles || c.xd != xd || c.cd != cd || (int)c.meshes.size() != n) continue;
        if (!std::equal(c.meshes.begin(), c.meshes.end(), ms)) continue;
        // move to the back (most recent)
        std::unique_ptr<BatchCtx> p = std::move(*it);
        g_batch_ctx.erase(it);
        g_batch_ctx.push_back(std::move(p));
        return g_batch_ctx.back().get();
    }
    return nullptr;
}

fem_status launch_batched(const fem_mesh *ms, int n, bool mixed, bool tiles, const void *const *X, fem_dtype xd,
                          const void *const *c, fem_dtype cd, void *const *vals, cudaStream_t s) {
    const int npe = ms[0]->npe;
    const bool elastic = ms[0]->opt.operator_kind == 2;
    for (int i = 1; i < n; ++i)
        if (ms[i]->npe != npe || (ms[i]->opt.operator_kind == 2) != elastic) {
            set_error("a batch must hold one element type and either scalar or elasticity meshes only");
            return FEM_ERR_ARG;
        }
    const fem_dtype want = mixed ? FEM_F32 : FEM_F64;
    if (xd != want || cd != want) {
        set_error("batched builds take %s X and c", mixed ? "float" : "double");
        return FEM_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(g_batch_mu);
    BatchCtx *ctx = find_ctx(ms, n, mixed, tiles, xd, cd);
    if (!ctx) {
        auto nc = std::make_unique<BatchCtx>();
        nc->meshes.assign(ms, ms + n);
        nc->mixed = mixed;
        nc->tiles = tiles;
        nc->xd = xd;
        nc->cd = cd;
        nc->npe = npe;
        nc->elastic = elastic;
        FEM_TRY(create_ctx(*nc, X, c, vals, s));
        if (g_batch_ctx.size() >= MAX_BATCH_CTX) g_batch_ctx.erase(g_batch_ctx.begin());
        g_batch_ctx.push_back(std::move(nc));
        ctx = g_batch_ctx.back().get();
    }
    fill_items(*ctx, X, c, vals);
    FEM_TRY(upload_items(*ctx, s));
    FEM_CUDA(cudaGraphLaunch(ctx->exec, s));
    count_launch();
    return FEM_OK;
}

fem_status batched_query(const fem_mesh *ms, int n, bool mixed, int *threads, int *blocks_per_sm, int *grid) {
    std::lock_guard<std::mutex> lock(g_batch_mu);
    for (auto &p : g_batch_ctx) {
        BatchCtx &c = *p;
        if (c.mixed != mixed || (int)c.meshes.size() != n || !std::equal(c.meshes.begin(), c.meshes.end(), ms))
            continue;
        if (threads) *threads = c.bl.threads;
        if (grid) *grid = c.bl.grid;
        if (blocks_per_sm) *blocks_per_sm = c.bl.grid / num_sms();
        return FEM_OK;
    }
    set_error("no batched build of these meshes has run");
    return FEM_ERR_STATE;
}

}  // namespace fem
