// primitives.cu -- status plumbing, budgeted allocation, and the device-wide
// scan and radix sort used by the symbolic phase.
#include <cstdarg>
#include <cstring>

#include "common.cuh"

namespace fem {

static thread_local char g_last_error[512] = "";
static int64_t g_launches = 0;

const char *last_error_text() { return g_last_error; }

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
}

fem_status cuda_status(cudaError_t e, const char *what) {
    set_error("%s: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? FEM_ERR_OOM : FEM_ERR_CUDA;
}

void count_launch(int n) { __atomic_add_fetch(&g_launches, n, __ATOMIC_RELAXED); }

int64_t launch_count(int reset) {
    return reset ? __atomic_exchange_n(&g_launches, 0, __ATOMIC_RELAXED)
                 : __atomic_load_n(&g_launches, __ATOMIC_RELAXED);
}

fem_status Arena::alloc(void **p, size_t bytes, const char *what) {
    *p = nullptr;
    const size_t need = bytes ? bytes : 1;
    // a kept block of at least the size and at most twice it (the smallest such)
    size_t best = pool.size();
    for (size_t i = 0; i < pool.size(); ++i)
        if (pool[i].second >= need && pool[i].second <= 2 * need &&
            (best == pool.size() || pool[i].second < pool[best].second))
            best = i;
    if (best < pool.size()) {
        *p = pool[best].first;
        const size_t sz = pool[best].second;
        pool.erase(pool.begin() + (std::ptrdiff_t)best);
        kept -= sz;
        live += sz;
        block[*p] = sz;
        if (live > peak) peak = live;
        return FEM_OK;
    }
    if (budget && live + kept + need > budget) trim();
    if (budget && live + need > budget) {
        set_error("memory budget: %s needs %zu bytes, %zu of %zu in use", what, bytes, live, budget);
        return FEM_ERR_BUDGET;
    }
    cudaError_t e = cudaMalloc(p, need);
    if (e != cudaSuccess && !pool.empty()) {
        cudaGetLastError();
        trim();
        e = cudaMalloc(p, need);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaMalloc(%zu) for %s: %s", bytes, what, cudaGetErrorString(e));
        *p = nullptr;
        return FEM_ERR_OOM;
    }
    live += need;
    block[*p] = need;
    if (live > peak) peak = live;
    return FEM_OK;
}

void Arena::release(void *p, size_t bytes) {
    (void)bytes;
    if (!p) return;
    auto it = block.find(p);
    const size_t sz = it != block.end() ? it->second : bytes;
    if (it != block.end()) block.erase(it);
    live -= sz;
    if (keep) {
        pool.emplace_back(p, sz);
        kept += sz;
        return;
    }
    cudaFree(p);
}

void Arena::trim() {
    for (auto &b : pool) cudaFree(b.first);
    pool.clear();
    kept = 0;
}

int num_sms() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

// ------------------------------------------------------------------------ scan
// Three passes: per-tile sums, one block scanning the tile sums, per-tile scan
// with the tile's offset.  Tile = 1024 threads x 4 values.
static constexpr int SCAN_THREADS = 1024;
static constexpr int SCAN_ITEMS = 4;
static constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

size_t scan_tmp_elems(int64_t n) { return (size_t)cdiv(n, SCAN_TILE) + 1; }

__device__ __forceinline__ int64_t warp_incl_scan(int64_t v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    return v;
}

// Block-wide exclusive scan of one value per thread (blockDim a multiple of 32);
// returns the block total.  All threads of the block must call it.
__device__ int64_t block_excl_scan(int64_t v, int64_t *excl) {
    __shared__ int64_t warp_sums[33];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    int64_t inc = warp_incl_scan(v);
    if (lane == 31) warp_sums[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int64_t w = lane < nw ? warp_sums[lane] : 0;
        int64_t wi = warp_incl_scan(w);
        warp_sums[lane] = wi - w;
        if (lane == 31) warp_sums[32] = wi;
    }
    __syncthreads();
    *excl = inc - v + warp_sums[warp];
    const int64_t total = warp_sums[32];
    __syncthreads();
    return total;
}

__global__ void scan_tile_sums(const int64_t *in, int64_t n, int64_t *tile_sums) {
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    int64_t s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        int64_t i = base + (int64_t)k * SCAN_THREADS + threadIdx.x;
        if (i < n) s += in[i];
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    __shared__ int64_t ws[32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        int64_t v = threadIdx.x < (SCAN_THREADS >> 5) ? ws[threadIdx.x] : 0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) tile_sums[blockIdx.x] = v;
    }
}

// One block: exclusive scan of the tile sums in place (any count), total at [nt].
__global__ void scan_tile_offsets(int64_t *tile_sums, int64_t nt) {
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < nt; base += blockDim.x) {
        int64_t i = base + threadIdx.x;
        int64_t v = i < nt ? tile_sums[i] : 0;
        int64_t ex;
        int64_t tot = block_excl_scan(v, &ex);
        if (i < nt) tile_sums[i] = ex + carry;
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) tile_sums[nt] = carry;
}

__global__ void scan_tiles(const int64_t *in, int64_t *out, int64_t n, const int64_t *tile_off,
                           bool with_total) {
    // each thread owns SCAN_ITEMS consecutive values
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    int64_t v[SCAN_ITEMS];
    int64_t s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        v[k] = (base + k < n) ? in[base + k] : 0;
        s += v[k];
    }
    int64_t ex;
    block_excl_scan(s, &ex);
    int64_t run = ex + tile_off[blockIdx.x];
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
    if (with_total && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = tile_off[gridDim.x];
}

fem_status scan_exclusive_i64(const int64_t *in, int64_t *out, int64_t n, bool with_total, int64_t *tmp,
                              cudaStream_t s) {
    if (n <= 0) {
        if (with_total) FEM_CUDA(cudaMemsetAsync(out, 0, sizeof(int64_t), s));
        return FEM_OK;
    }
    const int64_t nt = cdiv(n, SCAN_TILE);
    scan_tile_sums<<<(unsigned)nt, SCAN_THREADS, 0, s>>>(in, n, tmp);
    FEM_LAUNCHED("scan_tile_sums");
    scan_tile_offsets<<<1, SCAN_THREADS, 0, s>>>(tmp, nt);
    FEM_LAUNCHED("scan_tile_offsets");
    scan_tiles<<<(unsigned)nt, SCAN_THREADS, 0, s>>>(in, out, n, tmp, with_total);
    FEM_LAUNCHED("scan_tiles");
    return FEM_OK;
}

// ------------------------------------------------------------------ radix sort
// LSD, 8 bits per pass.  A tile is 256 threads x 8 rounds; position r*256 + t of
// a tile is handled by thread t in round r, so processing rounds in order and
// threads in order within a round visits keys in their input order, which keeps
// the sort stable.  hist is laid out digit-major: hist[d * ntiles + tile].
static constexpr int RS_THREADS = 256;
static constexpr int RS_ROUNDS = 8;
static constexpr int RS_TILE = RS_THREADS * RS_ROUNDS;
static constexpr int RS_WARPS = RS_THREADS / 32;

size_t radix_hist_elems(int64_t n) {
    const int64_t nh = 256 * cdiv(n > 0 ? n : 1, RS_TILE);
    return (size_t)nh + scan_tmp_elems(nh);  // histogram + the scan's scratch
}

__global__ void __launch_bounds__(RS_THREADS) rs_upsweep(const uint64_t *keys, int64_t n, int shift,
                                                          int64_t *hist, int64_t ntiles) {
    __shared__ unsigned cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
#pragma unroll
    for (int r = 0; r < RS_ROUNDS; ++r) {
        int64_t i = base + r * RS_THREADS + threadIdx.x;
        if (i < n) atomicAdd(&cnt[(unsigned)(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = cnt[threadIdx.x];
}

__global__ void __launch_bounds__(RS_THREADS) rs_downsweep(const uint64_t *keys_in, const uint32_t *vals_in,
                                                            uint64_t *keys_out, uint32_t *vals_out,
                                                            int64_t n, int shift, const int64_t *hist,
                                                            int64_t ntiles) {
    __shared__ int64_t base_off[256];   // global start of each digit for this tile (running)
    __shared__ unsigned wcnt[RS_WARPS][256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    base_off[threadIdx.x] = hist[(int64_t)threadIdx.x * ntiles + blockIdx.x];
    const int64_t tile0 = (int64_t)blockIdx.x * RS_TILE;
    const unsigned lt_mask = (1u << lane) - 1u;
    for (int r = 0; r < RS_ROUNDS; ++r) {
        for (int w = 0; w < RS_WARPS; ++w) wcnt[w][threadIdx.x] = 0;
        __syncthreads();
        const int64_t i = tile0 + r * RS_THREADS + threadIdx.x;
        const bool valid = i < n;
        uint64_t k = valid ? keys_in[i] : 0;
        uint32_t v = (valid && vals_in) ? vals_in[i] : 0;
        unsigned d = valid ? ((unsigned)(k >> shift) & 255u) : 256u;  // 256 = no key
        unsigned peers = __match_any_sync(0xffffffffu, d);
        unsigned rank_in_warp = __popc(peers & lt_mask);
        bool leader = (peers & lt_mask) == 0;
        if (valid && leader) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        if (valid) {
            int64_t pos = base_off[d] + rank_in_warp;
            for (int w = 0; w < warp; ++w) pos += wcnt[w][d];
            keys_out[pos] = k;
            if (vals_out) vals_out[pos] = v;
        }
        __syncthreads();
        {
            unsigned tot = 0;
            for (int w = 0; w < RS_WARPS; ++w) tot += wcnt[w][threadIdx.x];
            base_off[threadIdx.x] += tot;
        }
        __syncthreads();
    }
}

fem_status radix_sort_u64(uint64_t *keys, uint32_t *vals, int64_t n, int key_bits, uint64_t *alt_keys,
                          uint32_t *alt_vals, int64_t *hist, cudaStream_t s) {
    if (n <= 1) return FEM_OK;
    const int64_t ntiles = cdiv(n, RS_TILE);
    const int64_t nh = 256 * ntiles;
    uint64_t *kin = keys, *kout = alt_keys;
    uint32_t *vin = vals, *vout = vals ? alt_vals : nullptr;
    int passes = 0;
    for (int shift = 0; shift < key_bits; shift += 8, ++passes) {
        rs_upsweep<<<(unsigned)ntiles, RS_THREADS, 0, s>>>(kin, n, shift, hist, ntiles);
        FEM_LAUNCHED("rs_upsweep");
        // exclusive scan of the digit-major histogram in place (scratch after it)
        FEM_TRY(scan_exclusive_i64(hist, hist, nh, false, hist + nh, s));
        rs_downsweep<<<(unsigned)ntiles, RS_THREADS, 0, s>>>(kin, vin, kout, vout, n, shift, hist, ntiles);
        FEM_LAUNCHED("rs_downsweep");
        uint64_t *tk = kin; kin = kout; kout = tk;
        uint32_t *tv = vin; vin = vout; vout = tv;
    }
    if (passes & 1) {
        FEM_CUDA(cudaMemcpyAsync(keys, kin, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
        if (vals) FEM_CUDA(cudaMemcpyAsync(vals, vin, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    }
    return FEM_OK;
}

}  // namespace fem

extern "C" const char *fem_last_error(void) { return fem::last_error_text(); }
