// common.cuh -- internals shared by the libfem translation units: status
// plumbing, device-memory accounting under the mesh's budget, launch counting,
// and the device-wide primitives of the symbolic phase (exclusive scan, stable
// LSD radix sort).  Nothing here is part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <cstdio>
#include <string>
#include <unordered_map>
#include <utility>
#include <vector>

#include "fem.h"  // include/ is on the include path

namespace fem {

// ------------------------------------------------------------------ status plumbing
void set_error(const char *fmt, ...);
const char *last_error_text();
fem_status cuda_status(cudaError_t e, const char *what);
void count_launch(int n = 1);

#define FEM_TRY(expr)                                  \
    do {                                               \
        fem_status _s = (expr);                        \
        if (_s != FEM_OK) return _s;                   \
    } while (0)

#define FEM_CUDA(expr)                                                  \
    do {                                                                \
        cudaError_t _e = (expr);                                        \
        if (_e != cudaSuccess) return ::fem::cuda_status(_e, #expr);    \
    } while (0)

// A named NVTX range over a scope (API calls and symbolic phases appear on a
// profiler's timeline; without an attached tool a push is a no-op).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

#define FEM_LAUNCHED(what)                                                     \
    do {                                                                       \
        ::fem::count_launch();                                                 \
        cudaError_t _e = cudaGetLastError();                                   \
        if (_e != cudaSuccess) return ::fem::cuda_status(_e, what);            \
    } while (0)

// ------------------------------------------------------- budgeted device memory
// Every device allocation of a mesh goes through its Arena, which refuses to go
// beyond the mesh's budget (FEM_ERR_BUDGET) and frees everything on destroy.
//
// While a symbolic phase runs (one stream, synchronised before it returns),
// released blocks are kept for reuse instead of freed: cudaFree waits for the
// whole device, and the phase allocates and drops dozens of temporaries.  The
// kept blocks count against the budget (they are freed first when an allocation
// would exceed it) and are all freed when the phase ends.
struct Arena {
    size_t budget = 0;      // 0 = unlimited
    size_t live = 0, peak = 0;  // bytes in use by buffers; most ever in use (kept blocks are
                                // returned before an allocation would exceed the budget)
    size_t kept = 0;        // bytes of released blocks kept for reuse
    bool keep = false;      // keep released blocks (inside a symbolic phase)
    std::vector<std::pair<void *, size_t>> pool;        // kept blocks
    std::unordered_map<void *, size_t> block;           // size of every block handed out
    fem_status alloc(void **p, size_t bytes, const char *what);
    void release(void *p, size_t bytes);
    void trim();  // frees the kept blocks
    ~Arena() { trim(); }
};

// Keeps released blocks for the lifetime of the guard (a symbolic phase).
struct ArenaKeep {
    Arena &a;
    bool was;
    explicit ArenaKeep(Arena &ar) : a(ar), was(ar.keep) { a.keep = true; }
    ~ArenaKeep() {
        a.keep = was;
        if (!was) a.trim();
    }
};

template <typename T>
struct DevBuf {
    T *ptr = nullptr;
    size_t n = 0;
    Arena *arena = nullptr;
    fem_status alloc(Arena &a, size_t count, const char *what) {
        free();
        arena = &a;
        n = count;
        void *p = nullptr;
        fem_status s = a.alloc(&p, (count ? count : 1) * sizeof(T), what);
        ptr = static_cast<T *>(p);
        if (s != FEM_OK) n = 0;
        return s;
    }
    void free() {
        if (ptr && arena) arena->release(ptr, (n ? n : 1) * sizeof(T));
        ptr = nullptr;
        n = 0;
    }
    size_t bytes() const { return (n ? n : 1) * sizeof(T) * (ptr != nullptr); }
    ~DevBuf() { free(); }
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
};

// ------------------------------------------------------------ device primitives
// Exclusive prefix sum of n int64 values (in may equal out).  Writes the total to
// out[n] when with_total.  Uses `tmp` (>= scan_tmp_elems(n) int64) as scratch.
size_t scan_tmp_elems(int64_t n);
fem_status scan_exclusive_i64(const int64_t *in, int64_t *out, int64_t n, bool with_total,
                              int64_t *tmp, cudaStream_t s);

// Stable LSD radix sort of 64-bit keys on their low `key_bits` bits, with an
// optional 32-bit payload.  keys/vals are sorted in place; alt_keys/alt_vals
// are scratch of the same size; hist is scratch of radix_hist_elems(n) int64.
size_t radix_hist_elems(int64_t n);
fem_status radix_sort_u64(uint64_t *keys, uint32_t *vals, int64_t n, int key_bits, uint64_t *alt_keys,
                          uint32_t *alt_vals, int64_t *hist, cudaStream_t s);

// Ceil-div helper for grid sizes.
inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

int num_sms();

}  // namespace fem
