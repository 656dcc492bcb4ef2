// noalloc.cu -- the lower-CSR pattern of K without any device allocation.
//
// Some callers cannot allocate device memory at the time they need a matrix
// structure: code running under an external memory manager that owns the whole
// device heap, plugins that may only touch buffers handed to them, or callers
// that must not introduce allocation (and its implicit synchronisation) into
// their stream.  fem_pattern_noalloc serves them: the caller passes E and the
// output arrays, and the working memory of the symbolic phase (node degrees,
// node -> element incidence, row counts, scan partials) lives in one
// fixed-size array of device memory that is part of the library image.
#include "mesh.cuh"

namespace fem {
fem_status pattern_steps_validate(const int32_t *E, int64_t nel, int npe, int64_t N, unsigned long long *flags,
                                  cudaStream_t s);
fem_status pattern_steps_incidence(const int32_t *E, int64_t nel, int npe, int64_t N, int64_t *deg, int64_t *inc_ptr,
                                   unsigned int *cursor, int32_t *inc_elem, int64_t *scan_tmp,
                                   unsigned long long *mx, cudaStream_t s);
fem_status pattern_steps_rows(const int32_t *E, int npe, int64_t N, const int64_t *inc_ptr, const int32_t *inc_elem,
                              int cap, int64_t *cnt, const int64_t *rowptr, int32_t *col, cudaStream_t s);

// 16 MiB of scratch, held by every GPU that loads the library until the process
// exits.  In host code `g_pattern_scratch` is only a stand-in for the symbol:
// its device address comes from cudaGetSymbolAddress, with the device current.
static constexpr size_t NOALLOC_SCRATCH_BYTES = FEM_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_pattern_scratch[NOALLOC_SCRATCH_BYTES];

// Device address of the scratch array on the current device, looked up on every
// call (it allocates nothing and costs little): an address kept from an earlier
// call would dangle after a reset of the device's primary context, which loads
// the library's device code again.
static fem_status scratch_address(unsigned char **out) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_pattern_scratch);
    if (e != cudaSuccess) return cuda_status(e, "cudaGetSymbolAddress(pattern scratch)");
    *out = static_cast<unsigned char *>(p);
    return FEM_OK;
}

static size_t a256(size_t v) { return (v + 255) & ~(size_t)255; }

struct NoallocLayout {
    size_t flags, mx, deg, inc_ptr, cnt, scan_tmp, cursor, inc_elem, total;
};

static NoallocLayout layout_for(int64_t N, int64_t nel, int npe) {
    NoallocLayout L{};
    size_t o = 0;
    L.flags = o;    o = a256(o + 2 * sizeof(unsigned long long));
    L.mx = o;       o = a256(o + sizeof(unsigned long long));
    L.deg = o;      o = a256(o + (size_t)(N + 1) * sizeof(int64_t));
    L.inc_ptr = o;  o = a256(o + (size_t)(N + 1) * sizeof(int64_t));
    L.cnt = o;      o = a256(o + (size_t)(N + 1) * sizeof(int64_t));
    L.scan_tmp = o; o = a256(o + scan_tmp_elems(N + 1) * sizeof(int64_t));
    L.cursor = o;   o = a256(o + (size_t)N * sizeof(unsigned int));
    L.inc_elem = o; o = a256(o + (size_t)nel * npe * sizeof(int32_t));
    L.total = o;
    return L;
}

}  // namespace fem

using namespace fem;

extern "C" fem_status fem_pattern_noalloc(fem_elem type, int64_t n_nodes, int64_t n_elems, const int32_t *E,
                                          int64_t *rowptr, int32_t *col, int64_t col_capacity, int64_t *nnz_out,
                                          void *stream) {
    if (type != FEM_HEX8 && type != FEM_TET4) {
        set_error("element type must be FEM_HEX8 or FEM_TET4");
        return FEM_ERR_ARG;
    }
    if (n_nodes <= 0 || n_elems <= 0 || n_nodes >= (1ll << 31) || n_elems >= (1ll << 31)) {
        set_error("sizes must be in [1, 2^31)");
        return FEM_ERR_ARG;
    }
    if (!E || (reinterpret_cast<uintptr_t>(E) & 15) || !rowptr || (reinterpret_cast<uintptr_t>(rowptr) & 7) ||
        !nnz_out || col_capacity < 0 || (col_capacity > 0 && !col)) {
        set_error("E (16-byte aligned), rowptr (8-byte aligned) and nnz_out must be non-null");
        return FEM_ERR_ARG;
    }
    const int npe = (int)type;
    const NoallocLayout L = layout_for(n_nodes, n_elems, npe);
    if (L.total > NOALLOC_SCRATCH_BYTES) {
        set_error("mesh needs %zu bytes of pattern scratch; the allocation-free entry point has %zu", L.total,
                  NOALLOC_SCRATCH_BYTES);
        return FEM_ERR_BUDGET;
    }
    unsigned char *base = nullptr;
    FEM_TRY(scratch_address(&base));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    auto *flags = reinterpret_cast<unsigned long long *>(base + L.flags);
    auto *mx = reinterpret_cast<unsigned long long *>(base + L.mx);
    auto *deg = reinterpret_cast<int64_t *>(base + L.deg);
    auto *inc_ptr = reinterpret_cast<int64_t *>(base + L.inc_ptr);
    auto *cnt = reinterpret_cast<int64_t *>(base + L.cnt);
    auto *scan_tmp = reinterpret_cast<int64_t *>(base + L.scan_tmp);
    auto *cursor = reinterpret_cast<unsigned int *>(base + L.cursor);
    auto *inc_elem = reinterpret_cast<int32_t *>(base + L.inc_elem);

    // validation (every flag and counter that must start at zero is cleared here)
    FEM_TRY(pattern_steps_validate(E, n_elems, npe, n_nodes, flags, s));
    unsigned long long h[2];
    FEM_CUDA(cudaMemcpyAsync(h, flags, sizeof(h), cudaMemcpyDeviceToHost, s));
    FEM_CUDA(cudaStreamSynchronize(s));
    if (h[0] != ~0ull) {
        set_error("element %llu has a node id outside [0, %lld)", h[0], (long long)n_nodes);
        return FEM_ERR_INDEX;
    }
    if (h[1] != ~0ull) {
        set_error("element %llu repeats a node", h[1]);
        return FEM_ERR_DEGENERATE;
    }
    FEM_TRY(pattern_steps_incidence(E, n_elems, npe, n_nodes, deg, inc_ptr, cursor, inc_elem, scan_tmp, mx, s));
    unsigned long long max_deg = 0;
    FEM_CUDA(cudaMemcpyAsync(&max_deg, mx, sizeof(max_deg), cudaMemcpyDeviceToHost, s));
    FEM_CUDA(cudaStreamSynchronize(s));
    const int cap = (int)(max_deg * npe);
    if (cap > 64 * 32) {
        set_error("a node belongs to %llu elements; at most %d are supported", max_deg, 64 * 32 / npe);
        return FEM_ERR_UNSUPPORTED;
    }
    FEM_TRY(pattern_steps_rows(E, npe, n_nodes, inc_ptr, inc_elem, cap, cnt, nullptr, nullptr, s));
    FEM_TRY(scan_exclusive_i64(cnt, rowptr, n_nodes, true, scan_tmp, s));
    int64_t nnz = 0;
    FEM_CUDA(cudaMemcpyAsync(&nnz, rowptr + n_nodes, sizeof(nnz), cudaMemcpyDeviceToHost, s));
    FEM_CUDA(cudaStreamSynchronize(s));
    *nnz_out = nnz;
    if (nnz > col_capacity) {
        set_error("col holds %lld entries; the pattern has %lld", (long long)col_capacity, (long long)nnz);
        return FEM_ERR_ARG;
    }
    FEM_TRY(pattern_steps_rows(E, npe, n_nodes, inc_ptr, inc_elem, cap, nullptr, rowptr, col, s));
    FEM_CUDA(cudaStreamSynchronize(s));
    return FEM_OK;
}
