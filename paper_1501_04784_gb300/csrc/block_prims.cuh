// block_prims.cuh -- block-wide primitives of the symbolic kernels: ascending
// bitonic sorts of a power-of-two number of 32- or 64-bit keys in shared memory
// and an in-place exclusive prefix sum.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fem {

__host__ __device__ inline int pow2_at_least(int n) {
    int p = 1;
    while (p < n) p <<= 1;
    return p;
}

// ----------------------------------------------------------- block primitives
// Ascending bitonic sort of n (a power of two) keys in shared memory.
__device__ inline void block_bitonic(uint32_t *keys, int n) {
    for (int k = 2; k <= n; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const uint32_t a = keys[i], b = keys[ixj];
                    const bool up = (i & k) == 0;
                    if ((a > b) == up) {
                        keys[i] = b;
                        keys[ixj] = a;
                    }
                }
            }
            __syncthreads();
        }
}

// The same for 64-bit keys.
__device__ inline void block_bitonic64(uint64_t *keys, int n) {
    for (int k = 2; k <= n; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const uint64_t a = keys[i], b = keys[ixj];
                    const bool up = (i & k) == 0;
                    if ((a > b) == up) {
                        keys[i] = b;
                        keys[ixj] = a;
                    }
                }
            }
            __syncthreads();
        }
}

// In-place exclusive prefix sum of n ints in shared memory; returns the total to
// every thread.  ws: 32 ints of shared scratch.
__device__ inline int block_scan(int *a, int n, int *ws) {
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, w = tid >> 5, nw = nt >> 5;
    const int per = (n + nt - 1) / nt;
    const int b = min(n, tid * per), e = min(n, b + per);
    int s = 0;
    for (int i = b; i < e; ++i) s += a[i];
    int x = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[w] = x;
    __syncthreads();
    if (w == 0) {
        int v = lane < nw ? ws[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        if (lane < nw) ws[lane] = v;
    }
    __syncthreads();
    int run = (w > 0 ? ws[w - 1] : 0) + x - s;
    for (int i = b; i < e; ++i) {
        const int v = a[i];
        a[i] = run;
        run += v;
    }
    const int total = ws[nw - 1];
    __syncthreads();
    return total;
}

}  // namespace fem
