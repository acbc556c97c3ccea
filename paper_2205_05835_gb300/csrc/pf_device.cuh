// Device helpers shared by the kernels: periodic indexing and deterministic
// block reductions finished by the last block of a fixed-size grid.
#pragma once

#include "pf_internal.h"

namespace pf {

__device__ __forceinline__ int wrapi(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// Cell coordinates of a linear index (x fastest).
struct Cell {
    int i, j, k;
};

__device__ __forceinline__ Cell decode(int idx, const Dims& g) {
    Cell c;
    c.i = idx % g.nx;
    int t = idx / g.nx;
    c.j = t % g.ny;
    c.k = t / g.ny;
    return c;
}

// Wrapped neighbour index for offsets |o| <= 3 along each axis (n >= 4).
template <int DIM>
struct Nbr {
    int nx, ny, nz;
    int im[7], jm[7], km[7];   // wrapped coordinates for offsets -3..3
    __device__ __forceinline__ Nbr(const Cell& c, const Dims& g) : nx(g.nx), ny(g.ny), nz(g.nz) {
#pragma unroll
        for (int o = -3; o <= 3; ++o) {
            im[o + 3] = wrapi(c.i + o, g.nx);
            jm[o + 3] = wrapi(c.j + o, g.ny);
            km[o + 3] = (DIM == 3) ? wrapi(c.k + o, g.nz) : 0;
        }
    }
    __device__ __forceinline__ int at(int di, int dj, int dk) const {
        return (km[dk + 3] * ny + jm[dj + 3]) * nx + im[di + 3];
    }
    // offset o along axis d
    __device__ __forceinline__ int ax(int d, int o) const {
        return d == 0 ? at(o, 0, 0) : (d == 1 ? at(0, o, 0) : at(0, 0, o));
    }
    // offsets o1 along d1 and o2 along d2 (d1 != d2)
    __device__ __forceinline__ int ax2(int d1, int o1, int d2, int o2) const {
        int di = (d1 == 0 ? o1 : 0) + (d2 == 0 ? o2 : 0);
        int dj = (d1 == 1 ? o1 : 0) + (d2 == 1 ? o2 : 0);
        int dk = (d1 == 2 ? o1 : 0) + (d2 == 2 ? o2 : 0);
        return at(di, dj, dk);
    }
};

template <typename T>
__device__ __forceinline__ T ldg(const T* p, int i) { return __ldg(p + i); }

// Sum of K values over the block (deterministic order). Result valid in thread 0.
template <int K>
__device__ __forceinline__ void block_reduce_sum(double (&v)[K], double* smem /* K*32 */) {
#pragma unroll
    for (int q = 0; q < K; ++q)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < K; ++q) smem[q * 32 + warp] = v[q];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int q = 0; q < K; ++q) {
            double t = lane < nw ? smem[q * 32 + lane] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
            v[q] = t;
        }
    }
    __syncthreads();
}

template <int K>
__device__ __forceinline__ void block_reduce_max(double (&v)[K], double* smem) {
#pragma unroll
    for (int q = 0; q < K; ++q)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[q] = fmax(v[q], __shfl_down_sync(0xffffffffu, v[q], o));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < K; ++q) smem[q * 32 + warp] = v[q];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int q = 0; q < K; ++q) {
            double t = lane < nw ? smem[q * 32 + lane] : -1.0e308;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t = fmax(t, __shfl_down_sync(0xffffffffu, t, o));
            v[q] = t;
        }
    }
    __syncthreads();
}

// Stores the block's K partials; returns true in every thread of the last
// block to finish, after which `tot` holds the grid totals (fixed order).
// Mode per value: 0 sum, 1 max.
template <int K>
__device__ __forceinline__ bool grid_reduce(double (&v)[K], const int (&mode)[K], RedBuf rb,
                                            double (&tot)[K]) {
    __shared__ double smem[K * 32];
    __shared__ bool last;
    double s[K], m[K];
#pragma unroll
    for (int q = 0; q < K; ++q) {
        s[q] = mode[q] == 0 ? v[q] : 0.0;
        m[q] = mode[q] == 1 ? v[q] : -1.0e308;
    }
    block_reduce_sum<K>(s, smem);
    block_reduce_max<K>(m, smem);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < K; ++q) rb.part[blockIdx.x * K + q] = mode[q] == 0 ? s[q] : m[q];
        __threadfence();
        unsigned t = atomicAdd(rb.counter, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
#pragma unroll
    for (int q = 0; q < K; ++q) {
        s[q] = 0.0;
        m[q] = -1.0e308;
    }
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
#pragma unroll
        for (int q = 0; q < K; ++q) {
            double t = __ldcg(rb.part + b * K + q);
            if (mode[q] == 0) s[q] += t; else m[q] = fmax(m[q], t);
        }
    }
    block_reduce_sum<K>(s, smem);
    block_reduce_max<K>(m, smem);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < K; ++q) tot[q] = mode[q] == 0 ? s[q] : m[q];
        *rb.counter = 0u;
    }
    return true;
}

inline int red_grid(int n) {
    int b = (n + kThreads - 1) / kThreads;
    return b < kRedBlocks ? (b < 1 ? 1 : b) : kRedBlocks;
}

inline int lin_grid(int n) {
    int b = (n + kThreads - 1) / kThreads;
    return b < 1 ? 1 : b;
}

}  // namespace pf
