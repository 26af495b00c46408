// Block-level reductions (sum, max, arg-max) in float64 and the deterministic "last block"
// completion used to finish grid reductions inside the kernel that produced the partials.
#pragma once

#include "common.cuh"

namespace pb {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Larger value wins; equal values go to the smaller index.  NaN never wins (the non-finite
// flag reports it separately).
__device__ __forceinline__ void argmax_merge(double& v, long long& i, double v2, long long i2) {
    if (v2 > v || (v2 == v && i2 < i)) { v = v2; i = i2; }
}

__device__ __forceinline__ void warp_argmax(double& v, long long& i) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        double v2 = __shfl_xor_sync(0xffffffffu, v, o);
        long long i2 = __shfl_xor_sync(0xffffffffu, i, o);
        argmax_merge(v, i, v2, i2);
    }
}

// Sums NV values over the block; the result is valid in thread 0.  All threads must call.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV]) {
    __shared__ double red[NV][32];
    const int nt = blockDim.x * blockDim.y * blockDim.z;
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int lane = tid & 31, warp = tid >> 5, nw = (nt + 31) >> 5;
#pragma unroll
    for (int a = 0; a < NV; ++a) v[a] = warp_sum(v[a]);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int a = 0; a < NV; ++a) red[a][warp] = v[a];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int a = 0; a < NV; ++a) {
            double x = lane < nw ? red[a][lane] : 0.0;
            v[a] = warp_sum(x);
        }
    }
}

__device__ __forceinline__ void block_argmax(double& v, long long& i) {
    __shared__ double rv[32];
    __shared__ long long ri[32];
    const int nt = blockDim.x * blockDim.y * blockDim.z;
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int lane = tid & 31, warp = tid >> 5, nw = (nt + 31) >> 5;
    warp_argmax(v, i);
    __syncthreads();
    if (lane == 0) { rv[warp] = v; ri[warp] = i; }
    __syncthreads();
    if (warp == 0) {
        // empty lanes carry -inf, below any value a caller merges (|F| >= 0, or -bound)
        v = lane < nw ? rv[lane] : -(1.0 / 0.0);
        i = lane < nw ? ri[lane] : 0x7fffffffffffffffLL;
        warp_argmax(v, i);
    }
}

// Returns true in every thread of the block that completes the grid (the last one to arrive).
// Partials written before the call by thread 0 of each block are visible to that block.
__device__ __forceinline__ bool last_block(unsigned int* counter, int nblocks) {
    __shared__ int am_last;
    __threadfence();
    __syncthreads();
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    if (tid == 0) {
        unsigned int prev = atomicAdd(counter, 1u);
        am_last = (prev == (unsigned int)(nblocks - 1));
    }
    __syncthreads();
    if (am_last) __threadfence();
    return am_last != 0;
}

// Sums NV doubles over `count` partial records (stride `stride` doubles) in a fixed order; the
// result is valid in thread 0.  Called by one whole block.
template <int NV>
__device__ __forceinline__ void sum_partials(const double* part, int count, int stride, double (&v)[NV]) {
    const int nt = blockDim.x * blockDim.y * blockDim.z;
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
#pragma unroll
    for (int a = 0; a < NV; ++a) v[a] = 0.0;
    for (int b = tid; b < count; b += nt)
#pragma unroll
        for (int a = 0; a < NV; ++a) v[a] += __ldcg(part + (size_t)b * stride + a);
    block_sum<NV>(v);
}

}  // namespace pb
