// Deterministic block reduction helpers: a fixed grid accumulates per-thread
// grid-stride sums, reduces them warp-wise with shuffles in a fixed pattern and
// writes one partial per block; a single block then sums the partials in order.
#pragma once

#include <cuda_runtime.h>

namespace nek {

template <int NT>
__device__ __forceinline__ double block_sum(double v, double* sh /* NT/32 doubles */)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double t = 0.0;
    if (wid == 0) {
        t = lane < NT / 32 ? sh[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    __syncthreads();
    return t;  // valid in thread 0
}

// Sum of nparts partials (in a fixed order) by one block of NT threads.  The
// unrolled loop issues a thread's loads together; the adds stay in order.
template <int NT>
__device__ __forceinline__ double sum_partials(const double* __restrict__ parts, int nparts, double* sh)
{
    double v = 0.0;
#pragma unroll 8
    for (int q = threadIdx.x; q < nparts; q += NT) v += parts[q];
    return block_sum<NT>(v, sh);
}

// out[e] = sum of the values v of element e's threads (thread t belongs to
// element t / TPE).  Each element's TPE values are summed in a fixed order
// (lane-strided, then a shuffle tree), so the result depends on nx only, not on
// the number of elements per CTA.  sh: blockDim doubles of shared memory that
// no thread reads any more.
template <int TPE, int EPB>
__device__ __forceinline__ void element_sums(double v, double* sh, double* __restrict__ out, int ne)
{
    __syncthreads();
    sh[threadIdx.x] = v;
    __syncthreads();
    if constexpr (TPE >= 32) {
        if (threadIdx.x < EPB * 32) {  // whole warps: the block has EPB * TPE >= EPB * 32 threads
            const int e = threadIdx.x >> 5, lane = threadIdx.x & 31;
            double t = 0.0;
            for (int q = lane; q < TPE; q += 32) t += sh[e * TPE + q];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if (lane == 0 && e < ne) out[e] = t;
        }
    } else {
        if (threadIdx.x < EPB) {
            double t = 0.0;
            for (int q = 0; q < TPE; q++) t += sh[threadIdx.x * TPE + q];
            if ((int)threadIdx.x < ne) out[threadIdx.x] = t;
        }
    }
}

}  // namespace nek
