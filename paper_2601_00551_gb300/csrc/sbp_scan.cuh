// Block-wide inclusive scans used by the trace finalisation and the adjoint
// preparation (int64, exact).
#pragma once

#include <cuda_runtime.h>

// Inclusive scan over the block of one int64 per thread; returns the
// inclusive prefix of the calling thread and the block total in `total`.
// `warp_tot` must hold 32 int64 of shared memory. Contains __syncthreads().
__device__ __forceinline__ long long sbp_block_incl_scan(long long v, long long* warp_tot,
                                                         long long& total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    if (lane == 31) warp_tot[wid] = v;
    __syncthreads();
    if (wid == 0) {
        long long w = lane < nw ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        warp_tot[lane] = w;
    }
    __syncthreads();
    total = warp_tot[nw - 1];
    const long long off = wid > 0 ? warp_tot[wid - 1] : 0;
    __syncthreads();  // warp_tot may be reused by the caller right away
    return v + off;
}
