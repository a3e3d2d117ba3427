// Device work queue of the persistent blend kernels.
//
// A persistent launch runs as many CTAs as fit on the GPU at once. Each CTA
// takes the next item (a position in the launch order of the batch's (frame,
// tile) pairs) with one atomic increment of queue[0] and loops until the items
// are exhausted; no CTA ever waits for another. The queue is two caller-owned
// counters, zero before the first launch: queue[1] counts the CTAs that have
// finished, and the last one to finish puts both counters back to zero, so
// the next launch in stream order starts from an empty queue without a clear.
#pragma once

#include <cuda_runtime.h>

#include <atomic>

#include "gs_internal.cuh"

namespace gs {

// Next item for this CTA (uniform across the CTA). s_item holds two slots that
// alternate between loop iterations, so one barrier per item suffices: a
// thread re-reads slot (it & 1) only after every thread has passed the
// barrier of iteration it + 1.
__device__ __forceinline__ int queue_next(unsigned *queue, int *s_item, int it) {
    if (threadIdx.x == 0) s_item[it & 1] = (int)atomicAdd(queue, 1u);
    __syncthreads();
    return s_item[it & 1];
}

// Called once by every CTA after its last (failed) fetch.
__device__ __forceinline__ void queue_exit(unsigned *queue) {
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(queue + 1, 1u) == gridDim.x - 1) {  // every CTA has made its last fetch
            atomicExch(queue, 0u);
            atomicExch(queue + 1, 0u);
        }
    }
}

// Grid of a persistent launch of KERNEL: resident CTAs per SM x SMs (the
// occupancy is read once per device and kernel; the first call comes before
// any stream capture), never more CTAs than items.
template <auto KERNEL>
cudaError_t persistent_grid(int threads, size_t smem, int items, int *grid) {
    static std::atomic<int> cached[64];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    int per_sm = dev < 64 ? cached[dev].load(std::memory_order_relaxed) : 0;
    if (per_sm == 0) {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, KERNEL, threads, smem);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) per_sm = 1;
        if (dev < 64) cached[dev].store(per_sm, std::memory_order_relaxed);
    }
    const long long g = (long long)per_sm * device_sm_count();
    *grid = (int)(g < items ? g : (items > 0 ? items : 1));
    return cudaSuccess;
}

}  // namespace gs
