// kt_sched.cu -- longest-first order of the persistent work queue.
//
// The cost of one cell-integration varies by two orders of magnitude across a batch
// (sub-step counts follow the density and temperature of the cell), while the lanes
// of a warp advance in lockstep and a persistent launch ends with its slowest warp.
// Taking cells from the queue in index order leaves the expensive cells that happen to
// come last running alone at the end of the launch.  Handing out the expensive cells
// first (the longest-processing-time rule of list scheduling) removes most of that
// tail.  The cost estimate is the Newton-iteration count the previous call left for
// each cell; cells are grouped into buckets of a quarter octave of that count (a
// counting sort: histogram, descending scan, scatter).  Results do not depend on the
// order: every cell's integration is the same computation whichever lane runs it.
#include <cuda_runtime.h>

#include <cstdint>

#include "kt_internal.h"

namespace kt {
namespace {

// Quarter-octave bucket of a non-negative count: 4 floor(log2(x)) + the two bits after
// the leading one, x = count + 1 (bucket 0 for count 0).
__device__ __forceinline__ int cost_bucket(int count)
{
    const unsigned x = static_cast<unsigned>(count < 0 ? 0 : count) + 1u;
    const int msb = 31 - __clz(x);
    const unsigned frac = msb >= 2 ? (x >> (msb - 2)) & 3u : (x << (2 - msb)) & 3u;
    const int b = 4 * msb + static_cast<int>(frac);
    return b < kSchedBuckets ? b : kSchedBuckets - 1;
}

__global__ void sched_hist(const int *__restrict__ count, long long n, unsigned *__restrict__ hist)
{
    __shared__ unsigned sh[kSchedBuckets];
    for (int i = threadIdx.x; i < kSchedBuckets; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    for (long long c = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; c < n;
         c += static_cast<long long>(gridDim.x) * blockDim.x)
        atomicAdd(&sh[cost_bucket(count[c])], 1u);
    __syncthreads();
    for (int i = threadIdx.x; i < kSchedBuckets; i += blockDim.x)
        if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

// cursor[b] = number of cells in buckets above b (the most expensive bucket first).
__global__ void sched_scan(const unsigned *__restrict__ hist, unsigned *__restrict__ cursor)
{
    if (threadIdx.x == 0) {
        unsigned run = 0;
        for (int b = kSchedBuckets - 1; b >= 0; --b) {
            cursor[b] = run;
            run += hist[b];
        }
    }
}

__global__ void sched_scatter(const int *__restrict__ count, long long n, unsigned *__restrict__ cursor,
                              int *__restrict__ order)
{
    const long long c = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    const bool live = c < n;
    const int b = live ? cost_bucket(count[c]) : -1;
    // one atomic per distinct bucket in the warp
    const unsigned peers = __match_any_sync(0xffffffffu, b);
    const int leader = __ffs(peers) - 1;
    const int lane = threadIdx.x & 31;
    unsigned base = 0;
    if (live && lane == leader) base = atomicAdd(&cursor[b], static_cast<unsigned>(__popc(peers)));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (live) order[base + __popc(peers & ((1u << lane) - 1u))] = static_cast<int>(c);
}

}  // namespace

int launch_schedule(const int *count, long long ncells, unsigned *work, int *order, void *stream)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (ncells <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(work, 0, 2 * kSchedBuckets * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    const int threads = 256;
    long long blocks = (ncells + threads - 1) / threads;
    const long long hist_blocks = blocks < 1024 ? blocks : 1024;
    sched_hist<<<static_cast<unsigned>(hist_blocks), threads, 0, s>>>(count, ncells, work);
    sched_scan<<<1, 32, 0, s>>>(work, work + kSchedBuckets);
    sched_scatter<<<static_cast<unsigned>(blocks), threads, 0, s>>>(count, ncells, work + kSchedBuckets, order);
    return cudaGetLastError();
}

}  // namespace kt
