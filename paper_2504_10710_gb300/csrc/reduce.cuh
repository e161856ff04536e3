// Block-level FP64 reductions shared by the kernels: a warp-shuffle block
// sum, the "last block" ticket, and the fixed-order sum of block partials
// (results do not depend on block scheduling).
#pragma once
#include <cuda_runtime.h>

namespace glls {
namespace {

__device__ __forceinline__ double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) s += red[w];
    return s;   // valid in thread 0
}

// Ticket increment with acquire-release semantics at GPU scope: the calling
// thread's earlier writes (its block's partial sums) are visible to whichever
// thread observes a later ticket value, and that thread sees all of them.
__device__ __forceinline__ unsigned ticket_add_acq_rel(unsigned* ticket) {
    unsigned prev;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(prev) : "l"(ticket) : "memory");
    return prev;
}

// Every block writes its partial sums (thread 0 writes them); the last block
// to finish (atomic ticket) adds the partials in block order, so the result
// does not depend on scheduling, and resets the ticket for the next launch.
// Only thread 0's writes need ordering, so no block-wide fence is issued.
__device__ __forceinline__ bool last_block(unsigned* ticket) {
    __shared__ bool is_last;
    __syncthreads();
    if (threadIdx.x == 0) is_last = ticket_add_acq_rel(ticket) == gridDim.x - 1;
    __syncthreads();
    return is_last;
}

// As last_block, for a launch of `total` blocks (multi-dimensional grids).
__device__ __forceinline__ bool last_block_of(unsigned* ticket, unsigned total) {
    __shared__ bool is_last_n;
    __syncthreads();
    if (threadIdx.x == 0) is_last_n = ticket_add_acq_rel(ticket) == total - 1;
    __syncthreads();
    return is_last_n;
}

__device__ __forceinline__ void finalize_partials(const double* part, int ndots, int nblocks, double* S, int slot0, int slot1,
                                  double* red) {
    for (int d = 0; d < ndots; ++d) {
        double s = 0.0;
        for (int i = threadIdx.x; i < nblocks; i += blockDim.x) s += __ldcg(part + d * nblocks + i);
        double t = block_sum(s, red);
        if (threadIdx.x == 0) S[d == 0 ? slot0 : slot1] = t;
    }
}

}  // namespace
}  // namespace glls
