// Deterministic FP64 reductions over a grid of blocks (the norm and inner-product sums of
// the power iteration, FISTA's objective pieces and the unrolled gradient's lambda term).
// Every block sums a fixed set of elements in a fixed tree order and leaves its pair in
// part[]; the block that takes the last ticket adds the partials in block order.  The
// result depends only on the element count and the grid, never on which block finishes
// first.  Blocks must have kDotThreads threads.
#pragma once

namespace aexp {

constexpr int kDotThreads = 256;

// Block sum of (a, b) in a fixed tree order; the result is valid in thread 0.
__device__ __forceinline__ void block_sum2(double &a, double &b, double *sa, double *sb) {
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    if (lane == 0) {
        sa[warp] = a;
        sb[warp] = b;
    }
    __syncthreads();
    if (warp == 0) {
        a = lane < kDotThreads / 32 ? sa[lane] : 0.0;
        b = lane < kDotThreads / 32 ? sb[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            b += __shfl_xor_sync(0xffffffffu, b, o);
        }
    }
}

// Block `blk` of `nblk` contributes its per-thread (a, b).  Returns true in thread 0 of the
// block that finished last, with (a, b) the totals over all blocks; that block also resets
// the ticket, so the same part/ticket serve the next launch (also inside a replayed graph).
// Every thread of every block must call it.
__device__ __forceinline__ bool grid_sum2(double &a, double &b, int blk, int nblk, double *part,
                                          unsigned *ticket) {
    __shared__ double sa[kDotThreads / 32], sb[kDotThreads / 32];
    __shared__ bool last;
    block_sum2(a, b, sa, sb);
    if (threadIdx.x == 0) {
        part[2 * blk] = a;
        part[2 * blk + 1] = b;
        __threadfence();
        last = atomicAdd(ticket, 1u) == (unsigned)nblk - 1;
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    a = b = 0.0;
    for (int k = threadIdx.x; k < nblk; k += kDotThreads) {
        a += __ldcg(part + 2 * k);
        b += __ldcg(part + 2 * k + 1);
    }
    __syncthreads();  // the shared partials of the first block_sum2 are reused
    block_sum2(a, b, sa, sb);
    if (threadIdx.x == 0) *ticket = 0u;
    return threadIdx.x == 0;
}

}  // namespace aexp
