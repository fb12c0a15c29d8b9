// Bounded grid-wide barrier for cooperative launches.
#pragma once

#include <cuda_runtime.h>

#include "slim_kernels.h"

namespace slim {

// Grid-wide barrier of a cooperative launch (all blocks resident): arrival counter
// bar[0] and generation bar[1] in device memory.  The wait is bounded: after
// kBarrierPolls polls the block records SLIM_ERRBIT_TIMEOUT and returns false, and
// the kernel ends (the other blocks then time out at their next barrier).
constexpr int kBarrierPolls = 1 << 21;  // about 0.15 s of 64-ns sleeps
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned nblk, int* err, int* s_fail) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = bar + 1;
    const unsigned g0 = *vgen;
    __threadfence();
    int fail = 0;
    if (atomicAdd(bar, 1u) == nblk - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      int it = 0;
      while (*vgen == g0) {
        if (++it > kBarrierPolls) {
          fail = 1;
          atomicOr(err, (int)SLIM_ERRBIT_TIMEOUT);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    *s_fail = fail;
  }
  __syncthreads();
  return *s_fail == 0;
}

// Wait of one block of a cooperative launch for its neighbour blocks only: block b
// publishes done[b] = k once its stores of stage k are issued, then waits until
// done[n] >= k for every block n in its list s_nb[0, nn) (the blocks that own a
// triangle its triangles read).  Blocks that share no data never wait for each
// other, and no counter is contended.  Bounded like grid_barrier: after
// kBarrierPolls polls (16-ns sleeps between them: a waiter wakes sooner than with the
// barrier's 64 ns, 1% of the 2D run) a thread records SLIM_ERRBIT_TIMEOUT and the
// block returns false.  *s_fail must be 0 on entry.
__device__ __forceinline__ bool neighbour_wait(unsigned* done, unsigned k, const int* s_nb, int nn, int* err,
                                               int* s_fail) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicExch(done + blockIdx.x, k);
  }
  for (int j = threadIdx.x; j < nn; j += blockDim.x) {
    volatile unsigned* d = done + s_nb[j];
    int it = 0;
    while (*d < k) {
      if (++it > kBarrierPolls) {
        *s_fail = 1;
        atomicOr(err, (int)SLIM_ERRBIT_TIMEOUT);
        break;
      }
      __nanosleep(16);
    }
  }
  // only the threads that observed a counter fence; the block barrier then orders
  // every thread of the block after them
  if (threadIdx.x < nn) __threadfence();
  __syncthreads();
  return *s_fail == 0;
}

}  // namespace slim
