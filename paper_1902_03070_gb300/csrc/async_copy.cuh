// Asynchronous global -> shared copies (cp.async, 16-byte chunks): a CTA
// issues every chunk of a tile before waiting once, so the copy is bound by
// bandwidth rather than by one load's latency per thread.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace tnn {

// 16 bytes from gmem to smem; both addresses 16-byte aligned.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}

// Wait for all of this thread's cp.async copies (a __syncthreads must follow
// before other threads read them).
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;\n" ::: "memory");
}

// True when a contiguous copy of `count` floats between these addresses can
// go in 16-byte chunks.
__device__ __forceinline__ bool chunkable(const void* smem, const void* gmem, size_t count)
{
    return ((reinterpret_cast<uintptr_t>(smem) | reinterpret_cast<uintptr_t>(gmem)) & 15u) == 0 && count % 4 == 0;
}

// Contiguous copy of `count` floats (16-byte chunks when chunkable, else
// plain loads) by the threads tid = 0 .. nthr - 1; the caller waits with
// cp_async_wait_all and a barrier.
__device__ __forceinline__ void copy_to_shared(float* smem, const float* gmem, size_t count, int tid, int nthr)
{
    if (chunkable(smem, gmem, count)) {
        for (size_t e = (size_t)tid * 4; e < count; e += (size_t)nthr * 4) cp_async16(smem + e, gmem + e);
    } else {
        for (size_t e = tid; e < count; e += nthr) smem[e] = gmem[e];
    }
}

}  // namespace tnn
