// pool.cuh -- device memory of encoded matrices and solver workspaces.
//
// Every handle buffer and Krylov workspace comes from one stream-ordered
// memory pool per device, owned by the library and never trimmed: a server
// encodes and frees one matrix per request, and with the pool neither step
// calls into the driver's allocator (cudaMalloc) or synchronises the device
// (cudaFree).  Blocks are allocated on the stream that first uses them.  They
// are returned only after the caller has synchronised the device (gse_free
// does), so a block is never reused while queued work still reads it.
#pragma once

#include <cuda_runtime.h>

#include "../../include/gse.h"

namespace gse {

// The pool of the current device (created on first use; nullptr if it could
// not be created).
cudaMemPool_t device_pool();

// count elements of T from the pool, ordered on stream s; *acc += bytes.
template <typename T>
static int pool_alloc(T** p, size_t count, size_t* acc, cudaStream_t s) {
    if (count == 0) count = 1;
    const size_t bytes = count * sizeof(T);
    cudaMemPool_t pool = device_pool();
    if (!pool || cudaMallocFromPoolAsync((void**)p, bytes, pool, s) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return GSE_ERR_OOM;
    }
    if (acc) *acc += bytes;
    return GSE_OK;
}

// Returns a block to the pool; call only once no queued work uses it.
static inline void pool_free(void* p) {
    if (p) cudaFreeAsync(p, 0);
}

}  // namespace gse
