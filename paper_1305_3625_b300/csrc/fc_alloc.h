// Allocation wrappers of the fftconv library (defined in fc_lib.cu).  Every
// device and pinned allocation the library makes goes through them: they
// count live allocations and bytes (fc_mem_stats) and honour the host-side
// allocation-failure injection of fc_debug_inject (FC_INJECT_ALLOC), which
// makes the chosen allocation return cudaErrorMemoryAllocation.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

namespace fc {

cudaError_t dev_malloc(void** ptr, size_t bytes);
cudaError_t dev_malloc_async(void** ptr, size_t bytes, cudaStream_t s);
cudaError_t host_malloc(void** ptr, size_t bytes);
void dev_free(void* ptr);
void dev_free_async(void* ptr, cudaStream_t s);
void host_free(void* ptr);

}  // namespace fc
