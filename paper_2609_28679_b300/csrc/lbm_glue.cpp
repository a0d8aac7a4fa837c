// Device memory and streams from PyTorch's CUDA runtime (libc10_cuda): the
// library allocates through the caching allocator so that its buffers share
// the pool with the caller's tensors, and defaults to the caller's current
// stream.  The rest of the library sees only these three C functions.
#include <c10/cuda/CUDACachingAllocator.h>
#include <c10/cuda/CUDAStream.h>
#include <cuda_runtime.h>

extern "C" {

void* lbm_glue_alloc(size_t nbytes, void* stream)
{
    try {
        auto* alloc = c10::cuda::CUDACachingAllocator::get();
        if (alloc == nullptr || !alloc->initialized()) return nullptr;
        if (nbytes == 0) nbytes = 256;
        return alloc->raw_alloc_with_stream(nbytes, static_cast<cudaStream_t>(stream));
    } catch (...) {
        return nullptr;
    }
}

void lbm_glue_free(void* ptr)
{
    if (ptr == nullptr) return;
    try {
        c10::cuda::CUDACachingAllocator::raw_delete(ptr);
    } catch (...) {
    }
}

void* lbm_glue_current_stream(int device)
{
    try {
        return static_cast<void*>(c10::cuda::getCurrentCUDAStream(static_cast<c10::DeviceIndex>(device)).stream());
    } catch (...) {
        return nullptr;
    }
}

}  // extern "C"
