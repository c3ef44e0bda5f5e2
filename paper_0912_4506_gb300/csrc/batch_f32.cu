// Batched persistent kernel, f32 storage.
#include "batch_kernel.cuh"

namespace jac {

cudaError_t launch_batch_f32(const BatchArgs& a, int ctas, size_t smem, cudaStream_t st) {
    tb_batch_kernel<F32><<<ctas, kBatchNW * 32, smem, st>>>(a);
    return cudaGetLastError();
}

const void* batch_kernel_f32() { return reinterpret_cast<const void*>(&tb_batch_kernel<F32>); }

}  // namespace jac
