// Batched persistent kernel, bf16 storage.
#include "batch_kernel.cuh"

namespace jac {

cudaError_t launch_batch_bf16(const BatchArgs& a, int ctas, size_t smem, cudaStream_t st) {
    tb_batch_kernel<BF16><<<ctas, kBatchNW * 32, smem, st>>>(a);
    return cudaGetLastError();
}

const void* batch_kernel_bf16() { return reinterpret_cast<const void*>(&tb_batch_kernel<BF16>); }

}  // namespace jac
