// Uneven-batch kernel for the F_p groups (see bg_batch.cuh).
#include "bg_batch.cuh"

namespace bgk {
const void* batch_kernel_fp() { return reinterpret_cast<const void*>(&bg_batch_kernel<FpOps, kBlockFpBatch>); }
void launch_batch_fp(const BatchArgs& a, int blocks, cudaStream_t s) {
    bg_batch_kernel<FpOps, kBlockFpBatch><<<blocks, kBlockFpBatch, 0, s>>>(a);
}
}  // namespace bgk
