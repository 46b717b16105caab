// Uneven-batch kernels for the F_p groups (see bg_batch.cuh).
#include "bg_batch.cuh"

namespace bgk {
const void* batch_kernel_fp(bool wide) {
    return wide ? reinterpret_cast<const void*>(&bg_batch_kernel<FpOps, kBlockFpBatch, 1>)
                : reinterpret_cast<const void*>(&bg_batch_kernel<FpOps, kBlockFpBatch, kFpNarrowBlocks>);
}
void launch_batch_fp(const BatchArgs& a, int blocks, bool wide, cudaStream_t s) {
    if (wide) bg_batch_kernel<FpOps, kBlockFpBatch, 1><<<blocks, kBlockFpBatch, 0, s>>>(a);
    else bg_batch_kernel<FpOps, kBlockFpBatch, kFpNarrowBlocks><<<blocks, kBlockFpBatch, 0, s>>>(a);
}
}  // namespace bgk
