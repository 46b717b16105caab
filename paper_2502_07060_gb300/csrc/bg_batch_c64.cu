// Uneven-batch kernel for the complex FP64 groups (see bg_batch.cuh).
#include "bg_batch.cuh"

namespace bgk {
const void* batch_kernel_c64() { return reinterpret_cast<const void*>(&bg_batch_kernel<C64Ops, kBlockC64Batch, 1>); }
void launch_batch_c64(const BatchArgs& a, int blocks, cudaStream_t s) {
    bg_batch_kernel<C64Ops, kBlockC64Batch, 1><<<blocks, kBlockC64Batch, 0, s>>>(a);
}
}  // namespace bgk
