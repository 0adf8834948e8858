// The persistent batch kernel, f32 instance (see q2x_batch.cuh).
#include "q2x_batch.cuh"

namespace q2x {

cudaError_t batch_launch_f32(const BatchArgs& b, int grid, size_t smem, cudaStream_t st)
{
    cudaError_t e = cudaFuncSetAttribute(q2x_batch_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    q2x_batch_kernel<float><<<grid, BATCH_WARPS * 32, smem, st>>>(b);
    return cudaGetLastError();
}

cudaError_t batch_occupancy_f32(int* blocks_per_sm, size_t smem)
{
    cudaError_t e = cudaFuncSetAttribute(q2x_batch_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, q2x_batch_kernel<float>, BATCH_WARPS * 32, smem);
}

}  // namespace q2x
