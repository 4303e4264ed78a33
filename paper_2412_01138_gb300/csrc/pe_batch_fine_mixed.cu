// Mixed-precision instantiation of the batched persistent fine kernel.
#include "pe_batch_fine.cuh"

pe_status batch_launch_fine_mixed(const BProb* probs, const FineItem* items, int n_items, const int* active,
                                  int* counter, BatchArrays A, int grid, int threads, size_t smem, cudaStream_t st) {
  b_fine_kernel<PE_MIXED><<<grid, threads, smem, st>>>(probs, items, n_items, active, counter, A);
  PE_CUDA_TRY(cudaGetLastError());
  return PE_OK;
}

pe_status batch_fine_set_smem_mixed(size_t smem) {
  PE_CUDA_TRY(cudaFuncSetAttribute(b_fine_kernel<PE_MIXED>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  return PE_OK;
}
