// Float64 instantiation of the batched persistent fine kernel.
#include "pe_batch_fine.cuh"

pe_status batch_launch_fine_f64(const BProb* probs, const FineItem* items, int n_items, const int* active,
                                int* counter, BatchArrays A, int grid, int threads, size_t smem, cudaStream_t st) {
  b_fine_kernel<PE_FP64><<<grid, threads, smem, st>>>(probs, items, n_items, active, counter, A);
  PE_CUDA_TRY(cudaGetLastError());
  return PE_OK;
}

pe_status batch_fine_set_smem_mixed(size_t smem);

pe_status batch_fine_set_smem(int precision, size_t smem) {
  if (precision == PE_MIXED) return batch_fine_set_smem_mixed(smem);
  PE_CUDA_TRY(cudaFuncSetAttribute(b_fine_kernel<PE_FP64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  return PE_OK;
}
