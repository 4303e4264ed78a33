// Float64 instantiations of the batched persistent fine kernels (one per column class).
#include "pe_batch_fine.cuh"

pe_status batch_launch_fine_f64(int KC, const BProb* probs, const FineItem* items, int n_items, const int* active,
                                 int* counter, BatchArrays A, int grid, int threads, size_t smem, cudaStream_t st) {
  return b_fine_launch_class<PE_FP64>(KC, probs, items, n_items, active, counter, A, grid, threads, smem, st);
}
