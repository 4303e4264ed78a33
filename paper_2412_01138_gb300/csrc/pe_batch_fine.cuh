// Persistent fine-propagator kernel of the batched solver: CTAs pull
// (problem, slice, mode-tile) items from an atomic counter and run the tile
// body specialised for the problem's number of forcing terms R.
#pragma once
#include "pe_batch.h"
#include "pe_fine_kernels.cuh"

namespace {

// Tile bodies are compiled for R rounded up to a multiple of 4 (RC = 4..20); the
// padding terms carry zero weights.
template <int PREC, int RC>
__device__ __forceinline__ void run_tile(const FineTile& t, int R, double* smem) {
  if constexpr (PREC == PE_MIXED) {
    fine_mixed_tile<RC, (RC <= 16 ? 4 : 2)>(t, R, reinterpret_cast<float*>(smem));
  } else {
    fine_f64_tile<RC>(t, R, smem);
  }
}

template <int PREC>
__device__ __forceinline__ void dispatch_tile(int R, const FineTile& t, double* smem) {
  const int RC = (R + 3) / 4 * 4;
  switch (RC) {
    case 4: run_tile<PREC, 4>(t, R, smem); break;
    case 8: run_tile<PREC, 8>(t, R, smem); break;
    case 12: run_tile<PREC, 12>(t, R, smem); break;
    case 16: run_tile<PREC, 16>(t, R, smem); break;
    case 20: run_tile<PREC, 20>(t, R, smem); break;
    default: break;
  }
}

template <int PREC>
__global__ void __launch_bounds__(256) b_fine_kernel(const BProb* __restrict__ probs,
                                                     const FineItem* __restrict__ items, int n_items,
                                                     const int* __restrict__ active, int* __restrict__ counter,
                                                     BatchArrays A) {
  extern __shared__ __align__(16) double smem_d[];
  __shared__ int s_item;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    const int it = s_item;
    __syncthreads();
    if (it >= n_items) break;
    const FineItem f = items[it];
    const BProb& B = probs[f.p];
    if (!active[f.p]) continue;  // uniform over the CTA
    FineTile t{};
    t.g = B.g;
    t.M = B.M;
    t.q = B.q;
    t.base = f.J0;
    t.mchunk = B.mchunk;
    const int64_t slice_af = (int64_t)B.M * B.q * B.R;
    t.axisF = A.axisF + B.oAx;
    t.AFn = A.AF + B.oAF + (int64_t)f.n * slice_af;
    t.coefF = A.coefF + B.oCF;
    if (PREC == PE_MIXED) {
      t.axisF32 = A.axisF32 + B.oAx;
      t.AFn32 = A.AF32 + B.oAF + (int64_t)f.n * slice_af;
      t.coefF32 = A.coefF32 + B.oCF;
    }
    t.Un = A.U + B.oU + (int64_t)f.n * B.g.ndof;
    t.Fn = A.Fbar + B.oS + (int64_t)f.n * B.g.ndof;
    dispatch_tile<PREC>(B.R, t, smem_d);
  }
}

}  // namespace
