// Persistent fine-propagator kernels of the batched solver: CTAs pull
// (problem, slice, mode-tile) items from an atomic counter and run the tile
// body specialised for the column class KC of the launch.  Each tile is Eq. (1-7)
// applied M times in the stage-contracted form of the single-problem solver:
//   c <- E_F c + sum_k Y_k(T_n + m dt) W_{k,J},
// with the K per-mode stage weights W (one column per exponential source term,
// two per sinusoid) tabulated at preparation.  The slice's Y rows are staged in
// shared memory, zero-padded to KC = roundup(K, 4) (warp-wide broadcasts); W
// and E_F stay in registers.
// PE_MIXED: F^M(v) = E_F^M v (float64) + F^M(0) (float32, E_F as hi + lo).
#pragma once
#include "pe_batch.h"

namespace {

// Operands of one tile: one slice n of one problem, blockDim.x*MPT modes from `base`.
struct BFineTile {
  int64_t ndof;
  int M, mchunk, q, K;
  int64_t base;
  const float* W32;       // stage weights of the problem [K][ndof]
  const double* W;
  const float* Yn32;      // substep time factors of slice n [M][K]
  const double* Yn;
  const float* coefF32;   // E_hi, E_lo (rows of ndof)
  const double* coefF;    // E, dt*b_i, exp(-lam M dt) (rows of ndof)
  const double* Un;
  double* Fn;
};

template <int KC, int MPT>
__device__ __forceinline__ void b_fine_mixed_tile(const BFineTile& a, float* sY) {
  const int M = a.M, B = blockDim.x, K = a.K;
  const int64_t nd = a.ndof;
  const int64_t base = a.base + threadIdx.x;
  float W[MPT][KC];
  float eh[MPT], el[MPT], w[MPT];
#pragma unroll
  for (int k = 0; k < MPT; ++k) {
    const int64_t J = base + (int64_t)B * k;
    eh[k] = 0.f;
    el[k] = 0.f;
    w[k] = 0.f;
#pragma unroll
    for (int c = 0; c < KC; ++c) W[k][c] = (J < nd && c < K) ? a.W32[(int64_t)c * nd + J] : 0.f;
    if (J < nd) {
      eh[k] = a.coefF32[J];
      el[k] = a.coefF32[nd + J];
    }
  }
  for (int m0 = 0; m0 < M; m0 += a.mchunk) {
    const int mc = min(a.mchunk, M - m0);
    __syncthreads();
    for (int t = threadIdx.x; t < mc * KC; t += B) {
      const int row = t / KC, c = t - row * KC;
      sY[t] = c < K ? a.Yn32[(int64_t)(m0 + row) * K + c] : 0.f;
    }
    __syncthreads();
    for (int m = 0; m < mc; ++m) {
      const float4* y4 = reinterpret_cast<const float4*>(sY + m * KC);
      float acc[MPT];
#pragma unroll
      for (int k = 0; k < MPT; ++k) acc[k] = 0.f;
#pragma unroll
      for (int c4 = 0; c4 < KC / 4; ++c4) {
        if (4 * c4 < K) {
          const float4 v = y4[c4];
          const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
          for (int e = 0; e < 4; ++e)
#pragma unroll
            for (int k = 0; k < MPT; ++k) acc[k] = fmaf(vv[e], W[k][4 * c4 + e], acc[k]);
        }
      }
#pragma unroll
      for (int k = 0; k < MPT; ++k) w[k] = fmaf(eh[k], w[k], fmaf(el[k], w[k], acc[k]));
    }
  }
  const double* EM = a.coefF + (int64_t)(a.q + 1) * nd;
#pragma unroll
  for (int k = 0; k < MPT; ++k) {
    const int64_t J = base + (int64_t)B * k;
    if (J < nd) a.Fn[J] = fma(EM[J], a.Un[J], (double)w[k]);
  }
}

template <int KC>
__device__ __forceinline__ void b_fine_f64_tile(const BFineTile& a, double* sY) {
  const int M = a.M, B = blockDim.x, K = a.K;
  const int64_t nd = a.ndof;
  const int64_t J = a.base + threadIdx.x;
  const bool active = J < nd;
  double W[KC];
  double E = 0.0, c = 0.0;
#pragma unroll
  for (int k = 0; k < KC; ++k) W[k] = (active && k < K) ? a.W[(int64_t)k * nd + J] : 0.0;
  if (active) {
    E = a.coefF[J];
    c = a.Un[J];
  }
  for (int m0 = 0; m0 < M; m0 += a.mchunk) {
    const int mc = min(a.mchunk, M - m0);
    __syncthreads();
    for (int t = threadIdx.x; t < mc * KC; t += B) {
      const int row = t / KC, col = t - row * KC;
      sY[t] = col < K ? a.Yn[(int64_t)(m0 + row) * K + col] : 0.0;
    }
    __syncthreads();
    if (active) {
      for (int m = 0; m < mc; ++m) {
        const double* yp = sY + m * KC;
        double acc = 0.0;
#pragma unroll
        for (int k = 0; k < KC; ++k)
          if (k < K) acc = fma(yp[k], W[k], acc);
        c = fma(E, c, acc);
      }
    }
  }
  if (active) a.Fn[J] = c;
}

template <int PREC, int KC>
__device__ __forceinline__ void run_tile(const BFineTile& t, double* smem) {
  if constexpr (PREC == PE_MIXED) {
    b_fine_mixed_tile<KC, batch_mixed_mpt(KC)>(t, reinterpret_cast<float*>(smem));
  } else {
    b_fine_f64_tile<KC>(t, smem);
  }
}

// One launch per column class KC: every item of the list belongs to a problem with
// roundup(K, 4) == KC, so each class gets the registers its own tile needs.
template <int PREC, int KC>
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
    BFineTile t{};
    t.ndof = B.g.ndof;
    t.M = B.M;
    t.q = B.q;
    t.K = B.K;
    t.base = f.J0;
    t.mchunk = B.mchunk;
    const int64_t slice_y = (int64_t)B.M * B.K;
    t.W = A.W + B.oW;
    t.Yn = A.AF + B.oAF + (int64_t)f.n * slice_y;
    t.coefF = A.coefF + B.oCF;
    if (PREC == PE_MIXED) {
      t.W32 = A.W32 + B.oW;
      t.Yn32 = A.AF32 + B.oAF + (int64_t)f.n * slice_y;
      t.coefF32 = A.coefF32 + B.oCF;
    }
    t.Un = A.U + B.oU + (int64_t)f.n * B.g.ndof;
    t.Fn = A.Fbar + B.oS + (int64_t)f.n * B.g.ndof;
    run_tile<PREC, KC>(t, smem_d);
  }
}

}  // namespace

// Launch the class-KC kernel (KC = 4, 8, ..., 40) over its item list.
template <int PREC>
pe_status b_fine_launch_class(int KC, const BProb* probs, const FineItem* items, int n_items, const int* active,
                              int* counter, BatchArrays A, int grid, int threads, size_t smem, cudaStream_t st) {
  switch (KC) {
#define PE_B_CASE(X)                                                                                  \
  case X:                                                                                             \
    b_fine_kernel<PREC, X><<<grid, threads, smem, st>>>(probs, items, n_items, active, counter, A); \
    break;
    PE_B_CASE(4) PE_B_CASE(8) PE_B_CASE(12) PE_B_CASE(16) PE_B_CASE(20)
    PE_B_CASE(24) PE_B_CASE(28) PE_B_CASE(32) PE_B_CASE(36) PE_B_CASE(40)
#undef PE_B_CASE
    default:
      return pe_fail(PE_EINVAL, "batch: column class out of range");
  }
  PE_CUDA_TRY(cudaGetLastError());
  return PE_OK;
}
