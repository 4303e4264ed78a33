// Persistent fine-propagator kernels of the batched solver: CTAs pull
// (problem, mode-tile) items from an atomic counter and run, for every slice n
// of the problem in turn, Eq. (1-7) applied M times in the stage-contracted form
// of the single-problem solver:
//   c <- E_F c + sum_k Y_k(T_n + m dt) W_{k,J},
// with the K per-mode stage weights W (one column per exponential source term,
// two per sinusoid) tabulated at preparation.  W and E_F do not depend on the
// slice, so an item loads them into registers once and reuses them for all N
// slices; each slice's Y rows are staged in shared memory, zero-padded to
// KC = roundup(K, 4) (warp-wide broadcasts).  Items are ordered by decreasing
// slice count so that the longest start first.
// PE_MIXED: F^M(v) = E_F^M v (float64) + F^M(0) (float32, E_F as hi + lo).
#pragma once
#include "pe_batch.h"

namespace {

// Stage rows m0 .. m0+mc-1 of one slice's time factors (row length K, padded to KC).
template <typename T, int KC>
__device__ __forceinline__ void b_stage_rows(const T* __restrict__ Yn, int K, int m0, int mc, T* sY) {
  for (int t = threadIdx.x; t < mc * KC; t += blockDim.x) {
    const int row = t / KC, c = t - row * KC;
    sY[t] = c < K ? Yn[(int64_t)(m0 + row) * K + c] : T(0);
  }
}

// 16-byte asynchronous global -> shared copies (cp.async, waited on per group).
__device__ __forceinline__ void b_copy16(void* dst_smem, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void b_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int PENDING>
__device__ __forceinline__ void b_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(PENDING) : "memory"); }

// mc substeps of the float32 forced recurrence from staged rows sY[m*KC + k].
template <int KC, int MPT>
__device__ __forceinline__ void b_mixed_substeps(const float* sY, int mc, int K, const float (&W)[MPT][KC],
                                                 const float (&eh)[MPT], const float (&el)[MPT], float (&w)[MPT]) {
  // four substeps per trip: the later substeps' loads and FMA chains overlap the earlier ones' latency
#pragma unroll 4
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

// The float time table holds rows of KC floats (zero padded), so a slice's block is
// contiguous: when two whole blocks fit the staging buffer (P.dbuf), slice n + 1 is
// staged by cp.async into one half while slice n runs from the other.
template <int KC, int MPT>
__device__ __forceinline__ void b_fine_mixed_item(const BProb& P, int64_t J0, const BatchArrays& A, float* sY) {
  const int M = P.M, K = P.K, Bd = blockDim.x;
  const int64_t nd = P.g.ndof;
  const int64_t base = J0 + threadIdx.x;
  const float* W32 = A.W32 + P.oW;
  const float* cf32 = A.coefF32 + P.oCF;
  const double* EM = A.coefF + P.oCF + (int64_t)(P.q + 1) * nd;
  const float* Y = A.AF32 + P.oAF32;
  const int slab = M * KC;  // floats per slice, a multiple of 4
  float W[MPT][KC];
  float eh[MPT], el[MPT];
  double em[MPT];
#pragma unroll
  for (int k = 0; k < MPT; ++k) {
    const int64_t J = base + (int64_t)Bd * k;
    const bool on = J < nd;
#pragma unroll
    for (int c = 0; c < KC; ++c) W[k][c] = (on && c < K) ? W32[(int64_t)c * nd + J] : 0.f;
    eh[k] = on ? cf32[J] : 0.f;
    el[k] = on ? cf32[nd + J] : 0.f;
    em[k] = on ? EM[J] : 0.0;
  }
  auto stage = [&](int n, float* dst) {
    const float4* src = reinterpret_cast<const float4*>(Y + (int64_t)n * slab);
    float4* d4 = reinterpret_cast<float4*>(dst);
    for (int e = threadIdx.x; e < slab / 4; e += Bd) b_copy16(d4 + e, src + e);
    b_commit();
  };
  if (P.dbuf) {
    __syncthreads();  // the previous item's last reads of the buffer are done
    stage(0, sY);
  }
  for (int n = 0; n < P.N; ++n) {
    const double* Un = A.U + P.oU + (int64_t)n * nd;
    double* Fn = A.Fbar + P.oS + (int64_t)n * nd;
    double u[MPT];
#pragma unroll
    for (int k = 0; k < MPT; ++k) {
      const int64_t J = base + (int64_t)Bd * k;
      u[k] = J < nd ? Un[J] : 0.0;  // consumed after the recurrence: its latency is hidden
    }
    float w[MPT];
#pragma unroll
    for (int k = 0; k < MPT; ++k) w[k] = 0.f;
    if (P.dbuf) {
      float* cur = sY + (n & 1) * slab;
      // the other half was last read by slice n - 1, which ended with a barrier
      if (n + 1 < P.N) {
        stage(n + 1, sY + ((n + 1) & 1) * slab);
        b_wait<1>();
      } else {
        b_wait<0>();
      }
      __syncthreads();
      b_mixed_substeps<KC, MPT>(cur, M, K, W, eh, el, w);
      __syncthreads();
    } else {
      for (int m0 = 0; m0 < M; m0 += P.mchunk) {
        const int mc = min(P.mchunk, M - m0);
        __syncthreads();
        const float* src = Y + (int64_t)n * slab + (int64_t)m0 * KC;
        for (int t = threadIdx.x; t < mc * KC; t += Bd) sY[t] = src[t];
        __syncthreads();
        b_mixed_substeps<KC, MPT>(sY, mc, K, W, eh, el, w);
      }
    }
#pragma unroll
    for (int k = 0; k < MPT; ++k) {
      const int64_t J = base + (int64_t)Bd * k;
      if (J < nd) Fn[J] = fma(em[k], u[k], (double)w[k]);
    }
  }
}

template <int KC>
__device__ __forceinline__ void b_fine_f64_item(const BProb& P, int64_t J0, const BatchArrays& A, double* sY) {
  const int M = P.M, K = P.K;
  const int64_t nd = P.g.ndof;
  const int64_t J = J0 + threadIdx.x;
  const bool on = J < nd;
  const double* Wp = A.W + P.oW;
  double W[KC];
#pragma unroll
  for (int k = 0; k < KC; ++k) W[k] = (on && k < K) ? Wp[(int64_t)k * nd + J] : 0.0;
  const double E = on ? A.coefF[P.oCF + J] : 0.0;
  for (int n = 0; n < P.N; ++n) {
    const double* Yn = A.AF + P.oAF + (int64_t)n * M * K;
    double c = on ? A.U[P.oU + (int64_t)n * nd + J] : 0.0;
    for (int m0 = 0; m0 < M; m0 += P.mchunk) {
      const int mc = min(P.mchunk, M - m0);
      __syncthreads();
      b_stage_rows<double, KC>(Yn, K, m0, mc, sY);
      __syncthreads();
      if (on) {
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
    if (on) A.Fbar[P.oS + (int64_t)n * nd + J] = c;
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
    if (!active[f.p]) continue;  // uniform over the CTA
    const BProb& P = probs[f.p];
    if constexpr (PREC == PE_MIXED) {
      b_fine_mixed_item<KC, batch_mixed_mpt(KC)>(P, f.J0, A, reinterpret_cast<float*>(smem_d));
    } else {
      b_fine_f64_item<KC>(P, f.J0, A, smem_d);
    }
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
