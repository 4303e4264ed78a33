// Persistent fine-propagator kernel of the batched solver: CTAs pull
// (problem, slice, mode-tile) items from an atomic counter and run the tile
// body specialised for the problem's number of forcing terms R.  Each tile
// is Eq. (1-7) applied M times, the stage forcing summed per stage:
//   c <- E_F c + sum_{i<q} (dt b_i) sum_r A_r(T_n + (m + c_i) dt) P_{r,J}.
// The slice's time factors for all M*q stage times are staged in shared
// memory (warp-wide broadcasts); P, E_F, b_i stay in registers.
// PE_MIXED: F^M(v) = E_F^M v (float64) + F^M(0) (float32, E_F as hi + lo).
#pragma once
#include "pe_batch.h"

namespace {

// Operands of one fine-propagator tile: one slice n of one problem, blockDim.x*MPT
// modes starting at `base` (thread t owns base + t + k*blockDim.x, k < MPT, so every
// global access stays coalesced).
struct BFineTile {
  Geom g;
  int M, q, mchunk;
  int64_t base;
  const float* axisF32;   // per-axis modal factors (float)
  const double* axisF;    // per-axis modal factors (double)
  const float* AFn32;     // time factors of slice n [M][q][R] (float)
  const double* AFn;      // time factors of slice n [M][q][R] (double)
  const float* coefF32;   // E_hi, E_lo, dt*b_i  (rows of ndof)
  const double* coefF;    // E, dt*b_i, exp(-lam M dt) (rows of ndof)
  const double* Un;       // U^n
  double* Fn;             // F^M(U^n)
};

// P[r] = prod_a axisF[R*off[a] + r*n_a + j_a] for r < R, zero for R <= r < RC.
template <int RC, typename T>
__device__ __forceinline__ void b_load_P_rt(const Geom& g, int64_t J, const T* __restrict__ axisF, int R, T* P) {
  int j[PE_MAX_D];
  unflatten(g, J, j);
#pragma unroll
  for (int r = 0; r < RC; ++r) {
    T v = T(0);
    if (r < R) {
      v = axisF[(int64_t)R * g.off[0] + (int64_t)r * g.n[0] + j[0]];
      for (int a = 1; a < g.d; ++a) v *= axisF[(int64_t)R * g.off[a] + (int64_t)r * g.n[a] + j[a]];
    }
    P[r] = v;
  }
}

// Mixed precision, R <= RC forcing terms (RC a multiple of 4): each float4 broadcast
// load of four time factors feeds up to 4*MPT FMAs; staged rows are zero-padded to
// RC.  RX > 0: R == RX is known at compile time and the padding lanes are skipped.
template <int RC, int MPT, int RX = 0>
__device__ __forceinline__ void b_fine_mixed_tile(const BFineTile& a, int R, float* sAf) {
  static_assert(RC % 4 == 0, "RC must be a multiple of 4");
  const Geom& g = a.g;
  const int q = a.q, M = a.M, B = blockDim.x;
  const int64_t nd = g.ndof;
  const int64_t base = a.base + threadIdx.x;
  float P[MPT][RC];
  float b[MPT][PE_MAX_S];
  float eh[MPT], el[MPT], w[MPT];
#pragma unroll
  for (int k = 0; k < MPT; ++k) {
    const int64_t J = base + (int64_t)B * k;
    eh[k] = 0.f;
    el[k] = 0.f;
    w[k] = 0.f;
#pragma unroll
    for (int r = 0; r < RC; ++r) P[k][r] = 0.f;
#pragma unroll
    for (int i = 0; i < PE_MAX_S; ++i) b[k][i] = 0.f;
    if (J < nd) {
      b_load_P_rt<RC, float>(g, J, a.axisF32, R, P[k]);
      eh[k] = a.coefF32[J];
      el[k] = a.coefF32[nd + J];
#pragma unroll
      for (int i = 0; i < PE_MAX_S; ++i)
        if (i < q) b[k][i] = a.coefF32[(2 + i) * nd + J];
    }
  }
  for (int m0 = 0; m0 < M; m0 += a.mchunk) {
    const int mc = min(a.mchunk, M - m0);
    __syncthreads();
    for (int t = threadIdx.x; t < mc * q * RC; t += B) {
      const int row = t / RC, r = t - row * RC;
      sAf[t] = r < R ? a.AFn32[((int64_t)m0 * q + row) * R + r] : 0.f;
    }
    __syncthreads();
    for (int m = 0; m < mc; ++m) {
      float acc[MPT];
#pragma unroll
      for (int k = 0; k < MPT; ++k) acc[k] = 0.f;
#pragma unroll
      for (int i = 0; i < PE_MAX_S; ++i) {
        if (i < q) {
          const float4* a4 = reinterpret_cast<const float4*>(sAf + (m * q + i) * RC);
          float gk[MPT];
#pragma unroll
          for (int k = 0; k < MPT; ++k) gk[k] = 0.f;
#pragma unroll
          for (int c4 = 0; c4 < RC / 4; ++c4) {
            const float4 v = a4[c4];
            const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              if (RX == 0 || 4 * c4 + e < RX) {
#pragma unroll
                for (int k = 0; k < MPT; ++k) gk[k] = fmaf(vv[e], P[k][4 * c4 + e], gk[k]);
              }
            }
          }
#pragma unroll
          for (int k = 0; k < MPT; ++k) acc[k] = fmaf(b[k][i], gk[k], acc[k]);
        }
      }
#pragma unroll
      for (int k = 0; k < MPT; ++k) w[k] = fmaf(eh[k], w[k], fmaf(el[k], w[k], acc[k]));
    }
  }
  const double* EM = a.coefF + (int64_t)(q + 1) * nd;
#pragma unroll
  for (int k = 0; k < MPT; ++k) {
    const int64_t J = base + (int64_t)B * k;
    if (J < nd) a.Fn[J] = fma(EM[J], a.Un[J], (double)w[k]);
  }
}

// Float64, R <= RC forcing terms: one mode per thread, the plain recurrence of Eq. (1-7).
template <int RC>
__device__ __forceinline__ void b_fine_f64_tile(const BFineTile& a, int R, double* sA) {
  const Geom& g = a.g;
  const int q = a.q, M = a.M, B = blockDim.x;
  const int64_t nd = g.ndof;
  const int64_t J = a.base + threadIdx.x;
  const bool active = J < nd;
  double P[RC];
  double b[PE_MAX_S];
  double E = 0.0, c = 0.0;
  if (active) {
    b_load_P_rt<RC, double>(g, J, a.axisF, R, P);
    E = a.coefF[J];
#pragma unroll
    for (int i = 0; i < PE_MAX_S; ++i)
      if (i < q) b[i] = a.coefF[(1 + i) * nd + J];
    c = a.Un[J];
  }
  for (int m0 = 0; m0 < M; m0 += a.mchunk) {
    const int mc = min(a.mchunk, M - m0);
    __syncthreads();
    for (int t = threadIdx.x; t < mc * q * RC; t += B) {
      const int row = t / RC, r = t - row * RC;
      sA[t] = r < R ? a.AFn[((int64_t)m0 * q + row) * R + r] : 0.0;
    }
    __syncthreads();
    if (active) {
      for (int m = 0; m < mc; ++m) {
        double acc = 0.0;
#pragma unroll
        for (int i = 0; i < PE_MAX_S; ++i) {
          if (i < q) {
            const double* ap = sA + (m * q + i) * RC;
            double gi = 0.0;
#pragma unroll
            for (int r = 0; r < RC; ++r) gi = fma(ap[r], P[r], gi);
            acc = fma(b[i], gi, acc);
          }
        }
        c = fma(E, c, acc);
      }
    }
  }
  if (active) a.Fn[J] = c;
}


// Tile bodies are compiled for R rounded up to a multiple of 4 (RC = 4..20); the
// padding terms carry zero weights.
template <int PREC, int RC>
__device__ __forceinline__ void run_tile(const BFineTile& t, int R, double* smem) {
  if constexpr (PREC == PE_MIXED) {
    b_fine_mixed_tile<RC, (RC <= 16 ? 4 : 2)>(t, R, reinterpret_cast<float*>(smem));
  } else {
    b_fine_f64_tile<RC>(t, R, smem);
  }
}

template <int PREC>
__device__ __forceinline__ void dispatch_tile(int R, const BFineTile& t, double* smem) {
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
    BFineTile t{};
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
