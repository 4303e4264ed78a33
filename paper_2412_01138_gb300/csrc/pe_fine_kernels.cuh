// Fine propagator F^M of Algorithm 1 from every slice start at once (the
// parallel part of each Parareal iteration), Eq. (1-7) applied M times:
//   c <- E_F c + sum_{i<q} (dt b_i) ghat_J(T_n + (m + c_i) dt),  m = 0..M-1,
//   ghat_J(t) = sum_r A_r(t) P_{r,J}.
// One CTA owns one slice n and 256 (float64) or 256*MPT (mixed) modes.
// The slice's time factors A_r(t) for all M*q stage times are staged in
// shared memory and read as warp-wide broadcasts; the per-mode weights
// P_{r,J}, E_F and b_i stay in registers for the whole slice.  The kernel
// is bound by the FMA rate: q(R+1)+1 FMAs per mode and substep.
//
// PE_MIXED splits F^M(v) = E_F^M v + F^M(0) (the step is affine in v): the
// homogeneous part uses the float64 table value exp(-lam M dt), and the
// forced part runs the full M-substep recurrence in float32 from zero with
// E_F carried as a float32 hi + lo pair, so that rounding E_F does not
// compound over the M substeps.
#pragma once
#include "pe_internal.h"
#include "pe_sweep_common.cuh"

namespace {

// Operands of one fine-propagator tile: one slice n of one problem, blockDim.x*MPT
// modes starting at `base` (thread t owns base + t + k*blockDim.x, k < MPT, so every
// global access stays coalesced).
struct FineTile {
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
__device__ __forceinline__ void load_P_rt(const Geom& g, int64_t J, const T* __restrict__ axisF, int R, T* P) {
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
__device__ __forceinline__ void fine_mixed_tile(const FineTile& a, int R, float* sAf) {
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
      load_P_rt<RC, float>(g, J, a.axisF32, R, P[k]);
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
__device__ __forceinline__ void fine_f64_tile(const FineTile& a, int R, double* sA) {
  const Geom& g = a.g;
  const int q = a.q, M = a.M, B = blockDim.x;
  const int64_t nd = g.ndof;
  const int64_t J = a.base + threadIdx.x;
  const bool active = J < nd;
  double P[RC];
  double b[PE_MAX_S];
  double E = 0.0, c = 0.0;
  if (active) {
    load_P_rt<RC, double>(g, J, a.axisF, R, P);
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

template <int R, int MPT>
__global__ void __launch_bounds__(256) fine_mixed_kernel(FineTile t, int64_t slice_stride_af) {
  constexpr int RC = (R + 3) / 4 * 4;
  extern __shared__ __align__(16) float sAf[];
  const int n = blockIdx.y;
  const int64_t nd = t.g.ndof;
  t.base = (int64_t)blockIdx.x * (blockDim.x * MPT);
  t.AFn32 += (int64_t)n * slice_stride_af;
  t.Un += (int64_t)n * nd;
  t.Fn += (int64_t)n * nd;
  fine_mixed_tile<RC, MPT, R>(t, R, sAf);
}

template <int R>
__global__ void __launch_bounds__(256) fine_f64_kernel(FineTile t, int64_t slice_stride_af) {
  extern __shared__ __align__(16) double sA[];
  const int n = blockIdx.y;
  const int64_t nd = t.g.ndof;
  t.base = (int64_t)blockIdx.x * blockDim.x;
  t.AFn += (int64_t)n * slice_stride_af;
  t.Un += (int64_t)n * nd;
  t.Fn += (int64_t)n * nd;
  fine_f64_tile<R>(t, R, sA);
}

}  // namespace


template <int R>
pe_status fine_launch(pe_ctx* c, int precision) {
  const int threads = 256;
  FineTile t{};
  t.g = c->g;
  t.M = c->M;
  t.q = c->q;
  t.axisF32 = c->axisF32;
  t.axisF = c->axisF;
  t.AFn32 = c->AF32;
  t.AFn = c->AF;
  t.coefF32 = c->coefF32;
  t.coefF = c->coefF;
  t.Un = c->U;
  t.Fn = c->Fbar;
  const int64_t stride = (int64_t)c->M * c->q * R;
  if (precision == PE_MIXED) {
    constexpr int MPT = R <= 16 ? 4 : 2;
    constexpr int R4 = (R + 3) / 4 * 4;
    t.mchunk = pick_mchunk(c->M, c->q * R4, sizeof(float));
    const int64_t per_cta = (int64_t)threads * MPT;
    dim3 grid((unsigned)((c->g.ndof + per_cta - 1) / per_cta), c->N);
    fine_mixed_kernel<R, MPT><<<grid, threads, sizeof(float) * t.mchunk * c->q * R4, c->stream>>>(t, stride);
  } else {
    t.mchunk = pick_mchunk(c->M, c->q * R, sizeof(double));
    dim3 grid((unsigned)((c->g.ndof + threads - 1) / threads), c->N);
    fine_f64_kernel<R><<<grid, threads, sizeof(double) * t.mchunk * c->q * R, c->stream>>>(t, stride);
  }
  c->launches += 1;
  PE_CUDA_TRY(cudaGetLastError());
  return PE_OK;
}
