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

template <int R>
__global__ void __launch_bounds__(256) fine_f64_kernel(Geom g, int M, int q, int mchunk,
                                                       const double* __restrict__ axisF,
                                                       const double* __restrict__ AF,
                                                       const double* __restrict__ coefF,
                                                       const double* __restrict__ U, double* __restrict__ Fbar) {
  extern __shared__ double sA[];
  const int n = blockIdx.y;
  const int64_t nd = g.ndof;
  const int64_t J = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = J < nd;
  double P[R];
  double b[PE_MAX_S];
  double E = 0.0, c = 0.0;
  if (active) {
    load_P<R, double>(g, J, axisF, P);
    E = coefF[J];
#pragma unroll
    for (int i = 0; i < PE_MAX_S; ++i)
      if (i < q) b[i] = coefF[(1 + i) * nd + J];
    c = U[(int64_t)n * nd + J];
  }
  const int per_m = q * R;
  const double* An = AF + (int64_t)n * M * per_m;
  for (int m0 = 0; m0 < M; m0 += mchunk) {
    const int mc = min(mchunk, M - m0);
    __syncthreads();
    for (int t = threadIdx.x; t < mc * per_m; t += blockDim.x) sA[t] = An[(int64_t)m0 * per_m + t];
    __syncthreads();
    if (active) {
      for (int m = 0; m < mc; ++m) {
        double acc = 0.0;
#pragma unroll
        for (int i = 0; i < PE_MAX_S; ++i) {
          if (i < q) {
            const double* a = sA + (m * q + i) * R;
            double gi = 0.0;
#pragma unroll
            for (int r = 0; r < R; ++r) gi = fma(a[r], P[r], gi);
            acc = fma(b[i], gi, acc);
          }
        }
        c = fma(E, c, acc);
      }
    }
  }
  if (active) Fbar[(int64_t)n * nd + J] = c;
}

// MPT modes per thread (threadIdx.x + k * 256 within the CTA's 256*MPT modes, so
// every global access stays coalesced); each float4 broadcast load of four time
// factors feeds 4*MPT FMAs.  Rows of the staged table are padded to R4 floats.
template <int R, int MPT>
__global__ void __launch_bounds__(256) fine_mixed_kernel(Geom g, int M, int q, int mchunk,
                                                         const float* __restrict__ axisF32,
                                                         const float* __restrict__ AF32,
                                                         const float* __restrict__ coefF32,
                                                         const double* __restrict__ coefF,
                                                         const double* __restrict__ U, double* __restrict__ Fbar) {
  constexpr int R4 = (R + 3) / 4 * 4;
  extern __shared__ __align__(16) float sAf[];
  const int n = blockIdx.y;
  const int64_t nd = g.ndof;
  const int64_t base = (int64_t)blockIdx.x * (256 * MPT) + threadIdx.x;
  float P[MPT][R];
  float b[MPT][PE_MAX_S];
  float eh[MPT], el[MPT], w[MPT];
#pragma unroll
  for (int k = 0; k < MPT; ++k) {
    const int64_t J = base + 256 * k;
    eh[k] = 0.f;
    el[k] = 0.f;
    w[k] = 0.f;
#pragma unroll
    for (int r = 0; r < R; ++r) P[k][r] = 0.f;
#pragma unroll
    for (int i = 0; i < PE_MAX_S; ++i) b[k][i] = 0.f;
    if (J < nd) {
      load_P<R, float>(g, J, axisF32, P[k]);
      eh[k] = coefF32[J];
      el[k] = coefF32[nd + J];
#pragma unroll
      for (int i = 0; i < PE_MAX_S; ++i)
        if (i < q) b[k][i] = coefF32[(2 + i) * nd + J];
    }
  }
  const int per_m = q * R;
  const float* An = AF32 + (int64_t)n * M * per_m;
  for (int m0 = 0; m0 < M; m0 += mchunk) {
    const int mc = min(mchunk, M - m0);
    __syncthreads();
    for (int t = threadIdx.x; t < mc * q * R4; t += blockDim.x) {
      const int row = t / R4, r = t - row * R4;
      sAf[t] = r < R ? An[((int64_t)m0 * q + row) * R + r] : 0.f;
    }
    __syncthreads();
    for (int m = 0; m < mc; ++m) {
      float acc[MPT];
#pragma unroll
      for (int k = 0; k < MPT; ++k) acc[k] = 0.f;
#pragma unroll
      for (int i = 0; i < PE_MAX_S; ++i) {
        if (i < q) {
          const float4* a4 = reinterpret_cast<const float4*>(sAf + (m * q + i) * R4);
          float gk[MPT];
#pragma unroll
          for (int k = 0; k < MPT; ++k) gk[k] = 0.f;
#pragma unroll
          for (int c4 = 0; c4 < R4 / 4; ++c4) {
            const float4 v = a4[c4];
            const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              if (4 * c4 + e < R) {
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
  const int64_t off = (int64_t)n * nd;
  const double* EM = coefF + (int64_t)(q + 1) * nd;
#pragma unroll
  for (int k = 0; k < MPT; ++k) {
    const int64_t J = base + 256 * k;
    if (J < nd) Fbar[off + J] = fma(EM[J], U[off + J], (double)w[k]);
  }
}

inline int pick_mchunk(int M, int per_m, size_t elem) {
  const size_t budget = 48 * 1024;
  int mc = (int)(budget / (elem * (size_t)per_m));
  if (mc < 1) mc = 1;
  return mc < M ? mc : M;
}

}  // namespace

template <int R>
pe_status fine_launch(pe_ctx* c, int precision) {
  const int per_m = c->q * R;
  const int threads = 256;
  if (precision == PE_MIXED) {
    constexpr int MPT = R <= 16 ? 4 : 2;
    constexpr int R4 = (R + 3) / 4 * 4;
    const int mc = pick_mchunk(c->M, c->q * R4, sizeof(float));
    const int64_t per_cta = 256 * MPT;
    dim3 grid((unsigned)((c->g.ndof + per_cta - 1) / per_cta), c->N);
    fine_mixed_kernel<R, MPT><<<grid, threads, sizeof(float) * mc * c->q * R4, c->stream>>>(
        c->g, c->M, c->q, mc, c->axisF32, c->AF32, c->coefF32, c->coefF, c->U, c->Fbar);
  } else {
    const int mc = pick_mchunk(c->M, per_m, sizeof(double));
    dim3 grid((unsigned)((c->g.ndof + threads - 1) / threads), c->N);
    fine_f64_kernel<R><<<grid, threads, sizeof(double) * mc * per_m, c->stream>>>(
        c->g, c->M, c->q, mc, c->axisF, c->AF, c->coefF, c->U, c->Fbar);
  }
  c->launches += 1;
  PE_CUDA_TRY(cudaGetLastError());
  return PE_OK;
}
