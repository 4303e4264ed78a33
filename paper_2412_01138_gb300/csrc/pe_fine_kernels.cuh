// Fine propagator F^M of Algorithm 1 from every slice start at once (the
// parallel part of each Parareal iteration), Eq. (1-7) applied M times:
//   c <- E_F c + sum_{i<q} (dt b_i) ghat_J(T_n + (m + c_i) dt),  m = 0..M-1,
//   ghat_J(t) = sum_r A_r(t) P_{r,J}.
// One CTA owns one slice n and 256 (float64) or 512 (mixed) consecutive modes.
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

template <int R>
__global__ void __launch_bounds__(256) fine_mixed_kernel(Geom g, int M, int q, int mchunk,
                                                         const float* __restrict__ axisF32,
                                                         const float* __restrict__ AF32,
                                                         const float* __restrict__ coefF32,
                                                         const double* __restrict__ coefF,
                                                         const double* __restrict__ U, double* __restrict__ Fbar) {
  extern __shared__ float sAf[];
  const int n = blockIdx.y;
  const int64_t nd = g.ndof;
  const int64_t J0 = 2 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x);
  const int64_t J1 = J0 + 1;
  const bool a0 = J0 < nd, a1 = J1 < nd;
  float P0[R], P1[R];
  float b0[PE_MAX_S], b1[PE_MAX_S];
  float eh0 = 0.f, el0 = 0.f, eh1 = 0.f, el1 = 0.f;
#pragma unroll
  for (int r = 0; r < R; ++r) { P0[r] = 0.f; P1[r] = 0.f; }
#pragma unroll
  for (int i = 0; i < PE_MAX_S; ++i) { b0[i] = 0.f; b1[i] = 0.f; }
  if (a0) {
    load_P<R, float>(g, J0, axisF32, P0);
    eh0 = coefF32[J0];
    el0 = coefF32[nd + J0];
#pragma unroll
    for (int i = 0; i < PE_MAX_S; ++i)
      if (i < q) b0[i] = coefF32[(2 + i) * nd + J0];
  }
  if (a1) {
    load_P<R, float>(g, J1, axisF32, P1);
    eh1 = coefF32[J1];
    el1 = coefF32[nd + J1];
#pragma unroll
    for (int i = 0; i < PE_MAX_S; ++i)
      if (i < q) b1[i] = coefF32[(2 + i) * nd + J1];
  }
  float w0 = 0.f, w1 = 0.f;
  const int per_m = q * R;
  const float* An = AF32 + (int64_t)n * M * per_m;
  for (int m0 = 0; m0 < M; m0 += mchunk) {
    const int mc = min(mchunk, M - m0);
    __syncthreads();
    for (int t = threadIdx.x; t < mc * per_m; t += blockDim.x) sAf[t] = An[(int64_t)m0 * per_m + t];
    __syncthreads();
    for (int m = 0; m < mc; ++m) {
      float acc0 = 0.f, acc1 = 0.f;
#pragma unroll
      for (int i = 0; i < PE_MAX_S; ++i) {
        if (i < q) {
          const float* a = sAf + (m * q + i) * R;
          float g0 = 0.f, g1 = 0.f;
#pragma unroll
          for (int r = 0; r < R; ++r) {
            const float av = a[r];
            g0 = fmaf(av, P0[r], g0);
            g1 = fmaf(av, P1[r], g1);
          }
          acc0 = fmaf(b0[i], g0, acc0);
          acc1 = fmaf(b1[i], g1, acc1);
        }
      }
      w0 = fmaf(eh0, w0, fmaf(el0, w0, acc0));
      w1 = fmaf(eh1, w1, fmaf(el1, w1, acc1));
    }
  }
  const int64_t off = (int64_t)n * nd;
  const double* EM = coefF + (int64_t)(q + 1) * nd;
  if (a0) Fbar[off + J0] = fma(EM[J0], U[off + J0], (double)w0);
  if (a1) Fbar[off + J1] = fma(EM[J1], U[off + J1], (double)w1);
}

inline int pick_mchunk(int M, int per_m, size_t elem) {
  const size_t budget = 48 * 1024;
  int mc = (int)(budget / (elem * (size_t)per_m));
  if (mc < 1) mc = 1;
  return mc < M ? mc : M;
}

}  // namespace

template <int R>
pe_status fine_launch(pe_ctx* c) {
  const int per_m = c->q * R;
    if (c->precision == PE_MIXED) {
      const int mc = pick_mchunk(c->M, per_m, sizeof(float));
      const int threads = 256;
      const int64_t pairs = (c->g.ndof + 1) / 2;
      dim3 grid((unsigned)((pairs + threads - 1) / threads), c->N);
      fine_mixed_kernel<R><<<grid, threads, sizeof(float) * mc * per_m, c->stream>>>(
          c->g, c->M, c->q, mc, c->axisF32, c->AF32, c->coefF32, c->coefF, c->U, c->Fbar);
    } else {
      const int mc = pick_mchunk(c->M, per_m, sizeof(double));
      const int threads = 256;
      dim3 grid((unsigned)((c->g.ndof + threads - 1) / threads), c->N);
      fine_f64_kernel<R><<<grid, threads, sizeof(double) * mc * per_m, c->stream>>>(
          c->g, c->M, c->q, mc, c->axisF, c->AF, c->coefF, c->U, c->Fbar);
    }
  c->launches += 1;
  PE_CUDA_TRY(cudaGetLastError());
  return PE_OK;
}
