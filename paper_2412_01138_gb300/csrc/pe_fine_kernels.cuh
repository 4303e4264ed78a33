// Fine propagator F^M of Algorithm 1 from every slice start at once (the
// parallel part of each Parareal iteration), Eq. (1-7) applied M times:
//   c <- E_F c + sum_{i<q} (dt b_i) ghat_J(T_n + (m + c_i) dt),  m = 0..M-1,
//   ghat_J(t) = sum_r A_r(t) P_{r,J}.
//
// Stage contraction.  Every time factor of a separable source is shift
// invariant: exp(a(t+s)) = exp(at) exp(as) and
// sin(w(t+s)+phi) = sin(wt+phi) cos(ws) + cos(wt+phi) sin(ws).  Writing
// A_r(t + s) = sum_k Y_{r,k}(t) Z_{r,k}(s) (one column k for an exponential,
// two for a sinusoid; K columns in all), the stage sum of one substep is
//   sum_i dt b_i ghat_J(t_m + c_i dt) = sum_k Y_k(t_m) W_{k,J},
//   W_{k,J} = P_{r(k),J} sum_i dt b_i(-lam_J dt) Z_k(c_i dt),
// with the per-mode weights W tabulated once per problem (stage_weights_kernel)
// and Y_k at the substep starts t_m = T_n + m dt tabulated per slice.  This is
// the same sum, regrouped: every substep is still taken, at K + 1 FMAs per mode
// instead of q(R + 1) + 1.
//
// One CTA owns one slice n and 256 (float64) or 256*MPT (mixed) modes.  The
// slice's Y_k(t_m) are staged in shared memory and read as warp-wide broadcasts;
// W, E_F stay in registers for the whole slice.  The float64 kernel is bound
// by the FP64 FMA rate.
//
// PE_MIXED splits F^M(v) = E_F^M v + F^M(0) (the step is affine in v): the
// homogeneous part uses the float64 table value exp(-lam M dt), and the
// forced part runs the full M-substep recurrence in float32 from zero with
// E_F carried as a float32 hi + lo pair, so that rounding E_F does not
// compound over the M substeps.
#pragma once
#include "pe_internal.h"

namespace {

// Operands of one fine-propagator tile: one slice n, blockDim.x*MPT modes
// starting at `base` (thread t owns base + t + k*blockDim.x, k < MPT, so every
// global access stays coalesced).
struct FineTile {
  int64_t ndof;
  int M, mchunk;
  int64_t base;
  const float* W32;       // stage weights [K][ndof] (float)
  const double* W;        // stage weights [K][ndof] (double)
  const float* Yn32;      // substep time factors of slice n [M][K] (float)
  const double* Yn;       // substep time factors of slice n [M][K] (double)
  const float* coefF32;   // E_hi, E_lo (rows of ndof)
  const double* coefF;    // E, dt*b_i, exp(-lam M dt) (rows of ndof)
  int q;
  int from_zero;          // 1: propagate 0 instead of U^n (the forced part F^M(0))
  const double* Un;       // U^n
  double* Fn;             // F^M(U^n), or F^M(0) when from_zero
};

// Modes per thread of the mixed tile: as many as the registers allow (W takes MPT * K).
__host__ __device__ constexpr int fine_mixed_mpt(int K) { return K <= 17 ? 6 : (K <= 24 ? 4 : (K <= 40 ? 2 : 1)); }

// Mixed precision, K columns stored as KC = roundup(K, 4) floats per substep
// (zero padding, [N][M][KC] in the float time table) so that each float4
// broadcast load feeds 4*MPT FMAs; the padding lanes are skipped.
//
// W and the hi/lo E_F of the MPT modes base + k*blockDim.x (zero past the end).
template <int K, int MPT>
__device__ __forceinline__ void mixed_load_weights(const FineTile& a, int64_t base, float (&W)[MPT][K],
                                                   float (&eh)[MPT], float (&el)[MPT]) {
  const int64_t nd = a.ndof;
#pragma unroll
  for (int k = 0; k < MPT; ++k) {
    const int64_t J = base + (int64_t)blockDim.x * k;
    eh[k] = 0.f;
    el[k] = 0.f;
#pragma unroll
    for (int c = 0; c < K; ++c) W[k][c] = 0.f;
    if (J < nd) {
#pragma unroll
      for (int c = 0; c < K; ++c) W[k][c] = a.W32[(int64_t)c * nd + J];
      eh[k] = a.coefF32[J];
      el[k] = a.coefF32[nd + J];
    }
  }
}

// mc substeps of the float32 forced recurrence w <- E_F w + sum_k Y_k(t_m) W_k
// from the staged time factors sY[m*KC + k].
template <int K, int MPT>
__device__ __forceinline__ void mixed_substeps(const float* sY, int mc, const float (&W)[MPT][K],
                                               const float (&eh)[MPT], const float (&el)[MPT], float (&w)[MPT]) {
  constexpr int KC = (K + 3) / 4 * 4;
  // four substeps per trip: the later substeps' broadcast loads and FMA chains are
  // independent of the earlier ones' recurrence, so they overlap its latency
#pragma unroll 4
  for (int m = 0; m < mc; ++m) {
    const float4* y4 = reinterpret_cast<const float4*>(sY + m * KC);
    float acc[MPT];
#pragma unroll
    for (int k = 0; k < MPT; ++k) acc[k] = 0.f;
#pragma unroll
    for (int c4 = 0; c4 < KC / 4; ++c4) {
      const float4 v = y4[c4];
      const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        if (4 * c4 + e < K) {
#pragma unroll
          for (int k = 0; k < MPT; ++k) acc[k] = fmaf(vv[e], W[k][4 * c4 + e], acc[k]);
        }
      }
    }
#pragma unroll
    for (int k = 0; k < MPT; ++k) w[k] = fmaf(eh[k], w[k], fmaf(el[k], w[k], acc[k]));
  }
}

// F^M(U^n) = exp(-lam M dt) U^n + w (float64), or w alone when from_zero.
template <int MPT>
__device__ __forceinline__ void mixed_store(const FineTile& a, int64_t base, const double* Un, double* Fn,
                                            const float (&w)[MPT]) {
  const int64_t nd = a.ndof;
  const double* EM = a.coefF + (int64_t)(a.q + 1) * nd;
#pragma unroll
  for (int k = 0; k < MPT; ++k) {
    const int64_t J = base + (int64_t)blockDim.x * k;
    if (J < nd) Fn[J] = a.from_zero ? (double)w[k] : fma(EM[J], Un[J], (double)w[k]);
  }
}

template <int K, int MPT>
__device__ __forceinline__ void fine_mixed_tile(const FineTile& a, float* sY) {
  constexpr int KC = (K + 3) / 4 * 4;
  const int M = a.M, B = blockDim.x;
  const int64_t base = a.base + threadIdx.x;
  float W[MPT][K], eh[MPT], el[MPT], w[MPT];
  mixed_load_weights<K, MPT>(a, base, W, eh, el);
#pragma unroll
  for (int k = 0; k < MPT; ++k) w[k] = 0.f;
  for (int m0 = 0; m0 < M; m0 += a.mchunk) {
    const int mc = min(a.mchunk, M - m0);
    __syncthreads();
    for (int t = threadIdx.x; t < mc * KC; t += B) sY[t] = a.Yn32[(int64_t)m0 * KC + t];
    __syncthreads();
    mixed_substeps<K, MPT>(sY, mc, W, eh, el, w);
  }
  mixed_store<MPT>(a, base, a.Un, a.Fn, w);
}

// 16-byte asynchronous global -> shared copies (cp.async, waited on per group).
__device__ __forceinline__ void y_copy16(void* dst_smem, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void y_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int PENDING>
__device__ __forceinline__ void y_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(PENDING) : "memory"); }

// Persistent form of the mixed kernel.  The work items are (mode tile, slice)
// pairs, tile-major, I = tiles * N of them; CTA b runs the contiguous range
// [b I / G, (b+1) I / G) of a grid of G resident CTAs.  W and the hi/lo E_F stay
// in registers until the range crosses a tile boundary (once or twice per CTA
// instead of once per slice), and the next item's [M][KC] time factors are staged
// by cp.async into the other half of a double buffer while the current item runs.
//
// 128 threads per CTA; MPT = 6 (K <= 17) at three CTAs per SM, otherwise four CTAs per SM
// (at most 128 registers).
constexpr int kMixedThreads = 128;
template <int K, int MPT>
__global__ void __launch_bounds__(kMixedThreads, MPT >= 6 ? 3 : 4)
    fine_mixed_persistent_kernel(FineTile t, int N, int64_t n_items) {
  pdl_wait();
  constexpr int KC = (K + 3) / 4 * 4;
  extern __shared__ __align__(16) float sYb[];
  const int B = kMixedThreads;
  const int64_t nd = t.ndof;
  const int slab = t.M * KC;  // floats per slice, a multiple of 4
  const int64_t i0 = (int64_t)blockIdx.x * n_items / gridDim.x;
  const int64_t i1 = (int64_t)(blockIdx.x + 1) * n_items / gridDim.x;
  auto stage = [&](int64_t i, int buf) {
    const float4* src = reinterpret_cast<const float4*>(t.Yn32 + (i % N) * slab);
    float4* dst = reinterpret_cast<float4*>(sYb + buf * slab);
    for (int e = threadIdx.x; e < slab / 4; e += B) y_copy16(dst + e, src + e);
    y_commit();
  };
  float W[MPT][K], eh[MPT], el[MPT];
  int64_t loaded = -1;
  if (i0 < i1) stage(i0, 0);
  for (int64_t i = i0; i < i1; ++i) {
    const int buf = (int)((i - i0) & 1);
    const int64_t tile = i / N, n = i - tile * N;
    // the other buffer was last read by the previous item, which ended with a barrier
    if (i + 1 < i1) stage(i + 1, buf ^ 1);
    const int64_t base = tile * (int64_t)(B * MPT) + threadIdx.x;
    if (tile != loaded) {
      mixed_load_weights<K, MPT>(t, base, W, eh, el);
      loaded = tile;
    }
    if (i + 1 < i1) y_wait<1>();
    else y_wait<0>();
    __syncthreads();
    float w[MPT];
#pragma unroll
    for (int k = 0; k < MPT; ++k) w[k] = 0.f;
    mixed_substeps<K, MPT>(sYb + buf * slab, t.M, W, eh, el, w);
    mixed_store<MPT>(t, base, t.Un + n * nd, t.Fn + n * nd, w);
    __syncthreads();
  }
}

// Float64: one mode per thread, the contracted recurrence c <- E c + sum_k Y_k W_k.
template <int K>
__device__ __forceinline__ void fine_f64_tile(const FineTile& a, double* sY) {
  const int M = a.M, B = blockDim.x;
  const int64_t nd = a.ndof;
  const int64_t J = a.base + threadIdx.x;
  const bool active = J < nd;
  double W[K];
  double E = 0.0, c = 0.0;
#pragma unroll
  for (int k = 0; k < K; ++k) W[k] = 0.0;
  if (active) {
#pragma unroll
    for (int k = 0; k < K; ++k) W[k] = a.W[(int64_t)k * nd + J];
    E = a.coefF[J];
    c = a.from_zero ? 0.0 : a.Un[J];
  }
  for (int m0 = 0; m0 < M; m0 += a.mchunk) {
    const int mc = min(a.mchunk, M - m0);
    __syncthreads();
    for (int t = threadIdx.x; t < mc * K; t += B) sY[t] = a.Yn[(int64_t)m0 * K + t];
    __syncthreads();
    if (active) {
      for (int m = 0; m < mc; ++m) {
        const double* yp = sY + m * K;
        double acc = 0.0;
#pragma unroll
        for (int k = 0; k < K; ++k) acc = fma(yp[k], W[k], acc);
        c = fma(E, c, acc);
      }
    }
  }
  if (active) a.Fn[J] = c;
}

template <int K, int MPT>
__global__ void __launch_bounds__(256) fine_mixed_kernel(FineTile t, int64_t slice_stride_y) {
  pdl_wait();
  extern __shared__ __align__(16) float sYf[];
  const int n = blockIdx.y;
  const int64_t nd = t.ndof;
  t.base = (int64_t)blockIdx.x * (blockDim.x * MPT);
  t.Yn32 += (int64_t)n * slice_stride_y;
  t.Un += (int64_t)n * nd;
  t.Fn += (int64_t)n * nd;
  fine_mixed_tile<K, MPT>(t, sYf);
}

template <int K>
__global__ void __launch_bounds__(256) fine_f64_kernel(FineTile t, int64_t slice_stride_y) {
  pdl_wait();
  extern __shared__ __align__(16) double sY[];
  const int n = blockIdx.y;
  const int64_t nd = t.ndof;
  t.base = (int64_t)blockIdx.x * blockDim.x;
  t.Yn += (int64_t)n * slice_stride_y;
  t.Un += (int64_t)n * nd;
  t.Fn += (int64_t)n * nd;
  fine_f64_tile<K>(t, sY);
}

}  // namespace


// from_zero: write F^M(0) of every slice to `out` instead of F^M(U^n) to c->Fbar.
template <int K>
pe_status fine_launch(pe_ctx* c, int precision, int from_zero, double* out) {
  const int threads = 256;
  FineTile t{};
  t.ndof = c->g.ndof;
  t.M = c->M;
  t.q = c->q;
  t.W32 = c->Wst32;
  t.W = c->Wst;
  t.Yn32 = c->AF32;
  t.Yn = c->AF;
  t.coefF32 = c->coefF32;
  t.coefF = c->coefF;
  t.from_zero = from_zero;
  t.Un = c->U;
  t.Fn = out;
  if (precision == PE_MIXED) {
    constexpr int MPT = fine_mixed_mpt(K);
    constexpr int KC = (K + 3) / 4 * 4;
    const size_t slab_bytes = sizeof(float) * (size_t)c->M * KC;
    if (2 * slab_bytes <= 48 * 1024) {
      const int64_t per_cta = (int64_t)kMixedThreads * MPT;
      const int64_t tiles = (c->g.ndof + per_cta - 1) / per_cta;
      // persistent: one resident wave of CTAs over the (tile, slice) items
      int dev = 0, sms = 0, occ = 0;
      PE_CUDA_TRY(cudaGetDevice(&dev));
      PE_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
      PE_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fine_mixed_persistent_kernel<K, MPT>,
                                                                kMixedThreads, 2 * slab_bytes));
      if (occ < 1) return pe_fail(PE_EINVAL, "fine sweep: persistent kernel does not fit an SM");
      const int64_t items = tiles * c->N;
      const int64_t grid = items < (int64_t)sms * occ ? items : (int64_t)sms * occ;
      PE_CUDA_TRY(launch_pdl(fine_mixed_persistent_kernel<K, MPT>, dim3((unsigned)grid), dim3(kMixedThreads),
                             2 * slab_bytes, c->stream, t, c->N, items));
    } else {
      const int64_t per_cta = (int64_t)threads * MPT;
      const int64_t tiles = (c->g.ndof + per_cta - 1) / per_cta;
      t.mchunk = pick_mchunk(c->M, KC, sizeof(float));
      dim3 grid((unsigned)tiles, c->N);
      PE_CUDA_TRY(launch_pdl(fine_mixed_kernel<K, MPT>, grid, dim3(threads), sizeof(float) * t.mchunk * KC, c->stream,
                             t, (int64_t)c->M * KC));
    }
  } else {
    t.mchunk = pick_mchunk(c->M, K, sizeof(double));
    dim3 grid((unsigned)((c->g.ndof + threads - 1) / threads), c->N);
    PE_CUDA_TRY(launch_pdl(fine_f64_kernel<K>, grid, dim3(threads), sizeof(double) * t.mchunk * K, c->stream, t,
                           (int64_t)c->M * K));
  }
  c->launches += 1;
  PE_CUDA_TRY(cudaGetLastError());
  return PE_OK;
}
