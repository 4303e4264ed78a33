// Coarse sweep, correction and residual of Algorithm 1 (PEIFE-linear).
//
// In mode space every step of Eq. (1-7) is  c <- E c + sum_i (tau b_i) ghat(t_i)
// with ghat_J(t) = sum_r A_r(t) P_{r,J}, A_r(t) = amp_r time_r(t) and
// P_{r,J} = prod_a axisF[a][r][j_a].  Modes are independent, so one thread owns
// one mode and walks the slices n = 0..N-1 sequentially (the "sequential"
// parts of Algorithm 1 are sequential in n only).
//
//   coarse sweep   U^{n+1,(0)} = G(U^{n,(0)}) = E_G U^n + gG_n, stored G(U^{n,(0)});
//                  the coarse forcing gG_n (independent of the iterate) is kept.
//   correction     U^{n+1,(k+1)} = G(U^{n,(k+1)}) + Fbar^{n+1} - G(U^{n,(k)})
//                  and the float64 sums  sum mu^M_J (U^{new} - U^{old})^2, sum mu^M_J (U^{new})^2.
#include "pe_internal.h"

namespace {

// Coarse forcing of every slice, in parallel over slices: each thread owns one
// mode and SL consecutive slices; its weights P_{r,J} sit in a column of shared
// memory (R x blockDim doubles / floats), so R is a run-time value.  T = double
// on the float64 path; float in the mixed form, where gG only enters through
// G(U^{new}) - G(U^{old}), in which the same stored gG cancels.
template <typename T>
__global__ void __launch_bounds__(256) coarse_forcing_kernel(Geom g, int N, int p, int R, int SL,
                                                            const T* __restrict__ axisF, const T* __restrict__ AG,
                                                            const double* __restrict__ coefG,
                                                            double* __restrict__ gG) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sP = reinterpret_cast<T*>(smem_raw);  // [R][blockDim.x]
  const int64_t J = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (J >= g.ndof) return;
  const int64_t nd = g.ndof;
  const int tid = threadIdx.x, B = blockDim.x;
  int j[PE_MAX_D];
  unflatten(g, J, j);
  for (int r = 0; r < R; ++r) {
    T v = axisF[(int64_t)R * g.off[0] + (int64_t)r * g.n[0] + j[0]];
    for (int a = 1; a < g.d; ++a) v *= axisF[(int64_t)R * g.off[a] + (int64_t)r * g.n[a] + j[a]];
    sP[r * B + tid] = v;
  }
  T b[PE_MAX_S];
#pragma unroll
  for (int i = 0; i < PE_MAX_S; ++i)
    if (i < p) b[i] = (T)coefG[(1 + i) * nd + J];
  const int n0 = blockIdx.y * SL;
  const int n1 = min(N, n0 + SL);
  for (int n = n0; n < n1; ++n) {
    T acc = T(0);
#pragma unroll
    for (int i = 0; i < PE_MAX_S; ++i) {
      if (i < p) {
        const T* a = AG + ((int64_t)n * p + i) * R;
        T gi = T(0);
        for (int r = 0; r < R; ++r) gi = fma(__ldg(a + r), sP[r * B + tid], gi);
        acc = fma(b[i], gi, acc);
      }
    }
    gG[(int64_t)n * nd + J] = (double)acc;
  }
}

// Sequential coarse sweep U^{n+1,(0)} = E_G U^{n,(0)} + gG_n (one thread per mode).
__global__ void __launch_bounds__(256) coarse_recurrence_kernel(Geom g, int N, const double* __restrict__ coefG,
                                                               const double* __restrict__ gG,
                                                               double* __restrict__ U, double* __restrict__ Gold) {
  const int64_t J = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (J >= g.ndof) return;
  const int64_t nd = g.ndof;
  const double E = coefG[J];
  double c = U[J];
  double gn = gG[J];
  for (int n = 0; n < N; ++n) {
    const double gnext = n + 1 < N ? gG[(int64_t)(n + 1) * nd + J] : 0.0;
    c = fma(E, c, gn);
    U[(int64_t)(n + 1) * nd + J] = c;
    Gold[(int64_t)n * nd + J] = c;
    gn = gnext;
  }
}

template <typename T>
__device__ inline T block_sum(T v, T* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  T out = T(0);
  if (threadIdx.x < 32) {
    T x = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : T(0);
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    out = x;
  }
  __syncthreads();
  return out;
}

__global__ void __launch_bounds__(256) correction_kernel(Geom g, int N, const double* __restrict__ muM_axis,
                                                         const double* __restrict__ coefG,
                                                         const double* __restrict__ gG,
                                                         const double* __restrict__ Fbar, double* __restrict__ Gold,
                                                         double* __restrict__ U, double* __restrict__ partials) {
  __shared__ double sh[32];
  const int64_t J = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double sd = 0.0, su = 0.0;
  if (J < g.ndof) {
    const int64_t nd = g.ndof;
    int j[PE_MAX_D];
    unflatten(g, J, j);
    double w = muM_axis[g.off[0] + j[0]];
    for (int a = 1; a < g.d; ++a) w *= muM_axis[g.off[a] + j[a]];
    const double E = coefG[J];
    double unew = U[J];
    // the four streams of slice n+1 are loaded before slice n is combined, so
    // each thread keeps two slices of loads in flight (the recurrence itself only
    // carries unew)
    double g0 = gG[J], f0 = Fbar[J], o0 = Gold[J], u0 = U[nd + J];
    for (int n = 0; n < N; ++n) {
      const int64_t o = (int64_t)n * nd + J;
      double g1 = 0.0, f1 = 0.0, o1 = 0.0, u1 = 0.0;
      if (n + 1 < N) {
        g1 = gG[o + nd];
        f1 = Fbar[o + nd];
        o1 = Gold[o + nd];
        u1 = U[o + 2 * nd];
      }
      const double Gn = fma(E, unew, g0);
      const double nxt = (Gn + f0) - o0;
      Gold[o] = Gn;
      U[o + nd] = nxt;
      const double df = nxt - u0;
      sd = fma(w * df, df, sd);
      su = fma(w * nxt, nxt, su);
      unew = nxt;
      g0 = g1; f0 = f1; o0 = o1; u0 = u1;
    }
  }
  sd = block_sum(sd, sh);
  su = block_sum(su, sh);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = sd;
    partials[2 * blockIdx.x + 1] = su;
  }
}

__global__ void final_reduce_kernel(const double* __restrict__ partials, int nblocks, double* __restrict__ out) {
  __shared__ double sh[32];
  double sd = 0.0, su = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
    sd += partials[2 * b];
    su += partials[2 * b + 1];
  }
  sd = block_sum(sd, sh);
  su = block_sum(su, sh);
  if (threadIdx.x == 0) {
    out[0] = sd;
    out[1] = su;
  }
}

}  // namespace

pe_status launch_coarse_sweep(pe_ctx* c) {
  const int threads = 256;
  const unsigned blocks = (unsigned)((c->g.ndof + threads - 1) / threads);
  if (c->forcing_path == PE_FORCING_GENERAL) {
    PE_TRY(launch_general_coarse_forcing(c));
    coarse_recurrence_kernel<<<blocks, threads, 0, c->stream>>>(c->g, c->N, c->coefG, c->gG, c->U, c->Gold);
    c->launches += 1;
    PE_CUDA_TRY(cudaGetLastError());
    return PE_OK;
  }
  // slices per thread: enough CTAs to cover the GPU twice, at least one slice each
  int64_t want = (2 * 152 * 2 + blocks - 1) / blocks;
  int SL = (int)((c->N + want - 1) / want);
  SL = SL < 1 ? 1 : SL;
  dim3 grid(blocks, (unsigned)((c->N + SL - 1) / SL));
  if (c->precision == PE_MIXED) {
    const size_t smem = sizeof(float) * (size_t)c->R * threads;
    coarse_forcing_kernel<float><<<grid, threads, smem, c->stream>>>(c->g, c->N, c->p, c->R, SL, c->axisF32, c->AG32,
                                                                    c->coefG, c->gG);
  } else {
    const size_t smem = sizeof(double) * (size_t)c->R * threads;
    if (smem > 48 * 1024)
      PE_CUDA_TRY(cudaFuncSetAttribute(coarse_forcing_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem));
    coarse_forcing_kernel<double><<<grid, threads, smem, c->stream>>>(c->g, c->N, c->p, c->R, SL, c->axisF, c->AG,
                                                                     c->coefG, c->gG);
  }
  // learned correction G'(v) = G(v) + delta^ (no-op unless a trained network is attached)
  PE_TRY(launch_learned_correction(c));
  coarse_recurrence_kernel<<<blocks, threads, 0, c->stream>>>(c->g, c->N, c->coefG, c->gG, c->U, c->Gold);
  c->launches += 2;
  PE_CUDA_TRY(cudaGetLastError());
  return PE_OK;
}

pe_status launch_correction(pe_ctx* c, double* num, double* den) {
  const int threads = 256;
  const int blocks = (int)((c->g.ndof + threads - 1) / threads);
  if (blocks > c->max_blocks) return pe_fail(PE_EINVAL, "correction: partials buffer too small");
  correction_kernel<<<blocks, threads, 0, c->stream>>>(c->g, c->N, c->muM_axis, c->coefG, c->gG, c->Fbar, c->Gold,
                                                       c->U, c->partials);
  PE_CUDA_TRY(cudaGetLastError());
  final_reduce_kernel<<<1, 1024, 0, c->stream>>>(c->partials, blocks, c->red);
  c->launches += 2;
  PE_CUDA_TRY(cudaGetLastError());
  PE_CUDA_TRY(cudaMemcpyAsync(c->h_red, c->red, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  PE_CUDA_TRY(cudaStreamSynchronize(c->stream));
  *num = c->h_red[0];
  *den = c->h_red[1];
  return PE_OK;
}
