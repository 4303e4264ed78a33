// Coarse sweep, correction and residual of Algorithm 1 (PEIFE-linear).
//
// In mode space every step of Eq. (1-7) is  c <- E c + sum_i (tau b_i) ghat(t_i)
// with ghat_J(t) = sum_r A_r(t) P_{r,J}, A_r(t) = amp_r time_r(t) and
// P_{r,J} = prod_a axisF[a][r][j_a].  Modes are independent, so one thread owns
// one mode and walks the slices n = 0..N-1 sequentially (the "sequential"
// parts of Algorithm 1 are sequential in n only).
//
//   coarse sweep   U^{n+1,(0)} = G(U^{n,(0)}) = E_G U^n + gG_n.
//   correction     U^{n+1,(k+1)} = G(U^{n,(k+1)}) + Fbar^{n+1} - G(U^{n,(k)}).  G is affine
//                  in its argument, G(v) = E_G v + gG_n (a learned correction adds a term
//                  that does not depend on v), so the update is evaluated as
//                    U^{n+1,(k+1)} = Fbar^{n+1} + E_G (U^{n,(k+1)} - U^{n,(k)}):
//                  the same value, without G(U^{n,(k)}) stored between iterations and
//                  without the cancellation of the two G terms; it reads Fbar and the
//                  old U and writes the new U (3 words per mode and slice instead of 6).
//                  Float64 sums  sum mu^M_J (U^{new} - U^{old})^2, sum mu^M_J (U^{new})^2
//                  (per-CTA partial sums, added by the last CTA to finish).
#include "pe_internal.h"
#include "pe_learned.h"

namespace {

// Coarse forcing of every slice, in parallel over slices: each thread owns one
// mode and SL consecutive slices.  Its weights P_{r,J} sit in registers, padded
// with zeros to RB = roundup(R, 4) terms; the CTA's coarse time factors
// A_r(T_n + c_i dT) (n in its slice range) are staged in shared memory, rows of RB
// with zero padding, and read as float4 / double2 broadcasts.  T = double on the
// float64 path; float in the mixed form, where gG only enters through
// G(U^{new}) - G(U^{old}), in which the same stored gG cancels.
template <typename T, int RB>
__global__ void __launch_bounds__(256) coarse_forcing_kernel(Geom g, int N, int p, int R, int SL,
                                                            const T* __restrict__ axisF, const T* __restrict__ AG,
                                                            const double* __restrict__ coefG,
                                                            double* __restrict__ gG) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sA = reinterpret_cast<T*>(smem_raw);  // [SL * p][RB]
  const int n0 = blockIdx.y * SL;
  const int n1 = min(N, n0 + SL);
  for (int e = threadIdx.x; e < (n1 - n0) * p * RB; e += blockDim.x) {
    const int row = e / RB, r = e - row * RB;
    sA[e] = r < R ? AG[((int64_t)n0 * p + row) * R + r] : T(0);
  }
  __syncthreads();
  const int64_t J = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (J >= g.ndof) return;
  const int64_t nd = g.ndof;
  int j[PE_MAX_D];
  unflatten(g, J, j);
  T P[RB];
#pragma unroll
  for (int r = 0; r < RB; ++r) {
    T v = T(0);
    if (r < R) {
      v = axisF[(int64_t)R * g.off[0] + (int64_t)r * g.n[0] + j[0]];
#pragma unroll
      for (int a = 1; a < PE_MAX_D; ++a) if (a < g.d) v *= axisF[(int64_t)R * g.off[a] + (int64_t)r * g.n[a] + j[a]];
    }
    P[r] = v;
  }
  T b[PE_MAX_S];
#pragma unroll
  for (int i = 0; i < PE_MAX_S; ++i) b[i] = i < p ? (T)coefG[(1 + i) * nd + J] : T(0);
  for (int n = n0; n < n1; ++n) {
    T acc = T(0);
#pragma unroll
    for (int i = 0; i < PE_MAX_S; ++i) {
      if (i < p) {
        const T* a = sA + ((int64_t)(n - n0) * p + i) * RB;
        T gi = T(0);
        if constexpr (sizeof(T) == 4) {
#pragma unroll
          for (int r = 0; r < RB; r += 4) {
            const float4 v = *reinterpret_cast<const float4*>(a + r);
            gi = fmaf(v.x, P[r], gi);
            gi = fmaf(v.y, P[r + 1], gi);
            gi = fmaf(v.z, P[r + 2], gi);
            gi = fmaf(v.w, P[r + 3], gi);
          }
        } else {
#pragma unroll
          for (int r = 0; r < RB; r += 2) {
            const double2 v = *reinterpret_cast<const double2*>(a + r);
            gi = fma(v.x, P[r], gi);
            gi = fma(v.y, P[r + 1], gi);
          }
        }
        acc = fma(b[i], gi, acc);
      }
    }
    gG[(int64_t)n * nd + J] = (double)acc;
  }
}

// The instantiation with RB = roundup(R, 4) (at least 4); SL slices per thread,
// capped so that the staged time factors fit 48 KB.
template <typename T>
pe_status launch_coarse_forcing_t(pe_ctx* c, unsigned blocks, int threads, int SL, const T* axisF, const T* AG) {
  const int RB = c->R < 4 ? 4 : (c->R + 3) / 4 * 4;  // no source terms: one all-zero group
  const int sl_max = (int)((48 * 1024) / (sizeof(T) * (size_t)c->p * RB));
  SL = SL > sl_max ? sl_max : SL;
  const size_t smem = sizeof(T) * (size_t)SL * c->p * RB;
  const dim3 grid(blocks, (unsigned)((c->N + SL - 1) / SL));
  switch (RB) {
#define PE_CF_CASE(X)                                                                                        \
  case X:                                                                                                    \
    coarse_forcing_kernel<T, X><<<grid, threads, smem, c->stream>>>(c->g, c->N, c->p, c->R, SL, axisF, AG, \
                                                                    c->coefG, c->gG);                      \
    break;
    PE_CF_CASE(4) PE_CF_CASE(8) PE_CF_CASE(12) PE_CF_CASE(16) PE_CF_CASE(20) PE_CF_CASE(24) PE_CF_CASE(28)
    PE_CF_CASE(32)
#undef PE_CF_CASE
    default:
      return pe_fail(PE_EINVAL, "coarse forcing: too many source terms");
  }
  PE_CUDA_TRY(cudaGetLastError());
  return PE_OK;
}

// Coarse sweep of k = 0 with the coarse forcing made on the fly: one thread per mode walks
// the slices, forming gG_n = sum_i b_i sum_r A_r(T_n + c_i dT) P_{r,J} from its register
// weights and the time factors of all slices (staged in shared memory, rows of RB) and
// applying U^{n+1} = E_G U^n + gG_n, so gG is neither written nor read back.  LEARN adds the
// learned term of G' = G + delta^ per slice, sum_r (A_r cos_{r,n} + B_r sin_{r,n}) with
// A_r = P_{r,J} amp_r Im K^, B_r = P_{r,J} amp_r Re K^ (K^ interpolated linearly in
// log(lam dT) between the band centres) and the phase table staged beside the time factors:
// the same float32 sum, added to gG_n in float64, as the separate learned-correction kernel.
template <typename T, int RB, bool LEARN>
__global__ void __launch_bounds__(512) coarse_fused_kernel(Geom g, int N, int p, int R,
                                                          const T* __restrict__ axisF, const T* __restrict__ AG,
                                                          const double* __restrict__ coefG, double* __restrict__ U,
                                                          LearnedTerms L, const double* __restrict__ axisF64,
                                                          const double* __restrict__ lam) {
  pdl_wait();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* sCS = reinterpret_cast<float2*>(smem_raw);                // [N][RB] (LEARN only)
  T* sA = reinterpret_cast<T*>(smem_raw + (LEARN ? sizeof(float2) * (size_t)N * RB : 0));  // [N * p][RB]
  for (int e = threadIdx.x; e < N * p * RB; e += blockDim.x) {
    const int row = e / RB, r = e - row * RB;
    sA[e] = r < R ? AG[(int64_t)row * R + r] : T(0);
  }
  if constexpr (LEARN) {
    for (int e = threadIdx.x; e < N * RB; e += blockDim.x) {
      const int n = e / RB, r = e - n * RB;
      sCS[e] = r < R ? L.cs[(int64_t)r * N + n] : make_float2(0.f, 0.f);
    }
  }
  __syncthreads();
  const int64_t J = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (J >= g.ndof) return;
  const int64_t nd = g.ndof;
  int j[PE_MAX_D];
  unflatten(g, J, j);
  T P[RB];
#pragma unroll
  for (int r = 0; r < RB; ++r) {
    T v = T(0);
    if (r < R) {
      v = axisF[(int64_t)R * g.off[0] + (int64_t)r * g.n[0] + j[0]];
#pragma unroll
      for (int a = 1; a < PE_MAX_D; ++a) if (a < g.d) v *= axisF[(int64_t)R * g.off[a] + (int64_t)r * g.n[a] + j[a]];
    }
    P[r] = v;
  }
  float LA[LEARN ? RB : 1], LB[LEARN ? RB : 1];
  if constexpr (LEARN) {
    double pos = (log(lam[J] * L.dT) - L.loglo) / L.logstep;
    pos = fmin(fmax(pos, 0.0), (double)(L.NB - 1) - 1e-9);
    const int b0 = (int)pos;
    const double f = pos - (double)b0;
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      LA[r] = 0.f;
      LB[r] = 0.f;
      if (r < R && L.is_sin[r]) {
        double Pd = axisF64[(int64_t)R * g.off[0] + (int64_t)r * g.n[0] + j[0]];
#pragma unroll
        for (int a = 1; a < PE_MAX_D; ++a) if (a < g.d)
          Pd *= axisF64[(int64_t)R * g.off[a] + (int64_t)r * g.n[a] + j[a]];
        const double* k0 = L.Ktab + 2 * ((int64_t)r * L.NB + b0);
        const double Kre = (1.0 - f) * k0[0] + f * k0[2];
        const double Kim = (1.0 - f) * k0[1] + f * k0[3];
        const double cc = Pd * L.amp[r];
        LA[r] = (float)(cc * Kim);
        LB[r] = (float)(cc * Kre);
      }
    }
  }
  T b[PE_MAX_S];
#pragma unroll
  for (int i = 0; i < PE_MAX_S; ++i) b[i] = i < p ? (T)coefG[(1 + i) * nd + J] : T(0);
  const double E = coefG[J];
  double c = U[J];
  // two slices per pass: the forcing sums of the second overlap the float64 step of the first
  // (four measured slower: 20.3 against 18.4 us at 255^2)
#pragma unroll 2
  for (int n = 0; n < N; ++n) {
    T acc = T(0);
#pragma unroll
    for (int i = 0; i < PE_MAX_S; ++i) {
      if (i < p) {
        const T* a = sA + ((int64_t)n * p + i) * RB;
        T gi = T(0);
        if constexpr (sizeof(T) == 4) {
#pragma unroll
          for (int r = 0; r < RB; r += 4) {
            const float4 v = *reinterpret_cast<const float4*>(a + r);
            gi = fmaf(v.x, P[r], gi);
            gi = fmaf(v.y, P[r + 1], gi);
            gi = fmaf(v.z, P[r + 2], gi);
            gi = fmaf(v.w, P[r + 3], gi);
          }
        } else {
#pragma unroll
          for (int r = 0; r < RB; r += 2) {
            const double2 v = *reinterpret_cast<const double2*>(a + r);
            gi = fma(v.x, P[r], gi);
            gi = fma(v.y, P[r + 1], gi);
          }
        }
        acc = fma(b[i], gi, acc);
      }
    }
    double gn;
    if constexpr (sizeof(T) == 4) gn = widen_f32(acc);
    else gn = acc;
    if constexpr (LEARN) {
      float dl = 0.f;
      const float2* e = sCS + (int64_t)n * RB;
#pragma unroll
      for (int r = 0; r < RB; ++r) dl = fmaf(LA[r], e[r].x, fmaf(LB[r], e[r].y, dl));
      gn += widen_f32(dl);
    }
    c = fma(E, c, gn);
    U[(int64_t)(n + 1) * nd + J] = c;
  }
}

// The fused coarse sweep when its shared tables fit 48 KB; *done = false (nothing launched)
// otherwise.  L is null without a learned correction.
template <typename T>
pe_status launch_coarse_fused_t(pe_ctx* c, unsigned blocks, int threads, const T* axisF, const T* AG,
                                const LearnedTerms* L, bool* done) {
  *done = false;
  const int RB = c->R < 4 ? 4 : (c->R + 3) / 4 * 4;
  const size_t smem = sizeof(T) * (size_t)c->N * c->p * RB + (L ? sizeof(float2) * (size_t)c->N * RB : 0);
  if (smem > 48 * 1024) return PE_OK;
  const LearnedTerms Lv = L ? *L : LearnedTerms{};
  switch (RB) {
#define PE_CF_CASE(X)                                                                                          \
  case X:                                                                                                      \
    if (L)                                                                                                     \
      PE_CUDA_TRY(launch_pdl(coarse_fused_kernel<T, X, true>, dim3(blocks), dim3(threads), smem, c->stream, c->g, \
                             c->N, c->p, c->R, axisF, AG, (const double*)c->coefG, c->U, Lv,                    \
                             (const double*)c->axisF, (const double*)c->lam));                                  \
    else                                                                                                       \
      PE_CUDA_TRY(launch_pdl(coarse_fused_kernel<T, X, false>, dim3(blocks), dim3(threads), smem, c->stream, c->g, \
                             c->N, c->p, c->R, axisF, AG, (const double*)c->coefG, c->U, Lv,                     \
                             (const double*)c->axisF, (const double*)c->lam));                                   \
    break;
    PE_CF_CASE(4) PE_CF_CASE(8) PE_CF_CASE(12) PE_CF_CASE(16) PE_CF_CASE(20) PE_CF_CASE(24) PE_CF_CASE(28)
    PE_CF_CASE(32)
#undef PE_CF_CASE
    default:
      return pe_fail(PE_EINVAL, "coarse sweep: too many source terms");
  }
  PE_CUDA_TRY(cudaGetLastError());
  *done = true;
  return PE_OK;
}

// Slices of loads each thread keeps in flight in the sequential sweeps below.
// The recurrence carries one value per mode; its inputs do not depend on it,
// so the loads of the next kPF slices are issued while the current kPF are
// combined (one thread per mode leaves too few threads to cover HBM latency
// with one slice in flight).
constexpr int kPF = 4;

// Sequential coarse sweep U^{n+1,(0)} = E_G U^{n,(0)} + gG_n (one thread per mode).
__global__ void __launch_bounds__(256) coarse_recurrence_kernel(Geom g, int N, const double* __restrict__ coefG,
                                                               const double* __restrict__ gG,
                                                               double* __restrict__ U) {
  const int64_t J = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (J >= g.ndof) return;
  const int64_t nd = g.ndof;
  const double E = coefG[J];
  double c = U[J];
  double cur[kPF], nxt[kPF];
#pragma unroll
  for (int e = 0; e < kPF; ++e) cur[e] = e < N ? gG[(int64_t)e * nd + J] : 0.0;
  for (int n0 = 0; n0 < N; n0 += kPF) {
#pragma unroll
    for (int e = 0; e < kPF; ++e) {
      const int n = n0 + kPF + e;
      nxt[e] = n < N ? gG[(int64_t)n * nd + J] : 0.0;
    }
#pragma unroll
    for (int e = 0; e < kPF; ++e) {
      const int n = n0 + e;
      if (n < N) {
        c = fma(E, c, cur[e]);
        U[(int64_t)(n + 1) * nd + J] = c;
      }
    }
#pragma unroll
    for (int e = 0; e < kPF; ++e) cur[e] = nxt[e];
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

// Stopping decision of a device-resident loop, run by one thread after the residual sums are
// complete: r_k appended to the history, k advanced, and the graph's while condition set to
// continue while r > tol and k < max_iter (a non-finite sum stops the loop and is flagged).
__device__ void loop_decide(LoopCtl* L, unsigned long long handle, double num, double den) {
  const bool finite = isfinite(num) && isfinite(den);
  const double r = den > 0.0 ? sqrt(num) / sqrt(den) : sqrt(num);
  const int k = L->k;
  if (k < L->hist_cap) L->hist[k] = r;
  L->k = k + 1;
  L->r = r;
  if (!finite) L->nonfinite = 1;
  // the host reads k, r and the flag from its mapped mirror after the solve's one wait
  volatile LoopCtl* H = L->host;
  H->k = k + 1;
  H->r = r;
  if (!finite) H->nonfinite = 1;
  __threadfence_system();
  cudaGraphSetConditional((cudaGraphConditionalHandle)handle,
                          (finite && r > L->tol && k + 1 < L->max_iter) ? 1u : 0u);
}

__global__ void loop_init_kernel(LoopCtl* L, int max_iter, int hist_cap, double tol, double* hist,
                                 LoopCtl* host) {
  pdl_wait();
  if (threadIdx.x == 0) {
    L->k = 0;
    L->max_iter = max_iter;
    L->nonfinite = 0;
    L->hist_cap = hist_cap;
    L->tol = tol;
    L->r = INFINITY;
    L->hist = hist;
    L->host = host;
  }
}

// The correction: one thread per mode walks the slices.  With d = U^{n,(k+1)} - U^{n,(k)}
// (d = 0 at n = 0: U^0 is the same in every iterate)
//   U^{n+1,(k+1)} = fma(E_G, d, Fbar^{n+1}),   d <- U^{n+1,(k+1)} - U^{n+1,(k)},
// and the residual terms fma(d, d, sd), fma(U, U, su): four float64 operations per mode and
// slice.  GB300 executes float64 at 2 lanes per SM and clock, so this HBM-shaped step is bound
// by those operations (at 255^2 x 32 slices: about 13 us at the full float64 rate); the loads of
// the next kCorrPF slices are issued before the current kCorrPF are combined.
constexpr int kCorrPF = 8;

__global__ void __launch_bounds__(512) correction_kernel(Geom g, int N, const double* __restrict__ muM_axis,
                                                         const double* __restrict__ coefG,
                                                         const double* __restrict__ Fbar, double* __restrict__ U,
                                                         double* __restrict__ partials,
                                                         unsigned int* __restrict__ done, double* __restrict__ red,
                                                         LoopCtl* loop, unsigned long long handle) {
  pdl_wait();
  __shared__ double sh[32];
  __shared__ bool s_last;
  const int64_t J = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double sd = 0.0, su = 0.0, w = 0.0;
  if (J < g.ndof) {
    const int64_t nd = g.ndof;
    int j[PE_MAX_D];
    unflatten(g, J, j);
    w = muM_axis[g.off[0] + j[0]];
#pragma unroll
    for (int a = 1; a < PE_MAX_D; ++a) if (a < g.d) w *= muM_axis[g.off[a] + j[a]];
    const double E = coefG[J];
    double d = 0.0;
    // per slice n: Fbar^{n+1} = F(U^{n,(k)}) and the old U^{n+1}
    double f0[kCorrPF], o0[kCorrPF], f1[kCorrPF], o1[kCorrPF];
#pragma unroll
    for (int e = 0; e < kCorrPF; ++e) {
      const int64_t o = (int64_t)e * nd + J;
      const bool in = e < N;
      f0[e] = in ? Fbar[o] : 0.0;
      o0[e] = in ? U[o + nd] : 0.0;
    }
    for (int n0 = 0; n0 < N; n0 += kCorrPF) {
#pragma unroll
      for (int e = 0; e < kCorrPF; ++e) {
        const int n = n0 + kCorrPF + e;
        const int64_t o = (int64_t)n * nd + J;
        const bool in = n < N;
        f1[e] = in ? Fbar[o] : 0.0;
        o1[e] = in ? U[o + nd] : 0.0;
      }
#pragma unroll
      for (int e = 0; e < kCorrPF; ++e) {
        const int n = n0 + e;
        if (n < N) {
          const double un = fma(E, d, f0[e]);
          U[(int64_t)(n + 1) * nd + J] = un;
          d = un - o0[e];
          sd = fma(d, d, sd);
          su = fma(un, un, su);
        }
      }
#pragma unroll
      for (int e = 0; e < kCorrPF; ++e) {
        f0[e] = f1[e];
        o0[e] = o1[e];
      }
    }
  }
  // the weight mu^M_J is the same for every slice of the mode: applied once
  sd *= w;
  su *= w;
  sd = block_sum(sd, sh);
  su = block_sum(su, sh);
  // the last CTA to finish adds the per-CTA partial sums (in CTA order) and re-arms the counter
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = sd;
    partials[2 * blockIdx.x + 1] = su;
    __threadfence();
    s_last = atomicAdd(done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (s_last) {
    __threadfence();
    double td = 0.0, tu = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
      td += __ldcg(partials + 2 * b);
      tu += __ldcg(partials + 2 * b + 1);
    }
    td = block_sum(td, sh);
    tu = block_sum(tu, sh);
    if (threadIdx.x == 0) {
      red[0] = td;
      red[1] = tu;
      *done = 0u;
      if (loop) loop_decide(loop, handle, td, tu);
    }
  }
}

}  // namespace

pe_status launch_coarse_sweep(pe_ctx* c) {
  const int threads = 256;
  const unsigned blocks = (unsigned)((c->g.ndof + threads - 1) / threads);
  const int fthreads = per_mode_block(c->g.ndof, c->sms);
  const unsigned fblocks = (unsigned)((c->g.ndof + fthreads - 1) / fthreads);
  if (c->forcing_path == PE_FORCING_GENERAL) {
    PE_TRY(launch_general_coarse_forcing(c));
    coarse_recurrence_kernel<<<blocks, threads, 0, c->stream>>>(c->g, c->N, c->coefG, c->gG, c->U);
    c->launches += 1;
    PE_CUDA_TRY(cudaGetLastError());
    return PE_OK;
  }
  {
    // fused sweep; with a learned correction its band and phase tables are made first
    LearnedTerms L{};
    if (c->mlp) PE_TRY(launch_learned_tables(c, &L));
    const LearnedTerms* Lp = c->mlp ? &L : nullptr;
    bool done = false;
    if (c->precision == PE_MIXED) PE_TRY(launch_coarse_fused_t<float>(c, fblocks, fthreads, c->axisF32, c->AG32, Lp, &done));
    else PE_TRY(launch_coarse_fused_t<double>(c, fblocks, fthreads, c->axisF, c->AG, Lp, &done));
    if (done) {
      c->launches += 1;
      return PE_OK;
    }
  }
  // slices per thread: enough CTAs to cover the GPU twice, at least one slice each
  int64_t want = (2 * 152 * 2 + blocks - 1) / blocks;
  int SL = (int)((c->N + want - 1) / want);
  SL = SL < 1 ? 1 : SL;
  if (c->precision == PE_MIXED) PE_TRY(launch_coarse_forcing_t<float>(c, blocks, threads, SL, c->axisF32, c->AG32));
  else PE_TRY(launch_coarse_forcing_t<double>(c, blocks, threads, SL, c->axisF, c->AG));
  // learned correction G'(v) = G(v) + delta^ (no-op unless a trained network is attached)
  PE_TRY(launch_learned_correction(c));
  coarse_recurrence_kernel<<<blocks, threads, 0, c->stream>>>(c->g, c->N, c->coefG, c->gG, c->U);
  c->launches += 2;
  PE_CUDA_TRY(cudaGetLastError());
  return PE_OK;
}

pe_status launch_correction(pe_ctx* c, double* num, double* den, cudaEvent_t after) {
  PE_TRY(launch_correction_kernel(c, nullptr, 0ull));
  if (after) PE_CUDA_TRY(cudaEventRecord(after, c->stream));
  PE_CUDA_TRY(cudaMemcpyAsync(c->h_red, c->red, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  PE_CUDA_TRY(cudaStreamSynchronize(c->stream));
  *num = c->h_red[0];
  *den = c->h_red[1];
  return PE_OK;
}

pe_status launch_loop_init(pe_ctx* c, double tol) {
  PE_CUDA_TRY(launch_pdl(loop_init_kernel, dim3(1), dim3(32), 0, c->stream, c->loopctl, c->max_iter, c->N, tol,
                         c->loop_hist, c->h_loop_dev));
  c->launches += 1;
  return PE_OK;
}

pe_status launch_correction_kernel(pe_ctx* c, LoopCtl* loop, unsigned long long handle) {
  const int threads = per_mode_block(c->g.ndof, c->sms);
  const int64_t blocks = (c->g.ndof + threads - 1) / threads;
  if (blocks > (int64_t)c->max_blocks) return pe_fail(PE_EINVAL, "correction: partials buffer too small");
  PE_CUDA_TRY(launch_pdl(correction_kernel, dim3((unsigned)blocks), dim3(threads), 0, c->stream, c->g, c->N,
                         (const double*)c->muM_axis, (const double*)c->coefG, (const double*)c->Fbar, c->U,
                         c->partials, c->done_ctr, c->red, loop, handle));
  c->launches += 1;
  PE_CUDA_TRY(cudaGetLastError());
  return PE_OK;
}
