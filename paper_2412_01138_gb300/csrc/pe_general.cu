// General forcing path: P_h f(t) through nodal space at every stage time.
//
// For sources whose spatial factors move with t (the oscillating hat of Example 4
// of Sec. 5) the modal factors cannot be formed once.  At every stage time t of
// Eq. (1-7) this path (i) evaluates the consistent load F(t) by element
// Gauss-Legendre quadrature (per axis: a product of per-axis factors integrates as
// the product of 1D element integrals), (ii) applies the tensor DST-I V^T along
// every axis (batched over the stage times of a chunk of slices), and (iii) folds
// Lambda_M^{-1} into the stage weights of the fine and coarse recurrences.  The
// fine propagator then reads ghat(t) from HBM instead of forming it from
// per-axis factors: the step is memory-bound, and the transform dominates.
// In the mixed form the fine sweep's loads, assembly and transforms run in
// float32 (the coarse forcing, computed once per problem, stays float64).
//
// Slices are processed in chunks so that the stage-time loads of a chunk fit a
// fixed device budget.
#include <math.h>

#include <algorithm>

#include "pe_forcing_common.cuh"
#include "pe_internal.h"
#include "pe_sweep_common.cuh"

namespace {

// stage times of a chunk: fine (n0 + s / (M q), m, i) or coarse (s / p, i)
struct StageGen {
  int coarse;   // 0 fine, 1 coarse
  int n0;       // first slice of the chunk (fine)
  int M, s;     // substeps and nodes per step
  double t0, dT, dt;
  double c[PE_MAX_S];
};

__device__ inline double stage_time(const StageGen& G, int idx) {
  if (G.coarse) {
    const int n = idx / G.s, i = idx % G.s;
    const double Tn = G.t0 + (double)n * G.dT;
    return Tn + G.c[i] * G.dT;
  }
  const int per = G.M * G.s;
  const int n = G.n0 + idx / per, rem = idx % per;
  const int m = rem / G.s, i = rem % G.s;
  const double Tn = G.t0 + (double)n * G.dT;
  const double tl = Tn + (double)m * G.dt;
  return tl + G.c[i] * G.dt;
}

// L[st][R*off[a] + r*n_a + k] = int g_{r,a}(x, t_st) phi_{k+1}(x) dx  (grid: node blocks of
// 128, R*d, stages).  Element m = [lo + m h, lo + (m+1) h] contributes h int g s ds to its
// right node and h int g (1-s) ds to its left node; each element's quadrature is evaluated
// once (into shared memory) and node k sums the rising part of element k and the falling
// part of element k+1.  TL = float evaluates the factors in float32 (mixed precision).
// Per block (one term, axis and stage) the factor's parameters, the moving hat's centre at
// t_st and the quadrature weights w_q s_q, w_q (1 - s_q) are converted once into shared
// memory; per element only the node positions are formed in float64 (lo + m h + s_q h).

// The spatial factor at x from parameters already in TL (the moving hat's centre in p[0]).
template <typename TL>
__device__ __forceinline__ TL eval_factor(int kind, const TL* p, TL x) {
  switch (kind) {
    case PE_S_SIN: return sin(p[0] * x + p[1]);
    case PE_S_GAUSS: { const TL u = x - p[0]; return exp(-(u * u) / (TL(2) * p[1] * p[1])); }
    case PE_S_POLY: return p[0] + x * (p[1] + x * (p[2] + x * p[3]));
    case PE_S_MOVING_HAT: return fmax(TL(1) - fabs(x - p[0]) / p[3], TL(0));
    default: return TL(1);
  }
}

template <typename TL>
__global__ void __launch_bounds__(128) gen_loads_kernel(TermsDev T, Geom g, double lo0, double lo1, double lo2,
                                                        double h0, double h1, double h2, Gauss Q, StageGen SG,
                                                        int nsum, TL* __restrict__ L) {
  __shared__ TL rise[129], fall[129];
  __shared__ TL sp[4], sws[8], sw1s[8];
  __shared__ double ssh[8];
  __shared__ int skind;
  const int st = blockIdx.z;
  const int ra = blockIdx.y;
  const int r = ra / g.d, a = ra % g.d;
  if (r >= T.n) return;
  const int n = g.n[a];
  const int k0 = blockIdx.x * 128;
  if (k0 >= n) return;  // uniform over the block
  const double lo = a == 0 ? lo0 : (a == 1 ? lo1 : lo2);
  const double h = a == 0 ? h0 : (a == 1 ? h1 : h2);
  const int nq = Q.npts;
  if (threadIdx.x == 0) {
    const pe_term& tm = T.t[r];
    const int kind = tm.skind[a];
    const double* pd = tm.sp[a];
    double p0 = pd[0];
    if (kind == PE_S_MOVING_HAT) p0 = pd[0] + pd[1] * sinpi(2.0 * pd[2] * stage_time(SG, st));
    sp[0] = (TL)p0;
    sp[1] = (TL)pd[1];
    sp[2] = (TL)pd[2];
    sp[3] = (TL)pd[3];
    skind = kind;
  } else if (threadIdx.x <= 8) {
    const int q = threadIdx.x - 1;
    if (q < nq) {
      sws[q] = (TL)(Q.w[q] * Q.s[q]);
      sw1s[q] = (TL)(Q.w[q] * (1.0 - Q.s[q]));
      ssh[q] = Q.s[q] * h;
    }
  }
  __syncthreads();
  const int kind = skind;
  // elements k0 .. k0 + 128 (the last one only for its falling part); on a periodic axis
  // node k's elements are k-1 and k, i.e. k0-1 .. k0+127 taken modulo n
  const bool per = g.per[a] != 0;
  for (int i = threadIdx.x; i <= 128; i += blockDim.x) {
    int m = per ? k0 - 1 + i : k0 + i;
    if (per) m = (m + n) % n;
    TL up = TL(0), dn = TL(0);
    if (per || m <= n) {
      const double xm = fma((double)m, h, lo);
      for (int qi = 0; qi < nq; ++qi) {
        const TL gv = eval_factor<TL>(kind, sp, (TL)(xm + ssh[qi]));
        up += sws[qi] * gv;
        dn += sw1s[qi] * gv;
      }
    }
    rise[i] = up;
    fall[i] = dn;
  }
  __syncthreads();
  const int k = k0 + threadIdx.x;
  if (k < n)
    L[(int64_t)st * T.n * nsum + (int64_t)T.n * g.off[a] + (int64_t)r * n + k] =
        (TL)h * rise[threadIdx.x] + (TL)h * fall[threadIdx.x + 1];
}

// F[st][J] = sum_r amp_r time_r(t_st) prod_a L[st][...]  (nodal consistent load), as
// the rank-R product it is: with J = (o, j) split into the outer indices o and the last
// axis j, F[st][o][j] = sum_r P_r(o) q_r(j), P_r(o) = prod_{a<d-1} L_a[r][o_a] and
// q_r(j) = w_r L_{d-1}[r][j] (w_r = amp_r time_r(t_st)).  A block takes one stage and
// OC outer indices: thread j keeps q_r(j) in registers, the block tabulates P_r(o) in
// shared memory, and every output costs R FMAs (P read as a broadcast).
// R is a template parameter so that the R-term loops unroll without predicated FMAs.
constexpr int kAsmOC = 32;
template <typename Tout, int R>
__global__ void __launch_bounds__(256) gen_assemble_kernel(TermsDev T, Geom g, StageGen SG, int nsum, int count,
                                                           const Tout* __restrict__ L, Tout* __restrict__ F) {
  __shared__ Tout w[PE_MAX_TERMS];
  __shared__ Tout sP[kAsmOC][R];
  const int d = g.d, nl = g.n[d - 1];
  const int64_t outer = g.ndof / nl;
  const int64_t chunks = (outer + kAsmOC - 1) / kAsmOC;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  for (int64_t yy = blockIdx.y; yy < (int64_t)count * chunks; yy += gridDim.y) {
    const int st = (int)(yy / chunks);
    const int64_t o0 = (yy - (int64_t)st * chunks) * kAsmOC;
    const Tout* Ls = L + (int64_t)st * R * nsum;
    __syncthreads();  // the previous iteration's readers of w and sP are done
    if (threadIdx.x < R) {
      const pe_term& tm = T.t[threadIdx.x];
      w[threadIdx.x] = (Tout)(tm.amp * eval_time(tm, stage_time(SG, st)));
    }
    for (int e = threadIdx.x; e < kAsmOC * R; e += blockDim.x) {
      const int oc = e / R, r = e - oc * R;
      const int64_t o = o0 + oc;
      Tout P = Tout(1);
      if (o < outer) {
        int64_t rest = o;
        for (int a = d - 2; a >= 0; --a) {
          const int ja = (int)(rest % g.n[a]);
          rest /= g.n[a];
          P *= Ls[(int64_t)R * g.off[a] + (int64_t)r * g.n[a] + ja];
        }
      }
      sP[oc][r] = P;
    }
    __syncthreads();
    if (j < nl) {
      Tout q[R];
#pragma unroll
      for (int r = 0; r < R; ++r) q[r] = w[r] * Ls[(int64_t)R * g.off[d - 1] + (int64_t)r * nl + j];
      const int oend = (int)min((int64_t)kAsmOC, outer - o0);
      for (int oc = 0; oc < oend; ++oc) {
        Tout acc = Tout(0);
#pragma unroll
        for (int r = 0; r < R; ++r) acc = fma(sP[oc][r], q[r], acc);
        F[(int64_t)st * g.ndof + (o0 + oc) * nl + j] = acc;
      }
    }
  }
}

// fine propagator from the stored transformed loads: Gh[(n - n0) M q + m q + i][J] = (V^T F)_J
__global__ void __launch_bounds__(256) gen_fine_f64_kernel(Geom g, int n0, int M, int q,
                                                          const double* __restrict__ muM_axis,
                                                          const double* __restrict__ coefF,
                                                          const double* __restrict__ Gh,
                                                          const double* __restrict__ U, double* __restrict__ Fbar) {
  const int n = n0 + blockIdx.y;
  const int64_t nd = g.ndof;
  const int64_t J = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (J >= nd) return;
  int j[PE_MAX_D];
  unflatten(g, J, j);
  double mu = muM_axis[g.off[0] + j[0]];
#pragma unroll
  for (int a = 1; a < PE_MAX_D; ++a) if (a < g.d) mu *= muM_axis[g.off[a] + j[a]];
  const double E = coefF[J];
  double b[PE_MAX_S];
#pragma unroll
  for (int i = 0; i < PE_MAX_S; ++i)
    if (i < q) b[i] = coefF[(1 + i) * nd + J] / mu;
  double c = U[(int64_t)n * nd + J];
  const double* Gs = Gh + (int64_t)blockIdx.y * M * q * nd + J;
  for (int m = 0; m < M; ++m) {
    double acc = 0.0;
#pragma unroll
    for (int i = 0; i < PE_MAX_S; ++i)
      if (i < q) acc = fma(b[i], Gs[(int64_t)(m * q + i) * nd], acc);
    c = fma(E, c, acc);
  }
  Fbar[(int64_t)n * nd + J] = c;
}

__global__ void __launch_bounds__(256) gen_fine_mixed_kernel(Geom g, int n0, int M, int q,
                                                            const double* __restrict__ muM_axis,
                                                            const double* __restrict__ coefF,
                                                            const float* __restrict__ coefF32,
                                                            const float* __restrict__ Gh,
                                                            const double* __restrict__ U,
                                                            double* __restrict__ Fbar) {
  const int n = n0 + blockIdx.y;
  const int64_t nd = g.ndof;
  const int64_t J = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (J >= nd) return;
  int j[PE_MAX_D];
  unflatten(g, J, j);
  double mu = muM_axis[g.off[0] + j[0]];
#pragma unroll
  for (int a = 1; a < PE_MAX_D; ++a) if (a < g.d) mu *= muM_axis[g.off[a] + j[a]];
  const float eh = coefF32[J], el = coefF32[nd + J];
  float b[PE_MAX_S];
#pragma unroll
  for (int i = 0; i < PE_MAX_S; ++i)
    if (i < q) b[i] = (float)(coefF[(1 + i) * nd + J] / mu);
  float w = 0.f;
  const float* Gs = Gh + (int64_t)blockIdx.y * M * q * nd + J;
  for (int m = 0; m < M; ++m) {
    float acc = 0.f;
#pragma unroll
    for (int i = 0; i < PE_MAX_S; ++i)
      if (i < q) acc = fmaf(b[i], Gs[(int64_t)(m * q + i) * nd], acc);
    w = fmaf(eh, w, fmaf(el, w, acc));
  }
  const double EM = coefF[(int64_t)(q + 1) * nd + J];
  Fbar[(int64_t)n * nd + J] = fma(EM, U[(int64_t)n * nd + J], (double)w);
}

// coarse forcing gG[n][J] = sum_i (dT b_i / mu_J) (V^T F(T_n + c_i dT))_J
__global__ void gen_coarse_forcing_kernel(Geom g, int N, int p, const double* __restrict__ muM_axis,
                                          const double* __restrict__ coefG, const double* __restrict__ Gc,
                                          double* __restrict__ gG) {
  const int64_t J = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int n = blockIdx.y;
  if (J >= g.ndof || n >= N) return;
  const int64_t nd = g.ndof;
  int j[PE_MAX_D];
  unflatten(g, J, j);
  double mu = muM_axis[g.off[0] + j[0]];
#pragma unroll
  for (int a = 1; a < PE_MAX_D; ++a) if (a < g.d) mu *= muM_axis[g.off[a] + j[a]];
  double acc = 0.0;
  for (int i = 0; i < p; ++i) acc = fma(coefG[(1 + i) * nd + J] / mu, Gc[((int64_t)n * p + i) * nd + J], acc);
  gG[(int64_t)n * nd + J] = acc;
}

StageGen make_gen(const pe_ctx* c, int coarse, int n0) {
  StageGen G{};
  G.coarse = coarse;
  G.n0 = n0;
  G.M = c->M;
  G.s = coarse ? c->p : c->q;
  G.t0 = c->t0;
  G.dT = c->dT;
  G.dt = c->dt;
  for (int i = 0; i < PE_MAX_S; ++i) G.c[i] = coarse ? c->cG[i] : c->cF[i];
  return G;
}

template <typename T>
struct AssembleLaunch {
  template <int R>
  struct L {
    static pe_status run(dim3 grid, cudaStream_t st, TermsDev TD, Geom g, StageGen SG, int nsum, int count,
                         const T* Lp, T* F) {
      gen_assemble_kernel<T, R><<<grid, 256, 0, st>>>(TD, g, SG, nsum, count, Lp, F);
      return PE_OK;
    }
  };
};

// loads + nodal assembly + batched DST of `count` stage times into out (element type T)
template <typename T>
pe_status stage_transforms(pe_ctx* c, const StageGen& SG, int count, T* out, T* tmp) {
  TermsDev TD = pack_terms(c->terms, c->R);
  Gauss Q = make_gauss(c->quad_pts);
  int nmax = 1;
  for (int a = 0; a < c->g.d; ++a) nmax = std::max(nmax, c->g.n[a]);
  dim3 gl((nmax + 127) / 128, c->R * c->g.d, count);
  T* L = reinterpret_cast<T*>(c->gen_L);
  gen_loads_kernel<T><<<gl, 128, 0, c->stream>>>(TD, c->g, c->lo[0], c->lo[1], c->lo[2], c->h[0], c->h[1], c->h[2], Q,
                                                 SG, c->nsum, L);
  const int nl = c->g.n[c->g.d - 1];
  const int64_t chunks = (c->g.ndof / nl + kAsmOC - 1) / kAsmOC;
  dim3 ga((unsigned)((nl + 255) / 256), (unsigned)std::min<int64_t>((int64_t)count * chunks, 65535));
  // the assembled loads go to tmp or out so that the last DST pass lands in out
  T* F = (c->g.d % 2 == 1) ? tmp : out;
  PE_TRY(dispatch_R<AssembleLaunch<T>::template L>(c->R, ga, c->stream, TD, c->g, SG, c->nsum, count,
                                                   (const T*)L, F));
  c->launches += 2;
  PE_CUDA_TRY(cudaGetLastError());
  const T* src = F;
  for (int a = 0; a < c->g.d; ++a) {
    T* dst = (src == tmp) ? out : tmp;
    int64_t outer = count, inner = 1;
    for (int b = 0; b < a; ++b) outer *= c->g.n[b];
    for (int b = a + 1; b < c->g.d; ++b) inner *= c->g.n[b];
    if constexpr (sizeof(T) == 8)
      PE_TRY(dst_axis_f64(c->S[a], src, dst, outer, c->g.n[a], inner, c->stream, c->g.per[a]));
    else
      PE_TRY(dst_axis_f32(c->S32[a], src, dst, outer, c->g.n[a], inner, c->stream, c->g.per[a]));
    c->launches += 1;
    src = dst;
  }
  return PE_OK;
}

}  // namespace

// slices per chunk: the chunk's stage transforms (out + tmp) within 2 GiB, and at most
// 65535 stage times per chunk (grid dimension of the load kernels)
int general_slices_per_chunk(const pe_ctx* c) {
  const size_t elem = c->precision == PE_MIXED ? sizeof(float) : sizeof(double);
  const size_t per_slice = (size_t)c->M * c->q * (size_t)c->g.ndof * elem * 2;
  const size_t budget = (size_t)2 << 30;
  int ns = (int)std::max<size_t>(1, budget / std::max<size_t>(per_slice, 1));
  ns = std::min(ns, std::max(1, 65535 / (c->M * c->q)));
  return std::min(ns, c->N);
}

pe_status launch_general_coarse_forcing(pe_ctx* c) {
  const int count = c->N * c->p;
  StageGen SG = make_gen(c, 1, 0);
  double* out = c->gen_buf;   // the coarse stage transforms fit: N*p <= chunk stage capacity (checked at setup)
  double* tmp = c->gen_tmp;
  PE_TRY(stage_transforms<double>(c, SG, count, out, tmp));
  dim3 grid((unsigned)((c->g.ndof + 255) / 256), c->N);
  gen_coarse_forcing_kernel<<<grid, 256, 0, c->stream>>>(c->g, c->N, c->p, c->muM_axis, c->coefG, out, c->gG);
  c->launches += 1;
  PE_CUDA_TRY(cudaGetLastError());
  return PE_OK;
}

pe_status launch_general_fine_sweep(pe_ctx* c, int precision) {
  c->sweeps += 1;
  const int chunk = general_slices_per_chunk(c);
  for (int n0 = 0; n0 < c->N; n0 += chunk) {
    const int ns = std::min(chunk, c->N - n0);
    const int count = ns * c->M * c->q;
    StageGen SG = make_gen(c, 0, n0);
    dim3 grid((unsigned)((c->g.ndof + 255) / 256), ns);
    if (precision == PE_MIXED) {
      float* out = reinterpret_cast<float*>(c->gen_buf);
      float* tmp = reinterpret_cast<float*>(c->gen_tmp);
      PE_TRY(stage_transforms<float>(c, SG, count, out, tmp));
      gen_fine_mixed_kernel<<<grid, 256, 0, c->stream>>>(c->g, n0, c->M, c->q, c->muM_axis, c->coefF, c->coefF32,
                                                          out, c->U, c->Fbar);
    } else {
      PE_TRY(stage_transforms<double>(c, SG, count, c->gen_buf, c->gen_tmp));
      gen_fine_f64_kernel<<<grid, 256, 0, c->stream>>>(c->g, n0, c->M, c->q, c->muM_axis, c->coefF, c->gen_buf,
                                                        c->U, c->Fbar);
    }
    c->launches += 1;
    PE_CUDA_TRY(cudaGetLastError());
  }
  return PE_OK;
}
