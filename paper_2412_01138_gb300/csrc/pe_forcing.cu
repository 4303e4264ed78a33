// The load P_h f in mode space for separable sources, and the projection of u0.
//
// P_h is the L2 projection (Sec. 2.1, Eq. (3-11)); its modal coefficients are
// ghat = Lambda_M^{-1} V^T F with F_k = (f, phi_k) the consistent load.  For a
// separable term amp * time(t) * prod_a g_a(x_a) the load is the outer product
// of 1D loads F_a[k] = int g_a phi_k, so
//   ghat_J(t) = sum_r amp_r time_r(t) prod_a (S_a F_{r,a})_{j_a} / mu^M_a(j_a).
// 1D loads use a Gauss-Legendre rule with quad_pts points on each element.
// The per-axis modal factors, the time factors of the coarse stages and of the
// fine substep starts, and the per-mode stage weights of the fine step
// (Eq. (1-7), with the stage sum contracted as described in pe_fine_kernels.cuh)
// are tabulated here; the sweeps multiply them together on the fly.
#include <math.h>

#include "pe_internal.h"
#include "pe_forcing_common.cuh"

namespace {

// Time tables of one problem, one thread per entry:
//   AF[(n*M + m)*K + k] = Y_k(T_n + m dt)   (fine substep starts, stage-contracted columns;
//                                            the float copy AF32 has rows of roundup(K, 4))
//   AG[(n*p + i)*R + r] = amp_r time_r(T_n + c_i dT)   (coarse stage times)
//   Z[i*K + k]          = Z_k(c_i dt)       (shift of column k to fine stage i)
__global__ void time_tables_kernel(TermsDev T, StageCols C, int N, int M, int q, int p, double t0, double dT,
                                   double dt, Nodes cF, Nodes cG, double* __restrict__ AF,
                                   float* __restrict__ AF32, double* __restrict__ AG, float* __restrict__ AG32,
                                   double* __restrict__ Z) {
  pdl_wait();
  const int R = T.n, K = C.K;
  const int64_t nf = (int64_t)N * M * K;
  const int64_t ng = (int64_t)N * p * R;
  const int64_t nz = (int64_t)q * K;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < nf) {
    int64_t rest = idx;
    const int k = (int)(rest % K); rest /= K;
    const int m = (int)(rest % M); rest /= M;
    const int n = (int)rest;
    const double t = t0 + (double)n * dT + (double)m * dt;
    const pe_term& tr = T.t[C.term[k]];
    double v;
    if (C.kind[k] == 1) v = tr.amp * cos(tr.tp[0] * t + tr.tp[1]);  // partner of a sinusoid
    else v = tr.amp * eval_time(tr, t);
    AF[idx] = v;
    if (AF32) {
      // float copy padded to KC = roundup(K, 4) columns: [N][M][KC], zeros past K
      const int KC = (K + 3) & ~3;
      float* row = AF32 + ((int64_t)n * M + m) * KC;
      row[k] = (float)v;
      if (k == K - 1)
        for (int e = K; e < KC; ++e) row[e] = 0.f;
    }
  } else if (idx < nf + ng) {
    int64_t rest = idx - nf;
    const int r = (int)(rest % R); rest /= R;
    const int i = (int)(rest % p); rest /= p;
    const int n = (int)rest;
    const double Tn = t0 + (double)n * dT;
    const double t = Tn + cG.c[i] * dT;
    const double v = T.t[r].amp * eval_time(T.t[r], t);
    AG[idx - nf] = v;
    if (AG32) AG32[idx - nf] = (float)v;
  } else if (idx < nf + ng + nz) {
    const int64_t e = idx - nf - ng;
    const int k = (int)(e % K), i = (int)(e / K);
    const pe_term& tr = T.t[C.term[k]];
    const double s = cF.c[i] * dt;
    double v;
    if (tr.tkind == PE_T_SIN) v = C.kind[k] == 1 ? sin(tr.tp[0] * s) : cos(tr.tp[0] * s);
    else v = exp(tr.tp[0] * s);
    Z[e] = v;
  }
}

// W[k*ndof + J] = P_{r(k),J} sum_i (dt b_i)_J Z[i*K + k], with P_{r,J} = prod_a axisF[R off_a + r n_a + j_a],
// in the arithmetic of T (coefficient row i of dt b_i at coef + i * ndof).
template <typename T>
__global__ void stage_weights_kernel(Geom g, StageCols C, int R, int q, const T* __restrict__ axisF,
                                     const T* __restrict__ coef, const double* __restrict__ Z, T* __restrict__ W) {
  pdl_wait();
  // the shifts Z (converted to T once per CTA) and the column -> term map, in shared memory
  __shared__ T sZ[PE_MAX_S * 2 * PE_MAX_TERMS];
  __shared__ int sTerm[2 * PE_MAX_TERMS];
  for (int e = threadIdx.x; e < q * C.K; e += blockDim.x) sZ[e] = (T)Z[e];
  for (int e = threadIdx.x; e < C.K; e += blockDim.x) sTerm[e] = C.term[e];
  __syncthreads();
  const int64_t J = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (J >= g.ndof) return;
  const int64_t nd = g.ndof;
  int j[PE_MAX_D];
  unflatten(g, J, j);
  T b[PE_MAX_S];
#pragma unroll
  for (int i = 0; i < PE_MAX_S; ++i) b[i] = i < q ? coef[(int64_t)i * nd + J] : T(0);
  for (int k = 0; k < C.K; ++k) {
    const int r = sTerm[k];
    T P = axisF[(int64_t)R * g.off[0] + (int64_t)r * g.n[0] + j[0]];
#pragma unroll
    for (int a = 1; a < PE_MAX_D; ++a) if (a < g.d) P *= axisF[(int64_t)R * g.off[a] + (int64_t)r * g.n[a] + j[a]];
    T s = T(0);
#pragma unroll
    for (int i = 0; i < PE_MAX_S; ++i)
      if (i < q) s = fma(b[i], sZ[i * C.K + k], s);
    W[(int64_t)k * nd + J] = P * s;
  }
}

// 1D consistent loads of every (term, axis): out[R*off[a] + r*n_a + k] = int g_{r,a} phi_{k+1}.
// Eight lanes per node (blockDim = 8 x 32 nodes): lane s evaluates the quadrature points
// e = s, s + 8, ... of the node's 2 npts (its left element's points, then its right element's),
// and the eight partial sums are added by shuffles in a fixed order.  The float64 exponentials
// and sines of the factors thus spread over eight times more warps than a thread per node.
constexpr int kLoadLanes = 8;
__global__ void __launch_bounds__(256) loads_1d_kernel(TermsDev T, Geom g, double lo0, double lo1, double lo2,
                                                       double h0, double h1, double h2, Gauss G,
                                                       double* __restrict__ out) {
  pdl_wait();
  const int a = blockIdx.z;
  const int r = blockIdx.y;
  const int sub = threadIdx.x & (kLoadLanes - 1);
  const int k = blockIdx.x * (blockDim.x / kLoadLanes) + threadIdx.x / kLoadLanes;  // 0-based node
  if (a >= g.d || r >= T.n || k >= g.n[a]) return;  // whole groups of eight lanes leave together
  const double lo = a == 0 ? lo0 : (a == 1 ? lo1 : lo2);
  const double h = a == 0 ? h0 : (a == 1 ? h1 : h2);
  const pe_term& t = T.t[r];
  const int lk = T.lk[r][a];
  const unsigned grp = 0xFFu << (threadIdx.x & 24);  // this node's eight lanes of the warp
  if (lk != 0) {
    // lifting of Dirichlet data: the factor at full-grid nodes k, k+1, k+2 (x = lo + i h)
    if (sub == 0) {
      const double g0 = eval_space(t.skind[a], t.sp[a], lo + (double)k * h);
      const double g1 = eval_space(t.skind[a], t.sp[a], lo + (double)(k + 1) * h);
      const double g2 = eval_space(t.skind[a], t.sp[a], lo + (double)(k + 2) * h);
      double v = g1;
      if (lk == 1) v = (h / 6.0) * (g0 + 4.0 * g1 + g2);
      else if (lk == 2) v = (1.0 / h) * (2.0 * g1 - g0 - g2);
      out[(int64_t)T.n * g.off[a] + (int64_t)r * g.n[a] + k] = v;
    }
    return;
  }
  // Dirichlet: node k sits at lo + (k+1) h; element k ([lo + k h, lo + (k+1) h]) has it as
  // right vertex (shape s), element k+1 as left vertex (shape 1-s).  Periodic: node k sits
  // at lo + k h; the elements are k-1 (element n-1 for k = 0) and k.
  const int el = g.per[a] ? (k == 0 ? g.n[a] - 1 : k - 1) : k;
  const int er = g.per[a] ? k : k + 1;
  double part = 0.0;
  for (int e = sub; e < 2 * G.npts; e += kLoadLanes) {
    const bool left = e < G.npts;
    const int qi = left ? e : e - G.npts;
    const double x = lo + ((double)(left ? el : er) + G.s[qi]) * h;
    part += G.w[qi] * eval_space(t.skind[a], t.sp[a], x) * (left ? G.s[qi] : 1.0 - G.s[qi]);
  }
#pragma unroll
  for (int o = kLoadLanes / 2; o > 0; o >>= 1) part += __shfl_xor_sync(grp, part, o);
  if (sub == 0) out[(int64_t)T.n * g.off[a] + (int64_t)r * g.n[a] + k] = h * part;
}

// Per-axis source factors in matrix form, for grids whose axes are short: out[e],
// e = R off_a + r n_a + j (the layout of the per-axis tables), is sum_k S_a[j][k] L[R off_a + r
// n_a + k], times 1 / mu^M_a(j) when muInv is given.  A warp per output splits k (a row of the
// symmetric transform matrix and the term's loads, both contiguous: coalesced reads, all of a
// lane's loads in flight at once for n < 256, so a row read from HBM costs one latency); a shuffle
// sum in a fixed order.  The float64 work (n FMAs per output) spreads over every SM, where a
// half-length FFT per pencil pair runs one chain of dependent float64 latencies on a few SMs.
constexpr int kFactorLanes = 32;
__global__ void __launch_bounds__(256) axis_factor_matrix_kernel(Geom g, int R, const double* __restrict__ S0,
                                                                 const double* __restrict__ S1,
                                                                 const double* __restrict__ S2,
                                                                 const double* __restrict__ loads,
                                                                 const double* __restrict__ muInv,
                                                                 double* __restrict__ fac, float* __restrict__ fac32,
                                                                 int64_t total) {
  pdl_wait();
  const int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / kFactorLanes;
  const int sub = threadIdx.x & (kFactorLanes - 1);
  if (e >= total) return;  // whole warps leave together
  int a = 0;
  while (a + 1 < g.d && e >= (int64_t)R * g.off[a + 1]) ++a;
  const int n = g.n[a];
  const int64_t local = e - (int64_t)R * g.off[a];
  const int r = (int)(local / n), j = (int)(local - (int64_t)r * n);
  const double* S = a == 0 ? S0 : (a == 1 ? S1 : S2);
  const double* row = S + (int64_t)j * n;
  const double* L = loads + (int64_t)R * g.off[a] + (int64_t)r * n;
  double acc = 0.0;
#pragma unroll 8
  for (int k = sub; k < n; k += kFactorLanes) acc = fma(row[k], L[k], acc);
#pragma unroll
  for (int o = kFactorLanes / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
  if (sub == 0) {
    const double v = muInv ? acc * muInv[g.off[a] + j] : acc;
    fac[e] = v;
    if (fac32) fac32[e] = (float)v;
  }
}

__global__ void divide_axis_mu_kernel(Geom g, int R, const double* __restrict__ muM, double* __restrict__ x,
                                      float* __restrict__ x32) {
  const int a = blockIdx.z;
  const int r = blockIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= g.d || r >= R || j >= g.n[a]) return;
  const int64_t idx = (int64_t)R * g.off[a] + (int64_t)r * g.n[a] + j;
  const double v = x[idx] / muM[g.off[a] + j];
  x[idx] = v;
  if (x32) x32[idx] = (float)v;
}

// out[J] = sum_r w_r prod_a fac[R*off[a] + r*n_a + j_a]
__global__ void outer_sum_kernel(Geom g, int R, const double* __restrict__ fac, const double* __restrict__ w,
                                 double* __restrict__ out, int accumulate) {
  pdl_wait();
  const int64_t J = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (J >= g.ndof) return;
  int j[PE_MAX_D];
  unflatten(g, J, j);
  double acc = 0.0;
  for (int r = 0; r < R; ++r) {
    double P = fac[(int64_t)R * g.off[0] + (int64_t)r * g.n[0] + j[0]];
#pragma unroll
    for (int a = 1; a < PE_MAX_D; ++a) if (a < g.d) P *= fac[(int64_t)R * g.off[a] + (int64_t)r * g.n[a] + j[a]];
    acc += w[r] * P;
  }
  out[J] = accumulate ? out[J] + acc : acc;
}

__global__ void scale_mu_kernel(Geom g, const double* __restrict__ muM, double* __restrict__ x, int inverse) {
  const int64_t J = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (J >= g.ndof) return;
  int j[PE_MAX_D];
  unflatten(g, J, j);
  double mu = muM[g.off[0] + j[0]];
#pragma unroll
  for (int a = 1; a < PE_MAX_D; ++a) if (a < g.d) mu *= muM[g.off[a] + j[a]];
  x[J] = inverse ? x[J] / mu : x[J] * mu;
}

__global__ void weights_at_time_kernel(TermsDev T, double t, double* w) {
  const int r = threadIdx.x;
  if (r < T.n) w[r] = T.t[r].amp * eval_time(T.t[r], t);
}

__global__ void amps_kernel(TermsDev T, double* w) {
  pdl_wait();
  const int r = threadIdx.x;
  if (r < T.n) w[r] = T.t[r].amp;
}

}  // namespace

pe_status launch_time_tables(pe_ctx* c) {
  const int R = c->R;
  if (R == 0) return PE_OK;
  TermsDev T = pack_terms(c->terms, R);
  Nodes nF{}, nG{};
  for (int i = 0; i < PE_MAX_S; ++i) {
    nF.c[i] = c->cF[i];
    nG.c[i] = c->cG[i];
  }
  // stage-contracted columns: one per exponential term, two per sinusoid
  StageCols C{};
  for (int r = 0; r < R; ++r) {
    C.term[C.K] = (signed char)r;
    C.kind[C.K++] = 0;
    if (c->terms[r].tkind == PE_T_SIN) {
      C.term[C.K] = (signed char)r;
      C.kind[C.K++] = 1;
    }
  }
  c->cols = C;
  c->K = C.K;
  const int64_t total = (int64_t)c->N * c->M * C.K + (int64_t)c->N * c->p * R + (int64_t)c->q * C.K;
  const int threads = 256;
  PE_CUDA_TRY(launch_pdl(time_tables_kernel, dim3((unsigned)((total + threads - 1) / threads)), dim3(threads), 0,
                         c->stream, T, C, c->N, c->M, c->q, c->p, c->t0, c->dT, c->dt, nF, nG, c->AF,
                         c->precision == PE_MIXED ? c->AF32 : (float*)nullptr, c->AG,
                         c->precision == PE_MIXED ? c->AG32 : (float*)nullptr, c->Zst));
  c->launches += 1;
  PE_CUDA_TRY(cudaGetLastError());
  return PE_OK;
}

pe_status launch_stage_weights(pe_ctx* c) {
  const int K = c->K;
  if (K > c->Wcap) {
    // grown on demand (first problem, or a problem with more columns than before)
    PE_CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (c->Wst) cudaFree(c->Wst);
    if (c->Wst32) cudaFree(c->Wst32);
    c->Wst = nullptr;
    c->Wst32 = nullptr;
    c->Wcap = 0;
    const size_t n = (size_t)K * (size_t)c->g.ndof;
    if (cudaMalloc((void**)&c->Wst, n * sizeof(double)) != cudaSuccess ||
        (c->precision == PE_MIXED && cudaMalloc((void**)&c->Wst32, n * sizeof(float)) != cudaSuccess)) {
      cudaGetLastError();
      return pe_fail(PE_ENOMEM, "pe_set_problem: stage-weight table allocation failed");
    }
    c->Wcap = K;
  }
  const int threads = 256;
  const unsigned blocks = (unsigned)((c->g.ndof + threads - 1) / threads);
  if (c->precision == PE_MIXED && c->fine_engine == PE_FINE_TC && c->forcing_path == PE_FORCING_SEPARABLE) {
    // the tensor-core engine forms its float32 weights inside its operand split
    // (fine_tc_prepare); the float64 ones follow on the first float64 sweep (pe_refine)
    c->Wst_valid = false;
    return PE_OK;
  }
  if (c->precision == PE_MIXED) {
    // the float32 fine sweeps need only the float32 weights; the float64 ones follow on the
    // first float64 sweep (pe_refine)
    PE_CUDA_TRY(launch_pdl(stage_weights_kernel<float>, dim3(blocks), dim3(threads), 0, c->stream, c->g, c->cols, c->R,
                           c->q, (const float*)c->axisF32, (const float*)(c->coefF32 + 2 * c->g.ndof),
                           (const double*)c->Zst, c->Wst32));
    c->Wst_valid = false;
  } else {
    PE_CUDA_TRY(launch_pdl(stage_weights_kernel<double>, dim3(blocks), dim3(threads), 0, c->stream, c->g, c->cols,
                           c->R, c->q, (const double*)c->axisF, (const double*)(c->coefF + c->g.ndof),
                           (const double*)c->Zst, c->Wst));
    c->Wst_valid = true;
  }
  c->launches += 1;
  PE_CUDA_TRY(cudaGetLastError());
  return PE_OK;
}

pe_status launch_stage_weights_f64(pe_ctx* c) {
  if (c->Wst_valid) return PE_OK;
  const int threads = 256;
  stage_weights_kernel<double><<<(unsigned)((c->g.ndof + threads - 1) / threads), threads, 0, c->stream>>>(
      c->g, c->cols, c->R, c->q, c->axisF, c->coefF + c->g.ndof, c->Zst, c->Wst);
  c->launches += 1;
  PE_CUDA_TRY(cudaGetLastError());
  c->Wst_valid = true;
  return PE_OK;
}

// Rows of the whole-axis per-axis tables (layout of gf) that a sharded context owns, in its
// own layout (gl): out[R off_l[a] + r n_l[a] + j] = in[R off_f[a] + r n_f[a] + j + base_a],
// base_0 = the first owned axis-0 mode, base_a = 0 for the other axes.
__global__ void compact_axis_kernel(Geom gf, Geom gl, int base0, int R, const double* __restrict__ in,
                                    double* __restrict__ out, float* __restrict__ out32) {
  const int a = blockIdx.z;
  const int r = blockIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= gl.d || r >= R || j >= gl.n[a]) return;
  const int jf = j + (a == 0 ? base0 : 0);
  const double v = in[(int64_t)R * gf.off[a] + (int64_t)r * gf.n[a] + jf];
  const int64_t o = (int64_t)R * gl.off[a] + (int64_t)r * gl.n[a] + j;
  out[o] = v;
  if (out32) out32[o] = (float)v;
}

static pe_status separable_factors_whole(pe_ctx* c, const pe_term* terms, int nterms, double* axis_out, int mode,
                                         const signed char (*lk)[PE_MAX_D]);

pe_status compact_axis_tables(pe_ctx* c, int R, const double* in, double* out, float* out32) {
  int nmax = 1;
  for (int a = 0; a < c->g.d; ++a) nmax = c->g.n[a] > nmax ? c->g.n[a] : nmax;
  dim3 grid((nmax + 127) / 128, R, c->g.d);
  compact_axis_kernel<<<grid, 128, 0, c->stream>>>(c->gn, c->g, c->base0, R, in, out, out32);
  c->launches += 1;
  PE_CUDA_TRY(cudaGetLastError());
  return PE_OK;
}

// mode 0: 1D loads only (axis_out gets loads); mode 1: modal factors (S_a F)/mu^M;
// mode 2: S_a F only (the modal coefficients V^T y of a separable nodal vector y).
// lk (may be NULL): per-term, per-axis load kinds of the Dirichlet lifting (TermsDev).
// A sharded context computes the factors of the whole axes and keeps the rows of its modes.
pe_status launch_separable_factors(pe_ctx* c, const pe_term* terms, int nterms, double* axis_out, int mode,
                                   const signed char (*lk)[PE_MAX_D]) {
  if (!c->sharded) return separable_factors_whole(c, terms, nterms, axis_out, mode, lk);
  if (nterms == 0) return PE_OK;
  if (mode != 1) return pe_fail(PE_EINVAL, "a context that owns a block of modes takes separable modal factors only");
  const Geom gl = c->g;
  double* mu_l = c->muM_axis;
  c->g = c->gn;
  c->muM_axis = c->muM_full;
  const pe_status st = separable_factors_whole(c, terms, nterms, c->fac_full, 1, lk);
  c->g = gl;
  c->muM_axis = mu_l;
  PE_TRY(st);
  const bool f32 = (axis_out == c->axisF) && c->precision == PE_MIXED;
  return compact_axis_tables(c, nterms, c->fac_full, axis_out, f32 ? c->axisF32 : nullptr);
}

static pe_status separable_factors_whole(pe_ctx* c, const pe_term* terms, int nterms, double* axis_out, int mode,
                                         const signed char (*lk)[PE_MAX_D]) {
  if (nterms == 0) return PE_OK;
  TermsDev T = pack_terms(terms, nterms, lk);
  Gauss G = make_gauss(c->quad_pts);
  int nmax = 1;
  for (int a = 0; a < c->g.d; ++a) nmax = c->g.n[a] > nmax ? c->g.n[a] : nmax;
  dim3 grid((nmax + 127) / 128, nterms, c->g.d);
  dim3 lgrid((nmax + 31) / 32, nterms, c->g.d);  // 32 nodes of eight lanes per CTA
  double* loads = mode == 0 ? axis_out : c->loads;
  PE_CUDA_TRY(launch_pdl(loads_1d_kernel, lgrid, dim3(32 * kLoadLanes), 0, c->stream, T, c->g, c->lo[0], c->lo[1],
                         c->lo[2], c->h[0], c->h[1], c->h[2], G, loads));
  c->launches += 1;
  PE_CUDA_TRY(cudaGetLastError());
  if (mode == 0) return PE_OK;
  const bool f32 = (axis_out == c->axisF) && c->precision == PE_MIXED;
  // the matrix form over every SM while its float64 work stays small (R sum_a n_a^2 <= 8M FMAs)
  int64_t work = 0;
  for (int a = 0; a < c->g.d; ++a) work += (int64_t)nterms * c->g.n[a] * c->g.n[a];
  if (c->muM_inv && work <= ((int64_t)8 << 20)) {
    const int64_t total = (int64_t)nterms * (c->g.off[c->g.d - 1] + c->g.n[c->g.d - 1]);
    const unsigned blocks = (unsigned)((total * kFactorLanes + 255) / 256);
    PE_CUDA_TRY(launch_pdl(axis_factor_matrix_kernel, dim3(blocks), dim3(256), 0, c->stream, c->g, nterms,
                           (const double*)c->S[0], (const double*)(c->g.d > 1 ? c->S[1] : c->S[0]),
                           (const double*)(c->g.d > 2 ? c->S[2] : c->S[0]), (const double*)loads,
                           (const double*)(mode == 1 ? c->muM_inv : nullptr), axis_out,
                           mode == 1 && f32 ? c->axisF32 : (float*)nullptr, total));
    c->launches += 1;
    PE_CUDA_TRY(cudaGetLastError());
    return PE_OK;
  }
  if (mode == 1) {
    bool done = false;
    PE_TRY(axis_factors_fused(c, nterms, loads, axis_out, f32 ? c->axisF32 : nullptr, &done));
    if (done) return PE_OK;
  }
  for (int a = 0; a < c->g.d; ++a) {
    const int64_t base = (int64_t)nterms * c->g.off[a];
    PE_TRY(dst_axis_f64(c->S[a], loads + base, axis_out + base, nterms, c->g.n[a], 1, c->stream, c->g.per[a]));
    c->launches += 1;
  }
  if (mode == 2) return PE_OK;  // V^T of nodal values: no division by mu^M
  divide_axis_mu_kernel<<<grid, 128, 0, c->stream>>>(c->g, nterms, c->muM_axis, axis_out,
                                                     f32 ? c->axisF32 : nullptr);
  c->launches += 1;
  PE_CUDA_TRY(cudaGetLastError());
  return PE_OK;
}

// out[J] = sum_r amp_r prod_a fac_{r,a}[j_a] (nodal_loads: fac are 1D loads, out a nodal load vector)
pe_status launch_outer_sum(pe_ctx* c, const double* axis_fac, const pe_term* terms, int nterms, double* out,
                           int accumulate) {
  if (nterms == 0) return PE_OK;
  double* w = c->partials;  // at least PE_MAX_TERMS doubles
  TermsDev T = pack_terms(terms, nterms);
  PE_CUDA_TRY(launch_pdl(amps_kernel, dim3(1), dim3(PE_MAX_TERMS), 0, c->stream, T, w));
  const int threads = 256;
  PE_CUDA_TRY(launch_pdl(outer_sum_kernel, dim3((unsigned)((c->g.ndof + threads - 1) / threads)), dim3(threads), 0,
                         c->stream, c->g, nterms, axis_fac, (const double*)w, out, accumulate));
  c->launches += 2;
  PE_CUDA_TRY(cudaGetLastError());
  return PE_OK;
}

pe_status launch_forcing_modal(pe_ctx* c, double t, double* out) {
  double* w = c->partials;
  TermsDev T = pack_terms(c->terms, c->R);
  weights_at_time_kernel<<<1, PE_MAX_TERMS, 0, c->stream>>>(T, t, w);
  const int threads = 256;
  outer_sum_kernel<<<(unsigned)((c->g.ndof + threads - 1) / threads), threads, 0, c->stream>>>(c->g, c->R,
                                                                                               c->axisF, w, out, 0);
  c->launches += 2;
  PE_CUDA_TRY(cudaGetLastError());
  return PE_OK;
}

pe_status launch_scale_by_muM(pe_ctx* c, double* x, int inverse) {
  const int threads = 256;
  scale_mu_kernel<<<(unsigned)((c->g.ndof + threads - 1) / threads), threads, 0, c->stream>>>(c->g, c->muM_axis, x,
                                                                                              inverse);
  c->launches += 1;
  PE_CUDA_TRY(cudaGetLastError());
  return PE_OK;
}
